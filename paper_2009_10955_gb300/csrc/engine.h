// engine.h -- internal declarations shared by the C ABI and the CUDA code.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>

#include "../../include/graphpi.h"
#include "plan.h"

// The data graph: undirected, simple, sorted adjacency lists in CSR form,
// resident on one device (Section IV-E keeps the whole graph in memory).
struct gp_graph {
    int device = 0;
    int32_t n = 0;
    int64_t nnz = 0;              // directed entries = 2 |E|
    int32_t max_deg = 0;
    int64_t heavy_end = 0;        // CSR entries of the leading vertices of degree
                                  // >= kHeavyDegree (degree-ordered graphs only)
    int64_t* row_ptr = nullptr;   // device, n + 1
    int32_t* col = nullptr;       // device, nnz
    int32_t* labels = nullptr;      // device, n vertex labels (graph labelling) or null
    uint32_t* core_bits = nullptr;  // device, core_n x core_words: adjacency among
    int32_t core_n = 0;             // the core_n highest-degree vertices (ids
    int32_t core_words = 0;         // 0..core_n-1 of a degree-ordered graph)
    int32_t* perm = nullptr;      // device, n (new id -> input id) or null
    std::mutex mu;
    bool tri_done = false;
    uint64_t tri_cnt = 0;         // ordered triangles (6 x triangles)
};

namespace gp {

void set_error(const char* fmt, ...);
void count_launch(int n = 1);

// Device graph build from m pairs already on the device (graph.cu).
gp_status build_graph(const int32_t* d_src, const int32_t* d_dst, int64_t m, int32_t n,
                      bool degree_order, cudaStream_t st, gp_graph* g);
// Expand a device CSR to pairs (graph.cu).
gp_status csr_to_pairs(const int64_t* d_row_ptr, const int32_t* d_col, int32_t n, int64_t nnz,
                       int32_t* d_src, int32_t* d_dst, cudaStream_t st);
// Maximum degree of a device CSR (graph.cu).
gp_status max_degree(const int64_t* d_row_ptr, int32_t n, cudaStream_t st, int32_t* out);
// Adjacency bit matrix of vertices [0, core_n) among themselves (graph.cu).
gp_status build_core_bits(gp_graph* g, int32_t core_n, cudaStream_t st);
// First CSR entry of the first vertex whose degree is below min_deg, for a
// graph whose degrees do not increase with the id (graph.cu).
gp_status heavy_prefix(const int64_t* d_row_ptr, int32_t n, int32_t min_deg, cudaStream_t st,
                       int64_t* out);

// One counting job for the device (count.cu).
struct CountJob {
    GpPlan plan;
    const int64_t* row_ptr;
    const int32_t* col;
    int32_t n;
    int32_t slot_cap;        // elements per intermediate set (>= max degree)
    int64_t task_begin;      // first CSR entry (edge task) of this job
    int64_t ntasks;          // edge tasks of this job
    int64_t task_offset;     // first global work-item index of this job
    int64_t heavy;           // leading tasks of this job handed out one at a time
    int32_t split;           // parts each of those tasks is cut into (>= 1)
    int32_t pad0;
    int64_t nvirt;           // work items: heavy * split + (ntasks - heavy)
    const int32_t* labels;      // vertex labels (labelled plans), or null
    const uint32_t* core_bits;  // core adjacency bit matrix (null: none)
    int32_t core_n;
    int32_t core_words;
};

// Largest core (in vertices) whose adjacency bit matrix a graph keeps:
// 8192 x 8192 bits = 8 MB.
constexpr int32_t kCoreMax = 8192;

// Vertices of at least this degree start tasks heavy enough to be handed out
// one per grab (degree-ordered graphs put them first).
constexpr int32_t kHeavyDegree = 256;

struct LaunchOpts {
    int warps_per_block = 8;
    int blocks_per_sm = 0;   // 0 = occupancy maximum
    int chunk = 0;           // 0 = automatic
    int64_t budget_cycles = 0;
    bool stats = false;      // instrumented kernel that tallies algorithmic bytes and operations
    bool no_core = false;    // binary searches only (no core bit matrix)
    int64_t task_cycles = 0; // per-work-item cycle limit (0 = none)
    int bitmap_mode = 2;     // bitmap subtree: 0 warp per candidate, 1 lane per candidate (last two levels), 2 (default) also the lane three-level tail
    int lane_work = 0;       // 0 = default
};

// Run the jobs in one persistent launch. results[2 j], results[2 j + 1]
// receive job j's 128-bit count (lo, hi). *processed receives how many
// global tasks (from 0) were completed (< total only with a budget).
// With lo.stats, *algo_bytes receives the list-path bytes and *algo_ops the
// bitmap-subtree word operations of the launch. busy (2 words) receives the
// sum over warps of the cycles each spent before finding no work left, and
// the number of warps launched.
gp_status run_count(const CountJob* jobs, int njobs, const LaunchOpts& lo, cudaStream_t st,
                    uint64_t* results, int64_t* processed, float* kernel_ms = nullptr,
                    uint64_t* algo_bytes = nullptr, int* aborted = nullptr, uint64_t* algo_ops = nullptr,
                    uint64_t* busy = nullptr);

// run_count without allocating: results, job table and intermediate sets all
// live in the caller's device buffer d_scratch (256-byte aligned); the grid
// shrinks to what that buffer holds. GP_ERR_SCRATCH when not even one block
// fits.
gp_status run_count_in_scratch(const CountJob* jobs, int njobs, void* d_scratch, size_t scratch_bytes,
                               cudaStream_t st, uint64_t* results);

// The job of plan idx of s over all edge tasks of g, with g's device made
// current (capi.cu).
gp_status single_job(gp_graph* g, const gp_schedules* s, int32_t idx, CountJob* job);
// A job's count from its 128-bit device total (inclusion-exclusion plans are
// divided by their multiplicity); GP_ERR_OVERFLOW beyond 64 bits (capi.cu).
gp_status job_total(const CountJob& job, const uint64_t* res, uint64_t* out);

// Listing: the embeddings of the longest prefix of the job's tasks whose
// total fits `capacity` tuples, written to d_out (k int32 per embedding).
// *cut_tasks receives that prefix's length, *n_written its embeddings,
// *total the embeddings of all the job's tasks. capacity < 0: count only.
gp_status run_list(const CountJob& job, int32_t* d_out, int64_t capacity, cudaStream_t st,
                   int64_t* n_written, int64_t* cut_tasks, int64_t* total = nullptr);

// Key of the kernel build geometry() would pick for this job alone (its
// register budget and whether it carries general inclusion-exclusion); jobs
// with equal keys run best in one launch.
int kernel_variant(const CountJob& job, const LaunchOpts& opt);

// Device scratch run_count would allocate for these jobs and options.
gp_status scratch_bytes(const CountJob* jobs, int njobs, const LaunchOpts& lo, uint64_t* bytes);

}  // namespace gp

#define GP_CUDA_TRY(expr)                                                          \
    do {                                                                           \
        cudaError_t _e = (expr);                                                   \
        if (_e != cudaSuccess) {                                                   \
            gp::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e),  \
                          __FILE__, __LINE__);                                     \
            return GP_ERR_CUDA;                                                    \
        }                                                                          \
    } while (0)
