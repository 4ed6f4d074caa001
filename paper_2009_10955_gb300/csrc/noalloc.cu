// noalloc.cu -- gp_count_noalloc: a count that allocates no memory.
//
// Some callers cannot allocate device memory at the moment they need a
// count: code running under a memory pool or arena that owns every byte of
// the device, plugins whose host forbids cudaMalloc/cudaFree on its streams,
// or latency-critical loops where an allocation (and the synchronisation it
// may imply) is not acceptable. For them this file keeps one fixed scratch
// array in device memory for the whole life of the process, and
// gp_count_noalloc runs the ordinary counting kernel with its results, job
// table and intermediate sets placed inside that array.
//
// Costs and limits: every GPU that loads the library holds the array
// (kNoallocScratchBytes) until the process exits; the launch uses only as
// many blocks as the array has room for, so a count can be much slower than
// gp_count on large graphs; plans whose per-block scratch exceeds the array
// are rejected with GP_ERR_SCRATCH.
#include <mutex>

#include "engine.h"

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)64 << 20;   // 64 MiB

// The fixed scratch. In host code this name is only a stand-in for the
// device symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 128;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (with that device current) and cached.
gp_status scratch_address(void** out) {
    int dev = 0;
    GP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        gp::set_error("device ordinal %d beyond the supported %d", dev, kMaxDevices);
        return GP_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            gp::set_error("cudaGetSymbolAddress of the fixed scratch failed: %s", cudaGetErrorString(e));
            return GP_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return GP_OK;
}

}  // namespace

extern "C" gp_status gp_count_noalloc(gp_graph* g, const gp_schedules* s, int32_t idx, void* stream,
                                      uint64_t* out) {
    if (!out) { gp::set_error("out is null"); return GP_ERR_ARG; }
    gp::CountJob job;
    gp_status rc = gp::single_job(g, s, idx, &job);
    if (rc != GP_OK) return rc;
    void* scratch = nullptr;
    rc = scratch_address(&scratch);
    if (rc != GP_OK) return rc;
    uint64_t res[2] = {0, 0};
    rc = gp::run_count_in_scratch(&job, 1, scratch, kNoallocScratchBytes, static_cast<cudaStream_t>(stream), res);
    if (rc != GP_OK) return rc;
    uint64_t total = 0;
    rc = gp::job_total(job, res, &total);
    if (rc != GP_OK) return rc;
    *out = total;
    return GP_OK;
}
