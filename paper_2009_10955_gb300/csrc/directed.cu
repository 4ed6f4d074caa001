// directed.cu -- directed patterns on directed graphs.
//
// The paper names directed patterns as an extension without defining them.
// Reading taken here: a directed pattern has arcs a -> b; an embedding is an
// injective map f that sends every pattern arc a -> b to a graph arc
// f(a) -> f(b) (non-induced), and the count is the number of such maps
// divided by |Aut(P)|, Aut(P) being the arc-preserving permutations.
// Algorithm 1 (Section IV-A) runs on that group unchanged; where it finds no
// restriction set (a directed cycle's rotations have no usable 2-cycles)
// the plan keeps no restrictions and the total is divided by |Aut(P)|.
//
// Graph: every arc once, as sorted out-lists and sorted in-lists (CSR each),
// built on the device with one radix sort per direction (CUB).
//
// Count kernel: a persistent grid, one warp per root vertex taken from a
// global cursor; the warp runs the matching order depth-first. At depth d
// the candidates are the out- or in-list of the image of one earlier vertex
// joined to it by an arc; the 32 lanes test 32 candidates at a time (distinct
// from the matched vertices, the other arcs to matched vertices by binary
// search in out-lists, the restrictions as comparisons) and a ballot keeps
// the survivors; at the last depth the survivors are counted, not visited.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_select.cuh>

#include <algorithm>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "engine.h"
#include "planner.h"

struct gp_dgraph {
    int device = 0;
    int32_t n = 0;
    int64_t narcs = 0;
    int64_t* out_ptr = nullptr;   // device, n + 1
    int32_t* out_col = nullptr;   // device, narcs
    int64_t* in_ptr = nullptr;    // device, n + 1
    int32_t* in_col = nullptr;    // device, narcs
};

struct gp_dpattern {
    int k = 0;
    uint8_t arc[GP_MAX_K][GP_MAX_K] = {};   // arc[a][b]: a -> b
    gp::PatternInfo info;                   // underlying undirected pattern, arc-preserving group
};

namespace gp {
namespace {

constexpr int kDThreads = 256;
constexpr unsigned kAll = 0xffffffffu;

inline int dblocks_for(int64_t n) {
    int64_t b = (n + kDThreads - 1) / kDThreads;
    return (int)(b < 1 ? 1 : (b > (1 << 30) ? (1 << 30) : b));
}

int dbits_for(uint64_t x) {
    int b = 0;
    while (b < 64 && (x >> b)) ++b;
    return b;
}

gp_status dfail(gp_status s, const char* msg) {
    set_error("%s", msg);
    return s;
}

struct DScratch {
    cudaStream_t st;
    void* p = nullptr;
    explicit DScratch(cudaStream_t s) : st(s) {}
    ~DScratch() { if (p) cudaFreeAsync(p, st); }
    cudaError_t alloc(size_t bytes) { return cudaMallocAsync(&p, bytes ? bytes : 16, st); }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// ----------------------------------------------------------------- graph

// Arc keys (u << 32) | v; loops and out-of-range ids become the sentinel
// n << 32, which sorts after every real arc.
__global__ void k_arc_keys(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                           int32_t n, uint64_t* __restrict__ keys, int* __restrict__ bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = src[i], v = dst[i];
        const bool in_range = u >= 0 && u < n && v >= 0 && v < n;
        if (!in_range) atomicExch(bad, 1);
        keys[i] = (in_range && u != v) ? (((uint64_t)(uint32_t)u << 32) | (uint32_t)v)
                                       : ((uint64_t)(uint32_t)n << 32);
    }
}

// The same arcs keyed by their head: (v << 32) | u.
__global__ void k_swap_keys(const uint64_t* __restrict__ keys, int64_t a, uint64_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t x = keys[i];
        out[i] = ((x & 0xffffffffull) << 32) | (x >> 32);
    }
}

__global__ void k_low_words(const uint64_t* __restrict__ keys, int64_t a, int32_t* __restrict__ col) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a;
         i += (int64_t)gridDim.x * blockDim.x)
        col[i] = (int32_t)(uint32_t)(keys[i] & 0xffffffffull);
}

// ptr[v] = first key index whose high word is >= v, for v in [0, n].
__global__ void k_list_starts(const uint64_t* __restrict__ keys, int64_t a, int32_t n,
                              int64_t* __restrict__ ptr) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t target = (uint64_t)v << 32;
        int64_t lo = 0, hi = a;
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (keys[mid] < target) lo = mid + 1; else hi = mid;
        }
        ptr[v] = lo;
    }
}

// Sort keys (a entries of `in`, ids of n vertices) into `out` and lay them
// out as one CSR direction (ptr n + 1, col a), both freshly allocated.
gp_status keys_to_lists(uint64_t* keys, uint64_t* spare, int64_t a, int32_t n, cudaStream_t st,
                        int64_t** ptr, int32_t** col) {
    const int end_bit = 32 + dbits_for((uint64_t)(uint32_t)n);
    if (a > 0) {
        size_t tb = 0;
        GP_CUDA_TRY(cub::DeviceRadixSort::SortKeys(nullptr, tb, keys, spare, a, 0, end_bit, st));
        DScratch temp(st);
        GP_CUDA_TRY(temp.alloc(tb));
        GP_CUDA_TRY(cub::DeviceRadixSort::SortKeys(temp.p, tb, keys, spare, a, 0, end_bit, st));
        count_launch();
    }
    GP_CUDA_TRY(cudaMalloc(ptr, sizeof(int64_t) * ((size_t)n + 1)));
    GP_CUDA_TRY(cudaMalloc(col, sizeof(int32_t) * (size_t)std::max<int64_t>(a, 1)));
    k_list_starts<<<dblocks_for((int64_t)n + 1), kDThreads, 0, st>>>(spare, a, n, *ptr);
    count_launch();
    GP_CUDA_TRY(cudaGetLastError());
    if (a > 0) {
        k_low_words<<<dblocks_for(a), kDThreads, 0, st>>>(spare, a, *col);
        count_launch();
        GP_CUDA_TRY(cudaGetLastError());
    }
    return GP_OK;
}

gp_status build_dgraph(const int32_t* d_src, const int32_t* d_dst, int64_t m, int32_t n, cudaStream_t st,
                       gp_dgraph* g) {
    DScratch keys(st), sorted(st), bad(st), nsel(st);
    GP_CUDA_TRY(keys.alloc(sizeof(uint64_t) * (size_t)std::max<int64_t>(m, 1)));
    GP_CUDA_TRY(sorted.alloc(sizeof(uint64_t) * (size_t)std::max<int64_t>(m, 1)));
    GP_CUDA_TRY(bad.alloc(sizeof(int)));
    GP_CUDA_TRY(nsel.alloc(sizeof(int64_t)));
    GP_CUDA_TRY(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    int64_t a = 0;
    if (m > 0) {
        k_arc_keys<<<dblocks_for(m), kDThreads, 0, st>>>(d_src, d_dst, m, n, keys.as<uint64_t>(), bad.as<int>());
        count_launch();
        GP_CUDA_TRY(cudaGetLastError());
        int h_bad = 0;
        GP_CUDA_TRY(cudaMemcpyAsync(&h_bad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        GP_CUDA_TRY(cudaStreamSynchronize(st));
        if (h_bad) { set_error("arc endpoint outside [0, %d)", n); return GP_ERR_ARG; }
        // sort by tail, keep one copy of each arc, drop the sentinel
        const int end_bit = 32 + dbits_for((uint64_t)(uint32_t)n);
        size_t tb = 0, tb2 = 0;
        GP_CUDA_TRY(cub::DeviceRadixSort::SortKeys(nullptr, tb, keys.as<uint64_t>(), sorted.as<uint64_t>(),
                                                   m, 0, end_bit, st));
        GP_CUDA_TRY(cub::DeviceSelect::Unique(nullptr, tb2, sorted.as<uint64_t>(), keys.as<uint64_t>(),
                                              nsel.as<int64_t>(), m, st));
        DScratch temp(st);
        GP_CUDA_TRY(temp.alloc(std::max(tb, tb2)));
        GP_CUDA_TRY(cub::DeviceRadixSort::SortKeys(temp.p, tb, keys.as<uint64_t>(), sorted.as<uint64_t>(),
                                                   m, 0, end_bit, st));
        GP_CUDA_TRY(cub::DeviceSelect::Unique(temp.p, tb2, sorted.as<uint64_t>(), keys.as<uint64_t>(),
                                              nsel.as<int64_t>(), m, st));
        count_launch(2);
        int64_t h = 0;
        GP_CUDA_TRY(cudaMemcpyAsync(&h, nsel.p, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        GP_CUDA_TRY(cudaStreamSynchronize(st));
        uint64_t last = 0;
        if (h > 0) {
            GP_CUDA_TRY(cudaMemcpyAsync(&last, keys.as<uint64_t>() + (h - 1), sizeof(uint64_t),
                                        cudaMemcpyDeviceToHost, st));
            GP_CUDA_TRY(cudaStreamSynchronize(st));
        }
        a = h - ((h > 0 && last == ((uint64_t)(uint32_t)n << 32)) ? 1 : 0);
    }
    // keys holds the unique arcs by tail (a entries): out-lists; the same
    // arcs keyed by head give the in-lists
    DScratch rkeys(st);
    GP_CUDA_TRY(rkeys.alloc(sizeof(uint64_t) * (size_t)std::max<int64_t>(a, 1)));
    if (a > 0) {
        k_swap_keys<<<dblocks_for(a), kDThreads, 0, st>>>(keys.as<uint64_t>(), a, rkeys.as<uint64_t>());
        count_launch();
        GP_CUDA_TRY(cudaGetLastError());
    }
    gp_status rc = keys_to_lists(keys.as<uint64_t>(), sorted.as<uint64_t>(), a, n, st, &g->out_ptr, &g->out_col);
    if (rc != GP_OK) return rc;
    rc = keys_to_lists(rkeys.as<uint64_t>(), keys.as<uint64_t>(), a, n, st, &g->in_ptr, &g->in_col);
    if (rc != GP_OK) return rc;
    GP_CUDA_TRY(cudaStreamSynchronize(st));
    g->n = n;
    g->narcs = a;
    return GP_OK;
}

void free_dgraph(gp_dgraph* g) {
    if (!g) return;
    if (g->out_ptr) cudaFree(g->out_ptr);
    if (g->out_col) cudaFree(g->out_col);
    if (g->in_ptr) cudaFree(g->in_ptr);
    if (g->in_col) cudaFree(g->in_col);
    delete g;
}

// ------------------------------------------------------------------ plan

constexpr int kMaxChecks = 2 * GP_MAX_K;

struct DPlan {
    int k;
    int order[GP_MAX_K];
    int anchor[GP_MAX_K];                  // earlier depth whose image's list holds the candidates
    int anchor_out[GP_MAX_K];              // 1: its out-list, 0: its in-list
    int nchk[GP_MAX_K];
    int chk_depth[GP_MAX_K][kMaxChecks];   // further arcs to matched vertices ...
    int chk_fwd[GP_MAX_K][kMaxChecks];     // ... 1: image(j) -> v, 0: v -> image(j)
    int nres[GP_MAX_K];
    int res_depth[GP_MAX_K][GP_MAX_K];     // restrictions acting at depth d
    int res_gt[GP_MAX_K][GP_MAX_K];        // 1: v > image(j), 0: v < image(j)
};

// Compile a matching order (every prefix weakly connected) and a restriction
// set into a DPlan; false with a message otherwise.
bool compile_dplan(const gp_dpattern& p, const int8_t* sched, ResMask res, DPlan* out, std::string& err) {
    const int k = p.k;
    DPlan P;
    std::memset(&P, 0, sizeof(P));
    P.k = k;
    int pos[GP_MAX_K];
    bool seen[GP_MAX_K] = {};
    for (int d = 0; d < k; ++d) {
        const int x = sched[d];
        if (x < 0 || x >= k || seen[x]) { err = "order is not a permutation of the pattern vertices"; return false; }
        seen[x] = true;
        P.order[d] = x;
        pos[x] = d;
    }
    for (int d = 1; d < k; ++d) {
        const int x = P.order[d];
        P.anchor[d] = -1;
        for (int j = 0; j < d; ++j) {
            const int y = P.order[j];
            const bool to_x = p.arc[y][x], from_x = p.arc[x][y];
            if (!to_x && !from_x) continue;
            if (P.anchor[d] < 0) {
                P.anchor[d] = j;
                P.anchor_out[d] = to_x ? 1 : 0;   // y -> x: x is among the out-arcs of image(y)
                if (to_x && from_x) { P.chk_depth[d][P.nchk[d]] = j; P.chk_fwd[d][P.nchk[d]++] = 0; }
                continue;
            }
            if (to_x) { P.chk_depth[d][P.nchk[d]] = j; P.chk_fwd[d][P.nchk[d]++] = 1; }
            if (from_x) { P.chk_depth[d][P.nchk[d]] = j; P.chk_fwd[d][P.nchk[d]++] = 0; }
        }
        if (P.anchor[d] < 0) { err = "every prefix of the order must be weakly connected"; return false; }
    }
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) {
            if (!(res >> res_bit(a, b) & 1)) continue;     // id(a) > id(b)
            const int da = pos[a], db = pos[b];
            const int later = std::max(da, db);
            P.res_depth[later][P.nres[later]] = std::min(da, db);
            P.res_gt[later][P.nres[later]++] = (later == da) ? 1 : 0;
        }
    *out = P;
    return true;
}

// ---------------------------------------------------------------- kernel

__device__ __forceinline__ bool arc_in(const int64_t* __restrict__ out_ptr, const int32_t* __restrict__ out_col,
                                       int32_t u, int32_t v) {   // u -> v ?
    int64_t lo = out_ptr[u], hi = out_ptr[u + 1];
    const int64_t end = hi;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (out_col[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo < end && out_col[lo] == v;
}

__global__ void __launch_bounds__(kDThreads)
k_dcount(const __grid_constant__ DPlan P, int32_t n, const int64_t* __restrict__ out_ptr, const int32_t* __restrict__ out_col,
         const int64_t* __restrict__ in_ptr, const int32_t* __restrict__ in_col,
         unsigned long long* __restrict__ cursor, unsigned long long* __restrict__ result) {
    const int lane = threadIdx.x & 31;
    unsigned long long lo_acc = 0, hi_acc = 0;      // lane 0's 128-bit sum
    int32_t img[GP_MAX_K];
    const int32_t* lst[GP_MAX_K];
    int64_t len[GP_MAX_K], next[GP_MAX_K], taken[GP_MAX_K];
    unsigned mask[GP_MAX_K];
    for (;;) {
        unsigned long long root = 0;
        if (lane == 0) root = atomicAdd(cursor, 1ull);
        root = __shfl_sync(kAll, root, 0);
        if (root >= (unsigned long long)n) break;
        img[0] = (int32_t)root;
        int d = 1;
        auto open = [&](int dd) {
            const int32_t a = img[P.anchor[dd]];
            const int64_t* ptr = P.anchor_out[dd] ? out_ptr : in_ptr;
            const int32_t* col = P.anchor_out[dd] ? out_col : in_col;
            lst[dd] = col + ptr[a];
            len[dd] = ptr[a + 1] - ptr[a];
            next[dd] = 0;
            mask[dd] = 0;
        };
        open(1);
        while (d >= 1) {
            if (mask[d] == 0) {
                if (next[d] >= len[d]) { --d; continue; }
                const int64_t i = next[d] + lane;
                bool ok = false;
                if (i < len[d]) {
                    const int32_t v = lst[d][i];
                    ok = true;
                    for (int j = 0; j < d; ++j) ok = ok && (img[j] != v);                 // injective
                    for (int c = 0; c < P.nchk[d] && ok; ++c) {                         // other arcs
                        const int32_t o = img[P.chk_depth[d][c]];
                        ok = P.chk_fwd[d][c] ? arc_in(out_ptr, out_col, o, v) : arc_in(out_ptr, out_col, v, o);
                    }
                    for (int r = 0; r < P.nres[d] && ok; ++r) {                         // restrictions
                        const int32_t o = img[P.res_depth[d][r]];
                        ok = P.res_gt[d][r] ? (v > o) : (v < o);
                    }
                }
                const unsigned m = __ballot_sync(kAll, ok);
                taken[d] = next[d];
                next[d] += 32;
                if (d == P.k - 1) {                                   // last depth: count
                    if (lane == 0) {
                        const unsigned long long add = (unsigned long long)__popc(m);
                        lo_acc += add;
                        hi_acc += (lo_acc < add) ? 1ull : 0ull;
                    }
                    continue;
                }
                mask[d] = m;
                continue;
            }
            const int b = __ffs(mask[d]) - 1;
            mask[d] &= mask[d] - 1;
            img[d] = lst[d][taken[d] + b];
            ++d;
            open(d);
        }
    }
    if (lane == 0 && (lo_acc | hi_acc)) {
        const unsigned long long old = atomicAdd(result, lo_acc);
        const unsigned long long carry = (old + lo_acc < old) ? 1ull : 0ull;
        if (hi_acc + carry) atomicAdd(result + 1, hi_acc + carry);
    }
}

gp_status run_dcount(const gp_dgraph* g, const DPlan& P, uint64_t div, cudaStream_t st, uint64_t* out) {
    if (g->n == 0) { *out = 0; return GP_OK; }
    DScratch mem(st);
    GP_CUDA_TRY(mem.alloc(3 * sizeof(unsigned long long)));
    GP_CUDA_TRY(cudaMemsetAsync(mem.p, 0, 3 * sizeof(unsigned long long), st));
    unsigned long long* cursor = mem.as<unsigned long long>();
    unsigned long long* res = cursor + 1;
    int dev = 0, nsm = 0;
    GP_CUDA_TRY(cudaGetDevice(&dev));
    GP_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = std::max(1, nsm * 8);
    k_dcount<<<blocks, kDThreads, 0, st>>>(P, g->n, g->out_ptr, g->out_col, g->in_ptr, g->in_col, cursor, res);
    count_launch();
    GP_CUDA_TRY(cudaGetLastError());
    unsigned long long h[2] = {0, 0};
    GP_CUDA_TRY(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, st));
    GP_CUDA_TRY(cudaStreamSynchronize(st));
    const unsigned __int128 total = ((unsigned __int128)h[1] << 64) | h[0];
    if (div == 0 || total % div) return dfail(GP_ERR_INTERNAL, "map count is not a multiple of |Aut(P)|");
    const unsigned __int128 q = total / div;
    if (q >> 64) return dfail(GP_ERR_OVERFLOW, "count does not fit in 64 bits");
    *out = (uint64_t)q;
    return GP_OK;
}

cudaStream_t dstream(void* s) { return static_cast<cudaStream_t>(s); }

}  // namespace
}  // namespace gp

extern "C" {

gp_status gp_dgraph_create(const int32_t* src, const int32_t* dst, int64_t m, int32_t n, uint32_t flags,
                           void* stream, gp_dgraph** out) {
    using namespace gp;
    if (!out || m < 0 || n < 0 || n == INT32_MAX || (m > 0 && (!src || !dst)))
        return dfail(GP_ERR_ARG, "gp_dgraph_create: bad arguments");
    *out = nullptr;
    cudaStream_t st = dstream(stream);
    std::unique_ptr<gp_dgraph> g(new (std::nothrow) gp_dgraph);
    if (!g) return dfail(GP_ERR_NOMEM, "gp_dgraph_create: out of host memory");
    GP_CUDA_TRY(cudaGetDevice(&g->device));
    const int32_t* d_src = src;
    const int32_t* d_dst = dst;
    DScratch s_src(st), s_dst(st);
    if (!(flags & GP_DEVICE_PTRS) && m > 0) {
        GP_CUDA_TRY(s_src.alloc(sizeof(int32_t) * (size_t)m));
        GP_CUDA_TRY(s_dst.alloc(sizeof(int32_t) * (size_t)m));
        GP_CUDA_TRY(cudaMemcpyAsync(s_src.p, src, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, st));
        GP_CUDA_TRY(cudaMemcpyAsync(s_dst.p, dst, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, st));
        d_src = s_src.as<int32_t>();
        d_dst = s_dst.as<int32_t>();
    }
    gp_status rc = build_dgraph(d_src, d_dst, m, n, st, g.get());
    if (rc != GP_OK) {
        cudaStreamSynchronize(st);
        free_dgraph(g.release());
        return rc;
    }
    *out = g.release();
    return GP_OK;
}

gp_status gp_dgraph_stats(const gp_dgraph* g, int64_t* n, int64_t* narcs) {
    if (!g) return gp::dfail(GP_ERR_ARG, "gp_dgraph_stats: null graph");
    if (n) *n = g->n;
    if (narcs) *narcs = g->narcs;
    return GP_OK;
}

gp_status gp_dgraph_copy(const gp_dgraph* g, int64_t* out_ptr, int32_t* out_col, int64_t* in_ptr,
                         int32_t* in_col) {
    using namespace gp;
    if (!g) return dfail(GP_ERR_ARG, "gp_dgraph_copy: null graph");
    const size_t pb = sizeof(int64_t) * ((size_t)g->n + 1), cb = sizeof(int32_t) * (size_t)g->narcs;
    if (out_ptr) GP_CUDA_TRY(cudaMemcpy(out_ptr, g->out_ptr, pb, cudaMemcpyDeviceToHost));
    if (in_ptr) GP_CUDA_TRY(cudaMemcpy(in_ptr, g->in_ptr, pb, cudaMemcpyDeviceToHost));
    if (out_col && cb) GP_CUDA_TRY(cudaMemcpy(out_col, g->out_col, cb, cudaMemcpyDeviceToHost));
    if (in_col && cb) GP_CUDA_TRY(cudaMemcpy(in_col, g->in_col, cb, cudaMemcpyDeviceToHost));
    return GP_OK;
}

void gp_dgraph_destroy(gp_dgraph* g) { gp::free_dgraph(g); }

gp_status gp_dpattern_create(const uint8_t* adj, int32_t k, gp_dpattern** out) {
    using namespace gp;
    if (!adj || !out) return dfail(GP_ERR_ARG, "gp_dpattern_create: null argument");
    *out = nullptr;
    if (k < 3 || k > GP_MAX_K) return dfail(GP_ERR_PATTERN, "directed pattern needs 3 to 7 vertices");
    std::unique_ptr<gp_dpattern> p(new (std::nothrow) gp_dpattern);
    if (!p) return dfail(GP_ERR_NOMEM, "gp_dpattern_create: out of host memory");
    p->k = k;
    uint8_t und[GP_MAX_K * GP_MAX_K] = {};
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) {
            const uint8_t x = adj[a * k + b];
            if (x > 1 || (a == b && x)) return dfail(GP_ERR_PATTERN, "arcs must be 0/1 with a zero diagonal");
            p->arc[a][b] = x;
        }
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) und[a * k + b] = (p->arc[a][b] || p->arc[b][a]) ? 1 : 0;
    std::string err;
    if (!pattern_init(p->info, und, k, err)) return dfail(GP_ERR_PATTERN, err.c_str());   // weakly connected
    // the group: permutations of the underlying pattern that also keep every arc
    std::vector<Perm> keep;
    for (const Perm& q : p->info.auts) {
        bool ok = true;
        for (int a = 0; a < k && ok; ++a)
            for (int b = 0; b < k && ok; ++b)
                if (p->arc[a][b] && !p->arc[q[a]][q[b]]) ok = false;
        if (ok) keep.push_back(q);
    }
    p->info.auts = keep;
    *out = p.release();
    return GP_OK;
}

gp_status gp_dpattern_aut_count(const gp_dpattern* p, uint64_t* out) {
    if (!p || !out) return gp::dfail(GP_ERR_ARG, "gp_dpattern_aut_count: null argument");
    *out = (uint64_t)p->info.auts.size();
    return GP_OK;
}

void gp_dpattern_destroy(gp_dpattern* p) { delete p; }

gp_status gp_dcount(const gp_dgraph* g, gp_dpattern* p, const int32_t* order, const int32_t* restr,
                    int32_t n_restr, void* stream, uint64_t* out) {
    using namespace gp;
    if (!g || !p || !out || (order == nullptr && n_restr > 0) || n_restr < 0 || (n_restr > 0 && !restr))
        return dfail(GP_ERR_ARG, "gp_dcount: bad arguments");
    const int k = p->k;
    int8_t sched[GP_MAX_K];
    ResMask res = 0;
    uint64_t div = 1;
    if (order) {
        for (int d = 0; d < k; ++d) {
            if (order[d] < 0 || order[d] >= k) return dfail(GP_ERR_ARG, "gp_dcount: order out of range");
            sched[d] = (int8_t)order[d];
        }
        for (int r = 0; r < n_restr; ++r) {
            const int a = restr[2 * r], b = restr[2 * r + 1];
            if (a < 0 || a >= k || b < 0 || b >= k || a == b) return dfail(GP_ERR_ARG, "gp_dcount: bad restriction");
            res |= (ResMask)1 << res_bit(a, b);
        }
        if (n_restr == 0) div = (uint64_t)p->info.auts.size();
        else if (!validate_set(p->info, res))
            return dfail(GP_ERR_PATTERN, "gp_dcount: the restrictions do not identify each embedding once");
    } else {
        // the performance model's first choice among the efficient schedules
        // and Algorithm 1's sets, for the underlying pattern on a graph of
        // this size (triangle rate of the library's default statistics);
        // no set: no restrictions, divide by |Aut|
        const double V = (double)std::max<int32_t>(g->n, 1), E = (double)std::max<int64_t>(g->narcs, 1);
        std::vector<Config> cfg = rank_configs(p->info, V, E, 6.0 * E, 1);
        if (!cfg.empty()) {
            for (int d = 0; d < k; ++d) sched[d] = cfg[0].sched[d];
            res = cfg[0].res;
        } else {
            int kp = 0;
            const std::vector<Perm>& sc = efficient_schedules(p->info, &kp);
            if (sc.empty()) return dfail(GP_ERR_INTERNAL, "gp_dcount: no schedule");
            for (int d = 0; d < k; ++d) sched[d] = sc[0][d];
            div = (uint64_t)p->info.auts.size();
        }
    }
    DPlan P;
    std::string err;
    if (!compile_dplan(*p, sched, res, &P, err)) return dfail(GP_ERR_PATTERN, err.c_str());
    int cur = 0;
    GP_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != g->device) return dfail(GP_ERR_ARG, "gp_dcount: graph lives on another device");
    return run_dcount(g, P, div, dstream(stream), out);
}

}  // extern "C"
