// graph.cu -- device-side graph preprocessing: drop self loops, insert both
// directions, sort, deduplicate, optionally relabel by degree, and lay the
// result out as CSR with sorted neighbour lists (GraphPi Section IV-E).
//
// Each directed pair (u, v) travels as one 64-bit key (u << 32) | v, so a
// single radix sort orders the pairs by source and then by target, which is
// exactly the CSR order. The sort and the unique pass are CUB library calls.
#include <algorithm>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_select.cuh>

#include "engine.h"

namespace gp {

namespace {

constexpr int kThreads = 256;

inline int blocks_for(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    return (int)(b < 1 ? 1 : (b > (1 << 30) ? (1 << 30) : b));
}

int bits_for(uint64_t x) {     // bits needed to represent x
    int b = 0;
    while (b < 64 && (x >> b)) ++b;
    return b;
}

__global__ void k_check_ids(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                            int64_t m, int32_t n, int* __restrict__ bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t u = src[i], v = dst[i];
        if (u < 0 || u >= n || v < 0 || v >= n) atomicExch(bad, 1);
    }
}

// Pair i yields keys 2i (u -> v) and 2i + 1 (v -> u); a self loop yields two
// copies of the sentinel n << 32, which sorts after every real key.
__global__ void k_make_keys(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                            int64_t m, int32_t n, uint64_t* __restrict__ keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t u = (uint32_t)src[i], v = (uint32_t)dst[i];
        uint64_t a = (u << 32) | v, b = (v << 32) | u;
        if (u == v) a = b = (uint64_t)(uint32_t)n << 32;
        keys[2 * i] = a;
        keys[2 * i + 1] = b;
    }
}

// row_ptr[u] = first key whose source is >= u (binary search in sorted keys).
__global__ void k_row_ptr(const uint64_t* __restrict__ keys, int64_t nnz, int32_t n,
                          int64_t* __restrict__ row_ptr) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u <= n;
         u += (int64_t)gridDim.x * blockDim.x) {
        uint64_t target = (uint64_t)u << 32;
        int64_t lo = 0, hi = nnz;
        while (lo < hi) {
            int64_t mid = lo + ((hi - lo) >> 1);
            if (keys[mid] < target) lo = mid + 1; else hi = mid;
        }
        row_ptr[u] = lo;
    }
}

__global__ void k_col(const uint64_t* __restrict__ keys, int64_t nnz, int32_t* __restrict__ col) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz;
         i += (int64_t)gridDim.x * blockDim.x)
        col[i] = (int32_t)(uint32_t)keys[i];
}

__global__ void k_max_deg(const int64_t* __restrict__ row_ptr, int32_t n, int* __restrict__ out) {
    int best = 0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x)
        best = max(best, (int)(row_ptr[u + 1] - row_ptr[u]));
    for (int o = 16; o; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

// Degree-order key: (max_deg - deg) in the high half sorts high degrees first,
// the vertex id in the low half breaks ties by id.
__global__ void k_degree_keys(const int64_t* __restrict__ row_ptr, int32_t n, int32_t max_deg,
                              uint64_t* __restrict__ keys) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        uint64_t deg = (uint64_t)(row_ptr[u + 1] - row_ptr[u]);
        keys[u] = (((uint64_t)max_deg - deg) << 32) | (uint64_t)u;
    }
}

__global__ void k_perm_from_keys(const uint64_t* __restrict__ keys, int32_t n,
                                 int32_t* __restrict__ new2old, int32_t* __restrict__ old2new) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t old = (int32_t)(uint32_t)keys[i];
        new2old[i] = old;
        old2new[old] = (int32_t)i;
    }
}

// Entry e of row u becomes key (old2new[u] << 32) | old2new[col[e]].
__global__ void k_relabel_keys(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                               int32_t n, int64_t nnz, const int32_t* __restrict__ old2new,
                               uint64_t* __restrict__ keys) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n;                 // row of e: last u with row_ptr[u] <= e
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) >> 1;
            if (row_ptr[mid] <= e) lo = mid; else hi = mid;
        }
        keys[e] = ((uint64_t)(uint32_t)old2new[lo] << 32) | (uint32_t)old2new[col[e]];
    }
}

__global__ void k_pairs_from_csr(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                 int32_t n, int64_t nnz, int32_t* __restrict__ src,
                                 int32_t* __restrict__ dst) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n;
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) >> 1;
            if (row_ptr[mid] <= e) lo = mid; else hi = mid;
        }
        src[e] = (int32_t)lo;
        dst[e] = col[e];
    }
}

// Stream-ordered scratch that is released on every exit path.
struct Scratch {
    cudaStream_t st;
    void* p = nullptr;
    explicit Scratch(cudaStream_t s) : st(s) {}
    ~Scratch() { if (p) cudaFreeAsync(p, st); }
    cudaError_t alloc(size_t bytes) { return cudaMallocAsync(&p, bytes ? bytes : 16, st); }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// Sorted unique keys -> (row_ptr, col) allocated into g.
gp_status keys_to_csr(const uint64_t* d_keys, int64_t nnz, int32_t n, cudaStream_t st, gp_graph* g) {
    int64_t* row_ptr = nullptr;
    int32_t* col = nullptr;
    GP_CUDA_TRY(cudaMalloc(&row_ptr, sizeof(int64_t) * ((size_t)n + 1)));
    if (cudaMalloc(&col, sizeof(int32_t) * (size_t)(nnz ? nnz : 1)) != cudaSuccess) {
        cudaFree(row_ptr);
        set_error("cudaMalloc of %lld column ids failed", (long long)nnz);
        return GP_ERR_NOMEM;
    }
    k_row_ptr<<<blocks_for((int64_t)n + 1), kThreads, 0, st>>>(d_keys, nnz, n, row_ptr);
    if (nnz) k_col<<<blocks_for(nnz), kThreads, 0, st>>>(d_keys, nnz, col);
    count_launch(nnz ? 2 : 1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaFree(row_ptr); cudaFree(col);
        set_error("CSR kernels failed: %s", cudaGetErrorString(e));
        return GP_ERR_CUDA;
    }
    g->row_ptr = row_ptr;
    g->col = col;
    g->nnz = nnz;
    g->n = n;
    return GP_OK;
}

// One thread: binary search for the first vertex of degree < min_deg.
__global__ void k_heavy_prefix(const int64_t* __restrict__ row_ptr, int32_t n, int32_t min_deg,
                               int64_t* __restrict__ out) {
    int32_t lo = 0, hi = n;
    while (lo < hi) {
        int32_t mid = lo + ((hi - lo) >> 1);
        if (row_ptr[mid + 1] - row_ptr[mid] >= min_deg) lo = mid + 1; else hi = mid;
    }
    *out = row_ptr[lo];
}

// One warp per core vertex u: set bit x of row u for every neighbour x of u
// below core_n (a prefix of u's sorted list).
__global__ void k_core_bits(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            int32_t core_n, int32_t words, uint32_t* __restrict__ bits) {
    const int lane = threadIdx.x & 31;
    for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < core_n;
         u += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t b = row_ptr[u], e = row_ptr[u + 1];
        for (int64_t i = b + lane; i < e; i += 32) {
            const int32_t x = col[i];
            if (x >= core_n) break;
            atomicOr(bits + u * words + (x >> 5), 1u << (x & 31));
        }
    }
}

}  // namespace

gp_status build_core_bits(gp_graph* g, int32_t core_n, cudaStream_t st) {
    if (core_n <= 0) return GP_OK;
    // rows padded to a multiple of 4 words: 16-byte loads stay aligned
    const int32_t words = (((core_n + 31) / 32) + 3) & ~3;
    const size_t bytes = sizeof(uint32_t) * (size_t)core_n * (size_t)words;
    uint32_t* bits = nullptr;
    GP_CUDA_TRY(cudaMalloc(&bits, bytes));
    cudaError_t e = cudaMemsetAsync(bits, 0, bytes, st);
    if (e == cudaSuccess) {
        const int blocks = (int)std::min<int64_t>(((int64_t)core_n * 32 + kThreads - 1) / kThreads, 4096);
        k_core_bits<<<blocks, kThreads, 0, st>>>(g->row_ptr, g->col, core_n, words, bits);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(bits);
        set_error("core bit matrix: %s", cudaGetErrorString(e));
        return GP_ERR_CUDA;
    }
    g->core_bits = bits;
    g->core_n = core_n;
    g->core_words = words;
    return GP_OK;
}

gp_status heavy_prefix(const int64_t* d_row_ptr, int32_t n, int32_t min_deg, cudaStream_t st,
                       int64_t* out) {
    Scratch s(st);
    GP_CUDA_TRY(s.alloc(sizeof(int64_t)));
    k_heavy_prefix<<<1, 1, 0, st>>>(d_row_ptr, n, min_deg, s.as<int64_t>());
    count_launch();
    GP_CUDA_TRY(cudaGetLastError());
    int64_t h = 0;
    GP_CUDA_TRY(cudaMemcpyAsync(&h, s.p, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    GP_CUDA_TRY(cudaStreamSynchronize(st));
    *out = h;
    return GP_OK;
}

gp_status max_degree(const int64_t* d_row_ptr, int32_t n, cudaStream_t st, int32_t* out) {
    Scratch s(st);
    GP_CUDA_TRY(s.alloc(sizeof(int)));
    GP_CUDA_TRY(cudaMemsetAsync(s.p, 0, sizeof(int), st));
    if (n > 0) {
        int blocks = blocks_for(n);
        if (blocks > 4096) blocks = 4096;
        k_max_deg<<<blocks, kThreads, 0, st>>>(d_row_ptr, n, s.as<int>());
        count_launch();
        GP_CUDA_TRY(cudaGetLastError());
    }
    int h = 0;
    GP_CUDA_TRY(cudaMemcpyAsync(&h, s.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    GP_CUDA_TRY(cudaStreamSynchronize(st));
    *out = h;
    return GP_OK;
}

gp_status csr_to_pairs(const int64_t* d_row_ptr, const int32_t* d_col, int32_t n, int64_t nnz,
                       int32_t* d_src, int32_t* d_dst, cudaStream_t st) {
    if (nnz == 0) return GP_OK;
    k_pairs_from_csr<<<blocks_for(nnz), kThreads, 0, st>>>(d_row_ptr, d_col, n, nnz, d_src, d_dst);
    count_launch();
    GP_CUDA_TRY(cudaGetLastError());
    return GP_OK;
}

gp_status build_graph(const int32_t* d_src, const int32_t* d_dst, int64_t m, int32_t n,
                      bool degree_order, cudaStream_t st, gp_graph* g) {
    // 1. ids in range
    {
        Scratch bad(st);
        GP_CUDA_TRY(bad.alloc(sizeof(int)));
        GP_CUDA_TRY(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
        if (m > 0) {
            k_check_ids<<<blocks_for(m), kThreads, 0, st>>>(d_src, d_dst, m, n, bad.as<int>());
            count_launch();
            GP_CUDA_TRY(cudaGetLastError());
        }
        int h = 0;
        GP_CUDA_TRY(cudaMemcpyAsync(&h, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        GP_CUDA_TRY(cudaStreamSynchronize(st));
        if (h) { set_error("edge endpoint outside [0, %d)", n); return GP_ERR_ARG; }
    }
    const int64_t nkeys = 2 * m;
    const int end_bit = 32 + bits_for((uint64_t)(uint32_t)n);
    Scratch keys_a(st), keys_b(st), nsel(st), temp(st);
    GP_CUDA_TRY(keys_a.alloc(sizeof(uint64_t) * (size_t)nkeys));
    GP_CUDA_TRY(keys_b.alloc(sizeof(uint64_t) * (size_t)nkeys));
    GP_CUDA_TRY(nsel.alloc(sizeof(int64_t)));
    int64_t nnz = 0;
    if (m > 0) {
        // 2-3. both directions as 64-bit keys, self loops to the sentinel
        k_make_keys<<<blocks_for(m), kThreads, 0, st>>>(d_src, d_dst, m, n, keys_a.as<uint64_t>());
        count_launch();
        GP_CUDA_TRY(cudaGetLastError());
        // 4. radix sort (CUB)
        size_t tbytes = 0, tbytes2 = 0;
        GP_CUDA_TRY(cub::DeviceRadixSort::SortKeys(nullptr, tbytes, keys_a.as<uint64_t>(),
                                                   keys_b.as<uint64_t>(), nkeys, 0, end_bit, st));
        GP_CUDA_TRY(cub::DeviceSelect::Unique(nullptr, tbytes2, keys_b.as<uint64_t>(),
                                              keys_a.as<uint64_t>(), nsel.as<int64_t>(), nkeys, st));
        GP_CUDA_TRY(temp.alloc(tbytes > tbytes2 ? tbytes : tbytes2));
        GP_CUDA_TRY(cub::DeviceRadixSort::SortKeys(temp.p, tbytes, keys_a.as<uint64_t>(),
                                                   keys_b.as<uint64_t>(), nkeys, 0, end_bit, st));
        // 5. unique
        GP_CUDA_TRY(cub::DeviceSelect::Unique(temp.p, tbytes2, keys_b.as<uint64_t>(),
                                              keys_a.as<uint64_t>(), nsel.as<int64_t>(), nkeys, st));
        count_launch(2);
        int64_t h = 0;
        GP_CUDA_TRY(cudaMemcpyAsync(&h, nsel.p, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        uint64_t last = 0;
        GP_CUDA_TRY(cudaStreamSynchronize(st));
        if (h > 0) {
            GP_CUDA_TRY(cudaMemcpyAsync(&last, keys_a.as<uint64_t>() + (h - 1), sizeof(uint64_t),
                                        cudaMemcpyDeviceToHost, st));
            GP_CUDA_TRY(cudaStreamSynchronize(st));
        }
        nnz = h - ((h > 0 && last == ((uint64_t)(uint32_t)n << 32)) ? 1 : 0);
    }
    // 7. CSR from the sorted unique keys
    gp_status rc = keys_to_csr(keys_a.as<uint64_t>(), nnz, n, st, g);
    if (rc != GP_OK) return rc;
    rc = max_degree(g->row_ptr, n, st, &g->max_deg);
    if (rc != GP_OK) return rc;
    if (!degree_order || n == 0) return GP_OK;

    // 6. relabel by non-increasing degree, then rebuild the CSR
    Scratch vkeys(st), vkeys2(st), old2new(st), temp2(st);
    int32_t* new2old = nullptr;
    GP_CUDA_TRY(vkeys.alloc(sizeof(uint64_t) * (size_t)n));
    GP_CUDA_TRY(vkeys2.alloc(sizeof(uint64_t) * (size_t)n));
    GP_CUDA_TRY(old2new.alloc(sizeof(int32_t) * (size_t)n));
    GP_CUDA_TRY(cudaMalloc(&new2old, sizeof(int32_t) * (size_t)n));
    k_degree_keys<<<blocks_for(n), kThreads, 0, st>>>(g->row_ptr, n, g->max_deg, vkeys.as<uint64_t>());
    count_launch();
    size_t tb = 0, tb2 = 0;
    const int vend = 32 + bits_for((uint64_t)g->max_deg);
    GP_CUDA_TRY(cub::DeviceRadixSort::SortKeys(nullptr, tb, vkeys.as<uint64_t>(), vkeys2.as<uint64_t>(),
                                               (int64_t)n, 0, vend, st));
    if (nnz > 0)
        GP_CUDA_TRY(cub::DeviceRadixSort::SortKeys(nullptr, tb2, keys_b.as<uint64_t>(),
                                                   keys_a.as<uint64_t>(), nnz, 0, end_bit, st));
    GP_CUDA_TRY(temp2.alloc(tb > tb2 ? tb : tb2));
    GP_CUDA_TRY(cub::DeviceRadixSort::SortKeys(temp2.p, tb, vkeys.as<uint64_t>(), vkeys2.as<uint64_t>(),
                                               (int64_t)n, 0, vend, st));
    k_perm_from_keys<<<blocks_for(n), kThreads, 0, st>>>(vkeys2.as<uint64_t>(), n, new2old,
                                                         old2new.as<int32_t>());
    count_launch(2);
    if (nnz > 0) {
        k_relabel_keys<<<blocks_for(nnz), kThreads, 0, st>>>(g->row_ptr, g->col, n, nnz,
                                                             old2new.as<int32_t>(), keys_b.as<uint64_t>());
        GP_CUDA_TRY(cub::DeviceRadixSort::SortKeys(temp2.p, tb2, keys_b.as<uint64_t>(),
                                                   keys_a.as<uint64_t>(), nnz, 0, end_bit, st));
        count_launch(2);
    }
    GP_CUDA_TRY(cudaGetLastError());
    GP_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(g->row_ptr);
    cudaFree(g->col);
    g->row_ptr = nullptr;
    g->col = nullptr;
    rc = keys_to_csr(keys_a.as<uint64_t>(), nnz, n, st, g);
    if (rc != GP_OK) { cudaFree(new2old); return rc; }
    g->perm = new2old;
    rc = heavy_prefix(g->row_ptr, n, kHeavyDegree, st, &g->heavy_end);
    if (rc != GP_OK) return rc;
    return build_core_bits(g, std::min(n, kCoreMax), st);
}

}  // namespace gp
