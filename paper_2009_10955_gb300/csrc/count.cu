// count.cu -- the pattern-count kernel: a persistent, warp-per-task
// interpreter of the nested-loop search of GraphPi (Sections II-B, IV-B,
// IV-E), for sm_103a.
//
// Work decomposition (Section IV-E, fine-grained tasks + work stealing):
// every directed CSR entry (v0, v1) is one task that fixes the first two
// loops. Tasks of all jobs form one global index space; a warp grabs a chunk
// of consecutive tasks with one atomicAdd on a global cursor, so idle warps
// take the next work immediately (the device analogue of stealing).
//
// Inside a task one warp runs the remaining loops depth-first. Candidate
// sets are intersections of sorted neighbour lists, clipped to the window the
// restrictions impose (a restriction becomes a bound on a sorted list, the
// "break" of Section IV-B). Intersections are warp-cooperative: each lane
// takes one element of the shorter list and binary-searches it in the longer
// one, and ballot/popc compacts the matches. The innermost loop is never
// enumerated: its contribution is the size of its clipped candidate set
// minus the already-matched vertices inside it.
//
// Counts are accumulated per lane in 128 bits and reduced with warp shuffles;
// one atomic pair (low word, carry into the high word) per warp per job
// publishes them.
#include <algorithm>
#include <climits>
#include <vector>

#include "engine.h"

namespace gp {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = 8;   // warps per block
static_assert(sizeof(GpPlan) % 4 == 0, "plan is copied as 32-bit words");

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// First index i in [0, n) with a[i] >= x (n if none).
__device__ __forceinline__ int lower_bound(const int32_t* __restrict__ a, int n, int x) {
    int base = 0;
    while (n > 0) {
        int half = n >> 1;
        if (__ldg(a + base + half) < x) { base += half + 1; n -= half + 1; }
        else n = half;
    }
    return base;
}

// Algorithmic bytes of intersecting sorted lists of lengths na and nb: the
// cheaper of a merge (4 bytes per element of both) and a binary search of
// each element of the shorter list in the longer one, counted in 32-byte
// sectors (eight ids per sector, so about log2(n / 8) + 1 sectors a search).
__device__ __forceinline__ unsigned long long intersect_bytes(int na, int nb) {
    const int sh = min(na, nb), lo = max(na, nb);
    const unsigned long long merge = 4ull * (unsigned long long)(na + nb);
    const int sectors = (lo > 8) ? (32 - __clz((lo >> 3) | 1)) + 1 : 1;
    const unsigned long long search = (unsigned long long)sh * (4ull + 32ull * (unsigned long long)sectors);
    return merge < search ? merge : search;
}

struct Acc {   // per-lane 128-bit counter
    unsigned long long lo = 0, hi = 0;
    __device__ __forceinline__ void add(unsigned long long x) { lo += x; hi += (lo < x); }
    __device__ __forceinline__ void sub(unsigned long long x) { hi -= (lo < x); lo -= x; }
};

__device__ void flush(Acc& acc, unsigned long long* res) {
    unsigned long long lo = acc.lo, hi = acc.hi;
    for (int o = 16; o; o >>= 1) {
        unsigned long long l2 = __shfl_down_sync(kFull, lo, o);
        unsigned long long h2 = __shfl_down_sync(kFull, hi, o);
        lo += l2;
        hi += h2 + (lo < l2);
    }
    if ((threadIdx.x & 31) == 0 && (lo | hi)) {
        unsigned long long old = atomicAdd(res, lo);
        unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
        if (hi + carry) atomicAdd(res + 1, hi + carry);
    }
    acc.lo = acc.hi = 0;
}

// Warp-cooperative sorted intersection of A and B. Writes the (sorted)
// result to out when out != nullptr and returns its size (warp-uniform).
// With acc != nullptr each lane also adds its own matches to acc.
__device__ __forceinline__ int warp_intersect(const int32_t* __restrict__ A, int na,
                                              const int32_t* __restrict__ B, int nb,
                                              int32_t* __restrict__ out, int cap, Acc* acc,
                                              int lane, int* err, unsigned long long* sbytes) {
    if (na > nb) {
        const int32_t* t = A; A = B; B = t;
        int tn = na; na = nb; nb = tn;
    }
    int total = 0, from = 0;
    for (int base = 0; base < na; base += 32) {
        int i = base + lane;
        int x = 0, pos = nb;
        bool f = false;
        if (i < na) {
            x = __ldg(A + i);
            pos = from + lower_bound(B + from, nb - from, x);
            f = pos < nb && __ldg(B + pos) == x;
        }
        unsigned m = __ballot_sync(kFull, f);
        if (out && f) {
            int at = total + __popc(m & lanemask_lt());
            if (at < cap) out[at] = x; else atomicExch(err, 2);
        }
        if (acc && f) acc->add(1);
        total += __popc(m);
        int last = min(31, na - 1 - base);
        from = __shfl_sync(kFull, pos, last);   // later elements are larger
    }
    if (sbytes && lane == 0)
        *sbytes += intersect_bytes(na, nb) + (out ? 4ull * (unsigned long long)total : 0ull);
    return total;
}

struct Window { int lo, hi; };   // candidates c with lo < c < hi

__device__ __forceinline__ Window window(uint8_t lo_mask, uint8_t hi_mask, const int* v) {
    Window w{-1, INT_MAX};
    for (int j = 0; j < GP_MAX_K; ++j) {
        if (lo_mask >> j & 1) w.lo = max(w.lo, v[j]);
        if (hi_mask >> j & 1) w.hi = min(w.hi, v[j]);
    }
    return w;
}

// Clip a sorted list to a window: returns [b, e).
__device__ __forceinline__ void clip(const int32_t* a, int n, Window w, int& b, int& e) {
    b = (w.lo < 0) ? 0 : lower_bound(a, n, w.lo + 1);
    e = (w.hi == INT_MAX) ? n : lower_bound(a, n, w.hi);
    if (e < b) e = b;
}

struct TaskCtx {
    const GpPlan* P;
    const int64_t* __restrict__ row_ptr;
    const int32_t* __restrict__ col;
    int32_t* slots;        // this warp's intermediate sets
    int slot_cap;
    int n_vertices;
    int* slen;             // their lengths (shared memory, per warp)
    int lane;
    int* err;
    unsigned long long* sbytes;   // algorithmic-byte tally (instrumented kernel only)
};

__device__ __forceinline__ void nbr(const TaskCtx& c, int v, const int32_t*& p, int& n) {
    int64_t b = __ldg(c.row_ptr + v), e = __ldg(c.row_ptr + v + 1);
    p = c.col + b;
    n = (int)(e - b);
}

__device__ __forceinline__ void run_builds(const TaskCtx& c, int d, const int* v) {
    const GpLevel& L = c.P->lvl[d];
    for (int q = 0; q < L.nbuild; ++q) {
        const GpBuild& B = L.build[q];
        const int32_t* a; int na;
        if (B.base_kind == 1) nbr(c, v[B.base], a, na);
        else { a = c.slots + (size_t)B.base * c.slot_cap; na = c.slen[B.base]; }
        const int32_t* b; int nb;
        nbr(c, v[d], b, nb);
        Window w = window(B.lo_mask, B.hi_mask, v);
        int a0, a1, b0, b1;
        clip(a, na, w, a0, a1);
        clip(b, nb, w, b0, b1);
        int32_t* out = c.slots + (size_t)B.dst * c.slot_cap;
        int n = warp_intersect(a + a0, a1 - a0, b + b0, b1 - b0, out, c.slot_cap, nullptr, c.lane, c.err,
                               c.sbytes);
        if (c.lane == 0) c.slen[B.dst] = n;
        __syncwarp();
    }
}

// Is x in the sorted list a[0, n)?
__device__ __forceinline__ bool contains(const int32_t* a, int n, int x) {
    int p = lower_bound(a, n, x);
    return p < n && __ldg(a + p) == x;
}

// Contribution of the innermost loop given v[0..k-2].
__device__ __forceinline__ void count_last(const TaskCtx& c, const int* v, Acc& acc) {
    const GpPlan& P = *c.P;
    const int L = P.k - 1;
    const GpLevel& lv = P.lvl[L];
    Window w = window(lv.lo_mask, lv.hi_mask, v);
    if (P.last_count_only) {
        const int32_t* a; int na;
        if (P.last_base_kind == 1) nbr(c, v[P.last_base], a, na);
        else { a = c.slots + (size_t)P.last_base * c.slot_cap; na = c.slen[P.last_base]; }
        const int32_t* b; int nb;
        nbr(c, v[L - 1], b, nb);
        int a0, a1, b0, b1;
        clip(a, na, w, a0, a1);
        clip(b, nb, w, b0, b1);
        warp_intersect(a + a0, a1 - a0, b + b0, b1 - b0, nullptr, 0, &acc, c.lane, c.err, c.sbytes);
        // matched vertices inside the intersection are not new vertices
        bool hit = false;
        if (c.lane < L && (lv.excl_mask >> c.lane & 1)) {
            int x = v[c.lane];
            hit = x > w.lo && x < w.hi && contains(a + a0, a1 - a0, x) && contains(b + b0, b1 - b0, x);
        }
        unsigned h = __ballot_sync(kFull, hit);
        if (c.lane == 0) acc.sub(__popc(h));
    } else {
        const int32_t* a; int na;
        if (lv.src_kind == 1) nbr(c, v[lv.src], a, na);
        else { a = c.slots + (size_t)lv.src * c.slot_cap; na = c.slen[lv.src]; }
        int a0, a1;
        clip(a, na, w, a0, a1);
        bool hit = false;
        if (c.lane < L && (lv.excl_mask >> c.lane & 1)) {
            int x = v[c.lane];
            hit = x > w.lo && x < w.hi && contains(a + a0, a1 - a0, x);
        }
        unsigned h = __ballot_sync(kFull, hit);
        if (c.lane == 0) acc.add((unsigned long long)(a1 - a0) - __popc(h));
    }
}

// Per-lane sorted intersection size: binary search of the shorter list in
// the longer when their lengths differ a lot, a linear merge otherwise.
__device__ __forceinline__ int lane_intersect_count(const int32_t* __restrict__ A, int na,
                                                    const int32_t* __restrict__ B, int nb) {
    if (na > nb) {
        const int32_t* t = A; A = B; B = t;
        int tn = na; na = nb; nb = tn;
    }
    int cnt = 0;
    if (na == 0) return 0;
    if (nb > 16 * na) {
        int from = 0;
        for (int i = 0; i < na && from < nb; ++i) {
            int x = __ldg(A + i);
            from += lower_bound(B + from, nb - from, x);
            cnt += (from < nb && __ldg(B + from) == x);
        }
        return cnt;
    }
    int i = 0, j = 0;
    int x = __ldg(A), y = __ldg(B);
    for (;;) {
        if (x == y) {
            ++cnt;
            if (++i == na || ++j == nb) break;
            x = __ldg(A + i);
            y = __ldg(B + j);
        } else if (x < y) {
            if (++i == na) break;
            x = __ldg(A + i);
        } else {
            if (++j == nb) break;
            y = __ldg(B + j);
        }
    }
    return cnt;
}

// Work above which a lane hands its last-level count to the whole warp.
constexpr int kLaneWork = 192;

// Per-lane version of count_last: v[] is this lane's own matched vertices.
// Returns false (and counts nothing) when the work is large enough that the
// warp-cooperative count_last should take it.
__device__ __forceinline__ bool count_last_lane(const TaskCtx& c, const int* v, Acc& acc) {
    const GpPlan& P = *c.P;
    const int L = P.k - 1;
    const GpLevel& lv = P.lvl[L];
    Window w = window(lv.lo_mask, lv.hi_mask, v);
    if (P.last_count_only) {
        const int32_t* a; int na;
        if (P.last_base_kind == 1) nbr(c, v[P.last_base], a, na);
        else { a = c.slots + (size_t)P.last_base * c.slot_cap; na = c.slen[P.last_base]; }
        const int32_t* b; int nb;
        nbr(c, v[L - 1], b, nb);
        int a0, a1, b0, b1;
        clip(a, na, w, a0, a1);
        clip(b, nb, w, b0, b1);
        const int la = a1 - a0, lb = b1 - b0;
        const int sh = min(la, lb), lo = max(la, lb);
        const int work = (lo > 16 * sh) ? sh * (32 - __clz(lo | 1)) : la + lb;
        if (work > kLaneWork) return false;
        int cnt = lane_intersect_count(a + a0, la, b + b0, lb);
        for (int j = 0; j < L; ++j) {
            if (!(lv.excl_mask >> j & 1)) continue;
            int x = v[j];
            if (x > w.lo && x < w.hi && contains(a + a0, la, x) && contains(b + b0, lb, x)) --cnt;
        }
        acc.add((unsigned long long)cnt);
        if (c.sbytes) *c.sbytes += intersect_bytes(la, lb);
        return true;
    }
    const int32_t* a; int na;
    if (lv.src_kind == 1) nbr(c, v[lv.src], a, na);
    else { a = c.slots + (size_t)lv.src * c.slot_cap; na = c.slen[lv.src]; }
    int a0, a1;
    clip(a, na, w, a0, a1);
    int cnt = a1 - a0;
    for (int j = 0; j < L; ++j) {
        if (!(lv.excl_mask >> j & 1)) continue;
        int x = v[j];
        if (x > w.lo && x < w.hi && contains(a + a0, a1 - a0, x)) --cnt;
    }
    acc.add((unsigned long long)cnt);
    return true;
}

// The loop at depth k-2 with one candidate per lane: every lane counts the
// last level for its own candidate; candidates with heavy intersections are
// then counted one at a time by the whole warp.
__device__ __forceinline__ void lane_parallel_last_two(const TaskCtx& c, int* v, const int32_t* lst,
                                                       int beg, int end, Acc& acc) {
    const GpPlan& P = *c.P;
    const int d = P.k - 2;
    const uint8_t ex = P.lvl[d].excl_mask;
    for (int base = beg; base < end; base += 32) {
        const int i = base + c.lane;
        int x = -1;
        bool active = i < end;
        if (active) {
            x = __ldg(lst + i);
            for (int j = 0; j < d; ++j) active &= !(((ex >> j) & 1) && v[j] == x);
            if (c.sbytes) *c.sbytes += 4;
        }
        bool deferred = false;
        if (active) {
            v[d] = x;
            deferred = !count_last_lane(c, v, acc);
        }
        unsigned dm = __ballot_sync(kFull, deferred);
        while (dm) {
            const int src = __ffs(dm) - 1;
            dm &= dm - 1;
            v[d] = __shfl_sync(kFull, x, src);
            count_last(c, v, acc);
        }
    }
}

// Remaining loops of one edge task (v0, v1).
__device__ void run_task(const TaskCtx& c, int v0, int v1, Acc& acc) {
    const GpPlan& P = *c.P;
    const int k = P.k;
    int v[GP_MAX_K];
    const int32_t* lst[GP_MAX_K];
    int cur[GP_MAX_K], end[GP_MAX_K];
#pragma unroll
    for (int i = 0; i < GP_MAX_K; ++i) v[i] = -1;
    v[0] = v0;
    v[1] = v1;
    run_builds(c, 1, v);
    if (k == 3) { count_last(c, v, acc); return; }
    int d = 2;
    auto prepare = [&](int dd) {
        const GpLevel& L = P.lvl[dd];
        const int32_t* a; int na;
        if (L.src_kind == 1) nbr(c, v[L.src], a, na);
        else { a = c.slots + (size_t)L.src * c.slot_cap; na = c.slen[L.src]; }
        clip(a, na, window(L.lo_mask, L.hi_mask, v), cur[dd], end[dd]);
        lst[dd] = a;
    };
    const bool lane_last = P.lvl[k - 2].nbuild == 0;
    prepare(2);
    while (d >= 2) {
        if (lane_last && d == k - 2) {
            lane_parallel_last_two(c, v, lst[d], cur[d], end[d], acc);
            --d;
            continue;
        }
        if (cur[d] >= end[d]) { --d; continue; }
        int x = __ldg(lst[d] + cur[d]);
        ++cur[d];
        if (c.sbytes && c.lane == 0) *c.sbytes += 4;
        uint8_t ex = P.lvl[d].excl_mask;
        bool skip = false;
        for (int j = 0; j < d; ++j) skip |= ((ex >> j) & 1) && v[j] == x;
        if (skip) continue;
        v[d] = x;
        run_builds(c, d, v);
        if (d == k - 2) count_last(c, v, acc);
        else { ++d; prepare(d); }
    }
}

template <bool kStats, int kMinBlocks>
__global__ void __launch_bounds__(kWarps * 32, kMinBlocks)
k_count(const CountJob* __restrict__ jobs, int njobs, int64_t total,
        unsigned long long* __restrict__ cursor, unsigned long long* __restrict__ results,
        int32_t* __restrict__ slot_pool, int64_t warp_elems, int chunk, long long budget,
        int* __restrict__ err, unsigned long long* __restrict__ stats) {
    unsigned long long my_bytes = 0;
    __shared__ GpPlan s_plan[kWarps];
    __shared__ int s_len[kWarps][GP_MAX_SLOTS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * kWarps + w;
    TaskCtx c;
    c.P = &s_plan[w];
    c.slots = slot_pool + gw * warp_elems;
    c.slen = s_len[w];
    c.lane = lane;
    c.err = err;
    c.row_ptr = nullptr;
    c.col = nullptr;
    c.slot_cap = 0;
    c.n_vertices = 0;
    c.sbytes = kStats ? &my_bytes : nullptr;
    int cur_job = -1;
    int64_t job_lo = 0, job_hi = 0, job_begin = 0;
    Acc acc;
    const long long t_start = clock64();
    for (;;) {
        if (budget > 0 && clock64() - t_start > budget) break;
        // Grab one task while the cursor is inside some job's heavy prefix
        // (tasks of high-degree first vertices), a chunk otherwise.
        unsigned long long t0 = 0;
        int grab = chunk;
        if (lane == 0) {
            const int64_t peek = (int64_t)*(volatile unsigned long long*)cursor;
            if (peek < total) {
                int lo = 0, hi = njobs - 1;
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (jobs[mid].task_offset <= peek) lo = mid; else hi = mid - 1;
                }
                if (peek - jobs[lo].task_offset < jobs[lo].heavy) grab = 1;
            }
            t0 = atomicAdd(cursor, (unsigned long long)grab);
        }
        t0 = __shfl_sync(kFull, t0, 0);
        grab = __shfl_sync(kFull, grab, 0);
        if ((int64_t)t0 >= total) break;
        const int64_t t1 = min((int64_t)t0 + grab, total);
        int64_t t = (int64_t)t0;
        while (t < t1) {
            if (cur_job < 0 || t < job_lo || t >= job_hi) {
                int lo = 0, hi = njobs - 1;      // last job whose offset <= t
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (jobs[mid].task_offset <= t) lo = mid; else hi = mid - 1;
                }
                if (cur_job >= 0) flush(acc, results + 2 * cur_job);
                cur_job = lo;
                const CountJob& J = jobs[lo];
                const int* src = reinterpret_cast<const int*>(&J.plan);
                int* dst = reinterpret_cast<int*>(&s_plan[w]);
                for (int i = lane; i < (int)(sizeof(GpPlan) / 4); i += 32) dst[i] = src[i];
                __syncwarp();
                job_lo = J.task_offset;
                job_hi = J.task_offset + J.ntasks;
                job_begin = J.task_begin;
                c.row_ptr = J.row_ptr;
                c.col = J.col;
                c.slot_cap = J.slot_cap;
                c.n_vertices = J.n;
            }
            const int64_t tend = min(t1, job_hi);
            int64_t e = job_begin + (t - job_lo);
            const int64_t e_end = job_begin + (tend - job_lo);
            // source vertex of entry e: last u with row_ptr[u] <= e
            int lo = 0, hi = c.n_vertices - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (__ldg(c.row_ptr + mid) <= e) lo = mid; else hi = mid - 1;
            }
            int v0 = lo;
            int64_t row_end = __ldg(c.row_ptr + v0 + 1);
            const uint8_t lo1 = s_plan[w].lvl[1].lo_mask & 1, hi1 = s_plan[w].lvl[1].hi_mask & 1;
            if (s_plan[w].k == 3 && s_plan[w].lvl[1].nbuild == 0) {
                // one task per lane; heavy ones go to the whole warp
                int v[GP_MAX_K];
#pragma unroll
                for (int i = 0; i < GP_MAX_K; ++i) v[i] = -1;
                for (int64_t eb = e; eb < e_end; eb += 32) {
                    const int64_t my = eb + lane;
                    bool active = my < e_end;
                    int a0 = -1, a1 = -1;
                    if (active) {
                        int rl = v0, rh = c.n_vertices - 1;     // row of entry `my`
                        while (rl < rh) {
                            int mid = (rl + rh + 1) >> 1;
                            if (__ldg(c.row_ptr + mid) <= my) rl = mid; else rh = mid - 1;
                        }
                        a0 = rl;
                        a1 = __ldg(c.col + my);
                        if (lo1 && !(a1 > a0)) active = false;
                        if (hi1 && !(a1 < a0)) active = false;
                    }
                    bool deferred = false;
                    if (active) {
                        v[0] = a0;
                        v[1] = a1;
                        deferred = !count_last_lane(c, v, acc);
                    }
                    unsigned dm = __ballot_sync(kFull, deferred);
                    while (dm) {
                        const int src = __ffs(dm) - 1;
                        dm &= dm - 1;
                        v[0] = __shfl_sync(kFull, a0, src);
                        v[1] = __shfl_sync(kFull, a1, src);
                        count_last(c, v, acc);
                    }
                }
            } else {
                for (; e < e_end; ++e) {
                    while (e >= row_end) { ++v0; row_end = __ldg(c.row_ptr + v0 + 1); }
                    const int v1 = __ldg(c.col + e);
                    if (lo1 && !(v1 > v0)) continue;
                    if (hi1 && !(v1 < v0)) continue;
                    run_task(c, v0, v1, acc);
                }
            }
            t = tend;
        }
    }
    if (cur_job >= 0) flush(acc, results + 2 * cur_job);
    if (kStats) {
        for (int o = 16; o; o >>= 1) my_bytes += __shfl_down_sync(kFull, my_bytes, o);
        if (lane == 0 && my_bytes) atomicAdd(stats, my_bytes);
    }
}

}  // namespace

namespace {

using KernelFn = void (*)(const CountJob*, int, int64_t, unsigned long long*, unsigned long long*,
                          int32_t*, int64_t, int, long long, int*, unsigned long long*);

struct Geometry {
    KernelFn kern;
    int64_t blocks;
    int64_t warp_elems;     // scratch elements per warp
    size_t per_block;       // scratch bytes per block
    int64_t total;          // tasks over all jobs
};

// Grid of the persistent launch: SM count x resident blocks per SM, reduced
// (in whole waves of SMs) until the per-warp intermediate-set scratch fits in
// a quarter of the free device memory.
gp_status geometry(const CountJob* jobs, int njobs, const LaunchOpts& opt, Geometry* g) {
    g->total = 0;
    g->warp_elems = 1;
    for (int j = 0; j < njobs; ++j) {
        g->total += jobs[j].ntasks;
        g->warp_elems = std::max<int64_t>(g->warp_elems, (int64_t)jobs[j].plan.nslots * jobs[j].slot_cap);
    }
    int dev = 0, nsm = 0;
    GP_CUDA_TRY(cudaGetDevice(&dev));
    GP_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int occ = 0;
    // two register budgets: 64 registers (4 blocks per SM, the default: the
    // kernel is latency-bound and gains more from warps than from registers)
    // or about 96 (2 blocks per SM, when 1 or 2 blocks per SM are asked for)
    const bool dense = !(opt.blocks_per_sm == 1 || opt.blocks_per_sm == 2);
    g->kern = opt.stats ? (dense ? k_count<true, 4> : k_count<true, 1>)
                        : (dense ? k_count<false, 4> : k_count<false, 1>);
    GP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, g->kern, kWarps * 32, 0));
    int per_sm = opt.blocks_per_sm > 0 ? std::min(opt.blocks_per_sm, occ) : occ;
    if (per_sm < 1) per_sm = 1;
    g->blocks = (int64_t)nsm * per_sm;
    size_t free_b = 0, total_b = 0;
    GP_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    g->per_block = (size_t)kWarps * (size_t)g->warp_elems * sizeof(int32_t);
    while (g->blocks > nsm && g->per_block * (size_t)g->blocks > free_b / 4) g->blocks -= nsm;
    if (g->per_block * (size_t)g->blocks > free_b / 2) {
        set_error("intermediate sets need %zu bytes per block; %zu free", g->per_block, free_b);
        return GP_ERR_SCRATCH;
    }
    return GP_OK;
}

}  // namespace

gp_status scratch_bytes(const CountJob* jobs, int njobs, const LaunchOpts& opt, uint64_t* bytes) {
    Geometry g;
    gp_status rc = geometry(jobs, njobs, opt, &g);
    if (rc != GP_OK) return rc;
    *bytes = (uint64_t)g.per_block * (uint64_t)g.blocks;
    return GP_OK;
}

gp_status run_count(const CountJob* jobs, int njobs, const LaunchOpts& opt, cudaStream_t st,
                    uint64_t* results, int64_t* processed, float* kernel_ms, uint64_t* algo_bytes) {
    if (njobs <= 0) { set_error("no jobs"); return GP_ERR_ARG; }
    Geometry geo;
    gp_status grc = geometry(jobs, njobs, opt, &geo);
    if (grc != GP_OK) return grc;
    const int64_t total = geo.total, blocks = geo.blocks, warp_elems = geo.warp_elems;
    const size_t per_block = geo.per_block;
    auto kern = geo.kern;
    int chunk = opt.chunk;
    if (chunk <= 0) {
        int64_t per_warp = total / (blocks * kWarps * 64);
        chunk = (int)std::max<int64_t>(1, std::min<int64_t>(64, per_warp));
    }

    // device buffers: job table, results (2 per job), cursor, error word
    const size_t jobs_b = sizeof(CountJob) * (size_t)njobs;
    const size_t res_b = sizeof(unsigned long long) * (2 * (size_t)njobs + 3);
    void* d_mem = nullptr;
    int32_t* d_slots = nullptr;
    GP_CUDA_TRY(cudaMallocAsync(&d_mem, jobs_b + res_b + 64, st));
    if (cudaMallocAsync((void**)&d_slots, per_block * (size_t)blocks, st) != cudaSuccess) {
        cudaFreeAsync(d_mem, st);
        cudaGetLastError();
        set_error("cannot allocate %zu bytes of intermediate-set scratch", per_block * (size_t)blocks);
        return GP_ERR_NOMEM;
    }
    CountJob* d_jobs = static_cast<CountJob*>(d_mem);
    unsigned long long* d_res = reinterpret_cast<unsigned long long*>(static_cast<char*>(d_mem) + jobs_b);
    unsigned long long* d_cursor = d_res + 2 * njobs;
    int* d_err = reinterpret_cast<int*>(d_cursor + 1);
    unsigned long long* d_stats = d_cursor + 2;
    gp_status rc = GP_OK;
    std::vector<unsigned long long> h_res(2 * (size_t)njobs + 3, 0);
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (kernel_ms) {
        GP_CUDA_TRY(cudaEventCreate(&ev0));
        GP_CUDA_TRY(cudaEventCreate(&ev1));
    }
    cudaError_t e = cudaMemcpyAsync(d_jobs, jobs, jobs_b, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_res, 0, res_b, st);
    if (e == cudaSuccess && ev0) e = cudaEventRecord(ev0, st);
    if (e == cudaSuccess && total > 0) {
        kern<<<(unsigned)blocks, kWarps * 32, 0, st>>>(d_jobs, njobs, total, d_cursor, d_res, d_slots,
                                                      warp_elems, chunk, (long long)opt.budget_cycles,
                                                      d_err, d_stats);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && ev1) e = cudaEventRecord(ev1, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_res.data(), d_res, res_b, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && ev0) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, ev0, ev1);
        *kernel_ms = ms;
    }
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    cudaFreeAsync(d_slots, st);
    cudaFreeAsync(d_mem, st);
    if (e != cudaSuccess) {
        set_error("count kernel failed: %s", cudaGetErrorString(e));
        return GP_ERR_CUDA;
    }
    const int err_word = (int)(h_res[2 * njobs + 1] & 0xffffffffu);
    if (err_word) {
        set_error("count kernel reported internal error %d", err_word);
        return GP_ERR_INTERNAL;
    }
    for (int j = 0; j < 2 * njobs; ++j) results[j] = h_res[j];
    if (algo_bytes) *algo_bytes = h_res[2 * njobs + 2];
    int64_t done = (int64_t)std::min<unsigned long long>(h_res[2 * njobs], (unsigned long long)total);
    if (processed) *processed = total == 0 ? 0 : done;
    return rc;
}

gp_status run_count_in_scratch(const CountJob* jobs, int njobs, void* d_scratch, size_t scratch_bytes,
                               cudaStream_t st, uint64_t* results) {
    constexpr int kMaxJobs = 8;            // host result words live on the stack
    if (njobs <= 0 || njobs > kMaxJobs) { set_error("1 to %d jobs per call", kMaxJobs); return GP_ERR_ARG; }
    // layout: [result words | job table | intermediate sets], 256-byte aligned
    const size_t words_b = ((sizeof(unsigned long long) * (2 * (size_t)njobs + 3)) + 255) & ~(size_t)255;
    const size_t jobs_b = ((sizeof(CountJob) * (size_t)njobs) + 255) & ~(size_t)255;
    if (words_b + jobs_b > scratch_bytes) {
        set_error("%d jobs need %zu bytes of fixed scratch for results and job table; it holds %zu",
                  njobs, words_b + jobs_b, scratch_bytes);
        return GP_ERR_SCRATCH;
    }
    int64_t total = 0, warp_elems = 1;
    for (int j = 0; j < njobs; ++j) {
        total += jobs[j].ntasks;
        warp_elems = std::max<int64_t>(warp_elems, (int64_t)jobs[j].plan.nslots * jobs[j].slot_cap);
    }
    const size_t per_block = (size_t)kWarps * (size_t)warp_elems * sizeof(int32_t);
    const size_t slot_b = scratch_bytes - words_b - jobs_b;
    if (per_block > slot_b) {
        set_error("this plan and graph need %zu bytes of intermediate-set scratch per block; "
                  "the fixed scratch has %zu", per_block, slot_b);
        return GP_ERR_SCRATCH;
    }
    int dev = 0, nsm = 0, occ = 0;
    GP_CUDA_TRY(cudaGetDevice(&dev));
    GP_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    auto kern = k_count<false, 4>;
    GP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWarps * 32, 0));
    int64_t blocks = std::min<int64_t>((int64_t)nsm * std::max(occ, 1), (int64_t)(slot_b / per_block));
    int64_t per_warp = total / (blocks * kWarps * 64);
    const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(64, per_warp));
    char* base = static_cast<char*>(d_scratch);
    unsigned long long* d_res = reinterpret_cast<unsigned long long*>(base);
    unsigned long long* d_cursor = d_res + 2 * njobs;
    int* d_err = reinterpret_cast<int*>(d_cursor + 1);
    unsigned long long* d_stats = d_cursor + 2;
    CountJob* d_jobs = reinterpret_cast<CountJob*>(base + words_b);
    int32_t* d_slots = reinterpret_cast<int32_t*>(base + words_b + jobs_b);
    unsigned long long h_res[2 * kMaxJobs + 3] = {};
    const size_t nwords = 2 * (size_t)njobs + 3;
    GP_CUDA_TRY(cudaMemcpyAsync(d_jobs, jobs, sizeof(CountJob) * (size_t)njobs, cudaMemcpyHostToDevice, st));
    GP_CUDA_TRY(cudaMemsetAsync(d_res, 0, words_b, st));       // results, cursor, error word start at 0
    if (total > 0) {
        kern<<<(unsigned)blocks, kWarps * 32, 0, st>>>(d_jobs, njobs, total, d_cursor, d_res, d_slots,
                                                      warp_elems, chunk, 0, d_err, d_stats);
        count_launch();
        GP_CUDA_TRY(cudaGetLastError());
    }
    GP_CUDA_TRY(cudaMemcpyAsync(h_res, d_res, sizeof(unsigned long long) * nwords,
                                cudaMemcpyDeviceToHost, st));
    GP_CUDA_TRY(cudaStreamSynchronize(st));
    if ((int)(h_res[2 * njobs + 1] & 0xffffffffu)) {
        set_error("count kernel reported internal error %d", (int)(h_res[2 * njobs + 1] & 0xffffffffu));
        return GP_ERR_INTERNAL;
    }
    for (int j = 0; j < 2 * njobs; ++j) results[j] = h_res[j];
    return GP_OK;
}

}  // namespace gp
