// count.cu -- the pattern-count kernel: a persistent, warp-per-task
// interpreter of the nested-loop search of GraphPi (Sections II-B, IV-B,
// IV-E), for sm_103a.
//
// Work decomposition (Section IV-E, fine-grained tasks + work stealing):
// every directed CSR entry (v0, v1) is one task that fixes the first two
// loops. Tasks of all jobs form one global index space; a warp grabs tasks
// with one atomicAdd on a global cursor (one at a time while the cursor is in
// the high-degree prefix of a job, a chunk otherwise), so idle warps take the
// next work immediately (the device analogue of work stealing).
//
// Inside a task one warp runs the remaining loops depth-first. Candidate
// sets are intersections of sorted neighbour lists, clipped to the window the
// restrictions impose (a restriction becomes a bound on a sorted list, the
// "break" of Section IV-B). An intersection of lists of similar length is a
// tile merge; otherwise it iterates the shorter list and tests each element
// for membership in the other: with one bit probe when the other is the
// neighbour list of a "core" vertex (the highest-degree vertices of a
// degree-ordered graph, whose adjacency among themselves is kept as a bit
// matrix), else with a binary search. Plans switched to inclusion-exclusion
// (Section IV-D) stop kk >= 2 loops early and add the number of distinct
// kk-tuples from the inner candidate sets instead. Loops above the last two run one
// candidate at a time with the whole warp cooperating on each intersection;
// the loop at depth k-2 gives one candidate to each lane, which counts the
// last level alone (heavy candidates go back to the whole warp). The last
// loop is never enumerated: its contribution is the size of its clipped
// candidate set minus the already-matched vertices inside it. Plans whose
// later vertices all lie below v1 run, for tasks whose v1 is a core vertex,
// on shared-memory bitmaps instead (the bitmap subtree below).
//
// Counts are accumulated per lane in 128 bits and reduced with warp shuffles;
// one atomic pair (low word, carry into the high word) per warp per job
// publishes them.
#include <algorithm>
#include <climits>
#include <vector>

#include <cub/device/device_scan.cuh>

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
    __device__ __forceinline__ void add128(unsigned long long xl, unsigned long long xh) {
        lo += xl;
        hi += xh + (lo < xl);
    }
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

struct TaskCtx {
    const GpPlan* P;
    const int64_t* __restrict__ row_ptr;
    const int32_t* __restrict__ col;
    const uint32_t* __restrict__ core_bits;   // core_n x core_words adjacency bits
    int core_n;
    int core_words;
    int32_t* slots;        // this warp's intermediate sets
    int slot_cap;
    int n_vertices;
    int* slen;             // their lengths (shared memory, per warp)
    uint32_t* bm;          // this warp's bitmap sets (shared memory) or null
    int bm_stride;         // words per bitmap set
    bool lane_bitmap;      // bitmap last level: one candidate per lane
    bool lane_three;       // bitmap last three levels: one candidate per lane where the plan allows
    int lane;
    int lane_work;         // per-lane work limit before handing to the warp
    int* err;
    unsigned long long* sbytes;   // algorithmic-byte tally (instrumented kernel only)
    unsigned long long* sops;     // bitmap word-operation tally (instrumented kernel only)
    const int32_t* labels; // vertex labels (labelled plans in the listing kernel)
    long long* deadline;   // this warp's current work-item deadline (shared memory; 0 = none)
    long long task_cycles; // work-item cycle limit (0 = none)
    int* job_abort;        // abort flag of the current job (global memory)
    unsigned* iep_cnt;     // 32 counters per warp for inclusion-exclusion (shared memory)
};

// True (on every lane) once the current work item has outlived its cycle
// limit; the job is then marked abandoned. Call from warp-uniform code only.
__device__ __forceinline__ bool over(const TaskCtx& c) {
    const long long dl = *c.deadline;
    if (dl == 0) return false;
    const bool late = __any_sync(kFull, clock64() > dl);
    if (late && c.lane == 0) atomicExch(c.job_abort, 1);
    return late;
}

// A sorted list: [p, p + n). v >= 0 when it is (a window of) N(v).
struct List {
    const int32_t* p;
    int n;
    int v;
};

struct Window { int lo, hi; };   // candidates c with lo < c < hi

__device__ __forceinline__ Window window(uint8_t lo_mask, uint8_t hi_mask, const int* v) {
    Window w{-1, INT_MAX};
    for (int j = 0; j < GP_MAX_K; ++j) {
        if (lo_mask >> j & 1) w.lo = max(w.lo, v[j]);
        if (hi_mask >> j & 1) w.hi = min(w.hi, v[j]);
    }
    return w;
}

// Clip a sorted list to a window.
__device__ __forceinline__ List clip(List a, Window w) {
    int b = (w.lo < 0) ? 0 : lower_bound(a.p, a.n, w.lo + 1);
    int e = (w.hi == INT_MAX) ? a.n : lower_bound(a.p, a.n, w.hi);
    if (e < b) e = b;
    return List{a.p + b, e - b, a.v};
}

__device__ __forceinline__ List nbr(const TaskCtx& c, int v) {
    int64_t b = __ldg(c.row_ptr + v), e = __ldg(c.row_ptr + v + 1);
    return List{c.col + b, (int)(e - b), v};
}

__device__ __forceinline__ List slot(const TaskCtx& c, int s) {
    return List{c.slots + (size_t)s * c.slot_cap, c.slen[s], -1};
}

__device__ __forceinline__ bool is_core(const TaskCtx& c, int v) { return v >= 0 && v < c.core_n; }

// Is x (< core_n) a neighbour of core vertex v?
__device__ __forceinline__ bool core_bit(const TaskCtx& c, int v, int x) {
    const uint32_t w = __ldg(c.core_bits + (size_t)v * c.core_words + (x >> 5));
    return (w >> (x & 31)) & 1u;
}

// How an intersection runs: iterate `it` (clipped to the window) and test
// each element against `pr`, by bit probe when pr is a core vertex's
// neighbourhood (elements >= core_n are binary-searched in pr's tail), by
// binary search otherwise.
struct Probe {
    List it;
    List pr;        // by bitmap: full N(pr.v), searched from `tail`; else clipped
    int tail;
    bool bitmap;
};

__device__ __forceinline__ Probe choose(const TaskCtx& c, List a, List b, Window w) {
    const bool ca = is_core(c, a.v), cb = is_core(c, b.v);
    Probe q;
    if (ca || cb) {
        List it, pr;
        if (ca && cb) {            // both probe-able: iterate the shorter window
            List a2 = clip(a, w), b2 = clip(b, w);
            if (a2.n <= b2.n) { it = a2; pr = b; } else { it = b2; pr = a; }
        } else if (cb) {
            it = clip(a, w);
            pr = b;
        } else {
            it = clip(b, w);
            pr = a;
        }
        q.it = it;
        q.pr = pr;
        q.bitmap = true;
        // elements of `it` at or above core_n are searched in pr from there
        q.tail = (it.n > 0 && __ldg(it.p + it.n - 1) >= c.core_n) ? lower_bound(pr.p, pr.n, c.core_n) : pr.n;
        return q;
    }
    List a2 = clip(a, w), b2 = clip(b, w);
    if (a2.n <= b2.n) { q.it = a2; q.pr = b2; } else { q.it = b2; q.pr = a2; }
    q.bitmap = false;
    q.tail = 0;
    return q;
}

__device__ __forceinline__ void tally(const TaskCtx& c, List a, List b, Window w, unsigned long long extra) {
    if (c.sbytes) {
        List a2 = clip(a, w), b2 = clip(b, w);
        *c.sbytes += intersect_bytes(a2.n, b2.n) + extra;
    }
}

// Lists whose lengths differ by at most this factor are intersected by the
// tile merge below; longer ratios by binary search of the shorter list.
constexpr int kMergeRatio = 4;

// Tile merge of sorted lists A (na) and B (nb): each round loads 32 elements
// of each (coalesced), every lane finds its A element among the 32 B
// elements with a 5-step shuffle search, and the tile that ends first is
// consumed. Invariant: B elements before ib are below A[ia], so an A element
// not above the B tile's last element is matched exactly when it is in the
// tile. Writes matches to out (in order) when out != nullptr.
__device__ __forceinline__ int warp_merge(const TaskCtx& c, const int32_t* __restrict__ A, int na,
                                          const int32_t* __restrict__ B, int nb,
                                          int32_t* __restrict__ out, int cap, Acc* acc) {
    const int lane = c.lane;
    int ia = 0, ib = 0, total = 0;
    while (ia < na && ib < nb) {
        const int x = (ia + lane < na) ? __ldg(A + ia + lane) : INT_MAX;
        const int y = (ib + lane < nb) ? __ldg(B + ib + lane) : INT_MAX;
        const int amax = __shfl_sync(kFull, x, min(31, na - 1 - ia));
        const int bmax = __shfl_sync(kFull, y, min(31, nb - 1 - ib));
        int pos = 0;                                  // B elements of the tile below x
#pragma unroll
        for (int st = 16; st; st >>= 1)
            if (__shfl_sync(kFull, y, pos + st - 1) < x) pos += st;
        const int yp = __shfl_sync(kFull, y, pos);        // every lane takes part
        const bool mine = ia + lane < na && x <= bmax;   // resolved by this tile pair
        const bool f = mine && yp == x;
        const unsigned m = __ballot_sync(kFull, f);
        if (out && f) {
            const int at = total + __popc(m & lanemask_lt());
            if (at < cap) out[at] = x; else atomicExch(c.err, 2);
        }
        if (acc && f) acc->add(1);
        total += __popc(m);
        if (amax <= bmax) {                           // the A tile is resolved
            ia += 32;
            ib += __popc(__ballot_sync(kFull, ib + lane < nb && y <= amax));
        } else {                                      // the B tile is used up
            ia += __popc(__ballot_sync(kFull, mine));
            ib += 32;
        }
    }
    return total;
}

// Warp-cooperative intersection of a and b within window w. Writes the
// (sorted) result to out when out != nullptr and returns its size
// (warp-uniform). With acc != nullptr each lane also adds its own matches.
__device__ __forceinline__ int warp_intersect(const TaskCtx& c, List a, List b, Window w,
                                              int32_t* __restrict__ out, int cap, Acc* acc) {
    const Probe q = choose(c, a, b, w);
    if (!q.bitmap && q.it.n > 0 && q.pr.n <= kMergeRatio * q.it.n) {
        const int total = warp_merge(c, q.it.p, q.it.n, q.pr.p, q.pr.n, out, cap, acc);
        if (c.sbytes && c.lane == 0) tally(c, a, b, w, out ? 4ull * (unsigned long long)total : 0ull);
        return total;
    }
    const int n = q.it.n, lane = c.lane;
    int total = 0, from = q.bitmap ? q.tail : 0;
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        int x = 0, pos = q.pr.n;
        bool f = false, searched = false;
        if (i < n) {
            x = __ldg(q.it.p + i);
            if (q.bitmap && x < c.core_n) {
                f = core_bit(c, q.pr.v, x);
            } else {
                pos = from + lower_bound(q.pr.p + from, q.pr.n - from, x);
                f = pos < q.pr.n && __ldg(q.pr.p + pos) == x;
                searched = true;
            }
        }
        const unsigned m = __ballot_sync(kFull, f);
        if (out && f) {
            const int at = total + __popc(m & lanemask_lt());
            if (at < cap) out[at] = x; else atomicExch(c.err, 2);
        }
        if (acc && f) acc->add(1);
        total += __popc(m);
        // later elements are larger: narrow the searched range
        const int last = min(31, n - 1 - base);
        const int lpos = __shfl_sync(kFull, pos, last);
        if (__shfl_sync(kFull, (int)searched, last)) from = lpos;
    }
    if (c.sbytes && lane == 0) tally(c, a, b, w, out ? 4ull * (unsigned long long)total : 0ull);
    return total;
}

// Default work above which a lane hands its last-level count to the warp.
constexpr int kLaneWork = 192;

// Per-lane intersection size of a and b within w, or -1 when the estimated
// work exceeds kLaneWork (nothing is counted then).
__device__ __forceinline__ int lane_intersect_count(const TaskCtx& c, List a, List b, Window w) {
    const Probe q = choose(c, a, b, w);
    const int n = q.it.n;
    if (q.bitmap) {
        if (n > c.lane_work) return -1;
        int cnt = 0, from = q.tail;
        for (int i = 0; i < n; ++i) {
            const int x = __ldg(q.it.p + i);
            if (x < c.core_n) {
                cnt += core_bit(c, q.pr.v, x);
            } else {
                from += lower_bound(q.pr.p + from, q.pr.n - from, x);
                cnt += (from < q.pr.n && __ldg(q.pr.p + from) == x);
            }
        }
        return cnt;
    }
    const int sh = n, lo = q.pr.n;
    const bool search = lo > 16 * sh;
    const int work = search ? sh * (32 - __clz(lo | 1)) : sh + lo;
    if (work > c.lane_work) return -1;
    if (sh == 0) return 0;
    const int32_t* A = q.it.p;
    const int32_t* B = q.pr.p;
    int cnt = 0;
    if (search) {
        int from = 0;
        for (int i = 0; i < sh && from < lo; ++i) {
            const int x = __ldg(A + i);
            from += lower_bound(B + from, lo - from, x);
            cnt += (from < lo && __ldg(B + from) == x);
        }
        return cnt;
    }
    int i = 0, j = 0;
    int x = __ldg(A), y = __ldg(B);
    for (;;) {
        if (x == y) {
            ++cnt;
            if (++i == sh || ++j == lo) break;
            x = __ldg(A + i);
            y = __ldg(B + j);
        } else if (x < y) {
            if (++i == sh) break;
            x = __ldg(A + i);
        } else {
            if (++j == lo) break;
            y = __ldg(B + j);
        }
    }
    return cnt;
}

// Is x in list a (x already inside the window a was clipped to)?
__device__ __forceinline__ bool member(const TaskCtx& c, List a, int x) {
    if (is_core(c, a.v) && x < c.core_n) return core_bit(c, a.v, x);
    const int p = lower_bound(a.p, a.n, x);
    return p < a.n && __ldg(a.p + p) == x;
}

__device__ __forceinline__ void run_builds(const TaskCtx& c, int d, const int* v) {
    const GpLevel& L = c.P->lvl[d];
    for (int q = 0; q < L.nbuild; ++q) {
        const GpBuild& B = L.build[q];
        const List a = (B.base_kind == 1) ? nbr(c, v[B.base]) : slot(c, B.base);
        const Window w = window(B.lo_mask, B.hi_mask, v);
        int32_t* out = c.slots + (size_t)B.dst * c.slot_cap;
        const int n = warp_intersect(c, a, nbr(c, v[d]), w, out, c.slot_cap, nullptr);
        if (c.lane == 0) c.slen[B.dst] = n;
        __syncwarp();
    }
}

// Matched vertices that lie in the last level's candidate set: they are not
// new vertices (injectivity) and are subtracted from its size.
__device__ __forceinline__ int excluded_hits(const TaskCtx& c, const GpLevel& lv, int L, const int* v,
                                             Window w, List a, const List* b) {
    int hits = 0;
    for (int j = 0; j < L; ++j) {
        if (!(lv.excl_mask >> j & 1)) continue;
        const int x = v[j];
        if (x > w.lo && x < w.hi && member(c, a, x) && (!b || member(c, *b, x))) ++hits;
    }
    return hits;
}

// excluded_hits with one lane per matched vertex (warp-uniform call; the
// same value on every lane).
__device__ __forceinline__ int excluded_hits_warp(const TaskCtx& c, const GpLevel& lv, int L, const int* v,
                                                  Window w, List a, const List* b) {
    bool hit = false;
    if (c.lane < L && (lv.excl_mask >> c.lane & 1)) {
        const int x = v[c.lane];
        hit = x > w.lo && x < w.hi && member(c, a, x) && (!b || member(c, *b, x));
    }
    return __popc(__ballot_sync(kFull, hit));
}

// Contribution of the innermost loop given v[0..k-2] (warp-uniform).
__device__ __forceinline__ void count_last(const TaskCtx& c, const int* v, Acc& acc) {
    const GpPlan& P = *c.P;
    const int L = P.k - 1;
    const GpLevel& lv = P.lvl[L];
    const Window w = window(lv.lo_mask, lv.hi_mask, v);
    if (P.last_count_only) {
        const List a = (P.last_base_kind == 1) ? nbr(c, v[P.last_base]) : slot(c, P.last_base);
        const List b = nbr(c, v[L - 1]);
        warp_intersect(c, a, b, w, nullptr, 0, &acc);
        const List a2 = is_core(c, a.v) ? a : clip(a, w);
        const List b2 = is_core(c, b.v) ? b : clip(b, w);
        const int hits = excluded_hits_warp(c, lv, L, v, w, a2, &b2);
        if (c.lane == 0) acc.sub((unsigned long long)hits);
    } else {
        const List a = clip((lv.src_kind == 1) ? nbr(c, v[lv.src]) : slot(c, lv.src), w);
        const int hits = excluded_hits_warp(c, lv, L, v, w, a, nullptr);
        if (c.lane == 0) acc.add((unsigned long long)a.n - hits);
    }
}

// Per-lane count_last: v[] is this lane's own matched vertices. Returns
// false (and counts nothing) when the warp-cooperative version should run.
__device__ __forceinline__ bool count_last_lane(const TaskCtx& c, const int* v, Acc& acc) {
    const GpPlan& P = *c.P;
    const int L = P.k - 1;
    const GpLevel& lv = P.lvl[L];
    const Window w = window(lv.lo_mask, lv.hi_mask, v);
    if (P.last_count_only) {
        const List a = (P.last_base_kind == 1) ? nbr(c, v[P.last_base]) : slot(c, P.last_base);
        const List b = nbr(c, v[L - 1]);
        const int cnt = lane_intersect_count(c, a, b, w);
        if (cnt < 0) return false;
        const List a2 = is_core(c, a.v) ? a : clip(a, w);
        const List b2 = is_core(c, b.v) ? b : clip(b, w);
        acc.add((unsigned long long)(cnt - excluded_hits(c, lv, L, v, w, a2, &b2)));
        if (c.sbytes) { const List x = clip(a, w), y = clip(b, w); *c.sbytes += intersect_bytes(x.n, y.n); }
        return true;
    }
    const List a = clip((lv.src_kind == 1) ? nbr(c, v[lv.src]) : slot(c, lv.src), w);
    acc.add((unsigned long long)(a.n - excluded_hits(c, lv, L, v, w, a, nullptr)));
    return true;
}

// Inclusion-exclusion for the last two depths (Section IV-D, k = 2): with
// v[0..k-3] bound, the last two vertices range over S_a (depth k-2) and
// S_b (depth k-1), minus already-matched vertices, and must differ:
// |S_a| |S_b| - |S_a ∩ S_b|. The plan has no restriction acting at those
// depths; the host divides the job's total by the plan's iep_div.
// Is x in list a? Binary search from position `from` (x is not below a.p[from]
// when from > 0); *pos receives the search position for the next, larger x.
__device__ __forceinline__ bool member_from(const TaskCtx& c, List a, int x, int from, int* pos) {
    if (is_core(c, a.v) && x < c.core_n) { *pos = from; return core_bit(c, a.v, x); }
    const int p = from + lower_bound(a.p + from, a.n - from, x);
    *pos = p;
    return p < a.n && __ldg(a.p + p) == x;
}

// The fused form (plan.iep_fuse): one inner set F = base ∩ N(v_{k-3}) is
// never stored. One pass over the list choose() iterates counts |F| (the
// elements found in the probed list) and |F ∩ O| (those also in the other
// inner set O, searched with a window that narrows as the elements grow).
// Returns both, warp-uniform.
__device__ __forceinline__ int2 fused_counts(const TaskCtx& c, const Probe& q, List O) {
    const int n = q.it.n, lane = c.lane;
    int nf = 0, nfo = 0, from = q.bitmap ? q.tail : 0, from_o = 0;
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        int x = INT_MAX, pos = q.pr.n, pos_o = 0;
        bool f = false, searched = false;
        if (i < n) {
            x = __ldg(q.it.p + i);
            if (q.bitmap && x < c.core_n) {
                f = core_bit(c, q.pr.v, x);
            } else {
                pos = from + lower_bound(q.pr.p + from, q.pr.n - from, x);
                f = pos < q.pr.n && __ldg(q.pr.p + pos) == x;
                searched = true;
            }
        }
        bool fo = false;
        if (f) fo = member_from(c, O, x, from_o, &pos_o);
        nf += __popc(__ballot_sync(kFull, f));
        nfo += __popc(__ballot_sync(kFull, fo));
        // later elements are larger: narrow both searched ranges
        const int last = min(31, n - 1 - base);
        const int lpos = __shfl_sync(kFull, pos, last);
        if (__shfl_sync(kFull, (int)searched, last)) from = lpos;
        // the next batch's elements exceed lx: O's searches start at lx's
        // lower bound
        const int lx = __shfl_sync(kFull, x, last);
        int p0 = 0;
        if (lane == 0) p0 = from_o + lower_bound(O.p + from_o, O.n - from_o, lx);
        from_o = __shfl_sync(kFull, p0, 0);
    }
    if (c.sbytes && lane == 0) *c.sbytes += intersect_bytes(q.it.n, q.pr.n) + intersect_bytes(nf, O.n);
    return make_int2(nf, nfo);
}

// kFused: the launch's build carries the fused form (the general
// inclusion-exclusion build); other builds never see a fused plan.
template <bool kFused>
__device__ __forceinline__ void iep_count2(const TaskCtx& c, const int* v, Acc& acc) {
    const GpPlan& P = *c.P;
    const int da = P.k - 2, db = P.k - 1;
    const GpLevel& LA = P.lvl[da];
    const GpLevel& LB = P.lvl[db];
    if (kFused && P.iep_fuse) {
        const int dF = P.k - 3 + P.iep_fuse, dO = (dF == da) ? db : da;
        const GpLevel& LF = P.lvl[dF];
        const GpLevel& LO = P.lvl[dO];
        const GpBuild& Bf = P.iep_build;
        const List base = (Bf.base_kind == 1) ? nbr(c, v[Bf.base]) : slot(c, Bf.base);
        const List nd = nbr(c, v[P.k - 3]);
        const Window wf = window(Bf.lo_mask | LF.lo_mask, Bf.hi_mask | LF.hi_mask, v);
        const Window wo = window(LO.lo_mask, LO.hi_mask, v);
        const List O = clip((LO.src_kind == 1) ? nbr(c, v[LO.src]) : slot(c, LO.src), wo);
        const Probe q = choose(c, base, nd, wf);
        const int2 cnt = fused_counts(c, q, O);
        // matched vertices in F (in the window, in base and in N(v_{k-3})),
        // in O, and in both: lane j tests v_j for F, lane 16 + j for O
        const int j = c.lane & 15;
        const bool forF = c.lane < 16;
        bool in = false;
        if (j < da && ((forF ? LF.excl_mask : LO.excl_mask) >> j & 1)) {
            const int x = v[j];
            if (forF) {
                in = x > wf.lo && x < wf.hi && member(c, base, x) && member(c, nd, x);
            } else {
                in = x > wo.lo && x < wo.hi && member(c, O, x);
            }
        }
        const unsigned m = __ballot_sync(kFull, in);
        if (c.lane == 0) {
            const unsigned mf = m & 0xffffu, mo = m >> 16;
            const int a = cnt.x - __popc(mf), b = O.n - __popc(mo);
            acc.add((unsigned long long)a * (unsigned long long)b);
            acc.sub((unsigned long long)(cnt.y - __popc(mf & mo)));
        }
        return;
    }
    const Window wa = window(LA.lo_mask, LA.hi_mask, v), wb = window(LB.lo_mask, LB.hi_mask, v);
    const List A = clip((LA.src_kind == 1) ? nbr(c, v[LA.src]) : slot(c, LA.src), wa);
    const List B = clip((LB.src_kind == 1) ? nbr(c, v[LB.src]) : slot(c, LB.src), wb);
    const Window open{-1, INT_MAX};
    // the two sets are often one (both inner vertices adjacent to the same
    // outer vertices, as in K6-e): then S_a ∩ S_b = S_a
    const int ab = (A.p == B.p && A.n == B.n) ? A.n : warp_intersect(c, A, B, open, nullptr, 0, nullptr);
    // matched vertices inside S_a, S_b and both: a matched vertex can be in a
    // set only when the set's exclusion mask names its depth (operands and
    // window bounds exclude it), so lane j tests v_j against S_a and lane
    // 16 + j against S_b, all searches at once
    const int j = c.lane & 15;
    const bool forA = c.lane < 16;
    const GpLevel& L = forA ? LA : LB;
    const List S = forA ? A : B;
    const Window w = forA ? wa : wb;
    bool in = false;
    if (j < da && (L.excl_mask >> j & 1)) {
        const int x = v[j];
        in = x > w.lo && x < w.hi && member(c, S, x);
    }
    const unsigned m = __ballot_sync(kFull, in);
    if (c.lane == 0) {
        const unsigned ma = m & 0xffffu, mb = m >> 16;
        const int a = A.n - __popc(ma), b = B.n - __popc(mb);
        acc.add((unsigned long long)a * (unsigned long long)b);
        acc.sub((unsigned long long)(ab - __popc(ma & mb)));
    }
}

// Inclusion-exclusion for the last kk >= 3 depths (Section IV-D). With the
// outer depths 0 .. k-kk-1 bound, the inner vertices (pairwise non-adjacent,
// no restriction among them or towards the outer ones) take values in
// their candidate sets S_1 .. S_kk minus the matched outer vertices, and
// must be pairwise distinct. The number of such tuples is
//   sum over set partitions pi of {1..kk} of
//       prod over blocks B of pi of (-1)^(|B|-1) (|B|-1)! |∩_{i in B} S_i|,
// the terms of Algorithm 2's expansion grouped by the components they
// produce. Every intersection size comes from one pass: each element x of
// a set other than the largest gets the mask M(x) of the sets holding it
// (counted once, at the first iterated set that holds it), the warp tallies
// how many elements share each mask, and |∩_{i in T} S_i| is the sum of the
// tallies of the masks containing T. Arithmetic is in 128 bits; the host
// divides the job's total by the plan's iep_div.
__device__ __noinline__ void iep_count_sets(const TaskCtx& c, const int* v, Acc& acc) {
    const GpPlan& P = *c.P;
    const int k = P.k, kk = P.iep, d0 = k - kk;
    List S[GP_MAX_IEP];
    int big = 0, big_n = -1;
#pragma unroll
    for (int i = 0; i < GP_MAX_IEP; ++i) {
        S[i] = List{nullptr, 0, -1};
        if (i < kk) {
            const GpLevel& L = P.lvl[d0 + i];
            S[i] = clip((L.src_kind == 1) ? nbr(c, v[L.src]) : slot(c, L.src), window(L.lo_mask, L.hi_mask, v));
            if (S[i].n > big_n) { big = i; big_n = S[i].n; }
        }
    }
    unsigned* cnt = c.iep_cnt;
    cnt[c.lane] = 0u;
    __syncwarp();
#pragma unroll
    for (int i = 0; i < GP_MAX_IEP; ++i) {
        if (i >= kk || i == big) continue;
        int from[GP_MAX_IEP];
#pragma unroll
        for (int j = 0; j < GP_MAX_IEP; ++j) from[j] = 0;
        const int n = S[i].n;
        for (int base = 0; base < n; base += 32) {
            const int idx = base + c.lane;
            unsigned M = 0;
            int pos[GP_MAX_IEP];
#pragma unroll
            for (int j = 0; j < GP_MAX_IEP; ++j) pos[j] = from[j];
            if (idx < n) {
                const int x = __ldg(S[i].p + idx);
                bool dup = false;
                M = 1u << i;
#pragma unroll
                for (int j = 0; j < GP_MAX_IEP; ++j) {
                    if (j >= kk || j == i) continue;
                    if (member_from(c, S[j], x, from[j], &pos[j])) {
                        M |= 1u << j;
                        dup |= (j < i && j != big);     // counted at an earlier set
                    }
                }
                for (int j = 0; j < d0; ++j) dup |= (v[j] == x);   // a matched outer vertex
                if (dup) M = 0;
            }
            const unsigned grp = __match_any_sync(kFull, M);
            if (__popc(M) >= 2 && (__ffs(grp) - 1) == c.lane) cnt[M] += __popc(grp);
            // later elements are larger: narrow the searches
            const int last = min(31, n - 1 - base);
#pragma unroll
            for (int j = 0; j < GP_MAX_IEP; ++j) from[j] = __shfl_sync(kFull, pos[j], last);
        }
        if (c.sbytes && c.lane == 0)
            for (int j = 0; j < kk; ++j)
                if (j != i) *c.sbytes += intersect_bytes(n, S[j].n);
    }
    __syncwarp();
    // superset sums: lane T holds |∩_{i in T} S_i| (without matched vertices)
    unsigned long long val = cnt[c.lane];
    for (int b = 0; b < kk; ++b) {
        const unsigned long long o = __shfl_xor_sync(kFull, val, 1 << b);
        if (!(c.lane >> b & 1)) val += o;
    }
    if (__popc(c.lane) == 1) {                  // single sets: |S_i| minus matched vertices
        const int i = __ffs(c.lane) - 1;
        if (i < kk) {
            const GpLevel& L = P.lvl[d0 + i];
            const Window w = window(L.lo_mask, L.hi_mask, v);
            List si = S[0];
#pragma unroll
            for (int t = 1; t < GP_MAX_IEP; ++t) if (t == i) si = S[t];
            val = (unsigned long long)(si.n - excluded_hits(c, L, d0, v, w, si, nullptr));
        }
    }
    // every set partition of the kk sets as a restricted growth string
    // g_0 .. g_{kk-1} (3 bits each): g_0 = 0 and g_i <= 1 + max(g_0 .. g_{i-1});
    // block b holds the sets i with g_i = b. All lanes walk the same
    // partitions, so every shuffle below is uniform.
    __int128 total = 0;
    unsigned g = 0;
    for (;;) {
        __int128 term = 1;
        for (int blk = 0; blk < kk; ++blk) {
            unsigned mask = 0;
            for (int i = 0; i < kk; ++i)
                if (((g >> (3 * i)) & 7u) == (unsigned)blk) mask |= 1u << i;
            if (!mask) break;                     // blocks are numbered 0, 1, 2, ...
            const long long card = (long long)__shfl_sync(kFull, val, (int)mask);
            const int m = __popc(mask);
            long long mu = 1;                     // (-1)^(m-1) (m-1)!
            for (int t = 2; t < m; ++t) mu *= t;
            if (!(m & 1)) mu = -mu;
            term *= (__int128)(mu * card);
        }
        total += term;
        int i = kk - 1;                           // next growth string
        for (; i >= 1; --i) {
            unsigned mx = 0;
            for (int j = 0; j < i; ++j) mx = max(mx, (g >> (3 * j)) & 7u);
            if (((g >> (3 * i)) & 7u) <= mx) {
                g += 1u << (3 * i);
                g &= (1u << (3 * (i + 1))) - 1u;  // zero the tail
                break;
            }
        }
        if (i < 1) break;
    }
    if (c.lane == 0) {
        const unsigned __int128 r = (unsigned __int128)total;
        acc.add128((unsigned long long)r, (unsigned long long)(r >> 64));
    }
}

// kGeneralIep: the launch may hold plans with kk >= 3 or a fused two-loop
// form (kernels launched without such plans carry none of that code).
template <bool kGeneralIep>
__device__ __forceinline__ void iep_count(const TaskCtx& c, const int* v, Acc& acc) {
    if (!kGeneralIep || c.P->iep == 2) iep_count2<kGeneralIep>(c, v, acc);
    else iep_count_sets(c, v, acc);
}

// The loop at depth k-2 with one candidate per lane: every lane counts the
// last level for its own candidate; candidates with heavy intersections are
// then counted one at a time by the whole warp.
__device__ __forceinline__ void lane_parallel_last_two(const TaskCtx& c, int* v, List lst, Acc& acc) {
    const GpPlan& P = *c.P;
    const int d = P.k - 2;
    const uint8_t ex = P.lvl[d].excl_mask;
    for (int base = 0; base < lst.n; base += 32) {
        if (over(c)) return;
        const int i = base + c.lane;
        int x = -1;
        bool active = i < lst.n;
        if (active) {
            x = __ldg(lst.p + i);
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

// ---------------------------------------------------------------------------
// Bitmap subtree: used when every vertex searched after v1 is restricted
// below v1 and v1 is a core vertex. All later candidates are then core
// vertices below v1, so a candidate set is the AND of core adjacency rows
// (plus N(v0) scattered into a bitmap when v0 is not a core vertex), masked
// to its restriction window, held in shared memory (bit x = vertex x). Lanes
// work on 32-bit words; loops visit set bits in increasing order; the last
// level is a popcount.

__device__ __forceinline__ uint32_t window_bits(int w, int lo, int hi) {
    // bits b of word w with lo < 32 w + b < hi
    const int first = 32 * w;
    uint32_t m = 0xffffffffu;
    const int a = lo - first + 1;            // lowest allowed bit
    if (a > 0) m = (a >= 32) ? 0u : (m << a);
    const int b = hi - first;                // bits below b allowed
    if (b < 32) m &= (b <= 0) ? 0u : ((1u << b) - 1u);
    return m;
}

// Word w of N(v_j) restricted to the core (N(v0) comes from shared memory
// when v0 is not a core vertex).
__device__ __forceinline__ uint32_t operand_word(const TaskCtx& c, const int* v, int j, int w, bool n0_smem) {
    if (j == 0 && n0_smem) return c.bm[w];
    return __ldg(c.core_bits + (size_t)v[j] * c.core_words + w);
}

// S_d = AND of the rows of its operands, inside its window, without the
// already-matched vertices that may lie in it. Returns the number of words
// that can hold its bits (its window ends before that). With bm_inc the set
// is S_{d-1} AND the row of v_{d-1}.
__device__ __forceinline__ int bitmap_build(const TaskCtx& c, const int* v, int d, int W, int Wprev,
                                            bool n0_smem) {
    const GpLevel& L = c.P->lvl[d];
    const Window win = window(L.lo_mask, L.hi_mask, v);
    const int Wd = min(W, (win.hi == INT_MAX) ? W : ((win.hi + 31) >> 5));
    uint32_t* S = c.bm + (size_t)d * c.bm_stride;
    if (L.bm_inc && d >= 3) {
        const uint32_t* prev = c.bm + (size_t)(d - 1) * c.bm_stride;
        const uint32_t* row = c.core_bits + (size_t)v[d - 1] * c.core_words;
        const int Wi = min(Wd, Wprev);
        for (int w = c.lane; w < Wd; w += 32)
            S[w] = (w < Wi) ? (prev[w] & __ldg(row + w) & window_bits(w, win.lo, win.hi)) : 0u;
        if (c.sops && c.lane == 0) *c.sops += (unsigned long long)Wi;          // one AND per word
    } else {
        if (c.sops && c.lane == 0)                                             // operands - 1 ANDs per word
            *c.sops += (unsigned long long)Wd * (unsigned)max(0, __popc(L.op_mask & ((1u << d) - 1u)) - 1);
        for (int w = c.lane; w < Wd; w += 32) {
            uint32_t x = window_bits(w, win.lo, win.hi);
            for (int j = 0; j < d && x; ++j)
                if (L.op_mask >> j & 1) x &= operand_word(c, v, j, w, n0_smem);
            S[w] = x;
        }
    }
    __syncwarp();
    if (c.lane == 0)
        for (int j = 0; j < d; ++j)
            if ((L.excl_mask >> j & 1) && v[j] > win.lo && v[j] < win.hi && v[j] < 32 * Wd)
                S[v[j] >> 5] &= ~(1u << (v[j] & 31));
    __syncwarp();
    return Wd;
}

// Next set bit of S_d at or after the iteration state (word, remaining bits).
__device__ __forceinline__ int bitmap_next(const uint32_t* S, int W, int& word, uint32_t& bits) {
    while (bits == 0) {
        if (++word >= W) return -1;
        bits = S[word];
    }
    const int b = __ffs(bits) - 1;
    bits &= bits - 1;
    return 32 * word + b;
}

// Every candidate x of depth k-2 (set S_{k-2}, Wd words): add the size of
// the last level's set, the AND of its operand rows in its window (which may
// depend on x), minus matched vertices inside it. With bm_inc on the last
// level that set is S_{k-2} AND the row of x.
__device__ __forceinline__ void bitmap_last_two(const TaskCtx& c, int* v, int W, int Ws, bool n0_smem,
                                                Acc& acc, int part, int nparts) {
    const GpPlan& P = *c.P;
    const int d = P.k - 2, L = P.k - 1;
    const GpLevel& lv = P.lvl[L];
    const bool uses_x = lv.op_mask >> d & 1;
    const uint32_t* S = c.bm + (size_t)d * c.bm_stride;      // candidates x (Ws words)
    // the window's part that does not depend on x, and whether x bounds it
    const uint8_t xbit = (uint8_t)(1u << d);
    const Window base = window(lv.lo_mask & (uint8_t)~xbit, lv.hi_mask & (uint8_t)~xbit, v);
    const bool x_lo = lv.lo_mask & xbit, x_hi = lv.hi_mask & xbit;
    // words the last level's sets can use: its own window, which may be wider
    // than S's unless the plan builds it from S (bm_inc)
    const uint32_t* PP = S;
    int Wd = Ws;
    if (!(lv.bm_inc && d >= 2)) {
        Wd = min(W, (base.hi == INT_MAX) ? W : ((base.hi + 31) >> 5));
        uint32_t* pp = c.bm + (size_t)1 * c.bm_stride;   // operands other than x
        for (int w = c.lane; w < Wd; w += 32) {
            uint32_t m = 0xffffffffu;
            for (int j = 0; j < d && m; ++j)
                if (lv.op_mask >> j & 1) m &= operand_word(c, v, j, w, n0_smem);
            pp[w] = m;
        }
        __syncwarp();
        PP = pp;
        if (c.sops && c.lane == 0)
            *c.sops += (unsigned long long)Wd * (unsigned)max(0, __popc(lv.op_mask & ((1u << d) - 1u)) - 1);
    }
    const bool any_excl = (lv.excl_mask & (uint8_t)((2u << d) - 1)) != 0;
    if (c.lane_bitmap) {
        // one candidate per lane, the candidates ranked in increasing order:
        // lane l owns words [l per, (l + 1) per) of S, a warp scan of their
        // popcounts ranks every set bit, and each round hands the next 32
        // ranks of this part to the 32 lanes, so that every lane but those of
        // the last round has a candidate. Neighbouring ranks have similar
        // windows, so the lanes' row scans (16-byte loads over the rows and
        // sets, both padded to multiples of 4 words) stay balanced.
        const int per = (Ws + 31) >> 5;
        const int wb0 = min(Ws, c.lane * per), wb1 = min(Ws, wb0 + per);
        int own = 0;
        for (int w = wb0; w < wb1; ++w) own += __popc(S[w]);
        int incl = own;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if (c.lane >= o) incl += t;
        }
        const int T = __shfl_sync(kFull, incl, 31);
        const int excl = incl - own;
        const int np = (d == 2) ? nparts : 1, pt = (d == 2) ? part : 0;
        const int J = (T > pt) ? (T - pt + np - 1) / np : 0;   // this part's candidates
        const uint4* PP4 = reinterpret_cast<const uint4*>(PP);
        unsigned long long mine_cnt = 0;
        for (int j0 = 0; j0 < J; j0 += 32) {
            if (over(c)) return;
            const int j = j0 + c.lane;
            const int r = pt + np * min(j, J - 1);
            int ol = 0;                               // lane owning rank r
#pragma unroll
            for (int st = 16; st; st >>= 1) {
                const int e = __shfl_sync(kFull, excl, ol + st);
                if (e <= r) ol += st;
            }
            const int owner_excl = __shfl_sync(kFull, excl, ol);
            if (j >= J) continue;
            int rem = r - owner_excl;
            int w = ol * per;
            uint32_t bw = S[w];
            for (int pc = __popc(bw); rem >= pc; pc = __popc(bw)) { rem -= pc; bw = S[++w]; }
            int pos = 0;                              // the rem-th set bit of bw
#pragma unroll
            for (int h = 16; h; h >>= 1) {
                const int lowc = __popc(bw & ((1u << h) - 1u));
                if (rem >= lowc) { rem -= lowc; bw >>= h; pos += h; }
            }
            const int x = 32 * w + pos;
            const int lo = x_lo ? max(base.lo, x) : base.lo;
            const int hi = x_hi ? min(base.hi, x) : base.hi;
            const int w0 = max(0, (lo + 1) >> 5);
            const int w1 = min(Wd, (hi == INT_MAX) ? Wd : ((hi + 31) >> 5));
            const uint4* rx4 = reinterpret_cast<const uint4*>(c.core_bits + (size_t)x * c.core_words);
            int cnt = 0;
            if (w0 < w1) {
                const uint32_t m_first = window_bits(w0, lo, hi), m_last = window_bits(w1 - 1, lo, hi);
                const int q0 = w0 >> 2, q1 = (w1 - 1) >> 2;
                for (int q = q0; q <= q1; ++q) {
                    const uint4 a = PP4[q];
                    const uint4 rr = uses_x ? __ldg(rx4 + q) : make_uint4(~0u, ~0u, ~0u, ~0u);
                    uint32_t m[4] = {a.x & rr.x, a.y & rr.y, a.z & rr.z, a.w & rr.w};
                    if (q == q0 || q == q1) {         // words outside [w0, w1), partial end words
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            const int ww = 4 * q + t;
                            uint32_t keep = (ww < w0 || ww >= w1) ? 0u : ~0u;
                            if (ww == w0) keep &= m_first;
                            if (ww == w1 - 1) keep &= m_last;
                            m[t] &= keep;
                        }
                    }
                    cnt += __popc(m[0]) + __popc(m[1]) + __popc(m[2]) + __popc(m[3]);
                }
                if (c.sops) *c.sops += (unsigned long long)(w1 - w0) * (uses_x ? 2u : 1u);   // AND + POPC per word
            }
            if (any_excl) {
                for (int jj = 0; jj <= d; ++jj) {
                    if (!(lv.excl_mask >> jj & 1)) continue;
                    const int y = (jj == d) ? x : v[jj];
                    if (y <= lo || y >= hi || y >= 32 * Wd) continue;
                    bool in = (PP[y >> 5] >> (y & 31)) & 1u;
                    if (in && uses_x) in = (__ldg(c.core_bits + (size_t)x * c.core_words + (y >> 5)) >> (y & 31)) & 1u;
                    cnt -= in;
                }
            }
            mine_cnt += (unsigned)cnt;
        }
        acc.add(mine_cnt);
        return;
    }
    int word = -1;
    uint32_t bits = 0;
    int ordinal = 0;
    for (;;) {
        const int x = bitmap_next(S, Ws, word, bits);
        if (x < 0 || over(c)) break;
        if (d == 2 && (ordinal++ % nparts) != part) continue;   // another part's candidate
        v[d] = x;
        Window win = base;
        if (x_lo) win.lo = max(win.lo, x);
        if (x_hi) win.hi = min(win.hi, x);
        const int w0 = max(0, (win.lo + 1) >> 5);
        const int w1 = min(Wd, (win.hi == INT_MAX) ? Wd : ((win.hi + 31) >> 5));
        const uint32_t* rx = c.core_bits + (size_t)x * c.core_words;
        unsigned long long cnt = 0;
        for (int w = w0 + c.lane; w < w1; w += 32) {
            uint32_t m = PP[w] & window_bits(w, win.lo, win.hi);
            if (uses_x) m &= __ldg(rx + w);
            cnt += __popc(m);
        }
        if (c.sops && c.lane == 0 && w1 > w0) *c.sops += (unsigned long long)(w1 - w0) * (uses_x ? 2u : 1u);
        acc.add(cnt);
        if (any_excl && c.lane == 0) {
            int hits = 0;
            for (int j = 0; j <= d; ++j) {
                if (!(lv.excl_mask >> j & 1)) continue;
                const int y = v[j];
                if (y <= win.lo || y >= win.hi || y >= 32 * Wd) continue;
                bool in = (PP[y >> 5] >> (y & 31)) & 1u;
                if (in && uses_x) in = (__ldg(rx + (y >> 5)) >> (y & 31)) & 1u;
                hits += in;
            }
            acc.sub((unsigned long long)hits);
        }
    }
}

// Rank of a set bit of S (Ws words) for one lane, as the three-level lane
// tail uses it (the last-two lane path above runs the same scan inline):
// lane l owns words [l per, (l + 1) per); `excl` is the number of set bits
// in the words of lanes below l, `T` the total.
struct RankScan {
    int per, excl, T;
};

__device__ __forceinline__ RankScan rank_scan(const TaskCtx& c, const uint32_t* S, int Ws) {
    RankScan r;
    r.per = (Ws + 31) >> 5;
    const int wb0 = min(Ws, c.lane * r.per), wb1 = min(Ws, wb0 + r.per);
    int own = 0;
    for (int w = wb0; w < wb1; ++w) own += __popc(S[w]);
    int incl = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, o);
        if (c.lane >= o) incl += t;
    }
    r.T = __shfl_sync(kFull, incl, 31);
    r.excl = incl - own;
    return r;
}

// The set bit of rank r (0-based) of S. Called by every lane (r may differ).
__device__ __forceinline__ int rank_select(const uint32_t* S, const RankScan& rs, int r) {
    int ol = 0;                               // lane owning rank r
#pragma unroll
    for (int st = 16; st; st >>= 1) {
        const int e = __shfl_sync(kFull, rs.excl, ol + st);
        if (e <= r) ol += st;
    }
    int rem = r - __shfl_sync(kFull, rs.excl, ol);
    int w = ol * rs.per;
    uint32_t bw = S[w];
    for (int pc = __popc(bw); rem >= pc; pc = __popc(bw)) { rem -= pc; bw = S[++w]; }
    int pos = 0;                              // the rem-th set bit of bw
#pragma unroll
    for (int h = 16; h; h >>= 1) {
        const int lowc = __popc(bw & ((1u << h) - 1u));
        if (rem >= lowc) { rem -= lowc; bw >>= h; pos += h; }
    }
    return 32 * w + pos;
}

// The last three levels with one candidate of depth d = k-3 per lane, for
// plans whose last two levels are built incrementally (each is the set
// before it AND the row of the vertex bound before it, inside a window no
// wider than the one before). Lane-held x = v_d walks the set of depth k-2,
// S_d AND row(x) inside that level's window; for each member y it counts the
// last level's set, S_d AND row(x) AND row(y) inside its window. Matched
// vertices v_j (j < d) are removed from both sets where they lie inside
// them (x and y are never in their own rows). One round of the warp hands
// the next 32 candidates of this part to the lanes; each lane then runs its
// candidate's whole subtree without further warp-wide steps.
__device__ __forceinline__ void bitmap_last_three(const TaskCtx& c, int* v, int Ws, Acc& acc, int part,
                                                  int nparts) {
    const GpPlan& P = *c.P;
    const int d = P.k - 3, e = P.k - 2;
    const GpLevel& le = P.lvl[e];
    const GpLevel& lL = P.lvl[P.k - 1];
    const uint32_t* S = c.bm + (size_t)d * c.bm_stride;
    const uint8_t xb = (uint8_t)(1u << d), yb = (uint8_t)(1u << e);
    const Window be = window(le.lo_mask & (uint8_t)~xb, le.hi_mask & (uint8_t)~xb, v);
    const Window bL = window(lL.lo_mask & (uint8_t)~(xb | yb), lL.hi_mask & (uint8_t)~(xb | yb), v);
    const bool e_xlo = le.lo_mask & xb, e_xhi = le.hi_mask & xb;
    const bool L_xlo = lL.lo_mask & xb, L_xhi = lL.hi_mask & xb;
    const bool L_ylo = lL.lo_mask & yb, L_yhi = lL.hi_mask & yb;
    const uint8_t below = (uint8_t)((1u << d) - 1u);
    const uint8_t ex_e = le.excl_mask & below, ex_L = (uint8_t)((le.excl_mask | lL.excl_mask) & below);
    const RankScan rs = rank_scan(c, S, Ws);
    const int np = (d == 2) ? nparts : 1, pt = (d == 2) ? part : 0;
    const int J = (rs.T > pt) ? (rs.T - pt + np - 1) / np : 0;
    const uint4* S4 = reinterpret_cast<const uint4*>(S);
    unsigned long long mine = 0;
    for (int j0 = 0; j0 < J; j0 += 32) {
        if (over(c)) return;
        const int j = j0 + c.lane;
        const int x = rank_select(S, rs, pt + np * min(j, J - 1));
        if (j >= J) continue;
        const uint32_t* rx = c.core_bits + (size_t)x * c.core_words;
        const uint4* rx4 = reinterpret_cast<const uint4*>(rx);
        const int lo_e = e_xlo ? max(be.lo, x) : be.lo;
        const int hi_e = e_xhi ? min(be.hi, x) : be.hi;
        const int we0 = max(0, (lo_e + 1) >> 5);
        const int we1 = min(Ws, (hi_e == INT_MAX) ? Ws : ((hi_e + 31) >> 5));
        if (c.sops && we1 > we0) *c.sops += (unsigned long long)(we1 - we0);   // S AND row(x) per word
        for (int w = we0; w < we1; ++w) {
            uint32_t m = S[w] & __ldg(rx + w);
            if (w == we0 || w == we1 - 1) m &= window_bits(w, lo_e, hi_e);
            while (m) {
                const int y = 32 * w + __ffs(m) - 1;
                m &= m - 1;
                if (ex_e) {
                    bool skip = false;
                    for (int jj = 0; jj < d; ++jj) skip |= ((ex_e >> jj) & 1) && v[jj] == y;
                    if (skip) continue;
                }
                int lo = bL.lo, hi = bL.hi;
                if (L_xlo) lo = max(lo, x);
                if (L_ylo) lo = max(lo, y);
                if (L_xhi) hi = min(hi, x);
                if (L_yhi) hi = min(hi, y);
                const int w0 = max(0, (lo + 1) >> 5);
                const int w1 = min(Ws, (hi == INT_MAX) ? Ws : ((hi + 31) >> 5));
                const uint32_t* ry = c.core_bits + (size_t)y * c.core_words;
                const uint4* ry4 = reinterpret_cast<const uint4*>(ry);
                int cnt = 0;
                if (w0 < w1) {
                    const uint32_t m_first = window_bits(w0, lo, hi), m_last = window_bits(w1 - 1, lo, hi);
                    const int q0 = w0 >> 2, q1 = (w1 - 1) >> 2;
                    for (int q = q0; q <= q1; ++q) {
                        const uint4 a = S4[q], b = __ldg(rx4 + q), f = __ldg(ry4 + q);
                        uint32_t t4[4] = {a.x & b.x & f.x, a.y & b.y & f.y, a.z & b.z & f.z, a.w & b.w & f.w};
                        if (q == q0 || q == q1) {
#pragma unroll
                            for (int t = 0; t < 4; ++t) {
                                const int ww = 4 * q + t;
                                uint32_t keep = (ww < w0 || ww >= w1) ? 0u : ~0u;
                                if (ww == w0) keep &= m_first;
                                if (ww == w1 - 1) keep &= m_last;
                                t4[t] &= keep;
                            }
                        }
                        cnt += __popc(t4[0]) + __popc(t4[1]) + __popc(t4[2]) + __popc(t4[3]);
                    }
                    if (c.sops) *c.sops += 3ull * (unsigned long long)(w1 - w0);   // two ANDs + POPC per word
                }
                if (c.sops) *c.sops += 1;                                          // y taken from the set
                if (ex_L) {
                    for (int jj = 0; jj < d; ++jj) {
                        if (!((ex_L >> jj) & 1)) continue;
                        const int u = v[jj];
                        if (u <= lo || u >= hi || u >= 32 * Ws) continue;
                        const int uw = u >> 5;
                        cnt -= (int)((S[uw] & __ldg(rx + uw) & __ldg(ry + uw)) >> (u & 31) & 1u);
                    }
                }
                mine += (unsigned)cnt;
            }
        }
    }
    acc.add(mine);
}

__device__ void bitmap_task(const TaskCtx& c, int* v, Acc& acc, int part, int nparts) {
    const GpPlan& P = *c.P;
    const int k = P.k;
    const int W = (v[1] + 31) >> 5;          // every later candidate is below v1
    const bool n0_smem = v[0] >= c.core_n;
    if (n0_smem) {                           // N(v0) ∩ [0, v1) as a bitmap
        for (int w = c.lane; w < W; w += 32) c.bm[w] = 0u;
        __syncwarp();
        const List a = nbr(c, v[0]);
        const int n = lower_bound(a.p, a.n, v[1]);
        for (int i = c.lane; i < n; i += 32) {
            const int x = __ldg(a.p + i);
            atomicOr(c.bm + (x >> 5), 1u << (x & 31));
        }
        if (c.sops && c.lane == 0) *c.sops += (unsigned long long)n;           // one OR per element
        __syncwarp();
    }
    if (k == 4) {
        const int W2 = bitmap_build(c, v, 2, W, W, n0_smem);
        bitmap_last_two(c, v, W, W2, n0_smem, acc, part, nparts);
        return;
    }
    // the last three levels one candidate per lane when the last two sets
    // are incremental (clique-like tails)
    const bool three = c.lane_three && P.lvl[k - 2].bm_inc && P.lvl[k - 1].bm_inc;
    int word[GP_MAX_K], Wd[GP_MAX_K];
    uint32_t bits[GP_MAX_K];
    int d = 2, ordinal2 = 0;
    Wd[2] = bitmap_build(c, v, 2, W, W, n0_smem);
    if (three && k == 5) {
        bitmap_last_three(c, v, Wd[2], acc, part, nparts);
        return;
    }
    word[2] = -1;
    bits[2] = 0;
    while (d >= 2) {
        if (over(c)) return;
        const int x = bitmap_next(c.bm + (size_t)d * c.bm_stride, Wd[d], word[d], bits[d]);
        if (x < 0) { --d; continue; }
        if (c.sops && c.lane == 0) *c.sops += 1;                               // candidate taken from the set
        if (d == 2 && (ordinal2++ % nparts) != part) continue;  // another part's candidate
        v[d] = x;
        Wd[d + 1] = bitmap_build(c, v, d + 1, W, Wd[d], n0_smem);
        if (three && d + 1 == k - 3) {
            bitmap_last_three(c, v, Wd[d + 1], acc, 0, 1);
        } else if (d + 1 == k - 2) {
            bitmap_last_two(c, v, W, Wd[d + 1], n0_smem, acc, 0, 1);
        } else {
            ++d;
            word[d] = -1;
            bits[d] = 0;
        }
    }
}

// Remaining loops of one edge task (v0, v1), or of part `part` of `nparts`
// of it: the parts share out the candidates of depth 2.
template <bool kGeneralIep>
__device__ void run_task(const TaskCtx& c, int v0, int v1, Acc& acc, int part, int nparts) {
    const GpPlan& P = *c.P;
    const int k = P.k;
    if (c.task_cycles > 0) {                 // work-item cycle limit
        if (*(volatile int*)c.job_abort) return;
        const long long now = __shfl_sync(kFull, clock64(), 0);
        if (c.lane == 0) *c.deadline = now + c.task_cycles;
        __syncwarp();
    }
    int v[GP_MAX_K];
    List lst[GP_MAX_K];
    int cur[GP_MAX_K];
#pragma unroll
    for (int i = 0; i < GP_MAX_K; ++i) v[i] = -1;
    v[0] = v0;
    v[1] = v1;
    if (P.core_dfs && c.bm && v1 < c.core_n) { bitmap_task(c, v, acc, part, nparts); return; }
    const int d_iep = P.iep ? k - 1 - P.iep : -1;   // last outer depth of an inclusion-exclusion plan
    if (k == 3 || d_iep == 1) {
        if (part != 0) return;                 // no depth-2 loop to share out
        run_builds(c, 1, v);
        if (k == 3) count_last(c, v, acc);
        else iep_count<kGeneralIep>(c, v, acc);
        return;
    }
    run_builds(c, 1, v);
    auto prepare = [&](int dd) {
        const GpLevel& L = P.lvl[dd];
        lst[dd] = clip((L.src_kind == 1) ? nbr(c, v[L.src]) : slot(c, L.src), window(L.lo_mask, L.hi_mask, v));
        cur[dd] = 0;
    };
    const bool lane_last = !P.iep && P.lvl[k - 2].nbuild == 0;
    int d = 2;
    prepare(2);
    if (nparts > 1) {                          // this part's share of depth 2
        const int n = lst[2].n;
        const int b = (int)((int64_t)n * part / nparts), e = (int)((int64_t)n * (part + 1) / nparts);
        lst[2].p += b;
        lst[2].n = e - b;
    }
    while (d >= 2) {
        if (lane_last && d == k - 2) {
            lane_parallel_last_two(c, v, lst[d], acc);
            --d;
            continue;
        }
        if (cur[d] >= lst[d].n) { --d; continue; }
        if (over(c)) return;
        const int x = __ldg(lst[d].p + cur[d]);
        ++cur[d];
        if (c.sbytes && c.lane == 0) *c.sbytes += 4;
        const uint8_t ex = P.lvl[d].excl_mask;
        bool skip = false;
        for (int j = 0; j < d; ++j) skip |= ((ex >> j) & 1) && v[j] == x;
        if (skip) continue;
        v[d] = x;
        run_builds(c, d, v);
        if (d == d_iep) iep_count<kGeneralIep>(c, v, acc);
        else if (d == k - 2) count_last(c, v, acc);
        else { ++d; prepare(d); }
    }
}

template <bool kStats, int kMinBlocks, bool kGeneralIep>
__global__ void __launch_bounds__(kWarps * 32, kMinBlocks)
k_count(const CountJob* __restrict__ jobs, int njobs, int64_t total,
        unsigned long long* __restrict__ cursor, unsigned long long* __restrict__ results,
        int32_t* __restrict__ slot_pool, int64_t warp_elems, int chunk, long long budget,
        int* __restrict__ err, unsigned long long* __restrict__ stats, int lane_work, int use_core,
        int bm_stride, int bm_sets, long long task_cycles, int* __restrict__ aborts, int lane_bitmap) {
    unsigned long long my_bytes = 0, my_ops = 0;
    extern __shared__ uint32_t s_bitmaps[];   // bm_sets x bm_stride words per warp (may be empty)
    __shared__ GpPlan s_plan[kWarps];
    __shared__ int s_len[kWarps][GP_MAX_SLOTS];
    __shared__ long long s_deadline[kWarps];
    __shared__ unsigned s_iep[kWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * kWarps + w;
    TaskCtx c;
    c.P = &s_plan[w];
    c.iep_cnt = s_iep[w];
    c.slots = slot_pool + gw * warp_elems;
    c.slen = s_len[w];
    c.bm_stride = bm_stride;
    c.bm = (bm_stride > 0) ? s_bitmaps + (size_t)w * bm_sets * bm_stride : nullptr;
    c.lane = lane;
    c.lane_work = lane_work;
    c.deadline = &s_deadline[w];
    c.labels = nullptr;
    c.lane_bitmap = lane_bitmap != 0;
    c.lane_three = lane_bitmap == 2;
    const int bitmap_mode = lane_bitmap;    // 0 warp, 1 lane (last two levels), 2 lane (last three where allowed)
    c.task_cycles = task_cycles;
    c.job_abort = aborts;
    if (lane == 0) s_deadline[w] = 0;
    __syncwarp();
    c.err = err;
    c.row_ptr = nullptr;
    c.col = nullptr;
    c.core_bits = nullptr;
    c.core_n = 0;
    c.core_words = 0;
    c.slot_cap = 0;
    c.n_vertices = 0;
    c.sbytes = kStats ? &my_bytes : nullptr;
    c.sops = kStats ? &my_ops : nullptr;
    int cur_job = -1;
    int64_t job_lo = 0, job_hi = 0, job_begin = 0, job_heavy = 0;
    int job_split = 1;
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
                if (peek - jobs[lo].task_offset < jobs[lo].heavy * jobs[lo].split) grab = 1;
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
                c.job_abort = aborts + lo;
                const CountJob& J = jobs[lo];
                const int* src = reinterpret_cast<const int*>(&J.plan);
                int* dst = reinterpret_cast<int*>(&s_plan[w]);
                for (int i = lane; i < (int)(sizeof(GpPlan) / 4); i += 32) dst[i] = src[i];
                __syncwarp();
                job_lo = J.task_offset;
                job_hi = J.task_offset + J.nvirt;
                job_begin = J.task_begin;
                job_heavy = J.heavy;
                job_split = J.split > 0 ? J.split : 1;
                c.row_ptr = J.row_ptr;
                c.col = J.col;
                c.core_bits = J.core_bits;
                c.core_n = (use_core && J.core_bits) ? J.core_n : 0;
                // bitmap subtree: one candidate per lane (mode 1 or 2), and
                // in mode 2 the three-level lane tail where the plan allows
                c.lane_bitmap = bitmap_mode != 0;
                c.lane_three = bitmap_mode == 2;
                if (c.core_n == 0 || J.core_words > c.bm_stride) c.bm = nullptr;
                else if (bm_stride > 0 && J.plan.k - 1 <= bm_sets)
                    c.bm = s_bitmaps + (size_t)w * bm_sets * bm_stride;
                else c.bm = nullptr;
                c.core_words = J.core_words;
                c.slot_cap = J.slot_cap;
                c.n_vertices = J.n;
            }
            const int64_t tend = min(t1, job_hi);
            // work items of the split high-degree prefix: (task, part)
            const int64_t hp = job_heavy * job_split;
            int64_t lt = t - job_lo;
            const int64_t lt_end = tend - job_lo;
            const uint8_t lo1s = s_plan[w].lvl[1].lo_mask & 1, hi1s = s_plan[w].lvl[1].hi_mask & 1;
            for (; lt < lt_end && lt < hp; ++lt) {
                const int64_t eh = job_begin + lt / job_split;
                const int part = (int)(lt % job_split);
                int rl = 0, rh = c.n_vertices - 1;
                while (rl < rh) {
                    int mid = (rl + rh + 1) >> 1;
                    if (__ldg(c.row_ptr + mid) <= eh) rl = mid; else rh = mid - 1;
                }
                const int hv1 = __ldg(c.col + eh);
                if (lo1s && !(hv1 > rl)) continue;
                if (hi1s && !(hv1 < rl)) continue;
                run_task<kGeneralIep>(c, rl, hv1, acc, part, job_split);
            }
            if (lt >= lt_end) { t = tend; continue; }
            int64_t e = job_begin + job_heavy + (lt - hp);
            const int64_t e_end = job_begin + job_heavy + (lt_end - hp);
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
                    run_task<kGeneralIep>(c, v0, v1, acc, 0, 1);
                }
            }
            t = tend;
        }
    }
    if (cur_job >= 0) flush(acc, results + 2 * cur_job);
    // busy cycles: from this warp's start to the moment it found no work
    // left (the persistent loop's exit); summed over warps it measures the
    // launch's total work, independent of how evenly the work spread
    if (lane == 0) atomicAdd(stats + 2, (unsigned long long)(clock64() - t_start));
    if (kStats) {
        for (int o = 16; o; o >>= 1) my_bytes += __shfl_down_sync(kFull, my_bytes, o);
        if (lane == 0 && my_bytes) atomicAdd(stats, my_bytes);
        for (int o = 16; o; o >>= 1) my_ops += __shfl_down_sync(kFull, my_ops, o);
        if (lane == 0 && my_ops) atomicAdd(stats + 1, my_ops);
    }
}

// ---------------------------------------------------------------------------
// Listing (every embedding as a k-tuple). One warp per edge task, the loops
// of run_task without the per-lane and bitmap shortcuts; the last level's
// candidate set is materialised (in the spare slot `nslots`) and every
// element that is not an already-matched vertex is one embedding. Pass 1
// (kWrite = false) stores each task's embedding count; pass 2 writes task
// t's tuples from offset[t], in depth-first order, so the output is
// deterministic.

__device__ __forceinline__ int list_last(const TaskCtx& c, const int* v, int32_t* out, int64_t at,
                                         bool write) {
    const GpPlan& P = *c.P;
    const int L = P.k - 1;
    const GpLevel& lv = P.lvl[L];
    const Window w = window(lv.lo_mask, lv.hi_mask, v);
    List S;
    if (P.last_count_only) {
        const List a = (P.last_base_kind == 1) ? nbr(c, v[P.last_base]) : slot(c, P.last_base);
        int32_t* spare = c.slots + (size_t)P.nslots * c.slot_cap;
        const int m = warp_intersect(c, a, nbr(c, v[L - 1]), w, spare, c.slot_cap, nullptr);
        __syncwarp();
        S = List{spare, m, -1};
    } else {
        S = clip((lv.src_kind == 1) ? nbr(c, v[lv.src]) : slot(c, lv.src), w);
    }
    int total = 0;
    for (int base = 0; base < S.n; base += 32) {
        const int i = base + c.lane;
        int x = -1;
        bool keep = false;
        if (i < S.n) {
            x = __ldg(S.p + i);
            keep = true;
            for (int j = 0; j < L; ++j) keep &= !((lv.excl_mask >> j & 1) && v[j] == x);
            if (P.labeled) keep &= __ldg(c.labels + x) == P.label[L];
        }
        const unsigned m = __ballot_sync(kFull, keep);
        if (write && keep) {
            int32_t* t = out + (at + total + __popc(m & lanemask_lt())) * P.k;
            for (int d = 0; d < L; ++d) t[P.order[d]] = v[d];
            t[P.order[L]] = x;
        }
        total += __popc(m);
    }
    return total;
}

template <bool kWrite>
__global__ void __launch_bounds__(kWarps * 32, 4)
k_list(const CountJob* __restrict__ job, int64_t ntasks, unsigned long long* __restrict__ cursor,
       int64_t* __restrict__ per_task, int32_t* __restrict__ out, int32_t* __restrict__ slot_pool,
       int64_t warp_elems, int* __restrict__ err) {
    __shared__ GpPlan s_plan[kWarps];
    __shared__ int s_len[kWarps][GP_MAX_SLOTS];
    __shared__ long long s_deadline[kWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * kWarps + w;
    {
        const int* src = reinterpret_cast<const int*>(&job->plan);
        int* dst = reinterpret_cast<int*>(&s_plan[w]);
        for (int i = lane; i < (int)(sizeof(GpPlan) / 4); i += 32) dst[i] = src[i];
        if (lane == 0) s_deadline[w] = 0;
        __syncwarp();
    }
    TaskCtx c;
    c.P = &s_plan[w];
    c.iep_cnt = nullptr;                        // listing plans never use inclusion-exclusion
    c.row_ptr = job->row_ptr;
    c.col = job->col;
    c.core_bits = job->core_bits;
    c.core_n = job->core_bits ? job->core_n : 0;
    c.core_words = job->core_words;
    c.slots = slot_pool + gw * warp_elems;
    c.slot_cap = job->slot_cap;
    c.n_vertices = job->n;
    c.slen = s_len[w];
    c.bm = nullptr;
    c.bm_stride = 0;
    c.lane_bitmap = false;
    c.lane_three = false;
    c.lane = lane;
    c.lane_work = kLaneWork;
    c.err = err;
    c.sbytes = nullptr;
    c.sops = nullptr;
    c.deadline = &s_deadline[w];
    c.task_cycles = 0;
    c.job_abort = err;
    c.labels = job->labels;
    const GpPlan& P = s_plan[w];
    const int k = P.k;
    for (;;) {
        unsigned long long t0 = 0;
        if (lane == 0) t0 = atomicAdd(cursor, 1ull);
        t0 = __shfl_sync(kFull, t0, 0);
        if ((int64_t)t0 >= ntasks) break;
        const int64_t e = job->task_begin + (int64_t)t0;
        int rl = 0, rh = c.n_vertices - 1;           // source vertex of entry e
        while (rl < rh) {
            int mid = (rl + rh + 1) >> 1;
            if (__ldg(c.row_ptr + mid) <= e) rl = mid; else rh = mid - 1;
        }
        int v[GP_MAX_K];
#pragma unroll
        for (int i = 0; i < GP_MAX_K; ++i) v[i] = -1;
        v[0] = rl;
        v[1] = __ldg(c.col + e);
        int64_t found = 0;
        const int64_t at = kWrite ? per_task[t0] : 0;
        bool ok1 = !((P.lvl[1].lo_mask & 1) && !(v[1] > v[0])) && !((P.lvl[1].hi_mask & 1) && !(v[1] < v[0]));
        if (P.labeled)
            ok1 = ok1 && __ldg(c.labels + v[0]) == P.label[0] && __ldg(c.labels + v[1]) == P.label[1];
        if (ok1) {
            run_builds(c, 1, v);
            if (k == 3) {
                found += list_last(c, v, out, at + found, kWrite);
            } else {
                List lst[GP_MAX_K];
                int cur[GP_MAX_K];
                int d = 2;
                lst[2] = clip((P.lvl[2].src_kind == 1) ? nbr(c, v[P.lvl[2].src]) : slot(c, P.lvl[2].src),
                              window(P.lvl[2].lo_mask, P.lvl[2].hi_mask, v));
                cur[2] = 0;
                while (d >= 2) {
                    if (cur[d] >= lst[d].n) { --d; continue; }
                    const int x = __ldg(lst[d].p + cur[d]);
                    ++cur[d];
                    const uint8_t ex = P.lvl[d].excl_mask;
                    bool skip = false;
                    for (int j = 0; j < d; ++j) skip |= ((ex >> j) & 1) && v[j] == x;
                    if (P.labeled) skip |= __ldg(c.labels + x) != P.label[d];
                    if (skip) continue;
                    v[d] = x;
                    run_builds(c, d, v);
                    if (d == k - 2) {
                        found += list_last(c, v, out, at + found, kWrite);
                    } else {
                        ++d;
                        const GpLevel& L2 = P.lvl[d];
                        lst[d] = clip((L2.src_kind == 1) ? nbr(c, v[L2.src]) : slot(c, L2.src),
                                      window(L2.lo_mask, L2.hi_mask, v));
                        cur[d] = 0;
                    }
                }
            }
        }
        if (!kWrite && lane == 0) per_task[t0] = found;
    }
}

// Largest c <= ntasks with offsets[c] <= capacity (offsets is an exclusive
// prefix sum with ntasks + 1 entries): out[0] = c, out[1] = offsets[c].
__global__ void k_list_cut(const int64_t* __restrict__ offsets, int64_t ntasks, int64_t capacity,
                           int64_t* __restrict__ out) {
    int64_t lo = 0, hi = ntasks;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (offsets[mid] <= capacity) lo = mid; else hi = mid - 1;
    }
    out[0] = lo;
    out[1] = offsets[lo];
}

}  // namespace

namespace {

using KernelFn = void (*)(const CountJob*, int, int64_t, unsigned long long*, unsigned long long*,
                          int32_t*, int64_t, int, long long, int*, unsigned long long*, int, int, int, int,
                          long long, int*, int);

struct Geometry {
    KernelFn kern;
    int bm_stride;          // words per bitmap set (0: no bitmap subtree)
    int bm_sets;            // bitmap sets per warp (k - 1 of the largest such plan)
    size_t smem;            // dynamic shared memory per block
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
        g->total += jobs[j].nvirt;
        g->warp_elems = std::max<int64_t>(g->warp_elems, (int64_t)jobs[j].plan.nslots * jobs[j].slot_cap);
    }
    int dev = 0, nsm = 0;
    GP_CUDA_TRY(cudaGetDevice(&dev));
    GP_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int occ = 0;
    // three register budgets, chosen by the requested blocks per SM: 64
    // registers (4 blocks), 80 (3 blocks) or the compiler's choice (1 or 2).
    // Default: 3 blocks when some job runs the three-level lane tail of the
    // bitmap subtree, whose loop nest spills at 64 registers; otherwise 4
    // (the kernel is latency-bound and gains more from warps than from
    // registers)
    int want = opt.blocks_per_sm;
    if (want <= 0) {
        want = 4;
        if (!opt.no_core && opt.bitmap_mode == 2)
            for (int j = 0; j < njobs; ++j) {
                const GpPlan& P = jobs[j].plan;
                if (P.core_dfs && jobs[j].core_bits && P.k >= 5 && P.lvl[P.k - 2].bm_inc && P.lvl[P.k - 1].bm_inc)
                    want = 3;
            }
    }
    bool general_iep = false;              // some job replaces three or more loops or fuses two
    for (int j = 0; j < njobs; ++j) general_iep |= jobs[j].plan.iep >= 3 || jobs[j].plan.iep_fuse;
    if (opt.stats) {
        g->kern = (want == 1 || want == 2) ? k_count<true, 1, true>
                : (want == 3) ? k_count<true, 3, true> : k_count<true, 4, true>;
    } else if (general_iep) {
        g->kern = k_count<false, 4, true>;
    } else {
        g->kern = (want == 1 || want == 2) ? k_count<false, 1, false>
                : (want == 3) ? k_count<false, 3, false> : k_count<false, 4, false>;
    }
    // bitmap sets in shared memory when some job may search a core subtree
    g->bm_stride = 0;
    g->bm_sets = 0;
    if (!opt.no_core)
        for (int j = 0; j < njobs; ++j)
            if (jobs[j].plan.core_dfs && jobs[j].core_bits && jobs[j].core_n > 0) {
                g->bm_stride = std::max(g->bm_stride, (int)jobs[j].core_words);
                g->bm_sets = std::max(g->bm_sets, jobs[j].plan.k - 1);
            }
    g->smem = (size_t)kWarps * (size_t)g->bm_sets * (size_t)g->bm_stride * sizeof(uint32_t);
    // opt in beyond the 48 KB a block gets by default only when static and
    // dynamic shared memory together need it (seven-vertex cliques on a full
    // core: 48 KB of bitmaps alone); raising the limit for every launch moved
    // the shared-memory/L1 split and slowed L1-bound counts
    cudaFuncAttributes fa;
    GP_CUDA_TRY(cudaFuncGetAttributes(&fa, g->kern));
    if (g->smem + fa.sharedSizeBytes > 48 * 1024)
        GP_CUDA_TRY(cudaFuncSetAttribute(g->kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g->smem));
    GP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, g->kern, kWarps * 32, g->smem));
    int per_sm = std::min(want, occ);
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

int kernel_variant(const CountJob& job, const LaunchOpts& opt) {
    // the variant key geometry() would pick for this job alone: general
    // inclusion-exclusion, and the register budget of the default blocks
    // per SM (3 for the three-level lane tail, else 4)
    const GpPlan& P = job.plan;
    int want = opt.blocks_per_sm > 0 ? opt.blocks_per_sm : 4;
    if (opt.blocks_per_sm <= 0 && !opt.no_core && opt.bitmap_mode == 2 && P.core_dfs && job.core_bits && P.k >= 5 &&
        P.lvl[P.k - 2].bm_inc && P.lvl[P.k - 1].bm_inc)
        want = 3;
    return (P.iep >= 3 || P.iep_fuse ? 8 : 0) + want;
}

gp_status scratch_bytes(const CountJob* jobs, int njobs, const LaunchOpts& opt, uint64_t* bytes) {
    Geometry g;
    gp_status rc = geometry(jobs, njobs, opt, &g);
    if (rc != GP_OK) return rc;
    *bytes = (uint64_t)g.per_block * (uint64_t)g.blocks;
    return GP_OK;
}

gp_status run_count(const CountJob* jobs, int njobs, const LaunchOpts& opt, cudaStream_t st,
                    uint64_t* results, int64_t* processed, float* kernel_ms, uint64_t* algo_bytes,
                    int* aborted, uint64_t* algo_ops, uint64_t* busy) {
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
    // results (2 per job), cursor, error word, stats (bytes, operations, busy
    // warp cycles), then one abort flag per job
    const size_t res_b = sizeof(unsigned long long) * (2 * (size_t)njobs + 5) + sizeof(int) * (size_t)njobs;
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
    int* d_aborts = reinterpret_cast<int*>(d_stats + 3);
    gp_status rc = GP_OK;
    std::vector<unsigned long long> h_res((res_b + 7) / 8, 0);
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (kernel_ms) {
        GP_CUDA_TRY(cudaEventCreate(&ev0));
        GP_CUDA_TRY(cudaEventCreate(&ev1));
    }
    cudaError_t e = cudaMemcpyAsync(d_jobs, jobs, jobs_b, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_res, 0, res_b, st);
    if (e == cudaSuccess && ev0) e = cudaEventRecord(ev0, st);
    if (e == cudaSuccess && total > 0) {
        kern<<<(unsigned)blocks, kWarps * 32, geo.smem, st>>>(d_jobs, njobs, total, d_cursor, d_res, d_slots,
                                                      warp_elems, chunk, (long long)opt.budget_cycles,
                                                      d_err, d_stats, opt.lane_work > 0 ? opt.lane_work : kLaneWork,
                                                      opt.no_core ? 0 : 1, geo.bm_stride, geo.bm_sets,
                                                      (long long)opt.task_cycles, d_aborts, opt.bitmap_mode);
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
    if (algo_ops) *algo_ops = h_res[2 * njobs + 3];
    if (busy) { busy[0] = h_res[2 * njobs + 4]; busy[1] = (uint64_t)blocks * kWarps; }
    if (aborted) {
        const int* flags = reinterpret_cast<const int*>(h_res.data() + 2 * njobs + 5);
        for (int j = 0; j < njobs; ++j) aborted[j] = flags[j];
    }
    int64_t done = (int64_t)std::min<unsigned long long>(h_res[2 * njobs], (unsigned long long)total);
    if (processed) *processed = total == 0 ? 0 : done;
    return rc;
}

gp_status run_count_in_scratch(const CountJob* jobs, int njobs, void* d_scratch, size_t scratch_bytes,
                               cudaStream_t st, uint64_t* results) {
    constexpr int kMaxJobs = 8;            // host result words live on the stack
    if (njobs <= 0 || njobs > kMaxJobs) { set_error("1 to %d jobs per call", kMaxJobs); return GP_ERR_ARG; }
    // layout: [result words | job table | intermediate sets], 256-byte aligned
    const size_t words_b = ((sizeof(unsigned long long) * (2 * (size_t)njobs + 6)) + 255) & ~(size_t)255;
    const size_t jobs_b = ((sizeof(CountJob) * (size_t)njobs) + 255) & ~(size_t)255;
    if (words_b + jobs_b > scratch_bytes) {
        set_error("%d jobs need %zu bytes of fixed scratch for results and job table; it holds %zu",
                  njobs, words_b + jobs_b, scratch_bytes);
        return GP_ERR_SCRATCH;
    }
    int64_t total = 0, warp_elems = 1;
    for (int j = 0; j < njobs; ++j) {
        total += jobs[j].nvirt;
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
    bool general_iep = false;
    for (int j = 0; j < njobs; ++j) general_iep |= jobs[j].plan.iep >= 3 || jobs[j].plan.iep_fuse;
    auto kern = general_iep ? k_count<false, 4, true> : k_count<false, 4, false>;
    GP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWarps * 32, 0));
    int64_t blocks = std::min<int64_t>((int64_t)nsm * std::max(occ, 1), (int64_t)(slot_b / per_block));
    int64_t per_warp = total / (blocks * kWarps * 64);
    const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(64, per_warp));
    char* base = static_cast<char*>(d_scratch);
    unsigned long long* d_res = reinterpret_cast<unsigned long long*>(base);
    unsigned long long* d_cursor = d_res + 2 * njobs;
    int* d_err = reinterpret_cast<int*>(d_cursor + 1);
    unsigned long long* d_stats = d_cursor + 2;
    int* d_aborts = reinterpret_cast<int*>(d_stats + 3);       // unused: no cycle limit here
    CountJob* d_jobs = reinterpret_cast<CountJob*>(base + words_b);
    int32_t* d_slots = reinterpret_cast<int32_t*>(base + words_b + jobs_b);
    unsigned long long h_res[2 * kMaxJobs + 3] = {};
    const size_t nwords = 2 * (size_t)njobs + 3;
    GP_CUDA_TRY(cudaMemcpyAsync(d_jobs, jobs, sizeof(CountJob) * (size_t)njobs, cudaMemcpyHostToDevice, st));
    GP_CUDA_TRY(cudaMemsetAsync(d_res, 0, words_b, st));       // results, cursor, error word start at 0
    if (total > 0) {
        kern<<<(unsigned)blocks, kWarps * 32, 0, st>>>(d_jobs, njobs, total, d_cursor, d_res, d_slots,
                                                      warp_elems, chunk, 0, d_err, d_stats, kLaneWork, 1, 0, 0,
                                                      0, d_aborts, 2);
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

gp_status run_list(const CountJob& job, int32_t* d_out, int64_t capacity, cudaStream_t st,
                   int64_t* n_written, int64_t* cut_tasks, int64_t* total) {
    const bool count_only = capacity < 0;      // per-task counts and their sum only
    const int64_t T = job.ntasks;
    *n_written = 0;
    *cut_tasks = 0;
    if (total) *total = 0;
    if (T == 0) return GP_OK;
    int dev = 0, nsm = 0, occ = 0;
    GP_CUDA_TRY(cudaGetDevice(&dev));
    GP_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    GP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_list<false>, kWarps * 32, 0));
    const int64_t warp_elems = (int64_t)(job.plan.nslots + 1) * job.slot_cap;
    const size_t per_block = (size_t)kWarps * (size_t)warp_elems * sizeof(int32_t);
    size_t free_b = 0, total_b = 0;
    GP_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    int64_t blocks = (int64_t)nsm * std::max(occ, 1);
    while (blocks > nsm && per_block * (size_t)blocks > free_b / 4) blocks -= nsm;
    if (per_block * (size_t)blocks > free_b / 2) { set_error("listing scratch does not fit"); return GP_ERR_SCRATCH; }
    size_t scan_b = 0;
    GP_CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, scan_b, (int64_t*)nullptr, (int64_t*)nullptr, T + 1, st));
    void* mem = nullptr;
    const size_t head_b = 256;                       // job, cursor, error, cut
    const size_t cnt_b = sizeof(int64_t) * (size_t)(T + 1);
    GP_CUDA_TRY(cudaMallocAsync(&mem, head_b + sizeof(CountJob) + 2 * cnt_b + scan_b + 64, st));
    int32_t* slots = nullptr;
    if (cudaMallocAsync((void**)&slots, per_block * (size_t)blocks, st) != cudaSuccess) {
        cudaFreeAsync(mem, st);
        cudaGetLastError();
        set_error("cannot allocate listing scratch");
        return GP_ERR_NOMEM;
    }
    char* b = static_cast<char*>(mem);
    unsigned long long* cursor = reinterpret_cast<unsigned long long*>(b);
    int* err = reinterpret_cast<int*>(b + 8);
    int64_t* cut = reinterpret_cast<int64_t*>(b + 16);
    CountJob* d_job = reinterpret_cast<CountJob*>(b + head_b);
    int64_t* counts = reinterpret_cast<int64_t*>(b + head_b + ((sizeof(CountJob) + 63) & ~(size_t)63));
    int64_t* offsets = counts + (T + 1);
    void* scan_tmp = offsets + (T + 1);
    int64_t h[2] = {0, 0}, h_total = 0;
    int h_err = 0;
    cudaError_t e = cudaMemsetAsync(b, 0, head_b, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_job, &job, sizeof(CountJob), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, cnt_b, st);
    if (e == cudaSuccess) {
        k_list<false><<<(unsigned)blocks, kWarps * 32, 0, st>>>(d_job, T, cursor, counts, nullptr, slots,
                                                               warp_elems, err);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cub::DeviceScan::ExclusiveSum(scan_tmp, scan_b, counts, offsets, T + 1, st);
    if (e == cudaSuccess) {
        k_list_cut<<<1, 1, 0, st>>>(offsets, T, count_only ? 0 : capacity, cut);
        count_launch(2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, cut, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_total, offsets + T, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && h[0] > 0 && !count_only) {
        e = cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), st);
        if (e == cudaSuccess) {
            k_list<true><<<(unsigned)blocks, kWarps * 32, 0, st>>>(d_job, h[0], cursor, offsets, d_out, slots,
                                                                  warp_elems, err);
            count_launch();
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(slots, st);
    cudaFreeAsync(mem, st);
    if (e != cudaSuccess) { set_error("listing kernels failed: %s", cudaGetErrorString(e)); return GP_ERR_CUDA; }
    if (h_err) { set_error("listing kernel reported internal error %d", h_err); return GP_ERR_INTERNAL; }
    *cut_tasks = h[0];
    *n_written = h[1];
    if (total) *total = h_total;
    return GP_OK;
}

}  // namespace gp
