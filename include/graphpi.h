/* graphpi.h -- C ABI of libgraphpi_gb300.so, a GB300 (sm_103a) engine that
 * counts the embeddings of a small connected pattern in a large undirected
 * graph with the method of GraphPi (Shi, Zhai, Xu, Zhai, SC 2020).
 *
 * Problem (Section II-A): a pattern P = (V_p, E_p), 3 <= |V_p| <= 7, and a
 * data graph G = (V, E), both undirected and unlabeled. An embedding is a
 * distinct subgraph of G isomorphic to P under an injective map
 * id : V_p -> V that sends every pattern edge to a graph edge (non-induced).
 * Maps that differ by an automorphism of P are one embedding (Section II-B),
 * so the count is #maps / |Aut(P)|.
 *
 * Method: the count is produced by a nested-loop search in a matching order
 * (a "schedule", Section II-B) whose loops range over intersections of
 * sorted neighbour lists (Section IV-B, IV-E), pruned by asymmetric
 * restrictions id(a) > id(b) produced by 2-cycle automorphism elimination
 * (Algorithm 1, Section IV-A), with the configuration chosen by the
 * performance model of Section IV-C. As in the paper's overview (Section
 * III), the inputs are a pattern and a data graph given as adjacency lists.
 * Extensions below: vertex-labelled patterns, listing, inclusion-exclusion
 * counting (Section IV-D) and directed patterns on directed graphs.
 *
 * Conventions for every call:
 *  - Return value: GP_OK (0) on success, GP_PARTIAL (> 0) for a count that
 *    stopped early and can be resumed, a negative GP_ERR_* code otherwise.
 *    A failed call writes none of its outputs. gp_last_error() gives a
 *    human-readable detail for the calling thread's last failure.
 *  - Handles are opaque, created by the library and released by the
 *    matching *_destroy call (NULL is accepted and ignored). Handles are
 *    read-only after creation and may be shared between threads and
 *    streams, except that a graph must not be destroyed while a count on it
 *    is in flight, and that gp_schedule_set_iep, gp_graph_set_labels and a
 *    gp_pattern_restriction_sets call with another cap change their handle
 *    (each documents it).
 *  - Streams: a `void* stream` is a cudaStream_t (NULL = the legacy default
 *    stream). Device work runs on that stream. Every call documents whether
 *    it synchronises the stream before returning.
 *  - Array arguments are host pointers unless GP_DEVICE_PTRS is set, in
 *    which case they are device pointers on the current CUDA device.
 *  - Nothing is ever aborted: bad arguments return GP_ERR_ARG.
 */
#ifndef GRAPHPI_GB300_H
#define GRAPHPI_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t gp_status;

#define GP_OK            0
#define GP_PARTIAL       1   /* count stopped at its budget; resumable            */
#define GP_ERR_ARG      -1   /* bad argument (null pointer, size, id range)      */
#define GP_ERR_PATTERN  -2   /* pattern not symmetric 0/1, self loop, not
                                connected, or k outside [3, 7]                   */
#define GP_ERR_NOMEM    -3   /* host or device allocation failed                 */
#define GP_ERR_CUDA     -4   /* a CUDA call failed (detail in gp_last_error)     */
#define GP_ERR_OVERFLOW -5   /* the count does not fit in 64 bits                */
#define GP_ERR_TIMEOUT  -6   /* the device-side budget expired (see opts)       */
#define GP_ERR_SCRATCH  -7   /* scratch memory too small for this plan/graph     */
#define GP_ERR_INTERNAL -8   /* invariant broken inside the library              */

/* gp_graph_create_* flags */
#define GP_DEVICE_PTRS   1u  /* input arrays are device pointers                 */
#define GP_DEGREE_ORDER  2u  /* relabel vertices by non-increasing degree
                                (ties by id) before building the CSR; counts are
                                label-invariant, the relabel only speeds the
                                restricted loops                                  */
#define GP_ASSUME_CLEAN  4u  /* gp_graph_create_csr: lists are already sorted,
                                symmetric, loop-free and duplicate-free           */

typedef struct gp_graph gp_graph;
typedef struct gp_pattern gp_pattern;
typedef struct gp_schedules gp_schedules;  /* ranked plans of one pattern */

/* ------------------------------------------------------------------ graph */

/* Build the device-resident data graph from m undirected pairs over [0, n):
 * self loops dropped, both directions inserted, duplicates removed, every
 * neighbour list sorted ascending, stored as CSR with int64 row offsets and
 * int32 column ids (Section IV-E). src and dst have m entries each; n >= 0,
 * m >= 0, n < 2^31 - 1. Ids outside [0, n) give GP_ERR_ARG (checked on the
 * device before any output is produced). Input arrays are copied; the caller
 * keeps ownership. Runs on `stream` and synchronises it before returning. */
gp_status gp_graph_create_edges(const int32_t* src, const int32_t* dst, int64_t m, int32_t n,
                                uint32_t flags, void* stream, gp_graph** out);

/* Build the graph from an adjacency-list (CSR) description: row_ptr has
 * n + 1 non-decreasing int64 entries starting at 0, col has row_ptr[n]
 * int32 ids in [0, n). Unless GP_ASSUME_CLEAN is set the lists are cleaned
 * exactly as gp_graph_create_edges does (each (u, col) is one pair). Input
 * arrays are copied. Synchronises `stream`. */
gp_status gp_graph_create_csr(const int64_t* row_ptr, const int32_t* col, int32_t n,
                              uint32_t flags, void* stream, gp_graph** out);

/* Graph statistics used by the performance model (Section IV-C): vertex
 * count, undirected edge count |E|, maximum degree, and tri_cnt, the number
 * of triangles counted once per ordered vertex triple (6 x the number of
 * triangles). tri_cnt is computed on first request with the counting
 * kernel and cached; pass NULL to skip it. Synchronises `stream` when it has
 * to compute tri_cnt. */
gp_status gp_graph_stats(gp_graph* g, int64_t* n, int64_t* m_undirected, int32_t* max_deg,
                         uint64_t* tri_cnt, void* stream);

/* Copy the CSR back to host buffers (row_ptr: n + 1 entries, col: 2|E|
 * entries; either may be NULL) and, when GP_DEGREE_ORDER was used, the map
 * new id -> input id (perm: n entries, may be NULL; identity otherwise).
 * Synchronous. */
gp_status gp_graph_copy_csr(const gp_graph* g, int64_t* row_ptr, int32_t* col, int32_t* perm);

/* Device pointers of the CSR (valid until gp_graph_destroy). */
gp_status gp_graph_device_csr(const gp_graph* g, const int64_t** row_ptr, const int32_t** col,
                              int64_t* nnz);

void gp_graph_destroy(gp_graph* g);

/* ---------------------------------------------------------------- pattern */

/* Pattern from a k x k row-major 0/1 adjacency matrix (host memory),
 * 3 <= k <= 7, symmetric, zero diagonal, connected (else GP_ERR_PATTERN).
 * Computes the automorphism group (Section IV-A) on creation. */
gp_status gp_pattern_create(const uint8_t* adj, int32_t k, gp_pattern** out);

/* Vertex-labelled pattern (Section II-A: the method extends to labelled
 * graphs): as gp_pattern_create, plus labels[k]; a vertex matched to
 * pattern vertex a must carry labels[a], and automorphisms must preserve
 * labels. Labelled plans are counted by gp_count (which runs them through
 * the listing kernel's counting pass, without the bit-matrix shortcuts) and
 * listed by gp_list; the batched, time-sliced and no-allocation calls
 * reject them. */
gp_status gp_pattern_create_labeled(const uint8_t* adj, const int32_t* labels, int32_t k,
                                    gp_pattern** out);

/* Attach vertex labels to a graph: labels (host) has n entries in the
 * labelling of the input pairs (the library applies its degree relabel).
 * Replaces earlier labels, so it must not overlap a count on g.
 * Synchronous. */
gp_status gp_graph_set_labels(gp_graph* g, const int32_t* labels, void* stream);

/* |Aut(P)|: permutations of V_p that preserve E_p. */
gp_status gp_pattern_aut_count(const gp_pattern* p, uint64_t* out);

/* Restriction sets produced by Algorithm 1 (2-cycle based automorphism
 * elimination), each validated on the k-vertex complete graph. *count
 * receives how many there are: the search stops after `cap` sets (0 = the
 * default, 1024), and when it stops there the mirror image of every set
 * found (each restriction reversed, also valid) is added, so up to 2 x cap.
 * The pattern caches the sets of the last cap asked for (gp_schedule asks
 * for the default); asking for another cap recomputes them, so such a call
 * must not overlap another call on the same pattern. With pairs != NULL,
 * set `idx` is written as pairs[2r], pairs[2r+1] = (a, b) meaning
 * id(a) > id(b), r < *n_pairs <= 21. */
gp_status gp_pattern_restriction_sets(gp_pattern* p, int32_t cap, int32_t* count,
                                      int32_t idx, int32_t* pairs, int32_t* n_pairs);

/* Efficient schedules of Section IV-B (phase 1: every prefix connected;
 * phase 2: the last k' searched vertices pairwise non-adjacent, with k' the
 * largest value <= the maximum independent set size that keeps at least
 * one schedule). *count receives their number, *kprime the k' used; with
 * order != NULL schedule `idx` is written (k entries, pattern vertex ids in
 * search order). */
gp_status gp_pattern_schedules(const gp_pattern* p, int32_t* count, int32_t* kprime,
                               int32_t idx, int32_t* order);

void gp_pattern_destroy(gp_pattern* p);

/* ------------------------------------------------------------- schedules */

/* Rank every configuration (efficient schedule x restriction set) with the
 * performance model cost_i = l_i (1 - f_i) (c_i + cost_{i+1}),
 * cost_n = l_n (1 - f_n) (Section IV-C), using the graph's statistics
 * (g == NULL: |V| = 2^20, |E| = 8 |V|, tri_cnt = 6 |E|), and keep the top_k
 * (>= 1) cheapest as ready-to-run plans. May synchronise `stream` (tri_cnt). */
gp_status gp_schedule(const gp_pattern* p, gp_graph* g, int32_t top_k, void* stream,
                      gp_schedules** out);

/* A single explicit configuration: `order` (k pattern vertices in search
 * order; every prefix must be connected) and n_restr restrictions
 * restr[2r] > restr[2r+1]. The set must be valid (Algorithm 1, validate),
 * else GP_ERR_PATTERN. */
gp_status gp_schedule_explicit(const gp_pattern* p, const int32_t* order, const int32_t* restr,
                               int32_t n_restr, gp_schedules** out);

/* Switch the plans of s to (enable != 0) or from inclusion-exclusion
 * counting of the innermost loops (Section IV-D, Algorithm 2). A plan
 * qualifies when its last kk >= 2 searched vertices are pairwise
 * non-adjacent and at least two vertices are searched before them; the
 * library takes the largest such kk (at most 5) whose divisor is exact.
 * Once the outer vertices are bound, the count of kk distinct inner
 * vertices is the inclusion-exclusion sum over the set partitions of their
 * kk candidate sets (each term a product of intersection sizes). The
 * restrictions acting at the inner loops are dropped and the total is
 * divided by the number of automorphic copies of each embedding that the
 * remaining restrictions still admit. The paper computes that number with
 * no_conflict; here it is counted exactly over all k! relative vertex
 * orders, and a kk for which it is not the same for every order is not
 * used. *n_iep (may be NULL) receives how many plans switched. Counts over
 * part of the edge tasks (a task range, a budget, a time slice) are not
 * divisible on their own: those calls return the undivided 128-bit total
 * in gp_count_opts.raw_total; totals of disjoint ranges add up, and their
 * sum divided by the plan's divisor (gp_schedule_iep) is the count. With
 * kk = 5 the graph's maximum degree must be below 2^24 (GP_ERR_ARG
 * otherwise), so that every term stays inside 128 bits. This call changes
 * the handle (the one exception to read-only handles): it must not overlap
 * another call that uses s. */
gp_status gp_schedule_set_iep(gp_schedules* s, int32_t enable, int32_t* n_iep);

/* Inclusion-exclusion form of plan idx: *kk (may be NULL) receives the
 * number of innermost loops it replaces (0: plain enumeration) and
 * *divisor (may be NULL) the number by which its undivided totals are
 * divided (1 for plain plans). */
gp_status gp_schedule_iep(const gp_schedules* s, int32_t idx, int32_t* kk, uint32_t* divisor);

/* Number of plans held. */
gp_status gp_schedule_size(const gp_schedules* s, int32_t* count);

/* Plan idx: order[k], restrictions (restr[2r] > restr[2r+1], up to 21 pairs;
 * may be NULL), their number and the predicted cost (may be NULL). */
gp_status gp_schedule_get(const gp_schedules* s, int32_t idx, int32_t* order, int32_t* restr,
                          int32_t* n_restr, double* predicted_cost);

/* Performance-model cost of one configuration for given |V|, |E|
 * (undirected) and tri_cnt (ordered). */
gp_status gp_config_cost(const gp_pattern* p, const int32_t* order, const int32_t* restr,
                         int32_t n_restr, double n_vertices, double n_edges, double tri_cnt,
                         double* cost);

void gp_schedule_destroy(gp_schedules* s);

/* ----------------------------------------------------------------- count */

/* Optional tuning and control for gp_count / gp_count_batch. Zero fields
 * take the library defaults. */
typedef struct gp_count_opts {
    int32_t struct_size;      /* sizeof(gp_count_opts)                               */
    int32_t warps_per_block;  /* 1..32                                               */
    int32_t blocks_per_sm;    /* resident blocks per SM for the persistent grid       */
    int32_t chunk;            /* edge tasks claimed per work-queue grab               */
    int32_t split;            /* second-level split: every edge task whose first
                                 vertex has degree >= 256 is cut into this many
                                 parts that share out its depth-2 candidates, each
                                 handed to whichever warp is free (0/1 = no split;
                                 ignored with a budget and for 3-vertex patterns)   */
    int32_t flags;            /* GP_COUNT_STATS                                      */
    int64_t task_begin;       /* first edge task (CSR entry) to process              */
    int64_t task_end;         /* one past the last (0 = all)                         */
    int64_t budget_cycles;    /* per-warp clock64 budget; 0 = unlimited              */
    int64_t* resume_cursor;   /* host out: with GP_PARTIAL, where to resume          */
    float* kernel_ms;         /* host out (may be NULL): device time of the counting
                                 kernel, from CUDA events recorded around its launch
                                 on the caller's stream                               */
    uint64_t* algo_bytes;     /* host out (with GP_COUNT_STATS): algorithmic bytes of
                                 the count -- per intersection the cheaper of a merge
                                 (4 bytes per clipped operand element) and a binary
                                 search counted in 32-byte sectors, plus 4 bytes per
                                 stored result element and per iterated candidate    */
    int32_t lane_work;        /* probe/merge steps above which a lane hands its
                                 last-level count to the whole warp (0 = 192)        */
    int32_t reserved1;
    int64_t task_cycles;      /* per-work-item clock64 limit, checked inside the
                                 search loops (0 = none). A job whose work item
                                 outlives it is abandoned: gp_count and
                                 gp_count_batch return GP_ERR_TIMEOUT,
                                 gp_count_batch_ranges sets its next_task to -1.
                                 Other jobs of the same launch are unaffected.    */
    uint64_t* raw_total;      /* host out (may be NULL): the undivided 128-bit total
                                 of the processed tasks as (low, high) words, one
                                 pair per job in the batch calls. It equals the
                                 count for plain plans; for inclusion-exclusion
                                 plans it is the count times the plan's divisor
                                 (gp_schedule_iep). Required when an
                                 inclusion-exclusion plan counts part of the tasks
                                 (GP_ERR_ARG otherwise)                            */
    uint64_t* algo_ops;       /* host out (with GP_COUNT_STATS; may be NULL): word
                                 operations of the bitmap subtree -- one per 32-bit
                                 word ANDed, popcounted or scattered, and one per
                                 candidate taken from a set (the bitmap
                                 counterpart of algo_bytes, which then covers the
                                 list path only)                                   */
    uint64_t* busy_cycles;    /* host out (may be NULL), 2 words: the sum over the
                                 launch's warps of the SM cycles each spent before it
                                 found no work left, and the number of warps
                                 launched. The sum measures the launch's total work
                                 even when a few long tasks set its duration; a
                                 count over a task sample scales it to the whole  */
} gp_count_opts;

/* gp_count_opts.flags */
#define GP_COUNT_STATS 1   /* run the instrumented kernel that tallies algo_bytes
                              and algo_ops on the same paths as the plain kernel
                              (slower; for measurement only)                      */
#define GP_COUNT_NO_CORE 2 /* never use the core adjacency bit matrix: every
                              membership test is a binary search                  */
#define GP_COUNT_WARP_BITMAP 4 /* bitmap subtree: count the last level one
                              candidate at a time with the whole warp (default:
                              one candidate per lane, and for plans whose last
                              two sets are incremental one candidate of depth
                              k-3 per lane running the last three levels)         */
#define GP_COUNT_LANE_BITMAP 8 /* bitmap subtree: one candidate per lane for the
                              last two levels only (GP_COUNT_WARP_BITMAP wins
                              when both are set)                                  */

/* Count the embeddings of the pattern of `s` in `g` with plan `idx`.
 * Every embedding is counted exactly once (restrictions, Algorithm 1).
 * Writes *out (host) on GP_OK and GP_PARTIAL. GP_ERR_OVERFLOW when the
 * count needs more than 64 bits. An inclusion-exclusion plan counting part
 * of the tasks (opts->task_begin / task_end, or a budget that stops it)
 * writes 0 to *out and its undivided total to opts->raw_total. Runs on
 * `stream` and synchronises it before returning; the only device-to-host
 * traffic is the 16-byte result and an error word. */
gp_status gp_count(gp_graph* g, const gp_schedules* s, int32_t idx, const gp_count_opts* opts,
                   void* stream, uint64_t* out);

/* Count several (graph, schedule, plan) jobs in one persistent launch per
 * kernel build (jobs wanting the same register budget and inclusion-
 * exclusion code share one; at most four builds exist); work items of the
 * jobs of a launch share one device work queue. out[j] receives job j's
 * count. All graphs must live on the current device. With opts->raw_total
 * (2 x njobs words) each job's undivided 128-bit total is written there too,
 * and a count beyond 64 bits is not an error: its out[j] is 0 and the count
 * is raw_total / divisor. Synchronises. */
gp_status gp_count_batch(gp_graph* const* graphs, const gp_schedules* const* scheds,
                         const int32_t* idx, int32_t njobs, const gp_count_opts* opts,
                         void* stream, uint64_t* out);

/* Time-sliced batch: like gp_count_batch, but job j covers only its edge
 * tasks [task_begin[j], task_end[j]) (task_end[j] <= 0 means all) and
 * opts->budget_cycles may stop the launch early. Work items are handed out
 * in job order, so a stopped launch leaves every job with a processed
 * prefix: out[j] receives the count over that prefix and next_task[j] the
 * first unprocessed task (== the job's end when it is complete; -1 when the
 * job was abandoned under opts->task_cycles). Returns GP_OK when every job
 * completed, GP_PARTIAL otherwise; counts over disjoint
 * task ranges add up to the full count. Inclusion-exclusion jobs need
 * opts->raw_total (2 x njobs words): their out[j] is 0 and raw_total holds
 * their undivided partial totals. Synchronises `stream`. This is the
 * call a continuous-batching server issues once per time slice. */
gp_status gp_count_batch_ranges(gp_graph* const* graphs, const gp_schedules* const* scheds,
                                const int32_t* idx, const int64_t* task_begin,
                                const int64_t* task_end, int32_t njobs,
                                const gp_count_opts* opts, void* stream, uint64_t* out,
                                int64_t* next_task);

/* Device scratch (bytes) a gp_count of plan idx on g allocates for its
 * intermediate sets with the given options (for admission control). */
gp_status gp_count_scratch_bytes(const gp_graph* g, const gp_schedules* s, int32_t idx,
                                 const gp_count_opts* opts, uint64_t* bytes);

/* Listing (the embeddings themselves, Section II-A: "find all distinct
 * subgraphs"): the embeddings of plan idx whose edge tasks lie in
 * [task_begin, task_end) (task_end <= 0: all), each written once as k
 * int32 graph vertex ids, entry a being the image of pattern vertex a (ids
 * of the graph's own labelling: with GP_DEGREE_ORDER map them back with
 * gp_graph_copy_csr's perm). out is a device buffer of capacity embeddings
 * (capacity * k int32, owned by the caller). Back-pressure: a call writes
 * the embeddings of the longest prefix of the tasks that fits, in task
 * order and, within a task, in search order (so repeated calls with the
 * returned *next_task list every embedding exactly once, in the same order
 * as one large call); *n_written receives how many were written. Returns
 * GP_OK when the range is done, GP_PARTIAL when *next_task < task_end,
 * GP_ERR_SCRATCH when the first task alone needs more than capacity.
 * Inclusion-exclusion plans cannot list (GP_ERR_ARG). Synchronises. */
gp_status gp_list(gp_graph* g, const gp_schedules* s, int32_t idx, int64_t task_begin,
                  int64_t task_end, int32_t* out, int64_t capacity, void* stream,
                  int64_t* n_written, int64_t* next_task);

/* gp_count without any memory allocation, for callers that cannot allocate
 * device memory when they count (an arena or pool owns the device memory,
 * a host application forbids cudaMalloc/cudaFree on its streams, or the
 * allocation's latency is unacceptable). The paper has no counterpart: it
 * is an interface choice of this library. Results, job table and
 * intermediate sets go into one fixed 64 MiB device array that the library
 * holds on every GPU it is loaded on until the process exits; the launch
 * uses as many blocks as fit there, so it can be much slower than gp_count.
 * A plan and graph needing more than the array holds per block of 8 warps
 * (8 x intermediate sets x max degree x 4 bytes) fail with GP_ERR_SCRATCH.
 * The first call on a device looks up the array's device address (once per
 * device); make that first call before any stream capture. All calls share
 * the array and it keeps the last call's contents (each call clears what
 * must start at zero): calls that overlap on the GPU, from any thread or
 * stream, race and must be serialised by the caller. Counts all edge tasks;
 * writes *out on GP_OK; synchronises `stream`. Also: labelled plans give
 * GP_ERR_ARG (they count through the listing kernel, which allocates);
 * under CUDA's lazy module loading the driver creates the 64 MiB array when
 * the first call on a device loads this code, so that first call reserves
 * the memory; and the call makes the graph's device current and leaves it
 * current. */
gp_status gp_count_noalloc(gp_graph* g, const gp_schedules* s, int32_t idx, void* stream,
                           uint64_t* out);

/* -------------------------------------------------------------- directed */

/* Directed patterns on directed graphs. The paper names directed patterns
 * as an extension of the method (Section II-A) without defining them; the
 * reading here: a directed pattern has arcs a -> b, an embedding is an
 * injective map that sends every pattern arc to a graph arc (non-induced),
 * and the count divides the number of such maps by |Aut(P)|, the
 * arc-preserving permutations. Algorithm 1 (Section IV-A) runs on that
 * group; where it returns no restriction set (directed cycles: their
 * rotations have no usable 2-cycles) the count runs without restrictions
 * and divides by |Aut(P)|. */
typedef struct gp_dgraph gp_dgraph;
typedef struct gp_dpattern gp_dpattern;

/* Directed graph from m arcs src[i] -> dst[i] (int32, host memory, or device
 * memory with GP_DEVICE_PTRS): loops dropped, repeated arcs kept once, out-
 * and in-lists sorted. Ids outside [0, n) give GP_ERR_ARG. Synchronises
 * `stream`; the inputs may be released on return. */
gp_status gp_dgraph_create(const int32_t* src, const int32_t* dst, int64_t m, int32_t n, uint32_t flags,
                           void* stream, gp_dgraph** out);
/* n and the number of distinct arcs (either pointer may be NULL). */
gp_status gp_dgraph_stats(const gp_dgraph* g, int64_t* n, int64_t* narcs);
/* Copy the lists back (host buffers; out_ptr and in_ptr n + 1 entries,
 * out_col and in_col narcs entries; any may be NULL). Synchronous. */
gp_status gp_dgraph_copy(const gp_dgraph* g, int64_t* out_ptr, int32_t* out_col, int64_t* in_ptr,
                         int32_t* in_col);
void gp_dgraph_destroy(gp_dgraph* g);

/* Directed pattern from a k x k row-major 0/1 matrix (adj[a * k + b] = 1:
 * arc a -> b; host memory), 3 <= k <= 7, zero diagonal, weakly connected
 * (else GP_ERR_PATTERN). Computes the arc-preserving automorphisms. */
gp_status gp_dpattern_create(const uint8_t* adj, int32_t k, gp_dpattern** out);
gp_status gp_dpattern_aut_count(const gp_dpattern* p, uint64_t* out);
void gp_dpattern_destroy(gp_dpattern* p);

/* Count the embeddings of p in g. order == NULL: the configuration the
 * performance model ranks first for the underlying undirected pattern
 * (Section IV-C). Else order (k pattern vertices; every prefix weakly
 * connected) with n_restr restrictions restr[2r] > restr[2r+1]: a valid set
 * of Algorithm 1 (else GP_ERR_PATTERN), or none (n_restr = 0; the count
 * then divides by |Aut(P)|). Writes *out on GP_OK; synchronises `stream`. */
gp_status gp_dcount(const gp_dgraph* g, gp_dpattern* p, const int32_t* order, const int32_t* restr,
                    int32_t n_restr, void* stream, uint64_t* out);

/* ------------------------------------------------------------------ misc */

const char* gp_status_str(gp_status s);
const char* gp_last_error(void);
/* Number of kernel launches the library issued on this thread since the
 * last call of this function (a launch counter for benchmarking). */
int64_t gp_take_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* GRAPHPI_GB300_H */
