/* Oracle for the pattern-count path (plain C11 + pthreads). See oracle.h.
 *
 * TEST INFRASTRUCTURE ONLY: nothing in the counting library links or calls
 * this file. Every routine is the definition written out, with no blocking,
 * fusion or reordering beyond a depth-first walk over the pattern vertices.
 */
#include "oracle.h"

#include <pthread.h>
#include <stdatomic.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ CSR */

static int cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x > y) - (x < y);
}

int oracle_build_csr(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                     int64_t* row_ptr, int32_t* col, int64_t* nnz) {
    if (n < 0 || m < 0 || (m > 0 && (!src || !dst)) || !row_ptr || !nnz) return -1;
    uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(2 * m + 1));
    if (!key) return -2;
    int64_t cnt = 0;
    for (int64_t i = 0; i < m; ++i) {
        int32_t u = src[i], v = dst[i];
        if (u < 0 || u >= n || v < 0 || v >= n) { free(key); return -1; }
        if (u == v) continue;                      /* self loop: not an edge */
        key[cnt++] = ((uint64_t)(uint32_t)u << 32) | (uint32_t)v;   /* u -> v */
        key[cnt++] = ((uint64_t)(uint32_t)v << 32) | (uint32_t)u;   /* v -> u */
    }
    qsort(key, (size_t)cnt, sizeof(uint64_t), cmp_u64);
    int64_t out = 0;
    for (int64_t i = 0; i < cnt; ++i)
        if (i == 0 || key[i] != key[i - 1]) key[out++] = key[i];   /* dedup */
    for (int32_t v = 0; v <= n; ++v) row_ptr[v] = 0;
    for (int64_t i = 0; i < out; ++i) {
        row_ptr[(key[i] >> 32) + 1]++;
        col[i] = (int32_t)(uint32_t)key[i];
    }
    for (int32_t v = 0; v < n; ++v) row_ptr[v + 1] += row_ptr[v];
    *nnz = out;
    free(key);
    return 0;
}

/* ---------------------------------------------------------- automorphisms */

static int next_perm(int* p, int k) {           /* lexicographic successor */
    int i = k - 2;
    while (i >= 0 && p[i] >= p[i + 1]) --i;
    if (i < 0) return 0;
    int j = k - 1;
    while (p[j] <= p[i]) --j;
    int t = p[i]; p[i] = p[j]; p[j] = t;
    for (int a = i + 1, b = k - 1; a < b; ++a, --b) { t = p[a]; p[a] = p[b]; p[b] = t; }
    return 1;
}

int oracle_aut_count(int32_t k, const uint8_t* adj, uint64_t* out) {
    if (k < 1 || k > 10 || !adj || !out) return -1;
    int p[10];
    for (int i = 0; i < k; ++i) p[i] = i;
    uint64_t c = 0;
    do {
        int ok = 1;
        for (int a = 0; a < k && ok; ++a)
            for (int b = 0; b < k && ok; ++b)
                if (adj[a * k + b] && !adj[p[a] * k + p[b]]) ok = 0;
        c += (uint64_t)ok;
    } while (next_perm(p, k));
    *out = c;
    return 0;
}

/* -------------------------------------------------------- map enumeration */

typedef struct {
    int k;
    int order[8];          /* order[d]: pattern vertex searched at depth d      */
    int anchor[8];         /* depth whose image's neighbours are the candidates */
    int nchk[8];           /* other earlier-searched pattern neighbours ...     */
    int chk[8][8];         /* ... whose adjacency is verified by binary search  */
    int nres[8];           /* restrictions whose later endpoint is depth d:     */
    int res_other[8][32];  /*   the other endpoint's depth                      */
    int res_gt[8][32];     /*   1: image(d) > image(other); 0: image(d) < ...   */
    int32_t n;
    const int64_t* row_ptr;
    const int32_t* col;
    int32_t root_begin, root_end, root_stride;
    int64_t entry_begin, entry_end; /* entry mode: only the CSR entries (v0, v1) of   */
    int entry_mode;                 /* [entry_begin, entry_end) start the walk       */
    const int32_t* glab;   /* graph vertex labels, or NULL (unlabelled)        */
    int32_t plab[8];       /* label required at depth d                        */
    atomic_long cursor;    /* next root index (in stride units) to hand out */
} walk_t;

static int has_edge(const walk_t* w, int32_t u, int32_t v) {
    int64_t lo = w->row_ptr[u], hi = w->row_ptr[u + 1];
    while (lo < hi) {                            /* lower bound of v */
        int64_t mid = lo + (hi - lo) / 2;
        if (w->col[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo < w->row_ptr[u + 1] && w->col[lo] == v;
}

/* May v (a neighbour of the anchor's image) be the image at depth d? */
static int admit(const walk_t* w, int d, const int32_t* img, int32_t v) {
    for (int j = 0; j < d; ++j) if (img[j] == v) return 0;                 /* injective */
    for (int c = 0; c < w->nchk[d]; ++c)
        if (!has_edge(w, img[w->chk[d][c]], v)) return 0;                   /* edges */
    for (int r = 0; r < w->nres[d]; ++r) {
        int32_t o = img[w->res_other[d][r]];
        if (w->res_gt[d][r] ? !(v > o) : !(v < o)) return 0;                /* restriction */
    }
    if (w->glab && w->glab[v] != w->plab[d]) return 0;                     /* label */
    return 1;
}

static u128 walk(const walk_t* w, int d, int32_t* img) {
    if (d == w->k) return 1;                     /* every pattern vertex mapped */
    u128 total = 0;
    int32_t a = img[w->anchor[d]];
    for (int64_t e = w->row_ptr[a]; e < w->row_ptr[a + 1]; ++e) {
        int32_t v = w->col[e];
        if (!admit(w, d, img, v)) continue;
        img[d] = v;
        total += walk(w, d + 1, img);
    }
    return total;
}

/* Row of CSR entry e: the last u with row_ptr[u] <= e. */
static int32_t entry_row(const walk_t* w, int64_t e) {
    int32_t lo = 0, hi = w->n - 1;
    while (lo < hi) {
        int32_t mid = lo + (hi - lo + 1) / 2;
        if (w->row_ptr[mid] <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

typedef struct { walk_t* w; u128 sum; } worker_t;

static void* worker_main(void* arg) {
    worker_t* me = (worker_t*)arg;
    walk_t* w = me->w;
    int32_t img[8];
    const long chunk = 16;
    if (w->entry_mode) {                         /* the walk from single entries, */
        long count = (long)(w->entry_end - w->entry_begin);   /* one per grab      */
        for (;;) {
            long s = atomic_fetch_add(&w->cursor, 1);
            if (s >= count) break;
            long e = s + 1;
            for (long i = s; i < e; ++i) {
                int64_t x = w->entry_begin + i;
                img[0] = entry_row(w, x);
                if (w->glab && w->plab[0] != w->glab[img[0]]) continue;   /* root label */
                if (!admit(w, 1, img, w->col[x])) continue;
                img[1] = w->col[x];
                me->sum += walk(w, 2, img);
            }
        }
        return NULL;
    }
    long count = (w->root_end - w->root_begin + w->root_stride - 1) / w->root_stride;
    for (;;) {
        long s = atomic_fetch_add(&w->cursor, chunk);
        if (s >= count) break;
        long e = s + chunk < count ? s + chunk : count;
        for (long i = s; i < e; ++i) {
            img[0] = (int32_t)(w->root_begin + i * w->root_stride);
            if (w->glab && w->glab[img[0]] != w->plab[0]) continue;             /* root label */
            me->sum += walk(w, 1, img);
        }
    }
    return NULL;
}

static int run_walk(walk_t* w, int32_t nthreads, u128* out) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 512) nthreads = 512;
    worker_t* ws = (worker_t*)calloc((size_t)nthreads, sizeof(worker_t));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!ws || !th) { free(ws); free(th); return -2; }
    atomic_store(&w->cursor, 0);
    for (int t = 0; t < nthreads; ++t) { ws[t].w = w; ws[t].sum = 0; }
    /* a thread that fails to start leaves its roots to the others (shared cursor) */
    for (int t = 1; t < nthreads; ++t)
        if (pthread_create(&th[t], NULL, worker_main, &ws[t]) != 0) ws[t].w = NULL;
    worker_main(&ws[0]);
    for (int t = 1; t < nthreads; ++t) if (ws[t].w) pthread_join(th[t], NULL);
    u128 s = 0;
    for (int t = 0; t < nthreads; ++t) s += ws[t].sum;
    *out = s;
    free(ws); free(th);
    return 0;
}

/* Depth-first plan for a given matching order: the candidates at depth d are
 * the neighbours of the image of the first earlier-searched pattern
 * neighbour; edges to the other earlier-searched neighbours are checked. */
static int setup_walk(walk_t* w, int32_t k, const uint8_t* adj, const int32_t* order,
                      int32_t nres, const int32_t* res,
                      int32_t n, const int64_t* row_ptr, const int32_t* col) {
    if (k < 2 || k > 8 || !adj || !row_ptr || (n > 0 && !col) || n < 0) return -1;
    memset(w, 0, sizeof(*w));
    w->k = k; w->n = n; w->row_ptr = row_ptr; w->col = col;
    int pos[8];
    int seen[8] = {0};
    for (int d = 0; d < k; ++d) {
        if (order[d] < 0 || order[d] >= k || seen[order[d]]) return -1;
        seen[order[d]] = 1;
        w->order[d] = order[d];
        pos[order[d]] = d;
    }
    for (int a = 0; a < k; ++a) {
        if (adj[a * k + a]) return -1;
        for (int b = 0; b < k; ++b) if (adj[a * k + b] != adj[b * k + a]) return -1;
    }
    for (int d = 1; d < k; ++d) {
        w->anchor[d] = -1;
        for (int j = 0; j < d; ++j) {
            if (!adj[order[d] * k + order[j]]) continue;
            if (w->anchor[d] < 0) w->anchor[d] = j;
            else w->chk[d][w->nchk[d]++] = j;
        }
        if (w->anchor[d] < 0) return -1;      /* order must keep every prefix connected */
    }
    for (int r = 0; r < nres; ++r) {
        int a = res[2 * r], b = res[2 * r + 1];          /* id(a) > id(b) */
        if (a < 0 || a >= k || b < 0 || b >= k || a == b) return -1;
        int da = pos[a], db = pos[b];
        int later = da > db ? da : db;
        if (w->nres[later] >= 32) return -1;
        w->res_other[later][w->nres[later]] = da > db ? db : da;
        w->res_gt[later][w->nres[later]] = (later == da);
        w->nres[later]++;
    }
    return 0;
}

static void split128(u128 x, uint64_t* hi, uint64_t* lo) {
    *hi = (uint64_t)(x >> 64);
    *lo = (uint64_t)x;
}

/* Breadth-first order from pattern vertex 0: every later vertex has an
 * earlier neighbour when the pattern is connected. */
static int bfs_order(int32_t k, const uint8_t* adj, int32_t* order) {
    int seen[8] = {0};
    int head = 0, tail = 0;
    order[tail++] = 0; seen[0] = 1;
    while (head < tail) {
        int a = order[head++];
        for (int b = 0; b < k; ++b)
            if (adj[a * k + b] && !seen[b]) { seen[b] = 1; order[tail++] = b; }
    }
    return tail == k ? 0 : -1;
}

int oracle_count_maps(int32_t k, const uint8_t* adj,
                      int32_t n, const int64_t* row_ptr, const int32_t* col,
                      int32_t root_begin, int32_t root_end, int32_t root_stride,
                      int32_t nthreads, uint64_t* hi, uint64_t* lo) {
    if (!hi || !lo || k < 2 || k > 8 || !adj || root_stride < 1) return -1;
    int32_t order[8];
    if (bfs_order(k, adj, order)) return -1;
    walk_t* w = (walk_t*)malloc(sizeof(walk_t));
    if (!w) return -2;
    int rc = setup_walk(w, k, adj, order, 0, NULL, n, row_ptr, col);
    if (rc) { free(w); return rc; }
    if (root_begin < 0) root_begin = 0;
    if (root_end > n) root_end = n;
    if (root_end < root_begin) root_end = root_begin;
    w->root_begin = root_begin; w->root_end = root_end; w->root_stride = root_stride;
    u128 total = 0;
    rc = run_walk(w, nthreads, &total);
    free(w);
    if (rc) return rc;
    split128(total, hi, lo);
    return 0;
}

int oracle_count_restricted(int32_t k, const uint8_t* adj, const int32_t* order,
                            int32_t nres, const int32_t* res,
                            int32_t n, const int64_t* row_ptr, const int32_t* col,
                            int32_t root_begin, int32_t root_end,
                            int32_t nthreads, uint64_t* hi, uint64_t* lo) {
    if (!hi || !lo || !order || (nres > 0 && !res) || nres < 0) return -1;
    walk_t* w = (walk_t*)malloc(sizeof(walk_t));
    if (!w) return -2;
    int rc = setup_walk(w, k, adj, order, nres, res, n, row_ptr, col);
    if (rc) { free(w); return rc; }
    if (root_begin < 0) root_begin = 0;
    if (root_end > n) root_end = n;
    if (root_end < root_begin) root_end = root_begin;
    w->root_begin = root_begin; w->root_end = root_end; w->root_stride = 1;
    u128 total = 0;
    rc = run_walk(w, nthreads, &total);
    free(w);
    if (rc) return rc;
    split128(total, hi, lo);
    return 0;
}

/* --------------------------------------------------------------- labelled */

int oracle_aut_count_labeled(int32_t k, const uint8_t* adj, const int32_t* plabels, uint64_t* out) {
    if (k < 1 || k > 10 || !adj || !plabels || !out) return -1;
    int p[10];
    for (int i = 0; i < k; ++i) p[i] = i;
    uint64_t c = 0;
    do {
        int ok = 1;
        for (int a = 0; a < k && ok; ++a) {
            if (plabels[p[a]] != plabels[a]) ok = 0;
            for (int b = 0; b < k && ok; ++b)
                if (adj[a * k + b] && !adj[p[a] * k + p[b]]) ok = 0;
        }
        c += (uint64_t)ok;
    } while (next_perm(p, k));
    *out = c;
    return 0;
}

int oracle_count_labeled(int32_t k, const uint8_t* adj, const int32_t* plabels,
                         int32_t n, const int64_t* row_ptr, const int32_t* col,
                         const int32_t* glabels, int32_t nthreads, uint64_t* out) {
    if (!plabels || !glabels || !out) return -1;
    uint64_t aut;
    int rc = oracle_aut_count_labeled(k, adj, plabels, &aut);
    if (rc) return rc;
    int32_t order[8];
    if (bfs_order(k, adj, order)) return -1;
    walk_t* w = (walk_t*)malloc(sizeof(walk_t));
    if (!w) return -2;
    rc = setup_walk(w, k, adj, order, 0, NULL, n, row_ptr, col);
    if (rc) { free(w); return rc; }
    w->glab = glabels;
    for (int d = 0; d < k; ++d) w->plab[d] = plabels[order[d]];
    w->root_begin = 0; w->root_end = n; w->root_stride = 1;
    u128 maps = 0;
    rc = run_walk(w, nthreads, &maps);
    free(w);
    if (rc) return rc;
    if (maps % aut) return -3;
    u128 q = maps / aut;
    if (q >> 64) return -4;
    *out = (uint64_t)q;
    return 0;
}

/* ------------------------------------------------------------------ listing */

typedef struct { int32_t* out; int64_t cap; int64_t n; } list_sink;

static void list_walk(const walk_t* w, int d, int32_t* img, list_sink* sink) {
    if (d == w->k) {                             /* one embedding */
        if (sink->n < sink->cap)
            for (int j = 0; j < w->k; ++j) sink->out[sink->n * w->k + w->order[j]] = img[j];
        sink->n++;
        return;
    }
    int32_t a = img[w->anchor[d]];
    for (int64_t e = w->row_ptr[a]; e < w->row_ptr[a + 1]; ++e) {
        int32_t v = w->col[e];
        int ok = 1;
        for (int j = 0; j < d && ok; ++j) if (img[j] == v) ok = 0;
        for (int c = 0; c < w->nchk[d] && ok; ++c)
            if (!has_edge(w, img[w->chk[d][c]], v)) ok = 0;
        for (int r = 0; r < w->nres[d] && ok; ++r) {
            int32_t o = img[w->res_other[d][r]];
            if (w->res_gt[d][r] ? !(v > o) : !(v < o)) ok = 0;
        }
        if (!ok) continue;
        img[d] = v;
        list_walk(w, d + 1, img, sink);
    }
}

int oracle_count_restricted_entries(int32_t k, const uint8_t* adj, const int32_t* order,
                                    int32_t nres, const int32_t* res,
                                    int32_t n, const int64_t* row_ptr, const int32_t* col,
                                    int64_t entry_begin, int64_t entry_end,
                                    int32_t nthreads, uint64_t* hi, uint64_t* lo) {
    if (!hi || !lo || !order || (nres > 0 && !res) || nres < 0 || k < 2) return -1;
    walk_t* w = (walk_t*)malloc(sizeof(walk_t));
    if (!w) return -2;
    int rc = setup_walk(w, k, adj, order, nres, res, n, row_ptr, col);
    if (rc) { free(w); return rc; }
    int64_t nnz = n > 0 ? row_ptr[n] : 0;
    if (entry_begin < 0) entry_begin = 0;
    if (entry_end > nnz) entry_end = nnz;
    if (entry_end < entry_begin) entry_end = entry_begin;
    w->entry_mode = 1;
    w->entry_begin = entry_begin;
    w->entry_end = entry_end;
    u128 total = 0;
    rc = run_walk(w, nthreads, &total);
    free(w);
    if (rc) return rc;
    split128(total, hi, lo);
    return 0;
}

int oracle_list_restricted(int32_t k, const uint8_t* adj, const int32_t* order,
                           int32_t nres, const int32_t* res,
                           int32_t n, const int64_t* row_ptr, const int32_t* col,
                           int32_t root_begin, int32_t root_end,
                           int32_t* out, int64_t cap, int64_t* n_out) {
    if (!order || (nres > 0 && !res) || nres < 0 || !n_out || cap < 0 || (cap > 0 && !out)) return -1;
    walk_t* w = (walk_t*)malloc(sizeof(walk_t));
    if (!w) return -2;
    int rc = setup_walk(w, k, adj, order, nres, res, n, row_ptr, col);
    if (rc) { free(w); return rc; }
    if (root_begin < 0) root_begin = 0;
    if (root_end > n) root_end = n;
    list_sink sink = {out, cap, 0};
    int32_t img[8];
    for (int32_t r = root_begin; r < root_end; ++r) {
        img[0] = r;
        list_walk(w, 1, img, &sink);
    }
    *n_out = sink.n;
    free(w);
    return 0;
}

/* ---------------------------------------------------------------- triangles */

typedef struct {
    int32_t n; const int64_t* row_ptr; const int32_t* col;
    atomic_long cursor; int32_t nthreads;
} tri_t;
typedef struct { tri_t* t; uint64_t sum; } tri_worker_t;

static int tri_has_edge(const tri_t* t, int32_t u, int32_t v) {
    int64_t lo = t->row_ptr[u], hi = t->row_ptr[u + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (t->col[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo < t->row_ptr[u + 1] && t->col[lo] == v;
}

static void* tri_main(void* arg) {
    tri_worker_t* me = (tri_worker_t*)arg;
    tri_t* t = me->t;
    for (;;) {
        long s = atomic_fetch_add(&t->cursor, 64);
        if (s >= t->n) break;
        long e = s + 64 < t->n ? s + 64 : t->n;
        for (long a = s; a < e; ++a)                    /* a < b < c, all adjacent */
            for (int64_t i = t->row_ptr[a]; i < t->row_ptr[a + 1]; ++i) {
                int32_t b = t->col[i];
                if (b <= a) continue;
                for (int64_t j = t->row_ptr[a]; j < t->row_ptr[a + 1]; ++j) {
                    int32_t c = t->col[j];
                    if (c <= b) continue;
                    me->sum += (uint64_t)tri_has_edge(t, b, c);
                }
            }
    }
    return NULL;
}

int oracle_triangles(int32_t n, const int64_t* row_ptr, const int32_t* col,
                     int32_t nthreads, uint64_t* out) {
    if (n < 0 || !row_ptr || !out) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 512) nthreads = 512;
    tri_t t;
    t.n = n; t.row_ptr = row_ptr; t.col = col; t.nthreads = nthreads;
    atomic_store(&t.cursor, 0);
    tri_worker_t* ws = (tri_worker_t*)calloc((size_t)nthreads, sizeof(tri_worker_t));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!ws || !th) { free(ws); free(th); return -2; }
    for (int i = 0; i < nthreads; ++i) ws[i].t = &t;
    for (int i = 1; i < nthreads; ++i)
        if (pthread_create(&th[i], NULL, tri_main, &ws[i]) != 0) ws[i].t = NULL;
    tri_main(&ws[0]);
    uint64_t s = ws[0].sum;
    for (int i = 1; i < nthreads; ++i) if (ws[i].t) { pthread_join(th[i], NULL); s += ws[i].sum; }
    *out = s;
    free(ws); free(th);
    return 0;
}

/* ------------------------------------------------------ directed patterns */
/* A directed pattern has arcs a -> b (adj[a * k + b] = 1; not necessarily
 * symmetric). An embedding is an injective map f sending every pattern arc
 * a -> b to a graph arc f(a) -> f(b) (non-induced); the count is maps /
 * |Aut(P)|, Aut(P) being the arc-preserving permutations. The graph keeps
 * both the out-arcs and the in-arcs of every vertex as sorted lists. */

static int build_sorted_lists(int32_t n, int64_t m, const uint64_t* keys, int64_t* ptr, int32_t* col) {
    for (int32_t v = 0; v <= n; ++v) ptr[v] = 0;
    for (int64_t i = 0; i < m; ++i) ptr[(keys[i] >> 32) + 1]++;
    for (int32_t v = 0; v < n; ++v) ptr[v + 1] += ptr[v];
    for (int64_t i = 0; i < m; ++i) col[i] = (int32_t)(keys[i] & 0xffffffffu);
    return 0;
}

int oracle_build_dcsr(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                      int64_t* out_ptr, int32_t* out_col, int64_t* in_ptr, int32_t* in_col,
                      int64_t* narcs) {
    if (n < 0 || m < 0 || (m > 0 && (!src || !dst)) || !out_ptr || !in_ptr || !narcs) return -1;
    uint64_t* fwd = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(m + 1));
    uint64_t* rev = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(m + 1));
    if (!fwd || !rev) { free(fwd); free(rev); return -2; }
    int64_t cnt = 0;
    for (int64_t i = 0; i < m; ++i) {
        int32_t u = src[i], v = dst[i];
        if (u < 0 || u >= n || v < 0 || v >= n) { free(fwd); free(rev); return -1; }
        if (u != v)                                             /* a loop is not an arc */
            fwd[cnt++] = ((uint64_t)(uint32_t)u << 32) | (uint32_t)v;
    }
    qsort(fwd, (size_t)cnt, sizeof(uint64_t), cmp_u64);
    int64_t uniq = 0;
    for (int64_t i = 0; i < cnt; ++i)                            /* one copy of each arc */
        if (uniq == 0 || fwd[i] != fwd[uniq - 1]) fwd[uniq++] = fwd[i];
    for (int64_t i = 0; i < uniq; ++i)                           /* the same arcs by head */
        rev[i] = ((fwd[i] & 0xffffffffu) << 32) | (fwd[i] >> 32);
    qsort(rev, (size_t)uniq, sizeof(uint64_t), cmp_u64);
    build_sorted_lists(n, uniq, fwd, out_ptr, out_col);
    build_sorted_lists(n, uniq, rev, in_ptr, in_col);
    *narcs = uniq;
    free(fwd); free(rev);
    return 0;
}

int oracle_aut_count_directed(int32_t k, const uint8_t* adj, uint64_t* out) {
    if (k < 1 || k > 10 || !adj || !out) return -1;
    int p[10];
    for (int i = 0; i < k; ++i) p[i] = i;
    uint64_t c = 0;
    do {
        int keeps_arcs = 1;
        for (int a = 0; a < k; ++a)
            for (int b = 0; b < k; ++b)
                if (adj[a * k + b] && !adj[p[a] * k + p[b]]) keeps_arcs = 0;
        c += (uint64_t)keeps_arcs;
    } while (next_perm(p, k));
    *out = c;
    return 0;
}

typedef struct {
    int k;
    int order[8];
    int anchor[8];          /* earlier depth joined to depth d by an arc            */
    int from_out[8];        /* 1: candidates are the out-arcs of the anchor's image */
    int nchk[8];
    int chk_depth[8][16];   /* further arcs to verify at depth d ...                */
    int chk_fwd[8][16];     /* ... 1: image(j) -> v, 0: v -> image(j)              */
    int nres[8];
    int res_other[8][32];
    int res_gt[8][32];
    int32_t n;
    const int64_t *out_ptr, *in_ptr;
    const int32_t *out_col, *in_col;
    int32_t root_begin, root_end;
    atomic_long cursor;
} dwalk_t;

static int arc_present(const dwalk_t* w, int32_t u, int32_t v) {   /* u -> v ? */
    int64_t lo = w->out_ptr[u], hi = w->out_ptr[u + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (w->out_col[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo < w->out_ptr[u + 1] && w->out_col[lo] == v;
}

static u128 dwalk(const dwalk_t* w, int d, int32_t* img) {
    if (d == w->k) return 1;
    const int32_t a = img[w->anchor[d]];
    const int64_t* ptr = w->from_out[d] ? w->out_ptr : w->in_ptr;
    const int32_t* col = w->from_out[d] ? w->out_col : w->in_col;
    u128 total = 0;
    for (int64_t e = ptr[a]; e < ptr[a + 1]; ++e) {
        const int32_t v = col[e];
        int good = 1;
        for (int j = 0; j < d; ++j) good &= (img[j] != v);                      /* injective */
        for (int c = 0; c < w->nchk[d] && good; ++c) {
            const int32_t o = img[w->chk_depth[d][c]];
            good = w->chk_fwd[d][c] ? arc_present(w, o, v) : arc_present(w, v, o);
        }
        for (int r = 0; r < w->nres[d] && good; ++r) {
            const int32_t o = img[w->res_other[d][r]];
            good = w->res_gt[d][r] ? (v > o) : (v < o);
        }
        if (!good) continue;
        img[d] = v;
        total += dwalk(w, d + 1, img);
    }
    return total;
}

typedef struct { dwalk_t* w; u128 sum; } dworker_t;

static void* dworker_main(void* arg) {
    dworker_t* me = (dworker_t*)arg;
    int32_t img[8];
    for (;;) {
        long r = atomic_fetch_add(&me->w->cursor, 1) + me->w->root_begin;
        if (r >= me->w->root_end) break;
        img[0] = (int32_t)r;
        me->sum += dwalk(me->w, 1, img);
    }
    return NULL;
}

int oracle_count_directed(int32_t k, const uint8_t* adj, const int32_t* order,
                          int32_t nres, const int32_t* res,
                          int32_t n, const int64_t* out_ptr, const int32_t* out_col,
                          const int64_t* in_ptr, const int32_t* in_col,
                          int32_t root_begin, int32_t root_end, int32_t nthreads,
                          uint64_t* hi, uint64_t* lo) {
    if (k < 2 || k > 8 || !adj || !hi || !lo || n < 0 || !out_ptr || !in_ptr || (nres > 0 && !res))
        return -1;
    dwalk_t* w = (dwalk_t*)calloc(1, sizeof(dwalk_t));
    if (!w) return -2;
    w->k = k; w->n = n;
    w->out_ptr = out_ptr; w->out_col = out_col; w->in_ptr = in_ptr; w->in_col = in_col;
    int pos[8], seen[8] = {0};
    if (order) {
        for (int d = 0; d < k; ++d) {
            if (order[d] < 0 || order[d] >= k || seen[order[d]]) { free(w); return -1; }
            seen[order[d]] = 1;
            w->order[d] = order[d];
        }
    } else {                                  /* breadth-first over arcs of either direction */
        int head = 0, tail = 0;
        w->order[tail++] = 0; seen[0] = 1;
        while (head < tail) {
            const int x = w->order[head++];
            for (int y = 0; y < k; ++y)
                if ((adj[x * k + y] || adj[y * k + x]) && !seen[y]) { seen[y] = 1; w->order[tail++] = y; }
        }
        if (tail != k) { free(w); return -1; }
    }
    for (int d = 0; d < k; ++d) pos[w->order[d]] = d;
    for (int a = 0; a < k; ++a) if (adj[a * k + a]) { free(w); return -1; }
    for (int d = 1; d < k; ++d) {
        const int x = w->order[d];
        w->anchor[d] = -1;
        for (int j = 0; j < d; ++j) {
            const int y = w->order[j];
            const int to_x = adj[y * k + x], from_x = adj[x * k + y];
            if (!to_x && !from_x) continue;
            if (w->anchor[d] < 0) {
                w->anchor[d] = j;
                w->from_out[d] = to_x;        /* y -> x: x among the out-arcs of img(y) */
                if (to_x && from_x) {         /* the arc back still needs a check */
                    w->chk_depth[d][w->nchk[d]] = j; w->chk_fwd[d][w->nchk[d]++] = 0;
                }
                continue;
            }
            if (to_x) { w->chk_depth[d][w->nchk[d]] = j; w->chk_fwd[d][w->nchk[d]++] = 1; }
            if (from_x) { w->chk_depth[d][w->nchk[d]] = j; w->chk_fwd[d][w->nchk[d]++] = 0; }
        }
        if (w->anchor[d] < 0) { free(w); return -1; }   /* every prefix must be weakly connected */
    }
    for (int r = 0; r < nres; ++r) {
        const int a = res[2 * r], b = res[2 * r + 1];   /* id(a) > id(b) */
        if (a < 0 || a >= k || b < 0 || b >= k || a == b) { free(w); return -1; }
        const int da = pos[a], db = pos[b], later = da > db ? da : db;
        if (w->nres[later] >= 32) { free(w); return -1; }
        w->res_other[later][w->nres[later]] = da > db ? db : da;
        w->res_gt[later][w->nres[later]] = (later == da);
        w->nres[later]++;
    }
    if (root_begin < 0) root_begin = 0;
    if (root_end > n) root_end = n;
    if (root_end < root_begin) root_end = root_begin;
    w->root_begin = root_begin; w->root_end = root_end;
    atomic_store(&w->cursor, 0);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 512) nthreads = 512;
    dworker_t* ws = (dworker_t*)calloc((size_t)nthreads, sizeof(dworker_t));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!ws || !th) { free(ws); free(th); free(w); return -2; }
    for (int t = 0; t < nthreads; ++t) ws[t].w = w;
    for (int t = 1; t < nthreads; ++t)
        if (pthread_create(&th[t], NULL, dworker_main, &ws[t]) != 0) ws[t].w = NULL;
    dworker_main(&ws[0]);
    u128 s = ws[0].sum;
    for (int t = 1; t < nthreads; ++t) if (ws[t].w) { pthread_join(th[t], NULL); s += ws[t].sum; }
    split128(s, hi, lo);
    free(ws); free(th); free(w);
    return 0;
}
