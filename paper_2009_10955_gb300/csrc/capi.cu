// capi.cu -- the C ABI of libgraphpi_gb300.so (declared in include/graphpi.h).
// Argument checking, handle management and host<->device marshalling; all
// graph and counting work runs in the kernels of graph.cu and count.cu.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "engine.h"
#include "planner.h"

struct gp_pattern {
    gp::PatternInfo info;
};

struct gp_schedules {
    int k = 0;
    std::vector<gp::Config> configs;
    std::vector<GpPlan> plans;
    std::unique_ptr<gp::PatternInfo> info;   // for recompiling (inclusion-exclusion)
};

namespace gp {

namespace {
thread_local char t_error[512] = "";
thread_local int64_t t_launches = 0;
}  // namespace

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_error, sizeof(t_error), fmt, ap);
    va_end(ap);
}

void count_launch(int n) { t_launches += n; }

namespace {

gp_status fail(gp_status s, const char* msg) {
    set_error("%s", msg);
    return s;
}

// Stream-ordered device buffer released on scope exit.
struct DevBuf {
    void* p = nullptr;
    cudaStream_t st;
    explicit DevBuf(cudaStream_t s) : st(s) {}
    ~DevBuf() { if (p) cudaFreeAsync(p, st); }
};

void free_graph(gp_graph* g) {
    if (!g) return;
    if (g->labels) cudaFree(g->labels);
    if (g->row_ptr) cudaFree(g->row_ptr);
    if (g->col) cudaFree(g->col);
    if (g->perm) cudaFree(g->perm);
    if (g->core_bits) cudaFree(g->core_bits);
    delete g;
}

gp_status ensure_device(const gp_graph* g) {
    int cur = 0;
    GP_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != g->device) GP_CUDA_TRY(cudaSetDevice(g->device));
    return GP_OK;
}

// Triangle plan: schedule (0, 1, 2) with id(0) > id(1) > id(2).
gp_status triangle_count(gp_graph* g, cudaStream_t st, uint64_t* out) {
    static const uint8_t tri[9] = {0, 1, 1, 1, 0, 1, 1, 1, 0};
    PatternInfo info;
    std::string err;
    if (!pattern_init(info, tri, 3, err)) return fail(GP_ERR_INTERNAL, err.c_str());
    const int8_t sched[3] = {0, 1, 2};
    ResMask res = (1ull << res_bit(0, 1)) | (1ull << res_bit(1, 2));
    CountJob job;
    std::memset(&job, 0, sizeof(job));
    if (!compile_plan(info, sched, res, &job.plan, err)) return fail(GP_ERR_INTERNAL, err.c_str());
    job.row_ptr = g->row_ptr;
    job.col = g->col;
    job.n = g->n;
    job.slot_cap = g->max_deg > 0 ? g->max_deg : 1;
    job.task_begin = 0;
    job.ntasks = g->nnz;
    job.task_offset = 0;
    job.heavy = 0;                              // three-vertex plan: full chunks
    job.split = 1;
    job.nvirt = job.ntasks;
    job.core_bits = g->core_bits;
    job.core_n = g->core_n;
    job.core_words = g->core_words;
    uint64_t res2[2] = {0, 0};
    int64_t done = 0;
    gp_status rc = run_count(&job, 1, LaunchOpts(), st, res2, &done);
    if (rc != GP_OK) return rc;
    if (res2[1]) return fail(GP_ERR_OVERFLOW, "triangle count overflows 64 bits");
    *out = res2[0];
    return GP_OK;
}

gp_status make_job(gp_graph* g, const gp_schedules* s, int32_t idx, const gp_count_opts* opts,
                   CountJob* job) {
    if (!g || !s) return fail(GP_ERR_ARG, "null graph or schedule");
    if (idx < 0 || idx >= (int32_t)s->plans.size()) return fail(GP_ERR_ARG, "plan index out of range");
    std::memset(job, 0, sizeof(*job));
    job->plan = s->plans[idx];
    job->row_ptr = g->row_ptr;
    job->col = g->col;
    job->n = g->n;
    job->slot_cap = g->max_deg > 0 ? g->max_deg : 1;
    int64_t b = 0, e = g->nnz;
    if (opts) {
        if (opts->task_begin < 0 || opts->task_end < 0) return fail(GP_ERR_ARG, "negative task range");
        b = std::min<int64_t>(opts->task_begin, g->nnz);
        if (opts->task_end > 0) e = std::min<int64_t>(opts->task_end, g->nnz);
        if (e < b) e = b;
    }
    job->task_begin = b;
    job->ntasks = e - b;
    // single-task grabs only pay off where a task runs loops of its own; a
    // three-vertex plan handles one task per lane and wants full chunks
    job->heavy = job->plan.k == 3 ? 0 : std::min<int64_t>(std::max<int64_t>(g->heavy_end - b, 0), e - b);
    // parts per heavy task: only for counts that run to completion (a stop
    // inside a split task could not be resumed exactly)
    job->split = 1;
    if (opts && opts->split > 1 && opts->budget_cycles <= 0 && job->plan.k > 3)
        job->split = std::min(opts->split, 1024);
    job->nvirt = job->heavy * job->split + (job->ntasks - job->heavy);
    job->core_bits = g->core_bits;
    job->core_n = g->core_n;
    job->core_words = g->core_words;
    job->labels = g->labels;
    if (job->plan.labeled && !g->labels) return fail(GP_ERR_ARG, "labelled pattern on a graph without labels");
    // a term of the five-set inclusion-exclusion expansion multiplies five
    // set sizes: keep it inside 128 bits
    if (job->plan.iep == 5 && g->max_deg >= (1 << 24))
        return fail(GP_ERR_ARG, "five-loop inclusion-exclusion needs a maximum degree below 2^24");
    return GP_OK;
}

// True when a job covers every edge task of its graph.
bool whole_graph(const CountJob& job, const gp_graph* g) { return job.task_begin == 0 && job.ntasks == g->nnz; }

// A job's count from its 128-bit device total: inclusion-exclusion plans
// divide by their multiplicity, exactly.
gp_status finish_total(const GpPlan& plan, uint64_t lo, uint64_t hi, uint64_t* out) {
    unsigned __int128 t = ((unsigned __int128)hi << 64) | lo;
    if (plan.iep) {
        const unsigned __int128 d = plan.iep_div ? plan.iep_div : 1;
        if (t % d) return fail(GP_ERR_INTERNAL, "inclusion-exclusion total is not a multiple of its divisor");
        t /= d;
    }
    if (t >> 64) return fail(GP_ERR_OVERFLOW, "count does not fit in 64 bits");
    *out = (uint64_t)t;
    return GP_OK;
}

std::unique_ptr<PatternInfo> clone_pattern(const PatternInfo& p) {
    std::unique_ptr<PatternInfo> q(new (std::nothrow) PatternInfo());
    if (!q) return q;
    uint8_t adj[GP_MAX_K * GP_MAX_K];
    for (int a = 0; a < p.k; ++a)
        for (int b = 0; b < p.k; ++b) adj[a * p.k + b] = p.adj[a][b];
    std::string err;
    const bool ok = p.labeled ? pattern_init_labeled(*q, adj, p.labels, p.k, err) : pattern_init(*q, adj, p.k, err);
    if (!ok) q.reset();
    return q;
}

LaunchOpts launch_opts(const gp_count_opts* o) {
    LaunchOpts lo;
    if (o) {
        if (o->blocks_per_sm > 0) lo.blocks_per_sm = o->blocks_per_sm;
        if (o->chunk > 0) lo.chunk = o->chunk;
        if (o->budget_cycles > 0) lo.budget_cycles = o->budget_cycles;
        lo.stats = (o->flags & GP_COUNT_STATS) != 0;
        lo.no_core = (o->flags & GP_COUNT_NO_CORE) != 0;
        if (o->task_cycles > 0) lo.task_cycles = o->task_cycles;
        if (o->flags & GP_COUNT_WARP_BITMAP) lo.bitmap_mode = 0;
        else if (o->flags & GP_COUNT_LANE_BITMAP) lo.bitmap_mode = 1;
        if (o->lane_work > 0) lo.lane_work = o->lane_work;
    }
    return lo;
}

bool opts_ok(const gp_count_opts* o) {
    return !o || (o->struct_size == (int32_t)sizeof(gp_count_opts));
}

}  // namespace

gp_status single_job(gp_graph* g, const gp_schedules* s, int32_t idx, CountJob* job) {
    gp_status rc = make_job(g, s, idx, nullptr, job);
    if (rc != GP_OK) return rc;
    if (job->plan.labeled) return fail(GP_ERR_ARG, "labelled plans are counted by gp_count");
    return ensure_device(g);
}

gp_status job_total(const CountJob& job, const uint64_t* res, uint64_t* out) {
    return finish_total(job.plan, res[0], res[1], out);
}

}  // namespace gp

using namespace gp;

extern "C" {

const char* gp_status_str(gp_status s) {
    switch (s) {
        case GP_OK: return "GP_OK";
        case GP_PARTIAL: return "GP_PARTIAL";
        case GP_ERR_ARG: return "GP_ERR_ARG";
        case GP_ERR_PATTERN: return "GP_ERR_PATTERN";
        case GP_ERR_NOMEM: return "GP_ERR_NOMEM";
        case GP_ERR_CUDA: return "GP_ERR_CUDA";
        case GP_ERR_OVERFLOW: return "GP_ERR_OVERFLOW";
        case GP_ERR_TIMEOUT: return "GP_ERR_TIMEOUT";
        case GP_ERR_SCRATCH: return "GP_ERR_SCRATCH";
        case GP_ERR_INTERNAL: return "GP_ERR_INTERNAL";
        default: return "GP_UNKNOWN";
    }
}

const char* gp_last_error(void) { return t_error; }

int64_t gp_take_launch_count(void) {
    int64_t n = t_launches;
    t_launches = 0;
    return n;
}

gp_status gp_graph_create_edges(const int32_t* src, const int32_t* dst, int64_t m, int32_t n,
                                uint32_t flags, void* stream, gp_graph** out) {
    if (!out) return fail(GP_ERR_ARG, "out is null");
    if (n < 0 || n >= INT32_MAX || m < 0) return fail(GP_ERR_ARG, "bad n or m");
    if (m > 0 && (!src || !dst)) return fail(GP_ERR_ARG, "null edge arrays");
    if (flags & ~(GP_DEVICE_PTRS | GP_DEGREE_ORDER)) return fail(GP_ERR_ARG, "unknown flag");
    if (m > ((int64_t)1 << 40)) return fail(GP_ERR_ARG, "too many pairs");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::unique_ptr<gp_graph, void (*)(gp_graph*)> g(new (std::nothrow) gp_graph(), free_graph);
    if (!g) return fail(GP_ERR_NOMEM, "host allocation failed");
    GP_CUDA_TRY(cudaGetDevice(&g->device));
    const int32_t* ds = src;
    const int32_t* dd = dst;
    DevBuf bs(st), bd(st);
    if (!(flags & GP_DEVICE_PTRS) && m > 0) {
        GP_CUDA_TRY(cudaMallocAsync(&bs.p, sizeof(int32_t) * (size_t)m, st));
        GP_CUDA_TRY(cudaMallocAsync(&bd.p, sizeof(int32_t) * (size_t)m, st));
        GP_CUDA_TRY(cudaMemcpyAsync(bs.p, src, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, st));
        GP_CUDA_TRY(cudaMemcpyAsync(bd.p, dst, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, st));
        ds = static_cast<const int32_t*>(bs.p);
        dd = static_cast<const int32_t*>(bd.p);
    }
    gp_status rc = build_graph(ds, dd, m, n, (flags & GP_DEGREE_ORDER) != 0, st, g.get());
    if (rc != GP_OK) return rc;
    *out = g.release();
    return GP_OK;
}

gp_status gp_graph_create_csr(const int64_t* row_ptr, const int32_t* col, int32_t n,
                              uint32_t flags, void* stream, gp_graph** out) {
    if (!out || !row_ptr) return fail(GP_ERR_ARG, "null argument");
    if (n < 0 || n >= INT32_MAX) return fail(GP_ERR_ARG, "bad n");
    if (flags & ~(GP_DEVICE_PTRS | GP_DEGREE_ORDER | GP_ASSUME_CLEAN)) return fail(GP_ERR_ARG, "unknown flag");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool dev = (flags & GP_DEVICE_PTRS) != 0;
    int64_t nnz = 0;
    std::vector<int64_t> h_rp;
    if (dev) {
        GP_CUDA_TRY(cudaMemcpyAsync(&nnz, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        GP_CUDA_TRY(cudaStreamSynchronize(st));
    } else {
        if (row_ptr[0] != 0) return fail(GP_ERR_ARG, "row_ptr[0] must be 0");
        for (int32_t u = 0; u < n; ++u)
            if (row_ptr[u + 1] < row_ptr[u]) return fail(GP_ERR_ARG, "row_ptr must be non-decreasing");
        nnz = row_ptr[n];
    }
    if (nnz < 0) return fail(GP_ERR_ARG, "negative entry count");
    if (nnz > 0 && !col) return fail(GP_ERR_ARG, "null col");
    std::unique_ptr<gp_graph, void (*)(gp_graph*)> g(new (std::nothrow) gp_graph(), free_graph);
    if (!g) return fail(GP_ERR_NOMEM, "host allocation failed");
    GP_CUDA_TRY(cudaGetDevice(&g->device));
    DevBuf brp(st), bcol(st);
    const int64_t* drp = row_ptr;
    const int32_t* dcol = col;
    if (!dev) {
        GP_CUDA_TRY(cudaMallocAsync(&brp.p, sizeof(int64_t) * ((size_t)n + 1), st));
        GP_CUDA_TRY(cudaMallocAsync(&bcol.p, sizeof(int32_t) * (size_t)(nnz ? nnz : 1), st));
        GP_CUDA_TRY(cudaMemcpyAsync(brp.p, row_ptr, sizeof(int64_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, st));
        if (nnz) GP_CUDA_TRY(cudaMemcpyAsync(bcol.p, col, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, st));
        drp = static_cast<const int64_t*>(brp.p);
        dcol = static_cast<const int32_t*>(bcol.p);
    }
    if ((flags & GP_ASSUME_CLEAN) && !(flags & GP_DEGREE_ORDER)) {
        GP_CUDA_TRY(cudaMalloc(&g->row_ptr, sizeof(int64_t) * ((size_t)n + 1)));
        GP_CUDA_TRY(cudaMalloc(&g->col, sizeof(int32_t) * (size_t)(nnz ? nnz : 1)));
        GP_CUDA_TRY(cudaMemcpyAsync(g->row_ptr, drp, sizeof(int64_t) * ((size_t)n + 1), cudaMemcpyDeviceToDevice, st));
        if (nnz) GP_CUDA_TRY(cudaMemcpyAsync(g->col, dcol, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToDevice, st));
        g->n = n;
        g->nnz = nnz;
        gp_status rc = max_degree(g->row_ptr, n, st, &g->max_deg);
        if (rc != GP_OK) return rc;
        *out = g.release();
        return GP_OK;
    }
    DevBuf ps(st), pd(st);
    GP_CUDA_TRY(cudaMallocAsync(&ps.p, sizeof(int32_t) * (size_t)(nnz ? nnz : 1), st));
    GP_CUDA_TRY(cudaMallocAsync(&pd.p, sizeof(int32_t) * (size_t)(nnz ? nnz : 1), st));
    gp_status rc = csr_to_pairs(drp, dcol, n, nnz, static_cast<int32_t*>(ps.p), static_cast<int32_t*>(pd.p), st);
    if (rc != GP_OK) return rc;
    rc = build_graph(static_cast<int32_t*>(ps.p), static_cast<int32_t*>(pd.p), nnz, n,
                     (flags & GP_DEGREE_ORDER) != 0, st, g.get());
    if (rc != GP_OK) return rc;
    *out = g.release();
    return GP_OK;
}

gp_status gp_graph_stats(gp_graph* g, int64_t* n, int64_t* m_undirected, int32_t* max_deg,
                         uint64_t* tri_cnt, void* stream) {
    if (!g) return fail(GP_ERR_ARG, "null graph");
    if (tri_cnt) {
        std::lock_guard<std::mutex> lock(g->mu);
        if (!g->tri_done) {
            gp_status rc = ensure_device(g);
            if (rc != GP_OK) return rc;
            uint64_t t = 0;
            rc = triangle_count(g, static_cast<cudaStream_t>(stream), &t);
            if (rc != GP_OK) return rc;
            if (t > UINT64_MAX / 6) return fail(GP_ERR_OVERFLOW, "6 x triangles overflows 64 bits");
            g->tri_cnt = 6 * t;
            g->tri_done = true;
        }
        *tri_cnt = g->tri_cnt;
    }
    if (n) *n = g->n;
    if (m_undirected) *m_undirected = g->nnz / 2;
    if (max_deg) *max_deg = g->max_deg;
    return GP_OK;
}

gp_status gp_graph_copy_csr(const gp_graph* g, int64_t* row_ptr, int32_t* col, int32_t* perm) {
    if (!g) return fail(GP_ERR_ARG, "null graph");
    if (row_ptr) GP_CUDA_TRY(cudaMemcpy(row_ptr, g->row_ptr, sizeof(int64_t) * ((size_t)g->n + 1), cudaMemcpyDeviceToHost));
    if (col && g->nnz) GP_CUDA_TRY(cudaMemcpy(col, g->col, sizeof(int32_t) * (size_t)g->nnz, cudaMemcpyDeviceToHost));
    if (perm) {
        if (g->perm) GP_CUDA_TRY(cudaMemcpy(perm, g->perm, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDeviceToHost));
        else for (int32_t u = 0; u < g->n; ++u) perm[u] = u;
    }
    return GP_OK;
}

gp_status gp_graph_device_csr(const gp_graph* g, const int64_t** row_ptr, const int32_t** col,
                              int64_t* nnz) {
    if (!g) return fail(GP_ERR_ARG, "null graph");
    if (row_ptr) *row_ptr = g->row_ptr;
    if (col) *col = g->col;
    if (nnz) *nnz = g->nnz;
    return GP_OK;
}

void gp_graph_destroy(gp_graph* g) { free_graph(g); }

gp_status gp_pattern_create(const uint8_t* adj, int32_t k, gp_pattern** out) {
    if (!adj || !out) return fail(GP_ERR_ARG, "null argument");
    std::unique_ptr<gp_pattern> p(new (std::nothrow) gp_pattern());
    if (!p) return fail(GP_ERR_NOMEM, "host allocation failed");
    std::string err;
    if (!pattern_init(p->info, adj, k, err)) return fail(GP_ERR_PATTERN, err.c_str());
    *out = p.release();
    return GP_OK;
}

gp_status gp_pattern_create_labeled(const uint8_t* adj, const int32_t* labels, int32_t k, gp_pattern** out) {
    if (!adj || !labels || !out) return fail(GP_ERR_ARG, "null argument");
    std::unique_ptr<gp_pattern> p(new (std::nothrow) gp_pattern());
    if (!p) return fail(GP_ERR_NOMEM, "host allocation failed");
    std::string err;
    if (!pattern_init_labeled(p->info, adj, labels, k, err)) return fail(GP_ERR_PATTERN, err.c_str());
    *out = p.release();
    return GP_OK;
}

gp_status gp_graph_set_labels(gp_graph* g, const int32_t* labels, void* stream) {
    if (!g || (!labels && g->n > 0)) return fail(GP_ERR_ARG, "null argument");
    gp_status rc = ensure_device(g);
    if (rc != GP_OK) return rc;
    std::vector<int32_t> lab((size_t)g->n);
    if (g->perm) {                            // labels arrive in the input labelling
        std::vector<int32_t> perm((size_t)g->n);
        GP_CUDA_TRY(cudaMemcpy(perm.data(), g->perm, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDeviceToHost));
        for (int32_t i = 0; i < g->n; ++i) lab[i] = labels[perm[i]];
    } else {
        for (int32_t i = 0; i < g->n; ++i) lab[i] = labels[i];
    }
    int32_t* d = nullptr;
    GP_CUDA_TRY(cudaMalloc(&d, sizeof(int32_t) * (size_t)(g->n ? g->n : 1)));
    if (g->n) {
        cudaError_t e = cudaMemcpyAsync(d, lab.data(), sizeof(int32_t) * (size_t)g->n, cudaMemcpyHostToDevice,
                                        static_cast<cudaStream_t>(stream));
        if (e == cudaSuccess) e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) { cudaFree(d); set_error("label upload failed: %s", cudaGetErrorString(e)); return GP_ERR_CUDA; }
    }
    if (g->labels) cudaFree(g->labels);
    g->labels = d;
    return GP_OK;
}

gp_status gp_pattern_aut_count(const gp_pattern* p, uint64_t* out) {
    if (!p || !out) return fail(GP_ERR_ARG, "null argument");
    *out = p->info.auts.size();
    return GP_OK;
}

gp_status gp_pattern_restriction_sets(gp_pattern* p, int32_t cap, int32_t* count,
                                      int32_t idx, int32_t* pairs, int32_t* n_pairs) {
    if (!p || !count) return fail(GP_ERR_ARG, "null argument");
    const std::vector<ResMask>& sets = restriction_sets(p->info, cap);
    if (pairs || n_pairs) {
        if (idx < 0 || idx >= (int32_t)sets.size()) return fail(GP_ERR_ARG, "set index out of range");
        int r = 0;
        for (int a = 0; a < p->info.k; ++a)
            for (int b = 0; b < p->info.k; ++b)
                if (sets[idx] >> res_bit(a, b) & 1) {
                    if (pairs) { pairs[2 * r] = a; pairs[2 * r + 1] = b; }
                    ++r;
                }
        if (n_pairs) *n_pairs = r;
    }
    *count = (int32_t)sets.size();
    return GP_OK;
}

gp_status gp_pattern_schedules(const gp_pattern* p, int32_t* count, int32_t* kprime,
                               int32_t idx, int32_t* order) {
    if (!p || !count) return fail(GP_ERR_ARG, "null argument");
    int kp = 0;
    const std::vector<Perm>& sc = efficient_schedules(const_cast<gp_pattern*>(p)->info, &kp);
    if (order) {
        if (idx < 0 || idx >= (int32_t)sc.size()) return fail(GP_ERR_ARG, "schedule index out of range");
        for (int i = 0; i < p->info.k; ++i) order[i] = sc[idx][i];
    }
    *count = (int32_t)sc.size();
    if (kprime) *kprime = kp;
    return GP_OK;
}

void gp_pattern_destroy(gp_pattern* p) { delete p; }

gp_status gp_schedule(const gp_pattern* p, gp_graph* g, int32_t top_k, void* stream, gp_schedules** out) {
    if (!p || !out || top_k < 1) return fail(GP_ERR_ARG, "bad argument");
    double V = (double)(1 << 20), E = 8.0 * V, T = 6.0 * E;
    if (g) {
        uint64_t tri = 0;
        gp_status rc = gp_graph_stats(g, nullptr, nullptr, nullptr, &tri, stream);
        if (rc != GP_OK) return rc;
        V = g->n > 0 ? (double)g->n : 1.0;
        E = g->nnz > 0 ? (double)(g->nnz / 2) : 1.0;
        T = tri > 0 ? (double)tri : 1.0;       // keep p2 > 0 on triangle-free graphs
    }
    std::unique_ptr<gp_schedules> s(new (std::nothrow) gp_schedules());
    if (!s) return fail(GP_ERR_NOMEM, "host allocation failed");
    gp_pattern* pm = const_cast<gp_pattern*>(p);
    s->k = p->info.k;
    s->info = clone_pattern(p->info);
    if (!s->info) return fail(GP_ERR_NOMEM, "host allocation failed");
    s->configs = rank_configs(pm->info, V, E, T, top_k);
    if (s->configs.empty()) return fail(GP_ERR_PATTERN, "no configuration for this pattern");
    for (const Config& c : s->configs) {
        GpPlan plan;
        std::string err;
        if (!compile_plan(p->info, c.sched.data(), c.res, &plan, err)) return fail(GP_ERR_INTERNAL, err.c_str());
        s->plans.push_back(plan);
    }
    *out = s.release();
    return GP_OK;
}

gp_status gp_schedule_explicit(const gp_pattern* p, const int32_t* order, const int32_t* restr,
                               int32_t n_restr, gp_schedules** out) {
    if (!p || !order || !out || n_restr < 0 || (n_restr > 0 && !restr)) return fail(GP_ERR_ARG, "bad argument");
    const int k = p->info.k;
    Perm sched{};
    for (int i = 0; i < k; ++i) {
        if (order[i] < 0 || order[i] >= k) return fail(GP_ERR_ARG, "order entry outside the pattern");
        sched[i] = (int8_t)order[i];
    }
    ResMask res = 0;
    for (int r = 0; r < n_restr; ++r) {
        int a = restr[2 * r], b = restr[2 * r + 1];
        if (a < 0 || a >= k || b < 0 || b >= k || a == b) return fail(GP_ERR_ARG, "bad restriction");
        res |= 1ull << res_bit(a, b);
    }
    if (!validate_set(p->info, res)) return fail(GP_ERR_PATTERN, "restriction set fails validate");
    GpPlan plan;
    std::string err;
    if (!compile_plan(p->info, sched.data(), res, &plan, err)) return fail(GP_ERR_PATTERN, err.c_str());
    std::unique_ptr<gp_schedules> s(new (std::nothrow) gp_schedules());
    if (!s) return fail(GP_ERR_NOMEM, "host allocation failed");
    s->k = k;
    s->info = clone_pattern(p->info);
    if (!s->info) return fail(GP_ERR_NOMEM, "host allocation failed");
    s->configs.push_back({0.0, sched, res});
    s->plans.push_back(plan);
    *out = s.release();
    return GP_OK;
}

gp_status gp_schedule_size(const gp_schedules* s, int32_t* count) {
    if (!s || !count) return fail(GP_ERR_ARG, "null argument");
    *count = (int32_t)s->plans.size();
    return GP_OK;
}

gp_status gp_schedule_get(const gp_schedules* s, int32_t idx, int32_t* order, int32_t* restr,
                          int32_t* n_restr, double* predicted_cost) {
    if (!s) return fail(GP_ERR_ARG, "null schedule");
    if (idx < 0 || idx >= (int32_t)s->configs.size()) return fail(GP_ERR_ARG, "plan index out of range");
    const Config& c = s->configs[idx];
    if (order) for (int i = 0; i < s->k; ++i) order[i] = c.sched[i];
    int r = 0;
    for (int a = 0; a < s->k; ++a)
        for (int b = 0; b < s->k; ++b)
            if (c.res >> res_bit(a, b) & 1) {
                if (restr) { restr[2 * r] = a; restr[2 * r + 1] = b; }
                ++r;
            }
    if (n_restr) *n_restr = r;
    if (predicted_cost) *predicted_cost = c.cost;
    return GP_OK;
}

gp_status gp_config_cost(const gp_pattern* p, const int32_t* order, const int32_t* restr,
                         int32_t n_restr, double n_vertices, double n_edges, double tri_cnt,
                         double* cost) {
    if (!p || !order || !cost || n_restr < 0 || (n_restr > 0 && !restr)) return fail(GP_ERR_ARG, "bad argument");
    if (!(n_vertices > 0) || !(n_edges > 0) || !(tri_cnt >= 0)) return fail(GP_ERR_ARG, "bad graph statistics");
    const int k = p->info.k;
    int8_t sched[GP_MAX_K];
    for (int i = 0; i < k; ++i) {
        if (order[i] < 0 || order[i] >= k) return fail(GP_ERR_ARG, "order entry outside the pattern");
        sched[i] = (int8_t)order[i];
    }
    ResMask res = 0;
    for (int r = 0; r < n_restr; ++r) {
        int a = restr[2 * r], b = restr[2 * r + 1];
        if (a < 0 || a >= k || b < 0 || b >= k || a == b) return fail(GP_ERR_ARG, "bad restriction");
        res |= 1ull << res_bit(a, b);
    }
    *cost = config_cost(p->info, sched, res, n_vertices, n_edges, tri_cnt);
    return GP_OK;
}

void gp_schedule_destroy(gp_schedules* s) { delete s; }

gp_status gp_count(gp_graph* g, const gp_schedules* s, int32_t idx, const gp_count_opts* opts,
                   void* stream, uint64_t* out) {
    if (!out) return fail(GP_ERR_ARG, "out is null");
    if (!opts_ok(opts)) return fail(GP_ERR_ARG, "gp_count_opts.struct_size mismatch");
    CountJob job;
    gp_status rc = make_job(g, s, idx, opts, &job);
    if (rc != GP_OK) return rc;
    const bool iep_part = job.plan.iep && (!whole_graph(job, g) || (opts && opts->budget_cycles > 0));
    if (iep_part && !(opts && opts->raw_total))
        return fail(GP_ERR_ARG, "an inclusion-exclusion count over part of the tasks needs opts->raw_total");
    rc = ensure_device(g);
    if (rc != GP_OK) return rc;
    if (job.plan.labeled) {                  // labelled plans: the listing kernel's counting pass
        if (opts && opts->budget_cycles > 0) return fail(GP_ERR_ARG, "labelled counts take no budget");
        int64_t w = 0, cut = 0, total = 0;
        rc = run_list(job, nullptr, -1, static_cast<cudaStream_t>(stream), &w, &cut, &total);
        if (rc != GP_OK) return rc;
        if (opts && opts->resume_cursor) *opts->resume_cursor = job.task_begin + job.ntasks;
        *out = (uint64_t)total;
        return GP_OK;
    }
    uint64_t res[2] = {0, 0};
    int64_t done = 0;
    float ms = 0.f;
    uint64_t bytes = 0;
    const bool want_ms = opts && opts->kernel_ms;
    int aborted = 0;
    uint64_t ops = 0, busy[2] = {0, 0};
    rc = run_count(&job, 1, launch_opts(opts), static_cast<cudaStream_t>(stream), res, &done,
                   want_ms ? &ms : nullptr, &bytes, &aborted, &ops, busy);
    if (rc != GP_OK) return rc;
    if (aborted) return fail(GP_ERR_TIMEOUT, "a work item outlived opts.task_cycles; the count was abandoned");
    uint64_t total = 0;
    if (job.plan.iep && (iep_part || done < job.nvirt)) {
        total = 0;                           // only the undivided raw total is meaningful
    } else {
        rc = finish_total(job.plan, res[0], res[1], &total);
        if (rc != GP_OK) return rc;
    }
    if (opts && opts->raw_total) { opts->raw_total[0] = res[0]; opts->raw_total[1] = res[1]; }
    if (want_ms) *opts->kernel_ms = ms;
    if (opts && opts->algo_bytes && (opts->flags & GP_COUNT_STATS)) *opts->algo_bytes = bytes;
    if (opts && opts->algo_ops && (opts->flags & GP_COUNT_STATS)) *opts->algo_ops = ops;
    if (opts && opts->busy_cycles) { opts->busy_cycles[0] = busy[0]; opts->busy_cycles[1] = busy[1]; }
    if (done < job.nvirt) {
        if (opts && opts->resume_cursor) *opts->resume_cursor = job.task_begin + done;
        *out = total;
        return GP_PARTIAL;
    }
    if (opts && opts->resume_cursor) *opts->resume_cursor = job.task_begin + job.ntasks;
    *out = total;
    return GP_OK;
}

gp_status gp_count_batch(gp_graph* const* graphs, const gp_schedules* const* scheds,
                         const int32_t* idx, int32_t njobs, const gp_count_opts* opts,
                         void* stream, uint64_t* out) {
    if (!graphs || !scheds || !out || njobs < 1) return fail(GP_ERR_ARG, "bad argument");
    if (!opts_ok(opts)) return fail(GP_ERR_ARG, "gp_count_opts.struct_size mismatch");
    if (opts && (opts->task_begin || opts->task_end)) return fail(GP_ERR_ARG, "task ranges are per gp_count only");
    std::vector<CountJob> jobs((size_t)njobs);
    int64_t off = 0;
    for (int32_t j = 0; j < njobs; ++j) {
        gp_count_opts r;
        std::memset(&r, 0, sizeof(r));
        r.struct_size = sizeof(r);
        r.split = opts ? opts->split : 0;
        gp_status rc = make_job(graphs[j], scheds[j], idx ? idx[j] : 0, &r, &jobs[j]);
        if (rc != GP_OK) return rc;
        if (jobs[j].plan.labeled) return fail(GP_ERR_ARG, "labelled plans are counted by gp_count");
        if (graphs[j]->device != graphs[0]->device) return fail(GP_ERR_ARG, "graphs on different devices");
        jobs[j].task_offset = off;
        off += jobs[j].nvirt;
    }
    gp_status rc = ensure_device(graphs[0]);
    if (rc != GP_OK) return rc;
    std::vector<uint64_t> res(2 * (size_t)njobs, 0);
    LaunchOpts lo = launch_opts(opts);
    lo.budget_cycles = 0;
    float ms = 0.f;
    uint64_t bytes = 0;
    const bool want_ms = opts && opts->kernel_ms;
    std::vector<int> aborted((size_t)njobs, 0);
    uint64_t ops = 0, busy[2] = {0, 0};
    // one persistent launch per kernel build: jobs that want different
    // register budgets (or the general inclusion-exclusion code) would
    // otherwise all run with the build the most demanding one needs
    std::vector<int> key((size_t)njobs);
    for (int32_t j = 0; j < njobs; ++j) key[j] = kernel_variant(jobs[j], lo);
    std::vector<int> keys(key);
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    int nsm = 0, dev = 0;
    GP_CUDA_TRY(cudaGetDevice(&dev));
    GP_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int user_chunk = lo.chunk;
    for (int kv : keys) {
        std::vector<CountJob> group;
        std::vector<int32_t> members;
        int64_t goff = 0;
        // tasks per work-queue grab: the smallest any of the launch's jobs
        // would take alone (a chunk sized by the whole batch's task count
        // hands expensive tasks out in blocks of up to 64 and leaves long
        // tails); about 64 grabs per warp of a 4-block-per-SM grid
        int64_t chunk = 64;
        for (int32_t j = 0; j < njobs; ++j) {
            if (key[j] != kv) continue;
            group.push_back(jobs[j]);
            group.back().task_offset = goff;
            goff += jobs[j].nvirt;
            members.push_back(j);
            chunk = std::min<int64_t>(chunk, jobs[j].nvirt / ((int64_t)nsm * 4 * 8 * 64));
        }
        lo.chunk = user_chunk > 0 ? user_chunk : (int)std::max<int64_t>(1, chunk);
        std::vector<uint64_t> gres(2 * group.size(), 0);
        std::vector<int> gab(group.size(), 0);
        int64_t done = 0;
        float gms = 0.f;
        uint64_t gbytes = 0, gops = 0, gbusy[2] = {0, 0};
        rc = run_count(group.data(), (int)group.size(), lo, static_cast<cudaStream_t>(stream), gres.data(), &done,
                       want_ms ? &gms : nullptr, &gbytes, gab.data(), &gops, gbusy);
        if (rc != GP_OK) return rc;
        for (size_t q = 0; q < members.size(); ++q) {
            res[2 * members[q]] = gres[2 * q];
            res[2 * members[q] + 1] = gres[2 * q + 1];
            aborted[members[q]] = gab[q];
        }
        ms += gms;
        bytes += gbytes;
        ops += gops;
        busy[0] += gbusy[0];
        busy[1] = std::max(busy[1], gbusy[1]);
    }
    for (int32_t j = 0; j < njobs; ++j)
        if (aborted[j]) return fail(GP_ERR_TIMEOUT, "a work item outlived opts.task_cycles; the batch was abandoned");
    if (want_ms) *opts->kernel_ms = ms;
    if (opts && opts->algo_bytes && (opts->flags & GP_COUNT_STATS)) *opts->algo_bytes = bytes;
    if (opts && opts->algo_ops && (opts->flags & GP_COUNT_STATS)) *opts->algo_ops = ops;
    if (opts && opts->busy_cycles) { opts->busy_cycles[0] = busy[0]; opts->busy_cycles[1] = busy[1]; }
    std::vector<uint64_t> tot((size_t)njobs);
    for (int32_t j = 0; j < njobs; ++j) {
        rc = finish_total(jobs[j].plan, res[2 * j], res[2 * j + 1], &tot[j]);
        // with raw_total, a count beyond 64 bits is reported there alone
        if (rc == GP_ERR_OVERFLOW && opts && opts->raw_total) { tot[j] = 0; continue; }
        if (rc != GP_OK) return rc;
    }
    for (int32_t j = 0; j < njobs; ++j) out[j] = tot[j];
    if (opts && opts->raw_total)
        for (size_t w = 0; w < 2 * (size_t)njobs; ++w) opts->raw_total[w] = res[w];
    return GP_OK;
}

gp_status gp_count_batch_ranges(gp_graph* const* graphs, const gp_schedules* const* scheds,
                                const int32_t* idx, const int64_t* task_begin,
                                const int64_t* task_end, int32_t njobs,
                                const gp_count_opts* opts, void* stream, uint64_t* out,
                                int64_t* next_task) {
    if (!graphs || !scheds || !out || !next_task || njobs < 1) return fail(GP_ERR_ARG, "bad argument");
    if (!opts_ok(opts)) return fail(GP_ERR_ARG, "gp_count_opts.struct_size mismatch");
    std::vector<CountJob> jobs((size_t)njobs);
    int64_t off = 0;
    for (int32_t j = 0; j < njobs; ++j) {
        gp_count_opts r;
        std::memset(&r, 0, sizeof(r));
        r.struct_size = sizeof(r);
        r.task_begin = task_begin ? task_begin[j] : 0;
        r.task_end = task_end ? task_end[j] : 0;
        r.split = (opts && opts->budget_cycles <= 0) ? opts->split : 0;   // whole ranges only
        gp_status rc = make_job(graphs[j], scheds[j], idx ? idx[j] : 0, &r, &jobs[j]);
        if (rc != GP_OK) return rc;
        if (jobs[j].plan.iep && !(opts && opts->raw_total))
            return fail(GP_ERR_ARG, "inclusion-exclusion jobs of a time slice need opts->raw_total");
        if (jobs[j].plan.labeled) return fail(GP_ERR_ARG, "labelled plans are counted by gp_count");
        if (graphs[j]->device != graphs[0]->device) return fail(GP_ERR_ARG, "graphs on different devices");
        jobs[j].task_offset = off;
        off += jobs[j].nvirt;
    }
    gp_status rc = ensure_device(graphs[0]);
    if (rc != GP_OK) return rc;
    std::vector<uint64_t> res(2 * (size_t)njobs, 0);
    int64_t done = 0;
    float ms = 0.f;
    const bool want_ms = opts && opts->kernel_ms;
    std::vector<int> aborted((size_t)njobs, 0);
    uint64_t busy[2] = {0, 0};
    rc = run_count(jobs.data(), njobs, launch_opts(opts), static_cast<cudaStream_t>(stream), res.data(),
                   &done, want_ms ? &ms : nullptr, nullptr, aborted.data(), nullptr, busy);
    if (rc != GP_OK) return rc;
    for (int32_t j = 0; j < njobs; ++j)
        if (!jobs[j].plan.iep && res[2 * j + 1] && !aborted[j])
            return fail(GP_ERR_OVERFLOW, "a count does not fit in 64 bits");
    bool all = true;
    for (int32_t j = 0; j < njobs; ++j) {
        int64_t p = std::min(std::max<int64_t>(done - jobs[j].task_offset, 0), jobs[j].ntasks);
        out[j] = (aborted[j] || jobs[j].plan.iep) ? 0 : res[2 * j];
        if (opts && opts->raw_total) {
            opts->raw_total[2 * j] = aborted[j] ? 0 : res[2 * j];
            opts->raw_total[2 * j + 1] = aborted[j] ? 0 : res[2 * j + 1];
        }
        next_task[j] = aborted[j] ? -1 : jobs[j].task_begin + p;
        all = all && !aborted[j] && p == jobs[j].ntasks;
    }
    if (want_ms) *opts->kernel_ms = ms;
    if (opts && opts->busy_cycles) { opts->busy_cycles[0] = busy[0]; opts->busy_cycles[1] = busy[1]; }
    return all ? GP_OK : GP_PARTIAL;
}

gp_status gp_schedule_set_iep(gp_schedules* s, int32_t enable, int32_t* n_iep) {
    if (!s || !s->info) return fail(GP_ERR_ARG, "null schedule");
    std::vector<GpPlan> plans;
    int32_t n = 0;
    for (const Config& c : s->configs) {
        GpPlan plan;
        std::string err;
        bool iep = enable && compile_plan_iep(*s->info, c.sched.data(), c.res, &plan, err);
        if (!iep && !compile_plan(*s->info, c.sched.data(), c.res, &plan, err))
            return fail(GP_ERR_INTERNAL, err.c_str());
        n += iep;
        plans.push_back(plan);
    }
    s->plans = plans;
    if (n_iep) *n_iep = n;
    return GP_OK;
}

gp_status gp_schedule_iep(const gp_schedules* s, int32_t idx, int32_t* kk, uint32_t* divisor) {
    if (!s) return fail(GP_ERR_ARG, "null schedule");
    if (idx < 0 || idx >= (int32_t)s->plans.size()) return fail(GP_ERR_ARG, "plan index out of range");
    const GpPlan& P = s->plans[idx];
    if (kk) *kk = P.iep;
    if (divisor) *divisor = P.iep ? P.iep_div : 1u;
    return GP_OK;
}

gp_status gp_list(gp_graph* g, const gp_schedules* s, int32_t idx, int64_t task_begin,
                  int64_t task_end, int32_t* out, int64_t capacity, void* stream,
                  int64_t* n_written, int64_t* next_task) {
    if (!n_written || !next_task || capacity < 0 || (capacity > 0 && !out)) return fail(GP_ERR_ARG, "bad argument");
    gp_count_opts r;
    std::memset(&r, 0, sizeof(r));
    r.struct_size = sizeof(r);
    r.task_begin = task_begin;
    r.task_end = task_end;
    CountJob job;
    gp_status rc = make_job(g, s, idx, &r, &job);
    if (rc != GP_OK) return rc;
    if (job.plan.iep) return fail(GP_ERR_ARG, "inclusion-exclusion plans count; they cannot list");
    rc = ensure_device(g);
    if (rc != GP_OK) return rc;
    int64_t written = 0, cut = 0;
    rc = run_list(job, out, capacity, static_cast<cudaStream_t>(stream), &written, &cut);
    if (rc != GP_OK) return rc;
    if (cut == 0 && job.ntasks > 0) return fail(GP_ERR_SCRATCH, "the first task's embeddings exceed the capacity");
    *n_written = written;
    *next_task = job.task_begin + cut;
    return cut == job.ntasks ? GP_OK : GP_PARTIAL;
}

gp_status gp_count_scratch_bytes(const gp_graph* g, const gp_schedules* s, int32_t idx,
                                 const gp_count_opts* opts, uint64_t* bytes) {
    if (!g || !s || !bytes) return fail(GP_ERR_ARG, "null argument");
    if (idx < 0 || idx >= (int32_t)s->plans.size()) return fail(GP_ERR_ARG, "plan index out of range");
    if (!opts_ok(opts)) return fail(GP_ERR_ARG, "gp_count_opts.struct_size mismatch");
    CountJob job;
    std::memset(&job, 0, sizeof(job));
    job.plan = s->plans[idx];
    job.slot_cap = g->max_deg > 0 ? g->max_deg : 1;
    return scratch_bytes(&job, 1, launch_opts(opts), bytes);
}

}  // extern "C"
