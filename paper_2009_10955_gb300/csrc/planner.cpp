// planner.cpp -- configuration generation, performance model and plan
// compilation (GraphPi Sections IV-A, IV-B, IV-C).
#include "planner.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <unordered_set>

namespace gp {

namespace {

int factorial(int k) {
    int f = 1;
    for (int i = 2; i <= k; ++i) f *= i;
    return f;
}

// Acyclicity of a digraph on k <= 7 nodes given as out-neighbour bit masks:
// repeatedly peel nodes without incoming arcs.
bool acyclic(const uint8_t* out, int k) {
    uint8_t alive = (uint8_t)((1u << k) - 1);
    for (;;) {
        uint8_t has_in = 0;
        for (int v = 0; v < k; ++v)
            if (alive >> v & 1) has_in |= out[v] & alive;
        uint8_t sources = alive & (uint8_t)~has_in;
        if (!sources) return alive == 0;
        alive &= (uint8_t)~sources;
    }
}

// All k! relative orders (rank vectors) and, per ordered pair (a, b), the
// bit set of orders with rank[a] > rank[b]. Used for validate and for f_i.
struct OrderTable {
    int k = 0, n = 0, words = 0;
    std::vector<std::array<int8_t, GP_MAX_K>> perms;
    std::vector<uint64_t> gt;   // [(a * K + b) * words + w]
    const uint64_t* pair(int a, int b) const { return &gt[(size_t)(a * GP_MAX_K + b) * words]; }
};

const OrderTable& order_table(int k) {
    static std::mutex mu;
    static std::unique_ptr<OrderTable> tables[GP_MAX_K + 1];
    std::lock_guard<std::mutex> lock(mu);
    if (!tables[k]) {
        auto t = std::make_unique<OrderTable>();
        t->k = k;
        t->n = factorial(k);
        t->words = (t->n + 63) / 64;
        std::array<int8_t, GP_MAX_K> p{};
        for (int i = 0; i < k; ++i) p[i] = (int8_t)i;
        do { t->perms.push_back(p); } while (std::next_permutation(p.begin(), p.begin() + k));
        t->gt.assign((size_t)GP_MAX_K * GP_MAX_K * t->words, 0);
        for (int a = 0; a < k; ++a)
            for (int b = 0; b < k; ++b)
                for (int s = 0; s < t->n; ++s)
                    if (t->perms[s][a] > t->perms[s][b])
                        t->gt[(size_t)(a * GP_MAX_K + b) * t->words + s / 64] |= 1ull << (s % 64);
        tables[k] = std::move(t);
    }
    return *tables[k];
}

int popcount_words(const uint64_t* w, int n) {
    int c = 0;
    for (int i = 0; i < n; ++i) c += __builtin_popcountll(w[i]);
    return c;
}

}  // namespace

bool pattern_init(PatternInfo& p, const uint8_t* adj, int k, std::string& err) {
    if (k < 3 || k > GP_MAX_K) { err = "pattern size k must be in [3, 7]"; return false; }
    p.k = k;
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) {
            uint8_t x = adj[a * k + b];
            if (x > 1) { err = "pattern adjacency must be 0/1"; return false; }
            if (a == b && x) { err = "pattern has a self loop"; return false; }
            if (x != adj[b * k + a]) { err = "pattern adjacency is not symmetric"; return false; }
            p.adj[a][b] = x;
        }
    // connectivity (breadth-first from vertex 0)
    int seen = 1, stack[GP_MAX_K], top = 0;
    stack[top++] = 0;
    while (top) {
        int a = stack[--top];
        for (int b = 0; b < k; ++b)
            if (p.adj[a][b] && !(seen >> b & 1)) { seen |= 1 << b; stack[top++] = b; }
    }
    if (seen != (1 << k) - 1) { err = "pattern is not connected"; return false; }
    // automorphisms: permutations mapping every edge onto an edge
    Perm q{};
    for (int i = 0; i < k; ++i) q[i] = (int8_t)i;
    p.auts.clear();
    do {
        bool ok = true;
        for (int a = 0; a < k && ok; ++a)
            for (int b = 0; b < k && ok; ++b)
                if (p.adj[a][b] && !p.adj[q[a]][q[b]]) ok = false;
        if (ok) p.auts.push_back(q);
    } while (std::next_permutation(q.begin(), q.begin() + k));
    return true;
}

bool pattern_init_labeled(PatternInfo& p, const uint8_t* adj, const int32_t* labels, int k, std::string& err) {
    if (!pattern_init(p, adj, k, err)) return false;
    p.labeled = true;
    for (int i = 0; i < k; ++i) p.labels[i] = labels[i];
    std::vector<Perm> keep;
    for (const Perm& q : p.auts) {
        bool ok = true;
        for (int a = 0; a < k && ok; ++a) ok = p.labels[q[a]] == p.labels[a];
        if (ok) keep.push_back(q);
    }
    p.auts = keep;
    return true;
}

bool no_conflict(const Perm& perm, ResMask res, int k) {
    uint8_t out[GP_MAX_K] = {};
    for (ResMask m = res; m; m &= m - 1) {
        int bit = __builtin_ctzll(m);
        int a = bit / GP_MAX_K, b = bit % GP_MAX_K;
        out[a] |= (uint8_t)(1u << b);
        out[perm[a]] |= (uint8_t)(1u << perm[b]);
    }
    return acyclic(out, k);
}

bool validate_set(const PatternInfo& p, ResMask res) {
    const OrderTable& t = order_table(p.k);
    std::vector<uint64_t> alive((size_t)t.words, ~0ull);
    if (t.n % 64) alive.back() = (1ull << (t.n % 64)) - 1;
    for (ResMask m = res; m; m &= m - 1) {
        int bit = __builtin_ctzll(m);
        const uint64_t* g = t.pair(bit / GP_MAX_K, bit % GP_MAX_K);
        for (int w = 0; w < t.words; ++w) alive[w] &= g[w];
    }
    long ext = popcount_words(alive.data(), t.words);
    return ext * (long)p.auts.size() == (long)t.n;
}

// Algorithm 1. generate(pg, res_set) depends only on res_set: pg is exactly
// the automorphisms that no_conflict keeps under res_set, because a
// permutation that closes a cycle under a set also closes it under every
// superset. Each set is therefore explored once, and every validated leaf is
// added to one global result set.
const std::vector<ResMask>& restriction_sets(PatternInfo& p, int cap) {
    std::lock_guard<std::mutex> lock(p.mu);
    if (cap <= 0) cap = 1024;
    if (p.sets_done && p.sets_cap == cap) return p.sets;
    const int k = p.k;
    std::unordered_set<ResMask> visited, found;
    const size_t visit_cap = (size_t)1 << 21;
    std::vector<ResMask> stack{0};
    visited.insert(0);
    while (!stack.empty() && found.size() < (size_t)cap && visited.size() < visit_cap) {
        ResMask rs = stack.back();
        stack.pop_back();
        std::vector<const Perm*> pg;
        for (const Perm& q : p.auts)
            if (no_conflict(q, rs, k)) pg.push_back(&q);
        if (pg.size() > 1) {
            // pairs (a, b) with a < b are pushed last and so explored first
            for (const Perm* q : pg)
                for (int v = k - 1; v >= 0; --v) {
                    int w = (*q)[v];
                    if (w != v && (*q)[w] == v) {           // a 2-cycle (v, w)
                        ResMask ns = rs | (1ull << res_bit(v, w));
                        if (visited.insert(ns).second) stack.push_back(ns);
                    }
                }
        } else if (validate_set(p, rs)) {
            found.insert(rs);
        }
    }
    // Reversing every restriction of a valid set gives a valid set with the
    // same f_i under every schedule (Algorithm 1 adds both orientations of
    // each 2-cycle); when the search stopped at its cap, add the mirrors so
    // that the ranking can pick the orientation it prefers.
    if (found.size() >= (size_t)cap || visited.size() >= visit_cap) {
        std::vector<ResMask> mirrors;
        for (ResMask m : found) {
            ResMask r = 0;
            for (ResMask x = m; x; x &= x - 1) {
                int bit = __builtin_ctzll(x);
                r |= 1ull << res_bit(bit % GP_MAX_K, bit / GP_MAX_K);
            }
            mirrors.push_back(r);
        }
        for (ResMask r : mirrors) found.insert(r);
    }
    p.sets.assign(found.begin(), found.end());
    // deterministic order: by the sorted list of pairs, as (a, b) tuples
    auto key = [k](ResMask m) {
        std::vector<int> v;
        for (int a = 0; a < k; ++a)
            for (int b = 0; b < k; ++b)
                if (m >> res_bit(a, b) & 1) v.push_back(a * 16 + b);
        return v;
    };
    std::sort(p.sets.begin(), p.sets.end(), [&](ResMask x, ResMask y) { return key(x) < key(y); });
    p.sets_done = true;
    p.sets_cap = cap;
    return p.sets;
}

const std::vector<Perm>& efficient_schedules(PatternInfo& p, int* kprime) {
    std::lock_guard<std::mutex> lock(p.mu);
    if (!p.scheds_done) {
        const int k = p.k;
        std::vector<Perm> phase1;
        Perm s{};
        for (int i = 0; i < k; ++i) s[i] = (int8_t)i;
        do {
            bool ok = true;
            for (int i = 1; i < k && ok; ++i) {
                bool any = false;
                for (int j = 0; j < i; ++j) any |= p.adj[s[i]][s[j]] != 0;
                ok = any;
            }
            if (ok) phase1.push_back(s);
        } while (std::next_permutation(s.begin(), s.begin() + k));
        int mis = 0;
        for (int sub = 1; sub < (1 << k); ++sub) {
            bool indep = true;
            for (int a = 0; a < k && indep; ++a)
                for (int b = a + 1; b < k && indep; ++b)
                    if ((sub >> a & 1) && (sub >> b & 1) && p.adj[a][b]) indep = false;
            if (indep) mis = std::max(mis, __builtin_popcount(sub));
        }
        for (int kk = mis; kk >= 1; --kk) {
            p.scheds.clear();
            for (const Perm& q : phase1) {
                bool ok = true;
                for (int a = k - kk; a < k && ok; ++a)
                    for (int b = a + 1; b < k && ok; ++b)
                        if (p.adj[q[a]][q[b]]) ok = false;
                if (ok) p.scheds.push_back(q);
            }
            if (!p.scheds.empty()) { p.kprime = kk; break; }
        }
        p.scheds_done = true;
    }
    if (kprime) *kprime = p.kprime;
    return p.scheds;
}

double config_cost(const PatternInfo& p, const int8_t* sched, ResMask res,
                   double n_vertices, double n_edges, double tri_cnt) {
    const int k = p.k;
    const double V = n_vertices;
    const double p1 = 2.0 * n_edges / (V * V);
    const double p2 = tri_cnt * V / ((2.0 * n_edges) * (2.0 * n_edges));
    auto card = [&](int m) { return m == 0 ? V : V * p1 * std::pow(p2, (double)(m - 1)); };
    int ops[GP_MAX_K][GP_MAX_K], nops[GP_MAX_K];
    for (int i = 0; i < k; ++i) {
        nops[i] = 0;
        for (int j = 0; j < i; ++j)
            if (p.adj[sched[i]][sched[j]]) ops[i][nops[i]++] = j;
    }
    double l[GP_MAX_K] = {}, c[GP_MAX_K] = {}, f[GP_MAX_K] = {};
    for (int i = 0; i < k; ++i) l[i] = card(nops[i]);
    // c_i: distinct partial intersections computed in loop i
    for (int i = 0; i < k; ++i) {
        c[i] = 0.0;
        uint32_t built[GP_MAX_K * GP_MAX_K];
        int nbuilt = 0;
        for (int x = i + 1; x < k; ++x) {
            int at = -1;
            for (int q = 0; q < nops[x]; ++q) if (ops[x][q] == i) at = q;
            if (at < 1) continue;
            uint32_t prefix = 0;
            for (int q = 0; q <= at; ++q) prefix |= 1u << ops[x][q];
            bool dup = false;
            for (int b = 0; b < nbuilt; ++b) dup |= built[b] == prefix;
            if (dup) continue;
            built[nbuilt++] = prefix;
            c[i] += card(at) + card(1);
        }
    }
    // f_i: share of the still-alive relative orders removed in loop i
    const OrderTable& t = order_table(k);
    int pos[GP_MAX_K];
    for (int i = 0; i < k; ++i) pos[sched[i]] = i;
    std::vector<uint64_t> alive((size_t)t.words, ~0ull);
    if (t.n % 64) alive.back() = (1ull << (t.n % 64)) - 1;
    for (int i = 0; i < k; ++i) {
        int before = popcount_words(alive.data(), t.words);
        bool any = false;
        for (ResMask m = res; m; m &= m - 1) {
            int bit = __builtin_ctzll(m);
            int a = bit / GP_MAX_K, b = bit % GP_MAX_K;
            if (std::max(pos[a], pos[b]) != i) continue;
            any = true;
            const uint64_t* g = t.pair(a, b);
            for (int w = 0; w < t.words; ++w) alive[w] &= g[w];
        }
        int after = popcount_words(alive.data(), t.words);
        f[i] = (!any || before == 0) ? 0.0 : (double)(before - after) / (double)before;
    }
    double total = l[k - 1] * (1.0 - f[k - 1]);
    for (int i = k - 2; i >= 0; --i) total = l[i] * (1.0 - f[i]) * (c[i] + total);
    return total;
}

int upper_bound_restrictions(const int8_t* sched, ResMask res, int k) {
    int pos[GP_MAX_K];
    for (int i = 0; i < k; ++i) pos[sched[i]] = i;
    int n = 0;
    for (ResMask m = res; m; m &= m - 1) {
        int bit = __builtin_ctzll(m);
        int a = bit / GP_MAX_K, b = bit % GP_MAX_K;   // id(a) > id(b)
        n += pos[b] > pos[a];                         // later endpoint b is the smaller
    }
    return n;
}

bool compile_plan(const PatternInfo& p, const int8_t* sched, ResMask res, GpPlan* out,
                  std::string& err) {
    const int k = p.k;
    GpPlan plan;
    std::memset(&plan, 0, sizeof(plan));
    plan.k = k;
    int pos[GP_MAX_K];
    bool seen[GP_MAX_K] = {};
    for (int i = 0; i < k; ++i) {
        if (sched[i] < 0 || sched[i] >= k || seen[sched[i]]) { err = "schedule is not a permutation"; return false; }
        seen[sched[i]] = true;
        pos[sched[i]] = i;
        plan.order[i] = sched[i];
    }
    // transitive closure of the restriction order, in depth terms:
    // gt[x][j] = the restrictions force v_x > v_j
    bool gt[GP_MAX_K][GP_MAX_K] = {};
    for (ResMask m = res; m; m &= m - 1) {
        int bit = __builtin_ctzll(m);
        int a = bit / GP_MAX_K, b = bit % GP_MAX_K;
        if (a >= k || b >= k || a == b) { err = "restriction names a vertex outside the pattern"; return false; }
        gt[pos[a]][pos[b]] = true;
    }
    for (int m = 0; m < k; ++m)
        for (int x = 0; x < k; ++x)
            for (int y = 0; y < k; ++y)
                if (gt[x][m] && gt[m][y]) gt[x][y] = true;
    for (int x = 0; x < k; ++x)
        if (gt[x][x]) { err = "restriction set is cyclic"; return false; }

    struct SlotKey { uint8_t prefix, lo, hi; int8_t id; };
    std::vector<SlotKey> keys;
    int nslots = 0;
    auto find_slot = [&](uint8_t prefix, uint8_t lo, uint8_t hi) -> int {
        for (const SlotKey& s : keys)
            if (s.prefix == prefix && s.lo == lo && s.hi == hi) return s.id;
        return -1;
    };

    plan.lvl[0].src_kind = 0;
    for (int x = 1; x < k; ++x) {
        GpLevel& L = plan.lvl[x];
        int ops[GP_MAX_K], nops = 0;
        uint8_t lo = 0, hi = 0, opmask = 0;
        for (int j = 0; j < x; ++j) {
            if (p.adj[sched[x]][sched[j]]) { ops[nops++] = j; opmask |= (uint8_t)(1u << j); }
            if (gt[x][j]) lo |= (uint8_t)(1u << j);
            if (gt[j][x]) hi |= (uint8_t)(1u << j);
        }
        if (nops == 0) { err = "schedule prefix is not connected (phase 1)"; return false; }
        L.lo_mask = lo;
        L.hi_mask = hi;
        L.op_mask = opmask;
        L.excl_mask = (uint8_t)(((1u << x) - 1) & ~opmask & ~lo & ~hi);
        if (nops == 1) { L.src_kind = 1; L.src = (int8_t)ops[0]; continue; }
        int prev_slot = -1;
        for (int q = 1; q < nops; ++q) {
            int d = ops[q];
            uint8_t prefix = 0;
            for (int r = 0; r <= q; ++r) prefix |= (uint8_t)(1u << ops[r]);
            uint8_t below = (uint8_t)((1u << (d + 1)) - 1);
            uint8_t clo = lo & below, chi = hi & below;
            bool count_only = (x == k - 1 && q == nops - 1 && d == k - 2);
            if (count_only) {
                plan.last_count_only = 1;
                if (q == 1) { plan.last_base_kind = 1; plan.last_base = (int16_t)ops[0]; }
                else { plan.last_base_kind = 2; plan.last_base = (int16_t)prev_slot; }
                L.src_kind = 2;
                L.src = -1;
                break;
            }
            int id = find_slot(prefix, clo, chi);
            if (id < 0) {
                if (nslots >= GP_MAX_SLOTS) { err = "plan needs too many intermediate sets"; return false; }
                id = nslots++;
                keys.push_back({prefix, clo, chi, (int8_t)id});
                GpLevel& B = plan.lvl[d];
                if (B.nbuild >= GP_MAX_BUILDS) { err = "too many intersections in one loop"; return false; }
                GpBuild& b = B.build[B.nbuild++];
                b.dst = (int8_t)id;
                if (q == 1) { b.base_kind = 1; b.base = (int8_t)ops[0]; }
                else { b.base_kind = 2; b.base = (int8_t)prev_slot; }
                b.lo_mask = clo;
                b.hi_mask = chi;
            }
            prev_slot = id;
            if (q == nops - 1) { L.src_kind = 2; L.src = (int8_t)id; }
        }
    }
    plan.nslots = nslots;
    plan.labeled = p.labeled;
    for (int d = 0; d < k; ++d) plan.label[d] = p.labeled ? p.labels[sched[d]] : -1;
    for (int x = 3; x < k; ++x) {
        const GpLevel& A = plan.lvl[x - 1];
        const GpLevel& B = plan.lvl[x];
        plan.lvl[x].bm_inc = B.op_mask == (uint8_t)(A.op_mask | (1u << (x - 1))) &&
                             (B.lo_mask & A.lo_mask) == A.lo_mask && (B.hi_mask & A.hi_mask) == A.hi_mask;
    }
    plan.core_dfs = k >= 4 && !p.labeled;
    for (int x = 2; x < k; ++x)
        if (!gt[1][x]) plan.core_dfs = 0;      // some later vertex may exceed v_1
    *out = plan;
    return true;
}

bool iep_divisor(const PatternInfo& p, const int8_t* sched, ResMask res, int kk, ResMask* outer, uint32_t* div) {
    const int k = p.k;
    if (p.labeled || kk < 2 || kk > GP_MAX_IEP || k - kk < 2) return false;
    for (int a = k - kk; a < k; ++a)
        for (int b = a + 1; b < k; ++b)
            if (p.adj[sched[a]][sched[b]]) return false;
    int pos[GP_MAX_K];
    for (int i = 0; i < k; ++i) pos[sched[i]] = i;
    ResMask ro = 0;
    for (ResMask m = res; m; m &= m - 1) {
        const int bit = __builtin_ctzll(m);
        if (std::max(pos[bit / GP_MAX_K], pos[bit % GP_MAX_K]) < k - kk) ro |= 1ull << bit;
    }
    const OrderTable& t = order_table(k);
    long mult = -1;
    for (int o = 0; o < t.n; ++o) {             // rank pattern pi of the images
        const auto& pi = t.perms[o];
        long c = 0;
        for (const Perm& sg : p.auts) {         // maps f o sigma, sigma in Aut
            bool ok = true;
            for (ResMask m = ro; m && ok; m &= m - 1) {
                const int bit = __builtin_ctzll(m);
                ok = pi[sg[bit / GP_MAX_K]] > pi[sg[bit % GP_MAX_K]];
            }
            c += ok;
        }
        if (mult < 0) mult = c;
        else if (c != mult) return false;
    }
    if (mult <= 0) return false;
    *outer = ro;
    *div = (uint32_t)mult;
    return true;
}

namespace {

// Two-loop inclusion-exclusion: when an inner set is a slot built at the
// last outer depth and read by nothing but its inner level, drop that build
// and let the kernel count the set (and its intersection with the other
// inner set) in one pass instead of storing it.
void fuse_inner_set(GpPlan* P) {
    const int k = P->k, d = k - 3;
    if (d < 1) return;
    for (int which = 0; which < 2; ++which) {
        const int x = k - 2 + which;
        const GpLevel& L = P->lvl[x];
        if (L.src_kind != 2) continue;
        const int slot_id = L.src;
        if (P->lvl[k - 2 + (1 - which)].src_kind == 2 && P->lvl[k - 2 + (1 - which)].src == slot_id) continue;
        bool other_use = P->last_count_only && P->last_base_kind == 2 && P->last_base == slot_id;
        for (int y = 0; y < k; ++y) {
            if (y != x && P->lvl[y].src_kind == 2 && P->lvl[y].src == slot_id) other_use = true;
            for (int q = 0; q < P->lvl[y].nbuild; ++q)
                if (P->lvl[y].build[q].base_kind == 2 && P->lvl[y].build[q].base == slot_id) other_use = true;
        }
        if (other_use) continue;
        GpLevel& B = P->lvl[d];
        for (int q = 0; q < B.nbuild; ++q) {
            if (B.build[q].dst != slot_id) continue;
            P->iep_fuse = 1 + which;
            P->iep_build = B.build[q];
            for (int r = q + 1; r < B.nbuild; ++r) B.build[r - 1] = B.build[r];
            --B.nbuild;
            return;
        }
    }
}

}  // namespace

int iep_depth(const PatternInfo& p, const int8_t* sched) {
    const int k = p.k;
    int kk = 1;                                 // trailing vertices pairwise non-adjacent
    while (kk < k) {
        const int a = k - 1 - kk;
        bool free = true;
        for (int b = a + 1; b < k && free; ++b) free = !p.adj[sched[a]][sched[b]];
        if (!free) break;
        ++kk;
    }
    return std::min(kk, std::min(k - 2, GP_MAX_IEP));
}

bool compile_plan_iep(const PatternInfo& p, const int8_t* sched, ResMask res, GpPlan* out,
                      std::string& err) {
    // the largest kk whose multiplicity is the same for every relative order
    for (int kk = iep_depth(p, sched); kk >= 2; --kk) {
        ResMask ro = 0;
        uint32_t div = 0;
        if (!iep_divisor(p, sched, res, kk, &ro, &div)) continue;
        if (!compile_plan(p, sched, ro, out, err)) return false;
        const int k = p.k;
        out->iep = kk;
        out->iep_div = div;
        out->core_dfs = 0;
        // the inner vertices are never bound: only outer ones can be matched
        // vertices inside an inner candidate set
        const uint8_t outer_mask = (uint8_t)((1u << (k - kk)) - 1u);
        for (int x = k - kk; x < k; ++x) out->lvl[x].excl_mask &= outer_mask;
        if (kk == 2) fuse_inner_set(out);
        return true;
    }
    err = "inclusion-exclusion does not apply to this configuration";
    return false;
}

std::vector<Config> rank_configs(PatternInfo& p, double n_vertices, double n_edges,
                                 double tri_cnt, int top_k) {
    int kp = 0;
    const std::vector<Perm>& all_scheds = efficient_schedules(p, &kp);
    const std::vector<ResMask>& sets = restriction_sets(p, 0);
    // An automorphism pi maps configuration (sigma, S) to (pi o sigma, pi(S))
    // with the same cost and the same depth-indexed plan, and Algorithm 1's
    // output is closed under pi. Ranking one schedule per orbit under Aut
    // (its lexicographically smallest image) therefore loses nothing.
    std::vector<Perm> scheds;
    for (const Perm& s : all_scheds) {
        bool smallest = true;
        for (const Perm& a : p.auts) {
            Perm img = s;
            for (int i = 0; i < p.k; ++i) img[i] = a[s[i]];
            if (std::lexicographical_compare(img.begin(), img.begin() + p.k, s.begin(), s.begin() + p.k)) {
                smallest = false;
                break;
            }
        }
        if (smallest) scheds.push_back(s);
    }
    struct Row { double cost; int ub; size_t si, ri; };
    std::vector<Row> rows;
    rows.reserve(scheds.size() * sets.size());
    for (size_t si = 0; si < scheds.size(); ++si)
        for (size_t ri = 0; ri < sets.size(); ++ri) {
            double c = config_cost(p, scheds[si].data(), sets[ri], n_vertices, n_edges, tri_cnt);
            int ub = upper_bound_restrictions(scheds[si].data(), sets[ri], p.k);
            rows.push_back({c, ub, si, ri});
        }
    // cheapest first; among equal costs (mirror-image sets give identical
    // f_i) prefer restrictions that bound a sorted candidate list from
    // above, which a non-increasing-degree labelling turns into short lists.
    auto cmp = [](const Row& x, const Row& y) {
        double tol = 1e-12 * std::max(std::fabs(x.cost), std::fabs(y.cost));
        if (std::fabs(x.cost - y.cost) > tol) return x.cost < y.cost;
        if (x.ub != y.ub) return x.ub > y.ub;
        if (x.si != y.si) return x.si < y.si;
        return x.ri < y.ri;
    };
    size_t keep = std::min(rows.size(), (size_t)std::max(1, top_k));
    std::partial_sort(rows.begin(), rows.begin() + keep, rows.end(), cmp);
    std::vector<Config> out;
    for (size_t i = 0; i < keep; ++i)
        out.push_back({rows[i].cost, scheds[rows[i].si], sets[rows[i].ri]});
    return out;
}

}  // namespace gp
