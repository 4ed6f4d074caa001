// planner.h -- host-side configuration generation and performance model
// (GraphPi Sections IV-A to IV-C) and compilation of a configuration into
// the GpPlan that the counting kernel interprets.
#pragma once
#include <array>
#include <mutex>
#include <string>
#include <vector>

#include "plan.h"

namespace gp {

using Perm = std::array<int8_t, GP_MAX_K>;
// A restriction set as a bit mask: bit (a * GP_MAX_K + b) set means
// id(a) > id(b) for pattern vertices a, b.
using ResMask = uint64_t;

inline int res_bit(int a, int b) { return a * GP_MAX_K + b; }

struct PatternInfo {
    int k = 0;
    uint8_t adj[GP_MAX_K][GP_MAX_K] = {};
    bool labeled = false;
    int32_t labels[GP_MAX_K] = {};   // vertex labels when labeled
    std::vector<Perm> auts;          // automorphism group (Section IV-A)

    std::mutex mu;                   // guards the lazily computed members below
    bool sets_done = false;
    int sets_cap = 0;
    std::vector<ResMask> sets;       // Algorithm 1 output
    bool scheds_done = false;
    int kprime = 0;
    std::vector<Perm> scheds;        // efficient schedules (Section IV-B)
};

// Validates (3 <= k <= 7, symmetric 0/1, zero diagonal, connected) and
// enumerates the automorphisms. Returns false with a message on bad input.
bool pattern_init(PatternInfo& p, const uint8_t* adj, int k, std::string& err);
// Same for a vertex-labelled pattern: automorphisms must also preserve labels.
bool pattern_init_labeled(PatternInfo& p, const uint8_t* adj, const int32_t* labels, int k, std::string& err);

// Algorithm 1 restriction sets (cached on the pattern). cap <= 0: default.
const std::vector<ResMask>& restriction_sets(PatternInfo& p, int cap);

// Efficient schedules, 2-phase filter with phase 2 relaxed (cached).
const std::vector<Perm>& efficient_schedules(PatternInfo& p, int* kprime);

// no_conflict of Algorithm 1: true when perm survives the set.
bool no_conflict(const Perm& perm, ResMask res, int k);

// validate of Algorithm 1: #orderings of k labels obeying res == k!/|Aut|.
bool validate_set(const PatternInfo& p, ResMask res);

// Performance model cost_1 of one configuration.
double config_cost(const PatternInfo& p, const int8_t* sched, ResMask res,
                   double n_vertices, double n_edges, double tri_cnt);

// Number of restrictions whose later-searched endpoint must be SMALLER than
// the earlier one (an upper bound on a sorted candidate list).
int upper_bound_restrictions(const int8_t* sched, ResMask res, int k);

// Compile a configuration. Returns false (with a message) when the schedule
// has a disconnected prefix or the plan needs more slots than supported.
bool compile_plan(const PatternInfo& p, const int8_t* sched, ResMask res, GpPlan* out,
                  std::string& err);

// Inclusion-exclusion over the last kk depths (Section IV-D): applicable
// when the last kk searched vertices are pairwise non-adjacent, 2 <= kk <=
// GP_MAX_IEP and at least two vertices stay outside (the edge task binds
// them). The restrictions whose later endpoint is one of the kk inner
// vertices are dropped; every embedding is then found once per automorphism
// sigma whose relabelled map still obeys the remaining ("outer")
// restrictions. Dividing by that number is exact only if it is the same for
// all k! relative orders of the vertices; *div receives it and the call
// returns false when it varies.
bool iep_divisor(const PatternInfo& p, const int8_t* sched, ResMask res, int kk, ResMask* outer, uint32_t* div);

// Number of trailing vertices of the schedule that are pairwise
// non-adjacent, capped at min(k - 2, GP_MAX_IEP): the largest kk that
// inclusion-exclusion could replace.
int iep_depth(const PatternInfo& p, const int8_t* sched);

// compile_plan for the inclusion-exclusion form with the largest kk that has
// an exact divisor (false when none applies).
bool compile_plan_iep(const PatternInfo& p, const int8_t* sched, ResMask res, GpPlan* out,
                      std::string& err);

struct Config {
    double cost;
    Perm sched;
    ResMask res;
};

// Rank all configurations by predicted cost and keep the best top_k.
std::vector<Config> rank_configs(PatternInfo& p, double n_vertices, double n_edges,
                                 double tri_cnt, int top_k);

}  // namespace gp
