// plan.h -- the compiled form of one configuration (schedule + restriction
// set) that the counting kernel interprets. Shared by the host planner and
// the device code; plain POD so it can travel as a kernel parameter.
//
// Depth d is the position in the schedule (the paper's loop d+1). The
// candidate set of depth d is the intersection of the neighbour lists of the
// already-matched pattern neighbours of the depth-d vertex (Section IV-B),
// built incrementally as its operands become bound (the tmp_AB sets of the
// House example), clipped to the window that the restrictions impose
// (a restriction acts as a bound on a sorted candidate list, Section IV-B).
#pragma once
#include <stdint.h>

#define GP_MAX_K 7
#define GP_MAX_SLOTS 16
#define GP_MAX_BUILDS 8
#define GP_MAX_IEP 5     // most innermost loops that inclusion-exclusion replaces

// One incremental intersection: slot[dst] = base ∩ N(v_d), clipped to the
// window of the consuming depth that is already known at depth d.
struct GpBuild {
    int8_t dst;        // destination slot
    int8_t base_kind;  // 1: base = N(v_base) ; 2: base = slot[base]
    int8_t base;
    uint8_t lo_mask;   // depths j <= d with candidate > v_j
    uint8_t hi_mask;   // depths j <= d with candidate < v_j
    int8_t pad[3];
};

struct GpLevel {
    int8_t src_kind;   // 0: every vertex (depth 0), 1: N(v_src), 2: slot[src]
    int8_t src;
    uint8_t lo_mask;   // candidate > v_j for j in mask (restrictions, closed transitively)
    uint8_t hi_mask;   // candidate < v_j
    uint8_t excl_mask; // earlier depths whose vertex may lie in the set (injectivity)
    int8_t nbuild;     // builds executed after v_d is bound
    uint8_t op_mask;   // depths whose neighbourhoods are intersected for this set
    uint8_t bm_inc;    // set of depth d = set of depth d-1 ∩ N(v_{d-1}) (same
                       // operands plus d-1, window no wider): built incrementally
    GpBuild build[GP_MAX_BUILDS];
};

struct GpPlan {
    int32_t k;
    int32_t nslots;
    // 1 when the last depth's final operand is bound at depth k-2: the
    // intersection base ∩ N(v_{k-2}) is only counted, never stored. The base
    // is N(v_last_base) (last_base_kind 1) or slot[last_base] (kind 2).
    int32_t last_count_only;
    int16_t last_base_kind;
    int16_t last_base;
    int8_t order[GP_MAX_K];   // pattern vertex searched at depth d
    int8_t pad[1];
    // Inclusion-exclusion counting of the last iep (= kk >= 2, 0: off)
    // depths, whose vertices are pairwise non-adjacent (Section IV-D): once
    // the outer depths 0 .. k-kk-1 are bound, the number of ways to pick kk
    // distinct vertices from the inner candidate sets is added, expanded
    // over the set partitions of the kk sets (Algorithm 2 gives each term's
    // intersection). Restrictions acting at inner depths are dropped, and
    // the job's total is divided by iep_div.
    int32_t iep;
    uint32_t iep_div;
    // 1 when every vertex searched after depth 1 is restricted below v_1:
    // if v_1 is a core vertex the whole remaining search stays among core
    // vertices and runs on their adjacency bit matrix.
    int32_t core_dfs;
    // vertex-labelled pattern: the vertex matched at depth d must carry
    // label[d] (such plans run through the simple listing kernel)
    int32_t labeled;
    int32_t label[GP_MAX_K];
    GpLevel lvl[GP_MAX_K];
    // Two-loop inclusion-exclusion with one inner set never stored: that
    // set (depth k-3 + iep_fuse, 1 or 2) is iep_build's intersection of the
    // depth k-3 vertex's neighbours with its base, which no other level
    // reads; its size and its intersection with the other inner set are
    // counted in one pass (0: both inner sets are read from their lists).
    int32_t iep_fuse;
    GpBuild iep_build;
};
