/* Oracle for the pattern-count path: plain, slow, obviously correct CPU code.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may call this library. The counting library
 * never links, loads or calls it, and shares no code with it.
 *
 * What it computes (GraphPi, Section II-A, problem definition): a pattern
 * P = (V_p, E_p) with k vertices matches a data graph G when an injective map
 * id : V_p -> V sends every pattern edge to a graph edge (non-induced
 * matching). Maps that differ by an automorphism of P name the same embedding
 * (Section II-B), so the embedding count is
 *
 *     count(P, G) = #{injective edge-preserving maps V_p -> V} / |Aut(P)|.
 *
 * The data graph is the undirected simple graph of the input pairs: self loops
 * dropped, both directions kept, duplicates removed, each neighbour list sorted
 * ascending (compressed sparse row, Section IV-E).
 *
 * All functions return 0 on success and a negative value on bad arguments or
 * allocation failure.
 */
#ifndef GRAPHPI_ORACLE_H
#define GRAPHPI_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Undirected simple CSR from m sampled pairs over [0, n). row_ptr has n + 1
 * entries; col must hold 2 * m entries. *nnz receives the directed entry
 * count (twice the undirected edge count). */
int oracle_build_csr(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                     int64_t* row_ptr, int32_t* col, int64_t* nnz);

/* |Aut(P)|: permutations p of the k pattern vertices with (p(a), p(b)) in E_p
 * for every (a, b) in E_p (Section IV-A), by trying all k! permutations.
 * adj is k * k row-major 0/1. */
int oracle_aut_count(int32_t k, const uint8_t* adj, uint64_t* out);

/* Number of injective edge-preserving maps of the pattern into the graph
 * whose image of pattern vertex 0 is one of the roots root_begin,
 * root_begin + root_stride, ... below root_end (stride 1 = every root). The 128-bit
 * total is returned in (*hi, *lo). nthreads worker threads split the roots. */
int oracle_count_maps(int32_t k, const uint8_t* adj,
                      int32_t n, const int64_t* row_ptr, const int32_t* col,
                      int32_t root_begin, int32_t root_end, int32_t root_stride,
                      int32_t nthreads, uint64_t* hi, uint64_t* lo);

/* Maps enumerated in the given matching order (Section II-B) that also obey
 * every restriction id(res[2i]) > id(res[2i+1]) (Section II-B), with the
 * image of the first searched vertex in [root_begin, root_end). Vertices are
 * pattern vertex numbers; order is a permutation of 0..k-1 whose prefixes
 * are connected. With a correct restriction set and all roots this equals
 * count(P, G) (Algorithm 1, validate). */
int oracle_count_restricted(int32_t k, const uint8_t* adj, const int32_t* order,
                            int32_t nres, const int32_t* res,
                            int32_t n, const int64_t* row_ptr, const int32_t* col,
                            int32_t root_begin, int32_t root_end,
                            int32_t nthreads, uint64_t* hi, uint64_t* lo);

/* oracle_count_restricted over the maps whose first two searched vertices
 * are one CSR entry (v0, v1) of [entry_begin, entry_end): v0 the entry's
 * row, v1 its column (the second searched pattern vertex is adjacent to the
 * first in every order with connected prefixes). The entries of a root's
 * row split its count into disjoint parts. */
int oracle_count_restricted_entries(int32_t k, const uint8_t* adj, const int32_t* order,
                                    int32_t nres, const int32_t* res,
                                    int32_t n, const int64_t* row_ptr, const int32_t* col,
                                    int64_t entry_begin, int64_t entry_end,
                                    int32_t nthreads, uint64_t* hi, uint64_t* lo);

/* The embeddings found by oracle_count_restricted with roots in
 * [root_begin, root_end), single-threaded in depth-first order: embedding i
 * is written as out[i * k + a] = image of pattern vertex a, for at most cap
 * embeddings. *n_out receives how many there are in total (also beyond
 * cap). Listing is the enumeration of Section II-A, one tuple per embedding. */
int oracle_list_restricted(int32_t k, const uint8_t* adj, const int32_t* order,
                           int32_t nres, const int32_t* res,
                           int32_t n, const int64_t* row_ptr, const int32_t* col,
                           int32_t root_begin, int32_t root_end,
                           int32_t* out, int64_t cap, int64_t* n_out);

/* Vertex-labelled patterns and graphs (Section II-A notes that the method
 * extends to labelled graphs): a map must also send every pattern vertex to
 * a graph vertex of the same label. plabels has k entries, glabels n.
 * oracle_aut_count_labeled counts the automorphisms that preserve labels;
 * oracle_count_labeled returns maps / labelled |Aut|; it returns -3 when the
 * maps are not a multiple of it (impossible for a correct enumeration) and
 * -4 when the count does not fit in 64 bits. (The unlabelled count(P, G) =
 * maps / |Aut(P)| is taken in Python from oracle_count_maps and
 * oracle_aut_count, where it may exceed 64 bits.) */
int oracle_aut_count_labeled(int32_t k, const uint8_t* adj, const int32_t* plabels, uint64_t* out);
int oracle_count_labeled(int32_t k, const uint8_t* adj, const int32_t* plabels,
                         int32_t n, const int64_t* row_ptr, const int32_t* col,
                         const int32_t* glabels, int32_t nthreads, uint64_t* out);

/* Unordered triangles {a, b, c} of the graph (the cost model's tri_cnt,
 * Section IV-C, counts each triangle once per ordered traversal; see the
 * planner). */
int oracle_triangles(int32_t n, const int64_t* row_ptr, const int32_t* col,
                     int32_t nthreads, uint64_t* out);

/* Directed patterns and graphs (the paper mentions directed patterns without
 * defining them; reading: an embedding is an injective map sending every
 * pattern arc a -> b, adj[a * k + b] = 1, to a graph arc, non-induced, and
 * the count is maps / |Aut(P)| over arc-preserving permutations).
 * oracle_build_dcsr: m arcs src[i] -> dst[i] (loops dropped, repeats merged)
 * into out-lists (out_ptr n + 1, out_col) and in-lists (in_ptr, in_col),
 * each sorted; *narcs receives the number of distinct arcs.
 * oracle_aut_count_directed: |Aut(P)| over arc-preserving permutations.
 * oracle_count_directed: maps whose first searched vertex (order[0]; order
 * NULL = breadth-first over arcs of either direction from vertex 0) has its
 * image in [root_begin, root_end), obeying the restrictions id(res[2i]) >
 * id(res[2i+1]); every prefix of the order must be weakly connected. The
 * 128-bit total is returned in (*hi, *lo). */
int oracle_build_dcsr(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                      int64_t* out_ptr, int32_t* out_col, int64_t* in_ptr, int32_t* in_col,
                      int64_t* narcs);
int oracle_aut_count_directed(int32_t k, const uint8_t* adj, uint64_t* out);
int oracle_count_directed(int32_t k, const uint8_t* adj, const int32_t* order,
                          int32_t nres, const int32_t* res,
                          int32_t n, const int64_t* out_ptr, const int32_t* out_col,
                          const int64_t* in_ptr, const int32_t* in_col,
                          int32_t root_begin, int32_t root_end, int32_t nthreads,
                          uint64_t* hi, uint64_t* lo);

#ifdef __cplusplus
}
#endif

#endif
