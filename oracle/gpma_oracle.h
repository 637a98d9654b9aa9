/*
 * gpma_oracle.h -- plain, single-threaded CPU oracle of GPMA+ (Sha, Li, He, Tan,
 * "Accelerating Dynamic Graph Analytics on GPUs").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The product path (the
 * CUDA library under paper_1709_05061_gb300/) neither links nor calls it, and
 * the two share no source, header, table or helper.
 *
 * Every routine follows the paper step by step in its own order:
 *   - thresholds: Sec. 4.1 "Background of PMA" and the Fig. 3 table;
 *   - batch update: Algorithm "GPMA+ Segment-Oriented Insertion" (Sec. 5.2),
 *     with lazy deletion (Sec. 6.1, "Maintaining Dynamic Graph");
 *   - CSR with guard entries: Sec. 4.2, Example 4 / Fig. 5;
 *   - BFS / connected components / PageRank: Sec. 4.2 (Algorithm "BFS") and
 *     Sec. 6.1 "Applications".
 * Readings of places where the paper is silent or ambiguous are listed with
 * each routine in gpma_oracle.c.
 */
#ifndef GPMA_ORACLE_H
#define GPMA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_EMPTY 0xFFFFFFFFFFFFFFFFull
#define OR_RAW_KEYS 1u /* keys are opaque integers < 2^63: no guards, no analytics */
#define OR_DUAL_DELETE 2u /* deletion as the dual of insertion (lower thresholds kept) */

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2

#define OR_MAX_LEVELS 48

typedef struct or_pma or_pma;

typedef struct {
  uint64_t n_inserted;      /* inserts that took effect */
  uint64_t n_deleted;       /* deletes that took effect */
  uint64_t n_ignored;       /* raw inputs that took no effect (dups, cancelled, present/absent) */
  uint32_t levels_climbed;  /* highest level at which a segment merged; h_old+1 on resize */
  uint32_t resized;         /* 1 if the array was grown, 2 if it was shrunk (dual mode) */
  uint64_t alg_bytes;       /* algorithmic bytes of the batch (definition in gpma_oracle.c) */
  uint64_t touched_leaves;  /* distinct leaves holding an insert or delete after cancellation */
  uint64_t covered_leaves;  /* leaves rewritten by a merge (union of merged segments) */
  uint64_t merges[OR_MAX_LEVELS]; /* segments merged per level, in the paper's level order */
  uint64_t delete_leaves;   /* distinct leaves holding a delete that took effect */
} or_stats;

/* Threshold rule: per-level maximum/minimum entry counts for a tree of height h. */
void or_thresholds(uint32_t L, uint32_t h, uint32_t tau0, uint32_t tauh, uint32_t rho0,
                   uint32_t rhoh, uint64_t *max_out, uint64_t *min_out);

or_pma *or_create(uint32_t n_vertices, uint32_t L, uint32_t tau0, uint32_t tauh,
                  uint32_t rho0, uint32_t rhoh, uint32_t flags);
void or_destroy(or_pma *p);

int or_update(or_pma *p, const uint64_t *ins, uint64_t n_ins, const uint64_t *del,
              uint64_t n_del, or_stats *st);

uint64_t or_capacity(const or_pma *p);
uint32_t or_height(const or_pma *p);
uint64_t or_num_valid(const or_pma *p);            /* valid slots, guards included */
void or_layout(const or_pma *p, uint64_t *out);     /* raw C slots */
int or_import_layout(or_pma *p, const uint64_t *slots, uint64_t capacity);
uint64_t or_export_sorted(const or_pma *p, uint64_t *out); /* edges only (no guards) */
/* CSR: rowptr[V+1], col[E] (column = dst); returns E. */
uint64_t or_export_csr(const or_pma *p, uint64_t *rowptr, uint32_t *col);
/* slot index of guard(u) for every vertex (non-raw mode). */
void or_row_end(const or_pma *p, uint32_t *row_end);

int or_bfs(const or_pma *p, uint32_t src, int32_t *depth);
int or_cc(const or_pma *p, uint32_t *label);
int or_pagerank(const or_pma *p, uint32_t iters, double damping, double *rank);
/* the same three analytics over a plain list of edges (src << 32 | dst, any order,
   every id below V): for graphs too large to load into the oracle's PMA */
int or_bfs_edges(uint32_t V, const uint64_t *keys, uint64_t n, uint32_t src, int32_t *depth);
int or_cc_edges(uint32_t V, const uint64_t *keys, uint64_t n, uint32_t *label);
int or_pagerank_edges(uint32_t V, const uint64_t *keys, uint64_t n, uint32_t iters, double damping,
                      double *rank);

/* 0 if every checked property holds, else a code naming the first violated one.
   Dual mode adds: 5 a leaf with a hole (a valid key after an EMPTY slot). */
int or_check_invariants(const or_pma *p);

#ifdef __cplusplus
}
#endif
#endif
