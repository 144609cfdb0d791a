/*
 * CPU oracle for dynamic Leiden (ND / DS / DF) -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, sequential, obviously-correct restatement of the paper's
 * algorithms (Alg. "naive", "delta", "frontier", "leiden", "leidenlm",
 * "leidensr", "leidensp", "leidenre", "leidenag", "leidenmk", "update",
 * "leidentr"; Eq. 1 and Eq. 2), used by the tests, by smoke() and by the
 * benchmark's CPU-baseline leg.  The product path never links or calls it.
 *
 * Arithmetic is exact: integer edge weights, int64 degrees and community
 * totals, int128 delta-modularity numerators, one fp64 division at the end.
 * Two schedules:
 *   ORACLE_SEQ  -- Gauss-Seidel in ascending vertex order, in place (the
 *                  paper's loops run by one thread); the quality reference.
 *   ORACLE_SYNC -- snapshot (Jacobi) schedule whose result does not depend on
 *                  processing order; the CUDA path's deterministic mode must
 *                  reproduce it bit for bit.
 */
#ifndef LEIDEN_ORACLE_H
#define LEIDEN_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_SEQ = 0, ORACLE_SYNC = 1 };
enum { ORACLE_ND = 0, ORACLE_DS = 1, ORACLE_DF = 2 };
enum { ORACLE_OK = 0, ORACLE_ERR_ARG = 1, ORACLE_ERR_BATCH = 2, ORACLE_ERR_OOM = 3, ORACLE_ERR_STATE = 6 };

typedef struct {
  double tau;              /* iteration tolerance, 1e-2 */
  double tau_drop;         /* TOLERANCE_DECLINE_FACTOR, 10 */
  double tau_refine;       /* tau_re, 0.6 */
  int32_t max_iterations;  /* 20 */
  int32_t max_passes;      /* 10 */
  int32_t schedule;        /* ORACLE_SEQ or ORACLE_SYNC */
  int32_t classes;         /* SYNC: sub-sweeps per local-moving iteration, 4 */
  int32_t split_all;       /* ablation: split every community not refined (not only changed ones), 0 */
  int32_t converge_any;    /* ablation: leave the pass loop when l_i <= 1 OR nothing was refined
                              (the text's reading of the convergence test), 0 */
} oracle_params;

typedef struct oracle_state oracle_state;

/* Trace layout (int64 words): [0] passes run, [1] |dV| of the last call,
 * then per pass p (ORACLE_TRACE_PASS words each): n_level, l_i,
 * communities after refinement, refined_any, refine rounds, moves in LM
 * iteration 0..19. */
#define ORACLE_TRACE_PASS 25
#define ORACLE_TRACE_WORDS (2 + 10 * ORACLE_TRACE_PASS)

oracle_state *oracle_create(const oracle_params *p, int64_t n, const int64_t *off,
                            const int32_t *col, const int32_t *w /* NULL = unit */);
void oracle_destroy(oracle_state *s);
int oracle_static(oracle_state *s, int32_t *membership_out /* n or NULL */);
int oracle_update(oracle_state *s, const int32_t *del3, int64_t n_del, const int32_t *ins3,
                  int64_t n_ins, int mode, int32_t *membership_out);
int oracle_get_state(const oracle_state *s, int32_t *C, int64_t *K, int64_t *Sigma, int64_t *dSigma,
                     int64_t *m2);
int64_t oracle_graph_arcs(const oracle_state *s);
int oracle_get_graph(const oracle_state *s, int64_t *off, int32_t *col, int64_t *w);
int oracle_get_affected(const oracle_state *s, uint8_t *dV);
int oracle_get_trace(const oracle_state *s, int64_t *trace /* ORACLE_TRACE_WORDS */);

/* Eq. 1 on any weighted CSR: q = (2m*sum_c sigma_c - sum_c Sigma_c^2) / (2m)^2.
 * num_out (optional) receives the exact numerator as {low 64 bits, high 64 bits}. */
int oracle_modularity(int64_t n, const int64_t *off, const int32_t *col, const int64_t *w,
                      const int32_t *C, double *q_out, int64_t *num_out);

/* Eq. 2 scaled by 2m^2: the exact integer g with dQ = 2g/(2m)^2 for moving i
 * from its community C[i] to community c (self-loops of i excluded). */
int oracle_move_gain(int64_t n, const int64_t *off, const int32_t *col, const int64_t *w,
                     const int32_t *C, int64_t i, int32_t c, int64_t *gain_out /* {lo, hi} */);

/* Alg. "leidenag": super-vertex graph of the dense membership C (ids in
 * [0, ncomm)); rows sorted by neighbour.  Returns arcs written, or -1. */
int64_t oracle_aggregate(int64_t n, const int64_t *off, const int32_t *col, const int64_t *w,
                         const int32_t *C, int64_t ncomm, int64_t *off_out, int32_t *col_out,
                         int64_t *w_out);

/* Alg. "leidensp" (reading: min-vertex label of each connected component of
 * the communities whose flag split_c is set, edges restricted to the
 * community).  C is rewritten in place. */
int oracle_split(int64_t n, const int64_t *off, const int32_t *col, int32_t *C,
                 const uint8_t *split_c /* indexed by community id, length n */);

#ifdef __cplusplus
}
#endif
#endif
