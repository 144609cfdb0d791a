/*
 * CPU oracle for dynamic Leiden -- TEST INFRASTRUCTURE ONLY (see the header).
 *
 * Follows the paper's algorithms step by step, sequentially, with exact
 * integer arithmetic.  Section and algorithm names are the paper's; where the
 * paper is silent or garbled the reading taken is stated beside the code.
 *
 * Notation (Preliminaries): K_i weighted degree, Sigma_c total weight of the arcs
 * leaving community c, K_{i->c} weight from i to the members of c other than
 * i, M2 = 2m = sum of all arc weights.  Delta-modularity (Eq. 2) is kept as
 * the integer g = M2 (K_{i->c} - K_{i->d}) - K_i (K_i + Sigma_c - Sigma_d),
 * which equals Eq. 2 multiplied by 2m^2 = M2^2/2.
 */
#include "leiden_oracle.h"

#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

/* ------------------------------------------------------------------ utils */

static void *xcalloc(size_t n, size_t sz) { return calloc(n ? n : 1, sz); }
static void *xmalloc(size_t n) { return malloc(n ? n : 1); }

/* int128 -> double in a fixed operation order (|x| = hi*2^64 + lo): the CUDA
 * path converts with the same two steps, so both give the same double. */
static double i128_to_double(i128 x) {
  int neg = x < 0;
  unsigned __int128 u = neg ? (unsigned __int128)(-(x + 1)) + 1 : (unsigned __int128)x;
  double hi = (double)(uint64_t)(u >> 64);
  double lo = (double)(uint64_t)u;
  double r = hi * 18446744073709551616.0 + lo;
  return neg ? -r : r;
}

/* Delta-modularity of a sum of integer gains g: dQ = 2g / M2^2 (Eq. 2). */
static double gains_to_dq(i128 g, int64_t m2) {
  if (g == 0 || m2 == 0) return 0.0;
  double den = (double)m2 * (double)m2;
  return i128_to_double(2 * g) / den;
}

/* Weighted CSR at any level of the dendrogram (int64 weights). */
typedef struct {
  int64_t n;
  int64_t *off;
  int32_t *col;
  int64_t *w;
} ograph;

static void graph_free(ograph *g) {
  free(g->off); free(g->col); free(g->w);
  memset(g, 0, sizeof(*g));
}

/* The paper's "collision-free" per-thread hashtable (Approach, "Implementation details"): a dense
 * value array over all keys plus the list of keys touched. */
typedef struct {
  int64_t *val;
  int32_t *keys;
  int64_t nkeys;
} dense_ht;

static int ht_init(dense_ht *h, int64_t n) {
  h->val = (int64_t *)xcalloc((size_t)n, sizeof(int64_t));
  h->keys = (int32_t *)xmalloc((size_t)n * sizeof(int32_t));
  h->nkeys = 0;
  return h->val && h->keys ? 0 : -1;
}
static void ht_free(dense_ht *h) { free(h->val); free(h->keys); }
/* A key is "present" once added, even if its weight sums to zero: mark with a
 * separate flag array would cost memory, so presence is tracked by a
 * sentinel bit in a parallel byte array. */
typedef struct {
  dense_ht h;
  uint8_t *present;
} scan_ht;
static int sht_init(scan_ht *s, int64_t n) {
  s->present = (uint8_t *)xcalloc((size_t)n, 1);
  return (ht_init(&s->h, n) == 0 && s->present) ? 0 : -1;
}
static void sht_free(scan_ht *s) { ht_free(&s->h); free(s->present); }
static void sht_add(scan_ht *s, int32_t k, int64_t v) {
  if (!s->present[k]) { s->present[k] = 1; s->h.keys[s->h.nkeys++] = k; }
  s->h.val[k] += v;
}
static void sht_clear(scan_ht *s) {
  for (int64_t t = 0; t < s->h.nkeys; t++) { s->h.val[s->h.keys[t]] = 0; s->present[s->h.keys[t]] = 0; }
  s->h.nkeys = 0;
}

/* ---------------------------------------------------------- Eq. 1 (Q) */

static i128 modularity_numerator(const ograph *g, const int32_t *C, int64_t *m2_out) {
  /* sigma_c: intra-community arc weight; Sigma_c: weight of arcs leaving c */
  int64_t n = g->n;
  int64_t *Sig = (int64_t *)xcalloc((size_t)n, sizeof(int64_t));
  int64_t sigma = 0, m2 = 0;
  for (int64_t i = 0; i < n; i++) {
    for (int64_t a = g->off[i]; a < g->off[i + 1]; a++) {
      int64_t j = g->col[a];
      m2 += g->w[a];
      Sig[C[i]] += g->w[a];
      if (C[i] == C[j]) sigma += g->w[a];
    }
  }
  i128 sq = 0;
  for (int64_t c = 0; c < n; c++) sq += (i128)Sig[c] * Sig[c];
  free(Sig);
  *m2_out = m2;
  /* Q = sum_c sigma_c/2m - (Sigma_c/2m)^2 = (M2*sigma - sum Sigma_c^2) / M2^2 */
  return (i128)m2 * sigma - sq;
}

static double numerator_to_q(i128 num, int64_t m2) {
  if (m2 == 0) return 0.0;
  return i128_to_double(num) / ((double)m2 * (double)m2);
}

int oracle_modularity(int64_t n, const int64_t *off, const int32_t *col, const int64_t *w,
                      const int32_t *C, double *q_out, int64_t *num_out) {
  if (n < 0 || !off || !C) return ORACLE_ERR_ARG;
  for (int64_t i = 0; i < n; i++)
    if (C[i] < 0 || C[i] >= n) return ORACLE_ERR_ARG;
  ograph g = {n, (int64_t *)off, (int32_t *)col, (int64_t *)w};
  int64_t m2;
  i128 num = modularity_numerator(&g, C, &m2);
  if (q_out) *q_out = numerator_to_q(num, m2);
  if (num_out) {
    num_out[0] = (int64_t)(uint64_t)(unsigned __int128)num;
    num_out[1] = (int64_t)(num >> 64);
  }
  return ORACLE_OK;
}

/* ----------------------------------------------------- Eq. 2 (dQ) */

static inline i128 gain_full(int64_t m2, int64_t Kic, int64_t Kid, int64_t Ki, int64_t Sc, int64_t Sd) {
  return (i128)m2 * (Kic - Kid) - (i128)Ki * ((i128)Ki + Sc - Sd);
}
/* The part of g that depends on the target c (the rest is fixed per vertex). */
static inline i128 gain_rel(int64_t m2, int64_t Kic, int64_t Ki, int64_t Sc) {
  return (i128)m2 * Kic - (i128)Ki * Sc;
}

int oracle_move_gain(int64_t n, const int64_t *off, const int32_t *col, const int64_t *w,
                     const int32_t *C, int64_t i, int32_t c, int64_t *gain_out) {
  if (i < 0 || i >= n || c < 0 || c >= n) return ORACLE_ERR_ARG;
  int64_t m2 = 0;
  int64_t *Sig = (int64_t *)xcalloc((size_t)n, sizeof(int64_t));
  for (int64_t v = 0; v < n; v++)
    for (int64_t a = off[v]; a < off[v + 1]; a++) { m2 += w[a]; Sig[C[v]] += w[a]; }
  int64_t Ki = 0, Kic = 0, Kid = 0;
  int32_t d = C[i];
  for (int64_t a = off[i]; a < off[i + 1]; a++) {
    Ki += w[a];
    if (col[a] == i) continue; /* K_{i->c} excludes i itself */
    if (C[col[a]] == c) Kic += w[a];
    if (C[col[a]] == d) Kid += w[a];
  }
  i128 g = (c == d) ? 0 : gain_full(m2, Kic, Kid, Ki, Sig[c], Sig[d]);
  free(Sig);
  gain_out[0] = (int64_t)(uint64_t)(unsigned __int128)g;
  gain_out[1] = (int64_t)(g >> 64);
  return ORACLE_OK;
}

/* --------------------------------------------------------------- state */

struct oracle_state {
  oracle_params p;
  ograph g;         /* G^t */
  int64_t m2;       /* 2m of G^t */
  int32_t *C;       /* C^t */
  int64_t *K;       /* K^t */
  int64_t *S;       /* Sigma^t */
  int64_t *dS;      /* Delta Sigma^t */
  uint8_t *dV;      /* affected flags of the last call */
  int has_static;
  int64_t trace[ORACLE_TRACE_WORDS];
};

/* The per-call context handed to leiden(): the lambdas of Alg. naive/delta/
 * frontier become two flag arrays. */
typedef struct {
  int dynamic;              /* ND/DS/DF (1) or static (0) */
  const uint8_t *affected;  /* isAffected(i) */
  const uint8_t *in_range;  /* inAffectedRange(i); NULL = always 1 */
} leiden_ctx;

/* ------------------------------------------- Alg. leidenlm (local moving) */

/* Best community for vertex i among those linked to it (H holds K_{i->c}).
 * Reading: candidates are the neighbour communities other than d, the best
 * is the largest g with ties to the lowest community id; i moves only if
 * that g > 0 (staying has gain 0). */
static int32_t best_community(const scan_ht *H, int32_t d, int64_t m2, int64_t Ki, const int64_t *S,
                              i128 *rel_out) {
  int32_t best = -1;
  i128 bestv = 0;
  for (int64_t t = 0; t < H->h.nkeys; t++) {
    int32_t c = H->h.keys[t];
    if (c == d) continue;
    i128 v = gain_rel(m2, H->h.val[c], Ki, S[c]);
    if (best < 0 || v > bestv || (v == bestv && c < best)) { best = c; bestv = v; }
  }
  *rel_out = bestv;
  return best;
}

static void scan_communities(scan_ht *H, const ograph *g, const int32_t *C, int64_t i) {
  for (int64_t a = g->off[i]; a < g->off[i + 1]; a++) {
    int64_t j = g->col[a];
    if (j == i) continue; /* scanCommunities(self = false) */
    sht_add(H, C[j], g->w[a]);
  }
}

/* Mark the neighbours of i (other than i) unprocessed. */
static void mark_neighbours(const ograph *g, int64_t i, uint8_t *unproc) {
  for (int64_t a = g->off[i]; a < g->off[i + 1]; a++)
    if (g->col[a] != i) unproc[g->col[a]] = 1;
}

/* SEQ: the loop of Alg. leidenlm run by one thread in ascending order. */
static int leiden_move_seq(const ograph *g, int32_t *C, const int64_t *K, int64_t *S, uint8_t *dS,
                           uint8_t *unproc, const uint8_t *in_range, int dynamic, double tau,
                           int64_t m2, const oracle_params *p, scan_ht *H, int64_t *moves_trace) {
  int li;
  for (li = 0; li < p->max_iterations; li++) {
    i128 dq = 0;
    int64_t moves = 0;
    for (int64_t i = 0; i < g->n; i++) {
      if (!unproc[i]) continue;
      unproc[i] = 0; /* prune */
      if (in_range && !in_range[i]) continue;
      scan_communities(H, g, C, i);
      int32_t d = C[i];
      i128 rel;
      int32_t cs = best_community(H, d, m2, K[i], S, &rel);
      i128 gbest = 0;
      if (cs >= 0) gbest = gain_full(m2, H->h.val[cs], H->h.val[d], K[i], S[cs], S[d]);
      sht_clear(H);
      if (cs < 0 || gbest <= 0) continue; /* c* = C'[i] */
      S[d] -= K[i];
      S[cs] += K[i];
      C[i] = cs;
      dq += gbest;
      moves++;
      mark_neighbours(g, i, unproc);
      if (dynamic) dS[d] = 1;
    }
    if (li < 20 && moves_trace) moves_trace[li] = moves;
    if (gains_to_dq(dq, m2) <= tau) { li++; break; }
  }
  return li; /* reading: number of iterations executed */
}

/* SplitMix64 output function (Steele, Lea, Flood 2014) on x: a fixed hash
 * that spreads vertex ids over the SYNC schedule's classes. */
static inline uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* SYNC: an iteration is `classes` sub-sweeps (vertex i belongs to class
 * splitmix64(i) mod classes).  In sub-sweep k every unprocessed vertex of
 * class k decides from the state at the start of the sub-sweep, then all of
 * its moves apply together; neighbours marked unprocessed by them are taken
 * by a later class of the same iteration, or by the next iteration.  The
 * outcome does not depend on the order inside a sub-sweep.  One extra rule
 * keeps two singletons from swapping (Lu, Halappanavar, Kalyanaraman 2015):
 * a vertex alone in its community does not move into another single-vertex
 * community with a larger id. */
static int leiden_move_sync(const ograph *g, int32_t *C, const int64_t *K, int64_t *S, uint8_t *dS,
                            uint8_t *unproc, const uint8_t *in_range, int dynamic, double tau,
                            int64_t m2, const oracle_params *p, scan_ht *H, int64_t *moves_trace) {
  int64_t n = g->n;
  int classes = p->classes > 0 ? p->classes : 1;
  int32_t *size = (int32_t *)xcalloc((size_t)n, sizeof(int32_t));
  int32_t *target = (int32_t *)xmalloc((size_t)n * sizeof(int32_t));
  int64_t *list = (int64_t *)xmalloc((size_t)n * sizeof(int64_t));
  for (int64_t i = 0; i < n; i++) size[C[i]]++;
  int li;
  for (li = 0; li < p->max_iterations; li++) {
    i128 dq = 0;
    int64_t moves = 0;
    for (int k = 0; k < classes; k++) {
      int64_t cnt = 0;
      for (int64_t i = 0; i < n; i++)
        if (unproc[i] && (int64_t)(splitmix64((uint64_t)i) % (uint64_t)classes) == k) {
          unproc[i] = 0; /* prune */
          list[cnt++] = i;
        }
      for (int64_t t = 0; t < cnt; t++) {
        int64_t i = list[t];
        target[i] = -1;
        if (in_range && !in_range[i]) continue;
        scan_communities(H, g, C, i);
        int32_t d = C[i];
        i128 rel;
        int32_t cs = best_community(H, d, m2, K[i], S, &rel);
        i128 gbest = 0;
        if (cs >= 0) gbest = gain_full(m2, H->h.val[cs], H->h.val[d], K[i], S[cs], S[d]);
        sht_clear(H);
        if (cs < 0 || gbest <= 0) continue;
        if (size[d] == 1 && size[cs] == 1 && cs > d) continue;
        target[i] = cs;
        dq += gbest;
      }
      for (int64_t t = 0; t < cnt; t++) {
        int64_t i = list[t];
        int32_t cs = target[i];
        if (cs < 0) continue;
        int32_t d = C[i];
        S[d] -= K[i];
        S[cs] += K[i];
        size[d]--;
        size[cs]++;
        C[i] = cs;
        moves++;
        mark_neighbours(g, i, unproc);
        if (dynamic) dS[d] = 1;
      }
    }
    if (li < 20 && moves_trace) moves_trace[li] = moves;
    if (gains_to_dq(dq, m2) <= tau) { li++; break; }
  }
  free(size); free(target); free(list);
  return li;
}

/* ------------------------------------ Alg. leidensr (subset renumbering) */

/* Each community takes the id of one of its vertices -- reading: the
 * smallest -- and Sigma, dS, dR are re-keyed to it (others cleared). */
static void subset_renumber(int64_t n, int32_t *C, int64_t *S, uint8_t *dSp, uint8_t *dR) {
  int32_t *rep = (int32_t *)xmalloc((size_t)n * sizeof(int32_t));
  for (int64_t c = 0; c < n; c++) rep[c] = -1;
  for (int64_t i = 0; i < n; i++)
    if (rep[C[i]] < 0) rep[C[i]] = (int32_t)i; /* ascending scan: first = min */
  int64_t *S2 = (int64_t *)xcalloc((size_t)n, sizeof(int64_t));
  uint8_t *dS2 = (uint8_t *)xcalloc((size_t)n, 1);
  uint8_t *dR2 = (uint8_t *)xcalloc((size_t)n, 1);
  for (int64_t c = 0; c < n; c++) {
    if (rep[c] < 0) continue;
    S2[rep[c]] = S[c];
    dS2[rep[c]] = dSp[c];
    dR2[rep[c]] = dR[c];
  }
  for (int64_t i = 0; i < n; i++) C[i] = rep[C[i]];
  memcpy(S, S2, (size_t)n * sizeof(int64_t));
  memcpy(dSp, dS2, (size_t)n);
  memcpy(dR, dR2, (size_t)n);
  free(rep); free(S2); free(dS2); free(dR2);
}

/* ---------------------------------------------- Alg. leidensp (splitting) */

/* Communities c with split_c[c] are cut into their connected components
 * (edges with both ends in c).  Reading of the BFS labelling: a component
 * takes the id of its smallest vertex, which is what a sequential BFS from
 * the lowest unvisited vertex gives. */
static void split_components(const ograph *g, int32_t *C, const uint8_t *split_c) {
  int64_t n = g->n;
  uint8_t *vis = (uint8_t *)xcalloc((size_t)n, 1);
  int64_t *queue = (int64_t *)xmalloc((size_t)n * sizeof(int64_t));
  int32_t *Cold = (int32_t *)xmalloc((size_t)n * sizeof(int32_t));
  memcpy(Cold, C, (size_t)n * sizeof(int32_t));
  for (int64_t r = 0; r < n; r++) {
    if (vis[r] || !split_c[Cold[r]]) continue;
    int32_t c = Cold[r];
    int64_t qh = 0, qt = 0;
    queue[qt++] = r;
    vis[r] = 1;
    while (qh < qt) {
      int64_t u = queue[qh++];
      C[u] = (int32_t)r;
      for (int64_t a = g->off[u]; a < g->off[u + 1]; a++) {
        int64_t v = g->col[a];
        if (vis[v] || Cold[v] != c) continue;
        vis[v] = 1;
        queue[qt++] = v;
      }
    }
  }
  free(vis); free(queue); free(Cold);
}

int oracle_split(int64_t n, const int64_t *off, const int32_t *col, int32_t *C, const uint8_t *split_c) {
  ograph g = {n, (int64_t *)off, (int32_t *)col, NULL};
  for (int64_t i = 0; i < n; i++)
    if (C[i] < 0 || C[i] >= n) return ORACLE_ERR_ARG;
  split_components(&g, C, split_c);
  return ORACLE_OK;
}

/* -------------------------------------------- Alg. leidenre (refinement) */

static void scan_bounded(scan_ht *H, const ograph *g, const int32_t *CB, const int32_t *C, int64_t i) {
  for (int64_t a = g->off[i]; a < g->off[i + 1]; a++) {
    int64_t j = g->col[a];
    if (j == i) continue;
    if (CB[i] != CB[j]) continue;
    sht_add(H, C[j], g->w[a]);
  }
}

/* SEQ: the two loops of Alg. leidenre, one thread, ascending order. */
static int refine_seq(const ograph *g, const int32_t *CB, int32_t *C, const int64_t *K, int64_t *S,
                      const uint8_t *dR, int64_t m2, scan_ht *H) {
  int64_t n = g->n;
  for (int64_t i = 0; i < n; i++)
    if (dR[CB[i]]) { C[i] = (int32_t)i; S[i] = K[i]; }
  for (int64_t i = 0; i < n; i++) {
    int32_t c = C[i];
    if (!dR[CB[i]] || S[c] != K[i]) continue; /* only isolated vertices move */
    scan_bounded(H, g, CB, C, i);
    i128 rel;
    int32_t cs = best_community(H, c, m2, K[i], S, &rel);
    i128 gbest = 0;
    if (cs >= 0) gbest = gain_full(m2, H->h.val[cs], H->h.val[c], K[i], S[cs], S[c]);
    sht_clear(H);
    if (cs < 0 || gbest <= 0) continue;
    if (C[cs] != cs) continue; /* the representative of c* has moved away */
    /* atomicCAS(Sigma[c], K[i], 0) succeeds: i is still alone */
    S[c] = 0;
    S[cs] += K[i];
    C[i] = cs;
  }
  return 1;
}

/* SYNC: rounds.  In a round every isolated vertex in a refined bound picks
 * its best c* from the state at the start of the round (positive gain, ties
 * to the lowest id, representative of c* still in c*) or stays.  A vertex v
 * "holds" when it stays, or when it and p[v] chose each other and v has the
 * smaller id.  i -> c* is applied iff i does not hold and c* holds.  A moving
 * vertex therefore never receives a vertex in the same round, every
 * sub-community stays a star around a fixed vertex, and the result does not
 * depend on order.  Rounds repeat until none applies, at most
 * MAX_ITERATIONS times. */
static int refine_sync(const ograph *g, const int32_t *CB, int32_t *C, const int64_t *K, int64_t *S,
                       const uint8_t *dR, int64_t m2, int max_rounds, scan_ht *H) {
  int64_t n = g->n;
  int32_t *prop = (int32_t *)xmalloc((size_t)n * sizeof(int32_t));
  uint8_t *holds = (uint8_t *)xmalloc((size_t)n);
  for (int64_t i = 0; i < n; i++)
    if (dR[CB[i]]) { C[i] = (int32_t)i; S[i] = K[i]; }
  int rounds = 0;
  for (int r = 0; r < max_rounds; r++) {
    rounds++;
    for (int64_t i = 0; i < n; i++) {
      prop[i] = -1;
      int32_t c = C[i];
      if (!dR[CB[i]] || S[c] != K[i]) continue;
      scan_bounded(H, g, CB, C, i);
      i128 rel;
      int32_t cs = best_community(H, c, m2, K[i], S, &rel);
      i128 gbest = 0;
      if (cs >= 0) gbest = gain_full(m2, H->h.val[cs], H->h.val[c], K[i], S[cs], S[c]);
      sht_clear(H);
      if (cs < 0 || gbest <= 0) continue;
      if (C[cs] != cs) continue;
      prop[i] = cs;
    }
    for (int64_t v = 0; v < n; v++) {
      int32_t t = prop[v];
      holds[v] = (t < 0) || (prop[t] == v && v < t);
    }
    int64_t applied = 0;
    for (int64_t i = 0; i < n; i++) {
      int32_t cs = prop[i];
      if (cs < 0 || holds[i] || !holds[cs]) continue;
      int32_t c = C[i];
      S[c] -= K[i];
      S[cs] += K[i];
      C[i] = cs;
      applied++;
    }
    if (applied == 0) break;
  }
  free(prop); free(holds);
  return rounds;
}

/* ------------------------------------------------ renumber and aggregate */

/* Dense renumbering (Alg. leiden, "Renumber communities"): reading -- ids
 * are ranked in ascending order of the old id. */
static int64_t renumber_dense(int64_t n, int32_t *C) {
  int32_t *rank = (int32_t *)xmalloc((size_t)n * sizeof(int32_t));
  for (int64_t c = 0; c < n; c++) rank[c] = -1;
  for (int64_t i = 0; i < n; i++) rank[C[i]] = 0;
  int64_t k = 0;
  for (int64_t c = 0; c < n; c++)
    if (rank[c] == 0) rank[c] = (int32_t)k++;
  for (int64_t i = 0; i < n; i++) C[i] = rank[C[i]];
  free(rank);
  return k;
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return x < y ? -1 : x > y;
}

/* Alg. leidenag: community c of G' becomes super-vertex c; each arc (i, j, w)
 * of G' adds w to the super-arc (C[i], C[j]), self-loops included.  Rows are
 * emitted sorted by neighbour. */
static int aggregate_graph(const ograph *g, const int32_t *C, int64_t ncomm, ograph *out) {
  int64_t n = g->n;
  /* community vertices CSR (countCommunityVertices + exclusive scan) */
  int64_t *coff = (int64_t *)xcalloc((size_t)(ncomm + 1), sizeof(int64_t));
  int64_t *cv = (int64_t *)xmalloc((size_t)n * sizeof(int64_t));
  int64_t *cur = (int64_t *)xmalloc((size_t)(ncomm + 1) * sizeof(int64_t));
  for (int64_t i = 0; i < n; i++) coff[C[i] + 1]++;
  for (int64_t c = 0; c < ncomm; c++) coff[c + 1] += coff[c];
  memcpy(cur, coff, (size_t)(ncomm + 1) * sizeof(int64_t));
  for (int64_t i = 0; i < n; i++) cv[cur[C[i]]++] = i;
  /* upper bound of super-vertex degrees (communityTotalDegree + scan) */
  int64_t *yoff = (int64_t *)xcalloc((size_t)(ncomm + 1), sizeof(int64_t));
  for (int64_t i = 0; i < n; i++) yoff[C[i] + 1] += g->off[i + 1] - g->off[i];
  for (int64_t c = 0; c < ncomm; c++) yoff[c + 1] += yoff[c];
  int32_t *ycol = (int32_t *)xmalloc((size_t)yoff[ncomm] * sizeof(int32_t));
  int64_t *yw = (int64_t *)xmalloc((size_t)yoff[ncomm] * sizeof(int64_t));
  int64_t *ylen = (int64_t *)xcalloc((size_t)(ncomm + 1), sizeof(int64_t));
  scan_ht H;
  if (sht_init(&H, ncomm) != 0) return -1;
  for (int64_t c = 0; c < ncomm; c++) {
    for (int64_t t = coff[c]; t < coff[c + 1]; t++) {
      int64_t i = cv[t];
      for (int64_t a = g->off[i]; a < g->off[i + 1]; a++) sht_add(&H, C[g->col[a]], g->w[a]);
    }
    /* emit in ascending neighbour order */
    int64_t k = 0;
    qsort(H.h.keys, (size_t)H.h.nkeys, sizeof(int32_t), cmp_i32);
    for (int64_t x = 0; x < H.h.nkeys; x++) {
      ycol[yoff[c] + k] = H.h.keys[x];
      yw[yoff[c] + k] = H.h.val[H.h.keys[x]];
      k++;
    }
    ylen[c] = k;
    sht_clear(&H);
  }
  sht_free(&H);
  /* compact into a dense CSR */
  out->n = ncomm;
  out->off = (int64_t *)xcalloc((size_t)(ncomm + 1), sizeof(int64_t));
  for (int64_t c = 0; c < ncomm; c++) out->off[c + 1] = out->off[c] + ylen[c];
  out->col = (int32_t *)xmalloc((size_t)out->off[ncomm] * sizeof(int32_t));
  out->w = (int64_t *)xmalloc((size_t)out->off[ncomm] * sizeof(int64_t));
  for (int64_t c = 0; c < ncomm; c++) {
    memcpy(out->col + out->off[c], ycol + yoff[c], (size_t)ylen[c] * sizeof(int32_t));
    memcpy(out->w + out->off[c], yw + yoff[c], (size_t)ylen[c] * sizeof(int64_t));
  }
  free(coff); free(cv); free(cur); free(yoff); free(ycol); free(yw); free(ylen);
  return 0;
}

int64_t oracle_aggregate(int64_t n, const int64_t *off, const int32_t *col, const int64_t *w,
                         const int32_t *C, int64_t ncomm, int64_t *off_out, int32_t *col_out,
                         int64_t *w_out) {
  for (int64_t i = 0; i < n; i++)
    if (C[i] < 0 || C[i] >= ncomm) return -1;
  ograph g = {n, (int64_t *)off, (int32_t *)col, (int64_t *)w}, y;
  if (aggregate_graph(&g, C, ncomm, &y) != 0) return -1;
  int64_t arcs = y.off[ncomm];
  memcpy(off_out, y.off, (size_t)(ncomm + 1) * sizeof(int64_t));
  memcpy(col_out, y.col, (size_t)arcs * sizeof(int32_t));
  memcpy(w_out, y.w, (size_t)arcs * sizeof(int64_t));
  graph_free(&y);
  return arcs;
}

/* ------------------------------------------------ Alg. leidentr (tracking) */

/* Reading: the weighted Boyer-Moore vote is replaced by the exact weighted
 * overlap argmax (the vote's answer whenever a majority exists), ties to the
 * lowest id, in both directions.  New communities no old community picked
 * take the ids no old community used, the k-th smallest such id going to
 * the k-th smallest unmatched new id.  Returns the relabelled membership in
 * Cnew, and `matched_old[id]` = 1 for old ids that were kept. */
static void track_communities(int64_t n, int32_t *Cnew, const int32_t *Cold, const int64_t *K,
                              uint8_t *matched_old) {
  /* overlap weights: sort vertices by (old, new) */
  int64_t *ord = (int64_t *)xmalloc((size_t)n * sizeof(int64_t));
  /* counting sort by new, then stable counting sort by old */
  int64_t *cnt = (int64_t *)xcalloc((size_t)(n + 1), sizeof(int64_t));
  int64_t *tmp = (int64_t *)xmalloc((size_t)n * sizeof(int64_t));
  for (int64_t i = 0; i < n; i++) cnt[Cnew[i] + 1]++;
  for (int64_t c = 0; c < n; c++) cnt[c + 1] += cnt[c];
  for (int64_t i = 0; i < n; i++) tmp[cnt[Cnew[i]]++] = i;
  memset(cnt, 0, (size_t)(n + 1) * sizeof(int64_t));
  for (int64_t i = 0; i < n; i++) cnt[Cold[i] + 1]++;
  for (int64_t c = 0; c < n; c++) cnt[c + 1] += cnt[c];
  for (int64_t t = 0; t < n; t++) { int64_t i = tmp[t]; ord[cnt[Cold[i]]++] = i; }
  free(tmp); free(cnt);
  int32_t *best_new = (int32_t *)xmalloc((size_t)n * sizeof(int32_t)); /* by old id */
  int64_t *best_new_w = (int64_t *)xmalloc((size_t)n * sizeof(int64_t));
  uint8_t *old_used = (uint8_t *)xcalloc((size_t)n, 1);
  for (int64_t b = 0; b < n; b++) best_new[b] = -1;
  for (int64_t t = 0; t < n;) {
    int64_t u = t;
    int32_t b = Cold[ord[t]], c = Cnew[ord[t]];
    int64_t wsum = 0;
    while (u < n && Cold[ord[u]] == b && Cnew[ord[u]] == c) { wsum += K[ord[u]]; u++; }
    old_used[b] = 1;
    /* pairs arrive in ascending c for a fixed b, so '>' keeps the lowest c on ties */
    if (best_new[b] < 0 || wsum > best_new_w[b]) { best_new[b] = c; best_new_w[b] = wsum; }
    t = u;
  }
  free(ord);
  int32_t *best_old = (int32_t *)xmalloc((size_t)n * sizeof(int32_t)); /* by new id */
  int64_t *best_old_w = (int64_t *)xmalloc((size_t)n * sizeof(int64_t));
  uint8_t *new_used = (uint8_t *)xcalloc((size_t)n, 1);
  for (int64_t c = 0; c < n; c++) best_old[c] = -1;
  for (int64_t i = 0; i < n; i++) new_used[Cnew[i]] = 1;
  for (int64_t b = 0; b < n; b++) { /* ascending b: '>' keeps the lowest b on ties */
    int32_t c = best_new[b];
    if (c < 0) continue;
    if (best_old[c] < 0 || best_new_w[b] > best_old_w[c]) { best_old[c] = (int32_t)b; best_old_w[c] = best_new_w[b]; }
  }
  int32_t *map = (int32_t *)xmalloc((size_t)n * sizeof(int32_t));
  int64_t fr = 0; /* next free id candidate */
  memset(matched_old, 0, (size_t)n);
  for (int64_t c = 0; c < n; c++) {
    if (!new_used[c]) continue;
    if (best_old[c] >= 0) { map[c] = best_old[c]; matched_old[best_old[c]] = 1; continue; }
    while (old_used[fr]) fr++;
    map[c] = (int32_t)fr++;
  }
  for (int64_t i = 0; i < n; i++) Cnew[i] = map[Cnew[i]];
  free(best_new); free(best_new_w); free(old_used); free(best_old); free(best_old_w);
  free(new_used); free(map);
}

/* --------------------------------------------------------- Alg. leiden */

static int leiden_run(oracle_state *s, const int32_t *Cprev, uint8_t *dSp, uint8_t *dR,
                      const leiden_ctx *ctx, int32_t *Cout) {
  const oracle_params *p = &s->p;
  int64_t N = s->g.n;
  int64_t m2 = s->m2;
  memset(s->trace, 0, sizeof(s->trace));
  /* Mark affected vertices as unprocessed; C <- [0..N); C' <- C^{t-1}; K', Sigma' */
  uint8_t *unproc = (uint8_t *)xmalloc((size_t)N);
  for (int64_t i = 0; i < N; i++) unproc[i] = ctx->affected[i] ? 1 : 0;
  int32_t *Ctop = (int32_t *)xmalloc((size_t)N * sizeof(int32_t));
  for (int64_t i = 0; i < N; i++) Ctop[i] = (int32_t)i;
  int32_t *Cp = (int32_t *)xmalloc((size_t)N * sizeof(int32_t));
  memcpy(Cp, Cprev, (size_t)N * sizeof(int32_t));
  int64_t *Kp = (int64_t *)xmalloc((size_t)N * sizeof(int64_t));
  int64_t *Sp = (int64_t *)xmalloc((size_t)N * sizeof(int64_t));
  memcpy(Kp, s->K, (size_t)N * sizeof(int64_t));
  memcpy(Sp, s->S, (size_t)N * sizeof(int64_t));
  int32_t *CB = (int32_t *)xmalloc((size_t)N * sizeof(int32_t));
  ograph G = s->g; /* level graph; level 0 is borrowed, later levels owned */
  int owned = 0;
  double tau = p->tau;
  const uint8_t *in_range = ctx->in_range;
  int passes = 0;
  scan_ht H;
  if (sht_init(&H, N) != 0) return ORACLE_ERR_OOM;
  for (int lp = 0; lp < p->max_passes; lp++) {
    int64_t n = G.n;
    int64_t *tr = &s->trace[2 + lp * ORACLE_TRACE_PASS];
    passes++;
    tr[0] = n;
    int li;
    if (p->schedule == ORACLE_SYNC)
      li = leiden_move_sync(&G, Cp, Kp, Sp, dSp, unproc, lp == 0 ? in_range : NULL, ctx->dynamic, tau,
                            m2, p, &H, tr + 5);
    else
      li = leiden_move_seq(&G, Cp, Kp, Sp, dSp, unproc, lp == 0 ? in_range : NULL, ctx->dynamic, tau,
                           m2, p, &H, tr + 5);
    tr[1] = li;
    subset_renumber(n, Cp, Sp, dSp, dR);
    /* split communities marked in dS and not in dR (or, as an ablation, every
       community not in dR) */
    uint8_t *split_c = (uint8_t *)xcalloc((size_t)n, 1);
    for (int64_t c = 0; c < n; c++) split_c[c] = (p->split_all || dSp[c]) && !dR[c];
    split_components(&G, Cp, split_c);
    free(split_c);
    memcpy(CB, Cp, (size_t)n * sizeof(int32_t)); /* community bounds */
    int refined_any = 0;
    for (int64_t i = 0; i < n; i++)
      if (dR[CB[i]]) { refined_any = 1; break; }
    if (p->schedule == ORACLE_SYNC)
      tr[4] = refine_sync(&G, CB, Cp, Kp, Sp, dR, m2, p->max_iterations, &H);
    else
      tr[4] = refine_seq(&G, CB, Cp, Kp, Sp, dR, m2, &H);
    tr[3] = refined_any;
    {
      uint8_t *seen = (uint8_t *)xcalloc((size_t)n, 1);
      int64_t k = 0;
      for (int64_t i = 0; i < n; i++)
        if (!seen[Cp[i]]) { seen[Cp[i]] = 1; k++; }
      free(seen);
      tr[2] = k;
    }
    if (p->converge_any) {
      if (li <= 1 || !refined_any) break;
    } else {
      if (li <= 1 && !refined_any) break;
      if (li <= 1 && lp > 0) break;
    }
    int64_t ncomm = renumber_dense(n, Cp);
    for (int64_t v = 0; v < N; v++) Ctop[v] = Cp[Ctop[v]]; /* dendrogram lookup */
    ograph Y;
    if (aggregate_graph(&G, Cp, ncomm, &Y) != 0) return ORACLE_ERR_OOM;
    if (owned) graph_free(&G);
    G = Y;
    owned = 1;
    /* Sigma' <- K' <- weight of each super-vertex; all unprocessed;
     * C' <- identity; dR <- all; dS cleared; tau scaled */
    for (int64_t c = 0; c < ncomm; c++) {
      int64_t k = 0;
      for (int64_t a = G.off[c]; a < G.off[c + 1]; a++) k += G.w[a];
      Kp[c] = Sp[c] = k;
      unproc[c] = 1;
      Cp[c] = (int32_t)c;
      dR[c] = 1;
      dSp[c] = 0;
    }
    tau /= p->tau_drop;
  }
  sht_free(&H);
  for (int64_t v = 0; v < N; v++) Ctop[v] = Cp[Ctop[v]];
  s->trace[0] = passes;
  memcpy(Cout, Ctop, (size_t)N * sizeof(int32_t));
  if (owned) graph_free(&G);
  free(unproc); free(Ctop); free(Cp); free(Kp); free(Sp); free(CB);
  return ORACLE_OK;
}

/* Tracking, then Sigma^t from C^t and Delta Sigma re-keyed to the kept ids. */
static void finish_tracking(oracle_state *s, int32_t *Cnew) {
  int64_t N = s->g.n;
  uint8_t *matched_old = (uint8_t *)xmalloc((size_t)N);
  track_communities(N, Cnew, s->C, s->K, matched_old);
  memcpy(s->C, Cnew, (size_t)N * sizeof(int32_t));
  memset(s->S, 0, (size_t)N * sizeof(int64_t));
  for (int64_t i = 0; i < N; i++) s->S[s->C[i]] += s->K[i];
  for (int64_t c = 0; c < N; c++)
    if (!matched_old[c]) s->dS[c] = 0;
  free(matched_old);
}

/* --------------------------------------------------------------- API */

oracle_state *oracle_create(const oracle_params *p, int64_t n, const int64_t *off, const int32_t *col,
                            const int32_t *w) {
  if (!p || n < 0 || n > 0x7fffffff || !off) return NULL;
  int64_t arcs = off[n];
  for (int64_t i = 0; i < n; i++)
    if (off[i + 1] < off[i]) return NULL;
  for (int64_t a = 0; a < arcs; a++)
    if (col[a] < 0 || col[a] >= n || (w && w[a] <= 0)) return NULL;
  oracle_state *s = (oracle_state *)xcalloc(1, sizeof(oracle_state));
  s->p = *p;
  s->g.n = n;
  s->g.off = (int64_t *)xmalloc((size_t)(n + 1) * sizeof(int64_t));
  s->g.col = (int32_t *)xmalloc((size_t)arcs * sizeof(int32_t));
  s->g.w = (int64_t *)xmalloc((size_t)arcs * sizeof(int64_t));
  memcpy(s->g.off, off, (size_t)(n + 1) * sizeof(int64_t));
  memcpy(s->g.col, col, (size_t)arcs * sizeof(int32_t));
  for (int64_t a = 0; a < arcs; a++) s->g.w[a] = w ? w[a] : 1;
  s->C = (int32_t *)xcalloc((size_t)n, sizeof(int32_t));
  s->K = (int64_t *)xcalloc((size_t)n, sizeof(int64_t));
  s->S = (int64_t *)xcalloc((size_t)n, sizeof(int64_t));
  s->dS = (int64_t *)xcalloc((size_t)n, sizeof(int64_t));
  s->dV = (uint8_t *)xcalloc((size_t)n, 1);
  return s;
}

void oracle_destroy(oracle_state *s) {
  if (!s) return;
  graph_free(&s->g);
  free(s->C); free(s->K); free(s->S); free(s->dS); free(s->dV);
  free(s);
}

/* Static Leiden: the same leiden() with C^{t-1} = singletons, every vertex
 * affected, every community refined and nothing split. */
int oracle_static(oracle_state *s, int32_t *out) {
  int64_t N = s->g.n;
  s->m2 = 0;
  for (int64_t i = 0; i < N; i++) {
    int64_t k = 0;
    for (int64_t a = s->g.off[i]; a < s->g.off[i + 1]; a++) k += s->g.w[a];
    s->K[i] = k;
    s->S[i] = k;
    s->C[i] = (int32_t)i;
    s->dS[i] = 0;
    s->m2 += k;
  }
  uint8_t *dSp = (uint8_t *)xcalloc((size_t)N, 1);
  uint8_t *dR = (uint8_t *)xmalloc((size_t)N);
  memset(dR, 1, (size_t)N);
  memset(s->dV, 1, (size_t)N);
  leiden_ctx ctx = {0, s->dV, NULL};
  int32_t *Cnew = (int32_t *)xmalloc((size_t)N * sizeof(int32_t));
  int rc = leiden_run(s, s->C, dSp, dR, &ctx, Cnew);
  s->trace[1] = N;
  if (rc == ORACLE_OK) finish_tracking(s, Cnew);
  free(dSp); free(dR); free(Cnew);
  if (rc == ORACLE_OK) {
    s->has_static = 1;
    if (out) memcpy(out, s->C, (size_t)N * sizeof(int32_t));
  }
  return rc;
}

/* One arc of a canonical batch: (i, j, w), both directions present. */
typedef struct { int32_t i, j; int64_t w; } arc_t;

static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return x < y ? -1 : x > y;
}

static int64_t find_arc(const ograph *g, int64_t u, int64_t v) {
  for (int64_t a = g->off[u]; a < g->off[u + 1]; a++)
    if (g->col[a] == v) return a;
  return -1;
}

int oracle_update(oracle_state *s, const int32_t *del3, int64_t n_del, const int32_t *ins3, int64_t n_ins,
                  int mode, int32_t *out) {
  if (!s->has_static) return ORACLE_ERR_STATE;
  if (mode < ORACLE_ND || mode > ORACLE_DF || n_del < 0 || n_ins < 0) return ORACLE_ERR_ARG;
  int64_t N = s->g.n;
  /* ---- canonical batch (reading of the batch edge cases): ids in range,
   * no self-loops, insertion weights > 0, deletions must name existing
   * edges (their stored weight is used), repeated deletions collapse,
   * repeated insertions add up; deletions apply before insertions. */
  uint64_t *dk = (uint64_t *)xmalloc((size_t)n_del * sizeof(uint64_t));
  uint64_t *ik = (uint64_t *)xmalloc((size_t)n_ins * 2 * sizeof(uint64_t));
  for (int64_t e = 0; e < n_del; e++) {
    int64_t u = del3[3 * e], v = del3[3 * e + 1];
    if (u < 0 || u >= N || v < 0 || v >= N || u == v) { free(dk); free(ik); return ORACLE_ERR_BATCH; }
    int64_t x = u < v ? u : v, y = u < v ? v : u;
    dk[e] = ((uint64_t)x << 32) | (uint64_t)y;
  }
  for (int64_t e = 0; e < n_ins; e++) {
    int64_t u = ins3[3 * e], v = ins3[3 * e + 1], w = ins3[3 * e + 2];
    if (u < 0 || u >= N || v < 0 || v >= N || u == v || w <= 0) { free(dk); free(ik); return ORACLE_ERR_BATCH; }
    int64_t x = u < v ? u : v, y = u < v ? v : u;
    ik[2 * e] = ((uint64_t)x << 32) | (uint64_t)y;
    ik[2 * e + 1] = (uint64_t)w;
  }
  qsort(dk, (size_t)n_del, sizeof(uint64_t), cmp_u64);
  int64_t nd = 0;
  for (int64_t e = 0; e < n_del; e++)
    if (e == 0 || dk[e] != dk[e - 1]) dk[nd++] = dk[e];
  qsort(ik, (size_t)n_ins, 2 * sizeof(uint64_t), cmp_u64); /* sorts by key (first word) */
  int64_t ni = 0;
  for (int64_t e = 0; e < n_ins; e++) {
    if (ni > 0 && ik[2 * (ni - 1)] == ik[2 * e]) { ik[2 * (ni - 1) + 1] += ik[2 * e + 1]; continue; }
    ik[2 * ni] = ik[2 * e]; ik[2 * ni + 1] = ik[2 * e + 1]; ni++;
  }
  arc_t *dA = (arc_t *)xmalloc((size_t)(2 * nd) * sizeof(arc_t));
  arc_t *iA = (arc_t *)xmalloc((size_t)(2 * ni) * sizeof(arc_t));
  for (int64_t e = 0; e < nd; e++) {
    int32_t x = (int32_t)(dk[e] >> 32), y = (int32_t)(dk[e] & 0xffffffffu);
    int64_t a = find_arc(&s->g, x, y);
    if (a < 0) { free(dk); free(ik); free(dA); free(iA); return ORACLE_ERR_BATCH; }
    dA[2 * e] = (arc_t){x, y, s->g.w[a]};
    dA[2 * e + 1] = (arc_t){y, x, s->g.w[a]};
  }
  for (int64_t e = 0; e < ni; e++) {
    int32_t x = (int32_t)(ik[2 * e] >> 32), y = (int32_t)(ik[2 * e] & 0xffffffffu);
    iA[2 * e] = (arc_t){x, y, (int64_t)ik[2 * e + 1]};
    iA[2 * e + 1] = (arc_t){y, x, (int64_t)ik[2 * e + 1]};
  }
  free(dk); free(ik);
  int64_t nda = 2 * nd, nia = 2 * ni;

  /* ---- G^{t-1} + batch -> G^t (rebuild every row: plain and slow) */
  {
    int64_t *deg = (int64_t *)xcalloc((size_t)N, sizeof(int64_t));
    uint8_t *gone = (uint8_t *)xcalloc((size_t)s->g.off[N] + 1, 1);
    for (int64_t e = 0; e < nda; e++) gone[find_arc(&s->g, dA[e].i, dA[e].j)] = 1;
    for (int64_t i = 0; i < N; i++)
      for (int64_t a = s->g.off[i]; a < s->g.off[i + 1]; a++)
        if (!gone[a]) deg[i]++;
    /* insertions of edges that survive the deletions add to their weight */
    int64_t *add_at = (int64_t *)xmalloc((size_t)(nia + 1) * sizeof(int64_t));
    for (int64_t e = 0; e < nia; e++) {
      int64_t a = find_arc(&s->g, iA[e].i, iA[e].j);
      add_at[e] = (a >= 0 && !gone[a]) ? a : -1;
      if (add_at[e] < 0) deg[iA[e].i]++;
    }
    ograph G2;
    G2.n = N;
    G2.off = (int64_t *)xcalloc((size_t)(N + 1), sizeof(int64_t));
    for (int64_t i = 0; i < N; i++) G2.off[i + 1] = G2.off[i] + deg[i];
    G2.col = (int32_t *)xmalloc((size_t)G2.off[N] * sizeof(int32_t));
    G2.w = (int64_t *)xmalloc((size_t)G2.off[N] * sizeof(int64_t));
    for (int64_t e = 0; e < nia; e++)
      if (add_at[e] >= 0) s->g.w[add_at[e]] += iA[e].w;
    int64_t *pos = (int64_t *)xmalloc((size_t)N * sizeof(int64_t));
    for (int64_t i = 0; i < N; i++) {
      pos[i] = G2.off[i];
      for (int64_t a = s->g.off[i]; a < s->g.off[i + 1]; a++)
        if (!gone[a]) { G2.col[pos[i]] = s->g.col[a]; G2.w[pos[i]] = s->g.w[a]; pos[i]++; }
    }
    for (int64_t e = 0; e < nia; e++)
      if (add_at[e] < 0) { G2.col[pos[iA[e].i]] = iA[e].j; G2.w[pos[iA[e].i]] = iA[e].w; pos[iA[e].i]++; }
    free(pos); free(deg); free(gone); free(add_at);
    graph_free(&s->g);
    s->g = G2;
  }

  /* ---- affected vertices (Alg. naive / delta / frontier) */
  const int32_t *Cprev = s->C;
  uint8_t *dV = s->dV;
  memset(dV, 0, (size_t)N);
  const uint8_t *in_range = NULL;
  uint8_t *dE = NULL, *dCf = NULL;
  if (mode == ORACLE_ND) {
    memset(dV, 1, (size_t)N);
  } else if (mode == ORACLE_DF) {
    for (int64_t e = 0; e < nda; e++)
      if (Cprev[dA[e].i] == Cprev[dA[e].j]) dV[dA[e].i] = 1;
    for (int64_t e = 0; e < nia; e++)
      if (Cprev[iA[e].i] != Cprev[iA[e].j]) dV[iA[e].i] = 1;
  } else { /* DS, using K^{t-1}, Sigma^{t-1}, m^{t-1} (marking precedes updateWeights) */
    dE = (uint8_t *)xcalloc((size_t)N, 1);
    dCf = (uint8_t *)xcalloc((size_t)N, 1);
    for (int64_t e = 0; e < nda; e++)
      if (Cprev[dA[e].i] == Cprev[dA[e].j]) { dV[dA[e].i] = 1; dE[dA[e].i] = 1; dCf[Cprev[dA[e].j]] = 1; }
    /* per unique source of the insertions: hash C^{t-1}[j] -> sum w over
     * cross-community insertions, c* = largest delta-modularity (ties to the
     * lowest id); reading: i is marked only when that hash is non-empty */
    arc_t *sorted = (arc_t *)xmalloc((size_t)(nia + 1) * sizeof(arc_t));
    memcpy(sorted, iA, (size_t)nia * sizeof(arc_t));
    /* group by source: counting sort */
    int64_t *cnt = (int64_t *)xcalloc((size_t)(N + 1), sizeof(int64_t));
    for (int64_t e = 0; e < nia; e++) cnt[iA[e].i + 1]++;
    for (int64_t i = 0; i < N; i++) cnt[i + 1] += cnt[i];
    int64_t *cur = (int64_t *)xmalloc((size_t)(N + 1) * sizeof(int64_t));
    memcpy(cur, cnt, (size_t)(N + 1) * sizeof(int64_t));
    for (int64_t e = 0; e < nia; e++) sorted[cur[iA[e].i]++] = iA[e];
    free(cur);
    scan_ht H;
    sht_init(&H, N);
    for (int64_t i = 0; i < N; i++) {
      if (cnt[i] == cnt[i + 1]) continue;
      for (int64_t e = cnt[i]; e < cnt[i + 1]; e++)
        if (Cprev[i] != Cprev[sorted[e].j]) sht_add(&H, Cprev[sorted[e].j], sorted[e].w);
      if (H.h.nkeys == 0) continue;
      i128 rel;
      int32_t cs = best_community(&H, -1, s->m2, s->K[i], s->S, &rel);
      sht_clear(&H);
      dV[i] = 1; dE[i] = 1; dCf[cs] = 1;
    }
    sht_free(&H);
    free(cnt); free(sorted);
    for (int64_t i = 0; i < N; i++) /* expansion over neighbours and communities */
      if (dE[i])
        for (int64_t a = s->g.off[i]; a < s->g.off[i + 1]; a++) dV[s->g.col[a]] = 1;
    for (int64_t i = 0; i < N; i++)
      if (dCf[Cprev[i]]) dV[i] = 1;
    in_range = dV;
  }

  /* ---- Alg. update: updateWeights, updateChanges */
  for (int64_t e = 0; e < nda; e++) {
    s->K[dA[e].i] -= dA[e].w;
    s->S[Cprev[dA[e].i]] -= dA[e].w;
    s->m2 -= dA[e].w;
    s->dS[Cprev[dA[e].i]] += dA[e].w;
  }
  for (int64_t e = 0; e < nia; e++) {
    s->K[iA[e].i] += iA[e].w;
    s->S[Cprev[iA[e].i]] += iA[e].w;
    s->m2 += iA[e].w;
    s->dS[Cprev[iA[e].i]] += iA[e].w;
  }
  /* ---- Alg. leidenmk: dS for same-community deletions; dR for
   * same-community deletions and insertions with dSigma/Sigma > tau_re
   * (reading: flags are per community of the source), then dSigma of the
   * marked communities is reset to 0. */
  uint8_t *dSp = (uint8_t *)xcalloc((size_t)N, 1);
  uint8_t *dR = (uint8_t *)xcalloc((size_t)N, 1);
  for (int64_t e = 0; e < nda; e++)
    if (Cprev[dA[e].i] == Cprev[dA[e].j]) dSp[Cprev[dA[e].i]] = 1;
  for (int64_t t = 0; t < nda + nia; t++) {
    const arc_t *a = t < nda ? &dA[t] : &iA[t - nda];
    int32_t c = Cprev[a->i];
    if (c != Cprev[a->j]) continue;
    if ((double)s->dS[c] / (double)s->S[c] > s->p.tau_refine) dR[c] = 1;
  }
  for (int64_t c = 0; c < N; c++)
    if (dR[c]) s->dS[c] = 0;

  /* ---- Alg. leiden */
  int64_t naff = 0;
  for (int64_t i = 0; i < N; i++) naff += dV[i];
  leiden_ctx ctx = {1, dV, in_range};
  int32_t *Cnew = (int32_t *)xmalloc((size_t)N * sizeof(int32_t));
  int rc = leiden_run(s, Cprev, dSp, dR, &ctx, Cnew);
  s->trace[1] = naff;
  if (rc == ORACLE_OK) finish_tracking(s, Cnew);
  free(Cnew); free(dSp); free(dR); free(dA); free(iA); free(dE); free(dCf);
  if (rc == ORACLE_OK && out) memcpy(out, s->C, (size_t)N * sizeof(int32_t));
  return rc;
}

int oracle_get_state(const oracle_state *s, int32_t *C, int64_t *K, int64_t *Sigma, int64_t *dSigma, int64_t *m2) {
  int64_t N = s->g.n;
  if (C) memcpy(C, s->C, (size_t)N * sizeof(int32_t));
  if (K) memcpy(K, s->K, (size_t)N * sizeof(int64_t));
  if (Sigma) memcpy(Sigma, s->S, (size_t)N * sizeof(int64_t));
  if (dSigma) memcpy(dSigma, s->dS, (size_t)N * sizeof(int64_t));
  if (m2) *m2 = s->m2;
  return ORACLE_OK;
}

int64_t oracle_graph_arcs(const oracle_state *s) { return s->g.off[s->g.n]; }

/* Canonical form of G^t: rows sorted by neighbour. */
int oracle_get_graph(const oracle_state *s, int64_t *off, int32_t *col, int64_t *w) {
  int64_t N = s->g.n;
  memcpy(off, s->g.off, (size_t)(N + 1) * sizeof(int64_t));
  for (int64_t i = 0; i < N; i++) {
    int64_t lo = s->g.off[i], hi = s->g.off[i + 1];
    uint64_t *tmp = (uint64_t *)xmalloc((size_t)(hi - lo) * 2 * sizeof(uint64_t));
    for (int64_t a = lo; a < hi; a++) {
      tmp[2 * (a - lo)] = (uint64_t)s->g.col[a];
      tmp[2 * (a - lo) + 1] = (uint64_t)s->g.w[a];
    }
    qsort(tmp, (size_t)(hi - lo), 2 * sizeof(uint64_t), cmp_u64);
    for (int64_t a = lo; a < hi; a++) {
      col[a] = (int32_t)tmp[2 * (a - lo)];
      w[a] = (int64_t)tmp[2 * (a - lo) + 1];
    }
    free(tmp);
  }
  return ORACLE_OK;
}

int oracle_get_affected(const oracle_state *s, uint8_t *dV) {
  memcpy(dV, s->dV, (size_t)s->g.n);
  return ORACLE_OK;
}

int oracle_get_trace(const oracle_state *s, int64_t *trace) {
  memcpy(trace, s->trace, sizeof(s->trace));
  return ORACLE_OK;
}
