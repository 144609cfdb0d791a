/*
 * Seeded synthetic inputs for dynamic Leiden: graphs and batch updates.
 *
 * This module holds no part of the community-detection arithmetic.  It only
 * draws graphs and edge batches whose shapes follow the paper's workloads
 * (random batch updates with an 80:20 insertion:deletion mix, unit weights,
 * undirected, no new vertices -- Evaluation, "Batch generation"), and it is
 * the one piece of code shared by the CUDA path's tests and the CPU oracle's.
 *
 * Every random number is a pure function of (seed, stream, counter): the
 * SplitMix64 output function (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) applied to
 * seed + (counter + 1) * 0x9E3779B97F4A7C15, with the stream folded into the
 * seed.  The result does not depend on thread count or call order.
 *
 * All graphs are returned as symmetric CSR (int64 offsets, int32 columns and
 * int32 weights), rows sorted by column, without self-loops or duplicates.
 * Buffers are malloc'd here and released with synth_free().
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>
#include <unistd.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static inline uint64_t rng_u64(uint64_t seed, uint64_t stream, uint64_t ctr) {
  uint64_t s = mix64(seed ^ (stream * 0xD1B54A32D192ED03ULL + 0x8CB92BA72F3D8DD7ULL));
  return mix64(s + (ctr + 1) * GOLDEN);
}

/* Uniform integer in [0, n): Lemire's multiply-shift on the top 32 bits is
 * not enough for n > 2^32, so use the 128-bit product of a 64-bit draw. */
static inline uint64_t rng_below(uint64_t seed, uint64_t stream, uint64_t ctr, uint64_t n) {
  unsigned __int128 p = (unsigned __int128)rng_u64(seed, stream, ctr) * n;
  return (uint64_t)(p >> 64);
}

/* ---------------------------------------------------------------- CSR build */

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return x < y ? -1 : x > y;
}

static void sort_row(int32_t *r, int64_t len) {
  if (len > 48) { qsort(r, (size_t)len, sizeof(int32_t), cmp_i32); return; }
  for (int64_t i = 1; i < len; i++) { /* insertion sort for short rows */
    int32_t x = r[i];
    int64_t j = i - 1;
    while (j >= 0 && r[j] > x) { r[j + 1] = r[j]; j--; }
    r[j + 1] = x;
  }
}

/* ------------------------------------------------------------ threading */

static int n_threads(void) {
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  const char *e = getenv("SYNTH_THREADS");
  if (e && atoi(e) > 0) c = atoi(e);
  if (c < 1) c = 1;
  if (c > 64) c = 64;
  return (int)c;
}

typedef struct {
  int tid, nt;
  void *ctx;
  void (*fn)(void *ctx, int tid, int nt);
} job_t;

static void *job_main(void *p) {
  job_t *j = (job_t *)p;
  j->fn(j->ctx, j->tid, j->nt);
  return NULL;
}

/* Run fn(ctx, tid, nt) on nt threads; each thread takes a fixed share. */
static void parallel_run(void (*fn)(void *, int, int), void *ctx) {
  int nt = n_threads();
  pthread_t th[64];
  job_t jobs[64];
  for (int t = 0; t < nt; t++) {
    jobs[t] = (job_t){t, nt, ctx, fn};
    if (t > 0) pthread_create(&th[t], NULL, job_main, &jobs[t]);
  }
  job_main(&jobs[0]);
  for (int t = 1; t < nt; t++) pthread_join(th[t], NULL);
}

static inline void span(int64_t n, int tid, int nt, int64_t *lo, int64_t *hi) {
  *lo = n * tid / nt;
  *hi = n * (tid + 1) / nt;
}

/* Turn a list of undirected pairs (u, v) into a symmetric CSR with unit
 * weights: counting sort of both directions by source, then each row is
 * sorted; self-pairs are dropped and repeated pairs collapse.  The scatter
 * order inside a row depends on thread timing, the sorted rows do not. */
typedef struct {
  int64_t n, m;
  const int64_t *u, *v;
  int64_t *pos, *cur, *uniq;
  int32_t *tmp, *col;
  const int64_t *off;
  int phase;
} csr_ctx;

static void csr_work(void *p, int tid, int nt) {
  csr_ctx *c = (csr_ctx *)p;
  int64_t lo, hi;
  if (c->phase == 0) { /* degrees */
    span(c->m, tid, nt, &lo, &hi);
    for (int64_t e = lo; e < hi; e++) {
      if (c->u[e] == c->v[e]) continue;
      __atomic_fetch_add(&c->pos[c->u[e] + 1], 1, __ATOMIC_RELAXED);
      __atomic_fetch_add(&c->pos[c->v[e] + 1], 1, __ATOMIC_RELAXED);
    }
  } else if (c->phase == 1) { /* scatter */
    span(c->m, tid, nt, &lo, &hi);
    for (int64_t e = lo; e < hi; e++) {
      if (c->u[e] == c->v[e]) continue;
      c->tmp[__atomic_fetch_add(&c->cur[c->u[e]], 1, __ATOMIC_RELAXED)] = (int32_t)c->v[e];
      c->tmp[__atomic_fetch_add(&c->cur[c->v[e]], 1, __ATOMIC_RELAXED)] = (int32_t)c->u[e];
    }
  } else if (c->phase == 2) { /* sort and deduplicate each row in place */
    span(c->n, tid, nt, &lo, &hi);
    for (int64_t i = lo; i < hi; i++) {
      int32_t *r = c->tmp + c->pos[i];
      int64_t len = c->pos[i + 1] - c->pos[i], k = 0;
      sort_row(r, len);
      for (int64_t t = 0; t < len; t++)
        if (t == 0 || r[t] != r[t - 1]) r[k++] = r[t];
      c->uniq[i] = k;
    }
  } else { /* copy rows to their compact place */
    span(c->n, tid, nt, &lo, &hi);
    for (int64_t i = lo; i < hi; i++)
      memcpy(c->col + c->off[i], c->tmp + c->pos[i], (size_t)c->uniq[i] * sizeof(int32_t));
  }
}

static int build_csr_from_pairs(int64_t n, const int64_t *u, const int64_t *v, int64_t m,
                                int64_t **off_out, int32_t **col_out, int32_t **w_out,
                                int64_t *arcs_out) {
  csr_ctx c;
  memset(&c, 0, sizeof(c));
  c.n = n; c.m = m; c.u = u; c.v = v;
  c.pos = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
  c.cur = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
  c.uniq = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
  int64_t *off = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
  if (!c.pos || !c.cur || !c.uniq || !off) { free(c.pos); free(c.cur); free(c.uniq); free(off); return -1; }
  c.phase = 0;
  parallel_run(csr_work, &c);
  for (int64_t i = 0; i < n; i++) c.pos[i + 1] += c.pos[i];
  c.tmp = (int32_t *)malloc((size_t)(c.pos[n] + 1) * sizeof(int32_t));
  if (!c.tmp) { free(c.pos); free(c.cur); free(c.uniq); free(off); return -1; }
  memcpy(c.cur, c.pos, (size_t)(n + 1) * sizeof(int64_t));
  c.phase = 1;
  parallel_run(csr_work, &c);
  c.phase = 2;
  parallel_run(csr_work, &c);
  for (int64_t i = 0; i < n; i++) off[i + 1] = off[i] + c.uniq[i];
  int64_t k = off[n];
  c.col = (int32_t *)malloc((size_t)(k + 1) * sizeof(int32_t));
  int32_t *w = (int32_t *)malloc((size_t)(k + 1) * sizeof(int32_t));
  if (!c.col || !w) { free(c.pos); free(c.cur); free(c.uniq); free(off); free(c.tmp); free(c.col); free(w); return -1; }
  c.off = off;
  c.phase = 3;
  parallel_run(csr_work, &c);
  for (int64_t a = 0; a < k; a++) w[a] = 1;
  free(c.pos); free(c.cur); free(c.uniq); free(c.tmp);
  *off_out = off; *col_out = c.col; *w_out = w; *arcs_out = k;
  return 0;
}

void synth_free(void *p) { free(p); }

/* ------------------------------------------------------ planted partition */

typedef struct { uint64_t *k; int64_t cap; } keyset; /* open addressing, 0 = empty */

static int keyset_insert(keyset *s, uint64_t key) { /* key must be != 0; returns 1 if new */
  uint64_t h = mix64(key) & (uint64_t)(s->cap - 1);
  while (s->k[h]) {
    if (s->k[h] == key) return 0;
    h = (h + 1) & (uint64_t)(s->cap - 1);
  }
  s->k[h] = key;
  return 1;
}

static uint64_t pair_key(int64_t a, int64_t b) {
  int64_t x = a < b ? a : b, y = a < b ? b : a;
  return (((uint64_t)x << 32) | (uint64_t)y) + 1;
}

/* n vertices in `blocks` equal consecutive blocks; exactly round(n*k_in/2)
 * distinct edges drawn uniformly inside blocks and round(n*k_out/2) distinct
 * edges drawn uniformly across blocks, where k_in = (1-mu)*avg_deg and
 * k_out = mu*avg_deg (repeated pairs and self-pairs are redrawn). */
int synth_planted_partition(int64_t n, int64_t blocks, double avg_deg, double mu, uint64_t seed,
                            int64_t **off, int32_t **col, int32_t **w, int64_t *arcs) {
  if (n < 2 || blocks < 1 || blocks > n) return -1;
  int64_t bs = n / blocks;
  int64_t m_in = (int64_t)llround((double)n * (1.0 - mu) * avg_deg / 2.0);
  int64_t m_out = (int64_t)llround((double)n * mu * avg_deg / 2.0);
  if (blocks == 1) { m_in += m_out; m_out = 0; }
  /* cap the request at the number of available pairs */
  double in_pairs = (double)blocks * (double)bs * (double)(bs - 1) / 2.0;
  if ((double)m_in > 0.9 * in_pairs) m_in = (int64_t)(0.9 * in_pairs);
  int64_t m = m_in + m_out;
  int64_t *u = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));
  int64_t *v = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));
  int64_t cap = 16;
  while (cap < 2 * m + 16) cap <<= 1;
  keyset s = {(uint64_t *)calloc((size_t)cap, sizeof(uint64_t)), cap};
  if (!u || !v || !s.k) { free(u); free(v); free(s.k); return -1; }
  int64_t got = 0;
  for (uint64_t t = 0; got < m_in; t++) {
    int64_t b = (int64_t)rng_below(seed, 1, 3 * t, (uint64_t)blocks);
    int64_t lo = b * bs, sz = (b == blocks - 1) ? n - lo : bs;
    int64_t x = lo + (int64_t)rng_below(seed, 1, 3 * t + 1, (uint64_t)sz);
    int64_t y = lo + (int64_t)rng_below(seed, 1, 3 * t + 2, (uint64_t)sz);
    if (x == y || !keyset_insert(&s, pair_key(x, y))) continue;
    u[got] = x; v[got] = y; got++;
  }
  for (uint64_t t = 0; got < m; t++) {
    /* one endpoint uniform over all vertices, the other uniform inside a
     * uniformly chosen different block */
    int64_t x = (int64_t)rng_below(seed, 2, 3 * t, (uint64_t)n);
    int64_t bx = x / bs < blocks ? x / bs : blocks - 1;
    int64_t by = (bx + 1 + (int64_t)rng_below(seed, 2, 3 * t + 1, (uint64_t)(blocks - 1))) % blocks;
    int64_t lo = by * bs, sz = (by == blocks - 1) ? n - lo : bs;
    int64_t y = lo + (int64_t)rng_below(seed, 2, 3 * t + 2, (uint64_t)sz);
    if (!keyset_insert(&s, pair_key(x, y))) continue;
    u[got] = x; v[got] = y; got++;
  }
  free(s.k);
  int rc = build_csr_from_pairs(n, u, v, m, off, col, w, arcs);
  free(u); free(v);
  return rc;
}

/* ------------------------------------------------------------------ R-MAT */

typedef struct {
  int scale;
  int64_t m;
  uint64_t seed;
  uint32_t ta, tb, tc;
  const int64_t *perm;
  int64_t *u, *v;
} rmat_ctx;

/* Edges [lo, hi) of the R-MAT sample: edge e descends `scale` levels using
 * 16 bits per level of the draws (seed, 8, 8e + l/4). */
static void rmat_work(void *p, int tid, int nt) {
  rmat_ctx *c = (rmat_ctx *)p;
  int64_t lo, hi;
  span(c->m, tid, nt, &lo, &hi);
  for (int64_t e = lo; e < hi; e++) {
    int64_t x = 0, y = 0;
    uint64_t r = 0;
    for (int l = 0; l < c->scale; l++) {
      if ((l & 3) == 0) r = rng_u64(c->seed, 8, (uint64_t)e * 8 + (uint64_t)(l >> 2));
      uint32_t q = (uint32_t)(r & 0xffff);
      r >>= 16;
      int bx = 0, by = 0;
      if (q < c->ta) { } else if (q < c->tb) { by = 1; } else if (q < c->tc) { bx = 1; } else { bx = 1; by = 1; }
      x = (x << 1) | bx;
      y = (y << 1) | by;
    }
    c->u[e] = c->perm[x];
    c->v[e] = c->perm[y];
  }
}

/* R-MAT (Chakrabarti, Zhan, Faloutsos 2004): 2^scale vertices and
 * edge_factor * 2^scale sampled edges; each edge descends `scale` levels of
 * the adjacency quadrants with probabilities (a, b, c, 1-a-b-c).  Vertex IDs
 * are then relabelled by a seeded random permutation, as the Graph500
 * generator does, so that degree is not correlated with ID.  The result is
 * symmetrised and deduplicated, and self-loops are dropped. */
int synth_rmat(int scale, int64_t edge_factor, double a, double b, double c, uint64_t seed,
               int64_t **off, int32_t **col, int32_t **w, int64_t *arcs) {
  if (scale < 1 || scale > 30) return -1;
  int64_t n = (int64_t)1 << scale;
  int64_t m = edge_factor * n;
  uint32_t ta = (uint32_t)llround(a * 65536.0);
  uint32_t tb = (uint32_t)llround((a + b) * 65536.0);
  uint32_t tc = (uint32_t)llround((a + b + c) * 65536.0);
  int64_t *perm = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  int64_t *u = (int64_t *)malloc((size_t)m * sizeof(int64_t));
  int64_t *v = (int64_t *)malloc((size_t)m * sizeof(int64_t));
  if (!perm || !u || !v) { free(perm); free(u); free(v); return -1; }
  for (int64_t i = 0; i < n; i++) perm[i] = i;
  for (int64_t i = n - 1; i > 0; i--) { /* Fisher-Yates */
    int64_t j = (int64_t)rng_below(seed, 7, (uint64_t)i, (uint64_t)(i + 1));
    int64_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
  }
  rmat_ctx rc0 = {scale, m, seed, ta, tb, tc, perm, u, v};
  parallel_run(rmat_work, &rc0);
  free(perm);
  int rc = build_csr_from_pairs(n, u, v, m, off, col, w, arcs);
  free(u); free(v);
  return rc;
}

/* ------------------------------------ degree-corrected planted partition */

/* Expected value of min(X, cap) for X Pareto with shape a > 1 and scale xm
 * (density a xm^a / x^(a+1), x >= xm). */
static double pareto_capped_mean(double a, double xm, double cap) {
  if (cap <= xm) return cap;
  double t = pow(xm / cap, a);
  return xm * a / (a - 1.0) * (1.0 - pow(xm / cap, a - 1.0)) + cap * t;
}

/* Inverse-CDF draw from a Pareto(shape a, scale xm) bounded to [xm, cap]
 * (the tail above cap folded onto cap). */
static double pareto_draw(double a, double xm, double cap, uint64_t r) {
  double u = ((double)(r >> 11) + 0.5) * (1.0 / 9007199254740992.0); /* (0, 1) */
  double x = xm * pow(u, -1.0 / a);
  return x < cap ? x : cap;
}

typedef struct {
  int64_t n;
  uint64_t seed;
  double mu;
  const int64_t *deg, *cstart, *comm, *perm;
  const double *gcdf, *ccdf; /* cumulative degree: global, and inside each community */
  const int64_t *eoff;       /* first edge index of each vertex */
  int64_t *u, *v;
} dcpp_ctx;

static int64_t cdf_pick(const double *cdf, int64_t lo, int64_t hi, double x) {
  /* smallest i in [lo, hi) with cdf[i] > x */
  while (lo < hi - 1) {
    int64_t mid = (lo + hi) >> 1;
    if (cdf[mid - 1] > x) hi = mid; else lo = mid;
  }
  return lo;
}

static void dcpp_work(void *p, int tid, int nt) {
  dcpp_ctx *c = (dcpp_ctx *)p;
  int64_t lo, hi;
  span(c->n, tid, nt, &lo, &hi);
  for (int64_t x = lo; x < hi; x++) {
    int64_t k = c->comm[x], a = c->cstart[k], b = c->cstart[k + 1];
    double cbase = a > 0 ? c->ccdf[a - 1] : 0.0, ctot = c->ccdf[b - 1] - cbase;
    double gtot = c->gcdf[c->n - 1];
    for (int64_t e = c->eoff[x]; e < c->eoff[x + 1]; e++) {
      uint64_t r1 = rng_u64(c->seed, 21, 2 * (uint64_t)e), r2 = rng_u64(c->seed, 21, 2 * (uint64_t)e + 1);
      double coin = ((double)(r1 >> 11)) * (1.0 / 9007199254740992.0);
      double pick = ((double)(r2 >> 11)) * (1.0 / 9007199254740992.0);
      int64_t y;
      if (coin >= c->mu && b - a > 1) y = cdf_pick(c->ccdf, a, b, cbase + pick * ctot);
      else y = cdf_pick(c->gcdf, 0, c->n, pick * gtot);
      c->u[e] = c->perm[x];
      c->v[e] = c->perm[y];
    }
  }
}

/* Degree-corrected planted partition: expected degrees from a Pareto law of
 * exponent deg_exp (density ~ d^-deg_exp) bounded by max_deg, its scale set
 * so the mean is avg_deg; community sizes from a Pareto law of exponent
 * comm_exp bounded to [cmin, cmax], filled in order; each vertex x draws
 * ceil(d_x/2) edges whose other end is, with probability 1-mu, a member of
 * x's community and otherwise any vertex, chosen in proportion to expected
 * degree (Chung-Lu style).  Vertex ids are then randomly permuted.  Weights
 * are 1..wmax from a hash of the unordered pair, so both directions agree;
 * repeated pairs collapse and self-pairs are dropped. */
int synth_dcpp(int64_t n, double avg_deg, double deg_exp, double max_deg, double comm_exp, int64_t cmin,
               int64_t cmax, double mu, int32_t wmax, uint64_t seed, int64_t **off, int32_t **col, int32_t **w,
               int64_t *arcs) {
  if (n < 2 || deg_exp <= 2.0 || comm_exp <= 1.0 || cmin < 1 || cmax < cmin || wmax < 1) return -1;
  double a = deg_exp - 1.0, lo = 1e-3, hi = avg_deg;
  for (int it = 0; it < 200; it++) { /* scale of the degree law for the requested mean */
    double mid = 0.5 * (lo + hi);
    if (pareto_capped_mean(a, mid, max_deg) < avg_deg) lo = mid; else hi = mid;
  }
  double xm = 0.5 * (lo + hi);
  int64_t *deg = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  int64_t *comm = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  int64_t *cstart = (int64_t *)malloc((size_t)(n + 2) * sizeof(int64_t));
  int64_t *perm = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  int64_t *eoff = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
  double *gcdf = (double *)malloc((size_t)n * sizeof(double));
  double *ccdf = (double *)malloc((size_t)n * sizeof(double));
  if (!deg || !comm || !cstart || !perm || !eoff || !gcdf || !ccdf) {
    free(deg); free(comm); free(cstart); free(perm); free(eoff); free(gcdf); free(ccdf);
    return -1;
  }
  int64_t nc = 0, pos = 0;
  for (uint64_t t = 0; pos < n; t++) {
    int64_t sz = (int64_t)pareto_draw(comm_exp - 1.0, (double)cmin, (double)cmax, rng_u64(seed, 22, t));
    if (sz < cmin) sz = cmin;
    if (pos + sz > n) sz = n - pos;
    cstart[nc++] = pos;
    for (int64_t x = pos; x < pos + sz; x++) comm[x] = nc - 1;
    pos += sz;
  }
  cstart[nc] = n;
  eoff[0] = 0;
  for (int64_t x = 0; x < n; x++) {
    double d = pareto_draw(a, xm, max_deg, rng_u64(seed, 23, (uint64_t)x));
    deg[x] = (int64_t)llround(d) < 1 ? 1 : (int64_t)llround(d);
    gcdf[x] = (x ? gcdf[x - 1] : 0.0) + (double)deg[x];
    ccdf[x] = gcdf[x];
    eoff[x + 1] = eoff[x] + (deg[x] + 1) / 2;
  }
  for (int64_t i = 0; i < n; i++) perm[i] = i;
  for (int64_t i = n - 1; i > 0; i--) {
    int64_t j = (int64_t)rng_below(seed, 24, (uint64_t)i, (uint64_t)(i + 1));
    int64_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
  }
  int64_t m = eoff[n];
  int64_t *u = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));
  int64_t *v = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));
  int rc = -1;
  if (u && v) {
    dcpp_ctx c = {n, seed, mu, deg, cstart, comm, perm, gcdf, ccdf, eoff, u, v};
    parallel_run(dcpp_work, &c);
    rc = build_csr_from_pairs(n, u, v, m, off, col, w, arcs);
  }
  free(u); free(v);
  free(deg); free(comm); free(cstart); free(perm); free(eoff); free(gcdf); free(ccdf);
  if (rc == 0) { /* weights from the unordered pair */
    int64_t nn = n;
    for (int64_t x = 0; x < nn; x++)
      for (int64_t e = (*off)[x]; e < (*off)[x + 1]; e++) {
        int64_t y = (*col)[e];
        uint64_t key = x < y ? ((uint64_t)x << 32) | (uint64_t)y : ((uint64_t)y << 32) | (uint64_t)x;
        (*w)[e] = 1 + (int32_t)(mix64(key ^ (seed * 0x9E3779B97F4A7C15ULL)) % (uint64_t)wmax);
      }
  }
  return rc;
}

/* ---------------------------------------------------------- batch updates */

static int has_edge(const int64_t *off, const int32_t *col, int64_t u, int64_t v) {
  int64_t lo = off[u], hi = off[u + 1];
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (col[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo < off[u + 1] && col[lo] == v;
}

/* A random batch on the CSR graph (off, col) of n vertices: n_del distinct
 * existing undirected edges chosen uniformly (by drawing a uniform arc and
 * keeping its undirected edge once), and n_ins distinct vertex pairs u != v
 * chosen uniformly among pairs that are not edges of the graph, each with
 * weight drawn uniformly from [w_lo, w_hi].  Edges are written as (u, v, w)
 * triples, one per undirected edge, into del3 (w = stored weight) and ins3. */
int synth_batch(int64_t n, const int64_t *off, const int32_t *col, const int32_t *wt,
                int64_t n_del, int64_t n_ins, int32_t w_lo, int32_t w_hi, uint64_t seed,
                int32_t *del3, int32_t *ins3) {
  int64_t arcs = off[n];
  if (n < 2) return -1;
  if (n_del > arcs / 2) return -2;
  int64_t cap = 16;
  while (cap < 2 * (n_del + n_ins) + 16) cap <<= 1;
  keyset s = {(uint64_t *)calloc((size_t)cap, sizeof(uint64_t)), cap};
  if (!s.k) return -1;
  int64_t got = 0;
  for (uint64_t t = 0; got < n_del; t++) {
    if (t > (uint64_t)(64 * (n_del + 16))) { free(s.k); return -3; }
    int64_t a = (int64_t)rng_below(seed, 11, t, (uint64_t)arcs);
    int64_t lo = 0, hi = n; /* row of arc a */
    while (hi - lo > 1) {
      int64_t mid = (lo + hi) >> 1;
      if (off[mid] <= a) lo = mid; else hi = mid;
    }
    int64_t u = lo, v = col[a];
    if (!keyset_insert(&s, pair_key(u, v))) continue;
    del3[3 * got] = (int32_t)u; del3[3 * got + 1] = (int32_t)v; del3[3 * got + 2] = wt ? wt[a] : 1;
    got++;
  }
  got = 0;
  for (uint64_t t = 0; got < n_ins; t++) {
    if (t > (uint64_t)(64 * (n_ins + 16))) { free(s.k); return -3; }
    int64_t u = (int64_t)rng_below(seed, 12, 2 * t, (uint64_t)n);
    int64_t v = (int64_t)rng_below(seed, 12, 2 * t + 1, (uint64_t)n);
    if (u == v || has_edge(off, col, u, v)) continue;
    if (!keyset_insert(&s, pair_key(u, v))) continue;
    int32_t wv = w_lo;
    if (w_hi > w_lo) wv = w_lo + (int32_t)rng_below(seed, 13, t, (uint64_t)(w_hi - w_lo + 1));
    ins3[3 * got] = (int32_t)u; ins3[3 * got + 1] = (int32_t)v; ins3[3 * got + 2] = wv;
    got++;
  }
  free(s.k);
  return 0;
}

/* Uniform integers in [0, n) for (seed, stream): used by callers that need
 * seeded choices (e.g. which configuration sample to time). */
void synth_uniform(uint64_t seed, uint64_t stream, int64_t count, uint64_t n, int64_t *out) {
  for (int64_t i = 0; i < count; i++) out[i] = (int64_t)rng_below(seed, stream, (uint64_t)i, n);
}
