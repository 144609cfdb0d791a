// Local-moving phase (Alg. "leidenlm") and refinement phase (Alg.
// "leidenre") of Leiden on one level of the dendrogram.
//
// Each vertex scans its neighbours' communities into an open-addressing
// table (K_{i->c}), takes the community with the largest delta-modularity
// (Eq. 2 times 2m^2, exact in int128; ties to the lowest community id) and
// moves when the gain is positive.  Vertices are binned by degree: a warp
// with a shared-memory table (<= 128 arcs), a block with a shared table
// (<= 1024 arcs), a block with a table in global scratch (larger).
//
// Deterministic mode (snapshot schedule): moves found in a sub-sweep are
// applied by a separate kernel after all decisions, so every decision reads
// the state at the start of the sub-sweep.  Asynchronous mode applies each
// move as soon as it is found.
#include <algorithm>
#include <atomic>
#include <type_traits>

#include "internal.h"

namespace {

constexpr int WARPS_PER_BLOCK = 8;
constexpr int BLOCK_THREADS = 128;
constexpr int HUGE_THREADS = 256;  // a hub's decision reads only its distinct communities

enum Kind { KIND_MOVE = 0, KIND_REFINE = 1 };

struct Args {
  // level graph
  int64_t n;
  const int64_t *off;
  const int32_t *deg;
  const int32_t *col;
  const void *w;
  // state
  int32_t *C;
  int64_t *S;
  const int64_t *K;
  int32_t *size;
  const int32_t *CB;     // refinement bounds
  int32_t *prop;         // refinement proposals / async states
  uint8_t *dS;           // split flags (local moving, dynamic)
  uint32_t *unproc;      // bitmap
  const uint8_t *in_range;
  int32_t *movers, *mtarget;
  const int32_t *list;   // bin list
  const int32_t *count;  // bin count (device)
  const int32_t *list_tiny;   // bin 3 list (degree <= 8), used with bin 0
  const int32_t *count_tiny;
  int64_t m2;                 // 2m of the level graph (one graph)
  // batched handles (null otherwise): graph of each vertex, 2m per graph,
  // the gain of each deferred move, per-graph refinement counters
  const int32_t *gid;
  const int64_t *m2g;
  const uint8_t *lm_on;
  int64_t *mgain;
  int32_t *accg;
  uint8_t *refg;
  DevCounters *cnt;
  int dynamic;
  int async_mode;
  int classes_mask;
  // global scratch for the huge bin
  int32_t *gkeys;
  int64_t *gvals;
  int32_t *glist;  // filled slots of each table
  int32_t *gocc;   // number of filled slots of each listed vertex
};

// 2m of the graph vertex i belongs to.
__device__ __forceinline__ int64_t m2_of(const Args &A, int64_t i) { return A.gid ? A.m2g[A.gid[i]] : A.m2; }

__device__ __forceinline__ int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

__device__ __forceinline__ void table_insert(int32_t *keys, int64_t *vals, int tmask, int32_t c, int64_t w) {
  uint32_t s = ld_hash32((uint32_t)c) & (uint32_t)tmask;
  for (uint32_t probe = 0; ld_ok(probe <= (uint32_t)tmask, LD_CHK_PROBE); probe++) {
    int32_t k = atomicCAS(&keys[s], LD_EMPTY_KEY, c);
    if (k == LD_EMPTY_KEY || k == c) {
      atomicAdd((unsigned long long *)&vals[s], (unsigned long long)w);
      return;
    }
    s = (s + 1) & (uint32_t)tmask;
  }
}

// Decision of one vertex once its table is complete: the best community c*
// (other than the current d), K_{i->c*}, K_{i->d}.
struct Best {
  i128 v;
  int32_t c;
  int64_t kc;
  int64_t kd;
};

__device__ __forceinline__ void best_merge(Best &a, const Best &b) {
  if (ld_better(b.v, b.c, a.v, a.c)) { a.v = b.v; a.c = b.c; a.kc = b.kc; }
  a.kd += b.kd;
}

__device__ __forceinline__ Best warp_best(Best b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Best t;
    t.v = ld_shfl_xor_i128(b.v, o);
    t.c = __shfl_xor_sync(LD_FULL, b.c, o);
    t.kc = __shfl_xor_sync(LD_FULL, b.kc, o);
    t.kd = __shfl_xor_sync(LD_FULL, b.kd, o);
    best_merge(b, t);
  }
  return b;
}

// Scan arcs [lo, hi) of vertex i with `stride` threads starting at `t0`.
template <typename W, int KIND>
__device__ __forceinline__ void scan_arcs(const Args &A, int64_t i, int64_t base, int64_t dg, int t0, int stride,
                                          int32_t *keys, int64_t *vals, int tmask) {
  const W *w = (const W *)A.w;
  int32_t bi = KIND == KIND_REFINE ? A.CB[i] : 0;
  for (int64_t a = t0; a < dg; a += stride) {
    int32_t j = A.col[base + a];
    if (j == i) continue;
    if (KIND == KIND_REFINE && A.CB[j] != bi) continue;
    table_insert(keys, vals, tmask, A.C[j], (int64_t)w[base + a]);
  }
}

// The decision and its effects, run by one thread (the group leader).
// Returns the gain counted into dQ (0 if no move).
template <int KIND>
__device__ __forceinline__ i128 decide_leader(const Args &A, int64_t i, const Best &b) {
  int32_t d = A.C[i];
  int64_t Ki = A.K[i];
  int64_t m2 = m2_of(A, i);
  if (b.c < 0) return 0;
  i128 g = (i128)m2 * (b.kc - b.kd) - (i128)Ki * ((i128)Ki + A.S[b.c] - A.S[d]);
  if (g <= 0) return 0;
  if (KIND == KIND_MOVE) {
    if (A.size[d] == 1 && A.size[b.c] == 1 && b.c > d) return 0;
    if (A.async_mode) {
      A.C[i] = b.c;
      atomicAdd((unsigned long long *)&A.S[d], (unsigned long long)(-Ki));
      atomicAdd((unsigned long long *)&A.S[b.c], (unsigned long long)Ki);
      atomicSub(&A.size[d], 1);
      atomicAdd(&A.size[b.c], 1);
    } else {
      int32_t slot = atomicAdd(&A.cnt->movers, 1);
      A.movers[slot] = (int32_t)i;
      A.mtarget[slot] = b.c;
      if (A.mgain) { A.mgain[2 * slot] = (int64_t)(u128)g; A.mgain[2 * slot + 1] = (int64_t)((u128)g >> 64); }
    }
    if (A.dynamic) A.dS[d] = 1;
    return g;
  } else {
    // Refinement runs in proposal/accept rounds in both modes: an in-place
    // CAS scheme (pin the target, then leave) never merges mutual best
    // pairs, because both pin each other before either can leave, and such
    // pairs are common since the gain of joining a singleton is symmetric.
    if (A.C[b.c] != b.c) return 0;  // the representative of c* left it
    A.prop[i] = b.c;
    return g;
  }
}

__device__ __forceinline__ void mark_neighbours(const Args &A, int64_t i, int64_t base, int64_t dg, int t0,
                                                int stride) {
  for (int64_t a = t0; a < dg; a += stride) {
    int32_t j = A.col[base + a];
    if (j == i) continue;
    if (A.in_range && !A.in_range[j]) continue;
    ld_bit_set(A.unproc, j);
  }
}

__device__ __forceinline__ void add_counters(DevCounters *cnt, int kind, int64_t visits, int64_t arcs, int64_t moves,
                                             i128 dq) {
  if (kind == KIND_MOVE) {
    if (visits) atomicAdd((unsigned long long *)&cnt->processed, (unsigned long long)visits);
    if (arcs) atomicAdd((unsigned long long *)&cnt->arcs, (unsigned long long)arcs);
    if (moves) atomicAdd((unsigned long long *)&cnt->moves, (unsigned long long)moves);
    if (dq != 0) ld_atomic_add_i128(cnt->dq, dq);
  } else {
    if (visits) atomicAdd((unsigned long long *)&cnt->ref_processed, (unsigned long long)visits);
    if (arcs) atomicAdd((unsigned long long *)&cnt->ref_arcs, (unsigned long long)arcs);
  }
}

// Work counters of the timed local-moving kernels (algorithmic bytes as
// stated in the C header).
__device__ __forceinline__ void add_lmk(DevCounters *cnt, int k, int64_t visits, int64_t arcs, int64_t bytes) {
  if (visits) atomicAdd((unsigned long long *)&cnt->lmk_visits[k], (unsigned long long)visits);
  if (arcs) atomicAdd((unsigned long long *)&cnt->lmk_arcs[k], (unsigned long long)arcs);
  if (bytes) atomicAdd((unsigned long long *)&cnt->lmk_bytes[k], (unsigned long long)bytes);
}

// ---------------------------------------------------------------- bins 3 and 0: warp range
// Candidate with the values the decision needs carried along, so that the
// winner's Sigma and size are not loaded again after the reduction.
struct BestX {
  i128 v;
  int32_t c;
  int32_t szc;  // size of c (local moving)
  int64_t kc;
  int64_t kd;
  int64_t sc;   // Sigma of c
};

__device__ __forceinline__ void bestx_merge(BestX &a, const BestX &b) {
  if (ld_better(b.v, b.c, a.v, a.c)) { a.v = b.v; a.c = b.c; a.kc = b.kc; a.sc = b.sc; a.szc = b.szc; }
  a.kd += b.kd;
}

__device__ __forceinline__ int64_t shfl_xor_i64(int64_t v, int o) { return __shfl_xor_sync(LD_FULL, v, o); }

// Reduction over lanes that differ in the bits of `width` - 1 (width 8:
// within aligned groups of 8 lanes; 32: the whole warp).
template <int WIDTH>
__device__ __forceinline__ BestX bestx_reduce(BestX b) {
#pragma unroll
  for (int o = WIDTH / 2; o > 0; o >>= 1) {
    BestX t;
    t.v = ld_shfl_xor_i128(b.v, o);
    t.c = __shfl_xor_sync(LD_FULL, b.c, o);
    t.szc = __shfl_xor_sync(LD_FULL, b.szc, o);
    t.kc = shfl_xor_i64(b.kc, o);
    t.kd = shfl_xor_i64(b.kd, o);
    t.sc = shfl_xor_i64(b.sc, o);
    bestx_merge(b, t);
  }
  return b;
}

// The decision of vertex i in community d (K_i, Sigma_d, size_d given) for
// the reduced candidate b.  Returns the gain (Eq. 2 times 2m^2) when i moves
// (local moving) or proposes (refinement), else 0; the caller records a
// deferred move.
template <int KIND>
__device__ __forceinline__ i128 decide_x(const Args &A, int64_t i, int32_t d, int64_t Ki, int64_t Sd, int32_t szd,
                                         int64_t m2, BestX b) {
  if (b.c < 0) return 0;
  if (KIND == KIND_MOVE && A.async_mode) {
    // in-place moves: read the totals again, as late as possible
    Sd = A.S[d];
    b.sc = A.S[b.c];
    szd = A.size[d];
    b.szc = A.size[b.c];
  }
  i128 g = (i128)m2 * (b.kc - b.kd) - (i128)Ki * ((i128)Ki + b.sc - Sd);
  if (g <= 0) return 0;
  if (KIND == KIND_MOVE) {
    if (szd == 1 && b.szc == 1 && b.c > d) return 0;
    if (A.async_mode) {
      A.C[i] = b.c;
      atomicAdd((unsigned long long *)&A.S[d], (unsigned long long)(-Ki));
      atomicAdd((unsigned long long *)&A.S[b.c], (unsigned long long)Ki);
      atomicSub(&A.size[d], 1);
      atomicAdd(&A.size[b.c], 1);
    }
    if (A.dynamic) A.dS[d] = 1;
    return g;
  } else {
    if (A.C[b.c] != b.c) return 0;  // the representative of c* left it
    A.prop[i] = b.c;
    return g;
  }
}

// The outcome of decide_x<KIND_MOVE> in the snapshot schedule, without its
// writes: a pure function of the sub-sweep's starting state, so every
// thread of a group can evaluate it.
__device__ __forceinline__ bool would_move(int32_t d, int64_t Ki, int64_t Sd, int32_t szd, int64_t m2,
                                           const BestX &b) {
  if (b.c < 0) return false;
  i128 g = (i128)m2 * (b.kc - b.kd) - (i128)Ki * ((i128)Ki + b.sc - Sd);
  if (g <= 0) return false;
  return !(szd == 1 && b.szc == 1 && b.c > d);
}

// Deferred moves of the lanes with `mv` set (snapshot schedule): one
// counter update per warp.
__device__ __forceinline__ void record_movers(const Args &A, bool mv, int32_t i, int32_t c, i128 g) {
  uint32_t m = __ballot_sync(LD_FULL, mv);
  if (!m) return;
  int lane = threadIdx.x & 31;
  int32_t p0 = 0;
  if (lane == __ffs(m) - 1) p0 = atomicAdd(&A.cnt->movers, __popc(m));
  p0 = __shfl_sync(LD_FULL, p0, __ffs(m) - 1);
  if (mv) {
    int32_t slot = p0 + __popc(m & ((1u << lane) - 1u));
    A.movers[slot] = i;
    A.mtarget[slot] = c;
    if (A.mgain) { A.mgain[2 * slot] = (int64_t)(u128)g; A.mgain[2 * slot + 1] = (int64_t)((u128)g >> 64); }
  }
}

struct Tally {
  int64_t visits = 0, arcs = 0, moves = 0;
  i128 dq = 0;
};

// Per-block sums of the lanes' tallies, then one set of counter updates.
template <typename W, int KIND>
__device__ __forceinline__ void flush_tally(const Args &A, Tally t) {
  __shared__ unsigned long long sacc[6];
  if (threadIdx.x < 6) sacc[threadIdx.x] = 0;
  __syncthreads();
  int64_t v = ld_warp_sum_i64(t.visits), a = ld_warp_sum_i64(t.arcs), m = ld_warp_sum_i64(t.moves);
  i128 q = t.dq;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) q += ld_shfl_xor_i128(q, o);
  if ((threadIdx.x & 31) == 0 && v) {
    atomicAdd(&sacc[0], (unsigned long long)v);
    atomicAdd(&sacc[1], (unsigned long long)a);
    atomicAdd(&sacc[2], (unsigned long long)m);
    ld_atomic_add_i128(&sacc[3], q);
  }
  __syncthreads();
  if (threadIdx.x == 0 && sacc[0]) {
    i128 dq = (i128)(((u128)sacc[4] << 64) | (u128)sacc[3]);
    add_counters(A.cnt, KIND, (int64_t)sacc[0], (int64_t)sacc[1], (int64_t)sacc[2], dq);
    if (KIND == KIND_MOVE) {
      // algorithmic bytes: per visit the list entry, off, deg, C[i], K[i],
      // Sigma[C[i]], size[C[i]] (40 B); per arc col, C[j] and the weight
      add_lmk(A.cnt, KT_WARP, (int64_t)sacc[0], (int64_t)sacc[1], 40 * (int64_t)sacc[0] + (8 + (int64_t)sizeof(W)) * (int64_t)sacc[1]);
    }
  }
}

constexpr int TINY_LANES = 8;  // lanes per vertex of degree <= BIN_TINY_MAX (one arc each)

// Four vertices of degree <= 8 per warp, one arc per lane: lanes whose
// neighbours share a community find each other with __match_any_sync, so
// no table is built; each group's leader lanes hold K_{i->c} and Sigma_c.
template <typename W, int KIND>
__device__ __forceinline__ void tiny_step(const Args &A, int64_t item, int64_t ntiny, int lane, Tally &tl) {
  const W *w = (const W *)A.w;
  int grp = lane >> 3, sub = lane & 7, gl = lane & ~7;
  int64_t k = item * 4 + grp;
  bool has = k < ntiny;
  int32_t i = has ? A.list_tiny[k] : 0;
  int64_t base = 0, Ki = 0, Sd = 0, wj = 0, m2 = A.m2;
  int32_t dg = 0, d = 0, szd = 0, bi = 0, j = -1;
  if (has) {
    base = A.off[i];
    dg = A.deg[i];
    d = A.C[i];
    Ki = A.K[i];
    if (A.gid) m2 = A.m2g[A.gid[i]];
    if (KIND == KIND_REFINE) bi = A.CB[i];
  }
  bool arc = has && sub < dg;
  if (arc) { j = A.col[base + sub]; wj = (int64_t)w[base + sub]; }
  arc = arc && ld_ok((uint64_t)j < (uint64_t)A.n, LD_CHK_COL);
  if (has) {
    Sd = A.S[d];
    if (KIND == KIND_MOVE) szd = A.size[d];
  }
  bool valid = arc && j != i && (KIND != KIND_REFINE || A.CB[j] == bi);
  int32_t c = valid ? A.C[j] : 0;
  valid = valid && ld_ok((uint64_t)c < (uint64_t)A.n, LD_CHK_COMM);
  unsigned long long key = valid ? (((unsigned long long)grp << 32) | (uint32_t)c)
                                 : (0xffffffff00000000ull | (unsigned)lane);
  uint32_t peers = __match_any_sync(LD_FULL, key);
  int64_t kv = 0;  // peers lie within the lane's group of eight
#pragma unroll
  for (int q = 0; q < TINY_LANES; q++) {
    int64_t x = __shfl_sync(LD_FULL, wj, gl + q);
    if ((peers >> (gl + q)) & 1u) kv += x;
  }
  BestX b{0, -1, 0, 0, 0, 0};
  if (valid && ld_group_leader(peers)) {
    if (c == d) {
      b.kd = kv;
    } else {
      b.sc = A.S[c];
      b.v = (i128)m2 * kv - (i128)Ki * b.sc;
      b.c = c;
      b.kc = kv;
    }
  }
  b = bestx_reduce<TINY_LANES>(b);
  i128 g = 0;
  if (has && sub == 0) {
    // the winner's size matters only to the singleton rule (size_d == 1)
    if (KIND == KIND_MOVE && !A.async_mode && b.c > d && szd == 1) b.szc = A.size[b.c];
    g = decide_x<KIND>(A, i, d, Ki, Sd, szd, m2, b);
  }
  bool mv = g > 0;
  if (KIND == KIND_MOVE && !A.async_mode) record_movers(A, mv, i, b.c, g);
  int moved = __shfl_sync(LD_FULL, mv ? 1 : 0, gl);
  if (KIND == KIND_MOVE && moved && arc && j != i && (!A.in_range || A.in_range[j])) ld_bit_set(A.unproc, j);
  if (has && sub == 0) { tl.visits++; tl.arcs += dg; tl.moves += mv; tl.dq += g; }
}

// One vertex of degree 9..128 per warp with a warp-private shared table that
// records its filled slots and is emptied by the reads (so it is cleared
// once per launch, not per vertex).  Every lane keeps its up to four arcs in
// flight: their col, weight and C[j] loads are independent, and so are the
// Sigma loads of the up to four candidates each lane reads back.
constexpr int WARP_UNROLL = BIN_WARP_MAX / 32;

template <typename W, int KIND>
__device__ __forceinline__ void warp_step(const Args &A, int32_t i, int lane, WarpTable &T, Tally &tl) {
  const W *w = (const W *)A.w;
  int64_t base = A.off[i];
  int32_t dg = A.deg[i];
  int32_t d = A.C[i];
  int64_t Ki = A.K[i];
  int64_t Sd = A.S[d];
  int32_t szd = KIND == KIND_MOVE ? A.size[d] : 0;
  int32_t bi = KIND == KIND_REFINE ? A.CB[i] : 0;
  int64_t m2 = m2_of(A, i);
  int32_t j[WARP_UNROLL], c[WARP_UNROLL];
  int64_t wa[WARP_UNROLL];
  bool v[WARP_UNROLL];
#pragma unroll
  for (int u = 0; u < WARP_UNROLL; u++) {
    int a = lane + 32 * u;
    v[u] = a < dg;
    j[u] = v[u] ? A.col[base + a] : i;
    wa[u] = v[u] ? (int64_t)w[base + a] : 0;
  }
#pragma unroll
  for (int u = 0; u < WARP_UNROLL; u++) {
    v[u] = v[u] && j[u] != i && ld_ok((uint64_t)j[u] < (uint64_t)A.n, LD_CHK_COL);
    if (KIND == KIND_REFINE) v[u] = v[u] && A.CB[j[u]] == bi;
  }
#pragma unroll
  for (int u = 0; u < WARP_UNROLL; u++) {
    c[u] = v[u] ? A.C[j[u]] : 0;
    v[u] = v[u] && ld_ok((uint64_t)c[u] < (uint64_t)A.n, LD_CHK_COMM);
  }
#pragma unroll
  for (int u = 0; u < WARP_UNROLL; u++) wt_insert_lanes(T, v[u], c[u], wa[u]);
  int n = T.count;
  int32_t cc[WARP_UNROLL];
  int64_t kv[WARP_UNROLL], sc[WARP_UNROLL];
#pragma unroll
  for (int u = 0; u < WARP_UNROLL; u++) {
    int q = lane + 32 * u;
    cc[u] = -1;
    kv[u] = 0;
    if (q < n) {
      int32_t sl = T.list[q];
      cc[u] = T.keys[sl];
      kv[u] = T.vals[sl];
      T.keys[sl] = LD_EMPTY_KEY;
      T.vals[sl] = 0;
    }
  }
  __syncwarp();
  if (lane == 0) T.count = 0;
  __syncwarp();
#pragma unroll
  for (int u = 0; u < WARP_UNROLL; u++) sc[u] = cc[u] >= 0 && cc[u] != d ? A.S[cc[u]] : 0;
  BestX b{0, -1, 0, 0, 0, 0};
#pragma unroll
  for (int u = 0; u < WARP_UNROLL; u++) {
    if (cc[u] < 0) continue;
    if (cc[u] == d) { b.kd += kv[u]; continue; }
    i128 val = (i128)m2 * kv[u] - (i128)Ki * sc[u];
    if (ld_better(val, cc[u], b.v, b.c)) { b.v = val; b.c = cc[u]; b.kc = kv[u]; b.sc = sc[u]; }
  }
  b = bestx_reduce<32>(b);
  i128 g = 0;
  if (lane == 0) {
    // the winner's size matters only to the singleton rule (size_d == 1)
    if (KIND == KIND_MOVE && !A.async_mode && b.c > d && szd == 1) b.szc = A.size[b.c];
    g = decide_x<KIND>(A, i, d, Ki, Sd, szd, m2, b);
  }
  bool mv = g > 0;
  if (KIND == KIND_MOVE && !A.async_mode) record_movers(A, mv, i, b.c, g);
  int moved = __shfl_sync(LD_FULL, mv ? 1 : 0, 0);
  if (KIND == KIND_MOVE && moved) mark_neighbours(A, i, base, dg, lane, 32);
  if (lane == 0) { tl.visits++; tl.arcs += dg; tl.moves += mv; tl.dq += g; }
}

// Bins 3 (degree <= 8, groups of 8 lanes) and 0 (degree <= 128, a warp
// each) in one launch: items [0, ceil(n3/4)) are groups of four tiny
// vertices, the rest one warp-bin vertex each.
template <typename W, int KIND>
__global__ void __launch_bounds__(WARPS_PER_BLOCK * 32, 4) k_decide_warp(Args A) {
  __shared__ WarpTable WT[WARPS_PER_BLOCK];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  wt_init(WT[wid]);
  int64_t ntiny = *A.count_tiny, nwarp = *A.count;
  int64_t ngroups = (ntiny + 3) / 4, total = ngroups + nwarp;
  int64_t gw = (int64_t)blockIdx.x * WARPS_PER_BLOCK + wid, nw = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  Tally tl;
  for (int64_t t = gw; t < total; t += nw) {
    if (t < ngroups) tiny_step<W, KIND>(A, t, ntiny, lane, tl);
    else warp_step<W, KIND>(A, A.list[t - ngroups], lane, WT[wid], tl);
  }
  flush_tally<W, KIND>(A, tl);
}

// Block-wide merge of per-thread Best values (result valid in thread 0).
__device__ __forceinline__ Best block_best(Best b) {
  __shared__ Best sb[32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  b = warp_best(b);
  if (lane == 0) sb[wid] = b;
  __syncthreads();
  if (wid == 0) {
    Best x = lane < nw ? sb[lane] : Best{0, -1, 0, 0};
    x = warp_best(x);
    if (lane == 0) sb[0] = x;
  }
  __syncthreads();
  Best r = sb[0];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------- bin 1: block, shared stage
// One vertex of degree 129..1024 per block of BLOCK_THREADS.  Each thread
// keeps BLOCK_UNROLL arcs in flight (their col, weight and C[j] loads are
// independent), adds them into a shared open-addressing stage with shared
// atomics, and the block then reads the candidates from the stage's
// filled-slot list (the distinct neighbour communities only), emptying
// each slot as it reads it.
//
// Two barriers per vertex: B1 after the inserts, B2 after the per-warp
// candidates are posted.  The filled-slot count alternates between two
// words by vertex parity: the count of vertex k is read between B1(k) and
// B2(k) and reset by thread 0 after B2(k); it is next used by vertex k+2,
// whose inserts begin after B2(k+1).  The slots read (and emptied) for
// vertex k are all emptied before B2(k), so the inserts of vertex k+1 find
// the stage empty.
constexpr int BLOCK_UNROLL = 4;
struct BlockStage {
  int32_t keys[STAGE_SLOTS];
  int64_t vals[STAGE_SLOTS];
  int32_t list[STAGE_FILL];
  int32_t count[2];
};

__device__ __forceinline__ void bstage_insert(BlockStage &S, int32_t *count, bool valid, int32_t c, int64_t w) {
  if (!valid) return;
  uint32_t s = ld_hash32((uint32_t)c) & (uint32_t)(STAGE_SLOTS - 1);
  for (int probe = 0; ld_ok(probe < STAGE_SLOTS, LD_CHK_PROBE); probe++) {
    int32_t k = S.keys[s];
    if (k == LD_EMPTY_KEY) {
      k = atomicCAS(&S.keys[s], LD_EMPTY_KEY, c);
      if (k == LD_EMPTY_KEY) {
        S.list[atomicAdd(count, 1)] = (int32_t)s;
        k = c;
      }
    }
    if (k == c) {
      atomicAdd((unsigned long long *)&S.vals[s], (unsigned long long)w);
      return;
    }
    s = (s + 1) & (uint32_t)(STAGE_SLOTS - 1);
  }
}

template <typename W, int KIND>
__global__ void __launch_bounds__(BLOCK_THREADS) k_decide_block(Args A) {
  __shared__ BlockStage S;
  __shared__ BestX sb[BLOCK_THREADS / 32];
  __shared__ int moved_s;
  for (int s = threadIdx.x; s < STAGE_SLOTS; s += BLOCK_THREADS) { S.keys[s] = LD_EMPTY_KEY; S.vals[s] = 0; }
  if (threadIdx.x < 2) S.count[threadIdx.x] = 0;
  __syncthreads();
  const W *w = (const W *)A.w;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  int64_t count = *A.count;
  int64_t visits = 0, arcs = 0, moves = 0;
  i128 dq = 0;
  int par = 0;
  for (int64_t t = blockIdx.x; t < count; t += gridDim.x, par ^= 1) {
    int32_t i = A.list[t];
    int64_t base = A.off[i];
    int32_t dg = A.deg[i];
    int32_t d = A.C[i];
    int64_t Ki = A.K[i];
    int64_t Sd = A.S[d];
    int32_t szd = KIND == KIND_MOVE ? A.size[d] : 0;
    int32_t bi = KIND == KIND_REFINE ? A.CB[i] : 0;
    int64_t m2 = m2_of(A, i);
    int32_t *cnt = &S.count[par];
    for (int r0 = 0; r0 < dg; r0 += BLOCK_THREADS * BLOCK_UNROLL) {
      int32_t j[BLOCK_UNROLL], c[BLOCK_UNROLL];
      int64_t wa[BLOCK_UNROLL];
      bool v[BLOCK_UNROLL];
#pragma unroll
      for (int u = 0; u < BLOCK_UNROLL; u++) {
        int a = r0 + u * BLOCK_THREADS + tid;
        v[u] = a < dg;
        j[u] = v[u] ? A.col[base + a] : i;
        wa[u] = v[u] ? (int64_t)w[base + a] : 0;
      }
#pragma unroll
      for (int u = 0; u < BLOCK_UNROLL; u++) {
        v[u] = v[u] && j[u] != i && ld_ok((uint64_t)j[u] < (uint64_t)A.n, LD_CHK_COL);
        if (KIND == KIND_REFINE) v[u] = v[u] && A.CB[j[u]] == bi;
      }
#pragma unroll
      for (int u = 0; u < BLOCK_UNROLL; u++) {
        c[u] = v[u] ? A.C[j[u]] : 0;
        v[u] = v[u] && ld_ok((uint64_t)c[u] < (uint64_t)A.n, LD_CHK_COMM);
      }
#pragma unroll
      for (int u = 0; u < BLOCK_UNROLL; u++) bstage_insert(S, cnt, v[u], c[u], wa[u]);
    }
    __syncthreads();  // B1: the stage holds K_{i->c} for every neighbour community c
    int n = *cnt;
    BestX b{0, -1, 0, 0, 0, 0};
    for (int q0 = 0; q0 < n; q0 += BLOCK_THREADS * BLOCK_UNROLL) {
      int32_t cc[BLOCK_UNROLL];
      int64_t kv[BLOCK_UNROLL], sc[BLOCK_UNROLL];
#pragma unroll
      for (int u = 0; u < BLOCK_UNROLL; u++) {
        int q = q0 + u * BLOCK_THREADS + tid;
        cc[u] = -1;
        kv[u] = 0;
        if (q < n) {
          int32_t sl = S.list[q];
          cc[u] = S.keys[sl];
          kv[u] = S.vals[sl];
          S.keys[sl] = LD_EMPTY_KEY;
          S.vals[sl] = 0;
        }
      }
#pragma unroll
      for (int u = 0; u < BLOCK_UNROLL; u++) sc[u] = cc[u] >= 0 && cc[u] != d ? A.S[cc[u]] : 0;
#pragma unroll
      for (int u = 0; u < BLOCK_UNROLL; u++) {
        if (cc[u] < 0) continue;
        if (cc[u] == d) { b.kd += kv[u]; continue; }
        i128 val = (i128)m2 * kv[u] - (i128)Ki * sc[u];
        if (ld_better(val, cc[u], b.v, b.c)) { b.v = val; b.c = cc[u]; b.kc = kv[u]; b.sc = sc[u]; }
      }
    }
    b = bestx_reduce<32>(b);
    if (lane == 0) sb[wid] = b;
    __syncthreads();  // B2: every warp's best is posted, every read slot emptied
    if (tid == 0) S.count[par] = 0;
    BestX r = sb[0];
#pragma unroll
    for (int k = 1; k < BLOCK_THREADS / 32; k++) bestx_merge(r, sb[k]);
    // the winner's size matters only to the singleton rule (size_d == 1)
    if (KIND == KIND_MOVE && !A.async_mode && r.c > d && szd == 1) r.szc = A.size[r.c];
    bool mv;
    if (A.async_mode) {
      // in-place moves change the totals under the decision: one thread
      // decides and applies, the block learns the outcome
      if (tid == 0) {
        i128 g = decide_x<KIND>(A, i, d, Ki, Sd, szd, m2, r);
        moved_s = g > 0;
        visits++; arcs += dg; moves += g > 0; dq += g;
      }
      __syncthreads();
      mv = moved_s;
    } else {
      // snapshot schedule: the decision reads only the state at the start
      // of the sub-sweep, so every thread reaches the same one; thread 0
      // writes it
      i128 g = 0;
      if (tid == 0) {
        g = decide_x<KIND>(A, i, d, Ki, Sd, szd, m2, r);
        if (KIND == KIND_MOVE && g > 0) {
          int32_t slot = atomicAdd(&A.cnt->movers, 1);
          A.movers[slot] = i;
          A.mtarget[slot] = r.c;
          if (A.mgain) { A.mgain[2 * slot] = (int64_t)(u128)g; A.mgain[2 * slot + 1] = (int64_t)((u128)g >> 64); }
        }
        visits++; arcs += dg; moves += g > 0; dq += g;
      }
      mv = KIND == KIND_MOVE && would_move(d, Ki, Sd, szd, m2, r);
    }
    if (KIND == KIND_MOVE && mv) mark_neighbours(A, i, base, dg, tid, BLOCK_THREADS);
  }
  if (tid == 0) add_counters(A.cnt, KIND, visits, arcs, moves, dq);
  if (KIND == KIND_MOVE && tid == 0)
    add_lmk(A.cnt, KT_BLOCK, visits, arcs, 40 * visits + (8 + (int64_t)sizeof(W)) * arcs);
}

// ---------------------------------------------------------------- bin 2, split across blocks
// Vertices above BIN_BLOCK_MAX arcs: each gets its own table of
// pow2 >= 2*degree slots in global scratch and its arcs are cut into chunks
// of HUGE_CHUNK that any block may take, so one hub no longer runs on one SM.
constexpr int HUGE_CHUNK = TABLE_CHUNK;
constexpr int HUGE_UNROLL = 4;

// Global tables start clean (empty keys, zero values) and are cleaned again
// by the kernel that reads them; each records the slots it fills in a list
// (occ[k] entries at tab_off[k] in A.glist), so the decision visits only the
// distinct communities instead of the whole table.
__global__ void k_huge_zero_occ(const int32_t *count_p, int32_t *occ) {
  for (int64_t k = ld_gtid(); k < *count_p; k += ld_gstride()) occ[k] = 0;
}

// Warp table with 32-bit sums, for 32-bit arc weights: 64-bit shared atomics
// cost more than twice as much, and the smaller table and register footprint
// leave room for more resident warps.  A lane whose add carries the slot past
// 2^32 adds the carry straight into the vertex's global table, so the sums
// stay exact for any weights (a weight below 2^31 carries at most once).
struct WarpTable32 {
  int32_t keys[WT_SLOTS];
  uint32_t vals[WT_SLOTS];
  int32_t list[WT_SLOTS / 2];
  int32_t count;
};

__device__ __forceinline__ void wt_init(WarpTable32 &T) {
  int lane = threadIdx.x & 31;
  for (int s = lane; s < WT_SLOTS; s += 32) { T.keys[s] = LD_EMPTY_KEY; T.vals[s] = 0; }
  if (lane == 0) T.count = 0;
  __syncwarp();
}

__device__ __forceinline__ void wt_insert_lanes(WarpTable32 &T, bool valid, int32_t c, int64_t w, int32_t *gkeys,
                                                int64_t *gvals, int32_t *glist, int32_t *gocc, int gmask) {
  if (valid) {
    uint32_t s = ld_hash32((uint32_t)c) & (uint32_t)(WT_SLOTS - 1);
    for (int probe = 0; ld_ok(probe < WT_SLOTS, LD_CHK_PROBE); probe++) {
      int32_t k = T.keys[s];
      if (k == LD_EMPTY_KEY) {
        k = atomicCAS(&T.keys[s], LD_EMPTY_KEY, c);
        if (k == LD_EMPTY_KEY) {
          T.list[atomicAdd(&T.count, 1)] = (int32_t)s;
          k = c;
        }
      }
      if (k == c) {
        uint32_t add = (uint32_t)w;
        uint32_t old = atomicAdd(&T.vals[s], add);
        if (old + add < old) ld_gtable_insert(gkeys, gvals, glist, gocc, gmask, c, (int64_t)1 << 32);
        break;
      }
      s = (s + 1) & (uint32_t)(WT_SLOTS - 1);
    }
  }
  __syncwarp();
}

__device__ __forceinline__ void wt_flush(WarpTable32 &T, int32_t *gkeys, int64_t *gvals, int32_t *glist, int32_t *gocc,
                                         int gmask) {
  int lane = threadIdx.x & 31;
  __syncwarp();
  int n = T.count;
  for (int q0 = 0; q0 < n; q0 += 32 * GT_KEYS) {  // warp-uniform
    bool has[GT_KEYS];
    int32_t sl[GT_KEYS], key[GT_KEYS];
    int64_t v[GT_KEYS];
#pragma unroll
    for (int u = 0; u < GT_KEYS; u++) {
      int q = q0 + 32 * u + lane;
      has[u] = q < n;
      sl[u] = has[u] ? T.list[q] : 0;
      key[u] = has[u] ? T.keys[sl[u]] : 0;
      v[u] = has[u] ? (int64_t)T.vals[sl[u]] : 0;
    }
    ld_gtable_add_warp(has, false, gkeys, gvals, glist, gocc, gmask, key, v);
#pragma unroll
    for (int u = 0; u < GT_KEYS; u++) {
      if (has[u]) {
        T.keys[sl[u]] = LD_EMPTY_KEY;
        T.vals[sl[u]] = 0;
      }
    }
  }
  __syncwarp();
  if (lane == 0) T.count = 0;
  __syncwarp();
}

template <typename W, int KIND>
__global__ void __launch_bounds__(256) k_huge_scan(Args A, const int64_t *tab_off, const int64_t *ch_off) {
  // Each warp sums its arcs per community in a private shared table first
  // (the neighbours of a hub fall into few communities), then each distinct
  // community updates the vertex's global table once per flush.
  using Table = typename std::conditional<sizeof(W) == 4, WarpTable32, WarpTable>::type;
  __shared__ Table WT[8];
  Table &T8 = WT[threadIdx.x >> 5];
  wt_init(T8);
  int64_t count = *A.count;
  int64_t nch = ch_off[count];
  for (int64_t t = blockIdx.x; t < nch; t += gridDim.x) {
    int64_t lo = 0, hi = count - 1;  // vertex k with ch_off[k] <= t < ch_off[k+1]
    while (lo < hi) {
      int64_t mid = (lo + hi + 1) >> 1;
      if (ch_off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    int64_t i = A.list[lo];
    int64_t first = (t - ch_off[lo]) * HUGE_CHUNK;
    int64_t full = A.deg[i];
    int64_t last = first + HUGE_CHUNK < full ? first + HUGE_CHUNK : full;
    int64_t T = tab_off[lo + 1] - tab_off[lo];
    const W *w = (const W *)A.w;
    int64_t base = A.off[i] + first, len = last - first;
    int32_t bi = KIND == KIND_REFINE ? A.CB[i] : 0;
    int32_t *keys = A.gkeys + tab_off[lo], *list = A.glist + tab_off[lo];
    int64_t *vals = A.gvals + tab_off[lo];
    int lane = threadIdx.x & 31;
    // HUGE_UNROLL arcs per lane in flight: their col, weight and C[j] loads
    // are independent; the inserts follow one by one
    for (int64_t a0 = threadIdx.x & ~31; a0 < len; a0 += (int64_t)blockDim.x * HUGE_UNROLL) {  // warp-uniform
      int32_t j[HUGE_UNROLL], c[HUGE_UNROLL];
      int64_t wa[HUGE_UNROLL];
      bool valid[HUGE_UNROLL];
#pragma unroll
      for (int u = 0; u < HUGE_UNROLL; u++) {
        int64_t a = a0 + (int64_t)u * blockDim.x + lane;
        valid[u] = a < len;
        j[u] = valid[u] ? A.col[base + a] : (int32_t)i;
        wa[u] = valid[u] ? (int64_t)w[base + a] : 0;
      }
#pragma unroll
      for (int u = 0; u < HUGE_UNROLL; u++) {
        valid[u] = valid[u] && j[u] != i && ld_ok((uint64_t)j[u] < (uint64_t)A.n, LD_CHK_COL);
        if (KIND == KIND_REFINE) valid[u] = valid[u] && A.CB[j[u]] == bi;
      }
#pragma unroll
      for (int u = 0; u < HUGE_UNROLL; u++) {
        c[u] = valid[u] ? A.C[j[u]] : 0;
        valid[u] = valid[u] && ld_ok((uint64_t)c[u] < (uint64_t)A.n, LD_CHK_COMM);
      }
#pragma unroll
      for (int u = 0; u < HUGE_UNROLL; u++) {
        if (T8.count > WT_LIMIT) wt_flush(T8, keys, vals, list, &A.gocc[lo], (int)(T - 1));
        if constexpr (sizeof(W) == 4)
          wt_insert_lanes(T8, valid[u], c[u], wa[u], keys, vals, list, &A.gocc[lo], (int)(T - 1));
        else wt_insert_lanes(T8, valid[u], c[u], wa[u]);
      }
    }
    wt_flush(T8, keys, vals, list, &A.gocc[lo], (int)(T - 1));
    if (KIND == KIND_MOVE && threadIdx.x == 0)
      add_lmk(A.cnt, KT_HUGE_SCAN, first == 0 ? 1 : 0, len, (8 + (int64_t)sizeof(W)) * len);
  }
}

template <int KIND>
__global__ void __launch_bounds__(HUGE_THREADS) k_huge_decide(Args A, const int64_t *tab_off) {
  __shared__ int moved_s;
  int64_t count = *A.count;
  int64_t visits = 0, arcs = 0, moves = 0;
  i128 dq = 0;
  for (int64_t k = blockIdx.x; k < count; k += gridDim.x) {
    int64_t i = A.list[k];
    int64_t base = A.off[i], dg = A.deg[i];
    int32_t *keys = A.gkeys + tab_off[k], *list = A.glist + tab_off[k];
    int64_t *vals = A.gvals + tab_off[k];
    int32_t occ = A.gocc[k];
    int32_t d = A.C[i];
    int64_t m2 = m2_of(A, i), Ki = A.K[i];
    Best b{0, -1, 0, 0};
    for (int32_t t = threadIdx.x; t < occ; t += blockDim.x) {
      int32_t s = list[t];
      int32_t c = keys[s];
      int64_t kv = vals[s];
      if (c == d) { b.kd += kv; continue; }
      i128 v = (i128)m2 * kv - (i128)Ki * A.S[c];
      if (ld_better(v, c, b.v, b.c)) { b.v = v; b.c = c; b.kc = kv; }
    }
    b = block_best(b);
    for (int32_t t = threadIdx.x; t < occ; t += blockDim.x) {  // leave the table clean
      int32_t s = list[t];
      keys[s] = LD_EMPTY_KEY;
      vals[s] = 0;
    }
    if (threadIdx.x == 0) {
      i128 g = decide_leader<KIND>(A, i, b);
      moved_s = g > 0;
      visits++; arcs += dg; moves += g > 0; dq += g;
    }
    __syncthreads();
    if (KIND == KIND_MOVE && moved_s) mark_neighbours(A, i, base, dg, threadIdx.x, blockDim.x);
    __syncthreads();
  }
  if (threadIdx.x == 0) add_counters(A.cnt, KIND, visits, arcs, moves, dq);
}

// ---------------------------------------------------------------- collection
// Take the unprocessed vertices of class `cls` (clearing their bits) and
// append the in-range ones to the degree bins.
__global__ void k_collect(int64_t n, uint32_t *unproc, int cls, int classes_mask, const uint8_t *in_range,
                          const int32_t *deg, int32_t *bins, DevCounters *cnt, const int32_t *gid,
                          const uint8_t *lm_on, const int64_t *loff, leiden_tuning tn) {
  // Each lane reads one bitmap word and sorts its set bits into per-bin
  // masks; a warp scan over the lanes' counts then places every vertex, so
  // a warp appends the vertices of its 32 words in id order with one atomic
  // per bin, however sparse the frontier is.  The bits taken are cleared
  // with one write per word (each word belongs to one lane here).
  int lane = threadIdx.x & 31;
  int64_t nwords = (n + 31) >> 5;
  int64_t warp = ld_gtid() >> 5, nwarps = ld_gstride() >> 5;
  for (int64_t w0 = warp * 32; w0 < nwords; w0 += nwarps * 32) {  // warp-uniform
    int64_t wi = w0 + lane;
    uint32_t word = wi < nwords ? unproc[wi] : 0u, rest = word, taken = 0u;
    uint32_t bm[NBINS];
#pragma unroll
    for (int b = 0; b < NBINS; b++) bm[b] = 0u;
    while (rest) {
      int bit = __ffs(rest) - 1;
      rest &= rest - 1u;
      int64_t v = (wi << 5) + bit;
      if (v >= n) break;
      // batched handles: the class of a vertex is taken on its id within
      // its graph, and graphs whose iterations ended are skipped
      int64_t vl = gid ? v - loff[gid[v]] : v;
      if (ld_class_of(vl, classes_mask) != cls || (gid && !lm_on[gid[v]])) continue;
      taken |= 1u << bit;
      if (in_range && !in_range[v]) continue;
      // a vertex without arcs has no candidate community: taking it is its visit
      int dg = deg[v];
      if (dg == 0) continue;
      int bin = dg <= tn.tiny_max ? BIN_TINY : dg <= tn.warp_max ? BIN_WARP : dg <= tn.block_max ? BIN_BLOCK : BIN_HUGE;
#pragma unroll
      for (int b = 0; b < NBINS; b++)
        if (bin == b) bm[b] |= 1u << bit;
    }
#pragma unroll
    for (int b = 0; b < NBINS; b++) {
      int k = __popc(bm[b]), incl = k;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(LD_FULL, incl, o);
        if (lane >= o) incl += y;
      }
      int total = __shfl_sync(LD_FULL, incl, 31);
      if (total == 0) continue;  // warp-uniform
      int32_t pos0 = 0;
      if (lane == 31) pos0 = atomicAdd(&cnt->bin_count[b], total);
      pos0 = __shfl_sync(LD_FULL, pos0, 31) + incl - k;
      int32_t *dst = bins + (int64_t)b * n + pos0;
      for (uint32_t m = bm[b]; m; m &= m - 1u) *dst++ = (int32_t)((wi << 5) + __ffs(m) - 1);
    }
    if (taken) unproc[wi] = word & ~taken;
  }
}

// Deferred moves of a sub-sweep (deterministic mode).
// Batched handles also sum the gains and moves per graph (gid non-null).
__global__ void k_apply_moves(const int32_t *movers, const int32_t *target, const DevCounters *cnt_c, int32_t *C,
                              int64_t *S, const int64_t *K, int32_t *size, const int32_t *gid, const int64_t *mgain,
                              unsigned long long *dqg, int64_t *movesg) {
  int64_t m = cnt_c->movers;
  for (int64_t t0 = (ld_gtid() & ~31ll); t0 < m; t0 += ld_gstride()) {  // warp-uniform trip count
    int64_t t = t0 + (threadIdx.x & 31);
    bool has = t < m;
    int32_t i = 0, gi = 0;
    i128 gain = 0;
    if (has) {
      i = movers[t];
      int32_t c = target[t];
      int32_t d = C[i];
      C[i] = c;
      atomicAdd((unsigned long long *)&S[d], (unsigned long long)(-K[i]));
      atomicAdd((unsigned long long *)&S[c], (unsigned long long)K[i]);
      atomicSub(&size[d], 1);
      atomicAdd(&size[c], 1);
      if (gid) {
        gi = gid[i];
        gain = (i128)(((u128)(uint64_t)mgain[2 * t + 1] << 64) | (u128)(uint64_t)mgain[2 * t]);
      }
    }
    if (gid) {
      ld_graph_add_i128(dqg, has, gi, gain);
      ld_graph_add_i64(movesg, has, gi, 1);
    }
  }
}

// Community sizes; lanes with the same community add once (giant
// communities would otherwise serialise on one counter).
__global__ void k_sizes(const int32_t *C, int64_t n, int32_t *size) {
  int lane = threadIdx.x & 31;
  for (int64_t base = (ld_gtid() & ~31ll); base < n; base += ld_gstride()) {
    int64_t i = base + lane;
    int32_t c = i < n ? C[i] : -1 - lane;
    uint32_t peers = __match_any_sync(LD_FULL, c);
    if (i < n && ld_group_leader(peers)) atomicAdd(&size[c], __popc(peers));
  }
}

// ---- refinement
// Reset the vertices of refined bounds to singletons and list them.
__global__ void k_refine_reset(int64_t n, const int32_t *CB, const uint8_t *dR, int32_t *C, int64_t *S,
                               const int64_t *K, int32_t *prop, int32_t *cand, DevCounters *cnt, const int32_t *gid,
                               uint8_t *refg) {
  int lane = threadIdx.x & 31;
  for (int64_t base = (ld_gtid() & ~31ll); base < n; base += ld_gstride()) {
    int64_t i = base + lane;
    bool r = i < n && dR[CB[i]];
    if (i < n) prop[i] = r ? 0 : -1;
    if (r) { C[i] = (int32_t)i; S[i] = K[i]; }
    if (r && gid) refg[gid[i]] = 1;  // the graph has a vertex in a refined bound
    uint32_t m = __ballot_sync(LD_FULL, r);
    if (!m) continue;
    int32_t p0 = 0;
    if (lane == 0) p0 = atomicAdd(&cnt->cand_count[0], __popc(m));
    p0 = __shfl_sync(LD_FULL, p0, 0);
    if (r) cand[p0 + __popc(m & ((1u << lane) - 1u))] = (int32_t)i;
  }
}

// Keep the candidates that are still alone in their community and bin them
// by degree; reset their proposals.
__global__ void k_refine_collect(const int32_t *cand_in, const int32_t *count_in, int32_t *cand_out,
                                 int32_t *count_out, int64_t n, const int32_t *C, const int64_t *S, const int64_t *K,
                                 const int32_t *deg, int32_t *prop, int32_t *bins, DevCounters *cnt, leiden_tuning tn) {
  int lane = threadIdx.x & 31;
  int64_t m = *count_in;
  for (int64_t base = (ld_gtid() & ~31ll); base < m; base += ld_gstride()) {
    int64_t t = base + lane;
    int32_t i = t < m ? cand_in[t] : -1;
    bool keep = false;
    if (i >= 0) {
      prop[i] = -1;
      keep = S[C[i]] == K[i];
    }
    int bin = -1;
    if (keep) {
      int dg = deg[i];  // without arcs: no proposal (prop stays -1)
      bin = dg == 0 ? -1 : dg <= tn.tiny_max ? BIN_TINY : dg <= tn.warp_max ? BIN_WARP : dg <= tn.block_max ? BIN_BLOCK : BIN_HUGE;
    }
    uint32_t km = __ballot_sync(LD_FULL, keep);
    if (km) {
      int32_t p0 = 0;
      if (lane == __ffs(km) - 1) p0 = atomicAdd(count_out, __popc(km));
      p0 = __shfl_sync(LD_FULL, p0, __ffs(km) - 1);
      if (keep) cand_out[p0 + __popc(km & ((1u << lane) - 1u))] = i;
    }
#pragma unroll
    for (int b = 0; b < NBINS; b++) {
      uint32_t mm = __ballot_sync(LD_FULL, bin == b);
      if (!mm) continue;
      int32_t q0 = 0;
      if (lane == __ffs(mm) - 1) q0 = atomicAdd(&cnt->bin_count[b], __popc(mm));
      q0 = __shfl_sync(LD_FULL, q0, __ffs(mm) - 1);
      if (bin == b) bins[(int64_t)b * n + q0 + __popc(mm & ((1u << lane) - 1u))] = i;
    }
  }
}

// Snapshot rounds: i -> c* applies iff i does not hold and c* holds, where
// v holds when it proposed nothing, or when v and prop[v] chose each other
// and v has the smaller id.
__device__ __forceinline__ bool holds(const int32_t *prop, int32_t v) {
  int32_t t = prop[v];
  return t < 0 || (prop[t] == v && v < t);
}
__global__ void k_refine_accept(const int32_t *cand, const int32_t *count, const int32_t *prop, int32_t *C, int64_t *S,
                                const int64_t *K, DevCounters *cnt, const int32_t *gid, int32_t *accg) {
  int64_t m = *count;
  int32_t acc = 0;
  for (int64_t t0 = (ld_gtid() & ~31ll); t0 < m; t0 += ld_gstride()) {  // warp-uniform trip count
    int64_t t = t0 + (threadIdx.x & 31);
    bool took = false;
    int32_t i = 0;
    if (t < m) {
      i = cand[t];
      int32_t c = prop[i];
      if (c >= 0 && !holds(prop, i) && holds(prop, c)) {
        int32_t d = C[i];
        C[i] = c;
        atomicAdd((unsigned long long *)&S[d], (unsigned long long)(-K[i]));
        atomicAdd((unsigned long long *)&S[c], (unsigned long long)K[i]);
        acc++;
        took = true;
      }
    }
    if (gid) ld_graph_add_i32(accg, took, took ? gid[i] : 0, 1);
  }
  if (acc) atomicAdd(&cnt->accepted, acc);
}

__global__ void k_check_selftest() {
  if (threadIdx.x == 0) ld_ok(false, LD_CHK_SELFTEST);
}

Args make_args(leiden_handle *h, const LevelGraph &g) {
  Args A{};
  A.n = g.n;
  A.off = g.off;
  A.deg = g.deg;
  A.col = g.col;
  A.w = g.w;
  A.C = h->Cp;
  A.S = h->Sp;
  A.K = h->Kp;
  A.size = h->csize;
  A.CB = h->CB;
  A.prop = h->prop;
  A.dS = h->dS;
  A.unproc = h->unproc;
  A.movers = h->movers;
  A.mtarget = h->mtarget;
  A.cnt = h->dcnt;
  A.m2 = h->m2;
  if (g.gid) {
    A.gid = g.gid;
    A.m2g = h->gc.m2;
    A.mgain = h->mgain;
    A.accg = h->gc.accepted;
    A.refg = h->gc.refined;
  }
  A.async_mode = h->p.deterministic ? 0 : 1;
  A.classes_mask = lm_classes(h) - 1;
  return A;
}

// The block-bin kernels ask for the largest shared-memory carveout, so that
// seven 29 KB stages fit on an SM (set once per device of the process).
void block_kernel_carveout() {
  static std::atomic<uint64_t> done{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) { cudaGetLastError(); return; }
  if (done.load(std::memory_order_relaxed) & (1ull << dev)) return;
  int co = cudaSharedmemCarveoutMaxShared;
  cudaFuncSetAttribute(k_decide_block<int32_t, KIND_MOVE>, cudaFuncAttributePreferredSharedMemoryCarveout, co);
  cudaFuncSetAttribute(k_decide_block<int64_t, KIND_MOVE>, cudaFuncAttributePreferredSharedMemoryCarveout, co);
  cudaFuncSetAttribute(k_decide_block<int32_t, KIND_REFINE>, cudaFuncAttributePreferredSharedMemoryCarveout, co);
  cudaFuncSetAttribute(k_decide_block<int64_t, KIND_REFINE>, cudaFuncAttributePreferredSharedMemoryCarveout, co);
  cudaGetLastError();
  done.fetch_or(1ull << dev, std::memory_order_relaxed);
}

// The bins of one sub-sweep (or refinement round) read the same state and
// write disjoint outputs (deferred moves through one atomic counter,
// frontier bits through atomics), so the block bin and the hub path run on
// the handle's side streams beside the warp bin, joined before the caller
// launches anything else: each of these kernels is bound by the latency of
// its gathers and leaves most of the GPU idle in its tail.
template <int KIND>
void launch_bins(leiden_handle *h, const LevelGraph &g, Args A) {
  cudaStream_t s = h->stream;
  int sms = h->sm_count;
  bool need_block = g.maxdeg > h->tune.warp_max, need_hub = g.maxdeg > h->tune.block_max;
  // tables for every listed hub at once: at most huge_slots slots (taken
  // before the fork: growing them synchronises and frees)
  if (need_hub && !ensure_hslots(h, g.huge_slots)) {
    h->fatal = LEIDEN_ERR_OOM;
    h->err = "global table scratch";
    return;
  }
  // (the in-place mode keeps the bins in order: there a bin's moves are
  // seen by the bins launched after it)
  bool fork = h->tune.overlap && h->p.deterministic && (need_block || need_hub) && side_streams(h);
  cudaStream_t sblock = s, shub = s;
  if (fork) {
    cudaEventRecord(h->fork_ev, s);
    if (need_block) { sblock = h->side[0]; cudaStreamWaitEvent(sblock, h->fork_ev, 0); }
    if (need_hub) { shub = h->side[1]; cudaStreamWaitEvent(shub, h->fork_ev, 0); }
  }
  A.list_tiny = h->bins + (int64_t)BIN_TINY * g.n;
  A.count_tiny = &h->dcnt->bin_count[BIN_TINY];
  for (int b = 0; b < NBINS; b++) {
    A.list = h->bins + (int64_t)b * g.n;
    A.count = &h->dcnt->bin_count[b];
    if (b == BIN_TINY) continue;  // with the warp bin
    if (b == BIN_HUGE && g.maxdeg <= h->tune.block_max) continue;
    if (b == BIN_BLOCK && g.maxdeg <= h->tune.warp_max) continue;
    if (b == BIN_WARP) {
      int grid = sms * h->tune.warp_blocks_per_sm;  // default 4: one wave at four resident blocks per SM
      if (KIND == KIND_MOVE) kt_begin(h, KT_WARP);
      if (g.w64) ld_note_launch(), k_decide_warp<int64_t, KIND><<<grid, WARPS_PER_BLOCK * 32, 0, s>>>(A);
      else ld_note_launch(), k_decide_warp<int32_t, KIND><<<grid, WARPS_PER_BLOCK * 32, 0, s>>>(A);
      if (KIND == KIND_MOVE) kt_end(h);
    } else if (b == BIN_BLOCK) {
      // default 7 blocks per SM: the shared stage (29 KB) and 71 registers
      // for 128 threads admit 7, with the carveout set to favour shared memory
      block_kernel_carveout();
      int grid = sms * h->tune.block_blocks_per_sm;
      if (KIND == KIND_MOVE) kt_begin(h, KT_BLOCK, sblock);
      if (g.w64) ld_note_launch(), k_decide_block<int64_t, KIND><<<grid, BLOCK_THREADS, 0, sblock>>>(A);
      else ld_note_launch(), k_decide_block<int32_t, KIND><<<grid, BLOCK_THREADS, 0, sblock>>>(A);
      if (KIND == KIND_MOVE) kt_end(h, sblock);
    } else {
      A.gkeys = hs_keys(h);
      A.gvals = hs_vals(h);
      A.glist = hs_list(h);
      A.gocc = h->hocc;
      int64_t *tab_off = h->lbuf2, *ch_off = h->lbuf3;
      launch_table_plan(A.list, A.count, g.deg, nullptr, g.n, tab_off, ch_off, shub);  // keys: communities of the level
      ld_note_launch(), k_huge_zero_occ<<<sms, 256, 0, shub>>>(A.count, A.gocc);
      if (KIND == KIND_MOVE) kt_begin(h, KT_HUGE_SCAN, shub);
      int hg = sms * h->tune.hub_blocks_per_sm;
      if (g.w64) ld_note_launch(), k_huge_scan<int64_t, KIND><<<hg, 256, 0, shub>>>(A, tab_off, ch_off);
      else ld_note_launch(), k_huge_scan<int32_t, KIND><<<hg, 256, 0, shub>>>(A, tab_off, ch_off);
      if (KIND == KIND_MOVE) kt_end(h, shub);
      ld_note_launch(), k_huge_decide<KIND><<<sms * 8, HUGE_THREADS, 0, shub>>>(A, tab_off);
    }
  }
  if (fork) {
    for (int k = 0; k < 2; k++) {
      if ((k == 0 && !need_block) || (k == 1 && !need_hub)) continue;
      cudaEventRecord(h->join_ev[k], h->side[k]);
      cudaStreamWaitEvent(s, h->join_ev[k], 0);
    }
  }
}

}  // namespace

// The side streams and events of a handle, created on first use; false
// (and the bins stay on the handle's stream) if they cannot be had.
bool side_streams(leiden_handle *h) {
  if (h->side[1]) return true;
  if (h->side_failed) return false;
  bool ok = cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; k < 2 && ok; k++)
    ok = cudaStreamCreateWithFlags(&h->side[k], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&h->join_ev[k], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    for (int k = 0; k < 2; k++) {
      if (h->side[k]) cudaStreamDestroy(h->side[k]);
      if (h->join_ev[k]) cudaEventDestroy(h->join_ev[k]);
      h->side[k] = nullptr;
      h->join_ev[k] = nullptr;
    }
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    h->fork_ev = nullptr;
    h->side_failed = true;
  }
  return ok;
}

// Global table scratch of `slots` slots laid out as keys int32[S] | values
// int64[S] | slot lists int32[S] (16 B per slot).  Every user leaves the
// slots it touched empty again, so a new allocation is cleared once.
bool ensure_hslots(leiden_handle *h, int64_t slots) {
  if (slots <= h->hslots) return true;
  int64_t S = (slots + 1023) & ~(int64_t)1023;
  if (h->hscratch) {
    cudaStreamSynchronize(h->stream);
    for (auto &q : h->owned)
      if (q == h->hscratch) { cudaFree(q); q = nullptr; }
  }
  void *p = nullptr;
  if (cudaMalloc(&p, (size_t)S * 16) != cudaSuccess) {
    cudaGetLastError();
    h->hscratch = nullptr;
    h->hscratch_bytes = 0;
    h->hslots = 0;
    return false;
  }
  h->owned.push_back(p);
  h->hscratch = p;
  h->hscratch_bytes = (size_t)S * 16;
  h->hslots = S;
  cudaMemsetAsync(p, 0xff, (size_t)S * 4, h->stream);                   // keys: empty
  cudaMemsetAsync((char *)p + (size_t)S * 4, 0, (size_t)S * 8, h->stream);  // values: 0
  return true;
}

int32_t *hs_keys(leiden_handle *h) { return (int32_t *)h->hscratch; }
int64_t *hs_vals(leiden_handle *h) { return (int64_t *)((char *)h->hscratch + (size_t)h->hslots * 4); }
int32_t *hs_list(leiden_handle *h) { return (int32_t *)((char *)h->hscratch + (size_t)h->hslots * 12); }

void lm_prepare(leiden_handle *h, const LevelGraph &g, int sizes_from) {
  if (sizes_from == SIZES_ONES) {  // C' is the identity: every community is one vertex
    launch_fill_i32(h->csize, 1, g.n, h->stream);
  } else if (sizes_from == SIZES_KEPT) {  // C' = C^{t-1}: sizes kept by the last tracking
    cudaMemcpyAsync(h->csize, h->csize0, (size_t)g.n * sizeof(int32_t), cudaMemcpyDeviceToDevice, h->stream);
  } else {
    cudaMemsetAsync(h->csize, 0, (size_t)g.n * sizeof(int32_t), h->stream);
    ld_note_launch(), k_sizes<<<grid_for(g.n, 256), 256, 0, h->stream>>>(h->Cp, g.n, h->csize);
  }
}

void count_sizes(leiden_handle *h, const int32_t *C, int64_t n, int32_t *size) {
  cudaMemsetAsync(size, 0, (size_t)n * sizeof(int32_t), h->stream);
  ld_note_launch(), k_sizes<<<grid_for(n, 256), 256, 0, h->stream>>>(C, n, size);
}

void lm_subsweep(leiden_handle *h, const LevelGraph &g, int cls, const uint8_t *in_range, int dynamic) {
  cudaStream_t s = h->stream;
  cudaMemsetAsync(&h->dcnt->bin_count[0], 0, sizeof(int32_t) * 4 + sizeof(int32_t), s);  // bins + movers
  ld_note_launch(), k_collect<<<grid_for((g.n + 31) / 32, 256), 256, 0, s>>>(
      g.n, h->unproc, cls, lm_classes(h) - 1, in_range, g.deg, h->bins, h->dcnt, g.gid, h->gc.lm_on, h->d_loff,
      h->tune);
  Args A = make_args(h, g);
  A.in_range = in_range;
  A.dynamic = dynamic;
  launch_bins<KIND_MOVE>(h, g, A);
  if (h->p.deterministic)
    ld_note_launch(), k_apply_moves<<<h->sm_count * 4, 256, 0, s>>>(h->movers, h->mtarget, h->dcnt, h->Cp, h->Sp, h->Kp,
                                                                    h->csize, g.gid, h->mgain, h->gc.dq, h->gc.moves);
}

void refine_reset(leiden_handle *h, const LevelGraph &g) {
  cudaStream_t s = h->stream;
  cudaMemsetAsync(&h->dcnt->cand_count[0], 0, sizeof(int32_t), s);
  ld_note_launch(), k_refine_reset<<<grid_for(g.n, 256), 256, 0, s>>>(g.n, h->CB, h->dR, h->Cp, h->Sp, h->Kp, h->prop, h->cand,
                                                    h->dcnt, g.gid, h->gc.refined);
}

// One round on the candidates of list `slot` (cand + slot*n, count
// cand_count[slot]); the ones still alone go to the other list.
void refine_round(leiden_handle *h, const LevelGraph &g, int slot) {
  cudaStream_t s = h->stream;
  int32_t *in = h->cand + (int64_t)slot * g.n, *out = h->cand + (int64_t)(1 - slot) * g.n;
  int32_t *cin = &h->dcnt->cand_count[slot], *cout = &h->dcnt->cand_count[1 - slot];
  cudaMemsetAsync(&h->dcnt->bin_count[0], 0, sizeof(int32_t) * 4, s);
  cudaMemsetAsync(cout, 0, sizeof(int32_t), s);
  cudaMemsetAsync(&h->dcnt->accepted, 0, sizeof(int32_t), s);
  ld_note_launch(), k_refine_collect<<<grid_for(g.n, 256), 256, 0, s>>>(in, cin, out, cout, g.n, h->Cp, h->Sp, h->Kp, g.deg, h->prop,
                                                      h->bins, h->dcnt, h->tune);
  Args A = make_args(h, g);
  launch_bins<KIND_REFINE>(h, g, A);
  ld_note_launch(), k_refine_accept<<<h->sm_count * 4, 256, 0, s>>>(out, cout, h->prop, h->Cp, h->Sp, h->Kp, h->dcnt,
                                                                     g.gid, h->gc.accepted);
}

LD_CHECK_WORD_READER(check_word_move)

unsigned int check_selftest(cudaStream_t s) {
  ld_note_launch(), k_check_selftest<<<1, 32, 0, s>>>();
  cudaStreamSynchronize(s);
  return check_word_move();
}
