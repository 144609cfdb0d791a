// Device-side helpers shared by the kernels of the GB300 dynamic Leiden
// library.  Internal header: not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

typedef __int128 i128;
typedef unsigned __int128 u128;

#define LD_WARP 32
#define LD_FULL 0xffffffffu
#define LD_EMPTY_KEY (-1)

// ---------------------------------------------------------------- counters
// One block of device counters per handle, mirrored to pinned host memory at
// the few host synchronisation points of a call.
struct DevCounters {
  unsigned long long dq[2];       // sum of accepted gains g (int128, two's complement)
  int32_t bin_count[4];           // vertices in each degree bin of the current sub-sweep
  int32_t movers;                 // deferred moves of the current sub-sweep (SYNC)
  int32_t accepted;               // refinement moves applied in this round
  int32_t cand_count[2];          // refinement candidate lists (ping-pong)
  int32_t refined_any;            // a vertex lies in a refined bound
  int32_t error;                  // batch validation error (first offending arc + 1)
  int32_t overflow;               // a touched CSR row outgrew its capacity
  int32_t list_count;             // generic list length
  int32_t ncomm;                  // communities after dense renumbering
  int32_t split_count;            // vertices in communities to split
  int32_t max_count;              // max degree (level), max community degree
  int64_t processed;              // local-moving vertex visits
  int64_t arcs;                   // local-moving arcs scanned
  int64_t moves;                  // local-moving moves
  int64_t ref_processed;          // refinement vertex visits
  int64_t ref_arcs;               // refinement arcs scanned
  int64_t lmk_visits[3];          // local moving per timed kernel (warp range, block bin, hub scan):
  int64_t lmk_arcs[3];            //   vertex visits, arcs scanned and algorithmic bytes
  int64_t lmk_bytes[3];
  int64_t m2;                     // 2m (sum of arc weights), device copy
  int64_t sigma_intra;            // modularity: intra-community arc weight
  unsigned long long sq[2];       // modularity: sum of Sigma_c^2 (int128)
  int64_t batch_dw;               // batch: change of 2m
  int64_t huge_slots;             // table slots the vertices above the block bin need
  int32_t big_count;              // splitting: long rows left to the block kernel
  int32_t large_count;            // batch apply: touched rows merged in chunks
  int32_t tr_occ;                 // tracking: filled slots of the pair table
  int32_t mid_count;              // batch apply: touched rows merged by one block each
  int64_t arena_used;             // next free arc slot of G^t (relocated rows go here)
  int64_t bcounts[8];             // batch apply: unique deletions, unique insertions, new arcs,
                                  //   touched rows, merge-buffer arcs
  int32_t pass_ncomm[10];         // communities after refinement, per pass (trace)
  int64_t affected;               // |dV|: vertices flagged affected (counted into the frontier)
  int64_t split_arcs;             // splitting: arcs of the vertices listed for splitting
  int64_t deg_sum;                // degree sum of the level scanned by level_maxdeg (its arcs)
  int64_t xk_bytes[3];            // algorithmic bytes of the other timed kernels (split sampling,
                                  //   giant-community aggregation scan, block merge of touched rows)
  int64_t agg_tables[2];          // aggregation's per-community global tables: [0] hashed, [1] indexed
                                  //   by the key (the table has a slot per community)
};

// ---------------------------------------------------------------- checked build
// Built with -DLEIDEN_CHECKED, the kernels test conditions the algorithm
// guarantees -- an open-addressing probe ends within its table, neighbour and
// community ids lie in [0, n), a union-find chain is shorter than n -- and
// where one fails they record its code in a device word of their source
// file, skip the access and go on.  A broken invariant then ends the call
// with LEIDEN_ERR_STATE instead of a fault, a trap or an endless loop.  The
// default build compiles every test away (ld_ok is then always true).
enum { LD_CHK_PROBE = 1, LD_CHK_COL = 2, LD_CHK_COMM = 3, LD_CHK_CHAIN = 4, LD_CHK_SELFTEST = 0x5e1f };
#ifdef LEIDEN_CHECKED
static __device__ unsigned int ld_check_word;
__device__ __forceinline__ bool ld_ok(bool cond, unsigned int code) {
  if (!cond) atomicCAS(&ld_check_word, 0u, code);
  return cond;
}
// Host: the file's check word (after a stream sync), reset to 0.
#define LD_CHECK_WORD_READER(fn)                                      \
  unsigned int fn() {                                                 \
    unsigned int v = 0, z = 0;                                        \
    if (cudaMemcpyFromSymbol(&v, ld_check_word, sizeof(v)) != cudaSuccess) { cudaGetLastError(); return 0; } \
    cudaMemcpyToSymbol(ld_check_word, &z, sizeof(z));                 \
    return v;                                                         \
  }
#else
__device__ __forceinline__ bool ld_ok(bool, unsigned int) { return true; }
#define LD_CHECK_WORD_READER(fn) \
  unsigned int fn() { return 0; }
#endif

// ---------------------------------------------------------------- hashing
// SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014).
__host__ __device__ __forceinline__ uint64_t ld_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Sub-sweep class of a vertex in the snapshot schedule.
__device__ __forceinline__ int ld_class_of(int64_t v, int classes_mask) {
  return (int)(ld_splitmix64((uint64_t)v) & (uint64_t)classes_mask);
}

// Multiplicative hash of a community id into a power-of-two table.
__device__ __forceinline__ uint32_t ld_hash32(uint32_t k) {
  k *= 0x9E3779B1u;
  return k ^ (k >> 15);
}

// ---------------------------------------------------------------- int128
__device__ __forceinline__ void ld_atomic_add_i128(unsigned long long *p, i128 v) {
  unsigned long long lo = (unsigned long long)(u128)v;
  unsigned long long hi = (unsigned long long)((u128)v >> 64);
  if (lo == 0 && hi == 0) return;
  unsigned long long old = atomicAdd(&p[0], lo);
  unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
  if (hi + carry) atomicAdd(&p[1], hi + carry);
}

__device__ __forceinline__ i128 ld_shfl_xor_i128(i128 v, int mask) {
  long long lo = (long long)(unsigned long long)(u128)v;
  long long hi = (long long)((u128)v >> 64);
  lo = __shfl_xor_sync(LD_FULL, lo, mask);
  hi = __shfl_xor_sync(LD_FULL, hi, mask);
  return (i128)(((u128)(unsigned long long)hi << 64) | (u128)(unsigned long long)lo);
}

// Candidate (value, community) ordered by larger value, then smaller id.
// c < 0 means "no candidate".
__device__ __forceinline__ bool ld_better(i128 v1, int32_t c1, i128 v2, int32_t c2) {
  if (c1 < 0) return false;
  if (c2 < 0) return true;
  return v1 > v2 || (v1 == v2 && c1 < c2);
}

__device__ __forceinline__ int64_t ld_warp_sum_i64(int64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(LD_FULL, v, o);
  return v;
}

// Sum over the lanes that share a key (peers = __match_any_sync of the
// key).  Every lane of the warp must call it (full-mask shuffles); each
// lane receives its group's sum.  (The warp reduction unit, __reduce_add_sync
// with one mask per group, measured about twice as slow here: it serialises
// over the distinct masks of a warp.)
__device__ __forceinline__ int64_t ld_group_sum_i64(uint32_t peers, int64_t v) {
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < 32; k++) {
    int64_t x = __shfl_sync(LD_FULL, v, k);
    if ((peers >> k) & 1u) s += x;
  }
  return s;
}
// True in the lowest lane of the group.
__device__ __forceinline__ bool ld_group_leader(uint32_t peers) {
  return (__ffs(peers) - 1) == (int)(threadIdx.x & 31);
}

// Open-addressing insert into a global table (linear probing, key -1 =
// empty) that records each slot it fills in `list` (count in *occ), so the
// reader visits only filled slots and can empty them again afterwards.
__device__ __forceinline__ void ld_gtable_insert(int32_t *keys, int64_t *vals, int32_t *list, int32_t *occ, int tmask,
                                                 int32_t c, int64_t w) {
  // A slot's key only goes from empty to a key while a table is in use, so
  // a plain read from L2 decides every probe but the claim of an empty slot:
  // a key already in the table costs a load and an add whose result is not
  // waited for, instead of a compare-and-swap on a slot every warp touches.
  uint32_t s = ld_hash32((uint32_t)c) & (uint32_t)tmask;
  for (uint32_t probe = 0; ld_ok(probe <= (uint32_t)tmask, LD_CHK_PROBE); probe++) {
    int32_t k = __ldcg(&keys[s]);
    if (k == LD_EMPTY_KEY) {
      k = atomicCAS(&keys[s], LD_EMPTY_KEY, c);
      if (k == LD_EMPTY_KEY) {
        list[atomicAdd(occ, 1)] = (int32_t)s;
        k = c;
      }
    }
    if (k == c) {
      atomicAdd((unsigned long long *)&vals[s], (unsigned long long)w);
      return;
    }
    s = (s + 1) & (uint32_t)tmask;
  }
}

// The same for a table with a slot per key (slot = key): the key array
// only marks the slots already listed.
__device__ __forceinline__ void ld_gtable_add_direct(int32_t *keys, int64_t *vals, int32_t *list, int32_t *occ,
                                                     int32_t c, int64_t w) {
  if (__ldcg(&keys[c]) == LD_EMPTY_KEY && atomicCAS(&keys[c], LD_EMPTY_KEY, c) == LD_EMPTY_KEY)
    list[atomicAdd(occ, 1)] = c;
  atomicAdd((unsigned long long *)&vals[c], (unsigned long long)w);
}

// All 32 lanes, each with up to GT_KEYS keys (has[u]): add them to a global
// table (`direct`: slot = key; otherwise open addressing as above).  A key's
// slot is read first and claimed only when empty; the weight add is not
// waited for; a collision probes on.  The slots claimed by the warp are
// listed with one atomic on the fill count, which every warp flushing into
// the same table would otherwise hit once per new key.  GT_KEYS is 1: with
// more keys per lane in flight the loops' registers cost the hub scan more
// occupancy than the overlapped reads gained.
constexpr int GT_KEYS = 1;
__device__ __forceinline__ void ld_gtable_add_warp(const bool *has, bool direct, int32_t *keys, int64_t *vals,
                                                   int32_t *list, int32_t *occ, int tmask, const int32_t *c,
                                                   const int64_t *w) {
  int lane = threadIdx.x & 31;
  uint32_t s[GT_KEYS];
  int32_t k[GT_KEYS], claimed[GT_KEYS];
#pragma unroll
  for (int u = 0; u < GT_KEYS; u++) {
    s[u] = direct ? (uint32_t)c[u] : ld_hash32((uint32_t)c[u]) & (uint32_t)tmask;
    k[u] = has[u] ? __ldcg(&keys[s[u]]) : c[u];
    claimed[u] = -1;
  }
#pragma unroll
  for (int u = 0; u < GT_KEYS; u++) {
    if (has[u] && k[u] == LD_EMPTY_KEY) {
      k[u] = atomicCAS(&keys[s[u]], LD_EMPTY_KEY, c[u]);
      if (k[u] == LD_EMPTY_KEY) {
        claimed[u] = (int32_t)s[u];
        k[u] = c[u];
      }
    }
  }
  int mine = 0;
#pragma unroll
  for (int u = 0; u < GT_KEYS; u++) {
    if (!has[u]) continue;
    // a collision (hash tables only: a direct slot holds its own key or none)
    for (uint32_t probe = 1; k[u] != c[u] && ld_ok(probe <= (uint32_t)tmask, LD_CHK_PROBE); probe++) {
      s[u] = (s[u] + 1) & (uint32_t)tmask;
      k[u] = __ldcg(&keys[s[u]]);
      if (k[u] == LD_EMPTY_KEY) {
        k[u] = atomicCAS(&keys[s[u]], LD_EMPTY_KEY, c[u]);
        if (k[u] == LD_EMPTY_KEY) {
          claimed[u] = (int32_t)s[u];
          k[u] = c[u];
        }
      }
    }
    if (k[u] == c[u]) atomicAdd((unsigned long long *)&vals[s[u]], (unsigned long long)w[u]);
    mine += claimed[u] >= 0;
  }
  int incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(LD_FULL, incl, o);
    if (lane >= o) incl += y;
  }
  int total = __shfl_sync(LD_FULL, incl, 31);
  if (total == 0) return;  // warp-uniform
  int32_t base = 0;
  if (lane == 31) base = atomicAdd(occ, total);
  base = __shfl_sync(LD_FULL, base, 31) + incl - mine;
#pragma unroll
  for (int u = 0; u < GT_KEYS; u++)
    if (claimed[u] >= 0) list[base++] = claimed[u];
}

// Shared staging table of one block (local moving and refinement of the
// block bin): STAGE_SLOTS open-addressing slots, at most STAGE_FILL keys.
constexpr int STAGE_SLOTS = 2048;
constexpr int STAGE_FILL = 1024;  // distinct keys per use at most (load <= 1/2)

// Warp-private shared table: only the lanes of one warp touch it, so the
// only contention on a slot is between lanes with the same key.  Flushed
// into a global table before it passes half full.
constexpr int WT_SLOTS = 256;
constexpr int WT_LIMIT = WT_SLOTS / 2 - 32;  // flush above this many keys
struct WarpTable {
  int32_t keys[WT_SLOTS];
  int64_t vals[WT_SLOTS];
  int32_t list[WT_SLOTS / 2];
  int32_t count;
};

__device__ __forceinline__ void wt_init(WarpTable &T) {
  int lane = threadIdx.x & 31;
  for (int s = lane; s < WT_SLOTS; s += 32) { T.keys[s] = LD_EMPTY_KEY; T.vals[s] = 0; }
  if (lane == 0) T.count = 0;
  __syncwarp();
}

// All 32 lanes call it; each lane with a pair adds it on its own with a
// shared-memory atomic (lanes of one warp only, so the only contention is
// between lanes with the same key, which the atomic unit serialises) -- no
// key grouping and no shuffles.
__device__ __forceinline__ void wt_insert_lanes(WarpTable &T, bool valid, int32_t c, int64_t w) {
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
        atomicAdd((unsigned long long *)&T.vals[s], (unsigned long long)w);
        break;
      }
      s = (s + 1) & (uint32_t)(WT_SLOTS - 1);
    }
  }
  __syncwarp();
}

// All 32 lanes: move the pairs into a global table and empty the warp table.
__device__ __forceinline__ void wt_flush_to(WarpTable &T, bool direct, int32_t *gkeys, int64_t *gvals,
                                            int32_t *glist, int32_t *gocc, int gmask) {
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
      v[u] = has[u] ? T.vals[sl[u]] : 0;
    }
    ld_gtable_add_warp(has, direct, gkeys, gvals, glist, gocc, gmask, key, v);
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

__device__ __forceinline__ void wt_flush(WarpTable &T, int32_t *gkeys, int64_t *gvals, int32_t *glist, int32_t *gocc,
                                         int gmask) {
  wt_flush_to(T, false, gkeys, gvals, glist, gocc, gmask);
}

// All 32 lanes: move the pairs into a directly indexed table (slot = key,
// for keys below the table's size) and empty the warp table.
__device__ __forceinline__ void wt_flush_dense(WarpTable &T, int32_t *gkeys, int64_t *gvals, int32_t *glist,
                                               int32_t *gocc) {
  wt_flush_to(T, true, gkeys, gvals, glist, gocc, 0);
}

// Per-graph sums of a batched handle: every lane of the warp calls these;
// lanes with `has` add v into arr[g].  When the whole warp is on one graph
// (the common case: lists follow vertex order) one lane adds the warp's sum.
__device__ __forceinline__ void ld_graph_add_i64(int64_t *arr, bool has, int32_t g, int64_t v) {
  int32_t g0 = __shfl_sync(LD_FULL, has ? g : -1, __ffs(__ballot_sync(LD_FULL, has) | 0x80000000u) - 1);
  if (__all_sync(LD_FULL, !has || g == g0)) {
    int64_t s = has ? v : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(LD_FULL, s, o);
    if ((threadIdx.x & 31) == 0 && g0 >= 0 && s) atomicAdd((unsigned long long *)&arr[g0], (unsigned long long)s);
  } else if (has && v) {
    atomicAdd((unsigned long long *)&arr[g], (unsigned long long)v);
  }
}
__device__ __forceinline__ void ld_graph_add_i32(int32_t *arr, bool has, int32_t g, int32_t v) {
  int32_t g0 = __shfl_sync(LD_FULL, has ? g : -1, __ffs(__ballot_sync(LD_FULL, has) | 0x80000000u) - 1);
  if (__all_sync(LD_FULL, !has || g == g0)) {
    int32_t s = has ? v : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(LD_FULL, s, o);
    if ((threadIdx.x & 31) == 0 && g0 >= 0 && s) atomicAdd(&arr[g0], s);
  } else if (has && v) {
    atomicAdd(&arr[g], v);
  }
}
__device__ __forceinline__ void ld_graph_add_i128(unsigned long long *arr, bool has, int32_t g, i128 v) {
  int32_t g0 = __shfl_sync(LD_FULL, has ? g : -1, __ffs(__ballot_sync(LD_FULL, has) | 0x80000000u) - 1);
  if (__all_sync(LD_FULL, !has || g == g0)) {
    i128 s = has ? v : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += ld_shfl_xor_i128(s, o);
    if ((threadIdx.x & 31) == 0 && g0 >= 0 && s != 0) ld_atomic_add_i128(&arr[2 * g0], s);
  } else if (has && v != 0) {
    ld_atomic_add_i128(&arr[2 * g], v);
  }
}

// ---------------------------------------------------------------- bitmaps
__device__ __forceinline__ bool ld_bit_test(const uint32_t *bm, int64_t i) {
  return (bm[i >> 5] >> (i & 31)) & 1u;
}
// Sets bit i; returns true if it was clear.
__device__ __forceinline__ bool ld_bit_set(uint32_t *bm, int64_t i) {
  uint32_t m = 1u << (i & 31);
  return (atomicOr(&bm[i >> 5], m) & m) == 0;
}

// Weight load for level 0 (int32) and aggregated levels (int64).
template <typename W>
__device__ __forceinline__ int64_t ld_w(const W *w, int64_t a) {
  return (int64_t)w[a];
}

// Grid-stride helpers.
__device__ __forceinline__ int64_t ld_gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t ld_gstride() { return (int64_t)gridDim.x * blockDim.x; }
