// Per-pass phases between local moving and the next pass: subset
// renumbering (Alg. "leidensr"), splitting (Alg. "leidensp"), dense
// renumbering with dendrogram lookup (Alg. "leiden"), aggregation (Alg.
// "leidenag").
#include <algorithm>
#include <climits>

#include "internal.h"

namespace {

constexpr int TB = 256;

// ---------------------------------------------------------------- Alg. leidensr
__global__ void k_sr_init(int64_t n, int32_t *rep, int64_t *S2, uint8_t *dS2, uint8_t *dR2) {
  for (int64_t c = ld_gtid(); c < n; c += ld_gstride()) { rep[c] = INT_MAX; S2[c] = 0; dS2[c] = 0; dR2[c] = 0; }
}
// rep[c] = smallest member; a vertex only competes while it is below the
// value already there (a plain read first spares most atomics).
__global__ void k_sr_min(int64_t n, const int32_t *C, int32_t *rep) {
  for (int64_t i = ld_gtid(); i < n; i += ld_gstride()) {
    int32_t c = C[i];
    if ((int32_t)i < rep[c]) atomicMin(&rep[c], (int32_t)i);
  }
}
__global__ void k_sr_rekey(int64_t n, const int32_t *rep, const int64_t *S, const uint8_t *dS, const uint8_t *dR,
                           int64_t *S2, uint8_t *dS2, uint8_t *dR2) {
  for (int64_t c = ld_gtid(); c < n; c += ld_gstride()) {
    int32_t r = rep[c];
    if (r == INT_MAX) continue;
    S2[r] = S[c]; dS2[r] = dS[c]; dR2[r] = dR[c];
  }
}
__global__ void k_sr_remap(int64_t n, const int32_t *rep, int32_t *C) {
  for (int64_t i = ld_gtid(); i < n; i += ld_gstride()) C[i] = rep[C[i]];
}

// ---------------------------------------------------------------- Alg. leidensp
// Components of the flagged communities by lock-free union-find: a root is
// only ever hooked under a smaller root, so every component ends with its
// smallest vertex as root -- the label a BFS from the lowest vertex gives.
__global__ void k_split_init(int64_t n, const int32_t *C, const uint8_t *dS, const uint8_t *dR, const int32_t *deg,
                             int32_t *parent, int32_t *list, DevCounters *cnt, int split_all) {
  int lane = threadIdx.x & 31;
  int64_t arcs = 0;  // arcs of the listed vertices (work counter)
  for (int64_t base = (ld_gtid() & ~31ll); base < n; base += ld_gstride()) {
    int64_t i = base + lane;
    bool f = false;
    if (i < n) {
      int32_t c = C[i];
      f = (split_all || dS[c]) && !dR[c];
      if (f) { parent[i] = (int32_t)i; arcs += deg[i]; }
    }
    uint32_t m = __ballot_sync(LD_FULL, f);
    if (!m) continue;
    int32_t p0 = 0;
    if (lane == 0) p0 = atomicAdd(&cnt->split_count, __popc(m));
    p0 = __shfl_sync(LD_FULL, p0, 0);
    if (f) list[p0 + __popc(m & ((1u << lane) - 1u))] = (int32_t)i;
  }
  arcs = ld_warp_sum_i64(arcs);
  if (lane == 0 && arcs) atomicAdd((unsigned long long *)&cnt->split_arcs, (unsigned long long)arcs);
}

__device__ __forceinline__ int32_t uf_find(int32_t *parent, int32_t x) {
  while (true) {
    int32_t p = parent[x];
    if (p == x) return x;
    int32_t gp = parent[p];
    if (gp != p) parent[x] = gp;  // path halving (parents only decrease)
    x = p;
  }
}

__device__ __forceinline__ void uf_unite(int32_t *parent, int32_t a, int32_t b) {
  while (true) {
    a = uf_find(parent, a);
    b = uf_find(parent, b);
    if (a == b) return;
    if (a < b) { int32_t t = a; a = b; b = t; }
    if (atomicCAS(&parent[a], a, b) == a) return;
  }
}

// Sampling round (Afforest, Sutton et al. 2018): link each listed vertex to
// its first SPLIT_SAMPLES neighbours in the same community.  Which
// neighbours are sampled never changes the result (the link round that
// follows makes the components exact); sampling only joins most of a
// community's vertices to one tree cheaply.
constexpr int SPLIT_SAMPLES = 2;
constexpr int SPLIT_SAMPLE_SCAN = 64;
constexpr int SPLIT_LANES = 4;  // lanes per vertex; each reads two arcs of a window of eight
// Four lanes per vertex (eight vertices per warp) read its row prefix eight
// arcs at a time, two per lane with independent loads, and the lanes
// holding the first SPLIT_SAMPLES same-community neighbours link.
__global__ void k_split_sample(const int32_t *list, DevCounters *cnt, const int64_t *off, const int32_t *deg,
                               const int32_t *col, const int32_t *C, int32_t *parent) {
  int64_t m = cnt->split_count;
  int lane = threadIdx.x & 31, grp = lane / SPLIT_LANES, sub = lane % SPLIT_LANES;
  constexpr int GROUPS = 32 / SPLIT_LANES;
  uint32_t gmask = ((1u << SPLIT_LANES) - 1u) << (grp * SPLIT_LANES);
  int64_t ngroups = (ld_gstride() >> 5) * GROUPS;
  int64_t bytes = 0;  // algorithmic bytes (lane 0 of each group)
  for (int64_t t0 = (ld_gtid() >> 5) * GROUPS; t0 < m; t0 += ngroups) {  // warp-uniform trip count
    int64_t t = t0 + grp;
    bool has = t < m;
    int32_t i = 0, c = 0;
    int64_t b = 0, d = 0;
    if (has) {
      i = list[t];
      c = C[i];
      b = off[i];
      d = deg[i];
      if (d > SPLIT_SAMPLE_SCAN) d = SPLIT_SAMPLE_SCAN;  // sampling looks at a short prefix only
    }
    int got = 0;
    for (int64_t a0 = 0; a0 < SPLIT_SAMPLE_SCAN; a0 += 2 * SPLIT_LANES) {
      bool live = has && got < SPLIT_SAMPLES && a0 < d;
      if (!__any_sync(LD_FULL, live)) break;
      // arcs a0 + sub and a0 + SPLIT_LANES + sub: loads first, then the C gathers
      int64_t x0 = a0 + sub, x1 = a0 + SPLIT_LANES + sub;
      int32_t j0 = live && x0 < d ? col[b + x0] : -1;
      int32_t j1 = live && x1 < d ? col[b + x1] : -1;
      bool h0 = j0 >= 0 && j0 != i && C[j0] == c;
      bool h1 = j1 >= 0 && j1 != i && C[j1] == c;
      // arc order: the first half of the window (lanes' j0), then the second
      uint32_t hits0 = __ballot_sync(LD_FULL, h0) & gmask, hits1 = __ballot_sync(LD_FULL, h1) & gmask;
      uint32_t below = (1u << lane) - 1u;
      int need = SPLIT_SAMPLES - got;
      int r0 = __popc(hits0 & below), r1 = __popc(hits0) + __popc(hits1 & below);
      if (h0 && r0 < need) uf_unite(parent, i, j0);
      if (h1 && r1 < need) uf_unite(parent, i, j1);
      if (live) {
        got += __popc(hits0) + __popc(hits1);
        if (sub == 0) bytes += 8 * (d - a0 < 2 * SPLIT_LANES ? d - a0 : 2 * SPLIT_LANES);  // col and C of the arcs read
      }
    }
    if (has && sub == 0) bytes += 20;  // list entry, C, offset, degree
  }
  bytes = ld_warp_sum_i64(bytes);
  if (lane == 0 && bytes) atomicAdd((unsigned long long *)&cnt->xk_bytes[0], (unsigned long long)bytes);
}

__global__ void k_split_flatten(const int32_t *list, const DevCounters *cnt, int32_t *parent) {
  int64_t m = cnt->split_count;
  for (int64_t t = ld_gtid(); t < m; t += ld_gstride()) {
    int32_t i = list[t];
    parent[i] = uf_find(parent, i);
  }
}

// Warp per listed vertex.  The community id C[i] is its smallest member,
// which is always the root of its own component; a vertex already joined to
// it skips its arcs, every other vertex links along all of its arcs.  An edge
// with an endpoint outside that component is therefore always processed
// from that endpoint, so the final components are exact.
constexpr int SPLIT_BIG = 2048;  // longer rows go to the block kernel
__global__ void k_split_link_rest(const int32_t *list, DevCounters *cnt, const int64_t *off, const int32_t *deg,
                                  const int32_t *col, const int32_t *C, int32_t *parent, int32_t *big) {
  int lane = threadIdx.x & 31;
  int64_t m = cnt->split_count;
  // 32 listed vertices per warp: the root lookups run a lane each, then the
  // warp scans the arcs of the vertices that are not joined yet, one by one
  for (int64_t base = (ld_gtid() & ~31ll); base < m; base += ld_gstride()) {
    int64_t t = base + lane;
    int32_t i = 0, c = 0;
    bool need = false;
    if (t < m) {
      i = list[t];
      c = C[i];
      need = uf_find(parent, i) != c;
    }
    uint32_t todo = __ballot_sync(LD_FULL, need);
    while (todo) {
      int src = __ffs(todo) - 1;
      todo &= todo - 1;
      int32_t vi = __shfl_sync(LD_FULL, i, src), vc = __shfl_sync(LD_FULL, c, src);
      int64_t b = off[vi], d = deg[vi];
      if (d > SPLIT_BIG) {
        if (lane == 0) big[atomicAdd(&cnt->big_count, 1)] = vi;
        continue;
      }
      for (int64_t a = lane; a < d; a += 32) {
        int32_t j = col[b + a];
        if (j != vi && C[j] == vc) uf_unite(parent, vi, j);
      }
    }
  }
}

__global__ void __launch_bounds__(1024) k_split_link_big(const int32_t *big, const DevCounters *cnt,
                                                        const int64_t *off, const int32_t *deg, const int32_t *col,
                                                        const int32_t *C, int32_t *parent) {
  int64_t m = cnt->big_count;
  for (int64_t t = blockIdx.x; t < m; t += gridDim.x) {
    int32_t i = big[t];
    int32_t c = C[i];
    int64_t b = off[i], d = deg[i];
    for (int64_t a = threadIdx.x; a < d; a += blockDim.x) {
      int32_t j = col[b + a];
      if (j != i && C[j] == c) uf_unite(parent, i, j);
    }
  }
}

__global__ void k_split_compress(const int32_t *list, const DevCounters *cnt, int32_t *parent, int32_t *C) {
  int64_t m = cnt->split_count;
  for (int64_t t = ld_gtid(); t < m; t += ld_gstride()) {
    int32_t i = list[t];
    C[i] = uf_find(parent, i);
  }
}

// ---------------------------------------------------------------- renumber / lookup
// Batched handles (gid non-null): only the graphs that continue to the next
// pass are renumbered; the others are mapped to one spare id past the dense
// range (rank[n]), which aggregation leaves out.
__global__ void k_used(int64_t n, const int32_t *C, int32_t *used, const int32_t *gid, const uint8_t *cont) {
  for (int64_t i = ld_gtid(); i < n; i += ld_gstride())
    if (!gid || cont[gid[i]]) used[C[i]] = 1;
}
__global__ void k_rank(int64_t n, const int64_t *rank, int32_t *C, const int32_t *gid, const uint8_t *cont) {
  for (int64_t i = ld_gtid(); i < n; i += ld_gstride())
    C[i] = (int32_t)((!gid || cont[gid[i]]) ? rank[C[i]] : rank[n]);
}
__global__ void k_lookup(int64_t N, const int32_t *Cp, int32_t *Ctop, const int32_t *gid0, const uint8_t *cont) {
  for (int64_t v = ld_gtid(); v < N; v += ld_gstride())
    if (!gid0 || cont[gid0[v]]) Ctop[v] = Cp[Ctop[v]];
}
// Final lookup of the graphs that stop at this pass, with the community id
// moved from the level's range of the graph into its own vertex range (the
// order within the graph, all that tracking uses, is kept).
__global__ void k_break_lookup(int64_t N, const int32_t *Cp, int32_t *Ctop, const int32_t *gid0, const uint8_t *cont,
                               const int64_t *loff, const int64_t *voff) {
  for (int64_t v = ld_gtid(); v < N; v += ld_gstride()) {
    int32_t g = gid0[v];
    if (loff[g + 1] > loff[g] && !cont[g]) Ctop[v] = (int32_t)(Cp[Ctop[v]] - loff[g] + voff[g]);
  }
}
// Graph of each super-vertex and the graphs' ranges at the next level.
__global__ void k_level_ids(int64_t n, const int32_t *Cdense, const int32_t *gid, const uint8_t *cont,
                            int32_t *gid_next) {
  for (int64_t i = ld_gtid(); i < n; i += ld_gstride())
    if (cont[gid[i]]) gid_next[Cdense[i]] = gid[i];
}
__global__ void k_level_off(int G, const int64_t *loff, const int64_t *rank, int64_t *loff_next) {
  for (int64_t g = ld_gtid(); g <= G; g += ld_gstride()) loff_next[g] = rank[loff[g]];
}
// After refinement every community id is one of its members and that
// member keeps its own id (subset renumbering gives the smallest member,
// splitting the smallest vertex of a component, refinement a stationary
// representative), so the communities are the vertices with C[i] == i.
__global__ void k_count_roots(int64_t n, const int32_t *C, DevCounters *cnt, const int32_t *gid, int32_t *ncg) {
  int32_t local = 0;
  for (int64_t b = (ld_gtid() & ~31ll); b < n; b += ld_gstride()) {  // warp-uniform trip count
    int64_t i = b + (threadIdx.x & 31);
    bool root = i < n && C[i] == (int32_t)i;
    local += root;
    if (gid) ld_graph_add_i32(ncg, root, root ? gid[i] : 0, 1);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(LD_FULL, local, o);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(&cnt->list_count, local);
}

// ---------------------------------------------------------------- Alg. leidenag
// Members per community.  Lanes of a warp in one community are counted
// with one atomic; a block then sums its warps' counts in a small shared
// table before the global counters: a giant community has members in every
// warp, and one atomic per warp on its counter would serialise on one word.
// A community whose table slot another community holds goes straight to
// the global counter.
constexpr int MEMBER_SLOTS = 256;

__device__ __forceinline__ int32_t member_claim(int32_t *hk, int32_t c) {
  int s = (int)(ld_hash32((uint32_t)c) & (MEMBER_SLOTS - 1));
  int32_t k = hk[s];
  if (k == -1) {
    int32_t old = atomicCAS(&hk[s], -1, c);
    k = old == -1 ? c : old;
  }
  return k == c ? s : -1;
}

__global__ void __launch_bounds__(256) k_member_count(int64_t n, const int32_t *C, int32_t *cnt_c) {
  __shared__ int32_t hk[MEMBER_SLOTS], hv[MEMBER_SLOTS];
  for (int s = threadIdx.x; s < MEMBER_SLOTS; s += blockDim.x) { hk[s] = -1; hv[s] = 0; }
  __syncthreads();
  int lane = threadIdx.x & 31;
  for (int64_t base = (ld_gtid() & ~31ll); base < n; base += ld_gstride()) {
    int64_t i = base + lane;
    int32_t c = i < n ? C[i] : -1 - lane;
    uint32_t peers = __match_any_sync(LD_FULL, c);
    if (i < n && ld_group_leader(peers)) {
      int s = member_claim(hk, c);
      if (s >= 0) atomicAdd(&hv[s], __popc(peers));
      else atomicAdd(&cnt_c[c], __popc(peers));
    }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < MEMBER_SLOTS; s += blockDim.x)
    if (hk[s] != -1) atomicAdd(&cnt_c[hk[s]], hv[s]);
}

// cursor[c] starts at coff[c]; each member takes the next slot of its
// community (the order of members within a community does not matter
// downstream).  As in the count, a block first counts its members of the
// communities that hold a shared slot, takes their ranges with one atomic
// each, then places them from shared cursors; the others take their slots
// from the global cursor, one atomic per group of lanes.  Both sweeps of a
// block visit the same vertices.
__global__ void __launch_bounds__(256) k_member_fill(int64_t n, const int32_t *C, unsigned long long *cursor,
                                                     int32_t *cverts) {
  __shared__ int32_t hk[MEMBER_SLOTS], hv[MEMBER_SLOTS];
  __shared__ unsigned long long hb[MEMBER_SLOTS];
  for (int s = threadIdx.x; s < MEMBER_SLOTS; s += blockDim.x) { hk[s] = -1; hv[s] = 0; }
  __syncthreads();
  int lane = threadIdx.x & 31;
  for (int64_t base = (ld_gtid() & ~31ll); base < n; base += ld_gstride()) {  // warp-uniform trip count
    int64_t i = base + lane;
    int32_t c = i < n ? C[i] : -1 - lane;
    uint32_t peers = __match_any_sync(LD_FULL, c);
    if (i < n && ld_group_leader(peers)) {
      int s = member_claim(hk, c);
      if (s >= 0) atomicAdd(&hv[s], __popc(peers));
    }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < MEMBER_SLOTS; s += blockDim.x) {
    if (hk[s] != -1) hb[s] = atomicAdd(&cursor[hk[s]], (unsigned long long)hv[s]);
    hv[s] = 0;
  }
  __syncthreads();
  for (int64_t base = (ld_gtid() & ~31ll); base < n; base += ld_gstride()) {  // warp-uniform trip count
    int64_t i = base + lane;
    int32_t c = i < n ? C[i] : -1 - lane;
    uint32_t peers = __match_any_sync(LD_FULL, c);
    int leader = __ffs(peers) - 1;
    unsigned long long p0 = 0;
    if (i < n && lane == leader) {
      int s = (int)(ld_hash32((uint32_t)c) & (MEMBER_SLOTS - 1));
      if (hk[s] == c) p0 = hb[s] + (unsigned long long)atomicAdd(&hv[s], __popc(peers));
      else p0 = atomicAdd(&cursor[c], (unsigned long long)__popc(peers));
    }
    p0 = __shfl_sync(LD_FULL, p0, leader);
    if (i < n) cverts[(int64_t)p0 + __popc(peers & ((1u << lane) - 1u))] = (int32_t)i;
  }
}
__global__ void k_member_deg(int64_t n, const int32_t *cverts, const int32_t *deg, int32_t *mdeg) {
  for (int64_t t = ld_gtid(); t < n; t += ld_gstride()) mdeg[t] = deg[cverts[t]];
}
// super-row offsets: yoff[c] = flat offset of the community's first member
__global__ void k_yoff(int64_t ncomm, const int64_t *coff, const int64_t *cflat, int64_t *yoff, DevCounters *cnt) {
  for (int64_t c = ld_gtid(); c <= ncomm; c += ld_gstride()) {
    yoff[c] = cflat[coff[c]];
    if (c < ncomm) {
      int64_t d = cflat[coff[c + 1]] - cflat[coff[c]];
      atomicMax(&cnt->max_count, (int32_t)(d < INT_MAX ? d : INT_MAX));
      if (d > BIN_BLOCK_MAX) {  // table slots of the chunked path (at most ncomm distinct keys)
        int64_t keys = d < ncomm ? d : ncomm;
        int64_t t = 1;
        while (t < 2 * keys) t <<= 1;
        atomicAdd((unsigned long long *)&cnt->huge_slots, (unsigned long long)t);
      }
    }
  }
}

__device__ __forceinline__ void agg_insert(int32_t *keys, int64_t *vals, int tmask, int32_t c, int64_t w) {
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

struct AggArgs {
  int64_t ncomm;
  const int64_t *off;
  const int32_t *deg;
  const int32_t *col;
  const void *w;
  const int32_t *C;
  const int64_t *coff;
  const int32_t *cverts;
  const int64_t *cflat;
  const int64_t *yoff;
  int32_t *ydeg;
  int32_t *ycol;
  int64_t *yw;
  int64_t *Kout;
  const int32_t *list;
  const int32_t *count;
  int32_t *gkeys;
  int64_t *gvals;
  int32_t *glist;  // filled slots of each listed community's table
  int32_t *gocc;   // number of filled slots
  int64_t *xk_bytes;  // algorithmic bytes of the chunked scan
  int64_t *tables;    // [0] hashed and [1] directly indexed global tables emitted
};

// The members of a community are staged in batches (flat start, and row
// offset minus flat start), so that each thread finds the member of its
// flat arc by a search among the staged members and the arcs are spread
// evenly over the threads whatever the members' degrees.
constexpr int AGG_MB = 256;
constexpr int AGG_UNROLL = 4;

// The member k of a staged batch whose arcs hold flat arc f, given
// ms[0] <= f < ms[nb]: the last k with ms[k] <= f (members without arcs
// share their start with the next one and are passed over).
__device__ __forceinline__ int agg_member_of(const int64_t *ms, int nb, int64_t f) {
  int lo = 0, hi = nb - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (ms[mid] <= f) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int GROUP>
// Emit the table as the super-row of c and leave every slot empty again.
__device__ __forceinline__ void agg_emit(const AggArgs &A, int64_t c, int t0, int stride, int32_t *keys,
                                         int64_t *vals, int T, int32_t *rowcount, int64_t *rowsum) {
  int64_t base = A.yoff[c];
  for (int s = t0; s < T; s += stride) {
    int32_t k = keys[s];
    if (k == LD_EMPTY_KEY) continue;
    int64_t v = vals[s];
    keys[s] = LD_EMPTY_KEY;
    vals[s] = 0;
    int32_t p = atomicAdd(rowcount, 1);
    A.ycol[base + p] = k;
    A.yw[base + p] = v;
    atomicAdd((unsigned long long *)rowsum, (unsigned long long)v);
  }
}

constexpr int AGG_WARPS = 8;
constexpr int AGG_WARP_TABLE = 256;
constexpr int AGG_BLOCK_TABLE = 2048;

// Communities of at most BIN_WARP_MAX flat arcs, a warp each: the warp
// holds 32 members at a time in registers (lane i the i-th), and a lane
// finds the member of its flat arc with five shuffles.
template <typename W>
__global__ void __launch_bounds__(AGG_WARPS * 32) k_agg_warp(AggArgs A) {
  __shared__ int32_t skeys[AGG_WARPS][AGG_WARP_TABLE];
  __shared__ int64_t svals[AGG_WARPS][AGG_WARP_TABLE];
  __shared__ int32_t scount[AGG_WARPS];
  __shared__ int64_t ssum[AGG_WARPS];
  const W *w = (const W *)A.w;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t count = *A.count;
  for (int64_t t = (int64_t)blockIdx.x * AGG_WARPS + wid; t < count; t += (int64_t)gridDim.x * AGG_WARPS) {
    int64_t c = A.list[t];
    int64_t dg = A.yoff[c + 1] - A.yoff[c];
    int T = 32;
    while (T < 2 * dg) T <<= 1;
    for (int s = lane; s < T; s += 32) { skeys[wid][s] = LD_EMPTY_KEY; svals[wid][s] = 0; }
    if (lane == 0) { scount[wid] = 0; ssum[wid] = 0; }
    __syncwarp();
    int64_t m0 = A.coff[c], m1 = A.coff[c + 1];
    int64_t selfw = 0;  // arcs inside the community: summed in registers, added once
    for (int64_t ab = m0; ab < m1; ab += 32) {  // warp-uniform
      int nb = m1 - ab < 32 ? (int)(m1 - ab) : 32;
      int64_t s = 0, r = 0;
      if (lane < nb) {
        s = A.cflat[ab + lane];
        r = A.off[A.cverts[ab + lane]] - s;
      }
      int64_t bs = __shfl_sync(LD_FULL, s, 0), be = A.cflat[ab + nb];
      for (int64_t R = bs; R < be; R += 32 * AGG_UNROLL) {  // warp-uniform
        int32_t j[AGG_UNROLL];
        int64_t wa[AGG_UNROLL];
        bool valid[AGG_UNROLL];
#pragma unroll
        for (int u = 0; u < AGG_UNROLL; u++) {
          int64_t f = R + u * 32 + lane;
          valid[u] = f < be;
          int k = 0;  // last staged member with start <= f (all lanes shuffle)
#pragma unroll
          for (int step = 16; step > 0; step >>= 1) {
            int cand = k + step;
            int64_t sc = __shfl_sync(LD_FULL, s, cand & 31);
            if (cand < nb && sc <= f) k = cand;
          }
          int64_t row = __shfl_sync(LD_FULL, r, k) + f;
          j[u] = valid[u] ? A.col[row] : 0;
          wa[u] = valid[u] ? (int64_t)w[row] : 0;
        }
        int32_t cj[AGG_UNROLL];  // the C gathers of all of them in flight together
#pragma unroll
        for (int u = 0; u < AGG_UNROLL; u++) cj[u] = valid[u] ? A.C[j[u]] : -1;
#pragma unroll
        for (int u = 0; u < AGG_UNROLL; u++) {
          if (cj[u] == (int32_t)c) selfw += wa[u];
          else if (valid[u]) agg_insert(skeys[wid], svals[wid], T - 1, cj[u], wa[u]);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) selfw += __shfl_xor_sync(LD_FULL, selfw, o);
    if (lane == 0 && selfw) agg_insert(skeys[wid], svals[wid], T - 1, (int32_t)c, selfw);
    __syncwarp();
    agg_emit<32>(A, c, lane, 32, skeys[wid], svals[wid], T, &scount[wid], &ssum[wid]);
    __syncwarp();
    if (lane == 0) { A.ydeg[c] = scount[wid]; A.Kout[c] = ssum[wid]; }
    __syncwarp();
  }
}

// Communities of at most AGG_TINY flat arcs and AGG_TINY members, eight lanes
// each (four per warp): lane g holds member g and flat arc g, and equal keys
// are merged with shuffles inside the group -- no table to clear or scan.
constexpr int AGG_TINY = 8;

template <typename W>
__global__ void __launch_bounds__(256) k_agg_tiny(AggArgs A) {
  const W *w = (const W *)A.w;
  const int lane = threadIdx.x & 31, g = lane & 7, grp = lane >> 3;
  const uint32_t gmask = 0xffu << (grp * 8);
  int64_t count = *A.count;
  int64_t step = (int64_t)gridDim.x * (blockDim.x >> 5) * 4;  // groups in the grid
  for (int64_t t0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 4; t0 < count;
       t0 += step) {  // warp-uniform
    int64_t t = t0 + grp;
    bool on = t < count;
    int64_t c = on ? A.list[t] : 0;
    int64_t m0 = on ? A.coff[c] : 0, nm = on ? A.coff[c + 1] - m0 : 0;
    int64_t f0 = on ? A.yoff[c] : 0, dg = on ? A.yoff[c + 1] - f0 : 0;  // the super-row and the flat arcs
    bool mem = g < nm;
    int64_t s = mem ? A.cflat[m0 + g] : INT64_MAX;  // member g: first flat arc, row of flat 0
    int64_t row = mem ? A.off[A.cverts[m0 + g]] - s : 0;
    int64_t f = f0 + g;
    bool arc = g < dg;
    int k = 0;  // the last member with first flat arc <= f (all lanes shuffle)
#pragma unroll
    for (int d = 4; d > 0; d >>= 1) {
      int64_t sc = __shfl_sync(LD_FULL, s, k + d, 8);
      if (sc <= f) k += d;
    }
    int64_t rw = __shfl_sync(LD_FULL, row, k, 8) + f;
    int32_t key = -1;
    int64_t wv = 0;
    if (arc) {
      key = A.C[A.col[rw]];
      wv = (int64_t)w[rw];
    }
    int64_t sum = 0;  // the weight of this lane's key in the group; the first lane holding it emits
    bool first = arc;
#pragma unroll
    for (int j = 0; j < 8; j++) {
      int32_t kj = __shfl_sync(LD_FULL, key, j, 8);
      int64_t wj = __shfl_sync(LD_FULL, wv, j, 8);
      if (arc && kj == key) {
        sum += wj;
        if (j < g) first = false;
      }
    }
    uint32_t fm = __ballot_sync(LD_FULL, first) & gmask;
    if (first) {
      int pos = __popc(fm & ((1u << lane) - 1u));
      A.ycol[f0 + pos] = key;
      A.yw[f0 + pos] = sum;
    }
    int64_t ks = wv;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) ks += __shfl_xor_sync(LD_FULL, ks, o, 8);
    if (on && g == 0) {
      A.ydeg[c] = __popc(fm);
      A.Kout[c] = ks;
    }
  }
}

// Communities of BIN_WARP_MAX+1..BIN_BLOCK_MAX flat arcs, a block each, with
// the members staged AGG_MB at a time in shared memory.
template <typename W>
__global__ void __launch_bounds__(256) k_agg_block(AggArgs A) {
  __shared__ int32_t keys[AGG_BLOCK_TABLE];
  __shared__ int64_t vals[AGG_BLOCK_TABLE];
  __shared__ int64_t ms[AGG_MB + 1];
  __shared__ int64_t mr[AGG_MB];
  __shared__ int32_t rc;
  __shared__ int64_t rs;
  const W *w = (const W *)A.w;
  int64_t count = *A.count;
  for (int64_t t = blockIdx.x; t < count; t += gridDim.x) {
    int64_t c = A.list[t];
    int64_t dg = A.yoff[c + 1] - A.yoff[c];
    int T = 32;
    while (T < 2 * dg) T <<= 1;
    for (int s = threadIdx.x; s < T; s += blockDim.x) { keys[s] = LD_EMPTY_KEY; vals[s] = 0; }
    if (threadIdx.x == 0) { rc = 0; rs = 0; }
    int64_t m0 = A.coff[c], m1 = A.coff[c + 1];
    int64_t selfw = 0;  // arcs inside the community: summed in registers, added once per warp
    for (int64_t ab = m0; ab < m1; ab += AGG_MB) {  // block-uniform
      int nb = m1 - ab < AGG_MB ? (int)(m1 - ab) : AGG_MB;
      __syncthreads();  // the table is cleared and the previous batch has been read
      if ((int)threadIdx.x < nb) {
        int64_t s = A.cflat[ab + threadIdx.x];
        ms[threadIdx.x] = s;
        mr[threadIdx.x] = A.off[A.cverts[ab + threadIdx.x]] - s;
      }
      if (threadIdx.x == 0) ms[nb] = A.cflat[ab + nb];
      __syncthreads();
      int64_t be = ms[nb];
      for (int64_t R = ms[0]; R < be; R += 256 * AGG_UNROLL) {
        int32_t j[AGG_UNROLL];
        int64_t wa[AGG_UNROLL];
        bool valid[AGG_UNROLL];
#pragma unroll
        for (int u = 0; u < AGG_UNROLL; u++) {
          int64_t f = R + u * 256 + threadIdx.x;
          valid[u] = f < be;
          j[u] = 0;
          wa[u] = 0;
          if (valid[u]) {
            int64_t row = mr[agg_member_of(ms, nb, f)] + f;
            j[u] = A.col[row];
            wa[u] = (int64_t)w[row];
          }
        }
        int32_t cj[AGG_UNROLL];  // the C gathers of all of them in flight together
#pragma unroll
        for (int u = 0; u < AGG_UNROLL; u++) cj[u] = valid[u] ? A.C[j[u]] : -1;
#pragma unroll
        for (int u = 0; u < AGG_UNROLL; u++) {
          if (cj[u] == (int32_t)c) selfw += wa[u];
          else if (valid[u]) agg_insert(keys, vals, T - 1, cj[u], wa[u]);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) selfw += __shfl_xor_sync(LD_FULL, selfw, o);
    if ((threadIdx.x & 31) == 0 && selfw) agg_insert(keys, vals, T - 1, (int32_t)c, selfw);
    __syncthreads();
    agg_emit<256>(A, c, threadIdx.x, blockDim.x, keys, vals, T, &rc, &rs);
    __syncthreads();
    if (threadIdx.x == 0) { A.ydeg[c] = rc; A.Kout[c] = rs; }
    __syncthreads();
  }
}

// A table of at least ncomm slots is indexed by the key directly (dense);
// a smaller one is an open-addressing hash table.
__device__ __forceinline__ void agg_flush(WarpTable &T8, bool dense, int32_t *keys, int64_t *vals, int32_t *list,
                                          int32_t *occ, int tmask) {
  if (dense) wt_flush_dense(T8, keys, vals, list, occ);
  else wt_flush(T8, keys, vals, list, occ, tmask);
}

// Communities above BIN_BLOCK_MAX flat arcs: each has its own global table
// (tab_off) and its flat arcs are cut into chunks any block may take
// (ch_off).  Each warp of the block takes an eighth of the chunk on its own
// (no block barrier, so no warp waits for another): it finds the member
// holding its first arc with a 32-way search over the members' flat
// offsets, then takes the members 32 at a time, lane i holding member i's
// arcs clipped to the warp's range; members with at most AGG_SHORT arcs
// there are walked by their lanes, the others one at a time by the whole
// warp.  Arcs go into the warp's table, flushed into the community's
// global table when full; arcs inside the community are summed in
// registers and added once per warp, and the weight sum goes to the
// super-vertex's K.
constexpr int AGG_SHORT = 16;  // at most this many arcs in range: a lane walks the member's row
constexpr int AGG_SPAN = TABLE_CHUNK / 8;  // flat arcs of one warp in a chunk

template <typename W>
__device__ __forceinline__ void agg_take(const AggArgs &A, WarpTable &T8, bool dense, int32_t *keys, int64_t *vals,
                                         int32_t *list, int32_t *occ, int tmask, int32_t self, const bool *valid,
                                         const int32_t *j, const int64_t *wa, int64_t &ksum, int64_t &selfw) {
  int32_t cc[AGG_UNROLL];
#pragma unroll
  for (int u = 0; u < AGG_UNROLL; u++) cc[u] = valid[u] ? A.C[j[u]] : 0;
#pragma unroll
  for (int u = 0; u < AGG_UNROLL; u++) {
    bool own = valid[u] && cc[u] == self;
    ksum += wa[u];
    selfw += own ? wa[u] : 0;
    if (T8.count > WT_LIMIT) agg_flush(T8, dense, keys, vals, list, occ, tmask);
    wt_insert_lanes(T8, valid[u] && !own, cc[u], wa[u]);
  }
}

template <typename W>
__global__ void __launch_bounds__(256, 4) k_agg_chunk_scan(AggArgs A, const int64_t *tab_off, const int64_t *ch_off) {
  __shared__ WarpTable WT[8];  // per-warp sums by community
  WarpTable &T8 = WT[threadIdx.x >> 5];
  wt_init(T8);
  int64_t count = *A.count;
  int64_t nch = ch_off[count];
  const W *w = (const W *)A.w;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t t = blockIdx.x; t < nch; t += gridDim.x) {
    int64_t lo = 0, hi = count - 1;  // community k with ch_off[k] <= t < ch_off[k+1]
    while (lo < hi) {
      int64_t mid = (lo + hi + 1) >> 1;
      if (ch_off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    int64_t c = A.list[lo];
    int64_t m0 = A.coff[c], m1 = A.coff[c + 1];
    int64_t fc = A.cflat[m0] + (t - ch_off[lo]) * TABLE_CHUNK, fe = A.cflat[m1];
    int64_t f0 = fc + (int64_t)wid * AGG_SPAN, f1 = f0 + AGG_SPAN;  // this warp's arcs
    if (f1 > fc + TABLE_CHUNK) f1 = fc + TABLE_CHUNK;
    if (f1 > fe) f1 = fe;
    if (f0 >= f1) continue;  // warp-uniform: the chunk is short
    int64_t T = tab_off[lo + 1] - tab_off[lo];
    bool dense = T >= A.ncomm;  // every key (a community id) has its own slot
    int tmask = (int)(T - 1);
    int32_t *keys = A.gkeys + tab_off[lo], *list = A.glist + tab_off[lo];
    int64_t *vals = A.gvals + tab_off[lo];
    int32_t *occ = &A.gocc[lo];
    // the member holding f0: the last a in [m0, m1) with cflat[a] <= f0,
    // narrowed 32-fold per step (cflat[a0] <= f0 holds throughout)
    int64_t a0 = m0, span = m1 - m0;
    while (span > 1) {  // warp-uniform
      int64_t step = (span + 31) >> 5;
      int64_t p = a0 + lane * step;
      bool le = p < a0 + span && A.cflat[p] <= f0;
      int k = 31 - __clz(__ballot_sync(LD_FULL, le));
      a0 += k * step;
      span = span - k * step < step ? span - k * step : step;
    }
    int64_t ksum = 0, selfw = 0;
    for (int64_t ab = a0; ab < m1; ab += 32) {  // warp-uniform
      int64_t a = ab + lane;
      bool in = a < m1;
      int64_t s = in ? A.cflat[a] : f1;
      if (__shfl_sync(LD_FULL, s, 0) >= f1) break;  // past this warp's range
      int64_t e = in ? A.cflat[a + 1] : f1;
      int64_t cs = s > f0 ? s : f0, ce = e < f1 ? e : f1;
      int64_t len = ce > cs ? ce - cs : 0, row = 0;
      if (len > 0) row = A.off[A.cverts[a]] - s;  // row index of flat arc f: row + f
      // the member's arcs in range start at col + row + cs (32-bit offsets
      // from there: a range holds at most AGG_SPAN arcs)
      const int32_t *mcol = A.col + (row + cs);
      const W *mw = w + (row + cs);
      int ln = (int)len;
      bool shrt = ln <= AGG_SHORT;
      int maxs = __reduce_max_sync(LD_FULL, shrt ? (unsigned)ln : 0u);
      for (int jj = 0; jj < maxs; jj += AGG_UNROLL) {  // warp-uniform
        int32_t j[AGG_UNROLL];
        int64_t wa[AGG_UNROLL];
        bool valid[AGG_UNROLL];
#pragma unroll
        for (int u = 0; u < AGG_UNROLL; u++) {
          valid[u] = shrt && jj + u < ln;
          j[u] = valid[u] ? mcol[jj + u] : 0;
          wa[u] = valid[u] ? (int64_t)mw[jj + u] : 0;
        }
        agg_take<W>(A, T8, dense, keys, vals, list, occ, tmask, (int32_t)c, valid, j, wa, ksum, selfw);
      }
      for (uint32_t med = __ballot_sync(LD_FULL, !shrt); med; med &= med - 1u) {  // warp-uniform
        int src = __ffs(med) - 1;
        const int32_t *pc = (const int32_t *)__shfl_sync(LD_FULL, (unsigned long long)mcol, src);
        const W *pw = (const W *)__shfl_sync(LD_FULL, (unsigned long long)mw, src);
        int n = __shfl_sync(LD_FULL, ln, src);
        for (int r = 0; r < n; r += 32 * AGG_UNROLL) {  // warp-uniform
          int32_t j[AGG_UNROLL];
          int64_t wa[AGG_UNROLL];
          bool valid[AGG_UNROLL];
#pragma unroll
          for (int u = 0; u < AGG_UNROLL; u++) {
            int x = r + u * 32 + lane;
            valid[u] = x < n;
            j[u] = valid[u] ? pc[x] : 0;
            wa[u] = valid[u] ? (int64_t)pw[x] : 0;
          }
          agg_take<W>(A, T8, dense, keys, vals, list, occ, tmask, (int32_t)c, valid, j, wa, ksum, selfw);
        }
      }
    }
    agg_flush(T8, dense, keys, vals, list, occ, tmask);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ksum += __shfl_xor_sync(LD_FULL, ksum, o);
      selfw += __shfl_xor_sync(LD_FULL, selfw, o);
    }
    if (lane == 0) {
      if (ksum != 0) atomicAdd((unsigned long long *)&A.Kout[c], (unsigned long long)ksum);
      if (selfw != 0) {
        if (dense) ld_gtable_add_direct(keys, vals, list, occ, (int32_t)c, selfw);
        else ld_gtable_insert(keys, vals, list, occ, tmask, (int32_t)c, selfw);
      }
      // per flat arc: col, C of the neighbour and the weight
      atomicAdd((unsigned long long *)A.xk_bytes, (unsigned long long)((8 + sizeof(W)) * (f1 - f0)));
    }
  }
}

// Emission of the chunked path: a community's listed slots are cut into
// EMIT_CHUNK pieces any block may take; em_off[k] is the first piece of the
// k-th listed community (every community has at least one, which also
// writes its degree).
constexpr int EMIT_CHUNK = 2048;

__global__ void __launch_bounds__(1024) k_emit_plan(const int32_t *count_p, const int32_t *occ, int64_t *em_off) {
  __shared__ int64_t ws[32];
  __shared__ int64_t carry;
  int64_t count = *count_p;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < count; base += blockDim.x) {  // block-uniform
    int64_t k = base + threadIdx.x;
    int64_t x = k < count ? (occ[k] > 0 ? (occ[k] + EMIT_CHUNK - 1) / EMIT_CHUNK : 1) : 0;
    int64_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(LD_FULL, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) ws[wid] = incl;
    __syncthreads();
    int64_t before = carry;
    for (int q = 0; q < wid; q++) before += ws[q];
    if (k < count) em_off[k] = before + incl - x;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) em_off[count] = carry;
}

__global__ void __launch_bounds__(256) k_agg_list_emit(AggArgs A, const int64_t *tab_off, const int64_t *em_off) {
  int64_t count = *A.count;
  int64_t npc = em_off[count];
  for (int64_t t = blockIdx.x; t < npc; t += gridDim.x) {
    int64_t k = 0, hi = count - 1;  // community k with em_off[k] <= t < em_off[k+1]
    while (k < hi) {
      int64_t mid = (k + hi + 1) >> 1;
      if (em_off[mid] <= t) k = mid; else hi = mid - 1;
    }
    int64_t c = A.list[k];
    int32_t *keys = A.gkeys + tab_off[k], *list = A.glist + tab_off[k];
    int64_t *vals = A.gvals + tab_off[k];
    int64_t occ = A.gocc[k];
    bool dense = tab_off[k + 1] - tab_off[k] >= A.ncomm;  // the list holds the keys themselves
    int64_t q0 = (t - em_off[k]) * EMIT_CHUNK, q1 = q0 + EMIT_CHUNK < occ ? q0 + EMIT_CHUNK : occ;
    int64_t base = A.yoff[c];
    for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
      int32_t s = list[q];
      int32_t key = dense ? s : keys[s];
      keys[s] = LD_EMPTY_KEY;
      A.ycol[base + q] = key;
      A.yw[base + q] = vals[s];
      vals[s] = 0;
    }
    if (q0 == 0 && threadIdx.x == 0) {
      A.ydeg[c] = (int32_t)occ;
      atomicAdd((unsigned long long *)&A.tables[dense ? 1 : 0], 1ull);
    }
  }
}

// Before the chunked scan: empty fill counts, and zero the K of the listed
// communities (the scan adds its chunks' weight sums into it).
__global__ void k_zero_occ(const int32_t *count_p, const int32_t *list, int32_t *occ, int64_t *Kout) {
  for (int64_t k = ld_gtid(); k < *count_p; k += ld_gstride()) {
    occ[k] = 0;
    Kout[list[k]] = 0;
  }
}

__global__ void k_agg_bin(int64_t ncomm, const int64_t *yoff, const int64_t *coff, int32_t *bins, DevCounters *cnt) {
  int lane = threadIdx.x & 31;
  for (int64_t base = (ld_gtid() & ~31ll); base < ncomm; base += ld_gstride()) {
    int64_t c = base + lane;
    int bin = -1;
    if (c < ncomm) {
      int64_t d = yoff[c + 1] - yoff[c];
      bin = d <= AGG_TINY && coff[c + 1] - coff[c] <= AGG_TINY ? BIN_TINY
            : d <= BIN_WARP_MAX ? BIN_WARP : (d <= BIN_BLOCK_MAX ? BIN_BLOCK : BIN_HUGE);
    }
#pragma unroll
    for (int b = 0; b < NBINS; b++) {
      uint32_t m = __ballot_sync(LD_FULL, bin == b);
      if (!m) continue;
      int32_t p0 = 0;
      if (lane == __ffs(m) - 1) p0 = atomicAdd(&cnt->bin_count[b], __popc(m));
      p0 = __shfl_sync(LD_FULL, p0, __ffs(m) - 1);
      if (bin == b) bins[(int64_t)b * ncomm + p0 + __popc(m & ((1u << lane) - 1u))] = (int32_t)c;
    }
  }
}

// ---------------------------------------------------------------- pass reset
__global__ void k_next_pass(int64_t nc, const int64_t *Kout, int64_t *Kp, int64_t *Sp, int32_t *Cp, uint8_t *dR,
                            uint8_t *dS) {
  for (int64_t c = ld_gtid(); c < nc; c += ld_gstride()) {
    Kp[c] = Kout[c]; Sp[c] = Kout[c]; Cp[c] = (int32_t)c; dR[c] = 1; dS[c] = 0;
  }
}
__global__ void k_bits_all(int64_t n, uint32_t *bm) {
  int64_t words = (n + 31) >> 5;
  for (int64_t w = ld_gtid(); w < words; w += ld_gstride()) {
    int64_t rem = n - (w << 5);
    bm[w] = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
  }
}
// Start of the pass loop in one sweep: the affected flags become the
// frontier bitmap (and are counted), Ctop = identity, C' = C, K' = K,
// Sigma' = Sigma.  Four vertices per thread with 16-byte loads and stores
// (the arrays start 256-byte aligned); eight lanes make one bitmap word.
// A tail of n % 32 vertices is done one per lane by the first warp.
__global__ void k_pass_init(int64_t n, const uint8_t *dV, uint32_t *bm, int32_t *Ctop, const int32_t *C, int32_t *Cp,
                            const int64_t *K, int64_t *Kp, const int64_t *Sig, int64_t *Sp, DevCounters *cnt) {
  int lane = threadIdx.x & 31;
  int64_t set = 0;
  int64_t nq = (n >> 5) << 3;  // quads of whole 32-vertex words
  for (int64_t q0 = (ld_gtid() & ~31ll); q0 < nq; q0 += ld_gstride()) {  // warp-uniform trip count
    int64_t q = q0 + lane;
    uint32_t nib = 0;
    if (q < nq) {
      int64_t v = q << 2;
      uint32_t f = ((const uint32_t *)dV)[q];
      nib = (f & 0xffu ? 1u : 0u) | (f & 0xff00u ? 2u : 0u) | (f & 0xff0000u ? 4u : 0u) | (f & 0xff000000u ? 8u : 0u);
      ((int4 *)Ctop)[q] = make_int4((int)v, (int)v + 1, (int)v + 2, (int)v + 3);
      ((int4 *)Cp)[q] = ((const int4 *)C)[q];
      ((longlong2 *)Kp)[2 * q] = ((const longlong2 *)K)[2 * q];
      ((longlong2 *)Kp)[2 * q + 1] = ((const longlong2 *)K)[2 * q + 1];
      ((longlong2 *)Sp)[2 * q] = ((const longlong2 *)Sig)[2 * q];
      ((longlong2 *)Sp)[2 * q + 1] = ((const longlong2 *)Sig)[2 * q + 1];
    }
    uint32_t word = nib << ((lane & 7) * 4);  // lanes 8k..8k+7 hold word q/8
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) word |= __shfl_xor_sync(LD_FULL, word, o);
    if (q < nq && (lane & 7) == 0) {
      bm[q >> 3] = word;
      set += __popc(word);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x < 32) {  // the last partial word
    int64_t v = (nq << 2) + lane;
    bool in = v < n;
    uint32_t m = __ballot_sync(LD_FULL, in && dV[v]);
    if (in) {
      Ctop[v] = (int32_t)v;
      Cp[v] = C[v];
      Kp[v] = K[v];
      Sp[v] = Sig[v];
    }
    if (lane == 0 && (nq << 2) < n) {
      bm[nq >> 3] = m;
      set += __popc(m);
    }
  }
  set = ld_warp_sum_i64(set);
  if (lane == 0 && set) atomicAdd((unsigned long long *)&cnt->affected, (unsigned long long)set);
}

__global__ void k_maxdeg(int64_t n, const int32_t *deg, DevCounters *cnt, int block_max) {
  int32_t mx = 0;
  int64_t slots = 0, sum = 0;
  for (int64_t i = ld_gtid(); i < n; i += ld_gstride()) {
    int32_t d = deg[i];
    mx = max(mx, d);
    sum += d;
    if (d > block_max) {
      int64_t t = 1;
      while (t < 2 * (int64_t)d) t <<= 1;
      slots += t;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = max(mx, __shfl_xor_sync(LD_FULL, mx, o));
    slots += __shfl_xor_sync(LD_FULL, slots, o);
    sum += __shfl_xor_sync(LD_FULL, sum, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (mx) atomicMax(&cnt->max_count, mx);
    if (slots) atomicAdd((unsigned long long *)&cnt->huge_slots, (unsigned long long)slots);
    if (sum) atomicAdd((unsigned long long *)&cnt->deg_sum, (unsigned long long)sum);
  }
}

}  // namespace

void subset_renumber(leiden_handle *h, int64_t n) {
  cudaStream_t s = h->stream;
  int g = grid_for(n, TB);
  ld_note_launch(), k_sr_init<<<g, TB, 0, s>>>(n, h->rep, h->S2, h->dS2, h->dR2);
  ld_note_launch(), k_sr_min<<<g, TB, 0, s>>>(n, h->Cp, h->rep);
  ld_note_launch(), k_sr_rekey<<<g, TB, 0, s>>>(n, h->rep, h->Sp, h->dS, h->dR, h->S2, h->dS2, h->dR2);
  ld_note_launch(), k_sr_remap<<<g, TB, 0, s>>>(n, h->rep, h->Cp);
  std::swap(h->Sp, h->S2);
  std::swap(h->dS, h->dS2);
  std::swap(h->dR, h->dR2);
}

void split_communities(leiden_handle *h, const LevelGraph &g) {
  cudaStream_t s = h->stream;
  cudaMemsetAsync(&h->dcnt->split_count, 0, sizeof(int32_t), s);
  cudaMemsetAsync(&h->dcnt->split_arcs, 0, sizeof(int64_t), s);
  int32_t *list = h->ibuf1;
  ld_note_launch(), k_split_init<<<grid_for(g.n, TB), TB, 0, s>>>(g.n, h->Cp, h->dS, h->dR, g.deg, h->parent, list,
                                                                  h->dcnt, h->p.split_all);
  kt_begin(h, KT_SPLIT_SAMPLE);
  ld_note_launch(), k_split_sample<<<h->sm_count * 16, TB, 0, s>>>(list, h->dcnt, g.off, g.deg, g.col, h->Cp, h->parent);
  kt_end(h);
  ld_note_launch(), k_split_flatten<<<h->sm_count * 8, TB, 0, s>>>(list, h->dcnt, h->parent);
  cudaMemsetAsync(&h->dcnt->big_count, 0, sizeof(int32_t), s);
  ld_note_launch(), k_split_link_rest<<<h->sm_count * 8, TB, 0, s>>>(list, h->dcnt, g.off, g.deg, g.col, h->Cp, h->parent, h->ibuf2);
  ld_note_launch(), k_split_link_big<<<h->sm_count, 1024, 0, s>>>(h->ibuf2, h->dcnt, g.off, g.deg, g.col, h->Cp, h->parent);
  ld_note_launch(), k_split_compress<<<h->sm_count * 8, TB, 0, s>>>(list, h->dcnt, h->parent, h->Cp);
}

void count_communities(leiden_handle *h, int64_t n, const int32_t *gid) {
  cudaStream_t s = h->stream;
  cudaMemsetAsync(&h->dcnt->list_count, 0, sizeof(int32_t), s);
  ld_note_launch(), k_count_roots<<<grid_for(n, TB), TB, 0, s>>>(n, h->Cp, h->dcnt, gid, h->gc.ncomm);
}

void renumber_dense(leiden_handle *h, int64_t n, const int32_t *gid) {
  cudaStream_t s = h->stream;
  const uint8_t *cont = gid ? h->gc.cont : nullptr;
  cudaMemsetAsync(h->ibuf0, 0, (size_t)n * sizeof(int32_t), s);
  ld_note_launch(), k_used<<<grid_for(n, TB), TB, 0, s>>>(n, h->Cp, h->ibuf0, gid, cont);
  exclusive_scan_i32_to_i64(h->ibuf0, h->lbuf0, n, h->scan_tmp, s);
  ld_note_launch(), k_rank<<<grid_for(n, TB), TB, 0, s>>>(n, h->lbuf0, h->Cp, gid, cont);
}

void lookup_dendrogram(leiden_handle *h) {
  const uint8_t *cont = h->gid0 ? h->gc.cont : nullptr;
  ld_note_launch(), k_lookup<<<grid_for(h->n, TB), TB, 0, h->stream>>>(h->n, h->Cp, h->Ctop, h->gid0, cont);
}

void break_lookup(leiden_handle *h) {
  ld_note_launch(), k_break_lookup<<<grid_for(h->n, TB), TB, 0, h->stream>>>(h->n, h->Cp, h->Ctop, h->gid0, h->gc.cont,
                                                                               h->d_loff, h->d_voff);
}

void next_level_ids(leiden_handle *h, int64_t n, const int32_t *gid, int32_t *gid_next, int64_t *loff_next) {
  cudaStream_t s = h->stream;
  ld_note_launch(), k_level_ids<<<grid_for(n, TB), TB, 0, s>>>(n, h->Cp, gid, h->gc.cont, gid_next);
  ld_note_launch(), k_level_off<<<grid_for(h->G + 1, TB), TB, 0, s>>>(h->G, h->d_loff, h->lbuf0, loff_next);
}

// Aggregate level g by its dense membership Cp into slot `out`; K'' goes to
// h->S2.  Sets dcnt->max_count to the largest super-row capacity.
void aggregate(leiden_handle *h, const LevelGraph &g, int64_t ncomm, int out) {
  cudaStream_t s = h->stream;
  int64_t n = g.n;
  // community vertices CSR; batched handles carry the stopped graphs'
  // vertices in one spare community ncomm, listed last and not aggregated
  int64_t nc = ncomm + (g.gid ? 1 : 0);
  cudaMemsetAsync(h->ibuf0, 0, (size_t)nc * sizeof(int32_t), s);
  ld_note_launch(), k_member_count<<<grid_for(n, TB), TB, 0, s>>>(n, h->Cp, h->ibuf0);
  exclusive_scan_i32_to_i64(h->ibuf0, h->coff, nc, h->scan_tmp, s);
  cudaMemcpyAsync(h->lbuf0, h->coff, (size_t)nc * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
  ld_note_launch(), k_member_fill<<<grid_for(n, TB), TB, 0, s>>>(n, h->Cp, (unsigned long long *)h->lbuf0, h->cverts);
  // flat arc offsets of the members, and the super-row offsets
  ld_note_launch(), k_member_deg<<<grid_for(n, TB), TB, 0, s>>>(n, h->cverts, g.deg, h->ibuf1);
  exclusive_scan_i32_to_i64(h->ibuf1, h->cflat, n, h->scan_tmp, s);
  cudaMemsetAsync(&h->dcnt->max_count, 0, sizeof(int32_t), s);
  cudaMemsetAsync(&h->dcnt->huge_slots, 0, sizeof(int64_t), s);
  ld_note_launch(), k_yoff<<<grid_for(ncomm + 1, TB), TB, 0, s>>>(ncomm, h->coff, h->cflat, h->y_off[out], h->dcnt);
  cudaMemsetAsync(&h->dcnt->bin_count[0], 0, sizeof(int32_t) * 4, s);
  ld_note_launch(), k_agg_bin<<<grid_for(ncomm, TB), TB, 0, s>>>(ncomm, h->y_off[out], h->coff, h->bins, h->dcnt);
  cudaMemcpyAsync(&h->hcnt->max_count, &h->dcnt->max_count, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&h->hcnt->huge_slots, &h->dcnt->huge_slots, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  int32_t maxc = h->hcnt->max_count;
  AggArgs A{};
  A.ncomm = ncomm;
  A.off = g.off;
  A.deg = g.deg;
  A.col = g.col;
  A.w = g.w;
  A.C = h->Cp;
  A.coff = h->coff;
  A.cverts = h->cverts;
  A.cflat = h->cflat;
  A.yoff = h->y_off[out];
  A.ydeg = h->y_deg[out];
  A.ycol = h->y_col[out];
  A.yw = h->y_w[out];
  A.Kout = h->S2;
  int sms = h->sm_count;
  A.list = h->bins + (int64_t)BIN_TINY * ncomm;
  A.count = &h->dcnt->bin_count[BIN_TINY];
  if (g.w64) ld_note_launch(), k_agg_tiny<int64_t><<<sms * 8, 256, 0, s>>>(A);
  else ld_note_launch(), k_agg_tiny<int32_t><<<sms * 8, 256, 0, s>>>(A);
  A.list = h->bins;
  A.count = &h->dcnt->bin_count[BIN_WARP];
  if (g.w64) ld_note_launch(), k_agg_warp<int64_t><<<sms * 8, AGG_WARPS * 32, 0, s>>>(A);
  else ld_note_launch(), k_agg_warp<int32_t><<<sms * 8, AGG_WARPS * 32, 0, s>>>(A);
  if (maxc > BIN_WARP_MAX) {
    A.list = h->bins + ncomm;
    A.count = &h->dcnt->bin_count[BIN_BLOCK];
    if (g.w64) ld_note_launch(), k_agg_block<int64_t><<<sms * 4, 256, 0, s>>>(A);
    else ld_note_launch(), k_agg_block<int32_t><<<sms * 4, 256, 0, s>>>(A);
  }
  if (maxc > BIN_BLOCK_MAX) {
    // a table per listed community at once: at most huge_slots slots
    if (!ensure_hslots(h, h->hcnt->huge_slots)) { h->fatal = LEIDEN_ERR_OOM; h->err = "global table scratch"; return; }
    A.list = h->bins + 2 * ncomm;
    A.count = &h->dcnt->bin_count[BIN_HUGE];
    A.gkeys = hs_keys(h);
    A.gvals = hs_vals(h);
    A.glist = hs_list(h);
    A.gocc = h->hocc;
    int64_t *tab_off = h->lbuf2, *ch_off = h->lbuf3;
    // a community's super-row has at most one key per community
    launch_table_plan(A.list, A.count, nullptr, h->y_off[out], ncomm, tab_off, ch_off, s);
    ld_note_launch(), k_zero_occ<<<sms, 256, 0, s>>>(A.count, A.list, A.gocc, A.Kout);
    A.xk_bytes = &h->dcnt->xk_bytes[1];
    A.tables = h->dcnt->agg_tables;
    kt_begin(h, KT_AGG_CHUNK);
    if (g.w64) ld_note_launch(), k_agg_chunk_scan<int64_t><<<sms * 16, 256, 0, s>>>(A, tab_off, ch_off);
    else ld_note_launch(), k_agg_chunk_scan<int32_t><<<sms * 16, 256, 0, s>>>(A, tab_off, ch_off);
    kt_end(h);
    int64_t *em_off = h->lbuf0;  // free again after the member fill
    ld_note_launch(), k_emit_plan<<<1, 1024, 0, s>>>(A.count, A.gocc, em_off);
    ld_note_launch(), k_agg_list_emit<<<sms * 8, 256, 0, s>>>(A, tab_off, em_off);
  }
}

void reset_next_pass(leiden_handle *h, int64_t ncomm, int out) {
  (void)out;
  cudaStream_t s = h->stream;
  ld_note_launch(), k_next_pass<<<grid_for(ncomm, TB), TB, 0, s>>>(ncomm, h->S2, h->Kp, h->Sp, h->Cp, h->dR, h->dS);
  mark_all_unprocessed(h, ncomm);
}

void mark_all_unprocessed(leiden_handle *h, int64_t n) {
  ld_note_launch(), k_bits_all<<<grid_for((n + 31) / 32, TB), TB, 0, h->stream>>>(n, h->unproc);
}

void pass_init(leiden_handle *h) {
  cudaMemsetAsync(&h->dcnt->affected, 0, sizeof(int64_t), h->stream);
  ld_note_launch(), k_pass_init<<<grid_for(h->n, TB), TB, 0, h->stream>>>(h->n, h->dV, h->unproc, h->Ctop, h->C, h->Cp,
                                                                          h->K, h->Kp, h->Sig, h->Sp, h->dcnt);
}

void level_maxdeg(leiden_handle *h, const int32_t *deg, int64_t n) {
  cudaMemsetAsync(&h->dcnt->max_count, 0, sizeof(int32_t), h->stream);
  cudaMemsetAsync(&h->dcnt->huge_slots, 0, sizeof(int64_t), h->stream);
  cudaMemsetAsync(&h->dcnt->deg_sum, 0, sizeof(int64_t), h->stream);
  ld_note_launch(), k_maxdeg<<<grid_for(n, TB), TB, 0, h->stream>>>(n, deg, h->dcnt, h->tune.block_max);
}

LD_CHECK_WORD_READER(check_word_phases)
