// Batch update: canonicalise the batch, apply it to the slack CSR by sorted
// merge, mark affected vertices (ND / DS / DF, Appendix A.1-A.3), update
// K, Sigma and Delta Sigma (Alg. "update"), and mark communities to split /
// refine (Alg. "leidenmk").
#include <algorithm>

#include "internal.h"

namespace {

constexpr int TB = 256;
constexpr int MERGE_SMALL = 256;  // touched rows up to this new length merge in one warp (8 KB of
                                  // shared staging per block keeps many rows in flight)
constexpr int MERGE_MID = 4096;   // up to this length: one block, staged in shared memory, in place

__device__ __forceinline__ int64_t lower_bound_i32(const int32_t *a, int64_t n, int32_t x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t *a, int64_t n, uint64_t x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Mirror each undirected edge into two arcs keyed (src << vb) | dst and
// validate it.  error := 1 on any violation.  Deletions and insertions go
// into one array for one sort: the 2*n_del deletion arcs first (weight 0),
// then the insertion arcs with bit 2*vb set, so that after the sort the
// deletions come first and each part is sorted by its keys.
__global__ void k_expand(const leiden_edge *del, int64_t n_del, const leiden_edge *ins, int64_t n_ins,
                         int64_t n, int vb, uint64_t *key, int64_t *w, DevCounters *cnt, const int32_t *gid0) {
  const uint64_t ins_bit = 1ull << (2 * vb);
  for (int64_t e = ld_gtid(); e < n_del + n_ins; e += ld_gstride()) {
    bool is_del = e < n_del;
    leiden_edge x = is_del ? del[e] : ins[e - n_del];
    bool bad = x.u < 0 || x.u >= n || x.v < 0 || x.v >= n || x.u == x.v || (!is_del && x.w <= 0);
    if (!bad && gid0 && gid0[x.u] != gid0[x.v]) bad = true;  // batched: an edge between two graphs
    if (bad) {
      atomicExch(&cnt->error, 1);
      x.u = 0; x.v = 1 % (int32_t)(n > 1 ? n : 1); x.w = 1;
    }
    uint64_t k1 = ((uint64_t)x.u << vb) | (uint64_t)x.v;
    uint64_t k2 = ((uint64_t)x.v << vb) | (uint64_t)x.u;
    uint64_t tag = is_del ? 0ull : ins_bit;
    key[2 * e] = k1 | tag;
    key[2 * e + 1] = k2 | tag;
    w[2 * e] = is_del ? 0 : x.w;
    w[2 * e + 1] = is_del ? 0 : x.w;
  }
}

// Clear the insertion tag of the sorted insertion arcs.
__global__ void k_untag(uint64_t *key, int64_t n, uint64_t mask) {
  for (int64_t i = ld_gtid(); i < n; i += ld_gstride()) key[i] &= mask;
}

__global__ void k_head_flags(const uint64_t *key, int64_t n, int32_t *flag) {
  for (int64_t i = ld_gtid(); i < n; i += ld_gstride()) flag[i] = (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
}

// Unique keys (and summed payload) into out_key/out_w at the scanned positions.
__global__ void k_unique(const uint64_t *key, const int64_t *w, int64_t n, const int32_t *flag, const int64_t *pos,
                         uint64_t *out_key, int64_t *out_w) {
  for (int64_t i = ld_gtid(); i < n; i += ld_gstride()) {
    int64_t p = pos[i] + flag[i] - 1;
    if (flag[i]) out_key[p] = key[i];
    if (out_w) atomicAdd((unsigned long long *)&out_w[p], (unsigned long long)w[i]);
  }
}

// Deletions must name existing arcs; record the stored weight.
__global__ void k_check_deletions(const uint64_t *dkey, const int64_t *nd_p, int vb, const int64_t *off,
                                  const int32_t *deg, const int32_t *col, const int32_t *w, int64_t *dw,
                                  DevCounters *cnt) {
  uint64_t mask = (1ull << vb) - 1;
  int64_t nd = *nd_p;
  for (int64_t i = ld_gtid(); i < nd; i += ld_gstride()) {
    int32_t u = (int32_t)(dkey[i] >> vb), v = (int32_t)(dkey[i] & mask);
    const int32_t *row = col + off[u];
    int64_t p = lower_bound_i32(row, deg[u], v);
    if (p < deg[u] && row[p] == v) dw[i] = w[off[u] + p];
    else { dw[i] = 0; atomicExch(&cnt->error, 2); }
  }
}

// Insertions: existing arc (not deleted in this batch) -> state 1, position;
// otherwise state 0 (a new arc).
__global__ void k_classify_insertions(const uint64_t *ikey, const int64_t *ni_p, const uint64_t *dkey,
                                      const int64_t *nd_p, int vb, const int64_t *off, const int32_t *deg,
                                      const int32_t *col, int32_t *state, int64_t *ipos) {
  uint64_t mask = (1ull << vb) - 1;
  int64_t ni = *ni_p, nd = *nd_p;
  for (int64_t i = ld_gtid(); i < ni; i += ld_gstride()) {
    int32_t u = (int32_t)(ikey[i] >> vb), v = (int32_t)(ikey[i] & mask);
    const int32_t *row = col + off[u];
    int64_t p = lower_bound_i32(row, deg[u], v);
    bool found = p < deg[u] && row[p] == v;
    if (found) {
      int64_t q = lower_bound_u64(dkey, nd, ikey[i]);
      if (q < nd && dkey[q] == ikey[i]) found = false;  // deleted, then inserted again
    }
    state[i] = found ? 1 : 0;
    ipos[i] = found ? off[u] + p : -1;
  }
}

// Flags of the new arcs over the bound nb >= ni (zero past ni).
__global__ void k_new_flags(const int32_t *state, const int64_t *ni_p, int64_t nb, int32_t *flag) {
  int64_t ni = *ni_p;
  for (int64_t i = ld_gtid(); i < nb; i += ld_gstride()) flag[i] = i < ni && state[i] == 0 ? 1 : 0;
}

__global__ void k_compact_new(const uint64_t *ikey, const int64_t *iw, int64_t ni, const int32_t *flag,
                              const int64_t *pos, uint64_t *okey, int64_t *ow) {
  for (int64_t i = ld_gtid(); i < ni; i += ld_gstride())
    if (flag[i]) { okey[pos[i]] = ikey[i]; ow[pos[i]] = iw[i]; }
}

// Rows whose structure changes (sources of deletions and of new arcs), each
// listed once, in no particular order: the first arc of a source's run in
// either sorted list sets the source's bit, and the arc that found it clear
// appends the row.  Work is O(batch), not O(n).
__global__ void k_touched_rows(const uint64_t *dkey, const int64_t *nd_p, const uint64_t *nkey, const int64_t *nn_p,
                               int vb, uint32_t *bits, int32_t *rows, int64_t *nrows) {
  int64_t nd = *nd_p, nn = *nn_p;
  for (int64_t t = ld_gtid(); t < nd + nn; t += ld_gstride()) {
    bool del = t < nd;
    const uint64_t *K = del ? dkey : nkey;
    int64_t k = del ? t : t - nd;
    uint64_t u = K[k] >> vb;
    if (k > 0 && (K[k - 1] >> vb) == u) continue;
    uint32_t bit = 1u << (u & 31);
    if (!(atomicOr(&bits[u >> 5], bit) & bit))
      rows[atomicAdd((unsigned long long *)nrows, 1ull)] = (int32_t)u;
  }
}

// Leaves the row bitmap clear for the next call (every set bit belongs to a
// listed row).
__global__ void k_clear_row_bits(const int32_t *rows, const int64_t *nrows_p, uint32_t *bits) {
  int64_t nrows = *nrows_p;
  for (int64_t r = ld_gtid(); r < nrows; r += ld_gstride()) bits[rows[r] >> 5] = 0;
}

// New length of each touched row and its segments in the two arc lists.
// A row that outgrows its capacity moves to the spill arena at the end of
// the arc arrays with fresh slack (dst, newcap); if the arena is full the
// whole CSR is rebuilt instead (overflow flag).  Lengths are written up to
// the bound nb >= nrows (zero past nrows) so that their scan needs no host
// count.  A batch already found invalid takes no arena space.
__global__ void k_row_plan(const int32_t *rows, const int64_t *nrows_p, int64_t nb, int vb, const uint64_t *dkey,
                           const int64_t *nd_p, const uint64_t *nkey, const int64_t *nn_p, const int64_t *off,
                           const int32_t *deg, const int32_t *rcap, int32_t *dlo, int32_t *dhi, int32_t *ilo,
                           int32_t *ihi, int64_t *len, int64_t *dst, int32_t *newcap, double slack, int min_slack,
                           int64_t colcap, int32_t *olddeg, int32_t *large, int32_t *mid, DevCounters *cnt) {
  int64_t nrows = *nrows_p, nd = *nd_p, nn = *nn_p;
  bool invalid = cnt->error != 0;
  for (int64_t r = ld_gtid(); r < nb; r += ld_gstride()) {
    if (r >= nrows) { len[r] = 0; continue; }
    uint64_t u = (uint64_t)rows[r];
    int64_t a = lower_bound_u64(dkey, nd, u << vb), b = lower_bound_u64(dkey, nd, (u + 1) << vb);
    int64_t c = lower_bound_u64(nkey, nn, u << vb), d = lower_bound_u64(nkey, nn, (u + 1) << vb);
    dlo[r] = (int32_t)a; dhi[r] = (int32_t)b; ilo[r] = (int32_t)c; ihi[r] = (int32_t)d;
    int64_t L = (int64_t)deg[u] - (b - a) + (d - c);
    len[r] = L;
    olddeg[r] = deg[u];
    if (L > MERGE_MID) large[atomicAdd(&cnt->large_count, 1)] = (int32_t)r;
    else if (L > MERGE_SMALL) mid[atomicAdd(&cnt->mid_count, 1)] = (int32_t)r;
    dst[r] = off[u];
    newcap[r] = 0;
    if (L > rcap[u] && !invalid) {
      int64_t extra = (int64_t)((double)L * slack);
      if (extra < min_slack) extra = min_slack;
      int64_t cap = L + extra;
      int64_t p = (int64_t)atomicAdd((unsigned long long *)&cnt->arena_used, (unsigned long long)cap);
      if (p + cap > colcap) atomicExch(&cnt->overflow, 1);
      dst[r] = p;
      newcap[r] = (int32_t)cap;
    }
  }
}

__global__ void k_add_existing(const int64_t *ipos, const int32_t *state, const int64_t *iw, int64_t ni, int32_t *w) {
  for (int64_t i = ld_gtid(); i < ni; i += ld_gstride())
    if (state[i]) w[ipos[i]] += (int32_t)iw[i];
}

// Warp per touched row: old row minus deletions plus new arcs, by ranks.
__global__ void k_merge_rows(const int32_t *rows, const int64_t *nrows_p, int vb, const uint64_t *dkey,
                             const uint64_t *nkey, const int64_t *nw, const int32_t *dlo, const int32_t *dhi,
                             const int32_t *ilo, const int32_t *ihi, const int64_t *tmp_off, const int64_t *off,
                             const int32_t *deg, const int32_t *col, const int32_t *w, int32_t *tcol, int32_t *tw) {
  int64_t nrows = *nrows_p;
  int lane = threadIdx.x & 31;
  int64_t warp = ld_gtid() >> 5, nwarps = ld_gstride() >> 5;
  uint64_t mask = (1ull << vb) - 1;
  for (int64_t r = warp; r < nrows; r += nwarps) {
    int32_t u = rows[r];
    const int32_t *row = col + off[u];
    const int32_t *roww = w + off[u];
    int64_t dg = deg[u];
    const uint64_t *D = dkey + dlo[r];
    int64_t nD = dhi[r] - dlo[r];
    const uint64_t *I = nkey + ilo[r];
    const int64_t *IW = nw + ilo[r];
    int64_t nI = ihi[r] - ilo[r];
    int64_t base = tmp_off[r];
    uint64_t ubase = (uint64_t)u << vb;
    for (int64_t p = lane; p < dg; p += 32) {
      int32_t x = row[p];
      int64_t dless = lower_bound_u64(D, nD, ubase | (uint64_t)x);
      if (dless < nD && (D[dless] & mask) == (uint64_t)x) continue;  // deleted
      int64_t iless = lower_bound_u64(I, nI, ubase | (uint64_t)x);
      int64_t o = base + (p - dless) + iless;
      tcol[o] = x;
      tw[o] = roww[p];
    }
    for (int64_t k = lane; k < nI; k += 32) {
      int32_t y = (int32_t)(I[k] & mask);
      int64_t rless = lower_bound_i32(row, dg, y);
      int64_t dless = lower_bound_u64(D, nD, ubase | (uint64_t)y);
      int64_t o = base + k + (rless - dless);
      tcol[o] = y;
      tw[o] = (int32_t)IW[k];
    }
  }
}

// In-place merge of the touched rows that fit their capacity (no overflow).
// Output position of an old element x at p: p - |D < x| + |I < x|; of the
// k-th new arc y: k + |row < y| - |D < y|.  Rows of at most MERGE_SMALL
// arcs are merged by one warp through shared memory, longer rows by one
// block through the global merge buffer; each writes back after all its
// reads are done, so the old row is never overwritten while still read.
constexpr int MERGE_WARPS = 4;

struct MergeArgs {
  const int32_t *rows;
  const int64_t *nrows_p;
  int vb;
  const uint64_t *dkey, *nkey;
  const int64_t *nw;
  const int32_t *dlo, *dhi, *ilo, *ihi;
  const int64_t *len, *tmp_off, *off;
  int32_t *deg, *col, *w, *tcol, *tw;
  const int64_t *dst;     // where the merged row goes (its old place unless relocated)
  const int32_t *newcap;  // capacity of a relocated row, 0 otherwise
  int64_t *off_w;         // row starts (written after a row is relocated)
  int32_t *rcap;          // row capacities
};

// After the row's reads are done: record a relocation.
__device__ __forceinline__ void finish_row(const MergeArgs &A, int64_t r, int32_t u, int64_t L) {
  A.deg[u] = (int32_t)L;
  if (A.newcap[r]) {
    A.off_w[u] = A.dst[r];
    A.rcap[u] = A.newcap[r];
  }
}

// D, I: the row's deletion keys and new-arc keys (global or staged copies).
__device__ __forceinline__ void merge_row_into(const MergeArgs &A, int64_t r, int t0, int stride, int32_t *ocol,
                                               int32_t *ow, const uint64_t *D, const uint64_t *I) {
  uint64_t mask = (1ull << A.vb) - 1;
  int32_t u = A.rows[r];
  const int32_t *row = A.col + A.off[u];
  const int32_t *roww = A.w + A.off[u];
  int64_t dg = A.deg[u];
  int64_t nD = A.dhi[r] - A.dlo[r];
  const int64_t *IW = A.nw + A.ilo[r];
  int64_t nI = A.ihi[r] - A.ilo[r];
  uint64_t ubase = (uint64_t)u << A.vb;
  for (int64_t p = t0; p < dg; p += stride) {
    int32_t x = row[p];
    int64_t dless = nD ? lower_bound_u64(D, nD, ubase | (uint64_t)x) : 0;
    if (dless < nD && (D[dless] & mask) == (uint64_t)x) continue;
    int64_t iless = nI ? lower_bound_u64(I, nI, ubase | (uint64_t)x) : 0;
    int64_t o = (p - dless) + iless;
    ocol[o] = x;
    ow[o] = roww[p];
  }
  for (int64_t k = t0; k < nI; k += stride) {
    int32_t y = (int32_t)(I[k] & mask);
    int64_t rless = lower_bound_i32(row, dg, y);
    int64_t dless = nD ? lower_bound_u64(D, nD, ubase | (uint64_t)y) : 0;
    int64_t o = k + (rless - dless);
    ocol[o] = y;
    ow[o] = (int32_t)IW[k];
  }
}

__global__ void __launch_bounds__(MERGE_WARPS * 32) k_merge_small(MergeArgs A) {
  __shared__ int32_t scol[MERGE_WARPS][MERGE_SMALL];
  __shared__ int32_t sw[MERGE_WARPS][MERGE_SMALL];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t nrows = *A.nrows_p;
  for (int64_t r = (int64_t)blockIdx.x * MERGE_WARPS + wid; r < nrows; r += (int64_t)gridDim.x * MERGE_WARPS) {
    int64_t L = A.len[r];
    if (L > MERGE_SMALL) continue;
    merge_row_into(A, r, lane, 32, scol[wid], sw[wid], A.dkey + A.dlo[r], A.nkey + A.ilo[r]);
    __syncwarp();
    int32_t u = A.rows[r];
    int64_t o = A.dst[r];
    for (int64_t x = lane; x < L; x += 32) { A.col[o + x] = scol[wid][x]; A.w[o + x] = sw[wid][x]; }
    if (lane == 0) finish_row(A, r, u, L);
    __syncwarp();
  }
}

// Rows of MERGE_SMALL..MERGE_MID arcs: one block each, staged in shared
// memory and written back after all of the row's reads.
__global__ void __launch_bounds__(256) k_merge_mid(MergeArgs A, const int32_t *mid, const int32_t *count_p,
                                                   int64_t *xk_bytes) {
  __shared__ int32_t scol[MERGE_MID];
  __shared__ int32_t sw[MERGE_MID];
  int64_t count = *count_p;
  int64_t bytes = 0;  // algorithmic bytes (thread 0): old row read, new row written, the row's batch arcs
  for (int64_t k = blockIdx.x; k < count; k += gridDim.x) {
    int64_t r = mid[k];
    int64_t L = A.len[r];
    int32_t u = A.rows[r];
    if (threadIdx.x == 0) bytes += 8 * ((int64_t)A.deg[u] + L) + 16 * (A.dhi[r] - A.dlo[r] + A.ihi[r] - A.ilo[r]);
    merge_row_into(A, r, threadIdx.x, blockDim.x, scol, sw, A.dkey + A.dlo[r], A.nkey + A.ilo[r]);
    __syncthreads();
    int64_t o = A.dst[r];
    for (int64_t x = threadIdx.x; x < L; x += blockDim.x) { A.col[o + x] = scol[x]; A.w[o + x] = sw[x]; }
    if (threadIdx.x == 0) finish_row(A, r, u, L);
    __syncthreads();
  }
  if (threadIdx.x == 0 && bytes) atomicAdd((unsigned long long *)xk_bytes, (unsigned long long)bytes);
}

// Long rows in chunks any block may take (items k of `large`, chunk offsets
// ch_off over the old row): elements go to the merge buffer by rank; the
// first chunk of a row also places its new arcs.
__global__ void __launch_bounds__(256) k_merge_chunks_write(MergeArgs A, const int32_t *large,
                                                            const int32_t *count_p, const int64_t *ch_off) {
  int64_t count = *count_p;
  int64_t nch = ch_off[count];
  uint64_t mask = (1ull << A.vb) - 1;
  for (int64_t t = blockIdx.x; t < nch; t += gridDim.x) {
    int64_t lo = 0, hi = count - 1;
    while (lo < hi) {
      int64_t mid = (lo + hi + 1) >> 1;
      if (ch_off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    int64_t r = large[lo];
    int32_t u = A.rows[r];
    const int32_t *row = A.col + A.off[u];
    const int32_t *roww = A.w + A.off[u];
    int64_t dg = A.deg[u];
    const uint64_t *D = A.dkey + A.dlo[r];
    int64_t nD = A.dhi[r] - A.dlo[r];
    const uint64_t *I = A.nkey + A.ilo[r];
    const int64_t *IW = A.nw + A.ilo[r];
    int64_t nI = A.ihi[r] - A.ilo[r];
    uint64_t ubase = (uint64_t)u << A.vb;
    int32_t *ocol = A.tcol + A.tmp_off[r];
    int32_t *ow = A.tw + A.tmp_off[r];
    int64_t c = t - ch_off[lo];
    int64_t p0 = c * TABLE_CHUNK, p1 = p0 + TABLE_CHUNK < dg ? p0 + TABLE_CHUNK : dg;
    for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
      int32_t x = row[p];
      int64_t dless = nD ? lower_bound_u64(D, nD, ubase | (uint64_t)x) : 0;
      if (dless < nD && (D[dless] & mask) == (uint64_t)x) continue;
      int64_t iless = nI ? lower_bound_u64(I, nI, ubase | (uint64_t)x) : 0;
      int64_t o = (p - dless) + iless;
      ocol[o] = x;
      ow[o] = roww[p];
    }
    if (c == 0) {
      for (int64_t k = threadIdx.x; k < nI; k += blockDim.x) {
        int32_t y = (int32_t)(I[k] & mask);
        int64_t rless = lower_bound_i32(row, dg, y);
        int64_t dless = nD ? lower_bound_u64(D, nD, ubase | (uint64_t)y) : 0;
        int64_t o = k + (rless - dless);
        ocol[o] = y;
        ow[o] = (int32_t)IW[k];
      }
    }
  }
}

// Copy the merged long rows back (chunks over the new length) and record
// the new degree and any relocation.
__global__ void __launch_bounds__(256) k_merge_chunks_copy(MergeArgs A, const int32_t *large,
                                                           const int32_t *count_p, const int64_t *ch_off) {
  int64_t count = *count_p;
  int64_t nch = ch_off[count];
  for (int64_t t = blockIdx.x; t < nch; t += gridDim.x) {
    int64_t lo = 0, hi = count - 1;
    while (lo < hi) {
      int64_t mid = (lo + hi + 1) >> 1;
      if (ch_off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    int64_t r = large[lo];
    int64_t L = A.len[r];
    int64_t c = t - ch_off[lo];
    int64_t x0 = c * TABLE_CHUNK, x1 = x0 + TABLE_CHUNK < L ? x0 + TABLE_CHUNK : L;
    int64_t b = A.tmp_off[r], o = A.dst[r];
    for (int64_t x = x0 + threadIdx.x; x < x1; x += blockDim.x) {
      A.col[o + x] = A.tcol[b + x];
      A.w[o + x] = A.tw[b + x];
    }
    if (c == 0 && threadIdx.x == 0) finish_row(A, r, A.rows[r], L);
  }
}

// ----- rebuild with fresh slack (when a row outgrows its capacity)
__global__ void k_row_lengths(const int32_t *deg, int64_t n, int64_t *len) {
  for (int64_t i = ld_gtid(); i < n; i += ld_gstride()) len[i] = deg[i];
}
__global__ void k_touched_lengths(const int32_t *rows, const int64_t *nrows_p, const int64_t *rlen, int64_t *len) {
  for (int64_t r = ld_gtid(); r < *nrows_p; r += ld_gstride()) len[rows[r]] = rlen[r];
}
__global__ void k_capacity(const int64_t *len, int64_t n, double slack, int min_slack, int64_t *cap) {
  for (int64_t i = ld_gtid(); i < n; i += ld_gstride()) {
    int64_t L = len[i];
    int64_t extra = (int64_t)((double)L * slack);
    if (extra < min_slack) extra = min_slack;
    cap[i] = L + extra;
  }
}
// rowsrc[i] = index into the touched-row list, or -1
__global__ void k_copy_rows_rebuild(int64_t n, const int64_t *old_off, const int32_t *old_deg, const int32_t *old_col,
                                    const int32_t *old_w, const int32_t *rowsrc, const int64_t *tmp_off,
                                    const int64_t *rlen, const int32_t *tcol, const int32_t *tw,
                                    const int64_t *new_off, int32_t *new_deg, int32_t *new_col, int32_t *new_w) {
  int lane = threadIdx.x & 31;
  int64_t warp = ld_gtid() >> 5, nwarps = ld_gstride() >> 5;
  for (int64_t u = warp; u < n; u += nwarps) {
    int32_t r = rowsrc ? rowsrc[u] : -1;
    const int32_t *sc, *sw;
    int64_t L;
    if (r >= 0) { sc = tcol + tmp_off[r]; sw = tw + tmp_off[r]; L = rlen[r]; }
    else { sc = old_col + old_off[u]; sw = old_w + old_off[u]; L = old_deg[u]; }
    int64_t o = new_off[u];
    for (int64_t x = lane; x < L; x += 32) { new_col[o + x] = sc[x]; new_w[o + x] = sw[x]; }
    if (lane == 0) new_deg[u] = (int32_t)L;
  }
}
__global__ void k_set_rcap(const int64_t *cap, int64_t n, int32_t *rcap) {
  for (int64_t i = ld_gtid(); i < n; i += ld_gstride()) rcap[i] = (int32_t)cap[i];
}
__global__ void k_rowsrc(const int32_t *rows, const int64_t *nrows_p, int32_t *rowsrc) {
  for (int64_t r = ld_gtid(); r < *nrows_p; r += ld_gstride()) rowsrc[rows[r]] = (int32_t)r;
}

// ----- marking (uses C^{t-1}, and K^{t-1}, Sigma^{t-1}, 2m^{t-1} for DS)
__global__ void k_mark_df(const uint64_t *dkey, int64_t nd, const uint64_t *ikey, int64_t ni, int vb,
                          const int32_t *C, uint8_t *dV) {
  uint64_t mask = (1ull << vb) - 1;
  for (int64_t i = ld_gtid(); i < nd + ni; i += ld_gstride()) {
    bool del = i < nd;
    uint64_t k = del ? dkey[i] : ikey[i - nd];
    int32_t u = (int32_t)(k >> vb), v = (int32_t)(k & mask);
    bool same = C[u] == C[v];
    if (del ? same : !same) dV[u] = 1;
  }
}

__global__ void k_mark_ds_del(const uint64_t *dkey, int64_t nd, int vb, const int32_t *C, uint8_t *dV, uint8_t *dE,
                              uint8_t *dCf) {
  uint64_t mask = (1ull << vb) - 1;
  for (int64_t i = ld_gtid(); i < nd; i += ld_gstride()) {
    int32_t u = (int32_t)(dkey[i] >> vb), v = (int32_t)(dkey[i] & mask);
    if (C[u] == C[v]) { dV[u] = 1; dE[u] = 1; dCf[C[v]] = 1; }
  }
}

// (src, C[dst]) keys of the cross-community insertions; same-community
// arcs get the key ~0 and sort last.
__global__ void k_ds_keys(const uint64_t *ikey, const int64_t *iw, int64_t ni, int vb, const int32_t *C,
                          uint64_t *okey, int64_t *ow) {
  uint64_t mask = (1ull << vb) - 1;
  for (int64_t i = ld_gtid(); i < ni; i += ld_gstride()) {
    int32_t u = (int32_t)(ikey[i] >> vb), v = (int32_t)(ikey[i] & mask);
    if (C[u] != C[v]) { okey[i] = ((uint64_t)u << vb) | (uint64_t)C[v]; ow[i] = iw[i]; }
    else { okey[i] = ~0ull; ow[i] = 0; }
  }
}

// Sorted unique (src, c) pairs with summed weights H; warp per source run:
// c* = argmax 2m*H[c] - K_src*Sigma_c, ties to the lowest c.
__global__ void k_ds_best(const uint64_t *pkey, const int64_t *pw, const int64_t *np_p, int vb, const int64_t *K,
                          const int64_t *Sig, const DevCounters *cnt, uint8_t *dV, uint8_t *dE, uint8_t *dCf,
                          const int32_t *gid0, const int64_t *m2g) {
  int64_t np = *np_p;
  uint64_t mask = (1ull << vb) - 1;
  for (int64_t i = ld_gtid(); i < np; i += ld_gstride()) {
    if (pkey[i] == ~0ull) continue;
    uint64_t src = pkey[i] >> vb;
    if (i > 0 && (pkey[i - 1] >> vb) == src) continue;  // only the run head works
    int64_t m2 = gid0 ? m2g[gid0[src]] : cnt->m2;  // 2m^{t-1} of the source's graph
    int32_t best = -1;
    i128 bv = 0;
    for (int64_t j = i; j < np && pkey[j] != ~0ull && (pkey[j] >> vb) == src; j++) {
      int32_t c = (int32_t)(pkey[j] & mask);
      i128 v = (i128)m2 * pw[j] - (i128)K[src] * Sig[c];
      if (ld_better(v, c, bv, best)) { bv = v; best = c; }
    }
    dV[src] = 1; dE[src] = 1; dCf[best] = 1;
  }
}

// Warp per vertex with dE: neighbours of G^t become affected.
__global__ void k_ds_expand_neighbours(const uint8_t *dE, int64_t n, const int64_t *off, const int32_t *deg,
                                       const int32_t *col, uint8_t *dV) {
  int lane = threadIdx.x & 31;
  int64_t warp = ld_gtid() >> 5, nwarps = ld_gstride() >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    if (!dE[i]) continue;
    for (int64_t a = lane; a < deg[i]; a += 32) dV[col[off[i] + a]] = 1;
  }
}
__global__ void k_ds_expand_communities(const uint8_t *dCf, const int32_t *C, int64_t n, uint8_t *dV) {
  for (int64_t i = ld_gtid(); i < n; i += ld_gstride())
    if (dCf[C[i]]) dV[i] = 1;
}

// Alg. update (updateWeights, updateChanges) on both arc lists.
__global__ void k_update_weights(const uint64_t *dkey, const int64_t *dw, int64_t nd, const uint64_t *ikey,
                                 const int64_t *iw, int64_t ni, int vb, const int32_t *C, int64_t *K, int64_t *Sig,
                                 int64_t *dSig, DevCounters *cnt, const int32_t *gid0, int64_t *m2g) {
  int64_t acc = 0;
  for (int64_t i0 = (ld_gtid() & ~31ll); i0 < nd + ni; i0 += ld_gstride()) {  // warp-uniform trip count
    int64_t i = i0 + (threadIdx.x & 31);
    bool has = i < nd + ni;
    int64_t s = 0;
    int32_t u = 0;
    if (has) {
      bool del = i < nd;
      uint64_t k = del ? dkey[i] : ikey[i - nd];
      int64_t w = del ? dw[i] : iw[i - nd];
      u = (int32_t)(k >> vb);
      int32_t c = C[u];
      s = del ? -w : w;
      atomicAdd((unsigned long long *)&K[u], (unsigned long long)s);
      atomicAdd((unsigned long long *)&Sig[c], (unsigned long long)s);
      atomicAdd((unsigned long long *)&dSig[c], (unsigned long long)w);
      acc += s;
    }
    // batched: 2m per graph (a signed sum; the helper adds two's-complement values)
    if (gid0) ld_graph_add_i64(m2g, has, has ? gid0[u] : 0, s);
  }
  acc = ld_warp_sum_i64(acc);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd((unsigned long long *)&cnt->m2, (unsigned long long)acc);
}

// Alg. leidenmk: dS for same-community deletions; dR for same-community
// arcs of either list with dSigma/Sigma > tau_re.
__global__ void k_mark_communities(const uint64_t *dkey, int64_t nd, const uint64_t *ikey, int64_t ni, int vb,
                                   const int32_t *C, const int64_t *Sig, const int64_t *dSig, double tau_re,
                                   uint8_t *dS, uint8_t *dR) {
  uint64_t mask = (1ull << vb) - 1;
  for (int64_t i = ld_gtid(); i < nd + ni; i += ld_gstride()) {
    bool del = i < nd;
    uint64_t k = del ? dkey[i] : ikey[i - nd];
    int32_t u = (int32_t)(k >> vb), v = (int32_t)(k & mask);
    int32_t c = C[u];
    if (c != C[v]) continue;
    if (del) dS[c] = 1;
    if ((double)dSig[c] / (double)Sig[c] > tau_re) dR[c] = 1;
  }
}
__global__ void k_reset_changes(const uint64_t *dkey, int64_t nd, const uint64_t *ikey, int64_t ni, int vb,
                                const int32_t *C, const uint8_t *dR, int64_t *dSig) {
  for (int64_t i = ld_gtid(); i < nd + ni; i += ld_gstride()) {
    uint64_t k = i < nd ? dkey[i] : ikey[i - nd];
    int32_t c = C[(int32_t)(k >> vb)];
    if (dR[c]) dSig[c] = 0;
  }
}

int bits_for(int64_t n) {
  int b = 1;
  while (((int64_t)1 << b) < n) b++;
  return b;
}

template <typename T>
cudaError_t grow(leiden_handle *h, T **p, int64_t count) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, (size_t)std::max<int64_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  h->owned.push_back(q);
  *p = (T *)q;
  return cudaSuccess;
}

void release(leiden_handle *h, void *p) {
  if (!p) return;
  for (auto &q : h->owned)
    if (q == p) { cudaFree(q); q = nullptr; }
}

// Buffers that grow with the batch.  A larger set is allocated in full
// before the old one is freed: a failed allocation leaves the handle with its
// old, valid buffers and capacity (and frees what it got).
cudaError_t ensure_batch(leiden_handle *h, int64_t edges) {
  BatchBuffers &b = h->b;
  if (b.cap_edges > 0 && edges <= b.cap_edges) return cudaSuccess;  // the first call always allocates
  // geometric growth: a freed buffer synchronises the whole device, which
  // stalls every other stream of a serving process
  int64_t cap = std::max<int64_t>({edges, 2 * b.cap_edges, (int64_t)1024});
  int64_t arcs = 2 * cap;
  int64_t rows = std::min<int64_t>(2 * arcs, h->n) + 1;
  BatchBuffers nb = b;
  void **slot[] = {(void **)&nb.dkey, (void **)&nb.dkey_alt, (void **)&nb.ikey, (void **)&nb.ikey_alt,
                   (void **)&nb.iw, (void **)&nb.iw_alt, (void **)&nb.dw, (void **)&nb.flag, (void **)&nb.pos,
                   (void **)&nb.ins_state, (void **)&nb.ins_pos, (void **)&nb.rows, (void **)&nb.row_dlo,
                   (void **)&nb.row_dhi, (void **)&nb.row_ilo, (void **)&nb.row_ihi, (void **)&nb.row_len,
                   (void **)&nb.row_tmp_off, (void **)&nb.row_dst, (void **)&nb.row_newcap, (void **)&nb.row_olddeg,
                   (void **)&nb.row_large, (void **)&nb.row_mid, (void **)&nb.ds_key, (void **)&nb.ds_key_alt,
                   (void **)&nb.ds_w, (void **)&nb.ds_w_alt, (void **)&nb.ds_ukey, (void **)&nb.ds_uw};
  // dkey, dkey_alt, iw and iw_alt hold the deletion and insertion arcs of
  // one sort together (2 * arcs); ikey, ikey_alt and iw_alt's unique part
  // at most one kind
  size_t bytes[] = {16 * (size_t)arcs, 16 * (size_t)arcs, 8 * (size_t)arcs, 8 * (size_t)arcs, 16 * (size_t)arcs,
                    16 * (size_t)arcs, 8 * (size_t)arcs, 4 * (size_t)(arcs + 1), 8 * (size_t)(arcs + 1),
                    4 * (size_t)arcs, 8 * (size_t)arcs, 4 * (size_t)rows, 4 * (size_t)rows, 4 * (size_t)rows,
                    4 * (size_t)rows, 4 * (size_t)rows, 8 * (size_t)(rows + 1), 8 * (size_t)(rows + 1),
                    8 * (size_t)(rows + 1), 4 * (size_t)(rows + 1), 4 * (size_t)(rows + 1), 4 * (size_t)(rows + 1),
                    4 * (size_t)(rows + 1), 8 * (size_t)arcs, 8 * (size_t)arcs, 8 * (size_t)arcs, 8 * (size_t)arcs,
                    8 * (size_t)arcs, 8 * (size_t)arcs};
  constexpr int NB = sizeof(slot) / sizeof(slot[0]);
  static_assert(NB == sizeof(bytes) / sizeof(bytes[0]), "one size per batch buffer");
  void *fresh[NB] = {};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < NB && e == cudaSuccess; k++) e = cudaMalloc(&fresh[k], bytes[k]);
  if (e == cudaSuccess && !b.row_bits) {
    int64_t words = (h->n + 31) / 32;
    e = grow(h, &nb.row_bits, words);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(nb.row_bits, 0, (size_t)std::max<int64_t>(words, 1) * sizeof(uint32_t), h->stream);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    for (void *q : fresh)
      if (q) cudaFree(q);
    return e;
  }
  void *old[NB];
  for (int k = 0; k < NB; k++) {
    old[k] = *slot[k];
    *slot[k] = fresh[k];
    h->owned.push_back(fresh[k]);
  }
  for (void *q : old) release(h, q);
  nb.counts = h->dcnt->bcounts;
  nb.cap_edges = cap;
  b = nb;
  return cudaSuccess;
}

cudaError_t ensure_scan_tmp(leiden_handle *h, size_t bytes) {
  if (bytes <= h->scan_tmp_bytes) return cudaSuccess;
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) { cudaGetLastError(); return e; }  // the old scratch stays
  release(h, h->scan_tmp);
  h->owned.push_back(p);
  h->scan_tmp = p;
  h->scan_tmp_bytes = bytes;
  return cudaSuccess;
}

cudaError_t ensure_tmp_rows(leiden_handle *h, int64_t arcs) {
  BatchBuffers &b = h->b;
  if (arcs <= b.tmp_cap) return cudaSuccess;
  int64_t cap = std::max<int64_t>({arcs, 2 * b.tmp_cap, (int64_t)4096});
  int32_t *col = nullptr, *w = nullptr;
  cudaError_t e = cudaMalloc((void **)&col, (size_t)cap * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc((void **)&w, (size_t)cap * sizeof(int32_t));
  if (e != cudaSuccess) {  // the old buffers stay
    cudaGetLastError();
    if (col) cudaFree(col);
    return e;
  }
  release(h, b.tmp_col);
  release(h, b.tmp_w);
  h->owned.push_back(col);
  h->owned.push_back(w);
  b.tmp_col = col;
  b.tmp_w = w;
  b.tmp_cap = cap;
  return cudaSuccess;
}

leiden_status fail(leiden_handle *h, leiden_status st, const std::string &msg) {
  h->err = msg;
  return st;
}

}  // namespace

// Rebuild G^t with new capacities: rows keep their content (touched rows
// come from the merge buffer).
static leiden_status rebuild_graph(leiden_handle *h, int64_t nrows_host, const int64_t *nrows_dev) {
  cudaStream_t s = h->stream;
  int64_t n = h->n;
  BatchBuffers &b = h->b;
  int64_t *len = h->lbuf0, *cap = h->lbuf1;
  ld_note_launch(), k_row_lengths<<<grid_for(n, TB), TB, 0, s>>>(h->g_deg, n, len);
  ld_note_launch(), k_touched_lengths<<<grid_for(nrows_host, TB), TB, 0, s>>>(b.rows, nrows_dev, b.row_len, len);
  ld_note_launch(), k_capacity<<<grid_for(n, TB), TB, 0, s>>>(len, n, h->p.slack, h->p.min_slack, cap);
  int64_t *new_off = nullptr;
  if (grow(h, &new_off, n + 1) != cudaSuccess) return fail(h, LEIDEN_ERR_OOM, "rebuild: offsets");
  if (ensure_scan_tmp(h, scan_tmp_bytes(n + 1)) != cudaSuccess) return fail(h, LEIDEN_ERR_OOM, "scan tmp");
  exclusive_scan_i64(cap, new_off, n, h->scan_tmp, s);
  int64_t used = 0;
  cudaMemcpyAsync(&used, new_off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  int64_t total = used + spill_arena_size(used, h->p.arena_log2);
  int32_t *new_col = nullptr, *new_w = nullptr, *new_deg = nullptr;
  if (grow(h, &new_col, total) != cudaSuccess || grow(h, &new_w, total) != cudaSuccess ||
      grow(h, &new_deg, n) != cudaSuccess)
    return fail(h, LEIDEN_ERR_OOM, "rebuild: arcs");
  ld_note_launch(), k_set_rcap<<<grid_for(n, TB), TB, 0, s>>>(cap, n, h->g_rcap);
  cudaMemcpyAsync(&h->dcnt->arena_used, &used, sizeof(int64_t), cudaMemcpyHostToDevice, s);
  int32_t *rowsrc = h->ibuf2;
  launch_fill_i32(rowsrc, -1, n, s);
  ld_note_launch(), k_rowsrc<<<grid_for(nrows_host, TB), TB, 0, s>>>(b.rows, nrows_dev, rowsrc);
  ld_note_launch(), k_copy_rows_rebuild<<<grid_for(n * 32, TB), TB, 0, s>>>(n, h->g_off, h->g_deg, h->g_col, h->g_w, rowsrc,
                                                          b.row_tmp_off, b.row_len, b.tmp_col, b.tmp_w, new_off,
                                                          new_deg, new_col, new_w);
  cudaStreamSynchronize(s);
  release(h, h->g_off);
  release(h, h->g_col);
  release(h, h->g_w);
  release(h, h->g_deg);
  h->g_off = new_off;
  h->g_col = new_col;
  h->g_w = new_w;
  h->g_deg = new_deg;
  h->g_cap = total;
  return LEIDEN_OK;
}

leiden_status batch_apply_and_mark(leiden_handle *h, const leiden_edge *d_del, int64_t n_del,
                                   const leiden_edge *d_ins, int64_t n_ins, int mode) {
  cudaStream_t s = h->stream;
  int64_t n = h->n;
  BatchBuffers &b = h->b;
  int vb = bits_for(n);
  DevCounters *cnt = h->dcnt;
  if (ensure_batch(h, std::max(n_del, n_ins)) != cudaSuccess) return fail(h, LEIDEN_ERR_OOM, "batch buffers");
  int64_t nda = 2 * n_del, nia = 2 * n_ins;
  if (ensure_scan_tmp(h, std::max(sort_tmp_bytes(nda + nia), scan_tmp_bytes(n + 1))) != cudaSuccess)
    return fail(h, LEIDEN_ERR_OOM, "scan tmp");
  cudaMemsetAsync(&cnt->error, 0, sizeof(int32_t), s);
  cudaMemsetAsync(&cnt->overflow, 0, sizeof(int32_t), s);
  cudaMemsetAsync(&cnt->large_count, 0, sizeof(int32_t), s);
  cudaMemsetAsync(&cnt->mid_count, 0, sizeof(int32_t), s);
  // one sort of both: the deletion arcs sorted in dkey[0, nda), the
  // insertion arcs and their weights in dkey, iw [nda, nda + nia)
  if (n_del + n_ins > 0)
    ld_note_launch(), k_expand<<<grid_for(n_del + n_ins, TB), TB, 0, s>>>(d_del, n_del, d_ins, n_ins, n, vb, b.dkey,
                                                                          b.iw, cnt, h->gid0);
  radix_sort_u64(b.dkey, b.dkey_alt, b.iw, b.iw_alt, nda + nia, 2 * vb + 1, h->scan_tmp, s);
  uint64_t *SD = b.dkey, *SI = b.dkey + nda;
  int64_t *SIW = b.iw + nda;
  if (nia > 0) ld_note_launch(), k_untag<<<grid_for(nia, TB), TB, 0, s>>>(SI, nia, (1ull << (2 * vb)) - 1);
  // deduplicate: deletions collapse (-> DK), insertions add up (-> IK, IW).
  // The counts stay on the device until the one host read below: launches
  // are sized by the bounds nda, nia and read the counts themselves.
  int64_t *counts = b.counts;  // [0] nd, [1] ni, [2] new arcs, [3] touched rows, [4] merge-buffer arcs
  cudaMemsetAsync(counts, 0, 8 * sizeof(int64_t), s);
  uint64_t *DK = b.dkey_alt, *IK = b.ikey_alt;
  int64_t *IW = b.iw_alt, *DW = b.dw;
  if (nda > 0) {
    ld_note_launch(), k_head_flags<<<grid_for(nda, TB), TB, 0, s>>>(SD, nda, b.flag);
    exclusive_scan_i32_to_i64(b.flag, b.pos, nda, h->scan_tmp, s);
    ld_note_launch(), k_unique<<<grid_for(nda, TB), TB, 0, s>>>(SD, nullptr, nda, b.flag, b.pos, DK, nullptr);
    cudaMemcpyAsync(counts + 0, b.pos + nda, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
  }
  if (nia > 0) {
    ld_note_launch(), k_head_flags<<<grid_for(nia, TB), TB, 0, s>>>(SI, nia, b.flag);
    exclusive_scan_i32_to_i64(b.flag, b.pos, nia, h->scan_tmp, s);
    cudaMemsetAsync(IW, 0, (size_t)nia * sizeof(int64_t), s);
    ld_note_launch(), k_unique<<<grid_for(nia, TB), TB, 0, s>>>(SI, SIW, nia, b.flag, b.pos, IK, IW);
    cudaMemcpyAsync(counts + 1, b.pos + nia, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
  }
  // deletions must exist (stored weight -> DW); insertions: existing or new
  if (nda > 0)
    ld_note_launch(), k_check_deletions<<<grid_for(nda, TB), TB, 0, s>>>(DK, counts + 0, vb, h->g_off, h->g_deg,
                                                                         h->g_col, h->g_w, DW, cnt);
  uint64_t *NK = b.ikey;  // new insertions, compacted in sorted order
  int64_t *NW = b.iw;      // (the sorted raw arcs there are consumed by then)
  if (nia > 0) {
    ld_note_launch(), k_classify_insertions<<<grid_for(nia, TB), TB, 0, s>>>(IK, counts + 1, DK, counts + 0, vb,
                                                                             h->g_off, h->g_deg, h->g_col,
                                                                             b.ins_state, b.ins_pos);
    ld_note_launch(), k_new_flags<<<grid_for(nia, TB), TB, 0, s>>>(b.ins_state, counts + 1, nia, b.flag);
    exclusive_scan_i32_to_i64(b.flag, b.pos, nia, h->scan_tmp, s);
    ld_note_launch(), k_compact_new<<<grid_for(nia, TB), TB, 0, s>>>(IK, IW, nia, b.flag, b.pos, NK, NW);
    cudaMemcpyAsync(counts + 2, b.pos + nia, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
  }
  // rows whose structure changes: sources of deletions and of new arcs
  int64_t nb = std::min<int64_t>(n, nda + nia);  // bound on the touched rows
  if (nb > 0) {
    ld_note_launch(), k_touched_rows<<<grid_for(nda + nia, TB), TB, 0, s>>>(DK, counts + 0, NK, counts + 2, vb,
                                                                            b.row_bits, b.rows, counts + 3);
    ld_note_launch(), k_clear_row_bits<<<grid_for(nb, TB), TB, 0, s>>>(b.rows, counts + 3, b.row_bits);
    ld_note_launch(), k_row_plan<<<grid_for(nb, TB), TB, 0, s>>>(
        b.rows, counts + 3, nb, vb, DK, counts + 0, NK, counts + 2, h->g_off, h->g_deg, h->g_rcap, b.row_dlo,
        b.row_dhi, b.row_ilo, b.row_ihi, b.row_len, b.row_dst, b.row_newcap, h->p.slack, h->p.min_slack, h->g_cap,
        b.row_olddeg, b.row_large, b.row_mid, cnt);
    exclusive_scan_i64(b.row_len, b.row_tmp_off, nb, h->scan_tmp, s);
    cudaMemcpyAsync(counts + 4, b.row_tmp_off + nb, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
  }
  // the one host read before the graph changes: counts, validation, overflow
  cudaMemcpyAsync(h->hcnt, h->dcnt, sizeof(DevCounters), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  if (h->hcnt->error)
    return fail(h, LEIDEN_ERR_BATCH, h->hcnt->error == 2 ? "batch deletes an edge that does not exist"
                                                         : "batch edge out of range, self-loop or weight <= 0");
  const int64_t *hc = h->hcnt->bcounts;
  int64_t nd = hc[0], ni = hc[1], nn = hc[2], nrows = hc[3], tmp_total = hc[4];
  bool overflow = nrows > 0 && h->hcnt->overflow != 0;
  if (ensure_tmp_rows(h, tmp_total) != cudaSuccess) return fail(h, LEIDEN_ERR_OOM, "merge buffer");
  // ---- apply: from here on the handle changes
  if (ni > 0) ld_note_launch(), k_add_existing<<<grid_for(ni, TB), TB, 0, s>>>(b.ins_pos, b.ins_state, IW, ni, h->g_w);
  if (nrows > 0) {
    if (!overflow) {
      MergeArgs M{b.rows, counts + 3, vb, DK, NK, NW, b.row_dlo, b.row_dhi, b.row_ilo, b.row_ihi, b.row_len,
                  b.row_tmp_off, h->g_off, h->g_deg, h->g_col, h->g_w, b.tmp_col, b.tmp_w,
                  b.row_dst, b.row_newcap, h->g_off, h->g_rcap};
      // the three row classes write disjoint rows and merge-buffer ranges:
      // short rows on the handle's stream, mid rows and long rows on its
      // side streams, joined before the marking below
      bool fork = h->tune.overlap && side_streams(h);
      cudaStream_t smid = s, slong = s;
      if (fork) {
        cudaEventRecord(h->fork_ev, s);
        smid = h->side[0];
        slong = h->side[1];
        cudaStreamWaitEvent(smid, h->fork_ev, 0);
        cudaStreamWaitEvent(slong, h->fork_ev, 0);
      }
      ld_note_launch(), k_merge_small<<<grid_for((nrows + MERGE_WARPS - 1) / MERGE_WARPS, 1, h->sm_count * 16), MERGE_WARPS * 32, 0,
                      s>>>(M);
      kt_begin(h, KT_MERGE_MID, smid);
      ld_note_launch(), k_merge_mid<<<h->sm_count * 7, 256, 0, smid>>>(M, b.row_mid, &cnt->mid_count,  // 32 KB: 7 per SM
                                                                      &cnt->xk_bytes[2]);
      kt_end(h, smid);
      // long rows: chunks over the old row, then chunks over the new row
      int32_t *large = b.row_large;
      const int32_t *nlarge = &cnt->large_count;
      launch_table_plan(large, nlarge, b.row_olddeg, nullptr, INT64_MAX, h->lbuf0, h->lbuf1, slong);
      ld_note_launch(), k_merge_chunks_write<<<h->sm_count * 16, 256, 0, slong>>>(M, large, nlarge, h->lbuf1);
      launch_table_plan(large, nlarge, nullptr, b.row_tmp_off, INT64_MAX, h->lbuf2, h->lbuf3, slong);
      ld_note_launch(), k_merge_chunks_copy<<<h->sm_count * 16, 256, 0, slong>>>(M, large, nlarge, h->lbuf3);
      if (fork) {
        for (int k = 0; k < 2; k++) {
          cudaEventRecord(h->join_ev[k], h->side[k]);
          cudaStreamWaitEvent(s, h->join_ev[k], 0);
        }
      }
    } else {
      ld_note_launch(), k_merge_rows<<<grid_for(nrows * 32, TB), TB, 0, s>>>(b.rows, counts + 3, vb, DK, NK, NW, b.row_dlo,
                                                           b.row_dhi, b.row_ilo, b.row_ihi, b.row_tmp_off, h->g_off,
                                                           h->g_deg, h->g_col, h->g_w, b.tmp_col, b.tmp_w);
      leiden_status st = rebuild_graph(h, nrows, counts + 3);
      h->stats.rebuilds++;
      if (st != LEIDEN_OK) {
        h->broken = true;  // the batch was applied in part
        return st;
      }
    }
  }
  h->g_arcs = h->g_arcs - nd + nn;
  h->stats.batch_arcs = nd + ni;
  // ---- affected vertices (C^{t-1}; DS also K^{t-1}, Sigma^{t-1}, 2m^{t-1})
  uint8_t *dV = h->dV;
  if (mode == LEIDEN_ND) {
    cudaMemsetAsync(dV, 1, (size_t)n, s);
  } else {
    cudaMemsetAsync(dV, 0, (size_t)n, s);
    if (mode == LEIDEN_DF) {
      if (nd + ni > 0) ld_note_launch(), k_mark_df<<<grid_for(nd + ni, TB), TB, 0, s>>>(DK, nd, IK, ni, vb, h->C, dV);
    } else {
      cudaMemsetAsync(h->dE, 0, (size_t)n, s);
      cudaMemsetAsync(h->dCf, 0, (size_t)n, s);
      if (nd > 0) ld_note_launch(), k_mark_ds_del<<<grid_for(nd, TB), TB, 0, s>>>(DK, nd, vb, h->C, dV, h->dE, h->dCf);
      if (ni > 0) {
        // H of each insertion source: (src, C[dst]) pairs, sorted, runs summed
        ld_note_launch(), k_ds_keys<<<grid_for(ni, TB), TB, 0, s>>>(IK, IW, ni, vb, h->C, b.ds_key, b.ds_w);
        radix_sort_u64(b.ds_key, b.ds_key_alt, b.ds_w, b.ds_w_alt, ni, 64, h->scan_tmp, s);
        ld_note_launch(), k_head_flags<<<grid_for(ni, TB), TB, 0, s>>>(b.ds_key, ni, b.flag);
        exclusive_scan_i32_to_i64(b.flag, b.pos, ni, h->scan_tmp, s);
        cudaMemsetAsync(b.ds_uw, 0, (size_t)ni * sizeof(int64_t), s);
        ld_note_launch(), k_unique<<<grid_for(ni, TB), TB, 0, s>>>(b.ds_key, b.ds_w, ni, b.flag, b.pos, b.ds_ukey, b.ds_uw);
        ld_note_launch(), k_ds_best<<<grid_for(ni, TB), TB, 0, s>>>(b.ds_ukey, b.ds_uw, b.pos + ni, vb, h->K, h->Sig, cnt, dV, h->dE,
                                                  h->dCf, h->gid0, h->gc.m2);
      }
      ld_note_launch(), k_ds_expand_neighbours<<<grid_for(n * 32, TB), TB, 0, s>>>(h->dE, n, h->g_off, h->g_deg, h->g_col, dV);
      ld_note_launch(), k_ds_expand_communities<<<grid_for(n, TB), TB, 0, s>>>(h->dCf, h->C, n, dV);
    }
  }
  // ---- Alg. update, then Alg. leidenmk (dS, dR; reset dSigma of refined)
  cudaMemsetAsync(h->dS, 0, (size_t)n, s);
  cudaMemsetAsync(h->dR, 0, (size_t)n, s);
  if (nd + ni > 0) {
    ld_note_launch(), k_update_weights<<<grid_for(nd + ni, TB), TB, 0, s>>>(DK, DW, nd, IK, IW, ni, vb, h->C, h->K, h->Sig, h->dSig,
                                                           cnt, h->gid0, h->gc.m2);
    ld_note_launch(), k_mark_communities<<<grid_for(nd + ni, TB), TB, 0, s>>>(DK, nd, IK, ni, vb, h->C, h->Sig, h->dSig,
                                                             h->p.tau_refine, h->dS, h->dR);
    ld_note_launch(), k_reset_changes<<<grid_for(nd + ni, TB), TB, 0, s>>>(DK, nd, IK, ni, vb, h->C, h->dR, h->dSig);
  }
  // Algorithmic bytes of the batch phase: the edge triples read (12 B per
  // edge); per raw arc its expansion and sort (48 B: key and weight written,
  // then read and written once more) and deduplication (24 B); per unique
  // arc the existence check or classification (16 B) and the updates of K,
  // Sigma, Delta Sigma, 2m and the flags (40 B); per touched row its plan
  // (40 B) and per arc of a merged row its read and write (16 B); a full
  // rebuild copies every arc (16 B); marking: dV (1 B per vertex) plus, for
  // DF, both endpoints' communities per unique arc (16 B), for DS the
  // (source, community) pairs of the insertions and their sort (48 B per
  // arc), dE and the community sweep (7 B per vertex); dS and dR (2 B per
  // vertex).
  int64_t A = nda + nia, U = nd + ni;
  int64_t bytes = 12 * (n_del + n_ins) + 72 * A + 56 * U + 40 * nrows + 16 * tmp_total + 3 * n;
  if (overflow) bytes += 16 * h->g_arcs;
  if (mode == LEIDEN_DF) bytes += 16 * U;
  if (mode == LEIDEN_DS) bytes += 48 * ni + 7 * n;
  ph_bytes(h, LEIDEN_PHASE_BATCH, bytes);
  return LEIDEN_OK;
}
