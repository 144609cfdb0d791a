// Device primitives: exclusive scan, stable radix sort, fills.
#include "internal.h"

namespace {

constexpr int SCAN_BLOCK = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
  int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(LD_FULL, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive scan over the block of one value per thread; returns the
// thread's exclusive prefix and the block total in *total.
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *total) {
  __shared__ int64_t wsum[SCAN_BLOCK / 32];
  __shared__ int64_t wtotal;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t incl = warp_incl_scan(v);
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int nw = blockDim.x >> 5;
    int64_t x = lane < nw ? wsum[lane] : 0;
    int64_t xs = warp_incl_scan(x);
    if (lane < nw) wsum[lane] = xs - x;
    if (lane == 31) wtotal = xs;  // lanes >= nw add 0, so lane 31 holds the total
  }
  __syncthreads();
  int64_t res = incl - v + wsum[wid];
  *total = wtotal;
  __syncthreads();
  return res;
}

template <typename T>
__global__ void scan_tile_reduce(const T *in, int64_t n, int64_t *tile_sums) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++)
    if (base + k < n) s += (int64_t)in[base + k];
  int64_t total;
  block_excl_scan(s, &total);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// Single block: exclusive scan of the tile sums in place; writes the grand
// total to *grand.
__global__ void scan_tile_offsets(int64_t *tile_sums, int64_t ntiles, int64_t *grand) {
  int64_t carry = 0;
  for (int64_t base = 0; base < ntiles; base += SCAN_BLOCK) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < ntiles ? tile_sums[i] : 0;
    int64_t total;
    int64_t ex = block_excl_scan(v, &total);
    if (i < ntiles) tile_sums[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) *grand = carry;
}

template <typename T>
__global__ void scan_tile_apply(const T *in, int64_t *out, int64_t n, const int64_t *tile_offs) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t v[SCAN_ITEMS];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    v[k] = (base + k < n) ? (int64_t)in[base + k] : 0;
    s += v[k];
  }
  int64_t total;
  int64_t ex = block_excl_scan(s, &total) + tile_offs[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    if (base + k < n) out[base + k] = ex;
    ex += v[k];
  }
}

// Second step of the two-launch scan: each block adds up the sums of the
// tiles before its own (at most SCAN_PREFIX_MAX of them, read from L2) in
// place of a separate offsets launch; the last block writes the total.
constexpr int64_t SCAN_PREFIX_MAX = 4096;
template <typename T>
__global__ void scan_tile_apply_prefix(const T *in, int64_t *out, int64_t n, const int64_t *tile_sums) {
  __shared__ int64_t red[SCAN_BLOCK / 32];
  int64_t b = blockIdx.x;
  int64_t p = 0;
  for (int64_t k = threadIdx.x; k < b; k += blockDim.x) p += tile_sums[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(LD_FULL, p, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = p;
  __syncthreads();
  int64_t prefix = 0;
#pragma unroll 4
  for (int w = 0; w < SCAN_BLOCK / 32; w++) prefix += red[w];
  int64_t base = b * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t v[SCAN_ITEMS];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    v[k] = (base + k < n) ? (int64_t)in[base + k] : 0;
    s += v[k];
  }
  int64_t total;
  int64_t ex = block_excl_scan(s, &total) + prefix;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    if (base + k < n) out[base + k] = ex;
    ex += v[k];
  }
  if (b == gridDim.x - 1 && threadIdx.x == 0) out[n] = prefix + total;
}

// One block over all n <= SCAN_TILE values (the loads finish before the
// first barrier, so in == out is safe).
template <typename T>
__global__ void scan_single_tile(const T *in, int64_t *out, int64_t n) {
  int64_t base = (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t v[SCAN_ITEMS];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    v[k] = (base + k < n) ? (int64_t)in[base + k] : 0;
    s += v[k];
  }
  int64_t total;
  int64_t ex = block_excl_scan(s, &total);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    if (base + k < n) out[base + k] = ex;
    ex += v[k];
  }
  if (threadIdx.x == 0) out[n] = total;
}

// One launch for a single tile, two while a block can add up the tile sums
// before it, three (reduce, offsets, apply) beyond that.
template <typename T>
cudaError_t scan_impl(const T *in, int64_t *out, int64_t n, void *tmp, cudaStream_t s) {
  int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  int64_t *tile = (int64_t *)tmp;
  if (n <= 0) {
    cudaMemsetAsync(out, 0, sizeof(int64_t), s);
  } else if (ntiles == 1) {
    ld_note_launch(), scan_single_tile<T><<<1, SCAN_BLOCK, 0, s>>>(in, out, n);
  } else if (ntiles <= SCAN_PREFIX_MAX) {
    ld_note_launch(), scan_tile_reduce<T><<<(unsigned)ntiles, SCAN_BLOCK, 0, s>>>(in, n, tile);
    ld_note_launch(), scan_tile_apply_prefix<T><<<(unsigned)ntiles, SCAN_BLOCK, 0, s>>>(in, out, n, tile);
  } else {
    ld_note_launch(), scan_tile_reduce<T><<<(unsigned)ntiles, SCAN_BLOCK, 0, s>>>(in, n, tile);
    ld_note_launch(), scan_tile_offsets<<<1, SCAN_BLOCK, 0, s>>>(tile, ntiles, out + n);
    ld_note_launch(), scan_tile_apply<T><<<(unsigned)ntiles, SCAN_BLOCK, 0, s>>>(in, out, n, tile);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- radix sort
constexpr int RS_BLOCK = 256;
constexpr int RS_ROUNDS = 4;  // short tiles: a batch of 1e5 keys still spreads over ~100 blocks
constexpr int RS_TILE = RS_BLOCK * RS_ROUNDS;

__global__ void rs_hist(const uint64_t *keys, int64_t n, int shift, int64_t nblocks, int64_t *hist) {
  __shared__ int32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ROUNDS; r++) {
    int64_t i = base + (int64_t)r * RS_BLOCK + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: elements of a tile are taken 256 at a time in index order;
// inside a round, warp w's elements precede warp w+1's, and inside a warp the
// lane order decides (match_any gives the peers with the same digit).
__global__ void rs_scatter(const uint64_t *keys, const int64_t *vals, uint64_t *okeys, int64_t *ovals,
                           int64_t n, int shift, int64_t nblocks, const int64_t *offs) {
  __shared__ int64_t base_off[256];
  __shared__ int32_t wcnt[RS_BLOCK / 32][256];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  base_off[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
  int64_t tile = (int64_t)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ROUNDS; r++) {
    for (int k = threadIdx.x; k < (RS_BLOCK / 32) * 256; k += RS_BLOCK) (&wcnt[0][0])[k] = 0;
    __syncthreads();
    int64_t i = tile + (int64_t)r * RS_BLOCK + threadIdx.x;
    bool valid = i < n;
    uint64_t key = valid ? keys[i] : 0;
    uint32_t d = valid ? (uint32_t)((key >> shift) & 255) : 256u + lane;  // invalid: unique pseudo-digit
    uint32_t peers = __match_any_sync(LD_FULL, d);
    uint32_t lt = peers & ((1u << lane) - 1u);
    int rank = __popc(lt);
    if (valid && lt == 0) wcnt[wid][d] = __popc(peers);
    __syncthreads();
    // per digit: exclusive prefix over warps
    {
      int dd = threadIdx.x;  // RS_BLOCK == 256 digits
      int32_t run = 0;
#pragma unroll
      for (int w = 0; w < RS_BLOCK / 32; w++) {
        int32_t t = wcnt[w][dd];
        wcnt[w][dd] = run;
        run += t;
      }
      // stash the round total in the slot past the prefix: reuse a register
      __syncthreads();
      if (valid) {
        int64_t pos = base_off[d] + wcnt[wid][d] + rank;
        okeys[pos] = key;
        if (vals) ovals[pos] = vals[i];
      }
      __syncthreads();
      base_off[dd] += run;
    }
    __syncthreads();
  }
}

// Stable sort of at most SMALL_SORT_MAX keys (on their low bits) in one
// block: a bitonic network over (key, position) pairs, then the keys and
// values are gathered by position.  Equal keys keep their input order, so
// the output equals the radix sort's.
constexpr int SMALL_SORT_MAX = 2048;
__global__ void __launch_bounds__(1024) k_small_sort(uint64_t *keys, int64_t *vals, int n, uint64_t mask) {
  __shared__ uint64_t sk[SMALL_SORT_MAX];
  __shared__ int32_t si[SMALL_SORT_MAX];
  int P = 1;
  while (P < n) P <<= 1;
  for (int t = threadIdx.x; t < P; t += blockDim.x) {
    sk[t] = t < n ? (keys[t] & mask) : ~0ull;  // padding sorts last (its positions are larger)
    si[t] = t;
  }
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < P; t += blockDim.x) {
        int u = t ^ j;
        if (u <= t) continue;
        uint64_t a = sk[t], b = sk[u];
        int32_t ia = si[t], ib = si[u];
        bool greater = a > b || (a == b && ia > ib);
        if (greater == ((t & k) == 0)) { sk[t] = b; sk[u] = a; si[t] = ib; si[u] = ia; }
      }
      __syncthreads();
    }
  constexpr int PER = SMALL_SORT_MAX / 1024;
  uint64_t kk[PER];
  int64_t vv[PER];
#pragma unroll
  for (int r = 0; r < PER; r++) {
    int t = threadIdx.x + r * (int)blockDim.x;
    if (t < n) { kk[r] = keys[si[t]]; vv[r] = vals ? vals[si[t]] : 0; }
  }
  __syncthreads();  // every read of the input is done before it is overwritten
#pragma unroll
  for (int r = 0; r < PER; r++) {
    int t = threadIdx.x + r * (int)blockDim.x;
    if (t < n) { keys[t] = kk[r]; if (vals) vals[t] = vv[r]; }
  }
}

}  // namespace

size_t scan_tmp_bytes(int64_t n) { return (size_t)((n + SCAN_TILE - 1) / SCAN_TILE + 8) * sizeof(int64_t); }

cudaError_t exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, void *tmp, cudaStream_t s) {
  return scan_impl<int64_t>(in, out, n, tmp, s);
}

cudaError_t exclusive_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, void *tmp, cudaStream_t s) {
  return scan_impl<int32_t>(in, out, n, tmp, s);
}

size_t sort_tmp_bytes(int64_t n) {
  int64_t nblocks = (n + RS_TILE - 1) / RS_TILE;
  int64_t hist = 256 * nblocks + 1;
  return (size_t)(2 * hist) * sizeof(int64_t) + scan_tmp_bytes(256 * nblocks) + 256;
}

cudaError_t radix_sort_u64(uint64_t *keys, uint64_t *keys_alt, int64_t *vals, int64_t *vals_alt, int64_t n,
                           int bits, void *tmp, cudaStream_t s) {
  if (n <= 1) return cudaSuccess;
  if (n <= SMALL_SORT_MAX) {
    uint64_t mask = bits >= 64 ? ~0ull : ((1ull << bits) - 1);
    ld_note_launch(), k_small_sort<<<1, 1024, 0, s>>>(keys, vals, (int)n, mask);
    return cudaGetLastError();
  }
  int64_t nblocks = (n + RS_TILE - 1) / RS_TILE;
  int64_t hlen = 256 * nblocks;
  int64_t *hist = (int64_t *)tmp;
  int64_t *offs = hist + hlen + 1;
  void *stmp = (void *)(offs + hlen + 1);
  uint64_t *src = keys, *dst = keys_alt;
  int64_t *vsrc = vals, *vdst = vals_alt;
  int passes = 0;
  for (int shift = 0; shift < bits; shift += 8) {
    ld_note_launch(), rs_hist<<<(unsigned)nblocks, RS_BLOCK, 0, s>>>(src, n, shift, nblocks, hist);
    cudaError_t e = exclusive_scan_i64(hist, offs, hlen, stmp, s);
    if (e != cudaSuccess) return e;
    ld_note_launch(), rs_scatter<<<(unsigned)nblocks, RS_BLOCK, 0, s>>>(src, vsrc, dst, vdst, n, shift, nblocks, offs);
    uint64_t *t = src; src = dst; dst = t;
    int64_t *tv = vsrc; vsrc = vdst; vdst = tv;
    passes++;
  }
  if (passes & 1) {
    cudaMemcpyAsync(keys, src, (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
    if (vals) cudaMemcpyAsync(vals, vsrc, (size_t)n * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
  }
  return cudaGetLastError();
}

namespace {
// One block: table and chunk offsets of the listed items (exclusive prefix
// sums, totals at index count).  An item's size is deg32[v] or
// off64[v+1] - off64[v]; its table has pow2 >= 2*min(size, key_cap) slots
// (key_cap bounds the distinct keys an item can have, e.g. the number of
// communities) and it is cut into chunks of TABLE_CHUNK.
__global__ void __launch_bounds__(1024) k_table_plan(const int32_t *list, const int32_t *count_p,
                                                      const int32_t *deg32, const int64_t *off64, int64_t key_cap,
                                                      int64_t *tab_off, int64_t *ch_off) {
  __shared__ int64_t ws[32][2];
  __shared__ int64_t carry[2];
  int64_t count = *count_p;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) { carry[0] = 0; carry[1] = 0; }
  __syncthreads();
  for (int64_t base = 0; base < count; base += blockDim.x) {
    int64_t k = base + threadIdx.x;
    int64_t t = 0, c = 0;
    if (k < count) {
      int32_t v = list[k];
      int64_t d = deg32 ? (int64_t)deg32[v] : off64[v + 1] - off64[v];
      int64_t keys = d < key_cap ? d : key_cap;
      t = 1;
      while (t < 2 * keys) t <<= 1;
      c = d > 0 ? (d + TABLE_CHUNK - 1) / TABLE_CHUNK : 1;  // every item gets at least one chunk
    }
    int64_t it = t, ic = c;  // inclusive warp scans
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t xt = __shfl_up_sync(LD_FULL, it, o), xc = __shfl_up_sync(LD_FULL, ic, o);
      if (lane >= o) { it += xt; ic += xc; }
    }
    if (lane == 31) { ws[wid][0] = it; ws[wid][1] = ic; }
    __syncthreads();
    if (threadIdx.x == 0) {
      int64_t a = carry[0], b = carry[1];
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
        int64_t x = ws[w][0], y = ws[w][1];
        ws[w][0] = a; ws[w][1] = b;
        a += x; b += y;
      }
      carry[0] = a; carry[1] = b;
    }
    __syncthreads();
    if (k < count) { tab_off[k] = ws[wid][0] + it - t; ch_off[k] = ws[wid][1] + ic - c; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { tab_off[count] = carry[0]; ch_off[count] = carry[1]; }
}

__global__ void k_fill_i32(int32_t *p, int32_t v, int64_t n) {
  for (int64_t i = ld_gtid(); i < n; i += ld_gstride()) p[i] = v;
}
__global__ void k_fill_i64(int64_t *p, int64_t v, int64_t n) {
  for (int64_t i = ld_gtid(); i < n; i += ld_gstride()) p[i] = v;
}
__global__ void k_iota_i32(int32_t *p, int64_t n) {
  for (int64_t i = ld_gtid(); i < n; i += ld_gstride()) p[i] = (int32_t)i;
}
}  // namespace

int grid_for(int64_t n, int block, int max_blocks) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > max_blocks) g = max_blocks;
  return (int)g;
}

void launch_fill_i32(int32_t *p, int32_t v, int64_t n, cudaStream_t s) {
  if (n > 0) ld_note_launch(), k_fill_i32<<<grid_for(n, 256), 256, 0, s>>>(p, v, n);
}
void launch_fill_i64(int64_t *p, int64_t v, int64_t n, cudaStream_t s) {
  if (n > 0) ld_note_launch(), k_fill_i64<<<grid_for(n, 256), 256, 0, s>>>(p, v, n);
}
void launch_table_plan(const int32_t *list, const int32_t *count, const int32_t *deg32, const int64_t *off64,
                       int64_t key_cap, int64_t *tab_off, int64_t *ch_off, cudaStream_t s) {
  ld_note_launch(), k_table_plan<<<1, 1024, 0, s>>>(list, count, deg32, off64, key_cap, tab_off, ch_off);
}

void launch_iota_i32(int32_t *p, int64_t n, cudaStream_t s) {
  if (n > 0) ld_note_launch(), k_iota_i32<<<grid_for(n, 256), 256, 0, s>>>(p, n);
}
