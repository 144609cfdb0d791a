// Modularity of a membership on a caller-owned device CSR, without any
// device allocation: the per-community totals and the reduction counters
// live in one file-scope __device__ array of fixed size.
#include <mutex>
#include <string>

#include "internal.h"

namespace {

// Largest vertex count the entry point accepts: the scratch holds one int64
// community total per vertex id (32 MiB) plus NOALLOC_COUNTERS int64 words.
constexpr int64_t NOALLOC_MAX_VERTICES = (int64_t)1 << 22;
constexpr int64_t NOALLOC_COUNTERS = 6;
constexpr int64_t NOALLOC_WORDS = NOALLOC_MAX_VERTICES + NOALLOC_COUNTERS;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) int64_t g_noalloc_scratch[NOALLOC_WORDS];

// Host code must not pass g_noalloc_scratch to a kernel: on the host that
// name is a stand-in symbol, not a device address.  The device address is
// looked up once per device (with that device current) and cached here.
constexpr int MAX_DEVICES = 64;
int64_t *g_scratch_ptr[MAX_DEVICES] = {};
std::mutex g_scratch_mu;

// counters after the per-vertex totals
enum { C_M2 = 0, C_SIGMA = 1, C_SQ_LO = 2, C_SQ_HI = 3, C_BAD = 4, C_BADCOL = 5 };

__global__ void k_na_clear(int64_t n, int64_t *scr) {
  for (int64_t i = ld_gtid(); i < n; i += ld_gstride()) scr[i] = 0;
  if (ld_gtid() < NOALLOC_COUNTERS) scr[NOALLOC_MAX_VERTICES + ld_gtid()] = 0;
}

// Warp per vertex: K_i (row sum) into Sigma[C_i]; intra-community weight; 2m.
// A membership id outside [0, n) sets the C_BAD word and the vertex is
// skipped; a column outside [0, n) sets C_BADCOL (and is not read through).
// Either one turns the call into LEIDEN_ERR_ARG.
__global__ void k_na_rows(int64_t n, const int64_t *off, const int32_t *col, const int32_t *w, const int32_t *C,
                          int64_t *scr) {
  int lane = threadIdx.x & 31;
  int64_t warp = ld_gtid() >> 5, nw = ld_gstride() >> 5;
  int64_t m2 = 0, intra = 0;
  for (int64_t i = warp; i < n; i += nw) {
    int32_t c = C[i];
    if (c < 0 || c >= n) {
      if (lane == 0) atomicExch((unsigned long long *)&scr[NOALLOC_MAX_VERTICES + C_BAD], 1ull);
      continue;
    }
    int64_t k = 0;
    for (int64_t a = off[i] + lane; a < off[i + 1]; a += 32) {
      int64_t wa = w ? (int64_t)w[a] : 1;
      k += wa;
      int32_t j = col[a];
      if (j < 0 || j >= n) {
        atomicExch((unsigned long long *)&scr[NOALLOC_MAX_VERTICES + C_BADCOL], 1ull);
        continue;
      }
      if (C[j] == c) intra += wa;
    }
    k = ld_warp_sum_i64(k);
    if (lane == 0 && k) atomicAdd((unsigned long long *)&scr[c], (unsigned long long)k);
    m2 += k;  // identical in every lane after the reduction; lane 0 adds it
  }
  intra = ld_warp_sum_i64(intra);
  if (lane == 0) {
    if (m2) atomicAdd((unsigned long long *)&scr[NOALLOC_MAX_VERTICES + C_M2], (unsigned long long)m2);
    if (intra) atomicAdd((unsigned long long *)&scr[NOALLOC_MAX_VERTICES + C_SIGMA], (unsigned long long)intra);
  }
}

__global__ void k_na_sq(int64_t n, int64_t *scr) {
  i128 acc = 0;
  for (int64_t c = ld_gtid(); c < n; c += ld_gstride()) acc += (i128)scr[c] * scr[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += ld_shfl_xor_i128(acc, o);
  if ((threadIdx.x & 31) == 0) ld_atomic_add_i128((unsigned long long *)&scr[NOALLOC_MAX_VERTICES + C_SQ_LO], acc);
}

}  // namespace


extern "C" leiden_status leiden_modularity_noalloc(int64_t n, const int64_t *d_offsets, const int32_t *d_cols,
                                                   const int32_t *d_weights, const int32_t *d_membership,
                                                   void *cuda_stream, double *q_out) {
  if (!q_out || n < 1 || !d_offsets || !d_cols || !d_membership) {
    set_handle_free_error("leiden_modularity_noalloc: null pointer or n < 1");
    return LEIDEN_ERR_ARG;
  }
  if (n > NOALLOC_MAX_VERTICES) {
    set_handle_free_error("leiden_modularity_noalloc: n exceeds the fixed scratch of 4194304 vertices");
    return LEIDEN_ERR_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_handle_free_error(std::string("leiden_modularity_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    return LEIDEN_ERR_CUDA;
  }
  if (dev < 0 || dev >= MAX_DEVICES) {
    set_handle_free_error("leiden_modularity_noalloc: device ordinal " + std::to_string(dev) +
                          " is beyond the 64 devices whose scratch address is cached");
    return LEIDEN_ERR_CUDA;
  }
  int64_t *scr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        set_handle_free_error(std::string("leiden_modularity_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return LEIDEN_ERR_CUDA;
      }
      g_scratch_ptr[dev] = (int64_t *)p;
    }
    scr = g_scratch_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  ld_note_launch(), k_na_clear<<<grid_for(n, 256), 256, 0, s>>>(n, scr);
  ld_note_launch(), k_na_rows<<<sms * 16, 256, 0, s>>>(n, d_offsets, d_cols, d_weights, d_membership, scr);
  ld_note_launch(), k_na_sq<<<grid_for(n, 256), 256, 0, s>>>(n, scr);
  int64_t cnt[NOALLOC_COUNTERS] = {};
  e = cudaMemcpyAsync(cnt, scr + NOALLOC_MAX_VERTICES, sizeof(cnt), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_handle_free_error(std::string("leiden_modularity_noalloc: ") + cudaGetErrorString(e));
    return LEIDEN_ERR_CUDA;
  }
  if (cnt[C_BAD]) {
    set_handle_free_error("leiden_modularity_noalloc: membership id outside [0, n)");
    return LEIDEN_ERR_ARG;
  }
  if (cnt[C_BADCOL]) {
    set_handle_free_error("leiden_modularity_noalloc: column id outside [0, n)");
    return LEIDEN_ERR_ARG;
  }
  int64_t m2 = cnt[C_M2];
  if (m2 == 0) {
    *q_out = 0.0;
    return LEIDEN_OK;
  }
  i128 sq = (i128)(((u128)(uint64_t)cnt[C_SQ_HI] << 64) | (u128)(uint64_t)cnt[C_SQ_LO]);
  i128 num = (i128)m2 * cnt[C_SIGMA] - sq;
  *q_out = i128_to_double(num) / ((double)m2 * (double)m2);
  return LEIDEN_OK;
}

