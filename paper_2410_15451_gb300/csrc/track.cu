// Community tracking (Alg. "leidentr"), Sigma recomputation and the terms of
// modularity (Eq. 1).
#include <climits>

#include "internal.h"

namespace {

constexpr int TB = 256;
constexpr uint64_t EMPTY64 = ~0ull;

__device__ __forceinline__ uint64_t hash64(uint64_t k) { return ld_splitmix64(k); }

// Best successor of each old community o: the new community with the largest
// overlap weight W(o, c) = sum of K_i over i with C^{t-1}_i = o and C_i = c,
// ties to the lowest new id.  Most communities keep a strict majority of
// their weight in one new community, and that one is then the unique
// argmax: a candidate (the new label of any member) is checked with two
// coalesced sweeps, and only communities without a majority go through the
// pair table.
// Tracking's per-id arrays in one sweep: best weights -1, best ids INT_MAX,
// candidates -1, use flags and deviant weights 0.
__global__ void k_tr_init(int64_t N, long long *bw, int32_t *bc, long long *ow, int32_t *ob, int32_t *cand,
                          int32_t *used, int64_t *dev) {
  for (int64_t i = ld_gtid(); i < N; i += ld_gstride()) {
    bw[i] = -1;
    bc[i] = INT_MAX;
    ow[i] = -1;
    ob[i] = INT_MAX;
    cand[i] = -1;
    used[i] = 0;
    dev[i] = 0;
  }
}
__global__ void k_trc_cand(int64_t N, const int32_t *Cold, const int32_t *Cnew, int32_t *cand) {
  for (int64_t i = ld_gtid(); i < N; i += ld_gstride()) cand[Cold[i]] = Cnew[i];  // any member will do
}
// The weight of an old community is Sigma^{t-1} with K^t (the batch kept it
// current), so only the members whose new label differs from the candidate
// (the deviants) need adding up: ov = tot - deviant weight.
__global__ void k_trc_deviants(int64_t N, const int32_t *Cold, const int32_t *Cnew, const int64_t *K,
                               const int32_t *cand, int64_t *dev) {
  for (int64_t i = ld_gtid(); i < N; i += ld_gstride()) {
    int32_t o = Cold[i];
    if (Cnew[i] != cand[o]) {
      int64_t k = K[i];
      if (k) atomicAdd((unsigned long long *)&dev[o], (unsigned long long)k);
    }
  }
}
// bw/bc of the majority communities; the others are flagged: 1 = through
// the pair table, 2 = weight 0 (every member has K = 0, e.g. isolated
// vertices): every pair weighs 0, so the lowest new label of a member wins.
__global__ void k_trc_majority(int64_t N, const int32_t *cand, const int64_t *tot, const int64_t *dev,
                               long long *bw, int32_t *bc, int32_t *flag) {
  for (int64_t o = ld_gtid(); o < N; o += ld_gstride()) {
    int f = 0;
    if (cand[o] >= 0) {
      int64_t ov = tot[o] - dev[o];
      if (tot[o] == 0) { bw[o] = 0; f = 2; }
      else if (2 * ov > tot[o]) { bw[o] = ov; bc[o] = cand[o]; }
      else f = 1;
    }
    flag[o] = f;
  }
}
// Pair weights of the flagged communities.  The table is empty between
// calls; each filled slot is listed (count in *occ) and emptied by its reader.
__global__ void k_trc_insert(int64_t N, const int32_t *Cold, const int32_t *Cnew, const int64_t *K,
                             const int32_t *flag, int32_t *bc, int64_t cap, uint64_t *keys, int64_t *vals,
                             int32_t *list, int32_t *occ) {
  uint64_t mask = (uint64_t)cap - 1;
  int lane = threadIdx.x & 31;
  for (int64_t base = (ld_gtid() & ~31ll); base < N; base += ld_gstride()) {
    int64_t i = base + lane;
    bool take = false;
    uint64_t key = EMPTY64 - 1 - lane;
    int64_t kw = 0;
    if (i < N) {
      int32_t o = Cold[i];
      int f = flag[o];
      if (f == 1) {
        take = true;
        key = ((uint64_t)(uint32_t)o << 32) | (uint32_t)Cnew[i];
        kw = K[i];
      } else if (f == 2) {
        atomicMin(&bc[o], Cnew[i]);
      }
    }
    if (!__any_sync(LD_FULL, take)) continue;
    uint32_t peers = __match_any_sync(LD_FULL, (unsigned long long)key);
    int64_t sum = ld_group_sum_i64(peers, kw);
    // the warp lists the slots it claims with one atomic on occ
    int32_t claimed = -1;
    if (take && ld_group_leader(peers)) {
      uint64_t sl = hash64(key) & mask;
      for (uint64_t probe = 0; ld_ok(probe <= mask, LD_CHK_PROBE); probe++) {
        unsigned long long k = atomicCAS((unsigned long long *)&keys[sl], EMPTY64, key);
        if (k == EMPTY64) claimed = (int32_t)sl;
        if (k == EMPTY64 || k == key) {
          atomicAdd((unsigned long long *)&vals[sl], (unsigned long long)sum);
          break;
        }
        sl = (sl + 1) & mask;
      }
    }
    uint32_t m = __ballot_sync(LD_FULL, claimed >= 0);
    if (m) {
      int leader = __ffs(m) - 1;
      int32_t p0 = 0;
      if (lane == leader) p0 = atomicAdd(occ, __popc(m));
      p0 = __shfl_sync(LD_FULL, p0, leader);
      if (claimed >= 0) list[p0 + __popc(m & ((1u << lane) - 1u))] = claimed;
    }
  }
}
__global__ void k_trc_best_w(const int32_t *occ, const int32_t *list, const uint64_t *keys, const int64_t *vals,
                             long long *bw) {
  int64_t m = *occ;
  for (int64_t t = ld_gtid(); t < m; t += ld_gstride()) {
    int32_t sl = list[t];
    atomicMax(&bw[keys[sl] >> 32], (long long)vals[sl]);
  }
}
__global__ void k_trc_best_c(const int32_t *occ, const int32_t *list, uint64_t *keys, int64_t *vals,
                             const long long *bw, int32_t *bc) {
  int64_t m = *occ;
  for (int64_t t = ld_gtid(); t < m; t += ld_gstride()) {
    int32_t sl = list[t];
    uint64_t key = keys[sl];
    uint32_t o = (uint32_t)(key >> 32);
    if (vals[sl] == bw[o]) atomicMin(&bc[o], (int32_t)(key & 0xffffffffu));
    keys[sl] = EMPTY64;  // leave the table empty
    vals[sl] = 0;
  }
}
// For each new community: among the old communities that picked it, the
// largest overlap, then the lowest old id.
__global__ void k_tr_best_old_w(int64_t N, const int32_t *bc, const long long *bw, long long *ow) {
  for (int64_t b = ld_gtid(); b < N; b += ld_gstride())
    if (bc[b] != INT_MAX) atomicMax(&ow[bc[b]], bw[b]);
}
__global__ void k_tr_best_old_b(int64_t N, const int32_t *bc, const long long *bw, const long long *ow, int32_t *ob) {
  for (int64_t b = ld_gtid(); b < N; b += ld_gstride())
    if (bc[b] != INT_MAX && bw[b] == ow[bc[b]]) atomicMin(&ob[bc[b]], (int32_t)b);
}
__global__ void k_tr_new_used(int64_t N, const int32_t *Cnew, int32_t *used) {
  for (int64_t i = ld_gtid(); i < N; i += ld_gstride()) used[Cnew[i]] = 1;
}
// unmatched[c] (new id used, nobody picked it); free[id] (no old vertex had id)
__global__ void k_tr_flags(int64_t N, const int32_t *new_used, const int32_t *ob, const int32_t *bc,
                           int32_t *unmatched, int32_t *freef) {
  for (int64_t c = ld_gtid(); c < N; c += ld_gstride()) {
    unmatched[c] = (new_used[c] && ob[c] == INT_MAX) ? 1 : 0;
    freef[c] = bc[c] == INT_MAX ? 1 : 0;
  }
}
__global__ void k_tr_free_list(int64_t N, const int32_t *freef, const int64_t *frank, int32_t *flist) {
  for (int64_t id = ld_gtid(); id < N; id += ld_gstride())
    if (freef[id]) flist[frank[id]] = (int32_t)id;
}
// The k-th unmatched new community of a graph takes the k-th free id of that
// graph (batched handles: ranks counted from the graph's first id).
__global__ void k_tr_map(int64_t N, const int32_t *new_used, const int32_t *ob, const int64_t *urank,
                         const int64_t *frank, const int32_t *flist, int32_t *map, uint8_t *matched,
                         const int32_t *gid0, const int64_t *voff) {
  for (int64_t c = ld_gtid(); c < N; c += ld_gstride()) {
    if (!new_used[c]) continue;
    if (ob[c] != INT_MAX) {
      map[c] = ob[c];
      matched[ob[c]] = 1;
    } else if (!gid0) {
      map[c] = flist[urank[c]];
    } else {
      int64_t v0 = voff[gid0[c]];
      map[c] = flist[frank[v0] + urank[c] - urank[v0]];
    }
  }
}
// C^t = map[new label]; Sigma and the member counts follow the vertices
// whose id changes (Sigma^{t-1} is current with K^t, so the others add
// nothing).
__global__ void k_tr_relabel(int64_t N, const int32_t *Cnew, const int32_t *map, const int64_t *K, int32_t *C,
                             int64_t *Sig, int32_t *size) {
  for (int64_t i = ld_gtid(); i < N; i += ld_gstride()) {
    int32_t c = map[Cnew[i]], o = C[i];
    if (c == o) continue;
    C[i] = c;
    int64_t k = K[i];
    if (k) {
      atomicAdd((unsigned long long *)&Sig[o], (unsigned long long)(-k));
      atomicAdd((unsigned long long *)&Sig[c], (unsigned long long)k);
    }
    atomicSub(&size[o], 1);  // member counts of C^t, for the next call
    atomicAdd(&size[c], 1);
  }
}
__global__ void k_tr_dsig(int64_t N, const uint8_t *matched, int64_t *dSig) {
  for (int64_t id = ld_gtid(); id < N; id += ld_gstride())
    if (!matched[id]) dSig[id] = 0;
}

// ---- modularity
__global__ void k_sig_of(int64_t N, const int32_t *C, const int64_t *K, int64_t *Sig) {
  int lane = threadIdx.x & 31;
  for (int64_t base = (ld_gtid() & ~31ll); base < N; base += ld_gstride()) {
    int64_t i = base + lane;
    int32_t c = i < N ? C[i] : -1 - lane;
    int64_t k = i < N ? K[i] : 0;
    uint32_t peers = __match_any_sync(LD_FULL, c);
    int64_t s = ld_group_sum_i64(peers, k);
    if (i < N && ld_group_leader(peers) && s) atomicAdd((unsigned long long *)&Sig[c], (unsigned long long)s);
  }
}
// Batched handles (gid0 non-null) also sum per graph: sigg, sqg, m2g.
__global__ void k_sigma_intra(int64_t N, const int64_t *off, const int32_t *deg, const int32_t *col, const int32_t *w,
                              const int32_t *C, DevCounters *cnt, const int32_t *gid0, int64_t *sigg) {
  int lane = threadIdx.x & 31;
  int64_t warp = ld_gtid() >> 5, nw = ld_gstride() >> 5;
  int64_t acc = 0;
  for (int64_t i = warp; i < N; i += nw) {
    int32_t c = C[i];
    int64_t b = off[i], d = deg[i], vi = 0;
    for (int64_t a = lane; a < d; a += 32)
      if (C[col[b + a]] == c) vi += w[b + a];
    acc += vi;
    if (gid0) {
      vi = ld_warp_sum_i64(vi);
      if (lane == 0 && vi) atomicAdd((unsigned long long *)&sigg[gid0[i]], (unsigned long long)vi);
    }
  }
  acc = ld_warp_sum_i64(acc);
  if (lane == 0 && acc) atomicAdd((unsigned long long *)&cnt->sigma_intra, (unsigned long long)acc);
}
__global__ void k_sq(int64_t N, const int64_t *Sig, DevCounters *cnt, const int32_t *gid0, unsigned long long *sqg) {
  i128 acc = 0;
  for (int64_t c0 = (ld_gtid() & ~31ll); c0 < N; c0 += ld_gstride()) {  // warp-uniform trip count
    int64_t c = c0 + (threadIdx.x & 31);
    i128 v = c < N ? (i128)Sig[c] * Sig[c] : 0;
    acc += v;
    if (gid0) ld_graph_add_i128(sqg, c < N && v != 0, c < N ? gid0[c] : 0, v);
  }
  // warp reduce in two halves
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += ld_shfl_xor_i128(acc, o);
  if ((threadIdx.x & 31) == 0) ld_atomic_add_i128(cnt->sq, acc);
}

__global__ void k_rowsum(int64_t N, const int64_t *off, const int32_t *deg, const int32_t *w, int64_t *K,
                         DevCounters *cnt, const int32_t *gid0, int64_t *m2g) {
  int lane = threadIdx.x & 31;
  int64_t warp = ld_gtid() >> 5, nw = ld_gstride() >> 5;
  int64_t tot = 0;
  for (int64_t i = warp; i < N; i += nw) {
    int64_t b = off[i], d = deg[i], acc = 0;
    for (int64_t a = lane; a < d; a += 32) acc += w[b + a];
    acc = ld_warp_sum_i64(acc);
    if (lane == 0) K[i] = acc;
    if (lane == 0 && gid0 && acc) atomicAdd((unsigned long long *)&m2g[gid0[i]], (unsigned long long)acc);
    tot += acc;
  }
  if (lane == 0 && tot) atomicAdd((unsigned long long *)&cnt->m2, (unsigned long long)tot);
}

}  // namespace

// C^{t-1} = h->C, final top-level membership = h->Ctop  ->  h->C, h->Sig, h->dSig.
void track_communities(leiden_handle *h) {
  cudaStream_t s = h->stream;
  int64_t N = h->n;
  int gN = grid_for(N, TB);
  long long *bw = (long long *)h->lbuf0, *ow = (long long *)h->lbuf1;
  int32_t *bc = h->ibuf0, *ob = h->ibuf1, *used = h->ibuf2;
  int32_t *cand = h->mtarget, *flag = h->movers;
  int64_t *dev = h->Sp;
  ld_note_launch(), k_tr_init<<<gN, TB, 0, s>>>(N, bw, bc, ow, ob, cand, used, dev);
  cudaMemsetAsync(&h->dcnt->tr_occ, 0, sizeof(int32_t), s);
  ld_note_launch(), k_trc_cand<<<gN, TB, 0, s>>>(N, h->C, h->Ctop, cand);
  ld_note_launch(), k_trc_deviants<<<gN, TB, 0, s>>>(N, h->C, h->Ctop, h->K, cand, dev);
  ld_note_launch(), k_trc_majority<<<gN, TB, 0, s>>>(N, cand, h->Sig, dev, bw, bc, flag);
  int32_t *occ = &h->dcnt->tr_occ;
  ld_note_launch(), k_trc_insert<<<gN, TB, 0, s>>>(N, h->C, h->Ctop, h->K, flag, bc, h->tr_cap, h->tr_keys, h->tr_vals,
                                                   h->tr_list, occ);
  ld_note_launch(), k_trc_best_w<<<h->sm_count * 8, TB, 0, s>>>(occ, h->tr_list, h->tr_keys, h->tr_vals, bw);
  ld_note_launch(), k_trc_best_c<<<h->sm_count * 8, TB, 0, s>>>(occ, h->tr_list, h->tr_keys, h->tr_vals, bw, bc);
  ld_note_launch(), k_tr_best_old_w<<<gN, TB, 0, s>>>(N, bc, bw, ow);
  ld_note_launch(), k_tr_best_old_b<<<gN, TB, 0, s>>>(N, bc, bw, ow, ob);
  ld_note_launch(), k_tr_new_used<<<gN, TB, 0, s>>>(N, h->Ctop, used);
  int32_t *unmatched = h->rep, *freef = h->prop;
  ld_note_launch(), k_tr_flags<<<gN, TB, 0, s>>>(N, used, ob, bc, unmatched, freef);
  int64_t *urank = h->lbuf2, *frank = h->lbuf3;
  exclusive_scan_i32_to_i64(unmatched, urank, N, h->scan_tmp, s);
  exclusive_scan_i32_to_i64(freef, frank, N, h->scan_tmp, s);
  int32_t *flist = h->parent, *map = h->CB;
  ld_note_launch(), k_tr_free_list<<<gN, TB, 0, s>>>(N, freef, frank, flist);
  uint8_t *matched = h->dE;
  cudaMemsetAsync(matched, 0, (size_t)N, s);
  ld_note_launch(), k_tr_map<<<gN, TB, 0, s>>>(N, used, ob, urank, frank, flist, map, matched, h->gid0, h->d_voff);
  ld_note_launch(), k_tr_relabel<<<gN, TB, 0, s>>>(N, h->Ctop, map, h->K, h->C, h->Sig, h->csize0);
  ld_note_launch(), k_tr_dsig<<<gN, TB, 0, s>>>(N, matched, h->dSig);
}

// sigma (intra arcs) and sum Sigma_c^2 of membership C on G^t.
void modularity_terms(leiden_handle *h, const int32_t *C) {
  cudaStream_t s = h->stream;
  int64_t N = h->n;
  int64_t *Sig = h->lbuf0;
  cudaMemsetAsync(Sig, 0, (size_t)N * sizeof(int64_t), s);
  cudaMemsetAsync(&h->dcnt->sigma_intra, 0, sizeof(int64_t), s);
  cudaMemsetAsync(&h->dcnt->sq[0], 0, 2 * sizeof(unsigned long long), s);
  ld_note_launch(), k_sig_of<<<grid_for(N, TB), TB, 0, s>>>(N, C, h->K, Sig);
  if (h->gid0) {
    cudaMemsetAsync(h->gc.sigma, 0, (size_t)h->G * sizeof(int64_t), s);
    cudaMemsetAsync(h->gc.sq, 0, (size_t)h->G * 2 * sizeof(unsigned long long), s);
  }
  ld_note_launch(), k_sigma_intra<<<grid_for(N * 32, TB), TB, 0, s>>>(N, h->g_off, h->g_deg, h->g_col, h->g_w, C, h->dcnt,
                                                                      h->gid0, h->gc.sigma);
  ld_note_launch(), k_sq<<<grid_for(N, TB), TB, 0, s>>>(N, Sig, h->dcnt, h->gid0, h->gc.sq);
}

// Sigma = per-community sums of K for membership h->C.
void recompute_sigma(leiden_handle *h) {
  cudaStream_t s = h->stream;
  cudaMemsetAsync(h->Sig, 0, (size_t)h->n * sizeof(int64_t), s);
  ld_note_launch(), k_sig_of<<<grid_for(h->n, TB), TB, 0, s>>>(h->n, h->C, h->K, h->Sig);
}

// K = row sums of G^t and 2m.
void recompute_weights(leiden_handle *h) {
  cudaStream_t s = h->stream;
  cudaMemsetAsync(&h->dcnt->m2, 0, sizeof(int64_t), s);
  if (h->gid0) cudaMemsetAsync(h->gc.m2, 0, (size_t)h->G * sizeof(int64_t), s);
  ld_note_launch(), k_rowsum<<<grid_for(h->n * 32, TB), TB, 0, s>>>(h->n, h->g_off, h->g_deg, h->g_w, h->K, h->dcnt,
                                                                    h->gid0, h->gc.m2);
}

LD_CHECK_WORD_READER(check_word_track)
