// C ABI of the GB300 dynamic Leiden library and the pass loop of Alg.
// "leiden" (Appendix A.4) that drives the kernels.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>

#include "internal.h"

#include <atomic>
#include <thread>

static std::atomic<int64_t> g_launches{0};

void ld_note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// int128 -> double in a fixed order (|x| = hi*2^64 + lo, then the sign).
double i128_to_double(i128 x) {
  bool neg = x < 0;
  u128 u = neg ? (u128)(-(x + 1)) + 1 : (u128)x;
  double hi = (double)(uint64_t)(u >> 64);
  double lo = (double)(uint64_t)u;
  double r = hi * 18446744073709551616.0 + lo;
  return neg ? -r : r;
}

GraphCounters gc_layout(void *base, int G) {
  char *q = (char *)base;
  GraphCounters c;
  c.dq = (unsigned long long *)q;  q += 16 * (size_t)G;
  c.sq = (unsigned long long *)q;  q += 16 * (size_t)G;
  c.moves = (int64_t *)q;          q += 8 * (size_t)G;
  c.m2 = (int64_t *)q;             q += 8 * (size_t)G;
  c.sigma = (int64_t *)q;          q += 8 * (size_t)G;
  c.accepted = (int32_t *)q;       q += 4 * (size_t)G;
  c.ncomm = (int32_t *)q;          q += 4 * (size_t)G;
  c.refined = (uint8_t *)q;        q += (size_t)G;
  c.lm_on = (uint8_t *)q;          q += (size_t)G;
  c.cont = (uint8_t *)q;
  return c;
}

// 16+16+8+8+8+4+4+1+1+1 = 67 bytes per graph, rounded up.
size_t gc_block_bytes(int G) { return 72 * (size_t)G + 64; }

// Global table slots the vertices above the block bin need at level 0.
int64_t level0_huge_slots(const std::vector<int32_t> &deg) {
  int64_t slots = 1 << 16;
  for (int32_t d : deg)
    if (d > BIN_BLOCK_MAX) {
      int64_t t = 1;
      while (t < 2 * (int64_t)d) t <<= 1;
      slots += t;
    }
  return slots;
}

bool acquire_agg_buffers(leiden_handle *h, int64_t arcs) {
  if (h->y_col[0] && h->y_slots >= arcs + 1) return true;
  release_agg_buffers(h);
  size_t slots = (size_t)arcs + 1;
  for (int attempt = 0; attempt < 2; attempt++) {
    bool ok = true;
    for (int k = 0; k < 2 && ok; k++)
      ok = cudaMallocAsync((void **)&h->y_col[k], slots * sizeof(int32_t), h->stream) == cudaSuccess &&
           cudaMallocAsync((void **)&h->y_w[k], slots * sizeof(int64_t), h->stream) == cudaSuccess;
    if (ok) {
      h->y_slots = arcs + 1;
      return true;
    }
    cudaGetLastError();
    release_agg_buffers(h);
    // the pool keeps freed blocks cached; blocks of other sizes (other
    // graphs' calls) may hold the memory this one needs: return the unused
    // ones to the device and try once more
    cudaStreamSynchronize(h->stream);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, h->device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
    cudaGetLastError();
  }
  return false;
}

void release_agg_buffers(leiden_handle *h) {
  for (int k = 0; k < 2; k++) {
    if (h->y_col[k]) cudaFreeAsync(h->y_col[k], h->stream);
    if (h->y_w[k]) cudaFreeAsync(h->y_w[k], h->stream);
    h->y_col[k] = nullptr;
    h->y_w[k] = nullptr;
  }
  h->y_slots = 0;
}

void ph_mark(leiden_handle *h, int tag) {
  if (!(h->p.collect_stats & 1)) return;
  if (h->ph_ev.size() < (size_t)h->ph_used + 1) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return; }
    h->ph_ev.push_back(e);
  }
  if (h->ph_tag.size() < (size_t)h->ph_used + 1) h->ph_tag.resize(h->ph_used + 1);
  h->ph_tag[h->ph_used] = tag;
  cudaEventRecord(h->ph_ev[h->ph_used], h->stream);
  h->ph_used++;
}

void ph_resolve(leiden_handle *h) {
  for (int k = 0; k + 1 < h->ph_used; k++) {
    float ms = 0;
    if (h->ph_tag[k] >= PHASE_END) continue;
    if (cudaEventElapsedTime(&ms, h->ph_ev[k], h->ph_ev[k + 1]) == cudaSuccess) h->stats.phase_ms[h->ph_tag[k]] += ms;
    else cudaGetLastError();
  }
  h->ph_used = 0;
  leiden_stats &st = h->stats;
  st.ms_batch = st.phase_ms[LEIDEN_PHASE_BATCH];
  st.ms_move = st.phase_ms[LEIDEN_PHASE_MOVE];
  st.ms_refine = st.phase_ms[LEIDEN_PHASE_REFINE];
  st.ms_aggregate = st.phase_ms[LEIDEN_PHASE_AGGREGATE];
  st.ms_track = st.phase_ms[LEIDEN_PHASE_TRACK];
  st.ms_total = 0;
  for (int k = 0; k < 6; k++) st.ms_total += st.phase_ms[k];
}

// An event pair around one launch of a timed kernel, on the stream it is
// launched on (the handle's stream unless given).
void kt_begin(leiden_handle *h, int k, cudaStream_t s) {
  if (!(h->p.collect_stats & 2)) return;
  size_t need = 2 * (size_t)(h->kt_used + 1);
  while (h->kt_ev.size() < need) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return; }
    h->kt_ev.push_back(e);
  }
  if (h->kt_tag.size() < (size_t)h->kt_used + 1) h->kt_tag.resize(h->kt_used + 1);
  h->kt_tag[h->kt_used] = k;
  cudaEventRecord(h->kt_ev[2 * h->kt_used], s ? s : h->stream);
}

void kt_end(leiden_handle *h, cudaStream_t s) {
  if (!(h->p.collect_stats & 2) || h->kt_ev.size() < 2 * (size_t)(h->kt_used + 1)) return;
  cudaEventRecord(h->kt_ev[2 * h->kt_used + 1], s ? s : h->stream);
  h->kt_used++;
}

void kt_reset(leiden_handle *h) {
  h->kt_used = 0;
  for (int k = 0; k < KT_KERNELS; k++) { h->kt_ms[k] = 0; h->kt_launches[k] = 0; }
  cudaMemsetAsync(h->dcnt->xk_bytes, 0, sizeof(h->dcnt->xk_bytes), h->stream);
  cudaMemsetAsync(h->dcnt->agg_tables, 0, sizeof(h->dcnt->agg_tables), h->stream);
}

void kt_resolve(leiden_handle *h) {
  for (int k = 0; k < h->kt_used; k++) {
    float ms = 0;
    int t = h->kt_tag[k];
    if (cudaEventElapsedTime(&ms, h->kt_ev[2 * k], h->kt_ev[2 * k + 1]) == cudaSuccess) h->kt_ms[t] += ms;
    else cudaGetLastError();
    h->kt_launches[t]++;
  }
  h->kt_used = 0;
}

namespace {

thread_local std::string g_create_error;

// fn(lo, hi) over [0, n) split across the host's threads (small n: one call).
template <typename F>
void host_parallel(int64_t n, F fn) {
  int nt = (int)std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
  if (n < (1 << 16) || nt == 1) { fn(0, n); return; }
  std::vector<std::thread> ts;
  for (int t = 0; t < nt; t++) ts.emplace_back([&, t] { fn(n * t / nt, n * (t + 1) / nt); });
  for (auto &th : ts) th.join();
}

i128 read_i128(const unsigned long long *p) { return (i128)(((u128)p[1] << 64) | (u128)p[0]); }

// dQ of a sum of gains g (Eq. 2 times 2m^2): 2g / (2m)^2.
double gains_to_dq(i128 g, int64_t m2) {
  if (g == 0 || m2 == 0) return 0.0;
  return i128_to_double(2 * g) / ((double)m2 * (double)m2);
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                    \
      return e_ == cudaErrorMemoryAllocation ? LEIDEN_ERR_OOM : LEIDEN_ERR_CUDA;      \
    }                                                                                 \
  } while (0)

template <typename T>
cudaError_t dalloc(leiden_handle *h, T **p, int64_t count) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, (size_t)std::max<int64_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  h->owned.push_back(q);
  *p = (T *)q;
  return cudaSuccess;
}

void sync_counters(leiden_handle *h) {
  cudaMemcpyAsync(h->hcnt, h->dcnt, sizeof(DevCounters), cudaMemcpyDeviceToHost, h->stream);
  cudaStreamSynchronize(h->stream);
}

#define CKF()                             \
  do {                                    \
    if (h->fatal != LEIDEN_OK) {          \
      leiden_status f_ = h->fatal;        \
      h->fatal = LEIDEN_OK;               \
      return f_;                          \
    }                                     \
  } while (0)

LevelGraph level0(leiden_handle *h) {
  LevelGraph g;
  g.gid = h->gid0;
  g.n = h->n;
  g.off = h->g_off;
  g.deg = h->g_deg;
  g.col = h->g_col;
  g.w = h->g_w;
  g.w64 = false;
  g.maxdeg = h->g_maxdeg;
  g.huge_slots = h->g_huge_slots;
  return g;
}

constexpr int TRACE_WORDS = 2 + 10 * 25;

// Copies the per-graph counter block of a batched handle to its pinned host
// mirror (with the device counters) and waits.
void sync_all(leiden_handle *h) {
  cudaMemcpyAsync(h->hcnt, h->dcnt, sizeof(DevCounters), cudaMemcpyDeviceToHost, h->stream);
  if (h->G > 1) cudaMemcpyAsync(h->gc_host, h->gc.dq, h->gc_bytes, cudaMemcpyDeviceToHost, h->stream);
  cudaStreamSynchronize(h->stream);
}

// Alg. leiden: passes of local moving, subset renumbering, splitting,
// refinement, then renumbering, lookup and aggregation; finally lookup and
// tracking.  Expects: Cp = C^{t-1} copy source in h->C, Kp/Sp from h->K,
// h->Sig, dS/dR marked, dV = affected.
//
// A batched handle runs the same loop over all its graphs at once; each
// graph keeps its own iteration count and stops iterating when its own dQ
// reaches tau, keeps its own refinement rounds, and leaves the pass loop at
// its own break (its final lookup is done then and it is not aggregated).
leiden_status run_leiden(leiden_handle *h, int dynamic, const uint8_t *in_range) {
  cudaStream_t s = h->stream;
  const leiden_params &p = h->p;
  int64_t N = h->n;
  memset(h->trace, 0, sizeof(h->trace));
  const bool B = h->G > 1;
  const int G = h->G;
  GraphCounters hg = B ? gc_layout(h->gc_host, G) : GraphCounters{};
  std::vector<int64_t> loff_h;
  std::vector<int> li_g, rounds_g;
  std::vector<char> inlvl, lmon, refany, refdone, cont;
  if (B) {
    h->gtrace.assign((size_t)G * TRACE_WORDS, 0);
    loff_h = h->voff;
    h->d_loff = h->d_loffb[0];
    CK(cudaMemcpyAsync(h->d_loff, h->d_voff, (size_t)(G + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    inlvl.assign(G, 1);
    li_g.assign(G, 0);
    rounds_g.assign(G, 0);
    lmon.assign(G, 0);
    refany.assign(G, 0);
    refdone.assign(G, 0);
    cont.assign(G, 0);
  }
  auto gtr = [&](int gi, int lp) -> int64_t * { return &h->gtrace[(size_t)gi * TRACE_WORDS + 2 + lp * 25]; };
  // initialisation
  // Phase bytes below follow the algorithmic byte model: the bytes a phase
  // must move per unit of its work (vertex of the level, arc scanned, move,
  // listed vertex), with the sizes of the arrays it reads and writes.
  ph_mark(h, LEIDEN_PHASE_MOVE);
  ph_bytes(h, LEIDEN_PHASE_MOVE, 45 * N + N / 8);  // dV -> frontier bits; Ctop; copies of C', K', Sigma'
  pass_init(h);
  CK(cudaMemsetAsync(&h->dcnt->processed, 0, 14 * sizeof(int64_t), s));  // processed .. lmk_bytes
  int64_t m2 = h->m2;
  LevelGraph g = level0(h);
  double tau = p.tau;
  int slot = 0;
  int passes = 0;
  bool looked_up = false;  // batched: every graph had its final lookup
  leiden_stats &st = h->stats;
  int64_t moves_total = 0;
  int64_t subsweep_words = 0;     // frontier words read by the collection kernels
  int64_t level_arcs = h->g_arcs;  // arcs of the current level
  for (int lp = 0; lp < p.max_passes; lp++) {
    int64_t n = g.n;
    int64_t tr_spare[25];
    int64_t *tr = lp < 10 ? &h->trace[2 + lp * 25] : tr_spare;  // the trace keeps the first 10 passes
    passes++;
    tr[0] = n;
    if (B) {
      for (int gi = 0; gi < G; gi++) {
        lmon[gi] = inlvl[gi];
        li_g[gi] = p.max_iterations;
        rounds_g[gi] = 0;
        refany[gi] = 0;
        refdone[gi] = !inlvl[gi];
        if (inlvl[gi] && lp < 10) {
          gtr(gi, lp)[0] = loff_h[gi + 1] - loff_h[gi];
          h->gtrace[(size_t)gi * TRACE_WORDS] = lp + 1;
        }
      }
      memcpy(hg.lm_on, lmon.data(), (size_t)G);
      CK(cudaMemcpyAsync(h->gc.lm_on, hg.lm_on, (size_t)G, cudaMemcpyHostToDevice, s));
    }
    if (lp > 0) ph_mark(h, LEIDEN_PHASE_MOVE);
    ph_bytes(h, LEIDEN_PHASE_MOVE, (lp > 0 || !dynamic ? 4 : 8) * n);  // community sizes
    lm_prepare(h, g, lp > 0 || !dynamic ? SIZES_ONES : SIZES_KEPT);
    int li = p.max_iterations;
    for (int it = 0; it < p.max_iterations; it++) {
      CK(cudaMemsetAsync(&h->dcnt->dq[0], 0, 2 * sizeof(unsigned long long), s));
      CK(cudaMemsetAsync(&h->dcnt->moves, 0, sizeof(int64_t), s));
      if (B) {
        CK(cudaMemsetAsync(h->gc.dq, 0, (size_t)G * 2 * sizeof(unsigned long long), s));
        CK(cudaMemsetAsync(h->gc.moves, 0, (size_t)G * sizeof(int64_t), s));
      }
      for (int cls = 0; cls < lm_classes(h); cls++) lm_subsweep(h, g, cls, lp == 0 ? in_range : nullptr, dynamic);
      subsweep_words += (int64_t)lm_classes(h) * ((n + 31) / 32);
      sync_all(h);
      kt_resolve(h);
      CK(cudaGetLastError());
      CKF();
      i128 dq = read_i128(h->hcnt->dq);
      int64_t mv = h->hcnt->moves;
      if (it < 20) tr[5 + it] = mv;
      moves_total += mv;
      st.lm_iterations++;
      if (!B) {
        if (gains_to_dq(dq, m2) <= tau) { li = it + 1; break; }
        continue;
      }
      bool any = false;
      for (int gi = 0; gi < G; gi++) {
        if (!lmon[gi]) continue;
        if (lp < 10 && it < 20) gtr(gi, lp)[5 + it] = hg.moves[gi];
        if (gains_to_dq(read_i128(&hg.dq[2 * gi]), h->m2g[gi]) <= tau) {
          li_g[gi] = it + 1;
          lmon[gi] = 0;
        } else {
          any = true;
        }
      }
      if (!any) { li = it + 1; break; }
      memcpy(hg.lm_on, lmon.data(), (size_t)G);
      CK(cudaMemcpyAsync(h->gc.lm_on, hg.lm_on, (size_t)G, cudaMemcpyHostToDevice, s));
    }
    tr[1] = li;
    ph_mark(h, LEIDEN_PHASE_SPLIT);
    ph_bytes(h, LEIDEN_PHASE_SPLIT, 64 * n);  // subset renumbering (58 B per vertex), split flags (6 B)
    subset_renumber(h, n);
    split_communities(h, g);
    ph_mark(h, LEIDEN_PHASE_REFINE);
    ph_bytes(h, LEIDEN_PHASE_REFINE, 29 * n);  // bounds C'_B, reset of the refined bounds
    CK(cudaMemcpyAsync(h->CB, h->Cp, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (B) CK(cudaMemsetAsync(h->gc.refined, 0, (size_t)G, s));
    refine_reset(h, g);
    int rounds = 0;
    int refined_any = 0;
    // Both modes repeat rounds until no move applies: in the in-place mode a
    // singleton whose target was taken retries against the updated state.
    // A graph of a batch counts the rounds up to its first round without a
    // move (its state does not change after that).
    int max_rounds = p.max_iterations;
    for (int r = 0; r < max_rounds; r++) {
      if (B) CK(cudaMemsetAsync(h->gc.accepted, 0, (size_t)G * sizeof(int32_t), s));
      refine_round(h, g, r & 1);
      rounds++;
      sync_all(h);
      CK(cudaGetLastError());
      CKF();
      if (r == 0) refined_any = h->hcnt->cand_count[0] > 0;
      if (B) {
        for (int gi = 0; gi < G; gi++) {
          if (r == 0) refany[gi] = hg.refined[gi];
          if (refdone[gi]) continue;
          rounds_g[gi]++;
          if (hg.accepted[gi] == 0) refdone[gi] = 1;
        }
      }
      if (h->hcnt->accepted == 0) break;
    }
    tr[3] = refined_any;
    tr[4] = rounds;
    // listed vertices (parent, list, compress: 24 B) and their arcs (col, C: 8 B)
    ph_bytes(h, LEIDEN_PHASE_SPLIT, 24 * (int64_t)h->hcnt->split_count + 8 * h->hcnt->split_arcs);
    ph_mark(h, LEIDEN_PHASE_AGGREGATE);
    ph_bytes(h, LEIDEN_PHASE_AGGREGATE, 4 * n);  // community count
    if (B) {
      CK(cudaMemsetAsync(h->gc.ncomm, 0, (size_t)G * sizeof(int32_t), s));
      count_communities(h, n, g.gid);
      sync_all(h);
      tr[2] = h->hcnt->list_count;
    } else {
      // only the trace needs the count: it is read with the next host sync
      count_communities(h, n, g.gid);
      if (lp < 10)
        CK(cudaMemcpyAsync(&h->dcnt->pass_ncomm[lp], &h->dcnt->list_count, sizeof(int32_t),
                           cudaMemcpyDeviceToDevice, s));
    }
    if (!B) {
      if (p.converge_any && (li <= 1 || !refined_any)) break;
      if (li <= 1 && !refined_any) break;
      if (li <= 1 && lp > 0 && !p.converge_any) break;
      if (lp == p.max_passes - 1) {
        // the pass limit is reached: lookup with C' below, as when breaking
        break;
      }
    } else {
      bool any_cont = false;
      for (int gi = 0; gi < G; gi++) {
        cont[gi] = 0;
        if (!inlvl[gi]) continue;
        if (lp < 10) {
          int64_t *t = gtr(gi, lp);
          t[1] = li_g[gi];
          t[2] = hg.ncomm[gi];
          t[3] = refany[gi];
          t[4] = rounds_g[gi];
        }
        bool brk = p.converge_any ? (li_g[gi] <= 1 || !refany[gi])
                                  : ((li_g[gi] <= 1 && !refany[gi]) || (li_g[gi] <= 1 && lp > 0));
        brk = brk || lp == p.max_passes - 1;
        cont[gi] = !brk;
        any_cont = any_cont || !brk;
      }
      memcpy(hg.cont, cont.data(), (size_t)G);
      CK(cudaMemcpyAsync(h->gc.cont, hg.cont, (size_t)G, cudaMemcpyHostToDevice, s));
      break_lookup(h);
      if (!any_cont) { looked_up = true; break; }
    }
    renumber_dense(h, n, g.gid);
    int64_t *loff_next = B ? (h->d_loff == h->d_loffb[0] ? h->d_loffb[1] : h->d_loffb[0]) : nullptr;
    if (B) next_level_ids(h, n, g.gid, h->gidL[slot], loff_next);
    int64_t ncomm = 0;
    {
      int64_t tot = 0;
      CK(cudaMemcpyAsync(&tot, h->lbuf0 + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      if (B) CK(cudaMemcpyAsync(loff_h.data(), loff_next, (size_t)(G + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      ncomm = tot;
    }
    lookup_dendrogram(h);
    // every aggregated level has at most the arcs of G^t (held since the
    // call's start; re-taken only if the batch outgrew the bound)
    if (!acquire_agg_buffers(h, h->g_arcs)) { h->err = "aggregation buffers (stream-ordered pool)"; return LEIDEN_ERR_OOM; }
    aggregate(h, g, ncomm, slot);
    reset_next_pass(h, ncomm, slot);
    level_maxdeg(h, h->y_deg[slot], ncomm);
    sync_counters(h);
    CK(cudaGetLastError());
    CKF();
    {
      // dense renumbering (36 B per vertex), lookup (12 B per vertex of G),
      // community-vertex lists (56 B per vertex), per community offsets,
      // bins, K'' and the next pass's state (81 B + a frontier bit); per arc
      // in: col, C of the neighbour and the weight; per super-arc out: col
      // and an 8-byte weight
      int64_t super_arcs = h->hcnt->deg_sum;
      ph_bytes(h, LEIDEN_PHASE_AGGREGATE, 92 * n + 12 * N + 81 * ncomm + ncomm / 8 +
                                              (8 + (g.w64 ? 8 : 4)) * level_arcs + 12 * super_arcs);
      level_arcs = super_arcs;
    }
    LevelGraph y;
    y.n = ncomm;
    y.off = h->y_off[slot];
    y.deg = h->y_deg[slot];
    y.col = h->y_col[slot];
    y.w = h->y_w[slot];
    y.w64 = true;
    y.maxdeg = h->hcnt->max_count;
    y.huge_slots = h->hcnt->huge_slots;
    if (B) {
      y.gid = h->gidL[slot];
      h->d_loff = loff_next;
      for (int gi = 0; gi < G; gi++) inlvl[gi] = cont[gi];
    }
    g = y;
    slot ^= 1;
    tau /= p.tau_drop;
  }
  ph_mark(h, LEIDEN_PHASE_TRACK);
  ph_bytes(h, LEIDEN_PHASE_TRACK, (B ? 0 : 12 * N) + 234 * N);  // final lookup; tracking's sweeps
  if (!B) lookup_dendrogram(h);
  else if (!looked_up) { h->err = "batched pass loop ended without a final lookup"; return LEIDEN_ERR_STATE; }
  track_communities(h);
  ph_mark(h, PHASE_END);
  release_agg_buffers(h);
  sync_counters(h);
  CK(cudaGetLastError());
  ph_resolve(h);
  if (unsigned int code = check_word_move() | check_word_phases() | check_word_track()) {
    h->err = "a device-side check of the checked build failed (code " + std::to_string(code) + ")";
    return LEIDEN_ERR_STATE;
  }
  h->trace[0] = passes;
  if (!B)
    for (int lp = 0; lp < passes && lp < 10; lp++) h->trace[2 + lp * 25 + 2] = h->hcnt->pass_ncomm[lp];
  st.passes = passes;
  st.lm_vertices = h->hcnt->processed;
  st.lm_arcs = h->hcnt->arcs;
  st.lm_moves = moves_total;
  st.refine_vertices = h->hcnt->ref_processed;
  st.refine_arcs = h->hcnt->ref_arcs;
  kt_resolve(h);
  int64_t visits = 0, decide_bytes = 0;
  for (int k = 0; k < 3; k++) {
    st.xk_launches[k] = h->kt_launches[KT_SPLIT_SAMPLE + k];
    st.xk_ms[k] = h->kt_ms[KT_SPLIT_SAMPLE + k];
    st.xk_bytes[k] = h->hcnt->xk_bytes[k];
  }
  st.agg_tables[0] = h->hcnt->agg_tables[0];
  st.agg_tables[1] = h->hcnt->agg_tables[1];
  for (int k = 0; k < 3; k++) {
    st.lmk_vertices[k] = h->hcnt->lmk_visits[k];
    st.lmk_arcs[k] = h->hcnt->lmk_arcs[k];
    st.lmk_bytes[k] = h->hcnt->lmk_bytes[k];
    st.lmk_launches[k] = h->kt_launches[k];
    st.lmk_ms[k] = h->kt_ms[k];
    visits += h->hcnt->lmk_visits[k];
    decide_bytes += h->hcnt->lmk_bytes[k];
  }
  // local moving: frontier words, the decide kernels' own count, 8 B per
  // visit to bin it (degree, list entry), 44 B per applied move
  ph_bytes(h, LEIDEN_PHASE_MOVE, 4 * subsweep_words + decide_bytes + 8 * visits + 44 * moves_total);
  // refinement: per visit 40 B of vertex state plus 40 B to list, bin and
  // accept it; per arc col, C, C'_B of the neighbour and the weight
  ph_bytes(h, LEIDEN_PHASE_REFINE, 80 * st.refine_vertices + 16 * st.refine_arcs);
  st.affected = h->hcnt->affected;
  return LEIDEN_OK;
}

// Pinned host staging of at least `bytes` (grows geometrically); false if it
// cannot be had, and the caller copies from pageable memory instead.
bool ensure_pinned(leiden_handle *h, size_t bytes) {
  if (bytes <= h->pin_bytes) return true;
  size_t want = std::max(bytes, 2 * h->pin_bytes);
  if (h->pin) {
    cudaStreamSynchronize(h->stream);
    cudaFreeHost(h->pin);
    h->pin = nullptr;
    h->pin_bytes = 0;
  }
  if (cudaMallocHost(&h->pin, want) != cudaSuccess) {
    cudaGetLastError();
    h->pin = nullptr;
    return false;
  }
  h->pin_bytes = want;
  return true;
}

leiden_status finish_call(leiden_handle *h, int32_t *out, bool device_out) {
  cudaStream_t s = h->stream;
  size_t bytes = (size_t)h->n * sizeof(int32_t);
  if (out && !device_out && ensure_pinned(h, bytes)) {
    // device -> pinned at full link speed, then one host copy
    CK(cudaMemcpyAsync(h->pin, h->C, bytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    memcpy(out, h->pin, bytes);
    return LEIDEN_OK;
  }
  if (out) CK(cudaMemcpyAsync(out, h->C, bytes, device_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return LEIDEN_OK;
}

leiden_status do_update(leiden_handle *h, const leiden_edge *d_del, int64_t n_del, const leiden_edge *d_ins,
                        int64_t n_ins, leiden_mode mode) {
  h->stats = leiden_stats{};
  h->ph_used = 0;
  kt_reset(h);
  // the aggregation arcs are taken before anything changes, so that running
  // out of memory leaves the handle as it was; the batch adds at most two
  // arcs per inserted edge
  if (!acquire_agg_buffers(h, h->g_arcs + 2 * n_ins)) {
    h->err = "aggregation buffers (stream-ordered pool)";
    return LEIDEN_ERR_OOM;
  }
  ph_mark(h, LEIDEN_PHASE_BATCH);
  leiden_status st = batch_apply_and_mark(h, d_del, n_del, d_ins, n_ins, (int)mode);
  if (st != LEIDEN_OK) {
    release_agg_buffers(h);
    return st;
  }
  ph_bytes(h, LEIDEN_PHASE_BATCH, 4 * h->n);  // degrees scanned for the bins
  level_maxdeg(h, h->g_deg, h->n);
  sync_all(h);
  if (cudaError_t e = cudaGetLastError()) {
    h->err = std::string("after the batch: ") + cudaGetErrorString(e);
    h->broken = true;
    return LEIDEN_ERR_CUDA;
  }
  h->m2 = h->hcnt->m2;
  if (h->G > 1) {
    GraphCounters hg = gc_layout(h->gc_host, h->G);
    for (int gi = 0; gi < h->G; gi++) h->m2g[gi] = hg.m2[gi];
  }
  h->g_maxdeg = h->hcnt->max_count;
  h->g_huge_slots = h->hcnt->huge_slots;
  st = run_leiden(h, 1, mode == LEIDEN_DS ? h->dV : nullptr);
  if (st != LEIDEN_OK) {
    h->broken = true;
    release_agg_buffers(h);
  }
  return st;
}

leiden_status check_handle(leiden_handle *h) {
  if (!h) return LEIDEN_ERR_ARG;
  if (h->broken) {
    h->err = "an earlier call failed after it began to change the handle (see its status); destroy it and "
             "create a new one, or import a saved state into a new one";
    return LEIDEN_ERR_STATE;
  }
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) {
    h->err = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
    return LEIDEN_ERR_CUDA;
  }
  return LEIDEN_OK;
}

}  // namespace

void set_handle_free_error(const std::string &msg) { g_create_error = msg; }

extern "C" {

void leiden_default_params(leiden_params *p) {
  if (!p) return;
  p->tau = 1e-2;
  p->tau_drop = 10.0;
  p->tau_refine = 0.6;
  p->max_iterations = 20;
  p->max_passes = 10;
  p->deterministic = 1;
  p->classes = 4;
  p->slack = 0.25;
  p->min_slack = 4;
  p->collect_stats = 0;
  p->split_all = 0;
  p->converge_any = 0;
  p->arena_log2 = 20;
}

leiden_status leiden_create(const leiden_params *params, int64_t n, const int64_t *offsets, const int32_t *cols,
                            const int32_t *weights, void *cuda_stream, leiden_handle **out) {
  g_create_error.clear();
  if (!out) { g_create_error = "out is NULL"; return LEIDEN_ERR_ARG; }
  *out = nullptr;
  if (n < 1 || n > 0x7ffffffe || !offsets || (offsets[n] > 0 && !cols)) {
    g_create_error = "invalid n, offsets or cols";
    return LEIDEN_ERR_ARG;
  }
  leiden_params p;
  leiden_default_params(&p);
  if (params) p = *params;
  if (p.classes < 1 || (p.classes & (p.classes - 1)) || p.max_iterations < 1 || p.max_passes < 1 || p.slack < 0 ||
      p.min_slack < 0 || p.tau_drop <= 0 || p.arena_log2 < 0 || p.arena_log2 > 30) {
    g_create_error = "invalid parameters (classes must be a power of two)";
    return LEIDEN_ERR_ARG;
  }
  // host validation and canonical rows
  int64_t arcs = offsets[n];
  if (offsets[0] != 0 || arcs < 0) { g_create_error = "offsets[0] must be 0"; return LEIDEN_ERR_ARG; }
  std::vector<int64_t> cap_off(n + 1, 0);
  std::vector<int32_t> deg(n);
  for (int64_t i = 0; i < n; i++) {
    int64_t d = offsets[i + 1] - offsets[i];
    if (d < 0 || d > 0x7fffffff) { g_create_error = "offsets not monotone"; return LEIDEN_ERR_ARG; }
    deg[i] = (int32_t)d;
    int64_t extra = std::max<int64_t>((int64_t)((double)d * p.slack), p.min_slack);
    cap_off[i + 1] = cap_off[i] + d + extra;
  }
  int64_t cap = cap_off[n];
  std::vector<int32_t> hcol((size_t)std::max<int64_t>(cap, 1), 0), hw((size_t)std::max<int64_t>(cap, 1), 0);
  int32_t maxdeg = 0;
  for (int64_t i = 0; i < n; i++) maxdeg = std::max<int32_t>(maxdeg, deg[i]);
  // rows canonicalised (sorted by neighbour) and checked on all host threads
  std::atomic<int> bad{0};  // 1 range/self-loop/weight, 2 repeated arc, 3 not symmetric
  host_parallel(n, [&](int64_t lo, int64_t hi) {
    std::vector<std::pair<int32_t, int32_t>> row;
    for (int64_t i = lo; i < hi && !bad.load(std::memory_order_relaxed); i++) {
      row.clear();
      bool sorted = true;
      for (int64_t a = offsets[i]; a < offsets[i + 1]; a++) {
        int32_t j = cols[a];
        int32_t w = weights ? weights[a] : 1;
        if (j < 0 || j >= n || j == i || w <= 0) { bad = 1; return; }
        if (!row.empty() && j <= row.back().first) sorted = false;
        row.emplace_back(j, w);
      }
      if (!sorted) std::sort(row.begin(), row.end());
      for (size_t k = 1; k < row.size(); k++)
        if (row[k].first == row[k - 1].first) { bad = 2; return; }
      for (size_t k = 0; k < row.size(); k++) {
        hcol[cap_off[i] + k] = row[k].first;
        hw[cap_off[i] + k] = row[k].second;
      }
    }
  });
  // symmetry: every arc (i, j, w) must have (j, i, w)
  if (!bad)
    host_parallel(n, [&](int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi && !bad.load(std::memory_order_relaxed); i++) {
        for (int64_t k = 0; k < deg[i]; k++) {
          int32_t j = hcol[cap_off[i] + k];
          const int32_t *rb = hcol.data() + cap_off[j];
          const int32_t *re = rb + deg[j];
          const int32_t *it = std::lower_bound(rb, re, (int32_t)i);
          if (it == re || *it != i || hw[cap_off[j] + (it - rb)] != hw[cap_off[i] + k]) { bad = 3; return; }
        }
      }
    });
  if (bad) {
    g_create_error = bad == 1 ? "column out of range, self-loop or weight <= 0"
                     : bad == 2 ? "repeated arc" : "graph is not symmetric";
    return LEIDEN_ERR_ARG;
  }
  leiden_handle *h = new leiden_handle();
  h->p = p;
  h->n = n;
  h->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&h->device);
  cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
  auto bail = [&](leiden_status st, const std::string &m) {
    g_create_error = m.empty() ? h->err : m;
    leiden_destroy(h);
    return st;
  };
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t x) { if (x != cudaSuccess && e == cudaSuccess) e = x; };
  // row capacities end at `cap`; the spill arena follows for rows that grow
  int64_t total = cap + spill_arena_size(cap, p.arena_log2);
  std::vector<int32_t> rcap(n);
  for (int64_t i = 0; i < n; i++) rcap[i] = (int32_t)(cap_off[i + 1] - cap_off[i]);
  A(dalloc(h, &h->g_off, n + 1));
  A(dalloc(h, &h->g_deg, n));
  A(dalloc(h, &h->g_rcap, n));
  A(dalloc(h, &h->g_col, total));
  A(dalloc(h, &h->g_w, total));
  A(dalloc(h, &h->C, n));
  A(dalloc(h, &h->K, n));
  A(dalloc(h, &h->Sig, n));
  A(dalloc(h, &h->dSig, n));
  A(dalloc(h, &h->dV, n));
  int32_t **i32s[] = {&h->Cp, &h->CB, &h->Ctop, &h->csize, &h->csize0, &h->rep, &h->prop, &h->parent,
                      &h->ibuf0, &h->ibuf1, &h->ibuf2, &h->movers, &h->mtarget, &h->cverts};
  for (auto pp : i32s) A(dalloc(h, pp, n + 1));
  int64_t **i64s[] = {&h->Kp, &h->Sp, &h->S2, &h->lbuf0, &h->lbuf1, &h->lbuf2, &h->lbuf3, &h->coff, &h->cflat};
  for (auto pp : i64s) A(dalloc(h, pp, n + 2));
  uint8_t **u8s[] = {&h->dS, &h->dR, &h->dS2, &h->dR2, &h->dE, &h->dCf};
  for (auto pp : u8s) A(dalloc(h, pp, n + 1));
  A(dalloc(h, &h->unproc, n / 32 + 2));
  A(dalloc(h, &h->bins, (int64_t)NBINS * n));
  A(dalloc(h, &h->hocc, n + 1));
  A(dalloc(h, &h->cand, 2 * n));
  for (int k = 0; k < 2; k++) {
    A(dalloc(h, &h->y_off[k], n + 2));
    A(dalloc(h, &h->y_deg[k], n + 1));
  }
  {
    // keep the pool's memory cached between calls instead of returning it
    // to the driver at every synchronisation
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, h->device) == cudaSuccess) {
      uint64_t keep = ~0ull;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
  }
  int64_t tc = 1;
  while (tc < 2 * n) tc <<= 1;
  A(dalloc(h, &h->tr_keys, tc));
  A(dalloc(h, &h->tr_vals, tc));
  A(dalloc(h, &h->tr_list, n));
  h->tr_cap = tc;
  A(dalloc(h, &h->dcnt, 1));
  size_t stb = scan_tmp_bytes(2 * n + 2);
  void *stp = nullptr;
  A(cudaMalloc(&stp, stb));
  if (stp) { h->owned.push_back(stp); h->scan_tmp = stp; h->scan_tmp_bytes = stb; }
  A(cudaMallocHost((void **)&h->hcnt, sizeof(DevCounters)));
  if (e != cudaSuccess)
    return bail(e == cudaErrorMemoryAllocation ? LEIDEN_ERR_OOM : LEIDEN_ERR_CUDA,
                std::string("device allocation: ") + cudaGetErrorString(e));
  cudaStream_t s = h->stream;
  A(cudaMemcpyAsync(h->g_off, cap_off.data(), (size_t)(n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  A(cudaMemcpyAsync(h->g_deg, deg.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  A(cudaMemcpyAsync(h->g_col, hcol.data(), (size_t)cap * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  A(cudaMemcpyAsync(h->g_w, hw.data(), (size_t)cap * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  A(cudaMemcpyAsync(h->g_rcap, rcap.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  A(cudaMemsetAsync(h->dcnt, 0, sizeof(DevCounters), s));
  A(cudaMemsetAsync(h->tr_keys, 0xff, (size_t)h->tr_cap * sizeof(uint64_t), s));  // empty pair table
  A(cudaMemsetAsync(h->tr_vals, 0, (size_t)h->tr_cap * sizeof(int64_t), s));
  A(cudaMemcpyAsync(&h->dcnt->arena_used, &cap, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  A(cudaStreamSynchronize(s));
  if (e != cudaSuccess) return bail(LEIDEN_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
  h->g_cap = total;
  h->g_arcs = arcs;
  h->g_maxdeg = maxdeg;
  ensure_hslots(h, level0_huge_slots(deg));  // grows on demand for aggregated levels
  *out = h;
  return LEIDEN_OK;
}

leiden_status leiden_create_batched(const leiden_params *params, int32_t graphs, const int64_t *vertex_offsets,
                                    const int64_t *offsets, const int32_t *cols, const int32_t *weights,
                                    void *cuda_stream, leiden_handle **out) {
  g_create_error.clear();
  if (!out) { g_create_error = "out is NULL"; return LEIDEN_ERR_ARG; }
  *out = nullptr;
  if (graphs < 1 || !vertex_offsets || vertex_offsets[0] != 0) {
    g_create_error = "invalid graph count or vertex offsets";
    return LEIDEN_ERR_ARG;
  }
  for (int32_t gi = 0; gi < graphs; gi++)
    if (vertex_offsets[gi + 1] <= vertex_offsets[gi]) {
      g_create_error = "every graph needs at least one vertex (vertex offsets strictly increasing)";
      return LEIDEN_ERR_ARG;
    }
  if (params && !params->deterministic && graphs > 1) {
    g_create_error = "batched handles run the deterministic (snapshot) schedule";
    return LEIDEN_ERR_ARG;
  }
  int64_t n = vertex_offsets[graphs];
  if (n < 1 || n > 0x7ffffffe || !offsets) { g_create_error = "invalid vertex count"; return LEIDEN_ERR_ARG; }
  std::vector<int32_t> gid((size_t)n);
  for (int32_t gi = 0; gi < graphs; gi++)
    for (int64_t v = vertex_offsets[gi]; v < vertex_offsets[gi + 1]; v++) gid[v] = gi;
  for (int64_t v = 0; v < n; v++)
    for (int64_t a = offsets[v]; a < offsets[v + 1]; a++)
      if (cols && cols[a] >= 0 && cols[a] < n && gid[cols[a]] != gid[v]) {
        g_create_error = "an arc joins two graphs of the batch";
        return LEIDEN_ERR_ARG;
      }
  leiden_handle *h = nullptr;
  leiden_status st = leiden_create(params, n, offsets, cols, weights, cuda_stream, &h);
  if (st != LEIDEN_OK) return st;
  if (graphs == 1) { *out = h; return LEIDEN_OK; }
  h->G = graphs;
  h->voff.assign(vertex_offsets, vertex_offsets + graphs + 1);
  h->m2g.assign(graphs, 0);
  h->gc_bytes = gc_block_bytes(graphs);
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t x) { if (x != cudaSuccess && e == cudaSuccess) e = x; };
  void *gcd = nullptr;
  A(cudaMalloc(&gcd, h->gc_bytes));
  if (gcd) h->owned.push_back(gcd);
  A(cudaMallocHost(&h->gc_host, h->gc_bytes));
  A(dalloc(h, &h->d_voff, graphs + 1));
  A(dalloc(h, &h->d_loffb[0], graphs + 1));
  A(dalloc(h, &h->d_loffb[1], graphs + 1));
  A(dalloc(h, &h->gid0, n));
  A(dalloc(h, &h->gidL[0], n));
  A(dalloc(h, &h->gidL[1], n));
  A(dalloc(h, &h->mgain, 2 * n));
  if (e == cudaSuccess) {
    h->gc = gc_layout(gcd, graphs);
    h->d_loff = h->d_loffb[0];
    A(cudaMemsetAsync(gcd, 0, h->gc_bytes, h->stream));
    A(cudaMemcpyAsync(h->d_voff, vertex_offsets, (size_t)(graphs + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                      h->stream));
    A(cudaMemcpyAsync(h->gid0, gid.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    A(cudaStreamSynchronize(h->stream));
  }
  if (e != cudaSuccess) {
    g_create_error = std::string("batched allocation: ") + cudaGetErrorString(e);
    leiden_destroy(h);
    return e == cudaErrorMemoryAllocation ? LEIDEN_ERR_OOM : LEIDEN_ERR_CUDA;
  }
  *out = h;
  return LEIDEN_OK;
}

int32_t leiden_batch_graphs(const leiden_handle *h) { return h ? h->G : 0; }

int64_t leiden_footprint_bytes(const leiden_params *params, int64_t n, const int64_t *offsets) {
  if (n < 1 || !offsets) return -1;
  leiden_params p;
  leiden_default_params(&p);
  if (params) p = *params;
  int64_t cap = 0;
  std::vector<int32_t> deg((size_t)n);
  for (int64_t i = 0; i < n; i++) {
    int64_t d = offsets[i + 1] - offsets[i];
    deg[i] = (int32_t)d;
    cap += d + std::max<int64_t>((int64_t)((double)d * p.slack), p.min_slack);
  }
  int64_t total = cap + spill_arena_size(cap, p.arena_log2);
  int64_t tc = 1;
  while (tc < 2 * n) tc <<= 1;
  int64_t hs = (level0_huge_slots(deg) + 1023) & ~(int64_t)1023;
  int64_t b = 0;
  b += 8 * (n + 1) + 8 * n + 8 * total;                              // G^t: off, deg, rcap, col, w
  b += 4 * n + 24 * n + n;                                            // C, K, Sigma, dSigma, dV
  b += 56 * (n + 1) + 72 * (n + 2) + 6 * (n + 1);                     // per-pass work arrays
  b += 4 * (n / 32 + 2) + 16 * n + 4 * (n + 1) + 8 * n;               // frontier, bins, hocc, cand
  b += 2 * (8 * (n + 2) + 4 * (n + 1));                              // aggregated levels' offsets, degrees
  b += 16 * tc + 4 * n + (int64_t)scan_tmp_bytes(2 * n + 2);          // tracking, scans
  b += 16 * hs;                                                       // hub tables at level 0
  b += 8 * n + n / 8 + ((int64_t)32 << 20);                          // batch buffers, touched-row bits
  return b;
}

leiden_status leiden_batch_trace(leiden_handle *h, int32_t graph, int64_t *trace) {
  if (!h || !trace || graph < 0 || graph >= h->G) return LEIDEN_ERR_ARG;
  if (h->G == 1) return leiden_get_trace(h, trace);
  if (h->gtrace.size() < (size_t)h->G * TRACE_WORDS) { memset(trace, 0, TRACE_WORDS * sizeof(int64_t)); return LEIDEN_OK; }
  memcpy(trace, &h->gtrace[(size_t)graph * TRACE_WORDS], TRACE_WORDS * sizeof(int64_t));
  std::vector<uint8_t> dV((size_t)h->n);
  if (leiden_get_affected(h, dV.data()) == LEIDEN_OK) {
    int64_t k = 0;
    for (int64_t v = h->voff[graph]; v < h->voff[graph + 1]; v++) k += dV[v];
    trace[1] = k;
  }
  return LEIDEN_OK;
}

leiden_status leiden_batch_modularity(leiden_handle *h, double *q_out) {
  leiden_status st = check_handle(h);
  if (st != LEIDEN_OK) return st;
  if (!q_out) return LEIDEN_ERR_ARG;
  if (h->G == 1) return leiden_modularity(h, nullptr, q_out);
  modularity_terms(h, h->C);
  sync_all(h);
  CK(cudaGetLastError());
  GraphCounters hg = gc_layout(h->gc_host, h->G);
  for (int gi = 0; gi < h->G; gi++) {
    int64_t m2 = h->m2g[gi];
    if (m2 == 0) { q_out[gi] = 0.0; continue; }
    i128 num = (i128)m2 * hg.sigma[gi] - read_i128(&hg.sq[2 * gi]);
    q_out[gi] = i128_to_double(num) / ((double)m2 * (double)m2);
  }
  return LEIDEN_OK;
}

leiden_status leiden_static(leiden_handle *h, int32_t *membership_out) {
  leiden_status st = check_handle(h);
  if (st != LEIDEN_OK) return st;
  cudaStream_t s = h->stream;
  h->stats = leiden_stats{};
  h->ph_used = 0;
  kt_reset(h);
  if (!acquire_agg_buffers(h, h->g_arcs)) { h->err = "aggregation buffers (stream-ordered pool)"; return LEIDEN_ERR_OOM; }
  ph_mark(h, LEIDEN_PHASE_BATCH);
  int64_t N = h->n;
  // row sums (offsets, degree, K: 20 B per vertex; a weight per arc), degree
  // scan, C, sizes, Sigma, Delta Sigma and the flags
  ph_bytes(h, LEIDEN_PHASE_BATCH, 59 * N + 4 * h->g_arcs);
  recompute_weights(h);
  level_maxdeg(h, h->g_deg, N);
  launch_iota_i32(h->C, N, s);
  launch_fill_i32(h->csize0, 1, N, s);  // singletons: tracking updates the counts by the vertices that move
  CK(cudaMemcpyAsync(h->Sig, h->K, (size_t)N * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(h->dSig, 0, (size_t)N * sizeof(int64_t), s));
  CK(cudaMemsetAsync(h->dV, 1, (size_t)N, s));
  CK(cudaMemsetAsync(h->dS, 0, (size_t)N, s));
  CK(cudaMemsetAsync(h->dR, 1, (size_t)N, s));
  sync_all(h);
  CK(cudaGetLastError());
  h->m2 = h->hcnt->m2;
  if (h->G > 1) {
    GraphCounters hg = gc_layout(h->gc_host, h->G);
    for (int gi = 0; gi < h->G; gi++) h->m2g[gi] = hg.m2[gi];
  }
  h->g_maxdeg = h->hcnt->max_count;
  h->g_huge_slots = h->hcnt->huge_slots;
  st = run_leiden(h, 0, nullptr);
  if (st != LEIDEN_OK) {
    h->broken = true;
    release_agg_buffers(h);
    return st;
  }
  h->has_static = true;
  return finish_call(h, membership_out, false);
}

leiden_status leiden_update(leiden_handle *h, const leiden_edge *del, int64_t n_del, const leiden_edge *ins,
                            int64_t n_ins, leiden_mode mode, int32_t *membership_out) {
  leiden_status st = check_handle(h);
  if (st != LEIDEN_OK) return st;
  if (!h->has_static) { h->err = "leiden_update before leiden_static"; return LEIDEN_ERR_STATE; }
  if (n_del < 0 || n_ins < 0 || (n_del && !del) || (n_ins && !ins) || mode < LEIDEN_ND || mode > LEIDEN_DF) {
    h->err = "invalid batch arguments";
    return LEIDEN_ERR_ARG;
  }
  // stage the host batch in device memory (upload buffers grow on demand)
  int64_t need = std::max<int64_t>(std::max(n_del, n_ins), 1);
  if (need > h->up_cap) {
    need = std::max<int64_t>(need, 2 * h->up_cap);  // geometric growth (fewer device-wide frees)
    for (auto &q : h->owned)
      if (q && (q == h->up_del || q == h->up_ins)) { cudaFree(q); q = nullptr; }
    h->up_del = h->up_ins = nullptr;
    h->up_cap = 0;
    CK(dalloc(h, &h->up_del, need));
    CK(dalloc(h, &h->up_ins, need));
    h->up_cap = need;
  }
  leiden_edge *dd = h->up_del, *di = h->up_ins;
  size_t bd = (size_t)n_del * sizeof(leiden_edge), bi = (size_t)n_ins * sizeof(leiden_edge);
  CK(cudaStreamSynchronize(h->stream));  // the pinned buffer may still feed an earlier copy
  if (ensure_pinned(h, bd + bi)) {
    // host -> pinned, then one asynchronous copy each at full link speed
    char *pp = (char *)h->pin;
    if (n_del) { memcpy(pp, del, bd); CK(cudaMemcpyAsync(dd, pp, bd, cudaMemcpyHostToDevice, h->stream)); }
    if (n_ins) { memcpy(pp + bd, ins, bi); CK(cudaMemcpyAsync(di, pp + bd, bi, cudaMemcpyHostToDevice, h->stream)); }
  } else {
    if (n_del) CK(cudaMemcpyAsync(dd, del, bd, cudaMemcpyHostToDevice, h->stream));
    if (n_ins) CK(cudaMemcpyAsync(di, ins, bi, cudaMemcpyHostToDevice, h->stream));
  }
  st = do_update(h, dd, n_del, di, n_ins, mode);
  if (st != LEIDEN_OK) return st;
  return finish_call(h, membership_out, false);
}

leiden_status leiden_update_device(leiden_handle *h, const leiden_edge *del, int64_t n_del, const leiden_edge *ins,
                                   int64_t n_ins, leiden_mode mode, int32_t *membership_out) {
  leiden_status st = check_handle(h);
  if (st != LEIDEN_OK) return st;
  if (!h->has_static) { h->err = "leiden_update_device before leiden_static"; return LEIDEN_ERR_STATE; }
  if (n_del < 0 || n_ins < 0 || (n_del && !del) || (n_ins && !ins) || mode < LEIDEN_ND || mode > LEIDEN_DF) {
    h->err = "invalid batch arguments";
    return LEIDEN_ERR_ARG;
  }
  st = do_update(h, del, n_del, ins, n_ins, mode);
  if (st != LEIDEN_OK) return st;
  return finish_call(h, membership_out, true);
}

leiden_status leiden_modularity(leiden_handle *h, const int32_t *membership, double *q_out) {
  leiden_status st = check_handle(h);
  if (st != LEIDEN_OK) return st;
  if (!q_out) { h->err = "q_out is NULL"; return LEIDEN_ERR_ARG; }
  cudaStream_t s = h->stream;
  const int32_t *C = h->C;
  if (membership) {
    for (int64_t i = 0; i < h->n; i++)
      if (membership[i] < 0 || membership[i] >= h->n) { h->err = "membership id out of range"; return LEIDEN_ERR_ARG; }
    CK(cudaMemcpyAsync(h->ibuf2, membership, (size_t)h->n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    C = h->ibuf2;
  }
  // K must be the row sums of G^t (it is, after static/update); before the
  // first static call compute them.
  if (!h->has_static) {
    recompute_weights(h);
    sync_counters(h);
    h->m2 = h->hcnt->m2;
  }
  modularity_terms(h, C);
  sync_counters(h);
  CK(cudaGetLastError());
  int64_t m2 = h->m2;
  if (m2 == 0) { *q_out = 0.0; return LEIDEN_OK; }
  i128 num = (i128)m2 * h->hcnt->sigma_intra - read_i128(h->hcnt->sq);
  *q_out = i128_to_double(num) / ((double)m2 * (double)m2);
  return LEIDEN_OK;
}

leiden_status leiden_membership_device(leiden_handle *h, const int32_t **d_membership) {
  if (!h || !d_membership) return LEIDEN_ERR_ARG;
  *d_membership = h->C;
  return LEIDEN_OK;
}

leiden_status leiden_get_state(leiden_handle *h, int32_t *C, int64_t *K, int64_t *Sigma, int64_t *dSigma,
                               int64_t *m2) {
  leiden_status st = check_handle(h);
  if (st != LEIDEN_OK) return st;
  cudaStream_t s = h->stream;
  size_t n = (size_t)h->n;
  if (C) CK(cudaMemcpyAsync(C, h->C, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  if (K) CK(cudaMemcpyAsync(K, h->K, n * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  if (Sigma) CK(cudaMemcpyAsync(Sigma, h->Sig, n * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  if (dSigma) CK(cudaMemcpyAsync(dSigma, h->dSig, n * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (m2) *m2 = h->m2;
  return LEIDEN_OK;
}

leiden_status leiden_import_state(leiden_handle *h, const int32_t *C, const int64_t *dSigma) {
  leiden_status st = check_handle(h);
  if (st != LEIDEN_OK) return st;
  if (!C || !dSigma) return LEIDEN_ERR_ARG;
  int64_t N = h->n;
  for (int64_t i = 0; i < N; i++)
    if (C[i] < 0 || C[i] >= N) { h->err = "membership id out of range"; return LEIDEN_ERR_ARG; }
  if (h->G > 1)
    for (int32_t gi = 0; gi < h->G; gi++)
      for (int64_t i = h->voff[gi]; i < h->voff[gi + 1]; i++)
        if (C[i] < h->voff[gi] || C[i] >= h->voff[gi + 1]) {
          h->err = "membership id outside its graph's range";
          return LEIDEN_ERR_ARG;
        }
  cudaStream_t s = h->stream;
  // K and 2m from G^t, Sigma from K and C (Approach: the auxiliary
  // information is a function of the graph and the membership, plus the
  // accumulated Delta Sigma)
  recompute_weights(h);
  CK(cudaMemcpyAsync(h->C, C, (size_t)N * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->dSig, dSigma, (size_t)N * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));  // the host arrays may be freed on return
  recompute_sigma(h);
  count_sizes(h, h->C, N, h->csize0);
  sync_all(h);
  CK(cudaGetLastError());
  h->m2 = h->hcnt->m2;
  if (h->G > 1) {
    GraphCounters hg = gc_layout(h->gc_host, h->G);
    for (int gi = 0; gi < h->G; gi++) h->m2g[gi] = hg.m2[gi];
  }
  level_maxdeg(h, h->g_deg, N);
  sync_counters(h);
  h->g_maxdeg = h->hcnt->max_count;
  h->g_huge_slots = h->hcnt->huge_slots;
  h->has_static = true;
  return LEIDEN_OK;
}

void leiden_default_tuning(leiden_tuning *t) {
  if (t) *t = leiden_tuning{8, BIN_WARP_MAX, BIN_BLOCK_MAX, 4, 7, 16, 1};
}

leiden_status leiden_set_tuning(leiden_handle *h, const leiden_tuning *t) {
  if (!h || !t) return LEIDEN_ERR_ARG;
  if (t->tiny_max < 0 || t->tiny_max > 8 || t->warp_max < t->tiny_max || t->warp_max > BIN_WARP_MAX ||
      t->block_max < t->warp_max || t->block_max > BIN_BLOCK_MAX || t->warp_blocks_per_sm < 1 ||
      t->warp_blocks_per_sm > 8 || t->block_blocks_per_sm < 1 || t->block_blocks_per_sm > 8 ||
      t->hub_blocks_per_sm < 1 || t->hub_blocks_per_sm > 32 || t->overlap < 0 || t->overlap > 1) {
    h->err = "tuning outside its ranges";
    return LEIDEN_ERR_ARG;
  }
  h->tune = *t;
  // hub tables are sized for the vertices above block_max
  level_maxdeg(h, h->g_deg, h->n);
  sync_counters(h);
  h->g_maxdeg = h->hcnt->max_count;
  h->g_huge_slots = h->hcnt->huge_slots;
  return LEIDEN_OK;
}

int64_t leiden_graph_arcs(leiden_handle *h) { return h ? h->g_arcs : -1; }

leiden_status leiden_get_graph(leiden_handle *h, int64_t *off, int32_t *col, int64_t *w) {
  leiden_status st = check_handle(h);
  if (st != LEIDEN_OK) return st;
  if (!off || (h->g_arcs && (!col || !w))) { h->err = "null output"; return LEIDEN_ERR_ARG; }
  cudaStream_t s = h->stream;
  int64_t n = h->n;
  std::vector<int64_t> goff(n + 1);
  std::vector<int32_t> gdeg(n), gcol((size_t)h->g_cap), gw((size_t)h->g_cap);
  CK(cudaMemcpyAsync(goff.data(), h->g_off, (size_t)(n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(gdeg.data(), h->g_deg, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(gcol.data(), h->g_col, (size_t)h->g_cap * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(gw.data(), h->g_w, (size_t)h->g_cap * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  off[0] = 0;
  for (int64_t i = 0; i < n; i++) {
    off[i + 1] = off[i] + gdeg[i];
    for (int64_t k = 0; k < gdeg[i]; k++) {
      col[off[i] + k] = gcol[goff[i] + k];
      w[off[i] + k] = gw[goff[i] + k];
    }
  }
  if (off[n] != h->g_arcs) { h->err = "arc count mismatch"; return LEIDEN_ERR_STATE; }
  return LEIDEN_OK;
}

leiden_status leiden_get_affected(leiden_handle *h, uint8_t *dV) {
  leiden_status st = check_handle(h);
  if (st != LEIDEN_OK) return st;
  if (!dV) return LEIDEN_ERR_ARG;
  CK(cudaMemcpyAsync(dV, h->dV, (size_t)h->n, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return LEIDEN_OK;
}

leiden_status leiden_get_trace(leiden_handle *h, int64_t *trace) {
  if (!h || !trace) return LEIDEN_ERR_ARG;
  memcpy(trace, h->trace, sizeof(h->trace));
  // |dV| (computed on demand)
  std::vector<uint8_t> dV((size_t)h->n);
  if (leiden_get_affected(h, dV.data()) == LEIDEN_OK) {
    int64_t k = 0;
    for (uint8_t x : dV) k += x;
    trace[1] = k;
  }
  return LEIDEN_OK;
}

leiden_status leiden_get_stats(leiden_handle *h, leiden_stats *stats) {
  if (!h || !stats) return LEIDEN_ERR_ARG;
  *stats = h->stats;
  return LEIDEN_OK;
}

int64_t leiden_transient_bytes(int64_t n, const int64_t *offsets) {
  if (n < 1 || !offsets) return -1;
  return agg_buffer_bytes(offsets[n]);
}

int64_t leiden_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int32_t leiden_checked_build(void) {
#ifdef LEIDEN_CHECKED
  return 1;
#else
  return 0;
#endif
}

int32_t leiden_check_selftest(void *cuda_stream) { return (int32_t)check_selftest((cudaStream_t)cuda_stream); }

const char *leiden_last_error(leiden_handle *h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

void leiden_destroy(leiden_handle *h) {
  if (!h) return;
  cudaSetDevice(h->device);
  release_agg_buffers(h);
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (void *q : h->owned)
    if (q) cudaFree(q);
  if (h->hcnt) cudaFreeHost(h->hcnt);
  if (h->gc_host) cudaFreeHost(h->gc_host);
  if (h->pin) cudaFreeHost(h->pin);
  for (auto &ev : h->ph_ev)
    if (ev) cudaEventDestroy(ev);
  for (auto &ev : h->kt_ev)
    if (ev) cudaEventDestroy(ev);
  for (int k = 0; k < 2; k++) {
    if (h->side[k]) cudaStreamDestroy(h->side[k]);
    if (h->join_ev[k]) cudaEventDestroy(h->join_ev[k]);
  }
  if (h->fork_ev) cudaEventDestroy(h->fork_ev);
  delete h;
}

}  // extern "C"
