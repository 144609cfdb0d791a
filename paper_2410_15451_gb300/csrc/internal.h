// Internal host-side declarations of the GB300 dynamic Leiden library: the
// handle, its device buffers, and the launchers each .cu file provides.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/leiden_gb300.h"
#include "common.cuh"

// A level of the dendrogram as the kernels see it: rows off[i] .. off[i] + deg[i].
struct LevelGraph {
  int64_t n = 0;
  const int64_t *off = nullptr;
  const int32_t *deg = nullptr;
  const int32_t *col = nullptr;
  const void *w = nullptr;  // int32 at level 0, int64 above
  bool w64 = false;
  int32_t maxdeg = 0;
  int64_t huge_slots = 0;  // sum over vertices above BIN_BLOCK_MAX of pow2 >= 2*degree
  const int32_t *gid = nullptr;  // batched handles: graph of each vertex (null: one graph)
};

// Per-graph device counters of a batched handle (G graphs), one allocation.
struct GraphCounters {
  unsigned long long *dq = nullptr;  // [2G] local-moving gains of the iteration (int128)
  int64_t *moves = nullptr;          // [G] local-moving moves of the iteration
  int64_t *m2 = nullptr;             // [G] 2m of each graph
  int32_t *accepted = nullptr;       // [G] refinement moves accepted in the round
  int32_t *ncomm = nullptr;          // [G] communities after refinement
  int64_t *sigma = nullptr;          // [G] modularity: intra-community arc weight
  unsigned long long *sq = nullptr;  // [2G] modularity: sum of Sigma_c^2 (int128)
  uint8_t *refined = nullptr;        // [G] a vertex of the graph lies in a refined bound
  uint8_t *lm_on = nullptr;          // [G] still iterating local moving (host-written)
  uint8_t *cont = nullptr;           // [G] continues to the next pass (host-written)
};

// Degree bins of the vertex-centric kernels (local moving, refinement).
enum { BIN_WARP = 0, BIN_BLOCK = 1, BIN_HUGE = 2, BIN_TINY = 3, NBINS = 4 };
constexpr int BIN_TINY_MAX = 8;      // eight lanes, one arc per lane (local moving, refinement)
constexpr int BIN_WARP_MAX = 128;    // one warp, shared table of <= 256 slots
constexpr int BIN_BLOCK_MAX = 1024;  // one block, shared table of 2048 slots
// Kernels with their own live timer (event pairs, collect_stats bit 2) and
// algorithmic-byte counters: the three local-moving kernels, and the
// largest kernels of the other phases (split sampling, the chunked scan of
// giant communities in aggregation, the block merge of touched rows).
enum { KT_WARP = 0, KT_BLOCK = 1, KT_HUGE_SCAN = 2, KT_SPLIT_SAMPLE = 3, KT_AGG_CHUNK = 4, KT_MERGE_MID = 5,
       KT_KERNELS = 6 };

struct BatchBuffers {
  int64_t cap_edges = 0;  // capacity in undirected edges, per side
  uint64_t *dkey = nullptr, *dkey_alt = nullptr;         // deletion arcs (src<<32|dst)
  uint64_t *ikey = nullptr, *ikey_alt = nullptr;         // insertion arcs
  int64_t *iw = nullptr, *iw_alt = nullptr;              // insertion weights
  int64_t *dw = nullptr;                                 // stored weights of deleted arcs
  int32_t *flag = nullptr;                               // scan flags
  int64_t *pos = nullptr;                                // scan output
  int32_t *ins_state = nullptr;                          // 1 = existing arc, 0 = new arc
  int64_t *ins_pos = nullptr;                            // arc index of existing insertions
  int32_t *rows = nullptr;                               // touched rows
  int32_t *row_dlo = nullptr, *row_dhi = nullptr;        // deletion arc range of a row
  int32_t *row_ilo = nullptr, *row_ihi = nullptr;        // insertion arc range of a row
  int64_t *row_len = nullptr;                            // new row length
  int64_t *row_tmp_off = nullptr;                        // offset into the merge buffer
  int64_t *row_dst = nullptr;                            // where the merged row goes
  int32_t *row_newcap = nullptr;                         // capacity of a relocated row (0: stays)
  int32_t *row_olddeg = nullptr;                         // degree of the row before the batch
  int32_t *row_large = nullptr;                          // touched rows merged in chunks
  int32_t *row_mid = nullptr;                            // touched rows merged by one block each
  uint64_t *ds_key = nullptr, *ds_key_alt = nullptr, *ds_ukey = nullptr;  // DS (src, C[dst]) pairs
  int64_t *ds_w = nullptr, *ds_w_alt = nullptr, *ds_uw = nullptr;
  int64_t *counts = nullptr;                             // device counts of the batch pipeline (in DevCounters)
  uint32_t *row_bits = nullptr;                          // one bit per vertex, all clear between calls
  int32_t *tmp_col = nullptr;                            // merged rows
  int32_t *tmp_w = nullptr;
  int64_t tmp_cap = 0;
};

struct leiden_handle {
  leiden_params p{};
  leiden_tuning tune{8, BIN_WARP_MAX, BIN_BLOCK_MAX, 4, 7, 16, 1};
  cudaStream_t stream = nullptr;
  // side streams of the local-moving and refinement bins (created on first
  // use): the block bin and the hub path run beside the warp bin
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t fork_ev = nullptr, join_ev[2] = {nullptr, nullptr};
  bool side_failed = false;
  int device = 0;
  int sm_count = 152;
  int64_t n = 0;

  // G^t: device CSR with slack
  int64_t *g_off = nullptr;  // [n+1] row starts
  int32_t *g_deg = nullptr;  // [n]
  int32_t *g_rcap = nullptr; // [n] row capacities (rows that outgrow them move to the spill arena)
  int32_t *g_col = nullptr;  // [g_cap]
  int32_t *g_w = nullptr;    // [g_cap]
  int64_t g_cap = 0;
  int64_t g_arcs = 0;
  int32_t g_maxdeg = 0;
  int64_t g_huge_slots = 0;
  int64_t m2 = 0;            // 2m = sum of arc weights

  // auxiliary state {C, K, Sigma, Delta Sigma}
  int32_t *C = nullptr;
  int64_t *K = nullptr, *Sig = nullptr, *dSig = nullptr;
  uint8_t *dV = nullptr;
  bool has_static = false;
  // A call that failed after it began to change the handle's state (a
  // failed allocation or CUDA error mid-call) leaves it broken: every later
  // call that needs the state returns LEIDEN_ERR_STATE.
  bool broken = false;

  // per-vertex work arrays (length n or n+1)
  int32_t *Cp = nullptr, *CB = nullptr, *Ctop = nullptr, *csize = nullptr, *rep = nullptr;
  int32_t *csize0 = nullptr;  // [n] member counts of C^t (kept by tracking for the next call)
  int32_t *prop = nullptr, *parent = nullptr, *ibuf0 = nullptr, *ibuf1 = nullptr, *ibuf2 = nullptr;
  int64_t *Kp = nullptr, *Sp = nullptr, *S2 = nullptr, *lbuf0 = nullptr, *lbuf1 = nullptr;
  int64_t *lbuf2 = nullptr, *lbuf3 = nullptr;
  uint8_t *dS = nullptr, *dR = nullptr, *dS2 = nullptr, *dR2 = nullptr, *dE = nullptr, *dCf = nullptr;
  uint32_t *unproc = nullptr;  // bitmap, words = n/32 + 2
  int32_t *bins = nullptr;     // NBINS * n
  int32_t *movers = nullptr;   // [n]
  int32_t *mtarget = nullptr;  // [n]
  int32_t *cand = nullptr;     // 2 * n

  // aggregation (ping-pong super-vertex graphs)
  int64_t *coff = nullptr;   // [n+1] community vertex offsets
  int32_t *cverts = nullptr; // [n]
  int64_t *cflat = nullptr;  // [n+1] flat arc offsets in cverts order
  int64_t *y_off[2] = {nullptr, nullptr};
  int32_t *y_deg[2] = {nullptr, nullptr};
  // The arcs of the two aggregated levels (y_col, y_w: 12 B per arc of G^t
  // each) are drawn from the device's stream-ordered memory pool when a call
  // first aggregates and returned at its end, so a resident graph does not
  // hold them between calls (most DF updates never aggregate).
  int32_t *y_col[2] = {nullptr, nullptr};
  int64_t *y_w[2] = {nullptr, nullptr};
  int64_t y_slots = 0;  // arc slots of the buffers held (0: none)

  // global hash scratch for the largest vertices / communities (kept clean)
  void *hscratch = nullptr;
  size_t hscratch_bytes = 0;
  int64_t hslots = 0;
  int32_t *hocc = nullptr;  // [n] filled slots per listed vertex

  // tracking hash table of (old, new) pairs (empty between calls) and the
  // list of its filled slots
  uint64_t *tr_keys = nullptr;
  int64_t *tr_vals = nullptr;
  int32_t *tr_list = nullptr;
  int64_t tr_cap = 0;

  // scan scratch
  void *scan_tmp = nullptr;
  size_t scan_tmp_bytes = 0;

  DevCounters *dcnt = nullptr;  // device
  DevCounters *hcnt = nullptr;  // pinned host mirror

  // Batched handles: G graphs concatenated with vertex offsets voff (graph g
  // owns vertices and community ids [voff[g], voff[g+1])).  Every kernel
  // covers all graphs in one launch; 2m, convergence, pass breaks, tracking
  // ranges and traces are per graph.  G == 1: the single-graph path, and
  // gid0 / gidL / gc stay null.
  int G = 1;
  std::vector<int64_t> voff;          // host [G+1]
  int64_t *d_voff = nullptr;          // device [G+1]
  int32_t *gid0 = nullptr;            // device [n] graph of each vertex of G^t
  int32_t *gidL[2] = {nullptr, nullptr};  // graph of each super-vertex (ping-pong with y_*)
  int64_t *d_loff = nullptr;          // device [G+1] level offsets of the current level
  int64_t *d_loffb[2] = {nullptr, nullptr};  // the two buffers d_loff alternates between
  int64_t *mgain = nullptr;           // device [2n] gain (lo, hi) of each deferred move
  GraphCounters gc;                   // device
  void *gc_host = nullptr;            // pinned host copy of the gc block
  size_t gc_bytes = 0;
  std::vector<int64_t> m2g;           // host 2m of each graph
  std::vector<int64_t> gtrace;        // host per-graph traces, G x (2 + 10*25)

  BatchBuffers b;
  leiden_edge *up_del = nullptr, *up_ins = nullptr;  // staging of host batches
  int64_t up_cap = 0;
  void *pin = nullptr;      // pinned host staging: batches in, membership out
  size_t pin_bytes = 0;

  // Phase timer (collect_stats bit 1): an event recorded on the stream at
  // each phase boundary, tagged with the phase that starts there, and read
  // after the call's last host sync.
  std::vector<cudaEvent_t> ph_ev;
  std::vector<int> ph_tag;
  int ph_used = 0;
  // Kernel timer (collect_stats bit 2): event pairs around the launches of
  // the local-moving kernels, resolved at the next host sync.
  std::vector<cudaEvent_t> kt_ev;
  std::vector<int> kt_tag;  // timed kernel of each recorded pair
  int kt_used = 0;          // pairs recorded since the last resolve
  double kt_ms[KT_KERNELS] = {};
  int64_t kt_launches[KT_KERNELS] = {};
  leiden_stats stats{};
  int64_t trace[2 + 10 * 25] = {};
  std::string err;
  leiden_status fatal = LEIDEN_OK;  // set by a launcher that could not run
  std::vector<void *> owned;  // every cudaMalloc of the handle
};

// int128 -> double in a fixed order (|x| = hi*2^64 + lo, then the sign), so
// that every entry point turns the same exact numerator into the same double.
double i128_to_double(i128 x);

// Every kernel launch of the library is written `ld_note_launch(), k<<<...>>>(...)`
// so that leiden_kernel_launches() counts them.
void ld_note_launch();

// Kernel timer of the local-moving kernels: begin/end around a launch of
// kernel `k` (no-ops unless collect_stats has bit 2), resolve after a
// stream sync.
// Phase boundaries (tag: a leiden_phase, or PHASE_END after the last one)
// and their resolution after a stream sync into stats.phase_ms.
constexpr int PHASE_END = 6;
// Aggregation arcs from the stream-ordered pool (false: out of memory) and
// their return at the end of a call (a no-op when none are held).
// `arcs` bounds the arcs of G^t during the call (taken before a batch is
// applied, it must count the arcs the batch can add); buffers already held
// with enough slots are kept.
bool acquire_agg_buffers(leiden_handle *h, int64_t arcs);
void release_agg_buffers(leiden_handle *h);
// Bytes of those buffers for a graph of `arcs` arcs: every aggregated level
// has at most the arcs of G^t, and its rows are laid out by the members'
// degrees, so arcs + 1 slots per buffer suffice.
inline int64_t agg_buffer_bytes(int64_t arcs) { return 2 * 12 * (arcs + 1); }

void ph_mark(leiden_handle *h, int tag);
void ph_resolve(leiden_handle *h);
// Adds algorithmic bytes to stats.phase_bytes[phase].
inline void ph_bytes(leiden_handle *h, int phase, int64_t bytes) { h->stats.phase_bytes[phase] += bytes; }

bool side_streams(leiden_handle *h);
void kt_begin(leiden_handle *h, int k, cudaStream_t s = nullptr);
void kt_end(leiden_handle *h, cudaStream_t s = nullptr);
void kt_resolve(leiden_handle *h);
void kt_reset(leiden_handle *h);  // at the start of a call

// Layout of the per-graph counter block (device or its host mirror) at
// `base`; gc_block_bytes(G) bytes in all.
GraphCounters gc_layout(void *base, int G);
size_t gc_block_bytes(int G);
int64_t level0_huge_slots(const std::vector<int32_t> &deg);

// Message returned by leiden_last_error(NULL) (calls without a handle).
void set_handle_free_error(const std::string &msg);

// Checked build: each file's device check word (0 = every check held), read
// after a stream sync and reset; check_selftest records LD_CHK_SELFTEST on
// purpose and returns what the host reads back (0 in the default build).
unsigned int check_word_move();
unsigned int check_word_phases();
unsigned int check_word_track();
unsigned int check_selftest(cudaStream_t s);

// ------------------------------------------------------------ prims.cu
// Exclusive scan of n values; out[n] receives the total.  `tmp` must hold
// scan_tmp_bytes(n) bytes.  in == out is allowed.
size_t scan_tmp_bytes(int64_t n);
cudaError_t exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, void *tmp, cudaStream_t s);
cudaError_t exclusive_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, void *tmp, cudaStream_t s);
// Stable sort of 64-bit keys on their low `bits` bits, with an optional
// int64 payload: one block for at most 2048 keys, otherwise an LSD radix
// sort whose buffers are ping-ponged.  The result is written back to
// keys/vals.  `tmp` must hold sort_tmp_bytes(n) bytes.
size_t sort_tmp_bytes(int64_t n);
cudaError_t radix_sort_u64(uint64_t *keys, uint64_t *keys_alt, int64_t *vals, int64_t *vals_alt, int64_t n,
                           int bits, void *tmp, cudaStream_t s);
void launch_fill_i32(int32_t *p, int32_t v, int64_t n, cudaStream_t s);
void launch_fill_i64(int64_t *p, int64_t v, int64_t n, cudaStream_t s);
void launch_iota_i32(int32_t *p, int64_t n, cudaStream_t s);
// Per-item global tables and work chunks for the listed items (see prims.cu).
constexpr int TABLE_CHUNK = 4096;
// key_cap: the most distinct keys any item can have (tables take
// pow2 >= 2*min(size, key_cap) slots).
void launch_table_plan(const int32_t *list, const int32_t *count, const int32_t *deg32, const int64_t *off64,
                       int64_t key_cap, int64_t *tab_off, int64_t *ch_off, cudaStream_t s);
int grid_for(int64_t n, int block, int max_blocks = 152 * 16);

// ------------------------------------------------------------ batch.cu
leiden_status batch_apply_and_mark(leiden_handle *h, const leiden_edge *d_del, int64_t n_del,
                                   const leiden_edge *d_ins, int64_t n_ins, int mode);
// Spare arc slots kept after `used` slots for rows that outgrow their capacity.
inline int64_t spill_arena_size(int64_t used, int log2_min) { return used / 8 + ((int64_t)1 << log2_min); }

// Sub-sweeps per local-moving iteration: params.classes in the snapshot
// schedule; the in-place schedule uses at least 16 (fewer vertices move at
// once, so fewer decisions act on totals that other moves are changing).
inline int lm_classes(const leiden_handle *h) {
  return h->p.deterministic ? h->p.classes : (h->p.classes > 16 ? h->p.classes : 16);
}

// ------------------------------------------------------------ move.cu
// One local-moving sub-sweep of class `cls` (0 .. classes-1).
void lm_subsweep(leiden_handle *h, const LevelGraph &g, int cls, const uint8_t *in_range, int dynamic);
// Refinement: reset, then one round (SYNC) or one sweep (async) of moves.
void refine_reset(leiden_handle *h, const LevelGraph &g);
void refine_round(leiden_handle *h, const LevelGraph &g, int slot);
// Community sizes of C' for the singleton rule: all ones (C' the identity),
// the sizes kept by the last tracking (C' = C^{t-1}), or counted.
enum { SIZES_ONES = 0, SIZES_KEPT = 1, SIZES_COUNT = 2 };
void lm_prepare(leiden_handle *h, const LevelGraph &g, int sizes_from);
void count_sizes(leiden_handle *h, const int32_t *C, int64_t n, int32_t *size);
bool ensure_hslots(leiden_handle *h, int64_t slots);     // false: allocation failed
int32_t *hs_keys(leiden_handle *h);  // global table scratch: keys, values, slot lists
int64_t *hs_vals(leiden_handle *h);
int32_t *hs_list(leiden_handle *h);

// ------------------------------------------------------------ phases.cu
void subset_renumber(leiden_handle *h, int64_t n);
void split_communities(leiden_handle *h, const LevelGraph &g);
// Ranks in lbuf0, count in lbuf0[n]; batched (gid non-null): only the
// graphs flagged in gc.cont, the others mapped to the spare id lbuf0[n].
void renumber_dense(leiden_handle *h, int64_t n, const int32_t *gid);
// Distinct ids of Cp -> dcnt->list_count (and gc.ncomm per graph when batched).
void count_communities(leiden_handle *h, int64_t n, const int32_t *gid);
void lookup_dendrogram(leiden_handle *h);  // batched: the continuing graphs only
void break_lookup(leiden_handle *h);       // batched: final lookup of the stopping graphs
// Batched: graph ids of the next level's super-vertices and its graph ranges.
void next_level_ids(leiden_handle *h, int64_t n, const int32_t *gid, int32_t *gid_next, int64_t *loff_next);
void aggregate(leiden_handle *h, const LevelGraph &g, int64_t ncomm, int out_slot);
void reset_next_pass(leiden_handle *h, int64_t ncomm, int out_slot);
void mark_all_unprocessed(leiden_handle *h, int64_t n);
// Pass-loop start: frontier from dV (counted into affected), Ctop = identity,
// C' = C, K' = K, Sigma' = Sigma.
void pass_init(leiden_handle *h);
void level_maxdeg(leiden_handle *h, const int32_t *deg, int64_t n);  // into dcnt->max_count

// ------------------------------------------------------------ track.cu
void track_communities(leiden_handle *h);  // Ctop vs C -> C, Sig, dSig
void modularity_terms(leiden_handle *h, const int32_t *C);  // into dcnt->sigma_intra / sq
void recompute_weights(leiden_handle *h);  // K = row sums, m2 (device)
void recompute_sigma(leiden_handle *h);    // Sigma from K and C
