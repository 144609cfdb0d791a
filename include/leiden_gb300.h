/*
 * leiden_gb300.h -- C ABI of the GB300 (sm_103a) dynamic Leiden library.
 *
 * The library tracks the communities of one evolving undirected graph on one
 * GPU, following "Heuristic-based Dynamic Leiden Algorithm for Efficient
 * Tracking of Communities on Evolving Graphs" (Sahu, arXiv 2410.15451).  The
 * functions mirror the paper's statement of the problem: Alg. "naive",
 * "delta" and "frontier" (Appendix A.1-A.3) take the updated graph G^t, the
 * batch (deletions Delta^{t-}, insertions Delta^{t+}) and the auxiliary
 * state {C^{t-1}, K^{t-1}, Sigma^{t-1}, Delta Sigma^{t-1}}, and return
 * {C^t, K^t, Sigma^t, Delta Sigma^t}.  Here the handle owns G and that
 * state on the device, so a call passes only the batch.
 *
 * Conventions for every function:
 *  - Host pointers unless the name ends in _device; the library copies host
 *    inputs before returning and never keeps a caller pointer.
 *  - Vertex ids are int32 in [0, n); n is fixed for the life of a handle
 *    (the paper adds or removes no vertices: Evaluation, "Batch generation").  Edge weights
 *    are positive int32; degrees and community totals are exact int64.
 *  - Errors are reported by status code only; no exception or abort crosses
 *    the ABI.  leiden_last_error() gives a message for the last failure.
 *  - One handle is used by one host thread at a time; all its GPU work runs
 *    on the stream given at creation.  Different handles are independent.
 */
#ifndef LEIDEN_GB300_H
#define LEIDEN_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LEIDEN_OK = 0,
  LEIDEN_ERR_ARG = 1,      /* bad argument (null pointer, size, mode)           */
  LEIDEN_ERR_BATCH = 2,    /* invalid batch; the handle is left unchanged        */
  LEIDEN_ERR_OOM = 3,      /* device memory exhausted                            */
  LEIDEN_ERR_CUDA = 4,     /* a CUDA call failed (the message names it)          */
  LEIDEN_ERR_TIMEOUT = 5,  /* a bounded wait gave up (leiden_server_wait_for)    */
  LEIDEN_ERR_STATE = 6     /* call order violated (update before static)         */
} leiden_status;

/* Affected-vertex marking of the batch (Appendix A.1, A.2, A.3). */
typedef enum { LEIDEN_ND = 0, LEIDEN_DS = 1, LEIDEN_DF = 2 } leiden_mode;

/* One undirected edge; the library adds the reverse direction itself. */
typedef struct {
  int32_t u, v, w;
} leiden_edge;

typedef struct {
  double tau;             /* iteration tolerance of local moving, 1e-2 (Evaluation, "Configuration") */
  double tau_drop;        /* TOLERANCE_DECLINE_FACTOR, 10                                 */
  double tau_refine;      /* refinement tolerance tau_re, 0.6 (Approach, "Minimizing     */
                          /*    communities to refine")                                  */
  int32_t max_iterations; /* MAX_ITERATIONS per pass, 20                                  */
  int32_t max_passes;     /* MAX_PASSES, 10                                               */
  int32_t deterministic;  /* 1: snapshot schedule, bit-identical run to run (default);    */
                          /* 0: moves applied in place as vertices decide (the paper's    */
                          /*    asynchronous style; results may vary between runs)        */
  int32_t classes;        /* sub-sweeps per local-moving iteration, power of two, 4       */
                          /*    (the in-place schedule uses at least 16)                  */
  double slack;           /* spare CSR capacity per row as a fraction of its degree, 0.25 */
  int32_t min_slack;      /* minimum spare arcs per row, 4                                */
  int32_t collect_stats;  /* bit 1: time each phase with CUDA events recorded at the     */
                          /*    phase boundaries, read after the call's last host sync    */
                          /*    (no added syncs);                                         */
                          /* bit 2: time each launch of the local-moving kernels          */
                          /*    with an event pair on the stream (no added syncs); 0      */
  int32_t split_all;      /* ablation: split every community that is not refined, not     */
                          /*    only the changed ones (Approach, "Minimizing communities */
                          /*    to split", splits the changed ones); 0                   */
  int32_t converge_any;   /* ablation: leave the pass loop when l_i <= 1 OR no community  */
                          /*    was refined (the text's reading; the pseudocode's AND     */
                          /*    is the default); 0                                        */
  int32_t arena_log2;     /* spill arena for rows that outgrow their slack: used/8 +     */
                          /*    2^arena_log2 arc slots (0..30); when it is full the CSR   */
                          /*    is rebuilt with fresh slack; 20                           */
} leiden_params;

/* Counters and phase times of the last static/update call. */
typedef struct {
  int64_t passes;              /* Leiden passes run                                     */
  int64_t lm_iterations;       /* local-moving iterations, all passes                   */
  int64_t lm_vertices;         /* vertex visits in local moving                          */
  int64_t lm_arcs;             /* arcs scanned in local moving                           */
  int64_t lm_moves;            /* community changes in local moving                      */
  int64_t refine_vertices;     /* vertex visits in refinement                            */
  int64_t refine_arcs;         /* arcs scanned in refinement                             */
  int64_t aggregate_arcs;      /* arcs read by aggregation                               */
  int64_t affected;            /* |dV|: the affected set of pass 1 (all n for static/ND) */
  int64_t communities;         /* communities in C^t                                     */
  int64_t batch_arcs;          /* arcs applied (both directions, after deduplication)    */
  /* Phase times (collect_stats bit 1; device time on the stream between the
   * phase boundaries, ms): */
  double ms_total;             /* the whole call: the sum of the six phases below        */
  double ms_batch;             /* phase_ms[LEIDEN_PHASE_BATCH]                           */
  double ms_move;              /* phase_ms[LEIDEN_PHASE_MOVE]                            */
  double ms_refine;            /* phase_ms[LEIDEN_PHASE_REFINE]                          */
  double ms_aggregate;         /* phase_ms[LEIDEN_PHASE_AGGREGATE]                       */
  double ms_track;             /* phase_ms[LEIDEN_PHASE_TRACK]                           */
  /* The local-moving kernels, [0] vertices of degree <= 128 (a warp or 8 lanes
   * each), [1] degree 129..1024 (a block each), [2] the arc scan of vertices
   * above 1024 arcs (chunks spread over all SMs): */
  int64_t lmk_launches[3];     /* launches timed (collect_stats bit 2)                    */
  int64_t lmk_vertices[3];     /* vertex visits                                          */
  int64_t lmk_arcs[3];         /* arcs scanned                                           */
  int64_t lmk_bytes[3];        /* algorithmic bytes: per arc 8 (col, C of the neighbour) */
                               /* + the weight (4 at level 0, else 8); [0] and [1] add   */
                               /* 40 per visit (list entry, offset, degree, C, K, Sigma  */
                               /* and size of C)                                         */
  double lmk_ms[3];            /* summed device time of the timed launches               */
  int64_t rebuilds;            /* full CSR rebuilds (the spill arena was full)           */
  /* Per phase (index: leiden_phase): device time (collect_stats bit 1, else 0)
   * and algorithmic bytes (always), the bytes each phase must move as counted
   * from its work counters: per vertex of a level, per arc scanned, per batch
   * arc, per move, with the per-unit sizes of each phase's arrays (the byte
   * model is documented with the kernels).  Bytes / time is the phase's
   * achieved bandwidth for a roofline of the whole call. */
  double phase_ms[6];
  int64_t phase_bytes[6];
  /* The largest kernels of the other phases, timed like the local-moving
   * ones: [0] split sampling (per listed vertex 20 B: list entry, C, offset,
   * degree; per arc read 8 B: col, C of the neighbour), [1] the chunked scan
   * of communities above 1024 member arcs in aggregation (per arc: col, C of
   * the neighbour and the weight), [2] the block merge of touched rows of
   * 257..4096 arcs (per arc: the old row read and the new row written,
   * 16 B; per batch arc 16 B). */
  int64_t xk_launches[3];
  int64_t xk_bytes[3];
  double xk_ms[3];
  /* Communities above 1024 member arcs aggregated through a global table of
   * their own: [0] an open-addressing hash table (fewer slots than the
   * level has communities), [1] a table indexed by the community id itself
   * (a slot per community: one atomic add per key, no probing). */
  int64_t agg_tables[2];
} leiden_stats;

/* Phases of a call, as timed and counted in leiden_stats. */
typedef enum {
  LEIDEN_PHASE_BATCH = 0,     /* batch canonicalisation, sort, merge-apply, marking, weights */
  LEIDEN_PHASE_MOVE = 1,      /* local moving (Alg. leidenlm), all passes                     */
  LEIDEN_PHASE_SPLIT = 2,     /* subset renumbering and splitting (Alg. leidensr, leidensp)   */
  LEIDEN_PHASE_REFINE = 3,    /* refinement (Alg. leidenre)                                   */
  LEIDEN_PHASE_AGGREGATE = 4, /* community count, dense renumbering, lookup, aggregation      */
  LEIDEN_PHASE_TRACK = 5      /* final lookup and tracking (Alg. leidentr)                    */
} leiden_phase;

typedef struct leiden_handle leiden_handle;

/* Launch shapes of the local-moving and refinement kernels.  They change how
 * the work is spread over the GPU, never a result (the deterministic schedule
 * gives the same bits for every valid setting).  `overlap` lets kernels that
 * write disjoint data run at once on the handle's two side streams: the
 * block bin and the hub path beside the warp bin (deterministic schedule
 * only), and the merges of short, mid and long rows of a batch. */
typedef struct {
  int32_t tiny_max;           /* degree <= this: eight lanes per vertex; 0 or 1..8, 8       */
  int32_t warp_max;           /* degree <= this: a warp per vertex; tiny_max..128, 128      */
  int32_t block_max;          /* degree <= this: a block per vertex, above: spread over all */
                              /*    SMs; warp_max..1024, 1024                               */
  int32_t warp_blocks_per_sm; /* grid of the warp-range kernel, 1..8, 4                     */
  int32_t block_blocks_per_sm;/* grid of the block-bin kernel, 1..8, 7                      */
  int32_t hub_blocks_per_sm;  /* grid of the hub arc scan, 1..32, 16                        */
  int32_t overlap;            /* side streams: 0 or 1, 1                                    */
} leiden_tuning;

/* Fill *p with the defaults listed above. */
void leiden_default_params(leiden_params *p);

/* Defaults of leiden_tuning; set a handle's with leiden_set_tuning
 * (LEIDEN_ERR_ARG outside the ranges above).  `python bench.py --autotune`
 * searches them on a workload. */
void leiden_default_tuning(leiden_tuning *t);
leiden_status leiden_set_tuning(leiden_handle *h, const leiden_tuning *t);

/* Create a handle for the graph G^0 -- the graph before the first batch in
 * the problem statement of Alg. "naive", "delta" and "frontier" (Appendix
 * A.1-A.3, whose G^{t-1} it is at t = 1) -- given as symmetric CSR on the host:
 * offsets[n+1] (int64, offsets[0] = 0), cols[offsets[n]] (int32, in [0, n)),
 * weights[offsets[n]] (int32 > 0, NULL = unit).  Rows need not be sorted;
 * self-loops and repeated arcs are rejected (LEIDEN_ERR_ARG).  The graph is
 * copied to a device CSR with per-row slack.  cuda_stream is a cudaStream_t
 * (NULL = the legacy default stream).  On success *out owns all device state;
 * release it with leiden_destroy(). */
leiden_status leiden_create(const leiden_params *params, int64_t n, const int64_t *offsets,
                            const int32_t *cols, const int32_t *weights, void *cuda_stream,
                            leiden_handle **out);

/* Static Leiden (the baseline of Evaluation, "Measurement"; Alg. "leiden" with C^{t-1} = singletons,
 * every vertex affected, every community refined) on the current graph.
 * Resets the auxiliary state: C^t = result, K^t = weighted degrees,
 * Sigma^t = community totals, Delta Sigma^t = 0.  membership_out: host
 * int32[n] or NULL. */
leiden_status leiden_static(leiden_handle *h, int32_t *membership_out);

/* Apply one batch update and update the communities (Alg. "naive" / "delta" /
 * "frontier" with Alg. "leiden" and "leidenTrack").  del/ins are host arrays
 * of undirected edges.  Batch rules: ids in [0, n), u != v, insertion
 * weights > 0; a deletion must name an existing edge (its w is ignored and
 * the stored weight is removed); repeated deletions collapse, repeated
 * insertions add up; inserting an existing edge adds to its weight;
 * deletions apply before insertions.  Any violation returns
 * LEIDEN_ERR_BATCH with the handle unchanged.  Requires a prior
 * leiden_static (else LEIDEN_ERR_STATE).  membership_out: host int32[n] or
 * NULL (C^t stays on the device). */
leiden_status leiden_update(leiden_handle *h, const leiden_edge *del, int64_t n_del,
                            const leiden_edge *ins, int64_t n_ins, leiden_mode mode,
                            int32_t *membership_out);

/* As leiden_update, but del, ins and membership_out are device pointers on
 * the handle's device (membership_out may be NULL).  The call returns when
 * the result is complete on the device. */
leiden_status leiden_update_device(leiden_handle *h, const leiden_edge *del, int64_t n_del,
                                   const leiden_edge *ins, int64_t n_ins, leiden_mode mode,
                                   int32_t *membership_out);

/* Modularity Q of Eq. 1 on the current graph for `membership` (host
 * int32[n] with ids in [0, n); NULL = the handle's C^t).  Computed exactly in
 * integers (2m * sum sigma_c - sum Sigma_c^2) and divided once by (2m)^2. */
leiden_status leiden_modularity(leiden_handle *h, const int32_t *membership, double *q_out);

/* Modularity Q (Eq. 1, same exact-integer arithmetic and final division as
 * leiden_modularity) of the membership d_membership (device int32[n], ids in
 * [0, n)) on a caller-owned device CSR: d_offsets int64[n+1], d_cols
 * int32[d_offsets[n]] with ids in [0, n) (non-NULL even for a graph without
 * arcs), d_weights int32 or NULL for unit weights.  Work runs on cuda_stream
 * (NULL = legacy default stream); the call returns when *q_out is written.
 * A graph without arcs has Q = 0.
 *
 * The paper has no counterpart to this function.  It exists for callers that
 * may not allocate device memory: a serving loop that reserved all device
 * memory up front, code whose device memory belongs to another allocator
 * (e.g. a framework's caching pool), or a latency-critical path where the
 * implicit synchronisation of cudaMalloc/cudaFree is not acceptable.  It
 * allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 * Its scratch is one fixed array in the library's device memory, 32 MiB,
 * which every GPU that loads the library holds until the process exits; so n
 * may be at most 4,194,304 (larger n returns LEIDEN_ERR_ARG).  The first call
 * on each device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * All calls share the one array: calls whose GPU work overlaps (other
 * streams, other host threads) race and give wrong results; serialise them.
 * Errors: LEIDEN_ERR_ARG (null pointer, n out of range, a membership or
 * column id outside [0, n): found by the kernels, reported after the GPU
 * work, with no other effect), LEIDEN_ERR_CUDA; the message is in
 * leiden_last_error(NULL). */
leiden_status leiden_modularity_noalloc(int64_t n, const int64_t *d_offsets, const int32_t *d_cols,
                                        const int32_t *d_weights, const int32_t *d_membership,
                                        void *cuda_stream, double *q_out);

/* Resume from an exported state: a handle created from the exported graph
 * (leiden_get_graph) takes the exported membership C (int32[n]) and Delta
 * Sigma (int64[n], indexed by community id); K, Sigma and 2m are recomputed
 * from the graph (they are functions of it and of C).  The handle then
 * behaves as the exporting one did: leiden_update may follow directly, with
 * no leiden_static.  LEIDEN_ERR_ARG on ids out of range (or outside their
 * graph's range on a batched handle).  Library extension (checkpointing). */
leiden_status leiden_import_state(leiden_handle *h, const int32_t *C, const int64_t *dSigma);

/* Device pointer to the handle's current membership C^t (int32[n]); valid
 * until the next call on the handle. */
leiden_status leiden_membership_device(leiden_handle *h, const int32_t **d_membership);

/* Host copies of the auxiliary state {C^t, K^t, Sigma^t, Delta Sigma^t} and
 * 2m.  Any output pointer may be NULL. */
leiden_status leiden_get_state(leiden_handle *h, int32_t *C, int64_t *K, int64_t *Sigma,
                               int64_t *dSigma, int64_t *m2);

/* Number of arcs of G^t (twice the number of edges). */
int64_t leiden_graph_arcs(leiden_handle *h);

/* Host copy of G^t as compact CSR with rows sorted by neighbour:
 * off[n+1], col[arcs], w[arcs] (arcs from leiden_graph_arcs). */
leiden_status leiden_get_graph(leiden_handle *h, int64_t *off, int32_t *col, int64_t *w);

/* Affected flags dV (uint8[n]) of the last call (all ones for static/ND). */
leiden_status leiden_get_affected(leiden_handle *h, uint8_t *dV);

/* Per-pass trace of the last call, int64[2 + 10*25]: [0] passes, [1] |dV|,
 * then per pass: level vertex count, local-moving iterations, communities
 * after refinement, any community refined, refinement rounds, moves in
 * local-moving iterations 0..19. */
leiden_status leiden_get_trace(leiden_handle *h, int64_t *trace);

/* Counters and phase times of the last call: the work of the phases of
 * Alg. "leiden" (Appendix A.4: local moving, splitting, refinement,
 * aggregation), the affected set |dV| the evaluation reports per approach
 * (Evaluation, "Affected vertices and Marked communities"), and the phase times behind its runtime split.  Library
 * instrumentation; the paper measures with its own timers. */
leiden_status leiden_get_stats(leiden_handle *h, leiden_stats *stats);

/* ---- Batched handles: many graphs, one launch per kernel for all of them ----
 *
 * leiden_create_batched() takes G graphs concatenated with vertex offsets:
 * graph g owns the vertices vertex_offsets[g] .. vertex_offsets[g+1]-1 of one
 * symmetric CSR (offsets[n+1], cols, weights as in leiden_create, with
 * n = vertex_offsets[G]); no arc may join two graphs (LEIDEN_ERR_ARG).  Every
 * call on the handle then processes all graphs at once, each exactly as a
 * handle of its own would (Alg. "leiden": same passes, iterations, tau, 2m and
 * tracking per graph; the deterministic schedule gives the same memberships
 * bit for bit, offset by vertex_offsets[g]).  Batches passed to
 * leiden_update use the concatenated vertex ids; an edge between two graphs
 * is LEIDEN_ERR_BATCH.  Community ids of graph g stay in its vertex range.
 * Batched handles with G > 1 run the deterministic schedule only
 * (params->deterministic = 0 is LEIDEN_ERR_ARG).  Library extension: the
 * paper processes one graph at a time. */
leiden_status leiden_create_batched(const leiden_params *params, int32_t graphs, const int64_t *vertex_offsets,
                                    const int64_t *offsets, const int32_t *cols, const int32_t *weights,
                                    void *cuda_stream, leiden_handle **out);

/* Device bytes a handle for this graph (CSR offsets[n+1]) is expected to
 * hold: the allocations of leiden_create plus an allowance for batch buffers
 * and aggregated-level hash tables that grow on demand.  -1 on bad input.
 * Used by the server below to admit graphs by footprint.  The batch buffers
 * take about 160 B per arc of batch capacity (two arcs per edge, capacity
 * grown geometrically to at most twice the largest batch); the allowance
 * (8 B per vertex plus 32 MB) covers batches up to about 50k edges on a
 * small graph, more on a large one.  Not included: the arcs of the
 * aggregated levels, which a call draws from the device's stream-ordered
 * memory pool only while it aggregates (see the next). */
int64_t leiden_footprint_bytes(const leiden_params *params, int64_t n, const int64_t *offsets);

/* Device bytes a call on this graph draws from the stream-ordered pool while
 * it aggregates (two levels of arcs, 24 B per arc of the graph), returned at
 * the end of the call; -1 on bad input.  The server keeps room for `slots`
 * of these (the largest admitted graph's).  Library extension. */
int64_t leiden_transient_bytes(int64_t n, const int64_t *offsets);

/* Number of graphs of the handle (1 for leiden_create handles). */
int32_t leiden_batch_graphs(const leiden_handle *h);

/* Per-graph trace of the last call, same layout as leiden_get_trace ([1] is
 * |dV| of that graph). */
leiden_status leiden_batch_trace(leiden_handle *h, int32_t graph, int64_t *trace);

/* Modularity (Eq. 1) of each graph's current membership, q_out[G], with its
 * own 2m. */
leiden_status leiden_batch_modularity(leiden_handle *h, double *q_out);

/* ---- Serving: many tracked graphs resident on the device ----
 *
 * A server keeps every admitted graph's state (CSR with slack, C, K, Sigma,
 * Delta Sigma) on the device, each graph with a CUDA stream of its own, and
 * runs update requests on `slots` worker threads as soon as a slot is free.
 * Admission is by footprint (leiden_footprint_bytes): a graph waits until it
 * fits in the remaining `device_bytes` budget (graphs leave with
 * leiden_server_remove_graph), then gets its static Leiden.  Requests of one
 * graph run one at a time in submission order, so every result equals the
 * one the graph gets alone (bit for bit in the deterministic schedule);
 * requests of different graphs overlap on the device.  All functions are
 * thread-safe.  Library extension: the paper has no serving layer. */
typedef struct leiden_server leiden_server;

typedef struct {
  int64_t graphs_resident;   /* admitted and on the device                         */
  int64_t graphs_waiting;    /* waiting for device memory, or being admitted       */
  int64_t requests_queued;   /* submitted, not started                             */
  int64_t requests_running;  /* on a slot now (admissions included)                */
  int64_t requests_done;     /* finished                                           */
  int64_t bytes_used;        /* footprint of the resident graphs                   */
  int64_t bytes_budget;      /* device_bytes                                       */
} leiden_server_stats;

/* params as for leiden_create (shared by all graphs); 1 <= slots <= 256. */
leiden_status leiden_server_create(const leiden_params *params, int64_t device_bytes, int32_t slots,
                                   leiden_server **out);
/* Register a graph (host CSR as for leiden_create, copied); *graph_out is its
 * id.  LEIDEN_ERR_OOM if its footprint alone exceeds the budget.  A graph
 * that fails admission answers its requests with LEIDEN_ERR_OOM. */
leiden_status leiden_server_add_graph(leiden_server *s, int64_t n, const int64_t *offsets, const int32_t *cols,
                                      const int32_t *weights, int32_t *graph_out);
/* Queue an update of `graph` (batch copied); keep_membership != 0 keeps a host
 * copy of the resulting membership for leiden_server_wait. */
leiden_status leiden_server_submit(leiden_server *s, int32_t graph, const leiden_edge *del, int64_t n_del,
                                   const leiden_edge *ins, int64_t n_ins, leiden_mode mode, int32_t keep_membership,
                                   int64_t *ticket_out);
/* Wait for a request: its status; membership_out (n of the graph, or NULL),
 * latency from submission to completion and service time (ms, or NULL).
 * Each ticket is waited for once. */
leiden_status leiden_server_wait(leiden_server *s, int64_t ticket, int32_t *membership_out, double *latency_ms,
                                 double *service_ms);
/* The same with a limit: if the request is not done within timeout_ms
 * (< 0: no limit) the call returns LEIDEN_ERR_TIMEOUT and the ticket stays
 * valid, so it may be waited for again -- a caller's deadline, e.g. for a
 * request of a graph still waiting for memory, never blocks it for good. */
leiden_status leiden_server_wait_for(leiden_server *s, int64_t ticket, double timeout_ms, int32_t *membership_out,
                                     double *latency_ms, double *service_ms);
/* Current membership of a resident graph (after its queued requests). */
leiden_status leiden_server_membership(leiden_server *s, int32_t graph, int32_t *membership_out);
/* Remove a graph once its queued requests are done; its memory is freed and
 * waiting graphs may be admitted. */
leiden_status leiden_server_remove_graph(leiden_server *s, int32_t graph);
leiden_status leiden_server_get_stats(leiden_server *s, leiden_server_stats *out);
/* Message of the last failure on s (NULL: of the last failed create). */
const char *leiden_server_last_error(leiden_server *s);
/* Wait for running work, stop the workers, free everything (queued requests
 * are dropped). */
void leiden_server_destroy(leiden_server *s);

/* Number of CUDA kernels this library has launched in the process since it
 * was loaded, over all handles and threads (a relaxed atomic counter; read
 * it before and after a call to count that call's launches).  Library
 * bookkeeping with no counterpart in the paper. */
int64_t leiden_kernel_launches(void);

/* Checked build.  Compiled with -DLEIDEN_CHECKED, the kernels test the
 * invariants the algorithm guarantees (an open-addressing probe ends within
 * its table; neighbour and community ids lie in [0, n)); a failed test is
 * recorded in a device word, the access is skipped, and the call returns
 * LEIDEN_ERR_STATE -- no trap, no fault, no endless loop.  The default build
 * compiles the tests away.  leiden_checked_build() is 1 in the checked build,
 * else 0.  leiden_check_selftest() launches one kernel that fails a test on
 * purpose and returns the code the host reads back (and clears): 0x5e1f in
 * the checked build, 0 in the default one.  Library diagnostics with no
 * counterpart in the paper. */
int32_t leiden_checked_build(void);
int32_t leiden_check_selftest(void *cuda_stream);

/* Message for the last failed call on h (or for the last failed
 * leiden_create when h is NULL).  Never NULL. */
const char *leiden_last_error(leiden_handle *h);

/* Free all device and host memory of the handle (NULL is a no-op). */
void leiden_destroy(leiden_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* LEIDEN_GB300_H */
