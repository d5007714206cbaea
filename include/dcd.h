/*
 * dcd.h -- C ABI of the GB300 (sm_103a) library for incremental dynamic
 * community detection with Delta-screening (Zarayeneh & Kalyanaraman,
 * "A Fast and Efficient Incremental Approach toward Dynamic Community
 * Detection", arXiv 1904.08553).
 *
 * The calls follow the problem statement of Sec. III-B (detect C_t for every
 * G_t of a dynamic graph) and the incremental approach of Sec. III-D:
 *
 *   dcd_create(n)                      a dynamic graph on the vertex set [0, n)
 *   dcd_apply_batch(inserts, deletes)  stage the changes Delta_t of one step
 *   dcd_update()                       G_t <- G_{t-1} + Delta_t, then C_t and Q_t
 *
 * Conventions shared by every call:
 *   - Return value: DCD_OK (0) on success, a negative DCD_E* code otherwise.
 *     A call that fails leaves the context exactly as it was.
 *   - Vertex ids are int32 in [0, n); n <= 2^31 - 1.  Graphs are undirected:
 *     an edge (u, v) and (v, u) are the same edge.  Self-loops are rejected.
 *   - Weights are positive int32 (Sec. III-A allows any non-negative weight;
 *     integer weights keep every decision exact).  Repeated inserts of an
 *     edge add their weights (multiplicity).
 *   - Pointers marked "host" are ordinary CPU memory; pointers marked
 *     "device" are CUDA device memory of the context's device; "host or
 *     device" pointers are told apart with cudaPointerGetAttributes.
 *     The library never takes ownership of caller memory.
 *   - All device work is ordered on the CUDA stream given to dcd_create
 *     (NULL: a stream the context creates, see dcd_create).  Kernels with
 *     disjoint outputs may run on side streams the context owns, forked from
 *     that stream and joined back into it within the same call, so the caller
 *     sees one stream's order.  Every call returns with its work complete
 *     unless the call says otherwise.
 *   - Not thread-safe per context: one context, one host thread at a time.
 */
#ifndef DCD_H
#define DCD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define DCD_OK 0
#define DCD_EINVAL (-1)    /* bad argument: id out of range, u == v, w <= 0, n out of range */
#define DCD_ENOMEM (-2)    /* device or host allocation failed                              */
#define DCD_ECUDA (-3)     /* a CUDA runtime call failed (see dcd_last_cuda_error)          */
#define DCD_ESTATE (-4)    /* call not valid in the current state                           */
#define DCD_EOVERFLOW (-5) /* an edge weight above INT32_MAX, or 2m >= 2^62                  */
#define DCD_ETIMEOUT (-6)  /* a bounded device-side wait gave up                            */
#define DCD_EIO (-7)       /* a file could not be opened, written or renamed                 */

/* ---- modes (Sec. III-C, III-D) ---- */
#define DCD_MODE_STATIC 0  /* Static(G_t) from singletons every step (the naive approach)   */
#define DCD_MODE_BASE 1    /* dLouvain-base: inherit C_{t-1}, R_t = V_t                     */
#define DCD_MODE_DELTA 2   /* dLouvain-Delta-s: inherit C_{t-1}, R_t = Delta-screening      */
#define DCD_MODE_GIVEN_R 3 /* inherit C_{t-1}, R_t supplied by dcd_set_rset                */
#define DCD_MODE_LEARNED 4 /* inherit C_{t-1}, R_t from the network around Delta-screening  */

typedef struct {
  int32_t u, v; /* endpoints, u != v                               */
  int32_t w;    /* weight > 0 for inserts; ignored for deletes     */
} dcd_edge;

/* ---- host methods of the multi-level run (Sec. III-D applies
 * Delta-screening to both) ---- */
#define DCD_ALG_LOUVAIN 0  /* Louvain: Algorithm 1                                    */
#define DCD_ALG_SLM 1      /* smart local moving: dSLM (refinement of every community) */

typedef struct {
  int32_t mode;       /* DCD_MODE_*; default DCD_MODE_DELTA                          */
  int32_t max_iters;  /* local-move passes per level; default 500 (tau reading)       */
  int32_t max_levels; /* default 64                                                   */
  int32_t tau_inv;    /* a pass (level) gaining at most |N| / tau_inv stops it; 1e6  */
  int32_t alg;        /* DCD_ALG_*; default DCD_ALG_LOUVAIN                           */
  int32_t coarsen_full; /* 1: build level 0's coarse graph from every entry of G_t in
                           every update; 0 (default): from the previous update's one
                           when it allows (see dcd_step_stats.coarse0_delta)         */
  int32_t pass_loop;    /* 0 (default): the passes of a level run as one CUDA-graph
                           launch, the loop and its stop rule on the device; 1: the
                           host enqueues each pass and reads the stop rule after it
                           (same results; for tools that cannot look into a graph's
                           conditional nodes, such as a kernel profiler)             */
  int32_t reserved[9];
} dcd_config;

typedef struct {
  int64_t t;             /* time step just computed, 1-based                        */
  int64_t n;             /* |V_t|                                                   */
  int64_t nnz;           /* directed CSR entries of G_t (2 per undirected edge)      */
  int64_t m2;            /* 2 m_t = sum of weighted degrees                         */
  int64_t r_size;        /* |R_t|: vertices evaluated at level 0                    */
  int64_t levels;        /* levels run                                              */
  int64_t iters_total;   /* local-move passes, all levels                           */
  int64_t iters_level0;  /* local-move passes at level 0                            */
  int64_t moves_total;   /* single-vertex moves applied                             */
  int64_t edges_scanned; /* sum over passes of the active vertices' degrees          */
  int64_t verts_scanned; /* sum over passes of the active vertex counts              */
  int64_t communities;   /* |C_t|                                                   */
  int64_t n_lo, n_hi;    /* N = m2^2 Q as a two's-complement 128-bit integer         */
  double q;              /* modularity Q_t (Eq. 1), from N and m2 in FP64            */
  int64_t ins_records;   /* staged inserts in Delta_t                               */
  int64_t del_records;   /* staged deletes in Delta_t                               */
  int64_t launches;      /* CUDA kernel launches issued by this update               */
  int64_t r_screen;      /* |R_t| of plain Delta-screening (-1: not computed)        */
  int64_t pool;          /* vertices scored by the learned screen                   */
  int64_t fallback;      /* 1: the judge kept plain Delta-screening for this step   */
  double q_screen;       /* judged learned mode: Q of the other run (see dcd_set_screen) */
  float ms_total;        /* device time of the whole update (CUDA events)           */
  float ms_merge;        /* batch sort + CSR merge + degrees                        */
  float ms_screen;       /* Delta-screening + R_t build                             */
  float ms_local_move;   /* local-move kernels only (all levels)                    */
  float ms_apply;        /* move apply + modularity tracking                        */
  float ms_coarsen;      /* graph compaction (all levels)                           */
  float ms_finish;       /* label composition, canonical labels                     */
  float ms_bin[4];       /* 0: the degree bins of a pass run side by side in one graph launch, so their
                            times are not separated (edges_bin / verts_bin give their work) */
  float reserved_f[5];
  int64_t edges_bin[4];  /* entries scanned per degree bin (all passes)              */
  int64_t verts_bin[4];  /* vertices evaluated per degree bin (all passes)           */
  float ms_local_move0;  /* local-move kernels of level 0 only (the R_t level)        */
  float reserved_g;
  int64_t edges_level0;  /* entries scanned at level 0 (all its passes)             */
  int64_t verts_level0;  /* vertices evaluated at level 0 (all its passes)          */
  int64_t refine_iters;  /* DCD_ALG_SLM: local-move passes of the refinements       */
  int64_t refine_moves;  /* DCD_ALG_SLM: moves of the refinements                   */
  int64_t coarse0_delta; /* 1: level 0's coarse graph was updated from the previous
                            update's (same communities as a rebuild, Sec. III-D: R_t
                            only changes level 0): the coarse graph of G_{t-1} under
                            C_{t-1}, plus the batch's weight changes, plus the rows
                            of the vertices that level 0 moved.  Taken for a single
                            Louvain graph whose level-0 and previous communities
                            number at most 4096, after a non-static update        */
  int64_t coarse0_entries; /* entries that built level 0's coarse graph: nnz of G_t,
                              or batch pairs + rows of the moved vertices          */
  int64_t edges_level0_screen; /* of edges_level0, entries of the first level-0 pass
                                  not scanned again: Delta-screening sums a source's
                                  row by community under C_{t-1} on G_t, the state
                                  that pass reads, and hands over the source's move
                                  proposal (the same decision)                     */
  int64_t verts_level0_screen; /* of verts_level0, the vertices it covers             */
} dcd_step_stats;

typedef struct dcd_ctx dcd_ctx;

/* Default configuration (see the fields). */
void dcd_config_default(dcd_config* cfg);

/* Create a dynamic graph on vertices [0, n) with no edges (Sec. III-A:
 * G(V, E) as a sequence G_1..G_T).  cfg may be NULL (defaults); with
 * cfg->alg = DCD_ALG_SLM the multi-level run is smart local moving
 * (dSLM-Delta-s in DCD_MODE_DELTA), which needs n < 2^30 (a pass may name
 * n + v, the empty community of v) and does not take DCD_MODE_LEARNED or
 * training-data collection (dcd_update: DCD_ESTATE);
 * cuda_stream is the cudaStream_t the context's work runs on; with NULL the
 * context creates a stream of its own that is ordered with the legacy default
 * stream (the local-move passes run as CUDA graphs, which the legacy stream
 * cannot capture).  *out receives the context.
 * Errors: DCD_EINVAL (n <= 0 or n > 2^31 - 1, out NULL, an unknown alg, alg
 * DCD_ALG_SLM with n >= 2^30), DCD_ENOMEM, DCD_ECUDA. */
int dcd_create(int64_t n, const dcd_config* cfg, void* cuda_stream, dcd_ctx** out);

/* Release every resource of the context.  NULL is accepted. */
int dcd_destroy(dcd_ctx* ctx);

/* Stage one batch of Delta_t (Sec. III-A; Sec. III-E stores each change as
 * the ordered pairs (i,j) and (j,i) -- the library does that itself).
 * ins: n_ins host dcd_edge (u, v, w > 0); del: n_del host dcd_edge (u, v).
 * Deletes of the step act before its inserts; deleting an absent edge is a
 * no-op.  Several calls before one dcd_update concatenate.  The arrays are
 * copied to the device and checked there (ids in [0, n), u != v, w > 0 for
 * inserts) before the call returns; a batch with a bad record is not staged.
 * The caller keeps ownership.  Errors: DCD_EINVAL (any bad record: nothing
 * is staged), DCD_ENOMEM, DCD_ECUDA. */
int dcd_apply_batch(dcd_ctx* ctx, const dcd_edge* ins, int64_t n_ins, const dcd_edge* del,
                    int64_t n_del);

/* As dcd_apply_batch with device arrays.  The records are copied
 * device-to-device on the context stream; validation happens on the device
 * inside the next dcd_update, which fails with DCD_EINVAL (state unchanged,
 * staged batch dropped) if any record is bad. */
int dcd_apply_batch_device(dcd_ctx* ctx, const dcd_edge* d_ins, int64_t n_ins,
                           const dcd_edge* d_del, int64_t n_del);

/* Advance one time step (Sec. III-D): merge the staged batch into G_t, pick
 * R_t by the context mode (Algorithm 2 in DCD_MODE_DELTA), run the
 * multi-level local-move / compaction loop of Algorithm 1 with R_t at level 0,
 * and produce C_t with canonical labels (each community is named by its
 * smallest member id) and Q_t (Eq. 1).  The first update of a context is
 * static (step 1).  With nothing staged the step is valid and empty.
 * labels_out: n int32, host or device, may be NULL.  q_out, stats: host, may
 * be NULL.  Errors: DCD_EINVAL (bad device batch), DCD_EOVERFLOW, DCD_ENOMEM,
 * DCD_ECUDA; on error G and C are those of the previous step. */
int dcd_update(dcd_ctx* ctx, int32_t* labels_out, double* q_out, dcd_step_stats* stats);

/* Current labels C_t (n int32, host or device). */
int dcd_get_labels(dcd_ctx* ctx, int32_t* labels_out);

/* R_t of the last update: n bytes (host or device), 1 = evaluated at level 0. */
int dcd_get_rset(dcd_ctx* ctx, uint8_t* r_out);

/* Replace C_{t-1} (n int32 in [0, n), host).  A context that has not been
 * updated yet then counts as past step 1, so its next update inherits these
 * labels instead of running statically.  Errors: DCD_EINVAL. */
int dcd_set_labels(dcd_ctx* ctx, const int32_t* labels);

/* Supply R_t for the next update in DCD_MODE_GIVEN_R: n bytes, host. */
int dcd_set_rset(dcd_ctx* ctx, const uint8_t* r);

/* Change the mode for the following updates (DCD_MODE_*). */
int dcd_set_mode(dcd_ctx* ctx, int32_t mode);

/* ---- degree bins of the local-move kernels (no counterpart in the paper) ----
 * The local-move evaluation (Algorithm 1, the loop over vertices) splits the
 * active vertices into bins by degree (CSR entries of the row); each bin runs
 * one kernel variant DCD_LM_*, which accepts rows up to its limit.  A plan is
 * nb bins in increasing degree: bin b holds the degrees in (hi[b-1], hi[b]];
 * the last bin has hi = -1 (no limit) and variant DCD_LM_HUB.  Every plan
 * gives the same labels and modularity; only the time differs.
 * dcd_set_bins: errors DCD_EINVAL (nb outside 1..DCD_MAX_BINS, unknown
 * variant, hi not increasing or above the variant's limit, DCD_LM_HUB
 * anywhere but in the last bin, last bin not an unbounded DCD_LM_HUB).
 * dcd_get_bins: *nb, and nb entries of variant / hi (host, each may be NULL).  dcd_autotune: times one local-move evaluation of
 * every vertex of G_t under C_t (no move applied), reps times for each
 * candidate plan, and keeps the fastest; *best_ms (host, may be NULL)
 * receives its time per evaluation.  Errors: DCD_ESTATE before the first
 * update or for reps < 1, DCD_ENOMEM, DCD_ECUDA. */
#define DCD_MAX_BINS 12
#define DCD_LM_SEG16 0   /* <= 16 entries: 8 lanes per vertex, 4 vertices a warp   */
#define DCD_LM_SEG32 1   /* <= 32: 16 lanes per vertex, 2 vertices a warp          */
#define DCD_LM_SEG64 2   /* <= 64: 16 lanes per vertex, 2 vertices a warp          */
#define DCD_LM_WARP128 3 /* <= 128: a warp per vertex                              */
#define DCD_LM_WARP256 4 /* <= 256: a warp per vertex                              */
#define DCD_LM_CTA512 5  /* <= 512: a CTA of 128 threads per vertex                */
#define DCD_LM_CTA1K 6   /* <= 1024: a CTA of 256 threads per vertex               */
#define DCD_LM_CTA2K 7   /* <= 2048: a CTA of 512 threads per vertex               */
#define DCD_LM_CTA4K 8   /* <= 4096: a CTA of 512 threads per vertex               */
#define DCD_LM_HUB 9     /* any degree: a row split over many CTAs, global tables  */
int dcd_set_bins(dcd_ctx* ctx, int32_t nb, const int32_t* variant, const int64_t* hi);
int dcd_get_bins(const dcd_ctx* ctx, int32_t* nb, int32_t* variant, int64_t* hi);
int dcd_autotune(dcd_ctx* ctx, int32_t reps, float* best_ms);

/* Reserves device memory for graphs of up to nnz directed entries (two per
 * undirected edge) and batches of up to `records` records (inserts plus
 * deletes staged for one update): both CSR buffers, the batch staging
 * buffers and the per-update scratch arena.  Updates within those sizes then
 * take their memory from what is reserved instead of growing buffers on the
 * way (growth maps new device memory while the update waits); larger graphs
 * or batches still work, the buffers grow as before.  No counterpart in the
 * paper: a service for callers that keep allocation out of the update path.
 * G_t and a staged batch are kept.  Errors: DCD_EINVAL (ctx NULL, nnz or
 * records negative, records >= 2^30), DCD_ENOMEM, DCD_ECUDA. */
int dcd_reserve(dcd_ctx* ctx, int64_t nnz, int64_t records);

/* One local-move evaluation (the candidate scan of Algorithm 1's inner loop)
 * of every vertex of G_t under C_t with the bin plan in force, repeated reps
 * times with no move applied; each bin's kernels run alone, one bin after
 * another, timed with CUDA events on the context stream.  For measurement
 * and profiling: the per-kernel figures the overlapped bins of a pass hide.
 * Outputs (host, DCD_MAX_BINS entries each): *nb bins; variant[b], verts[b]
 * (vertices of positive degree in bin b), entries[b] (their degree sum) and
 * ms[b] (mean time of one evaluation of bin b).  Errors: DCD_EINVAL (a NULL
 * pointer), DCD_ESTATE (before the first update, reps < 1), DCD_ENOMEM,
 * DCD_ECUDA. */
int dcd_eval_bins(dcd_ctx* ctx, int32_t reps, int32_t* nb, int32_t* variant, int64_t* verts, int64_t* entries,
                  float* ms);

/* Level 0 of the last update's local move (Algorithm 1 over R_t), as run:
 * *nb bins of the plan in force; count[b] the active vertices of bin b;
 * per_sweep[b] the vertices one sweep of bin b's kernel grid covers (a bin
 * holding more runs its grid-stride loop more than once; for the hub bin it
 * equals the count); *side_by_side 1 when the bins ran concurrently on side
 * streams.  Outputs are host memory; count, per_sweep and side_by_side may
 * be NULL.  Before the first update *nb is 0.  Errors: DCD_EINVAL (ctx or nb
 * NULL). */
int dcd_get_level0_bins(const dcd_ctx* ctx, int32_t* nb, int64_t* count, int64_t* per_sweep,
                        int32_t* side_by_side);

/* The CSR of G_t: *nnz_out receives the entry count; when row_ptr/col/w are
 * non-NULL they receive n+1 int64, nnz int32 and nnz int32 (host memory). */
int dcd_get_graph(dcd_ctx* ctx, int64_t* nnz_out, int64_t* row_ptr, int32_t* col, int32_t* w);

/* ---- checkpoint / resume (no counterpart in the paper) ----
 * dcd_save writes to the file at path (host string) what the next step of
 * Sec. III-D reads from a context -- G_t as a CSR, C_t, the step counter t --
 * and its mode, configuration, degree-bin plan and last R_t.  A context that
 * dcd_load creates from the file (on cuda_stream, as dcd_create) continues
 * the stream exactly as the saved one would: the same labels, modularity,
 * R_t and step statistics for the same batches.  Not saved: a staged batch
 * (dcd_save refuses while one is staged), the learned screen (attach the
 * network again with dcd_set_screen; DCD_MODE_LEARNED updates fail with
 * DCD_ESTATE until then), training-data collection and a pending
 * dcd_set_rset.  The file is written under path + ".tmp" and renamed over
 * path at the end, so a failed save leaves an existing file as it was.
 * Format: little-endian; a 256-byte header (magic "DCDCKPT1", version 1,
 * flags, n, nnz, t, mode, plan size, dcd_config, plan), then row_ptr (n + 1
 * int64), col and w (nnz int32 each), labels (n int32) and R_t (n bytes,
 * when flag bit 0 is set), each padded with zeros to a multiple of 8 bytes,
 * then a 64-bit FNV-1a checksum over the 8-byte words before it.  dcd_load
 * checks every field and entry on the host before it reaches the device
 * (row_ptr from 0 to nnz without decreasing, columns in [0, n) increasing
 * along each row with no self-loop, weights > 0, labels in [0, n), R_t bytes
 * 0 or 1, the checksum, no trailing bytes).
 * Errors: DCD_EINVAL (NULL or empty argument; a file that is not a valid
 * checkpoint), DCD_ESTATE (dcd_save with a batch staged), DCD_EIO (the file
 * cannot be opened, written or renamed), DCD_ENOMEM, DCD_ECUDA. */
int dcd_save(dcd_ctx* ctx, const char* path);
int dcd_load(const char* path, void* cuda_stream, dcd_ctx** out);

/* The context's vertex count n, time steps computed t (the next update is
 * step t + 1) and mode; each output is host memory and may be NULL.
 * Errors: DCD_EINVAL (ctx NULL). */
int dcd_get_state(const dcd_ctx* ctx, int64_t* n_out, int64_t* t_out, int32_t* mode_out);

/* Kernel launches issued by the library in this process so far (all
 * contexts, all devices): lets a caller count the device work of a region. */
int64_t dcd_kernel_launches(void);

/* ---- learned screen: the network ----
 * A multilayer perceptron 12 -> 64 -> 64 -> 1 (ReLU, ReLU, sigmoid) that
 * scores a vertex's chance of changing community at level 0.  Not in the
 * paper: it widens or prunes the Delta-screening set R_t (DCD_MODE_LEARNED).
 * All products run on tensor cores with BF16 operands and FP32 accumulation;
 * training minimises the mean binary cross-entropy with Adam (beta 0.9 /
 * 0.999, eps 1e-8) on FP32 master weights; reductions are deterministic.
 * Parameter layout (DCD_MLP_PARAMS floats): W1[12][64] (row = input), b1[64],
 * W2[64][64] (row = input), b2[64], W3[64], b3.  Features are float32 rows of
 * DCD_MLP_FEATURES values (see dcd_get_screen_data). */
#define DCD_MLP_FEATURES 12
#define DCD_MLP_HIDDEN 64
#define DCD_MLP_PARAMS 5057
typedef struct dcd_mlp dcd_mlp;

/* New network with He-uniform weights from SplitMix64(seed), zero biases, on
 * the current device; work runs on cuda_stream (NULL = default stream). */
int dcd_mlp_create(uint64_t seed, void* cuda_stream, dcd_mlp** out);
int dcd_mlp_destroy(dcd_mlp* mlp);
/* Copy DCD_MLP_PARAMS host floats in / out; setting also resets Adam state. */
int dcd_mlp_set_params(dcd_mlp* mlp, const float* params);
int dcd_mlp_get_params(dcd_mlp* mlp, float* params_out);
/* d_p[r] = sigmoid(network(d_X[r])) for n rows (device float32, n x 12 in). */
int dcd_mlp_forward(dcd_mlp* mlp, const float* d_X, int64_t n, float* d_p);
/* Mean BCE of n rows against d_y (device, 0/1 float32) and its gradient
 * (host, DCD_MLP_PARAMS floats; may be NULL); no update. */
int dcd_mlp_grad(dcd_mlp* mlp, const float* d_X, const float* d_y, int64_t n, float* grad_out, double* loss_out);
/* epochs passes of Adam over rows [0, n) in consecutive minibatches of
 * `batch` rows (the caller shuffles); *loss_out = last minibatch loss. */
int dcd_mlp_train(dcd_mlp* mlp, const float* d_X, const float* d_y, int64_t n, int64_t batch, int32_t epochs,
                  float lr, double* loss_out);

/* The network's parameters to / from a file (host path): magic "DCDMLP01",
 * version 1 and DCD_MLP_PARAMS (uint32 each), the parameters as float32 in
 * the layout above plus one zero float, then a 64-bit FNV-1a checksum over
 * the 8-byte words before it.  The optimiser state is not saved.
 * dcd_mlp_load creates the network on cuda_stream (as dcd_mlp_create) and
 * rejects a file whose header, size, checksum or values (NaN, infinity) are
 * wrong.  Errors: DCD_EINVAL, DCD_EIO (open, write or rename failed),
 * DCD_ENOMEM, DCD_ECUDA. */
int dcd_mlp_save(dcd_mlp* mlp, const char* path);
int dcd_mlp_load(const char* path, void* cuda_stream, dcd_mlp** out);

/* Learned screen for DCD_MODE_LEARNED: every update also runs
 * Delta-screening (R_t), scores the pool (R_t, the vertices the batch touches
 * and their neighbours) with mlp, and evaluates R'_t = {v in R_t : p >=
 * theta_keep} + {v in pool \ R_t : p >= theta_add} at level 0.  With judge
 * set, the step is also run with R_t from the same state; when the learned
 * modularity is more than 1e-3 below it, the plain result is kept and
 * stats.fallback = 1 (q_screen then holds the rejected learned Q; otherwise
 * the plain run's Q).  mlp stays owned by the caller and must outlive its use.
 * Errors: DCD_EINVAL (a threshold outside [0, 1]). */
int dcd_set_screen(dcd_ctx* ctx, dcd_mlp* mlp, float theta_keep, float theta_add, int32_t judge);

/* Training data: with collection on, every update after the first computes
 * the pool features (as in DCD_MODE_LEARNED) under C_{t-1} on G_t and, after
 * the update, the move labels y = [community after level 0 != C_{t-1}] (train
 * on updates in DCD_MODE_BASE).  dcd_get_screen_data copies the last update's
 * rows: X_out (n x 12 float32), y_out (n float32), vertex_out (n int32), each
 * host or device and may be NULL; cap is their row capacity; *n_out (host)
 * receives n.  Errors: DCD_EINVAL (cap < n), DCD_ESTATE (no labels yet). */
int dcd_set_collect(dcd_ctx* ctx, int32_t on);
int dcd_get_screen_data(dcd_ctx* ctx, float* X_out, float* y_out, int32_t* vertex_out, int64_t cap,
                        int64_t* n_out);

/* ---- batched form: many independent dynamic graphs in one context ----
 * G graphs of n[g] vertices each (sum <= 2^31 - 1) advance together: one
 * update runs every kernel once for all graphs (they occupy disjoint vertex
 * ranges of one union graph), while 2m, the tracked modularity and the pass
 * and level stop rules of Algorithm 1 stay per graph, so every graph's result
 * is the one its own context would give.  Modes STATIC, BASE, DELTA only;
 * Louvain only (DCD_ALG_SLM: DCD_EINVAL).
 * dcd_group_apply_batch stages a batch of graph g (local ids in [0, n[g]),
 * host arrays); dcd_group_update advances every graph one step.
 * labels_out: sum(n) int32 (graph after graph, local canonical labels), host
 * or device, may be NULL; q_out: G doubles (host, may be NULL); stats_out: G
 * dcd_step_stats (host, may be NULL).  Errors as dcd_create / dcd_update;
 * DCD_EINVAL also for g out of range. */
typedef struct dcd_group dcd_group;
int dcd_group_create(int32_t G, const int64_t* n, const dcd_config* cfg, void* cuda_stream, dcd_group** out);
int dcd_group_destroy(dcd_group* grp);
int dcd_group_apply_batch(dcd_group* grp, int32_t g, const dcd_edge* ins, int64_t n_ins, const dcd_edge* del,
                          int64_t n_del);
int dcd_group_update(dcd_group* grp, int32_t* labels_out, double* q_out, dcd_step_stats* stats_out);
/* The degree bins of the group's local-move kernels, as dcd_set_bins /
 * dcd_get_bins / dcd_autotune for a context (the union of the G graphs). */
int dcd_group_set_bins(dcd_group* grp, int32_t nb, const int32_t* variant, const int64_t* hi);
int dcd_group_get_bins(const dcd_group* grp, int32_t* nb, int32_t* variant, int64_t* hi);
int dcd_group_autotune(dcd_group* grp, int32_t reps, float* best_ms);

/* ---- allocation-free evaluation ----
 * No counterpart in the paper: a service for callers that cannot allocate
 * device memory when they need the answer (their device memory is held by
 * another allocator, such as a framework's caching allocator, or they run
 * where cudaMalloc/cudaFree must not be called or must not synchronise).
 *
 * Modularity Q of the partition d_labels of the graph given as a device
 * CSR: d_row_ptr (n+1 int64), d_col and d_w (row_ptr[n] int32 each;
 * every undirected edge stored in both rows, positive weights), d_labels
 * (n int32 in [0, n)).  *q_out (host) receives Q, *m2_out (host, may be NULL)
 * 2m.  Work runs on cuda_stream (NULL = legacy default stream) and the call
 * returns when it is done.  No device memory is allocated: the scratch is a
 * fixed 8 MiB array that the library reserves on every GPU where it is loaded
 * and keeps until the process exits.  Every call looks up that array's
 * device address on the current device (the first lookup on a device loads
 * the library's device code there); make the first call on a device before
 * any stream capture.  Every call overwrites the array (each call clears what it needs),
 * so calls whose device work overlaps -- other streams, other host threads --
 * race and return wrong values.
 * Errors: DCD_EINVAL (n <= 0, n > DCD_NOALLOC_MAX_N, NULL pointer, a label or
 * column outside [0, n)), DCD_ECUDA. */
#define DCD_NOALLOC_MAX_N 1048056
int dcd_modularity_noalloc(int64_t n, const int64_t* d_row_ptr, const int32_t* d_col, const int32_t* d_w,
                           const int32_t* d_labels, void* cuda_stream, double* q_out, int64_t* m2_out);

/* ---- fault injection (no counterpart in the paper) ----
 * Makes the library's own error paths testable without a GPU fault: spec
 * "alloc:N" makes the N-th device allocation from now on fail (DCD_ENOMEM),
 * "cuda:N" the N-th checked CUDA runtime call (DCD_ECUDA, with
 * dcd_last_cuda_error naming the call); "alloc:N,cuda:M" arms both.  The
 * failing call is not made -- the library takes the error path a real
 * failure of that call would take -- and each armed kind fires once.  NULL
 * or "" disarms.  The environment variable DCD_FAULT, read when the library
 * loads, takes the same spec.  Process-wide; counts from every thread and
 * context.  Errors: DCD_EINVAL (a malformed spec: the armed state is kept). */
int dcd_set_fault(const char* spec);

/* Text of a status code (static storage). */
const char* dcd_strerror(int code);

/* Text of the last CUDA error seen by this thread (static storage). */
const char* dcd_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif
