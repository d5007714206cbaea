// state.cuh -- the context behind dcd_ctx and the internal interfaces between
// the library's translation units.
#pragma once

#include "common.cuh"

namespace dcd {

// A device CSR graph of one level.  Level 0 keeps int32 weights (the caller's
// multiplicities); compacted levels carry int64 weights.
template <typename W>
struct Csr {
  int64_t n = 0;
  int64_t nnz = 0;
  const int64_t* rp = nullptr;
  const int32_t* col = nullptr;
  const W* w = nullptr;
};

// Per-step scalars kept on the device (one struct, copied back in one go).
struct DevScalars {
  int64_t pad_[9];
  int32_t any_running;  // some graph's pass loop goes on
  int32_t stop_unused;
  int32_t nc;        // labels in use (coarsening)
  int32_t pad0;
  int64_t uniq;      // distinct coarse entries (coarsening)
  int64_t act_deg;   // sum of the active vertices' degrees
  int64_t ncomm;     // communities at the end
  int64_t nsrc;      // screening: distinct sources
  int64_t npairs;    // distinct (src, dst) pairs of the batch
  int64_t r_size;    // |R_t|
  uint32_t err;      // kErr* bits
  uint32_t pad1;
  int64_t bcnt[12];  // active vertices in each degree bin
  int64_t bdeg[12];  // sum of their degrees
  int64_t bmax[12];  // largest degree in the bin
  int32_t pass_id;   // local-move passes started in this update (moved-in-pass marks)
  int32_t level_passes;  // passes of the level running on the device
  unsigned long long stamp[2];  // globaltimer at the start of a pass and after its evaluation
  unsigned long long t_eval_ns, t_apply_ns;  // a level's evaluation and apply time, summed over its passes
  int32_t loop_err;  // the device pass loop hit its hard cap (cannot happen: the stop rule ends it first)
  int32_t pad3;
  int64_t pre_verts;  // level 0: active vertices whose first-pass proposal the screening made
  int64_t pre_deg;    // and the sum of their degrees
};

// Per-graph state of one update.  A context holds G graphs on disjoint vertex
// ranges (G = 1 for dcd_create, G > 1 for a dcd_group); every level-wide
// quantity of Algorithm 1 that the paper defines per graph lives here.
struct GraphState {
  int64_t m2;          // 2m of the graph (equal on every level)
  int64_t in_cur;      // sum_i e_{i->C(i)} of the current labels
  int64_t in_delta;    // change of in_cur produced by the last pass
  unsigned long long sq_lo, sq_hi;  // sum_C a_C^2 (unsigned 128-bit)
  int64_t n_cur_lo, n_cur_hi;       // N of the current labels
  int64_t n_start_lo, n_start_hi;   // N at the start of the level
  int64_t nc;          // labels in use at the end of the level
  int64_t nv;          // vertices of the graph at this level
  int64_t ncomm;       // communities at the end of the update
  int64_t moves_level; // movers summed over the passes of the level
  int32_t moves;       // movers of the last pass
  int32_t running;     // the graph's pass loop at this level goes on
  int32_t passes;      // passes at this level
  int32_t done;        // the graph's levels are over
};

__device__ __forceinline__ int graph_of(const int32_t* gid, int64_t v) { return gid ? gid[v] : 0; }

// Degree bins of the local-move kernels.  A bin holds the active vertices
// whose degree lies in (hi of the previous bin, hi]; each bin runs one kernel
// variant, which bounds the degree it accepts.  Every variant sums the
// neighbour communities of a row in a table in shared memory (louvain.cu):
//   kLmSeg16     1..16     8 lanes a vertex (4 vertices a warp), 2 entries a lane
//   kLmSeg32     ..32      16 lanes a vertex (2 vertices a warp), 2 entries a lane
//   kLmSeg64     ..64      16 lanes a vertex (2 vertices a warp), 4 entries a lane
//   kLmWarp128   ..128     one warp a vertex, 4 entries a lane
//   kLmWarp256   ..256     one warp a vertex, 8 entries a lane
//   kLmCta512    ..512     one CTA of 128 threads a vertex, 4 entries a thread
//   kLmCta1k     ..1024    one CTA of 256 threads, 4 entries a thread
//   kLmCta2k     ..2048    one CTA of 512 threads, 4 entries a thread
//   kLmCta4k     ..4096    one CTA of 512 threads, 8 entries a thread
//   kLmHub       any       a row split over many CTAs, table in global memory
constexpr int kMaxBins = 12;
enum LmVariant : int32_t {
  kLmSeg16 = 0,
  kLmSeg32,
  kLmSeg64,
  kLmWarp128,
  kLmWarp256,
  kLmCta512,
  kLmCta1k,
  kLmCta2k,
  kLmCta4k,
  kLmHub,
  kLmVariants
};
__host__ __device__ __forceinline__ int64_t lm_variant_max(int v) {
  return v == kLmSeg16 ? 16 : v == kLmSeg32 ? 32 : v == kLmSeg64 ? 64 : v == kLmWarp128 ? 128
       : v == kLmWarp256 ? 256 : v == kLmCta512 ? 512 : v == kLmCta1k ? 1024 : v == kLmCta2k ? 2048
       : v == kLmCta4k ? 4096 : INT64_MAX;
}
// The four classes the step statistics report (<= 32, 33..256, 257..4096, hub).
__host__ __device__ __forceinline__ int lm_variant_class(int v) {
  return v <= kLmSeg32 ? 0 : v <= kLmWarp256 ? 1 : v <= kLmCta4k ? 2 : 3;
}

static_assert(sizeof(DevScalars::bcnt) == kMaxBins * sizeof(int64_t), "one counter a bin");

struct BinPlan {
  int32_t nb = 0;
  int32_t var[kMaxBins] = {};
  int64_t hi[kMaxBins] = {};  // the last bin's is INT64_MAX
};

__host__ __device__ __forceinline__ int bin_of(const BinPlan& p, int64_t deg) {
  int b = 0;
  while (b < p.nb - 1 && deg > p.hi[b]) b++;
  return b;
}

// Every variant in degree order, each bin as wide as its kernel allows.
inline BinPlan default_bin_plan() {
  BinPlan p;
  p.nb = 0;
  for (int v = kLmSeg16; v < kLmVariants; v++) {
    p.var[p.nb] = v;
    p.hi[p.nb] = lm_variant_max(v);
    p.nb++;
  }
  return p;
}

// The screening kernels' source bins: 1..32 a warp, 33..256 a warp with a
// shared table, 257..4096 a CTA with a shared table, larger: hub tables in
// global memory (hub.cuh).
constexpr int kBinWarpMax = 32;
constexpr int kBinMidMax = 256;
constexpr int kBinLargeMax = 4096;
constexpr int kMidCap = 512;     // table_cap(kBinMidMax)
constexpr int kLargeCap = 8192;  // table_cap(kBinLargeMax)

}  // namespace dcd

struct dcd_ctx {
  int64_t n = 0;
  dcd_config cfg{};
  int32_t mode = DCD_MODE_DELTA;
  cudaStream_t stream = nullptr;
  bool own_stream = false;  // created by dcd_create (the caller passed none)
  int device = 0;
  int sms = 0;
  dcd::DevMem mem;
  int64_t t = 0;  // time steps computed

  // G_t (level 0), double-buffered so a failed update leaves G_{t-1} intact.
  int cur = 0;
  int64_t nnz = 0;
  dcd::Buf<int64_t> rp[2];
  dcd::Buf<int32_t> col[2];
  dcd::Buf<int32_t> w[2];

  dcd::Buf<int32_t> labels;     // C_t (canonical)
  dcd::Buf<int32_t> labels_nx;  // C_{t+1} under construction
  dcd::Buf<uint8_t> rset;       // R_t of the last update
  dcd::Buf<uint8_t> rset_nx;    // R_t under construction
  dcd::Buf<uint8_t> rgiven;     // R_t for DCD_MODE_GIVEN_R
  bool has_rgiven = false;

  // staged Delta_t
  dcd::Buf<dcd_edge> ins, del;
  int64_t n_ins = 0, n_del = 0;
  bool staged_on_device = false;  // some records still need device validation

  // device scalars + pinned host mirror
  dcd::Buf<dcd::DevScalars> dsc;
  dcd::DevScalars* hsc = nullptr;

  // graphs of the context: G vertex ranges starting at goff[g] (goff[G] = n);
  // gid[v] = graph of vertex v (absent when G = 1)
  int32_t G = 1;
  dcd::Buf<int32_t> gid;
  dcd::Buf<int64_t> goff_d;
  int64_t* goff = nullptr;            // host, G + 1
  dcd::Buf<dcd::GraphState> gs;       // device, G
  dcd::GraphState* hgs = nullptr;     // pinned host mirror, G
  int64_t* hscratch = nullptr;  // pinned, 64 words

  dcd::Buf<int32_t> iota;  // 0..n-1 (singleton labels)

  // learned screen (DCD_MODE_LEARNED) and training-data collection
  struct dcd_mlp* mlp = nullptr;
  float theta_keep = 0.5f, theta_add = 0.5f;
  int32_t judge = 0;
  int32_t collect = 0;
  dcd::Buf<float> feat_X;     // pool rows x 12
  dcd::Buf<float> feat_y;     // pool rows (move labels)
  dcd::Buf<int32_t> feat_v;   // vertex of each pool row
  dcd::Buf<int32_t> level0;   // level-0 labels of the last collected update
  int64_t feat_n = 0;
  bool feat_has_y = false;

  cudaEvent_t ev[24] = {};
  // the local-move bins of a captured pass run on side streams (fork / join)
  bool have_side = false;
  cudaStream_t side[dcd::kMaxBins] = {};
  cudaEvent_t bin_start[dcd::kMaxBins] = {};
  cudaEvent_t join_ev[dcd::kMaxBins] = {};
  cudaEvent_t fork_ev = nullptr;
  dcd::BinPlan bin_plan = dcd::default_bin_plan();  // degree bins of the local-move kernels
  // sum_i e_{i->C(i)} of C_t on G_t per graph, kept by the last update so the
  // next merge need not gather every entry's label (in_valid: it is current;
  // cleared by anything that replaces C_t other than a Louvain update)
  bool in_valid = false;
  dcd::Buf<int64_t> in_prev, in_next;
  // Per-step delta coarsening of level 0 (dense coarse graphs only): K is
  // the coarse graph of G_t under C_t (the last committed labels) as a dense
  // kc_n x kc_n matrix over the communities of C_t in label order; kc_idx maps
  // a label to its row (-1: no community); kc_lab is the inverse.  The next
  // update builds its level-0 coarse graph from K, the batch's weight changes
  // and the rows of the vertices that changed community at level 0, instead
  // of from every entry of G_{t+1}.  The *_nx copies are built during an
  // update and take over at its commit.
  bool kc_valid = false;
  int64_t kc_n = 0, kc_n_nx = 0;
  bool kc_nx_ready = false;
  dcd::Buf<unsigned long long> kc_mat, kc_mat_nx;
  dcd::Buf<int32_t> kc_idx, kc_idx_nx, kc_lab, kc_lab_nx;
  // this update's inputs and level-0 matrix for it
  struct {
    bool track = false;            // build K for the next update
    bool usable = false;           // K holds G_{t-1} under the start labels
    const uint64_t* pkey = nullptr;  // the batch's pairs and their weight changes
    const int64_t* pdelta = nullptr;
    int64_t P = 0;
    const int32_t* cprev = nullptr;  // C_{t-1}
    bool used = false;             // this update took the delta path
    int64_t entries = 0;           // entries the level-0 coarsening read
    bool h0_ready = false;         // h0 holds this update's level-0 matrix
    int64_t h0_nc = 0;
    bool h0_wide = false;          // 64-bit cells
  } n1;
  dcd::Buf<unsigned char> h0;      // level-0 dense coarse matrix of this update
  dcd::Buf<int32_t> h0_ccid;       // level-1 vertex of every vertex
  // level 0 of the last update's local move (dcd_get_level0_bins): active
  // vertices per bin, vertices one sweep of each bin's grid covers, and
  // whether the bins ran side by side
  int32_t l0_nb = 0, l0_side = 0;
  int64_t l0_cnt[dcd::kMaxBins] = {}, l0_sweep[dcd::kMaxBins] = {};
};

namespace dcd {

// merge.cu: sort the staged batch, merge it into G_t (new buffers of ctx at
// index 1 - cur), compute k (weighted degrees), m2 and in under labels0.
// merge.cu: check staged records on the device (ids in [0, n), no self
// loop, positive insert weight); *ok false when one fails.  Synchronises.
int validate_batch(dcd_ctx* c, const dcd_edge* ins, int64_t n_ins, const dcd_edge* del, int64_t n_del, bool* ok);

// api.cu: create the context's side streams and their events once (outside
// stream capture); dcd_destroy releases them.
int side_streams(dcd_ctx* c);

// Kernels with disjoint outputs, run side by side on the context's side
// streams.  fork() marks the point of the context stream every side stream
// starts from; on(x) gives side stream x, made to wait for that point once;
// join() brings every side stream used back into the context stream.  The
// destructor joins whatever is left, so an error return never leaves side
// work unjoined; declare it after the buffers the side work uses, so that
// they are released (stream-ordered, on the context stream) after the join.
// Below kForkMin items the kernels are too small to gain from running side
// by side and the fork would only add its events: everything then stays on
// the context stream.
constexpr int64_t kForkMin = (int64_t)1 << 16;

struct SideBySide {
  dcd_ctx* c;
  bool enabled;
  unsigned used = 0;
  SideBySide(dcd_ctx* cc, int64_t items) : c(cc), enabled(items >= kForkMin) {}
  SideBySide(const SideBySide&) = delete;
  SideBySide& operator=(const SideBySide&) = delete;
  int fork() {
    if (!enabled) return DCD_OK;
    DCD_TRY(side_streams(c));
    DCD_TRY_CUDA(cudaEventRecord(c->fork_ev, c->stream));
    return DCD_OK;
  }
  int on(int x, cudaStream_t* out) {
    if (!enabled) {
      *out = c->stream;
      return DCD_OK;
    }
    if (!(used & (1u << x))) {
      DCD_TRY_CUDA(cudaStreamWaitEvent(c->side[x], c->fork_ev, 0));
      used |= 1u << x;
    }
    *out = c->side[x];
    return DCD_OK;
  }
  int join() {
    for (int x = 0; x < kMaxBins; x++)
      if (used & (1u << x)) {
        DCD_TRY_CUDA(cudaEventRecord(c->join_ev[x], c->side[x]));
        DCD_TRY_CUDA(cudaStreamWaitEvent(c->stream, c->join_ev[x], 0));
        used &= ~(1u << x);
      }
    return DCD_OK;
  }
  ~SideBySide() {
    for (int x = 0; x < kMaxBins; x++)
      if (used & (1u << x)) {
        cudaEventRecord(c->join_ev[x], c->side[x]);
        cudaStreamWaitEvent(c->stream, c->join_ev[x], 0);
      }
  }
};

// api.cu: one time step of a context (or of a group's union graph).  Before
// the step is committed (G_t, C_t, R_t and t replaced), finish(c, user) runs
// when given: it reads the step's results in c->labels_nx, c->rset_nx and
// c->rp/col/w[1 - c->cur] and writes the caller's outputs, so that a failure
// there still leaves the context as it was.
using UpdateFinish = int (*)(dcd_ctx* c, void* user);
int update_impl(dcd_ctx* c, dcd_step_stats* st, dcd_step_stats* per_graph, UpdateFinish finish, void* user);

struct MergeOut {
  Buf<int64_t> k;          // n weighted degrees of G_t
  Buf<uint64_t> pkey;      // distinct (src << 32 | dst) pairs, sorted
  Buf<int64_t> pw;         // summed insert weight per pair (0 = no insert)
  Buf<uint8_t> pflag;      // bit0 insert, bit1 delete, bit2 edge was in G_{t-1}
  Buf<int64_t> pair_ptr;   // n + 1: pairs of source u are [pair_ptr[u], pair_ptr[u+1])
  Buf<int64_t> pdelta;     // per pair: its weight in G_t minus its weight in G_{t-1}
  int64_t npairs = 0;
};
int merge_batch(dcd_ctx* c, const int32_t* labels0, bool static_start, MergeOut* out);

// screen.cu: Algorithm 2 plus the deletion rule -> rset (n bytes).
// size and pre may be NULL; with pre, the first local-move pass's proposal of
// every source whose row phase A sums is written to pre[source] (others -1;
// the caller fills pre with -1).
int screen_batch(dcd_ctx* c, const Csr<int32_t>& g, const int32_t* labels0, const int64_t* k,
                 const int64_t* a, const MergeOut& mo, uint8_t* rset, const int32_t* size = nullptr,
                 int32_t* pre = nullptr);

// louvain.cu: Algorithm 1 from level-0 labels (modified in place into the
// level-0 result), level-0 active flags (NULL = all), k and m2 of G_t.
// Writes canonical labels to out_labels and fills stats.
// a0 / size0 (may be NULL): community sums of labels0, when the caller has them.
int run_louvain(dcd_ctx* c, const Csr<int32_t>& g, int32_t* labels0, const uint8_t* active0,
                Buf<int64_t>& k, int32_t* out_labels, dcd_step_stats* st, int32_t* level0_out = nullptr,
                dcd_step_stats* per_graph = nullptr, const int64_t* a0 = nullptr, const int32_t* size0 = nullptr,
                const int32_t* pre0 = nullptr);

// louvain.cu: multi-level smart local moving (dSLM) from level-0 labels and
// level-0 active flags (NULL = all), k and 2m of G_t (one graph a context).
int run_slm(dcd_ctx* c, const Csr<int32_t>& g0, int32_t* labels0, const uint8_t* active0, Buf<int64_t>& k0,
            int32_t* out_labels, dcd_step_stats* st);

// louvain.cu: statistics of the learned screen's pool (mask over vertices):
// the local-move evaluation of every pool vertex of positive degree, without
// moving, in degree-bin order.  list[i] is the vertex of row i.
struct PoolStats {
  Buf<int32_t> list;
  Buf<int64_t> eC, eB;  // e_{v->C\v}, e_{v->D*}
  Buf<int32_t> dB;      // D* (-1: no other community)
  Buf<double> sB;       // S(v -> D*)
  int64_t count = 0;
};
int pool_stats(dcd_ctx* c, const Csr<int32_t>& g, const int32_t* L, const int64_t* k, const int64_t* a,
               const int32_t* size, const uint8_t* mask, PoolStats* out);

// features.cu: the learned screen's pool, features, R'_t and move labels.
struct LearnedPool {
  PoolStats st;
};
int screen_features(dcd_ctx* c, const Csr<int32_t>& g, const int32_t* L0, const int64_t* k, const int64_t* a,
                    const int32_t* size, const MergeOut& mo, const uint8_t* rds, LearnedPool* out);
int learned_rset_build(dcd_ctx* c, const LearnedPool& lp, const uint8_t* rds, const float* p, uint8_t* r,
                       int64_t* r_size);
int screen_labels(dcd_ctx* c, const int32_t* before, const int32_t* after);

// mlp.cu: forward pass of the network on a given stream (no synchronisation).
int mlp_forward_on(struct dcd_mlp* m, const float* X, int64_t n, float* p, cudaStream_t s);

// louvain.cu: one local-move evaluation of every vertex of g under labels L
// (no move applied) timed for each candidate bin plan; the fastest becomes the
// context's plan.  ms[x] receives candidate x's time per evaluation.
int tune_bins(dcd_ctx* c, const Csr<int32_t>& g, const int32_t* L, const BinPlan* cands, int ncand, int reps,
              float* ms, int* best);
int eval_bins(dcd_ctx* c, const Csr<int32_t>& g, const int32_t* L, int reps, int32_t* nb, int32_t* var,
              int64_t* verts, int64_t* entries, float* ms);

// louvain.cu: community sums a (by label) and sizes from k and labels.
int community_sums(dcd_ctx* c, int64_t n, const int32_t* labels, const int64_t* k, int64_t* a,
                   int32_t* size);

}  // namespace dcd
