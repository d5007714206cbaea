// api.cu -- the extern "C" entry points of dcd.h and the per-step driver
// (Sec. III-D: G_t <- G_{t-1} + Delta_t; R_t; multi-level run; C_t, Q_t).
#include <chrono>
#include <cerrno>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "prims.cuh"
#include "state.cuh"

namespace dcd {

std::atomic<int64_t> g_launches{0};
std::atomic<int64_t> g_fault_left[kFaultKinds];

bool fault_fire(int kind) {
  int64_t v = g_fault_left[kind].load(std::memory_order_relaxed);
  while (v > 0)
    if (g_fault_left[kind].compare_exchange_weak(v, v - 1, std::memory_order_relaxed)) return v == 1;
  return false;
}

namespace {
// "alloc:N,cuda:M" (either, both, or empty = disarmed); N, M >= 1
int parse_fault(const char* spec, int64_t left[kFaultKinds]) {
  for (int k = 0; k < kFaultKinds; k++) left[k] = 0;
  if (!spec) return DCD_OK;
  const char* p = spec;
  while (*p) {
    const char* colon = strchr(p, ':');
    if (!colon) return DCD_EINVAL;
    const size_t len = (size_t)(colon - p);
    const int kind = (len == 5 && !strncmp(p, "alloc", 5)) ? kFaultAlloc
                     : (len == 4 && !strncmp(p, "cuda", 4)) ? kFaultCuda
                                                             : -1;
    if (kind < 0) return DCD_EINVAL;
    char* end = nullptr;
    errno = 0;
    const long long v = strtoll(colon + 1, &end, 10);
    if (end == colon + 1 || errno || v < 1) return DCD_EINVAL;
    left[kind] = v;
    if (*end == ',') p = end + 1;
    else if (*end == '\0') p = end;
    else return DCD_EINVAL;
  }
  return DCD_OK;
}

// DCD_FAULT arms the injector when the library loads
const int g_fault_from_env = [] {
  int64_t left[kFaultKinds];
  if (parse_fault(getenv("DCD_FAULT"), left) == DCD_OK)
    for (int k = 0; k < kFaultKinds; k++) g_fault_left[k].store(left[k]);
  return 0;
}();
}  // namespace

namespace {
thread_local char g_last_cuda[512] = "no CUDA error";
int g_sms_cache = 0;

__global__ void iota_kernel(int32_t* x, int64_t n) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    x[v] = (int32_t)v;
}

// Grow a staging buffer while keeping its first `keep` elements.
template <typename T>
int grow_keep(DevMem* mem, Buf<T>& b, size_t need, size_t keep, cudaStream_t s) {
  if (b.p && b.n >= need) return DCD_OK;
  Buf<T> nb;
  DCD_TRY(nb.ensure(mem, need + need / 2 + 1024));
  if (keep && b.p) DCD_TRY_CUDA(cudaMemcpyAsync(nb.p, b.p, keep * sizeof(T), cudaMemcpyDeviceToDevice, s));
  b.reset();
  b.p = nb.p;
  b.n = nb.n;
  b.mem = mem;
  nb.p = nullptr;
  nb.n = 0;
  return DCD_OK;
}

}  // namespace

void trace(const char* what) {
  static const bool on = getenv("DCD_TRACE") != nullptr;
  if (!on) return;
  using clk = std::chrono::steady_clock;
  static thread_local clk::time_point last = clk::now();
  const clk::time_point now = clk::now();
  fprintf(stderr, "[dcd] %-28s %9.3f ms\n", what, std::chrono::duration<double, std::milli>(now - last).count());
  last = now;
}

bool trace_on() {
  static const bool on = getenv("DCD_TRACE") != nullptr;
  return on;
}

void tracef(const char* fmt, ...) {
  if (!trace_on()) return;
  va_list ap;
  va_start(ap, fmt);
  fprintf(stderr, "[dcd] ");
  vfprintf(stderr, fmt, ap);
  fprintf(stderr, "\n");
  va_end(ap);
}

void note_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_last_cuda, sizeof(g_last_cuda), "%s: %s (%s:%d)", cudaGetErrorString(e), what, file, line);
}

int num_sms() {
  if (!g_sms_cache) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms_cache, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms_cache <= 0) g_sms_cache = 1;
  }
  return g_sms_cache;
}

int side_streams(dcd_ctx* c) {
  if (c->have_side) return DCD_OK;
  for (int x = 0; x < kMaxBins; x++) {
    if (!c->side[x]) DCD_TRY_CUDA(cudaStreamCreateWithFlags(&c->side[x], cudaStreamNonBlocking));
    if (!c->bin_start[x]) DCD_TRY_CUDA(cudaEventCreate(&c->bin_start[x]));
    if (!c->join_ev[x]) DCD_TRY_CUDA(cudaEventCreateWithFlags(&c->join_ev[x], cudaEventDisableTiming));
  }
  if (!c->fork_ev) DCD_TRY_CUDA(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
  c->have_side = true;
  return DCD_OK;
}

int resident_blocks(const void* kernel, int threads, size_t smem) {
  struct Entry {
    const void* k;
    int threads, dev;
    size_t smem;
    int blocks;
  };
  static thread_local std::vector<Entry> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  for (const Entry& e : cache)
    if (e.k == kernel && e.threads == threads && e.smem == smem && e.dev == dev) return e.blocks;
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem) != cudaSuccess || b < 1) {
    cudaGetLastError();
    b = 1;  // the launch itself reports what is wrong
  }
  cache.push_back(Entry{kernel, threads, dev, smem, b});
  return b;
}

int grid_for(int64_t items, int threads, int per_sm) {
  int64_t b = cdiv(items > 0 ? items : 1, threads);
  int64_t cap = (int64_t)num_sms() * per_sm;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

int DevMem::alloc_persistent(void** p, size_t bytes) {
  if (fault_hit(kFaultAlloc)) {
    *p = nullptr;
    return DCD_ENOMEM;
  }
  cudaError_t e = pool ? cudaMallocFromPoolAsync(p, bytes, pool, stream) : cudaMallocAsync(p, bytes, stream);
  if (e != cudaSuccess) {
    note_cuda_error(e, "cudaMallocAsync", __FILE__, __LINE__);
    cudaGetLastError();
    *p = nullptr;
    return DCD_ENOMEM;
  }
  return DCD_OK;
}

int DevMem::alloc(void** p, size_t bytes) {
  const size_t b = (bytes + 255) & ~(size_t)255;
  if (in_step && arena && arena_off + b <= arena_size) {
    if (fault_hit(kFaultAlloc)) {
      *p = nullptr;
      return DCD_ENOMEM;
    }
    *p = arena + arena_off;
    arena_off += b;
    return DCD_OK;
  }
  if (in_step) overflow += b;
  return alloc_persistent(p, bytes);
}

void DevMem::release(void* p) {
  if (!p) return;
  if (arena && static_cast<char*>(p) >= arena && static_cast<char*>(p) < arena + arena_size) return;
  cudaFreeAsync(p, stream);
}

int DevMem::begin_step(size_t hint) {
  // grow by doubling, and only when the last step came near the end (or
  // overflowed), so a slowly growing graph re-sizes the arena rarely
  if (arena_size < hint || last_use > arena_size - arena_size / 8) {
    size_t target = 2 * last_use;
    if (hint + hint / 2 > target) target = hint + hint / 2;
    if (arena) cudaFreeAsync(arena, stream);
    arena = nullptr;
    arena_size = 0;
    void* q = nullptr;
    DCD_TRY(alloc_persistent(&q, target));
    arena = static_cast<char*>(q);
    arena_size = target;
  }
  arena_off = 0;
  overflow = 0;
  in_step = true;
  return DCD_OK;
}

int DevMem::reserve(size_t bytes) {
  if (in_step) return DCD_ESTATE;
  if (arena_size >= bytes) return DCD_OK;
  if (arena) cudaFreeAsync(arena, stream);
  arena = nullptr;
  arena_size = 0;
  void* q = nullptr;
  DCD_TRY(alloc_persistent(&q, bytes));
  arena = static_cast<char*>(q);
  arena_size = bytes;
  last_use = 0;
  return DCD_OK;
}

void DevMem::end_step() {
  if (in_step) last_use = arena_off + overflow;
  arena_off = 0;
  in_step = false;
}

namespace {
__global__ void count_bytes(const uint8_t* r, int64_t n, unsigned long long* out) {
  unsigned long long c = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    c += r[v] != 0;
  c = warp_sum(c);
  if (lane_id() == 0 && c) atomicAdd(out, c);
}
}  // namespace

}  // namespace dcd

using namespace dcd;

#define DCD_SCOPE(c) DCD_TRY_CUDA(cudaSetDevice((c)->device))

extern "C" {

void dcd_config_default(dcd_config* cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof(*cfg));
  cfg->mode = DCD_MODE_DELTA;
  cfg->max_iters = 500;
  cfg->max_levels = 64;
  cfg->tau_inv = 1000000;
}

const char* dcd_strerror(int code) {
  switch (code) {
    case DCD_OK: return "ok";
    case DCD_EINVAL: return "invalid argument";
    case DCD_ENOMEM: return "out of memory";
    case DCD_ECUDA: return "CUDA error";
    case DCD_ESTATE: return "invalid state";
    case DCD_EOVERFLOW: return "integer overflow (weight above INT32_MAX or 2m >= 2^62)";
    case DCD_ETIMEOUT: return "device wait timed out";
    case DCD_EIO: return "file could not be opened, written or renamed";
    default: return "unknown error";
  }
}

const char* dcd_last_cuda_error(void) { return dcd::g_last_cuda; }

int dcd_set_fault(const char* spec) {
  int64_t left[dcd::kFaultKinds];
  DCD_TRY(dcd::parse_fault(spec, left));
  for (int k = 0; k < dcd::kFaultKinds; k++) dcd::g_fault_left[k].store(left[k]);
  return DCD_OK;
}

int64_t dcd_kernel_launches(void) { return dcd::g_launches.load(std::memory_order_relaxed); }

int dcd_create(int64_t n, const dcd_config* cfg, void* cuda_stream, dcd_ctx** out) {
  if (!out || n <= 0 || n > INT32_MAX) return DCD_EINVAL;
  *out = nullptr;
  dcd_config cf;
  dcd_config_default(&cf);
  if (cfg) cf = *cfg;
  if (cf.mode < DCD_MODE_STATIC || cf.mode > DCD_MODE_LEARNED || cf.max_iters <= 0 || cf.max_levels <= 0 ||
      cf.tau_inv <= 0 || (cf.alg != DCD_ALG_LOUVAIN && cf.alg != DCD_ALG_SLM) ||
      (cf.coarsen_full != 0 && cf.coarsen_full != 1) || (cf.pass_loop != 0 && cf.pass_loop != 1))
    return DCD_EINVAL;
  if (cf.alg == DCD_ALG_SLM && n >= ((int64_t)1 << 30)) return DCD_EINVAL;
  dcd_ctx* c = new (std::nothrow) dcd_ctx();
  if (!c) return DCD_ENOMEM;
  c->n = n;
  c->cfg = cf;
  c->mode = cf.mode;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->mem.stream = c->stream;
  int rc = DCD_OK;
  do {
    {
      const cudaError_t ee = cudaGetDevice(&c->device);
      if (ee != cudaSuccess) {
        note_cuda_error(ee, "cudaGetDevice", __FILE__, __LINE__);
        rc = DCD_ECUDA;
        break;
      }
    }
    c->sms = num_sms();
    if (!c->stream) {
      // the local-move passes are replayed as CUDA graphs, which cannot be
      // captured on the legacy default stream: use a stream of our own that
      // is ordered with it (blocking), so device batches written there first
      // are still seen
      const cudaError_t es = cudaStreamCreate(&c->stream);
      if (es != cudaSuccess) {
        note_cuda_error(es, "cudaStreamCreate", __FILE__, __LINE__);
        c->stream = nullptr;
        rc = DCD_ECUDA;
        break;
      }
      c->own_stream = true;
      c->mem.stream = c->stream;
    }
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = c->device;
    if (cudaMemPoolCreate(&c->mem.pool, &props) != cudaSuccess) {
      // many contexts in one process: share the device's default pool
      cudaGetLastError();
      c->mem.pool = nullptr;
    } else {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(c->mem.pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    if (cudaMallocHost(&c->hsc, sizeof(DevScalars)) != cudaSuccess) { rc = DCD_ENOMEM; break; }
    if (cudaMallocHost(&c->hscratch, 64 * sizeof(int64_t)) != cudaSuccess) { rc = DCD_ENOMEM; break; }
    for (auto& e : c->ev) {
      const cudaError_t ee = cudaEventCreate(&e);
      if (ee != cudaSuccess) {
        note_cuda_error(ee, "cudaEventCreate", __FILE__, __LINE__);
        rc = DCD_ECUDA;
        break;
      }
    }
    if (rc) break;
    if ((rc = c->dsc.alloc(&c->mem, 1))) break;
    if ((rc = c->gs.alloc(&c->mem, 1))) break;
    if ((rc = c->goff_d.alloc(&c->mem, 2))) break;
    if (cudaMallocHost(&c->hgs, sizeof(GraphState)) != cudaSuccess) { rc = DCD_ENOMEM; break; }
    c->goff = new (std::nothrow) int64_t[2];
    if (!c->goff) { rc = DCD_ENOMEM; break; }
    c->goff[0] = 0;
    c->goff[1] = n;
    if (cudaMemcpyAsync(c->goff_d.get(), c->goff, 2 * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream) !=
        cudaSuccess) { rc = DCD_ECUDA; break; }
    if ((rc = c->labels.alloc(&c->mem, n))) break;
    if ((rc = c->iota.alloc(&c->mem, n))) break;
    if ((rc = c->rset.alloc(&c->mem, n))) break;
    if ((rc = c->rp[0].alloc(&c->mem, n + 1))) break;
    if ((rc = c->col[0].alloc(&c->mem, 1))) break;
    if ((rc = c->w[0].alloc(&c->mem, 1))) break;
    ::dcd::count_launch(), iota_kernel<<<grid_for(n, 256), 256, 0, c->stream>>>(c->iota.get(), n);
    if (cudaMemcpyAsync(c->labels.get(), c->iota.get(), n * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream) !=
        cudaSuccess) { rc = DCD_ECUDA; break; }
    if (cudaMemsetAsync(c->rp[0].get(), 0, (n + 1) * sizeof(int64_t), c->stream) != cudaSuccess) { rc = DCD_ECUDA; break; }
    if (cudaMemsetAsync(c->rset.get(), 0, n, c->stream) != cudaSuccess) { rc = DCD_ECUDA; break; }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { note_cuda_error(e, "dcd_create", __FILE__, __LINE__); rc = DCD_ECUDA; break; }
  } while (0);
  if (rc) {
    dcd_destroy(c);
    return rc;
  }
  *out = c;
  return DCD_OK;
}

int dcd_destroy(dcd_ctx* c) {
  if (!c) return DCD_OK;
  cudaSetDevice(c->device);
  {
    cudaStreamSynchronize(c->stream);
    c->rp[0].reset(); c->rp[1].reset();
    c->col[0].reset(); c->col[1].reset();
    c->w[0].reset(); c->w[1].reset();
    c->labels.reset(); c->labels_nx.reset(); c->rset.reset(); c->rgiven.reset();
    c->ins.reset(); c->del.reset(); c->dsc.reset(); c->iota.reset(); c->rset_nx.reset();
    c->feat_X.reset(); c->feat_y.reset(); c->feat_v.reset(); c->level0.reset();
    c->gs.reset(); c->goff_d.reset(); c->gid.reset();
    c->in_prev.reset(); c->in_next.reset();
    c->kc_mat.reset(); c->kc_mat_nx.reset(); c->kc_idx.reset(); c->kc_idx_nx.reset();
    c->kc_lab.reset(); c->kc_lab_nx.reset(); c->h0.reset(); c->h0_ccid.reset();
    if (c->mem.arena) cudaFreeAsync(c->mem.arena, c->stream);
    c->mem.arena = nullptr;
    cudaStreamSynchronize(c->stream);
  }
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  for (int x = 0; x < kMaxBins; x++) {
    if (c->side[x]) cudaStreamDestroy(c->side[x]);
    if (c->bin_start[x]) cudaEventDestroy(c->bin_start[x]);
    if (c->join_ev[x]) cudaEventDestroy(c->join_ev[x]);
  }
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->hsc) cudaFreeHost(c->hsc);
  if (c->hgs) cudaFreeHost(c->hgs);
  delete[] c->goff;
  if (c->hscratch) cudaFreeHost(c->hscratch);
  if (c->mem.pool) cudaMemPoolDestroy(c->mem.pool);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return DCD_OK;
}

int dcd_apply_batch(dcd_ctx* c, const dcd_edge* ins, int64_t n_ins, const dcd_edge* del, int64_t n_del) {
  if (!c || n_ins < 0 || n_del < 0 || (n_ins && !ins) || (n_del && !del)) return DCD_EINVAL;
  if ((c->n_ins + n_ins + c->n_del + n_del) * 2 >= (int64_t)INT32_MAX) return DCD_EINVAL;
  DCD_SCOPE(c);
  DCD_TRY(grow_keep(&c->mem, c->ins, c->n_ins + n_ins, c->n_ins, c->stream));
  DCD_TRY(grow_keep(&c->mem, c->del, c->n_del + n_del, c->n_del, c->stream));
  if (n_ins)
    DCD_TRY_CUDA(cudaMemcpyAsync(c->ins.get() + c->n_ins, ins, n_ins * sizeof(dcd_edge), cudaMemcpyHostToDevice,
                                 c->stream));
  if (n_del)
    DCD_TRY_CUDA(cudaMemcpyAsync(c->del.get() + c->n_del, del, n_del * sizeof(dcd_edge), cudaMemcpyHostToDevice,
                                 c->stream));
  // the new records are checked on the device (one pass, then a
  // synchronisation); a bad batch is not counted, so the staged state stays
  bool ok = true;
  DCD_TRY(validate_batch(c, c->ins.get() + c->n_ins, n_ins, c->del.get() + c->n_del, n_del, &ok));
  if (!ok) return DCD_EINVAL;
  c->n_ins += n_ins;
  c->n_del += n_del;
  return DCD_OK;
}

int dcd_apply_batch_device(dcd_ctx* c, const dcd_edge* ins, int64_t n_ins, const dcd_edge* del, int64_t n_del) {
  if (!c || n_ins < 0 || n_del < 0 || (n_ins && !ins) || (n_del && !del)) return DCD_EINVAL;
  if ((c->n_ins + n_ins + c->n_del + n_del) * 2 >= (int64_t)INT32_MAX) return DCD_EINVAL;
  DCD_SCOPE(c);
  DCD_TRY(grow_keep(&c->mem, c->ins, c->n_ins + n_ins, c->n_ins, c->stream));
  DCD_TRY(grow_keep(&c->mem, c->del, c->n_del + n_del, c->n_del, c->stream));
  if (n_ins)
    DCD_TRY_CUDA(cudaMemcpyAsync(c->ins.get() + c->n_ins, ins, n_ins * sizeof(dcd_edge), cudaMemcpyDeviceToDevice,
                                 c->stream));
  if (n_del)
    DCD_TRY_CUDA(cudaMemcpyAsync(c->del.get() + c->n_del, del, n_del * sizeof(dcd_edge), cudaMemcpyDeviceToDevice,
                                 c->stream));
  c->n_ins += n_ins;
  c->n_del += n_del;
  if (n_ins + n_del) c->staged_on_device = true;
  return DCD_OK;
}

}  // extern "C"

namespace dcd {

// Candidate bin plans of the autotuner: the default (every variant from a warp
// per vertex on), with the half-warp variant in front, and coarser layouts
// that drop variants (fewer launches, larger tables).
static std::vector<BinPlan> candidate_plans() {
  const int32_t lists[][kMaxBins] = {
      {kLmSeg16, kLmSeg32, kLmSeg64, kLmWarp128, kLmWarp256, kLmCta512, kLmCta1k, kLmCta2k, kLmCta4k, kLmHub},
      {kLmSeg32, kLmSeg64, kLmWarp128, kLmWarp256, kLmCta512, kLmCta1k, kLmCta2k, kLmCta4k, kLmHub},
      {kLmSeg16, kLmSeg32, kLmWarp128, kLmWarp256, kLmCta512, kLmCta1k, kLmCta2k, kLmCta4k, kLmHub},
      {kLmSeg16, kLmSeg32, kLmSeg64, kLmWarp128, kLmWarp256, kLmCta1k, kLmCta4k, kLmHub},
      {kLmSeg16, kLmSeg32, kLmSeg64, kLmWarp128, kLmWarp256, kLmCta512, kLmCta1k, kLmCta2k, kLmHub},
      {kLmSeg32, kLmWarp256, kLmCta4k, kLmHub},
      {kLmSeg16, kLmSeg32, kLmSeg64, kLmWarp128, kLmWarp256, kLmHub},
  };
  const int lens[] = {10, 9, 9, 8, 9, 4, 6};
  std::vector<BinPlan> out;
  for (int x = 0; x < (int)(sizeof(lens) / sizeof(lens[0])); x++) {
    BinPlan p;
    p.nb = lens[x];
    for (int b = 0; b < p.nb; b++) {
      p.var[b] = lists[x][b];
      p.hi[b] = b == p.nb - 1 ? INT64_MAX : lm_variant_max(lists[x][b]);
    }
    out.push_back(p);
  }
  return out;
}

// Times one local-move evaluation of every vertex of the current graph under
// the current labels for each candidate plan and keeps the fastest.  Every
// plan gives the same proposals; only the time differs.
__global__ void save_in(const GraphState* __restrict__ gs, int G, int64_t* __restrict__ out) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) out[g] = gs[g].in_cur;
}

int autotune_impl(dcd_ctx* c, int32_t reps, float* best_ms) {
  if (c->t == 0 || reps < 1) return DCD_ESTATE;
  const std::vector<BinPlan> cands = candidate_plans();
  std::vector<float> ms(cands.size(), 0.f);
  int best = -1;
  DCD_TRY(c->mem.begin_step((size_t)(32 * c->n) + ((size_t)64 << 20)));
  const int k = c->cur;
  const Csr<int32_t> g{c->n, c->nnz, c->rp[k].get(), c->col[k].get(), c->w[k].get()};
  const int rc = tune_bins(c, g, c->labels.get(), cands.data(), (int)cands.size(), reps, ms.data(), &best);
  c->mem.end_step();
  if (rc) return rc;
  if (trace_on())
    for (size_t x = 0; x < cands.size(); x++)
      tracef("autotune plan %d: %.3f ms%s", (int)x, ms[x], (int)x == best ? " *" : "");
  if (best_ms) *best_ms = best >= 0 ? ms[best] : 0.f;
  return DCD_OK;
}
}  // namespace dcd

int dcd::update_impl(dcd_ctx* c, dcd_step_stats* st, dcd_step_stats* per_graph, UpdateFinish finish, void* user) {
  cudaStream_t s = c->stream;
  const int64_t n = c->n;
  DevScalars* d = c->dsc.get();
  const bool first = c->t == 0;
  const int mode = first ? DCD_MODE_STATIC : c->mode;
  if (mode == DCD_MODE_GIVEN_R && !c->has_rgiven) return DCD_ESTATE;
  // the learned screen and its training data are defined on Louvain's level 0
  if (c->cfg.alg == DCD_ALG_SLM && (mode == DCD_MODE_LEARNED || (c->collect && !first))) return DCD_ESTATE;
  trace("update: enter");
  DCD_TRY_CUDA(cudaEventRecord(c->ev[0], s));
  DCD_TRY_CUDA(cudaMemsetAsync(d, 0, sizeof(DevScalars), s));

  // labels of level 0: singletons (static) or C_{t-1}; the run overwrites them
  Buf<int32_t> L0;
  DCD_TRY(L0.alloc(&c->mem, n));
  const int32_t* src_labels = (mode == DCD_MODE_STATIC) ? c->iota.get() : c->labels.get();
  DCD_TRY_CUDA(cudaMemcpyAsync(L0.get(), src_labels, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));

  MergeOut mo;
  DCD_TRY(merge_batch(c, src_labels, mode == DCD_MODE_STATIC, &mo));
  const int nxt = 1 - c->cur;
  DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch + 8, c->rp[nxt].get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  DCD_TRY_CUDA(cudaMemcpyAsync(c->hsc, d, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
  DCD_TRY_CUDA(cudaMemcpyAsync(c->hgs, c->gs.get(), c->G * sizeof(GraphState), cudaMemcpyDeviceToHost, s));
  DCD_TRY_CUDA(cudaEventRecord(c->ev[1], s));
  DCD_TRY_CUDA(cudaStreamSynchronize(s));
  trace("update: merge done");
  if (c->hsc->err & kErrBadRecord) return DCD_EINVAL;
  if (c->hsc->err & kErrOverflow) return DCD_EOVERFLOW;
  for (int x = 0; x < c->G; x++)
    if (c->hgs[x].m2 < 0 || c->hgs[x].m2 >= ((int64_t)1 << 62)) return DCD_EOVERFLOW;
  // per-graph state after the merge (2m, sum e_{i->C(i)} under C_{t-1}): a
  // second run from the same state starts from this copy
  std::vector<GraphState> gs0(c->hgs, c->hgs + c->G);
  const int64_t nnz_new = c->hscratch[8];
  Csr<int32_t> g{n, nnz_new, c->rp[nxt].get(), c->col[nxt].get(), c->w[nxt].get()};

  // ---- R_t ----
  Buf<uint8_t>& rnew = c->rset_nx;
  DCD_TRY(rnew.ensure(&c->mem, n));
  const uint8_t* active = nullptr;
  int64_t r_size = n, r_screen = -1;
  const bool learned = mode == DCD_MODE_LEARNED;
  const bool collect = c->collect && !first;
  if (learned && !c->mlp) return DCD_ESTATE;
  DCD_TRY_CUDA(cudaEventRecord(c->ev[9], s));
  Buf<uint8_t> rds;  // R_t of Delta-screening
  Buf<int64_t> a;
  Buf<int32_t> size;
  LearnedPool lp;
  // the first level-0 pass of a Delta-screening update reads the state the
  // screening reads (C_{t-1}, its sums on G_t): the screening hands over its
  // proposals for the sources whose rows it sums (one Louvain graph)
  Buf<int32_t> pre;
  const bool use_pre = mode == DCD_MODE_DELTA && !collect && c->G == 1 && c->cfg.alg == DCD_ALG_LOUVAIN;
  if (mode == DCD_MODE_DELTA || learned || collect) {
    DCD_TRY(a.alloc(&c->mem, n));
    DCD_TRY(size.alloc(&c->mem, n));
    DCD_TRY(rds.alloc(&c->mem, n));
    if (use_pre) {
      DCD_TRY(pre.alloc(&c->mem, n));
      DCD_TRY_CUDA(cudaMemsetAsync(pre.get(), 0xff, n * sizeof(int32_t), s));  // -1: none
    }
    DCD_TRY(community_sums(c, n, src_labels, mo.k.get(), a.get(), size.get()));
    DCD_TRY(screen_batch(c, g, src_labels, mo.k.get(), a.get(), mo, rds.get(), size.get(),
                         use_pre ? pre.get() : nullptr));
    DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch + 9, &d->r_size, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    DCD_TRY_CUDA(cudaStreamSynchronize(s));
    r_screen = c->hscratch[9];
  }
  if (learned || collect) {
    DCD_TRY(screen_features(c, g, src_labels, mo.k.get(), a.get(), size.get(), mo, rds.get(), &lp));
    c->feat_has_y = false;
  }
  if (mode == DCD_MODE_DELTA) {
    DCD_TRY_CUDA(cudaMemcpyAsync(rnew.get(), rds.get(), n, cudaMemcpyDeviceToDevice, s));
    r_size = r_screen;
    active = rnew.get();
  } else if (learned) {
    Buf<float> p;
    DCD_TRY(p.alloc(&c->mem, c->feat_n > 0 ? c->feat_n : 1));
    DCD_TRY(mlp_forward_on(c->mlp, c->feat_X.get(), c->feat_n, p.get(), s));
    DCD_TRY(learned_rset_build(c, lp, rds.get(), p.get(), rnew.get(), &r_size));
    active = rnew.get();
  } else if (mode == DCD_MODE_GIVEN_R) {
    DCD_TRY_CUDA(cudaMemcpyAsync(rnew.get(), c->rgiven.get(), n, cudaMemcpyDeviceToDevice, s));
    active = rnew.get();
    DCD_TRY_CUDA(cudaMemsetAsync(&d->r_size, 0, sizeof(int64_t), s));
    ::dcd::count_launch(), count_bytes<<<grid_for(n, 256), 256, 0, s>>>(rnew.get(), n, (unsigned long long*)&d->r_size);
    DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch + 9, &d->r_size, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    DCD_TRY_CUDA(cudaStreamSynchronize(s));
    r_size = c->hscratch[9];
  } else {
    DCD_TRY_CUDA(cudaMemsetAsync(rnew.get(), 1, n, s));
  }
  DCD_TRY_CUDA(cudaEventRecord(c->ev[10], s));
  trace("update: R_t done");

  // ---- Algorithm 1 with R_t at level 0 ----
  // level-0 delta coarsening: usable when K holds G_{t-1} under the start
  // labels; K is rebuilt for the next update unless a judge may replace the
  // labels this run commits
  {
    const bool on = c->cfg.alg == DCD_ALG_LOUVAIN && c->G == 1 && !c->cfg.coarsen_full;
    c->n1 = decltype(c->n1){};
    c->kc_nx_ready = false;
    c->n1.track = on && !(learned && c->judge);
    c->n1.usable = on && mode != DCD_MODE_STATIC && c->kc_valid;
    c->n1.pkey = mo.pkey.get();
    c->n1.pdelta = mo.pdelta.get();
    c->n1.P = mo.npairs;
    c->n1.cprev = c->labels.get();
  }
  DCD_TRY(c->labels_nx.ensure(&c->mem, n));
  if (collect) DCD_TRY(c->level0.ensure(&c->mem, n));
  // the screening's community sums are those of C_{t-1} on G_t, the start of level 0
  if (c->cfg.alg == DCD_ALG_SLM)
    DCD_TRY(run_slm(c, g, L0.get(), active, mo.k, c->labels_nx.get(), st));
  else
    DCD_TRY(run_louvain(c, g, L0.get(), active, mo.k, c->labels_nx.get(), st,
                        collect ? c->level0.get() : nullptr, per_graph, a.n ? a.get() : nullptr,
                        size.n ? size.get() : nullptr, pre.n ? pre.get() : nullptr));
  if (collect) DCD_TRY(screen_labels(c, src_labels, c->level0.get()));
  if (learned && c->judge && st) {
    // the judge: plain Delta-screening from the same state; keep it when the
    // learned set loses more than 1e-3 of modularity
    dcd_step_stats st2;
    memset(&st2, 0, sizeof(st2));
    Buf<int32_t> L0b, lab2;
    DCD_TRY(L0b.alloc(&c->mem, n));
    DCD_TRY(lab2.alloc(&c->mem, n));
    DCD_TRY_CUDA(cudaMemcpyAsync(L0b.get(), src_labels, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    memcpy(c->hgs, gs0.data(), c->G * sizeof(GraphState));
    DCD_TRY_CUDA(cudaMemcpyAsync(c->gs.get(), c->hgs, c->G * sizeof(GraphState), cudaMemcpyHostToDevice, s));
    DCD_TRY(run_louvain(c, g, L0b.get(), rds.get(), mo.k, lab2.get(), &st2));
    st->q_screen = st2.q;
    if (st->q < st2.q - 1e-3) {
      const double ql = st->q;
      *st = st2;
      st->q_screen = ql;  // on a fallback, q_screen reports the rejected learned Q
      st->fallback = 1;
      r_size = r_screen;
      DCD_TRY_CUDA(cudaMemcpyAsync(c->labels_nx.get(), lab2.get(), n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
      DCD_TRY_CUDA(cudaMemcpyAsync(rnew.get(), rds.get(), n, cudaMemcpyDeviceToDevice, s));
    }
  }
  DCD_TRY_CUDA(cudaEventRecord(c->ev[11], s));
  DCD_TRY_CUDA(cudaEventSynchronize(c->ev[11]));
  trace("update: louvain done");
  if (st) {
    st->r_screen = r_screen;
    st->pool = (learned || collect) ? c->feat_n : 0;
    st->coarse0_delta = c->n1.used ? 1 : 0;
    st->coarse0_entries = c->n1.entries;
  }

  // sum_i e_{i->C(i)} of C_t on G_t, kept for the next merge: Louvain's
  // tracked value, except after a judged learned step (its device state then
  // holds the second run) and after SLM (which does not track it)
  const bool keep_in = c->cfg.alg == DCD_ALG_LOUVAIN && !(learned && c->judge);
  if (keep_in) {
    DCD_TRY(c->in_next.ensure(&c->mem, c->G));
    ::dcd::count_launch(), save_in<<<cdiv(c->G, 128), 128, 0, s>>>(c->gs.get(), c->G, c->in_next.get());
    DCD_LAUNCH_CHECK();
  }

  if (finish) DCD_TRY(finish(c, user));

  // ---- commit ----
  if (keep_in) {
    std::swap(c->in_prev.p, c->in_next.p);
    std::swap(c->in_prev.n, c->in_next.n);
    std::swap(c->in_prev.mem, c->in_next.mem);
  }
  c->in_valid = keep_in;
  if (c->kc_nx_ready) {
    std::swap(c->kc_mat.p, c->kc_mat_nx.p);
    std::swap(c->kc_mat.n, c->kc_mat_nx.n);
    std::swap(c->kc_mat.mem, c->kc_mat_nx.mem);
    std::swap(c->kc_idx.p, c->kc_idx_nx.p);
    std::swap(c->kc_idx.n, c->kc_idx_nx.n);
    std::swap(c->kc_idx.mem, c->kc_idx_nx.mem);
    std::swap(c->kc_lab.p, c->kc_lab_nx.p);
    std::swap(c->kc_lab.n, c->kc_lab_nx.n);
    std::swap(c->kc_lab.mem, c->kc_lab_nx.mem);
    c->kc_n = c->kc_n_nx;
  }
  c->kc_valid = c->kc_nx_ready;
  c->kc_nx_ready = false;
  c->cur = nxt;
  c->nnz = nnz_new;
  std::swap(c->labels.p, c->labels_nx.p);
  std::swap(c->labels.n, c->labels_nx.n);
  std::swap(c->rset.p, c->rset_nx.p);
  std::swap(c->rset.n, c->rset_nx.n);
  c->t += 1;
  if (st) {
    float t_all = 0.f, t_merge = 0.f, t_screen = 0.f;
    cudaEventElapsedTime(&t_all, c->ev[0], c->ev[11]);
    cudaEventElapsedTime(&t_merge, c->ev[0], c->ev[1]);
    cudaEventElapsedTime(&t_screen, c->ev[9], c->ev[10]);
    st->t = c->t;
    st->n = n;
    st->nnz = nnz_new;
    st->r_size = r_size;
    st->ins_records = c->n_ins;
    st->del_records = c->n_del;
    st->ms_total = t_all;
    st->ms_merge = t_merge;
    st->ms_screen = t_screen;
  }
  return DCD_OK;
}

extern "C" {

// Device bytes the step arena of an update needs: G_t of at most nnz_cap
// entries, a batch of R directed records.
static size_t step_bytes(const dcd_ctx* c, int64_t nnz_cap, int64_t R) {
  return (size_t)(40 * nnz_cap + 64 * c->n + 48 * R) + ((size_t)64 << 20);
}

int dcd_reserve(dcd_ctx* c, int64_t nnz, int64_t records) {
  if (!c || nnz < 0 || records < 0 || records >= (int64_t)INT32_MAX / 2) return DCD_EINVAL;
  DCD_SCOPE(c);
  const int cur = c->cur, nxt = 1 - c->cur;
  // the buffers of G_t keep their entries; the other pair is empty
  DCD_TRY(grow_keep(&c->mem, c->col[cur], (size_t)nnz, (size_t)c->nnz, c->stream));
  DCD_TRY(grow_keep(&c->mem, c->w[cur], (size_t)nnz, (size_t)c->nnz, c->stream));
  DCD_TRY(c->rp[nxt].ensure(&c->mem, c->n + 1));
  DCD_TRY(c->col[nxt].ensure(&c->mem, nnz));
  DCD_TRY(c->w[nxt].ensure(&c->mem, nnz));
  DCD_TRY(grow_keep(&c->mem, c->ins, (size_t)records, (size_t)c->n_ins, c->stream));
  DCD_TRY(grow_keep(&c->mem, c->del, (size_t)records, (size_t)c->n_del, c->stream));
  DCD_TRY(c->mem.reserve(step_bytes(c, nnz, 2 * records)));
  DCD_TRY_CUDA(cudaStreamSynchronize(c->stream));
  return DCD_OK;
}

int dcd_update(dcd_ctx* c, int32_t* labels_out, double* q_out, dcd_step_stats* stats) {
  if (!c) return DCD_EINVAL;
  DCD_SCOPE(c);
  dcd_step_stats st;
  memset(&st, 0, sizeof(st));
  const int64_t launches0 = dcd::g_launches.load();
  const int64_t R = 2 * (c->n_ins + c->n_del);
  const int64_t nnz_cap = c->nnz + 2 * c->n_ins;
  int rc = c->mem.begin_step(step_bytes(c, nnz_cap, R));
  if (rc == DCD_OK) {
    // labels_out is written before the commit: a failed copy fails the step
    const UpdateFinish copy_labels = [](dcd_ctx* cc, void* out) -> int {
      if (out) {
        DCD_TRY_CUDA(cudaMemcpyAsync(out, cc->labels_nx.get(), cc->n * sizeof(int32_t), cudaMemcpyDefault,
                                     cc->stream));
        DCD_TRY_CUDA(cudaStreamSynchronize(cc->stream));
      }
      return DCD_OK;
    };
    rc = update_impl(c, &st, nullptr, copy_labels, labels_out);
    c->mem.end_step();
  }
  st.launches = dcd::g_launches.load() - launches0;
  // the staged batch is consumed by the attempt, successful or not
  c->n_ins = c->n_del = 0;
  c->staged_on_device = false;
  if (rc != DCD_OK) {
    cudaStreamSynchronize(c->stream);
    cudaGetLastError();
    return rc;
  }
  if (q_out) *q_out = st.q;
  if (stats) *stats = st;
  return DCD_OK;
}

int dcd_get_labels(dcd_ctx* c, int32_t* out) {
  if (!c || !out) return DCD_EINVAL;
  DCD_SCOPE(c);
  DCD_TRY_CUDA(cudaMemcpyAsync(out, c->labels.get(), c->n * sizeof(int32_t), cudaMemcpyDefault, c->stream));
  DCD_TRY_CUDA(cudaStreamSynchronize(c->stream));
  return DCD_OK;
}

int dcd_get_rset(dcd_ctx* c, uint8_t* out) {
  if (!c || !out) return DCD_EINVAL;
  DCD_SCOPE(c);
  DCD_TRY_CUDA(cudaMemcpyAsync(out, c->rset.get(), c->n, cudaMemcpyDefault, c->stream));
  DCD_TRY_CUDA(cudaStreamSynchronize(c->stream));
  return DCD_OK;
}

int dcd_set_labels(dcd_ctx* c, const int32_t* labels) {
  if (!c || !labels) return DCD_EINVAL;
  for (int64_t v = 0; v < c->n; v++)
    if (labels[v] < 0 || labels[v] >= c->n) return DCD_EINVAL;
  DCD_SCOPE(c);
  c->in_valid = false;  // the kept sum_i e_{i->C(i)} belongs to the replaced labels
  c->kc_valid = false;  // and so does the kept coarse graph
  DCD_TRY_CUDA(cudaMemcpyAsync(c->labels.get(), labels, c->n * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
  DCD_TRY_CUDA(cudaStreamSynchronize(c->stream));
  if (c->t == 0) c->t = 1;
  return DCD_OK;
}

int dcd_set_rset(dcd_ctx* c, const uint8_t* r) {
  if (!c || !r) return DCD_EINVAL;
  DCD_SCOPE(c);
  DCD_TRY(c->rgiven.ensure(&c->mem, c->n));
  DCD_TRY_CUDA(cudaMemcpyAsync(c->rgiven.get(), r, c->n, cudaMemcpyHostToDevice, c->stream));
  DCD_TRY_CUDA(cudaStreamSynchronize(c->stream));
  c->has_rgiven = true;
  return DCD_OK;
}

int dcd_set_mode(dcd_ctx* c, int32_t mode) {
  if (!c || mode < DCD_MODE_STATIC || mode > DCD_MODE_LEARNED) return DCD_EINVAL;
  c->mode = mode;
  return DCD_OK;
}

static_assert(DCD_MAX_BINS == kMaxBins && DCD_LM_SEG16 == kLmSeg16 && DCD_LM_SEG32 == kLmSeg32 &&
                  DCD_LM_SEG64 == kLmSeg64 && DCD_LM_WARP128 == kLmWarp128 && DCD_LM_WARP256 == kLmWarp256 &&
                  DCD_LM_CTA512 == kLmCta512 && DCD_LM_CTA1K == kLmCta1k && DCD_LM_CTA2K == kLmCta2k &&
                  DCD_LM_CTA4K == kLmCta4k && DCD_LM_HUB == kLmHub,
              "variant ids of dcd.h and the kernels agree");

int dcd_set_bins(dcd_ctx* c, int32_t nb, const int32_t* variant, const int64_t* hi) {
  if (!c || nb < 1 || nb > kMaxBins || !variant || !hi) return DCD_EINVAL;
  BinPlan p;
  p.nb = nb;
  for (int b = 0; b < nb; b++) {
    const bool last = b == nb - 1;
    const int64_t h = last ? INT64_MAX : hi[b];
    if (variant[b] < 0 || variant[b] >= kLmVariants) return DCD_EINVAL;
    if (last ? (hi[b] != -1 || variant[b] != kLmHub) : (h < 1 || h > lm_variant_max(variant[b]) || variant[b] == kLmHub))
      return DCD_EINVAL;
    if (b > 0 && h <= p.hi[b - 1]) return DCD_EINVAL;
    p.var[b] = variant[b];
    p.hi[b] = h;
  }
  c->bin_plan = p;
  return DCD_OK;
}

int dcd_get_bins(const dcd_ctx* c, int32_t* nb, int32_t* variant, int64_t* hi) {
  if (!c || !nb) return DCD_EINVAL;
  *nb = c->bin_plan.nb;
  for (int b = 0; b < c->bin_plan.nb; b++) {
    if (variant) variant[b] = c->bin_plan.var[b];
    if (hi) hi[b] = c->bin_plan.hi[b] == INT64_MAX ? -1 : c->bin_plan.hi[b];
  }
  return DCD_OK;
}

int dcd_get_level0_bins(const dcd_ctx* c, int32_t* nb, int64_t* count, int64_t* per_sweep, int32_t* side_by_side) {
  if (!c || !nb) return DCD_EINVAL;
  *nb = c->l0_nb;
  for (int b = 0; b < c->l0_nb; b++) {
    if (count) count[b] = c->l0_cnt[b];
    if (per_sweep) per_sweep[b] = c->l0_sweep[b];
  }
  if (side_by_side) *side_by_side = c->l0_side;
  return DCD_OK;
}

int dcd_autotune(dcd_ctx* c, int32_t reps, float* best_ms) {
  if (!c) return DCD_EINVAL;
  DCD_SCOPE(c);
  return autotune_impl(c, reps, best_ms);
}

int dcd_eval_bins(dcd_ctx* c, int32_t reps, int32_t* nb, int32_t* variant, int64_t* verts, int64_t* entries,
                  float* ms) {
  if (!c || !nb || !variant || !verts || !entries || !ms) return DCD_EINVAL;
  if (c->t == 0 || reps < 1) return DCD_ESTATE;
  DCD_SCOPE(c);
  DCD_TRY(c->mem.begin_step((size_t)(32 * c->n) + ((size_t)64 << 20)));
  const int k = c->cur;
  const Csr<int32_t> g{c->n, c->nnz, c->rp[k].get(), c->col[k].get(), c->w[k].get()};
  const int rc = eval_bins(c, g, c->labels.get(), reps, nb, variant, verts, entries, ms);
  c->mem.end_step();
  return rc;
}

int dcd_set_screen(dcd_ctx* c, dcd_mlp* mlp, float theta_keep, float theta_add, int32_t judge) {
  if (!c || !(theta_keep >= 0.f && theta_keep <= 1.f) || !(theta_add >= 0.f && theta_add <= 1.f)) return DCD_EINVAL;
  c->mlp = mlp;
  c->theta_keep = theta_keep;
  c->theta_add = theta_add;
  c->judge = judge ? 1 : 0;
  return DCD_OK;
}

int dcd_set_collect(dcd_ctx* c, int32_t on) {
  if (!c) return DCD_EINVAL;
  c->collect = on ? 1 : 0;
  return DCD_OK;
}

int dcd_get_screen_data(dcd_ctx* c, float* X_out, float* y_out, int32_t* vertex_out, int64_t cap, int64_t* n_out) {
  if (!c || !n_out) return DCD_EINVAL;
  *n_out = c->feat_n;
  if (!X_out && !y_out && !vertex_out) return DCD_OK;
  if (cap < c->feat_n) return DCD_EINVAL;
  if (y_out && !c->feat_has_y) return DCD_ESTATE;
  DCD_SCOPE(c);
  const int64_t m = c->feat_n;
  if (m > 0) {
    if (X_out)
      DCD_TRY_CUDA(cudaMemcpyAsync(X_out, c->feat_X.get(), m * 12 * sizeof(float), cudaMemcpyDefault, c->stream));
    if (y_out) DCD_TRY_CUDA(cudaMemcpyAsync(y_out, c->feat_y.get(), m * sizeof(float), cudaMemcpyDefault, c->stream));
    if (vertex_out)
      DCD_TRY_CUDA(cudaMemcpyAsync(vertex_out, c->feat_v.get(), m * sizeof(int32_t), cudaMemcpyDefault, c->stream));
  }
  DCD_TRY_CUDA(cudaStreamSynchronize(c->stream));
  return DCD_OK;
}

int dcd_get_graph(dcd_ctx* c, int64_t* nnz_out, int64_t* row_ptr, int32_t* col, int32_t* w) {
  if (!c) return DCD_EINVAL;
  if (nnz_out) *nnz_out = c->nnz;
  DCD_SCOPE(c);
  const int k = c->cur;
  if (row_ptr)
    DCD_TRY_CUDA(cudaMemcpyAsync(row_ptr, c->rp[k].get(), (c->n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost,
                                 c->stream));
  if (col && c->nnz)
    DCD_TRY_CUDA(cudaMemcpyAsync(col, c->col[k].get(), c->nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  if (w && c->nnz)
    DCD_TRY_CUDA(cudaMemcpyAsync(w, c->w[k].get(), c->nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  DCD_TRY_CUDA(cudaStreamSynchronize(c->stream));
  return DCD_OK;
}

}  // extern "C"
