// group.cu -- many independent dynamic graphs advanced together.
//
// The G graphs occupy consecutive vertex ranges of one context (the union
// graph has no edge between two ranges), so every kernel of the update runs
// once for all graphs: the batch sort-merge, Delta-screening, the local-move
// passes, the apply and compaction launches.  What Algorithm 1 defines per
// graph -- 2m, the tracked modularity N, the pass and level stop rules -- is
// kept per graph (GraphState), so each graph's communities are exactly those
// of its own single-graph run.  A graph whose levels are over stays inactive
// while the others continue.
#include <cstring>
#include <new>
#include <vector>

#include "prims.cuh"
#include "state.cuh"

struct dcd_group {
  dcd_ctx* ctx = nullptr;
  int32_t G = 0;
  std::vector<int64_t> off;  // G + 1
  std::vector<dcd_edge> ins, del;
};

namespace dcd {
namespace {

__global__ void fill_gid(const int64_t* __restrict__ off, int G, int32_t* __restrict__ gid) {
  for (int g = blockIdx.x; g < G; g += gridDim.x)
    for (int64_t v = off[g] + threadIdx.x; v < off[g + 1]; v += blockDim.x) gid[v] = g;
}

__global__ void to_local(int64_t n, const int32_t* __restrict__ lab, const int32_t* __restrict__ gid,
                         const int64_t* __restrict__ off, int32_t* __restrict__ out) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    out[v] = lab[v] - (int32_t)off[gid[v]];
}

__global__ void per_graph_counts(int G, const int64_t* __restrict__ off, const int64_t* __restrict__ rp,
                                 const uint8_t* __restrict__ r, long long* __restrict__ nnz,
                                 unsigned long long* __restrict__ rsz) {
  for (int g = blockIdx.x; g < G; g += gridDim.x) {
    unsigned long long c = 0;
    for (int64_t v = off[g] + threadIdx.x; v < off[g + 1]; v += blockDim.x) c += r[v] != 0;
    c = warp_sum(c);
    if (lane_id() == 0 && c) atomicAdd(&rsz[g], c);
    if (threadIdx.x == 0) nnz[g] = rp[off[g + 1]] - rp[off[g]];
  }
}

// The group's outputs, written before the step is committed (update_impl's
// finish): per-graph entry counts and |R_t|, and the local labels.
struct GroupOut {
  int G;
  int32_t* labels_out;
  long long* hn;
  unsigned long long* hr;
};

int group_finish(dcd_ctx* c, void* user) {
  const GroupOut* o = static_cast<const GroupOut*>(user);
  cudaStream_t s = c->stream;
  const int G = o->G;
  Buf<long long> nnz;
  Buf<unsigned long long> rsz;
  DCD_TRY(nnz.alloc(&c->mem, G));
  DCD_TRY(rsz.alloc(&c->mem, G));
  DCD_TRY_CUDA(cudaMemsetAsync(rsz.get(), 0, G * sizeof(unsigned long long), s));
  count_launch(), per_graph_counts<<<G < 4096 ? G : 4096, 256, 0, s>>>(G, c->goff_d.get(), c->rp[1 - c->cur].get(),
                                                                      c->rset_nx.get(), nnz.get(), rsz.get());
  DCD_LAUNCH_CHECK();
  DCD_TRY_CUDA(cudaMemcpyAsync(o->hn, nnz.get(), G * sizeof(long long), cudaMemcpyDeviceToHost, s));
  DCD_TRY_CUDA(cudaMemcpyAsync(o->hr, rsz.get(), G * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  if (o->labels_out) {
    Buf<int32_t> loc;
    DCD_TRY(loc.alloc(&c->mem, c->n));
    count_launch(), to_local<<<grid_for(c->n, 256), 256, 0, s>>>(c->n, c->labels_nx.get(), c->gid.get(),
                                                                 c->goff_d.get(), loc.get());
    DCD_LAUNCH_CHECK();
    DCD_TRY_CUDA(cudaMemcpyAsync(o->labels_out, loc.get(), c->n * sizeof(int32_t), cudaMemcpyDefault, s));
  }
  DCD_TRY_CUDA(cudaStreamSynchronize(s));
  return DCD_OK;
}

}  // namespace

int autotune_impl(dcd_ctx* c, int32_t reps, float* best_ms);

}  // namespace dcd

using namespace dcd;

extern "C" {

int dcd_group_create(int32_t G, const int64_t* n, const dcd_config* cfg, void* cuda_stream, dcd_group** out) {
  if (!out || G <= 0 || !n) return DCD_EINVAL;
  *out = nullptr;
  int64_t tot = 0;
  for (int32_t g = 0; g < G; g++) {
    if (n[g] <= 0) return DCD_EINVAL;
    tot += n[g];
    if (tot > INT32_MAX) return DCD_EINVAL;
  }
  dcd_config cf;
  dcd_config_default(&cf);
  if (cfg) cf = *cfg;
  if (cf.mode == DCD_MODE_GIVEN_R || cf.mode == DCD_MODE_LEARNED || cf.alg != DCD_ALG_LOUVAIN) return DCD_EINVAL;
  dcd_group* grp = new (std::nothrow) dcd_group();
  if (!grp) return DCD_ENOMEM;
  grp->G = G;
  grp->off.resize(G + 1);
  grp->off[0] = 0;
  for (int32_t g = 0; g < G; g++) grp->off[g + 1] = grp->off[g] + n[g];
  int rc = dcd_create(tot, &cf, cuda_stream, &grp->ctx);
  if (rc) {
    delete grp;
    return rc;
  }
  dcd_ctx* c = grp->ctx;
  cudaStream_t s = c->stream;
  do {
    c->G = G;
    delete[] c->goff;
    c->goff = new (std::nothrow) int64_t[G + 1];
    if (!c->goff) { rc = DCD_ENOMEM; break; }
    memcpy(c->goff, grp->off.data(), (G + 1) * sizeof(int64_t));
    if ((rc = c->goff_d.alloc(&c->mem, G + 1))) break;
    if ((rc = c->gs.alloc(&c->mem, G))) break;
    if ((rc = c->gid.alloc(&c->mem, tot))) break;
    cudaFreeHost(c->hgs);
    c->hgs = nullptr;
    if (cudaMallocHost(&c->hgs, G * sizeof(GraphState)) != cudaSuccess) { rc = DCD_ENOMEM; break; }
    if (cudaMemcpyAsync(c->goff_d.get(), c->goff, (G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s) !=
        cudaSuccess) { rc = DCD_ECUDA; break; }
    count_launch(), fill_gid<<<G < 4096 ? G : 4096, 256, 0, s>>>(c->goff_d.get(), G, c->gid.get());
    if (cudaStreamSynchronize(s) != cudaSuccess) { rc = DCD_ECUDA; break; }
  } while (0);
  if (rc) {
    dcd_group_destroy(grp);
    return rc;
  }
  *out = grp;
  return DCD_OK;
}

int dcd_group_destroy(dcd_group* grp) {
  if (!grp) return DCD_OK;
  dcd_destroy(grp->ctx);
  delete grp;
  return DCD_OK;
}

int dcd_group_apply_batch(dcd_group* grp, int32_t g, const dcd_edge* ins, int64_t n_ins, const dcd_edge* del,
                          int64_t n_del) {
  if (!grp || g < 0 || g >= grp->G || n_ins < 0 || n_del < 0 || (n_ins && !ins) || (n_del && !del))
    return DCD_EINVAL;
  const int64_t o = grp->off[g], n = grp->off[g + 1] - o;
  for (int64_t i = 0; i < n_ins; i++) {
    const dcd_edge e = ins[i];
    if (e.u < 0 || e.v < 0 || e.u >= n || e.v >= n || e.u == e.v || e.w <= 0) return DCD_EINVAL;
  }
  for (int64_t i = 0; i < n_del; i++) {
    const dcd_edge e = del[i];
    if (e.u < 0 || e.v < 0 || e.u >= n || e.v >= n || e.u == e.v) return DCD_EINVAL;
  }
  for (int64_t i = 0; i < n_ins; i++)
    grp->ins.push_back(dcd_edge{(int32_t)(ins[i].u + o), (int32_t)(ins[i].v + o), ins[i].w});
  for (int64_t i = 0; i < n_del; i++) grp->del.push_back(dcd_edge{(int32_t)(del[i].u + o), (int32_t)(del[i].v + o), 0});
  return DCD_OK;
}

int dcd_group_autotune(dcd_group* grp, int32_t reps, float* best_ms) {
  if (!grp) return DCD_EINVAL;
  DCD_TRY_CUDA(cudaSetDevice(grp->ctx->device));
  return autotune_impl(grp->ctx, reps, best_ms);
}

int dcd_group_set_bins(dcd_group* grp, int32_t nb, const int32_t* variant, const int64_t* hi) {
  return grp ? dcd_set_bins(grp->ctx, nb, variant, hi) : DCD_EINVAL;
}

int dcd_group_get_bins(const dcd_group* grp, int32_t* nb, int32_t* variant, int64_t* hi) {
  return grp ? dcd_get_bins(grp->ctx, nb, variant, hi) : DCD_EINVAL;
}

int dcd_group_update(dcd_group* grp, int32_t* labels_out, double* q_out, dcd_step_stats* stats_out) {
  if (!grp) return DCD_EINVAL;
  dcd_ctx* c = grp->ctx;
  DCD_TRY_CUDA(cudaSetDevice(c->device));
  int rc = dcd_apply_batch(c, grp->ins.data(), (int64_t)grp->ins.size(), grp->del.data(), (int64_t)grp->del.size());
  grp->ins.clear();
  grp->del.clear();
  if (rc) return rc;
  const int G = grp->G;
  std::vector<dcd_step_stats> pg(G);
  memset(pg.data(), 0, G * sizeof(dcd_step_stats));
  dcd_step_stats st;
  memset(&st, 0, sizeof(st));
  const int64_t launches0 = g_launches.load();
  {
    const int64_t R = 2 * (c->n_ins + c->n_del);
    const int64_t nnz_cap = c->nnz + 2 * c->n_ins;
    rc = c->mem.begin_step((size_t)(40 * nnz_cap + 64 * c->n + 48 * R) + ((size_t)64 << 20));
    if (rc) {
      c->n_ins = c->n_del = 0;  // the attempt consumes the staged batches, as a failed update does
      c->staged_on_device = false;
      return rc;
    }
  }
  std::vector<long long> hn(G);
  std::vector<unsigned long long> hr(G);
  GroupOut go{G, labels_out, hn.data(), hr.data()};
  rc = update_impl(c, &st, pg.data(), group_finish, &go);
  c->mem.end_step();
  c->n_ins = c->n_del = 0;
  c->staged_on_device = false;
  if (rc) {
    cudaStreamSynchronize(c->stream);
    cudaGetLastError();
    return rc;
  }
  const int64_t launches = g_launches.load() - launches0;
  for (int g = 0; g < G; g++) {
    dcd_step_stats& o = pg[g];
    o.t = c->t;
    o.n = grp->off[g + 1] - grp->off[g];
    o.nnz = hn[g];
    o.r_size = (int64_t)hr[g];
    o.launches = launches;  // shared by the whole group
    if (q_out) q_out[g] = o.q;
  }
  if (stats_out) memcpy(stats_out, pg.data(), G * sizeof(dcd_step_stats));
  return DCD_OK;
}

}  // extern "C"
