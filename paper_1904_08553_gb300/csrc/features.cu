// features.cu -- the learned screen around Delta-screening (not in the paper).
//
// Pool P = R_t of Delta-screening, plus every vertex touched by the batch and
// its neighbours in G_t.  For each pool vertex of positive degree, under
// C_{t-1} on G_t, twelve features:
//   0 log1p(degree)            1 log1p(d_w)             2 log1p(inserted pairs)
//   3 log1p(deleted pairs)     4 inserted weight / d_w  5 e_{v->C\v} / d_w
//   6 e_{v->D*} / d_w          7 S(v->D*) / (d_w 2m)    8 a_C / 2m
//   9 a_{D*} / 2m             10 log1p(|C|)            11 [v in R_t]
// where D* is the best other neighbouring community by the exact gain S.  The
// network scores each row; R'_t = (R_t with p >= theta_keep) + (P \ R_t with
// p >= theta_add).  Labels for training: 1 when the vertex's community after
// the level-0 local moving of a full re-evaluation (R_t = V) differs from
// C_{t-1}.
#include "agg.cuh"
#include "prims.cuh"
#include "state.cuh"

namespace dcd {
namespace {

constexpr uint8_t kPairIns = 1, kPairDel = 2, kPairPresent = 4;

// pool[v] = R_t[v] | (v has a pair) | (v is a neighbour of a vertex with a pair)
__global__ void pool_mark(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                          const int64_t* __restrict__ pair_ptr, const uint8_t* __restrict__ rds,
                          uint8_t* __restrict__ pool) {
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
    if (lane_id() == 0 && rds[u]) pool[u] = 1;
    if (pair_ptr[u + 1] == pair_ptr[u]) continue;
    if (lane_id() == 0) pool[u] = 1;
    for (int64_t e = rp[u] + lane_id(); e < rp[u + 1]; e += 32) pool[col[e]] = 1;
  }
}

__global__ void assemble(int64_t m, const int32_t* __restrict__ list, const int64_t* __restrict__ rp,
                         const int64_t* __restrict__ k, const int32_t* __restrict__ L, const int64_t* __restrict__ a,
                         const int32_t* __restrict__ size, const int64_t* __restrict__ pair_ptr,
                         const uint8_t* __restrict__ pflag, const int64_t* __restrict__ pw,
                         const int64_t* __restrict__ eC, const int64_t* __restrict__ eB,
                         const int32_t* __restrict__ dB, const double* __restrict__ sB,
                         const uint8_t* __restrict__ rds, int64_t m2, float* __restrict__ X) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = list[i];
    const int64_t deg = rp[v + 1] - rp[v];
    const int64_t kv = k[v];
    const int32_t C = L[v];
    int64_t nins = 0, ndel = 0, wins = 0;
    for (int64_t q = pair_ptr[v]; q < pair_ptr[v + 1]; q++) {
      const uint8_t f = pflag[q];
      if (f & kPairIns) {
        nins++;
        wins += pw[q];
      }
      if ((f & kPairDel) && (f & kPairPresent)) ndel++;
    }
    const float fk = (float)kv, fm = (float)m2;
    const int32_t D = dB[i];
    float* x = X + i * 12;
    x[0] = log1pf((float)deg);
    x[1] = log1pf(fk);
    x[2] = log1pf((float)nins);
    x[3] = log1pf((float)ndel);
    x[4] = kv > 0 ? fminf((float)wins / fk, 1.f) : 0.f;
    x[5] = kv > 0 ? (float)eC[i] / fk : 0.f;
    x[6] = kv > 0 ? (float)eB[i] / fk : 0.f;
    x[7] = (kv > 0 && m2 > 0) ? (float)(sB[i] / ((double)kv * (double)m2)) : 0.f;
    x[8] = m2 > 0 ? (float)a[C] / fm : 0.f;
    x[9] = (m2 > 0 && D >= 0) ? (float)a[D] / fm : 0.f;
    x[10] = log1pf((float)size[C]);
    x[11] = rds[v] ? 1.f : 0.f;
  }
}

__global__ void learned_rset(int64_t m, const int32_t* __restrict__ list, const float* __restrict__ p,
                             const uint8_t* __restrict__ rds, float theta_keep, float theta_add,
                             uint8_t* __restrict__ r, unsigned long long* __restrict__ count) {
  unsigned long long c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = list[i];
    const uint8_t x = rds[v] ? (p[i] >= theta_keep) : (p[i] >= theta_add);
    r[v] = x;
    c += x;
  }
  c = warp_sum(c);
  if (lane_id() == 0 && c) atomicAdd(count, c);
}

__global__ void move_labels(int64_t m, const int32_t* __restrict__ list, const int32_t* __restrict__ before,
                            const int32_t* __restrict__ after, float* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = list[i];
    y[i] = before[v] != after[v] ? 1.f : 0.f;
  }
}

}  // namespace

int screen_features(dcd_ctx* c, const Csr<int32_t>& g, const int32_t* L0, const int64_t* k, const int64_t* a,
                    const int32_t* size, const MergeOut& mo, const uint8_t* rds, LearnedPool* out) {
  cudaStream_t s = c->stream;
  const int64_t n = g.n;
  const int T = 256;
  Buf<uint8_t> pool;
  DCD_TRY(pool.alloc(&c->mem, n));
  DCD_TRY_CUDA(cudaMemsetAsync(pool.get(), 0, n, s));
  count_launch(), pool_mark<<<grid_for(n * 32, T, 16), T, 0, s>>>(n, g.rp, g.col, mo.pair_ptr.get(), rds, pool.get());
  DCD_LAUNCH_CHECK();
  DCD_TRY(pool_stats(c, g, L0, k, a, size, pool.get(), &out->st));
  const int64_t m = out->st.count;
  DCD_TRY(c->feat_X.ensure(&c->mem, 12 * (m > 0 ? m : 1)));
  DCD_TRY(c->feat_v.ensure(&c->mem, m > 0 ? m : 1));
  if (m > 0) {
    count_launch(), assemble<<<grid_for(m, T), T, 0, s>>>(
        m, out->st.list.get(), g.rp, k, L0, a, size, mo.pair_ptr.get(), mo.pflag.get(), mo.pw.get(),
        out->st.eC.get(), out->st.eB.get(), out->st.dB.get(), out->st.sB.get(), rds, c->hgs[0].m2, c->feat_X.get());
    DCD_LAUNCH_CHECK();
    DCD_TRY_CUDA(cudaMemcpyAsync(c->feat_v.get(), out->st.list.get(), m * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  }
  c->feat_n = m;
  return DCD_OK;
}

int learned_rset_build(dcd_ctx* c, const LearnedPool& lp, const uint8_t* rds, const float* p, uint8_t* r,
                       int64_t* r_size) {
  cudaStream_t s = c->stream;
  DevScalars* d = c->dsc.get();
  const int64_t n = c->n;
  const int64_t m = lp.st.count;
  DCD_TRY_CUDA(cudaMemsetAsync(r, 0, n, s));
  DCD_TRY_CUDA(cudaMemsetAsync(&d->r_size, 0, sizeof(int64_t), s));
  if (m > 0) {
    count_launch(), learned_rset<<<grid_for(m, 256), 256, 0, s>>>(m, lp.st.list.get(), p, rds, c->theta_keep,
                                                                   c->theta_add, r, (unsigned long long*)&d->r_size);
    DCD_LAUNCH_CHECK();
  }
  DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch + 11, &d->r_size, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  DCD_TRY_CUDA(cudaStreamSynchronize(s));
  *r_size = c->hscratch[11];
  return DCD_OK;
}

int screen_labels(dcd_ctx* c, const int32_t* before, const int32_t* after) {
  const int64_t m = c->feat_n;
  DCD_TRY(c->feat_y.ensure(&c->mem, m > 0 ? m : 1));
  if (m > 0) {
    count_launch(), move_labels<<<grid_for(m, 256), 256, 0, c->stream>>>(m, c->feat_v.get(), before, after,
                                                                          c->feat_y.get());
    DCD_LAUNCH_CHECK();
  }
  c->feat_has_y = true;
  return DCD_OK;
}

}  // namespace dcd
