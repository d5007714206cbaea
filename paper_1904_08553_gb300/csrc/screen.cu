// screen.cu -- Delta-screening (Algorithm 2, Sec. III-E) and the deletion
// rule, on G_t with the inherited labels C_{t-1}; then R_t.
//
// Per source i of the batch (the distinct (source, sink) pairs are already
// sorted by source):
//   inserts: j* = argmax over the insert sinks j of S(i -> C(j)) (S = 0 when
//     C(j) = C(i); ties to the smaller C(j), then the smaller j -- the paper
//     fixes no tie rule); gain1 = S(i -> C(j*)), gain2 = S(j* -> C(i)); when
//     gain1 >= gain2 and gain1 > 0: mark i, j*, Gamma(i), flag C(j*).
//   deletes (not in the paper; reading): for each deleted pair (i, j) whose
//     edge was in G_{t-1}: mark i and j; if C(i) = C(j) also mark Gamma(i).
// R_t = marked vertices plus the members of flagged communities.  Screening
// changes no label.
#include "agg.cuh"
#include "prims.cuh"
#include "state.cuh"

namespace dcd {

namespace {

constexpr uint8_t kPairIns = 1, kPairDel = 2, kPairPresent = 4;

struct SV {
  const int64_t* rp;
  const int32_t* col;
  const int32_t* w;
  const int64_t* k;
  const int32_t* L;
  const int64_t* a;
  const uint64_t* pkey;
  const uint8_t* pflag;
  const int64_t* pair_ptr;
  int64_t m2;
  uint8_t* mark;
  uint8_t* cflag;
};

// (S, D, j) order of the j* choice: larger gain, then smaller C(j), then smaller j.
template <typename ST>
__device__ __forceinline__ bool better3(ST s1, int32_t d1, int32_t j1, ST s2, int32_t d2, int32_t j2) {
  return s1 > s2 || (s1 == s2 && (d1 < d2 || (d1 == d2 && j1 < j2)));
}

template <typename ST>
__device__ __forceinline__ void warp_argmax3(ST& S, int32_t& D, int32_t& J) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ST s2 = shfl_xor_st(S, o);
    int32_t d2 = __shfl_xor_sync(0xffffffffu, D, o);
    int32_t j2 = __shfl_xor_sync(0xffffffffu, J, o);
    if (better3(s2, d2, j2, S, D, J)) {
      S = s2;
      D = d2;
      J = j2;
    }
  }
}

// gain2 = S(j* -> C(i)) from one scan of row j*: weights into C(i) and into
// C(j*) without j*'s self entries.  Returns the two sums through the warp.
__device__ __forceinline__ void row_two_sums(const SV& g, int32_t j, int32_t Ci, int32_t Cj, int64_t* e_i,
                                             int64_t* e_j, int tid, int nthreads) {
  int64_t s1 = 0, s2 = 0;
  const int64_t b = g.rp[j], e1 = g.rp[j + 1];
  for (int64_t e = b + tid; e < e1; e += nthreads) {
    const int32_t y = g.col[e];
    if (y == j) continue;
    const int32_t ly = g.L[y];
    if (ly == Ci) s1 += g.w[e];
    if (ly == Cj) s2 += g.w[e];
  }
  *e_i = s1;
  *e_j = s2;
}

__device__ __forceinline__ void mark_row(const SV& g, int32_t u, int tid, int nthreads) {
  const int64_t b = g.rp[u], e1 = g.rp[u + 1];
  for (int64_t e = b + tid; e < e1; e += nthreads) g.mark[g.col[e]] = 1;
}

// ---- one warp per source of degree <= 32 in G_t ----
template <typename ST>
__global__ void __launch_bounds__(256) screen_warp(SV g, const int32_t* __restrict__ src, int64_t cnt) {
  const int lane = lane_id();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < cnt; i += nw) {
    const int32_t u = src[i];
    const int32_t C = g.L[u];
    const int64_t p0 = g.pair_ptr[u], p1 = g.pair_ptr[u + 1];
    bool intra = false, has_ins = false;
    for (int64_t q = p0 + lane; q < p1; q += 32) {
      const uint8_t f = g.pflag[q];
      has_ins |= (f & kPairIns) != 0;
      if ((f & kPairDel) && (f & kPairPresent)) {
        const int32_t j = (int32_t)(g.pkey[q] & 0xffffffffu);
        g.mark[j] = 1;
        g.mark[u] = 1;
        intra |= g.L[j] == C;
      }
    }
    intra = __any_sync(0xffffffffu, intra);
    has_ins = __any_sync(0xffffffffu, has_ins);
    bool mark_gamma = intra;
    if (has_ins) {
      // lanes hold row u (degree <= 32): group by label
      const int64_t b = g.rp[u];
      const int d = (int)(g.rp[u + 1] - b);
      bool valid = lane < d;
      const int32_t y = valid ? g.col[b + lane] : -1;
      valid = valid && y != u;
      const int32_t lab = valid ? g.L[y] : -1;
      const int32_t wt = valid ? g.w[b + lane] : 0;
      const unsigned peers = __match_any_sync(0xffffffffu, lab);
      const int64_t e = group_sum_exact(peers, wt);
      const bool leader = valid && (int)(__ffs(peers) - 1) == lane;
      const unsigned leaders = __ballot_sync(0xffffffffu, leader);
      const unsigned cm = __ballot_sync(0xffffffffu, leader && lab == C);
      const int64_t eCx = __shfl_sync(0xffffffffu, e, cm ? __ffs(cm) - 1 : 0);
      const int64_t eC = cm ? eCx : 0;
      const int64_t ku = g.k[u], aC = g.a[C];
      ST S = gain_lowest<ST>();
      int32_t D = INT_MAX, J = INT_MAX;
      for (int64_t q0 = p0; q0 < p1; q0 += 32) {
        const int64_t q = q0 + lane;
        const bool sink = q < p1 && (g.pflag[q] & kPairIns);
        const int32_t j = sink ? (int32_t)(g.pkey[q] & 0xffffffffu) : -1;
        const int32_t Dj = sink ? g.L[j] : -1;
        int64_t eD = 0;
        for (unsigned lm = leaders; lm; lm &= lm - 1) {
          const int l = __ffs(lm) - 1;
          const int32_t ll = __shfl_sync(0xffffffffu, lab, l);
          const int64_t el = __shfl_sync(0xffffffffu, e, l);
          if (ll == Dj) eD = el;
        }
        if (sink) {
          const ST x = (Dj == C) ? ST(0) : gain<ST>(g.m2, ku, eD, eC, g.a[Dj], aC);
          if (better3(x, Dj, j, S, D, J)) {
            S = x;
            D = Dj;
            J = j;
          }
        }
      }
      warp_argmax3(S, D, J);
      // gain2 = S(j* -> C(i))
      int64_t e_i = 0, e_j = 0;
      row_two_sums(g, J, C, D, &e_i, &e_j, lane, 32);
      e_i = warp_sum((long long)e_i);
      e_j = warp_sum((long long)e_j);
      const ST g2 = (D == C) ? ST(0) : gain<ST>(g.m2, g.k[J], e_i, e_j, aC, g.a[D]);
      if (S >= g2 && S > 0) {
        if (lane == 0) {
          g.mark[u] = 1;
          g.mark[J] = 1;
          g.cflag[D] = 1;
        }
        mark_gamma = true;
      }
    }
    if (mark_gamma) {
      if (lane == 0) g.mark[u] = 1;
      mark_row(g, u, lane, 32);
    }
  }
}

// ---- one CTA per source of degree > 32: table in shared or global memory ----
template <typename ST, int THREADS>
__global__ void __launch_bounds__(THREADS) screen_block(SV g, const int32_t* __restrict__ src, int64_t cnt,
                                                        int32_t* __restrict__ gkeys,
                                                        unsigned long long* __restrict__ gvals, int64_t gcap) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NW = THREADS / 32;
  __shared__ ST redS[NW];
  __shared__ int32_t redD[NW], redJ[NW];
  __shared__ long long red1[NW], red2[NW];
  __shared__ int s_flags;
  __shared__ long long s_eC;
  const int tid = threadIdx.x, lane = lane_id(), wid = tid >> 5;
  for (int64_t i = blockIdx.x; i < cnt; i += gridDim.x) {
    const int32_t u = src[i];
    const int32_t C = g.L[u];
    const int64_t p0 = g.pair_ptr[u], p1 = g.pair_ptr[u + 1];
    if (tid == 0) s_flags = 0;
    __syncthreads();
    int fl = 0;
    for (int64_t q = p0 + tid; q < p1; q += THREADS) {
      const uint8_t f = g.pflag[q];
      if (f & kPairIns) fl |= 2;
      if ((f & kPairDel) && (f & kPairPresent)) {
        const int32_t j = (int32_t)(g.pkey[q] & 0xffffffffu);
        g.mark[j] = 1;
        g.mark[u] = 1;
        if (g.L[j] == C) fl |= 1;
      }
    }
    if (fl) atomicOr(&s_flags, fl);
    __syncthreads();
    const int flags = s_flags;
    bool mark_gamma = flags & 1;
    if (flags & 2) {
      const int64_t b = g.rp[u];
      const int64_t d = g.rp[u + 1] - b;
      const uint32_t cap = table_cap(d), mask = cap - 1;
      int32_t* keys;
      unsigned long long* vals;
      if (gcap == 0) {
        vals = reinterpret_cast<unsigned long long*>(smem);
        keys = reinterpret_cast<int32_t*>(smem + (size_t)cap * sizeof(unsigned long long));
      } else {
        keys = gkeys + (int64_t)blockIdx.x * gcap;
        vals = gvals + (int64_t)blockIdx.x * gcap;
      }
      for (uint32_t s = tid; s < cap; s += THREADS) {
        keys[s] = -1;
        vals[s] = 0;
      }
      __syncthreads();
      for (int64_t e0 = 0; e0 < d; e0 += THREADS) {
        const int64_t e = e0 + tid;
        bool valid = e < d;
        const int32_t y = valid ? g.col[b + e] : -1;
        valid = valid && y != u;
        const int32_t lab = valid ? g.L[y] : -1;
        const int32_t wt = valid ? g.w[b + e] : 0;
        const unsigned peers = __match_any_sync(0xffffffffu, lab);
        const int64_t sum = group_sum_exact(peers, wt);
        if (valid && (int)(__ffs(peers) - 1) == lane) tbl_add(keys, vals, mask, lab, (unsigned long long)sum);
      }
      __syncthreads();
      if (tid == 0) s_eC = tbl_get(keys, vals, mask, C);
      __syncthreads();
      const int64_t eC = s_eC, ku = g.k[u], aC = g.a[C];
      ST S = gain_lowest<ST>();
      int32_t D = INT_MAX, J = INT_MAX;
      for (int64_t q = p0 + tid; q < p1; q += THREADS) {
        if (!(g.pflag[q] & kPairIns)) continue;
        const int32_t j = (int32_t)(g.pkey[q] & 0xffffffffu);
        const int32_t Dj = g.L[j];
        const ST x = (Dj == C) ? ST(0) : gain<ST>(g.m2, ku, tbl_get(keys, vals, mask, Dj), eC, g.a[Dj], aC);
        if (better3(x, Dj, j, S, D, J)) {
          S = x;
          D = Dj;
          J = j;
        }
      }
      warp_argmax3(S, D, J);
      if (lane == 0) {
        redS[wid] = S;
        redD[wid] = D;
        redJ[wid] = J;
      }
      __syncthreads();
      S = lane < NW ? redS[lane] : gain_lowest<ST>();
      D = lane < NW ? redD[lane] : INT_MAX;
      J = lane < NW ? redJ[lane] : INT_MAX;
      warp_argmax3(S, D, J);  // every warp computes the same result
      int64_t e_i = 0, e_j = 0;
      row_two_sums(g, J, C, D, &e_i, &e_j, tid, THREADS);
      e_i = warp_sum((long long)e_i);
      e_j = warp_sum((long long)e_j);
      if (lane == 0) {
        red1[wid] = e_i;
        red2[wid] = e_j;
      }
      __syncthreads();
      e_i = lane < NW ? red1[lane] : 0;
      e_j = lane < NW ? red2[lane] : 0;
      e_i = warp_sum((long long)e_i);
      e_j = warp_sum((long long)e_j);
      const ST g2 = (D == C) ? ST(0) : gain<ST>(g.m2, g.k[J], e_i, e_j, aC, g.a[D]);
      if (S >= g2 && S > 0) {
        if (tid == 0) {
          g.mark[u] = 1;
          g.mark[J] = 1;
          g.cflag[D] = 1;
        }
        mark_gamma = true;
      }
    }
    if (mark_gamma) {
      if (tid == 0) g.mark[u] = 1;
      mark_row(g, u, tid, THREADS);
    }
    __syncthreads();
  }
}

// Sources (vertices with at least one pair) binned by their degree in G_t.
__global__ void src_bins(int64_t n, const int64_t* __restrict__ pair_ptr, const int64_t* __restrict__ rp,
                         int32_t* __restrict__ cursor, int32_t* __restrict__ lst_small,
                         int32_t* __restrict__ lst_mid, int32_t* __restrict__ lst_hub,
                         unsigned long long* __restrict__ hub_max) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x) + (threadIdx.x & ~31); base < n; base += stride) {
    const int64_t v = base + lane_id();
    int bin = -1;
    if (v < n && pair_ptr[v + 1] > pair_ptr[v]) {
      const int64_t deg = rp[v + 1] - rp[v];
      bin = deg <= kBinWarpMax ? 0 : deg <= kBinLargeMax ? 1 : 2;
      if (bin == 2) atomicMax(hub_max, (unsigned long long)deg);
    }
#pragma unroll
    for (int b = 0; b < 3; b++) {
      const unsigned bal = __ballot_sync(0xffffffffu, bin == b);
      if (!bal) continue;
      int32_t slot = 0;
      if (lane_id() == 0) slot = atomicAdd(&cursor[b], __popc(bal));
      slot = __shfl_sync(0xffffffffu, slot, 0);
      int32_t* lst = b == 0 ? lst_small : b == 1 ? lst_mid : lst_hub;
      if (bin == b) lst[slot + __popc(bal & lanemask_lt())] = (int32_t)v;
    }
  }
}

__global__ void build_rset(int64_t n, const uint8_t* __restrict__ mark, const uint8_t* __restrict__ cflag,
                           const int32_t* __restrict__ L, uint8_t* __restrict__ r,
                           unsigned long long* __restrict__ count) {
  unsigned long long c = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t x = mark[v] | cflag[L[v]];
    r[v] = x;
    c += x;
  }
  c = warp_sum(c);
  if (lane_id() == 0 && c) atomicAdd(count, c);
}

}  // namespace

int screen_batch(dcd_ctx* c, const Csr<int32_t>& g, const int32_t* labels0, const int64_t* k, const int64_t* a,
                 const MergeOut& mo, uint8_t* rset) {
  cudaStream_t s = c->stream;
  DevScalars* d = c->dsc.get();
  const int64_t n = g.n;
  const int T = 256;
  Buf<uint8_t> mark, cflag;
  Buf<int32_t> lists, cursor;
  Buf<unsigned long long> hubmax;
  DCD_TRY(mark.alloc(&c->mem, n));
  DCD_TRY(cflag.alloc(&c->mem, n));
  DCD_TRY(lists.alloc(&c->mem, 3 * n));
  DCD_TRY(cursor.alloc(&c->mem, 4));
  DCD_TRY(hubmax.alloc(&c->mem, 1));
  DCD_TRY_CUDA(cudaMemsetAsync(mark.get(), 0, n, s));
  DCD_TRY_CUDA(cudaMemsetAsync(cflag.get(), 0, n, s));
  DCD_TRY_CUDA(cudaMemsetAsync(cursor.get(), 0, 4 * sizeof(int32_t), s));
  DCD_TRY_CUDA(cudaMemsetAsync(hubmax.get(), 0, sizeof(unsigned long long), s));
  int32_t* l0 = lists.get();
  int32_t* l1 = l0 + n;
  int32_t* l2 = l1 + n;
  if (mo.npairs > 0) {
    ::dcd::count_launch(), src_bins<<<grid_for(n, T), T, 0, s>>>(n, mo.pair_ptr.get(), g.rp, cursor.get(), l0, l1, l2, hubmax.get());
    DCD_LAUNCH_CHECK();
    DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch, cursor.get(), 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch + 2, hubmax.get(), sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    DCD_TRY_CUDA(cudaStreamSynchronize(s));
    const int32_t* cnts = reinterpret_cast<const int32_t*>(c->hscratch);
    const int64_t c0 = cnts[0], c1 = cnts[1], c2 = cnts[2];
    const int64_t hub_max = c->hscratch[2];
    SV sv{g.rp, g.col, g.w, k, labels0, a, mo.pkey.get(), mo.pflag.get(), mo.pair_ptr.get(), c->hsc->m2,
          mark.get(), cflag.get()};
    const bool wide = sv.m2 >= ((int64_t)1 << 31);
    const size_t smem = (size_t)kLargeCap * 12;
    Buf<int32_t> hkeys;
    Buf<unsigned long long> hvals;
    int64_t hub_cap = 0, hub_ctas = 0;
    if (c2) {
      hub_cap = table_cap(hub_max);
      hub_ctas = ((int64_t)1 << 30) / (hub_cap * 12);
      if (hub_ctas < 1) hub_ctas = 1;
      if (hub_ctas > c2) hub_ctas = c2;
      if (hub_ctas > 4 * (int64_t)c->sms) hub_ctas = 4 * (int64_t)c->sms;
      DCD_TRY(hkeys.alloc(&c->mem, hub_ctas * hub_cap));
      DCD_TRY(hvals.alloc(&c->mem, hub_ctas * hub_cap));
    }
#define DCD_SCREEN(ST)                                                                                           \
  do {                                                                                                           \
    DCD_TRY_CUDA(cudaFuncSetAttribute(screen_block<ST, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,        \
                                      (int)smem));                                                               \
    if (c0) ::dcd::count_launch(), screen_warp<ST><<<grid_for(c0 * 32, T, 16), T, 0, s>>>(sv, l0, c0);                                  \
    if (c1)                                                                                                      \
      ::dcd::count_launch(), screen_block<ST, 256><<<(unsigned)(c1 < 2 * c->sms ? c1 : 2 * c->sms), 256, smem, s>>>(sv, l1, c1, nullptr, \
                                                                                             nullptr, 0);        \
    if (c2)                                                                                                      \
      ::dcd::count_launch(), screen_block<ST, 512><<<(unsigned)hub_ctas, 512, 0, s>>>(sv, l2, c2, hkeys.get(), hvals.get(), hub_cap);   \
  } while (0)
    if (wide) DCD_SCREEN(i128);
    else DCD_SCREEN(long long);
#undef DCD_SCREEN
    DCD_LAUNCH_CHECK();
  }
  DCD_TRY_CUDA(cudaMemsetAsync(&d->r_size, 0, sizeof(int64_t), s));
  ::dcd::count_launch(), build_rset<<<grid_for(n, T), T, 0, s>>>(n, mark.get(), cflag.get(), labels0, rset,
                                           (unsigned long long*)&d->r_size);
  DCD_LAUNCH_CHECK();
  return DCD_OK;
}

}  // namespace dcd
