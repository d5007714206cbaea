// merge.cu -- Delta_t into G_t: batch records, radix sort by (source, sink),
// distinct pairs, and a row-parallel sort-merge of the CSR that also produces
// the weighted degrees d_w (Sec. III-A), 2m and sum_i e_{i->C(i)} under the
// inherited labels.
//
// The changes are stored as ordered pairs (i,j) and (j,i) (Sec. III-E).  The
// paper only adds edges; the reading for deletions is: every delete of the
// step acts first and removes the whole edge, then every insert adds its
// weight (a new edge or a larger multiplicity).
#include "prims.cuh"
#include "state.cuh"

namespace dcd {

namespace {

constexpr uint8_t kPairIns = 1, kPairDel = 2, kPairPresent = 4, kPairAdded = 8, kPairRemoved = 16;

__global__ void validate_records(const dcd_edge* __restrict__ ins, int64_t n_ins,
                                 const dcd_edge* __restrict__ del, int64_t n_del, int64_t n,
                                 uint32_t* __restrict__ err) {
  int64_t tot = n_ins + n_del;
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    dcd_edge e = i < n_ins ? ins[i] : del[i - n_ins];
    bad |= e.u < 0 || e.v < 0 || e.u >= n || e.v >= n || e.u == e.v || (i < n_ins && e.w <= 0);
  }
  if (__any_sync(0xffffffffu, bad) && lane_id() == 0) atomicOr(err, kErrBadRecord);
}

// Record r: inserts first (2i, 2i+1 = both orientations of insert i), then
// deletes.  key = source << 32 | sink, value = r.
__global__ void make_records(const dcd_edge* __restrict__ ins, int64_t n_ins, const dcd_edge* __restrict__ del,
                             int64_t n_del, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  int64_t tot = n_ins + n_del;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    dcd_edge e = i < n_ins ? ins[i] : del[i - n_ins];
    uint64_t a = (uint64_t)(uint32_t)e.u, b = (uint64_t)(uint32_t)e.v;
    keys[2 * i] = a << 32 | b;
    keys[2 * i + 1] = b << 32 | a;
    vals[2 * i] = (uint32_t)(2 * i);
    vals[2 * i + 1] = (uint32_t)(2 * i + 1);
  }
}

// Records sorted by source with a counting sort, then each source's segment
// by sink with a rank sort (a record's place = the records of its segment
// with a smaller key, or an equal key and a smaller index).  Used when no
// source holds more than kRankSortMax records (the rank sort costs the square
// of a segment); otherwise the batch takes the LSD radix sort.
constexpr int64_t kRankSortMax = 4096;

__global__ void rec_count(const dcd_edge* __restrict__ ins, int64_t n_ins, const dcd_edge* __restrict__ del,
                          int64_t n_del, int32_t* __restrict__ cnt) {
  const int64_t tot = n_ins + n_del;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    const dcd_edge e = i < n_ins ? ins[i] : del[i - n_ins];
    atomicAdd(&cnt[e.u], 1);
    atomicAdd(&cnt[e.v], 1);
  }
}

__global__ void rec_maxseg(const int32_t* __restrict__ cnt, int64_t n, int32_t* __restrict__ mx) {
  int32_t m = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    m = cnt[v] > m ? cnt[v] : m;
  m = (int32_t)__reduce_max_sync(0xffffffffu, (unsigned)m);
  if (lane_id() == 0 && m) atomicMax(mx, m);
}

__global__ void rec_scatter(const dcd_edge* __restrict__ ins, int64_t n_ins, const dcd_edge* __restrict__ del,
                            int64_t n_del, const int32_t* __restrict__ off, int32_t* __restrict__ cur,
                            uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t tot = n_ins + n_del;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    const dcd_edge e = i < n_ins ? ins[i] : del[i - n_ins];
    const uint64_t a = (uint64_t)(uint32_t)e.u, b = (uint64_t)(uint32_t)e.v;
    const int32_t pa = off[e.u] + atomicAdd(&cur[e.u], 1);
    keys[pa] = a << 32 | b;
    vals[pa] = (uint32_t)(2 * i);
    const int32_t pb = off[e.v] + atomicAdd(&cur[e.v], 1);
    keys[pb] = b << 32 | a;
    vals[pb] = (uint32_t)(2 * i + 1);
  }
}

// Segments longer than kRankSmall are sorted by rec_bitonic instead (a CTA
// each, a bitonic network in shared memory).
constexpr int kRankSmall = 64;

__global__ void rec_rank(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin, int64_t R,
                         const int32_t* __restrict__ off, uint64_t* __restrict__ kout, uint32_t* __restrict__ vout) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < R; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = kin[i];
    const int32_t src = (int32_t)(k >> 32);
    const int64_t a = off[src], b = off[src + 1];
    if (b - a > kRankSmall) continue;
    int64_t r = 0;
    for (int64_t j = a; j < b; j++) {
      const uint64_t kj = kin[j];
      r += (kj < k || (kj == k && j < i)) ? 1 : 0;
    }
    kout[a + r] = k;
    vout[a + r] = vin[i];
  }
}

// sources whose segment is longer than kRankSmall
__global__ void rec_big_list(const int32_t* __restrict__ off, int64_t n, int32_t* __restrict__ list,
                             int32_t* __restrict__ cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x) + (threadIdx.x & ~31); base < n; base += stride) {
    const int64_t v = base + lane_id();
    const bool big = v < n && off[v + 1] - off[v] > kRankSmall;
    const unsigned bal = __ballot_sync(0xffffffffu, big);
    if (!bal) continue;
    int32_t slot = 0;
    if (lane_id() == 0) slot = atomicAdd(cnt, __popc(bal));
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (big) list[slot + __popc(bal & lanemask_lt())] = (int32_t)v;
  }
}

// One CTA per long segment (at most kRankSortMax records): a bitonic sort in
// shared memory, padded to a power of two with the largest key.
__global__ void __launch_bounds__(1024) rec_bitonic(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                    const int32_t* __restrict__ off, const int32_t* __restrict__ list,
                                                    const int32_t* __restrict__ cnt, uint64_t* __restrict__ kout,
                                                    uint32_t* __restrict__ vout) {
  __shared__ uint64_t sk[kRankSortMax];
  __shared__ uint32_t sv[kRankSortMax];
  const int64_t nl = *cnt;
  for (int64_t i = blockIdx.x; i < nl; i += gridDim.x) {
    const int32_t v = list[i];
    const int64_t a = off[v];
    const int len = (int)(off[v + 1] - a);
    int P = 1;
    while (P < len) P <<= 1;
    for (int x = threadIdx.x; x < P; x += blockDim.x) {
      sk[x] = x < len ? kin[a + x] : ~0ull;
      sv[x] = x < len ? vin[a + x] : 0u;
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int x = threadIdx.x; x < P; x += blockDim.x) {
          const int y = x ^ j;
          if (y > x) {
            const bool up = (x & k) == 0;
            const uint64_t kx = sk[x], ky = sk[y];
            if ((kx > ky) == up) {
              sk[x] = ky;
              sk[y] = kx;
              const uint32_t t = sv[x];
              sv[x] = sv[y];
              sv[y] = t;
            }
          }
        }
        __syncthreads();
      }
    for (int x = threadIdx.x; x < len; x += blockDim.x) {
      kout[a + x] = sk[x];
      vout[a + x] = sv[x];
    }
    __syncthreads();
  }
}

__global__ void run_heads(const uint64_t* __restrict__ keys, int64_t R, int32_t* __restrict__ head) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < R; e += (int64_t)gridDim.x * blockDim.x)
    head[e] = (e == 0 || keys[e] != keys[e - 1]) ? 1 : 0;
}

// One thread per run of equal keys: sum of insert weights, delete flag.
__global__ void reduce_pairs(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t R,
                             const int32_t* __restrict__ head, const int32_t* __restrict__ pid,
                             const dcd_edge* __restrict__ ins, int64_t n_ins, uint64_t* __restrict__ pkey,
                             int64_t* __restrict__ pw, uint8_t* __restrict__ pflag) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < R; e += (int64_t)gridDim.x * blockDim.x) {
    if (!head[e]) continue;
    uint64_t k = keys[e];
    int64_t W = 0;
    uint8_t f = 0;
    for (int64_t x = e; x < R && keys[x] == k; x++) {
      uint32_t r = vals[x];
      if ((int64_t)r < 2 * n_ins) {
        W += ins[r >> 1].w;
        f |= kPairIns;
      } else {
        f |= kPairDel;
      }
    }
    int32_t p = pid[e];
    pkey[p] = k;
    pw[p] = W;
    pflag[p] = f;
  }
}

__device__ __forceinline__ int64_t lower_bound_i32(const int32_t* __restrict__ a, int64_t lo, int64_t hi, int32_t x) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t* __restrict__ a, int64_t lo, int64_t hi, uint64_t x) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Per pair: was the edge in G_{t-1}; does the merge add or remove a row entry.
// With lab0 (C_{t-1}) given, also the change the pair makes to
// sum_i e_{i->C(i)} under C_{t-1}: its new weight minus its old one when both
// ends share a community, added into in_delta[graph].
__global__ void pair_status(const uint64_t* __restrict__ pkey, const int64_t* __restrict__ pw,
                            uint8_t* __restrict__ pflag, int64_t P, const int64_t* __restrict__ rp,
                            const int32_t* __restrict__ col, const int32_t* __restrict__ w,
                            int32_t* __restrict__ added, int32_t* __restrict__ removed,
                            int64_t* __restrict__ src_cnt, uint32_t* __restrict__ err,
                            const int32_t* __restrict__ lab0, const int32_t* __restrict__ gid,
                            int64_t* __restrict__ in_delta) {
  // warp-uniform trip count: the lanes of a warp sum their in_delta changes
  // per graph before one lane adds them (most pairs of a step add into the
  // same word)
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31u); p0 < P; p0 += stride) {
    const int64_t p = p0 + lane_id();
    int64_t dlt = 0;
    int32_t graph = 0, src = -1;
    if (p < P) {
      uint64_t k = pkey[p];
      int32_t u = (int32_t)(k >> 32), v = (int32_t)(k & 0xffffffffu);
      int64_t b = rp[u], e = rp[u + 1];
      int64_t pos = lower_bound_i32(col, b, e, v);
      bool present = pos < e && col[pos] == v;
      uint8_t f = pflag[p];
      bool isins = f & kPairIns, isdel = f & kPairDel;
      bool add = isins && !present;
      bool rem = !isins && isdel && present;
      if (isins) {
        int64_t nw = (present && !isdel) ? (int64_t)w[pos] + pw[p] : pw[p];
        if (nw > INT32_MAX) atomicOr(err, kErrOverflow);
      }
      if (lab0 && lab0[u] == lab0[v]) {
        // deletes remove the whole edge first, then inserts add their weight
        const int64_t w_old = present ? (int64_t)w[pos] : 0;
        const int64_t w_new = ((present && !isdel) ? w_old : 0) + (isins ? pw[p] : 0);
        dlt = w_new - w_old;
        graph = graph_of(gid, u);
      }
      f |= (present ? kPairPresent : 0) | (add ? kPairAdded : 0) | (rem ? kPairRemoved : 0);
      pflag[p] = f;
      added[p] = add;
      removed[p] = rem;
      src = u;
    }
    {
      // pairs are sorted by source: one add per run of equal sources
      const unsigned same = __match_any_sync(0xffffffffu, src);
      if (src >= 0 && (int)(__ffs(same) - 1) == (int)lane_id())
        atomicAdd((unsigned long long*)&src_cnt[src], (unsigned long long)__popc(same));
    }
    if (lab0) {
      const unsigned peers = __match_any_sync(0xffffffffu, graph);
      // two's-complement sum of the peers' changes, 16 bits at a time
      const unsigned long long x = (unsigned long long)dlt;
      unsigned long long sum = 0;
#pragma unroll
      for (int q = 0; q < 4; q++)
        sum += (unsigned long long)__reduce_add_sync(peers, (unsigned)(x >> (16 * q)) & 0xffffu) << (16 * q);
      if (sum != 0 && (int)(__ffs(peers) - 1) == (int)lane_id())
        atomicAdd((unsigned long long*)&in_delta[graph], sum);
    }
  }
}

// sum_i e_{i->C(i)} under C_{t-1} on G_t from its value on G_{t-1} (kept by
// the previous update) and the batch's change.
__global__ void seed_in(GraphState* __restrict__ gs, int G, const int64_t* __restrict__ in_prev,
                        const int64_t* __restrict__ in_delta) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x)
    gs[g].in_cur += in_prev[g] + in_delta[g];
}

// Rows longer than kLongRow entries (old or new) are merged by a CTA each
// (merge_long) instead of by G lanes: a hub row would otherwise hold its
// group for thousands of iterations and set the kernel's length.
constexpr int64_t kLongRow = 512;

__global__ void new_degrees(const int64_t* __restrict__ rp, const int64_t* __restrict__ pair_ptr,
                            const int32_t* __restrict__ pA, const int32_t* __restrict__ pR, int64_t n,
                            int64_t* __restrict__ deg, int32_t* __restrict__ long_rows,
                            int32_t* __restrict__ long_cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x) + (threadIdx.x & ~31); base < n; base += stride) {
    const int64_t u = base + lane_id();
    bool lng = false;
    if (u < n) {
      const int64_t p0 = pair_ptr[u], p1 = pair_ptr[u + 1];
      const int64_t od = rp[u + 1] - rp[u];
      const int64_t nd = od + (pA[p1] - pA[p0]) - (pR[p1] - pR[p0]);
      deg[u] = nd;
      lng = od > kLongRow || nd > kLongRow;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, lng);
    if (bal) {
      int32_t slot = 0;
      if (lane_id() == 0) slot = atomicAdd(long_cnt, __popc(bal));
      slot = __shfl_sync(0xffffffffu, slot, 0);
      if (lng) long_rows[slot + __popc(bal & lanemask_lt())] = (int32_t)u;
    }
  }
}

// One CTA per long row (the list from new_degrees): the row's pairs are staged
// in shared memory when they fit, the entries are placed as in merge_rows, and
// k_u, 2m and sum_i e_{i->C(i)} are reduced over the CTA.
constexpr int kLongPairs = 1024;

template <int THREADS>
__global__ void __launch_bounds__(THREADS) merge_long(
    const int32_t* __restrict__ long_rows, const int32_t* __restrict__ long_cnt, const int64_t* __restrict__ rp_o,
    const int32_t* __restrict__ col_o, const int32_t* __restrict__ w_o, const int64_t* __restrict__ rp_n,
    int32_t* __restrict__ col_n, int32_t* __restrict__ w_n, const int64_t* __restrict__ pair_ptr,
    const uint64_t* __restrict__ pkey, const int64_t* __restrict__ pw, const uint8_t* __restrict__ pflag,
    const int32_t* __restrict__ pA, const int32_t* __restrict__ pR, const int32_t* __restrict__ lab,
    int64_t* __restrict__ kdeg, const int32_t* __restrict__ gid, GraphState* __restrict__ gs) {
  __shared__ int32_t s_pc[kLongPairs];
  __shared__ int32_t s_pa[kLongPairs + 1], s_pr[kLongPairs + 1];
  __shared__ long long red_k[THREADS / 32], red_i[THREADS / 32];
  const int tid = threadIdx.x, lane = lane_id(), wid = tid >> 5;
  const int64_t cnt = *long_cnt;
  for (int64_t i = blockIdx.x; i < cnt; i += gridDim.x) {
    const int32_t u = long_rows[i];
    const int64_t ob = rp_o[u], oe = rp_o[u + 1], nb = rp_n[u];
    const int64_t p0 = pair_ptr[u], p1 = pair_ptr[u + 1];
    const int64_t np = p1 - p0;
    const int32_t Lu = lab ? lab[u] : 0;
    const int32_t rA0 = pA[p0], rR0 = pR[p0];  // prefix arrays hold P + 1 entries
    const bool staged = np <= kLongPairs;
    if (staged) {
      for (int64_t q = tid; q <= np; q += THREADS) {
        s_pa[q] = pA[p0 + q] - rA0;
        s_pr[q] = pR[p0 + q] - rR0;
        if (q < np) s_pc[q] = (int32_t)(pkey[p0 + q] & 0xffffffffu);
      }
    }
    __syncthreads();
    int64_t ks = 0, is = 0;
    const uint64_t hi = (uint64_t)(uint32_t)u << 32;
    for (int64_t e = ob + tid; e < oe; e += THREADS) {
      const int32_t c = col_o[e];
      int64_t q;
      bool match;
      int32_t aq, rq;
      if (staged) {
        int64_t lo = 0, hi2 = np;
        while (lo < hi2) {
          const int64_t mid = (lo + hi2) >> 1;
          if (s_pc[mid] < c) lo = mid + 1; else hi2 = mid;
        }
        q = p0 + lo;
        match = lo < np && s_pc[lo] == c;
        aq = s_pa[lo];
        rq = s_pr[lo];
      } else {
        q = lower_bound_u64(pkey, p0, p1, hi | (uint32_t)c);
        match = q < p1 && pkey[q] == (hi | (uint32_t)c);
        aq = pA[q] - rA0;
        rq = pR[q] - rR0;
      }
      const uint8_t f = match ? pflag[q] : 0;
      if (f & kPairRemoved) continue;
      int64_t wv = w_o[e];
      if (match && (f & kPairIns)) wv = (f & kPairDel) ? pw[q] : wv + pw[q];
      const int64_t pos = nb + (e - ob) - rq + aq;
      col_n[pos] = c;
      w_n[pos] = (int32_t)wv;
      ks += wv;
      if (lab && lab[c] == Lu) is += wv;
    }
    for (int64_t q = p0 + tid; q < p1; q += THREADS) {
      if (!(pflag[q] & kPairAdded)) continue;
      const int32_t c = (int32_t)(pkey[q] & 0xffffffffu);
      const int64_t o = lower_bound_i32(col_o, ob, oe, c) - ob;
      const int64_t pos = nb + o - (pR[q] - rR0) + (pA[q] - rA0);
      const int64_t wv = pw[q];
      col_n[pos] = c;
      w_n[pos] = (int32_t)wv;
      ks += wv;
      if (lab && lab[c] == Lu) is += wv;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ks += __shfl_xor_sync(0xffffffffu, ks, o);
      is += __shfl_xor_sync(0xffffffffu, is, o);
    }
    if (lane == 0) {
      red_k[wid] = ks;
      red_i[wid] = is;
    }
    __syncthreads();
    if (tid == 0) {
      long long tk = 0, ti = 0;
      for (int x = 0; x < THREADS / 32; x++) {
        tk += red_k[x];
        ti += red_i[x];
      }
      kdeg[u] = tk;
      const int gu = graph_of(gid, u);
      atomicAdd((unsigned long long*)&gs[gu].m2, (unsigned long long)tk);
      atomicAdd((unsigned long long*)&gs[gu].in_cur, (unsigned long long)ti);
    }
    __syncthreads();
  }
}

template <int G>
__device__ __forceinline__ int64_t group_sum(int64_t x) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o, G);
  return x;
}

// G lanes per row.  An untouched row is copied; a touched row is merged with
// its pairs: an old entry lands at its old offset minus the removed pairs and
// plus the added pairs that sort before it; an added pair lands after the old
// entries below it, corrected the same way.
template <int G>
__global__ void __launch_bounds__(256, 5) merge_rows(
    int64_t n, const int64_t* __restrict__ rp_o, const int32_t* __restrict__ col_o, const int32_t* __restrict__ w_o,
    const int64_t* __restrict__ rp_n, int32_t* __restrict__ col_n, int32_t* __restrict__ w_n,
    const int64_t* __restrict__ pair_ptr, const uint64_t* __restrict__ pkey, const int64_t* __restrict__ pw,
    const uint8_t* __restrict__ pflag, const int32_t* __restrict__ pA, const int32_t* __restrict__ pR,
    const int32_t* __restrict__ lab, int64_t* __restrict__ kdeg, const int32_t* __restrict__ gid,
    GraphState* __restrict__ gs) {
  const int g = threadIdx.x % G;
  // warp-uniform loop: every lane reaches the group shuffles
  const int64_t gid0 = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * (32 / G);
  const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / G;
  // 2m and sum_i e_{i->C(i)} per graph: accumulated while consecutive rows of
  // a group stay in one graph, flushed by the group leader when it changes
  int64_t m2_loc = 0, in_loc = 0;
  int cur_g = -1;
  for (int64_t ubase = gid0; ubase < n; ubase += ngroups) {
    const int64_t u = ubase + (int64_t)(lane_id() / G);
    int64_t ks = 0, is = 0;
    const bool lng = u < n && (rp_o[u + 1] - rp_o[u] > kLongRow || rp_n[u + 1] - rp_n[u] > kLongRow);
    if (u >= n || lng) {
      // idle group in the warp's last round, or a long row (merge_long)
    } else if (pair_ptr[u] == pair_ptr[u + 1]) {
      int64_t ob = rp_o[u], oe = rp_o[u + 1], nb = rp_n[u];
      int32_t Lu = lab ? lab[u] : 0;
      for (int64_t e = ob + g; e < oe; e += G) {
        int32_t c = col_o[e];
        int32_t wv = w_o[e];
        col_n[nb + (e - ob)] = c;
        w_n[nb + (e - ob)] = wv;
        ks += wv;
        if (lab && lab[c] == Lu) is += wv;
      }
    } else if (pair_ptr[u + 1] - pair_ptr[u] < G) {
      // few pairs: the group's lanes hold them (lane q: pair p0 + q, and the
      // prefix counts up to it), so an entry finds its place among them with
      // shuffles instead of a binary search in global memory
      const int64_t ob = rp_o[u], oe = rp_o[u + 1], nb = rp_n[u];
      const int64_t p0 = pair_ptr[u];
      const int np = (int)(pair_ptr[u + 1] - p0);
      const int32_t Lu = lab ? lab[u] : 0;
      const int32_t rA0 = pA[p0], rR0 = pR[p0];
      const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane_id() & ~(G - 1)));
      int32_t pc = INT_MAX, pa = 0, pr = 0;
      uint32_t pf = 0;
      long long pwv = 0;
      if (g <= np) {
        pa = pA[p0 + g] - rA0;
        pr = pR[p0 + g] - rR0;
        if (g < np) {
          pc = (int32_t)(pkey[p0 + g] & 0xffffffffu);
          pf = pflag[p0 + g];
          pwv = pw[p0 + g];
        }
      }
      for (int64_t e0 = ob; e0 < oe; e0 += G) {
        const int64_t e = e0 + g;
        const bool valid = e < oe;
        const int32_t c = valid ? col_o[e] : INT_MAX;
        // pairs of the row with a smaller column: the lanes hold the pair
        // columns in ascending order (INT_MAX past the last), so a branch-free
        // binary search over the G lanes counts them
        int q = 0;
#pragma unroll
        for (int stp = G / 2; stp > 0; stp >>= 1)
          if (__shfl_sync(gmask, pc, q + stp - 1, G) < c) q += stp;
        const int32_t kq = __shfl_sync(gmask, pc, q, G);
        const uint32_t fq = __shfl_sync(gmask, pf, q, G);
        const long long wq = __shfl_sync(gmask, pwv, q, G);
        const int32_t aq = __shfl_sync(gmask, pa, q, G), rq = __shfl_sync(gmask, pr, q, G);
        const bool match = valid && kq == c;
        const uint32_t f = match ? fq : 0u;
        if (!valid || (f & kPairRemoved)) continue;
        int64_t wv = w_o[e];
        if (match && (f & kPairIns)) wv = (f & kPairDel) ? (int64_t)wq : wv + (int64_t)wq;
        const int64_t pos = nb + (e - ob) - rq + aq;
        col_n[pos] = c;
        w_n[pos] = (int32_t)wv;
        ks += wv;
        if (lab && lab[c] == Lu) is += wv;
      }
      for (int64_t q = p0 + g; q < p0 + np; q += G) {
        if (!(pflag[q] & kPairAdded)) continue;
        const int32_t c = (int32_t)(pkey[q] & 0xffffffffu);
        const int64_t o = lower_bound_i32(col_o, ob, oe, c) - ob;
        const int64_t pos = nb + o - (pR[q] - rR0) + (pA[q] - rA0);
        const int64_t wv = pw[q];
        col_n[pos] = c;
        w_n[pos] = (int32_t)wv;
        ks += wv;
        if (lab && lab[c] == Lu) is += wv;
      }
    } else {
      int64_t ob = rp_o[u], oe = rp_o[u + 1], nb = rp_n[u];
      int64_t p0 = pair_ptr[u], p1 = pair_ptr[u + 1];
      int32_t Lu = lab ? lab[u] : 0;
      int32_t rA0 = pA[p0], rR0 = pR[p0];
      uint64_t hi = (uint64_t)(uint32_t)u << 32;
      for (int64_t e = ob + g; e < oe; e += G) {
        int32_t c = col_o[e];
        int64_t q = lower_bound_u64(pkey, p0, p1, hi | (uint32_t)c);
        bool match = q < p1 && pkey[q] == (hi | (uint32_t)c);
        uint8_t f = match ? pflag[q] : 0;
        if (f & kPairRemoved) continue;
        int64_t wv = w_o[e];
        if (match && (f & kPairIns)) wv = (f & kPairDel) ? pw[q] : wv + pw[q];
        int64_t pos = nb + (e - ob) - (pR[q] - rR0) + (pA[q] - rA0);
        col_n[pos] = c;
        w_n[pos] = (int32_t)wv;
        ks += wv;
        if (lab && lab[c] == Lu) is += wv;
      }
      for (int64_t q = p0 + g; q < p1; q += G) {
        if (!(pflag[q] & kPairAdded)) continue;
        int32_t c = (int32_t)(pkey[q] & 0xffffffffu);
        int64_t o = lower_bound_i32(col_o, ob, oe, c) - ob;
        int64_t pos = nb + o - (pR[q] - rR0) + (pA[q] - rA0);
        int64_t wv = pw[q];
        col_n[pos] = c;
        w_n[pos] = (int32_t)wv;
        ks += wv;
        if (lab && lab[c] == Lu) is += wv;
      }
    }
    ks = group_sum<G>(ks);
    is = group_sum<G>(is);
    if (g == 0 && u < n && !lng) {
      kdeg[u] = ks;
      const int gu = graph_of(gid, u);
      if (gu != cur_g) {
        if (cur_g >= 0 && (m2_loc | in_loc)) {
          atomicAdd((unsigned long long*)&gs[cur_g].m2, (unsigned long long)m2_loc);
          atomicAdd((unsigned long long*)&gs[cur_g].in_cur, (unsigned long long)in_loc);
        }
        cur_g = gu;
        m2_loc = in_loc = 0;
      }
      m2_loc += ks;
      in_loc += is;
    }
  }
  if (g == 0 && cur_g >= 0 && (m2_loc | in_loc)) {
    atomicAdd((unsigned long long*)&gs[cur_g].m2, (unsigned long long)m2_loc);
    atomicAdd((unsigned long long*)&gs[cur_g].in_cur, (unsigned long long)in_loc);
  }
}

}  // namespace

int validate_batch(dcd_ctx* c, const dcd_edge* ins, int64_t n_ins, const dcd_edge* del, int64_t n_del, bool* ok) {
  cudaStream_t s = c->stream;
  uint32_t* err = &c->dsc.get()->err;
  *ok = true;
  if (n_ins + n_del == 0) return DCD_OK;
  DCD_TRY_CUDA(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
  ::dcd::count_launch(), validate_records<<<grid_for(n_ins + n_del, 256), 256, 0, s>>>(ins, n_ins, del, n_del, c->n,
                                                                                       err);
  DCD_LAUNCH_CHECK();
  DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  DCD_TRY_CUDA(cudaStreamSynchronize(s));
  *ok = !(*reinterpret_cast<uint32_t*>(c->hscratch) & kErrBadRecord);
  return DCD_OK;
}

int merge_batch(dcd_ctx* c, const int32_t* labels0, bool static_start, MergeOut* out) {
  cudaStream_t s = c->stream;
  const int64_t n = c->n;
  const int64_t n_ins = c->n_ins, n_del = c->n_del;
  const int64_t R = 2 * (n_ins + n_del);
  DevScalars* d = c->dsc.get();
  uint32_t* err = &d->err;
  const int T = 256;

  if (c->staged_on_device && n_ins + n_del > 0) {
    // device-staged records are checked before any kernel indexes with them
    ::dcd::count_launch(), validate_records<<<grid_for(n_ins + n_del, T), T, 0, s>>>(c->ins.get(), n_ins, c->del.get(), n_del, n, err);
    DCD_LAUNCH_CHECK();
    DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    DCD_TRY_CUDA(cudaStreamSynchronize(s));
    if (*reinterpret_cast<uint32_t*>(c->hscratch) & kErrBadRecord) return DCD_EINVAL;
  }

  trace("merge: validated");
  // ---- records sorted by (source, sink) ----
  Buf<uint64_t> k0, k1;
  Buf<uint32_t> v0, v1;
  Buf<int32_t> head, pid;
  Buf<uint32_t> stmp;
  DCD_TRY(k0.alloc(&c->mem, R));
  DCD_TRY(k1.alloc(&c->mem, R));
  DCD_TRY(v0.alloc(&c->mem, R));
  DCD_TRY(v1.alloc(&c->mem, R));
  DCD_TRY(head.alloc(&c->mem, R + 1));
  DCD_TRY(pid.alloc(&c->mem, R + 1));
  int64_t scan_words = sort_tmp_words(R) + scan_tmp_count(n + 1) * 2 + scan_tmp_count(R + 1) * 2 + 64;
  DCD_TRY(stmp.alloc(&c->mem, scan_words));
  int64_t* stmp64 = reinterpret_cast<int64_t*>(stmp.get());

  uint64_t* keys = k0.get();
  uint32_t* vals = v0.get();
  int64_t P = 0;
  if (R > 0) {
    // counting sort by source: per-source counts, offsets, the longest segment
    Buf<int32_t> cnt, cur;
    DCD_TRY(cnt.alloc(&c->mem, n + 1));
    DCD_TRY(cur.alloc(&c->mem, n + 1));
    DCD_TRY_CUDA(cudaMemsetAsync(cnt.get(), 0, (n + 1) * sizeof(int32_t), s));
    DCD_TRY_CUDA(cudaMemsetAsync(cur.get(), 0, (n + 1) * sizeof(int32_t), s));
    ::dcd::count_launch(), rec_count<<<grid_for(R / 2, T), T, 0, s>>>(c->ins.get(), n_ins, c->del.get(), n_del,
                                                                       cnt.get());
    ::dcd::count_launch(), rec_maxseg<<<grid_for(n, T), T, 0, s>>>(cnt.get(), n, cur.get() + n);
    DCD_LAUNCH_CHECK();
    DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch, cur.get() + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    DCD_TRY(exclusive_scan<int32_t>(cnt.get(), cnt.get(), n + 1, nullptr, reinterpret_cast<int32_t*>(stmp.get()), s));
    DCD_TRY_CUDA(cudaStreamSynchronize(s));
    const int64_t maxseg = *reinterpret_cast<int32_t*>(c->hscratch);
    if (maxseg <= kRankSortMax && R < (int64_t)INT32_MAX) {
      DCD_TRY_CUDA(cudaMemsetAsync(cur.get() + n, 0, sizeof(int32_t), s));
      ::dcd::count_launch(), rec_scatter<<<grid_for(R / 2, T), T, 0, s>>>(c->ins.get(), n_ins, c->del.get(), n_del,
                                                                           cnt.get(), cur.get(), k1.get(), v1.get());
      ::dcd::count_launch(), rec_rank<<<grid_for(R, T), T, 0, s>>>(k1.get(), v1.get(), R, cnt.get(), k0.get(),
                                                                    v0.get());
      if (maxseg > kRankSmall) {
        Buf<int32_t> big;
        DCD_TRY(big.alloc(&c->mem, n));
        DCD_TRY_CUDA(cudaMemsetAsync(cur.get() + n, 0, sizeof(int32_t), s));
        ::dcd::count_launch(), rec_big_list<<<grid_for(n, T), T, 0, s>>>(cnt.get(), n, big.get(), cur.get() + n);
        ::dcd::count_launch(), rec_bitonic<<<2 * c->sms, 1024, 0, s>>>(k1.get(), v1.get(), cnt.get(), big.get(),
                                                                        cur.get() + n, k0.get(), v0.get());
      }
      DCD_LAUNCH_CHECK();
    } else {
      ::dcd::count_launch(), make_records<<<grid_for(R / 2, T), T, 0, s>>>(c->ins.get(), n_ins, c->del.get(), n_del,
                                                                          k0.get(), v0.get());
      DCD_LAUNCH_CHECK();
      int b = bits_for(n - 1);
      int ranges[4] = {0, b, 32, 32 + b};
      bool in1 = false;
      DCD_TRY(sort_pairs<uint32_t>(k0.get(), v0.get(), k1.get(), v1.get(), R, ranges, 2, stmp.get(), &in1, s));
      if (in1) {
        keys = k1.get();
        vals = v1.get();
      }
    }
    ::dcd::count_launch(), run_heads<<<grid_for(R, T), T, 0, s>>>(keys, R, head.get());
    DCD_TRY(exclusive_scan<int32_t>(head.get(), pid.get(), R, pid.get() + R, reinterpret_cast<int32_t*>(stmp.get()), s));
    DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch, pid.get() + R, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    DCD_TRY_CUDA(cudaStreamSynchronize(s));
    P = (int64_t)(*reinterpret_cast<int32_t*>(c->hscratch));
  }
  trace("merge: sorted + pairs counted");
  out->npairs = P;

  DCD_TRY(out->pkey.alloc(&c->mem, P));
  DCD_TRY(out->pw.alloc(&c->mem, P));
  DCD_TRY(out->pflag.alloc(&c->mem, P));
  DCD_TRY(out->pair_ptr.alloc(&c->mem, n + 1));
  Buf<int32_t> added, removed;
  DCD_TRY(added.alloc(&c->mem, P + 1));
  DCD_TRY(removed.alloc(&c->mem, P + 1));
  DCD_TRY_CUDA(cudaMemsetAsync(out->pair_ptr.get(), 0, (n + 1) * sizeof(int64_t), s));

  // sum_i e_{i->C(i)} under the start labels on G_t: zero for a static start
  // (singletons, no self-loops); from the previous update's value plus the
  // batch's change when the context kept it (in_valid); else summed over
  // every entry by the merge, which then gathers the label of each column
  const bool from_prev = !static_start && c->in_valid;
  const int32_t* lab_gather = (static_start || from_prev) ? nullptr : labels0;
  Buf<int64_t> in_delta;
  DCD_TRY(in_delta.alloc(&c->mem, c->G));
  DCD_TRY_CUDA(cudaMemsetAsync(in_delta.get(), 0, c->G * sizeof(int64_t), s));

  const int cur = c->cur, nxt = 1 - c->cur;
  const int64_t* rp_o = c->rp[cur].get();
  const int32_t* col_o = c->col[cur].get();
  const int32_t* w_o = c->w[cur].get();

  if (P > 0) {
    ::dcd::count_launch(), reduce_pairs<<<grid_for(R, T), T, 0, s>>>(keys, vals, R, head.get(), pid.get(), c->ins.get(), n_ins,
                                              out->pkey.get(), out->pw.get(), out->pflag.get());
    ::dcd::count_launch(), pair_status<<<grid_for(P, T), T, 0, s>>>(out->pkey.get(), out->pw.get(), out->pflag.get(), P, rp_o, col_o, w_o,
                                             added.get(), removed.get(), out->pair_ptr.get(), err,
                                             from_prev ? labels0 : nullptr, c->G > 1 ? c->gid.get() : nullptr,
                                             in_delta.get());
    DCD_LAUNCH_CHECK();
  }
  // pair_ptr: per-source counts -> exclusive scan (n + 1 entries)
  DCD_TRY(exclusive_scan<int64_t>(out->pair_ptr.get(), out->pair_ptr.get(), n + 1, nullptr, stmp64, s));
  DCD_TRY(exclusive_scan<int32_t>(added.get(), added.get(), P + 1, nullptr, reinterpret_cast<int32_t*>(stmp.get()), s));
  DCD_TRY(exclusive_scan<int32_t>(removed.get(), removed.get(), P + 1, nullptr,
                                  reinterpret_cast<int32_t*>(stmp.get()), s));

  // ---- new row pointers ----
  const int64_t cap = c->nnz + 2 * n_ins;
  DCD_TRY(c->rp[nxt].ensure(&c->mem, n + 1));
  DCD_TRY(c->col[nxt].ensure(&c->mem, cap));
  DCD_TRY(c->w[nxt].ensure(&c->mem, cap));
  int64_t* rp_n = c->rp[nxt].get();
  Buf<int32_t> long_rows, long_cnt;
  DCD_TRY(long_rows.alloc(&c->mem, n));
  DCD_TRY(long_cnt.alloc(&c->mem, 1));
  DCD_TRY_CUDA(cudaMemsetAsync(long_cnt.get(), 0, sizeof(int32_t), s));
  ::dcd::count_launch(), new_degrees<<<grid_for(n, T), T, 0, s>>>(rp_o, out->pair_ptr.get(), added.get(), removed.get(),
                                                                   n, rp_n, long_rows.get(), long_cnt.get());
  DCD_LAUNCH_CHECK();
  DCD_TRY(exclusive_scan<int64_t>(rp_n, rp_n, n + 1, nullptr, stmp64, s));

  // ---- merge rows, degrees, m2, in ----
  DCD_TRY(out->k.alloc(&c->mem, n));
  DCD_TRY_CUDA(cudaMemsetAsync(c->gs.get(), 0, c->G * sizeof(GraphState), s));
  const int64_t avg = (cap + n - 1) / n;
  const int64_t* pp = out->pair_ptr.get();
  // merge_rows skips the rows above kLongRow entries, which merge_long takes:
  // the two write disjoint rows (and add into 2m and sum e_{i->C(i)} with
  // atomics), so they run side by side
  SideBySide par(c, n);
  DCD_TRY(par.fork());
  cudaStream_t s_long;
  DCD_TRY(par.on(0, &s_long));
  ::dcd::count_launch(), merge_long<256><<<4 * c->sms, 256, 0, s_long>>>(
      long_rows.get(), long_cnt.get(), rp_o, col_o, w_o, rp_n, c->col[nxt].get(), c->w[nxt].get(), pp,
      out->pkey.get(), out->pw.get(), out->pflag.get(), added.get(), removed.get(), lab_gather, out->k.get(),
      c->G > 1 ? c->gid.get() : nullptr, c->gs.get());
#define DCD_MERGE(Gs)                                                                                       \
  ::dcd::count_launch(), merge_rows<Gs><<<wave_grid(merge_rows<Gs>, n * Gs, T), T, 0, s>>>(n, rp_o, col_o, w_o, rp_n, c->col[nxt].get(),            \
                                                   c->w[nxt].get(), pp, out->pkey.get(), out->pw.get(),     \
                                                   out->pflag.get(), added.get(), removed.get(), lab_gather, \
                                                   out->k.get(), c->G > 1 ? c->gid.get() : nullptr,         \
                                                   c->gs.get())
  if (avg <= 6) DCD_MERGE(4);
  else if (avg <= 12) DCD_MERGE(8);
  else if (avg <= 24) DCD_MERGE(16);
  else DCD_MERGE(32);
#undef DCD_MERGE
  DCD_LAUNCH_CHECK();
  DCD_TRY(par.join());
  if (from_prev) {
    ::dcd::count_launch(), seed_in<<<cdiv(c->G, 128), 128, 0, s>>>(c->gs.get(), c->G, c->in_prev.get(),
                                                                    in_delta.get());
    DCD_LAUNCH_CHECK();
  }
  return DCD_OK;
}

}  // namespace dcd
