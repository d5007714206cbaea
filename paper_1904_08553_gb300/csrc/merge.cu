// merge.cu -- Delta_t into G_t: batch records, radix sort by (source, sink),
// distinct pairs, and a tiled merge of the CSR with the pairs that also produces
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
                            int64_t* __restrict__ in_delta, int64_t* __restrict__ pdelta) {
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
      // deletes remove the whole edge first, then inserts add their weight
      const int64_t w_old = present ? (int64_t)w[pos] : 0;
      const int64_t w_new = ((present && !isdel) ? w_old : 0) + (isins ? pw[p] : 0);
      pdelta[p] = w_new - w_old;
      if (lab0 && lab0[u] == lab0[v]) {
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

// ---- tiled merge ----
//
// The merge as one merge of two sorted sequences: the old entries (key =
// source << 32 | sink, in CSR order) and the pairs (same keys), an entry
// before a pair of equal key.  With A(q), R(q) the added and removed pairs
// among the first q, an old entry e lands at e + A(q) - R(q) (q: pairs of
// smaller key) and an added pair q at i + A(q) - R(q) (i: old entries of
// smaller key), so rows need not be merged one by one: the merged sequence is
// cut into tiles of kMergeTile items, a CTA each, whatever rows they cover.
constexpr int kMergeTile = 2048;
constexpr int kMergeThreads = 256;
constexpr int kMergeRows = 1024;  // row starts staged per tile (more: searched in global memory)

// Row u's start in the new CSR: rp_o[u] + A(pair_ptr[u]) - R(pair_ptr[u]).
__global__ void new_rows(const int64_t* __restrict__ rp_o, const int64_t* __restrict__ pair_ptr,
                         const int32_t* __restrict__ pA, const int32_t* __restrict__ pR, int64_t n,
                         int64_t* __restrict__ rp_n) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u <= n; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = pair_ptr[u];
    rp_n[u] = rp_o[u] + pA[p] - pR[p];
  }
}

// Tile t starts at merged item d = t * kMergeTile: se[t] old entries and sq[t]
// pairs come before it, su[t] is the row of item d.  Rows are found on
// W(u) = rp_o[u] + pair_ptr[u] (the merged items of rows before u), then
// the split inside the row by a merge-path search over its sinks.
__global__ void merge_split(int64_t n, const int64_t* __restrict__ rp_o, const int32_t* __restrict__ col_o,
                            const int64_t* __restrict__ pp, const uint64_t* __restrict__ pkey, int64_t nt,
                            int64_t total, int64_t* __restrict__ se, int64_t* __restrict__ sq,
                            int64_t* __restrict__ su) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t <= nt; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t dd = t * kMergeTile < total ? t * kMergeTile : total;
    if (dd == total) {
      se[t] = rp_o[n];
      sq[t] = pp[n];
      su[t] = n > 0 ? n - 1 : 0;
      continue;
    }
    int64_t lo = 0, hi = n - 1;  // last row with W(u) <= dd
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (rp_o[mid] + pp[mid] <= dd) lo = mid; else hi = mid - 1;
    }
    const int64_t u = lo;
    const int64_t ob = rp_o[u], deg = rp_o[u + 1] - ob, p0 = pp[u], np = pp[u + 1] - p0;
    const int64_t r = dd - ob - p0;  // items of row u before dd: i entries, r - i pairs
    int64_t a = r - np > 0 ? r - np : 0, b = r < deg ? r : deg;
    while (a < b) {
      const int64_t mid = (a + b) >> 1;
      if (col_o[ob + mid] <= (int32_t)(pkey[p0 + r - 1 - mid] & 0xffffffffu)) a = mid + 1; else b = mid;
    }
    se[t] = ob + a;
    sq[t] = p0 + r - a;
    su[t] = u;
  }
}

__device__ __forceinline__ int lower_bound_smem(const uint64_t* a, int n, uint64_t x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Adds a row's share of the weights into kdeg: lanes of one row sum with
// redux (exact from 16-bit slices) and the lowest adds.
__device__ __forceinline__ void add_row_weight(int64_t* kdeg, int64_t u, int64_t wv) {
  const unsigned peers = __match_any_sync(0xffffffffu, u);
  const unsigned lo = (unsigned)wv & 0xffffu, hi = (unsigned)(wv >> 16);
  const unsigned long long sum =
      (unsigned long long)__reduce_add_sync(peers, lo) + ((unsigned long long)__reduce_add_sync(peers, hi) << 16);
  if (u >= 0 && sum != 0 && (int)(__ffs(peers) - 1) == (int)lane_id())
    atomicAdd((unsigned long long*)&kdeg[u], sum);
}

// One tile of the merge.  Weights written are int32 (checked by pair_status),
// so a lane's weight is below 2^31 and the slice sums above are exact.
__global__ void __launch_bounds__(kMergeThreads) merge_tile(
    int64_t n, const int64_t* __restrict__ rp_o, const int32_t* __restrict__ col_o,
    const int32_t* __restrict__ w_o, const int64_t* __restrict__ se, const int64_t* __restrict__ sq,
    const int64_t* __restrict__ su, const uint64_t* __restrict__ pkey, const int64_t* __restrict__ pw,
    const uint8_t* __restrict__ pflag, const int32_t* __restrict__ pA, const int32_t* __restrict__ pR, int64_t P,
    int32_t* __restrict__ col_n, int32_t* __restrict__ w_n, const int32_t* __restrict__ lab,
    int64_t* __restrict__ kdeg, const int32_t* __restrict__ gid, GraphState* __restrict__ gs) {
  __shared__ uint64_t s_pk[kMergeTile];
  __shared__ uint64_t s_ek[kMergeTile];
  __shared__ int64_t s_rp[kMergeRows + 1];
  __shared__ unsigned long long s_red[2][kMergeThreads / 32];
  __shared__ int s_uni;
  const int tid = threadIdx.x;
  const int64_t t = blockIdx.x;
  const int64_t e0 = se[t], q0 = sq[t], ua = su[t], ub = su[t + 1];
  const int ne = (int)(se[t + 1] - e0), np = (int)(sq[t + 1] - q0);
  const int64_t nr = ub - ua + 1;  // rows ua..ub hold the tile's entries
  const bool staged = nr + 1 <= kMergeRows + 1;
  for (int j = tid; j < np; j += kMergeThreads) s_pk[j] = pkey[q0 + j];
  if (staged)
    for (int j = tid; j <= nr; j += kMergeThreads) s_rp[j] = rp_o[ua + j];
  __syncthreads();
  // entry keys
  for (int j = tid; j < ne; j += kMergeThreads) {
    const int64_t e = e0 + j;
    int64_t u;
    if (staged) {
      int lo = 0, hi = (int)nr - 1;  // last row start <= e
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_rp[mid] <= e) lo = mid; else hi = mid - 1;
      }
      u = ua + lo;
    } else {
      int64_t lo = ua, hi = ub;
      while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (rp_o[mid] <= e) lo = mid; else hi = mid - 1;
      }
      u = lo;
    }
    s_ek[j] = (uint64_t)u << 32 | (uint32_t)ld_stream(col_o + e);
  }
  __syncthreads();
  int cur_g = -1;
  long long m2_loc = 0, in_loc = 0;
  auto account = [&](int64_t u, int32_t cc, int64_t wv) {
    const int gu = graph_of(gid, u);
    if (gu != cur_g) {
      if (cur_g >= 0 && (m2_loc | in_loc)) {
        atomicAdd((unsigned long long*)&gs[cur_g].m2, (unsigned long long)m2_loc);
        atomicAdd((unsigned long long*)&gs[cur_g].in_cur, (unsigned long long)in_loc);
      }
      cur_g = gu;
      m2_loc = in_loc = 0;
    }
    m2_loc += wv;
    if (lab && lab[cc] == lab[u]) in_loc += wv;
  };
  // old entries (warp-uniform trip count for the row sums)
  for (int j0 = 0; j0 < ne; j0 += kMergeThreads) {
    const int j = j0 + tid;
    int64_t u = -1, wv = 0;
    if (j < ne) {
      const int64_t e = e0 + j;
      const uint64_t key = s_ek[j];
      const int64_t q = q0 + lower_bound_smem(s_pk, np, key);
      // the equal pair follows its entry, possibly in the next tile
      const bool match = q - q0 < np ? s_pk[q - q0] == key : (q < P && pkey[q] == key);
      const uint32_t f = match ? pflag[q] : 0u;
      if (!(f & kPairRemoved)) {
        const int32_t cc = (int32_t)(key & 0xffffffffu);
        wv = ld_stream(w_o + e);
        if (match && (f & kPairIns)) wv = (f & kPairDel) ? pw[q] : wv + pw[q];
        const int64_t pos = e + pA[q] - pR[q];
        st_stream(col_n + pos, cc);
        st_stream(w_n + pos, (int32_t)wv);
        u = (int64_t)(key >> 32);
        account(u, cc, wv);
      }
    }
    add_row_weight(kdeg, u, wv);
  }
  // added pairs
  for (int j0 = 0; j0 < np; j0 += kMergeThreads) {
    const int j = j0 + tid;
    int64_t u = -1, wv = 0;
    if (j < np) {
      const int64_t q = q0 + j;
      if (pflag[q] & kPairAdded) {
        const uint64_t key = s_pk[j];
        const int64_t i = e0 + lower_bound_smem(s_ek, ne, key);
        const int32_t cc = (int32_t)(key & 0xffffffffu);
        wv = pw[q];
        const int64_t pos = i + pA[q] - pR[q];
        st_stream(col_n + pos, cc);
        st_stream(w_n + pos, (int32_t)wv);
        u = (int64_t)(key >> 32);
        account(u, cc, wv);
      }
    }
    add_row_weight(kdeg, u, wv);
  }
  // 2m and sum_i e_{i->C(i)}: one add per CTA when the tile lies in one graph
  const int g0 = cur_g;
  if (tid == 0) s_uni = -2;
  __syncthreads();
  if (g0 >= 0) atomicCAS(&s_uni, -2, g0);
  __syncthreads();
  const int gref = s_uni;
  const bool uni = __syncthreads_and(g0 < 0 || g0 == gref);
  if (uni) {
    unsigned long long a = (unsigned long long)m2_loc, b = (unsigned long long)in_loc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane_id() == 0) {
      s_red[0][tid >> 5] = a;
      s_red[1][tid >> 5] = b;
    }
    __syncthreads();
    if (tid == 0 && gref >= 0) {
      unsigned long long sa = 0, sb = 0;
      for (int x = 0; x < kMergeThreads / 32; x++) {
        sa += s_red[0][x];
        sb += s_red[1][x];
      }
      if (sa | sb) {
        atomicAdd((unsigned long long*)&gs[gref].m2, sa);
        atomicAdd((unsigned long long*)&gs[gref].in_cur, sb);
      }
    }
  } else if (cur_g >= 0 && (m2_loc | in_loc)) {
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
  DCD_TRY(out->pdelta.alloc(&c->mem, P));
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
                                             in_delta.get(), out->pdelta.get());
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
  ::dcd::count_launch(), new_rows<<<grid_for(n + 1, T), T, 0, s>>>(rp_o, out->pair_ptr.get(), added.get(),
                                                                    removed.get(), n, rp_n);
  DCD_LAUNCH_CHECK();

  // ---- merge (tiles of the merged sequence), degrees, m2, in ----
  DCD_TRY(out->k.alloc(&c->mem, n));
  DCD_TRY_CUDA(cudaMemsetAsync(out->k.get(), 0, n * sizeof(int64_t), s));
  DCD_TRY_CUDA(cudaMemsetAsync(c->gs.get(), 0, c->G * sizeof(GraphState), s));
  const int64_t total = c->nnz + P;
  const int64_t nt = cdiv(total, (int64_t)kMergeTile);
  if (nt > 0) {
    Buf<int64_t> split;
    DCD_TRY(split.alloc(&c->mem, 3 * (nt + 1)));
    int64_t* se = split.get();
    int64_t* sq = se + (nt + 1);
    int64_t* su = sq + (nt + 1);
    ::dcd::count_launch(), merge_split<<<grid_for(nt + 1, T), T, 0, s>>>(n, rp_o, col_o, out->pair_ptr.get(),
                                                                          out->pkey.get(), nt, total, se, sq, su);
    DCD_LAUNCH_CHECK();
    ::dcd::count_launch(), merge_tile<<<(unsigned)nt, kMergeThreads, 0, s>>>(
        n, rp_o, col_o, w_o, se, sq, su, out->pkey.get(), out->pw.get(), out->pflag.get(), added.get(),
        removed.get(), P, c->col[nxt].get(), c->w[nxt].get(), lab_gather, out->k.get(),
        c->G > 1 ? c->gid.get() : nullptr, c->gs.get());
    DCD_LAUNCH_CHECK();
  }
  if (from_prev) {
    ::dcd::count_launch(), seed_in<<<cdiv(c->G, 128), 128, 0, s>>>(c->gs.get(), c->G, c->in_prev.get(),
                                                                    in_delta.get());
    DCD_LAUNCH_CHECK();
  }
  return DCD_OK;
}

}  // namespace dcd
