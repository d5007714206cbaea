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
//
// GPU schedule (same decisions, reordered work):
//   A  per source: aggregate row i by community, pick j*, gain1; deletes.
//   B  sources with gain1 > 0 sorted by j* (radix sort), grouped.
//   C  per distinct j*: aggregate row j* once, then gain2 for every source of
//      the group (a hub chosen as j* by many sources is read once, not once
//      per source).
//   D  per source: mark Gamma(i), i, j*, flag C(j*).
#include "agg.cuh"
#include "hub.cuh"
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
  int64_t m2;                   // 2m when the context holds one graph
  const int32_t* gid;           // graph of each vertex (several graphs)
  const GraphState* gs;
  __device__ __forceinline__ int64_t m2_of(int64_t v) const { return gid ? gs[gid[v]].m2 : m2; }
  uint8_t* mark;
  uint8_t* cflag;
  // phase A outputs / phase C inputs, indexed by position in the source list
  const int32_t* src;
  int32_t* jstar;
  long long* g1;   // two words per source (low, high) of gain1
  uint8_t* flags;  // bit0: intra-community delete (mark Gamma(i)); bit1: winner
  // first-pass proposals (may be NULL): phase A sums a source's row by
  // community under C_{t-1} on G_t, the state the first local-move pass of
  // level 0 reads, so it also takes that pass's choice for the source (the
  // best neighbouring community, the S > 0 rule and the singleton guard) and
  // stores it in pre[source]; sources it does not sum keep -1
  const int32_t* size;
  int32_t* pre;
};

// (S, D, j) order of the j* choice: larger gain, then smaller C(j), then smaller j.
template <typename ST>
__device__ __forceinline__ bool better3(ST s1, int32_t d1, int32_t j1, ST s2, int32_t d2, int32_t j2) {
  return s1 > s2 || (s1 == s2 && (d1 < d2 || (d1 == d2 && j1 < j2)));
}

__device__ __forceinline__ void warp_argmax3(i128& S, int32_t& D, int32_t& J) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    i128 s2 = shfl_xor_st(S, o);
    int32_t d2 = __shfl_xor_sync(0xffffffffu, D, o);
    int32_t j2 = __shfl_xor_sync(0xffffffffu, J, o);
    if (better3(s2, d2, j2, S, D, J)) {
      S = s2;
      D = d2;
      J = j2;
    }
  }
}

// 64-bit gains: full-warp redux.sync steps with neutral values (no
// divergence): the largest gain (high word, then low word), then the
// smallest C(j) among the lanes holding it, then the smallest j (D and J are
// >= 0 where a lane has a candidate; the sentinel is INT_MAX).
__device__ __forceinline__ void warp_argmax3(long long& S, int32_t& D, int32_t& J) {
  const unsigned long long u = (unsigned long long)S ^ 0x8000000000000000ull;
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
  const unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
  const bool top = hi == mhi && lo == mlo;
  const unsigned dmin = __reduce_min_sync(0xffffffffu, top ? (unsigned)D : 0xffffffffu);
  const bool top2 = top && (unsigned)D == dmin;
  const unsigned jmin = __reduce_min_sync(0xffffffffu, top2 ? (unsigned)J : 0xffffffffu);
  S = (long long)((((unsigned long long)mhi << 32) | mlo) ^ 0x8000000000000000ull);
  D = (int32_t)dmin;
  J = (int32_t)jmin;
}

__device__ __forceinline__ void st_gain(long long* p, long long x) {
  p[0] = x;
  p[1] = x < 0 ? -1 : 0;
}
__device__ __forceinline__ void st_gain(long long* p, i128 x) {
  p[0] = (long long)(unsigned long long)x;
  p[1] = (long long)(unsigned long long)((unsigned __int128)x >> 64);
}
template <typename ST>
__device__ __forceinline__ ST ld_gain(const long long* p);
template <>
__device__ __forceinline__ long long ld_gain<long long>(const long long* p) {
  return p[0];
}
template <>
__device__ __forceinline__ i128 ld_gain<i128>(const long long* p) {
  return (i128)(((unsigned __int128)(unsigned long long)p[1] << 64) | (unsigned long long)p[0]);
}

// ---- row aggregation helpers ----

// Lanes of one warp hold row v (degree <= 32): neighbour label (-1: none or a
// self loop) and weight.
struct LaneRow {
  int32_t lab;
  int32_t wt;
};

__device__ __forceinline__ LaneRow lane_row(const SV& g, int32_t v) {
  const int lane = lane_id();
  const int64_t b = g.rp[v];
  const int d = (int)(g.rp[v + 1] - b);
  bool valid = lane < d;
  const int32_t y = valid ? ld_stream(g.col + b + lane) : -1;
  valid = valid && y != v;
  LaneRow r;
  r.lab = valid ? g.L[y] : -1;
  r.wt = valid ? ld_stream(g.w + b + lane) : 0;
  return r;
}

// Weight from the row into community D (D the same in every lane): one
// reduction over the warp.
template <typename ST>
__device__ __forceinline__ int64_t lane_get(const LaneRow& r, int32_t D) {
  return group_sum<ST>(0xffffffffu, r.lab == D ? r.wt : 0);
}

// Weight from the row into each lane's own community D (lanes with want):
// one reduction per distinct D among them.
template <typename ST>
__device__ __forceinline__ int64_t lane_get_each(const LaneRow& r, int32_t D, bool want) {
  int64_t out = 0;
  unsigned todo = __ballot_sync(0xffffffffu, want);
  while (todo) {
    const int32_t Dl = __shfl_sync(0xffffffffu, D, __ffs(todo) - 1);
    const int64_t el = group_sum<ST>(0xffffffffu, r.lab == Dl ? r.wt : 0);
    const bool hit = want && D == Dl;
    if (hit) out = el;
    todo &= ~__ballot_sync(0xffffffffu, hit);
  }
  return out;
}

// A shared table (keys, sums) with the list of the slots it claimed; empty
// between uses: it is cleared once when a kernel starts and afterwards only
// the listed slots are emptied, so a row costs its own entries, not the
// table's capacity.  VT: 32-bit sums on the 64-bit gain path (2m < 2^31).
template <typename VT>
struct SlotTable {
  int32_t* keys;
  VT* vals;
  uint16_t* slots;
  int32_t* ns;
};

template <typename VT>
__device__ __forceinline__ SlotTable<VT> slot_table(unsigned char* base, int cap) {
  SlotTable<VT> t;
  t.vals = reinterpret_cast<VT*>(base);
  t.keys = reinterpret_cast<int32_t*>(base + (size_t)cap * sizeof(VT));
  t.slots = reinterpret_cast<uint16_t*>(base + (size_t)cap * (sizeof(VT) + 4));
  t.ns = reinterpret_cast<int32_t*>(base + (size_t)cap * (sizeof(VT) + 6));
  return t;
}
template <typename VT>
__host__ __device__ constexpr size_t slot_table_bytes(int cap) {
  return ((size_t)cap * (sizeof(VT) + 6) + 16 + 7) / 8 * 8;
}

// The whole table empty (NT threads, tid in [0, NT)); the caller synchronises.
template <typename VT>
__device__ __forceinline__ void slot_table_init(const SlotTable<VT>& t, int cap, int tid, int NT) {
  for (int x = tid; x < cap; x += NT) {
    t.keys[x] = -1;
    t.vals[x] = 0;
  }
  if (tid == 0) *t.ns = 0;
}

// Row v added into t by NT cooperating threads (whole warps): each thread
// inserts its own entries -- a CAS claims the slot of a new label, a shared
// atomic adds the weight, and the claimed slots are listed (one reservation
// per warp and round) -- except the entries of label `skip` (the row vertex's
// own community, most of a row), whose weight the thread sums in a register
// and returns for the caller to reduce.  No warp-wide grouping runs per
// entry.  The caller synchronises before and after.
template <typename ST, typename VT>
__device__ __forceinline__ VT slot_table_fill(const SV& g, int32_t v, const SlotTable<VT>& t, uint32_t mask, int tid,
                                              int NT, int32_t skip) {
  const int64_t b = g.rp[v];
  const int64_t d = g.rp[v + 1] - b;
  VT acc = 0;
  for (int64_t e0 = 0; e0 < d; e0 += NT) {
    const int64_t e = e0 + tid;
    bool valid = e < d;
    const int32_t y = valid ? ld_stream(g.col + b + e) : -1;
    valid = valid && y != v;
    const int32_t lab = valid ? g.L[y] : -1;
    const int32_t wt = valid ? ld_stream(g.w + b + e) : 0;
    bool claimed = false;
    uint32_t sl = 0;
    if (valid) {
      if (lab == skip) {
        acc += (VT)wt;
      } else {
        sl = probe_claim(t.keys, mask, lab, claimed);
        atomicAdd(&t.vals[sl], (VT)wt);
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, claimed);
    int at = 0;
    if (lane_id() == 0 && bal) at = atomicAdd(t.ns, __popc(bal));
    at = __shfl_sync(0xffffffffu, at, 0);
    if (claimed) t.slots[at + __popc(bal & lanemask_lt())] = (uint16_t)sl;
  }
  return acc;
}

// Sum over a CTA of one value per thread (red: NW words of shared memory);
// every thread gets the total.  Synchronises twice.
template <int NW, typename VT>
__device__ __forceinline__ int64_t cta_total(VT x, VT* red) {
  const int64_t w = seg_total<32>(x, 0xffffffffu);
  if (lane_id() == 0) red[threadIdx.x >> 5] = (VT)w;
  __syncthreads();
  int64_t t = 0;
#pragma unroll
  for (int i = 0; i < NW; i++) t += (int64_t)red[i];
  __syncthreads();
  return t;
}

// Empty the listed slots (after a synchronisation that ends the table's reads);
// the count is reset by thread 0 after the next synchronisation.
template <typename VT>
__device__ __forceinline__ void slot_table_clear(const SlotTable<VT>& t, int tid, int NT) {
  const int nd = *t.ns;
  for (int x = tid; x < nd; x += NT) {
    const uint32_t sl = t.slots[x];
    t.keys[sl] = -1;
    t.vals[sl] = 0;
  }
}

// Deleted pairs of source u: mark the endpoints; return whether one of them
// is an intra-community delete (then Gamma(u) is marked in phase D).
__device__ __forceinline__ bool scan_deletes(const SV& g, int32_t u, int64_t p0, int64_t p1, int tid, int NT,
                                             bool* has_ins) {
  const int32_t C = g.L[u];
  bool intra = false, ins = false;
  for (int64_t q = p0 + tid; q < p1; q += NT) {
    const uint8_t f = g.pflag[q];
    ins |= (f & kPairIns) != 0;
    if ((f & kPairDel) && (f & kPairPresent)) {
      const int32_t j = (int32_t)(g.pkey[q] & 0xffffffffu);
      g.mark[j] = 1;
      g.mark[u] = 1;
      intra |= g.L[j] == C;
    }
  }
  *has_ins = ins;
  return intra;
}

// ---- phase A: j* and gain1 per source ----

// Sources of degree <= 32: one warp, lanes hold the row.
template <typename ST>
__global__ void __launch_bounds__(256) scr_a_warp(SV g, int64_t off, int64_t cnt) {
  const int lane = lane_id();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < cnt; i += nw) {
    const int64_t idx = off + i;
    const int32_t u = g.src[idx];
    const int32_t C = g.L[u];
    const int64_t p0 = g.pair_ptr[u], p1 = g.pair_ptr[u + 1];
    bool has_ins;
    const bool intra = __any_sync(0xffffffffu, scan_deletes(g, u, p0, p1, lane, 32, &has_ins));
    has_ins = __any_sync(0xffffffffu, has_ins);
    int32_t J = -1;
    ST S = 0;
    if (has_ins) {
      const LaneRow r = lane_row(g, u);
      const int64_t eC = lane_get<ST>(r, C);
      const int64_t ku = g.k[u], aC = g.a[C];
      if (g.pre) {
        // the local move's choice (the lanes hold the row): lanes grouped by
        // neighbouring community, the first lane of each group takes its
        // gain, one argmax over the warp
        const bool cand = r.lab >= 0 && r.lab != C;
        const unsigned peers = __match_any_sync(0xffffffffu, cand ? r.lab : -1);
        const int64_t el = group_sum<ST>(peers, r.wt);
        ST Sb = gain_lowest<ST>();
        int32_t Db = INT_MAX;
        if (cand && (int)(__ffs(peers) - 1) == lane) {
          Sb = gain<ST>(g.m2_of(u), ku, el, eC, g.a[r.lab], aC);
          Db = r.lab;
        }
        warp_argmax(Sb, Db);
        if (lane == 0) g.pre[u] = move_proposal(Sb, Db, C, g.size);
      }
      int32_t D = INT_MAX;
      J = INT_MAX;
      S = gain_lowest<ST>();
      for (int64_t q0 = p0; q0 < p1; q0 += 32) {
        const int64_t q = q0 + lane;
        const bool sink = q < p1 && (g.pflag[q] & kPairIns);
        const int32_t j = sink ? (int32_t)(g.pkey[q] & 0xffffffffu) : -1;
        const int32_t Dj = sink ? g.L[j] : -2;
        const int64_t eD = lane_get_each<ST>(r, Dj, sink);
        if (sink) {
          const ST x = (Dj == C) ? ST(0) : gain<ST>(g.m2_of(u), ku, eD, eC, g.a[Dj], aC);
          if (better3(x, Dj, j, S, D, J)) {
            S = x;
            D = Dj;
            J = j;
          }
        }
      }
      warp_argmax3(S, D, J);
    }
    if (lane == 0) {
      g.jstar[idx] = J;
      st_gain(&g.g1[2 * idx], S);
      g.flags[idx] = intra ? 1 : 0;
    }
  }
}

// Sources of degree 33..256: one warp with a warp-private shared table.
template <typename ST>
__global__ void __launch_bounds__(256) scr_a_wtbl(SV g, int64_t off, int64_t cnt) {
  using VT = typename TblVal<ST>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = lane_id(), wib = threadIdx.x >> 5;
  const SlotTable<VT> t = slot_table<VT>(smem + (size_t)wib * slot_table_bytes<VT>(kMidCap), kMidCap);
  slot_table_init(t, kMidCap, lane, 32);
  __syncwarp();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < cnt; i += nw) {
    const int64_t idx = off + i;
    const int32_t u = g.src[idx];
    const int32_t C = g.L[u];
    const int64_t p0 = g.pair_ptr[u], p1 = g.pair_ptr[u + 1];
    bool has_ins;
    const bool intra = __any_sync(0xffffffffu, scan_deletes(g, u, p0, p1, lane, 32, &has_ins));
    has_ins = __any_sync(0xffffffffu, has_ins);
    int32_t J = -1;
    ST S = 0;
    if (has_ins) {
      const uint32_t mask = table_cap(g.rp[u + 1] - g.rp[u]) - 1;
      const VT own = slot_table_fill<ST, VT>(g, u, t, mask, lane, 32, C);
      __syncwarp();
      const int64_t eC = seg_total<32>(own, 0xffffffffu);
      const int64_t ku = g.k[u], aC = g.a[C];
      if (g.pre) {  // the local move's choice over the table's communities
        ST Sb = gain_lowest<ST>();
        int32_t Db = INT_MAX;
        const int nd = *t.ns;
        for (int x = lane; x < nd; x += 32) {
          const uint32_t sl = t.slots[x];
          const int32_t key = t.keys[sl];
          const ST y = gain<ST>(g.m2_of(u), ku, (int64_t)t.vals[sl], eC, g.a[key], aC);
          if (better(y, key, Sb, Db)) {
            Sb = y;
            Db = key;
          }
        }
        warp_argmax(Sb, Db);
        if (lane == 0) g.pre[u] = move_proposal(Sb, Db, C, g.size);
      }
      int32_t D = INT_MAX;
      J = INT_MAX;
      S = gain_lowest<ST>();
      for (int64_t q = p0 + lane; q < p1; q += 32) {
        if (!(g.pflag[q] & kPairIns)) continue;
        const int32_t j = (int32_t)(g.pkey[q] & 0xffffffffu);
        const int32_t Dj = g.L[j];
        const ST x = (Dj == C) ? ST(0) : gain<ST>(g.m2_of(u), ku, tbl_get(t.keys, t.vals, mask, Dj), eC, g.a[Dj], aC);
        if (better3(x, Dj, j, S, D, J)) {
          S = x;
          D = Dj;
          J = j;
        }
      }
      warp_argmax3(S, D, J);
      __syncwarp();
      slot_table_clear(t, lane, 32);
      __syncwarp();
      if (lane == 0) *t.ns = 0;
      __syncwarp();
    }
    if (lane == 0) {
      g.jstar[idx] = J;
      st_gain(&g.g1[2 * idx], S);
      g.flags[idx] = intra ? 1 : 0;
    }
  }
}

// Sources above 256 entries: one CTA, table in shared memory (<= 4096
// entries) or in a per-CTA region of global memory.
template <typename ST, int THREADS>
__global__ void __launch_bounds__(THREADS) scr_a_block(SV g, int64_t off, int64_t cnt, int cap) {
  using VT = typename TblVal<ST>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NW = THREADS / 32;
  __shared__ ST redS[NW];
  __shared__ int32_t redD[NW], redJ[NW];
  __shared__ VT redE[NW];
  __shared__ ST preS[NW];
  __shared__ int32_t preD[NW];
  __shared__ int s_flags;
  const int tid = threadIdx.x, lane = lane_id(), wid = tid >> 5;
  const SlotTable<VT> t = slot_table<VT>(smem, cap);
  slot_table_init(t, cap, tid, THREADS);
  __syncthreads();
  for (int64_t i = blockIdx.x; i < cnt; i += gridDim.x) {
    const int64_t idx = off + i;
    const int32_t u = g.src[idx];
    const int32_t C = g.L[u];
    const int64_t p0 = g.pair_ptr[u], p1 = g.pair_ptr[u + 1];
    if (tid == 0) s_flags = 0;
    __syncthreads();
    bool has_ins;
    const bool intra = scan_deletes(g, u, p0, p1, tid, THREADS, &has_ins);
    if (intra || has_ins) atomicOr(&s_flags, (intra ? 1 : 0) | (has_ins ? 2 : 0));
    __syncthreads();
    const int flags = s_flags;
    int32_t J = -1;
    ST S = 0;
    if (flags & 2) {
      const uint32_t mask = table_cap(g.rp[u + 1] - g.rp[u]) - 1;
      const VT own = slot_table_fill<ST, VT>(g, u, t, mask, tid, THREADS, C);
      const int64_t eC = cta_total<NW>(own, redE);
      const int64_t ku = g.k[u], aC = g.a[C];
      if (g.pre) {  // the local move's choice over the table's communities
        ST Sb = gain_lowest<ST>();
        int32_t Db = INT_MAX;
        const int nd = *t.ns;
        for (int x = tid; x < nd; x += THREADS) {
          const uint32_t sl = t.slots[x];
          const int32_t key = t.keys[sl];
          const ST y = gain<ST>(g.m2_of(u), ku, (int64_t)t.vals[sl], eC, g.a[key], aC);
          if (better(y, key, Sb, Db)) {
            Sb = y;
            Db = key;
          }
        }
        warp_argmax(Sb, Db);
        if (lane == 0) {
          preS[wid] = Sb;
          preD[wid] = Db;
        }
      }
      int32_t D = INT_MAX;
      J = INT_MAX;
      S = gain_lowest<ST>();
      for (int64_t q = p0 + tid; q < p1; q += THREADS) {
        if (!(g.pflag[q] & kPairIns)) continue;
        const int32_t j = (int32_t)(g.pkey[q] & 0xffffffffu);
        const int32_t Dj = g.L[j];
        const ST x = (Dj == C) ? ST(0) : gain<ST>(g.m2_of(u), ku, tbl_get(t.keys, t.vals, mask, Dj), eC, g.a[Dj], aC);
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
      warp_argmax3(S, D, J);
      if (g.pre && wid == 0) {
        ST Sb = lane < NW ? preS[lane] : gain_lowest<ST>();
        int32_t Db = lane < NW ? preD[lane] : INT_MAX;
        warp_argmax(Sb, Db);
        if (lane == 0) g.pre[u] = move_proposal(Sb, Db, C, g.size);
      }
      slot_table_clear(t, tid, THREADS);
      __syncthreads();
      if (tid == 0) *t.ns = 0;
    }
    if (tid == 0) {
      g.jstar[idx] = J;
      st_gain(&g.g1[2 * idx], S);
      g.flags[idx] = (flags & 1) ? 1 : 0;
    }
    __syncthreads();
  }
}

// Hub sources (rows above 4096 entries): the rows were summed into per-hub
// global tables by hub_agg (many CTAs per row); one CTA per source then
// reads its deletes and evaluates its insert sinks by table lookups.
template <typename ST, int THREADS>
__global__ void __launch_bounds__(THREADS) scr_a_hub(SV g, int64_t off, int64_t cnt, HubTables t) {
  constexpr int NW = THREADS / 32;
  __shared__ ST redS[NW];
  __shared__ int32_t redD[NW], redJ[NW];
  __shared__ int s_flags;
  const int tid = threadIdx.x, lane = lane_id(), wid = tid >> 5;
  for (int64_t h = blockIdx.x; h < cnt; h += gridDim.x) {
    const int64_t idx = off + h;
    const int32_t u = g.src[idx];
    const int32_t C = g.L[u];
    const int64_t p0 = g.pair_ptr[u], p1 = g.pair_ptr[u + 1];
    if (tid == 0) s_flags = 0;
    __syncthreads();
    bool has_ins;
    const bool intra = scan_deletes(g, u, p0, p1, tid, THREADS, &has_ins);
    if (intra || has_ins) atomicOr(&s_flags, (intra ? 1 : 0) | (has_ins ? 2 : 0));
    __syncthreads();
    const int flags = s_flags;
    int32_t J = -1;
    ST S = 0;
    if (flags & 2) {
      const uint32_t mask = (uint32_t)(t.toff[h + 1] - t.toff[h]) - 1;
      const int32_t* keys = t.keys + t.toff[h];
      const unsigned long long* vals = t.vals + t.toff[h];
      const int64_t eC = tbl_get(keys, vals, mask, C);
      const int64_t ku = g.k[u], aC = g.a[C];
      int32_t D = INT_MAX;
      J = INT_MAX;
      S = gain_lowest<ST>();
      for (int64_t q = p0 + tid; q < p1; q += THREADS) {
        if (!(g.pflag[q] & kPairIns)) continue;
        const int32_t j = (int32_t)(g.pkey[q] & 0xffffffffu);
        const int32_t Dj = g.L[j];
        const ST x = (Dj == C) ? ST(0) : gain<ST>(g.m2_of(u), ku, tbl_get(keys, vals, mask, Dj), eC, g.a[Dj], aC);
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
      warp_argmax3(S, D, J);
    }
    if (tid == 0) {
      g.jstar[idx] = J;
      st_gain(&g.g1[2 * idx], S);
      g.flags[idx] = (flags & 1) ? 1 : 0;
    }
    __syncthreads();
  }
}

// ---- phase B: group the sources with gain1 > 0 by j* ----

template <typename ST>
__global__ void cand_keys(SV g, int64_t nsrc, int64_t n, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nsrc; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t j = g.jstar[i];
    const bool cand = j >= 0 && ld_gain<ST>(&g.g1[2 * i]) > 0;
    keys[i] = cand ? (uint64_t)j : (uint64_t)n;
    vals[i] = (uint32_t)i;
  }
}

// group heads of candidate keys (< n) -> group start offsets (compacted)
__global__ void group_heads(const uint64_t* __restrict__ keys, int64_t m, int64_t n, int32_t* __restrict__ head) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    head[e] = (keys[e] < (uint64_t)n && (e == 0 || keys[e] != keys[e - 1])) ? 1 : 0;
}

__global__ void group_starts(const int32_t* __restrict__ head, const int32_t* __restrict__ hpos, int64_t m,
                             int32_t* __restrict__ gstart) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    if (head[e]) gstart[hpos[e]] = (int32_t)e;
}

// lower bound of the sentinel key n in the sorted keys (one warp)
__global__ void close_groups(const uint64_t* __restrict__ keys, int64_t m, int64_t n, int32_t* __restrict__ out) {
  if (threadIdx.x != 0) return;
  int64_t lo = 0, hi = m;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (keys[mid] < (uint64_t)n) lo = mid + 1; else hi = mid;
  }
  *out = (int32_t)lo;
}

// groups binned by the degree of their j*
__global__ void group_bins(const uint64_t* __restrict__ keys, const int32_t* __restrict__ gstart, int64_t ng,
                           const int64_t* __restrict__ rp, int32_t* __restrict__ cursor, int32_t* __restrict__ lists,
                           int64_t cap_per_bin) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x) + (threadIdx.x & ~31); base < ng; base += stride) {
    const int64_t gi = base + lane_id();
    int bin = -1;
    if (gi < ng) {
      const int64_t j = (int64_t)keys[gstart[gi]];
      const int64_t deg = rp[j + 1] - rp[j];
      bin = deg <= kBinWarpMax ? 0 : deg <= kBinMidMax ? 1 : deg <= kBinLargeMax ? 2 : 3;
    }
#pragma unroll
    for (int b = 0; b < 4; b++) {
      const unsigned bal = __ballot_sync(0xffffffffu, bin == b);
      if (!bal) continue;
      int32_t slot = 0;
      if (lane_id() == 0) slot = atomicAdd(&cursor[b], __popc(bal));
      slot = __shfl_sync(0xffffffffu, slot, 0);
      if (bin == b) lists[b * cap_per_bin + slot + __popc(bal & lanemask_lt())] = (int32_t)gi;
    }
  }
}

// ---- phase C: gain2 per source, one aggregation of row j* per group ----

struct GroupView {
  const uint64_t* keys;  // sorted candidate keys (j*)
  const uint32_t* vals;  // source-list positions in key order
  const int32_t* gstart; // ng + 1 group starts
  const int32_t* glist;  // groups of this bin
};

template <typename ST>
__device__ __forceinline__ void decide(const SV& g, int64_t idx, int32_t j, int64_t e1, int64_t e2) {
  const int32_t i = g.src[idx];
  const int32_t Ci = g.L[i], Cj = g.L[j];
  const ST g2 = (Cj == Ci) ? ST(0) : gain<ST>(g.m2_of(j), g.k[j], e1, e2, g.a[Ci], g.a[Cj]);
  if (ld_gain<ST>(&g.g1[2 * idx]) >= g2) g.flags[idx] |= 2;
}

template <typename ST>
__global__ void __launch_bounds__(256) scr_c_warp(SV g, GroupView gv, int64_t cnt) {
  const int lane = lane_id();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < cnt; i += nw) {
    const int32_t gi = gv.glist[i];
    const int64_t m0 = gv.gstart[gi], m1 = gv.gstart[gi + 1];
    const int32_t j = (int32_t)gv.keys[m0];
    const LaneRow r = lane_row(g, j);
    const int64_t e2 = lane_get<ST>(r, g.L[j]);
    for (int64_t q0 = m0; q0 < m1; q0 += 32) {
      const int64_t q = q0 + lane;
      const int64_t idx = q < m1 ? (int64_t)gv.vals[q] : -1;
      const int32_t Ci = idx >= 0 ? g.L[g.src[idx]] : -2;
      const int64_t e1 = lane_get_each<ST>(r, Ci, idx >= 0);
      if (idx >= 0) decide<ST>(g, idx, j, e1, e2);
    }
  }
}

template <typename ST>
__global__ void __launch_bounds__(256) scr_c_wtbl(SV g, GroupView gv, int64_t cnt) {
  using VT = typename TblVal<ST>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = lane_id(), wib = threadIdx.x >> 5;
  const SlotTable<VT> t = slot_table<VT>(smem + (size_t)wib * slot_table_bytes<VT>(kMidCap), kMidCap);
  slot_table_init(t, kMidCap, lane, 32);
  __syncwarp();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < cnt; i += nw) {
    const int32_t gi = gv.glist[i];
    const int64_t m0 = gv.gstart[gi], m1 = gv.gstart[gi + 1];
    const int32_t j = (int32_t)gv.keys[m0];
    const int32_t Cj = g.L[j];
    const uint32_t mask = table_cap(g.rp[j + 1] - g.rp[j]) - 1;
    const VT own = slot_table_fill<ST, VT>(g, j, t, mask, lane, 32, Cj);
    __syncwarp();
    const int64_t e2 = seg_total<32>(own, 0xffffffffu);
    for (int64_t q = m0 + lane; q < m1; q += 32) {
      const int64_t idx = gv.vals[q];
      const int32_t Ci = g.L[g.src[idx]];
      decide<ST>(g, idx, j, Ci == Cj ? e2 : tbl_get(t.keys, t.vals, mask, Ci), e2);
    }
    __syncwarp();
    slot_table_clear(t, lane, 32);
    __syncwarp();
    if (lane == 0) *t.ns = 0;
    __syncwarp();
  }
}

template <typename ST, int THREADS>
__global__ void __launch_bounds__(THREADS) scr_c_block(SV g, GroupView gv, int64_t cnt, int cap) {
  using VT = typename TblVal<ST>::type;
  constexpr int NW = THREADS / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ VT redE[NW];
  const int tid = threadIdx.x;
  const SlotTable<VT> t = slot_table<VT>(smem, cap);
  slot_table_init(t, cap, tid, THREADS);
  __syncthreads();
  for (int64_t i = blockIdx.x; i < cnt; i += gridDim.x) {
    const int32_t gi = gv.glist[i];
    const int64_t m0 = gv.gstart[gi], m1 = gv.gstart[gi + 1];
    const int32_t j = (int32_t)gv.keys[m0];
    const int32_t Cj = g.L[j];
    const uint32_t mask = table_cap(g.rp[j + 1] - g.rp[j]) - 1;
    const VT own = slot_table_fill<ST, VT>(g, j, t, mask, tid, THREADS, Cj);
    const int64_t e2 = cta_total<NW>(own, redE);
    for (int64_t q = m0 + tid; q < m1; q += THREADS) {
      const int64_t idx = gv.vals[q];
      const int32_t Ci = g.L[g.src[idx]];
      decide<ST>(g, idx, j, Ci == Cj ? e2 : tbl_get(t.keys, t.vals, mask, Ci), e2);
    }
    __syncthreads();
    slot_table_clear(t, tid, THREADS);
    __syncthreads();
    if (tid == 0) *t.ns = 0;
    __syncthreads();
  }
}

// j* of each hub group (the vertex whose row hub_agg sums).
__global__ void group_vertices(const uint64_t* __restrict__ keys, const int32_t* __restrict__ gstart,
                               const int32_t* __restrict__ glist, int64_t cnt, int32_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int32_t)keys[gstart[glist[i]]];
}

// Hub j* (rows above 4096 entries) summed into per-hub tables by hub_agg; one
// CTA per group evaluates gain2 for its sources by lookups.
template <typename ST, int THREADS>
__global__ void __launch_bounds__(THREADS) scr_c_hub(SV g, GroupView gv, int64_t cnt, HubTables t) {
  for (int64_t h = blockIdx.x; h < cnt; h += gridDim.x) {
    const int32_t gi = gv.glist[h];
    const int64_t m0 = gv.gstart[gi], m1 = gv.gstart[gi + 1];
    const int32_t j = t.list[h];
    const uint32_t mask = (uint32_t)(t.toff[h + 1] - t.toff[h]) - 1;
    const int32_t* keys = t.keys + t.toff[h];
    const unsigned long long* vals = t.vals + t.toff[h];
    const int64_t e2 = tbl_get(keys, vals, mask, g.L[j]);
    for (int64_t q = m0 + threadIdx.x; q < m1; q += THREADS) {
      const int64_t idx = gv.vals[q];
      decide<ST>(g, idx, j, tbl_get(keys, vals, mask, g.L[g.src[idx]]), e2);
    }
  }
}

// ---- phase D: marks ----
// Sources [lo, hi) of the list, a warp each.
__global__ void __launch_bounds__(256) scr_mark(SV g, int64_t lo, int64_t hi) {
  const int lane = lane_id();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t idx = lo + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); idx < hi; idx += nw) {
    const uint8_t f = g.flags[idx];
    if (!f) continue;
    const int32_t u = g.src[idx];
    if (lane == 0) {
      g.mark[u] = 1;
      if (f & 2) {
        const int32_t j = g.jstar[idx];
        g.mark[j] = 1;
        g.cflag[g.L[j]] = 1;
      }
    }
    const int64_t e1 = g.rp[u + 1];
    for (int64_t e = g.rp[u] + lane; e < e1; e += 32) g.mark[g.col[e]] = 1;
  }
}

// Hub sources [lo, hi) of the list (rows above 4096 entries): kMarkSlices
// CTAs per source, each marking one slice of the row.
constexpr int kMarkSlices = 16;
__global__ void __launch_bounds__(256) scr_mark_hub(SV g, int64_t lo, int64_t hi) {
  for (int64_t b = blockIdx.x; b < (hi - lo) * kMarkSlices; b += gridDim.x) {
    const int64_t idx = lo + b / kMarkSlices;
    const int sl = (int)(b % kMarkSlices);
    const uint8_t f = g.flags[idx];
    if (!f) continue;
    const int32_t u = g.src[idx];
    if (sl == 0 && threadIdx.x == 0) {
      g.mark[u] = 1;
      if (f & 2) {
        const int32_t j = g.jstar[idx];
        g.mark[j] = 1;
        g.cflag[g.L[j]] = 1;
      }
    }
    const int64_t r0 = g.rp[u], d = g.rp[u + 1] - r0;
    const int64_t e0 = r0 + d * sl / kMarkSlices, e1 = r0 + d * (sl + 1) / kMarkSlices;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) g.mark[g.col[e]] = 1;
  }
}

// Sources (vertices with at least one pair) binned by their degree in G_t.
__global__ void src_bins(int64_t n, const int64_t* __restrict__ pair_ptr, const int64_t* __restrict__ rp,
                         int32_t* __restrict__ cursor, int32_t* __restrict__ lists, int64_t cap_per_bin) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x) + (threadIdx.x & ~31); base < n; base += stride) {
    const int64_t v = base + lane_id();
    int bin = -1;
    if (v < n && pair_ptr[v + 1] > pair_ptr[v]) {
      const int64_t deg = rp[v + 1] - rp[v];
      bin = deg <= kBinWarpMax ? 0 : deg <= kBinMidMax ? 1 : deg <= kBinLargeMax ? 2 : 3;
    }
#pragma unroll
    for (int b = 0; b < 4; b++) {
      const unsigned bal = __ballot_sync(0xffffffffu, bin == b);
      if (!bal) continue;
      int32_t slot = 0;
      if (lane_id() == 0) slot = atomicAdd(&cursor[b], __popc(bal));
      slot = __shfl_sync(0xffffffffu, slot, 0);
      if (bin == b) lists[b * cap_per_bin + slot + __popc(bal & lanemask_lt())] = (int32_t)v;
    }
  }
}

// Packs the four per-bin segments into one list (bin order).
__global__ void pack_bins(const int32_t* __restrict__ lists, int64_t cap_per_bin, int64_t c0, int64_t c1, int64_t c2,
                          int64_t c3, int32_t* __restrict__ out) {
  const int64_t tot = c0 + c1 + c2 + c3;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    int b = 0;
    int64_t r = i;
    if (r >= c0) { r -= c0; b = 1;
      if (r >= c1) { r -= c1; b = 2;
        if (r >= c2) { r -= c2; b = 3; } } }
    out[i] = lists[b * cap_per_bin + r];
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


template <typename ST>
int screen_impl(dcd_ctx* c, SV& sv, const Csr<int32_t>& g, const int64_t* cnt, int64_t nsrc) {
  cudaStream_t s = c->stream;
  const int T = 256;
  const int64_t n = g.n;
  using VT = typename TblVal<ST>::type;
  const size_t wsmem = (size_t)8 * slot_table_bytes<VT>(kMidCap), bsmem = slot_table_bytes<VT>(kLargeCap);
  DCD_TRY_CUDA(cudaFuncSetAttribute(scr_a_wtbl<ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsmem));
  DCD_TRY_CUDA(cudaFuncSetAttribute(scr_c_wtbl<ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsmem));
  DCD_TRY_CUDA(cudaFuncSetAttribute(scr_a_block<ST, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsmem));
  DCD_TRY_CUDA(cudaFuncSetAttribute(scr_c_block<ST, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsmem));
  const int64_t off1 = cnt[0], off2 = off1 + cnt[1], off3 = off2 + cnt[2];
  const int sm2 = 2 * c->sms;

  // ---- A ----
  // the four source classes write disjoint slices of the per-source outputs:
  // they run side by side (the hub tables are set up before the fork)
  {
    HubBufs hb;
    if (cnt[3]) DCD_TRY(hub_setup(c, sv.src + off3, cnt[3], g.rp, &hb));
    SideBySide par(c, nsrc);
    DCD_TRY(par.fork());
    cudaStream_t sx;
    if (cnt[0]) {
      DCD_TRY(par.on(0, &sx));
      count_launch(), scr_a_warp<ST><<<wave_grid(scr_a_warp<ST>, cnt[0] * 32, T), T, 0, sx>>>(sv, 0, cnt[0]);
    }
    if (cnt[1]) {
      DCD_TRY(par.on(1, &sx));
      count_launch(), scr_a_wtbl<ST><<<wave_grid(scr_a_wtbl<ST>, cnt[1] * 32, T, wsmem), T, wsmem, sx>>>(sv, off1,
                                                                                                       cnt[1]);
    }
    if (cnt[2]) {
      DCD_TRY(par.on(2, &sx));
      count_launch(), scr_a_block<ST, 256><<<(unsigned)(cnt[2] < sm2 ? cnt[2] : sm2), 256, bsmem, sx>>>(
                          sv, off2, cnt[2], kLargeCap);
    }
    if (cnt[3]) {
      DCD_TRY(par.on(3, &sx));
      count_launch(), hub_agg<int32_t, ST><<<hub_grid(c, hb), 256, 0, sx>>>(sv, hb.t);
      count_launch(), scr_a_hub<ST, 512><<<(unsigned)(cnt[3] < 4 * c->sms ? cnt[3] : 4 * c->sms), 512, 0, sx>>>(
                          sv, off3, cnt[3], hb.t);
    }
    DCD_LAUNCH_CHECK();
    DCD_TRY(par.join());
  }

  trace("screen: phase A");
  // ---- B ----
  Buf<uint64_t> k0, k1;
  Buf<uint32_t> v0, v1, stmp;
  Buf<int32_t> head, hpos, gstart;  // gstart: ng + 1 group starts
  DCD_TRY(k0.alloc(&c->mem, nsrc));
  DCD_TRY(k1.alloc(&c->mem, nsrc));
  DCD_TRY(v0.alloc(&c->mem, nsrc));
  DCD_TRY(v1.alloc(&c->mem, nsrc));
  DCD_TRY(head.alloc(&c->mem, nsrc + 1));
  DCD_TRY(hpos.alloc(&c->mem, nsrc + 1));
  DCD_TRY(stmp.alloc(&c->mem, sort_tmp_words(nsrc) + scan_tmp_count(nsrc + 1) + 64));
  count_launch(), cand_keys<ST><<<grid_for(nsrc, T), T, 0, s>>>(sv, nsrc, n, k0.get(), v0.get());
  DCD_LAUNCH_CHECK();
  const int b = bits_for(n);
  int ranges[2] = {0, b};
  bool in1 = false;
  DCD_TRY(sort_pairs<uint32_t>(k0.get(), v0.get(), k1.get(), v1.get(), nsrc, ranges, 1, stmp.get(), &in1, s));
  const uint64_t* keys = in1 ? k1.get() : k0.get();
  const uint32_t* vals = in1 ? v1.get() : v0.get();
  count_launch(), group_heads<<<grid_for(nsrc, T), T, 0, s>>>(keys, nsrc, n, head.get());
  DCD_LAUNCH_CHECK();
  DCD_TRY(exclusive_scan<int32_t>(head.get(), hpos.get(), nsrc, hpos.get() + nsrc,
                                  reinterpret_cast<int32_t*>(stmp.get()), s));
  // number of candidates = first position with the sentinel key: count heads, then members
  DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch, hpos.get() + nsrc, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  DCD_TRY_CUDA(cudaStreamSynchronize(s));
  const int64_t ng = *reinterpret_cast<int32_t*>(c->hscratch);
  if (ng > 0) {
    DCD_TRY(gstart.alloc(&c->mem, ng + 1));
    count_launch(), group_starts<<<grid_for(nsrc, T), T, 0, s>>>(head.get(), hpos.get(), nsrc, gstart.get());
    DCD_LAUNCH_CHECK();
    // end of the last group: number of candidate keys (< n)
    Buf<int32_t> gl, gcur;
    DCD_TRY(gl.alloc(&c->mem, 4 * ng));
    DCD_TRY(gcur.alloc(&c->mem, 4));
    DCD_TRY_CUDA(cudaMemsetAsync(gcur.get(), 0, 4 * sizeof(int32_t), s));
    count_launch(), group_bins<<<grid_for(ng, T), T, 0, s>>>(keys, gstart.get(), ng, g.rp, gcur.get(), gl.get(), ng);
    DCD_LAUNCH_CHECK();
    DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch, gcur.get(), 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    DCD_TRY_CUDA(cudaStreamSynchronize(s));
    const int32_t* gc = reinterpret_cast<const int32_t*>(c->hscratch);
    const int64_t gcnt[4] = {gc[0], gc[1], gc[2], gc[3]};
    // gstart[ng] = number of candidates = lower bound of the sentinel key
    count_launch(), close_groups<<<1, 32, 0, s>>>(keys, nsrc, n, gstart.get() + ng);
    DCD_LAUNCH_CHECK();
    // ---- C ----
    // each candidate group is in one class and a source in one group, so the
    // classes write disjoint flags: side by side, as in phase A
    GroupView gv{keys, vals, gstart.get(), gl.get()};
    Buf<int32_t> jl;
    HubBufs hb;
    if (gcnt[3]) {
      DCD_TRY(jl.alloc(&c->mem, gcnt[3]));
      count_launch(), group_vertices<<<grid_for(gcnt[3], T), T, 0, s>>>(keys, gstart.get(), gl.get() + 3 * ng,
                                                                        gcnt[3], jl.get());
      DCD_TRY(hub_setup(c, jl.get(), gcnt[3], g.rp, &hb));
    }
    SideBySide par(c, nsrc);
    DCD_TRY(par.fork());
    cudaStream_t sx;
    if (gcnt[0]) {
      DCD_TRY(par.on(0, &sx));
      count_launch(), scr_c_warp<ST><<<wave_grid(scr_c_warp<ST>, gcnt[0] * 32, T), T, 0, sx>>>(sv, gv, gcnt[0]);
    }
    gv.glist = gl.get() + ng;
    if (gcnt[1]) {
      DCD_TRY(par.on(1, &sx));
      count_launch(), scr_c_wtbl<ST><<<wave_grid(scr_c_wtbl<ST>, gcnt[1] * 32, T, wsmem), T, wsmem, sx>>>(sv, gv,
                                                                                                       gcnt[1]);
    }
    gv.glist = gl.get() + 2 * ng;
    if (gcnt[2]) {
      DCD_TRY(par.on(2, &sx));
      count_launch(), scr_c_block<ST, 256><<<(unsigned)(gcnt[2] < sm2 ? gcnt[2] : sm2), 256, bsmem, sx>>>(
                          sv, gv, gcnt[2], kLargeCap);
    }
    gv.glist = gl.get() + 3 * ng;
    if (gcnt[3]) {
      DCD_TRY(par.on(3, &sx));
      count_launch(), hub_agg<int32_t, ST><<<hub_grid(c, hb), 256, 0, sx>>>(sv, hb.t);
      count_launch(), scr_c_hub<ST, 512><<<(unsigned)(gcnt[3] < 4 * c->sms ? gcnt[3] : 4 * c->sms), 512, 0, sx>>>(
                          sv, gv, gcnt[3], hb.t);
    }
    DCD_LAUNCH_CHECK();
    DCD_TRY(par.join());
  }
  trace("screen: phases B, C");
  // ---- D ----
  if (off3) count_launch(), scr_mark<<<wave_grid(scr_mark, off3 * 32, T), T, 0, s>>>(sv, 0, off3);
  if (cnt[3]) count_launch(), scr_mark_hub<<<grid_for(cnt[3] * kMarkSlices * T, T, 8), T, 0, s>>>(sv, off3, nsrc);
  DCD_LAUNCH_CHECK();
  return DCD_OK;
}

}  // namespace

int screen_batch(dcd_ctx* c, const Csr<int32_t>& g, const int32_t* labels0, const int64_t* k, const int64_t* a,
                 const MergeOut& mo, uint8_t* rset, const int32_t* size, int32_t* pre) {
  cudaStream_t s = c->stream;
  DevScalars* d = c->dsc.get();
  const int64_t n = g.n;
  const int T = 256;
  Buf<uint8_t> mark, cflag;
  DCD_TRY(mark.alloc(&c->mem, n));
  DCD_TRY(cflag.alloc(&c->mem, n));
  DCD_TRY_CUDA(cudaMemsetAsync(mark.get(), 0, n, s));
  DCD_TRY_CUDA(cudaMemsetAsync(cflag.get(), 0, n, s));
  if (mo.npairs > 0) {
    Buf<int32_t> lists, cursor, src;
    DCD_TRY(lists.alloc(&c->mem, 4 * n));
    DCD_TRY(cursor.alloc(&c->mem, 4));
    DCD_TRY_CUDA(cudaMemsetAsync(cursor.get(), 0, 4 * sizeof(int32_t), s));
    count_launch(), src_bins<<<grid_for(n, T), T, 0, s>>>(n, mo.pair_ptr.get(), g.rp, cursor.get(), lists.get(), n);
    DCD_LAUNCH_CHECK();
    DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch, cursor.get(), 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    DCD_TRY_CUDA(cudaStreamSynchronize(s));
    const int32_t* cn = reinterpret_cast<const int32_t*>(c->hscratch);
    const int64_t cnt[4] = {cn[0], cn[1], cn[2], cn[3]};
    const int64_t nsrc = cnt[0] + cnt[1] + cnt[2] + cnt[3];
    DCD_TRY(src.alloc(&c->mem, nsrc));
    count_launch(), pack_bins<<<grid_for(nsrc, T), T, 0, s>>>(lists.get(), n, cnt[0], cnt[1], cnt[2], cnt[3], src.get());
    DCD_LAUNCH_CHECK();
    lists.reset();
    Buf<int32_t> jstar;
    Buf<long long> g1;
    Buf<uint8_t> flags;
    DCD_TRY(jstar.alloc(&c->mem, nsrc));
    DCD_TRY(g1.alloc(&c->mem, 2 * nsrc));
    DCD_TRY(flags.alloc(&c->mem, nsrc));
    int64_t m2max = 0;
    for (int x = 0; x < c->G; x++) m2max = c->hgs[x].m2 > m2max ? c->hgs[x].m2 : m2max;
    SV sv{g.rp, g.col, g.w, k, labels0, a, mo.pkey.get(), mo.pflag.get(), mo.pair_ptr.get(), c->hgs[0].m2,
          c->G > 1 ? c->gid.get() : nullptr, c->gs.get(), mark.get(), cflag.get(), src.get(), jstar.get(),
          g1.get(), flags.get(), size, pre};
    if (m2max >= ((int64_t)1 << 31)) DCD_TRY(screen_impl<i128>(c, sv, g, cnt, nsrc));
    else DCD_TRY(screen_impl<long long>(c, sv, g, cnt, nsrc));
  }
  DCD_TRY_CUDA(cudaMemsetAsync(&d->r_size, 0, sizeof(int64_t), s));
  count_launch(), build_rset<<<grid_for(n, T), T, 0, s>>>(n, mark.get(), cflag.get(), labels0, rset,
                                                          (unsigned long long*)&d->r_size);
  DCD_LAUNCH_CHECK();
  return DCD_OK;
}

}  // namespace dcd
