// louvain.cu -- Algorithm 1 (multi-level local moving with graph compaction)
// on the GPU, with the level-0 active set R_t of Sec. III-D.
//
// Schedule (the paper's code visits vertices one by one in an arbitrary order;
// this library takes the synchronous reading): every pass reads one snapshot
// of (labels, a_C, |C|); each active vertex picks the neighbour community of
// largest gain S (ties to the smaller label; a singleton does not move into a
// singleton of larger label), moving only on S > 0; all moves apply together.
// The pass loop of a level stops when no vertex moves, when the pass gained at
// most |N| / tau_inv (tau is not given in the paper; the state is kept), or
// after max_iters passes.  N = m2^2 Q is tracked exactly: the moved rows give
// the change of sum_i e_{i->C(i)}, a full reduction gives sum_C a_C^2.
//
// Kernels (degree-binned; a bin is a list of active vertex ids, see BinPlan):
//   lm_seg       rows of at most 16 .. 256 entries: a segment of 8, 16 or 32
//                lanes per vertex, each segment with its own table in shared
//                memory
//   lm_cta       rows of at most 512 .. 4096 entries: a CTA per vertex with a
//                shared table
//   hub_*        longer rows: split into chunks over many CTAs, per-hub tables
//                in global memory
// Compaction (graph of the next level): dense nc x nc sums for few
// communities, sort-by-key reduction for many; level 0 of an update can be
// built from the previous update's coarse graph (delta coarsening, below).
#include <cstdio>
#include <type_traits>
#include <vector>

#include "agg.cuh"
#include "hub.cuh"
#include "prims.cuh"
#include "state.cuh"

namespace dcd {

namespace {

template <typename W>
struct LV {
  const int64_t* rp;
  const int32_t* col;
  const W* w;
  const int64_t* k;
  const int32_t* L;
  const int64_t* a;
  const int32_t* size;
  int64_t m2;                   // 2m when the context holds one graph
  const int32_t* gid = nullptr;  // graph of each vertex (several graphs)
  const GraphState* gs = nullptr;
  __device__ __forceinline__ int64_t m2_of(int64_t v) const { return gid ? gs[gid[v]].m2 : m2; }
  // optional per-list-position statistics for the learned screen's features:
  // e_{v->C\v}, e_{v->D*}, D* (-1: none) and S(v -> D*) of the best other
  // community D* (the greedy choice before the S > 0 test and the guard)
  int64_t* f_eC = nullptr;
  int64_t* f_eB = nullptr;
  int32_t* f_dB = nullptr;
  double* f_sB = nullptr;
  // level 0 of a Delta-screening update: pre[v] >= 0 is v's proposal of the
  // level's first pass, taken by the screening from the same state; while
  // *first == 0 (no pass of the level has ended) the kernels store it
  // instead of evaluating v's row again
  const int32_t* pre = nullptr;
  const int32_t* first = nullptr;
  __device__ __forceinline__ int32_t pre_of(int32_t v) const { return (pre && *first == 0) ? pre[v] : -1; }
};

__device__ __forceinline__ double to_double(long long x) { return (double)x; }
__device__ __forceinline__ double to_double(i128 x) {
  const long long hi = (long long)(x >> 64);
  const unsigned long long lo = (unsigned long long)x;
  return (double)hi * 18446744073709551616.0 + (double)lo;
}

// The proposal of a vertex from its best (S, D): move on S > 0, subject to
// the guard.  Evaluated by every lane of the (uniform) argmax result, so the
// caller stores it with a predicated write instead of a divergent branch.
template <typename ST>
__device__ __forceinline__ int32_t proposal(ST S, int32_t D, int32_t C, const int32_t* size) {
  return move_proposal(S, D, C, size);
}

// ---------------------------------------------------------------- local move
//
// Rows up to 4096 entries: the neighbour communities of a row are summed in
// an open-addressing table in shared memory (community label -> summed edge
// weight), written by every lane for its own entries: a lane probes for its
// entry's label, claims an empty slot with a CAS when the label is new, and
// adds its weight with a shared-memory atomic.  The vertex's own community C
// never enters the table: e_{v->C\v} is summed in registers and reduced once.
// A lane that claims a slot appends it to the row's list of distinct labels
// (one ballot per entry position), so the gain step visits only the distinct
// communities and then empties exactly the slots it used.  No warp-wide
// grouping instruction (match) runs per entry: round trips to the table are
// ordinary shared-memory operations, which the SM issues at a far higher rate.
//
// The table of a row of at most R entries has seg_cap(R) >= 2R slots, so at
// most half of it is ever in use and every probe sequence ends at the key or
// at an empty slot.

__host__ __device__ constexpr int seg_cap(int row) {
  int c = 32;
  while (c < 2 * row) c <<= 1;
  return c;
}

// Shared memory of one row table: keys (int32), sums (VT), the claimed-slot
// list (one uint16 per row entry); a multiple of 16 bytes.
template <int ROW, typename VT>
__host__ __device__ constexpr size_t row_tbl_bytes() {
  return ((size_t)seg_cap(ROW) * (4 + sizeof(VT)) + (size_t)ROW * 2 + 15) / 16 * 16;
}

// The learned screen's per-row statistics (see LV).
template <typename W, typename ST, typename VT>
__device__ __forceinline__ void put_features(const LV<W>& g, int64_t i, int64_t eC, const int32_t* keys,
                                             const VT* vals, uint32_t mask, ST S, int32_t D) {
  g.f_eC[i] = eC;
  g.f_eB[i] = D == INT_MAX ? 0 : tbl_get(keys, vals, mask, D);
  g.f_dB[i] = D == INT_MAX ? -1 : D;
  g.f_sB[i] = D == INT_MAX ? 0.0 : to_double(S);
}

// S lanes per vertex (32 / S vertices a warp), Q entries per lane: rows of at
// most S x Q entries.  Each segment owns a table in shared memory; the
// segments of a warp run in lockstep on their own rows.
//
// The rows of a segment are software-pipelined, so that the dependent chain
// list -> row_ptr -> col -> L of a row is spread over several iterations
// instead of waiting in one.  With Q <= 4 (four stages): while row k is
// aggregated in the table, the neighbour communities of row k+1 are being
// gathered (with its k_v, a_C, |C| and 2m), the entries and community of row
// k+2 loaded, the bounds of row k+3 read and the list entry of row k+4
// fetched.  With Q = 8 the entries of two rows would not fit the register
// budget of four resident CTAs, so one stage less: row k's communities are
// gathered at the start of its iteration, while row k+1's entries, row k+2's
// bounds and row k+3's list entry are in flight.
// S lanes per vertex (32 / S vertices a warp), Q entries per lane: rows of at
// most S x Q entries.  Each segment owns a table in shared memory; the
// segments of a warp run in lockstep on their own rows.
template <typename W, typename ST, int S, int Q>
__global__ void __launch_bounds__(256) lm_seg(LV<W> g, const int32_t* __restrict__ list, int64_t cnt,
                                              int32_t* __restrict__ prop) {
  static_assert(S == 8 || S == 16 || S == 32, "segments of 8, 16 or 32 lanes");
  using VT = typename TblVal<ST>::type;
  constexpr int P = 32 / S, ROW = S * Q, CAP = seg_cap(ROW);
  constexpr size_t SB = row_tbl_bytes<ROW, VT>();
  constexpr uint32_t mask = CAP - 1;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = lane_id(), sub = lane / S, sl = lane % S, wib = threadIdx.x >> 5;
  const unsigned smask = S == 32 ? 0xffffffffu : (((1u << S) - 1u) << (sub * S));
  unsigned char* base = smem + ((size_t)wib * P + sub) * SB;
  int32_t* keys = reinterpret_cast<int32_t*>(base);
  VT* vals = reinterpret_cast<VT*>(base + (size_t)CAP * 4);
  uint16_t* slots = reinterpret_cast<uint16_t*>(base + (size_t)CAP * (4 + sizeof(VT)));
  for (int s = sl; s < CAP; s += S) {
    keys[s] = -1;
    vals[s] = 0;
  }
  __syncwarp();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t wb = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * P; wb < cnt; wb += nw * P) {
    const int64_t i = wb + sub;
    const bool has = i < cnt;
    const int32_t v = has ? ld_stream(list + i) : 0;
    const int32_t pv = has ? g.pre_of(v) : -1;  // the screening's first-pass proposal
    const int64_t b = g.rp[v];
    const int d = (has && pv < 0) ? (int)(g.rp[v + 1] - b) : 0;
    const int dmax = S == 32 ? d : (int)__reduce_max_sync(0xffffffffu, (unsigned)d);
    const int32_t C = g.L[v];
    int32_t lab[Q];
    W wt[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) {
      const int e = q * S + sl;
      lab[q] = -1;
      wt[q] = W(0);
      if (e < d) {
        lab[q] = ld_stream(g.col + b + e);
        wt[q] = ld_stream(g.w + b + e);
      }
    }
#pragma unroll
    for (int q = 0; q < Q; q++) {
      const int32_t u = lab[q];
      lab[q] = (u >= 0 && u != v) ? g.L[u] : -1;  // a coarse self-loop is no neighbour
    }
    VT eCl = 0;
    int nd = 0;
#pragma unroll
    for (int q = 0; q < Q; q++) {
      if (q * S < dmax) {
        const bool isC = lab[q] == C;
        eCl += isC ? (VT)wt[q] : VT(0);
        bool claimed = false;
        uint32_t s = 0;
        if (lab[q] >= 0 && !isC) {
          s = probe_claim(keys, mask, lab[q], claimed);
          atomicAdd(&vals[s], (VT)wt[q]);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, claimed) & smask;
        if (claimed) slots[nd + __popc(bal & lanemask_lt())] = (uint16_t)s;
        nd += __popc(bal);
      }
    }
    __syncwarp();
    const int64_t eC = seg_total<S>(eCl, smask);
    const int64_t kv = g.k[v], aC = g.a[C], m2v = g.m2_of(v);
    ST Sb = gain_lowest<ST>();
    int32_t D = INT_MAX;
    for (int j = sl; j < nd; j += S) {
      const uint32_t s = slots[j];
      const int32_t key = keys[s];
      const ST x = gain<ST>(m2v, kv, (int64_t)vals[s], eC, g.a[key], aC);
      if (better(x, key, Sb, D)) {
        Sb = x;
        D = key;
      }
    }
    seg_argmax<S>(Sb, D, smask);
    const int32_t pr = pv >= 0 ? pv : proposal(Sb, D, C, g.size);
    if (sl == 0 && has) {
      prop[i] = pr;
      if (g.f_eC) put_features(g, i, eC, keys, vals, mask, Sb, D);
    }
    __syncwarp();
    for (int j = sl; j < nd; j += S) {
      const uint32_t s = slots[j];
      keys[s] = -1;
      vals[s] = 0;
    }
    __syncwarp();
  }
}

// One CTA of T threads per vertex, Q entries per thread: rows of at most
// T x Q entries, one table of seg_cap(T x Q) slots in shared memory.
template <int T, int Q, typename VT>
__host__ __device__ constexpr size_t cta_tbl_bytes() {
  return row_tbl_bytes<T * Q, VT>();
}

template <typename W, typename ST, int T, int Q>
__global__ void __launch_bounds__(T) lm_cta(LV<W> g, const int32_t* __restrict__ list, int64_t cnt,
                                            int32_t* __restrict__ prop) {
  using VT = typename TblVal<ST>::type;
  constexpr int NW = T / 32, ROW = T * Q, CAP = seg_cap(ROW);
  constexpr uint32_t mask = CAP - 1;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ ST redS[NW];
  __shared__ int32_t redD[NW];
  __shared__ VT redC[NW];
  __shared__ int32_t s_nd;
  int32_t* keys = reinterpret_cast<int32_t*>(smem);
  VT* vals = reinterpret_cast<VT*>(smem + (size_t)CAP * 4);
  uint16_t* slots = reinterpret_cast<uint16_t*>(smem + (size_t)CAP * (4 + sizeof(VT)));
  const int tid = threadIdx.x, lane = lane_id(), wid = tid >> 5;
  for (int s = tid; s < CAP; s += T) {
    keys[s] = -1;
    vals[s] = 0;
  }
  if (tid == 0) s_nd = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x; i < cnt; i += gridDim.x) {
    const int32_t v = list[i];
    const int32_t pv = g.pre_of(v);  // the screening's first-pass proposal
    const int64_t b = g.rp[v];
    const int d = pv < 0 ? (int)(g.rp[v + 1] - b) : 0;
    const int32_t C = g.L[v];
    int32_t lab[Q];
    W wt[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) {
      const int e = q * T + tid;
      lab[q] = -1;
      wt[q] = W(0);
      if (e < d) {
        lab[q] = ld_stream(g.col + b + e);
        wt[q] = ld_stream(g.w + b + e);
      }
    }
#pragma unroll
    for (int q = 0; q < Q; q++) {
      const int32_t u = lab[q];
      lab[q] = (u >= 0 && u != v) ? g.L[u] : -1;
    }
    VT eCl = 0;
#pragma unroll
    for (int q = 0; q < Q; q++) {
      if (q * T < d) {
        const bool isC = lab[q] == C;
        eCl += isC ? (VT)wt[q] : VT(0);
        bool claimed = false;
        uint32_t s = 0;
        if (lab[q] >= 0 && !isC) {
          s = probe_claim(keys, mask, lab[q], claimed);
          atomicAdd(&vals[s], (VT)wt[q]);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, claimed);
        int at = 0;
        if (lane == 0 && bal) at = atomicAdd(&s_nd, __popc(bal));
        at = __shfl_sync(0xffffffffu, at, 0);
        if (claimed) slots[at + __popc(bal & lanemask_lt())] = (uint16_t)s;
      }
    }
    const int64_t ew = seg_total<32>(eCl, 0xffffffffu);
    if (lane == 0) redC[wid] = (VT)ew;
    __syncthreads();
    const int nd = s_nd;
    int64_t eC = 0;
#pragma unroll
    for (int x = 0; x < NW; x++) eC += (int64_t)redC[x];
    const int64_t kv = g.k[v], aC = g.a[C], m2v = g.m2_of(v);
    ST Sb = gain_lowest<ST>();
    int32_t D = INT_MAX;
    for (int j = tid; j < nd; j += T) {
      const uint32_t s = slots[j];
      const int32_t key = keys[s];
      const ST x = gain<ST>(m2v, kv, (int64_t)vals[s], eC, g.a[key], aC);
      if (better(x, key, Sb, D)) {
        Sb = x;
        D = key;
      }
    }
    warp_argmax(Sb, D);
    if (lane == 0) {
      redS[wid] = Sb;
      redD[wid] = D;
    }
    __syncthreads();
    if (wid == 0) {
      Sb = lane < NW ? redS[lane] : gain_lowest<ST>();
      D = lane < NW ? redD[lane] : INT_MAX;
      warp_argmax(Sb, D);
      if (lane == 0) {
        prop[i] = pv >= 0 ? pv : proposal(Sb, D, C, g.size);
        if (g.f_eC) put_features(g, i, eC, keys, vals, mask, Sb, D);
      }
    }
    __syncthreads();
    for (int j = tid; j < nd; j += T) {
      const uint32_t s = slots[j];
      keys[s] = -1;
      vals[s] = 0;
    }
    if (tid == 0) s_nd = 0;
    __syncthreads();
  }
}

// ---------------------------------------------------------------- hub rows
//
// Rows of the hub bin (hub.cuh): hub_agg sums each row into its hub's global
// table, chunk by chunk over many CTAs; then
//   hub_gain    chunk c of hub h: the gains of h's claimed slots in slice c
//               (the distinct labels are at most the degree), CTA argmax into
//               a partial per chunk;
//   hub_pick    warp per hub: argmax of the partials, the proposal;
//   hub_clear   chunk c: empty the slots listed in slice c (the table is
//               clean again for the next pass).

__device__ __forceinline__ void st_part(long long* p, long long S, int32_t D) {
  p[0] = S;
  p[1] = S < 0 ? -1 : 0;
  p[2] = D;
}
__device__ __forceinline__ void st_part(long long* p, i128 S, int32_t D) {
  p[0] = (long long)(unsigned long long)S;
  p[1] = (long long)(unsigned long long)((unsigned __int128)S >> 64);
  p[2] = D;
}
template <typename ST>
__device__ __forceinline__ ST ld_part(const long long* p);
template <>
__device__ __forceinline__ long long ld_part<long long>(const long long* p) {
  return p[0];
}
template <>
__device__ __forceinline__ i128 ld_part<i128>(const long long* p) {
  return (i128)(((unsigned __int128)(unsigned long long)p[1] << 64) | (unsigned long long)p[0]);
}

template <typename W, typename ST>
__global__ void __launch_bounds__(256) hub_gain(LV<W> g, HubTables t) {
  constexpr int NW = 256 / 32;
  __shared__ ST redS[NW];
  __shared__ int32_t redD[NW];
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  const int64_t nch = t.coff[t.H];
  for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
    const int64_t h = hub_of_chunk(t, c);
    const int32_t v = t.list[h];
    const int32_t C = g.L[v];
    const uint32_t mask = (uint32_t)(t.toff[h + 1] - t.toff[h]) - 1;
    const int32_t* keys = t.keys + t.toff[h];
    const unsigned long long* vals = t.vals + t.toff[h];
    const int32_t* slots = t.slots + t.soff[h];
    const int64_t nd = t.nslot[h];
    const int64_t s0 = (c - t.coff[h]) * kHubChunk, s1 = s0 + kHubChunk < nd ? s0 + kHubChunk : nd;
    const int64_t eC = tbl_get(keys, vals, mask, C);
    const int64_t kv = g.k[v], aC = g.a[C], m2v = g.m2_of(v);
    ST S = gain_lowest<ST>();
    int32_t D = INT_MAX;
    for (int64_t j = s0 + threadIdx.x; j < s1; j += blockDim.x) {
      const uint32_t sl = (uint32_t)slots[j];
      const int32_t key = keys[sl];
      if (key != C) {
        const ST x = gain<ST>(m2v, kv, (int64_t)vals[sl], eC, g.a[key], aC);
        if (better(x, key, S, D)) {
          S = x;
          D = key;
        }
      }
    }
    warp_argmax(S, D);
    if (lane == 0) {
      redS[wid] = S;
      redD[wid] = D;
    }
    __syncthreads();
    if (wid == 0) {
      S = lane < NW ? redS[lane] : gain_lowest<ST>();
      D = lane < NW ? redD[lane] : INT_MAX;
      warp_argmax(S, D);
      if (lane == 0) st_part(t.part + 3 * c, S, D);
    }
    __syncthreads();
  }
}

template <typename W, typename ST>
__global__ void __launch_bounds__(256) hub_pick(LV<W> g, HubTables t, int32_t* __restrict__ prop) {
  const int lane = lane_id();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t h = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; h < t.H; h += nw) {
    const int32_t v = t.list[h];
    const int32_t C = g.L[v];
    ST S = gain_lowest<ST>();
    int32_t D = INT_MAX;
    for (int64_t c = t.coff[h] + lane; c < t.coff[h + 1]; c += 32) {
      const ST x = ld_part<ST>(t.part + 3 * c);
      const int32_t y = (int32_t)t.part[3 * c + 2];
      if (better(x, y, S, D)) {
        S = x;
        D = y;
      }
    }
    warp_argmax(S, D);
    const int32_t pv = proposal(S, D, C, g.size);
    if (lane == 0) {
      prop[h] = pv;
      if (g.f_eC) {
        const uint32_t mask = (uint32_t)(t.toff[h + 1] - t.toff[h]) - 1;
        const int32_t* keys = t.keys + t.toff[h];
        const unsigned long long* vals = t.vals + t.toff[h];
        g.f_eC[h] = tbl_get(keys, vals, mask, C);
        g.f_eB[h] = D == INT_MAX ? 0 : tbl_get(keys, vals, mask, D);
        g.f_dB[h] = D == INT_MAX ? -1 : D;
        g.f_sB[h] = D == INT_MAX ? 0.0 : to_double(S);
      }
      t.nprev[h] = t.nslot[h];
      t.nslot[h] = 0;
    }
  }
}

__global__ void __launch_bounds__(256) hub_clear(HubTables t) {
  const int64_t nch = t.coff[t.H];
  for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
    const int64_t h = hub_of_chunk(t, c);
    int32_t* keys = t.keys + t.toff[h];
    unsigned long long* vals = t.vals + t.toff[h];
    const int32_t* slots = t.slots + t.soff[h];
    const int64_t nd = t.nprev[h];
    const int64_t s0 = (c - t.coff[h]) * kHubChunk, s1 = s0 + kHubChunk < nd ? s0 + kHubChunk : nd;
    for (int64_t j = s0 + threadIdx.x; j < s1; j += blockDim.x) {
      const uint32_t sl = (uint32_t)slots[j];
      keys[sl] = -1;
      vals[sl] = 0;
    }
  }
}

// ---------------------------------------------------------------- apply + N

// Moves of one pass (proposals of graphs whose pass loop has stopped are
// dropped).  Community sums change by warp-aggregated atomics (one per distinct
// community of the warp); movers of long rows (list positions from big_from
// on) go to a separate list for block-per-row processing; per-graph mover
// counts feed the stop rule.
__global__ void lm_apply(const int32_t* __restrict__ list, int64_t cnt, int64_t big_from,
                         const int32_t* __restrict__ prop, int32_t* __restrict__ L, const int64_t* __restrict__ k,
                         unsigned long long* __restrict__ a, int32_t* __restrict__ size, int32_t* __restrict__ Lprev,
                         int32_t* __restrict__ mvit, const int32_t* __restrict__ pass_id,
                         int32_t* __restrict__ moved, int32_t* __restrict__ moved_cnt,
                         int32_t* __restrict__ moved_big, int32_t* __restrict__ moved_big_cnt,
                         const int32_t* __restrict__ gid, GraphState* __restrict__ gs) {
  const int32_t iter = *pass_id;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t base0 = (blockIdx.x * (int64_t)blockDim.x) & ~31ll;
  for (int64_t base = base0 + (threadIdx.x & ~31); base < cnt; base += stride) {
    const int64_t i = base + lane_id();
    bool mv = false;
    int32_t v = 0, c = -1, p = -1, gv = -1;
    int64_t kv = 0;
    if (i < cnt) {
      v = list[i];
      p = prop[i];
      c = L[v];
      gv = graph_of(gid, v);
      if (p != c && gs[gv].running) {
        mv = true;
        Lprev[v] = c;
        L[v] = p;
        mvit[v] = iter;
        kv = k[v];
      } else {
        c = p = -1;
      }
    }
    {  // leaving c
      const unsigned peers = __match_any_sync(0xffffffffu, c);
      const int64_t sk = group_sum_exact(peers, kv);
      if (mv && (int)(__ffs(peers) - 1) == (int)lane_id()) {
        atomicAdd(&a[c], 0ull - (unsigned long long)sk);
        atomicSub(&size[c], __popc(peers));
      }
    }
    {  // joining p
      const unsigned peers = __match_any_sync(0xffffffffu, p);
      const int64_t sk = group_sum_exact(peers, kv);
      if (mv && (int)(__ffs(peers) - 1) == (int)lane_id()) {
        atomicAdd(&a[p], (unsigned long long)sk);
        atomicAdd(&size[p], __popc(peers));
      }
    }
    {  // movers per graph
      const unsigned peers = __match_any_sync(0xffffffffu, mv ? gv : -1);
      if (mv && (int)(__ffs(peers) - 1) == (int)lane_id()) atomicAdd(&gs[gv].moves, __popc(peers));
    }
    const bool big = mv && i >= big_from;
    const bool small = mv && !big;
    unsigned bal = __ballot_sync(0xffffffffu, small);
    int32_t slot = 0;
    if (lane_id() == 0 && bal) slot = atomicAdd(moved_cnt, __popc(bal));
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (small) moved[slot + __popc(bal & lanemask_lt())] = v;
    bal = __ballot_sync(0xffffffffu, big);
    slot = 0;
    if (lane_id() == 0 && bal) slot = atomicAdd(moved_big_cnt, __popc(bal));
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (big) moved_big[slot + __popc(bal & lanemask_lt())] = v;
  }
}

// Change of sum_i e_{i->C(i)} from the rows of the moved vertices: an entry
// (x, y) with y unmoved also stands for its mirror (y, x), hence weight 2.
template <typename W>
__device__ __forceinline__ int64_t moved_row_delta(const LV<W>& g, int32_t x, const int32_t* __restrict__ Lprev,
                                                   const int32_t* __restrict__ mvit, int32_t iter, int tid, int nt) {
  const int32_t ox = Lprev[x], nx = g.L[x];
  const int64_t e1 = g.rp[x + 1];
  int64_t acc = 0;
  for (int64_t e = g.rp[x] + tid; e < e1; e += nt) {
    const int32_t y = ld_stream(g.col + e);
    const int64_t wt = (int64_t)ld_stream(g.w + e);
    const bool ym = mvit[y] == iter;
    const int32_t ny = g.L[y];
    const int32_t oy = ym ? Lprev[y] : ny;
    acc += ((int)(nx == ny) - (int)(ox == oy)) * wt * (ym ? 1 : 2);
  }
  return acc;
}

template <typename W>
__global__ void __launch_bounds__(256) lm_delta_in(LV<W> g, const int32_t* __restrict__ moved,
                                                   const int32_t* __restrict__ moved_cnt,
                                                   const int32_t* __restrict__ Lprev, const int32_t* __restrict__ mvit,
                                                   const int32_t* __restrict__ pass_id, GraphState* __restrict__ gs) {
  const int64_t cnt = *moved_cnt;
  const int32_t iter = *pass_id;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < cnt; i += nw) {
    const int32_t x = moved[i];
    const int64_t acc = (int64_t)warp_sum((long long)moved_row_delta(g, x, Lprev, mvit, iter, lane_id(), 32));
    if (lane_id() == 0 && acc != 0) atomicAdd((unsigned long long*)&gs[graph_of(g.gid, x)].in_delta, (unsigned long long)acc);
  }
}

// As lm_delta_in with one CTA per moved vertex (rows above 256 entries).
template <typename W>
__global__ void __launch_bounds__(256) lm_delta_in_block(LV<W> g, const int32_t* __restrict__ moved,
                                                         const int32_t* __restrict__ moved_cnt,
                                                         const int32_t* __restrict__ Lprev,
                                                         const int32_t* __restrict__ mvit,
                                                         const int32_t* __restrict__ pass_id,
                                                         GraphState* __restrict__ gs) {
  const int64_t cnt = *moved_cnt;
  const int32_t iter = *pass_id;
  for (int64_t i = blockIdx.x; i < cnt; i += gridDim.x) {
    const int32_t x = moved[i];
    const int64_t acc = (int64_t)warp_sum((long long)moved_row_delta(g, x, Lprev, mvit, iter, threadIdx.x, blockDim.x));
    if (lane_id() == 0 && acc != 0) atomicAdd((unsigned long long*)&gs[graph_of(g.gid, x)].in_delta, (unsigned long long)acc);
  }
}

__device__ __forceinline__ void add128(unsigned long long* lo, unsigned long long* hi, unsigned __int128 v) {
  const unsigned long long vlo = (unsigned long long)v, vhi = (unsigned long long)(v >> 64);
  if (!(vlo | vhi)) return;
  const unsigned long long old = atomicAdd(lo, vlo);
  const unsigned long long carry = (old + vlo < old) ? 1ull : 0ull;
  if (vhi + carry) atomicAdd(hi, vhi + carry);
}

// sum over labels of a^2 per graph, unsigned 128-bit: every contribution is
// added with a carry into the high word, so the total is exact in any order.
// One graph: a CTA reduction then one addition per CTA; several graphs: one
// addition per community in use.
__global__ void __launch_bounds__(256) sumsq_acc(const int64_t* __restrict__ a, int64_t n,
                                                 const int32_t* __restrict__ gid, GraphState* __restrict__ gs) {
  if (gid) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
      const unsigned long long x = (unsigned long long)a[c];
      if (x) {
        GraphState& G = gs[gid[c]];
        add128(&G.sq_lo, &G.sq_hi, (unsigned __int128)x * x);
      }
    }
    return;
  }
  __shared__ unsigned long long slo[8], shi[8];
  unsigned __int128 s = 0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long x = (unsigned long long)a[c];
    s += (unsigned __int128)x * x;
  }
  unsigned long long lo = (unsigned long long)s, hi = (unsigned long long)(s >> 64);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long lo2 = __shfl_xor_sync(0xffffffffu, lo, o), hi2 = __shfl_xor_sync(0xffffffffu, hi, o);
    unsigned long long nlo = lo + lo2;
    hi = hi + hi2 + (nlo < lo ? 1ull : 0ull);
    lo = nlo;
  }
  if (lane_id() == 0) {
    slo[threadIdx.x >> 5] = lo;
    shi[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned __int128 t = 0;
    for (int w = 0; w < 8; w++) t += ((unsigned __int128)shi[w] << 64) | slo[w];
    add128(&gs[0].sq_lo, &gs[0].sq_hi, t);
  }
}

__device__ __forceinline__ bool below_tau(i128 gain, i128 base, int64_t tau_inv) {
  const i128 y = base < 0 ? -base : base;
  return gain <= y / (i128)tau_inv;
}

__device__ __forceinline__ i128 ld128(const int64_t* lo) {
  return (i128)(((unsigned __int128)(unsigned long long)lo[1] << 64) | (unsigned long long)lo[0]);
}
__device__ __forceinline__ void st128(int64_t* lo, i128 x) {
  lo[0] = (int64_t)(unsigned long long)x;
  lo[1] = (int64_t)(unsigned long long)((unsigned __int128)x >> 64);
}

// Per-pass accumulators back to zero (one thread per graph).
__global__ void gs_reset_pass(GraphState* __restrict__ gs, int G, int32_t* __restrict__ pass_id) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *pass_id += 1;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    gs[g].in_delta = 0;
    gs[g].sq_lo = gs[g].sq_hi = 0;
    gs[g].moves = 0;
  }
}

// The pass decision per graph (one thread per graph).  mode 0: level start
// (N_start = N_cur = m2 in - sq; graphs whose levels are over do not run);
// mode 1: after a pass.  any_running <- some graph goes on.
__global__ void lm_decide(GraphState* __restrict__ gs, int G, int mode, int32_t max_iters, int64_t tau_inv,
                          int32_t* __restrict__ any_running) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    GraphState& X = gs[g];
    const unsigned __int128 sq = ((unsigned __int128)X.sq_hi << 64) | X.sq_lo;
    if (mode == 0) {
      const i128 N = (i128)X.m2 * (i128)X.in_cur - (i128)sq;
      st128(&X.n_cur_lo, N);
      st128(&X.n_start_lo, N);
      X.running = X.done ? 0 : 1;
      X.passes = 0;
      X.moves = 0;
      X.moves_level = 0;
      if (X.running) atomicOr(any_running, 1);
      continue;
    }
    if (!X.running) continue;
    X.passes++;
    X.moves_level += X.moves;
    if (X.moves == 0) {
      X.running = 0;
      continue;
    }
    const int64_t in_new = X.in_cur + X.in_delta;
    const i128 N_new = (i128)X.m2 * (i128)in_new - (i128)sq;
    const i128 N_old = ld128(&X.n_cur_lo);
    X.in_cur = in_new;
    st128(&X.n_cur_lo, N_new);
    if (below_tau(N_new - N_old, N_old, tau_inv) || X.passes >= max_iters) X.running = 0;
    if (X.running) atomicOr(any_running, 1);
  }
}

// ---------------------------------------------------------------- device pass loop
//
// A level's passes run inside one CUDA graph: a 'while' conditional node
// around the pass body.  The body's first and middle kernels stamp the
// global timer; its last kernel adds the pass's evaluation and apply times,
// counts the pass, and keeps the loop going while some graph's pass loop goes
// on (the stop rule of lm_decide).  The stop rule ends every level within
// max_iters passes; the cap here is a second bound that can only be reached
// if that rule were broken, and it is reported.

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void pass_stamp(DevScalars* d, int k) { d->stamp[k] = global_ns(); }

__global__ void pass_end(DevScalars* d, cudaGraphConditionalHandle h, int32_t cap, int in_graph) {
  const unsigned long long t = global_ns();
  d->t_eval_ns += d->stamp[1] - d->stamp[0];
  d->t_apply_ns += t - d->stamp[1];
  d->level_passes += 1;
  const bool more = d->any_running != 0;
  const bool capped = more && d->level_passes >= cap;
  if (capped) d->loop_err = 1;
  // outside a graph the host reads any_running and loop_err after the pass
  if (in_graph) cudaGraphSetConditional(h, (more && !capped) ? 1u : 0u);
}

// ---------------------------------------------------------------- binning

// Active vertices per degree bin, their degree sums and largest degree.  The
// lanes of a warp are grouped by bin (match_any); each group's leader updates
// the warp's own counters (leaders hold distinct bins, so no two update one
// counter), and the warps' counters meet in shared memory, then in global
// memory, once per CTA.
__global__ void __launch_bounds__(256) bin_count(const int64_t* __restrict__ rp, int64_t n,
                                                 const uint8_t* __restrict__ active, DevScalars* d,
                                                 const int32_t* __restrict__ gid,
                                                 const GraphState* __restrict__ gs, BinPlan plan,
                                                 const int32_t* __restrict__ pre) {
  constexpr int NW = 256 / 32;
  __shared__ unsigned long long wc[NW][kMaxBins], wdb[NW][kMaxBins];
  __shared__ long long wmax[NW][kMaxBins];
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  for (int b = lane; b < kMaxBins; b += 32) {
    wc[wid][b] = 0;
    wdb[wid][b] = 0;
    wmax[wid][b] = 0;
  }
  __syncwarp();
  unsigned long long deg_sum = 0, act = 0, pre_deg = 0, pre_cnt = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x) + (threadIdx.x & ~31); base < n; base += stride) {
    const int64_t v = base + lane;
    bool ok = v < n && (!active || active[v]) && (!gid || gs[gid[v]].running);
    const int64_t deg = ok ? rp[v + 1] - rp[v] : 0;
    deg_sum += (unsigned long long)deg;
    act += ok ? 1 : 0;
    // a first-pass proposal from the screening, which the table kernels take
    // (the hub kernels evaluate their rows all the same)
    if (pre && deg > 0 && pre[v] >= 0 && plan.var[bin_of(plan, deg)] != kLmHub) {
      pre_deg += (unsigned long long)deg;
      pre_cnt += 1;
    }
    const int bin = (ok && deg > 0) ? bin_of(plan, deg) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, bin);
    const int64_t ds = group_sum_exact(peers, deg);
    const unsigned mx = __reduce_max_sync(peers, (unsigned)deg);
    if (bin >= 0 && (int)(__ffs(peers) - 1) == lane) {
      wc[wid][bin] += __popc(peers);
      wdb[wid][bin] += (unsigned long long)ds;
      if ((long long)mx > wmax[wid][bin]) wmax[wid][bin] = (long long)mx;
    }
    __syncwarp();
  }
  deg_sum = warp_sum(deg_sum);
  act = warp_sum(act);
  if (pre) {
    pre_deg = warp_sum(pre_deg);
    pre_cnt = warp_sum(pre_cnt);
    if (lane == 0 && pre_cnt) {
      atomicAdd((unsigned long long*)&d->pre_deg, pre_deg);
      atomicAdd((unsigned long long*)&d->pre_verts, pre_cnt);
    }
  }
  __syncthreads();
  if (threadIdx.x < plan.nb) {
    const int b = threadIdx.x;
    unsigned long long c = 0, db = 0;
    long long mx = 0;
    for (int x = 0; x < NW; x++) {
      c += wc[x][b];
      db += wdb[x][b];
      mx = wmax[x][b] > mx ? wmax[x][b] : mx;
    }
    if (c) {
      atomicAdd((unsigned long long*)&d->bcnt[b], c);
      atomicAdd((unsigned long long*)&d->bdeg[b], db);
      atomicMax((long long*)&d->bmax[b], mx);
    }
  }
  if (lane == 0 && act) {
    atomicAdd((unsigned long long*)&d->act_deg, deg_sum);
    atomicAdd((unsigned long long*)&d->ncomm, act);
  }
}

__global__ void bin_scatter(const int64_t* __restrict__ rp, int64_t n, const uint8_t* __restrict__ active,
                            const DevScalars* __restrict__ d, int32_t* __restrict__ cursor,
                            int32_t* __restrict__ list, const int32_t* __restrict__ gid,
                            const GraphState* __restrict__ gs, BinPlan plan) {
  __shared__ int32_t off[kMaxBins];
  if (threadIdx.x == 0) {
    int64_t o = 0;
    for (int b = 0; b < plan.nb; b++) {
      off[b] = (int32_t)o;
      o += d->bcnt[b];
    }
  }
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t base0 = (blockIdx.x * (int64_t)blockDim.x) + (threadIdx.x & ~31);
  for (int64_t base = base0; base < n; base += stride) {
    const int64_t v = base + lane_id();
    int bin = -1;
    if (v < n && (!active || active[v]) && (!gid || gs[gid[v]].running)) {
      const int64_t deg = rp[v + 1] - rp[v];
      if (deg > 0) bin = bin_of(plan, deg);
    }
    for (int b = 0; b < plan.nb; b++) {
      const unsigned bal = __ballot_sync(0xffffffffu, bin == b);
      if (!bal) continue;
      int32_t slot = 0;
      if (lane_id() == 0) slot = atomicAdd(&cursor[b], __popc(bal));
      slot = __shfl_sync(0xffffffffu, slot, 0);
      if (bin == b) list[off[b] + slot + __popc(bal & lanemask_lt())] = (int32_t)v;
    }
  }
}

// ---------------------------------------------------------------- sums

// a_C and |C| of every label: each warp groups its 32 vertices by label,
// each CTA adds the group sums into a shared table (labels of a CTA repeat
// heavily when communities are large), and the table goes to global memory
// once per CTA; labels that find no slot within a few probes go there
// directly.
constexpr int kCsSlots = 2048;
constexpr int kCsThreads = 1024;

__global__ void __launch_bounds__(kCsThreads) comm_sums(int64_t n, const int32_t* __restrict__ L,
                                                        const int64_t* __restrict__ k,
                                                        unsigned long long* __restrict__ a, int32_t* __restrict__ size) {
  __shared__ int32_t tk[kCsSlots];
  __shared__ int32_t tc[kCsSlots];
  __shared__ unsigned long long tv[kCsSlots];
  for (int x = threadIdx.x; x < kCsSlots; x += blockDim.x) {
    tk[x] = -1;
    tc[x] = 0;
    tv[x] = 0;
  }
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x) + (threadIdx.x & ~31); base < n; base += stride) {
    const int64_t v = base + lane_id();
    const int32_t c = v < n ? L[v] : -1;
    const int64_t kv = v < n ? k[v] : 0;
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    const int64_t sk = group_sum_exact(peers, kv);
    if (c >= 0 && (int)(__ffs(peers) - 1) == (int)lane_id()) {
      uint32_t sl = hash_label(c, kCsSlots - 1);
      bool done = false;
      for (int probe = 0; probe < 8 && !done; probe++) {
        const int32_t key = tk[sl];
        if (key == c) {
          done = true;
        } else if (key == -1) {
          const int32_t old = atomicCAS(&tk[sl], -1, c);
          done = old == -1 || old == c;
        }
        if (done) {
          atomicAdd(&tv[sl], (unsigned long long)sk);
          atomicAdd(&tc[sl], __popc(peers));
        }
        sl = (sl + 1) & (kCsSlots - 1);
      }
      if (!done) {
        atomicAdd(&a[c], (unsigned long long)sk);
        atomicAdd(&size[c], __popc(peers));
      }
    }
  }
  __syncthreads();
  for (int x = threadIdx.x; x < kCsSlots; x += blockDim.x)
    if (tk[x] >= 0) {
      atomicAdd(&a[tk[x]], tv[x]);
      atomicAdd(&size[tk[x]], tc[x]);
    }
}

__global__ void fill_iota(int32_t* __restrict__ x, int64_t n) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    x[v] = (int32_t)v;
}

__global__ void fill_i32(int32_t* __restrict__ x, int64_t n, int32_t val) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    x[v] = val;
}

// ---------------------------------------------------------------- compaction

__global__ void mark_used(int64_t n, const int32_t* __restrict__ L, int32_t* __restrict__ used) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    if (!used[L[v]]) used[L[v]] = 1;  // a read first: most labels are already marked
}

// The same flags from the tracked community sizes: label x is used iff
// |x| > 0.  A coalesced pass over the labels, where mark_used writes a few
// hundred hot addresses from every vertex when communities are large.
__global__ void used_from_size(int64_t n, const int32_t* __restrict__ size, int32_t* __restrict__ used) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
    used[x] = size[x] > 0 ? 1 : 0;
}

// Row of entry e for the entry-linear walks below: a warp walks a range of
// consecutive entries, finds the row of its first entry by binary search,
// then advances 32 entries at a time with the row ends of the next 32 rows
// in its lanes.
struct RowWalk {
  int64_t r;     // row of the chunk's first entry
  int64_t rb;    // lane i holds the end of row rb + i (valid while chunks stay below `last`)
  int64_t bk, last;
  __device__ __forceinline__ void load(const int64_t* __restrict__ rp, int64_t n, int64_t r0) {
    rb = r0;
    bk = (r0 + 1 + lane_id() <= n) ? rp[r0 + 1 + lane_id()] : INT64_MAX;
    last = __shfl_sync(0xffffffffu, bk, 31);
  }
  __device__ __forceinline__ void start(const int64_t* __restrict__ rp, int64_t n, int64_t E0) {
    int64_t x = 0;
    if (lane_id() == 0) {  // last row whose start is <= E0
      int64_t lo = 0, hi = n - 1;
      while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (rp[mid] <= E0) lo = mid; else hi = mid - 1;
      }
      x = lo;
    }
    r = __shfl_sync(0xffffffffu, x, 0);
    load(rp, n, r);
  }
  // row of entry c0 + lane (entries past the segment get the last row); the
  // ends of 32 rows stay in the lanes across chunks and are reloaded only when
  // a chunk runs past them
  __device__ __forceinline__ int64_t row(const int64_t* __restrict__ rp, int64_t n, int64_t c0, bool valid) {
    const int lane = lane_id();
    const int64_t e = c0 + lane;
    if (last <= c0 + 31) load(rp, n, r);
    int64_t rw;
    if (last <= c0 + 31) {
      // more than 31 rows end inside this chunk (empty rows): search per lane
      int64_t lo = r, hi = n - 1, x = valid ? e : c0;
      while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (rp[mid] <= x) lo = mid; else hi = mid - 1;
      }
      rw = lo;
    } else {
      int cntv = 0;
      const int64_t x = valid ? e : c0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int64_t v = __shfl_sync(0xffffffffu, bk, cntv + step - 1);
        if (v <= x) cntv += step;
      }
      rw = rb + cntv;
    }
    r = __shfl_sync(0xffffffffu, rw, 31);
    return rw;
  }
};

// Coarse entries of one level (sort path): every entry (u, y, w) becomes the
// key cid(L(u)) * nc + cid(L(y)) with weight w.  Equal keys are summed twice
// before they are written: within a warp's 32-entry chunk (match_any + redux),
// then across the warp's whole range of entries in a warp-private hash table
// in shared memory (the chunk's leaders hold distinct keys, so their updates
// of the table never contend).  A warp writes its table out when it passes
// half full, and at the end.  A level that collapses into few communities --
// level 0 of a step that starts from the previous step's communities -- then
// writes a few hundred pairs per warp instead of one per chunk, and the sort
// that follows has little to do.
constexpr int kEmitThreads = 256;

// Warp table slots: 512 when key and sum are 32-bit (4 KB a warp), 256
// otherwise, so a CTA's tables stay within 48 KB of static shared memory.
template <typename KT, typename VT>
__host__ __device__ constexpr int emit_slots() {
  return sizeof(KT) + sizeof(VT) == 8 ? 512 : 256;
}
template <int BITS>
__device__ __forceinline__ uint32_t emit_hash(uint32_t k) {
  return (k * 0x9E3779B1u) >> (32 - BITS);
}
template <int BITS>
__device__ __forceinline__ uint32_t emit_hash(unsigned long long k) {
  return (uint32_t)((k * 0x9E3779B97F4A7C15ull) >> (64 - BITS));
}

template <typename W, typename KT, typename VT>
__global__ void __launch_bounds__(kEmitThreads) emit_coarse(int64_t n, int64_t m, const int64_t* __restrict__ rp,
                                                            const int32_t* __restrict__ col,
                                                            const W* __restrict__ w,
                                                            const int32_t* __restrict__ ccid, uint64_t nc,
                                                            int64_t per_warp, uint64_t* __restrict__ keys,
                                                            uint64_t* __restrict__ vals,
                                                            unsigned long long* __restrict__ count) {
  constexpr int NW = kEmitThreads / 32;
  constexpr KT kEmpty = ~KT(0);
  constexpr int kSlots = emit_slots<KT, VT>();
  constexpr int kBits = kSlots == 512 ? 9 : 8;
  static_assert(kSlots == (1 << kBits), "hash bits");
  __shared__ KT stk[NW][kSlots];
  __shared__ VT stv[NW][kSlots];
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  KT* tk = stk[wid];
  VT* tv = stv[wid];
  for (int s = lane; s < kSlots; s += 32) {
    tk[s] = kEmpty;
    tv[s] = 0;
  }
  __syncwarp();
  int used = 0;  // slots in use (warp-uniform)
  // write the table's pairs out (one output reservation per 32 slots) and
  // empty it
  auto flush = [&]() {
    __syncwarp();
    for (int s0 = 0; s0 < kSlots; s0 += 32) {
      const int s = s0 + lane;
      const KT k = tk[s];
      const bool occ = k != kEmpty;
      const unsigned bal = __ballot_sync(0xffffffffu, occ);
      unsigned long long at = 0;
      if (lane == 0 && bal) at = atomicAdd(count, (unsigned long long)__popc(bal));
      at = __shfl_sync(0xffffffffu, at, 0);
      if (occ) {
        const unsigned long long pos = at + __popc(bal & lanemask_lt());
        keys[pos] = (uint64_t)k;
        vals[pos] = (uint64_t)tv[s];
        tk[s] = kEmpty;
        tv[s] = 0;
      }
    }
    __syncwarp();
    used = 0;
  };
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t W0 = gw * per_warp, W1 = W0 + per_warp < m ? W0 + per_warp : m;
  if (W0 < W1) {
    RowWalk rw;
    rw.start(rp, n, W0);
    for (int64_t c0 = W0; c0 < W1; c0 += 32) {
      const int64_t e = c0 + lane;
      const bool valid = e < W1;
      const int64_t row = rw.row(rp, n, c0, valid);
      KT key = kEmpty;
      W wt = W(0);
      if (valid) {
        key = (KT)((uint64_t)ccid[row] * nc + (uint64_t)ccid[col[e]]);
        wt = w[e];
      }
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      // VT = 32 bits: 2m < 2^31 bounds every sum of weights
      const VT sum = sizeof(VT) == 4 ? (VT)__reduce_add_sync(peers, (unsigned)wt)
                                     : (VT)group_sum_exact(peers, (int64_t)wt);
      const bool lead = valid && (int)(__ffs(peers) - 1) == lane;
      bool claimed = false;
      if (lead) {
        // leaders hold distinct keys, so a slot is claimed by at most one of
        // them, and each adds to its own slot
        uint32_t s = emit_hash<kBits>(key);
        for (;;) {
          const KT k = tk[s];
          if (k == key) break;
          if (k == kEmpty && atomicCAS(&tk[s], kEmpty, key) == kEmpty) {
            claimed = true;
            break;
          }
          s = (s + 1) & (kSlots - 1);
        }
        tv[s] += sum;
      }
      __syncwarp();
      // at most 32 new keys a chunk: flushing above half minus one chunk keeps
      // the table at most half full, so every probe ends
      used += __popc(__ballot_sync(0xffffffffu, claimed));
      if (used > kSlots / 2 - 32) flush();
    }
  }
  flush();
}

// Dense coarsening, for levels that collapse into at most kDenseNc
// communities (level 0 of a Delta-screening step starts from the previous
// step's communities): the coarse graph is an nc x nc matrix of sums that
// stays in L2.  Warps walk the fine entries as emit_coarse does, sum equal
// keys of a 32-entry chunk with match_any + redux, and the chunk's leaders
// add straight into the matrix; two row-per-warp passes then count and write
// the non-zero cells in column order.  No key list, no sort.
constexpr int64_t kDenseNc = 4096;
constexpr size_t kDenseSmem = 96 * 1024;  // the CTA copy of the matrix (emit_dense<..., true>)

// SMEM: the CTA first sums into its own copy of the matrix in shared memory
// (nc x nc cells, for the smallest nc) and adds its non-zero cells into the
// global matrix once at the end.  A level-0 matrix receives most of its
// weight in the nc diagonal cells, and without the CTA copy every row's
// chunks would queue on those few L2 lines.
template <typename W, typename VT, bool SMEM>
__global__ void __launch_bounds__(kEmitThreads) emit_dense(int64_t n, int64_t m, const int64_t* __restrict__ rp,
                                                           const int32_t* __restrict__ col,
                                                           const W* __restrict__ w,
                                                           const int32_t* __restrict__ ccid, uint32_t nc,
                                                           int64_t per_warp, VT* __restrict__ dense) {
  extern __shared__ __align__(16) unsigned char smem[];
  VT* local = reinterpret_cast<VT*>(smem);
  const uint32_t cells = nc * nc;
  if (SMEM) {
    for (uint32_t x = threadIdx.x; x < cells; x += blockDim.x) local[x] = 0;
    __syncthreads();
  }
  const int lane = lane_id();
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t W0 = gw * per_warp, W1 = W0 + per_warp < m ? W0 + per_warp : m;
  if (W0 < W1) {
    RowWalk rw;
    rw.start(rp, n, W0);
    for (int64_t c0 = W0; c0 < W1; c0 += 32) {
      const int64_t e = c0 + lane;
      const bool valid = e < W1;
      const int64_t row = rw.row(rp, n, c0, valid);
      uint32_t key = 0xffffffffu;
      W wt = W(0);
      if (valid) {
        key = (uint32_t)ccid[row] * nc + (uint32_t)ccid[col[e]];
        wt = w[e];
      }
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      // VT = 32 bits: 2m < 2^31 bounds every sum of weights
      const VT sum = sizeof(VT) == 4 ? (VT)__reduce_add_sync(peers, (unsigned)wt)
                                     : (VT)group_sum_exact(peers, (int64_t)wt);
      if (valid && (int)(__ffs(peers) - 1) == lane) atomicAdd(SMEM ? &local[key] : &dense[key], sum);
    }
  }
  if (SMEM) {
    __syncthreads();
    for (uint32_t x = threadIdx.x; x < cells; x += blockDim.x)
      if (local[x]) atomicAdd(&dense[x], local[x]);
  }
}

// Non-zero cells of each matrix row (a warp a row).
template <typename VT>
__global__ void dense_count(const VT* __restrict__ dense, int64_t nc, int64_t* __restrict__ rowcnt) {
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < nc; r += nw) {
    int64_t cnt = 0;
    for (int64_t c0 = 0; c0 < nc; c0 += 32) {
      const int64_t cc = c0 + lane_id();
      cnt += __popc(__ballot_sync(0xffffffffu, cc < nc && dense[r * nc + cc] != 0));
    }
    if (lane_id() == 0) rowcnt[r] = cnt;
  }
}

// The non-zero cells written as the coarse CSR (columns ascending).
template <typename VT>
__global__ void dense_write(const VT* __restrict__ dense, int64_t nc, const int64_t* __restrict__ rp,
                            int32_t* __restrict__ ccol, int64_t* __restrict__ cw) {
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < nc; r += nw) {
    int64_t pos = rp[r];
    for (int64_t c0 = 0; c0 < nc; c0 += 32) {
      const int64_t cc = c0 + lane_id();
      const VT x = cc < nc ? dense[r * nc + cc] : VT(0);
      const unsigned bal = __ballot_sync(0xffffffffu, x != 0);
      if (x != 0) {
        const int64_t at = pos + __popc(bal & lanemask_lt());
        ccol[at] = (int32_t)cc;
        cw[at] = (int64_t)x;
      }
      pos += __popc(bal);
    }
  }
}

// coarse vertex of every vertex: cid of its label (one gather per entry in the
// emit instead of two dependent ones)
__global__ void coarse_of(int64_t n, const int32_t* __restrict__ L, const int32_t* __restrict__ cid,
                          int32_t* __restrict__ ccid) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    ccid[v] = cid[L[v]];
}

__global__ void key_heads(const uint64_t* __restrict__ keys, int64_t m, int32_t* __restrict__ head) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    head[e] = (e == 0 || keys[e] != keys[e - 1]) ? 1 : 0;
}

// Sum of each run of equal keys: a thread folds 16 consecutive entries and
// flushes one atomic per run piece.  Also writes the coarse column and the
// per-row entry counts at run heads.
constexpr int kRunItems = 16;
__global__ void reduce_runs(const uint64_t* __restrict__ keys, const uint64_t* __restrict__ vals, int64_t m,
                            uint64_t nc, const int32_t* __restrict__ head, const int32_t* __restrict__ uid,
                            unsigned long long* __restrict__ cw, int32_t* __restrict__ ccol,
                            int64_t* __restrict__ rowcnt) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t e0 = t * kRunItems;
  if (e0 >= m) return;
  const int64_t e1 = e0 + kRunItems < m ? e0 + kRunItems : m;
  int32_t cur = -1;
  unsigned long long acc = 0;
  for (int64_t e = e0; e < e1; e++) {
    const int32_t id = uid[e];
    if (head[e]) {
      ccol[id] = (int32_t)(keys[e] % nc);
      atomicAdd((unsigned long long*)&rowcnt[keys[e] / nc], 1ull);
    }
    if (id != cur) {
      if (cur >= 0) atomicAdd(&cw[cur], acc);
      cur = id;
      acc = 0;
    }
    acc += vals[e];
  }
  if (cur >= 0) atomicAdd(&cw[cur], acc);
}

__global__ void gs_reset_nc(GraphState* __restrict__ gs, int G) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    gs[g].nc = 0;
    gs[g].ncomm = 0;
  }
}

// Labels in use per graph (after the used-label scan: c is used when
// cid[c + 1] != cid[c]) and the graph of every coarse vertex.
__global__ void count_used(int64_t n, const int32_t* __restrict__ cid, const int32_t* __restrict__ gid,
                           GraphState* __restrict__ gs, int32_t* __restrict__ gid_next) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x) + (threadIdx.x & ~31); base < n; base += stride) {
    const int64_t c = base + lane_id();
    const bool used = c < n && cid[c + 1] != cid[c];
    const int g = used ? graph_of(gid, c) : -1;
    if (used && gid_next) gid_next[cid[c]] = g;
    const unsigned peers = __match_any_sync(0xffffffffu, g);
    if (used && (int)(__ffs(peers) - 1) == (int)lane_id())
      atomicAdd((unsigned long long*)&gs[g].nc, (unsigned long long)__popc(peers));
  }
}

// k of a coarse vertex = a of its community; compose the original vertices.
__global__ void coarse_k(int64_t n, const int32_t* __restrict__ cid, const int64_t* __restrict__ a,
                         int64_t* __restrict__ kc) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
    if (cid[c + 1] != cid[c]) kc[cid[c]] = a[c];
}

__global__ void compose(int64_t n0, int32_t* __restrict__ comp, const int32_t* __restrict__ L,
                        const int32_t* __restrict__ cid) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n0; v += (int64_t)gridDim.x * blockDim.x)
    comp[v] = cid[L[comp[v]]];
}

// ---------------------------------------------------------------- finish

__global__ void final_min(int64_t n0, const int32_t* __restrict__ comp, const int32_t* __restrict__ L,
                          int32_t* __restrict__ minid) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x) + (threadIdx.x & ~31); base < n0; base += stride) {
    const int64_t v = base + lane_id();
    const int32_t c = v < n0 ? L[comp[v]] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    const unsigned mn = __reduce_min_sync(peers, v < n0 ? (unsigned)v : 0xffffffffu);
    // labels of large communities repeat across the grid: read first, and
    // only a smaller id pays for the atomic
    if (c >= 0 && (int)(__ffs(peers) - 1) == (int)lane_id() && (int32_t)mn < minid[c])
      atomicMin(&minid[c], (int32_t)mn);
  }
}

// Canonical labels (smallest member id, a vertex id of the context) and the
// number of communities per graph.
__global__ void final_labels(int64_t n0, const int32_t* __restrict__ comp, const int32_t* __restrict__ L,
                             const int32_t* __restrict__ minid, int32_t* __restrict__ out,
                             const int32_t* __restrict__ gid, GraphState* __restrict__ gs) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x) + (threadIdx.x & ~31); base < n0; base += stride) {
    const int64_t v = base + lane_id();
    int g = -1;
    bool head = false;
    if (v < n0) {
      const int32_t x = minid[L[comp[v]]];
      head = x == (int32_t)v;
      g = graph_of(gid, v);
      out[v] = x;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, head ? g : -1);
    if (head && (int)(__ffs(peers) - 1) == (int)lane_id())
      atomicAdd((unsigned long long*)&gs[g].ncomm, (unsigned long long)__popc(peers));
  }
}

// ---------------------------------------------------------------- host side

inline i128 h128(int64_t lo, int64_t hi) {
  return (i128)(((unsigned __int128)(unsigned long long)hi << 64) | (unsigned long long)lo);
}

inline bool h_below_tau(i128 gain, i128 base, int64_t tau_inv) {
  i128 y = base < 0 ? -base : base;
  return gain <= y / (i128)tau_inv;
}

// State of one level (labels, sums, scratch) and its pass loop.
struct LevelRun {
  int64_t passes = 0, moves = 0, edges = 0, verts = 0;
  float ms_lm = 0.f, ms_apply = 0.f;
  float ms_bin[4] = {0.f, 0.f, 0.f, 0.f};
  int64_t edges_bin[4] = {0, 0, 0, 0}, verts_bin[4] = {0, 0, 0, 0};
  int64_t edges_pre = 0, verts_pre = 0;  // first-pass evaluations the screening supplied
};

// Degree bins of the active vertices of one level and the hub tables.
struct Bins {
  BinPlan plan;
  Buf<int32_t> list;
  int64_t cnt[kMaxBins] = {}, deg[kMaxBins] = {}, maxd[kMaxBins] = {}, off[kMaxBins + 1] = {};
  int64_t total = 0, act_deg = 0, n_active = 0;
  int64_t pre_verts = 0, pre_deg = 0;  // of them, first-pass proposals from the screening
  HubBufs hub;  // tables of the hub bin (hub.cuh)
};

template <typename W>
int make_bins(dcd_ctx* c, const Csr<W>& g, const uint8_t* active, Bins* b, const int32_t* gid = nullptr,
              const int32_t* pre = nullptr) {
  cudaStream_t s = c->stream;
  DevScalars* d = c->dsc.get();
  const int64_t nv = g.n;
  const int T = 256;
  b->plan = c->bin_plan;
  const BinPlan& plan = b->plan;
  DCD_TRY_CUDA(cudaMemsetAsync(&d->act_deg, 0, 2 * sizeof(int64_t), s));  // act_deg, ncomm
  DCD_TRY_CUDA(cudaMemsetAsync(&d->bcnt[0], 0, 3 * kMaxBins * sizeof(int64_t), s));  // bcnt, bdeg, bmax
  DCD_TRY_CUDA(cudaMemsetAsync(&d->pre_verts, 0, 2 * sizeof(int64_t), s));           // pre_verts, pre_deg
  ::dcd::count_launch(), bin_count<<<grid_for(nv, T), T, 0, s>>>(g.rp, nv, active, d, gid, c->gs.get(), plan, pre);
  DCD_LAUNCH_CHECK();
  DCD_TRY_CUDA(cudaMemcpyAsync(c->hsc, d, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
  DCD_TRY_CUDA(cudaStreamSynchronize(s));
  b->total = 0;
  for (int x = 0; x < plan.nb; x++) {
    b->cnt[x] = c->hsc->bcnt[x];
    b->deg[x] = c->hsc->bdeg[x];
    b->maxd[x] = c->hsc->bmax[x];
    b->off[x] = b->total;
    b->total += b->cnt[x];
  }
  b->off[plan.nb] = b->total;
  b->act_deg = c->hsc->act_deg;
  b->n_active = c->hsc->ncomm;  // bin_count leaves the active count here
  b->pre_verts = c->hsc->pre_verts;
  b->pre_deg = c->hsc->pre_deg;
  Buf<int32_t> cursor;
  DCD_TRY(b->list.alloc(&c->mem, b->total));
  DCD_TRY(cursor.alloc(&c->mem, kMaxBins));
  DCD_TRY_CUDA(cudaMemsetAsync(cursor.get(), 0, kMaxBins * sizeof(int32_t), s));
  if (b->total > 0) {
    ::dcd::count_launch(), bin_scatter<<<grid_for(nv, T), T, 0, s>>>(g.rp, nv, active, d, cursor.get(),
                                                                       b->list.get(), gid, c->gs.get(), plan);
    DCD_LAUNCH_CHECK();
  }
  // tables of the hub bin: a region per hub, sized by its degree
  for (int x = 0; x < plan.nb; x++)
    if (plan.var[x] == kLmHub && b->cnt[x])
      DCD_TRY(hub_setup(c, b->list.get() + b->off[x], b->cnt[x], g.rp, &b->hub));
  return DCD_OK;
}

template <typename W, typename ST, int S, int Q>
constexpr size_t seg_smem() {
  return (size_t)8 * (32 / S) * row_tbl_bytes<S * Q, typename TblVal<ST>::type>();
}

template <typename W, typename ST, int S, int Q>
int launch_seg(cudaStream_t s, const LV<W>& g, const int32_t* lst, int64_t cnt, int32_t* prop, int64_t* sweep) {
  constexpr int T = 256, P = 32 / S;
  constexpr size_t smem = seg_smem<W, ST, S, Q>();
  const int grid = wave_grid(lm_seg<W, ST, S, Q>, cdiv(cnt, P) * 32, T, smem);
  *sweep = (int64_t)grid * (T / 32) * P;
  count_launch(), lm_seg<W, ST, S, Q><<<grid, T, smem, s>>>(g, lst, cnt, prop);
  return DCD_OK;
}

template <typename W, typename ST, int T, int Q>
int launch_cta(cudaStream_t s, const LV<W>& g, const int32_t* lst, int64_t cnt, int32_t* prop, int64_t* sweep) {
  constexpr size_t smem = cta_tbl_bytes<T, Q, typename TblVal<ST>::type>();
  const int grid = wave_grid(lm_cta<W, ST, T, Q>, cnt * T, T, smem);
  *sweep = grid;
  count_launch(), lm_cta<W, ST, T, Q><<<grid, T, smem, s>>>(g, lst, cnt, prop);
  return DCD_OK;
}

template <typename K>
int table_kernel_attrs(K* kernel, int threads, size_t smem) {
  DCD_TRY_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  DCD_TRY_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    (int)cudaSharedmemCarveoutMaxShared));
  // occupancy of the grid-stride kernel, looked up here so that no query runs
  // while a pass is being captured
  resident_blocks(reinterpret_cast<const void*>(kernel), threads, smem);
  return DCD_OK;
}

// Shared-memory limits and occupancy of the table kernels (host calls, made
// before any launch and outside stream capture).
template <typename W, typename ST>
int prepare_lm_st() {
  using VT = typename TblVal<ST>::type;
  DCD_TRY(table_kernel_attrs(lm_seg<W, ST, 8, 2>, 256, seg_smem<W, ST, 8, 2>()));
  DCD_TRY(table_kernel_attrs(lm_seg<W, ST, 16, 2>, 256, seg_smem<W, ST, 16, 2>()));
  DCD_TRY(table_kernel_attrs(lm_seg<W, ST, 16, 4>, 256, seg_smem<W, ST, 16, 4>()));
  DCD_TRY(table_kernel_attrs(lm_seg<W, ST, 32, 4>, 256, seg_smem<W, ST, 32, 4>()));
  DCD_TRY(table_kernel_attrs(lm_seg<W, ST, 32, 8>, 256, seg_smem<W, ST, 32, 8>()));
  DCD_TRY(table_kernel_attrs(lm_cta<W, ST, 128, 4>, 128, cta_tbl_bytes<128, 4, VT>()));
  DCD_TRY(table_kernel_attrs(lm_cta<W, ST, 256, 4>, 256, cta_tbl_bytes<256, 4, VT>()));
  DCD_TRY(table_kernel_attrs(lm_cta<W, ST, 512, 4>, 512, cta_tbl_bytes<512, 4, VT>()));
  DCD_TRY(table_kernel_attrs(lm_cta<W, ST, 512, 8>, 512, cta_tbl_bytes<512, 8, VT>()));
  return DCD_OK;
}

// One local-move evaluation of every binned vertex (proposals in prop[]);
// bin_ev[x] is recorded after bin x (with ev_flags: external records inside
// stream capture).  With fork, the bins run side by side: they read the same
// labels and sums and write disjoint slices of prop[], so each non-empty bin
// runs on a side stream of its own between a fork from and a join to the
// context stream, between c->bin_start[x] and bin_ev[x] (the ramp-up and tail
// of one bin's kernels overlap the others'; a small bin fills SMs a large one
// leaves idle).
template <typename W, typename ST>
int launch_lm_bins(dcd_ctx* c, const LV<W>& lv, Bins& b, int32_t* prop, cudaEvent_t* bin_ev, unsigned ev_flags,
                   bool fork, unsigned* forked, int64_t* sweep_out) {
  int64_t sweep_tmp[kMaxBins];
  int64_t* sweep = sweep_out ? sweep_out : sweep_tmp;
  const cudaStream_t s0 = c->stream;
  const int T = 256;
  const int32_t* lst0 = b.list.get();
  if (fork) DCD_TRY_CUDA(cudaEventRecord(c->fork_ev, s0));
  for (int x = 0; x < b.plan.nb; x++) {
    const int64_t cnt = b.cnt[x], o = b.off[x];
    const cudaStream_t s = fork && cnt ? c->side[x] : s0;
    if (fork && cnt) {
      DCD_TRY_CUDA(cudaStreamWaitEvent(s, c->fork_ev, 0));
      *forked |= 1u << x;
    }
    // a bin's interval starts on its own stream (forked or not), so every
    // interval the caller times has both its events recorded
    if (bin_ev) DCD_TRY_CUDA(cudaEventRecordWithFlags(c->bin_start[x], s, ev_flags));
    if (cnt) {
      LV<W> g = lv;  // feature outputs shifted to the bin's list offset
      if (g.f_eC) {
        g.f_eC += o;
        g.f_eB += o;
        g.f_dB += o;
        g.f_sB += o;
      }
      const int32_t* lst = lst0 + o;
      int32_t* pr = prop + o;
      switch (b.plan.var[x]) {
        case kLmSeg16: DCD_TRY((launch_seg<W, ST, 8, 2>(s, g, lst, cnt, pr, &sweep[x]))); break;
        case kLmSeg32: DCD_TRY((launch_seg<W, ST, 16, 2>(s, g, lst, cnt, pr, &sweep[x]))); break;
        case kLmSeg64: DCD_TRY((launch_seg<W, ST, 16, 4>(s, g, lst, cnt, pr, &sweep[x]))); break;
        case kLmWarp128: DCD_TRY((launch_seg<W, ST, 32, 4>(s, g, lst, cnt, pr, &sweep[x]))); break;
        case kLmWarp256: DCD_TRY((launch_seg<W, ST, 32, 8>(s, g, lst, cnt, pr, &sweep[x]))); break;
        case kLmCta512: DCD_TRY((launch_cta<W, ST, 128, 4>(s, g, lst, cnt, pr, &sweep[x]))); break;
        case kLmCta1k: DCD_TRY((launch_cta<W, ST, 256, 4>(s, g, lst, cnt, pr, &sweep[x]))); break;
        case kLmCta2k: DCD_TRY((launch_cta<W, ST, 512, 4>(s, g, lst, cnt, pr, &sweep[x]))); break;
        case kLmCta4k: DCD_TRY((launch_cta<W, ST, 512, 8>(s, g, lst, cnt, pr, &sweep[x]))); break;
        default: {
          sweep[x] = cnt;
          const unsigned ch = hub_grid(c, b.hub);
          count_launch(), hub_agg<W, ST><<<ch, 256, 0, s>>>(g, b.hub.t);
          count_launch(), hub_gain<W, ST><<<ch, 256, 0, s>>>(g, b.hub.t);
          count_launch(), hub_pick<W, ST><<<grid_for(cnt * 32, T), T, 0, s>>>(g, b.hub.t, pr);
          count_launch(), hub_clear<<<ch, 256, 0, s>>>(b.hub.t);
          break;
        }
      }
      DCD_LAUNCH_CHECK();
    }
    if (bin_ev) DCD_TRY_CUDA(cudaEventRecordWithFlags(bin_ev[x], s, ev_flags));
    if (fork && cnt) {
      DCD_TRY_CUDA(cudaEventRecord(c->join_ev[x], s));
      DCD_TRY_CUDA(cudaStreamWaitEvent(s0, c->join_ev[x], 0));
      *forked &= ~(1u << x);
    }
  }
  return DCD_OK;
}

template <typename W, typename ST>
int launch_lm_st(dcd_ctx* c, const LV<W>& lv, Bins& b, int32_t* prop, cudaEvent_t* bin_ev, unsigned ev_flags,
                 bool fork = false, int64_t* sweep = nullptr) {
  unsigned forked = 0;
  const int rc = launch_lm_bins<W, ST>(c, lv, b, prop, bin_ev, ev_flags, fork, &forked, sweep);
  // an error between a fork and its join: join the side streams all the same,
  // so that a stream capture in progress ends with every stream back home
  for (int x = 0; x < kMaxBins; x++)
    if (forked & (1u << x)) {
      cudaEventRecord(c->join_ev[x], c->side[x]);
      cudaStreamWaitEvent(c->stream, c->join_ev[x], 0);
    }
  return rc;
}

template <typename W>
int prepare_lm(const LV<W>& lv) {
  if (lv.m2 >= ((int64_t)1 << 31)) return prepare_lm_st<W, i128>();
  return prepare_lm_st<W, long long>();
}

template <typename W>
int launch_lm(dcd_ctx* c, const LV<W>& lv, Bins& b, int32_t* prop, cudaEvent_t* bin_ev = nullptr,
              unsigned ev_flags = 0) {
  DCD_TRY(prepare_lm<W>(lv));
  if (lv.m2 >= ((int64_t)1 << 31)) return launch_lm_st<W, i128>(c, lv, b, prop, bin_ev, ev_flags);
  return launch_lm_st<W, long long>(c, lv, b, prop, bin_ev, ev_flags);
}

template <typename W>
int launch_lm_nocfg(dcd_ctx* c, const LV<W>& lv, Bins& b, int32_t* prop, cudaEvent_t* bin_ev, unsigned ev_flags,
                    bool fork, int64_t* sweep) {
  if (lv.m2 >= ((int64_t)1 << 31)) return launch_lm_st<W, i128>(c, lv, b, prop, bin_ev, ev_flags, fork, sweep);
  return launch_lm_st<W, long long>(c, lv, b, prop, bin_ev, ev_flags, fork, sweep);
}

// Per-graph counters of one update (host).
struct GraphTally {
  std::vector<int64_t> passes, passes0, moves, levels;
  explicit GraphTally(int G) : passes(G, 0), passes0(G, 0), moves(G, 0), levels(G, 0) {}
};

template <typename W>
int run_level(dcd_ctx* c, const Csr<W>& g, int32_t* L, Buf<int64_t>& kbuf, Buf<int64_t>& a, Buf<int32_t>& size,
              const uint8_t* active, const int32_t* gid, int level, LevelRun* out, GraphTally* tally,
              const int32_t* pre = nullptr) {
  cudaStream_t s = c->stream;
  DevScalars* d = c->dsc.get();
  GraphState* gs = c->gs.get();
  const int G = c->G;
  const int64_t nv = g.n;
  const int T = 256;

  // level start: N_start = N_cur per graph, running = not done
  DCD_TRY_CUDA(cudaMemsetAsync(&d->any_running, 0, sizeof(int32_t), s));
  ::dcd::count_launch(), lm_decide<<<cdiv(G, 128), 128, 0, s>>>(gs, G, 0, c->cfg.max_iters, c->cfg.tau_inv,
                                                                 &d->any_running);
  DCD_LAUNCH_CHECK();
  Bins bins;
  DCD_TRY(make_bins<W>(c, g, active, &bins, gid, pre));
  trace("level: binned");
  const int64_t total = bins.total;
  // list positions from big_from on hold rows longer than 256 entries: their
  // movers' delta of sum_i e_{i->C(i)} is taken by a CTA each
  int64_t big_from = 0;
  for (int x = 0; x < bins.plan.nb; x++)
    if (bins.plan.var[x] <= kLmWarp256) big_from += bins.cnt[x];
  const int64_t n_big = total - big_from;
  Buf<int32_t> prop, Lprev, mvit, moved, moved_cnt, moved_big, moved_big_cnt;
  DCD_TRY(prop.alloc(&c->mem, total));
  DCD_TRY(Lprev.alloc(&c->mem, nv));
  DCD_TRY(mvit.alloc(&c->mem, nv));
  DCD_TRY(moved.alloc(&c->mem, total));
  DCD_TRY(moved_cnt.alloc(&c->mem, 1));
  DCD_TRY(moved_big.alloc(&c->mem, n_big));
  DCD_TRY(moved_big_cnt.alloc(&c->mem, 1));
  ::dcd::count_launch(), fill_i32<<<grid_for(nv, T), T, 0, s>>>(mvit.get(), nv, -1);
  DCD_LAUNCH_CHECK();
  const int sq_ctas = grid_for(nv, T, 4);
  LV<W> lv{g.rp, g.col, g.w, kbuf.get(), L, a.get(), size.get(), G == 1 ? c->hgs[0].m2 : 0};
  lv.gid = gid;
  lv.gs = gid ? gs : nullptr;
  if (pre) {  // the first pass takes the screening's proposals
    lv.pre = pre;
    lv.first = &d->level_passes;
  }
  int64_t m2max = 0;
  for (int x = 0; x < G; x++) m2max = c->hgs[x].m2 > m2max ? c->hgs[x].m2 : m2max;
  LV<W> lvl = lv;
  lvl.m2 = G == 1 ? lv.m2 : m2max;  // gain width chosen by the largest graph
  const int32_t* lst = bins.list.get();
  bool any = total > 0;
  int64_t sweep[kMaxBins] = {};
  // One pass: evaluate, apply, tracked N, stop rule, then the loop condition.
  // Every pass of a level enqueues the same work (the pass number lives on
  // the device), so the body is captured once, into the body of a 'while'
  // conditional node, and the whole pass loop of the level is one graph
  // launch.  With dcd_config.pass_loop = 1 the host enqueues the same body
  // once per pass instead and reads the loop condition back after it.
  auto enqueue_pass = [&](cudaGraphConditionalHandle h, bool in_graph) -> int {
    ::dcd::count_launch(), gs_reset_pass<<<cdiv(G, 128), 128, 0, s>>>(gs, G, &d->pass_id);
    DCD_TRY_CUDA(cudaMemsetAsync(moved_cnt.get(), 0, sizeof(int32_t), s));
    DCD_TRY_CUDA(cudaMemsetAsync(moved_big_cnt.get(), 0, sizeof(int32_t), s));
    DCD_TRY_CUDA(cudaMemsetAsync(&d->any_running, 0, sizeof(int32_t), s));
    ::dcd::count_launch(), pass_stamp<<<1, 1, 0, s>>>(d, 0);
    if (any) DCD_TRY(launch_lm_nocfg<W>(c, lvl, bins, prop.get(), nullptr, 0, total >= kForkMin, sweep));
    ::dcd::count_launch(), pass_stamp<<<1, 1, 0, s>>>(d, 1);
    if (total) {
      ::dcd::count_launch(), lm_apply<<<grid_for(total, T), T, 0, s>>>(
          lst, total, big_from, prop.get(), L, kbuf.get(), (unsigned long long*)a.get(), size.get(),
          Lprev.get(), mvit.get(), &d->pass_id, moved.get(), moved_cnt.get(), moved_big.get(), moved_big_cnt.get(),
          gid, gs);
      if (big_from)
        ::dcd::count_launch(), lm_delta_in<W><<<grid_for(big_from * 32, T, 16), T, 0, s>>>(
            lv, moved.get(), moved_cnt.get(), Lprev.get(), mvit.get(), &d->pass_id, gs);
      if (n_big)
        ::dcd::count_launch(), lm_delta_in_block<W><<<grid_for(n_big * T, T, 4), T, 0, s>>>(
            lv, moved_big.get(), moved_big_cnt.get(), Lprev.get(), mvit.get(), &d->pass_id, gs);
    }
    ::dcd::count_launch(), sumsq_acc<<<sq_ctas, T, 0, s>>>(a.get(), nv, gid, gs);
    ::dcd::count_launch(), lm_decide<<<cdiv(G, 128), 128, 0, s>>>(gs, G, 1, c->cfg.max_iters, c->cfg.tau_inv,
                                                                   &d->any_running);
    ::dcd::count_launch(), pass_end<<<1, 1, 0, s>>>(d, h, c->cfg.max_iters + 2, in_graph ? 1 : 0);
    DCD_LAUNCH_CHECK();
    return DCD_OK;
  };
  if (any) DCD_TRY(prepare_lm<W>(lvl));
  DCD_TRY(side_streams(c));
  struct GraphGuard {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    cudaStream_t s = nullptr;
    ~GraphGuard() {
      if (x) {
        cudaStreamSynchronize(s);  // an error path may leave a launch of it in flight
        cudaGraphExecDestroy(x);
      }
      if (g) cudaGraphDestroy(g);
    }
  } gg;
  gg.s = s;
  {
    int64_t body_launches = 0;
    DCD_TRY_CUDA(cudaMemsetAsync(&d->level_passes, 0, sizeof(int32_t), s));
    DCD_TRY_CUDA(cudaMemsetAsync(&d->t_eval_ns, 0, 2 * sizeof(unsigned long long), s));
    if (c->cfg.pass_loop == 0) {
      DCD_TRY_CUDA(cudaGraphCreate(&gg.g, 0));
      cudaGraphConditionalHandle h;
      // the condition starts at 1 on every launch: a level runs at least one
      // pass, even with nothing to evaluate, as the sequential definition does
      DCD_TRY_CUDA(cudaGraphConditionalHandleCreate(&h, gg.g, 1, cudaGraphCondAssignDefault));
      cudaGraphNodeParams np{};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      cudaGraphNode_t node;
      DCD_TRY_CUDA(cudaGraphAddNode(&node, gg.g, nullptr, nullptr, 0, &np));
      cudaGraph_t body = np.conditional.phGraph_out[0];
      DCD_TRY_CUDA(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      const int64_t l0 = g_launches.load();
      const int rc = enqueue_pass(h, true);
      cudaGraph_t captured = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(s, &captured);
      body_launches = g_launches.load() - l0;
      g_launches -= body_launches;  // counted below, once per pass that ran
      if (rc != DCD_OK) return rc;
      DCD_TRY_CUDA(ec);
      DCD_TRY_CUDA(cudaGraphInstantiate(&gg.x, gg.g, 0));
      trace("level: pass loop instantiated");
      DCD_TRY_CUDA(cudaGraphLaunch(gg.x, s));
      DCD_TRY_CUDA(cudaMemcpyAsync(c->hsc, d, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
      DCD_TRY_CUDA(cudaMemcpyAsync(c->hgs, gs, G * sizeof(GraphState), cudaMemcpyDeviceToHost, s));
      DCD_TRY_CUDA(cudaStreamSynchronize(s));
    } else {
      // the same pass, enqueued by the host once per pass; the stop rule is
      // read back after each (pass_end caps the loop as in the graph)
      for (;;) {
        const int64_t l0 = g_launches.load();
        DCD_TRY(enqueue_pass(cudaGraphConditionalHandle{}, false));
        body_launches = g_launches.load() - l0;
        g_launches -= body_launches;
        DCD_TRY_CUDA(cudaMemcpyAsync(c->hsc, d, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
        DCD_TRY_CUDA(cudaMemcpyAsync(c->hgs, gs, G * sizeof(GraphState), cudaMemcpyDeviceToHost, s));
        DCD_TRY_CUDA(cudaStreamSynchronize(s));
        if (c->hsc->loop_err || !c->hsc->any_running) break;
      }
    }
    trace("level: pass loop ran");
    if (level == 0) {  // the level-0 bin record (dcd_get_level0_bins)
      c->l0_nb = bins.plan.nb;
      c->l0_side = any && total >= kForkMin;
      for (int x = 0; x < kMaxBins; x++) {
        c->l0_cnt[x] = x < bins.plan.nb ? bins.cnt[x] : 0;
        c->l0_sweep[x] = x < bins.plan.nb ? sweep[x] : 0;
      }
    }
    if (c->hsc->loop_err) {
      note_cuda_error(cudaErrorUnknown, "local-move pass loop passed its cap", __FILE__, __LINE__);
      return DCD_ETIMEOUT;
    }
    const int64_t passes = c->hsc->level_passes;
    g_launches += body_launches * passes;
    out->passes = passes;
    out->ms_lm = (float)(c->hsc->t_eval_ns * 1e-6);
    out->ms_apply = (float)(c->hsc->t_apply_ns * 1e-6);
    out->edges = bins.act_deg * passes;
    out->verts = bins.n_active * passes;
    out->edges_pre = pre ? bins.pre_deg : 0;
    out->verts_pre = pre ? bins.pre_verts : 0;
    for (int x = 0; x < bins.plan.nb; x++) {
      const int k = lm_variant_class(bins.plan.var[x]);
      out->edges_bin[k] += bins.deg[x] * passes;
      out->verts_bin[k] += bins.cnt[x] * passes;
    }
    if (trace_on()) {
      char buf[1024];
      int o = 0;
      for (int x = 0; x < bins.plan.nb && o < 900; x++)
        o += snprintf(buf + o, sizeof(buf) - o, " [<=%lld: %lld v %lld e]",
                      bins.plan.hi[x] == INT64_MAX ? -1LL : (long long)bins.plan.hi[x], (long long)bins.cnt[x],
                      (long long)bins.deg[x]);
      tracef("level %d: %lld passes, evaluation %.3f ms, apply %.3f ms:%s", level, (long long)passes, out->ms_lm,
             out->ms_apply, buf);
    }
  }
  for (int x = 0; x < G; x++) {
    tally->moves[x] += c->hgs[x].moves_level;
    tally->passes[x] += c->hgs[x].passes;
    if (level == 0) tally->passes0[x] = c->hgs[x].passes;
  }
  trace("level: passes done");
  return DCD_OK;
}

// Compaction of one level: returns nc; fills the coarse graph when nc < n.
template <typename W>
int used_labels(dcd_ctx* c, const Csr<W>& g, const int32_t* L, Buf<int32_t>& cid, int64_t* nc,
                const int32_t* gid, Buf<int32_t>* gid_next, const int32_t* size = nullptr) {
  cudaStream_t s = c->stream;
  const int T = 256;
  const int64_t nv = g.n;
  DCD_TRY(cid.alloc(&c->mem, nv + 1));
  Buf<int32_t> tmp;
  DCD_TRY(tmp.alloc(&c->mem, scan_tmp_count(nv + 1)));
  DCD_TRY_CUDA(cudaMemsetAsync(cid.get(), 0, (nv + 1) * sizeof(int32_t), s));
  if (size) ::dcd::count_launch(), used_from_size<<<grid_for(nv, T), T, 0, s>>>(nv, size, cid.get());
  else ::dcd::count_launch(), mark_used<<<grid_for(nv, T), T, 0, s>>>(nv, L, cid.get());
  DCD_LAUNCH_CHECK();
  DCD_TRY(exclusive_scan<int32_t>(cid.get(), cid.get(), nv + 1, nullptr, tmp.get(), s));
  ::dcd::count_launch(), gs_reset_nc<<<cdiv(c->G, 128), 128, 0, s>>>(c->gs.get(), c->G);
  DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch, cid.get() + nv, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  DCD_TRY_CUDA(cudaStreamSynchronize(s));
  *nc = *reinterpret_cast<int32_t*>(c->hscratch);
  if (gid_next) DCD_TRY(gid_next->alloc(&c->mem, *nc > 0 ? *nc : 1));
  ::dcd::count_launch(), count_used<<<grid_for(nv, T), T, 0, s>>>(nv, cid.get(), gid, c->gs.get(),
                                                                   gid_next ? gid_next->get() : nullptr);
  DCD_LAUNCH_CHECK();
  DCD_TRY_CUDA(cudaMemcpyAsync(c->hgs, c->gs.get(), c->G * sizeof(GraphState), cudaMemcpyDeviceToHost, s));
  DCD_TRY_CUDA(cudaStreamSynchronize(s));
  return DCD_OK;
}

// run id of entry e: heads before-or-at e, minus one
__global__ void incl_from_excl(const int32_t* __restrict__ head, int32_t* __restrict__ uid, int64_t m) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    uid[e] = uid[e] + head[e] - 1;
}

struct CoarseGraph {
  Buf<int64_t> rp;
  Buf<int32_t> col;
  Buf<int64_t> w;
  Csr<int64_t> view;
};

// One wave of emit CTAs, every warp taking an equal contiguous range of
// entries (a multiple of 32).
template <typename W, typename KT, typename VT>
int launch_emit(dcd_ctx* c, const Csr<W>& g, int64_t m0, const int32_t* ccid, int64_t nc, uint64_t* keys,
                uint64_t* vals, unsigned long long* cnt) {
  const int grid = wave_grid(emit_coarse<W, KT, VT>, cdiv(m0, 32) * 32, kEmitThreads);
  const int64_t warps = (int64_t)grid * (kEmitThreads / 32);
  const int64_t per_warp = cdiv(cdiv(m0, warps), 32) * 32;
  ::dcd::count_launch(), emit_coarse<W, KT, VT><<<grid, kEmitThreads, 0, c->stream>>>(
      g.n, m0, g.rp, g.col, g.w, ccid, (uint64_t)nc, per_warp, keys, vals, cnt);
  DCD_LAUNCH_CHECK();
  return DCD_OK;
}

// ---- per-step delta coarsening of level 0 ----
//
// R_t changes level 0 only (Sec. III-D); above it the run works on the
// coarse graph.  The coarse graph of G_t under the level-0 labels L0 equals
// K (the coarse graph of G_{t-1} under C_{t-1}, kept by the last update),
// plus every pair's weight change in cell (C_{t-1}(u), C_{t-1}(v)), plus, for
// every vertex v with L0(v) != C_{t-1}(v), its row moved from the cells of
// C_{t-1} to those of L0 (with the mirror entries of neighbours that stayed).
// Level 0 only assigns labels of existing communities, so every label of L0
// has a row in K; the result is folded onto the compacted ids of L0 and is
// the same matrix the full emit produces.  Cells are added modulo the width
// of VT (weight changes can be negative); the final cells are the exact sums.

// Two's-complement sum over the lanes of `peers`, modulo the width of VT.
__device__ __forceinline__ unsigned peer_sum(unsigned peers, long long x, unsigned) {
  return __reduce_add_sync(peers, (unsigned)x);
}
__device__ __forceinline__ unsigned long long peer_sum(unsigned peers, long long x, unsigned long long) {
  const unsigned long long u = (unsigned long long)x;
  unsigned long long sum = 0;
#pragma unroll
  for (int q = 0; q < 4; q++)
    sum += (unsigned long long)__reduce_add_sync(peers, (unsigned)(u >> (16 * q)) & 0xffffu) << (16 * q);
  return sum;
}

// One add per distinct cell of the warp (cell < 0: nothing).
template <typename VT>
__device__ __forceinline__ void cell_add(VT* D, long long cell, long long x) {
  const unsigned peers = __match_any_sync(0xffffffffu, (unsigned long long)cell);
  const VT sum = peer_sum(peers, x, VT(0));
  if (cell >= 0 && sum != VT(0) && (int)(__ffs(peers) - 1) == (int)lane_id()) atomicAdd(&D[cell], sum);
}

template <typename VT>
__global__ void n1_load(const unsigned long long* __restrict__ K, int64_t cells, VT* __restrict__ D) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cells; i += (int64_t)gridDim.x * blockDim.x)
    D[i] = (VT)K[i];
}

// The batch: pair (u, v) adds its weight change to cell (C(u), C(v)).
template <typename VT>
__global__ void n1_pairs(const uint64_t* __restrict__ pkey, const int64_t* __restrict__ pdelta, int64_t P,
                         const int32_t* __restrict__ cprev, const int32_t* __restrict__ kidx, int64_t nk,
                         VT* __restrict__ D, uint32_t* __restrict__ bad) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31u); p0 < P; p0 += stride) {
    const int64_t p = p0 + lane_id();
    long long cell = -1, x = 0;
    if (p < P) {
      x = pdelta[p];
      if (x != 0) {
        const uint64_t k = pkey[p];
        const long long a = kidx[cprev[(int32_t)(k >> 32)]], b = kidx[cprev[(int32_t)(k & 0xffffffffu)]];
        if (a >= 0 && b >= 0) cell = a * nk + b;
        else atomicOr(bad, 1u);
      }
    }
    cell_add(D, cell, x);
  }
}

// Vertices whose level-0 label differs from C_{t-1}: their rows as work
// items of at most kN1Chunk entries (v << 32 | chunk), so that a moved hub
// does not hold one warp for its whole row.
constexpr int kN1Chunk = 256;

__global__ void n1_movers_list(int64_t n, const int32_t* __restrict__ L0, const int32_t* __restrict__ cprev,
                               const int64_t* __restrict__ rp, int64_t* __restrict__ items,
                               int32_t* __restrict__ cnt, unsigned long long* __restrict__ entries) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int lane = lane_id();
  for (int64_t b0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31u); b0 < n; b0 += stride) {
    const int64_t v = b0 + lane;
    const bool mv = v < n && L0[v] != cprev[v];
    if (!__any_sync(0xffffffffu, mv)) continue;
    const int64_t d = mv ? rp[v + 1] - rp[v] : 0;
    const int nch = (int)((d + kN1Chunk - 1) / kN1Chunk);
    int incl = nch;  // inclusive prefix of the chunk counts over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const unsigned long long dsum = peer_sum(0xffffffffu, (long long)d, 0ull);
    int32_t base = 0;
    if (lane == 0 && total > 0) {
      base = atomicAdd(cnt, total);
      atomicAdd(entries, dsum);
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int j = 0; j < nch; j++) items[base + incl - nch + j] = (int64_t)v << 32 | (uint32_t)j;
  }
}

// A warp per item (a chunk of a moved vertex v's row): entry (v, u, w)
// leaves cell (C v, C u) for (L0 v, L0 u); when u stayed, its mirror entry
// (u, v) leaves (C u, C v) for (C u, L0 v).  (When u moved too, u's own row
// carries the mirror.)
template <typename VT>
__global__ void n1_movers(const int64_t* __restrict__ items, const int32_t* __restrict__ cnt,
                          const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                          const int32_t* __restrict__ w, const int32_t* __restrict__ L0,
                          const int32_t* __restrict__ cprev, const int32_t* __restrict__ kidx, int64_t nk,
                          VT* __restrict__ D, uint32_t* __restrict__ bad) {
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t M = *cnt;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < M; i += nw) {
    const int64_t it = items[i];
    const int32_t v = (int32_t)(it >> 32);
    const int64_t b = rp[v] + (int64_t)(uint32_t)it * kN1Chunk;
    const int64_t rest = rp[v + 1] - b;
    const int d = rest < kN1Chunk ? (int)rest : kN1Chunk;
    const long long cv = kidx[cprev[v]], lv = kidx[L0[v]];
    for (int e0 = 0; e0 < d; e0 += 32) {
      const int e = e0 + lane_id();
      long long c1 = -1, c2 = -1, c3 = -1, c4 = -1, x = 0;
      const int32_t u = e < d ? col[b + e] : 0;
      const long long cu = e < d ? kidx[cprev[u]] : 0, lu = e < d ? kidx[L0[u]] : 0;
      if (e < d && (cv < 0 || lv < 0 || cu < 0 || lu < 0)) atomicOr(bad, 1u);
      else if (e < d) {
        x = w[b + e];
        c1 = cv * nk + cu;
        c2 = lv * nk + lu;
        if (cu == lu) {
          c3 = cu * nk + cv;
          c4 = cu * nk + lv;
        }
      }
      cell_add(D, c1, -x);
      cell_add(D, c2, x);
      cell_add(D, c3, -x);
      cell_add(D, c4, x);
    }
  }
}

// Cell (a, b) of K's index space to (cid(label a), cid(label b)) of L0.
template <typename VT>
__global__ void n1_compact(const VT* __restrict__ D, int64_t nk, const int32_t* __restrict__ klab,
                           const int32_t* __restrict__ cid, const int32_t* __restrict__ L0, int64_t nc,
                           VT* __restrict__ H, uint32_t* __restrict__ bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nk * nk; i += (int64_t)gridDim.x * blockDim.x) {
    const VT x = D[i];
    if (x == VT(0)) continue;
    // a non-zero cell has members on both sides: their labels are in use
    const int32_t la = klab[i / nk], lb = klab[i % nk];
    const int64_t a = cid[la], b = cid[lb];
    if (a < 0 || a >= nc || b < 0 || b >= nc) {
      atomicOr(bad, 1u);
      continue;
    }
    H[a * nc + b] = x;
  }
}

// K for the next update, from this update's level-0 matrix H (nc0 x nc0):
// F(i) = the final label of level-1 vertex i (any member's), then the cells
// of H folded onto the final communities in label order.  A final label is
// its community's smallest member, so label v is in use exactly when
// fin[v] == v.  The members of a level-1 vertex share one final label: each
// CTA keeps the first it sees per level-1 vertex in shared memory (nc0 <=
// 4096 entries) and writes those once, so the few hundred cells of F are not
// written by every vertex.
__global__ void n1_final_of(int64_t n, int64_t nc0, const int32_t* __restrict__ ccid,
                            const int32_t* __restrict__ fin, int32_t* __restrict__ F, int32_t* __restrict__ used) {
  extern __shared__ int32_t fs[];
  for (int64_t i = threadIdx.x; i < nc0; i += blockDim.x) fs[i] = -1;
  __syncthreads();
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t f = fin[v];
    used[v] = f == (int32_t)v ? 1 : 0;
    const int32_t c = ccid[v];
    if (fs[c] < 0) fs[c] = f;  // every writer of fs[c] writes the same value
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < nc0; i += blockDim.x)
    if (fs[i] >= 0 && F[i] != fs[i]) F[i] = fs[i];
}

__global__ void n1_index(int64_t n, const int32_t* __restrict__ used, const int32_t* __restrict__ idx,
                         int32_t* __restrict__ kidx, int32_t* __restrict__ klab) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
    const bool u = used[l] != 0;
    kidx[l] = u ? idx[l] : -1;
    if (u) klab[idx[l]] = (int32_t)l;
  }
}

template <typename VT>
__global__ void n1_fold(const VT* __restrict__ H, int64_t nc0, const int32_t* __restrict__ F,
                        const int32_t* __restrict__ kidx, int64_t nk, unsigned long long* __restrict__ K) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc0 * nc0;
       i += (int64_t)gridDim.x * blockDim.x) {
    const VT x = H[i];
    if (x != VT(0))
      atomicAdd(&K[(int64_t)kidx[F[i / nc0]] * nk + kidx[F[i % nc0]]], (unsigned long long)x);
  }
}

// Level 0's coarse matrix by the delta rule into H (nc x nc, zeroed).
// *ok false (H unusable) when an index check failed: a label without a row
// of K, which the rule excludes; the caller then rebuilds from every entry.
template <typename VT>
int n1_build(dcd_ctx* c, const Csr<int32_t>& g, const int32_t* L0, const int32_t* cid, int64_t nc, VT* H,
             unsigned long long* entries, bool* ok) {
  cudaStream_t s = c->stream;
  const int T = 256;
  const int64_t nk = c->kc_n;
  Buf<VT> D;
  Buf<int64_t> items;
  Buf<int32_t> cnt;
  Buf<uint32_t> bad;
  DCD_TRY(D.alloc(&c->mem, nk * nk));
  DCD_TRY(items.alloc(&c->mem, g.n + g.nnz / kN1Chunk + 32));
  DCD_TRY(cnt.alloc(&c->mem, 1));
  DCD_TRY(bad.alloc(&c->mem, 1));
  DCD_TRY_CUDA(cudaMemsetAsync(cnt.get(), 0, sizeof(int32_t), s));
  DCD_TRY_CUDA(cudaMemsetAsync(bad.get(), 0, sizeof(uint32_t), s));
  ::dcd::count_launch(), n1_load<VT><<<grid_for(nk * nk, T), T, 0, s>>>(c->kc_mat.get(), nk * nk, D.get());
  if (c->n1.P > 0)
    ::dcd::count_launch(), n1_pairs<VT><<<grid_for(c->n1.P, T), T, 0, s>>>(
        c->n1.pkey, c->n1.pdelta, c->n1.P, c->n1.cprev, c->kc_idx.get(), nk, D.get(), bad.get());
  ::dcd::count_launch(), n1_movers_list<<<grid_for(g.n, T), T, 0, s>>>(g.n, L0, c->n1.cprev, g.rp, items.get(),
                                                                        cnt.get(), entries);
  ::dcd::count_launch(), n1_movers<VT><<<wave_grid(n1_movers<VT>, g.n * 32, T), T, 0, s>>>(
      items.get(), cnt.get(), g.rp, g.col, g.w, L0, c->n1.cprev, c->kc_idx.get(), nk, D.get(), bad.get());
  ::dcd::count_launch(), n1_compact<VT><<<grid_for(nk * nk, T), T, 0, s>>>(D.get(), nk, c->kc_lab.get(), cid, L0,
                                                                            nc, H, bad.get());
  DCD_LAUNCH_CHECK();
  DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch + 2, bad.get(), sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch + 3, cnt.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  DCD_TRY_CUDA(cudaStreamSynchronize(s));
  *ok = *reinterpret_cast<uint32_t*>(c->hscratch + 2) == 0;
  tracef("level-0 delta rule: %lld pairs, %d row chunks of moved vertices, %lld x %lld kept cells", (long long)c->n1.P,
         *reinterpret_cast<int32_t*>(c->hscratch + 3), (long long)nk, (long long)nk);
  return DCD_OK;
}

// K of this update's final labels (into the *_nx buffers; taken at commit).
template <typename VT>
int n1_keep_t(dcd_ctx* c, int64_t n, const int32_t* fin) {
  cudaStream_t s = c->stream;
  const int T = 256;
  const int64_t nc0 = c->n1.h0_nc;
  Buf<int32_t> F, used, idx;
  Buf<int32_t> stmp;
  DCD_TRY(F.alloc(&c->mem, nc0 > 0 ? nc0 : 1));
  DCD_TRY(used.alloc(&c->mem, n + 1));
  DCD_TRY(idx.alloc(&c->mem, n + 1));
  DCD_TRY(stmp.alloc(&c->mem, scan_tmp_count(n + 1) + 1));
  DCD_TRY_CUDA(cudaMemsetAsync(used.get() + n, 0, sizeof(int32_t), s));
  {
    const int64_t blocks = cdiv(n, (int64_t)T);
    const int grid = (int)(blocks < 4 * c->sms ? blocks : 4 * c->sms);
    ::dcd::count_launch(), n1_final_of<<<grid > 0 ? grid : 1, T, nc0 * sizeof(int32_t), s>>>(
        n, nc0, c->h0_ccid.get(), fin, F.get(), used.get());
  }
  DCD_LAUNCH_CHECK();
  DCD_TRY(exclusive_scan<int32_t>(used.get(), idx.get(), n + 1, nullptr, stmp.get(), s));
  DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch, idx.get() + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  DCD_TRY_CUDA(cudaStreamSynchronize(s));
  const int64_t nk = *reinterpret_cast<int32_t*>(c->hscratch);
  if (nk > kDenseNc) return DCD_OK;  // cannot happen (nk <= nc0); kept out of K's size bound
  DCD_TRY(c->kc_idx_nx.ensure(&c->mem, n));
  DCD_TRY(c->kc_lab_nx.ensure(&c->mem, nk > 0 ? nk : 1));
  DCD_TRY(c->kc_mat_nx.ensure(&c->mem, nk * nk > 0 ? nk * nk : 1));
  DCD_TRY_CUDA(cudaMemsetAsync(c->kc_mat_nx.get(), 0, nk * nk * sizeof(unsigned long long), s));
  ::dcd::count_launch(), n1_index<<<grid_for(n, T), T, 0, s>>>(n, used.get(), idx.get(), c->kc_idx_nx.get(),
                                                                c->kc_lab_nx.get());
  ::dcd::count_launch(), n1_fold<VT><<<grid_for(nc0 * nc0, T), T, 0, s>>>(
      reinterpret_cast<const VT*>(c->h0.get()), nc0, F.get(), c->kc_idx_nx.get(), nk, c->kc_mat_nx.get());
  DCD_LAUNCH_CHECK();
  c->kc_n_nx = nk;
  c->kc_nx_ready = true;
  return DCD_OK;
}

int n1_keep(dcd_ctx* c, int64_t n, const int32_t* fin) {
  c->kc_nx_ready = false;
  if (!c->n1.track || !c->n1.h0_ready) return DCD_OK;
  return c->n1.h0_wide ? n1_keep_t<unsigned long long>(c, n, fin) : n1_keep_t<unsigned>(c, n, fin);
}

// Dense coarsening (nc <= kDenseNc): matrix, emit, count, scan, write.
template <typename W, typename VT>
int coarsen_dense(dcd_ctx* c, const Csr<W>& g, const int32_t* ccid, int64_t nc, CoarseGraph* out, bool level0,
                  const int32_t* L, const int32_t* cid) {
  cudaStream_t s = c->stream;
  const int T = 256;
  const int64_t m0 = g.nnz;
  Buf<VT> dense_local;
  Buf<int64_t> stmp;
  Buf<unsigned long long> ent;
  VT* dense = nullptr;
  // level 0 keeps its matrix for the next update's delta coarsening
  const bool keep = level0 && c->n1.track;
  if (keep) {
    DCD_TRY(c->h0.ensure(&c->mem, (size_t)nc * nc * sizeof(VT) + 16));
    dense = reinterpret_cast<VT*>(c->h0.get());
    c->n1.h0_nc = nc;
    c->n1.h0_wide = sizeof(VT) == 8;
  } else {
    DCD_TRY(dense_local.alloc(&c->mem, nc * nc));
    dense = dense_local.get();
  }
  DCD_TRY(stmp.alloc(&c->mem, scan_tmp_count(nc + 1) + 1));
  DCD_TRY(ent.alloc(&c->mem, 1));
  DCD_TRY_CUDA(cudaMemsetAsync(dense, 0, nc * nc * sizeof(VT), s));
  DCD_TRY_CUDA(cudaMemsetAsync(ent.get(), 0, sizeof(unsigned long long), s));
  bool delta = false;
  if constexpr (std::is_same<W, int32_t>::value) {
    if (level0 && c->n1.usable && c->kc_valid) {
      bool ok = false;
      DCD_TRY(n1_build<VT>(c, g, L, cid, nc, dense, ent.get(), &ok));
      delta = ok;
      if (!ok) {  // rebuild from every entry
        DCD_TRY_CUDA(cudaMemsetAsync(dense, 0, nc * nc * sizeof(VT), s));
        DCD_TRY_CUDA(cudaMemsetAsync(ent.get(), 0, sizeof(unsigned long long), s));
      }
    }
  }
  if (!delta && m0 > 0) {
    // a CTA copy of the matrix when it fits in shared memory (two CTAs an SM)
    const size_t msm = (size_t)nc * nc * sizeof(VT);
    if (msm <= kDenseSmem) {
      DCD_TRY_CUDA(cudaFuncSetAttribute(emit_dense<W, VT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kDenseSmem));
      const int grid = wave_grid(emit_dense<W, VT, true>, cdiv(m0, 32) * 32, kEmitThreads, msm);
      const int64_t per_warp = cdiv(cdiv(m0, (int64_t)grid * (kEmitThreads / 32)), 32) * 32;
      ::dcd::count_launch(), emit_dense<W, VT, true><<<grid, kEmitThreads, msm, s>>>(
          g.n, m0, g.rp, g.col, g.w, ccid, (uint32_t)nc, per_warp, dense);
    } else {
      const int grid = wave_grid(emit_dense<W, VT, false>, cdiv(m0, 32) * 32, kEmitThreads);
      const int64_t per_warp = cdiv(cdiv(m0, (int64_t)grid * (kEmitThreads / 32)), 32) * 32;
      ::dcd::count_launch(), emit_dense<W, VT, false><<<grid, kEmitThreads, 0, s>>>(
          g.n, m0, g.rp, g.col, g.w, ccid, (uint32_t)nc, per_warp, dense);
    }
    DCD_LAUNCH_CHECK();
  }
  DCD_TRY(out->rp.alloc(&c->mem, nc + 1));
  DCD_TRY_CUDA(cudaMemsetAsync(out->rp.get(), 0, (nc + 1) * sizeof(int64_t), s));
  ::dcd::count_launch(), dense_count<VT><<<grid_for(nc * 32, T), T, 0, s>>>(dense, nc, out->rp.get());
  DCD_LAUNCH_CHECK();
  DCD_TRY(exclusive_scan<int64_t>(out->rp.get(), out->rp.get(), nc + 1, nullptr, stmp.get(), s));
  DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch, out->rp.get() + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch + 1, ent.get(), sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  DCD_TRY_CUDA(cudaStreamSynchronize(s));
  const int64_t U = c->hscratch[0];
  if (level0) {
    c->n1.used = delta;
    c->n1.entries = delta ? c->n1.P + c->hscratch[1] : m0;
    c->n1.h0_ready = keep;
    tracef("level-0 coarse graph: %s, %lld entries read, %lld communities", delta ? "delta rule" : "every entry",
           (long long)c->n1.entries, (long long)nc);
  }
  DCD_TRY(out->col.alloc(&c->mem, U));
  DCD_TRY(out->w.alloc(&c->mem, U));
  ::dcd::count_launch(), dense_write<VT><<<grid_for(nc * 32, T), T, 0, s>>>(dense, nc, out->rp.get(),
                                                                             out->col.get(), out->w.get());
  DCD_LAUNCH_CHECK();
  out->view = Csr<int64_t>{nc, U, out->rp.get(), out->col.get(), out->w.get()};
  return DCD_OK;
}

// level0: the coarsening of G_t's level-0 labels (the delta rule may apply,
// and the matrix is kept for the next update).
template <typename W>
int coarsen(dcd_ctx* c, const Csr<W>& g, const int32_t* L, const int32_t* cid, int64_t nc, CoarseGraph* out,
            bool level0 = false) {
  cudaStream_t s = c->stream;
  const int T = 256;
  const int64_t m0 = g.nnz;
  if (level0) c->n1.entries = m0;
  if (nc <= kDenseNc) {
    Buf<int32_t> ccid_local;
    int32_t* ccid = nullptr;
    if (level0 && c->n1.track) {
      DCD_TRY(c->h0_ccid.ensure(&c->mem, g.n > 0 ? g.n : 1));
      ccid = c->h0_ccid.get();
    } else {
      DCD_TRY(ccid_local.alloc(&c->mem, g.n > 0 ? g.n : 1));
      ccid = ccid_local.get();
    }
    if (g.n > 0) {
      ::dcd::count_launch(), coarse_of<<<grid_for(g.n, T), T, 0, s>>>(g.n, L, cid, ccid);
      DCD_LAUNCH_CHECK();
    }
    int64_t m2max = 0;
    for (int x = 0; x < c->G; x++) m2max = c->hgs[x].m2 > m2max ? c->hgs[x].m2 : m2max;
    if (m2max < ((int64_t)1 << 31)) return coarsen_dense<W, unsigned>(c, g, ccid, nc, out, level0, L, cid);
    return coarsen_dense<W, unsigned long long>(c, g, ccid, nc, out, level0, L, cid);
  }
  Buf<uint64_t> k0, k1, v0, v1;
  Buf<int32_t> head, uid;
  Buf<uint32_t> stmp;
  Buf<unsigned long long> cnt;
  DCD_TRY(k0.alloc(&c->mem, m0));
  DCD_TRY(v0.alloc(&c->mem, m0));
  DCD_TRY(cnt.alloc(&c->mem, 1));
  DCD_TRY_CUDA(cudaMemsetAsync(cnt.get(), 0, sizeof(unsigned long long), s));
  if (m0 > 0) {
    Buf<int32_t> ccid;
    DCD_TRY(ccid.alloc(&c->mem, g.n));
    ::dcd::count_launch(), coarse_of<<<grid_for(g.n, T), T, 0, s>>>(g.n, L, cid, ccid.get());
    int64_t m2max = 0;
    for (int x = 0; x < c->G; x++) m2max = c->hgs[x].m2 > m2max ? c->hgs[x].m2 : m2max;
    const bool narrow = m2max < ((int64_t)1 << 31), small = nc < 65536;
    if (narrow && small)
      DCD_TRY((launch_emit<W, uint32_t, unsigned>(c, g, m0, ccid.get(), nc, k0.get(), v0.get(), cnt.get())));
    else if (narrow)
      DCD_TRY((launch_emit<W, unsigned long long, unsigned>(c, g, m0, ccid.get(), nc, k0.get(), v0.get(),
                                                             cnt.get())));
    else if (small)
      DCD_TRY((launch_emit<W, uint32_t, unsigned long long>(c, g, m0, ccid.get(), nc, k0.get(), v0.get(),
                                                             cnt.get())));
    else
      DCD_TRY((launch_emit<W, unsigned long long, unsigned long long>(c, g, m0, ccid.get(), nc, k0.get(),
                                                                       v0.get(), cnt.get())));
    DCD_LAUNCH_CHECK();
  }
  DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch, cnt.get(), sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  DCD_TRY_CUDA(cudaStreamSynchronize(s));
  const int64_t m = c->hscratch[0];
  DCD_TRY(k1.alloc(&c->mem, m));
  DCD_TRY(v1.alloc(&c->mem, m));
  DCD_TRY(head.alloc(&c->mem, m + 1));
  DCD_TRY(uid.alloc(&c->mem, m + 1));
  DCD_TRY(stmp.alloc(&c->mem, sort_tmp_words(m) + 2 * scan_tmp_count(m + nc + 2) + 64));
  const int b = bits_for(nc * nc - 1);
  int ranges[2] = {0, b};
  bool in1 = false;
  DCD_TRY(sort_pairs<uint64_t>(k0.get(), v0.get(), k1.get(), v1.get(), m, ranges, 1, stmp.get(), &in1, s));
  const uint64_t* keys = in1 ? k1.get() : k0.get();
  const uint64_t* vals = in1 ? v1.get() : v0.get();
  ::dcd::count_launch(), key_heads<<<grid_for(m, T), T, 0, s>>>(keys, m, head.get());
  DCD_LAUNCH_CHECK();
  DCD_TRY(exclusive_scan<int32_t>(head.get(), uid.get(), m, uid.get() + m, reinterpret_cast<int32_t*>(stmp.get()), s));
  DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch, uid.get() + m, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  DCD_TRY_CUDA(cudaStreamSynchronize(s));
  const int64_t U = *reinterpret_cast<int32_t*>(c->hscratch);
  // run id of every entry = heads up to and including it, minus one
  ::dcd::count_launch(), incl_from_excl<<<grid_for(m, T), T, 0, s>>>(head.get(), uid.get(), m);
  DCD_LAUNCH_CHECK();
  DCD_TRY(out->rp.alloc(&c->mem, nc + 1));
  DCD_TRY(out->col.alloc(&c->mem, U));
  DCD_TRY(out->w.alloc(&c->mem, U));
  DCD_TRY_CUDA(cudaMemsetAsync(out->rp.get(), 0, (nc + 1) * sizeof(int64_t), s));
  DCD_TRY_CUDA(cudaMemsetAsync(out->w.get(), 0, U * sizeof(int64_t), s));
  if (m > 0) {
    ::dcd::count_launch(), reduce_runs<<<(unsigned)cdiv(cdiv(m, kRunItems), T), T, 0, s>>>(
        keys, vals, m, (uint64_t)nc, head.get(), uid.get(), (unsigned long long*)out->w.get(), out->col.get(),
        out->rp.get());
    DCD_LAUNCH_CHECK();
  }
  DCD_TRY(exclusive_scan<int64_t>(out->rp.get(), out->rp.get(), nc + 1, nullptr, reinterpret_cast<int64_t*>(stmp.get()),
                                  s));
  out->view = Csr<int64_t>{nc, U, out->rp.get(), out->col.get(), out->w.get()};
  return DCD_OK;
}

}  // namespace

int hub_setup(dcd_ctx* c, const int32_t* list, int64_t H, const int64_t* rp, HubBufs* b) {
  cudaStream_t s = c->stream;
  const int T = 256;
  Buf<int64_t> deg, tmp;
  DCD_TRY(b->toff.alloc(&c->mem, H + 1));
  DCD_TRY(b->soff.alloc(&c->mem, H + 1));
  DCD_TRY(b->coff.alloc(&c->mem, H + 1));
  DCD_TRY(deg.alloc(&c->mem, H + 1));
  DCD_TRY(tmp.alloc(&c->mem, scan_tmp_count(H + 1) + 1));
  DCD_TRY_CUDA(cudaMemsetAsync(b->toff.get() + H, 0, sizeof(int64_t), s));
  DCD_TRY_CUDA(cudaMemsetAsync(b->coff.get() + H, 0, sizeof(int64_t), s));
  DCD_TRY_CUDA(cudaMemsetAsync(deg.get() + H, 0, sizeof(int64_t), s));
  ::dcd::count_launch(), hub_sizes<0><<<grid_for(H, T), T, 0, s>>>(list, H, rp, b->toff.get(), deg.get(),
                                                                    b->coff.get());
  DCD_LAUNCH_CHECK();
  DCD_TRY(exclusive_scan<int64_t>(b->toff.get(), b->toff.get(), H + 1, nullptr, tmp.get(), s));
  DCD_TRY(exclusive_scan<int64_t>(deg.get(), b->soff.get(), H + 1, nullptr, tmp.get(), s));
  DCD_TRY(exclusive_scan<int64_t>(b->coff.get(), b->coff.get(), H + 1, nullptr, tmp.get(), s));
  DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch, b->toff.get() + H, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch + 1, b->soff.get() + H, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch + 2, b->coff.get() + H, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  DCD_TRY_CUDA(cudaStreamSynchronize(s));
  const int64_t tcap = c->hscratch[0], scap = c->hscratch[1];
  b->chunks = c->hscratch[2];
  DCD_TRY(b->keys.alloc(&c->mem, tcap));
  DCD_TRY(b->vals.alloc(&c->mem, tcap));
  DCD_TRY(b->slots.alloc(&c->mem, scap));
  DCD_TRY(b->nslot.alloc(&c->mem, H));
  DCD_TRY(b->nprev.alloc(&c->mem, H));
  DCD_TRY(b->part.alloc(&c->mem, 3 * b->chunks));
  DCD_TRY_CUDA(cudaMemsetAsync(b->keys.get(), 0xff, tcap * sizeof(int32_t), s));
  DCD_TRY_CUDA(cudaMemsetAsync(b->vals.get(), 0, tcap * sizeof(unsigned long long), s));
  DCD_TRY_CUDA(cudaMemsetAsync(b->nslot.get(), 0, H * sizeof(int32_t), s));
  HubTables& t = b->t;
  t.list = list;
  t.H = H;
  t.toff = b->toff.get();
  t.soff = b->soff.get();
  t.coff = b->coff.get();
  t.keys = b->keys.get();
  t.vals = b->vals.get();
  t.slots = b->slots.get();
  t.nslot = b->nslot.get();
  t.nprev = b->nprev.get();
  t.part = b->part.get();
  return DCD_OK;
}

unsigned hub_grid(dcd_ctx* c, const HubBufs& b) {
  const int64_t cap = 16 * (int64_t)c->sms;
  return (unsigned)(b.chunks < cap ? (b.chunks > 0 ? b.chunks : 1) : cap);
}

int pool_stats(dcd_ctx* c, const Csr<int32_t>& g, const int32_t* L, const int64_t* k, const int64_t* a,
               const int32_t* size, const uint8_t* mask, PoolStats* out) {
  Bins bins;
  DCD_TRY(make_bins<int32_t>(c, g, mask, &bins));
  const int64_t m = bins.total;
  out->count = m;
  DCD_TRY(out->eC.alloc(&c->mem, m));
  DCD_TRY(out->eB.alloc(&c->mem, m));
  DCD_TRY(out->dB.alloc(&c->mem, m));
  DCD_TRY(out->sB.alloc(&c->mem, m));
  Buf<int32_t> prop;
  DCD_TRY(prop.alloc(&c->mem, m));
  LV<int32_t> lv{g.rp, g.col, g.w, k, L, a, size, c->hgs[0].m2};
  lv.f_eC = out->eC.get();
  lv.f_eB = out->eB.get();
  lv.f_dB = out->dB.get();
  lv.f_sB = out->sB.get();
  if (m) DCD_TRY(launch_lm<int32_t>(c, lv, bins, prop.get()));
  out->list.reset();
  out->list.p = bins.list.p;
  out->list.n = bins.list.n;
  out->list.mem = bins.list.mem;
  bins.list.p = nullptr;
  bins.list.n = 0;
  return DCD_OK;
}

namespace {
__global__ void row_sums(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ w,
                         int64_t* __restrict__ k) {
  const int lane = lane_id();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; v < n; v += nw) {
    int64_t x = 0;
    for (int64_t e = rp[v] + lane; e < rp[v + 1]; e += 32) x += w[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) k[v] = x;
  }
}
}  // namespace

int tune_bins(dcd_ctx* c, const Csr<int32_t>& g, const int32_t* L, const BinPlan* cands, int ncand, int reps,
              float* ms, int* best) {
  cudaStream_t s = c->stream;
  const int T = 256;
  const int64_t n = g.n;
  const int G = c->G;
  Buf<int64_t> k, a;
  Buf<int32_t> size, prop;
  DCD_TRY(k.alloc(&c->mem, n));
  DCD_TRY(a.alloc(&c->mem, n));
  DCD_TRY(size.alloc(&c->mem, n));
  DCD_TRY(prop.alloc(&c->mem, n));
  ::dcd::count_launch(), row_sums<<<grid_for(n * 32, T), T, 0, s>>>(n, g.rp, g.w, k.get());
  DCD_LAUNCH_CHECK();
  DCD_TRY(community_sums(c, n, L, k.get(), a.get(), size.get()));
  int64_t m2max = 0;
  for (int x = 0; x < G; x++) m2max = c->hgs[x].m2 > m2max ? c->hgs[x].m2 : m2max;
  LV<int32_t> lv{g.rp, g.col, g.w, k.get(), L, a.get(), size.get(), m2max};
  if (G > 1) {
    lv.gid = c->gid.get();
    lv.gs = c->gs.get();
  }
  const BinPlan keep = c->bin_plan;
  *best = -1;
  for (int x = 0; x < ncand; x++) {
    c->bin_plan = cands[x];
    Bins bins;
    DCD_TRY(make_bins<int32_t>(c, g, nullptr, &bins));
    if (bins.total) DCD_TRY(launch_lm<int32_t>(c, lv, bins, prop.get()));  // warm-up
    DCD_TRY_CUDA(cudaEventRecord(c->ev[20], s));
    for (int r = 0; r < reps; r++)
      if (bins.total) DCD_TRY(launch_lm<int32_t>(c, lv, bins, prop.get()));
    DCD_TRY_CUDA(cudaEventRecord(c->ev[21], s));
    DCD_TRY_CUDA(cudaEventSynchronize(c->ev[21]));
    float t = 0.f;
    DCD_TRY_CUDA(cudaEventElapsedTime(&t, c->ev[20], c->ev[21]));
    ms[x] = t / (reps > 0 ? reps : 1);
    if (*best < 0 || ms[x] < ms[*best]) *best = x;
  }
  c->bin_plan = *best >= 0 ? cands[*best] : keep;
  return DCD_OK;
}

// One local-move evaluation of every vertex of g under L with the plan in
// force, reps times; each bin's kernels run alone, one bin after another, and
// are timed with CUDA events on the context stream.  Outputs per bin: vertices,
// entries (degree sum) and the mean time of one evaluation.  No move is
// applied.
int eval_bins(dcd_ctx* c, const Csr<int32_t>& g, const int32_t* L, int reps, int32_t* nb, int32_t* var,
              int64_t* verts, int64_t* entries, float* ms) {
  cudaStream_t s = c->stream;
  const int T = 256;
  const int64_t n = g.n;
  Buf<int64_t> k, a;
  Buf<int32_t> size, prop;
  DCD_TRY(k.alloc(&c->mem, n));
  DCD_TRY(a.alloc(&c->mem, n));
  DCD_TRY(size.alloc(&c->mem, n));
  DCD_TRY(prop.alloc(&c->mem, n));
  ::dcd::count_launch(), row_sums<<<grid_for(n * 32, T), T, 0, s>>>(n, g.rp, g.w, k.get());
  DCD_LAUNCH_CHECK();
  DCD_TRY(community_sums(c, n, L, k.get(), a.get(), size.get()));
  int64_t m2max = 0;
  for (int x = 0; x < c->G; x++) m2max = c->hgs[x].m2 > m2max ? c->hgs[x].m2 : m2max;
  LV<int32_t> lv{g.rp, g.col, g.w, k.get(), L, a.get(), size.get(), m2max};
  if (c->G > 1) {
    lv.gid = c->gid.get();
    lv.gs = c->gs.get();
  }
  Bins bins;
  DCD_TRY(make_bins<int32_t>(c, g, nullptr, &bins));
  *nb = bins.plan.nb;
  struct Events {
    cudaEvent_t e[kMaxBins] = {};
    ~Events() {
      for (auto x : e)
        if (x) cudaEventDestroy(x);
    }
  } end;
  for (int x = 0; x < bins.plan.nb; x++) {
    DCD_TRY_CUDA(cudaEventCreate(&end.e[x]));
    var[x] = bins.plan.var[x];
    verts[x] = bins.cnt[x];
    entries[x] = bins.deg[x];
    ms[x] = 0.f;
  }
  if (bins.total) DCD_TRY(launch_lm<int32_t>(c, lv, bins, prop.get()));  // warm-up
  for (int r = 0; r < reps; r++) {
    if (bins.total) DCD_TRY(launch_lm<int32_t>(c, lv, bins, prop.get(), end.e));
    DCD_TRY_CUDA(cudaStreamSynchronize(s));
    for (int x = 0; x < bins.plan.nb; x++) {
      float t = 0.f;
      if (bins.cnt[x]) DCD_TRY_CUDA(cudaEventElapsedTime(&t, c->bin_start[x], end.e[x]));
      ms[x] += t / (float)reps;
    }
  }
  return DCD_OK;
}

int community_sums(dcd_ctx* c, int64_t n, const int32_t* labels, const int64_t* k, int64_t* a, int32_t* size) {
  cudaStream_t s = c->stream;
  DCD_TRY_CUDA(cudaMemsetAsync(a, 0, n * sizeof(int64_t), s));
  DCD_TRY_CUDA(cudaMemsetAsync(size, 0, n * sizeof(int32_t), s));
  ::dcd::count_launch(), comm_sums<<<grid_for(n, kCsThreads, 2), kCsThreads, 0, s>>>(n, labels, k,
                                                                                   (unsigned long long*)a, size);
  DCD_LAUNCH_CHECK();
  return DCD_OK;
}

int run_louvain(dcd_ctx* c, const Csr<int32_t>& g0, int32_t* labels0, const uint8_t* active0, Buf<int64_t>& k0,
                int32_t* out_labels, dcd_step_stats* st, int32_t* level0_out, dcd_step_stats* per_graph,
                const int64_t* a0, const int32_t* size0, const int32_t* pre0) {
  cudaStream_t s = c->stream;
  GraphState* gs = c->gs.get();
  const int G = c->G;
  const int T = 256;
  const int64_t n0 = g0.n;
  const int64_t tau = c->cfg.tau_inv;
  const int32_t* gid0 = G > 1 ? c->gid.get() : nullptr;

  Buf<int64_t> a;
  Buf<int32_t> size, comp;
  DCD_TRY(a.alloc(&c->mem, n0));
  DCD_TRY(size.alloc(&c->mem, n0));
  DCD_TRY(comp.alloc(&c->mem, n0));
  if (a0 && size0) {
    DCD_TRY_CUDA(cudaMemcpyAsync(a.get(), a0, n0 * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    DCD_TRY_CUDA(cudaMemcpyAsync(size.get(), size0, n0 * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  } else {
    DCD_TRY(community_sums(c, n0, labels0, k0.get(), a.get(), size.get()));
  }
  ::dcd::count_launch(), fill_iota<<<grid_for(n0, T), T, 0, s>>>(comp.get(), n0);
  ::dcd::count_launch(), gs_reset_pass<<<cdiv(G, 128), 128, 0, s>>>(gs, G, &c->dsc.get()->pass_id);
  ::dcd::count_launch(), sumsq_acc<<<grid_for(n0, T, 4), T, 0, s>>>(a.get(), n0, gid0, gs);
  DCD_LAUNCH_CHECK();

  // per-graph host state of the level loop
  std::vector<int64_t> nv(G);
  std::vector<i128> N_start(G);
  for (int x = 0; x < G; x++) nv[x] = c->goff[x + 1] - c->goff[x];
  GraphTally tally(G);

  int64_t level = 0, passes_total = 0, passes0 = 0, edges_total = 0, verts_total = 0;
  float ms_bin[4] = {0.f, 0.f, 0.f, 0.f};
  int64_t edges_bin[4] = {0, 0, 0, 0}, verts_bin[4] = {0, 0, 0, 0};
  float ms_lm = 0.f, ms_apply = 0.f, ms_coarsen = 0.f, ms_lm0 = 0.f;
  int64_t edges0 = 0, verts0 = 0, edges0_pre = 0, verts0_pre = 0;
  bool first_level = true;

  // current level: level 0 uses g0 / labels0 / k0; later levels own their data
  CoarseGraph cg[2];
  Buf<int64_t> kc[2];
  Buf<int32_t> Lc[2], gidc[2];
  int which = 0;
  const Csr<int32_t>* g_l0 = &g0;
  const Csr<int64_t>* g_lc = nullptr;
  int32_t* L = labels0;
  Buf<int64_t>* kcur = &k0;
  const uint8_t* active = active0;
  const int32_t* gid = gid0;
  int64_t nvu = n0;  // vertices of the union at this level

  for (;;) {
    LevelRun lr;
    if (level == 0) {
      DCD_TRY(run_level<int32_t>(c, *g_l0, L, *kcur, a, size, active, gid, (int)level, &lr, &tally, pre0));
      if (level0_out)
        DCD_TRY_CUDA(cudaMemcpyAsync(level0_out, L, n0 * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    } else {
      DCD_TRY(run_level<int64_t>(c, *g_lc, L, *kcur, a, size, nullptr, gid, (int)level, &lr, &tally));
    }
    if (first_level) {
      for (int x = 0; x < G; x++) N_start[x] = h128(c->hgs[x].n_start_lo, c->hgs[x].n_start_hi);
      first_level = false;
    }
    passes_total += lr.passes;
    if (level == 0) {
      passes0 = lr.passes;
      ms_lm0 = lr.ms_lm;
      edges0 = lr.edges;
      verts0 = lr.verts;
      edges0_pre = lr.edges_pre;
      verts0_pre = lr.verts_pre;
    }
    edges_total += lr.edges;
    verts_total += lr.verts;
    for (int x = 0; x < 4; x++) {
      ms_bin[x] += lr.ms_bin[x];
      edges_bin[x] += lr.edges_bin[x];
      verts_bin[x] += lr.verts_bin[x];
    }
    ms_lm += lr.ms_lm;
    ms_apply += lr.ms_apply;

    DCD_TRY_CUDA(cudaEventRecord(c->ev[5], s));
    Buf<int32_t> cid;
    int64_t nc = 0;
    const int nx = which ^ 1;
    Buf<int32_t>* gnext = G > 1 ? &gidc[nx] : nullptr;
    // the level's tracked sizes give the used labels
    if (level == 0) DCD_TRY(used_labels<int32_t>(c, *g_l0, L, cid, &nc, gid, gnext, size.get()));
    else DCD_TRY(used_labels<int64_t>(c, *g_lc, L, cid, &nc, gid, gnext, size.get()));
    trace("level: labels counted");
    level++;
    // level stop per graph: nothing merged, or (from the second level on) a
    // gain of at most |N_start| / tau_inv, or the level cap
    bool all_done = true;
    for (int x = 0; x < G; x++) {
      GraphState& X = c->hgs[x];
      if (X.done) continue;
      tally.levels[x] = level;
      const i128 N_end = h128(X.n_cur_lo, X.n_cur_hi);
      if (X.nc == nv[x] || (level >= 2 && h_below_tau(N_end - N_start[x], N_start[x], tau)) ||
          level >= c->cfg.max_levels)
        X.done = 1;
      else
        all_done = false;
      N_start[x] = N_end;
      nv[x] = X.nc;
    }
    if (all_done) {
      DCD_TRY_CUDA(cudaEventRecord(c->ev[6], s));
      DCD_TRY_CUDA(cudaEventSynchronize(c->ev[6]));
      float tc = 0.f;
      cudaEventElapsedTime(&tc, c->ev[5], c->ev[6]);
      ms_coarsen += tc;
      break;
    }
    DCD_TRY_CUDA(cudaMemcpyAsync(gs, c->hgs, G * sizeof(GraphState), cudaMemcpyHostToDevice, s));
    // ---- compact: next level (all graphs together; finished graphs only
    // carry their labels along) ----
    if (level == 1) DCD_TRY(coarsen<int32_t>(c, *g_l0, L, cid.get(), nc, &cg[nx], G == 1));
    else DCD_TRY(coarsen<int64_t>(c, *g_lc, L, cid.get(), nc, &cg[nx]));
    DCD_TRY(kc[nx].alloc(&c->mem, nc));
    DCD_TRY(Lc[nx].alloc(&c->mem, nc));
    ::dcd::count_launch(), coarse_k<<<grid_for(nvu, T), T, 0, s>>>(nvu, cid.get(), a.get(), kc[nx].get());
    ::dcd::count_launch(), compose<<<grid_for(n0, T), T, 0, s>>>(n0, comp.get(), L, cid.get());
    ::dcd::count_launch(), fill_iota<<<grid_for(nc, T), T, 0, s>>>(Lc[nx].get(), nc);
    DCD_LAUNCH_CHECK();
    // next level starts from singletons: a = k, |C| = 1; in and sum a^2 carry over
    DCD_TRY_CUDA(cudaMemcpyAsync(a.get(), kc[nx].get(), nc * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    ::dcd::count_launch(), fill_i32<<<grid_for(nc, T), T, 0, s>>>(size.get(), nc, 1);
    DCD_LAUNCH_CHECK();
    DCD_TRY_CUDA(cudaEventRecord(c->ev[6], s));
    DCD_TRY_CUDA(cudaEventSynchronize(c->ev[6]));
    float tc = 0.f;
    cudaEventElapsedTime(&tc, c->ev[5], c->ev[6]);
    ms_coarsen += tc;
    trace("level: coarsened");
    // free the previous coarse level
    cg[which].rp.reset();
    cg[which].col.reset();
    cg[which].w.reset();
    kc[which].reset();
    Lc[which].reset();
    gidc[which].reset();
    which = nx;
    g_lc = &cg[which].view;
    L = Lc[which].get();
    kcur = &kc[which];
    gid = G > 1 ? gidc[which].get() : nullptr;
    nvu = nc;
    active = nullptr;
  }

  // ---- compose + canonical labels (smallest member id) ----
  DCD_TRY_CUDA(cudaEventRecord(c->ev[7], s));
  {
    Buf<int32_t> minid;
    DCD_TRY(minid.alloc(&c->mem, nvu));
    ::dcd::count_launch(), fill_i32<<<grid_for(nvu, T), T, 0, s>>>(minid.get(), nvu, INT32_MAX);
    ::dcd::count_launch(), final_min<<<grid_for(n0, T), T, 0, s>>>(n0, comp.get(), L, minid.get());
    ::dcd::count_launch(), gs_reset_nc<<<cdiv(G, 128), 128, 0, s>>>(gs, G);
    ::dcd::count_launch(), final_labels<<<grid_for(n0, T), T, 0, s>>>(n0, comp.get(), L, minid.get(), out_labels,
                                                                       gid0, gs);
    DCD_LAUNCH_CHECK();
    DCD_TRY_CUDA(cudaEventRecord(c->ev[8], s));
    DCD_TRY_CUDA(cudaMemcpyAsync(c->hgs, gs, G * sizeof(GraphState), cudaMemcpyDeviceToHost, s));
    DCD_TRY_CUDA(cudaStreamSynchronize(s));
  }
  if (G == 1) DCD_TRY(n1_keep(c, n0, out_labels));
  float tf = 0.f;
  cudaEventElapsedTime(&tf, c->ev[7], c->ev[8]);
  auto fill = [&](dcd_step_stats* o, int x) {
    const GraphState& X = c->hgs[x];
    const i128 N = h128(X.n_cur_lo, X.n_cur_hi);
    o->levels = tally.levels[x];
    o->iters_total = tally.passes[x];
    o->iters_level0 = tally.passes0[x];
    o->moves_total = tally.moves[x];
    o->communities = X.ncomm;
    o->n_lo = (int64_t)(unsigned long long)N;
    o->n_hi = (int64_t)(unsigned long long)((unsigned __int128)N >> 64);
    o->m2 = X.m2;
    o->q = X.m2 == 0 ? 0.0 : (double)N / ((double)X.m2 * (double)X.m2);
  };
  if (per_graph)
    for (int x = 0; x < G; x++) fill(&per_graph[x], x);
  if (st) {
    if (G == 1) {
      fill(st, 0);
      st->iters_total = passes_total;
      st->iters_level0 = passes0;
    } else {
      st->levels = level;
      st->iters_total = passes_total;
      st->iters_level0 = passes0;
      int64_t mv = 0, nc = 0;
      for (int x = 0; x < G; x++) {
        mv += tally.moves[x];
        nc += c->hgs[x].ncomm;
      }
      st->moves_total = mv;
      st->communities = nc;
    }
    st->edges_scanned = edges_total;
    st->verts_scanned = verts_total;
    for (int x = 0; x < 4; x++) {
      st->ms_bin[x] = ms_bin[x];
      st->edges_bin[x] = edges_bin[x];
      st->verts_bin[x] = verts_bin[x];
    }
    st->ms_local_move = ms_lm;
    st->ms_local_move0 = ms_lm0;
    st->edges_level0 = edges0;
    st->verts_level0 = verts0;
    st->edges_level0_screen = edges0_pre;
    st->verts_level0_screen = verts0_pre;
    st->ms_apply = ms_apply;
    st->ms_coarsen = ms_coarsen;
    st->ms_finish = tf;
  }
  return DCD_OK;
}


// ================================================================ dSLM-Delta-s
//
// Smart local moving, the paper's second host method (Sec. III-D applies
// Delta-screening to it as to Louvain), in the synchronous exact-integer form
// the oracle fixes:
//   - a pass moves vertices in one direction only: even passes to smaller
//     labels, odd passes to larger ones; in an odd pass a vertex of a
//     community of two or more may also move into an empty community (label
//     n + v) when that gains more than every neighbouring community; staying
//     wins ties, the smaller label wins ties between communities; after the
//     pass every community is renamed to its smallest member;
//   - a level stops after a down-and-up cycle that moved nothing or gained at
//     most |N| / tau_inv, or after max_iters passes;
//   - refinement: every community is split by the same local moving from
//     singletons, a vertex seeing only neighbours of its own community, with
//     the whole graph's k_v and 2m;
//   - aggregation: sub-communities become vertices, each starting in the
//     community that holds it (named by the coarse vertex of the community's
//     smallest member); the run stops when every sub-community is a single
//     vertex, when a level >= 1 gained at most |N| / tau_inv, or at
//     max_levels;
//   - R_t restricts the local moving of level 0 only.

namespace {

// The SLM choice of v from its row's sums: the best neighbouring community
// in the pass direction (S > 0 to move, ties to the smaller label), then, in
// an upward pass, the empty community n + v when it gains more.
template <typename ST>
__device__ __forceinline__ int32_t slm_choice(ST S, int32_t D, int32_t C, int up, int64_t m2, int64_t kv, int64_t eC,
                                              int64_t aC, int32_t sizeC, int64_t n, int32_t v) {
  int32_t best = C;
  ST bestS = 0;
  if (D != INT_MAX && S > 0) {
    best = D;
    bestS = S;
  }
  if (up && sizeC > 1) {
    const ST s0 = gain<ST>(m2, kv, 0, eC, 0, aC);  // into an empty community
    if (s0 > bestS) best = (int32_t)(n + v);
  }
  return best;
}

// Rows of at most 32 x Q entries: one warp per vertex, the row's sums in a
// warp-private shared table (the local move's scheme); parent (may be NULL)
// limits the row to neighbours of v's parent community.
template <typename W, typename ST, int Q>
__global__ void __launch_bounds__(256) slm_warp(LV<W> g, const int32_t* __restrict__ parent, int up, int64_t n,
                                                const int32_t* __restrict__ list, int64_t cnt,
                                                int32_t* __restrict__ prop) {
  using VT = typename TblVal<ST>::type;
  constexpr int ROW = 32 * Q, CAP = seg_cap(ROW);
  constexpr size_t SB = row_tbl_bytes<ROW, VT>();
  constexpr uint32_t mask = CAP - 1;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = lane_id(), wib = threadIdx.x >> 5;
  unsigned char* base = smem + (size_t)wib * SB;
  int32_t* keys = reinterpret_cast<int32_t*>(base);
  VT* vals = reinterpret_cast<VT*>(base + (size_t)CAP * 4);
  uint16_t* slots = reinterpret_cast<uint16_t*>(base + (size_t)CAP * (4 + sizeof(VT)));
  for (int s = lane; s < CAP; s += 32) {
    keys[s] = -1;
    vals[s] = 0;
  }
  __syncwarp();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < cnt; i += nw) {
    const int32_t v = list[i];
    const int64_t b = g.rp[v];
    const int d = (int)(g.rp[v + 1] - b);
    const int32_t C = g.L[v], pv = parent ? parent[v] : 0;
    int32_t lab[Q];
    W wt[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) {
      const int e = q * 32 + lane;
      lab[q] = -1;
      wt[q] = W(0);
      if (e < d) {
        lab[q] = g.col[b + e];
        wt[q] = g.w[b + e];
      }
    }
#pragma unroll
    for (int q = 0; q < Q; q++) {
      const int32_t u = lab[q];
      lab[q] = (u >= 0 && u != v && (!parent || parent[u] == pv)) ? g.L[u] : -1;
    }
    VT eCl = 0;
    int nd = 0;
#pragma unroll
    for (int q = 0; q < Q; q++) {
      if (q * 32 < d) {
        const bool isC = lab[q] == C;
        eCl += isC ? (VT)wt[q] : VT(0);
        bool claimed = false;
        uint32_t s = 0;
        if (lab[q] >= 0 && !isC) {
          s = probe_claim(keys, mask, lab[q], claimed);
          atomicAdd(&vals[s], (VT)wt[q]);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, claimed);
        if (claimed) slots[nd + __popc(bal & lanemask_lt())] = (uint16_t)s;
        nd += __popc(bal);
      }
    }
    __syncwarp();
    const int64_t eC = seg_total<32>(eCl, 0xffffffffu);
    const int64_t kv = g.k[v], aC = g.a[C], m2 = g.m2;
    ST S = gain_lowest<ST>();
    int32_t D = INT_MAX;
    for (int j = lane; j < nd; j += 32) {
      const uint32_t s = slots[j];
      const int32_t key = keys[s];
      if (up ? key > C : key < C) {
        const ST x = gain<ST>(m2, kv, (int64_t)vals[s], eC, g.a[key], aC);
        if (better(x, key, S, D)) {
          S = x;
          D = key;
        }
      }
    }
    warp_argmax(S, D);
    if (lane == 0) prop[i] = slm_choice<ST>(S, D, C, up, m2, kv, eC, aC, g.size[C], n, v);
    __syncwarp();
    for (int j = lane; j < nd; j += 32) {
      const uint32_t s = slots[j];
      keys[s] = -1;
      vals[s] = 0;
    }
    __syncwarp();
  }
}

// Rows of any length: one CTA per vertex, the table in a region of global
// memory private to the CTA (tcap slots, at least twice the longest row of
// the bin).  Keys are read around L1 (__ldcg): the region is emptied and
// reused vertex after vertex.
template <typename W, typename ST>
__global__ void __launch_bounds__(256) slm_cta(LV<W> g, const int32_t* __restrict__ parent, int up, int64_t n,
                                               const int32_t* __restrict__ list, int64_t cnt,
                                               int32_t* __restrict__ prop, int32_t* __restrict__ tkeys,
                                               typename TblVal<ST>::type* __restrict__ tvals,
                                               uint32_t* __restrict__ tslots, uint32_t tcap) {
  using VT = typename TblVal<ST>::type;
  constexpr int T = 256, NW = T / 32;
  __shared__ ST redS[NW];
  __shared__ int32_t redD[NW];
  __shared__ VT redE[NW];
  __shared__ int32_t s_nd;
  const int tid = threadIdx.x, lane = lane_id(), wid = tid >> 5;
  int32_t* keys = tkeys + (size_t)blockIdx.x * tcap;
  VT* vals = tvals + (size_t)blockIdx.x * tcap;
  uint32_t* slots = tslots + (size_t)blockIdx.x * tcap;
  const uint32_t mask = tcap - 1;
  for (uint32_t s = tid; s < tcap; s += T) {
    keys[s] = -1;
    vals[s] = 0;
  }
  if (tid == 0) s_nd = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x; i < cnt; i += gridDim.x) {
    const int32_t v = list[i];
    const int64_t b = g.rp[v];
    const int64_t d = g.rp[v + 1] - b;
    const int32_t C = g.L[v], pv = parent ? parent[v] : 0;
    VT eCl = 0;
    for (int64_t e0 = 0; e0 < d; e0 += T) {
      const int64_t e = e0 + tid;
      bool valid = e < d;
      const int32_t u = valid ? g.col[b + e] : -1;
      valid = valid && u != v && (!parent || parent[u] == pv);
      const int32_t lab = valid ? g.L[u] : -1;
      const W wt = valid ? g.w[b + e] : W(0);
      bool claimed = false;
      uint32_t s = 0;
      if (valid) {
        if (lab == C) {
          eCl += (VT)wt;
        } else {
          s = hash_label(lab, mask);
          for (;;) {
            const int32_t k = __ldcg(&keys[s]);
            if (k == lab) break;
            if (k == -1) {
              const int32_t old = atomicCAS(&keys[s], -1, lab);
              if (old == -1) {
                claimed = true;
                break;
              }
              if (old == lab) break;
            }
            s = (s + 1) & mask;
          }
          atomicAdd(&vals[s], (VT)wt);
        }
      }
      const unsigned bal = __ballot_sync(0xffffffffu, claimed);
      int at = 0;
      if (lane == 0 && bal) at = atomicAdd(&s_nd, __popc(bal));
      at = __shfl_sync(0xffffffffu, at, 0);
      if (claimed) slots[at + __popc(bal & lanemask_lt())] = s;
    }
    const int64_t ew = seg_total<32>(eCl, 0xffffffffu);
    if (lane == 0) redE[wid] = (VT)ew;
    __syncthreads();
    int64_t eC = 0;
#pragma unroll
    for (int x = 0; x < NW; x++) eC += (int64_t)redE[x];
    const int nd = s_nd;
    const int64_t kv = g.k[v], aC = g.a[C], m2 = g.m2;
    ST S = gain_lowest<ST>();
    int32_t D = INT_MAX;
    for (int j = tid; j < nd; j += T) {
      const uint32_t s = slots[j];
      const int32_t key = __ldcg(&keys[s]);
      if (up ? key > C : key < C) {
        const ST x = gain<ST>(m2, kv, (int64_t)__ldcg(&vals[s]), eC, g.a[key], aC);
        if (better(x, key, S, D)) {
          S = x;
          D = key;
        }
      }
    }
    warp_argmax(S, D);
    if (lane == 0) {
      redS[wid] = S;
      redD[wid] = D;
    }
    __syncthreads();
    if (wid == 0) {
      S = lane < NW ? redS[lane] : gain_lowest<ST>();
      D = lane < NW ? redD[lane] : INT_MAX;
      warp_argmax(S, D);
      if (lane == 0) prop[i] = slm_choice<ST>(S, D, C, up, m2, kv, eC, aC, g.size[C], n, v);
    }
    for (int j = tid; j < nd; j += T) {
      const uint32_t s = slots[j];
      keys[s] = -1;
      vals[s] = 0;
    }
    __syncthreads();
    if (tid == 0) s_nd = 0;
    __syncthreads();
  }
}

// next = L with the proposals of the listed vertices; movers counted.
__global__ void slm_apply(const int32_t* __restrict__ list, int64_t cnt, const int32_t* __restrict__ prop,
                          int32_t* __restrict__ next, const int32_t* __restrict__ L,
                          unsigned long long* __restrict__ moves) {
  unsigned long long mv = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = list[i], p = prop[i];
    next[v] = p;
    mv += p != L[v];
  }
  mv = warp_sum(mv);
  if (lane_id() == 0 && mv) atomicAdd(moves, mv);
}

// Canonical labels: every community renamed to its smallest member
// (labels in [0, 2n) in, [0, n) out).
__global__ void canon_min(int64_t n, const int32_t* __restrict__ next, int32_t* __restrict__ minid) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    atomicMin(&minid[next[v]], (int32_t)v);
}
__global__ void canon_apply(int64_t n, const int32_t* __restrict__ next, const int32_t* __restrict__ minid,
                            int32_t* __restrict__ L) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    L[v] = minid[next[v]];
}

// sum_i e_{i->C(i)} of labels L (self-loop entries included, as in Eq. 1's
// double count), a warp per row.
template <typename W>
__global__ void slm_in_sum(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const W* __restrict__ w, const int32_t* __restrict__ L,
                           unsigned long long* __restrict__ in) {
  unsigned long long acc = 0;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
    const int32_t Lu = L[u];
    for (int64_t e = rp[u] + lane_id(); e < rp[u + 1]; e += 32)
      if (L[col[e]] == Lu) acc += (unsigned long long)w[e];
  }
  acc = warp_sum(acc);
  if (lane_id() == 0 && acc) atomicAdd(in, acc);
}

// sum over labels of a^2 as an unsigned 128-bit integer (lo, hi).
__global__ void slm_sumsq(const int64_t* __restrict__ a, int64_t n, unsigned long long* __restrict__ lohi) {
  unsigned __int128 s = 0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long x = (unsigned long long)a[c];
    s += (unsigned __int128)x * x;
  }
  unsigned long long lo = (unsigned long long)s, hi = (unsigned long long)(s >> 64);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long lo2 = __shfl_xor_sync(0xffffffffu, lo, o), hi2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const unsigned long long nlo = lo + lo2;
    hi = hi + hi2 + (nlo < lo ? 1ull : 0ull);
    lo = nlo;
  }
  if (lane_id() == 0) add128(&lohi[0], &lohi[1], ((unsigned __int128)hi << 64) | lo);
}

// Start labels of the next level: the coarse vertex of sub-community s starts
// in the community of its members, named by the coarse vertex of that
// community's smallest member.
__global__ void slm_parent_start(int64_t n, const int32_t* __restrict__ sub, const int32_t* __restrict__ L,
                                 const int32_t* __restrict__ cid, int32_t* __restrict__ Lc) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    Lc[cid[sub[v]]] = cid[sub[L[v]]];
}

__global__ void count_heads(int64_t n, const int32_t* __restrict__ x, unsigned long long* __restrict__ out) {
  unsigned long long c = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    c += x[v] == (int32_t)v;
  c = warp_sum(c);
  if (lane_id() == 0 && c) atomicAdd(out, c);
}

constexpr int kSlmQ = 8;            // slm_warp rows: at most 256 entries
constexpr int64_t kSlmWarpMax = 32 * kSlmQ;
constexpr int kSlmThreads = 256;

// State and scratch of the SLM local moving on one graph.
template <typename W>
struct SlmLevel {
  dcd_ctx* c;
  Csr<W> g;
  const int64_t* k;
  int64_t m2;
  Buf<int64_t> a;
  Buf<int32_t> size, next, minid, prop;
  Buf<unsigned long long> scal;  // [0] moves, [1] in, [2..3] sum a^2
  int64_t passes = 0, moves = 0, edges = 0;

  int init() {
    DCD_TRY(a.alloc(&c->mem, g.n));
    DCD_TRY(size.alloc(&c->mem, g.n));
    DCD_TRY(next.alloc(&c->mem, g.n));
    DCD_TRY(minid.alloc(&c->mem, 2 * g.n));
    DCD_TRY(prop.alloc(&c->mem, g.n));
    DCD_TRY(scal.alloc(&c->mem, 4));
    return DCD_OK;
  }

  // a, size of labels L (in [0, n))
  int sums(const int32_t* L) {
    DCD_TRY_CUDA(cudaMemsetAsync(a.get(), 0, g.n * sizeof(int64_t), c->stream));
    DCD_TRY_CUDA(cudaMemsetAsync(size.get(), 0, g.n * sizeof(int32_t), c->stream));
    ::dcd::count_launch(), comm_sums<<<grid_for(g.n, kCsThreads, 2), kCsThreads, 0, c->stream>>>(
        g.n, L, k, (unsigned long long*)a.get(), size.get());
    DCD_LAUNCH_CHECK();
    return DCD_OK;
  }

  // N = m2 * in - sum a^2 of labels L (Eq. 1 scaled by m2^2), exact
  int modularity_N(const int32_t* L, i128* N) {
    const int T = 256;
    DCD_TRY(sums(L));
    DCD_TRY_CUDA(cudaMemsetAsync(scal.get() + 1, 0, 3 * sizeof(unsigned long long), c->stream));
    ::dcd::count_launch(), slm_in_sum<W><<<grid_for(g.n * 32, T), T, 0, c->stream>>>(g.n, g.rp, g.col, g.w, L,
                                                                                      scal.get() + 1);
    ::dcd::count_launch(), slm_sumsq<<<grid_for(g.n, T, 4), T, 0, c->stream>>>(a.get(), g.n, scal.get() + 2);
    DCD_LAUNCH_CHECK();
    DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch + 20, scal.get() + 1, 3 * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, c->stream));
    DCD_TRY_CUDA(cudaStreamSynchronize(c->stream));
    const unsigned long long in = (unsigned long long)c->hscratch[20];
    const unsigned __int128 sq = ((unsigned __int128)(unsigned long long)c->hscratch[22] << 64) |
                                 (unsigned long long)c->hscratch[21];
    *N = (i128)m2 * (i128)in - (i128)sq;
    return DCD_OK;
  }

  // The local moving of one level over the vertices of `active` (NULL: all)
  // with positive degree, from canonical labels L (modified in place).
  template <typename ST>
  int run(int32_t* L, const int32_t* parent, const uint8_t* active) {
    cudaStream_t s = c->stream;
    DevScalars* d = c->dsc.get();
    const int T = 256;
    const int64_t n = g.n;
    // the vertices to evaluate, split at kSlmWarpMax and kLargeRows entries
    BinPlan plan;
    plan.nb = 2;
    plan.var[0] = kLmWarp256;
    plan.hi[0] = kSlmWarpMax;
    plan.var[1] = kLmHub;
    plan.hi[1] = INT64_MAX;
    DCD_TRY_CUDA(cudaMemsetAsync(&d->act_deg, 0, 2 * sizeof(int64_t), s));
    DCD_TRY_CUDA(cudaMemsetAsync(&d->bcnt[0], 0, 3 * kMaxBins * sizeof(int64_t), s));
    ::dcd::count_launch(), bin_count<<<grid_for(n, T), T, 0, s>>>(g.rp, n, active, d, nullptr, nullptr, plan,
                                                                   nullptr);
    DCD_LAUNCH_CHECK();
    DCD_TRY_CUDA(cudaMemcpyAsync(c->hsc, d, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    DCD_TRY_CUDA(cudaStreamSynchronize(s));
    const int64_t cnt0 = c->hsc->bcnt[0], cnt1 = c->hsc->bcnt[1], maxd1 = c->hsc->bmax[1];
    const int64_t act_deg = c->hsc->act_deg, total = cnt0 + cnt1;
    Buf<int32_t> list, cursor;
    DCD_TRY(list.alloc(&c->mem, total > 0 ? total : 1));
    DCD_TRY(cursor.alloc(&c->mem, kMaxBins));
    DCD_TRY_CUDA(cudaMemsetAsync(cursor.get(), 0, kMaxBins * sizeof(int32_t), s));
    if (total)
      ::dcd::count_launch(), bin_scatter<<<grid_for(n, T), T, 0, s>>>(g.rp, n, active, d, cursor.get(), list.get(),
                                                                       nullptr, nullptr, plan);
    // CTA tables in global memory for the long rows
    using VT = typename TblVal<ST>::type;
    const uint32_t tcap = cnt1 ? table_cap(maxd1) : 64;
    const int64_t by_mem = ((int64_t)512 << 20) / ((int64_t)tcap * (4 + sizeof(VT) + 4));
    int64_t ctas = cnt1 < 2 * (int64_t)c->sms ? cnt1 : 2 * (int64_t)c->sms;
    if (ctas > by_mem) ctas = by_mem > 0 ? by_mem : 1;
    Buf<int32_t> tk;
    Buf<VT> tv;
    Buf<uint32_t> tsl;
    if (cnt1) {
      DCD_TRY(tk.alloc(&c->mem, (size_t)ctas * tcap));
      DCD_TRY(tv.alloc(&c->mem, (size_t)ctas * tcap));
      DCD_TRY(tsl.alloc(&c->mem, (size_t)ctas * tcap));
    }
    constexpr size_t smem = (size_t)8 * row_tbl_bytes<kSlmWarpMax, VT>();
    DCD_TRY_CUDA(cudaFuncSetAttribute(slm_warp<W, ST, kSlmQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    LV<W> lv{g.rp, g.col, g.w, k, L, a.get(), size.get(), m2};
    i128 N_old = 0;
    DCD_TRY(modularity_N(L, &N_old));
    int64_t cycle_moves = 0;
    while (passes < c->cfg.max_iters) {
      const int up = (int)(passes & 1);
      DCD_TRY(sums(L));
      if (cnt0)
        ::dcd::count_launch(), slm_warp<W, ST, kSlmQ><<<grid_for(cnt0 * 32, T), T, smem, s>>>(
            lv, parent, up, n, list.get(), cnt0, prop.get());
      if (cnt1)
        ::dcd::count_launch(), slm_cta<W, ST><<<(unsigned)ctas, kSlmThreads, 0, s>>>(
            lv, parent, up, n, list.get() + cnt0, cnt1, prop.get() + cnt0, tk.get(), tv.get(), tsl.get(), tcap);
      DCD_LAUNCH_CHECK();
      DCD_TRY_CUDA(cudaMemcpyAsync(next.get(), L, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
      DCD_TRY_CUDA(cudaMemsetAsync(scal.get(), 0, sizeof(unsigned long long), s));
      if (total)
        ::dcd::count_launch(), slm_apply<<<grid_for(total, T), T, 0, s>>>(list.get(), total, prop.get(), next.get(), L,
                                                                          scal.get());
      ::dcd::count_launch(), fill_i32<<<grid_for(2 * n, T), T, 0, s>>>(minid.get(), 2 * n, INT32_MAX);
      ::dcd::count_launch(), canon_min<<<grid_for(n, T), T, 0, s>>>(n, next.get(), minid.get());
      ::dcd::count_launch(), canon_apply<<<grid_for(n, T), T, 0, s>>>(n, next.get(), minid.get(), L);
      DCD_LAUNCH_CHECK();
      DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch + 24, scal.get(), sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                   s));
      DCD_TRY_CUDA(cudaStreamSynchronize(s));
      const int64_t mv = c->hscratch[24];
      passes++;
      edges += act_deg;
      moves += mv;
      cycle_moves += mv;
      if (!up) continue;
      if (cycle_moves == 0) break;
      cycle_moves = 0;
      i128 N_new = 0;
      DCD_TRY(modularity_N(L, &N_new));
      if (h_below_tau(N_new - N_old, N_old, c->cfg.tau_inv)) break;
      N_old = N_new;
    }
    return DCD_OK;
  }
};

template <typename W>
int slm_level(dcd_ctx* c, const Csr<W>& g, const int64_t* k, int64_t m2, int32_t* L, const int32_t* parent,
              const uint8_t* active, int64_t* passes, int64_t* moves, int64_t* edges) {
  SlmLevel<W> lv{c, g, k, m2};
  DCD_TRY(lv.init());
  if (m2 >= ((int64_t)1 << 31)) DCD_TRY(lv.template run<i128>(L, parent, active));
  else DCD_TRY(lv.template run<long long>(L, parent, active));
  *passes = lv.passes;
  *moves = lv.moves;
  if (edges) *edges = lv.edges;
  return DCD_OK;
}

template <typename W>
int slm_N(dcd_ctx* c, const Csr<W>& g, const int64_t* k, int64_t m2, const int32_t* L, i128* N) {
  SlmLevel<W> lv{c, g, k, m2};
  DCD_TRY(lv.init());
  return lv.modularity_N(L, N);
}

}  // namespace

// Multi-level SLM from level-0 labels (canonical or not), level-0 active
// flags (NULL = all), k and 2m of G_t (one graph a context).  Canonical
// labels to out_labels; stats as run_louvain's.
int run_slm(dcd_ctx* c, const Csr<int32_t>& g0, int32_t* labels0, const uint8_t* active0, Buf<int64_t>& k0,
            int32_t* out_labels, dcd_step_stats* st) {
  cudaStream_t s = c->stream;
  const int T = 256;
  const int64_t n0 = g0.n;
  const int64_t m2 = c->hgs[0].m2;
  Buf<int32_t> comp, L, minid;
  DCD_TRY(comp.alloc(&c->mem, n0));
  DCD_TRY(L.alloc(&c->mem, n0));
  DCD_TRY(minid.alloc(&c->mem, 2 * n0));
  ::dcd::count_launch(), fill_iota<<<grid_for(n0, T), T, 0, s>>>(comp.get(), n0);
  ::dcd::count_launch(), fill_i32<<<grid_for(2 * n0, T), T, 0, s>>>(minid.get(), 2 * n0, INT32_MAX);
  ::dcd::count_launch(), canon_min<<<grid_for(n0, T), T, 0, s>>>(n0, labels0, minid.get());
  ::dcd::count_launch(), canon_apply<<<grid_for(n0, T), T, 0, s>>>(n0, labels0, minid.get(), L.get());
  DCD_LAUNCH_CHECK();
  i128 N_start = 0, N_end = 0;
  DCD_TRY(slm_N<int32_t>(c, g0, k0.get(), m2, L.get(), &N_start));
  int64_t level = 0, iters_total = 0, iters0 = 0, moves_total = 0, edges_total = 0, refine_iters = 0,
          refine_moves = 0;
  float ms_lm = 0.f, ms_coarsen = 0.f;
  CoarseGraph cg[2];
  Buf<int64_t> kc[2];
  Buf<int32_t> Lc[2];
  int which = 0;
  const Csr<int64_t>* gc = nullptr;
  int32_t* Lcur = L.get();
  const int64_t* kcur = k0.get();
  const uint8_t* active = active0;
  int64_t nv = n0;
  for (;;) {
    DCD_TRY_CUDA(cudaEventRecord(c->ev[2], s));
    int64_t it = 0, mv = 0, ed = 0, rit = 0, rmv = 0;
    Buf<int32_t> sub;
    DCD_TRY(sub.alloc(&c->mem, nv));
    if (level == 0) {
      DCD_TRY(slm_level<int32_t>(c, g0, kcur, m2, Lcur, nullptr, active, &it, &mv, &ed));
      DCD_TRY(slm_N<int32_t>(c, g0, kcur, m2, Lcur, &N_end));
      ::dcd::count_launch(), fill_iota<<<grid_for(nv, T), T, 0, s>>>(sub.get(), nv);
      DCD_TRY(slm_level<int32_t>(c, g0, kcur, m2, sub.get(), Lcur, nullptr, &rit, &rmv, nullptr));
    } else {
      DCD_TRY(slm_level<int64_t>(c, *gc, kcur, m2, Lcur, nullptr, nullptr, &it, &mv, &ed));
      DCD_TRY(slm_N<int64_t>(c, *gc, kcur, m2, Lcur, &N_end));
      ::dcd::count_launch(), fill_iota<<<grid_for(nv, T), T, 0, s>>>(sub.get(), nv);
      DCD_TRY(slm_level<int64_t>(c, *gc, kcur, m2, sub.get(), Lcur, nullptr, &rit, &rmv, nullptr));
    }
    DCD_TRY_CUDA(cudaEventRecord(c->ev[3], s));
    iters_total += it;
    if (level == 0) iters0 = it;
    moves_total += mv;
    edges_total += ed;
    refine_iters += rit;
    refine_moves += rmv;
    // sub-communities (canonical: one head each)
    Buf<unsigned long long> heads;
    DCD_TRY(heads.alloc(&c->mem, 1));
    DCD_TRY_CUDA(cudaMemsetAsync(heads.get(), 0, sizeof(unsigned long long), s));
    ::dcd::count_launch(), count_heads<<<grid_for(nv, T), T, 0, s>>>(nv, sub.get(), heads.get());
    DCD_LAUNCH_CHECK();
    DCD_TRY_CUDA(cudaMemcpyAsync(c->hscratch + 25, heads.get(), sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    DCD_TRY_CUDA(cudaStreamSynchronize(s));
    float t1 = 0.f;
    cudaEventElapsedTime(&t1, c->ev[2], c->ev[3]);
    ms_lm += t1;
    const int64_t ns = c->hscratch[25];
    level++;
    const bool stop = ns == nv || (level >= 2 && h_below_tau(N_end - N_start, N_start, c->cfg.tau_inv)) ||
                      level >= c->cfg.max_levels;
    if (stop) break;
    // aggregation by the sub-communities
    DCD_TRY_CUDA(cudaEventRecord(c->ev[5], s));
    Buf<int32_t> cid;
    int64_t nc = 0;
    const int nx = which ^ 1;
    if (level == 1) {
      DCD_TRY(used_labels<int32_t>(c, g0, sub.get(), cid, &nc, nullptr, nullptr));
      DCD_TRY(coarsen<int32_t>(c, g0, sub.get(), cid.get(), nc, &cg[nx]));
    } else {
      DCD_TRY(used_labels<int64_t>(c, *gc, sub.get(), cid, &nc, nullptr, nullptr));
      DCD_TRY(coarsen<int64_t>(c, *gc, sub.get(), cid.get(), nc, &cg[nx]));
    }
    DCD_TRY(kc[nx].alloc(&c->mem, nc));
    DCD_TRY(Lc[nx].alloc(&c->mem, nc));
    {
      // coarse k = sum of k over a sub-community
      Buf<int64_t> asub;
      Buf<int32_t> ssub;
      DCD_TRY(asub.alloc(&c->mem, nv));
      DCD_TRY(ssub.alloc(&c->mem, nv));
      DCD_TRY(community_sums(c, nv, sub.get(), kcur, asub.get(), ssub.get()));
      ::dcd::count_launch(), coarse_k<<<grid_for(nv, T), T, 0, s>>>(nv, cid.get(), asub.get(), kc[nx].get());
    }
    ::dcd::count_launch(), compose<<<grid_for(n0, T), T, 0, s>>>(n0, comp.get(), sub.get(), cid.get());
    ::dcd::count_launch(), slm_parent_start<<<grid_for(nv, T), T, 0, s>>>(nv, sub.get(), Lcur, cid.get(),
                                                                           Lc[nx].get());
    DCD_LAUNCH_CHECK();
    DCD_TRY_CUDA(cudaEventRecord(c->ev[6], s));
    DCD_TRY_CUDA(cudaEventSynchronize(c->ev[6]));
    float tc = 0.f;
    cudaEventElapsedTime(&tc, c->ev[5], c->ev[6]);
    ms_coarsen += tc;
    cg[which].rp.reset();
    cg[which].col.reset();
    cg[which].w.reset();
    kc[which].reset();
    Lc[which].reset();
    which = nx;
    gc = &cg[which].view;
    Lcur = Lc[which].get();
    kcur = kc[which].get();
    nv = nc;
    active = nullptr;
    N_start = N_end;
  }
  // compose + canonical labels (smallest member id)
  DCD_TRY_CUDA(cudaEventRecord(c->ev[7], s));
  {
    Buf<int32_t> mid;
    DCD_TRY(mid.alloc(&c->mem, nv));
    ::dcd::count_launch(), fill_i32<<<grid_for(nv, T), T, 0, s>>>(mid.get(), nv, INT32_MAX);
    ::dcd::count_launch(), final_min<<<grid_for(n0, T), T, 0, s>>>(n0, comp.get(), Lcur, mid.get());
    ::dcd::count_launch(), gs_reset_nc<<<1, 128, 0, s>>>(c->gs.get(), 1);
    ::dcd::count_launch(), final_labels<<<grid_for(n0, T), T, 0, s>>>(n0, comp.get(), Lcur, mid.get(), out_labels,
                                                                       nullptr, c->gs.get());
    DCD_LAUNCH_CHECK();
    DCD_TRY_CUDA(cudaEventRecord(c->ev[8], s));
    DCD_TRY_CUDA(cudaMemcpyAsync(c->hgs, c->gs.get(), sizeof(GraphState), cudaMemcpyDeviceToHost, s));
    DCD_TRY_CUDA(cudaStreamSynchronize(s));
  }
  float tf = 0.f;
  cudaEventElapsedTime(&tf, c->ev[7], c->ev[8]);
  if (st) {
    st->levels = level;
    st->iters_total = iters_total;
    st->iters_level0 = iters0;
    st->moves_total = moves_total;
    st->communities = c->hgs[0].ncomm;
    st->n_lo = (int64_t)(unsigned long long)N_end;
    st->n_hi = (int64_t)(unsigned long long)((unsigned __int128)N_end >> 64);
    st->m2 = m2;
    st->q = m2 == 0 ? 0.0 : (double)N_end / ((double)m2 * (double)m2);
    st->edges_scanned = edges_total;
    st->verts_scanned = 0;
    st->refine_iters = refine_iters;
    st->refine_moves = refine_moves;
    st->ms_local_move = ms_lm;
    st->ms_coarsen = ms_coarsen;
    st->ms_finish = tf;
  }
  return DCD_OK;
}

}  // namespace dcd
