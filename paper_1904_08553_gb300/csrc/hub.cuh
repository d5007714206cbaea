// hub.cuh -- aggregation of very long rows (hubs) over many CTAs, shared by
// the local-move kernels and the screening kernels.
//
// A hub's row is split into chunks of kHubChunk entries, so that many CTAs
// work on one hub at once (one CTA per hub would leave the largest hub setting
// the kernel's length).  Each hub owns a region of a global open-addressing
// table (capacity: 2 x degree rounded up to a power of two, so probing always
// ends) and of a list of the slots it claimed:
//   hub_agg   chunk c of hub h: group the chunk's labels by warp (match_any),
//             add the group sums into h's table, list new keys.
// The caller then reads the tables (gains, lookups) and, to reuse them,
// empties the claimed slots.  The view V has rp, col, w and L.
#pragma once

#include "agg.cuh"
#include "state.cuh"

namespace dcd {

constexpr int64_t kHubChunk = 4096;

struct HubTables {
  const int32_t* list = nullptr;  // hub vertices (the bin's list segment)
  int64_t H = 0;                  // hubs
  const int64_t* toff = nullptr;  // table offset of hub h (H + 1)
  const int64_t* soff = nullptr;  // claimed-slot list offset of hub h (H + 1)
  const int64_t* coff = nullptr;  // first chunk of hub h (H + 1)
  int32_t* keys = nullptr;        // all tables (-1: empty)
  unsigned long long* vals = nullptr;
  int32_t* slots = nullptr;       // claimed-slot lists (table-relative slot)
  int32_t* nslot = nullptr;       // claimed slots of hub h (this pass)
  int32_t* nprev = nullptr;       // the same, kept for hub_clear
  long long* part = nullptr;      // per chunk: gain (2 words), label
};

__device__ __forceinline__ int64_t hub_of_chunk(const HubTables& t, int64_t c) {
  int64_t lo = 0, hi = t.H - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (t.coff[mid] <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename W, typename ST, typename V>
__global__ void __launch_bounds__(256) hub_agg(V g, HubTables t) {
  const int lane = lane_id(), wib = threadIdx.x >> 5;
  const int64_t nch = t.coff[t.H];
  for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
    const int64_t h = hub_of_chunk(t, c);
    const int32_t v = t.list[h];
    const int64_t b = g.rp[v], d = g.rp[v + 1] - b;
    const int64_t e0 = (c - t.coff[h]) * kHubChunk, e1 = e0 + kHubChunk < d ? e0 + kHubChunk : d;
    const uint32_t mask = (uint32_t)(t.toff[h + 1] - t.toff[h]) - 1;
    int32_t* keys = t.keys + t.toff[h];
    unsigned long long* vals = t.vals + t.toff[h];
    int32_t* slots = t.slots + t.soff[h];
    for (int64_t q0 = e0 + wib * 32; q0 < e1; q0 += blockDim.x) {
      const int64_t e = q0 + lane;
      bool valid = e < e1;
      const int32_t u = valid ? ld_stream(g.col + b + e) : -1;
      valid = valid && u != v;
      const int32_t lab = valid ? g.L[u] : -1;
      const W wt = valid ? ld_stream(g.w + b + e) : W(0);
      const unsigned peers = __match_any_sync(0xffffffffu, lab);
      const int64_t sum = group_sum<ST>(peers, wt);
      if (valid && (int)(__ffs(peers) - 1) == lane) {
        uint32_t sl = hash_label(lab, mask);
        for (;;) {
          const int32_t k = keys[sl];
          if (k == lab) {
            atomicAdd(&vals[sl], (unsigned long long)sum);
            break;
          }
          if (k == -1) {
            const int32_t old = atomicCAS(&keys[sl], -1, lab);
            if (old == -1) slots[atomicAdd(&t.nslot[h], 1)] = (int32_t)sl;
            if (old == -1 || old == lab) {
              atomicAdd(&vals[sl], (unsigned long long)sum);
              break;
            }
          }
          sl = (sl + 1) & mask;
        }
      }
    }
  }
}


// sizes of the hub tables (hub h: table 2 x degree rounded up to a power of
// two, slot list = degree, chunks = degree / kHubChunk rounded up)
template <int UNUSED>
__global__ void hub_sizes(const int32_t* __restrict__ list, int64_t H, const int64_t* __restrict__ rp,
                          int64_t* __restrict__ cap, int64_t* __restrict__ deg, int64_t* __restrict__ nch) {
  for (int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; h < H; h += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = list[h];
    const int64_t d = rp[v + 1] - rp[v];
    cap[h] = table_cap(d);
    deg[h] = d;
    nch[h] = cdiv(d, kHubChunk);
  }
}

// Device buffers behind a HubTables view (step arena).
struct HubBufs {
  Buf<int64_t> toff, soff, coff;
  Buf<int32_t> keys, slots, nslot, nprev;
  Buf<unsigned long long> vals;
  Buf<long long> part;
  int64_t chunks = 0;
  HubTables t;
};

// louvain.cu: sizes, offsets and empty tables for the H hubs of list.
int hub_setup(dcd_ctx* c, const int32_t* list, int64_t H, const int64_t* rp, HubBufs* b);
// CTAs for a launch over the hubs' chunks.
unsigned hub_grid(dcd_ctx* c, const HubBufs& b);

}  // namespace dcd
