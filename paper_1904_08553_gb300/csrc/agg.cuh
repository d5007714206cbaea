// agg.cuh -- neighbour-community aggregation shared by the local-move and
// screening kernels: exact group sums inside a warp, open-addressing tables
// (community label -> summed edge weight) in shared or global memory, the
// exact integer gain S and a total-order argmax.
#pragma once

#include <climits>

#include "common.cuh"

namespace dcd {

// Gain of moving v from C to D (Sec. III-A; expanded form in the appendix
// proof of Lemma 3.2):  S = m2 (e_{v->D} - e_{v->C\v}) - k_v (a_D - (a_C - k_v)),
// i.e. (2m)^2 times the paper's Delta Q_{v->D}.  ST = int64 is exact when
// m2 < 2^31 (both products stay below 2^62); otherwise ST = int128.
template <typename ST>
__device__ __forceinline__ ST gain(int64_t m2, int64_t kv, int64_t eD, int64_t eC, int64_t aD, int64_t aC) {
  return (ST)m2 * (ST)(eD - eC) - (ST)kv * (ST)(aD - aC + kv);
}

template <typename ST>
__device__ __forceinline__ ST gain_lowest();
template <>
__device__ __forceinline__ long long gain_lowest<long long>() {
  return LLONG_MIN;
}
template <>
__device__ __forceinline__ i128 gain_lowest<i128>() {
  return -((i128)1 << 126) * 2;
}

__device__ __forceinline__ long long shfl_xor_st(long long x, int o) { return __shfl_xor_sync(0xffffffffu, x, o); }
__device__ __forceinline__ i128 shfl_xor_st(i128 x, int o) {
  unsigned long long lo = (unsigned long long)x, hi = (unsigned long long)(x >> 64);
  lo = __shfl_xor_sync(0xffffffffu, lo, o);
  hi = __shfl_xor_sync(0xffffffffu, hi, o);
  return (i128)(((unsigned __int128)hi << 64) | lo);
}
__device__ __forceinline__ long long shfl_st(long long x, int src) { return __shfl_sync(0xffffffffu, x, src); }
__device__ __forceinline__ i128 shfl_st(i128 x, int src) {
  unsigned long long lo = (unsigned long long)x, hi = (unsigned long long)(x >> 64);
  lo = __shfl_sync(0xffffffffu, lo, src);
  hi = __shfl_sync(0xffffffffu, hi, src);
  return (i128)(((unsigned __int128)hi << 64) | lo);
}

// The move a vertex in community C proposes from its best (S, D) over the
// neighbouring communities D != C (Algorithm 1's rule, synchronous reading):
// move iff S > 0 (staying wins ties); a singleton does not move into a
// singleton of larger label (the minimum-label guard against two singletons
// swapping).  size: community sizes under the pass's snapshot.
template <typename ST>
__device__ __forceinline__ int32_t move_proposal(ST S, int32_t D, int32_t C, const int32_t* size) {
  const bool mv = D != INT_MAX && S > 0;
  const int32_t Dm = mv ? D : C;
  const int32_t sC = size[C], sD = size[Dm];
  return (mv && sC == 1 && sD == 1 && Dm > C) ? C : Dm;
}

// (S, D) order of the greedy choice: larger gain first, then smaller label.
template <typename ST>
__device__ __forceinline__ bool better(ST s1, int32_t d1, ST s2, int32_t d2) {
  return s1 > s2 || (s1 == s2 && d1 < d2);
}

// Whole-warp argmax of (S, D); every lane ends with the result (128-bit gains).
__device__ __forceinline__ void warp_argmax(i128& S, int32_t& D) {
  using ST = i128;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ST s2 = shfl_xor_st(S, o);
    int32_t d2 = __shfl_xor_sync(0xffffffffu, D, o);
    if (better(s2, d2, S, D)) {
      S = s2;
      D = d2;
    }
  }
}

// Whole-warp argmax of (S, D) for 64-bit gains with redux.sync over the full
// warp: the maximum of the high words, then of the low words among the lanes
// holding that high word, then the smallest label among the lanes holding
// the maximum (labels are >= 0, the sentinel INT_MAX).  Lanes outside each
// step contribute the neutral value, so no lane diverges.
__device__ __forceinline__ void warp_argmax(long long& S, int32_t& D) {
  const unsigned long long u = (unsigned long long)S ^ 0x8000000000000000ull;
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
  const unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
  const bool top = hi == mhi && lo == mlo;
  const unsigned dmin = __reduce_min_sync(0xffffffffu, top ? (unsigned)D : 0xffffffffu);
  S = (long long)((((unsigned long long)mhi << 32) | mlo) ^ 0x8000000000000000ull);
  D = (int32_t)dmin;
}

// Argmax of (S, D) over the SEG-lane segment of the calling lane (mask: that
// segment's lanes); SEG = 32 is the whole warp.
template <int SEG>
__device__ __forceinline__ void seg_argmax(long long& S, int32_t& D, unsigned mask) {
  const unsigned long long u = (unsigned long long)S ^ 0x8000000000000000ull;
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned mhi = __reduce_max_sync(mask, hi);
  const unsigned mlo = __reduce_max_sync(mask, hi == mhi ? lo : 0u);
  const bool top = hi == mhi && lo == mlo;
  const unsigned dmin = __reduce_min_sync(mask, top ? (unsigned)D : 0xffffffffu);
  S = (long long)((((unsigned long long)mhi << 32) | mlo) ^ 0x8000000000000000ull);
  D = (int32_t)dmin;
}
template <int SEG>
__device__ __forceinline__ void seg_argmax(i128& S, int32_t& D, unsigned) {
#pragma unroll
  for (int o = SEG / 2; o > 0; o >>= 1) {
    const i128 s2 = shfl_xor_st(S, o);
    const int32_t d2 = __shfl_xor_sync(0xffffffffu, D, o);
    if (better(s2, d2, S, D)) {
      S = s2;
      D = d2;
    }
  }
}

// Exact sum of non-negative weights over the lanes of `peers` (a match_any
// group), from 16-bit slices reduced with redux.sync: no slice sum can carry
// out of 32 bits, so the result is exact for any int32/int64 weight.
__device__ __forceinline__ int64_t group_sum_exact(unsigned peers, int32_t w) {
  unsigned lo = (unsigned)w & 0xffffu, hi = (unsigned)w >> 16;
  unsigned slo = __reduce_add_sync(peers, lo);
  unsigned shi = __reduce_add_sync(peers, hi);
  return (int64_t)slo + ((int64_t)shi << 16);
}
__device__ __forceinline__ int64_t group_sum_exact(unsigned peers, int64_t w) {
  unsigned long long x = (unsigned long long)w;
  int64_t s = 0;
#pragma unroll
  for (int q = 0; q < 4; q++) {
    unsigned part = (unsigned)(x >> (16 * q)) & 0xffffu;
    s += (int64_t)__reduce_add_sync(peers, part) << (16 * q);
  }
  return s;
}

// Sum of weights over the lanes of `peers` as the gain arithmetic needs it:
// with 64-bit gains 2m < 2^31, so every sum of a vertex's weights is below
// 2^31 and one 32-bit reduction is exact; with 128-bit gains the sum is
// taken exactly from 16-bit slices.
template <typename ST, typename W>
__device__ __forceinline__ int64_t group_sum(unsigned peers, W w);
template <>
__device__ __forceinline__ int64_t group_sum<long long, int32_t>(unsigned peers, int32_t w) {
  return (int64_t)__reduce_add_sync(peers, (unsigned)w);
}
template <>
__device__ __forceinline__ int64_t group_sum<long long, int64_t>(unsigned peers, int64_t w) {
  return (int64_t)__reduce_add_sync(peers, (unsigned)w);
}
template <>
__device__ __forceinline__ int64_t group_sum<i128, int32_t>(unsigned peers, int32_t w) {
  return group_sum_exact(peers, w);
}
template <>
__device__ __forceinline__ int64_t group_sum<i128, int64_t>(unsigned peers, int64_t w) {
  return group_sum_exact(peers, w);
}

// ---- open-addressing table: key -1 = empty; capacity a power of two that is
// at least twice the number of distinct keys, so probing always ends. ----
__device__ __forceinline__ void tbl_add(int32_t* keys, unsigned long long* vals, uint32_t mask, int32_t lab,
                                        unsigned long long x) {
  uint32_t s = hash_label(lab, mask);
  for (;;) {
    int32_t k = keys[s];
    if (k == lab) {
      atomicAdd(&vals[s], x);
      return;
    }
    if (k == -1) {
      int32_t old = atomicCAS(&keys[s], -1, lab);
      if (old == -1 || old == lab) {
        atomicAdd(&vals[s], x);
        return;
      }
    }
    s = (s + 1) & mask;
  }
}

// tbl_add that also appends each newly claimed slot to slots[] (counter *ns),
// so the distinct keys can be visited, and the table emptied again, without a
// scan over the whole capacity.
template <typename VT>
__device__ __forceinline__ void tbl_add_list(int32_t* keys, VT* vals, uint16_t* slots, int32_t* ns, uint32_t mask,
                                             int32_t lab, VT x) {
  uint32_t s = hash_label(lab, mask);
  for (;;) {
    int32_t k = keys[s];
    if (k == lab) {
      atomicAdd(&vals[s], x);
      return;
    }
    if (k == -1) {
      const int32_t old = atomicCAS(&keys[s], -1, lab);
      if (old == -1) slots[atomicAdd(ns, 1)] = (uint16_t)s;
      if (old == -1 || old == lab) {
        atomicAdd(&vals[s], x);
        return;
      }
    }
    s = (s + 1) & mask;
  }
}

template <typename VT>
__device__ __forceinline__ int64_t tbl_get(const int32_t* keys, const VT* vals, uint32_t mask, int32_t lab) {
  uint32_t s = hash_label(lab, mask);
  for (;;) {
    int32_t k = keys[s];
    if (k == lab) return (int64_t)vals[s];
    if (k == -1) return 0;
    s = (s + 1) & mask;
  }
}

// Width of the shared-table sums: with 64-bit gains 2m < 2^31 bounds every
// sum of a vertex's weights, so 32 bits hold them exactly (smaller tables,
// more warps per SM); with 128-bit gains the sums are 64-bit.
template <typename ST>
struct TblVal {
  using type = unsigned long long;
};
template <>
struct TblVal<long long> {
  using type = unsigned;
};

// The slot of `lab` in the table (claimed when absent); `claimed` is set when
// this call took an empty slot for it.
__device__ __forceinline__ uint32_t probe_claim(int32_t* keys, uint32_t mask, int32_t lab, bool& claimed) {
  uint32_t s = hash_label(lab, mask);
  for (;;) {
    const int32_t k = keys[s];
    if (k == lab) return s;
    if (k == -1) {
      const int32_t old = atomicCAS(&keys[s], -1, lab);
      if (old == -1) {
        claimed = true;
        return s;
      }
      if (old == lab) return s;
    }
    s = (s + 1) & mask;
  }
}

// Sum over the S lanes of the calling lane's segment: 32-bit sums are exact
// with 64-bit gains (every sum of a vertex's weights is below 2m < 2^31),
// 64-bit sums with 128-bit gains.
template <int S>
__device__ __forceinline__ int64_t seg_total(unsigned x, unsigned smask) {
  return (int64_t)__reduce_add_sync(smask, x);
}
template <int S>
__device__ __forceinline__ int64_t seg_total(unsigned long long x, unsigned) {
#pragma unroll
  for (int o = S / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return (int64_t)x;
}

__host__ __device__ __forceinline__ uint32_t table_cap(int64_t deg) {
  uint32_t c = 64;
  while ((int64_t)c < 2 * deg) c <<= 1;
  return c;
}

}  // namespace dcd
