// prims.cuh -- data-parallel primitives written for this library: a
// device-wide exclusive scan and an LSD radix sort of (uint64 key, value)
// pairs.  Both are deterministic (the sort is stable).
#pragma once

#include "common.cuh"

namespace dcd {

// ----------------------------------------------------------------------------
// Exclusive scan.  Tiles of 256 threads x 8 items: (1) per-tile totals,
// (2) one CTA scans the totals, (3) each tile scans itself from its offset.
// ----------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if ((int)lane_id() >= o) x += y;
  }
  return x;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Block-wide exclusive scan of one value per thread; returns the exclusive
// prefix and writes the block total to *total (shared memory).
// blockDim.x == kScanThreads.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T x, T* total) {
  constexpr int NW = kScanThreads / 32;
  __shared__ T warp_off[NW];
  T incl = warp_incl_scan(x);
  int w = threadIdx.x >> 5;
  if (lane_id() == 31) warp_off[w] = incl;
  __syncthreads();
  if (w == 0) {
    T t = lane_id() < NW ? warp_off[lane_id()] : T(0);
    T ti = warp_incl_scan(t);
    if (lane_id() < NW) warp_off[lane_id()] = ti - t;
    if (lane_id() == NW - 1) *total = ti;
  }
  __syncthreads();
  T r = incl - x + warp_off[w];
  __syncthreads();
  return r;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_tile_totals(const T* __restrict__ in, int64_t n,
                                                                 T* __restrict__ tot) {
  __shared__ T red[kScanThreads / 32];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  T s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
    if (idx < n) s += in[idx];
  }
  s = warp_sum(s);
  if (lane_id() == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    T t = threadIdx.x < kScanThreads / 32 ? red[threadIdx.x] : T(0);
    t = warp_sum(t);
    if (threadIdx.x == 0) tot[blockIdx.x] = t;
  }
}

// One CTA: exclusive scan of the tile totals in place; grand total -> *total.
template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_totals(T* __restrict__ tot, int64_t ntiles,
                                                            T* __restrict__ total) {
  __shared__ T carry_s;
  T carry = 0;
  for (int64_t base = 0; base < ntiles; base += kScanThreads) {
    int64_t idx = base + threadIdx.x;
    T x = idx < ntiles ? tot[idx] : T(0);
    T btot;
    T ex = block_excl_scan(x, &carry_s);
    btot = carry_s;
    if (idx < ntiles) tot[idx] = carry + ex;
    carry += btot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_tiles(const T* __restrict__ in, T* __restrict__ out,
                                                           int64_t n, const T* __restrict__ tile_off) {
  __shared__ T buf[kScanTile];
  __shared__ T tot_s;
  int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
    buf[i * kScanThreads + threadIdx.x] = idx < n ? in[idx] : T(0);
  }
  __syncthreads();
  T v[kScanItems];
  T s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    v[i] = buf[threadIdx.x * kScanItems + i];
    s += v[i];
  }
  T ex = block_excl_scan(s, &tot_s) + tile_off[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    buf[threadIdx.x * kScanItems + i] = ex;
    ex += v[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
    if (idx < n) out[idx] = buf[i * kScanThreads + threadIdx.x];
  }
}

// out[i] = sum_{j<i} in[i]; *total (device, may be NULL) = sum of all.
// out may alias in.  tmp needs scan_tmp_count(n) elements of T.
inline int64_t scan_tmp_count(int64_t n) { return cdiv(n, kScanTile) + 1; }

template <typename T>
int exclusive_scan(const T* in, T* out, int64_t n, T* total, T* tmp, cudaStream_t s) {
  if (n <= 0) {
    if (total) DCD_TRY_CUDA(cudaMemsetAsync(total, 0, sizeof(T), s));
    return DCD_OK;
  }
  int64_t ntiles = cdiv(n, kScanTile);
  ::dcd::count_launch(), scan_tile_totals<T><<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, n, tmp);
  ::dcd::count_launch(), scan_totals<T><<<1, kScanThreads, 0, s>>>(tmp, ntiles, total);
  ::dcd::count_launch(), scan_tiles<T><<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, out, n, tmp);
  DCD_LAUNCH_CHECK();
  return DCD_OK;
}

// ----------------------------------------------------------------------------
// LSD radix sort, 8-bit digits.  Per pass: per-tile digit histograms, a scan
// of the (digit-major) histogram table, and a stable scatter that ranks keys
// inside a tile with warp match + per-warp digit counts.
// ----------------------------------------------------------------------------
constexpr int kRsThreads = 256;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems;
constexpr int kRsWarps = kRsThreads / 32;

static __global__ void __launch_bounds__(kRsThreads) rs_histogram(const uint64_t* __restrict__ keys, int64_t n,
                                                           int shift, uint32_t* __restrict__ counts,
                                                           int64_t ntiles) {
  __shared__ uint32_t hist[256];
  hist[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kRsTile;
#pragma unroll
  for (int i = 0; i < kRsItems; i++) {
    int64_t idx = base + (int64_t)i * kRsThreads + threadIdx.x;
    if (idx < n) atomicAdd(&hist[(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = hist[threadIdx.x];
}

template <typename V>
__global__ void __launch_bounds__(kRsThreads) rs_scatter(const uint64_t* __restrict__ kin,
                                                         const V* __restrict__ vin, uint64_t* __restrict__ kout,
                                                         V* __restrict__ vout, int64_t n, int shift,
                                                         const uint32_t* __restrict__ offsets, int64_t ntiles) {
  __shared__ uint32_t base_s[256];
  __shared__ uint32_t round_s[256];
  __shared__ uint32_t wcnt[kRsWarps][256];
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  base_s[t] = offsets[(int64_t)t * ntiles + blockIdx.x];
#pragma unroll
  for (int x = 0; x < kRsWarps; x++) wcnt[x][t] = 0;
  __syncthreads();
  int64_t tile0 = (int64_t)blockIdx.x * kRsTile;
  for (int r = 0; r < kRsItems; r++) {
    int64_t idx = tile0 + (int64_t)r * kRsThreads + t;
    bool valid = idx < n;
    uint64_t k = valid ? kin[idx] : 0;
    V v = valid ? vin[idx] : V(0);
    uint32_t d = valid ? (uint32_t)((k >> shift) & 255u) : 256u;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    unsigned rank = __popc(peers & lanemask_lt());
    if (valid && rank == 0) wcnt[w][d] = __popc(peers);
    __syncthreads();
    {  // thread t owns digit t: exclusive prefix over warps
      uint32_t run = 0;
#pragma unroll
      for (int x = 0; x < kRsWarps; x++) {
        uint32_t c = wcnt[x][t];
        wcnt[x][t] = run;
        run += c;
      }
      round_s[t] = base_s[t];
      base_s[t] += run;
    }
    __syncthreads();
    if (valid) {
      uint32_t pos = round_s[d] + wcnt[w][d] + rank;
      kout[pos] = k;
      vout[pos] = v;
    }
    __syncthreads();
#pragma unroll
    for (int x = 0; x < kRsWarps; x++) wcnt[x][t] = 0;
    __syncthreads();
  }
  (void)lane;
}

// Temporary storage (in uint32 words) for sort_pairs of n items.
inline int64_t sort_tmp_words(int64_t n) {
  int64_t ntiles = cdiv(n > 0 ? n : 1, kRsTile);
  return 256 * ntiles + scan_tmp_count(256 * ntiles) + 2;
}

// Sorts (keys, vals) by the key bits in [lo0, hi0) then [lo1, hi1) (bits
// outside both ranges must be equal across keys or be ignorable).  Ping-pongs
// between (k0, v0) and (k1, v1); *result_in_1 tells which holds the output.
template <typename V>
int sort_pairs(uint64_t* k0, V* v0, uint64_t* k1, V* v1, int64_t n, const int* bit_ranges, int nranges,
               uint32_t* tmp, bool* result_in_1, cudaStream_t s) {
  *result_in_1 = false;
  if (n <= 1) return DCD_OK;
  if (n >= (int64_t)UINT32_MAX) return DCD_EINVAL;
  int64_t ntiles = cdiv(n, kRsTile);
  uint32_t* counts = tmp;
  uint32_t* scan_tmp = tmp + 256 * ntiles;
  uint64_t* ka = k0;
  uint64_t* kb = k1;
  V* va = v0;
  V* vb = v1;
  for (int r = 0; r < nranges; r++) {
    for (int b = bit_ranges[2 * r]; b < bit_ranges[2 * r + 1]; b += 8) {
      ::dcd::count_launch(), rs_histogram<<<(unsigned)ntiles, kRsThreads, 0, s>>>(ka, n, b, counts, ntiles);
      DCD_TRY(exclusive_scan<uint32_t>(counts, counts, 256 * ntiles, nullptr, scan_tmp, s));
      ::dcd::count_launch(), rs_scatter<V><<<(unsigned)ntiles, kRsThreads, 0, s>>>(ka, va, kb, vb, n, b, counts, ntiles);
      DCD_LAUNCH_CHECK();
      uint64_t* tk = ka;
      ka = kb;
      kb = tk;
      V* tv = va;
      va = vb;
      vb = tv;
      *result_in_1 = !*result_in_1;
    }
  }
  return DCD_OK;
}

inline int bits_for(int64_t maxval) {
  int b = 0;
  while (b < 63 && ((int64_t)1 << b) <= maxval) b++;
  return b;
}

}  // namespace dcd
