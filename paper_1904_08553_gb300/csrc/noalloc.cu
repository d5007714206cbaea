// noalloc.cu -- dcd_modularity_noalloc: modularity of a partition on a
// caller-owned device CSR, computed without allocating any device memory.
//
// Why it exists: some callers cannot allocate device memory at the moment
// they need an answer -- code whose device memory is already fully reserved
// by another allocator (a framework's caching allocator holding the free
// memory), code running where cudaMalloc/cudaFree must not be called (a host
// callback on a stream) or must not add their implicit synchronisation.  This
// entry point takes its scratch (community degree sums and reduction
// partials) from one fixed array in device memory that the library reserves
// at load time, on every GPU that loads it, until the process exits.
//
// Limits and sharing: at most kNoAllocMaxN labels (the array holds 8 MiB).
// Every call on a device uses the same array and leaves its contents behind;
// each call clears what it needs first, so consecutive calls are independent,
// but two calls whose device work overlaps (different streams, or different
// host threads) race on the array and give wrong results.
#include <cstring>

#include "prims.cuh"
#include "state.cuh"

namespace dcd {
namespace {

constexpr int64_t kNoAllocWords = (int64_t)1 << 20;  // 8 MiB of 64-bit words
constexpr int kNoAllocCtas = 256;                     // partials of the sum of squares
constexpr int64_t kNoAllocTail = 8;                   // m2, in, N lo/hi, error word
constexpr int64_t kNoAllocMaxN = kNoAllocWords - 2 * kNoAllocCtas - kNoAllocTail;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocWords];

// tail words: [0] m2, [1] in, [2] N lo, [3] N hi, [4] error flag
__global__ void na_clear(unsigned long long* s, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s[i] = 0;
  if (blockIdx.x == 0 && threadIdx.x < kNoAllocTail) s[kNoAllocWords - kNoAllocTail + threadIdx.x] = 0;
}

// Per row u: d_w(u), the intra-community weight of the row, and a_C += d_w(u).
__global__ void na_rows(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                        const int32_t* __restrict__ w, const int32_t* __restrict__ L, unsigned long long* s) {
  unsigned long long* tail = s + kNoAllocWords - kNoAllocTail;
  unsigned long long m2 = 0, in = 0;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
    const int32_t Lu = L[u];
    const bool ok = Lu >= 0 && Lu < n;
    unsigned long long ks = 0, is = 0;
    for (int64_t e = rp[u] + lane_id(); e < rp[u + 1]; e += 32) {
      const int32_t y = col[e];
      const unsigned long long wv = (unsigned long long)(int64_t)w[e];
      ks += wv;
      if (y >= 0 && y < n && L[y] == Lu) is += wv;
      if (y < 0 || y >= n) tail[4] = 1;
    }
    ks = warp_sum(ks);
    is = warp_sum(is);
    if (lane_id() == 0) {
      if (ok) atomicAdd(&s[Lu], ks);
      else tail[4] = 1;
    }
    m2 += ks;
    in += is;
  }
  if (lane_id() == 0) {
    atomicAdd(&tail[0], m2);
    atomicAdd(&tail[1], in);
  }
}

__global__ void na_sumsq(int64_t n, unsigned long long* s) {
  __shared__ unsigned long long lo_s[8], hi_s[8];
  unsigned __int128 acc = 0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
    acc += (unsigned __int128)s[c] * s[c];
  unsigned long long lo = (unsigned long long)acc, hi = (unsigned long long)(acc >> 64);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long lo2 = __shfl_xor_sync(0xffffffffu, lo, o), hi2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const unsigned long long nl = lo + lo2;
    hi = hi + hi2 + (nl < lo ? 1ull : 0ull);
    lo = nl;
  }
  if (lane_id() == 0) {
    lo_s[threadIdx.x >> 5] = lo;
    hi_s[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned __int128 t = 0;
    for (int x = 0; x < 8; x++) t += ((unsigned __int128)hi_s[x] << 64) | lo_s[x];
    s[n + 2 * blockIdx.x] = (unsigned long long)t;
    s[n + 2 * blockIdx.x + 1] = (unsigned long long)(t >> 64);
  }
}

__global__ void na_final(int64_t n, unsigned long long* s) {
  unsigned long long* tail = s + kNoAllocWords - kNoAllocTail;
  unsigned __int128 sq = 0;
  for (int b = 0; b < kNoAllocCtas; b++) sq += ((unsigned __int128)s[n + 2 * b + 1] << 64) | s[n + 2 * b];
  const __int128 N = (__int128)(long long)tail[0] * (__int128)(long long)tail[1] - (__int128)sq;
  tail[2] = (unsigned long long)N;
  tail[3] = (unsigned long long)((unsigned __int128)N >> 64);
}

// Device address of the scratch array on the current device.  Looked up on
// every call (the lookup allocates nothing and is cheap): a cached address
// would be shared by host threads without synchronisation and would outlive
// a device reset.  The first lookup on a device loads the module there.
int scratch_for_current_device(unsigned long long** out) {
  void* p = nullptr;
  DCD_TRY_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
  *out = static_cast<unsigned long long*>(p);
  return DCD_OK;
}

}  // namespace
}  // namespace dcd

static_assert(dcd::kNoAllocMaxN == DCD_NOALLOC_MAX_N, "header limit and scratch layout disagree");

extern "C" int dcd_modularity_noalloc(int64_t n, const int64_t* d_row_ptr, const int32_t* d_col,
                                      const int32_t* d_w, const int32_t* d_labels, void* cuda_stream,
                                      double* q_out, int64_t* m2_out) {
  using namespace dcd;
  if (n <= 0 || n > kNoAllocMaxN || !d_row_ptr || !d_col || !d_w || !d_labels || !q_out) return DCD_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  unsigned long long* sc = nullptr;
  DCD_TRY(scratch_for_current_device(&sc));
  const int T = 256;
  count_launch(), na_clear<<<grid_for(n, T), T, 0, s>>>(sc, n);
  count_launch(), na_rows<<<grid_for(n * 32, T), T, 0, s>>>(n, d_row_ptr, d_col, d_w, d_labels, sc);
  count_launch(), na_sumsq<<<kNoAllocCtas, T, 0, s>>>(n, sc);
  count_launch(), na_final<<<1, 1, 0, s>>>(n, sc);
  DCD_LAUNCH_CHECK();
  unsigned long long tail[kNoAllocTail];
  DCD_TRY_CUDA(cudaMemcpyAsync(tail, sc + kNoAllocWords - kNoAllocTail, sizeof(tail), cudaMemcpyDeviceToHost, s));
  DCD_TRY_CUDA(cudaStreamSynchronize(s));
  if (tail[4]) return DCD_EINVAL;
  const int64_t m2 = (int64_t)tail[0];
  const __int128 N = (__int128)(((unsigned __int128)tail[3] << 64) | tail[2]);
  *q_out = m2 == 0 ? 0.0 : (double)N / ((double)m2 * (double)m2);
  if (m2_out) *m2_out = m2;
  return DCD_OK;
}
