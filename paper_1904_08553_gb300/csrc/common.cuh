// common.cuh -- shared device helpers of the dcd library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "dcd.h"

typedef __int128 i128;

namespace dcd {

constexpr int kWarp = 32;

// Process-wide count of kernel launches (dcd_kernel_launches); every launch
// site of the library is written `count_launch(), kernel<<<...>>>(...)`.
extern std::atomic<int64_t> g_launches;
inline void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Host-side phase trace: with the environment variable DCD_TRACE set, prints
// the host time since the previous trace point (a debugging aid; off by default).
void trace(const char* what);
bool trace_on();
void tracef(const char* fmt, ...);

// Records the failing CUDA call for dcd_last_cuda_error().
void note_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// Host-side fault injection (dcd_set_fault, environment variable DCD_FAULT),
// for tests of the error paths: an armed kind counts its events -- device
// allocations, checked CUDA calls -- and the N-th one reports failure instead
// of being made.  Disarmed, the cost is one relaxed load per event.
enum FaultKind : int { kFaultAlloc = 0, kFaultCuda = 1, kFaultKinds = 2 };
extern std::atomic<int64_t> g_fault_left[kFaultKinds];
bool fault_fire(int kind);
inline bool fault_hit(int kind) {
  return g_fault_left[kind].load(std::memory_order_relaxed) > 0 && fault_fire(kind);
}

#define DCD_TRY_CUDA(expr)                                                                          \
  do {                                                                                              \
    const bool f_ = ::dcd::fault_hit(::dcd::kFaultCuda);                                            \
    cudaError_t e_ = f_ ? cudaErrorUnknown : (expr);                                                \
    if (e_ != cudaSuccess) {                                                                        \
      ::dcd::note_cuda_error(e_, f_ ? "injected fault instead of: " #expr : #expr, __FILE__, __LINE__); \
      return DCD_ECUDA;                                                                             \
    }                                                                                               \
  } while (0)

#define DCD_TRY(expr)        \
  do {                       \
    int rc_ = (expr);        \
    if (rc_ != DCD_OK) {     \
      return rc_;            \
    }                        \
  } while (0)

#define DCD_LAUNCH_CHECK() DCD_TRY_CUDA(cudaGetLastError())

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Grid size for grid-stride kernels: enough CTAs to fill every SM several
// times over, never more than the work needs.
int grid_for(int64_t items, int threads, int per_sm = 8);
int num_sms();

// Blocks of a kernel resident on one SM at `threads` threads and `smem`
// bytes of dynamic shared memory (the occupancy query, cached per thread and
// device).  At least 1.
int resident_blocks(const void* kernel, int threads, size_t smem);

// Grid of a grid-stride kernel whose CTAs all do the same share of the work:
// exactly one wave (resident blocks x SMs), never more CTAs than the items
// need.  A grid above one wave that is not a whole number of waves leaves a
// partial last wave at low occupancy, which a grid-stride loop cannot
// rebalance.
template <typename K>
inline int wave_grid(K* kernel, int64_t items, int threads, size_t smem = 0) {
  const int64_t need = cdiv(items > 0 ? items : 1, threads);
  const int64_t wave = (int64_t)resident_blocks(reinterpret_cast<const void*>(kernel), threads, smem) * num_sms();
  return (int)(need < wave ? need : wave);
}

// Device-side error word bits (ctx->d_err).
enum : uint32_t {
  kErrBadRecord = 1u,   // invalid batch record
  kErrOverflow = 2u,    // weight above INT32_MAX or 2m too large
  kErrTableFull = 4u,   // aggregation table overflow (cannot happen when sized by degree)
};

// ---- device memory of a context ----
// Persistent buffers (the graph, labels, staging) come from the context's own
// stream-ordered pool.  Scratch of one update comes from a step arena: one
// block sized from the previous step's use (plus a margin), handed out by a
// bump pointer and released as a whole when the update ends, so a step makes
// no allocator calls once the arena has grown to the workload.
struct DevMem {
  cudaStream_t stream = nullptr;
  cudaMemPool_t pool = nullptr;
  char* arena = nullptr;
  size_t arena_size = 0, arena_off = 0, overflow = 0, last_use = 0;
  bool in_step = false;
  int alloc(void** p, size_t bytes);             // arena inside a step, else pool
  int alloc_persistent(void** p, size_t bytes);  // pool
  void release(void* p);                         // no-op for arena memory
  int begin_step(size_t hint);
  void end_step();
  int reserve(size_t bytes);  // an arena of at least bytes, outside a step
};

template <typename T>
struct Buf {
  T* p = nullptr;
  size_t n = 0;
  DevMem* mem = nullptr;
  Buf() = default;
  Buf(const Buf&) = delete;
  Buf& operator=(const Buf&) = delete;
  ~Buf() { reset(); }
  int alloc(DevMem* m, size_t count) {
    reset();
    mem = m;
    n = count;
    void* q = nullptr;
    int rc = m->alloc(&q, (count ? count : 1) * sizeof(T));
    p = static_cast<T*>(q);
    return rc;
  }
  void reset() {
    if (p && mem) mem->release(p);
    p = nullptr;
    n = 0;
  }
  // Persistent buffer: keep the allocation when it is already large enough.
  int ensure(DevMem* m, size_t count) {
    if (p && n >= count) return DCD_OK;
    reset();
    mem = m;
    n = count + count / 4 + 64;
    void* q = nullptr;
    int rc = m->alloc_persistent(&q, n * sizeof(T));
    p = static_cast<T*>(q);
    return rc;
  }
  T* get() const { return p; }
};

// ---- small device helpers ----
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Loads of data that a pass reads once (CSR columns and weights, bin lists):
// the streaming cache operator, which allocates the lines evict-first in L1
// and L2, so that streaming G_t (far larger than L2) does not push out the
// arrays the same kernels gather from at random (labels, community sums,
// degrees, row bounds).
__device__ __forceinline__ int32_t ld_stream(const int32_t* p) {
  int32_t v;
  asm("ld.global.cs.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ int64_t ld_stream(const int64_t* p) {
  int64_t v;
  asm("ld.global.cs.s64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}

// Stores of data that the kernel writes once and a later pass reads once
// (the next CSR): the streaming cache operator, evict-first as above.
__device__ __forceinline__ void st_stream(int32_t* p, int32_t v) {
  asm volatile("st.global.cs.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Multiplicative hash of a label into a power-of-two table.
__device__ __forceinline__ uint32_t hash_label(int32_t x, uint32_t mask) {
  return ((uint32_t)x * 0x9E3779B1u) >> 7 & mask;
}

}  // namespace dcd
