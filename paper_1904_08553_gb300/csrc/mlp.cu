// mlp.cu -- the learned screen's network on tensor cores: 12 -> 64 -> 64 -> 1,
// ReLU hidden units, sigmoid output, mean binary cross-entropy.
//
// Every product runs as mma.sync m16n8k16 with BF16 operands and FP32
// accumulators.  A warp owns 16 rows: layer-1 and layer-2 accumulator tiles
// are turned into the next product's A fragments in registers (bias, ReLU,
// BF16 pack).  Training adds the backward pass in the same kernel: the
// activation gradients stay in registers, the weight gradients of a CTA's 64
// rows are formed with mma from shared-memory tiles, and per-CTA partial
// gradients are reduced in a fixed order (deterministic), then Adam updates
// the FP32 master weights and refreshes the BF16 copies.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

namespace dcd {
namespace {

constexpr int NF = 12, NH = 64, NP = 5057;
constexpr int OFF_W1 = 0, OFF_B1 = 768, OFF_W2 = 832, OFF_B2 = 4928, OFF_W3 = 4992, OFF_B3 = 5056;
constexpr int kRowsPerCta = 64;  // 4 warps x 16 rows

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float lo_f(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float hi_f(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }
__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ uint32_t two(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// BF16 operand copies: w1t[64][16] (output-major, inputs 12..15 zero),
// w2[64][64] (input-major), w2t[64][64] (output-major), w3[64].
struct Weights {
  const __nv_bfloat16* w1t;
  const __nv_bfloat16* w2;
  const __nv_bfloat16* w2t;
  const __nv_bfloat16* w3;
  const float* P;  // FP32 master (biases are read from here)
};

__global__ void prepare(const float* __restrict__ P, __nv_bfloat16* __restrict__ w1t, __nv_bfloat16* __restrict__ w2,
                        __nv_bfloat16* __restrict__ w2t, __nv_bfloat16* __restrict__ w3) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 64 * 64; i += gridDim.x * blockDim.x) {
    const int a = i / 64, b = i % 64;  // W2[a][b]
    const __nv_bfloat16 v = __float2bfloat16_rn(P[OFF_W2 + i]);
    w2[i] = v;
    w2t[b * 64 + a] = v;
    if (i < 64 * 16) {
      const int o = i / 16, k = i % 16;  // w1t[o][k] = W1[k][o]
      w1t[i] = __float2bfloat16_rn(k < NF ? P[OFF_W1 + k * NH + o] : 0.f);
    }
    if (i < 64) w3[i] = __float2bfloat16_rn(P[OFF_W3 + i]);
  }
}

struct Smem {
  __nv_bfloat16 w1t[64 * 16];
  __nv_bfloat16 w2[64 * 64];
  __nv_bfloat16 w2t[64 * 64];
  float w3f[64];
  __nv_bfloat16 w3[64];
  float b1[64], b2[64];
};

__device__ __forceinline__ void load_weights(Smem& s, const Weights& W) {
  for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
    s.w2[i] = W.w2[i];
    s.w2t[i] = W.w2t[i];
    if (i < 64 * 16) s.w1t[i] = W.w1t[i];
    if (i < 64) {
      s.w3[i] = W.w3[i];
      s.w3f[i] = __bfloat162float(W.w3[i]);
      s.b1[i] = W.P[OFF_B1 + i];
      s.b2[i] = W.P[OFF_B2 + i];
    }
  }
  __syncthreads();
}

// Forward of one 16-row tile.  Outputs: the X fragment, the layer-1
// activations as layer-2 A fragments, h2 (BF16-rounded, C layout) and z.
struct Fwd {
  uint32_t xa[4];
  uint32_t h1a[4][4];
  float h2[8][4];
  float z0, z1;  // logits of rows g and g + 8
};

__device__ __forceinline__ void forward_tile(const Smem& s, const float* __restrict__ X, int64_t r0, int64_t n,
                                             float b3, Fwd& f) {
  const int lane = lane_id(), g = lane >> 2, t = lane & 3;
  const int64_t ra = r0 + g, rb = r0 + g + 8;
  auto xv = [&](int64_t r, int c) -> float { return (r < n && c < NF) ? X[r * NF + c] : 0.f; };
  f.xa[0] = pack_bf16(xv(ra, 2 * t), xv(ra, 2 * t + 1));
  f.xa[1] = pack_bf16(xv(rb, 2 * t), xv(rb, 2 * t + 1));
  f.xa[2] = pack_bf16(xv(ra, 2 * t + 8), xv(ra, 2 * t + 9));
  f.xa[3] = pack_bf16(xv(rb, 2 * t + 8), xv(rb, 2 * t + 9));
  float c1[8][4];
#pragma unroll
  for (int j = 0; j < 8; j++) {
    c1[j][0] = c1[j][1] = c1[j][2] = c1[j][3] = 0.f;
    const __nv_bfloat16* col = s.w1t + (8 * j + g) * 16;
    mma16816(c1[j], f.xa, ld_pair(col + 2 * t), ld_pair(col + 2 * t + 8));
  }
#pragma unroll
  for (int kk = 0; kk < 4; kk++) {
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int j = 2 * kk + h, c = 8 * j + 2 * t;
      const float v00 = fmaxf(c1[j][0] + s.b1[c], 0.f), v01 = fmaxf(c1[j][1] + s.b1[c + 1], 0.f);
      const float v10 = fmaxf(c1[j][2] + s.b1[c], 0.f), v11 = fmaxf(c1[j][3] + s.b1[c + 1], 0.f);
      f.h1a[kk][2 * h] = pack_bf16(v00, v01);
      f.h1a[kk][2 * h + 1] = pack_bf16(v10, v11);
    }
  }
  float c2[8][4];
#pragma unroll
  for (int j = 0; j < 8; j++) c2[j][0] = c2[j][1] = c2[j][2] = c2[j][3] = 0.f;
#pragma unroll
  for (int kk = 0; kk < 4; kk++)
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const __nv_bfloat16* col = s.w2t + (8 * j + g) * 64 + 16 * kk;
      mma16816(c2[j], f.h1a[kk], ld_pair(col + 2 * t), ld_pair(col + 2 * t + 8));
    }
  float za = 0.f, zb = 0.f;
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const int c = 8 * j + 2 * t;
    f.h2[j][0] = bf16r(fmaxf(c2[j][0] + s.b2[c], 0.f));
    f.h2[j][1] = bf16r(fmaxf(c2[j][1] + s.b2[c + 1], 0.f));
    f.h2[j][2] = bf16r(fmaxf(c2[j][2] + s.b2[c], 0.f));
    f.h2[j][3] = bf16r(fmaxf(c2[j][3] + s.b2[c + 1], 0.f));
    za += f.h2[j][0] * s.w3f[c] + f.h2[j][1] * s.w3f[c + 1];
    zb += f.h2[j][2] * s.w3f[c] + f.h2[j][3] * s.w3f[c + 1];
  }
  za += __shfl_xor_sync(0xffffffffu, za, 1);
  za += __shfl_xor_sync(0xffffffffu, za, 2);
  zb += __shfl_xor_sync(0xffffffffu, zb, 1);
  zb += __shfl_xor_sync(0xffffffffu, zb, 2);
  f.z0 = za + b3;
  f.z1 = zb + b3;
}

__device__ __forceinline__ float sigmoidf_(float z) { return 1.f / (1.f + __expf(-z)); }

__global__ void __launch_bounds__(128) mlp_infer(Weights W, const float* __restrict__ X, int64_t n,
                                                 float* __restrict__ p) {
  __shared__ Smem s;
  load_weights(s, W);
  const float b3 = W.P[OFF_B3];
  const int lane = lane_id(), g = lane >> 2, t = lane & 3;
  const int64_t tiles = cdiv(n, 16);
  for (int64_t tile = blockIdx.x * 4 + (threadIdx.x >> 5); tile < tiles; tile += (int64_t)gridDim.x * 4) {
    Fwd f;
    forward_tile(s, X, tile * 16, n, b3, f);
    if (t == 0) {
      const int64_t ra = tile * 16 + g, rb = ra + 8;
      if (ra < n) p[ra] = sigmoidf_(f.z0);
      if (rb < n) p[rb] = sigmoidf_(f.z1);
    }
  }
}

// Per-CTA gradient partials: grid = rows / 64; part[cta][NP] and lpart[cta].
__global__ void __launch_bounds__(128) mlp_grad_cta(Weights W, const float* __restrict__ X,
                                                    const float* __restrict__ Y, int64_t n, float inv_n,
                                                    float* __restrict__ part, double* __restrict__ lpart) {
  __shared__ Smem s;
  __shared__ __nv_bfloat16 h1s[kRowsPerCta * 64], dh2s[kRowsPerCta * 64], dh1s[kRowsPerCta * 64];
  __shared__ __nv_bfloat16 xs[kRowsPerCta * 16];
  __shared__ float wpart[4][66];  // per warp: dW3[64], db3, loss
  load_weights(s, W);
  const float b3 = W.P[OFF_B3];
  const int lane = lane_id(), g = lane >> 2, t = lane & 3, wid = threadIdx.x >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * kRowsPerCta + wid * 16;
  Fwd f;
  forward_tile(s, X, r0, n, b3, f);
  const int64_t ra = r0 + g, rb = r0 + g + 8;
  const float ya = ra < n ? Y[ra] : 0.f, yb = rb < n ? Y[rb] : 0.f;
  const float pa = sigmoidf_(f.z0), pb = sigmoidf_(f.z1);
  const float dza = ra < n ? (pa - ya) * inv_n : 0.f, dzb = rb < n ? (pb - yb) * inv_n : 0.f;
  float la = 0.f, lb = 0.f;
  if (t == 0) {
    if (ra < n) la = fmaxf(f.z0, 0.f) - f.z0 * ya + log1pf(__expf(-fabsf(f.z0)));
    if (rb < n) lb = fmaxf(f.z1, 0.f) - f.z1 * yb + log1pf(__expf(-fabsf(f.z1)));
  }
  // layer 3: dW3 partial (rows of the warp) and dh2 = (h2 > 0) * dz * w3
  float dw3[8][2];
  uint32_t dh2a[4][4];
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const int c = 8 * j + 2 * t;
    dw3[j][0] = f.h2[j][0] * dza + f.h2[j][2] * dzb;
    dw3[j][1] = f.h2[j][1] * dza + f.h2[j][3] * dzb;
    const float d00 = f.h2[j][0] > 0.f ? dza * s.w3f[c] : 0.f, d01 = f.h2[j][1] > 0.f ? dza * s.w3f[c + 1] : 0.f;
    const float d10 = f.h2[j][2] > 0.f ? dzb * s.w3f[c] : 0.f, d11 = f.h2[j][3] > 0.f ? dzb * s.w3f[c + 1] : 0.f;
    const int kk = j >> 1, h = j & 1;
    dh2a[kk][2 * h] = pack_bf16(d00, d01);
    dh2a[kk][2 * h + 1] = pack_bf16(d10, d11);
  }
  // dh1 = dh2 W2^T, masked by h1 > 0
  float c3[8][4];
#pragma unroll
  for (int j = 0; j < 8; j++) c3[j][0] = c3[j][1] = c3[j][2] = c3[j][3] = 0.f;
#pragma unroll
  for (int kk = 0; kk < 4; kk++)
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const __nv_bfloat16* row = s.w2 + (8 * j + g) * 64 + 16 * kk;  // B[k][n] = W2[n][k]
      mma16816(c3[j], dh2a[kk], ld_pair(row + 2 * t), ld_pair(row + 2 * t + 8));
    }
  // stage x, h1, dh2, dh1 of the warp's 16 rows in shared memory (row-major)
  const int la_ = wid * 16 + g, lb_ = la_ + 8;
  {
    const uint32_t* xa = f.xa;
    *reinterpret_cast<uint32_t*>(&xs[la_ * 16 + 2 * t]) = xa[0];
    *reinterpret_cast<uint32_t*>(&xs[lb_ * 16 + 2 * t]) = xa[1];
    *reinterpret_cast<uint32_t*>(&xs[la_ * 16 + 2 * t + 8]) = xa[2];
    *reinterpret_cast<uint32_t*>(&xs[lb_ * 16 + 2 * t + 8]) = xa[3];
  }
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const int c = 8 * j + 2 * t, kk = j >> 1, h = j & 1;
    const uint32_t h1_a = f.h1a[kk][2 * h], h1_b = f.h1a[kk][2 * h + 1];
    *reinterpret_cast<uint32_t*>(&h1s[la_ * 64 + c]) = h1_a;
    *reinterpret_cast<uint32_t*>(&h1s[lb_ * 64 + c]) = h1_b;
    *reinterpret_cast<uint32_t*>(&dh2s[la_ * 64 + c]) = dh2a[kk][2 * h];
    *reinterpret_cast<uint32_t*>(&dh2s[lb_ * 64 + c]) = dh2a[kk][2 * h + 1];
    const float e00 = lo_f(h1_a) > 0.f ? c3[j][0] : 0.f, e01 = hi_f(h1_a) > 0.f ? c3[j][1] : 0.f;
    const float e10 = lo_f(h1_b) > 0.f ? c3[j][2] : 0.f, e11 = hi_f(h1_b) > 0.f ? c3[j][3] : 0.f;
    *reinterpret_cast<uint32_t*>(&dh1s[la_ * 64 + c]) = pack_bf16(e00, e01);
    *reinterpret_cast<uint32_t*>(&dh1s[lb_ * 64 + c]) = pack_bf16(e10, e11);
  }
  // warp partials of dW3 (sum over the 8 row groups), db3 and loss
#pragma unroll
  for (int j = 0; j < 8; j++)
#pragma unroll
    for (int e = 0; e < 2; e++) {
      float v = dw3[j][e];
      v += __shfl_xor_sync(0xffffffffu, v, 4);
      v += __shfl_xor_sync(0xffffffffu, v, 8);
      v += __shfl_xor_sync(0xffffffffu, v, 16);
      if (g == 0) wpart[wid][8 * j + 2 * t + e] = v;
    }
  {
    float db = (t == 0) ? dza + dzb : 0.f, ls = la + lb;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      db += __shfl_xor_sync(0xffffffffu, db, o);
      ls += __shfl_xor_sync(0xffffffffu, ls, o);
    }
    if (lane == 0) {
      wpart[wid][64] = db;
      wpart[wid][65] = ls;
    }
  }
  __syncthreads();
  float* out = part + (int64_t)blockIdx.x * NP;
  // dW2[i][j] = sum_r h1[r][i] dh2[r][j]: warp wid owns i in [16 wid, 16 wid + 16)
  {
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; j++) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    const int i0 = 16 * wid + g;
#pragma unroll
    for (int kk = 0; kk < 4; kk++) {
      const int r = 16 * kk + 2 * t;
      uint32_t a[4];
      a[0] = two(h1s[r * 64 + i0], h1s[(r + 1) * 64 + i0]);
      a[1] = two(h1s[r * 64 + i0 + 8], h1s[(r + 1) * 64 + i0 + 8]);
      a[2] = two(h1s[(r + 8) * 64 + i0], h1s[(r + 9) * 64 + i0]);
      a[3] = two(h1s[(r + 8) * 64 + i0 + 8], h1s[(r + 9) * 64 + i0 + 8]);
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const int cj = 8 * j + g;
        mma16816(acc[j], a, two(dh2s[r * 64 + cj], dh2s[(r + 1) * 64 + cj]),
                 two(dh2s[(r + 8) * 64 + cj], dh2s[(r + 9) * 64 + cj]));
      }
    }
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int c = 8 * j + 2 * t;
      out[OFF_W2 + i0 * 64 + c] = acc[j][0];
      out[OFF_W2 + i0 * 64 + c + 1] = acc[j][1];
      out[OFF_W2 + (i0 + 8) * 64 + c] = acc[j][2];
      out[OFF_W2 + (i0 + 8) * 64 + c + 1] = acc[j][3];
    }
  }
  // dW1[i][j] = sum_r x[r][i] dh1[r][j]: warp wid owns output columns [16 wid, 16 wid + 16)
  {
    float acc[2][4];
#pragma unroll
    for (int j = 0; j < 2; j++) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 4; kk++) {
      const int r = 16 * kk + 2 * t;
      uint32_t a[4];
      a[0] = two(xs[r * 16 + g], xs[(r + 1) * 16 + g]);
      a[1] = two(xs[r * 16 + g + 8], xs[(r + 1) * 16 + g + 8]);
      a[2] = two(xs[(r + 8) * 16 + g], xs[(r + 9) * 16 + g]);
      a[3] = two(xs[(r + 8) * 16 + g + 8], xs[(r + 9) * 16 + g + 8]);
#pragma unroll
      for (int jj = 0; jj < 2; jj++) {
        const int cj = 16 * wid + 8 * jj + g;
        mma16816(acc[jj], a, two(dh1s[r * 64 + cj], dh1s[(r + 1) * 64 + cj]),
                 two(dh1s[(r + 8) * 64 + cj], dh1s[(r + 9) * 64 + cj]));
      }
    }
#pragma unroll
    for (int jj = 0; jj < 2; jj++) {
      const int c = 16 * wid + 8 * jj + 2 * t;
      if (g < NF) {
        out[OFF_W1 + g * NH + c] = acc[jj][0];
        out[OFF_W1 + g * NH + c + 1] = acc[jj][1];
      }
      if (g + 8 < NF) {
        out[OFF_W1 + (g + 8) * NH + c] = acc[jj][2];
        out[OFF_W1 + (g + 8) * NH + c + 1] = acc[jj][3];
      }
    }
  }
  // biases, W3, loss (fixed-order sums)
  if (threadIdx.x < 64) {
    const int j = threadIdx.x;
    float s1 = 0.f, s2 = 0.f;
    for (int r = 0; r < kRowsPerCta; r++) {
      s1 += __bfloat162float(dh1s[r * 64 + j]);
      s2 += __bfloat162float(dh2s[r * 64 + j]);
    }
    out[OFF_B1 + j] = s1;
    out[OFF_B2 + j] = s2;
    out[OFF_W3 + j] = wpart[0][j] + wpart[1][j] + wpart[2][j] + wpart[3][j];
  }
  if (threadIdx.x == 64) {
    out[OFF_B3] = wpart[0][64] + wpart[1][64] + wpart[2][64] + wpart[3][64];
    lpart[blockIdx.x] = (double)wpart[0][65] + wpart[1][65] + wpart[2][65] + wpart[3][65];
  }
}

// grad[k] = sum over CTAs (in CTA order) of part[cta][k]; loss likewise.
__global__ void grad_reduce(const float* __restrict__ part, int ncta, float* __restrict__ grad,
                            const double* __restrict__ lpart, double* __restrict__ loss, double inv_n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < NP; k += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int c = 0; c < ncta; c++) s += part[(int64_t)c * NP + k];
    grad[k] = s;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double l = 0;
    for (int c = 0; c < ncta; c++) l += lpart[c];
    *loss = l * inv_n;
  }
}

__global__ void adam(float* __restrict__ P, float* __restrict__ m, float* __restrict__ v,
                     const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < NP; k += gridDim.x * blockDim.x) {
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    P[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
  }
}

}  // namespace
}  // namespace dcd

struct dcd_mlp {
  cudaStream_t stream = nullptr;
  int device = 0;
  float* P = nullptr;  // master params
  float* m = nullptr;
  float* v = nullptr;
  float* grad = nullptr;
  double* loss = nullptr;
  __nv_bfloat16* w1t = nullptr;
  __nv_bfloat16* w2 = nullptr;
  __nv_bfloat16* w2t = nullptr;
  __nv_bfloat16* w3 = nullptr;
  float* part = nullptr;
  double* lpart = nullptr;
  int64_t part_ctas = 0;
  int64_t adam_t = 0;
};

namespace {
using namespace dcd;

Weights weights_of(const dcd_mlp* m) { return Weights{m->w1t, m->w2, m->w2t, m->w3, m->P}; }

int refresh(dcd_mlp* m) {
  count_launch(), prepare<<<16, 256, 0, m->stream>>>(m->P, m->w1t, m->w2, m->w2t, m->w3);
  DCD_LAUNCH_CHECK();
  return DCD_OK;
}

int ensure_parts(dcd_mlp* m, int64_t ctas) {
  if (ctas <= m->part_ctas) return DCD_OK;
  if (m->part) cudaFree(m->part);
  if (m->lpart) cudaFree(m->lpart);
  m->part = nullptr;
  m->lpart = nullptr;
  DCD_TRY_CUDA(cudaMalloc(&m->part, (size_t)ctas * NP * sizeof(float)));
  DCD_TRY_CUDA(cudaMalloc(&m->lpart, (size_t)ctas * sizeof(double)));
  m->part_ctas = ctas;
  return DCD_OK;
}

// Mean BCE gradient of rows [0, n) into m->grad and m->loss.
int grad_pass(dcd_mlp* m, const float* X, const float* Y, int64_t n) {
  const int64_t ctas = cdiv(n, kRowsPerCta);
  DCD_TRY(ensure_parts(m, ctas));
  count_launch(), mlp_grad_cta<<<(unsigned)ctas, 128, 0, m->stream>>>(weights_of(m), X, Y, n, 1.f / (float)n,
                                                                       m->part, m->lpart);
  count_launch(), grad_reduce<<<(NP + 255) / 256, 256, 0, m->stream>>>(m->part, (int)ctas, m->grad, m->lpart, m->loss,
                                                                        1.0 / (double)n);
  DCD_LAUNCH_CHECK();
  return DCD_OK;
}

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

}  // namespace

namespace dcd {
int mlp_forward_on(dcd_mlp* m, const float* X, int64_t n, float* p, cudaStream_t s) {
  if (n <= 0) return DCD_OK;
  const int64_t tiles = cdiv(n, 16);
  const int64_t ctas = cdiv(tiles, 4) < 8 * (int64_t)num_sms() ? cdiv(tiles, 4) : 8 * (int64_t)num_sms();
  count_launch(), mlp_infer<<<(unsigned)ctas, 128, 0, s>>>(weights_of(m), X, n, p);
  DCD_LAUNCH_CHECK();
  return DCD_OK;
}
}  // namespace dcd

extern "C" {

int dcd_mlp_create(uint64_t seed, void* cuda_stream, dcd_mlp** out) {
  if (!out) return DCD_EINVAL;
  *out = nullptr;
  dcd_mlp* m = new (std::nothrow) dcd_mlp();
  if (!m) return DCD_ENOMEM;
  m->stream = static_cast<cudaStream_t>(cuda_stream);
  int rc = DCD_OK;
  do {
    if (cudaGetDevice(&m->device) != cudaSuccess) { rc = DCD_ECUDA; break; }
    if (cudaMalloc(&m->P, NP * sizeof(float)) != cudaSuccess || cudaMalloc(&m->m, NP * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&m->v, NP * sizeof(float)) != cudaSuccess || cudaMalloc(&m->grad, NP * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&m->loss, sizeof(double)) != cudaSuccess ||
        cudaMalloc(&m->w1t, 64 * 16 * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc(&m->w2, 64 * 64 * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc(&m->w2t, 64 * 64 * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc(&m->w3, 64 * sizeof(__nv_bfloat16)) != cudaSuccess) {
      cudaGetLastError();
      rc = DCD_ENOMEM;
      break;
    }
    // He-uniform initialisation from SplitMix64; biases zero
    std::vector<float> P(NP, 0.f);
    uint64_t s = seed;
    auto unif = [&](float lim) { return (float)(((splitmix(s) >> 11) * (1.0 / 9007199254740992.0)) * 2 - 1) * lim; };
    for (int i = 0; i < NF * NH; i++) P[OFF_W1 + i] = unif(std::sqrt(6.f / NF));
    for (int i = 0; i < NH * NH; i++) P[OFF_W2 + i] = unif(std::sqrt(6.f / NH));
    for (int i = 0; i < NH; i++) P[OFF_W3 + i] = unif(std::sqrt(6.f / NH));
    rc = dcd_mlp_set_params(m, P.data());
  } while (0);
  if (rc) {
    dcd_mlp_destroy(m);
    return rc;
  }
  *out = m;
  return DCD_OK;
}

int dcd_mlp_destroy(dcd_mlp* m) {
  if (!m) return DCD_OK;
  cudaStreamSynchronize(m->stream);
  for (void* p : {(void*)m->P, (void*)m->m, (void*)m->v, (void*)m->grad, (void*)m->loss, (void*)m->w1t, (void*)m->w2,
                  (void*)m->w2t, (void*)m->w3, (void*)m->part, (void*)m->lpart})
    if (p) cudaFree(p);
  delete m;
  return DCD_OK;
}

int dcd_mlp_set_params(dcd_mlp* m, const float* params) {
  if (!m || !params) return DCD_EINVAL;
  DCD_TRY_CUDA(cudaMemcpyAsync(m->P, params, NP * sizeof(float), cudaMemcpyHostToDevice, m->stream));
  DCD_TRY_CUDA(cudaMemsetAsync(m->m, 0, NP * sizeof(float), m->stream));
  DCD_TRY_CUDA(cudaMemsetAsync(m->v, 0, NP * sizeof(float), m->stream));
  m->adam_t = 0;
  DCD_TRY(refresh(m));
  DCD_TRY_CUDA(cudaStreamSynchronize(m->stream));
  return DCD_OK;
}

int dcd_mlp_get_params(dcd_mlp* m, float* params_out) {
  if (!m || !params_out) return DCD_EINVAL;
  DCD_TRY_CUDA(cudaMemcpyAsync(params_out, m->P, NP * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
  DCD_TRY_CUDA(cudaStreamSynchronize(m->stream));
  return DCD_OK;
}

int dcd_mlp_forward(dcd_mlp* m, const float* d_X, int64_t n, float* d_p) {
  if (!m || n < 0 || (n && (!d_X || !d_p))) return DCD_EINVAL;
  if (n == 0) return DCD_OK;
  const int64_t tiles = cdiv(n, 16);
  const int64_t ctas = cdiv(tiles, 4) < 8 * (int64_t)num_sms() ? cdiv(tiles, 4) : 8 * (int64_t)num_sms();
  count_launch(), mlp_infer<<<(unsigned)ctas, 128, 0, m->stream>>>(weights_of(m), d_X, n, d_p);
  DCD_LAUNCH_CHECK();
  DCD_TRY_CUDA(cudaStreamSynchronize(m->stream));
  return DCD_OK;
}

int dcd_mlp_grad(dcd_mlp* m, const float* d_X, const float* d_y, int64_t n, float* grad_out, double* loss_out) {
  if (!m || n <= 0 || !d_X || !d_y) return DCD_EINVAL;
  DCD_TRY(grad_pass(m, d_X, d_y, n));
  if (grad_out)
    DCD_TRY_CUDA(cudaMemcpyAsync(grad_out, m->grad, NP * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
  if (loss_out) DCD_TRY_CUDA(cudaMemcpyAsync(loss_out, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  DCD_TRY_CUDA(cudaStreamSynchronize(m->stream));
  return DCD_OK;
}

int dcd_mlp_train(dcd_mlp* m, const float* d_X, const float* d_y, int64_t n, int64_t batch, int32_t epochs,
                  float lr, double* loss_out) {
  if (!m || n <= 0 || batch <= 0 || epochs <= 0 || !d_X || !d_y || !(lr > 0.f)) return DCD_EINVAL;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  double last = 0;
  for (int32_t ep = 0; ep < epochs; ep++) {
    for (int64_t r = 0; r < n; r += batch) {
      const int64_t nb = (r + batch <= n) ? batch : n - r;
      DCD_TRY(grad_pass(m, d_X + r * NF, d_y + r, nb));
      m->adam_t++;
      const float c1 = 1.f - std::pow(b1, (float)m->adam_t), c2 = 1.f - std::pow(b2, (float)m->adam_t);
      count_launch(), adam<<<(NP + 255) / 256, 256, 0, m->stream>>>(m->P, m->m, m->v, m->grad, lr, b1, b2, eps, c1, c2);
      DCD_LAUNCH_CHECK();
      DCD_TRY(refresh(m));
    }
  }
  DCD_TRY_CUDA(cudaMemcpyAsync(&last, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  DCD_TRY_CUDA(cudaStreamSynchronize(m->stream));
  if (loss_out) *loss_out = last;
  return DCD_OK;
}

}  // extern "C"
