// Per-MCU kernels of the differentiable float chain (not in the paper; it extends the
// decode of Sec. 4.3 to a float, unclamped, unrounded map that gradients can flow through):
//   F = bilinear(RGB(upsample(IDCT_f(c) + 128)))
// with IDCT_f the orthonormal 8x8 DCT-III, f = A c A^T, A[x][u] = C(u)/2 cos((2x+1)u pi/16),
// C(0) = 1/sqrt(2); chroma replicated 2x2 within the 16x16 MCU; the JFIF colour matrix.
// The map from c to F is affine, so the backward pass needs no stored activations:
//   texel gradients (scattered by the screen pass) -> colour^T -> upsample^T (2x2 sums)
//   -> A^T g A per data unit.
//
// k_float_tiles    one warp per needed MCU: 384 coefficients -> 16x16 float4 texels (the
//                  forward pass; the backward pass is in pixel_kernels.cu and needs no tiles).
// The transform is two passes of 8-term dot products in shared memory; lane l always
// produces column l % 8 (pass 1) and rows l / 8 and l / 8 + 4 (pass 2), so it keeps the
// basis entries it needs in registers.
#include <cuda_runtime.h>

#include "jt_internal.cuh"

namespace jt {
namespace {


__device__ __forceinline__ uint32_t frame_count(const FrameState* st) {
  return *reinterpret_cast<const volatile uint32_t*>(&st->count);
}

__global__ void __launch_bounds__(kFloatWarps * 32) k_float_tiles(const __grid_constant__ FloatArgs a) {
  __shared__ __align__(16) float buf[kFloatWarps][2][384];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* c = buf[warp][0];
  float* t = buf[warp][1];
  const int x = lane & 7, y0 = lane >> 3;
  float Ax[8], Ay0[8], Ay1[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    Ax[k] = a.basis[x * 8 + k];
    Ay0[k] = a.basis[y0 * 8 + k];
    Ay1[k] = a.basis[(y0 + 4) * 8 + k];
  }
  const uint32_t count = frame_count(a.state);
  bool over = false;
  for (uint32_t j = blockIdx.x * kFloatWarps + warp; j < count; j += gridDim.x * kFloatWarps) {
    const uint32_t m = a.work[j] - a.coef_gid_base;
    if (m >= a.coef_mcus) continue;  // not a coefficient MCU
    if (j >= a.tile_cap) {
      over = true;
      continue;
    }
    const float4* src = reinterpret_cast<const float4*>(a.coef + (size_t)m * 384);
#pragma unroll
    for (int i = 0; i < 3; ++i) reinterpret_cast<float4*>(c)[lane + 32 * i] = __ldg(src + lane + 32 * i);
    __syncwarp();
    // pass 1: t[d][v][x] = sum_u A[x][u] c[d][v][u]
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      const int o = lane + 32 * i;
      const float* row = c + (o & ~7);
      float s = 0.f;
#pragma unroll
      for (int u = 0; u < 8; ++u) s = fmaf(Ax[u], row[u], s);
      t[o] = s;
    }
    __syncwarp();
    // pass 2: f[d][y][x] = sum_v A[y][v] t[d][v][x]  (y = y0 for even i, y0 + 4 for odd i)
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      const int o = lane + 32 * i;
      const float* col = t + (o & ~63) + x;
      float s = 0.f;
#pragma unroll
      for (int v = 0; v < 8; ++v) s = fmaf((i & 1) ? Ay1[v] : Ay0[v], col[v * 8], s);
      c[o] = s;
    }
    __syncwarp();
    // upsample + colour: texel q = (ty, tx) of the 16 x 16 MCU
    float4* dst = a.tiles + (size_t)j * 256;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int q = lane + 32 * i, ty = q >> 4, tx = q & 15;
      const float Y = c[((ty >> 3) * 2 + (tx >> 3)) * 64 + (ty & 7) * 8 + (tx & 7)] + 128.f;
      const int ci = (ty >> 1) * 8 + (tx >> 1);
      const float cb = c[256 + ci], cr = c[320 + ci];
      dst[q] = make_float4(Y + kCr2R * cr, Y - kCb2G * cb - kCr2G * cr, Y + kCb2B * cb, 0.f);
    }
    __syncwarp();
  }
  if (over) atomicOr(&a.state->err, JT_DEVERR_CAPACITY);
}

}  // namespace

void launch_float_tiles(const FloatArgs& a, int grid, cudaStream_t s) {
  k_float_tiles<<<grid, kFloatWarps * 32, 0, s>>>(a);
}

}  // namespace jt
