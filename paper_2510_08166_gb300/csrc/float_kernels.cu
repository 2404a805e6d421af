// Per-MCU kernels of the differentiable float chain (not in the paper; it extends the
// decode of Sec. 4.3 to a float, unclamped, unrounded map that gradients can flow through):
//   F = bilinear(RGB(upsample(IDCT_f(c) + 128)))
// with IDCT_f the orthonormal 8x8 DCT-III, f = A c A^T, A[x][u] = C(u)/2 cos((2x+1)u pi/16),
// C(0) = 1/sqrt(2); chroma replicated 2x2 within the 16x16 MCU; the JFIF colour matrix.
// The map from c to F is affine, so the backward pass needs no stored activations:
//   texel gradients (scattered by the screen pass) -> colour^T -> upsample^T (2x2 sums)
//   -> A^T g A per data unit.
//
// k_float_tiles    one warp per needed MCU: 384 coefficients -> 16x16 float4 texels.
// k_float_zero     clears the texel-gradient tiles of the needed MCUs.
// k_float_adjoint  one pass over EVERY coefficient MCU, writing each MCU's 384 gradients
//                  once: A^T g A of its texel gradients when it is needed, zeros otherwise.
//                  A warp owns a run of kAdjChunk consecutive MCUs and merges it with the
//                  ascending work list (one binary search per run), so the 4 x larger
//                  zero fill streams at write bandwidth with no second pass.
// Both transforms are two passes of 8-term dot products in shared memory; lane l always
// produces column l % 8 (pass 1) and rows l / 8 and l / 8 + 4 (pass 2), so it keeps the
// basis entries it needs in registers.
#include <cuda_runtime.h>

#include "jt_internal.cuh"

namespace jt {
namespace {

constexpr float kCr2R = 1.402f, kCb2G = 0.344136f, kCr2G = 0.714136f, kCb2B = 1.772f;
constexpr uint32_t kAdjChunk = 32;

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

__global__ void k_float_zero(const __grid_constant__ FloatArgs a) {
  const uint32_t n = min(frame_count(a.state), a.tile_cap) * 256u;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a.tiles[i] = z;
}

__global__ void __launch_bounds__(kFloatWarps * 32) k_float_adjoint(const __grid_constant__ FloatArgs a) {
  __shared__ __align__(16) float buf[kFloatWarps][2][384];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* g = buf[warp][0];
  float* s1 = buf[warp][1];
  const int u = lane & 7, v0 = lane >> 3;
  float Au[8], Av0[8], Av1[8];  // column u of A; columns v0, v0 + 4 of A
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    Au[k] = a.basis[k * 8 + u];
    Av0[k] = a.basis[k * 8 + v0];
    Av1[k] = a.basis[k * 8 + v0 + 4];
  }
  const uint32_t count = frame_count(a.state);
  const uint32_t nchunks = (a.coef_mcus + kAdjChunk - 1) / kAdjChunk;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  bool over = false;
  for (uint32_t ch = blockIdx.x * kFloatWarps + warp; ch < nchunks; ch += gridDim.x * kFloatWarps) {
    const uint32_t m0 = ch * kAdjChunk, m1 = min(m0 + kAdjChunk, a.coef_mcus);
    // first work position whose gid is >= the run's first gid (the list ascends)
    uint32_t lo = 0, hi = count;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (__ldg(a.work + mid) < a.coef_gid_base + m0)
        lo = mid + 1;
      else
        hi = mid;
    }
    uint32_t p = lo;
    uint32_t next = p < count ? __ldg(a.work + p) : 0xFFFFFFFFu;
    for (uint32_t m = m0; m < m1; ++m) {
      float4* dst = reinterpret_cast<float4*>(a.grad_coef + (size_t)m * 384);
      const bool needed = next == a.coef_gid_base + m;
      if (!needed || p >= a.tile_cap) {
#pragma unroll
        for (int i = 0; i < 3; ++i) dst[lane + 32 * i] = z;
        if (needed) {
          over = true;
          ++p;
          next = p < count ? __ldg(a.work + p) : 0xFFFFFFFFu;
        }
        continue;
      }
      // colour^T and upsample^T: lane owns chroma samples s = lane and lane + 32 and the
      // four texels each covers
      const float4* acc = a.tiles + (size_t)p * 256;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int sidx = lane + 32 * h, sy = sidx >> 3, sx = sidx & 7;
        float gcb = 0.f, gcr = 0.f;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
          for (int dx = 0; dx < 2; ++dx) {
            const int ty = 2 * sy + dy, tx = 2 * sx + dx;
            const float4 gt = acc[ty * 16 + tx];
            g[((ty >> 3) * 2 + (tx >> 3)) * 64 + (ty & 7) * 8 + (tx & 7)] = gt.x + gt.y + gt.z;
            gcb += kCb2B * gt.z - kCb2G * gt.y;
            gcr += kCr2R * gt.x - kCr2G * gt.y;
          }
        g[256 + sidx] = gcb;
        g[320 + sidx] = gcr;
      }
      __syncwarp();
      // pass 1: s1[d][y][u] = sum_x g[d][y][x] A[x][u]
#pragma unroll
      for (int i = 0; i < 12; ++i) {
        const int o = lane + 32 * i;
        const float* row = g + (o & ~7);
        float s = 0.f;
#pragma unroll
        for (int xx = 0; xx < 8; ++xx) s = fmaf(Au[xx], row[xx], s);
        s1[o] = s;
      }
      __syncwarp();
      // pass 2: grad[d][v][u] = sum_y A[y][v] s1[d][y][u]  (v = v0 for even i, v0 + 4 for odd i)
      float* out = a.grad_coef + (size_t)m * 384;
#pragma unroll
      for (int i = 0; i < 12; ++i) {
        const int o = lane + 32 * i;
        const float* col = s1 + (o & ~63) + u;
        float s = 0.f;
#pragma unroll
        for (int y = 0; y < 8; ++y) s = fmaf((i & 1) ? Av1[y] : Av0[y], col[y * 8], s);
        out[o] = s;
      }
      __syncwarp();
      ++p;
      next = p < count ? __ldg(a.work + p) : 0xFFFFFFFFu;
    }
  }
  if (over) atomicOr(&a.state->err, JT_DEVERR_CAPACITY);
}

}  // namespace

void launch_float_tiles(const FloatArgs& a, int grid, cudaStream_t s) {
  k_float_tiles<<<grid, kFloatWarps * 32, 0, s>>>(a);
}
void launch_float_zero_tiles(const FloatArgs& a, int grid, cudaStream_t s) { k_float_zero<<<grid, 256, 0, s>>>(a); }
void launch_float_adjoint(const FloatArgs& a, int grid, cudaStream_t s) {
  k_float_adjoint<<<grid, kFloatWarps * 32, 0, s>>>(a);
}

}  // namespace jt
