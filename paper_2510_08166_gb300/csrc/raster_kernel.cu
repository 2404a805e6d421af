// Scene rasteriser: writes the G-buffer (uv, texture id, mip level) of a procedural scene, a
// perspective ground plane of 2 m texture cells under projective screen-space quads. It
// stands in for the renderer's geometry pass (paper Sec. 4) so that a whole frame, geometry
// included, runs on the GPU.
//
// Every arithmetic step is an explicitly rounded fp32 operation (no contraction) in a fixed
// order, and levels are chosen by exact power-of-two thresholds on the squared footprint, so
// the result is reproducible on any IEEE fp32 implementation of the same steps.
//
// One CTA per 32 x 8 pixel tile: the CTA first lists, in drawing order, the quads whose
// pixel bounds meet the tile (ordered compaction by warp ballots), then each thread takes
// one pixel: the last listed quad containing it, else the ground, else sky.
#include <cuda_runtime.h>

#include "jt_internal.cuh"

namespace jt {
namespace {

constexpr int kTileX = 32, kTileY = 8, kThreads = kTileX * kTileY;

__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }

// SplitMix64 (Steele, Lea, Flood 2014): the ground cells' texture and uv offset come from
// two steps of it keyed by the cell coordinates.
__device__ __forceinline__ uint64_t splitmix_next(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t cell_hash(uint64_t seed, uint64_t a, uint64_t b) {
  uint64_t s = seed ^ (a * 0xD1B54A32D192ED03ull) ^ (b * 0x8CB92BA72F3D8DD7ull);
  splitmix_next(s);
  return splitmix_next(s);
}

// Ground hit of the camera ray through pixel coordinate (px, py); uv = world (x, z) / 2.
__device__ __forceinline__ bool ground(const RasterArgs& a, float px, float py, float& u, float& v) {
  const float* R = a.rot;
  const float sx = fmul(fsub(fmul(px, a.ax), 1.0f), a.tan_x);
  const float sy = fmul(fsub(1.0f, fmul(py, a.ay)), a.tan_y);
  const float dx = fsub(fadd(fmul(R[0], sx), fmul(R[1], sy)), R[2]);
  const float dy = fsub(fadd(fmul(R[3], sx), fmul(R[4], sy)), R[5]);
  const float dz = fsub(fadd(fmul(R[6], sx), fmul(R[7], sy)), R[8]);
  if (!(dy < -1e-9f)) return false;
  const float t = fdiv(-a.cam[1], dy);
  if (t > a.max_t) return false;
  u = fmul(fadd(a.cam[0], fmul(t, dx)), 0.5f);
  v = fmul(fadd(a.cam[2], fmul(t, dz)), 0.5f);
  return true;
}

// floor(log2(sqrt(r2)) + 1/2) clamped to [0, L-1]: the count of k >= 1 with r2 >= 2^(2k-1).
__device__ __forceinline__ int level_of(float r2, int L) {
  if (!(r2 > 0.0f)) return 0;
  int m = 0;
#pragma unroll 1
  while (m + 1 <= L - 1 && r2 >= __int_as_float((127 + 2 * (m + 1) - 1) << 23)) ++m;
  return m;
}

__device__ __forceinline__ float footprint(float u0, float v0, float u1, float v1, int w, int h) {
  const float du = fmul(fsub(u1, u0), (float)w), dv = fmul(fsub(v1, v0), (float)h);
  return fadd(fmul(du, du), fmul(dv, dv));
}

__device__ __forceinline__ void quad_uv(const SceneQuad& q, float x, float y, float& u, float& v) {
  float s = fadd(fadd(fmul(q.h[0], x), fmul(q.h[1], y)), q.h[2]);
  float t = fadd(fadd(fmul(q.h[3], x), fmul(q.h[4], y)), q.h[5]);
  const float w = fadd(fadd(fmul(q.h[6], x), fmul(q.h[7], y)), q.h[8]);
  s = fdiv(s, w);
  t = fdiv(t, w);
  u = fadd(q.ou, fmul(q.rep, fsub(fmul(q.cs, s), fmul(q.sn, t))));
  v = fadd(q.ov, fmul(q.rep, fadd(fmul(q.sn, s), fmul(q.cs, t))));
}

__device__ __forceinline__ bool inside(const SceneQuad& q, float x, float y) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (fsub(fmul(q.ex[i], fsub(y, q.cy[i])), fmul(q.ey[i], fsub(x, q.cx[i]))) < 0.0f) return false;
  return true;
}

__global__ void __launch_bounds__(kThreads) k_raster(const __grid_constant__ RasterArgs a) {
  __shared__ uint16_t list[kMaxSceneQuads];
  __shared__ uint32_t warp_count[kThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tx0 = blockIdx.x * kTileX, ty0 = blockIdx.y * kTileY;
  const int tx1 = min(tx0 + kTileX, a.width) - 1, ty1 = min(ty0 + kTileY, a.height) - 1;

  // the quads that may cover the tile, in drawing order
  uint32_t count = 0;
#pragma unroll 1
  for (int base = 0; base < a.nquads; base += kThreads) {
    const int n = base + tid;
    bool meets = false;
    if (n < a.nquads) {
      const SceneQuad& q = a.quads[n];
      meets = q.x0 <= tx1 && q.x1 >= tx0 && q.y0 <= ty1 && q.y1 >= ty0;
    }
    const uint32_t b = __ballot_sync(0xFFFFFFFFu, meets);
    if (lane == 0) warp_count[warp] = __popc(b);
    __syncthreads();
    uint32_t before = count;
    for (int w = 0; w < warp; ++w) before += warp_count[w];
    if (meets) list[before + __popc(b & ((1u << lane) - 1u))] = (uint16_t)n;
    uint32_t total = 0;
    for (int w = 0; w < kThreads / 32; ++w) total += warp_count[w];
    count += total;
    __syncthreads();
  }

  const int x = tx0 + (tid & (kTileX - 1)), y = ty0 + tid / kTileX;
  if (x >= a.width || y >= a.height) return;
  const float fx = fadd((float)x, 0.5f), fy = fadd((float)y, 0.5f);
  const float qx = fsub(fmul(fx, a.kx), a.shift), qy = fmul(fy, a.ky);
  int hit = -1;
#pragma unroll 1
  for (int i = (int)count - 1; i >= 0; --i) {  // the last quad drawn wins
    const SceneQuad& q = a.quads[list[i]];
    if (x >= q.x0 && x <= q.x1 && y >= q.y0 && y <= q.y1 && inside(q, qx, qy)) {
      hit = list[i];
      break;
    }
  }
  float u = 0.f, v = 0.f;
  int t = JT_EMPTY_TEXTURE, lvl = 0;
  if (hit >= 0) {
    const SceneQuad& q = a.quads[hit];
    t = q.tex;
    quad_uv(q, qx, qy, u, v);
    if (a.use_mips) {
      const float hx = fmul(a.kx, 0.5f), hy = fmul(a.ky, 0.5f);
      float u0, v0, u1, v1, u2, v2, u3, v3;
      quad_uv(q, fsub(qx, hx), qy, u0, v0);
      quad_uv(q, fadd(qx, hx), qy, u1, v1);
      quad_uv(q, qx, fsub(qy, hy), u2, v2);
      quad_uv(q, qx, fadd(qy, hy), u3, v3);
      const float rx = footprint(u0, v0, u1, v1, a.tex_w[t], a.tex_h[t]);
      const float ry = footprint(u2, v2, u3, v3, a.tex_w[t], a.tex_h[t]);
      lvl = level_of(fmaxf(rx, ry), a.tex_levels[t]);
    }
  } else if (ground(a, fx, fy, u, v)) {
    const int64_t cx = (int64_t)floorf(u), cz = (int64_t)floorf(v);  // 2 m cells
    const uint64_t hs = cell_hash(a.cell_seed, (uint64_t)cx, (uint64_t)cz);
    t = (int)(hs % (uint64_t)a.ntex);
    u = fadd(u, fmul((float)((hs >> 16) & 0xFFFFu), 1.0f / 65536.0f));
    v = fadd(v, fmul((float)((hs >> 32) & 0xFFFFu), 1.0f / 65536.0f));
    if (a.use_mips) {
      float u0, v0, u1, v1, u2, v2, u3, v3;
      const bool ok = ground(a, (float)x, fy, u0, v0) && ground(a, fadd((float)x, 1.0f), fy, u1, v1) &&
                      ground(a, fx, (float)y, u2, v2) && ground(a, fx, fadd((float)y, 1.0f), u3, v3);
      if (!ok) {
        lvl = a.tex_levels[t] - 1;
      } else {
        const float rx = footprint(u0, v0, u1, v1, a.tex_w[t], a.tex_h[t]);
        const float ry = footprint(u2, v2, u3, v3, a.tex_w[t], a.tex_h[t]);
        lvl = level_of(fmaxf(rx, ry), a.tex_levels[t]);
      }
    }
  }
  const size_t p = (size_t)y * a.width + x;
  a.uv[p] = make_float2(u, v);
  a.tex[p] = (uint16_t)t;
  a.mip[p] = (uint8_t)lvl;
}

}  // namespace

void launch_raster(const RasterArgs& a, cudaStream_t s) {
  const dim3 grid((a.width + kTileX - 1) / kTileX, (a.height + kTileY - 1) / kTileY);
  k_raster<<<grid, kThreads, 0, s>>>(a);
}

}  // namespace jt
