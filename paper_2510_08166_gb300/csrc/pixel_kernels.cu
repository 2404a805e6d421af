// Screen-space passes over the deferred G-buffer: Mark (paper Sec. 4.2) and Resolve /
// colourise (Sec. 4.4), for one or several views in one launch.
//
// Both are HBM-bound streams over the G-buffer (11 B/px read; colourise also writes 4 B/px
// and gathers texels from the block cache). Each thread handles a quad of 4 consecutive
// pixels with 32 B + 8 B + 4 B vector loads (and one 16 B store), in a grid-stride loop
// over all views' quads; views are passed by value (__grid_constant__).
//
// Texel addressing (shared by both passes and fixed in fp32 with explicit rounding so it
// is the same on every device): nearest x = floor(u * w) floor-mod w; bilinear
// xs = u * w - 1/2, x0 = floor(xs), fx = xs - x0, taps x0 and x0 + 1 (floor-mod w); the MCU
// of texel (x, y) is x / mw + (y / mw) * mcus_x with mw = 16 (4:2:0) or 8 (4:4:4), and its
// key is the level's gid_base + MCU (Sec. 4.6).
#include <cuda_runtime.h>

#include "jt_internal.cuh"

namespace jt {
namespace {

constexpr uint32_t kNoGid = 0xFFFFFFFFu;

__device__ __forceinline__ int floor_mod_i(int a, int w) {
  int r = a % w;
  return r < 0 ? r + w : r;
}

struct LevelInfo {
  uint32_t gid_base;
  int w, h, mcus_x, mw;
  uint32_t units;
  int sampling;
};

// (tex, mip) -> level; false when the pair was never uploaded.
__device__ __forceinline__ bool lookup_level(const TexLookup& tl, uint32_t tex, uint32_t mip, LevelInfo& L) {
  if (tex >= tl.map_ntex || mip >= JT_MAX_LEVELS) return false;
  int di = __ldg(&tl.desc_map[tex * JT_MAX_LEVELS + mip]);
  if (di < 0) return false;
  const DevDesc* d = tl.descs + di;
  L.gid_base = __ldg(&d->gid_base);
  L.w = __ldg(&d->width);
  L.h = __ldg(&d->height);
  L.mcus_x = __ldg(&d->mcus_x);
  L.sampling = __ldg(&d->sampling);
  L.units = __ldg(&d->units);
  L.mw = L.sampling == kSampling444 ? 8 : 16;
  return true;
}

__device__ __forceinline__ void nearest_texel(float u, float v, const LevelInfo& L, int& x, int& y) {
  float uw = __fmul_rn(u, (float)L.w);
  float vh = __fmul_rn(v, (float)L.h);
  x = floor_mod_i(__float2int_rd(uw), L.w);  // cvt.rmi saturates out-of-range values
  y = floor_mod_i(__float2int_rd(vh), L.h);
}

__device__ __forceinline__ void bilinear_taps(float u, float v, const LevelInfo& L, int& xa, int& xb, int& ya,
                                              int& yb, float& fx, float& fy) {
  float xs = __fsub_rn(__fmul_rn(u, (float)L.w), 0.5f);
  float ys = __fsub_rn(__fmul_rn(v, (float)L.h), 0.5f);
  float x0 = floorf(xs), y0 = floorf(ys);
  fx = __fsub_rn(xs, x0);
  fy = __fsub_rn(ys, y0);
  xa = floor_mod_i(__float2int_rd(x0), L.w);
  ya = floor_mod_i(__float2int_rd(y0), L.h);
  xb = xa + 1 == L.w ? 0 : xa + 1;
  yb = ya + 1 == L.h ? 0 : ya + 1;
}

// Locates the view of global quad q (views are few and sorted by quad_begin).
__device__ __forceinline__ int view_of(const ViewSet& vs, uint32_t q) {
  int vi = 0;
#pragma unroll 1
  for (int i = 1; i < vs.n; ++i)
    if (q >= vs.v[i].quad_begin) vi = i;
  return vi;
}

// Loads the 4 pixels of quad `lq` of view V (n = pixels present, 0..4).
__device__ __forceinline__ int load_quad(const View& V, uint32_t lq, float u[4], float v[4], uint32_t t[4],
                                         uint32_t m[4]) {
  uint32_t p0 = lq * 4;
  int n = (int)min(4u, V.npx - p0);
  if (n == 4) {
    float4 a = __ldg(V.uv + 2 * lq), b = __ldg(V.uv + 2 * lq + 1);
    u[0] = a.x; v[0] = a.y; u[1] = a.z; v[1] = a.w;
    u[2] = b.x; v[2] = b.y; u[3] = b.z; v[3] = b.w;
    uint2 tt = __ldg(reinterpret_cast<const uint2*>(V.tex) + lq);
    t[0] = tt.x & 0xFFFF; t[1] = tt.x >> 16; t[2] = tt.y & 0xFFFF; t[3] = tt.y >> 16;
    uint32_t mm = __ldg(reinterpret_cast<const uint32_t*>(V.mip) + lq);
    m[0] = mm & 255; m[1] = (mm >> 8) & 255; m[2] = (mm >> 16) & 255; m[3] = mm >> 24;
  } else {
    const float* uvs = reinterpret_cast<const float*>(V.uv);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (i < n) {
        u[i] = __ldg(uvs + 2 * (p0 + i));
        v[i] = __ldg(uvs + 2 * (p0 + i) + 1);
        t[i] = __ldg(V.tex + p0 + i);
        m[i] = __ldg(V.mip + p0 + i);
      } else {
        u[i] = v[i] = 0.f;
        t[i] = JT_EMPTY_TEXTURE;
        m[i] = 0;
      }
    }
  }
  return n;
}

// ---------------------------------------------------------------------------------------
// Mark
// ---------------------------------------------------------------------------------------
template <int FILTER>
__global__ void k_mark(const __grid_constant__ MarkArgs a) {
  const int lane = threadIdx.x & 31;
  const uint32_t stride = gridDim.x * blockDim.x;
  const uint32_t total = a.views.total_quads;
  uint32_t last[4] = {kNoGid, kNoGid, kNoGid, kNoGid};
  bool missing = false;
  // warp-uniform loop bound so every lane takes part in the neighbour shuffles
  for (uint32_t q0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); q0 < total; q0 += stride) {
    const uint32_t q = q0 + lane;
    float u[4], v[4];
    uint32_t t[4], m[4];
    int n = 0;
    if (q < total) {
      const int vi = view_of(a.views, q);
      n = load_quad(a.views.v[vi], q - a.views.v[vi].quad_begin, u, v, t, m);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      uint32_t g[4] = {kNoGid, kNoGid, kNoGid, kNoGid};
      uint32_t units = 0;
      if (i < n && t[i] != JT_EMPTY_TEXTURE && (a.only_tex < 0 || (int)t[i] == a.only_tex)) {
        LevelInfo L;
        bool ok = lookup_level(a.tl, t[i], m[i], L);
        if (ok && ((L.sampling == kSamplingCoef) != (a.coef_mode != 0))) ok = false;
        if (!ok) {
          missing = true;
        } else {
          units = L.units;
          if (FILTER == JT_FILTER_NEAREST) {
            int x, y;
            nearest_texel(u[i], v[i], L, x, y);
            g[0] = L.gid_base + x / L.mw + (y / L.mw) * L.mcus_x;
          } else {
            int xa, xb, ya, yb;
            float fx, fy;
            bilinear_taps(u[i], v[i], L, xa, xb, ya, yb, fx, fy);
            int mxa = xa / L.mw, mxb = xb / L.mw, mya = ya / L.mw, myb = yb / L.mw;
            g[0] = L.gid_base + mxa + mya * L.mcus_x;
            if (mxb != mxa) g[1] = L.gid_base + mxb + mya * L.mcus_x;
            if (myb != mya) g[2] = L.gid_base + mxa + myb * L.mcus_x;
            if (mxb != mxa && myb != mya) g[3] = L.gid_base + mxb + myb * L.mcus_x;
          }
        }
      }
      // Store a flag unless this thread just stored the same gid or the neighbouring lane
      // (the pixels just left of ours) holds it: consecutive pixels mostly share MCUs.
#pragma unroll
      for (int j = 0; j < (FILTER == JT_FILTER_NEAREST ? 1 : 4); ++j) {
        const uint32_t nb = __shfl_up_sync(0xFFFFFFFFu, g[j], 1);
        if (g[j] != kNoGid) {
          if (g[j] != last[j] && !(lane > 0 && nb == g[j])) a.flags[g[j]] = (uint8_t)units;
          last[j] = g[j];
        }
      }
    }
  }
  if (missing) atomicOr(&a.state->err, JT_DEVERR_MISSING);
}

// ---------------------------------------------------------------------------------------
// Colourise
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t fetch_texel(const ColorizeArgs& a, const LevelInfo& L, int x, int y,
                                                bool& bad) {
  const uint32_t gid = L.gid_base + x / L.mw + (y / L.mw) * L.mcus_x;
  const uint32_t off = __ldg(&a.slot[gid]);
  if (off + L.units > a.cap_units) {
    bad = true;
    return 0xFF000000u;
  }
  const uint32_t* tile = reinterpret_cast<const uint32_t*>(a.cache + (size_t)off * kUnitBytes);
  return __ldg(tile + (y & (L.mw - 1)) * L.mw + (x & (L.mw - 1)));
}

__device__ __forceinline__ uint32_t blend(uint32_t c00, uint32_t c10, uint32_t c01, uint32_t c11, float fx,
                                          float fy) {
  uint32_t out = 0xFF000000u;
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    const int sh = 8 * ch;
    float a0 = (float)((c00 >> sh) & 255), a1 = (float)((c10 >> sh) & 255);
    float b0 = (float)((c01 >> sh) & 255), b1 = (float)((c11 >> sh) & 255);
    float top = fmaf(fx, a1 - a0, a0);
    float bot = fmaf(fx, b1 - b0, b0);
    float c = fmaf(fy, bot - top, top);
    int iv = __float2int_rd(c + 0.5f);
    iv = min(255, max(0, iv));
    out |= (uint32_t)iv << sh;
  }
  return out;
}

template <int FILTER>
__global__ void k_colorize(const __grid_constant__ ColorizeArgs a) {
  const uint32_t stride = gridDim.x * blockDim.x;
  const uint32_t total = a.views.total_quads;
  bool missing = false, bad = false;
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += stride) {
    const int vi = view_of(a.views, q);
    const View& V = a.views.v[vi];
    const uint32_t lq = q - V.quad_begin;
    float u[4], v[4];
    uint32_t t[4], m[4];
    const int n = load_quad(V, lq, u, v, t, m);
    uint32_t px[4];
    bool write[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      px[i] = 0xFF000000u;
      write[i] = i < n && (a.only_tex < 0 || (int)t[i] == a.only_tex);
      if (!write[i] || t[i] == JT_EMPTY_TEXTURE) continue;
      LevelInfo L;
      if (!lookup_level(a.tl, t[i], m[i], L) || L.sampling == kSamplingCoef) {
        missing = true;
        continue;
      }
      if (FILTER == JT_FILTER_NEAREST) {
        int x, y;
        nearest_texel(u[i], v[i], L, x, y);
        px[i] = fetch_texel(a, L, x, y, bad);
      } else {
        int xa, xb, ya, yb;
        float fx, fy;
        bilinear_taps(u[i], v[i], L, xa, xb, ya, yb, fx, fy);
        uint32_t c00 = fetch_texel(a, L, xa, ya, bad), c10 = fetch_texel(a, L, xb, ya, bad);
        uint32_t c01 = fetch_texel(a, L, xa, yb, bad), c11 = fetch_texel(a, L, xb, yb, bad);
        px[i] = blend(c00, c10, c01, c11, fx, fy);
      }
    }
    if (n == 4 && write[0] && write[1] && write[2] && write[3]) {
      V.out[lq] = make_uint4(px[0], px[1], px[2], px[3]);
    } else {
      uint32_t* o = reinterpret_cast<uint32_t*>(V.out) + (size_t)lq * 4;
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (write[i]) o[i] = px[i];
    }
  }
  if (missing) atomicOr(&a.state->err, JT_DEVERR_MISSING);
  if (bad) atomicOr(&a.state->err, JT_DEVERR_CAPACITY);
}

}  // namespace

void launch_mark(const MarkArgs& a, int threads, int grid, cudaStream_t s) {
  if (a.filter == JT_FILTER_NEAREST)
    k_mark<JT_FILTER_NEAREST><<<grid, threads, 0, s>>>(a);
  else
    k_mark<JT_FILTER_BILINEAR><<<grid, threads, 0, s>>>(a);
}

void launch_colorize(const ColorizeArgs& a, int threads, int grid, cudaStream_t s) {
  if (a.filter == JT_FILTER_NEAREST)
    k_colorize<JT_FILTER_NEAREST><<<grid, threads, 0, s>>>(a);
  else
    k_colorize<JT_FILTER_BILINEAR><<<grid, threads, 0, s>>>(a);
}

}  // namespace jt
