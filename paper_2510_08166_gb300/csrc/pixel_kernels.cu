// Screen-space passes over the deferred G-buffer: Mark (paper Sec. 4.2) and Resolve /
// colourise (Sec. 4.4), for one or several views in one launch.
//
// Both stream the G-buffer (11 B/px read; colourise also writes 4 B/px and gathers texels
// from the block cache). A persistent grid walks the views in 128 x 32 pixel tiles, one
// warp per 128-pixel row segment and one quad of 4 pixels per lane (32 B + 8 B + 4 B vector
// loads, one 16 B store). Pixels of a tile share MCUs, so Mark keeps a 1024-entry table of
// the gids its CTA already flagged in shared memory and stores each flag about once per CTA
// instead of once per pixel (the byte stores of every SM to the same flag lines otherwise
// dominate the pass). A pixel's (texture, level) record is one 16-byte load, kept in
// registers while consecutive pixels share it; levels whose sides are powers of two (all
// mip chains of power-of-two textures) wrap with a mask, MCU coordinates are shifts.
//
// Texel addressing (fixed in fp32 with explicit rounding so it is the same on every
// device): nearest x = floor(u * w) floor-mod w; bilinear xs = u * w - 1/2, x0 = floor(xs),
// fx = xs - x0, taps x0 and x0 + 1 (floor-mod w); the MCU of texel (x, y) is
// x / mw + (y / mw) * mcus_x with mw = 16 (4:2:0) or 8 (4:4:4), and its key is the level's
// gid_base + MCU (Sec. 4.6).
#include <cuda_runtime.h>

#include <type_traits>

#include "jt_internal.cuh"

namespace jt {
namespace {

constexpr uint32_t kNoGid = 0xFFFFFFFFu;

__device__ __forceinline__ int floor_mod_i(int a, int w) {
  int r = a % w;
  return r < 0 ? r + w : r;
}

struct Lvl {
  uint32_t gid_base;
  int w, h, mcus_x, shift;
  uint32_t units, sampling;
  bool wp2, hp2;
  float wf, hf;
};

constexpr uint32_t kNoKey = 0xFFFFFFFFu;

// Key of a pixel's (texture, level) record, or kNoKey for pixels that are absent, empty,
// filtered out (only_tex) or name a texture id / level beyond the table.
__device__ __forceinline__ uint32_t level_key(const TexLookup& tl, bool present, uint32_t tex, uint32_t mip,
                                              int only_tex) {
  if (!present || tex == JT_EMPTY_TEXTURE || (only_tex >= 0 && (int)tex != only_tex)) return kNoKey;
  if (tex >= tl.map_ntex || mip >= JT_MAX_LEVELS) return kNoKey - 1;  // missing
  return tex * JT_MAX_LEVELS + mip;
}

// Level record for a key (w == 0 when the key is absent or the level was never uploaded).
__device__ __forceinline__ Lvl load_level(const TexLookup& tl, uint32_t key) {
  Lvl L;
  const uint4 r = key < kNoKey - 1 ? __ldg(tl.levels + key) : make_uint4(0, 0, 0, 0);
  L.gid_base = r.x;
  L.w = (int)(r.y & 0xFFFF);
  L.h = (int)(r.y >> 16);
  L.mcus_x = (int)(r.z & 0xFFFF);
  L.shift = (int)((r.z >> 16) & 15);
  L.units = (r.z >> 20) & 15;
  L.sampling = (r.z >> 24) & 15;
  L.wp2 = (r.z >> 28) & 1;
  L.hp2 = (r.z >> 29) & 1;
  L.wf = (float)L.w;
  L.hf = (float)L.h;
  return L;
}

// Keys of a quad's pixels.
struct QuadLevels {
  uint32_t key[4];
};

__device__ __forceinline__ void quad_levels(const TexLookup& tl, int n, const uint32_t t[4], const uint32_t m[4],
                                            int only_tex, QuadLevels& q) {
#pragma unroll
  for (int i = 0; i < 4; ++i) q.key[i] = level_key(tl, i < n, t[i], m[i], only_tex);
}

// Floor-mod of a texel coordinate; P2: the side is a power of two (a mask). The choice is
// made once per quad (warp-uniform), so the division-free path costs nothing extra.
template <bool P2>
__device__ __forceinline__ int wrap(int a, int w) {
  if (P2) return a & (w - 1);
  return floor_mod_i(a, w);
}

template <bool P2>
__device__ __forceinline__ void nearest_texel(float u, float v, const Lvl& L, int& x, int& y) {
  x = wrap<P2>(__float2int_rd(__fmul_rn(u, L.wf)), L.w);  // cvt.rmi saturates out-of-range values
  y = wrap<P2>(__float2int_rd(__fmul_rn(v, L.hf)), L.h);
}

template <bool P2>
__device__ __forceinline__ void bilinear_taps(float u, float v, const Lvl& L, int& xa, int& xb, int& ya, int& yb,
                                              float& fx, float& fy) {
  const float xs = __fsub_rn(__fmul_rn(u, L.wf), 0.5f);
  const float ys = __fsub_rn(__fmul_rn(v, L.hf), 0.5f);
  fx = __fsub_rn(xs, floorf(xs));
  fy = __fsub_rn(ys, floorf(ys));
  xa = wrap<P2>(__float2int_rd(xs), L.w);  // = floor(xs), saturated like floor then convert
  ya = wrap<P2>(__float2int_rd(ys), L.h);
  xb = xa + 1 == L.w ? 0 : xa + 1;
  yb = ya + 1 == L.h ? 0 : ya + 1;
}

// Calls f(P2, L, i) for the quad's pixels i = 0..3 with the level record of each, P2 a
// std::integral_constant telling whether the levels may be wrapped with a mask: known for
// the whole context, else decided per warp by a vote (so only one instantiation runs). A
// lane loads a level record only when its key differs from the previous pixel's (the
// pixels of a quad nearly always share one). Warp-collective: all 32 lanes must call it
// (lanes without pixels have empty keys).
template <bool P2, typename F>
__device__ __forceinline__ void quad_pixels_with(const TexLookup& tl, const QuadLevels& q, F&& f) {
  Lvl L = load_level(tl, kNoKey);
  uint32_t lk = kNoKey;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (q.key[i] != lk) {
      L = load_level(tl, q.key[i]);
      lk = q.key[i];
    }
    f(std::integral_constant<bool, P2>{}, L, i);
  }
}

template <typename F>
__device__ __forceinline__ void for_quad_pixels(const TexLookup& tl, const QuadLevels& q, F&& f) {
  bool p2 = true;
  if (!tl.all_p2) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (q.key[i] < kNoKey - 1) p2 &= ((__ldg(&tl.levels[q.key[i]].z) >> 28) & 3u) == 3u;
    p2 = __all_sync(0xFFFFFFFFu, p2);
  }
  if (p2)
    quad_pixels_with<true>(tl, q, f);
  else
    quad_pixels_with<false>(tl, q, f);
}

// Locates the view of global tile `tile` (views are few and sorted by tile_begin).
__device__ __forceinline__ int view_of_tile(const ViewSet& vs, uint32_t tile) {
  int vi = 0;
#pragma unroll 1
  for (int i = 1; i < vs.n; ++i)
    if (tile >= vs.v[i].tile_begin) vi = i;
  return vi;
}

// Loads up to 4 pixels of row y starting at column x (n = pixels present, 0..4).
__device__ __forceinline__ int load_px4(const View& V, int y, int x, float u[4], float v[4], uint32_t t[4],
                                        uint32_t m[4]) {
  const int n = (y < V.height && x < V.width) ? min(4, V.width - x) : 0;
  const uint32_t p0 = (uint32_t)y * (uint32_t)V.width + (uint32_t)x;
  if (n == 4 && (V.width & 3) == 0) {
    const uint32_t lq = p0 >> 2;
    const float4 a = __ldg(V.uv + 2 * lq), b = __ldg(V.uv + 2 * lq + 1);
    u[0] = a.x; v[0] = a.y; u[1] = a.z; v[1] = a.w;
    u[2] = b.x; v[2] = b.y; u[3] = b.z; v[3] = b.w;
    const uint2 tt = __ldg(reinterpret_cast<const uint2*>(V.tex) + lq);
    t[0] = tt.x & 0xFFFF; t[1] = tt.x >> 16; t[2] = tt.y & 0xFFFF; t[3] = tt.y >> 16;
    const uint32_t mm = __ldg(reinterpret_cast<const uint32_t*>(V.mip) + lq);
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

// Iterates the (view, row, column) of this thread's quads over the CTA's tiles:
// f(V, y, x) for every row segment a warp owns; warps take rows w, w + nwarps, ...
template <typename F>
__device__ __forceinline__ void for_each_quad(const ViewSet& vs, F&& f) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
#pragma unroll 1
  for (uint32_t tile = blockIdx.x; tile < vs.total_tiles; tile += gridDim.x) {
    const int vi = view_of_tile(vs, tile);
    const View& V = vs.v[vi];
    const uint32_t lt = tile - V.tile_begin;
    const int x = (int)(lt % V.tiles_x) * kTileW + lane * 4;
    const int y0 = (int)(lt / V.tiles_x) * kTileH;
#pragma unroll 1
    for (int r = warp; r < kTileH; r += nwarps) f(V, y0 + r, x);
  }
}

// ---------------------------------------------------------------------------------------
// Mark
// ---------------------------------------------------------------------------------------
constexpr int kSeen = 1024;  // per-CTA table of recently flagged gids

template <int FILTER>
__global__ void k_mark(const __grid_constant__ MarkArgs a) {
  __shared__ uint32_t seen[kSeen];
  for (int i = threadIdx.x; i < kSeen; i += blockDim.x) seen[i] = kNoGid;
  __syncthreads();
  bool missing = false;
  // flags gid g unless this CTA already did (racy by design: a duplicate store writes the
  // same byte)
  auto flag = [&](uint32_t g, uint32_t units) {
    uint32_t* e = &seen[(g ^ (g >> 10)) & (kSeen - 1)];
    if (*e != g) {
      *e = g;
      a.flags[g] = (uint8_t)units;
    }
  };
  for_each_quad(a.views, [&](const View& V, int y, int x) {
    float u[4], v[4];
    uint32_t t[4], m[4];
    const int n = load_px4(V, y, x, u, v, t, m);
    QuadLevels q;
    quad_levels(a.tl, n, t, m, a.only_tex, q);
    for_quad_pixels(a.tl, q, [&](auto p2, const Lvl& L, int i) {
      constexpr bool P2 = decltype(p2)::value;
      const uint32_t key = q.key[i];
      const bool ok = key < kNoKey - 1 && L.w != 0 && ((L.sampling == kSamplingCoef) == (a.coef_mode != 0));
      missing |= key != kNoKey && !ok;
      if (!ok) return;
      if (FILTER == JT_FILTER_NEAREST) {
        int tx, ty;
        nearest_texel<P2>(u[i], v[i], L, tx, ty);
        flag(L.gid_base + (tx >> L.shift) + (ty >> L.shift) * L.mcus_x, L.units);
      } else {
        int xa, xb, ya, yb;
        float fx, fy;
        bilinear_taps<P2>(u[i], v[i], L, xa, xb, ya, yb, fx, fy);
        const int mxa = xa >> L.shift, mxb = xb >> L.shift;
        const int mya = ya >> L.shift, myb = yb >> L.shift;
        const uint32_t row_a = L.gid_base + mya * L.mcus_x;
        flag(row_a + mxa, L.units);
        if (mxb != mxa) flag(row_a + mxb, L.units);  // the footprint straddles MCUs (rare)
        if (myb != mya) {
          const uint32_t row_b = L.gid_base + myb * L.mcus_x;
          flag(row_b + mxa, L.units);
          if (mxb != mxa) flag(row_b + mxb, L.units);
        }
      }
    });
  });
  if (missing) atomicOr(&a.state->err, JT_DEVERR_MISSING);
}

// ---------------------------------------------------------------------------------------
// Colourise
// ---------------------------------------------------------------------------------------
// Channel `ch` of an RGBA8 texel as float, exactly: the byte is placed under the exponent
// of 2^23 (PRMT) and the bias subtracted (full-rate ops instead of an int-to-float
// conversion).
__device__ __forceinline__ float chan(uint32_t c, int ch) {
  return __int_as_float((int)__byte_perm(c, 0x4B00u, 0x5440u | (uint32_t)ch)) - 8388608.0f;
}

// Bilinear blend in fp32 (lerp along x, then y); each channel rounds half up:
// floor(c + 1/2), computed as the low byte of (c + 1/2) + 2^23 rounded down.
__device__ __forceinline__ uint32_t blend(uint32_t c00, uint32_t c10, uint32_t c01, uint32_t c11, float fx,
                                          float fy) {
  uint32_t out = 0xFF000000u;
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    const float a0 = chan(c00, ch), a1 = chan(c10, ch), b0 = chan(c01, ch), b1 = chan(c11, ch);
    const float top = fmaf(fx, a1 - a0, a0);
    const float bot = fmaf(fx, b1 - b0, b0);
    const float c = fmaf(fy, bot - top, top);  // in [0, 255] up to rounding
    const uint32_t iv = (uint32_t)__float_as_int(__fadd_rd(__fadd_rn(c, 0.5f), 8388608.0f)) & 0x1FFu;
    out |= min(iv, 255u) << (8 * ch);
  }
  return out;
}

template <int FILTER>
__global__ void k_colorize(const __grid_constant__ ColorizeArgs a) {
  bool missing = false, bad = false;
  uint32_t last_gid = kNoGid, last_off = 0;  // slot of the last MCU looked up
  const uint32_t* cache = reinterpret_cast<const uint32_t*>(a.cache);
  // cache-unit offset of gid g (0 and `bad` when it would read past the cache)
  auto slot = [&](uint32_t g, uint32_t units) -> uint32_t {
    if (g != last_gid) {
      last_gid = g;
      last_off = __ldg(&a.slot[g]);
    }
    const bool fits = last_off + units <= a.cap_units;
    bad |= !fits;
    return fits ? last_off : 0u;
  };
  for_each_quad(a.views, [&](const View& V, int y, int x) {
    float u[4], v[4];
    uint32_t t[4], m[4];
    const int n = load_px4(V, y, x, u, v, t, m);
    QuadLevels q;
    quad_levels(a.tl, n, t, m, a.only_tex, q);
    uint32_t px[4];
    for_quad_pixels(a.tl, q, [&](auto p2, const Lvl& L, int i) {
      constexpr bool P2 = decltype(p2)::value;
      const uint32_t key = q.key[i];
      const bool ok = key < kNoKey - 1 && L.w != 0 && L.sampling != kSamplingCoef;
      missing |= key != kNoKey && !ok;
      px[i] = 0xFF000000u;  // empty pixel
      if (!ok) return;
      const int mwm = (1 << L.shift) - 1;
      if (FILTER == JT_FILTER_NEAREST) {
        int tx, ty;
        nearest_texel<P2>(u[i], v[i], L, tx, ty);
        const uint32_t off = slot(L.gid_base + (tx >> L.shift) + (ty >> L.shift) * L.mcus_x, L.units);
        px[i] = __ldg(cache + (size_t)off * (kUnitBytes / 4) + (((ty & mwm) << L.shift) | (tx & mwm)));
      } else if (FILTER == JT_FILTER_BILINEAR_CLAMP) {
        // bilinear taps clamped to the nearest texel's MCU: along each axis a tap in
        // another MCU moves onto the nearest texel's column or row (one MCU, one slot)
        int nx, ny, xa, xb, ya, yb;
        float fx, fy;
        nearest_texel<P2>(u[i], v[i], L, nx, ny);
        bilinear_taps<P2>(u[i], v[i], L, xa, xb, ya, yb, fx, fy);
        const int mx = nx >> L.shift, my = ny >> L.shift;
        xa = (xa >> L.shift) == mx ? xa : nx;
        xb = (xb >> L.shift) == mx ? xb : nx;
        ya = (ya >> L.shift) == my ? ya : ny;
        yb = (yb >> L.shift) == my ? yb : ny;
        const uint32_t* tile = cache + (size_t)slot(L.gid_base + mx + my * L.mcus_x, L.units) * (kUnitBytes / 4);
        const int ia = (ya & mwm) << L.shift, ib = (yb & mwm) << L.shift;
        const int ja = xa & mwm, jb = xb & mwm;
        px[i] = blend(__ldg(tile + (ia | ja)), __ldg(tile + (ia | jb)), __ldg(tile + (ib | ja)),
                      __ldg(tile + (ib | jb)), fx, fy);
      } else {
        int xa, xb, ya, yb;
        float fx, fy;
        bilinear_taps<P2>(u[i], v[i], L, xa, xb, ya, yb, fx, fy);
        const int mxa = xa >> L.shift, mxb = xb >> L.shift;
        const int mya = ya >> L.shift, myb = yb >> L.shift;
        const uint32_t row_a = L.gid_base + mya * L.mcus_x;
        const uint32_t o00 = slot(row_a + mxa, L.units);
        uint32_t o10 = o00, o01 = o00, o11 = o00;
        if (mxb != mxa || myb != mya) {  // the footprint straddles MCUs (rare)
          const uint32_t row_b = L.gid_base + myb * L.mcus_x;
          o10 = slot(row_a + mxb, L.units);
          o01 = slot(row_b + mxa, L.units);
          o11 = slot(row_b + mxb, L.units);
        }
        const int ia = (ya & mwm) << L.shift, ib = (yb & mwm) << L.shift;
        const int ja = xa & mwm, jb = xb & mwm;
        const uint32_t c00 = __ldg(cache + (size_t)o00 * (kUnitBytes / 4) + (ia | ja));
        const uint32_t c10 = __ldg(cache + (size_t)o10 * (kUnitBytes / 4) + (ia | jb));
        const uint32_t c01 = __ldg(cache + (size_t)o01 * (kUnitBytes / 4) + (ib | ja));
        const uint32_t c11 = __ldg(cache + (size_t)o11 * (kUnitBytes / 4) + (ib | jb));
        px[i] = blend(c00, c10, c01, c11, fx, fy);
      }
    });
    if (n == 0) return;
    bool write[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) write[i] = i < n && (a.only_tex < 0 || (int)t[i] == a.only_tex);
    const uint32_t p0 = (uint32_t)y * (uint32_t)V.width + (uint32_t)x;
    if (n == 4 && (V.width & 3) == 0 && write[0] && write[1] && write[2] && write[3]) {
      V.out[p0 >> 2] = make_uint4(px[0], px[1], px[2], px[3]);
    } else {
      uint32_t* o = reinterpret_cast<uint32_t*>(V.out) + p0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (write[i]) o[i] = px[i];
    }
  });
  if (missing) atomicOr(&a.state->err, JT_DEVERR_MISSING);
  if (bad) atomicOr(&a.state->err, JT_DEVERR_CAPACITY);
}

// ---------------------------------------------------------------------------------------
// Float chain (differentiable colourise, not in the paper): bilinear taps as above over
// the float tiles of the coefficient textures; weights (1-fx)(1-fy), fx(1-fy), (1-fx)fy, fx fy.
// The forward pass blends the four texels; the backward pass scatters w * dL/dF into the
// four texels' gradient tiles (float4 atomics; their order is the only non-determinism).
// ---------------------------------------------------------------------------------------
struct FloatTaps {
  uint32_t idx[4];  // float4 index into the tiles (tile * 256 + texel)
  float w[4];
  bool ok;
};

// Taps of one pixel; ok = false (and `missing`/`over` updated) when the pixel is empty,
// names a texture that is not a coefficient texture, or a tap's tile is past the capacity.
template <bool P2>
__device__ __forceinline__ FloatTaps float_taps(const FloatArgs& a, const Lvl& L, uint32_t key, float u, float v,
                                                bool& missing, bool& over) {
  FloatTaps T;
  T.ok = key < kNoKey - 1 && L.w != 0 && L.sampling == kSamplingCoef;
  missing |= key != kNoKey && !T.ok;
  int xa, xb, ya, yb;
  float fx, fy;
  bilinear_taps<P2>(u, v, L, xa, xb, ya, yb, fx, fy);
  const int xs[4] = {xa, xb, xa, xb}, ys[4] = {ya, ya, yb, yb};
  T.w[0] = (1.f - fx) * (1.f - fy);
  T.w[1] = fx * (1.f - fy);
  T.w[2] = (1.f - fx) * fy;
  T.w[3] = fx * fy;
  bool fit = true;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t g = L.gid_base + (xs[i] >> 4) + (ys[i] >> 4) * L.mcus_x;
    const uint32_t tile = T.ok ? __ldg(a.slot + g) : 0u;
    fit &= tile < a.tile_cap;
    T.idx[i] = (tile < a.tile_cap ? tile : 0u) * 256u + (uint32_t)(((ys[i] & 15) << 4) | (xs[i] & 15));
  }
  over |= T.ok && !fit;
  T.ok = T.ok && fit;
  return T;
}

template <bool BACKWARD>
__global__ void k_float_pixels(const __grid_constant__ FloatArgs a) {
  bool missing = false, over = false;
  for_each_quad(a.views, [&](const View& V, int y, int x) {
    float u[4], v[4];
    uint32_t t[4], m[4];
    const int n = load_px4(V, y, x, u, v, t, m);
    QuadLevels q;
    quad_levels(a.tl, n, t, m, -1, q);
    // every lane goes on to for_quad_pixels (it may vote); lanes without pixels touch no memory
    const uint32_t p0 = (uint32_t)y * (uint32_t)V.width + (uint32_t)x;
    float* fr = a.frame + (size_t)p0 * 3;  // 12 floats of the quad, 16-byte aligned when p0 % 4 == 0
    const bool vec = n == 4 && (V.width & 3) == 0;
    float rgb[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) rgb[i] = 0.f;
    if (BACKWARD && n > 0) {
      if (vec) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const float4 g4 = __ldg(reinterpret_cast<const float4*>(fr) + i);
          rgb[4 * i] = g4.x; rgb[4 * i + 1] = g4.y; rgb[4 * i + 2] = g4.z; rgb[4 * i + 3] = g4.w;
        }
      } else {
#pragma unroll
        for (int i = 0; i < 12; ++i) rgb[i] = i < 3 * n ? __ldg(fr + i) : 0.f;
      }
    }
    for_quad_pixels(a.tl, q, [&](auto p2, const Lvl& L, int i) {
      const FloatTaps T = float_taps<decltype(p2)::value>(a, L, q.key[i], u[i], v[i], missing, over);
      if (BACKWARD) {
        if (T.ok) {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            atomicAdd(a.tiles + T.idx[k], make_float4(T.w[k] * rgb[3 * i], T.w[k] * rgb[3 * i + 1],
                                                      T.w[k] * rgb[3 * i + 2], 0.f));
        }
      } else {
        float r = 0.f, gg = 0.f, b = 0.f;
        if (T.ok) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float4 c = __ldg(a.tiles + T.idx[k]);
            r = fmaf(T.w[k], c.x, r);
            gg = fmaf(T.w[k], c.y, gg);
            b = fmaf(T.w[k], c.z, b);
          }
        }
        rgb[3 * i] = r;
        rgb[3 * i + 1] = gg;
        rgb[3 * i + 2] = b;
      }
    });
    if (!BACKWARD && n > 0) {
      if (vec) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
          reinterpret_cast<float4*>(fr)[i] = make_float4(rgb[4 * i], rgb[4 * i + 1], rgb[4 * i + 2], rgb[4 * i + 3]);
      } else {
#pragma unroll
        for (int i = 0; i < 12; ++i)
          if (i < 3 * n) fr[i] = rgb[i];
      }
    }
  });
  if (missing) atomicOr(&a.state->err, JT_DEVERR_MISSING);
  if (over) atomicOr(&a.state->err, JT_DEVERR_CAPACITY);
}

}  // namespace

void launch_float_colorize(const FloatArgs& a, int threads, int grid, cudaStream_t s) {
  k_float_pixels<false><<<grid, threads, 0, s>>>(a);
}

void launch_float_scatter(const FloatArgs& a, int threads, int grid, cudaStream_t s) {
  k_float_pixels<true><<<grid, threads, 0, s>>>(a);
}

void launch_mark(const MarkArgs& a, int threads, int grid, cudaStream_t s) {
  // the clamped filter reads only the nearest texel's MCU
  if (a.filter == JT_FILTER_NEAREST || a.filter == JT_FILTER_BILINEAR_CLAMP)
    k_mark<JT_FILTER_NEAREST><<<grid, threads, 0, s>>>(a);
  else
    k_mark<JT_FILTER_BILINEAR><<<grid, threads, 0, s>>>(a);
}

void launch_colorize(const ColorizeArgs& a, int threads, int grid, cudaStream_t s) {
  if (a.filter == JT_FILTER_NEAREST)
    k_colorize<JT_FILTER_NEAREST><<<grid, threads, 0, s>>>(a);
  else if (a.filter == JT_FILTER_BILINEAR_CLAMP)
    k_colorize<JT_FILTER_BILINEAR_CLAMP><<<grid, threads, 0, s>>>(a);
  else
    k_colorize<JT_FILTER_BILINEAR><<<grid, threads, 0, s>>>(a);
}

}  // namespace jt
