// Screen-space passes over the deferred G-buffer: Mark (paper Sec. 4.2) and Resolve /
// colourise (Sec. 4.4), for one or several views in one launch.
//
// Both stream the G-buffer (11 B/px read; colourise also writes 4 B/px and gathers texels
// from the block cache). A persistent grid walks the views in 128 x 32 pixel tiles, one warp
// per 128-pixel row.
//
// Mark: one quad of 4 pixels per lane (32 B + 8 B + 4 B vector loads). Pixels of a tile
// share MCUs, so Mark keeps a 1024-entry table of the gids its CTA already flagged in shared
// memory and stores each flag about once per CTA instead of once per pixel (the byte stores
// of every SM to the same flag lines otherwise dominate the pass). A pixel's (texture,
// level) record is one 16-byte load, kept in registers while consecutive pixels share it;
// levels whose sides are powers of two (all mip chains of power-of-two textures) wrap with a
// mask, MCU coordinates are shifts.
//
// Colourise: a lane owns pixels 32 apart (lane + 32 k), so the 32 addresses of one texel
// gather instruction are 32 consecutive pixels' taps, which fall in two or three tiles (half
// the L1 wavefronts of quads per lane); the next step's G-buffer is loaded before the current
// one is shaded; a pixel's level comes from a 32-byte record that needs no decoding; the
// bilinear blend runs in fp16 pairs within a proven 1-LSB bound.
//
// Texel addressing (fixed in fp32 with explicit rounding so it is the same on every
// device): nearest x = floor(u * w) floor-mod w; bilinear xs = u * w - 1/2, x0 = floor(xs),
// fx = xs - x0, taps x0 and x0 + 1 (floor-mod w); the MCU of texel (x, y) is
// x / mw + (y / mw) * mcus_x with mw = 16 (4:2:0) or 8 (4:4:4), and its key is the level's
// gid_base + MCU (Sec. 4.6).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstring>
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
// Texel addressing of Colourise
// ---------------------------------------------------------------------------------------
// floor(x) for |x| < 2^22 by one round-down add: t = x + 1.5 * 2^23 rounded down is exactly
// floor(x) + 1.5 * 2^23 (the sum lies in [2^23, 2^24), where floats are the integers), so
// t - 1.5 * 2^23 is floor(x) as a float, and the bit pattern of t is that of 1.5 * 2^23
// (a multiple of 2^22) plus floor(x): masked by w - 1 (w a power of two below 2^22) it is
// floor(x) floor-mod w. Pixels outside that range, and levels whose sides are not powers of
// two, take the general path (conversion instructions, which saturate, and a division).
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23

// A pixel's level, from its PixRec (two vector loads; all fields zero for keys outside the
// table, so every address derived from them stays in range).
struct PixL {
  uint32_t gid_base;
  float wf, hf;
  uint32_t masks;  // (w - 1) | (h - 1) << 16
  uint32_t mcus_x;
  uint32_t shift;
  uint32_t info;   // units | kPixJpeg | kPixCoef | kPixPow2
  uint32_t wh;     // w | h << 16
};

__device__ __forceinline__ PixL pix_level(const TexLookup& tl, uint32_t tm) {
  const uint32_t tex = tm & 0xFFFFu, mip = tm >> 16;
  const uint32_t key =
      (tex < tl.map_ntex && mip < JT_MAX_LEVELS) ? tex * JT_MAX_LEVELS + mip : tl.map_ntex * JT_MAX_LEVELS;
  const uint4 r0 = __ldg(tl.pix + 2 * key), r1 = __ldg(tl.pix + 2 * key + 1);
  PixL P;
  P.gid_base = r0.x;
  P.wf = __uint_as_float(r0.y);
  P.hf = __uint_as_float(r0.z);
  P.masks = r0.w;
  P.mcus_x = r1.x;
  P.shift = r1.y;
  P.info = r1.z;
  P.wh = r1.w;
  return P;
}

// Bilinear taps on the fast path: a power-of-two level and |u w|, |v h| < 2^22 (returns
// false otherwise; every tap is then still inside the level, so loads made from it stay in
// range, but the caller must redo the pixel on the general path). Columns xa, xb = xa + 1,
// rows ya, yb = ya + 1 (repeat wrap), fractions fx, fy.
__device__ __forceinline__ bool taps_fast(const PixL& P, float u, float v, int& xa, int& xb, int& ya, int& yb,
                                          float& fx, float& fy) {
  const float xs = __fsub_rn(__fmul_rn(u, P.wf), 0.5f), ys = __fsub_rn(__fmul_rn(v, P.hf), 0.5f);
  const float tx = __fadd_rd(xs, kMagic), ty = __fadd_rd(ys, kMagic);
  fx = __fsub_rn(xs, __fsub_rn(tx, kMagic));
  fy = __fsub_rn(ys, __fsub_rn(ty, kMagic));
  const int wm = (int)(P.masks & 0xFFFFu), hm = (int)(P.masks >> 16);
  xa = __float_as_int(tx) & wm;
  ya = __float_as_int(ty) & hm;
  xb = (xa + 1) & wm;
  yb = (ya + 1) & hm;
  return (P.info & kPixPow2) && fabsf(xs) < 4194304.0f && fabsf(ys) < 4194304.0f;
}

// Nearest texel on the fast path (same conditions as taps_fast).
__device__ __forceinline__ bool nearest_fast(const PixL& P, float u, float v, int& x, int& y) {
  const float xn = __fmul_rn(u, P.wf), yn = __fmul_rn(v, P.hf);
  x = __float_as_int(__fadd_rd(xn, kMagic)) & (int)(P.masks & 0xFFFFu);
  y = __float_as_int(__fadd_rd(yn, kMagic)) & (int)(P.masks >> 16);
  return (P.info & kPixPow2) && fabsf(xn) < 4194304.0f && fabsf(yn) < 4194304.0f;
}

// The same taps for any level and coordinate (conversion instructions, floor-mod by
// division): the general path.
__device__ __forceinline__ void taps_any(const PixL& P, float u, float v, int& xa, int& xb, int& ya, int& yb,
                                         float& fx, float& fy) {
  const int w = (int)(P.wh & 0xFFFFu), h = (int)(P.wh >> 16);
  const float xs = __fsub_rn(__fmul_rn(u, P.wf), 0.5f), ys = __fsub_rn(__fmul_rn(v, P.hf), 0.5f);
  fx = __fsub_rn(xs, floorf(xs));
  fy = __fsub_rn(ys, floorf(ys));
  xa = floor_mod_i(__float2int_rd(xs), w);  // cvt.rmi saturates out-of-range values
  ya = floor_mod_i(__float2int_rd(ys), h);
  xb = xa + 1 == w ? 0 : xa + 1;
  yb = ya + 1 == h ? 0 : ya + 1;
}

__device__ __forceinline__ void nearest_any(const PixL& P, float u, float v, int& x, int& y) {
  x = floor_mod_i(__float2int_rd(__fmul_rn(u, P.wf)), (int)(P.wh & 0xFFFFu));
  y = floor_mod_i(__float2int_rd(__fmul_rn(v, P.hf)), (int)(P.wh >> 16));
}

// Walks the views' tiles: CTA tiles blockIdx.x, + gridDim.x, ...; warp rows w, w + nwarps,
// ... of each tile. A row of a tile is 128 pixels, taken in SPR steps of 128 / SPR pixels
// (the unit of work of a warp). The tile origin is recomputed only when the tile changes.
template <int SPR>
struct TileWalk {
  uint32_t tile;
  int r, h;    // row in the tile, step in the row
  int vi;      // view of the tile
  int x0, y0;  // tile origin
  __device__ __forceinline__ bool valid(const ViewSet& vs) const { return tile < vs.total_tiles; }
  __device__ __forceinline__ void set_tile(const ViewSet& vs) {
    if (tile >= vs.total_tiles) return;
    vi = view_of_tile(vs, tile);
    const View& V = vs.v[vi];
    const uint32_t lt = tile - V.tile_begin;
    const uint32_t ty = lt / V.tiles_x;
    x0 = (int)(lt - ty * V.tiles_x) * kTileW;
    y0 = (int)ty * kTileH;
  }
  __device__ __forceinline__ void start(const ViewSet& vs) {
    tile = blockIdx.x;
    r = threadIdx.x >> 5;
    h = 0;
    vi = 0;
    x0 = y0 = 0;
    set_tile(vs);
  }
  __device__ __forceinline__ void advance(const ViewSet& vs) {
    if (++h < SPR) return;
    h = 0;
    r += blockDim.x >> 5;
    if (r >= kTileH) {
      r = threadIdx.x >> 5;
      tile += gridDim.x;
      set_tile(vs);
    }
  }
  __device__ __forceinline__ int x() const { return x0 + h * (kTileW / SPR); }  // first pixel of the step
  __device__ __forceinline__ int y() const { return y0 + r; }
};

// G-buffer of a lane's pixels of the next step, loaded one step ahead of its use so that
// its HBM reads are in flight while the lane works on the current one.
template <int NPX>
struct RowG {  // Colourise: pixels x + lane + 32 k, k < NPX, of one step of a row
  float u[NPX], v[NPX];
  uint32_t tm[NPX];  // texture id | mip level << 16 (JT_EMPTY_TEXTURE past the view)
  uint32_t p0;       // index of pixel k = 0 in the view
  uint32_t n;        // pixels present: those with k < n
};

template <int NPX>
__device__ __forceinline__ void load_row(const View& V, int x, int y, bool valid, RowG<NPX>& g) {
  g.n = (valid && y < V.height && x < V.width) ? (uint32_t)min(NPX, (V.width - x + 31) >> 5) : 0u;
  g.p0 = (uint32_t)y * (uint32_t)V.width + (uint32_t)x;
  const float2* uv = reinterpret_cast<const float2*>(V.uv) + g.p0;
  const uint16_t* tx = V.tex + g.p0;
  const uint8_t* mp = V.mip + g.p0;
#pragma unroll
  for (int k = 0; k < NPX; ++k) {
    g.u[k] = g.v[k] = 0.f;
    g.tm[k] = JT_EMPTY_TEXTURE;
    if ((uint32_t)k < g.n) {
      const float2 t = __ldg(uv + 32 * k);
      g.u[k] = t.x;
      g.v[k] = t.y;
      g.tm[k] = (uint32_t)__ldg(tx + 32 * k) | ((uint32_t)__ldg(mp + 32 * k) << 16);
    }
  }
}

// ---------------------------------------------------------------------------------------
// Mark
// ---------------------------------------------------------------------------------------
constexpr int kSeen = 1024;  // per-CTA table of recently flagged gids

template <int FILTER, bool MULTI>
__global__ void k_mark(const __grid_constant__ MarkArgs a) {
  __shared__ uint32_t seen[kSeen];
  pdl_launch_dependents();
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
__device__ __forceinline__ __half2 u32_as_h2(uint32_t w) {
  __half2 h;
  memcpy(&h, &w, 4);
  return h;
}
__device__ __forceinline__ uint32_t h2_as_u32(__half2 h) {
  uint32_t w;
  memcpy(&w, &h, 4);
  return w;
}

// Bilinear blend of four RGBA8 texels with weights from fx, fy, rounded to bytes; alpha is
// 255 (every texel's). Channels are blended two at a time in fp16 pairs: a byte b becomes
// the half 1024 + b exactly (one byte permute under the exponent of 1024), differences of
// two such halves are exact, and each lerp a + f (b - a) is one fused fp16 multiply-add.
// The result c is rounded by adding 1536, whose binade [1024, 2048) has unit spacing, so
// the low byte of the sum is round(c). Error bound: fx, fy carry at most 2^-12 absolute
// error after the conversion to fp16 (255 * 2^-12 < 0.063 per lerp), each fp16 lerp and
// difference of values below 256 rounds by at most 1/16, so |c - c_exact| < 0.32 over the
// three lerps and one difference, and the byte differs from floor(c_exact + 1/2) by at most
// one. c stays within [-0.32, 255.32], so c + 1536 never leaves [1024, 2048).
__device__ __forceinline__ uint32_t blend_h(uint32_t c00, uint32_t c10, uint32_t c01, uint32_t c11, float fx,
                                            float fy) {
  const __half2 in_bias = u32_as_h2(0x64006400u);   // (1024, 1024)
  const __half2 out_bias = u32_as_h2(0x66006600u);  // (1536, 1536)
  const __half2 hx = __float2half2_rn(fx), hy = __float2half2_rn(fy);
  auto lerp_x = [&](uint32_t a, uint32_t b, uint32_t sel) {
    const __half2 ha = u32_as_h2(__byte_perm(a, 0x64646464u, sel));
    const __half2 hb = u32_as_h2(__byte_perm(b, 0x64646464u, sel));
    return __hfma2(hx, __hsub2(hb, ha), __hsub2(ha, in_bias));
  };
  const __half2 top_rg = lerp_x(c00, c10, 0x5140u), bot_rg = lerp_x(c01, c11, 0x5140u);  // (R, G)
  const __half2 top_ba = lerp_x(c00, c10, 0x5342u), bot_ba = lerp_x(c01, c11, 0x5342u);  // (B, A)
  const __half2 rg = __hadd2(__hfma2(hy, __hsub2(bot_rg, top_rg), top_rg), out_bias);
  const __half2 ba = __hadd2(__hfma2(hy, __hsub2(bot_ba, top_ba), top_ba), out_bias);
  return __byte_perm(h2_as_u32(rg), h2_as_u32(ba), 0x6420u);
}

// Slot at a, or 0 without touching memory when p is false: a predicated load, so that no
// branch orders one pixel's loads behind another's.
__device__ __forceinline__ uint32_t ldg_slot_if(bool p, const uint32_t* a) {
  uint32_t v;
  asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\tmov.u32 %0, 0;\n\t@q ld.global.nc.u32 %0, [%1];\n\t}"
      : "=r"(v)
      : "l"(a), "r"((uint32_t)p));
  return v;
}

// One pixel's colour from its taps: slots of up to four MCUs (predicated loads, the ones
// beyond the first only when the footprint straddles MCUs) and four texel gathers, then the
// blend (bilinear) or the texel itself (nearest). Branch-free: a pixel that is not shaded
// (ok false) reads no slot and gathers its texels from unit 0 (the cache holds at least one
// block), so the pixels of a lane overlap their chains.
template <int FILTER>
__device__ __forceinline__ uint32_t shade(const uint32_t* __restrict__ slot, const uint32_t* __restrict__ cache,
                                          const PixL& P, bool ok, int xa, int xb, int ya, int yb, float fx,
                                          float fy) {
  const uint32_t s = P.shift, mwm = (1u << s) - 1u;
  const uint32_t xas = (uint32_t)xa >> s, xbs = (uint32_t)xb >> s;
  const uint32_t rowa = P.gid_base + ((uint32_t)ya >> s) * P.mcus_x;
  const uint32_t o00 = ldg_slot_if(ok, slot + rowa + xas);
  const uint32_t ia = ((uint32_t)ya & mwm) << s, ja = (uint32_t)xa & mwm;
  if (FILTER == JT_FILTER_NEAREST) return __ldg(cache + (size_t)o00 * (kUnitBytes / 4) + (ia | ja));
  const uint32_t rowb = P.gid_base + ((uint32_t)yb >> s) * P.mcus_x;
  const bool sx = xbs != xas, sy = rowb != rowa;
  const uint32_t l10 = ldg_slot_if(ok && sx, slot + rowa + xbs);
  const uint32_t l01 = ldg_slot_if(ok && sy, slot + rowb + xas);
  const uint32_t l11 = ldg_slot_if(ok && sx && sy, slot + rowb + xbs);
  const uint32_t o10 = sx ? l10 : o00, o01 = sy ? l01 : o00;
  const uint32_t o11 = sx ? (sy ? l11 : o10) : o01;
  const uint32_t ib = ((uint32_t)yb & mwm) << s, jb = (uint32_t)xb & mwm;
  const uint32_t c00 = __ldg(cache + (size_t)o00 * (kUnitBytes / 4) + (ia | ja));
  const uint32_t c10 = __ldg(cache + (size_t)o10 * (kUnitBytes / 4) + (ia | jb));
  const uint32_t c01 = __ldg(cache + (size_t)o01 * (kUnitBytes / 4) + (ib | ja));
  const uint32_t c11 = __ldg(cache + (size_t)o11 * (kUnitBytes / 4) + (ib | jb));
  return blend_h(c00, c10, c01, c11, fx, fy);
}

// Taps of the clamped filter: along each axis a tap in another MCU than the nearest texel's
// moves onto the nearest texel's column or row (one MCU).
__device__ __forceinline__ void clamp_taps(uint32_t s, int nx, int ny, int& xa, int& xb, int& ya, int& yb) {
  const int mx = nx >> s, my = ny >> s;
  xa = (xa >> s) == mx ? xa : nx;
  xb = (xb >> s) == mx ? xb : nx;
  ya = (ya >> s) == my ? ya : ny;
  yb = (yb >> s) == my ? yb : ny;
}

// The general path of one pixel (any level, any coordinate; out of line).
template <int FILTER>
__device__ __noinline__ uint32_t colour_any(const uint32_t* slot, const uint32_t* cache, const PixL& P, float u,
                                            float v) {
  int xa, xb, ya, yb;
  float fx = 0.f, fy = 0.f;
  if (FILTER == JT_FILTER_NEAREST) {
    nearest_any(P, u, v, xa, ya);
    xb = xa;
    yb = ya;
  } else {
    taps_any(P, u, v, xa, xb, ya, yb, fx, fy);
    if (FILTER == JT_FILTER_BILINEAR_CLAMP) {
      int nx, ny;
      nearest_any(P, u, v, nx, ny);
      clamp_taps(P.shift, nx, ny, xa, xb, ya, yb);
    }
  }
  return shade<FILTER>(slot, cache, P, true, xa, xb, ya, yb, fx, fy);
}

// A lane owns pixel lane + 32 k (k < NPX) of each step of a row (32 NPX pixels), so a warp's
// texel gathers for one tap fall in the two or three tiles its 32 consecutive pixels cover
// (few L1 wavefronts per load), and the lane's NPX pixels are independent chains (level
// record, slot, texels) that overlap. The next step's G-buffer is loaded before the
// current one is shaded. The fast path has no data-dependent branch: the level record is
// loaded per pixel (an L1 hit), slots beyond the first tap's MCU are predicated loads, and
// pixels it cannot address (sides not powers of two, |u w| or |v h| >= 2^22) are redone on
// the general path. Warps whose pixels all lack a texture skip the arithmetic. Slots are in
// range by construction (the compaction and the cache update never write a slot whose tile
// would end past the cache), and the all-zero record of keys outside the table addresses
// unit 0, so no load needs a bound check.
template <int FILTER, bool MULTI, int NPX>
__global__ void __launch_bounds__(512, 2) k_colorize(const __grid_constant__ ColorizeArgs a) {
  const uint32_t* __restrict__ cache = reinterpret_cast<const uint32_t*>(a.cache);
  const uint32_t* __restrict__ slot = a.slot;
  const ViewSet& vs = a.views;
  bool missing = false;
  const int lx = threadIdx.x & 31;
  TileWalk<4 / NPX> it;
  it.start(vs);
  RowG<NPX> g;
  load_row(vs.v[MULTI ? it.vi : 0], it.x() + lx, it.y(), it.valid(vs), g);
#pragma unroll 1
  while (it.valid(vs)) {
    TileWalk<4 / NPX> nx = it;
    nx.advance(vs);
    RowG<NPX> ng;
    load_row(vs.v[MULTI ? nx.vi : 0], nx.x() + lx, nx.y(), nx.valid(vs), ng);
    uint32_t sel = 0, use = 0;
#pragma unroll
    for (int k = 0; k < NPX; ++k) {
      const uint32_t tex = g.tm[k] & 0xFFFFu;
      const bool sk = (uint32_t)k < g.n && (a.only_tex < 0 || (int)tex == a.only_tex);
      sel |= sk ? (1u << k) : 0u;
      use |= sk && tex != JT_EMPTY_TEXTURE ? (1u << k) : 0u;
    }
    uint32_t px[NPX];
#pragma unroll
    for (int k = 0; k < NPX; ++k) px[k] = 0xFF000000u;  // empty pixels
    if (__any_sync(0xFFFFFFFFu, use != 0)) {
      uint32_t slow = 0;
#pragma unroll
      for (int k = 0; k < NPX; ++k) {
        const PixL P = pix_level(a.tl, g.tm[k]);
        const bool ok = (use >> k & 1u) && (P.info & kPixJpeg);
        missing |= (use >> k & 1u) && !(P.info & kPixJpeg);
        int xa, xb, ya, yb;
        float fx = 0.f, fy = 0.f;
        bool fast;
        if (FILTER == JT_FILTER_NEAREST) {
          fast = nearest_fast(P, g.u[k], g.v[k], xa, ya);
          xb = xa;
          yb = ya;
        } else {
          fast = taps_fast(P, g.u[k], g.v[k], xa, xb, ya, yb, fx, fy);
          if (FILTER == JT_FILTER_BILINEAR_CLAMP) {
            int nxp, nyp;
            fast &= nearest_fast(P, g.u[k], g.v[k], nxp, nyp);
            clamp_taps(P.shift, nxp, nyp, xa, xb, ya, yb);
          }
        }
        const uint32_t c = shade<FILTER>(slot, cache, P, ok, xa, xb, ya, yb, fx, fy);
        px[k] = ok ? c : px[k];
        slow |= (ok && !fast) ? (1u << k) : 0u;
      }
      if (slow) {  // rare: redo those pixels on the general path
#pragma unroll
        for (int k = 0; k < NPX; ++k)
          if (slow & (1u << k)) px[k] = colour_any<FILTER>(slot, cache, pix_level(a.tl, g.tm[k]), g.u[k], g.v[k]);
      }
    }
    uint32_t* out = reinterpret_cast<uint32_t*>(vs.v[MULTI ? it.vi : 0].out) + g.p0;
#pragma unroll
    for (int k = 0; k < NPX; ++k)
      if (sel & (1u << k)) out[32 * k] = px[k];
    it = nx;
    g = ng;
  }
  if (missing) atomicOr(&a.state->err, JT_DEVERR_MISSING);
}

// ---------------------------------------------------------------------------------------
// Float chain (differentiable colourise, not in the paper): bilinear taps as above over the
// texels of the coefficient textures; weights (1-fx)(1-fy), fx(1-fy), (1-fx)fy, fx fy. Neither
// pass stores anything per texel: each pixel is bucketed under the needed MCUs its taps touch,
// and one warp per MCU transforms it once and serves its bucket (below): the forward adds the
// weighted texels into the pixels' values, the backward the pixels' weighted gradients into
// the MCU's.
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

// ---- Forward and backward passes over buckets of pixels per MCU ----
//
// F at a pixel is sum_k w_k colour(texel_k), each texel from f = A c A^T of its MCU; dL/dc of a
// coefficient MCU is A^T g A per data unit, g the MCU's texel gradients after colour^T and
// upsample^T, and those are the w dL/dF of the pixels whose taps fall in it. Both passes
// therefore invert the pixel -> MCU map rather than going through per-texel tiles:
//   k_float_buckets<count>  per pixel, +1 to the count of each distinct needed MCU among its
//                           four taps (the MCU's work position);
//   k_bucket_sums, k_bucket_offsets   exclusive offsets of the counts (two passes, the
//                           second also turns the counts back into zeroed fill cursors);
//   k_float_buckets<fill>   the same visits again, each writing a 32 B entry into the MCU's
//                           bucket: for each of the pixel's four taps the texel and weight when
//                           the tap falls in that MCU (weight 0 when it does not), and the
//                           pixel's index (forward) or its dL/dF after colour^T (backward:
//                           luma, Cb and Cr terms; the colour transform is per pixel);
//   k_float_gather_fwd      one warp per run of coefficient MCUs: a needed MCU is transformed
//                           once in shared memory and its bucket's pixels get their weighted
//                           texels added into their values (global atomics);
//   k_float_gather          one warp per run of coefficient MCUs (every MCU written once): a
//                           needed MCU's bucket terms are added into its 384 gradients in
//                           shared memory (luma per texel, chroma per 2x2 sample; shared
//                           atomics, upsample^T), then A^T g A; an MCU no pixel needs gets zeros.
// The sums' order (atomics) is the only non-determinism.

constexpr int kBucketCount = 0, kBucketGrad = 1, kBucketPixel = 2;

template <int MODE>
__global__ void k_float_buckets(const __grid_constant__ FloatArgs a) {
  constexpr bool FILL = MODE != kBucketCount;
  bool missing = false, over = false;
  for_each_quad(a.views, [&](const View& V, int y, int x) {
    float u[4], v[4];
    uint32_t t[4], m[4];
    const int n = load_px4(V, y, x, u, v, t, m);
    QuadLevels q;
    quad_levels(a.tl, n, t, m, -1, q);
    const uint32_t p0 = (uint32_t)y * (uint32_t)V.width + (uint32_t)x;
    for_quad_pixels(a.tl, q, [&](auto p2, const Lvl& L, int i) {
      const FloatTaps T = float_taps<decltype(p2)::value>(a, L, q.key[i], u[i], v[i], missing, over);
      if (!T.ok) return;
      float gy = 0.f, gcb = 0.f, gcr = 0.f;  // colour^T of the pixel's dL/dF
      if (MODE == kBucketGrad) {
        const float* gf = a.frame + 3 * (size_t)(p0 + (uint32_t)i);
        const float r = __ldg(gf), gg = __ldg(gf + 1), b = __ldg(gf + 2);
        gy = r + gg + b;
        gcb = kCb2B * b - kCb2G * gg;
        gcr = kCr2R * r - kCr2G * gg;
      }
      auto visit = [&](uint32_t tile) {
        if (FILL) {
          const uint32_t pos = a.bucket_off[tile] + atomicAdd(a.bucket_cnt + tile, 1u);
          if (pos < a.bucket_cap) {
            uint32_t texels = 0;
            float w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const bool in = (T.idx[k] >> 8) == tile;
              texels |= (in ? (T.idx[k] & 255u) : 0u) << (8 * k);
              w[k] = in ? T.w[k] : 0.f;
            }
            uint4* e = reinterpret_cast<uint4*>(a.bucket) + 2 * (size_t)pos;
            e[0] = MODE == kBucketGrad
                       ? make_uint4(__float_as_uint(gy), __float_as_uint(gcb), __float_as_uint(gcr), texels)
                       : make_uint4(p0 + (uint32_t)i, 0u, 0u, texels);
            e[1] = make_uint4(__float_as_uint(w[0]), __float_as_uint(w[1]), __float_as_uint(w[2]), __float_as_uint(w[3]));
          }
        } else {
          atomicAdd(a.bucket_cnt + tile, 1u);
        }
      };
      const uint32_t ta = T.idx[0] >> 8, tb = T.idx[1] >> 8, tc = T.idx[2] >> 8, td = T.idx[3] >> 8;
      visit(ta);
      if (tb != ta) visit(tb);
      if (tc != ta && tc != tb) visit(tc);
      if (td != ta && td != tb && td != tc) visit(td);
    });
  });
  if (!FILL && missing) atomicOr(&a.state->err, JT_DEVERR_MISSING);
  if (!FILL && over) atomicOr(&a.state->err, JT_DEVERR_CAPACITY);
}

__device__ __forceinline__ uint32_t needed_tiles(const FloatArgs& a) {
  return min(*reinterpret_cast<const volatile uint32_t*>(&a.state->count), a.tile_cap);
}

// Block-wide sum of one value per thread (256 threads).
__device__ __forceinline__ uint32_t block_sum256(uint32_t v, uint32_t* s_part) {
  v = __reduce_add_sync(0xFFFFFFFFu, v);
  if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = v;
  __syncthreads();
  uint32_t t = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) t += s_part[i];
  __syncthreads();
  return t;
}

// Counts [b * kBucketScan, (b + 1) * kBucketScan) of the n needed MCUs, four per thread.
__device__ __forceinline__ uint4 bucket_counts(const FloatArgs& a, uint32_t n, uint32_t first) {
  uint32_t c[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) c[k] = first + k < n ? a.bucket_cnt[first + k] : 0u;
  return make_uint4(c[0], c[1], c[2], c[3]);
}

__global__ void __launch_bounds__(256) k_bucket_sums(const __grid_constant__ FloatArgs a) {
  __shared__ uint32_t s_part[8];
  const uint32_t n = needed_tiles(a);
  const uint4 c = bucket_counts(a, n, blockIdx.x * kBucketScan + threadIdx.x * 4);
  const uint32_t t = block_sum256(c.x + c.y + c.z + c.w, s_part);
  if (threadIdx.x == 0) a.bucket_bsum[blockIdx.x] = t;
}

__global__ void __launch_bounds__(256) k_bucket_offsets(const __grid_constant__ FloatArgs a) {
  __shared__ uint32_t s_part[8], s_warp[8];
  const uint32_t n = needed_tiles(a);
  const uint32_t b = blockIdx.x, first = b * kBucketScan + threadIdx.x * 4;
  if (b * kBucketScan > n) return;  // past the last offset (index n)
  uint32_t pre = 0;  // sums of the blocks before this one
  for (uint32_t j = threadIdx.x; j < b; j += 256) pre += a.bucket_bsum[j];
  pre = block_sum256(pre, s_part);
  const uint4 c = bucket_counts(a, n, first);
  const uint32_t mine = c.x + c.y + c.z + c.w;
  // block-wide exclusive scan of the threads' sums
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = mine;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, inc, d);
    if (lane >= d) inc += o;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  uint32_t before = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) before += i < warp ? s_warp[i] : 0u;
  uint32_t off = pre + before + inc - mine;
  const uint32_t cc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t i = first + k;
    if (i <= n) a.bucket_off[i] = off;  // index n: the total
    if (i < n) a.bucket_cnt[i] = 0;      // the fill pass's cursor
    off += cc[k];
  }
}

// consecutive coefficient MCUs per warp task (lane l < kGatherChunk checks MCU l): with 8
// rather than 32 the 262,144 MCUs of sixteen 2048^2 coefficient textures make four times the
// tasks, so the grid's last wave is nearly full (their backward over a 1920x1080 plane: 0.308 ms
// with 8, 0.315 with 16, 0.364 with 32)
constexpr uint32_t kGatherChunk = 8;

// The weighted terms of bucket entry (c, wv) added into g (see k_float_gather).
__device__ __forceinline__ void gather_entry(float* g, const uint4& c, const uint4& wv) {
  const float gy = __uint_as_float(c.x), gcb = __uint_as_float(c.y), gcr = __uint_as_float(c.z);
  const float w[4] = {__uint_as_float(wv.x), __uint_as_float(wv.y), __uint_as_float(wv.z), __uint_as_float(wv.w)};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (w[k] == 0.f) continue;  // the tap falls in another MCU (or weighs nothing)
    const uint32_t t = (c.w >> (8 * k)) & 255u;
    const uint32_t tx = t & 15u, ty = t >> 4, s = (ty >> 1) * 8 + (tx >> 1);
    atomicAdd(g + ((ty >> 3) * 2 + (tx >> 3)) * 64 + (ty & 7) * 8 + (tx & 7), w[k] * gy);
    atomicAdd(g + 256 + s, w[k] * gcb);
    atomicAdd(g + 320 + s, w[k] * gcr);
  }
}

__device__ __forceinline__ void load_entry(const FloatArgs& a, uint32_t e, uint32_t e1, uint4& c, uint4& wv) {
  if (e < e1) {
    const uint4* ent = reinterpret_cast<const uint4*>(a.bucket) + 2 * (size_t)e;
    c = __ldg(ent);
    wv = __ldg(ent + 1);
  } else {
    c = make_uint4(0, 0, 0, 0);
    wv = make_uint4(0, 0, 0, 0);  // all weights zero: adds nothing
  }
}

__global__ void __launch_bounds__(kFloatWarps * 32) k_float_gather(const __grid_constant__ FloatArgs a) {
  __shared__ __align__(16) float buf[kFloatWarps][2][384];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* g = buf[warp][0];
  float* s1 = buf[warp][1];
  // the transforms: lane l owns, in data units d0, d0 + 2, d0 + 4, the four outputs at
  // columns ug .. ug + 3 of row r (pass 1: rows of g times A; pass 2: A^T times columns)
  const int ug = 4 * (lane & 1), r = (lane >> 1) & 7, d0 = lane >> 4;
  float A4[8][4], Ar[8];  // A[x][ug + j]; A[y][r]
#pragma unroll
  for (int x = 0; x < 8; ++x) {
#pragma unroll
    for (int j = 0; j < 4; ++j) A4[x][j] = a.basis[x * 8 + ug + j];
    Ar[x] = a.basis[x * 8 + r];
  }
  const uint32_t count = needed_tiles(a);
  const uint32_t nchunks = (a.coef_mcus + kGatherChunk - 1) / kGatherChunk;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  for (uint32_t ch = blockIdx.x * kFloatWarps + warp; ch < nchunks; ch += gridDim.x * kFloatWarps) {
    const uint32_t m0 = ch * kGatherChunk, nm = min(kGatherChunk, a.coef_mcus - m0);
    // lane l: is MCU m0 + l needed? Its work position is its slot when the work list holds
    // its gid there (slots of MCUs no pixel needs are stale)
    const uint32_t gid = a.coef_gid_base + m0 + (uint32_t)lane;
    uint32_t pl = 0, ob = 0, oe = 0;
    bool nd = false;
    if ((uint32_t)lane < nm) {
      pl = __ldg(a.slot + gid);
      nd = pl < count && __ldg(a.work + pl) == gid;
    }
    if (nd) {  // its bucket
      ob = __ldg(a.bucket_off + pl);
      oe = min(__ldg(a.bucket_off + pl + 1), a.bucket_cap);
    }
    const uint32_t need = __ballot_sync(0xFFFFFFFFu, nd);
    // MCUs no pixel needs: zeros
#pragma unroll 1
    for (uint32_t rest = ((nm == 32 ? 0xFFFFFFFFu : (1u << nm) - 1u)) & ~need; rest; rest &= rest - 1) {
      float4* dst = reinterpret_cast<float4*>(a.grad_coef + (size_t)(m0 + __ffs(rest) - 1) * 384);
#pragma unroll
      for (int i = 0; i < 3; ++i) dst[lane + 32 * i] = z;
    }
    // needed MCUs in order; the first 32 entries of the next one are loaded while the
    // current one is accumulated and transformed
    uint32_t cur = need;
    uint4 c, wv;
    if (cur) {
      const int i0 = __ffs(cur) - 1;
      load_entry(a, __shfl_sync(0xFFFFFFFFu, ob, i0) + lane, __shfl_sync(0xFFFFFFFFu, oe, i0), c, wv);
    }
#pragma unroll 1
    while (cur) {
      const int i = __ffs(cur) - 1;
      cur &= cur - 1;
      const uint32_t e0 = __shfl_sync(0xFFFFFFFFu, ob, i), e1 = __shfl_sync(0xFFFFFFFFu, oe, i);
      uint4 cn = make_uint4(0, 0, 0, 0), wn = make_uint4(0, 0, 0, 0);
      if (cur) {
        const int j = __ffs(cur) - 1;
        load_entry(a, __shfl_sync(0xFFFFFFFFu, ob, j) + lane, __shfl_sync(0xFFFFFFFFu, oe, j), cn, wn);
      }
      // the bucket's weighted terms, accumulated in g: luma texel (tx, ty) of data unit
      // (ty / 8) * 2 + tx / 8 at 64 d + (ty % 8) * 8 + tx % 8; chroma sample (tx / 2, ty / 2)
      // at 256 + s (Cb) and 320 + s (Cr), the sum over its four texels (upsample^T)
#pragma unroll
      for (int k = 0; k < 12; ++k) g[lane + 32 * k] = 0.f;
      __syncwarp();
      gather_entry(g, c, wv);
#pragma unroll 1
      for (uint32_t e = e0 + 32 + lane; e < e1; e += 32) {  // beyond the first 32 entries
        uint4 cx, wx;
        load_entry(a, e, e1, cx, wx);
        gather_entry(g, cx, wx);
      }
      __syncwarp();
      // pass 1: s1[d][r][u] = sum_x g[d][r][x] A[x][u], u = ug .. ug + 3
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int o = (d0 + 2 * k) * 64 + r * 8;
        const float4 ga = *reinterpret_cast<const float4*>(g + o), gb = *reinterpret_cast<const float4*>(g + o + 4);
        const float gx[8] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z, gb.w};
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int x = 0; x < 8; ++x)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) acc[jj] = fmaf(gx[x], A4[x][jj], acc[jj]);
        *reinterpret_cast<float4*>(s1 + o + ug) = make_float4(acc[0], acc[1], acc[2], acc[3]);
      }
      __syncwarp();
      // pass 2: grad[d][r][u] = sum_y A[y][r] s1[d][y][u], u = ug .. ug + 3
      float* out = a.grad_coef + (size_t)(m0 + (uint32_t)i) * 384;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int d = d0 + 2 * k;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int y = 0; y < 8; ++y) {
          const float4 sv = *reinterpret_cast<const float4*>(s1 + d * 64 + y * 8 + ug);
          acc[0] = fmaf(Ar[y], sv.x, acc[0]);
          acc[1] = fmaf(Ar[y], sv.y, acc[1]);
          acc[2] = fmaf(Ar[y], sv.z, acc[2]);
          acc[3] = fmaf(Ar[y], sv.w, acc[3]);
        }
        *reinterpret_cast<float4*>(out + d * 64 + r * 8 + ug) = make_float4(acc[0], acc[1], acc[2], acc[3]);
      }
      __syncwarp();
      c = cn;
      wv = wn;
    }
  }
}

// Forward gather: one warp per run of kGatherChunk coefficient MCUs; each needed MCU is
// transformed once in shared memory (f = A c A^T per data unit, two passes) and each pixel of
// its bucket gets, added into its frame value (zeroed before), the sum over its taps in this
// MCU of w times the texel's colour (computed from f on demand: Y = f + 128, chroma of the
// 2x2 sample, the JFIF matrix; the same fp32 operations as the per-texel form). A pixel whose
// taps all lie in one MCU gets exactly the fused sum in tap order.
__global__ void __launch_bounds__(kFloatWarps * 32) k_float_gather_fwd(const __grid_constant__ FloatArgs a) {
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
  const uint32_t count = needed_tiles(a);
  const uint32_t nchunks = (a.coef_mcus + kGatherChunk - 1) / kGatherChunk;
  for (uint32_t ch = blockIdx.x * kFloatWarps + warp; ch < nchunks; ch += gridDim.x * kFloatWarps) {
    const uint32_t m0 = ch * kGatherChunk, nm = min(kGatherChunk, a.coef_mcus - m0);
    const uint32_t gid = a.coef_gid_base + m0 + (uint32_t)lane;
    uint32_t pl = 0, ob = 0, oe = 0;
    bool nd = false;
    if ((uint32_t)lane < nm) {
      pl = __ldg(a.slot + gid);
      nd = pl < count && __ldg(a.work + pl) == gid;
    }
    if (nd) {
      ob = __ldg(a.bucket_off + pl);
      oe = min(__ldg(a.bucket_off + pl + 1), a.bucket_cap);
    }
    // needed MCUs in order; the next one's coefficients are loaded while the current one is
    // transformed and served
    uint32_t cur = __ballot_sync(0xFFFFFFFFu, nd);
    float4 cf[3];
    if (cur) {
      const float4* src = reinterpret_cast<const float4*>(a.coef + (size_t)(m0 + __ffs(cur) - 1) * 384);
#pragma unroll
      for (int k = 0; k < 3; ++k) cf[k] = __ldg(src + lane + 32 * k);
    }
#pragma unroll 1
    for (; cur; cur &= cur - 1) {
      const int i = __ffs(cur) - 1;
      const uint32_t e0 = __shfl_sync(0xFFFFFFFFu, ob, i), e1 = __shfl_sync(0xFFFFFFFFu, oe, i);
#pragma unroll
      for (int k = 0; k < 3; ++k) reinterpret_cast<float4*>(c)[lane + 32 * k] = cf[k];
      const uint32_t rest = cur & (cur - 1);
      if (rest) {
        const float4* src = reinterpret_cast<const float4*>(a.coef + (size_t)(m0 + __ffs(rest) - 1) * 384);
#pragma unroll
        for (int k = 0; k < 3; ++k) cf[k] = __ldg(src + lane + 32 * k);
      }
      __syncwarp();
      // pass 1: t[d][v][x] = sum_u A[x][u] c[d][v][u]
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const int o = lane + 32 * k;
        const float* row = c + (o & ~7);
        float sum = 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) sum = fmaf(Ax[u], row[u], sum);
        t[o] = sum;
      }
      __syncwarp();
      // pass 2: f[d][y][x] = sum_v A[y][v] t[d][v][x]  (y = y0 for even k, y0 + 4 for odd k)
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const int o = lane + 32 * k;
        const float* col = t + (o & ~63) + x;
        float sum = 0.f;
#pragma unroll
        for (int v = 0; v < 8; ++v) sum = fmaf((k & 1) ? Ay1[v] : Ay0[v], col[v * 8], sum);
        c[o] = sum;
      }
      __syncwarp();
#pragma unroll 1
      for (uint32_t e = e0 + lane; e < e1; e += 32) {
        const uint4* ent = reinterpret_cast<const uint4*>(a.bucket) + 2 * (size_t)e;
        const uint4 ce = __ldg(ent), wv = __ldg(ent + 1);
        const float w[4] = {__uint_as_float(wv.x), __uint_as_float(wv.y), __uint_as_float(wv.z), __uint_as_float(wv.w)};
        float r = 0.f, gg = 0.f, b = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (w[k] == 0.f) continue;  // the tap falls in another MCU (or weighs nothing)
          const uint32_t tq = (ce.w >> (8 * k)) & 255u, tx = tq & 15u, ty = tq >> 4;
          const float Y = c[((ty >> 3) * 2 + (tx >> 3)) * 64 + (ty & 7) * 8 + (tx & 7)] + 128.f;
          const uint32_t ci = (ty >> 1) * 8 + (tx >> 1);
          const float cb = c[256 + ci], cr = c[320 + ci];
          r = fmaf(w[k], Y + kCr2R * cr, r);
          gg = fmaf(w[k], Y - kCb2G * cb - kCr2G * cr, gg);
          b = fmaf(w[k], Y + kCb2B * cb, b);
        }
        float* out = a.frame + 3 * (size_t)ce.x;
        atomicAdd(out, r);
        atomicAdd(out + 1, gg);
        atomicAdd(out + 2, b);
      }
      __syncwarp();
    }
  }
}

}  // namespace

// The forward and backward passes after the needed set and its compaction; bucket_cnt must
// be zero on entry (and the frame, for the forward).
void launch_float_forward(const FloatArgs& a, int threads, int pixel_grid, int mcu_grid, cudaStream_t s) {
  const int sblocks = (int)((a.tile_cap + 1 + kBucketScan - 1) / kBucketScan);
  k_float_buckets<kBucketCount><<<pixel_grid, threads, 0, s>>>(a);
  k_bucket_sums<<<sblocks, 256, 0, s>>>(a);
  k_bucket_offsets<<<sblocks, 256, 0, s>>>(a);
  k_float_buckets<kBucketPixel><<<pixel_grid, threads, 0, s>>>(a);
  k_float_gather_fwd<<<mcu_grid, kFloatWarps * 32, 0, s>>>(a);
}

void launch_float_backward(const FloatArgs& a, int threads, int pixel_grid, int mcu_grid, cudaStream_t s) {
  const int sblocks = (int)((a.tile_cap + 1 + kBucketScan - 1) / kBucketScan);
  k_float_buckets<kBucketCount><<<pixel_grid, threads, 0, s>>>(a);
  k_bucket_sums<<<sblocks, 256, 0, s>>>(a);
  k_bucket_offsets<<<sblocks, 256, 0, s>>>(a);
  k_float_buckets<kBucketGrad><<<pixel_grid, threads, 0, s>>>(a);
  k_float_gather<<<mcu_grid, kFloatWarps * 32, 0, s>>>(a);
}

void launch_mark(const MarkArgs& a, int threads, int grid, cudaStream_t s) {
  // the clamped filter reads only the nearest texel's MCU
  const bool nearest = a.filter == JT_FILTER_NEAREST || a.filter == JT_FILTER_BILINEAR_CLAMP;
  if (a.views.n > 1) {
    if (nearest)
      k_mark<JT_FILTER_NEAREST, true><<<grid, threads, 0, s>>>(a);
    else
      k_mark<JT_FILTER_BILINEAR, true><<<grid, threads, 0, s>>>(a);
  } else {
    if (nearest)
      k_mark<JT_FILTER_NEAREST, false><<<grid, threads, 0, s>>>(a);
    else
      k_mark<JT_FILTER_BILINEAR, false><<<grid, threads, 0, s>>>(a);
  }
}

// pixels per lane per step: two (60 registers, 32 warps per SM) measured faster than four
// (74 registers) on the 4K frame
constexpr int kColorizePx = 2;

template <bool MULTI>
void launch_colorize_views(const ColorizeArgs& a, int threads, int grid, cudaStream_t s) {
  constexpr int N = kColorizePx;
  if (a.filter == JT_FILTER_NEAREST)
    k_colorize<JT_FILTER_NEAREST, MULTI, N><<<grid, threads, 0, s>>>(a);
  else if (a.filter == JT_FILTER_BILINEAR_CLAMP)
    k_colorize<JT_FILTER_BILINEAR_CLAMP, MULTI, N><<<grid, threads, 0, s>>>(a);
  else
    k_colorize<JT_FILTER_BILINEAR, MULTI, N><<<grid, threads, 0, s>>>(a);
}

void launch_colorize(const ColorizeArgs& a, int threads, int grid, cudaStream_t s) {
  if (a.views.n > 1)
    launch_colorize_views<true>(a, threads, grid, s);
  else
    launch_colorize_views<false>(a, threads, grid, s);
}

}  // namespace jt
