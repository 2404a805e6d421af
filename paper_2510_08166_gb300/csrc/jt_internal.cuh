// Internal device-side data model of the texture path (shared by the kernels and the
// host implementation of the C ABI in jt_api.cu).
//
// HBM layout
//   descs      DevDesc[ndesc]        one per uploaded (texture, level), sorted by gid_base
//   desc_map   int32[ntex * 16]      (tex_id, level) -> desc index, -1 when absent
//   streams    per level: uint32 words of the unstuffed entropy stream + >= 64 zero bytes
//   index      per level: packed 10-byte {bit_offset, dc_pred[3]} entries
//   huff       HuffSet[nh]           decode LUTs, deduplicated by content
//   quant      uint16[nq][2][64]     quantisation tables in zig-zag order
//   flags      uint8[ngid]           per-frame marks: cache units of the MCU (4, 1) or 0
//   slot       uint32[ngid]          cache-unit offset of each needed gid
//   work       uint32[ngid]          work list (needed gids, ascending)
//   cache      uint8[cap_units*256]  RGBA8 tiles; a 4:2:0 MCU = 4 units, 4:4:4 = 1 unit
//   state      FrameState            counts, work counter, error word
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "jt.h"

namespace jt {

// ---- programmatic dependent launch ----
// The frame's compaction (or cache update) and decode are launched with programmatic stream
// serialisation (colourise is not: its CTAs, launched early, would wait on the SMs the decode
// is using, and the 4K frame measured 0.181 ms with it against 0.176 ms without):
// a kernel may start while the one before it in the stream is still running, and waits on
// the device (pdl_wait) before it reads or writes anything an earlier kernel of the stream
// produces or consumes. Each kernel lets its dependents launch as soon as it starts
// (pdl_launch_dependents); a dependent's CTAs are only scheduled once every CTA of the
// running grid has started, so they never hold resources that grid still needs. Without
// the attribute (or after a non-kernel operation) both instructions are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

constexpr int kLutBits = 10;                 // first-level Huffman LUT: next 10 bits
constexpr int kLutSize = 1 << kLutBits;
constexpr int kLut2Size = 1024;              // second-level LUT for longer codes
constexpr int kStreamPadBytes = 64;          // zero padding after each entropy stream
constexpr uint32_t kUnitBytes = 256;         // cache unit
constexpr int kSampling420 = 0, kSampling444 = 1, kSamplingCoef = 2;

// Decode tables of one Huffman spec (T.81 Annex C canonical codes). A symbol entry is 16
// bits: code length l (bits 0..4), value-bit count s (bits 5..8), run r (bits 9..14):
//   AC value  (r, s)   -> store at k + r, advance k by r + 1
//   ZRL       (15, 0)  -> advance 16 (the skipped slots are zero)
//   EOB       (63, 0)  -> advance 64 (store a zero at slot 63, which is zero already)
//   DC        (0, s)   -> difference, advance 1
// The s value bits follow the code in the stream; the decoder cuts them from its 32-bit
// window itself (T.81 EXTEND), so an entry depends on the code alone. 0 = no entry.
//   lut[i]   entry of the code that starts the next kLutBits bits i (codes up to kLutBits)
//   lut2[j]  entry of the longer code whose 16-bit left-aligned prefix is first16 + j: in
//            canonical order the longer codes are the numerically largest, so they occupy
//            the top n2 of the 65536 16-bit prefixes (n2 <= kLut2Size, else 0)
// The decoder reads both entries for every symbol (the two reads are independent), so a
// long code costs no branch. Codes without an entry (invalid codes, long codes of tables
// whose range exceeds kLut2Size) and symbols invalid for the table's class (DC category >
// 11, AC size > 10, AC size 0 with a run other than 0 or 15) go to the MAXCODE walk of
// T.81 F.2.2.3, which decodes or rejects them.
__host__ __device__ constexpr uint16_t huff_entry(uint32_t l, uint32_t s, uint32_t r) {
  return (uint16_t)(l | (s << 5) | (r << 9));
}
constexpr uint32_t kRunEob = 63;
struct HuffTable {
  uint16_t lut[kLutSize];
  uint16_t lut2[kLut2Size];
  uint32_t first16;     // 16-bit left-aligned value of the first code longer than kLutBits
  uint32_t n2;          // entries of lut2 in use (0: no longer codes, or too many)
  int32_t maxcode[17];  // -1 when no code of length l
  int32_t valoff[17];
  uint8_t vals[256];
};

// Four tables: DC luma, AC luma, DC chroma, AC chroma.
struct HuffSet {
  HuffTable t[4];
};

struct DevDesc {
  const uint32_t* stream;      // big-endian words (word i = bytes 4i..4i+3)
  // standard form: packed 10-byte entries, read as 5 halfwords. Compact form: the side
  // table [abs uint32 x G][rel uint16 x 8G][DC records uint32 x (ceil(36 n / 32) + 1)],
  // G = ceil(n / 9)
  const uint16_t* index;
  uint32_t gid_base;
  uint32_t nmcu;
  uint32_t nwords;             // readable words including padding
  uint32_t nbits;              // coded bits
  uint16_t width, height;
  uint16_t mcus_x, mcus_y;
  uint8_t sampling;            // kSampling420 / kSampling444 / kSamplingCoef
  uint8_t units;               // cache units per MCU: 4 or 1
  uint8_t hset, qset;
  uint8_t compact;             // 1: the compact form (byte-aligned MCUs, stored DCs)
  uint8_t reduce;              // r > 0: tiles at 1/2^r from the lowest N x N frequencies, N = 8 >> r
  uint8_t pad0[2];
  const uint16_t* du_index;    // optional data-unit starts [mcu][ndu - 1] (bits from the MCU start)
  uint64_t pad1;
};
static_assert(sizeof(DevDesc) == 64, "descriptor layout");

struct FrameState {
  uint32_t count;        // needed MCUs after the last compaction
  uint32_t units;        // cache units they occupy
  uint32_t decode_next;  // next work item for the persistent decoder
  uint32_t err;          // JT_DEVERR_* bits
  uint32_t spare;        // unused
  uint32_t pad[3];
};

// Screen passes walk each view in tiles of kTileW x kTileH pixels (one CTA per tile at a
// time, one warp per 128-pixel row segment), so a CTA's pixels share MCUs.
constexpr int kTileW = 128, kTileH = 32;

// One view of a (possibly batched) frame, passed by value in the kernel parameters.
struct View {
  const float4* uv;      // two pixels per float4
  const uint16_t* tex;
  const uint8_t* mip;
  uint4* out;            // four RGBA8 pixels per uint4
  uint32_t npx;
  uint32_t quad_begin;   // prefix sum of ceil(npx/4) over earlier views
  int32_t width, height;
  uint32_t tiles_x;      // ceil(width / kTileW)
  uint32_t tile_begin;   // prefix sum of tile counts over earlier views
};

struct ViewSet {
  View v[JT_MAX_VIEWS];
  int n;
  uint32_t total_quads;
  uint32_t total_tiles;
};

// Per-(texture, level) record for the screen passes, indexed directly by
// tex_id * JT_MAX_LEVELS + level; 16 bytes, one vector load. w == 0 marks a missing level.
//   x: gid_base
//   y: width (16) | height (16)
//   z: mcus_x (16) | mcu shift (4: 4 at 4:2:0, 3 at 4:4:4) | units (4) | sampling (4) |
//      width is a power of two (1) | height is a power of two (1)
//   w: unused
struct LevelRec {
  uint32_t gid_base;
  uint32_t wh;
  uint32_t info;
  uint32_t pad;
};
__host__ __device__ inline uint32_t level_info(uint32_t mcus_x, uint32_t shift, uint32_t units, uint32_t sampling,
                                               bool wpow2, bool hpow2) {
  return (mcus_x & 0xFFFF) | (shift << 16) | (units << 20) | (sampling << 24) | ((wpow2 ? 1u : 0u) << 28) |
         ((hpow2 ? 1u : 0u) << 29);
}

// The screen passes' record of one (texture, level): 32 bytes (two vector loads that hit
// L1, since a warp's pixels mostly share a level), every field in the form the texel
// addressing uses, so no per-pixel branch or decoding is needed. Indexed by
// tex * JT_MAX_LEVELS + level; record map_ntex * JT_MAX_LEVELS is all zero, the record of
// every key outside the table (empty pixels, unknown textures or levels).
struct PixRec {
  uint32_t gid_base;
  float wf, hf;     // sides as floats
  uint32_t masks;   // (w - 1) | (h - 1) << 16: floor-mod masks of power-of-two sides
  uint32_t mcus_x;
  uint32_t shift;   // log2 of the MCU side in texels
  uint32_t info;    // units | kPixJpeg | kPixCoef | kPixPow2
  uint32_t wh;      // w | h << 16
};
static_assert(sizeof(PixRec) == 32, "screen-pass record layout");
constexpr uint32_t kPixJpeg = 1u << 16;  // an uploaded JPEG level (colourise, mark)
constexpr uint32_t kPixCoef = 1u << 17;  // a coefficient level (mark of the float chain)
constexpr uint32_t kPixPow2 = 1u << 18;  // both sides are powers of two

struct TexLookup {
  const DevDesc* descs;
  const int32_t* desc_map;
  const uint4* levels;  // LevelRec per (tex, level), same indexing as desc_map
  const uint4* pix;     // PixRec per (tex, level) as two uint4, then the all-zero record
  uint32_t map_ntex;
  uint32_t all_p2;      // every level has power-of-two sides
};

// ---- launchers (defined in the kernel translation units) ----
struct MarkArgs {
  ViewSet views;
  TexLookup tl;
  uint8_t* flags;
  FrameState* state;
  int filter;
  int only_tex;   // -1: all textures; otherwise only pixels with this texture id
  int coef_mode;  // 0: JPEG levels only; 1: coefficient textures only
};
void launch_mark(const MarkArgs& a, int threads, int grid, cudaStream_t s);

struct ScanArgs {
  uint8_t* flags;        // flags of gids [gid_lo, gid_lo + n)
  uint32_t gid_lo;
  uint32_t n;
  uint32_t* slot;        // indexed by gid
  uint32_t* work;
  uint32_t work_cap;
  uint64_t* tile_status; // one word per tile: its (count << 32 | units)
  FrameState* state;
  uint32_t cap_units;
};
constexpr int kScanThreads = 256;
constexpr int kScanPerThread = 16;  // one 16-byte load
constexpr int kScanTile = kScanThreads * kScanPerThread;  // 4096 flags
void launch_scan(const ScanArgs& a, cudaStream_t s);  // two launches; tile_status: one word per tile

// Cross-frame block cache (Sec. 4.1, Sec. 4.5): a residency bitmap over the gids; a resident
// gid's slot (4 x its block) is the one the previous frame gave it; free blocks in a ring,
// positions [head, head + free_count) modulo nblocks. A block is 4 cache units. Every counter
// but head, free_count, visible and evicted is zero between frames.
struct CacheState {
  uint32_t head;         // ring position of the first free block
  uint32_t free_count;   // free blocks
  uint32_t taken;        // misses of the current update (blocks asked for)
  uint32_t spare;        // (unused)
  uint32_t evict_n;      // blocks evicted by the current update
  uint32_t visible_acc;  // MCUs the current update has seen needed
  uint32_t done;         // CTAs of the current update that have finished
  uint32_t visible;      // MCUs the last frame needed
  uint32_t evicted;      // blocks evicted since the counter was last cleared
};
struct CacheArgs {
  uint8_t* flags;  // flags[gid], cleared by the update
  uint32_t n;      // gids
  uint16_t* resbits;    // residency bitmap, 16 gids per word ...
  uint32_t* resbits32;  // ... the same memory as 32-bit words (a whole number of them)
  uint32_t* ring;       // [nblocks] free blocks
  uint32_t* deferred;   // [nblocks] misses waiting for a block evicted by the same update
  uint32_t nblocks;
  uint32_t* slot;
  uint32_t* work;
  uint32_t work_cap;
  FrameState* state;
  CacheState* cs;
};
constexpr int kCacheThreads = 256;
void launch_cache_update(const CacheArgs& a, int max_grid, cudaStream_t s);  // one launch

// Scene rasteriser (geometry-pass stand-in): one quad, laid out as jt_scene_quad.
struct SceneQuad {
  float cx[4], cy[4], ex[4], ey[4], h[9], rep, cs, sn, ou, ov;
  int32_t tex, x0, y0, x1, y1;
};
static_assert(sizeof(SceneQuad) == 140, "scene quad layout");
constexpr int kMaxSceneQuads = 4096;
struct RasterArgs {
  int32_t width, height;
  float cam[3], rot[9];
  float ax, ay, tan_x, tan_y, max_t, kx, ky, shift;
  uint64_t cell_seed;
  int32_t ntex, use_mips, nquads;
  const int32_t* tex_w;       // device copies
  const int32_t* tex_h;
  const int32_t* tex_levels;
  const SceneQuad* quads;
  float2* uv;
  uint16_t* tex;
  uint8_t* mip;
};
void launch_raster(const RasterArgs& a, cudaStream_t s);

struct DecodeArgs {
  const DevDesc* descs;
  uint32_t ndesc;
  const uint32_t* desc_of_gid;  // descriptor index of each gid
  int mcus_per_warp;      // M, the buffer width: 4, 8, 16 or 32 (batches may be smaller)
  int unit_mode;          // some level has data-unit starts: the kernel that decodes them in parallel
  int short_lists;        // the kernel that decodes short lists MCU by MCU with whole warps
  const HuffSet* huff;    // set 0 is staged in shared memory
  const uint16_t* quant;  // [nq][2][64] zig-zag order
  const uint32_t* work;
  uint32_t work_cap;
  const uint32_t* slot;
  uint8_t* cache;
  uint32_t cap_units;
  FrameState* state;
};
size_t decode_smem_bytes(int warps, int mcus_per_warp);
void launch_decode(const DecodeArgs& a, int warps, int grid, cudaStream_t s);
int decode_max_ctas_per_sm(int warps, int mcus_per_warp);

struct ColorizeArgs {
  ViewSet views;
  TexLookup tl;
  const uint32_t* slot;
  const uint8_t* cache;
  uint32_t cap_units;
  FrameState* state;
  int filter;
  int only_tex;
};
void launch_colorize(const ColorizeArgs& a, int threads, int grid, cudaStream_t s);

// Float chain (differentiable colourise; not in the paper). Coefficient textures are
// 4:2:0 level-0 textures whose MCUs are marked with 1 unit each, so after the compaction
// slot[gid] is the MCU's position in the work list and the index of its float tile.
struct FloatArgs {
  ViewSet views;          // one view
  TexLookup tl;
  const uint32_t* slot;   // gid -> work position = float tile index
  const uint32_t* work;
  const float* coef;      // [T][my][mx][6][64], natural order k = v*8+u
  uint32_t coef_gid_base; // gid of coefficient texture 0, MCU 0
  uint32_t coef_mcus;     // MCUs of all coefficient textures
  uint32_t tile_cap;      // needed coefficient MCUs a pass can serve (more: JT_DEVERR_CAPACITY)
  float* frame;           // [npx][3]: forward output (zero on entry), or the backward's dL/dF
  float* grad_coef;       // [T][my][mx][6][64]: backward output
  FrameState* state;
  // the view's pixels bucketed under the needed MCUs (work positions) their taps touch
  uint32_t* bucket_cnt;   // [tile_cap + 1] per-MCU counts, then fill cursors; zero on entry
  uint32_t* bucket_off;   // [tile_cap + 1] exclusive offsets into bucket
  uint32_t* bucket_bsum;  // [ceil((tile_cap + 1) / kBucketScan)] per-block sums of the counts
  uint32_t* bucket;       // [bucket_cap][8]: the pixel's index (forward) or its colour^T terms
                          // (3 floats, backward), its taps' texels (4 bytes), their weights
                          // (4 floats, 0 for a tap in another MCU)
  uint32_t bucket_cap;    // entries, >= 4 pixels of the view (a pixel's taps touch at most 4 MCUs)
  float basis[64];        // A[x][u] = C(u)/2 cos((2x+1)u pi/16), C(0) = 1/sqrt(2); x*8+u
};
// JFIF colour of the float chain: R = Y + kCr2R Cr, G = Y - kCb2G Cb - kCr2G Cr, B = Y + kCb2B Cb
constexpr float kCr2R = 1.402f, kCb2G = 0.344136f, kCr2G = 0.714136f, kCb2B = 1.772f;
constexpr int kFloatWarps = 8;     // warps per CTA of the per-MCU float kernels
constexpr int kBucketScan = 1024;  // counts per CTA of the bucket-offset scan (256 threads x 4)
// count pass, offsets, fill pass, then the per-MCU gather (forward: weighted texels into the
// pixels; backward: the adjoint into the coefficients)
void launch_float_forward(const FloatArgs& a, int threads, int pixel_grid, int mcu_grid, cudaStream_t s);
void launch_float_backward(const FloatArgs& a, int threads, int pixel_grid, int mcu_grid, cudaStream_t s);

// The integer IDCT constants the decode kernel is compiled with, for the host-side check
// against round(8192 cos(k pi / 16)), k = 1..7.
void idct_constants(int out[8]);

}  // namespace jt
