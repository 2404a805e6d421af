/*
 * jt.h — C ABI of the GB300 variable-rate (JPEG) texture path.
 *
 * Textures stay in GPU memory as baseline-JPEG entropy streams plus a per-MCU index.
 * Each frame runs against a deferred G-buffer (uv, texture id, mip level per pixel):
 *   jt_mark      — flag the MCUs (JPEG blocks) the pixels touch           (paper Sec. 4.2)
 *   jt_decode    — compact the flags into a work list, then Huffman-decode, dequantise,
 *                  IDCT, upsample chroma and convert to RGB into the block cache
 *                                                                        (Sec. 4.3, Sec. 5.2)
 *   jt_colorize  — look up each pixel's texel(s) in the block cache      (Sec. 4.4)
 * Textures, levels and the cache key follow Sec. 4.6; the index follows Sec. 5.1/5.3.
 *
 * Conventions
 *  - All functions return a jt_status. On failure jt_last_error() describes the cause.
 *  - "device" pointers are CUDA device (or managed) memory on the context's device.
 *    "host" pointers are ordinary host memory. Nothing is retained past the call unless
 *    stated; work enqueued on a stream reads caller buffers until that stream reaches it.
 *  - A jt_stream is a cudaStream_t (NULL = the legacy default stream).
 *  - A context is not thread-safe; calls on one context must be serialised by the caller
 *    and its frames must not overlap on different streams.
 *  - Device-side problems (a corrupt stream, a capacity overflow, a pixel naming a level
 *    that was never uploaded) never trap: kernels finish with bounded loops and set bits
 *    in a device error word. jt_get_stats() synchronises, reads and clears that word and
 *    returns the matching status.
 */
#ifndef JT_H
#define JT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  JT_OK = 0,
  JT_ERR_INVALID_ARG = 1,    /* bad argument; nothing was enqueued */
  JT_ERR_CUDA = 2,           /* a CUDA runtime call failed (no device, launch failure) */
  JT_ERR_OOM = 3,            /* device allocation failed */
  JT_ERR_CORRUPT_STREAM = 4, /* an MCU's bits are not a valid baseline coding */
  JT_ERR_CAPACITY = 5,       /* needed blocks exceed the block cache */
  JT_ERR_UNSUPPORTED = 6,    /* e.g. a pixel names a (texture, level) never uploaded */
  JT_ERR_STATE = 7           /* call out of order (e.g. jt_decode without jt_mark) */
} jt_status;

/* Bits of jt_stats.error_bits (the device error word). */
#define JT_DEVERR_CORRUPT 0x1u     /* invalid code, category or run, or bits past the stream */
#define JT_DEVERR_CAPACITY 0x2u    /* needed cache units > capacity; extra tiles not written */
#define JT_DEVERR_MISSING 0x4u     /* a pixel names a (texture, level) that does not exist */
#define JT_DEVERR_TIMEOUT 0x8u     /* a bounded wait gave up (reserved: no kernel of this
                                      library waits on another CTA or launch) */

/* Texture filters. BILINEAR_CLAMP (Sec. 4.4, the linear-interpolation mode timed in
 * Sec. 6.2): the bilinear taps, except that along each axis a tap lying in another MCU than
 * the nearest texel is moved onto the nearest texel's column or row, so one MCU serves all
 * four fetches and the mark pass flags only the nearest texel's MCU. */
#define JT_FILTER_NEAREST 0
#define JT_FILTER_BILINEAR 1
#define JT_FILTER_BILINEAR_CLAMP 2
#define JT_MAX_VIEWS 16
#define JT_MAX_LEVELS 16
#define JT_EMPTY_TEXTURE 0xFFFFu

typedef struct jt_ctx jt_ctx;
typedef struct jt_graph jt_graph;
typedef void* jt_stream;

/* One entry of the random-access index (Sec. 5.1, Sec. 5.3): the MCU's first bit in the
 * unstuffed entropy stream and the DC value each component (Y, Cb, Cr) had just before
 * this MCU. Packed, 10 bytes. */
#pragma pack(push, 2)
typedef struct {
  uint32_t bit_offset;
  int16_t dc_pred[3];
} jt_block_index;
#pragma pack(pop)

/* A Huffman table specification as in a JPEG DHT segment (T.81 B.2.4.2): bits[i] = number
 * of codes of length i+1, vals = symbols in code order (sum(bits) <= 256). */
typedef struct {
  uint8_t bits[16];
  uint8_t vals[256];
} jt_huff_spec;

/* Deferred G-buffer (Sec. 4 "Geometry Pass"), structure of arrays, caller-owned device
 * memory, row-major [height][width]:
 *   uv     float32 pairs (u, v); repeat wrap; 16-byte aligned
 *   tex_id uint16, JT_EMPTY_TEXTURE for pixels without texture;  8-byte aligned
 *   mip    uint8 mip level;                                       4-byte aligned
 * The passes only read it; jt_raster_scene writes it. */
typedef struct {
  const float* uv;
  const uint16_t* tex_id;
  const uint8_t* mip;
  int32_t width;
  int32_t height;
} jt_gbuffer;

/* One view of a batched frame: its G-buffer and its RGBA8 output (device, 16-byte
 * aligned, [height][width][4]). */
typedef struct {
  jt_gbuffer g;
  uint8_t* out_rgba;
} jt_view;

typedef struct {
  uint64_t needed_blocks;   /* MCUs in the last compaction's work list (decoded by the frame) */
  uint64_t cache_units;     /* 256-byte block-cache units those MCUs occupy */
  uint64_t capacity_units;  /* block-cache capacity in 256-byte units */
  uint64_t total_blocks;    /* MCUs over all uploaded levels (the key space) */
  uint32_t levels;          /* uploaded (texture, level) pairs */
  uint32_t error_bits;      /* JT_DEVERR_* bits seen since the last jt_get_stats */
  uint64_t visible_blocks;  /* MCUs the last frame needed (= needed_blocks without the block cache) */
  uint64_t resident_blocks; /* MCUs resident in the cross-frame block cache (0 without it) */
  uint64_t evicted_blocks;  /* blocks evicted since the last jt_get_stats (0 without the cache) */
} jt_stats;

/* Launch configuration picked by the autotuner (or set by hand). */
typedef struct {
  int32_t decode_mcus_per_warp; /* most MCUs a decode warp takes at a time (its buffer
                                   width): 4, 8, 16 or 32; a short list runs fewer per warp */
  int32_t decode_warps;         /* warps per decode CTA: 1..16 (the CTA must fit shared memory) */
  int32_t decode_ctas_per_sm;   /* resident decode CTAs per SM of the persistent grid (>= 1) */
  int32_t pixel_threads;        /* threads per CTA of mark and colourise (64..1024, mult. of 32) */
  int32_t pixel_ctas_per_sm;    /* CTAs per SM of the grid-stride mark and colourise grids */
  int32_t decode_short_lists;   /* 1: a frame whose work list has at most 4 MCUs per decode warp
                                   decodes it one MCU per warp, each by the whole warp (a
                                   separate kernel); 0: one MCU per lane always; -1 (default):
                                   1 with the cross-frame block cache, 0 without */
} jt_tuning;

/* ---- context ------------------------------------------------------------------------- */

/* Creates a context on CUDA device `device` with a block cache of `max_cache_blocks`
 * 16x16 RGBA8 blocks (1 KiB each; a 4:4:4 MCU of 8x8 texels takes a quarter block).
 * Owns all device memory it allocates; the caller owns *out and frees it with jt_destroy. */
jt_status jt_create(jt_ctx** out, int device, uint64_t max_cache_blocks);
jt_status jt_destroy(jt_ctx* ctx);
const char* jt_last_error(const jt_ctx* ctx);
const char* jt_status_string(jt_status s);

/* ---- textures (Sec. 4.6, Sec. 5.1) --------------------------------------------------- */

/* Uploads one mip level of one texture: the unstuffed entropy-coded segment of a baseline
 * sequential JPEG scan (bytes 0xFF 0x00 replaced by 0xFF, no markers, no restart
 * intervals; `nbits` coded bits in `nbytes` bytes), its per-MCU index (`nblocks` =
 * ceil(width/mw) * ceil(height/mw) entries, MCU order row-major, mw = 16 at 4:2:0, 8 at
 * 4:4:4), two quantisation tables (luma, chroma; 64 entries each in natural row-major
 * order, `qt` points to 128 uint16) and four Huffman specs (DC luma, AC luma, DC chroma,
 * AC chroma). Components: Y uses table 0, Cb and Cr table 1.
 * `sampling` is 420 (MCU = 4 Y + Cb + Cr data units, 16x16 texels) or 444 (Y, Cb, Cr,
 * 8x8 texels). All pointers are host memory and are copied; they may be freed on return.
 * MCUs of the level get consecutive global ids (gids) in upload order: the first level
 * uploaded starts at gid 0 and each level starts where the previous one ended.
 * 0 <= tex_id < 0xFFFF, 0 <= level < JT_MAX_LEVELS, 1 <= width, height <= 65535,
 * nbytes < 2^29 (bit offsets are 32-bit); a (tex_id, level) pair may be uploaded once.
 * Not allowed between jt_mark and jt_decode. */
jt_status jt_upload_texture(jt_ctx* ctx, int tex_id, int level, int width, int height, int sampling,
                            const uint8_t* bitstream, uint64_t nbytes, uint64_t nbits,
                            const jt_block_index* index, uint64_t nblocks, const uint16_t* qt,
                            const jt_huff_spec huff[4]);

/* Uploads one mip level in the paper's compact random-access form (Sec. 5.1 "Indexing
 * Table", Sec. 5.3 "Memory Overhead"), as an alternative to jt_upload_texture; both forms
 * may be mixed in one context and decode to identical tiles.
 *  - `stream` (nbytes bytes, unstuffed): MCU m starts on byte
 *    start(m) = abs_offsets[m / 9] + (m % 9 ? rel_offsets[8 (m / 9) + m % 9 - 1] : 0),
 *    and its bits end at or before start(m + 1) (the last MCU: at or before nbytes).
 *    Its data units are coded as in a baseline scan, except that the first luma data unit
 *    and the chroma data units have no DC difference: their DCs are stored in dc_records.
 *    The other luma data units code their DC as the difference to the previous luma data
 *    unit of the same MCU.
 *  - abs_offsets: ceil(nblocks / 9) uint32; rel_offsets: 8 ceil(nblocks / 9) uint16
 *    (entries past the last MCU are ignored). Starts must not decrease and must be at most
 *    nbytes; otherwise JT_ERR_INVALID_ARG.
 *  - dc_records: ceil(36 nblocks / 32) uint32 words holding a bit array (bit b is bit
 *    b % 32 of word b / 32); MCU m's first-luma, Cb and Cr DCs are the 12-bit two's
 *    complement values at bits 36 m, 36 m + 12 and 36 m + 24.
 * Everything else (sizes, tables, limits, gids, ownership) is as for jt_upload_texture. */
jt_status jt_upload_texture_compact(jt_ctx* ctx, int tex_id, int level, int width, int height, int sampling,
                                    const uint8_t* stream, uint64_t nbytes, const uint32_t* abs_offsets,
                                    const uint16_t* rel_offsets, const uint32_t* dc_records, uint64_t nblocks,
                                    const uint16_t* qt, const jt_huff_spec huff[4]);

/* Index extension (not in the paper): records where each data unit of each MCU of a level
 * uploaded with jt_upload_texture starts, so that the decoder can run an MCU's data units
 * on six lanes at once instead of one chain (each unit's DC difference is chained
 * afterwards). du_offsets: host, count = nblocks * (ndu - 1) uint16, [mcu][unit 1..ndu-1],
 * bits from the MCU's first bit, non-decreasing within an MCU (ndu = 6 at 4:2:0, 3 at
 * 4:4:4); copied. Reduced levels made from the level use them too. A unit that runs past
 * the next unit's start sets JT_DEVERR_CORRUPT. Not for compact or reduced levels; not
 * allowed between jt_mark and jt_decode. */
jt_status jt_set_du_offsets(jt_ctx* ctx, int tex_id, int level, const uint16_t* du_offsets, uint64_t count);

/* Registers level `level` of texture `tex_id` as the reduced-resolution decode of the
 * stored level `src_level` (the mip alternative of Sec. 7: a lower resolution from the
 * lowest frequencies only). Each data unit of the source gives N x N texels (N = 8 >> reduce,
 * reduce = 1, 2 or 3; 3 = the DC alone) by the N-point IDCT of its N x N lowest-frequency
 * coefficients with the 8-point normalisation (the block at 1/2^reduce scale) and the same
 * integer rounding as the full decode; an MCU becomes a (mw >> reduce)^2 tile, 4:2:0 chroma
 * replicated 2x2 as at full size. The level is max(1, w >> reduce) x max(1, h >> reduce)
 * texels on the source's MCU grid, gets its own gids (as many as the source has MCUs) and
 * shares the source's stream, index and tables. The source must be a level uploaded with
 * jt_upload_texture or jt_upload_texture_compact; `level` must not exist yet. Not allowed
 * between jt_mark and jt_decode. */
jt_status jt_add_reduced_level(jt_ctx* ctx, int tex_id, int src_level, int reduce, int level);

/* ---- geometry-pass stand-in --------------------------------------------------------- */

/* One screen-space quad of a procedural scene (fp32; "reference units" are a frame
 * 1000 units high, scaled to pixels by kx, ky of the scene). */
typedef struct {
  float cx[4], cy[4]; /* corners, counter-clockwise on screen (y down), reference units */
  float ex[4], ey[4]; /* edge vectors corner i -> corner (i + 1) % 4 */
  float h[9];         /* row-major map (x, y, 1) -> (s, t, w); (s/w, t/w) in the unit square */
  float rep, cs, sn, ou, ov; /* uv = (ou, ov) + rep * [[cs, -sn], [sn, cs]] (s, t) */
  int32_t tex;        /* texture id */
  int32_t x0, y0, x1, y1; /* inclusive pixel bounds; pixels outside are not tested */
} jt_scene_quad;

/* A procedural scene: a ground plane y = 0 of 2 m cells seen from a pinhole camera, under
 * screen-space quads drawn in order (the last one covering a pixel wins). */
typedef struct {
  int32_t width, height;   /* G-buffer size */
  float cam[3];            /* camera position (metres) */
  float rot[9];            /* row-major: world ray = rot * (sx, sy, -1) */
  float ax, ay;            /* 2 / width, 2 / height */
  float tan_x, tan_y;      /* sx = (px * ax - 1) * tan_x, sy = (1 - py * ay) * tan_y at pixel coordinate (px, py) */
  float max_t;             /* farthest ground hit (ray parameter) */
  float kx, ky, shift;     /* quad reference units per pixel; quad x = px * kx - shift */
  uint64_t cell_seed;      /* ground cell (i, j) takes hash = SplitMix64 mix of (cell_seed, i, j) */
  int32_t ntex;            /* textures: cell texture = hash % ntex */
  int32_t use_mips;        /* 0: every level 0 */
  const int32_t* tex_w;    /* host, ntex: level-0 size and level count of each texture */
  const int32_t* tex_h;
  const int32_t* tex_levels;
  const jt_scene_quad* quads; /* host, nquads <= 4096 */
  int32_t nquads;
  int32_t reserved;
} jt_scene;

/* Writes the G-buffer of `scene` into `out` (device, width x height of the scene), standing
 * in for the geometry pass that precedes the path (Sec. 4). Per pixel at centre
 * (px, py) = (x + 1/2, y + 1/2), all arithmetic in fp32 with each operation rounded in the
 * order written:
 *  - quads: the last quad in drawing order whose bounds hold (x, y) and whose four edge
 *    tests ex[i] (qy - cy[i]) - ey[i] (qx - cx[i]) are >= 0 at qx = px kx - shift, qy = py ky;
 *    uv from h and the uv map; the footprint from uv at qx -+ kx/2 and qy -+ ky/2;
 *  - else the ground: the ray hits y = 0 at t = -cam_y / d_y if d_y < -1e-9 and
 *    t <= max_t; uv = (x, z) / 2 plus the cell's offset ((hash >> 16) & 0xFFFF,
 *    (hash >> 32) & 0xFFFF) / 65536, texture hash % ntex; the footprint from the hits at
 *    (x, py), (x + 1, py), (px, y), (px, y + 1), the last level when one of them misses;
 *  - else sky: uv (0, 0), texture 0xFFFF, level 0.
 * The level is floor(log2(rho) + 1/2) clamped to [0, levels - 1], rho^2 = the larger
 * squared texel-space footprint (uv differences times the level-0 size), decided exactly by
 * comparing rho^2 with 2^(2k-1). Errors: JT_ERR_INVALID_ARG for a bad size, null pointer,
 * more than 4096 quads, a quad texture outside [0, ntex) or a level count outside [1, 16]. */
jt_status jt_raster_scene(jt_ctx* ctx, const jt_scene* scene, const jt_gbuffer* out, jt_stream stream);

/* ---- per-frame path -------------------------------------------------------------------- */

/* Mark (Sec. 4.2): for every pixel with a texture, computes the texel(s) its uv falls on at
 * its mip level — nearest: x = floor(u*w) mod w; bilinear: the four texels around
 * u*w - 1/2; bilinear clamped: the nearest texel — and flags the MCUs that hold them. Flags accumulate over calls until the
 * next jt_decode, so several views marked in turn are decoded once (union). */
jt_status jt_mark(jt_ctx* ctx, const jt_gbuffer* g, int filter, jt_stream stream);

/* Compact + decode (Sec. 4.3): turns the flags into a work list of gids in ascending order
 * (exclusive prefix sum, which also assigns each needed MCU its block-cache slot) and
 * clears the flags; then decodes every listed MCU into its slot: Huffman decode from the
 * MCU's index entry, dequantise, 8x8 integer IDCT, 4:2:0 chroma replication, YCbCr->RGB,
 * RGBA8 tile (alpha 255). Needs no host synchronisation: the count stays on the device. */
jt_status jt_decode(jt_ctx* ctx, jt_stream stream);

/* Resolve (Sec. 4.4): writes RGBA8 per pixel from the block cache (nearest, or bilinear
 * with fp32 weights and round-half-up, with or without the clamp to the nearest MCU). Pixels without texture get (0,0,0,255). `filter`
 * must match the jt_mark call(s) of this frame. out_rgba: device, [height][width][4],
 * 16-byte aligned. */
jt_status jt_colorize(jt_ctx* ctx, const jt_gbuffer* g, int filter, uint8_t* out_rgba, jt_stream stream);

/* Synchronises the last stream used, reads the counts and the device error word (and
 * clears it). Returns JT_ERR_CORRUPT_STREAM / JT_ERR_CAPACITY / JT_ERR_UNSUPPORTED when the
 * corresponding error bit was set, else JT_OK; *out is filled either way. */
jt_status jt_get_stats(jt_ctx* ctx, jt_stats* out);

/* ---- batched frames, CUDA graphs, autotuning ------------------------------------------- */

/* One frame over `nviews` views (<= JT_MAX_VIEWS): one mark launch over all views into the
 * shared flags (an MCU needed by several views is decoded once), one compaction, one
 * persistent decode over the merged work list, one colourise launch over all views. */
jt_status jt_frame(jt_ctx* ctx, const jt_view* views, int nviews, int filter, jt_stream stream);

/* The same frame captured once into a CUDA graph; replay with jt_graph_launch. The views'
 * pointers are baked into the graph: their contents may change between launches, the
 * buffers may not move. The context's own tables are baked in too: an upload of any kind
 * (jt_upload_texture, jt_upload_texture_compact, jt_add_reduced_level, jt_set_du_offsets,
 * jt_register_coeff_textures) or a jt_set_block_cache call after the capture makes
 * jt_graph_launch refuse the graph with JT_ERR_STATE (nothing is launched); capture it
 * again. The graph belongs to ctx and must be destroyed before it. */
jt_status jt_frame_graph(jt_ctx* ctx, const jt_view* views, int nviews, int filter, jt_stream stream,
                         jt_graph** out);
jt_status jt_graph_launch(jt_graph* g, jt_stream stream);
jt_status jt_graph_destroy(jt_graph* g);

/* Reference form for comparison: per view and per texture id present in the frame, a
 * mark, compaction, decode and colourise restricted to that texture (4 launches each,
 * plus one colourise per view for empty pixels). Same output as jt_frame. */
jt_status jt_frame_plain(jt_ctx* ctx, const jt_view* views, int nviews, int filter, jt_stream stream);

jt_status jt_get_tuning(const jt_ctx* ctx, jt_tuning* out);
jt_status jt_set_tuning(jt_ctx* ctx, const jt_tuning* t);

/* Times `reps` graph replays of the frame for each candidate launch configuration (decode
 * MCUs per warp x warps per CTA x CTAs per SM, then the pixel-kernel shape), keeps the
 * fastest in the context and returns it with its median frame time in milliseconds. */
jt_status jt_autotune(jt_ctx* ctx, const jt_view* views, int nviews, int filter, jt_stream stream, int reps,
                      jt_tuning* best, float* best_ms);

/* ---- cross-frame block cache (Sec. 4.1 "Texture Block Cache", Sec. 4.5 "Update Cache") ----- */

/* persistent = 1: decoded MCUs stay in the block cache between frames, each in a 1 KiB block
 * (a quarter used at 4:4:4). A frame's compaction step becomes a cache update: the blocks
 * of resident MCUs that no pixel of the frame needs are evicted, the needed MCUs that are
 * not resident get free blocks and are the only ones decoded, and every needed MCU's slot
 * points at its block. Frames, graphs and jt_mark/jt_decode use it; jt_frame_plain refuses
 * it. Block numbers and the work-list order depend on atomic order; tiles and pixels do
 * not. More needed MCUs than blocks set JT_DEVERR_CAPACITY. An upload empties the cache.
 * persistent = 0 (the default): every frame decodes its whole needed set.
 * Switching mode empties the cache; the call synchronises the device. */
jt_status jt_set_block_cache(jt_ctx* ctx, int persistent);

/* ---- inspection (tests, tools) ---------------------------------------------------------- */

/* Pass timing. While enabled, every frame enqueued by jt_frame / jt_frame_graph (graphs
 * captured while enabled) records CUDA events on its stream at the pass boundaries; the
 * events belong to the context. jt_profile_read waits for the last recorded frame and
 * returns its durations in milliseconds: ms[0] mark, ms[1] compaction, ms[2] decode,
 * ms[3] colourise. The events between the passes also keep the compaction and the decode
 * from starting before the pass ahead of them ends (programmatic launch), so a profiled
 * frame takes longer than an unprofiled one. */
jt_status jt_profile(jt_ctx* ctx, int enable);
jt_status jt_profile_read(jt_ctx* ctx, float ms[4]);

/* Copies the last work list (gids, ascending) to dst (host or device), at most cap entries;
 * *count receives the full length. Synchronises. */
jt_status jt_read_work_list(jt_ctx* ctx, uint32_t* dst, uint64_t cap, uint64_t* count);
/* Copies the cache-unit offset of each gid in [gid_begin, gid_begin + n) to dst (valid for
 * gids in the last work list). Synchronises. */
jt_status jt_read_slots(jt_ctx* ctx, uint64_t gid_begin, uint64_t n, uint32_t* dst);
/* Copies 256-byte cache units [unit_begin, unit_begin + n) to dst. A 4:2:0 MCU is 4 units
 * (16 rows of 16 RGBA8 texels), a 4:4:4 MCU one unit (8 rows of 8). Synchronises. */
jt_status jt_read_cache(jt_ctx* ctx, uint64_t unit_begin, uint64_t n, uint8_t* dst);

/* ---- compaction without allocation (no counterpart in the paper) ------------------------- */

/* Largest n accepted by jt_compact_static: 4096 scan tiles of 4096 flags. */
#define JT_STATIC_COMPACT_MAX_FLAGS 16777216u

/* The compaction step of jt_decode (flags -> work list and cache slots: an exclusive prefix
 * sum over the flags), on caller-owned buffers, for callers that must not allocate device memory at the
 * call: a frame loop that cannot afford the device-wide synchronisation cudaMalloc/cudaFree
 * may cause, code under memory pressure, or code running inside an allocator. It makes no
 * allocating call (no cudaMalloc/cudaFree, no library allocator); its scratch is a fixed
 * array in the library's device image. No context is needed; the current device is used.
 *
 *  flags    device uint8[n], 16-byte aligned: cache units each index needs (0 = not needed).
 *           Zeroed by the call (as jt_decode leaves a context's flags).
 *  slot     device uint32[n]: slot[i] = sum of flags[j] for j < i, written where flags[i] != 0.
 *  work     device uint32[work_cap]: the indices i with flags[i] != 0, ascending; entries
 *           past work_cap are dropped (and JT_DEVERR_CAPACITY is set in totals[2]).
 *  totals   device uint32[3]: {count of flagged indices, sum of flags, JT_DEVERR_* bits}.
 *  All four stay caller-owned and must stay valid until the stream reaches the work.
 * Returns JT_ERR_CAPACITY for n > JT_STATIC_COMPACT_MAX_FLAGS and JT_ERR_INVALID_ARG for a
 * null or misaligned buffer, both before enqueueing anything; JT_ERR_CUDA if a CUDA call fails
 * (jt_last_error needs a context and does not apply), including when a launch error of the
 * caller's is already pending on this thread: that error is left pending for the caller to
 * read and nothing is enqueued. Enqueues a memset, two kernels and two
 * device-to-device copies on `stream`, which stays asynchronous.
 * The first call on each device looks up the scratch address and must happen outside any
 * stream capture. Calls share the scratch: two calls in flight at once on one device race
 * and corrupt each other's results, so order them (one stream, or events). */
jt_status jt_compact_static(uint8_t* flags, uint32_t n, uint32_t* slot, uint32_t* work, uint32_t work_cap,
                            uint32_t* totals, jt_stream stream);

/* ---- differentiable colourise (float chain; not in the paper) ---------------------------- */

/* Registers `count` coefficient textures with ids first_tex_id.. first_tex_id+count-1, each
 * width x height texels at 4:2:0, level 0, whose content is given per call as dequantised
 * DCT coefficients: float32 [count][height/16][width/16][6][64] (data units Y00 Y01 Y10
 * Y11 Cb Cr, coefficient k = v*8+u in natural order). width and height must be multiples
 * of 16. They share the gid space with uploaded textures but are only valid for the two
 * calls below. */
jt_status jt_register_coeff_textures(jt_ctx* ctx, int first_tex_id, int count, int width, int height);

/* Forward of the float chain F = bilinear(RGB(upsample(IDCT_f(c) + 128))) with the
 * orthonormal 8x8 IDCT, JFIF colour matrix, chroma replication and bilinear weights of
 * jt_colorize, without rounding or clamping. coeffs: device float32 as registered;
 * out_rgb: device float32 [height][width][3], overwritten; empty pixels get 0. The view's
 * pixels are bucketed under the MCUs their taps touch (as in jt_colorize_backward); the sum
 * of a pixel whose taps span two or more MCUs is added in float atomics, so its last bits
 * may differ between calls. At most max_cache_blocks needed coefficient MCUs are served;
 * beyond that the error word gets JT_DEVERR_CAPACITY and those pixels get 0. */
jt_status jt_colorize_float(jt_ctx* ctx, const jt_gbuffer* g, const float* coeffs, float* out_rgb,
                            jt_stream stream);

/* Adjoint of jt_colorize_float: grad_coeffs = J^T grad_frame, where grad_frame is
 * float32 [height][width][3] (device). grad_coeffs (device, the coefficients' shape) is
 * overwritten: zero except for the MCUs the frame touches. Recomputes the needed set
 * from the G-buffer; stores no decoded blocks and no per-texel gradients: the view's
 * pixels are bucketed under the MCUs their taps touch and each MCU gathers its bucket.
 * The bucket array (four 32-byte entries per pixel of the view) is grown on the first call
 * with a larger view, which synchronises the stream once. */
jt_status jt_colorize_backward(jt_ctx* ctx, const jt_gbuffer* g, const float* grad_frame, float* grad_coeffs,
                               jt_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* JT_H */
