// Host implementation of the C ABI declared in include/jt.h: context and memory
// management, texture upload (decode-table construction), the per-frame launch sequence,
// batched frames, CUDA-graph capture, the per-texture reference pipeline and autotuning.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "jt_internal.cuh"

using namespace jt;

namespace {

enum class Phase { Idle, Marked, Decoded };

struct Level {
  int tex, level;
  void* stream_mem = nullptr;
  void* index_mem = nullptr;
  void* du_mem = nullptr;  // data-unit starts (jt_set_du_offsets)
};

}  // namespace

struct jt_ctx {
  int device = 0;
  int sm_count = 0;
  uint64_t cap_units = 0;
  std::string last_error;
  cudaStream_t last_stream = nullptr;
  Phase phase = Phase::Idle;
  // Bumped whenever a device table or buffer that a captured graph bakes in is freed,
  // moved or rewritten by an upload (descriptors, level tables, Huffman and quantisation
  // sets, frame buffers, the block cache's arrays): graphs captured before are refused.
  uint64_t generation = 0;
  jt_tuning tuning{};
  int decode_occ[33][17] = {};  // resident decode CTAs per SM by [MCUs per warp][warps per CTA]

  // textures
  std::vector<DevDesc> descs;
  std::vector<Level> levels;
  DevDesc* d_descs = nullptr;
  size_t d_descs_cap = 0;
  uint32_t* d_desc_of_gid = nullptr;  // descriptor index of every gid (the decoder's lookup)
  uint64_t desc_of_gid_cap = 0;
  std::vector<int32_t> map;  // [map_ntex * 16]
  std::vector<LevelRec> lrec;  // [map_ntex * 16]
  std::vector<PixRec> prec;    // [map_ntex * 16 + 1], the last one all zero
  uint32_t map_ntex = 0;
  int32_t* d_map = nullptr;
  LevelRec* d_lrec = nullptr;
  PixRec* d_prec = nullptr;
  std::vector<HuffSet> hsets;
  HuffSet* d_huff = nullptr;
  std::vector<std::vector<uint16_t>> qsets;  // zig-zag order, 128 entries
  uint16_t* d_quant = nullptr;
  uint64_t ngid = 0;

  // per-frame buffers
  uint8_t* flags = nullptr;
  uint32_t* slot = nullptr;
  uint32_t* work = nullptr;
  uint64_t* tile_status = nullptr;
  uint64_t gid_cap = 0;
  uint8_t* cache = nullptr;
  FrameState* state = nullptr;

  // cross-frame block cache (jt_set_block_cache)
  bool persistent = false;
  bool unit_mode = false;  // some level has data-unit starts
  uint32_t* resbits = nullptr;    // residency bitmap, one bit per gid
  uint32_t* ring = nullptr;       // [nblocks] free blocks
  uint32_t* deferred = nullptr;   // [nblocks]
  uint32_t nblocks = 0;
  uint64_t resident_ngid = 0;     // gids covered by the residency bitmap
  CacheState* cstate = nullptr;

  // coefficient textures (float chain)
  int coef_first = -1, coef_count = 0, coef_w = 0, coef_h = 0;
  uint32_t coef_gid_base = 0;
  uint32_t float_tile_cap = 0;     // needed coefficient MCUs a float pass can serve
  uint32_t* bucket_cnt = nullptr;   // [float_tile_cap + 1], cleared at the start of each backward call
  uint32_t* bucket_off = nullptr;   // [float_tile_cap + 1]
  uint32_t* bucket_bsum = nullptr;  // one per kBucketScan counts
  uint32_t* bucket = nullptr;       // [bucket_cap] 32-byte entries
  uint64_t bucket_cap = 0;
  cudaStream_t capture_stream = nullptr;

  // scene rasteriser inputs (jt_raster_scene)
  uint8_t* raster_buf = nullptr;
  size_t raster_cap = 0;

  // pass timing (jt_profile)
  bool profiling = false;
  cudaEvent_t prof[5] = {};
};

struct jt_graph {
  jt_ctx* ctx;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t generation = 0;  // the context's generation at capture
};

namespace {

constexpr uint64_t kMaxGids = 1ull << 26;   // MCUs over all levels: unit sums of 4 per MCU stay below 2^28
constexpr uint64_t kMaxUnits = 1ull << 28;  // block cache of at most 64 GiB (2^28 units of 256 B)

jt_status fail(jt_ctx* c, jt_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->last_error = buf;
  }
  return s;
}

#define JT_CUDA(c, call)                                                                          \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return fail((c), JT_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

template <typename T>
jt_status dev_alloc(jt_ctx* c, T** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? JT_ERR_OOM : JT_ERR_CUDA, "cudaMalloc(%zu): %s", bytes,
                cudaGetErrorString(e));
  }
  return JT_OK;
}

template <typename T>
void dev_free(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

// Natural index of the k-th zig-zag coefficient (inverse of the kernel's closed form).
void zigzag_natural(int nat[64]) {
  for (int r = 0; r < 8; ++r)
    for (int c = 0; c < 8; ++c) {
      const int s = r + c;
      const int before = s <= 7 ? s * (s + 1) / 2 : 64 - (15 - s) * (16 - s) / 2;
      const int along = (s & 1) ? r - (s > 7 ? s - 7 : 0) : (s < 7 ? s : 7) - r;
      nat[before + along] = r * 8 + c;
    }
}

// Table entry of symbol `sym` with a code of length l (0 when the symbol is invalid for the
// table's class; the decoder's MAXCODE walk then rejects it).
uint16_t symbol_entry(bool dc, int l, uint8_t sym) {
  const int r = dc ? 0 : sym >> 4, s = dc ? sym : sym & 15;
  if ((dc && s > 11) || (!dc && s > 10) || (!dc && s == 0 && r != 0 && r != 15)) return 0;
  if (!dc && s == 0) return huff_entry((uint32_t)l, 0, r == 0 ? kRunEob : 15u);
  return huff_entry((uint32_t)l, (uint32_t)s, (uint32_t)r);
}

// Canonical decode tables of one Huffman spec (T.81 Annex C code assignment).
bool build_table(const jt_huff_spec& spec, bool dc, HuffTable& t, std::string& why) {
  std::memset(&t, 0, sizeof t);
  int n = 0;
  uint64_t kraft = 0;
  for (int l = 1; l <= 16; ++l) {
    n += spec.bits[l - 1];
    kraft += (uint64_t)spec.bits[l - 1] << (16 - l);
  }
  if (n == 0 || n > 256) {
    why = "Huffman spec with no symbols or more than 256";
    return false;
  }
  if (kraft > (1u << 16)) {
    why = "Huffman code lengths violate the Kraft inequality";
    return false;
  }
  std::memcpy(t.vals, spec.vals, n);
  // left-aligned start of the codes longer than kLutBits = Kraft mass of the shorter ones
  uint32_t first16 = 0;
  for (int l = 1; l <= kLutBits; ++l) first16 += (uint32_t)spec.bits[l - 1] << (16 - l);
  t.first16 = first16;
  t.n2 = (first16 < 65536u && 65536u - first16 <= (uint32_t)kLut2Size) ? 65536u - first16 : 0u;
  int code = 0, k = 0;
  for (int l = 1; l <= 16; ++l) {
    const int nl = spec.bits[l - 1];
    if (nl == 0) {
      t.maxcode[l] = -1;
      t.valoff[l] = 0;
    } else {
      t.valoff[l] = k - code;
      for (int i = 0; i < nl; ++i, ++k, ++code) {
        const uint16_t e = symbol_entry(dc, l, spec.vals[k]);
        if (l <= kLutBits) {
          const int first = code << (kLutBits - l), cnt = 1 << (kLutBits - l);
          for (int j = 0; j < cnt; ++j) t.lut[first + j] = e;
        } else if (t.n2) {
          const uint32_t first = ((uint32_t)code << (16 - l)) - first16, cnt = 1u << (16 - l);
          for (uint32_t j = 0; j < cnt; ++j) t.lut2[first + j] = e;
        }
      }
      t.maxcode[l] = code - 1;
    }
    code <<= 1;
  }
  t.maxcode[0] = -1;
  return true;
}

jt_status grow_frame_buffers(jt_ctx* c, uint64_t need) {
  if (need <= c->gid_cap) return JT_OK;
  ++c->generation;
  uint64_t cap = std::max<uint64_t>(need, c->gid_cap + c->gid_cap / 2);
  cap = std::min<uint64_t>(std::max<uint64_t>(cap, 4096), kMaxGids);
  cap = (cap + 15) & ~15ull;
  dev_free(c->flags);
  dev_free(c->slot);
  dev_free(c->work);
  dev_free(c->tile_status);
  c->gid_cap = 0;
  jt_status s;
  if ((s = dev_alloc(c, &c->flags, cap + 16)) != JT_OK) return s;
  if ((s = dev_alloc(c, &c->slot, cap * 4)) != JT_OK) return s;
  if ((s = dev_alloc(c, &c->work, cap * 4)) != JT_OK) return s;
  const uint64_t tiles = cap / kScanTile + 2;
  if ((s = dev_alloc(c, &c->tile_status, tiles * 8)) != JT_OK) return s;
  JT_CUDA(c, cudaMemset(c->flags, 0, cap + 16));
  JT_CUDA(c, cudaMemset(c->slot, 0, cap * 4));
  JT_CUDA(c, cudaMemset(c->work, 0, cap * 4));
  JT_CUDA(c, cudaMemset(c->tile_status, 0, tiles * 8));
  c->gid_cap = cap;
  return JT_OK;
}

jt_status sync_descs(jt_ctx* c) {
  ++c->generation;  // the level tables below are reallocated
  if (c->descs.size() > c->d_descs_cap) {
    dev_free(c->d_descs);
    size_t cap = std::max<size_t>(64, c->descs.size() * 2);
    jt_status s = dev_alloc(c, &c->d_descs, cap * sizeof(DevDesc));
    if (s != JT_OK) return s;
    c->d_descs_cap = cap;
  }
  JT_CUDA(c, cudaMemcpy(c->d_descs, c->descs.data(), c->descs.size() * sizeof(DevDesc), cudaMemcpyHostToDevice));
  dev_free(c->d_map);
  dev_free(c->d_lrec);
  jt_status s = dev_alloc(c, &c->d_map, c->map.size() * 4);
  if (s != JT_OK) return s;
  if ((s = dev_alloc(c, &c->d_lrec, c->lrec.size() * sizeof(LevelRec))) != JT_OK) return s;
  dev_free(c->d_prec);
  c->prec.resize(c->lrec.size() + 1, PixRec{});
  c->prec.back() = PixRec{};  // the record of keys outside the table
  if ((s = dev_alloc(c, &c->d_prec, c->prec.size() * sizeof(PixRec))) != JT_OK) return s;
  JT_CUDA(c, cudaMemcpy(c->d_prec, c->prec.data(), c->prec.size() * sizeof(PixRec), cudaMemcpyHostToDevice));
  if (!c->map.empty()) {
    JT_CUDA(c, cudaMemcpy(c->d_map, c->map.data(), c->map.size() * 4, cudaMemcpyHostToDevice));
    JT_CUDA(c, cudaMemcpy(c->d_lrec, c->lrec.data(), c->lrec.size() * sizeof(LevelRec), cudaMemcpyHostToDevice));
  }
  return JT_OK;
}

jt_status sync_tables(jt_ctx* c) {
  ++c->generation;
  dev_free(c->d_huff);
  jt_status s = dev_alloc(c, &c->d_huff, std::max<size_t>(1, c->hsets.size()) * sizeof(HuffSet));
  if (s != JT_OK) return s;
  if (!c->hsets.empty())
    JT_CUDA(c, cudaMemcpy(c->d_huff, c->hsets.data(), c->hsets.size() * sizeof(HuffSet), cudaMemcpyHostToDevice));
  dev_free(c->d_quant);
  if ((s = dev_alloc(c, &c->d_quant, std::max<size_t>(1, c->qsets.size()) * 256)) != JT_OK) return s;
  for (size_t i = 0; i < c->qsets.size(); ++i)
    JT_CUDA(c, cudaMemcpy(c->d_quant + i * 128, c->qsets[i].data(), 256, cudaMemcpyHostToDevice));
  return JT_OK;
}

bool pow2(uint32_t v) { return v && !(v & (v - 1)); }

TexLookup lookup(const jt_ctx* c) {
  bool all_p2 = true;
  for (const DevDesc& d : c->descs) all_p2 &= pow2(d.width) && pow2(d.height);
  return TexLookup{c->d_descs, c->d_map, reinterpret_cast<const uint4*>(c->d_lrec),
                   reinterpret_cast<const uint4*>(c->d_prec), c->map_ntex, all_p2 ? 1u : 0u};
}


bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

jt_status check_gbuffer(jt_ctx* c, const jt_gbuffer* g) {
  if (!g || !g->uv || !g->tex_id || !g->mip) return fail(c, JT_ERR_INVALID_ARG, "null G-buffer pointer");
  if (g->width <= 0 || g->height <= 0) return fail(c, JT_ERR_INVALID_ARG, "empty G-buffer");
  if ((uint64_t)g->width * g->height >= (1ull << 31)) return fail(c, JT_ERR_INVALID_ARG, "G-buffer too large");
  if (!aligned(g->uv, 16) || !aligned(g->tex_id, 8) || !aligned(g->mip, 4))
    return fail(c, JT_ERR_INVALID_ARG, "G-buffer arrays must be 16/8/4-byte aligned (uv/tex_id/mip)");
  return JT_OK;
}

jt_status make_views(jt_ctx* c, const jt_view* views, int n, bool need_out, ViewSet& vs) {
  if (!views || n <= 0 || n > JT_MAX_VIEWS) return fail(c, JT_ERR_INVALID_ARG, "need 1..%d views", JT_MAX_VIEWS);
  std::memset(&vs, 0, sizeof vs);
  uint64_t quads = 0, tiles = 0;
  for (int i = 0; i < n; ++i) {
    jt_status s = check_gbuffer(c, &views[i].g);
    if (s != JT_OK) return s;
    if (need_out && (!views[i].out_rgba || !aligned(views[i].out_rgba, 16)))
      return fail(c, JT_ERR_INVALID_ARG, "view %d: output must be a 16-byte aligned device pointer", i);
    View& v = vs.v[i];
    v.uv = reinterpret_cast<const float4*>(views[i].g.uv);
    v.tex = views[i].g.tex_id;
    v.mip = views[i].g.mip;
    v.out = reinterpret_cast<uint4*>(views[i].out_rgba);
    v.npx = (uint32_t)((uint64_t)views[i].g.width * views[i].g.height);
    v.quad_begin = (uint32_t)quads;
    quads += (v.npx + 3) / 4;
    v.width = views[i].g.width;
    v.height = views[i].g.height;
    v.tiles_x = (uint32_t)((v.width + kTileW - 1) / kTileW);
    v.tile_begin = (uint32_t)tiles;
    tiles += (uint64_t)v.tiles_x * ((v.height + kTileH - 1) / kTileH);
  }
  if (quads >= (1ull << 31)) return fail(c, JT_ERR_INVALID_ARG, "views too large");
  vs.n = n;
  vs.total_quads = (uint32_t)quads;
  vs.total_tiles = (uint32_t)tiles;
  return JT_OK;
}

// Persistent grid for the tiled screen passes: at most one CTA per tile.
int pixel_grid(const jt_ctx* c, const ViewSet& vs) {
  const uint64_t cap = (uint64_t)c->sm_count * std::max(1, c->tuning.pixel_ctas_per_sm);
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(vs.total_tiles, cap));
}

jt_status check_launch(jt_ctx* c, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, JT_ERR_CUDA, "%s launch: %s", what, cudaGetErrorString(e));
  return JT_OK;
}

jt_status enqueue_mark(jt_ctx* c, const ViewSet& vs, int filter, int only_tex, int coef_mode, cudaStream_t s) {
  if (c->descs.empty()) return fail(c, JT_ERR_STATE, "no textures uploaded");
  MarkArgs a{};
  a.views = vs;
  a.tl = lookup(c);
  a.flags = c->flags;
  a.state = c->state;
  a.filter = filter;
  a.only_tex = only_tex;
  a.coef_mode = coef_mode;
  launch_mark(a, c->tuning.pixel_threads, pixel_grid(c, vs), s);
  return check_launch(c, "mark");
}

jt_status enqueue_scan(jt_ctx* c, uint64_t gid_lo, uint64_t gid_hi, cudaStream_t s) {
  gid_lo &= ~15ull;  // 16-byte aligned vector access to the flags
  ScanArgs a{};
  a.flags = c->flags + gid_lo;
  a.gid_lo = (uint32_t)gid_lo;
  a.n = (uint32_t)(gid_hi - gid_lo);
  a.slot = c->slot;
  a.work = c->work;
  a.work_cap = (uint32_t)c->gid_cap;
  a.tile_status = c->tile_status;
  a.state = c->state;
  a.cap_units = (uint32_t)c->cap_units;
  launch_scan(a, s);
  return check_launch(c, "scan");
}

// Frees the cross-frame block cache's arrays.
void cache_free(jt_ctx* c) {
  ++c->generation;
  dev_free(c->resbits);
  dev_free(c->ring);
  dev_free(c->deferred);
  dev_free(c->cstate);
  c->nblocks = 0;
  c->resident_ngid = 0;
}

// (Re)builds an empty cross-frame block cache over the current gids and the whole block cache.
jt_status cache_reset(jt_ctx* c) {
  cache_free(c);
  c->nblocks = (uint32_t)(c->cap_units / 4);
  c->resident_ngid = c->ngid;
  jt_status s;
  if (c->nblocks == 0) return fail(c, JT_ERR_INVALID_ARG, "the block cache needs at least one block");
  const uint64_t nbits = std::max<uint64_t>(1, (c->ngid + 31) / 32) * 4;  // whole 32-bit words
  if ((s = dev_alloc(c, &c->resbits, nbits)) != JT_OK) return s;
  if ((s = dev_alloc(c, &c->ring, (size_t)c->nblocks * 4)) != JT_OK) return s;
  if ((s = dev_alloc(c, &c->deferred, (size_t)c->nblocks * 4)) != JT_OK) return s;
  if ((s = dev_alloc(c, &c->cstate, sizeof(CacheState))) != JT_OK) return s;
  std::vector<uint32_t> fl(c->nblocks);
  for (uint32_t i = 0; i < c->nblocks; ++i) fl[i] = i;  // blocks are handed out 0, 1, 2, ...
  CacheState cs{};
  cs.free_count = c->nblocks;
  JT_CUDA(c, cudaMemset(c->resbits, 0, nbits));
  JT_CUDA(c, cudaMemcpy(c->ring, fl.data(), (size_t)c->nblocks * 4, cudaMemcpyHostToDevice));
  JT_CUDA(c, cudaMemcpy(c->cstate, &cs, sizeof cs, cudaMemcpyHostToDevice));
  return JT_OK;
}

// The cache update of a persistent-cache frame, in place of the compaction: evict the blocks
// of MCUs the frame does not need, give the needed non-resident ones blocks and a place in the
// work list, set every needed MCU's slot.
jt_status enqueue_cache_update(jt_ctx* c, cudaStream_t s) {
  if (c->resident_ngid != c->ngid) {  // levels were uploaded since: start over
    jt_status st = cache_reset(c);
    if (st != JT_OK) return st;
  }
  CacheArgs a{};
  a.flags = c->flags;
  a.n = (uint32_t)c->ngid;
  a.resbits = reinterpret_cast<uint16_t*>(c->resbits);
  a.resbits32 = c->resbits;
  a.ring = c->ring;
  a.deferred = c->deferred;
  a.nblocks = c->nblocks;
  a.slot = c->slot;
  a.work = c->work;
  a.work_cap = (uint32_t)c->gid_cap;
  a.state = c->state;
  a.cs = c->cstate;
  launch_cache_update(a, c->sm_count * 8, s);
  return check_launch(c, "cache update");
}

// The frame's compaction step: the prefix-sum scan, or the cache update in persistent mode.
jt_status enqueue_compact(jt_ctx* c, cudaStream_t s) {
  return c->persistent ? enqueue_cache_update(c, s) : enqueue_scan(c, 0, c->ngid, s);
}

jt_status enqueue_decode(jt_ctx* c, cudaStream_t s) {
  DecodeArgs a{};
  a.descs = c->d_descs;
  a.ndesc = (uint32_t)c->descs.size();
  a.desc_of_gid = c->d_desc_of_gid;
  a.mcus_per_warp = c->tuning.decode_mcus_per_warp;
  a.unit_mode = c->unit_mode ? 1 : 0;
  a.short_lists = c->tuning.decode_short_lists < 0 ? (c->persistent ? 1 : 0) : c->tuning.decode_short_lists;
  a.huff = c->d_huff;
  a.quant = c->d_quant;
  a.work = c->work;
  a.work_cap = (uint32_t)c->gid_cap;
  a.slot = c->slot;
  a.cache = c->cache;
  a.cap_units = (uint32_t)c->cap_units;
  a.state = c->state;
  const int w = c->tuning.decode_warps;
  const int per_sm = std::max(1, std::min(c->tuning.decode_ctas_per_sm, c->decode_occ[a.mcus_per_warp][w]));
  launch_decode(a, w, c->sm_count * per_sm, s);
  return check_launch(c, "decode");
}

jt_status enqueue_colorize(jt_ctx* c, const ViewSet& vs, int filter, int only_tex, cudaStream_t s) {
  ColorizeArgs a{};
  a.views = vs;
  a.tl = lookup(c);
  a.slot = c->slot;
  a.cache = c->cache;
  a.cap_units = (uint32_t)c->cap_units;
  a.state = c->state;
  a.filter = filter;
  a.only_tex = only_tex;
  launch_colorize(a, c->tuning.pixel_threads, pixel_grid(c, vs), s);
  return check_launch(c, "colorize");
}

jt_status enqueue_frame(jt_ctx* c, const ViewSet& vs, int filter, cudaStream_t s) {
  jt_status st;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (c->profiling) cudaStreamIsCapturing(s, &cap);
  // while capturing, only an "external" record becomes an event-record node of the graph
  const unsigned rec_flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
  auto mark_time = [&](int i) {
    if (c->profiling) cudaEventRecordWithFlags(c->prof[i], s, rec_flags);
  };
  mark_time(0);
  if ((st = enqueue_mark(c, vs, filter, -1, 0, s)) != JT_OK) return st;
  mark_time(1);
  if ((st = enqueue_compact(c, s)) != JT_OK) return st;
  mark_time(2);
  if ((st = enqueue_decode(c, s)) != JT_OK) return st;
  mark_time(3);
  if ((st = enqueue_colorize(c, vs, filter, -1, s)) != JT_OK) return st;
  mark_time(4);
  return check_launch(c, "event record");
}

bool valid_filter(int f) {
  return f == JT_FILTER_NEAREST || f == JT_FILTER_BILINEAR || f == JT_FILTER_BILINEAR_CLAMP;
}

const int kMcusPerWarp[] = {4, 8, 16, 32};
// warps per decode CTA the autotuner tries (any 1..16 is valid); the odd counts let the
// 32-MCU shape fill an SM's shared memory (seven warps of 28 KiB)
const int kDecodeWarps[] = {2, 3, 4, 5, 6, 7, 8, 12, 16};

bool valid_tuning(const jt_ctx* c, const jt_tuning& t) {
  const int M = t.decode_mcus_per_warp, W = t.decode_warps;
  const bool m_ok = M == 4 || M == 8 || M == 16 || M == 32;
  const bool w_ok = W >= 1 && W <= 16;
  return m_ok && w_ok && c->decode_occ[M][W] > 0 && t.decode_ctas_per_sm >= 1 && t.pixel_threads >= 64 &&
         t.pixel_threads <= 1024 && t.pixel_threads % 32 == 0 && t.pixel_ctas_per_sm >= 1 &&
         t.pixel_ctas_per_sm <= 32 && t.decode_short_lists >= -1 && t.decode_short_lists <= 1;
}

// Shared set-up of the two float calls: checks, the view, the float-chain arguments.
jt_status float_setup(jt_ctx* c, const jt_gbuffer* g, const float* in, const float* frame_ptr, FloatArgs& a) {
  if (c->coef_first < 0) return fail(c, JT_ERR_STATE, "no coefficient textures registered");
  if (c->phase == Phase::Marked) return fail(c, JT_ERR_STATE, "a marked frame is pending");
  if (!in || !frame_ptr || !aligned(in, 16) || !aligned(frame_ptr, 16))
    return fail(c, JT_ERR_INVALID_ARG, "coefficient and frame buffers must be 16-byte aligned device pointers");
  jt_view v{};
  if (g) v.g = *g;
  std::memset(&a, 0, sizeof a);
  jt_status s = make_views(c, &v, 1, false, a.views);
  if (s != JT_OK) return s;
  a.tl = lookup(c);
  a.slot = c->slot;
  a.work = c->work;
  a.coef_gid_base = c->coef_gid_base;
  a.coef_mcus = (uint32_t)((uint64_t)c->coef_count * (c->coef_w / 16) * (c->coef_h / 16));
  a.tile_cap = c->float_tile_cap;
  a.bucket_cnt = c->bucket_cnt;
  a.bucket_off = c->bucket_off;
  a.bucket_bsum = c->bucket_bsum;
  a.state = c->state;
  // orthonormal 8-point DCT-III basis, A[x][u] = C(u)/2 cos((2x+1) u pi / 16)
  const double pi = 3.14159265358979323846;
  for (int x = 0; x < 8; ++x)
    for (int u = 0; u < 8; ++u)
      a.basis[x * 8 + u] = (float)((u == 0 ? std::sqrt(0.5) : 1.0) * 0.5 * std::cos((2 * x + 1) * u * pi / 16.0));
  return JT_OK;
}

// Needed set of the coefficient textures (bilinear taps) and its compaction, then the
// buckets' room (a pixel's taps touch at most four MCUs; grown, stream-ordered, when a larger
// view comes) and their zeroed counts.
jt_status enqueue_float_needed(jt_ctx* c, FloatArgs& a, cudaStream_t st) {
  jt_status s;
  const uint64_t need = 4ull * a.views.v[0].width * a.views.v[0].height;
  if (need > c->bucket_cap) {
    JT_CUDA(c, cudaStreamSynchronize(st));
    dev_free(c->bucket);
    c->bucket_cap = 0;
    if ((s = dev_alloc(c, &c->bucket, std::max<uint64_t>(need, 1) * 32)) != JT_OK) return s;
    c->bucket_cap = need;
  }
  a.bucket = c->bucket;
  a.bucket_cap = (uint32_t)std::min<uint64_t>(c->bucket_cap, 0xFFFFFFFFull);
  if ((s = enqueue_mark(c, a.views, JT_FILTER_BILINEAR, -1, 1, st)) != JT_OK) return s;
  if ((s = enqueue_scan(c, c->coef_gid_base, (uint64_t)c->coef_gid_base + a.coef_mcus, st)) != JT_OK) return s;
  JT_CUDA(c, cudaMemsetAsync(c->bucket_cnt, 0, ((size_t)c->float_tile_cap + 1) * 4, st));
  return JT_OK;
}

}  // namespace

extern "C" {

const char* jt_status_string(jt_status s) {
  switch (s) {
    case JT_OK: return "ok";
    case JT_ERR_INVALID_ARG: return "invalid argument";
    case JT_ERR_CUDA: return "CUDA error";
    case JT_ERR_OOM: return "out of device memory";
    case JT_ERR_CORRUPT_STREAM: return "corrupt entropy-coded stream";
    case JT_ERR_CAPACITY: return "block cache capacity exceeded";
    case JT_ERR_UNSUPPORTED: return "unsupported";
    case JT_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

const char* jt_last_error(const jt_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

jt_status jt_create(jt_ctx** out, int device, uint64_t max_cache_blocks) {
  if (!out) return JT_ERR_INVALID_ARG;
  *out = nullptr;
  if (max_cache_blocks == 0 || max_cache_blocks * 4 > kMaxUnits) return JT_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return JT_ERR_CUDA;
  }
  DeviceGuard g(device);
  if (!g.ok) return JT_ERR_CUDA;
  jt_ctx* c = new jt_ctx();
  c->device = device;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    delete c;
    return JT_ERR_CUDA;
  }
  c->sm_count = prop.multiProcessorCount;
  // the kernel's IDCT constants must be round(8192 cos(k pi / 16))
  int kc[8];
  idct_constants(kc);
  for (int k = 1; k < 8; ++k)
    if (kc[k] != (int)std::lround(8192.0 * std::cos(k * M_PI / 16.0))) {
      delete c;
      return JT_ERR_UNSUPPORTED;
    }
  for (int M : kMcusPerWarp)
    for (int W = 1; W <= 16; ++W) c->decode_occ[M][W] = decode_max_ctas_per_sm(W, M);
  cudaGetLastError();
  c->tuning.decode_mcus_per_warp = 32;
  c->tuning.decode_warps = 4;
  c->tuning.decode_ctas_per_sm = std::max(1, c->decode_occ[32][4]);
  c->tuning.pixel_threads = 256;
  c->tuning.pixel_ctas_per_sm = 8;
  c->tuning.decode_short_lists = -1;
  c->cap_units = max_cache_blocks * 4;
  if (dev_alloc(c, &c->cache, c->cap_units * kUnitBytes) != JT_OK || dev_alloc(c, &c->state, sizeof(FrameState)) != JT_OK ||
      cudaMemset(c->state, 0, sizeof(FrameState)) != cudaSuccess || cudaMemset(c->cache, 0, c->cap_units * kUnitBytes) != cudaSuccess ||
      grow_frame_buffers(c, 4096) != JT_OK || sync_tables(c) != JT_OK) {
    jt_destroy(c);
    return JT_ERR_OOM;
  }
  c->map_ntex = 0;
  if (sync_descs(c) != JT_OK) {
    jt_destroy(c);
    return JT_ERR_OOM;
  }
  *out = c;
  return JT_OK;
}

jt_status jt_destroy(jt_ctx* c) {
  if (!c) return JT_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  cudaDeviceSynchronize();
  for (Level& l : c->levels) {
    if (l.stream_mem) cudaFree(l.stream_mem);
    if (l.index_mem) cudaFree(l.index_mem);
    if (l.du_mem) cudaFree(l.du_mem);
  }
  dev_free(c->d_descs);
  dev_free(c->d_map);
  dev_free(c->d_lrec);
  dev_free(c->d_prec);
  dev_free(c->d_huff);
  dev_free(c->d_quant);
  dev_free(c->flags);
  dev_free(c->slot);
  dev_free(c->work);
  dev_free(c->tile_status);
  dev_free(c->cache);
  dev_free(c->d_desc_of_gid);
  cache_free(c);
  dev_free(c->state);
  dev_free(c->bucket_cnt);
  dev_free(c->bucket_off);
  dev_free(c->bucket_bsum);
  dev_free(c->bucket);
  dev_free(c->raster_buf);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  for (cudaEvent_t& e : c->prof)
    if (e) cudaEventDestroy(e);
  delete c;
  return JT_OK;
}

jt_status jt_profile(jt_ctx* c, int enable) {
  if (!c) return JT_ERR_INVALID_ARG;
  DeviceGuard dg(c->device);
  if (enable && !c->prof[0])
    for (cudaEvent_t& e : c->prof) JT_CUDA(c, cudaEventCreate(&e));
  c->profiling = enable != 0;
  return JT_OK;
}

jt_status jt_profile_read(jt_ctx* c, float ms[4]) {
  if (!c || !ms) return JT_ERR_INVALID_ARG;
  if (!c->prof[0]) return fail(c, JT_ERR_STATE, "profiling was never enabled");
  DeviceGuard dg(c->device);
  JT_CUDA(c, cudaEventSynchronize(c->prof[4]));
  for (int i = 0; i < 4; ++i) JT_CUDA(c, cudaEventElapsedTime(&ms[i], c->prof[i], c->prof[i + 1]));
  return JT_OK;
}

// The screen passes' record of an uploaded level (see PixRec).
static PixRec pix_rec(const DevDesc& d) {
  PixRec p{};
  p.gid_base = d.gid_base;
  p.wf = (float)d.width;
  p.hf = (float)d.height;
  p.masks = (uint32_t)(d.width - 1) | ((uint32_t)(d.height - 1) << 16);
  p.mcus_x = d.mcus_x;
  p.shift = (d.sampling == kSampling444 ? 3u : 4u) - d.reduce;
  p.info = (uint32_t)d.units | (d.sampling == kSamplingCoef ? kPixCoef : kPixJpeg) |
           (pow2(d.width) && pow2(d.height) ? kPixPow2 : 0u);
  p.wh = (uint32_t)d.width | ((uint32_t)d.height << 16);
  return p;
}

static jt_status add_level(jt_ctx* c, int tex_id, int level, DevDesc d, Level L) {
  if ((uint32_t)tex_id >= c->map_ntex) {
    uint32_t n = std::max<uint32_t>((uint32_t)tex_id + 1, c->map_ntex * 2);
    n = std::min<uint32_t>(n, 0xFFFF);
    c->map.resize((size_t)n * JT_MAX_LEVELS, -1);
    c->lrec.resize((size_t)n * JT_MAX_LEVELS, LevelRec{0, 0, 0, 0});
    c->prec.assign((size_t)n * JT_MAX_LEVELS + 1, PixRec{});
    for (size_t i = 0; i < c->descs.size(); ++i) c->prec[(size_t)c->levels[i].tex * JT_MAX_LEVELS + c->levels[i].level] = pix_rec(c->descs[i]);
    c->map_ntex = n;
  }
  c->map[(size_t)tex_id * JT_MAX_LEVELS + level] = (int32_t)c->descs.size();
  LevelRec& r = c->lrec[(size_t)tex_id * JT_MAX_LEVELS + level];
  r.gid_base = d.gid_base;
  r.wh = (uint32_t)d.width | ((uint32_t)d.height << 16);
  r.info = level_info(d.mcus_x, (d.sampling == kSampling444 ? 3u : 4u) - d.reduce, d.units, d.sampling, pow2(d.width),
                      pow2(d.height));
  r.pad = 0;
  c->prec[(size_t)tex_id * JT_MAX_LEVELS + level] = pix_rec(d);
  c->descs.push_back(d);
  c->levels.push_back(L);
  const uint64_t g0 = c->ngid;
  c->ngid += d.nmcu;
  jt_status s = grow_frame_buffers(c, c->ngid);
  if (s != JT_OK) return s;
  // gid -> descriptor index for the new level's MCUs
  if (c->ngid > c->desc_of_gid_cap) {
    const uint64_t cap = std::max<uint64_t>(c->ngid, c->desc_of_gid_cap * 2);
    uint32_t* nb = nullptr;
    if ((s = dev_alloc(c, &nb, cap * 4)) != JT_OK) return s;
    if (g0) JT_CUDA(c, cudaMemcpy(nb, c->d_desc_of_gid, g0 * 4, cudaMemcpyDeviceToDevice));
    dev_free(c->d_desc_of_gid);
    c->d_desc_of_gid = nb;
    c->desc_of_gid_cap = cap;
  }
  {
    const std::vector<uint32_t> di(d.nmcu, (uint32_t)(c->descs.size() - 1));
    JT_CUDA(c, cudaMemcpy(c->d_desc_of_gid + g0, di.data(), (size_t)d.nmcu * 4, cudaMemcpyHostToDevice));
  }
  return sync_descs(c);
}

// Shared by both texture forms: checks, tables, device copies of the stream and of the side
// table (side_bytes of `side`, already in the device layout), descriptor.
static jt_status upload_level(jt_ctx* c, int tex_id, int level, int width, int height, int sampling,
                              const uint8_t* bitstream, uint64_t nbytes, uint64_t nbits, const void* side,
                              uint64_t side_bytes, uint64_t nblocks, bool compact, const uint16_t* qt,
                              const jt_huff_spec huff[4]) {
  if (c->phase == Phase::Marked) return fail(c, JT_ERR_STATE, "upload between jt_mark and jt_decode");
  if (tex_id < 0 || tex_id >= 0xFFFF || level < 0 || level >= JT_MAX_LEVELS)
    return fail(c, JT_ERR_INVALID_ARG, "texture id %d / level %d out of range", tex_id, level);
  if (width <= 0 || height <= 0 || width > 65535 || height > 65535)
    return fail(c, JT_ERR_INVALID_ARG, "bad size %dx%d", width, height);
  if (sampling != 420 && sampling != 444) return fail(c, JT_ERR_INVALID_ARG, "sampling must be 420 or 444");
  if (!bitstream || !side || !qt || !huff) return fail(c, JT_ERR_INVALID_ARG, "null upload pointer");
  if (nbits > nbytes * 8 || nbytes >= (1ull << 29)) return fail(c, JT_ERR_INVALID_ARG, "bad stream size");
  if ((uint32_t)tex_id < c->map_ntex && c->map[(size_t)tex_id * JT_MAX_LEVELS + level] >= 0)
    return fail(c, JT_ERR_INVALID_ARG, "texture %d level %d already uploaded", tex_id, level);
  const int mw = sampling == 420 ? 16 : 8;
  const uint64_t mx = (width + mw - 1) / mw, my = (height + mw - 1) / mw;
  if (nblocks != mx * my) return fail(c, JT_ERR_INVALID_ARG, "index has %llu entries, expected %llu",
                                      (unsigned long long)nblocks, (unsigned long long)(mx * my));
  if (c->ngid + nblocks > kMaxGids) return fail(c, JT_ERR_UNSUPPORTED, "more than 2^26 MCUs in one context");
  DeviceGuard g(c->device);
  if (!g.ok) return fail(c, JT_ERR_CUDA, "cannot select device %d", c->device);

  // decode tables (deduplicated by content)
  HuffSet hs;
  std::string why;
  for (int t = 0; t < 4; ++t)
    if (!build_table(huff[t], t % 2 == 0, hs.t[t], why))
      return fail(c, JT_ERR_INVALID_ARG, "Huffman table %d: %s", t, why.c_str());
  int hset = -1;
  for (size_t i = 0; i < c->hsets.size(); ++i)
    if (std::memcmp(&c->hsets[i], &hs, sizeof hs) == 0) hset = (int)i;
  int nat[64];
  zigzag_natural(nat);
  std::vector<uint16_t> qz(128);
  for (int comp = 0; comp < 2; ++comp)
    for (int k = 0; k < 64; ++k) qz[comp * 64 + k] = qt[comp * 64 + nat[k]];
  int qset = -1;
  for (size_t i = 0; i < c->qsets.size(); ++i)
    if (c->qsets[i] == qz) qset = (int)i;
  bool tables_changed = false;
  if (hset < 0) {
    if (c->hsets.size() >= 255) return fail(c, JT_ERR_UNSUPPORTED, "more than 255 distinct Huffman table sets");
    c->hsets.push_back(hs);
    hset = (int)c->hsets.size() - 1;
    tables_changed = true;
  }
  if (qset < 0) {
    if (c->qsets.size() >= 255) return fail(c, JT_ERR_UNSUPPORTED, "more than 255 distinct quantisation tables");
    c->qsets.push_back(qz);
    qset = (int)c->qsets.size() - 1;
    tables_changed = true;
  }
  if (tables_changed) {
    jt_status s = sync_tables(c);
    if (s != JT_OK) return s;
  }

  // stream words (zero padded) and side table
  Level L{tex_id, level};
  const uint64_t words = (nbytes + 3) / 4 + kStreamPadBytes / 4;
  jt_status s;
  if ((s = dev_alloc(c, reinterpret_cast<uint8_t**>(&L.stream_mem), words * 4)) != JT_OK) return s;
  if ((s = dev_alloc(c, reinterpret_cast<uint8_t**>(&L.index_mem), side_bytes + 16)) != JT_OK) {
    cudaFree(L.stream_mem);
    return s;
  }
  if (cudaMemset(L.stream_mem, 0, words * 4) != cudaSuccess ||
      cudaMemcpy(L.stream_mem, bitstream, nbytes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(L.index_mem, side, side_bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(L.stream_mem);
    cudaFree(L.index_mem);
    return fail(c, JT_ERR_CUDA, "upload copy failed");
  }
  DevDesc d{};
  d.stream = static_cast<const uint32_t*>(L.stream_mem);
  d.index = static_cast<const uint16_t*>(L.index_mem);
  d.gid_base = (uint32_t)c->ngid;
  d.nmcu = (uint32_t)nblocks;
  d.nwords = (uint32_t)words;
  d.nbits = (uint32_t)nbits;
  d.width = (uint16_t)width;
  d.height = (uint16_t)height;
  d.mcus_x = (uint16_t)mx;
  d.mcus_y = (uint16_t)my;
  d.sampling = sampling == 420 ? kSampling420 : kSampling444;
  d.units = sampling == 420 ? 4 : 1;
  d.hset = (uint8_t)hset;
  d.qset = (uint8_t)qset;
  d.compact = compact ? 1 : 0;
  return add_level(c, tex_id, level, d, L);
}

jt_status jt_upload_texture(jt_ctx* c, int tex_id, int level, int width, int height, int sampling,
                            const uint8_t* bitstream, uint64_t nbytes, uint64_t nbits, const jt_block_index* index,
                            uint64_t nblocks, const uint16_t* qt, const jt_huff_spec huff[4]) {
  if (!c) return JT_ERR_INVALID_ARG;
  return upload_level(c, tex_id, level, width, height, sampling, bitstream, nbytes, nbits, index,
                      nblocks * sizeof(jt_block_index), nblocks, false, qt, huff);
}

jt_status jt_upload_texture_compact(jt_ctx* c, int tex_id, int level, int width, int height, int sampling,
                                    const uint8_t* stream, uint64_t nbytes, const uint32_t* abs_offsets,
                                    const uint16_t* rel_offsets, const uint32_t* dc_records, uint64_t nblocks,
                                    const uint16_t* qt, const jt_huff_spec huff[4]) {
  if (!c) return JT_ERR_INVALID_ARG;
  if (!abs_offsets || !rel_offsets || !dc_records) return fail(c, JT_ERR_INVALID_ARG, "null upload pointer");
  if (nblocks == 0 || nblocks > kMaxGids) return fail(c, JT_ERR_INVALID_ARG, "bad MCU count");
  // MCU starts must be non-decreasing and inside the stream
  const uint64_t ng = (nblocks + 8) / 9;
  uint64_t prev = 0;
  for (uint64_t m = 0; m < nblocks; ++m) {
    const uint64_t j = m / 9, i = m % 9;
    const uint64_t st = (uint64_t)abs_offsets[j] + (i ? rel_offsets[8 * j + i - 1] : 0u);
    if (st < prev || st > nbytes)
      return fail(c, JT_ERR_INVALID_ARG, "MCU %llu starts at byte %llu (previous %llu, stream %llu)",
                  (unsigned long long)m, (unsigned long long)st, (unsigned long long)prev,
                  (unsigned long long)nbytes);
    prev = st;
  }
  // device layout: [abs x ng][rel x 8 ng][DC records + one zero word]
  const uint64_t ndc = (36 * nblocks + 31) / 32;
  std::vector<uint32_t> side(ng + 4 * ng + ndc + 1, 0u);
  std::memcpy(side.data(), abs_offsets, ng * 4);
  std::memcpy(side.data() + ng, rel_offsets, ng * 16);
  std::memcpy(side.data() + 5 * ng, dc_records, ndc * 4);
  return upload_level(c, tex_id, level, width, height, sampling, stream, nbytes, nbytes * 8, side.data(),
                      side.size() * 4, nblocks, true, qt, huff);
}

jt_status jt_set_du_offsets(jt_ctx* c, int tex_id, int level, const uint16_t* du_offsets, uint64_t count) {
  if (!c) return JT_ERR_INVALID_ARG;
  if (c->phase == Phase::Marked) return fail(c, JT_ERR_STATE, "upload between jt_mark and jt_decode");
  if (tex_id < 0 || tex_id >= 0xFFFF || level < 0 || level >= JT_MAX_LEVELS || !du_offsets)
    return fail(c, JT_ERR_INVALID_ARG, "bad texture id, level or pointer");
  const int di = (uint32_t)tex_id < c->map_ntex ? c->map[(size_t)tex_id * JT_MAX_LEVELS + level] : -1;
  if (di < 0) return fail(c, JT_ERR_INVALID_ARG, "texture %d level %d is not uploaded", tex_id, level);
  DevDesc& d = c->descs[di];
  if (d.sampling == kSamplingCoef || d.compact || d.reduce)
    return fail(c, JT_ERR_INVALID_ARG, "texture %d level %d is not a standard-form stored level", tex_id, level);
  const int ndu = d.sampling == kSampling420 ? 6 : 3;
  if (count != (uint64_t)d.nmcu * (ndu - 1))
    return fail(c, JT_ERR_INVALID_ARG, "%llu offsets, expected %llu", (unsigned long long)count,
                (unsigned long long)d.nmcu * (ndu - 1));
  for (uint64_t m = 0; m < d.nmcu; ++m)  // starts must not decrease inside an MCU
    for (int i = 1; i < ndu - 1; ++i)
      if (du_offsets[m * (ndu - 1) + i] < du_offsets[m * (ndu - 1) + i - 1])
        return fail(c, JT_ERR_INVALID_ARG, "MCU %llu: data-unit starts decrease", (unsigned long long)m);
  DeviceGuard g(c->device);
  if (!g.ok) return fail(c, JT_ERR_CUDA, "cannot select device %d", c->device);
  Level& L = c->levels[di];
  if (L.du_mem) {
    cudaFree(L.du_mem);
    L.du_mem = nullptr;
  }
  jt_status s;
  if ((s = dev_alloc(c, reinterpret_cast<uint8_t**>(&L.du_mem), count * 2 + 16)) != JT_OK) return s;
  JT_CUDA(c, cudaMemcpy(L.du_mem, du_offsets, count * 2, cudaMemcpyHostToDevice));
  // the level and the reduced levels decoded from it (they share its stream)
  for (DevDesc& o : c->descs)
    if (o.stream == d.stream) o.du_index = static_cast<const uint16_t*>(L.du_mem);
  c->unit_mode = true;
  return sync_descs(c);
}

jt_status jt_add_reduced_level(jt_ctx* c, int tex_id, int src_level, int reduce, int level) {
  if (!c) return JT_ERR_INVALID_ARG;
  if (c->phase == Phase::Marked) return fail(c, JT_ERR_STATE, "upload between jt_mark and jt_decode");
  if (reduce < 1 || reduce > 3) return fail(c, JT_ERR_INVALID_ARG, "reduce must be 1, 2 or 3");
  if (tex_id < 0 || tex_id >= 0xFFFF || src_level < 0 || src_level >= JT_MAX_LEVELS || level < 0 ||
      level >= JT_MAX_LEVELS)
    return fail(c, JT_ERR_INVALID_ARG, "texture id %d / level %d / %d out of range", tex_id, src_level, level);
  const int si = (uint32_t)tex_id < c->map_ntex ? c->map[(size_t)tex_id * JT_MAX_LEVELS + src_level] : -1;
  if (si < 0) return fail(c, JT_ERR_INVALID_ARG, "texture %d level %d is not uploaded", tex_id, src_level);
  const DevDesc& src = c->descs[si];
  if (src.sampling == kSamplingCoef || src.reduce != 0)
    return fail(c, JT_ERR_INVALID_ARG, "texture %d level %d is not a stored JPEG level", tex_id, src_level);
  if (c->map[(size_t)tex_id * JT_MAX_LEVELS + level] >= 0)
    return fail(c, JT_ERR_INVALID_ARG, "texture %d level %d already exists", tex_id, level);
  if (c->ngid + src.nmcu > kMaxGids) return fail(c, JT_ERR_UNSUPPORTED, "more than 2^26 MCUs in one context");
  DeviceGuard g(c->device);
  if (!g.ok) return fail(c, JT_ERR_CUDA, "cannot select device %d", c->device);
  DevDesc d = src;  // same stream, index and tables; the source level owns the memory
  d.gid_base = (uint32_t)c->ngid;
  d.width = (uint16_t)std::max(1, (int)src.width >> reduce);
  d.height = (uint16_t)std::max(1, (int)src.height >> reduce);
  d.units = 1;  // at most 8 x 8 texels
  d.reduce = (uint8_t)reduce;
  return add_level(c, tex_id, level, d, Level{tex_id, level});
}

static_assert(sizeof(jt_scene_quad) == sizeof(SceneQuad), "jt_scene_quad layout");
static_assert(sizeof(jt_scene) == 144, "jt_scene layout");

jt_status jt_raster_scene(jt_ctx* c, const jt_scene* sc, const jt_gbuffer* out, jt_stream stream) {
  if (!c) return JT_ERR_INVALID_ARG;
  if (!sc || !out) return fail(c, JT_ERR_INVALID_ARG, "null scene or G-buffer");
  if (sc->width <= 0 || sc->height <= 0 || out->width != sc->width || out->height != sc->height)
    return fail(c, JT_ERR_INVALID_ARG, "G-buffer %dx%d does not match the scene's %dx%d", out->width, out->height,
                sc->width, sc->height);
  if (!out->uv || !out->tex_id || !out->mip) return fail(c, JT_ERR_INVALID_ARG, "null G-buffer pointer");
  if (sc->ntex <= 0 || sc->ntex > 0xFFFF || !sc->tex_w || !sc->tex_h || !sc->tex_levels)
    return fail(c, JT_ERR_INVALID_ARG, "bad texture table");
  if (sc->nquads < 0 || sc->nquads > kMaxSceneQuads || (sc->nquads > 0 && !sc->quads))
    return fail(c, JT_ERR_INVALID_ARG, "bad quad list (%d quads, at most %d)", sc->nquads, kMaxSceneQuads);
  for (int t = 0; t < sc->ntex; ++t)
    if (sc->tex_levels[t] < 1 || sc->tex_levels[t] > JT_MAX_LEVELS || sc->tex_w[t] <= 0 || sc->tex_h[t] <= 0)
      return fail(c, JT_ERR_INVALID_ARG, "texture %d: bad size or level count", t);
  for (int n = 0; n < sc->nquads; ++n)
    if (sc->quads[n].tex < 0 || sc->quads[n].tex >= sc->ntex)
      return fail(c, JT_ERR_INVALID_ARG, "quad %d names texture %d", n, sc->quads[n].tex);
  DeviceGuard dg(c->device);
  if (!dg.ok) return fail(c, JT_ERR_CUDA, "cannot select device %d", c->device);
  // device copies of the texture table and the quads: [w][h][levels] x ntex, then quads
  const size_t tbytes = (size_t)sc->ntex * 4, qoff = (3 * tbytes + 15) & ~(size_t)15;
  const size_t need = qoff + (size_t)sc->nquads * sizeof(SceneQuad);
  if (need > c->raster_cap) {
    dev_free(c->raster_buf);
    c->raster_buf = nullptr;
    c->raster_cap = 0;
    jt_status s = dev_alloc(c, &c->raster_buf, need);
    if (s != JT_OK) return s;
    c->raster_cap = need;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  JT_CUDA(c, cudaMemcpyAsync(c->raster_buf, sc->tex_w, tbytes, cudaMemcpyHostToDevice, st));
  JT_CUDA(c, cudaMemcpyAsync(c->raster_buf + tbytes, sc->tex_h, tbytes, cudaMemcpyHostToDevice, st));
  JT_CUDA(c, cudaMemcpyAsync(c->raster_buf + 2 * tbytes, sc->tex_levels, tbytes, cudaMemcpyHostToDevice, st));
  if (sc->nquads)
    JT_CUDA(c, cudaMemcpyAsync(c->raster_buf + qoff, sc->quads, (size_t)sc->nquads * sizeof(SceneQuad),
                               cudaMemcpyHostToDevice, st));
  RasterArgs a{};
  a.width = sc->width;
  a.height = sc->height;
  std::memcpy(a.cam, sc->cam, sizeof a.cam);
  std::memcpy(a.rot, sc->rot, sizeof a.rot);
  a.ax = sc->ax;
  a.ay = sc->ay;
  a.tan_x = sc->tan_x;
  a.tan_y = sc->tan_y;
  a.max_t = sc->max_t;
  a.kx = sc->kx;
  a.ky = sc->ky;
  a.shift = sc->shift;
  a.cell_seed = sc->cell_seed;
  a.ntex = sc->ntex;
  a.use_mips = sc->use_mips;
  a.nquads = sc->nquads;
  a.tex_w = reinterpret_cast<const int32_t*>(c->raster_buf);
  a.tex_h = reinterpret_cast<const int32_t*>(c->raster_buf + tbytes);
  a.tex_levels = reinterpret_cast<const int32_t*>(c->raster_buf + 2 * tbytes);
  a.quads = reinterpret_cast<const SceneQuad*>(c->raster_buf + qoff);
  // the G-buffer record is declared read-only for the passes that consume it; here it is
  // the output
  a.uv = reinterpret_cast<float2*>(const_cast<float*>(out->uv));
  a.tex = const_cast<uint16_t*>(out->tex_id);
  a.mip = const_cast<uint8_t*>(out->mip);
  launch_raster(a, st);
  JT_CUDA(c, cudaGetLastError());
  c->last_stream = st;
  return JT_OK;
}

jt_status jt_mark(jt_ctx* c, const jt_gbuffer* g, int filter, jt_stream stream) {
  if (!c) return JT_ERR_INVALID_ARG;
  if (!valid_filter(filter)) return fail(c, JT_ERR_INVALID_ARG, "bad filter %d", filter);
  jt_view v{};
  if (g) v.g = *g;
  ViewSet vs;
  jt_status s = make_views(c, &v, 1, false, vs);
  if (s != JT_OK) return s;
  DeviceGuard dg(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((s = enqueue_mark(c, vs, filter, -1, 0, st)) != JT_OK) return s;
  c->phase = Phase::Marked;
  c->last_stream = st;
  return JT_OK;
}

jt_status jt_decode(jt_ctx* c, jt_stream stream) {
  if (!c) return JT_ERR_INVALID_ARG;
  if (c->phase != Phase::Marked) return fail(c, JT_ERR_STATE, "jt_decode needs a preceding jt_mark");
  DeviceGuard dg(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  jt_status s;
  if ((s = enqueue_compact(c, st)) != JT_OK) return s;
  if ((s = enqueue_decode(c, st)) != JT_OK) return s;
  c->phase = Phase::Decoded;
  c->last_stream = st;
  return JT_OK;
}

jt_status jt_colorize(jt_ctx* c, const jt_gbuffer* g, int filter, uint8_t* out_rgba, jt_stream stream) {
  if (!c) return JT_ERR_INVALID_ARG;
  if (c->phase != Phase::Decoded) return fail(c, JT_ERR_STATE, "jt_colorize needs a preceding jt_decode");
  if (!valid_filter(filter)) return fail(c, JT_ERR_INVALID_ARG, "bad filter %d", filter);
  jt_view v{};
  if (g) v.g = *g;
  v.out_rgba = out_rgba;
  ViewSet vs;
  jt_status s = make_views(c, &v, 1, true, vs);
  if (s != JT_OK) return s;
  DeviceGuard dg(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((s = enqueue_colorize(c, vs, filter, -1, st)) != JT_OK) return s;
  c->last_stream = st;
  return JT_OK;
}

jt_status jt_get_stats(jt_ctx* c, jt_stats* out) {
  if (!c || !out) return JT_ERR_INVALID_ARG;
  DeviceGuard dg(c->device);
  JT_CUDA(c, cudaStreamSynchronize(c->last_stream));
  FrameState fs;
  JT_CUDA(c, cudaMemcpy(&fs, c->state, sizeof fs, cudaMemcpyDeviceToHost));
  JT_CUDA(c, cudaMemset(&c->state->err, 0, sizeof(uint32_t)));
  JT_CUDA(c, cudaDeviceSynchronize());
  out->needed_blocks = fs.count;
  out->cache_units = fs.units;
  out->capacity_units = c->cap_units;
  out->total_blocks = c->ngid;
  out->levels = (uint32_t)c->descs.size();
  out->error_bits = fs.err;
  out->visible_blocks = fs.count;
  out->resident_blocks = 0;
  out->evicted_blocks = 0;
  if (c->persistent && c->cstate) {
    CacheState cs;
    JT_CUDA(c, cudaMemcpy(&cs, c->cstate, sizeof cs, cudaMemcpyDeviceToHost));
    JT_CUDA(c, cudaMemset(&c->cstate->evicted, 0, sizeof(uint32_t)));
    out->visible_blocks = cs.visible;
    out->resident_blocks = c->nblocks - cs.free_count;
    out->evicted_blocks = cs.evicted;
  }
  if (fs.err & JT_DEVERR_CORRUPT) return fail(c, JT_ERR_CORRUPT_STREAM, "corrupt entropy-coded data in a needed MCU");
  if (fs.err & JT_DEVERR_CAPACITY) return fail(c, JT_ERR_CAPACITY, "needed %u cache units, capacity %llu", fs.units,
                                              (unsigned long long)c->cap_units);
  if (fs.err & JT_DEVERR_MISSING) return fail(c, JT_ERR_UNSUPPORTED, "a pixel names a texture level that was not uploaded");
  if (fs.err & JT_DEVERR_TIMEOUT) return fail(c, JT_ERR_CUDA, "compaction wait timed out");
  return JT_OK;
}

jt_status jt_frame(jt_ctx* c, const jt_view* views, int nviews, int filter, jt_stream stream) {
  if (!c) return JT_ERR_INVALID_ARG;
  if (!valid_filter(filter)) return fail(c, JT_ERR_INVALID_ARG, "bad filter %d", filter);
  if (c->phase == Phase::Marked) return fail(c, JT_ERR_STATE, "a marked frame is pending");
  ViewSet vs;
  jt_status s = make_views(c, views, nviews, true, vs);
  if (s != JT_OK) return s;
  DeviceGuard dg(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((s = enqueue_frame(c, vs, filter, st)) != JT_OK) return s;
  c->phase = Phase::Decoded;
  c->last_stream = st;
  return JT_OK;
}

jt_status jt_frame_graph(jt_ctx* c, const jt_view* views, int nviews, int filter, jt_stream stream, jt_graph** out) {
  if (!c || !out) return JT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!valid_filter(filter)) return fail(c, JT_ERR_INVALID_ARG, "bad filter %d", filter);
  if (c->phase == Phase::Marked) return fail(c, JT_ERR_STATE, "a marked frame is pending");
  ViewSet vs;
  jt_status s = make_views(c, views, nviews, true, vs);
  if (s != JT_OK) return s;
  if (c->descs.empty()) return fail(c, JT_ERR_STATE, "no textures uploaded");
  DeviceGuard dg(c->device);
  if (c->persistent && c->resident_ngid != c->ngid) {  // levels uploaded since: start the cache over
    s = cache_reset(c);                                // here, since no allocation may run in a capture
    if (s != JT_OK) return s;
  }
  if (!c->capture_stream) JT_CUDA(c, cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
  cudaStream_t cs = c->capture_stream;
  // capture on the context's own stream (the caller's may be the legacy default stream)
  JT_CUDA(c, cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  JT_CUDA(c, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  s = enqueue_frame(c, vs, filter, cs);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &graph);
  if (s != JT_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return fail(c, JT_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  jt_graph* gr = new jt_graph();
  gr->ctx = c;
  gr->graph = graph;
  gr->generation = c->generation;
  e = cudaGraphInstantiate(&gr->exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    delete gr;
    return fail(c, JT_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  *out = gr;
  return JT_OK;
}

jt_status jt_graph_launch(jt_graph* g, jt_stream stream) {
  if (!g || !g->exec) return JT_ERR_INVALID_ARG;
  jt_ctx* c = g->ctx;
  if (c->phase == Phase::Marked) return fail(c, JT_ERR_STATE, "a marked frame is pending");
  if (g->generation != c->generation)
    return fail(c, JT_ERR_STATE, "the context's tables moved since the graph was captured (an upload or a "
                                 "block-cache switch): capture it again");
  DeviceGuard dg(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  JT_CUDA(c, cudaGraphLaunch(g->exec, st));
  c->phase = Phase::Decoded;
  c->last_stream = st;
  return JT_OK;
}

jt_status jt_graph_destroy(jt_graph* g) {
  if (!g) return JT_ERR_INVALID_ARG;
  DeviceGuard dg(g->ctx->device);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
  return JT_OK;
}

jt_status jt_frame_plain(jt_ctx* c, const jt_view* views, int nviews, int filter, jt_stream stream) {
  if (!c) return JT_ERR_INVALID_ARG;
  if (!valid_filter(filter)) return fail(c, JT_ERR_INVALID_ARG, "bad filter %d", filter);
  if (c->phase == Phase::Marked) return fail(c, JT_ERR_STATE, "a marked frame is pending");
  if (c->descs.empty()) return fail(c, JT_ERR_STATE, "no textures uploaded");
  if (c->persistent) return fail(c, JT_ERR_STATE, "the per-texture pipeline needs the per-frame cache mode");
  ViewSet all;
  jt_status s = make_views(c, views, nviews, true, all);
  if (s != JT_OK) return s;
  DeviceGuard dg(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // gid range of each texture id (over its levels)
  std::map<int, std::pair<uint64_t, uint64_t>> ranges;
  for (size_t i = 0; i < c->descs.size(); ++i) {
    if (c->descs[i].sampling == kSamplingCoef) continue;
    const uint64_t lo = c->descs[i].gid_base, hi = lo + c->descs[i].nmcu;
    auto it = ranges.find(c->levels[i].tex);
    if (it == ranges.end())
      ranges[c->levels[i].tex] = {lo, hi};
    else
      it->second = {std::min(it->second.first, lo), std::max(it->second.second, hi)};
  }
  for (int v = 0; v < nviews; ++v) {
    ViewSet one;
    if ((s = make_views(c, views + v, 1, true, one)) != JT_OK) return s;
    if ((s = enqueue_colorize(c, one, filter, JT_EMPTY_TEXTURE, st)) != JT_OK) return s;
    for (const auto& kv : ranges) {
      if ((s = enqueue_mark(c, one, filter, kv.first, 0, st)) != JT_OK) return s;
      if ((s = enqueue_scan(c, kv.second.first, kv.second.second, st)) != JT_OK) return s;
      if ((s = enqueue_decode(c, st)) != JT_OK) return s;
      if ((s = enqueue_colorize(c, one, filter, kv.first, st)) != JT_OK) return s;
    }
  }
  c->phase = Phase::Decoded;
  c->last_stream = st;
  return JT_OK;
}

jt_status jt_get_tuning(const jt_ctx* c, jt_tuning* out) {
  if (!c || !out) return JT_ERR_INVALID_ARG;
  *out = c->tuning;
  return JT_OK;
}

jt_status jt_set_tuning(jt_ctx* c, const jt_tuning* t) {
  if (!c || !t) return JT_ERR_INVALID_ARG;
  if (!valid_tuning(c, *t)) return fail(c, JT_ERR_INVALID_ARG, "invalid tuning");
  c->tuning = *t;
  return JT_OK;
}

jt_status jt_autotune(jt_ctx* c, const jt_view* views, int nviews, int filter, jt_stream stream, int reps,
                      jt_tuning* best, float* best_ms) {
  if (!c) return JT_ERR_INVALID_ARG;
  if (reps < 1 || reps > 1000) return fail(c, JT_ERR_INVALID_ARG, "reps must be 1..1000");
  DeviceGuard dg(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  JT_CUDA(c, cudaEventCreate(&e0));
  JT_CUDA(c, cudaEventCreate(&e1));
  const jt_tuning saved = c->tuning;
  auto measure = [&](const jt_tuning& t, float& ms) -> jt_status {
    c->tuning = t;
    jt_graph* g = nullptr;
    jt_status s = jt_frame_graph(c, views, nviews, filter, stream, &g);
    if (s != JT_OK) return s;
    std::vector<float> times;
    for (int i = 0; i < reps + 2; ++i) {
      cudaEventRecord(e0, st);
      cudaGraphLaunch(g->exec, st);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float t_ms = 0;
      cudaEventElapsedTime(&t_ms, e0, e1);
      if (i >= 2) times.push_back(t_ms);
    }
    jt_graph_destroy(g);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, JT_ERR_CUDA, "autotune run: %s", cudaGetErrorString(e));
    std::sort(times.begin(), times.end());
    ms = times[times.size() / 2];
    return JT_OK;
  };
  jt_tuning cur = saved, top = saved;
  float top_ms = 1e30f;
  jt_status s = JT_OK;
  // stage 1: decode shape (MCUs per warp x warps per CTA at full occupancy, then fewer CTAs)
  for (int M : kMcusPerWarp) {
    for (int W : kDecodeWarps) {
      const int occ = c->decode_occ[M][W];
      if (occ <= 0) continue;
      for (int per : {occ, std::max(1, occ / 2)}) {
        cur = saved;
        cur.decode_mcus_per_warp = M;
        cur.decode_warps = W;
        cur.decode_ctas_per_sm = per;
        float ms;
        if ((s = measure(cur, ms)) != JT_OK) goto done;
        if (ms < top_ms) {
          top_ms = ms;
          top = cur;
        }
        if (occ == 1) break;
      }
    }
  }
  // stage 2: pixel-kernel shape
  for (int th : {128, 256, 512}) {
    for (int per : {4, 8, 16}) {
      if (th * per > 2048 * 2) continue;
      cur = top;
      cur.pixel_threads = th;
      cur.pixel_ctas_per_sm = per;
      float ms;
      if ((s = measure(cur, ms)) != JT_OK) goto done;
      if (ms < top_ms) {
        top_ms = ms;
        top = cur;
      }
    }
  }
done:
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != JT_OK) {
    c->tuning = saved;
    return s;
  }
  c->tuning = top;
  if (best) *best = top;
  if (best_ms) *best_ms = top_ms;
  return JT_OK;
}

jt_status jt_read_work_list(jt_ctx* c, uint32_t* dst, uint64_t cap, uint64_t* count) {
  if (!c || !count) return JT_ERR_INVALID_ARG;
  DeviceGuard dg(c->device);
  JT_CUDA(c, cudaStreamSynchronize(c->last_stream));
  FrameState fs;
  JT_CUDA(c, cudaMemcpy(&fs, c->state, sizeof fs, cudaMemcpyDeviceToHost));
  *count = fs.count;
  const uint64_t n = std::min<uint64_t>({cap, (uint64_t)fs.count, c->gid_cap});
  if (n && dst) JT_CUDA(c, cudaMemcpy(dst, c->work, n * 4, cudaMemcpyDefault));
  return JT_OK;
}

jt_status jt_read_slots(jt_ctx* c, uint64_t gid_begin, uint64_t n, uint32_t* dst) {
  if (!c || (!dst && n)) return JT_ERR_INVALID_ARG;
  if (gid_begin + n > c->ngid) return fail(c, JT_ERR_INVALID_ARG, "gid range beyond the uploaded levels");
  DeviceGuard dg(c->device);
  JT_CUDA(c, cudaStreamSynchronize(c->last_stream));
  if (n) JT_CUDA(c, cudaMemcpy(dst, c->slot + gid_begin, n * 4, cudaMemcpyDefault));
  return JT_OK;
}

jt_status jt_read_cache(jt_ctx* c, uint64_t unit_begin, uint64_t n, uint8_t* dst) {
  if (!c || (!dst && n)) return JT_ERR_INVALID_ARG;
  if (unit_begin + n > c->cap_units) return fail(c, JT_ERR_INVALID_ARG, "unit range beyond the cache");
  DeviceGuard dg(c->device);
  JT_CUDA(c, cudaStreamSynchronize(c->last_stream));
  if (n) JT_CUDA(c, cudaMemcpy(dst, c->cache + unit_begin * kUnitBytes, n * kUnitBytes, cudaMemcpyDefault));
  return JT_OK;
}

jt_status jt_set_block_cache(jt_ctx* c, int persistent) {
  if (!c) return JT_ERR_INVALID_ARG;
  if (persistent != 0 && persistent != 1) return fail(c, JT_ERR_INVALID_ARG, "mode must be 0 or 1");
  if (c->phase == Phase::Marked) return fail(c, JT_ERR_STATE, "a marked frame is pending");
  DeviceGuard dg(c->device);
  JT_CUDA(c, cudaDeviceSynchronize());
  cache_free(c);
  c->persistent = persistent == 1;
  c->phase = Phase::Idle;
  return c->persistent ? cache_reset(c) : JT_OK;
}

// ---- float chain ------------------------------------------------------------------------

jt_status jt_register_coeff_textures(jt_ctx* c, int first_tex_id, int count, int width, int height) {
  if (!c) return JT_ERR_INVALID_ARG;
  if (c->coef_first >= 0) return fail(c, JT_ERR_STATE, "coefficient textures are already registered");
  if (c->phase == Phase::Marked) return fail(c, JT_ERR_STATE, "registration between jt_mark and jt_decode");
  if (count <= 0 || first_tex_id < 0 || (int64_t)first_tex_id + count > 0xFFFF)
    return fail(c, JT_ERR_INVALID_ARG, "texture ids %d..%d out of range", first_tex_id, first_tex_id + count - 1);
  if (width <= 0 || height <= 0 || width % 16 || height % 16 || width > 65520 || height > 65520)
    return fail(c, JT_ERR_INVALID_ARG, "coefficient textures must be multiples of 16 texels, got %dx%d", width,
                height);
  for (int t = first_tex_id; t < first_tex_id + count; ++t)
    if ((uint32_t)t < c->map_ntex && c->map[(size_t)t * JT_MAX_LEVELS] >= 0)
      return fail(c, JT_ERR_INVALID_ARG, "texture %d level 0 already exists", t);
  const uint64_t mx = width / 16, my = height / 16, per = mx * my;
  if (c->ngid + per * count > kMaxGids) return fail(c, JT_ERR_UNSUPPORTED, "more than 2^26 MCUs in one context");
  DeviceGuard dg(c->device);
  if (!dg.ok) return fail(c, JT_ERR_CUDA, "cannot select device %d", c->device);
  const uint64_t cap = std::min<uint64_t>(per * count, c->cap_units / 4);
  jt_status s;
  if ((s = dev_alloc(c, &c->bucket_cnt, (cap + 1) * 4)) != JT_OK) return s;
  if ((s = dev_alloc(c, &c->bucket_off, (cap + 1) * 4)) != JT_OK) return s;
  if ((s = dev_alloc(c, &c->bucket_bsum, ((cap + 1 + kBucketScan - 1) / kBucketScan) * 4)) != JT_OK) return s;
  c->float_tile_cap = (uint32_t)cap;
  c->coef_gid_base = (uint32_t)c->ngid;
  for (int t = 0; t < count; ++t) {
    DevDesc d{};
    d.gid_base = (uint32_t)c->ngid;
    d.nmcu = (uint32_t)per;
    d.width = (uint16_t)width;
    d.height = (uint16_t)height;
    d.mcus_x = (uint16_t)mx;
    d.mcus_y = (uint16_t)my;
    d.sampling = kSamplingCoef;
    d.units = 1;  // one flag unit per MCU: the compaction's slot is the work position
    if ((s = add_level(c, first_tex_id + t, 0, d, Level{first_tex_id + t, 0})) != JT_OK) return s;
  }
  c->coef_first = first_tex_id;
  c->coef_count = count;
  c->coef_w = width;
  c->coef_h = height;
  return JT_OK;
}

jt_status jt_colorize_float(jt_ctx* c, const jt_gbuffer* g, const float* coeffs, float* out_rgb, jt_stream stream) {
  if (!c) return JT_ERR_INVALID_ARG;
  FloatArgs a;
  jt_status s = float_setup(c, g, coeffs, out_rgb, a);
  if (s != JT_OK) return s;
  a.coef = coeffs;
  a.frame = out_rgb;
  DeviceGuard dg(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((s = enqueue_float_needed(c, a, st)) != JT_OK) return s;
  JT_CUDA(c, cudaMemsetAsync(out_rgb, 0, (size_t)a.views.v[0].width * a.views.v[0].height * 3 * sizeof(float), st));
  launch_float_forward(a, c->tuning.pixel_threads, pixel_grid(c, a.views), c->sm_count * 8, st);
  if ((s = check_launch(c, "float forward")) != JT_OK) return s;
  c->phase = Phase::Idle;  // the work list now describes coefficient MCUs
  c->last_stream = st;
  return JT_OK;
}

jt_status jt_colorize_backward(jt_ctx* c, const jt_gbuffer* g, const float* grad_frame, float* grad_coeffs,
                               jt_stream stream) {
  if (!c) return JT_ERR_INVALID_ARG;
  FloatArgs a;
  jt_status s = float_setup(c, g, grad_coeffs, grad_frame, a);
  if (s != JT_OK) return s;
  a.frame = const_cast<float*>(grad_frame);  // read only in the backward kernels
  a.grad_coef = grad_coeffs;
  DeviceGuard dg(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((s = enqueue_float_needed(c, a, st)) != JT_OK) return s;
  launch_float_backward(a, c->tuning.pixel_threads, pixel_grid(c, a.views), c->sm_count * 8, st);
  if ((s = check_launch(c, "float backward")) != JT_OK) return s;
  c->phase = Phase::Idle;
  c->last_stream = st;
  return JT_OK;
}

}  // extern "C"
