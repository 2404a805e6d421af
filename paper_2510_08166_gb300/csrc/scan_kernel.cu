// Compaction of the marked MCUs into the decode work list (the paper's decode queue,
// Sec. 4.2 and the pipeline overview: every needed MCU enqueued once).
//
// The flags hold, per global MCU id (gid), the number of 256-byte cache units the MCU
// needs (4 at 4:2:0, 1 at 4:4:4) or 0. An exclusive scan over the flag bytes gives each
// needed gid its work-list position (count prefix) and its cache slot (units prefix):
// work[count_prefix] = gid, slot[gid] = units_prefix. The list is therefore in ascending
// gid order and deterministic. The same pass clears the flags for the next frame.
//
// Two passes over tiles of 4096 flags (256 threads, one 16-byte load each), with no waiting
// between CTAs of one launch:
//   k_tile_sums    every tile's (count, units) into one 64-bit word, count << 32 | units;
//   k_scan_scatter every tile adds up its predecessors' words (up to ntiles / 256 loads
//                  per thread, independent, four in flight, from L2), scans its own flags, writes slots
//                  and work-list entries and clears the flags; the last tile writes the
//                  totals into the frame state.
// A single-pass scan with decoupled look-back was measured slower here: with a few
// hundred tiles its prefix crosses the grid one poll round trip per window, while the
// second pass's loads all go out at once. Counts stay below 2^26 (the gid limit) and unit
// sums below 2^32 (at most 255 per flag over 2^24 flags, or 4 per MCU over 2^26 MCUs).
#include <cuda_runtime.h>

#include "jt_internal.cuh"

namespace jt {
namespace {

// Byte statistics of one 32-bit word of flags: number of non-zero bytes, sum of bytes.
__device__ __forceinline__ void word_stats(uint32_t w, uint32_t& cnt, uint32_t& sum) {
  cnt += __popc(__vcmpne4(w, 0u)) >> 3;
  sum += (w & 255) + ((w >> 8) & 255) + ((w >> 16) & 255) + (w >> 24);
}

// The thread's 16 flags of tile `tile` as four words (zero past n).
__device__ __forceinline__ void load_flags(const ScanArgs& a, uint32_t first, uint32_t w[4]) {
  if (first + kScanPerThread <= a.n) {
    const uint4 v = *reinterpret_cast<const uint4*>(a.flags + first);
    w[0] = v.x;
    w[1] = v.y;
    w[2] = v.z;
    w[3] = v.w;
  } else {
    w[0] = w[1] = w[2] = w[3] = 0;
    for (int i = 0; i < kScanPerThread; ++i)
      if (first + i < a.n) w[i >> 2] |= (uint32_t)a.flags[first + i] << (8 * (i & 3));
  }
}

// Block-wide sum of a (count, units) pair packed as count << 32 | units.
__device__ __forceinline__ uint64_t block_sum(uint64_t v, uint64_t* s_part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, d);
  if (lane == 0) s_part[warp] = v;
  __syncthreads();
  uint64_t t = 0;
#pragma unroll
  for (int i = 0; i < kScanThreads / 32; ++i) t += s_part[i];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(kScanThreads) k_tile_sums(const __grid_constant__ ScanArgs a) {
  __shared__ uint64_t s_part[kScanThreads / 32];
  pdl_launch_dependents();
  pdl_wait();  // the flags come from the kernel before
  const uint32_t ntiles = (a.n + kScanTile - 1) / kScanTile;
  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    uint32_t w[4], cnt = 0, sum = 0;
    load_flags(a, tile * kScanTile + threadIdx.x * kScanPerThread, w);
#pragma unroll
    for (int i = 0; i < 4; ++i) word_stats(w[i], cnt, sum);
    const uint64_t t = block_sum(((uint64_t)cnt << 32) | sum, s_part);
    if (threadIdx.x == 0) a.tile_status[tile] = t;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_scatter(const __grid_constant__ ScanArgs a) {
  __shared__ uint64_t s_part[kScanThreads / 32];
  __shared__ uint32_t s_cnt[kScanThreads / 32], s_sum[kScanThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t ntiles = (a.n + kScanTile - 1) / kScanTile;
  pdl_launch_dependents();
  pdl_wait();  // the tile sums come from k_tile_sums
  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // predecessors' totals: thread i adds tiles i, i + 256, ... below this one, four loads in
    // flight at a time
    uint64_t p0 = 0, p1 = 0, p2 = 0, p3 = 0;
    uint32_t t = tid;
    for (; t + 3 * kScanThreads < tile; t += 4 * kScanThreads) {
      p0 += a.tile_status[t];
      p1 += a.tile_status[t + kScanThreads];
      p2 += a.tile_status[t + 2 * kScanThreads];
      p3 += a.tile_status[t + 3 * kScanThreads];
    }
    for (; t < tile; t += kScanThreads) p0 += a.tile_status[t];
    const uint64_t pre = block_sum((p0 + p1) + (p2 + p3), s_part);
    const uint32_t first = tile * kScanTile + tid * kScanPerThread;  // relative to gid_lo
    uint32_t w[4], cnt = 0, sum = 0;
    load_flags(a, first, w);
#pragma unroll
    for (int i = 0; i < 4; ++i) word_stats(w[i], cnt, sum);
    // block-wide exclusive scan of (cnt, sum)
    uint32_t ic = cnt, is = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t c = __shfl_up_sync(0xFFFFFFFFu, ic, d), s = __shfl_up_sync(0xFFFFFFFFu, is, d);
      if (lane >= d) {
        ic += c;
        is += s;
      }
    }
    if (lane == 31) {
      s_cnt[warp] = ic;
      s_sum[warp] = is;
    }
    __syncthreads();
    uint32_t wc = 0, ws = 0, tot_c = 0, tot_s = 0;
#pragma unroll
    for (int i = 0; i < kScanThreads / 32; ++i) {
      if (i < warp) {
        wc += s_cnt[i];
        ws += s_sum[i];
      }
      tot_c += s_cnt[i];
      tot_s += s_sum[i];
    }
    __syncthreads();  // s_cnt / s_sum are reused by the next tile
    uint32_t pos = (uint32_t)(pre >> 32) + wc + ic - cnt, off = (uint32_t)pre + ws + is - sum;
    if (cnt) {
#pragma unroll
      for (int i = 0; i < kScanPerThread; ++i) {
        const uint32_t f = (w[i >> 2] >> (8 * (i & 3))) & 255;
        if (f) {
          const uint32_t gid = a.gid_lo + first + i;
          // a tile that would end past the cache points at unit 0 instead (the overflow is
          // reported through the error word), so every slot a later pass reads is in range
          a.slot[gid] = (uint64_t)off + f <= a.cap_units ? off : 0u;
          if (pos < a.work_cap) a.work[pos] = gid;
          off += f;
          ++pos;
        }
      }
      // clear for the next frame
      if (first + kScanPerThread <= a.n) {
        *reinterpret_cast<uint4*>(a.flags + first) = make_uint4(0, 0, 0, 0);
      } else {
        for (int i = 0; i < kScanPerThread; ++i)
          if (first + i < a.n) a.flags[first + i] = 0;
      }
    }
    if (tile == ntiles - 1 && tid == 0) {
      const uint32_t total_c = (uint32_t)(pre >> 32) + tot_c, total_s = (uint32_t)pre + tot_s;
      a.state->count = total_c;
      a.state->units = total_s;
      a.state->decode_next = 0;
      if (total_s > a.cap_units || total_c > a.work_cap) atomicOr(&a.state->err, JT_DEVERR_CAPACITY);
    }
  }
  if (a.n == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
    a.state->count = 0;
    a.state->units = 0;
    a.state->decode_next = 0;
  }
}

}  // namespace

// Both passes, one CTA per tile (at least one CTA, so that an empty range still resets the
// counts). tile_status must hold ntiles words.
void launch_scan(const ScanArgs& a, cudaStream_t s) {
  const uint32_t ntiles = (a.n + kScanTile - 1) / kScanTile;
  const int grid = (int)(ntiles ? ntiles : 1);
  launch_pdl(k_tile_sums, grid, kScanThreads, 0, s, a);
  launch_pdl(k_scan_scatter, grid, kScanThreads, 0, s, a);
}

}  // namespace jt
