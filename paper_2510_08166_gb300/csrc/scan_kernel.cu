// Compaction of the marked MCUs into the decode work list (the paper's decode queue,
// Sec. 4.2 and the pipeline overview: every needed MCU enqueued once).
//
// The flags hold, per global MCU id (gid), the number of 256-byte cache units the MCU
// needs (4 at 4:2:0, 1 at 4:4:4) or 0. One single-pass exclusive scan over the flag bytes
// gives each needed gid its work-list position (count prefix) and its cache slot (units
// prefix): work[count_prefix] = gid, slot[gid] = units_prefix. The list is therefore in
// ascending gid order and deterministic. The same pass clears the flags for the next frame.
//
// Single pass: decoupled look-back (Merrill & Garland 2016). Each 65536-flag tile
// publishes its aggregate, then a warp of the tile looks back over up to 32 predecessor
// tiles at a time until it meets an inclusive prefix. The grid is persistent (every CTA
// resident) and CTAs take tiles in increasing order, so every awaited predecessor is being
// processed by a running CTA. Waits are bounded: after kSpinLimit polls the tile gives up,
// sets JT_DEVERR_TIMEOUT and uses what it has. The last CTA to finish clears the status
// words, so every launch (including CUDA-graph replays) starts from "nothing published".
//
// Status word of a tile (64 bit): flag (2) | units (28) | count (26); flag 0 = not yet.
#include <cuda_runtime.h>

#include "jt_internal.cuh"

namespace jt {
namespace {

constexpr uint64_t kFlagAgg = 1, kFlagIncl = 2;
constexpr int kSpinLimit = 1 << 20;

__device__ __forceinline__ uint64_t pack_status(uint64_t flag, uint32_t units, uint32_t count) {
  return (flag << 54) | ((uint64_t)(units & 0x0FFFFFFF) << 26) | (uint64_t)(count & 0x03FFFFFF);
}
__device__ __forceinline__ uint64_t st_flag(uint64_t w) { return (w >> 54) & 3; }
__device__ __forceinline__ uint32_t st_units(uint64_t w) { return (uint32_t)((w >> 26) & 0x0FFFFFFF); }
__device__ __forceinline__ uint32_t st_count(uint64_t w) { return (uint32_t)(w & 0x03FFFFFF); }

__device__ __forceinline__ void store_status(uint64_t* p, uint64_t w) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}
__device__ __forceinline__ uint64_t load_status(const uint64_t* p) {
  uint64_t w;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
  return w;
}

// Byte statistics of one 32-bit word of flags: number of non-zero bytes, sum of bytes.
__device__ __forceinline__ void word_stats(uint32_t w, uint32_t& cnt, uint32_t& sum) {
  cnt += __popc(__vcmpne4(w, 0u)) >> 3;
  sum += (w & 255) + ((w >> 8) & 255) + ((w >> 16) & 255) + (w >> 24);
}

__global__ void __launch_bounds__(kScanThreads, 1) k_scan(const __grid_constant__ ScanArgs a) {
  __shared__ uint32_t s_cnt[kScanThreads / 32], s_sum[kScanThreads / 32];
  __shared__ uint32_t s_pre_cnt, s_pre_sum;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t ntiles = (a.n + kScanTile - 1) / kScanTile;
  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint32_t first = tile * kScanTile + tid * kScanPerThread;  // relative to gid_lo
    constexpr int kWords = kScanPerThread / 4;
    uint32_t w[kWords];
    if (first + kScanPerThread <= a.n) {
#pragma unroll
      for (int j = 0; j < kWords / 4; ++j) {
        const uint4 v = reinterpret_cast<const uint4*>(a.flags + first)[j];
        w[4 * j] = v.x; w[4 * j + 1] = v.y; w[4 * j + 2] = v.z; w[4 * j + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < kWords; ++j) w[j] = 0;
      for (int i = 0; i < kScanPerThread; ++i)
        if (first + i < a.n) w[i >> 2] |= (uint32_t)a.flags[first + i] << (8 * (i & 3));
    }
    uint32_t cnt = 0, sum = 0;
#pragma unroll
    for (int i = 0; i < kWords; ++i) word_stats(w[i], cnt, sum);
    // block-wide exclusive scan of (cnt, sum)
    uint32_t ic = cnt, is = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      uint32_t c = __shfl_up_sync(0xFFFFFFFFu, ic, d), s = __shfl_up_sync(0xFFFFFFFFu, is, d);
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
    uint32_t ex_c = wc + ic - cnt, ex_s = ws + is - sum;
    // look-back by warp 0
    if (warp == 0) {
      uint64_t* status = a.tile_status;
      uint32_t pre_c = 0, pre_s = 0;
      if (tile == 0) {
        if (lane == 0) store_status(status, pack_status(kFlagIncl, tot_s, tot_c));
      } else {
        if (lane == 0) store_status(status + tile, pack_status(kFlagAgg, tot_s, tot_c));
        int end = (int)tile - 1;  // predecessor window [end - 31, end]
        int spins = 0;
        bool gave_up = false;
        while (end >= 0) {
          const int idx = end - lane;
          uint64_t sw = idx >= 0 ? load_status(status + idx) : pack_status(kFlagIncl, 0, 0);
          const bool valid = st_flag(sw) != 0;
          const uint32_t incl = __ballot_sync(0xFFFFFFFFu, valid && st_flag(sw) == kFlagIncl);
          const int stop = incl ? __ffs(incl) - 1 : 31;  // nearest inclusive predecessor
          const uint32_t need = stop == 31 ? 0xFFFFFFFFu : ((2u << stop) - 1u);
          const uint32_t ok = __ballot_sync(0xFFFFFFFFu, valid);
          if ((ok & need) != need) {
            if (++spins > kSpinLimit) {
              gave_up = true;
              break;
            }
            continue;  // a predecessor has not published yet
          }
          uint32_t c = lane <= stop ? st_count(sw) : 0, s = lane <= stop ? st_units(sw) : 0;
#pragma unroll
          for (int d = 16; d > 0; d >>= 1) {
            c += __shfl_xor_sync(0xFFFFFFFFu, c, d);
            s += __shfl_xor_sync(0xFFFFFFFFu, s, d);
          }
          pre_c += c;
          pre_s += s;
          if (incl) break;
          end -= 32;
        }
        if (lane == 0) {
          store_status(status + tile, pack_status(kFlagIncl, pre_s + tot_s, pre_c + tot_c));
          if (gave_up) atomicOr(&a.state->err, JT_DEVERR_TIMEOUT);
        }
      }
      if (lane == 0) {
        s_pre_cnt = pre_c;
        s_pre_sum = pre_s;
      }
    }
    __syncthreads();
    uint32_t pos = s_pre_cnt + ex_c, off = s_pre_sum + ex_s;
    if (cnt) {
#pragma unroll
      for (int i = 0; i < kScanPerThread; ++i) {
        const uint32_t f = (w[i >> 2] >> (8 * (i & 3))) & 255;
        if (f) {
          const uint32_t gid = a.gid_lo + first + i;
          a.slot[gid] = off;
          if (pos < a.work_cap) a.work[pos] = gid;
          off += f;
          ++pos;
        }
      }
      // clear for the next frame
      if (first + kScanPerThread <= a.n) {
#pragma unroll
        for (int j = 0; j < kWords / 4; ++j) reinterpret_cast<uint4*>(a.flags + first)[j] = make_uint4(0, 0, 0, 0);
      } else {
        for (int i = 0; i < kScanPerThread; ++i)
          if (first + i < a.n) a.flags[first + i] = 0;
      }
    }
    if (tile == ntiles - 1 && tid == 0) {
      const uint32_t total_c = s_pre_cnt + tot_c, total_s = s_pre_sum + tot_s;
      a.state->count = total_c;
      a.state->units = total_s;
      a.state->decode_next = 0;
      if (total_s > a.cap_units || total_c > a.work_cap) atomicOr(&a.state->err, JT_DEVERR_CAPACITY);
    }
    __syncthreads();  // shared scratch is reused by the next tile
  }
  if (a.n == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
    a.state->count = 0;
    a.state->units = 0;
    a.state->decode_next = 0;
  }
  // the last CTA to finish (all look-backs done) clears the status words for the next launch
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&a.state->scan_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    for (uint32_t t = threadIdx.x; t < ntiles; t += blockDim.x) store_status(a.tile_status + t, 0);
    if (threadIdx.x == 0) a.state->scan_done = 0;
  }
}

}  // namespace

void launch_scan(const ScanArgs& a, int grid, cudaStream_t s) { k_scan<<<grid, kScanThreads, 0, s>>>(a); }

// Resident scan CTAs per SM: the look-back needs every CTA of the grid running at once.
int scan_max_ctas_per_sm() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_scan, kScanThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

}  // namespace jt
