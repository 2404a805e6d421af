// Cross-frame texture block cache (paper Sec. 4.1 "Texture Block Cache" and Sec. 4.5
// "Update Cache"): decoded MCUs stay resident in 1 KiB blocks of the block cache between
// frames; a frame decodes only the needed MCUs that are not resident, and blocks of MCUs no
// pixel of the frame needs are evicted (the paper evicts what is not visible).
//
// The paper keys a GPU hash map by a packed 32-bit MCU key. Our keys are the dense global
// MCU ids (gids, one range per uploaded level), so the map is a direct array resident[gid]
// (block index or kNone), with its inverse block_gid[block] and a stack of free blocks.
//
// Per frame, after the mark pass has set flags[gid] (cache units needed, 0 = not needed):
//   k_cache_evict  every resident block whose gid is not flagged returns to the free stack
//   k_cache_alloc  every flagged gid: if resident, its slot is its block; else it takes a
//                  free block and joins the decode work list. Flags are cleared.
// The decode and colourise passes then run unchanged on the work list and slot map.
// Work-list order and block numbers depend on atomic order (the decoded tiles and pixels do
// not); a frame that needs more blocks than are free sets JT_DEVERR_CAPACITY.
#include <cuda_runtime.h>

#include "jt_internal.cuh"

namespace jt {
namespace {

constexpr uint32_t kNone = 0xFFFFFFFFu;

__global__ void k_cache_evict(const __grid_constant__ CacheArgs a) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.state->count = 0;
    a.state->decode_next = 0;
    a.cs->taken = 0;
    a.cs->visible = 0;
  }
  uint32_t evicted = 0;
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < a.nblocks; b += gridDim.x * blockDim.x) {
    const uint32_t g = a.block_gid[b];
    if (g != kNone && a.flags[g] == 0) {
      a.resident[g] = kNone;
      a.block_gid[b] = kNone;
      a.free_list[atomicAdd(&a.cs->free_count, 1u)] = b;
      ++evicted;
    }
  }
  if (evicted) atomicAdd(&a.cs->evicted, evicted);
}

__global__ void k_cache_alloc(const __grid_constant__ CacheArgs a) {
  const uint32_t free_now = a.cs->free_count;  // after the eviction pass (stream order)
  uint32_t visible = 0;
  bool over = false;
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w * 16 < a.n; w += gridDim.x * blockDim.x) {
    const uint32_t first = w * 16;
    uint4 v;
    if (first + 16 <= a.n) {
      v = reinterpret_cast<const uint4*>(a.flags)[w];
    } else {
      uint32_t t[4] = {0, 0, 0, 0};
      for (uint32_t i = 0; first + i < a.n; ++i) t[i >> 2] |= (uint32_t)a.flags[first + i] << (8 * (i & 3));
      v = make_uint4(t[0], t[1], t[2], t[3]);
    }
    if ((v.x | v.y | v.z | v.w) == 0) continue;
    const uint32_t words[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      if (((words[i >> 2] >> (8 * (i & 3))) & 255) == 0) continue;
      const uint32_t g = first + i;
      ++visible;
      uint32_t b = a.resident[g];
      if (b == kNone) {
        const uint32_t pos = atomicAdd(&a.cs->taken, 1u);
        if (pos >= free_now) {
          over = true;
          continue;
        }
        b = a.free_list[free_now - 1 - pos];
        a.resident[g] = b;
        a.block_gid[b] = g;
        const uint32_t item = atomicAdd(&a.state->count, 1u);
        if (item < a.work_cap)
          a.work[item] = g;
        else
          over = true;
      }
      a.slot[g] = b * 4;  // a block is 4 cache units
    }
    // clear for the next frame
    if (first + 16 <= a.n)
      reinterpret_cast<uint4*>(a.flags)[w] = make_uint4(0, 0, 0, 0);
    else
      for (uint32_t i = 0; first + i < a.n; ++i) a.flags[first + i] = 0;
  }
  if (visible) atomicAdd(&a.cs->visible, visible);
  if (over) atomicOr(&a.state->err, JT_DEVERR_CAPACITY);
}

// Pops the blocks taken by the allocation pass off the free stack.
__global__ void k_cache_commit(const __grid_constant__ CacheArgs a) {
  const uint32_t taken = min(a.cs->taken, a.cs->free_count);
  a.cs->free_count -= taken;
  a.state->units = 4 * a.state->count;
}

}  // namespace

void launch_cache_update(const CacheArgs& a, int grid, cudaStream_t s) {
  k_cache_evict<<<grid, 256, 0, s>>>(a);
  k_cache_alloc<<<grid, 256, 0, s>>>(a);
  k_cache_commit<<<1, 1, 0, s>>>(a);
}

}  // namespace jt
