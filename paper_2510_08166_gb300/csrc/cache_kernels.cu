// Cross-frame texture block cache (paper Sec. 4.1 "Texture Block Cache" and Sec. 4.5
// "Update Cache"): decoded MCUs stay resident in 1 KiB blocks of the block cache between
// frames; a frame decodes only the needed MCUs that are not resident, and blocks of MCUs no
// pixel of the frame needs are evicted (the paper evicts what is not visible).
//
// The paper keys a GPU hash map by a packed 32-bit MCU key. Our keys are the dense global
// MCU ids (gids, one range per uploaded level), so the map is a residency bitmap over the
// gids plus the slot array itself: a resident MCU was needed by the frame before (the cache
// keeps nothing a frame does not need), so its slot from that frame still holds its block
// (slot = 4 x block). Free blocks sit in a ring: positions [head, head + free_count) modulo
// the block count.
//
// Per frame, after the mark pass has set flags[gid] (cache units needed, 0 = not needed), ONE
// launch updates the cache. Each thread owns 16 gids (16 flag bytes and a 16-bit word of the
// bitmap), so the decisions for one gid never race:
//   flagged and resident      nothing to do: its slot already points at its block (a hit);
//   flagged, not resident     it takes the next free block of the ring and joins the work
//                             list (a miss);
//   resident, not flagged     its block goes back to the ring, behind the blocks that were
//                             free when the frame began (an eviction).
// Misses take blocks that were free at the start of the frame; evictions are pushed behind
// them, so the two never touch the same ring entry. Misses beyond the free blocks are
// deferred: the last CTA to finish (a completion counter) hands them the blocks this frame
// evicted, then moves the ring's head, writes the frame's totals and resets the counters for
// the next frame. The frame therefore fits whenever its needed set fits in the cache, as with
// an evict-then-allocate order, without a second launch. The flags are cleared on the way.
// Work-list order and block numbers depend on atomic order (the decoded tiles and pixels do
// not); a frame that needs more blocks than the cache holds sets JT_DEVERR_CAPACITY, and its
// MCUs that found no block are neither decoded nor given a slot outside the cache.
#include <cuda_runtime.h>

#include "jt_internal.cuh"

namespace jt {
namespace {

// Ring entry at position p < 2 nblocks (every position used is head plus less than nblocks).
__device__ __forceinline__ uint32_t* ring_at(const CacheArgs& a, uint32_t p) {
  return a.ring + (p >= a.nblocks ? p - a.nblocks : p);
}

__global__ void __launch_bounds__(kCacheThreads) k_cache_update(const __grid_constant__ CacheArgs a) {
  __shared__ bool s_last;
  pdl_launch_dependents();
  pdl_wait();  // the flags come from the mark pass
  const uint32_t head = a.cs->head, free0 = a.cs->free_count;  // fixed until the last CTA
  uint32_t visible = 0;
  bool over = false, wrote = false;
  const uint32_t nw = (a.n + 15) / 16;
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) {
    const uint32_t first = w * 16;
    uint4 v;
    if (first + 16 <= a.n) {
      v = reinterpret_cast<const uint4*>(a.flags)[w];
    } else {
      uint32_t t[4] = {0, 0, 0, 0};
      for (uint32_t i = 0; first + i < a.n; ++i) t[i >> 2] |= (uint32_t)a.flags[first + i] << (8 * (i & 3));
      v = make_uint4(t[0], t[1], t[2], t[3]);
    }
    const uint32_t rb = a.resbits[w];
    const bool any_flag = (v.x | v.y | v.z | v.w) != 0;
    if (!any_flag && rb == 0) continue;
    // masks over the 16 gids: flagged, hit, miss, eviction
    uint32_t fm = 0;
    const uint32_t words[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t nz = __vcmpne4(words[q], 0u);
      fm |= (((nz >> 7) & 1u) | ((nz >> 14) & 2u) | ((nz >> 21) & 4u) | ((nz >> 28) & 8u)) << (4 * q);
    }
    const uint32_t hit = fm & rb, miss = fm & ~rb, evm = rb & ~fm;
    visible += __popc(fm);
    auto clear_flags = [&] {  // for the next frame
      if (first + 16 <= a.n)
        reinterpret_cast<uint4*>(a.flags)[w] = make_uint4(0, 0, 0, 0);
      else
        for (uint32_t i = 0; first + i < a.n; ++i) a.flags[first + i] = 0;
    };
    if (fm == hit && evm == 0) {  // only hits: their slots already hold their blocks
      if (any_flag) clear_flags();
      continue;
    }
    // the 16 gids' slots in one go when some are evicted (the slot array holds whole groups
    // of 16): an evicted MCU's block is its slot / 4
    uint32_t res[16];
    if (evm) {
      const uint4* rp = reinterpret_cast<const uint4*>(a.slot + first);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint4 r4 = rp[q];
        res[4 * q] = r4.x >> 2;
        res[4 * q + 1] = r4.y >> 2;
        res[4 * q + 2] = r4.z >> 2;
        res[4 * q + 3] = r4.w >> 2;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) res[q] = 0;
    }
    // one counter update per thread and kind: misses take ring positions pos0, pos0 + 1, ...
    // (the first ones, below free0, at once, at the same places of the work list; the rest
    // are deferred), evictions e0, e0 + 1, ...
    const uint32_t nmiss = __popc(miss), nev = __popc(evm);
    const uint32_t pos0 = nmiss ? atomicAdd(&a.cs->taken, nmiss) : 0u;
    const uint32_t e0 = nev ? atomicAdd(&a.cs->evict_n, nev) : 0u;
    const uint32_t nnow = pos0 < free0 ? min(nmiss, free0 - pos0) : 0u;
    wrote = true;
    uint32_t nrb = rb & ~evm;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const uint32_t bit = 1u << i, g = first + i;
      if (miss & bit) {
        const uint32_t rank = __popc(miss & (bit - 1u)), pos = pos0 + rank;
        if (rank < nnow) {
          const uint32_t b = *ring_at(a, head + pos);
          a.slot[g] = b * 4;  // a block is 4 cache units
          nrb |= bit;
          if (pos < a.work_cap)
            a.work[pos] = g;
          else
            over = true;
        } else if (pos - free0 < a.nblocks) {
          a.deferred[pos - free0] = g;  // the last CTA gives it a block evicted by this update
        } else {
          a.slot[g] = 0;
          over = true;
        }
      }
      if (evm & bit) *ring_at(a, head + free0 + e0 + __popc(evm & (bit - 1u))) = res[i];
    }
    if (nrb != rb) a.resbits[w] = (uint16_t)nrb;
    if (any_flag) clear_flags();
  }
  visible = __reduce_add_sync(0xFFFFFFFFu, visible);
  if ((threadIdx.x & 31) == 0 && visible) atomicAdd(&a.cs->visible_acc, visible);
  if (__any_sync(0xFFFFFFFFu, over) && (threadIdx.x & 31) == 0) atomicOr(&a.state->err, JT_DEVERR_CAPACITY);

  // ---- the last CTA to finish: deferred misses, ring head, totals, counters ----
  if (wrote || visible || over) __threadfence();  // this thread's writes before the count
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&a.cs->done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  volatile CacheState* cs = a.cs;
  const uint32_t taken = cs->taken, ev = cs->evict_n, items = min(taken, free0);
  const uint32_t nd = taken > free0 ? min(taken - free0, a.nblocks) : 0u;  // deferred misses stored
  const uint32_t served = min(nd, ev);
  bool dover = false;
  for (uint32_t j = threadIdx.x; j < nd; j += blockDim.x) {
    const uint32_t g = a.deferred[j];
    if (j < served) {
      const uint32_t b = *ring_at(a, head + free0 + j);
      a.slot[g] = b * 4;
      atomicOr(&a.resbits32[g >> 5], 1u << (g & 31));
      if (items + j < a.work_cap)
        a.work[items + j] = g;
      else
        dover = true;
    } else {
      a.slot[g] = 0;
      dover = true;
    }
  }
  if (dover) atomicOr(&a.state->err, JT_DEVERR_CAPACITY);
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t popped = min(taken, free0) + served;  // ring entries handed out this frame
    const uint32_t count = min(items + served, a.work_cap);
    cs->head = head + popped >= a.nblocks ? head + popped - a.nblocks : head + popped;
    cs->free_count = free0 + ev - popped;
    cs->visible = cs->visible_acc;
    cs->evicted += ev;
    cs->taken = 0;
    cs->evict_n = 0;
    cs->visible_acc = 0;
    cs->done = 0;
    a.state->count = count;
    a.state->units = 4 * count;
    a.state->decode_next = 0;
  }
}

}  // namespace

void launch_cache_update(const CacheArgs& a, int max_grid, cudaStream_t s) {
  const uint32_t nw = (a.n + 15) / 16;
  const int grid = (int)std::max<uint32_t>(1, std::min<uint32_t>((nw + kCacheThreads - 1) / kCacheThreads, (uint32_t)max_grid));
  launch_pdl(k_cache_update, grid, kCacheThreads, 0, s, a);
}

}  // namespace jt
