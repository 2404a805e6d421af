// jt_compact_static: the compaction scan (the same two passes over the flag bytes that a
// context launches) run on caller buffers with its scratch taken from a
// file-scope __device__ array instead of device memory the library allocates. The paper
// has no counterpart.
//
// Who needs it: callers that must not allocate device memory at the point of the call.
// cudaMalloc and cudaFree may synchronise the whole device, which stalls every other
// stream of a real-time frame loop; a caller under memory pressure may see them fail; and
// an allocator hook or a memory-accounting layer (e.g. code that runs inside a caching
// allocator's callbacks) must not re-enter the allocator. This entry point makes no
// allocating call of its own, neither CUDA nor any library's: it only clears its scratch,
// launches and copies three words out, all asynchronously on the caller's stream.
//
// Scratch: one fixed array per device image, 256 B of frame state then one 64-bit word per
// scan tile (4096 flags: its count and unit sum), for at most kMaxTiles = 4096 tiles
// (16,777,216 flags, 33 KB). Its device address is looked up once per device (cudaGetSymbolAddress, which
// may load the module lazily and so must first run outside any stream capture) and cached.
// Because
// the array is shared, two calls in flight at once on one device (two streams, or two
// host threads without ordering) race on it and give wrong results: callers serialise.
#include <cuda_runtime.h>

#include <mutex>

#include "jt_internal.cuh"

namespace jt {
namespace {

constexpr uint32_t kMaxFlags = JT_STATIC_COMPACT_MAX_FLAGS;
constexpr uint32_t kMaxTiles = kMaxFlags / (uint32_t)kScanTile;
static_assert(kMaxTiles * (uint32_t)kScanTile == kMaxFlags, "the limit is a whole number of scan tiles");
constexpr size_t kStateBytes = 256;  // FrameState, padded so the status words stay 256-B aligned
static_assert(sizeof(FrameState) <= kStateBytes, "frame state fits its slot");

// [0, 256): FrameState; [256, 256 + 8 * kMaxTiles): tile words.
__device__ __align__(256) uint64_t g_compact_scratch[kStateBytes / 8 + kMaxTiles];

constexpr int kMaxDevices = 64;
struct DeviceSlot {
  uint8_t* scratch = nullptr;
};
DeviceSlot g_slots[kMaxDevices];
std::mutex g_slots_mutex;

// Looks the scratch address up once per device (with that device current).
jt_status device_slot(DeviceSlot& out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return JT_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_slots_mutex);
  DeviceSlot& s = g_slots[dev];
  if (!s.scratch) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_compact_scratch) != cudaSuccess || !p) return JT_ERR_CUDA;
    s.scratch = static_cast<uint8_t*>(p);
  }
  out = s;
  return JT_OK;
}

}  // namespace
}  // namespace jt

extern "C" jt_status jt_compact_static(uint8_t* flags, uint32_t n, uint32_t* slot, uint32_t* work, uint32_t work_cap,
                                       uint32_t* totals, jt_stream stream) {
  using namespace jt;
  if (n > kMaxFlags) return JT_ERR_CAPACITY;  // the scratch holds kMaxTiles tile words
  if (!totals || (n && (!flags || !slot || (!work && work_cap)))) return JT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(flags) % 16) return JT_ERR_INVALID_ARG;  // 16-byte flag loads
  DeviceSlot d;
  if (device_slot(d) != JT_OK) return JT_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // a launch error the caller left pending is theirs to read: report it, leave it pending,
  // enqueue nothing (so the error checked after the launch below is this call's own)
  if (cudaPeekAtLastError() != cudaSuccess) return JT_ERR_CUDA;
  // what the scan expects at zero: the frame state (counters and error word); its first pass
  // writes every tile word the second pass reads
  if (cudaMemsetAsync(d.scratch, 0, kStateBytes, s) != cudaSuccess) return JT_ERR_CUDA;
  FrameState* state = reinterpret_cast<FrameState*>(d.scratch);
  ScanArgs a{};
  a.flags = flags;
  a.gid_lo = 0;
  a.n = n;
  a.slot = slot;
  a.work = work;
  a.work_cap = work_cap;
  a.tile_status = reinterpret_cast<uint64_t*>(d.scratch + kStateBytes);
  a.state = state;
  a.cap_units = 0xFFFFFFFFu;  // no cache behind these slots: only the work list can overflow
  launch_scan(a, s);
  if (cudaGetLastError() != cudaSuccess) return JT_ERR_CUDA;
  // totals = {count, units, error bits}: FrameState holds count, units at words 0, 1 and err at word 3
  if (cudaMemcpyAsync(totals, &state->count, 2 * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(totals + 2, &state->err, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return JT_ERR_CUDA;
  return JT_OK;
}
