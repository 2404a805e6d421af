// Decode (paper Sec. 4.3): every MCU of the work list is Huffman-decoded from its index
// entry (bit offset + DC predictors, Sec. 5.1 / Sec. 5.3), dequantised, inverse-DCT'd,
// chroma-upsampled, colour-converted and written as an RGBA8 tile into the block cache.
//
// GB300 design (the paper's one 64-thread block per MCU with a 32-lane code compare,
// Sec. 5.2, is prior art here):
//  * persistent grid, warps fetch 32 work items at a time from a device counter, so the
//    uneven MCU sizes balance dynamically and the count never goes to the host;
//  * one lane per MCU runs that MCU's serial entropy chain: a 64-bit bit buffer refilled
//    by aligned 32-bit loads, one 10-bit first-level LUT lookup per symbol in shared
//    memory (codes longer than 10 bits take a short MAXCODE walk), value bits extracted
//    together with the code;
//  * the 32 lanes step through the MCU's data units in lockstep; coefficients go to a
//    transposed per-warp buffer coef[k][lane] (int16, zig-zag order k, conflict-free);
//  * each lane then runs the 8x8 integer IDCT on its own column with even/odd butterflies
//    (an exact integer factorisation of the matrix product of the decode spec);
//  * pixels go to a per-lane shared buffer; finally the warp writes each of its 32 tiles
//    cooperatively (32 lanes x 32 B = one 1 KiB 4:2:0 tile per step, coalesced).
//
// Decode spec (identical in the oracle): dequantised d = clamp16(q * Q); column pass
// t = clamp16(floor((sum_v K[y][v] d[v][u] + 2^8) / 2^9)); row pass
// p = clamp(floor((sum_u K[x][u] t[y][u] + 2^18) / 2^19) + 128, 0, 255) with
// K[x][u] = round(2^14 c_u cos((2x+1) u pi / 16)); JFIF colour in 16-bit fixed point;
// 4:2:0 chroma replicated within the MCU; DC values wrap modulo 2^16.
#include <cuda_runtime.h>

#include "jt_internal.cuh"

namespace jt {
namespace {

// ---- integer IDCT constants: round(8192 cos(k pi / 16)), k = 1..7 ----
constexpr int C1 = 8035, C2 = 7568, C3 = 6811, C4 = 5793, C5 = 4551, C6 = 3135, C7 = 1598;

// Position in zig-zag order of natural index r*8+c (closed form: cells before the
// anti-diagonal s = r+c, plus the offset along it; odd diagonals run downwards).
__host__ __device__ constexpr int zz_pos(int r, int c) {
  const int s = r + c;
  const int before = s <= 7 ? s * (s + 1) / 2 : 64 - (15 - s) * (16 - s) / 2;
  const int along = (s & 1) ? r - (s > 7 ? s - 7 : 0) : (s < 7 ? s : 7) - r;
  return before + along;
}
static_assert(zz_pos(0, 0) == 0 && zz_pos(0, 1) == 1 && zz_pos(1, 0) == 2 && zz_pos(2, 0) == 3 &&
                  zz_pos(0, 2) == 5 && zz_pos(7, 6) == 62 && zz_pos(7, 7) == 63 && zz_pos(3, 4) == 31 && zz_pos(4, 3) == 32,
              "zig-zag positions");

// 1-D 8-point IDCT: out[x] = sum_u K[x][u] in[u], K as above, by even/odd parts.
// K[7-x][u] = (-1)^u K[x][u] exactly, so out[x] = E[x] + O[x], out[7-x] = E[x] - O[x].
__device__ __forceinline__ void idct8(const int in[8], int out[8]) {
  const int a0 = C4 * (in[0] + in[4]), a1 = C4 * (in[0] - in[4]);
  const int b0 = C2 * in[2] + C6 * in[6], b1 = C6 * in[2] - C2 * in[6];
  const int e0 = a0 + b0, e3 = a0 - b0, e1 = a1 + b1, e2 = a1 - b1;
  const int o0 = C1 * in[1] + C3 * in[3] + C5 * in[5] + C7 * in[7];
  const int o1 = C3 * in[1] - C7 * in[3] - C1 * in[5] - C5 * in[7];
  const int o2 = C5 * in[1] - C1 * in[3] + C7 * in[5] + C3 * in[7];
  const int o3 = C7 * in[1] - C5 * in[3] + C3 * in[5] - C1 * in[7];
  out[0] = e0 + o0; out[7] = e0 - o0;
  out[1] = e1 + o1; out[6] = e1 - o1;
  out[2] = e2 + o2; out[5] = e2 - o2;
  out[3] = e3 + o3; out[4] = e3 - o3;
}

__device__ __forceinline__ int sat16(int v) { return min(32767, max(-32768, v)); }
__device__ __forceinline__ uint32_t clamp255(int v) { return (uint32_t)min(255, max(0, v)); }

constexpr int kCoefWords = 64 * 32 / 2;  // int16 [64][32] per warp
constexpr int kPixStride = 97;           // words per lane: Y 64 + Cb 16 + Cr 16, +1 pad

struct BitReader {
  uint64_t buf;  // valid bits MSB-aligned
  int cnt;
  uint32_t wp;   // next word to load
  const uint32_t* words;
  uint32_t nwords;

  __device__ __forceinline__ void load_word() {
    uint32_t w = wp < nwords ? __ldg(words + wp) : 0u;
    ++wp;
    buf |= (uint64_t)__byte_perm(w, 0, 0x0123) << (32 - cnt);
    cnt += 32;
  }
  __device__ __forceinline__ void init(uint32_t bitpos) {
    wp = bitpos >> 5;
    buf = 0;
    cnt = 0;
    load_word();
    load_word();
    const int skip = bitpos & 31;
    buf <<= skip;
    cnt -= skip;
  }
  // afterwards at least 32 bits are buffered (a symbol needs at most 16 + 11)
  __device__ __forceinline__ void refill() {
    if (cnt <= 32) load_word();
  }
  __device__ __forceinline__ uint64_t position() const { return (uint64_t)wp * 32 - (uint64_t)cnt; }
};

// Decodes one data unit of `lane`'s MCU into col[k * 32] (k in zig-zag order, dequantised,
// saturated to int16). Returns false on an invalid coding.
__device__ __forceinline__ bool decode_du(BitReader& br, const HuffTable* dct, const HuffTable* act,
                                          const uint16_t* __restrict__ qz, int16_t& pred, int16_t* col) {
  int k = 0;
#pragma unroll 1
  while (k < 64) {
    br.refill();
    const HuffTable* t = k == 0 ? dct : act;
    const uint32_t top = (uint32_t)(br.buf >> 48);
    const uint32_t e = t->lut[top >> (16 - kLutBits)];
    uint32_t len = e >> 8, sym = e & 255;
    if (len == 0) {  // code longer than kLutBits
#pragma unroll 1
      for (int l = kLutBits + 1; l <= 16; ++l) {
        const int code = (int)(top >> (16 - l));
        if (code <= t->maxcode[l]) {
          const int vi = code + t->valoff[l];
          if (vi < 0 || vi > 255) return false;
          len = l;
          sym = t->vals[vi];
          break;
        }
      }
      if (len == 0) return false;
    }
    uint32_t r, s;
    if (k == 0) {
      r = 0;
      s = sym;
      if (s > 11) return false;
    } else {
      r = sym >> 4;
      s = sym & 15;
      if (s > 10) return false;
    }
    const uint32_t total = len + s;
    const uint32_t bits = (uint32_t)(br.buf >> (64 - total));
    br.buf <<= total;
    br.cnt -= (int)total;
    const uint32_t mag = bits & ((1u << s) - 1u);
    const int v = (int)mag - ((mag < ((1u << s) >> 1)) ? (int)((1u << s) - 1u) : 0);
    if (k == 0) {
      pred = (int16_t)(uint16_t)((int)pred + v);
      col[0] = (int16_t)sat16((int)pred * (int)__ldg(qz));
      k = 1;
    } else if (s) {
      k += (int)r;
      if (k > 63) return false;
      col[k * 32] = (int16_t)sat16(v * (int)__ldg(qz + k));
      ++k;
    } else if (r == 15) {
      k += 16;
      if (k > 63) return false;
    } else {
      k = 64;  // end of block
    }
  }
  return true;
}

// 8x8 integer IDCT of the lane's column; writes 8 rows of 8 pixels as word pairs at
// dst[y * row_words], dst[y * row_words + 1].
__device__ __forceinline__ void idct_du(int16_t* col, uint32_t* dst, int row_words) {
#pragma unroll
  for (int u = 0; u < 8; ++u) {  // column pass
    int in[8], out[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) in[v] = col[zz_pos(v, u) * 32];
    idct8(in, out);
#pragma unroll
    for (int y = 0; y < 8; ++y) col[zz_pos(y, u) * 32] = (int16_t)sat16((out[y] + 256) >> 9);
  }
#pragma unroll
  for (int y = 0; y < 8; ++y) {  // row pass
    int in[8], out[8];
#pragma unroll
    for (int x = 0; x < 8; ++x) in[x] = col[zz_pos(y, x) * 32];
    idct8(in, out);
    uint32_t w0 = 0, w1 = 0;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      w0 |= clamp255(((out[x] + (1 << 18)) >> 19) + 128) << (8 * x);
      w1 |= clamp255(((out[x + 4] + (1 << 18)) >> 19) + 128) << (8 * x);
    }
    dst[y * row_words] = w0;
    dst[y * row_words + 1] = w1;
  }
}

__device__ __forceinline__ uint32_t ycc_pixel(uint32_t Y, int ro, int go, int bo) {
  return clamp255((int)Y + ro) | (clamp255((int)Y + go) << 8) | (clamp255((int)Y + bo) << 16) | 0xFF000000u;
}

__device__ __forceinline__ void chroma_offsets(uint32_t cb8, uint32_t cr8, int& ro, int& go, int& bo) {
  const int cb = (int)cb8 - 128, cr = (int)cr8 - 128;
  ro = (91881 * cr + 32768) >> 16;
  go = (-22554 * cb - 46802 * cr + 32768) >> 16;
  bo = (116130 * cb + 32768) >> 16;
}

__device__ __forceinline__ int find_desc(const DevDesc* descs, int n, uint32_t gid) {
  int lo = 0, hi = n - 1;
#pragma unroll 1
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&descs[mid].gid_base) <= gid)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <int W>
__global__ void __launch_bounds__(W * 32) k_decode(const __grid_constant__ DecodeArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  HuffSet* sh = reinterpret_cast<HuffSet*>(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int16_t* coef = reinterpret_cast<int16_t*>(smem + sizeof(HuffSet)) + warp * (kCoefWords * 2);
  uint32_t* pix = reinterpret_cast<uint32_t*>(smem + sizeof(HuffSet) + W * kCoefWords * 4) + warp * 32 * kPixStride;

  {  // stage Huffman set 0 (the set shared by every texture coded with the same tables)
    const uint4* src = reinterpret_cast<const uint4*>(a.huff);
    uint4* dst = reinterpret_cast<uint4*>(sh);
    for (int i = threadIdx.x; i < (int)(sizeof(HuffSet) / 16); i += W * 32) dst[i] = __ldg(src + i);
  }
  __syncthreads();

  const uint32_t count = min(*(volatile uint32_t*)&a.state->count, a.work_cap);
  bool any_bad = false;

#pragma unroll 1
  for (;;) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&a.state->decode_next, 32u);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (base >= count) break;

    const uint32_t item = base + lane;
    bool act = item < count;
    int samp = kSampling420, ndu = 6;
    uint32_t off = 0;
    bool store = false, bad = false;
    BitReader br;
    int16_t pred[3] = {0, 0, 0};
    const HuffTable* hs = sh->t;
    const uint16_t* qz = a.quant;
    uint32_t nbits = 0;
    if (act) {
      const uint32_t gid = __ldg(a.work + item);
      const DevDesc d = a.descs[find_desc(a.descs, (int)a.ndesc, gid)];
      samp = d.sampling;
      const uint32_t mcu = gid - d.gid_base;
      if (samp == kSamplingCoef || mcu >= d.nmcu) {
        act = false;  // not a JPEG level: nothing to decode
      } else {
        ndu = samp == kSampling420 ? 6 : 3;
        off = __ldg(a.slot + gid);
        store = off + d.units <= a.cap_units;
        const uint16_t* ix = d.index + (size_t)mcu * 5;
        const uint32_t bitpos = (uint32_t)__ldg(ix) | ((uint32_t)__ldg(ix + 1) << 16);
        pred[0] = (int16_t)__ldg(ix + 2);
        pred[1] = (int16_t)__ldg(ix + 3);
        pred[2] = (int16_t)__ldg(ix + 4);
        br.words = d.stream;
        br.nwords = d.nwords;
        nbits = d.nbits;
        br.init(bitpos);
        if (d.hset != 0) hs = a.huff[d.hset].t;
        qz = a.quant + (size_t)d.qset * 128;
      }
    }

#pragma unroll 1
    for (int du = 0; du < 6; ++du) {
      {  // clear the warp's coefficient buffer (4 KiB, 8 x 16 B per lane)
        uint4* z = reinterpret_cast<uint4*>(coef);
#pragma unroll
        for (int i = 0; i < 8; ++i) z[lane + 32 * i] = make_uint4(0, 0, 0, 0);
      }
      __syncwarp();
      const bool mine = act && du < ndu;
      const int comp = du < ndu - 2 ? 0 : (du == ndu - 2 ? 1 : 2);
      if (mine && !bad) {
        const int tb = comp == 0 ? 0 : 2;
        if (!decode_du(br, hs + tb, hs + tb + 1, qz + (comp == 0 ? 0 : 64), pred[comp], coef + lane)) bad = true;
      }
      __syncwarp();
      if (mine) {
        uint32_t* dst;
        int row_words;
        if (samp == kSampling420) {
          dst = pix + lane * kPixStride + (du < 4 ? ((du >> 1) * 8) * 4 + (du & 1) * 2 : 64 + (du - 4) * 16);
          row_words = du < 4 ? 4 : 2;
        } else {
          dst = pix + lane * kPixStride + (du == 0 ? 0 : (du == 1 ? 64 : 80));
          row_words = 2;
        }
        idct_du(coef + lane, dst, row_words);
      }
      __syncwarp();
    }
    if (act && !bad && br.position() > nbits) bad = true;
    any_bad |= bad;

    // colour conversion + coalesced tile stores, one MCU of the warp at a time
#pragma unroll 1
    for (int m = 0; m < 32; ++m) {
      const bool st_m = __shfl_sync(0xFFFFFFFFu, act && store, m);
      if (!st_m) continue;
      const int samp_m = __shfl_sync(0xFFFFFFFFu, samp, m);
      const uint32_t off_m = __shfl_sync(0xFFFFFFFFu, off, m);
      const uint32_t* P = pix + m * kPixStride;
      uint8_t* tile = a.cache + (size_t)off_m * kUnitBytes;
      if (samp_m == kSampling420) {
        const int r = lane >> 1, h = lane & 1;
        const uint32_t y0 = P[r * 4 + h * 2], y1 = P[r * 4 + h * 2 + 1];
        const uint32_t cbw = P[64 + (r >> 1) * 2 + h], crw = P[80 + (r >> 1) * 2 + h];
        uint32_t o[8];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          int ro, go, bo;
          chroma_offsets((cbw >> (8 * j)) & 255, (crw >> (8 * j)) & 255, ro, go, bo);
          const uint32_t yw = j < 2 ? y0 : y1;
          const int sh0 = 16 * (j & 1);
          o[2 * j] = ycc_pixel((yw >> sh0) & 255, ro, go, bo);
          o[2 * j + 1] = ycc_pixel((yw >> (sh0 + 8)) & 255, ro, go, bo);
        }
        uint4* dst = reinterpret_cast<uint4*>(tile + r * 64 + h * 32);
        dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
        dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
      } else {
        const int r = lane >> 2, q = lane & 3;
        const int wi = r * 2 + (q >> 1), sh0 = 16 * (q & 1);
        const uint32_t yw = P[wi], cbw = P[64 + wi], crw = P[80 + wi];
        uint32_t o[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          int ro, go, bo;
          chroma_offsets((cbw >> (sh0 + 8 * i)) & 255, (crw >> (sh0 + 8 * i)) & 255, ro, go, bo);
          o[i] = ycc_pixel((yw >> (sh0 + 8 * i)) & 255, ro, go, bo);
        }
        *reinterpret_cast<uint2*>(tile + r * 32 + q * 8) = make_uint2(o[0], o[1]);
      }
    }
    __syncwarp();
  }
  if (any_bad) atomicOr(&a.state->err, JT_DEVERR_CORRUPT);
}

// The dynamic shared-memory attribute is set by decode_max_ctas_per_sm(), which the
// context calls for every variant on its device before the first launch.
template <int W>
void launch_w(const DecodeArgs& a, int grid, cudaStream_t s) {
  k_decode<W><<<grid, W * 32, decode_smem_bytes(W), s>>>(a);
}

template <int W>
int max_ctas() {
  const size_t smem = decode_smem_bytes(W);
  cudaFuncSetAttribute(k_decode<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_decode<W>, W * 32, smem) != cudaSuccess) return 0;
  return n;
}

}  // namespace

size_t decode_smem_bytes(int warps) {
  return sizeof(HuffSet) + (size_t)warps * kCoefWords * 4 + (size_t)warps * 32 * kPixStride * 4;
}

void launch_decode(const DecodeArgs& a, int warps, int grid, cudaStream_t s) {
  switch (warps) {
    case 2: launch_w<2>(a, grid, s); break;
    case 4: launch_w<4>(a, grid, s); break;
    case 6: launch_w<6>(a, grid, s); break;
    case 8: launch_w<8>(a, grid, s); break;
    default: launch_w<4>(a, grid, s); break;
  }
}

int decode_max_ctas_per_sm(int warps) {
  switch (warps) {
    case 2: return max_ctas<2>();
    case 4: return max_ctas<4>();
    case 6: return max_ctas<6>();
    case 8: return max_ctas<8>();
    default: return max_ctas<4>();
  }
}

void idct_constants(int out[8]) {
  const int c[8] = {0, C1, C2, C3, C4, C5, C6, C7};
  for (int i = 0; i < 8; ++i) out[i] = c[i];
}

}  // namespace jt
