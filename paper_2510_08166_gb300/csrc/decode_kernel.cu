// Decode (paper Sec. 4.3): every MCU of the work list is Huffman-decoded from its index
// entry (bit offset + DC predictors, Sec. 5.1 / Sec. 5.3), dequantised, inverse-DCT'd,
// chroma-upsampled, colour-converted and written as an RGBA8 tile into the block cache.
//
// GB300 design (the paper's one 64-thread block per MCU with a 32-lane code compare,
// Sec. 5.2, is prior art here):
//  * persistent grid; each warp fetches M work items (M = 4, 8, 16 or 32 MCUs per warp) at
//    a time from a device counter, so uneven MCU sizes balance dynamically and the count
//    never goes to the host. Small M gives many warps for frames with few needed MCUs
//    (latency hiding); large M amortises per-warp overhead for full decodes;
//  * entropy phase: lane m < M runs MCU m's serial entropy chain over all its data units —
//    a 64-bit bit buffer refilled from a two-word prefetch queue of aligned 32-bit loads,
//    one 10-bit first-level LUT lookup per symbol in shared memory whose entry usually
//    carries the decoded value (codes longer than 10 bits take a short MAXCODE walk) —
//    and writes the quantised coefficients in zig-zag order into a per-warp buffer
//    coef[du][k][m] (int16). Nothing but the LUT and the stream is read on this serial
//    chain: dequantisation waits for the IDCT phase;
//  * IDCT phase: all 32 lanes share the 8x8 integer IDCTs of the warp's 6M data units; for
//    each column index u (then row index y) in turn, every lane transforms that column of
//    one or more data units, so all zig-zag positions are compile-time constants. Columns
//    are dequantised on load with the MCU's quantisation table (staged per warp in shared
//    memory); even/odd butterflies give an exact integer factorisation of the matrix
//    product of the decode spec; rows of pixels go to a per-MCU shared buffer;
//  * colour phase: the warp writes each MCU's RGBA8 tile cooperatively (32 lanes x 32 B =
//    one 1 KiB 4:2:0 tile per step, coalesced).
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

// Words of an MCU's entropy-coded data copied to shared memory before its serial decode.
// Random loads from HBM take thousands of cycles and would otherwise sit on the serial
// chain once per refill; staging issues them all at once (one latency per work chunk).
constexpr int kStageWords = 64;  // 256 B per MCU; longer MCUs read their tail from global memory

constexpr int kPixStride = 97;  // words per MCU: Y 64 + Cb 16 + Cr 16, +1 pad

// Shared memory of one warp: coefficients [6][64][M] int16 (zig-zag order), pixels
// [M][97] words, quantisation tables [M][2][64] uint16 (zig-zag order), per-MCU cache
// offset and descriptor bits, staged entropy-coded words [M][kStageWords].
__host__ __device__ constexpr size_t warp_smem(int M) {
  return (size_t)6 * 64 * M * 2 + (size_t)M * kPixStride * 4 + (size_t)M * 256 + (size_t)M * 8 +
         (size_t)M * kStageWords * 4;
}

__device__ __forceinline__ uint32_t lds_u32(uint32_t saddr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(saddr));
  return v;
}

// Bit reader: a 64-bit window (hi:lo, big-endian words) read at bit `pos` of hi with one
// funnel shift, and a queue of the next three raw words. Words come from the lane's staged
// copy in shared memory (words [base, base + nstage)), else from global memory.
struct BitReader {
  uint32_t hi, lo;
  uint32_t pos;         // bit offset into hi, < 32 after refill()
  uint32_t q0, q1, q2;  // raw (as loaded) next words
  uint32_t wp;          // next word to request
  const uint32_t* words;
  uint32_t nwords;
  uint32_t base, nstage, stage_sa;

  __device__ __forceinline__ uint32_t fetch() {
    const uint32_t i = wp - base;
    uint32_t w;
    if (i < nstage)
      w = lds_u32(stage_sa + i * 4u);
    else
      w = wp < nwords ? __ldg(words + wp) : 0u;
    ++wp;
    return w;
  }
  __device__ __forceinline__ static uint32_t be(uint32_t w) { return __byte_perm(w, 0, 0x0123); }
  __device__ __forceinline__ void init(uint32_t bitpos) {
    wp = bitpos >> 5;
    hi = be(fetch());
    lo = be(fetch());
    q0 = fetch();
    q1 = fetch();
    q2 = fetch();
    pos = bitpos & 31;
  }
  // afterwards the window holds at least 33 unread bits (a symbol needs at most 16 + 11)
  __device__ __forceinline__ void refill() {
    if (pos >= 32) {
      hi = lo;
      lo = be(q0);
      q0 = q1;
      q1 = q2;
      q2 = fetch();
      pos -= 32;
    }
  }
  // the next 32 bits
  __device__ __forceinline__ uint32_t peek() const { return __funnelshift_l(lo, hi, pos); }
  // bit position of the next unread bit in the stream
  __device__ __forceinline__ uint64_t position() const { return (uint64_t)(wp - 5) * 32 + pos; }
};

// Slow path of a symbol (slow LUT entry): a code longer than kLutBits (found by the
// MAXCODE walk) or value bits beyond the LUT window. Cuts code and value bits from the
// 32-bit window w (at most 16 + 11 bits) and returns the equivalent fast entry, or
// kLutSlow for a code that matches nothing or a symbol invalid for the table's class.
__device__ __noinline__ uint32_t slow_symbol(const HuffTable* t, uint32_t w, uint32_t e, bool dc) {
  uint32_t L = e & 31, sym = (e >> 20) & 255;
  if (L == 0) {
    const uint32_t top = w >> 16;
#pragma unroll 1
    for (int l = kLutBits + 1; l <= 16; ++l) {
      const int code = (int)(top >> (16 - l));
      if (code <= t->maxcode[l]) {
        const int vi = code + t->valoff[l];
        if (vi < 0 || vi > 255) return kLutSlow;
        sym = t->vals[vi];
        L = (uint32_t)l;
        break;
      }
    }
    if (L == 0) return kLutSlow;
  }
  const uint32_t r = dc ? 0 : sym >> 4, s = dc ? sym : sym & 15;
  if (s > (dc ? 11u : 10u)) return kLutSlow;
  if (!dc && s == 0) {
    if (r == 0) return lut_fast(L, 64, 63, false, 0);   // end of block
    if (r == 15) return lut_fast(L, 16, 15, false, 0);  // zero run of 16
    return kLutSlow;
  }
  const uint32_t bits = s ? (w << L) >> (32 - s) : 0u;
  const int v = s ? ((int)bits - ((bits < (1u << (s - 1))) ? (int)((1u << s) - 1u) : 0)) : 0;
  return dc ? lut_fast(L + s, 1, 0, false, v) : lut_fast(L + s, r + 1, r, true, v);
}

// Entropy-decodes all data units of one MCU into coef[(du * 64 + k) * M] (quantised, zig-zag
// k; the buffer must be zero on entry). One symbol per loop iteration. The common symbol —
// an AC value, end of block, zero run or DC difference whose code and value bits fit the
// 10-bit window — is one LUT read and a fixed straight sequence: consume, (DC: add the
// component's predictor), store at k + offset, advance k. hs: the lane's table set; hs_sa:
// its shared-memory address when it is the staged set, else 0 (generic reads).
// Returns false on an invalid coding.
template <int M>
__device__ __forceinline__ bool decode_mcu(BitReader& br, const HuffTable* hs, uint32_t hs_sa, int ndu, int16_t& p0,
                                           int16_t& p1, int16_t& p2, int16_t* coef) {
  int du = 0, k = 0, comp = 0;
  int pc = p0;  // DC predictor of the current data unit's component
  uint32_t dct = 0;  // table index of the component's DC table (0 luma, 2 chroma)
  bool bad = false;
  int16_t* blk = coef;
#pragma unroll 1
  for (int it = 0; it < 64 * 6; ++it) {  // at most 64 symbols per data unit
    br.refill();
    const uint32_t w = br.peek();
    const bool dc = k == 0;
    const uint32_t ti = dct + (dc ? 0u : 1u);
    const uint32_t li = w >> (32 - kLutBits);
    uint32_t e = hs_sa ? lds_u32(hs_sa + ti * (uint32_t)sizeof(HuffTable) + li * 4u) : hs[ti].lut[li];
    if (e & kLutSlow) {
      e = slow_symbol(hs + ti, w, e, dc);
      if (e & kLutSlow) return false;
    }
    const uint32_t nb = e & 31, adv = (e >> 5) & 127, sofs = (e >> 12) & 63;
    const bool chk = (e >> 18) & 1;
    int v = (int)e >> 20;
    br.pos += nb;
    if (dc) {
      pc = (int16_t)(uint16_t)(pc + v);  // DC values wrap modulo 2^16
      v = pc;
    }
    const int kst = k + (int)sofs;
    bad |= chk && kst > 63;
    blk[min(kst, 63) * M] = (int16_t)v;
    k += (int)adv;
    if (k >= 64) {  // data unit done
      if (bad) return false;
      if (comp == 0) p0 = (int16_t)pc;
      if (comp == 1) p1 = (int16_t)pc;
      if (comp == 2) p2 = (int16_t)pc;
      if (++du == ndu) return true;
      comp = du < ndu - 2 ? 0 : (du == ndu - 2 ? 1 : 2);
      pc = comp == 0 ? p0 : (comp == 1 ? p1 : p2);
      dct = comp == 0 ? 0u : 2u;
      blk += 64 * M;
      k = 0;
    }
  }
  return false;
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

// Word offset of row y of data unit d inside an MCU's pixel buffer, and the row pitch.
__device__ __forceinline__ int pix_row(int d, int y, bool s420) {
  if (s420) return d < 4 ? ((d >> 1) * 8 + y) * 4 + (d & 1) * 2 : 64 + (d - 4) * 16 + y * 2;
  return (d == 0 ? 0 : (d == 1 ? 64 : 80)) + y * 2;
}

template <int M>
__global__ void k_decode(const __grid_constant__ DecodeArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  HuffSet* sh = reinterpret_cast<HuffSet*>(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* wbase = smem + sizeof(HuffSet) + 64 + (size_t)warp * warp_smem(M);
  int16_t* coef = reinterpret_cast<int16_t*>(wbase);                       // [6][64][M]
  uint32_t* pix = reinterpret_cast<uint32_t*>(wbase + 6 * 64 * M * 2);     // [M][97]
  uint16_t* qtab = reinterpret_cast<uint16_t*>(pix + M * kPixStride);      // [M][2][64] zig-zag
  uint32_t* moff = reinterpret_cast<uint32_t*>(qtab + M * 128);            // [M] cache unit offset
  uint32_t* minfo = moff + M;  // [M] ndu | 420 << 4 | store << 5 | qset << 8
  uint32_t* stage = minfo + M;  // [M][kStageWords] entropy-coded words

  {  // stage Huffman set 0
    const uint4* src = reinterpret_cast<const uint4*>(a.huff);
    uint4* dst = reinterpret_cast<uint4*>(sh);
    for (int i = threadIdx.x; i < (int)(sizeof(HuffSet) / 16); i += blockDim.x) dst[i] = __ldg(src + i);
  }
  __syncthreads();

  const uint32_t count = min(*(volatile uint32_t*)&a.state->count, a.work_cap);
  bool any_bad = false;

#pragma unroll 1
  for (;;) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&a.state->decode_next, (uint32_t)M);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (base >= count) break;

    // ---- set-up: lane m < M takes item base + m ----
    const uint32_t item = base + lane;
    bool act = lane < M && item < count;
    const uint32_t gid = act ? __ldg(a.work + item) : 0u;
    int d0 = 0;  // the first item's level is shared by nearly all lanes (the list is sorted)
    if (lane == 0) d0 = find_desc(a.descs, (int)a.ndesc, gid);
    d0 = __shfl_sync(0xFFFFFFFFu, d0, 0);
    int ndu = 0;
    bool s420 = true, store = false, bad = false;
    uint32_t off = 0, nbits = 0, qset = 0;
    BitReader br;
    int16_t pr0 = 0, pr1 = 0, pr2 = 0;
    const HuffTable* hs = sh->t;
    if (act) {
      int di = d0;
      const uint32_t b0 = __ldg(&a.descs[d0].gid_base);
      if (gid < b0 || gid - b0 >= __ldg(&a.descs[d0].nmcu)) di = find_desc(a.descs, (int)a.ndesc, gid);
      const DevDesc d = a.descs[di];
      const uint32_t mcu = gid - d.gid_base;
      if (d.sampling == kSamplingCoef || mcu >= d.nmcu) {
        act = false;  // not a JPEG level: nothing to decode
      } else {
        s420 = d.sampling == kSampling420;
        ndu = s420 ? 6 : 3;
        off = __ldg(a.slot + gid);
        store = off + d.units <= a.cap_units;
        const uint16_t* ix = d.index + (size_t)mcu * 5;
        const uint32_t bitpos = (uint32_t)__ldg(ix) | ((uint32_t)__ldg(ix + 1) << 16);
        pr0 = (int16_t)__ldg(ix + 2);
        pr1 = (int16_t)__ldg(ix + 3);
        pr2 = (int16_t)__ldg(ix + 4);
        br.words = d.stream;
        br.nwords = d.nwords;
        nbits = d.nbits;
        // stage the MCU's words (from its first word, 16 B aligned, to the next MCU's start
        // plus the reader's look-ahead) with independent vector loads
        const uint32_t endbit = mcu + 1 < d.nmcu ? ((uint32_t)__ldg(ix + 5) | ((uint32_t)__ldg(ix + 6) << 16)) : d.nbits;
        const uint32_t w0 = (bitpos >> 5) & ~3u;
        uint32_t want = (max(endbit, bitpos) >> 5) + 6 - w0;
        want = min((want + 3) & ~3u, (uint32_t)kStageWords);
        if (w0 + want > d.nwords) want = d.nwords > w0 ? (d.nwords - w0) & ~3u : 0u;
        br.base = w0;
        br.nstage = want;
        br.stage_sa = (uint32_t)__cvta_generic_to_shared(stage + lane * kStageWords);
        const uint4* src4 = reinterpret_cast<const uint4*>(d.stream + w0);
        uint4* dst4 = reinterpret_cast<uint4*>(stage + lane * kStageWords);
#pragma unroll 1
        for (uint32_t j = 0; j < want / 4; j += 4) {
          uint4 r[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) r[t] = j + t < want / 4 ? __ldg(src4 + j + t) : make_uint4(0, 0, 0, 0);
#pragma unroll
          for (int t = 0; t < 4; ++t)
            if (j + t < want / 4) dst4[j + t] = r[t];
        }
        br.init(bitpos);
        if (d.hset != 0) hs = a.huff[d.hset].t;
        qset = d.qset;
      }
    }
    if (lane < M) {
      moff[lane] = off;
      minfo[lane] = act ? ((uint32_t)ndu | (s420 ? 16u : 0u) | (store ? 32u : 0u) | (qset << 8)) : 0u;
    }
    {  // clear the coefficient buffer (768 M bytes)
      uint4* z = reinterpret_cast<uint4*>(coef);
#pragma unroll
      for (int i = lane; i < 48 * M; i += 32) z[i] = make_uint4(0, 0, 0, 0);
    }
    __syncwarp();
    {  // stage each MCU's quantisation tables (256 B = 16 x 16 B per MCU)
      const uint4* qsrc = reinterpret_cast<const uint4*>(a.quant);
      uint4* qdst = reinterpret_cast<uint4*>(qtab);
#pragma unroll
      for (int i = lane; i < 16 * M; i += 32) qdst[i] = __ldg(qsrc + (size_t)(minfo[i >> 4] >> 8) * 16 + (i & 15));
    }

    // ---- entropy phase: each active lane decodes all data units of its MCU ----
    if (act) {
      const uint32_t hs_sa = hs == sh->t ? (uint32_t)__cvta_generic_to_shared(sh->t) : 0u;
      if (!decode_mcu<M>(br, hs, hs_sa, ndu, pr0, pr1, pr2, coef + lane)) bad = true;
      if (!bad && br.position() > nbits) bad = true;
      any_bad |= bad;
    }
    __syncwarp();

    // ---- IDCT column pass: for each column u, the 6M data units spread over the lanes.
    // Dequantise on load: d = clamp16(q * Q[k]); t = clamp16(floor((sum + 2^8) / 2^9)),
    // written back in place (column u of t occupies the zig-zag slots of column u).
#pragma unroll
    for (int u = 0; u < 8; ++u) {
#pragma unroll 1
      for (int j = lane; j < 6 * M; j += 32) {
        const int d = j / M, m = j % M;
        const uint32_t info = minfo[m];
        if (d >= (int)(info & 7)) continue;
        int16_t* blk = coef + (size_t)d * 64 * M + m;
        const uint16_t* Q = qtab + m * 128 + (d < (int)(info & 7) - 2 ? 0 : 64);
        int in[8], out[8];
        int any = 0;
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          const int k = zz_pos(v, u);
          const int q = blk[k * M];
          any |= q;
          in[v] = sat16(q * (int)Q[k]);
        }
        if (any == 0) continue;  // an all-zero column stays zero
        idct8(in, out);
#pragma unroll
        for (int y = 0; y < 8; ++y) blk[zz_pos(y, u) * M] = (int16_t)sat16((out[y] + 256) >> 9);
      }
    }
    __syncwarp();

    // ---- IDCT row pass: for each row y, the 6M data units spread over the lanes -> pixels
#pragma unroll
    for (int y = 0; y < 8; ++y) {
#pragma unroll 1
      for (int j = lane; j < 6 * M; j += 32) {
        const int d = j / M, m = j % M;
        const uint32_t info = minfo[m];
        if (d >= (int)(info & 7)) continue;
        const int16_t* blk = coef + (size_t)d * 64 * M + m;
        int in[8], out[8];
#pragma unroll
        for (int x = 0; x < 8; ++x) in[x] = blk[zz_pos(y, x) * M];
        idct8(in, out);
        uint32_t w0 = 0, w1 = 0;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          w0 |= clamp255(((out[x] + (1 << 18)) >> 19) + 128) << (8 * x);
          w1 |= clamp255(((out[x + 4] + (1 << 18)) >> 19) + 128) << (8 * x);
        }
        uint32_t* dst = pix + m * kPixStride + pix_row(d, y, (info & 16) != 0);
        dst[0] = w0;
        dst[1] = w1;
      }
    }
    __syncwarp();

    // ---- colour conversion + coalesced tile stores, one MCU at a time ----
#pragma unroll 1
    for (int m = 0; m < M; ++m) {
      const uint32_t info = minfo[m];
      if (!(info & 32)) continue;
      const uint32_t* P = pix + m * kPixStride;
      uint8_t* tile = a.cache + (size_t)moff[m] * kUnitBytes;
      if (info & 16) {  // 4:2:0, 16x16: lane = (row r, half h)
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
      } else {  // 4:4:4, 8x8: lane = (row r, quarter q)
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

size_t smem_bytes(int warps, int M) { return sizeof(HuffSet) + 64 + (size_t)warps * warp_smem(M); }

template <int M>
int occupancy(int warps) {
  const size_t smem = smem_bytes(warps, M);
  if (smem > 227 * 1024) return 0;
  if (cudaFuncSetAttribute(k_decode<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_decode<M>, warps * 32, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace

size_t decode_smem_bytes(int warps, int mcus_per_warp) { return smem_bytes(warps, mcus_per_warp); }

// The dynamic shared-memory attribute of each variant is set by decode_max_ctas_per_sm(),
// which the context calls for every (warps, M) on its device before the first launch.
void launch_decode(const DecodeArgs& a, int warps, int grid, cudaStream_t s) {
  const size_t smem = smem_bytes(warps, a.mcus_per_warp);
  switch (a.mcus_per_warp) {
    case 4: k_decode<4><<<grid, warps * 32, smem, s>>>(a); break;
    case 8: k_decode<8><<<grid, warps * 32, smem, s>>>(a); break;
    case 16: k_decode<16><<<grid, warps * 32, smem, s>>>(a); break;
    default: k_decode<32><<<grid, warps * 32, smem, s>>>(a); break;
  }
}

int decode_max_ctas_per_sm(int warps, int mcus_per_warp) {
  switch (mcus_per_warp) {
    case 4: return occupancy<4>(warps);
    case 8: return occupancy<8>(warps);
    case 16: return occupancy<16>(warps);
    case 32: return occupancy<32>(warps);
  }
  return 0;
}

void idct_constants(int out[8]) {
  const int c[8] = {0, C1, C2, C3, C4, C5, C6, C7};
  for (int i = 0; i < 8; ++i) out[i] = c[i];
}

}  // namespace jt
