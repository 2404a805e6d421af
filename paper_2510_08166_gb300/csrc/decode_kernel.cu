// Decode (paper Sec. 4.3): every MCU of the work list is Huffman-decoded from its index
// entry (bit offset + DC predictors, Sec. 5.1 / Sec. 5.3), dequantised, inverse-DCT'd,
// chroma-upsampled, colour-converted and written as an RGBA8 tile into the block cache.
//
// GB300 design (the paper's one 64-thread block per MCU with a 32-lane code compare,
// Sec. 5.2, is prior art here):
//  * persistent grid; each warp takes batches of m_eff work items (one per lane), m_eff the
//    smallest power of two up to M (4, 8, 16 or 32, the buffer width) that covers the list
//    in one batch per warp, and a long list fills the lanes. A short list (a frame under
//    motion with a warm block cache: at most kWarpMcuMax MCUs per warp) goes one MCU at a
//    time, each decoded by the whole warp (decode_mcu_warp, mcu_warp_pixels), spread first
//    over the SMs. The first batch of each warp is fixed by its rank, later ones come from a
//    device counter, so uneven MCU sizes balance dynamically and the count never goes to
//    the host;
//  * entropy phase: lane m < m_eff runs MCU m's serial entropy chain over all its data
//    units from a byte-swapped copy of its words staged in shared memory (a per-warp pool
//    shared out by a prefix sum). Per symbol: one funnel shift of a two-word window, one
//    10-bit LUT read (16-bit entries: code length, value size, run) together with an
//    independent read of the second-level entry for codes longer than 10 bits, the value
//    cut from the same window without a branch, and a select to advance the window. The
//    quantised coefficients go in zig-zag order into a per-warp buffer coef[du][k][m]
//    (int16). Nothing but the LUT and the stream is read on this serial chain:
//    dequantisation waits for the IDCT phase;
//  * IDCT phase: the batch's data units are shared out over all 32 lanes, one (data unit,
//    MCU) pair per lane and round; lanes of one round read consecutive columns of the
//    buffer (conflict-free), and all zig-zag positions are compile-time constants. Columns
//    are dequantised on load with the MCU's quantisation table (read through L1); even/odd
//    butterflies give an exact integer factorisation of the matrix product of the decode
//    spec; the row pass writes each row's pixels in place over the slots it just read;
//  * colour phase: 4:2:0 tiles are shared out as (MCU, group of four texels) pairs, 16-byte
//    stores; 4:4:4 and reduced-resolution tiles are written by the MCU's own lane.
//    The buffers per MCU are 768 B of coefficients plus 128 B of staged words, so up to
//    seven 32-MCU warps fit on an SM.
//
// Decode spec (identical in the oracle): dequantised d = clamp16(q * Q); column pass
// t = clamp16(floor((sum_v K[y][v] d[v][u] + 2^8) / 2^9)); row pass
// p = clamp(floor((sum_u K[x][u] t[y][u] + 2^18) / 2^19) + 128, 0, 255) with
// K[x][u] = round(2^14 c_u cos((2x+1) u pi / 16)); JFIF colour in 16-bit fixed point;
// 4:2:0 chroma replicated within the MCU; DC values wrap modulo 2^16.
#include <cuda_runtime.h>

#include <cstddef>

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

// N-point IDCT of the N lowest frequencies, N = 4, 2, 1 (reduced-resolution decode):
// out[x] = sum_u K_N[x][u] in[u] with K_N[x][u] = round(2^14 c_u cos((2x+1) u pi / (2N))) and
// the 8-point c_u. The N-point cosines are the 8-point ones at even multiples, so N = 4 is
// the even half of idct8 (inputs at 0, 2, 4, 6), N = 2 its first butterfly, N = 1 the DC term.
template <int N>
__device__ __forceinline__ void idct_small(const int in[4], int out[4]) {
  if (N == 4) {
    const int a0 = C4 * (in[0] + in[2]), a1 = C4 * (in[0] - in[2]);
    const int b0 = C2 * in[1] + C6 * in[3], b1 = C6 * in[1] - C2 * in[3];
    out[0] = a0 + b0; out[1] = a1 + b1; out[2] = a1 - b1; out[3] = a0 - b0;
  } else if (N == 2) {
    out[0] = C4 * (in[0] + in[1]);
    out[1] = C4 * (in[0] - in[1]);
  } else {
    out[0] = C4 * in[0];
  }
}

// Words of the MCUs' entropy-coded data copied to shared memory before their serial decode
// (random loads from HBM take thousands of cycles and would otherwise sit on the serial
// chain once per word). A warp has kStageWords words per MCU as one pool, shared out by a
// prefix sum over its lanes, so a long MCU can use what short ones leave (the mean MCU of a
// scene needs about a quarter). Words are stored big-endian-swapped; a lane whose MCU does
// not fit reads the rest from global memory.
constexpr int kStageWords = 32;

// Shared memory of one warp: coefficients [6][64][M] int16 (zig-zag order k, lane m at
// column m; after the row pass each data unit's slots hold its pixels, see below) and the
// staged entropy-coded words [M * kStageWords].
__host__ __device__ constexpr size_t warp_smem(int M) {
  return (size_t)6 * 64 * M * 2 + (size_t)M * kStageWords * 4;
}

__device__ __forceinline__ uint32_t bswap(uint32_t w) { return __byte_perm(w, 0, 0x0123); }

// Stream word i (relative to the lane's first staged word): from the staged copy when it is
// there, else from global memory (past the end of the stream: 0).
__device__ __forceinline__ uint32_t lds_u32(uint32_t saddr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(saddr));
  return v;
}
__device__ __forceinline__ uint32_t lds_u16(uint32_t saddr) {
  uint16_t v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(saddr));
  return v;
}

// Stream word i (relative to the lane's first staged word): from the staged copy (shared
// memory address st) when it is there, else from global memory (past the end: 0).
struct Words {
  uint32_t st;            // shared-memory address of the staged, byte-swapped words
  uint32_t nst;           // words staged
  const uint32_t* gw;     // stream words from the first staged word on
  uint32_t ngw;           // readable words from gw on
  __device__ __forceinline__ uint32_t operator()(uint32_t i) const {
    if (i < nst) return lds_u32(st + 4 * i);
    return i < ngw ? bswap(__ldg(gw + i)) : 0u;
  }
};

// Reads of the table set on the serial chain: explicit shared-memory loads for the staged
// set (address hs_sa), generic loads through hs otherwise.
template <bool SH>
struct Tables {
  const HuffTable* hs;
  uint32_t hs_sa;
  __device__ __forceinline__ uint32_t lut(uint32_t ti, uint32_t i) const {
    return SH ? lds_u16(hs_sa + ti * (uint32_t)sizeof(HuffTable) + i * 2) : (uint32_t)hs[ti].lut[i];
  }
  __device__ __forceinline__ uint32_t lut2(uint32_t ti, uint32_t j) const {
    return SH ? lds_u16(hs_sa + ti * (uint32_t)sizeof(HuffTable) + (uint32_t)offsetof(HuffTable, lut2) + j * 2)
              : (uint32_t)hs[ti].lut2[j];
  }
  __device__ __forceinline__ uint32_t first16(uint32_t ti) const {
    return SH ? lds_u32(hs_sa + ti * (uint32_t)sizeof(HuffTable) + (uint32_t)offsetof(HuffTable, first16))
              : hs[ti].first16;
  }
  __device__ __forceinline__ uint32_t n2(uint32_t ti) const {
    return SH ? lds_u32(hs_sa + ti * (uint32_t)sizeof(HuffTable) + (uint32_t)offsetof(HuffTable, n2)) : hs[ti].n2;
  }
  // table ti as a byte address (shared) or byte offset from hs (global), and reads through it
  __device__ __forceinline__ uint32_t base(uint32_t ti) const {
    return (SH ? hs_sa : 0u) + ti * (uint32_t)sizeof(HuffTable);
  }
  __device__ __forceinline__ uint32_t lut_at(uint32_t b, uint32_t i) const {
    return SH ? lds_u16(b + i * 2) : (uint32_t)*reinterpret_cast<const uint16_t*>(reinterpret_cast<const char*>(hs) + b + i * 2);
  }
  __device__ __forceinline__ uint32_t lut2_at(uint32_t b, uint32_t j) const {
    const uint32_t o = b + (uint32_t)offsetof(HuffTable, lut2) + j * 2;
    return SH ? lds_u16(o) : (uint32_t)*reinterpret_cast<const uint16_t*>(reinterpret_cast<const char*>(hs) + o);
  }
};

// Symbol entry by the MAXCODE walk (T.81 F.2.2.3), or 0 for an invalid code or a symbol
// invalid for the table's class. Only codes without a LUT entry come here.
__device__ __noinline__ uint32_t walk_symbol(const HuffTable* t, uint32_t w, bool dc) {
  const uint32_t top = w >> 16;
#pragma unroll 1
  for (int l = 1; l <= 16; ++l) {
    const int code = (int)(top >> (16 - l));
    if (code <= t->maxcode[l]) {
      const int vi = code + t->valoff[l];
      if (vi < 0 || vi > 255) return 0;
      const uint32_t sym = t->vals[vi];
      const uint32_t r = dc ? 0 : sym >> 4, s = dc ? sym : sym & 15;
      if (s > (dc ? 11u : 10u)) return 0;
      if (!dc && s == 0) return r == 0 ? huff_entry(l, 0, kRunEob) : (r == 15 ? huff_entry(l, 0, 15) : 0u);
      return huff_entry(l, s, r);
    }
  }
  return 0;
}

// Entropy-decodes all data units of one MCU into coef[(du * 64 + k) * M] (quantised, zig-zag
// k; the buffer must be zero on entry). One symbol per iteration, on a short dependent
// chain: a funnel shift cuts the next 32 bits from the two-word window (hi:lo), one LUT
// read gives (l, s, r), the s value bits are cut from the same window (T.81 EXTEND without
// a branch), and the window advances by a select; the next stream word is read ahead. The
// move to the next data unit (predictor save/restore, table choice) is also branch-free.
// hs: the lane's tables (shared or global memory). CPT: the compact form, where the first
// luma data unit and the chroma data units carry no DC difference and their DCs are
// p0, p1, p2 as given. Returns the bit position after the MCU relative to the first staged
// word, or 0xFFFFFFFF on an invalid coding.
template <int M, bool SH, bool CPT>
__device__ __forceinline__ uint32_t decode_mcu(const Words& W, uint32_t bit0, const Tables<SH>& T, int ndu,
                                               int16_t& p0, int16_t& p1, int16_t& p2, int16_t* coef) {
  constexpr bool cpt = CPT;
  uint32_t widx = bit0 >> 5, pos = bit0 & 31;
  uint32_t hi = W(widx), lo = W(widx + 1), nx = W(widx + 2);
  // second-level ranges of the four tables, held in registers so that no table read other
  // than the two LUT entries sits on the chain
  const uint32_t F0 = T.first16(0), F1 = T.first16(1), F2 = T.first16(2), F3 = T.first16(3);
  const uint32_t N0 = T.n2(0), N1 = T.n2(1), N2 = T.n2(2), N3 = T.n2(3);
  int du = 0, k = cpt ? 1 : 0, comp = 0, pc = p0, q0 = p0, q1 = p1, q2 = p2;
  // the table of the symbol being decoded (0 DC luma, 1 AC luma, 2 DC chroma, 3 AC chroma),
  // its address and second-level range. The two possible successors (the next data unit's
  // first table, or this one's AC table) are prepared before the symbol is read, so the
  // symbol only has to select between them: a short dependent chain from one LUT read to the
  // next.
  uint32_t tcur = cpt ? 1u : 0u;
  uint32_t bcur = T.base(tcur), fcur = cpt ? F1 : F0, ncur = cpt ? N1 : N0;
  uint32_t boff = 0;
  if (cpt) coef[0] = (int16_t)pc;
  bool bad = false;
#pragma unroll 1
  for (int it = 0; it < 64 * 6; ++it) {  // at most 64 symbols per data unit
    // successors, off the chain: the next data unit's component and first table, and the
    // AC table of this data unit
    const int cn1 = du + 1 < ndu - 2 ? 0 : (du + 1 == ndu - 2 ? 1 : 2);
    const uint32_t tA = cn1 ? (cpt ? 3u : 2u) : 0u, tB = tcur | 1u;
    const uint32_t bA = T.base(tA), bB = T.base(tB);
    const uint32_t fA = cn1 ? (cpt ? F3 : F2) : F0, fB = (tcur & 2u) ? F3 : F1;
    const uint32_t nA = cn1 ? (cpt ? N3 : N2) : N0, nB = (tcur & 2u) ? N3 : N1;
    const int lim = 63 - k;  // the data unit ends when the run reaches it
    const bool dc = k == 0;

    const uint32_t w = __funnelshift_l(lo, hi, pos);
    // both levels read at once (independent loads): the first-level entry when the code is
    // short, else the second-level entry of the 16-bit prefix
    const uint32_t e1 = T.lut_at(bcur, w >> (32 - kLutBits));
    const uint32_t j = (w >> 16) - fcur;
    const uint32_t e2 = T.lut2_at(bcur, min(j, (uint32_t)kLut2Size - 1u));
    uint32_t e = (e1 & 31u) ? e1 : (j < ncur ? e2 : 0u);
    if (e == 0) {  // no table entry: the MAXCODE walk decodes or rejects it
      e = walk_symbol(T.hs + tcur, w, dc);
      if (e == 0) {
        bad = true;
        break;
      }
    }
    const uint32_t l = e & 31u, sz = (e >> 5) & 15u, r = e >> 9;
    const bool done = (int)r >= lim;  // data unit complete
    tcur = done ? tA : tB;
    bcur = done ? bA : bB;
    fcur = done ? fA : fB;
    ncur = done ? nA : nB;
    const uint32_t tw = w << l;
    // EXTEND: the s bits after the code; a leading 0 bit makes the value negative
    int v = (int)__funnelshift_l(tw, 0u, sz) + (int)(~((int)tw >> 31) & (int)(1u - (1u << sz)));
    pos += l + sz;
    const bool step = pos >= 32;
    hi = step ? lo : hi;
    lo = step ? nx : lo;
    pos = step ? pos - 32 : pos;
    widx += step ? 1u : 0u;
    nx = W(widx + 2);
    const int dcv = (int16_t)(uint16_t)(pc + v);  // DC values wrap modulo 2^16
    v = dc ? dcv : v;
    pc = dc ? dcv : pc;
    const int kst = k + (int)r;
    bad |= sz != 0 && kst > 63;
    coef[(boff + (uint32_t)min(kst, 63)) * M] = (int16_t)v;
    q0 = done && comp == 0 ? pc : q0;
    q1 = done && comp == 1 ? pc : q1;
    q2 = done && comp == 2 ? pc : q2;
    du += done ? 1 : 0;
    pc = done ? (cn1 == 0 ? q0 : (cn1 == 1 ? q1 : q2)) : pc;
    comp = done ? cn1 : comp;
    boff += done ? 64u : 0u;
    k = done ? ((cpt && cn1 != 0) ? 1 : 0) : kst + 1;
    if (du == ndu || bad) break;
    if (cpt && done && cn1 != 0) coef[boff * M] = (int16_t)pc;  // compact form: a stored chroma DC
  }
  p0 = (int16_t)q0;
  p1 = (int16_t)q1;
  p2 = (int16_t)q2;
  return (bad || du != ndu) ? 0xFFFFFFFFu : widx * 32 + pos;
}

// Entropy-decodes one data unit of component comp (0 luma, else chroma) from bit0 into
// coef[k * M] (zig-zag k; zero on entry); its DC slot receives the DC *difference* (the
// caller chains it). Same symbol step as decode_mcu, without data-unit transitions: the DC
// table for the first symbol, then the AC table. Returns the bit position after the unit
// relative to the first staged word, or 0xFFFFFFFF on an invalid coding.
template <int M, bool SH>
__device__ __forceinline__ uint32_t decode_unit(const Words& W, uint32_t bit0, const Tables<SH>& T, int comp,
                                                int16_t* coef) {
  uint32_t widx = bit0 >> 5, pos = bit0 & 31;
  uint32_t hi = W(widx), lo = W(widx + 1), nx = W(widx + 2);
  const uint32_t tdc = comp ? 2u : 0u, tac = tdc | 1u;
  const uint32_t bac = T.base(tac), fac = T.first16(tac), nac = T.n2(tac);
  uint32_t tcur = tdc, bcur = T.base(tdc), fcur = T.first16(tdc), ncur = T.n2(tdc);
  int k = 0;
  bool bad = false;
#pragma unroll 1
  for (int it = 0; it < 64; ++it) {  // every symbol advances k by at least one
    const uint32_t w = __funnelshift_l(lo, hi, pos);
    const uint32_t e1 = T.lut_at(bcur, w >> (32 - kLutBits));
    const uint32_t j = (w >> 16) - fcur;
    const uint32_t e2 = T.lut2_at(bcur, min(j, (uint32_t)kLut2Size - 1u));
    uint32_t e = (e1 & 31u) ? e1 : (j < ncur ? e2 : 0u);
    if (e == 0) {
      e = walk_symbol(T.hs + tcur, w, k == 0);
      if (e == 0) {
        bad = true;
        break;
      }
    }
    const uint32_t l = e & 31u, sz = (e >> 5) & 15u, r = e >> 9;
    const uint32_t tw = w << l;
    const int v = (int)__funnelshift_l(tw, 0u, sz) + (int)(~((int)tw >> 31) & (int)(1u - (1u << sz)));
    pos += l + sz;
    const bool step = pos >= 32;
    hi = step ? lo : hi;
    lo = step ? nx : lo;
    pos = step ? pos - 32 : pos;
    widx += step ? 1u : 0u;
    nx = W(widx + 2);
    const int kst = k + (int)r;
    bad |= sz != 0 && kst > 63;
    coef[min(kst, 63) * M] = (int16_t)v;
    k = kst + 1;
    tcur = tac;
    bcur = bac;
    fcur = fac;
    ncur = nac;
    if (k >= 64 || bad) break;
  }
  return (bad || k < 64) ? 0xFFFFFFFFu : widx * 32 + pos;
}

// ---- one MCU decoded by a whole warp (short work lists) ----
//
// A warp that holds a single MCU would run its serial chain on one lane, and every step of
// that chain (window cut, LUT read, length, position, coefficient store) waits for the one
// before. Here the 32 lanes instead decode, for every bit offset of a 256-bit window of the
// stream, the AC symbol that would start there (entries independent of each other, 8 per
// lane, loads issued before any store), and the chain that remains is one shared-memory read
// per one or two symbols: the slot at the current position holds the byte offset of the slot
// after its symbol (code + value bits), its run and its value, and the same for the symbol
// after it, so a read serves two symbols unless the first ends the data unit. All lanes follow the chain in
// step, so its state is warp-uniform; symbol s of a data unit is kept in registers by lane
// s mod 32, and the coefficients are stored once the data unit ends (a store on the chain
// would hold the next table read behind it). The DC symbol of each data unit is decoded
// directly on the chain. The window is rebuilt when the position leaves it or the component
// class (luma, chroma) changes.
constexpr int kWinBits = 256;    // window of symbol entries, bits (128 when the buffer is 4 MCUs wide)
constexpr int kWarpMcuMax = 4;   // lists of at most this many MCUs per warp are decoded MCU by MCU

// LUT entry of the code at the top of w in table ti (0 when it has none).
template <bool SH>
__device__ __forceinline__ uint32_t lut_entry(const Tables<SH>& T, uint32_t ti, uint32_t f, uint32_t n, uint32_t w) {
  const uint32_t b = T.base(ti);
  const uint32_t e1 = T.lut_at(b, w >> (32 - kLutBits));
  const uint32_t j = (w >> 16) - f;
  const uint32_t e2 = T.lut2_at(b, min(j, (uint32_t)kLut2Size - 1u));
  return (e1 & 31u) ? e1 : (j < n ? e2 : 0u);
}

// Signed value of the sz bits after the l-bit code at the top of w (T.81 EXTEND).
__device__ __forceinline__ int symbol_value(uint32_t w, uint32_t l, uint32_t sz) {
  const uint32_t tw = w << l;
  return (int)__funnelshift_l(tw, 0u, sz) + (int)(~((int)tw >> 31) & (int)(1u - (1u << sz)));
}

// Window slot of symbol entry e read at w, window offset o, in a window of WIN bits (16-byte
// slots). First word: byte offset in the window of the slot after the symbol, clamped to the
// last slot (bits 0-11), run (12-17), value bits present (18), the next symbol starts past
// the window (19), the next symbol's window offset (20-28); 0 for no symbol (an invalid
// code), never 0 otherwise (the next offset is at least 1). Second word: the value.
template <int WIN>
__device__ __forceinline__ uint2 win_entry(uint32_t e, uint32_t w, uint32_t o) {
  const uint32_t l = e & 31u, sz = (e >> 5) & 15u, r = e >> 9, nx = o + l + sz;
  const uint32_t x = (min(nx, (uint32_t)WIN - 1u) * 16u) | (r << 12) | (sz ? 1u << 18 : 0u) |
                     (nx >= (uint32_t)WIN ? 1u << 19 : 0u) | (nx << 20);
  return e ? make_uint2(x, (uint32_t)symbol_value(w, l, sz)) : make_uint2(0u, 0u);
}

__device__ __forceinline__ uint2 lds_u64(uint32_t saddr) {
  uint2 v;
  asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(saddr));
  return v;
}
__device__ __forceinline__ uint4 lds_u128(uint32_t saddr) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(saddr));
  return v;
}

// Stream words of a warp-decoded MCU that is staged whole (every word its symbols can reach
// is in shared memory): reads need no bounds branch; an index past the stage (only an invalid
// coding gets there) is clamped into the stage.
struct StagedWords {
  uint32_t st, last;  // shared address of the staged words, index of the last one
  __device__ __forceinline__ uint32_t operator()(uint32_t i) const { return lds_u32(st + 4 * min(i, last)); }
};

// The 32 stream bits from bit position p on (relative to the first staged word).
template <class WS>
__device__ __forceinline__ uint32_t bits32w(const WS& W, uint32_t p) {
  return __funnelshift_l(W((p >> 5) + 1), W(p >> 5), p & 31u);
}

// Entropy-decodes all data units of one MCU with the whole warp (every lane calls it with the
// same arguments). Coefficients go to cc[du * 64 + k] (contiguous, zig-zag k; zero on entry);
// tbl_sa is the 16-byte aligned shared address of WIN 16-byte slots of scratch. Slot o holds
// the symbol starting at window offset o and, when it stays in the window, the symbol right
// after it, so one read serves two symbols unless the first ends the data unit. Same
// results and the same invalid codings as decode_mcu. Returns the bit position after the
// MCU relative to the first staged word, or 0xFFFFFFFF on an invalid coding.
template <bool SH, bool CPT, int WIN, class WS>
__device__ __forceinline__ uint32_t decode_mcu_warp(const WS& W, uint32_t bit0, const Tables<SH>& T, int ndu,
                                                    int p0, int p1, int p2, int16_t* cc, uint32_t tbl_sa,
                                                    int lane) {
  constexpr int J = WIN / 32;  // slots per lane
  const uint32_t F0 = T.first16(0), F1 = T.first16(1), F2 = T.first16(2), F3 = T.first16(3);
  const uint32_t N0 = T.n2(0), N1 = T.n2(1), N2 = T.n2(2), N3 = T.n2(3);
  int pred0 = p0, pred1 = p1, pred2 = p2;
  uint32_t pos = bit0, wb = 0;
  int wcls = -1;  // component class of the window's entries (none yet)
  bool bad = false;
#pragma unroll 1
  for (int du = 0; du < ndu && !bad; ++du) {
    const int comp = du < ndu - 2 ? 0 : (du == ndu - 2 ? 1 : 2);
    const int cls = comp ? 1 : 0;
    const uint32_t tdc = cls ? 2u : 0u, tac = tdc | 1u;
    const uint32_t fdc = cls ? F2 : F0, ndc = cls ? N2 : N0, fac = cls ? F3 : F1, nac = cls ? N3 : N1;
    int16_t* cd = cc + du * 64;
    int pv = comp == 0 ? pred0 : (comp == 1 ? pred1 : pred2);
    if (!(CPT && (du == 0 || comp != 0))) {  // the compact form stores these DCs, no difference
      const uint32_t w = bits32w(W, pos);
      uint32_t e = lut_entry(T, tdc, fdc, ndc, w);
      if (e == 0) e = walk_symbol(T.hs + tdc, w, true);
      if (e == 0) {
        bad = true;
        break;
      }
      const uint32_t l = e & 31u, sz = (e >> 5) & 15u;
      pv = (int16_t)(uint16_t)(pv + symbol_value(w, l, sz));  // DC values wrap modulo 2^16
      pos += l + sz;
    }
    pred0 = comp == 0 ? pv : pred0;
    pred1 = comp == 1 ? pv : pred1;
    pred2 = comp == 2 ? pv : pred2;
    // AC symbols: symbol s of the unit is kept by lane s % 32 as k << 16 | value (0: none)
    uint32_t keep0 = 0, keep1 = 0;
    int k = 1, s = 0, kst = 0;
#pragma unroll 1
    while (true) {
      if (wcls != cls || pos - wb >= (uint32_t)WIN) {
        // rebuild the window at pos: every lane's loads first, then its entries
        __syncwarp();  // every lane has read the old window
        wb = pos;
        wcls = cls;
        uint32_t w[J], e[J];
#pragma unroll
        for (int j = 0; j < J; ++j) w[j] = bits32w(W, wb + (uint32_t)(lane + 32 * j));
        bool none = false;
#pragma unroll
        for (int j = 0; j < J; ++j) {
          e[j] = lut_entry(T, tac, fac, nac, w[j]);
          none |= e[j] == 0;
        }
        if (none) {  // codes without a LUT entry: the MAXCODE walk decodes or rejects them
#pragma unroll
          for (int j = 0; j < J; ++j)
            if (e[j] == 0) e[j] = walk_symbol(T.hs + tac, w[j], false);
        }
        uint2 we[J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const uint32_t o = (uint32_t)(lane + 32 * j);
          we[j] = win_entry<WIN>(e[j], w[j], o);
          asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(tbl_sa + 16 * o), "r"(we[j].x), "r"(we[j].y));
        }
        __syncwarp();
        // second halves: the symbol after each slot's symbol, when it starts in the window
        uint2 nb[J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const bool in = we[j].x != 0 && (we[j].x & (1u << 19)) == 0;
          nb[j] = lds_u64(tbl_sa + (we[j].x & 4095u));  // a slot in the window either way
          nb[j] = in ? nb[j] : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int j = 0; j < J; ++j)
          asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(tbl_sa + 16 * (uint32_t)(lane + 32 * j) + 8),
                       "r"(nb[j].x), "r"(nb[j].y));
        __syncwarp();
      }
      // symbols while the position stays in the window, one or two per read; the next
      // slot's read goes out before this one is taken apart (a lone warp issues in order);
      // a read past the window is clamped into it and dropped
      uint4 ent = lds_u128(tbl_sa + 16 * (pos - wb));
      uint32_t nofs = pos - wb;  // window offset of the next symbol
      bool more;
      do {
        const int kstA = k + (int)((ent.x >> 12) & 63u);
        const bool two = kstA < 63 && ent.z != 0;  // the second symbol belongs to this unit
        const uint4 nxt = lds_u128(tbl_sa + ((two ? ent.z : ent.x) & 4095u));
        const bool valA = (ent.x & (1u << 18)) != 0, valB = (ent.z & (1u << 18)) != 0;
        const int kstB = kstA + 1 + (int)((ent.z >> 12) & 63u);
        const uint32_t kvA = valA ? ((uint32_t)kstA << 16) | (ent.y & 0xFFFFu) : 0u;
        const uint32_t kvB = (two && valB) ? ((uint32_t)kstB << 16) | (ent.w & 0xFFFFu) : 0u;
        keep0 = s == lane ? kvA : (s + 1 == lane ? kvB : keep0);
        keep1 = s == lane + 32 ? kvA : (s + 1 == lane + 32 ? kvB : keep1);
        bad |= ent.x == 0 || (valA && kstA > 63) || (two && valB && kstB > 63);
        kst = two ? kstB : kstA;
        s += two ? 2 : 1;
        k = kst + 1;
        const uint32_t last = two ? ent.z : ent.x;
        nofs = last >> 20;
        more = kst < 63 && !bad && (last & (1u << 19)) == 0;
        ent = nxt;
      } while (more);
      pos = wb + nofs;
      if (kst >= 63 || bad) break;
    }
    if (lane == 0) cd[0] = (int16_t)pv;
    if (keep0 != 0 && (keep0 >> 16) <= 63u) cd[keep0 >> 16] = (int16_t)(keep0 & 0xFFFFu);
    if (keep1 != 0 && (keep1 >> 16) <= 63u) cd[keep1 >> 16] = (int16_t)(keep1 & 0xFFFFu);
  }
  return bad ? 0xFFFFFFFFu : pos;
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


// Pixels after the row pass, in place: the row pass of data unit d, row y has just read
// the 8 slots zz_pos(y, 0..7) (no other row reads them) and writes pixels x = 2i, 2i+1 as the
// low and high byte of slot zz_pos(y, i), i < 4. pixel2(d, y, i) reads that pair.
template <int M>
__device__ __forceinline__ uint32_t pixel2(const int16_t* col, int d, int y, int i) {
  return (uint16_t)col[(d * 64 + zz_pos(y, i)) * M];
}

// Reduced-resolution IDCT of one data unit (N = 8 >> R) in place over the buffer: the same
// dequantisation and rounding as the full transform on the N x N lowest frequencies; the
// row pass leaves pixel pairs (x = 2i, 2i+1) in slots zz_pos(y, i), i < N/2 (N = 1: the
// pixel in the low byte of slot 0), which pixel2() reads as for the full size.
template <int M, int R>
__device__ __forceinline__ void idct_reduced(int16_t* blk, const uint16_t* Qd) {
  constexpr int N = 8 >> R;
#pragma unroll
  for (int u = 0; u < N; ++u) {
    int in[4] = {0, 0, 0, 0}, out[4];
#pragma unroll
    for (int v = 0; v < N; ++v) {
      const int k = zz_pos(v, u);
      in[v] = sat16(blk[k * M] * (int)__ldg(Qd + k));
    }
    idct_small<N>(in, out);
#pragma unroll
    for (int y = 0; y < N; ++y) blk[zz_pos(y, u) * M] = (int16_t)sat16((out[y] + 256) >> 9);
  }
#pragma unroll
  for (int y = 0; y < N; ++y) {
    int in[4] = {0, 0, 0, 0}, out[4];
#pragma unroll
    for (int x = 0; x < N; ++x) in[x] = blk[zz_pos(y, x) * M];
    idct_small<N>(in, out);
    if (N == 1) {
      blk[zz_pos(y, 0) * M] = (int16_t)clamp255(((out[0] + (1 << 18)) >> 19) + 128);
    } else {
#pragma unroll
      for (int i = 0; i < N / 2; ++i)
        blk[zz_pos(y, i) * M] = (int16_t)(clamp255(((out[2 * i] + (1 << 18)) >> 19) + 128) |
                                          (clamp255(((out[2 * i + 1] + (1 << 18)) >> 19) + 128) << 8));
    }
  }
}

// Colour conversion of a reduced tile ((mw >> r)^2 texels, mw = 16 at 4:2:0, 8 at 4:4:4),
// chroma replicated 2x2 at 4:2:0 as at full size; one 4-byte store per texel.
template <int M>
__device__ __noinline__ void colour_reduced(const int16_t* col, bool s420, int red, uint32_t* tile) {
  const int n = 8 >> red, tw = (s420 ? 16 : 8) >> red;
  auto pix = [&](int d, int y, int x) { return (pixel2<M>(col, d, y, x >> 1) >> (8 * (x & 1))) & 255u; };
#pragma unroll 1
  for (int ty = 0; ty < tw; ++ty)
#pragma unroll 1
    for (int tx = 0; tx < tw; ++tx) {
      uint32_t Y, cb, cr;
      if (s420) {
        Y = pix((ty / n) * 2 + tx / n, ty % n, tx % n);
        cb = pix(4, ty >> 1, tx >> 1);
        cr = pix(5, ty >> 1, tx >> 1);
      } else {
        Y = pix(0, ty, tx);
        cb = pix(1, ty, tx);
        cr = pix(2, ty, tx);
      }
      int ro, go, bo;
      chroma_offsets(cb, cr, ro, go, bo);
      tile[ty * tw + tx] = ycc_pixel(Y, ro, go, bo);
    }
}

// Full-size IDCT of one data unit in place over the buffer: column pass with dequantisation
// on load, t = clamp16(floor((sum_v K[y][v] clamp16(q Q) + 2^8) / 2^9)), then the row pass
// p = clamp(floor((sum_u K[x][u] t[y][u] + 2^18) / 2^19) + 128, 0, 255), whose pixel pairs
// land in the slots the row just read (see pixel2).
template <int M>
__device__ __forceinline__ void idct_full(int16_t* blk, const uint16_t* Qd) {
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    int in[8], out[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const int k = zz_pos(v, u);
      in[v] = sat16(blk[k * M] * (int)__ldg(Qd + k));
    }
    idct8(in, out);
#pragma unroll
    for (int y = 0; y < 8; ++y) blk[zz_pos(y, u) * M] = (int16_t)sat16((out[y] + 256) >> 9);
  }
#pragma unroll
  for (int y = 0; y < 8; ++y) {
    int in[8], out[8];
#pragma unroll
    for (int x = 0; x < 8; ++x) in[x] = blk[zz_pos(y, x) * M];
    idct8(in, out);
#pragma unroll
    for (int i = 0; i < 4; ++i)
      blk[zz_pos(y, i) * M] = (int16_t)(clamp255(((out[2 * i] + (1 << 18)) >> 19) + 128) |
                                        (clamp255(((out[2 * i + 1] + (1 << 18)) >> 19) + 128) << 8));
  }
}

// IDCT and colour of one full-size MCU held by a whole warp (after decode_mcu_warp): the
// column passes are shared out over the lanes as (data unit, column) pairs, the row passes as
// (data unit, row) pairs, the tile as half rows of texels; same arithmetic as idct_full and
// the per-MCU colour stores. cc: quantised coefficients [ndu][64] in zig-zag order; tmp
// (16-byte aligned, [ndu][64] int16) and pix ([ndu][64] bytes) are scratch in natural order;
// Q: the MCU's quantisation tables (luma, then chroma, zig-zag order); tile: its cache block.
__device__ __forceinline__ void mcu_warp_pixels(const int16_t* cc, int16_t* tmp, uint8_t* pix, int ndu, bool s420,
                                                const uint16_t* Q, uint8_t* tile, int lane) {
  const int nluma = s420 ? 4 : 1;
#pragma unroll 1
  for (int q = lane; q < 8 * ndu; q += 32) {  // column u of data unit d, dequantised on load
    const int d = q >> 3, u = q & 7;
    const uint16_t* Qd = Q + (d < nluma ? 0 : 64);
    int in[8], out[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const int k = zz_pos(v, u);
      in[v] = sat16(cc[d * 64 + k] * (int)__ldg(Qd + k));
    }
    idct8(in, out);
#pragma unroll
    for (int v = 0; v < 8; ++v) tmp[d * 64 + v * 8 + u] = (int16_t)sat16((out[v] + 256) >> 9);
  }
  __syncwarp();
#pragma unroll 1
  for (int q = lane; q < 8 * ndu; q += 32) {  // row y of data unit d
    const int d = q >> 3, y = q & 7;
    const uint4 r = *reinterpret_cast<const uint4*>(tmp + d * 64 + y * 8);
    const uint32_t rw[4] = {r.x, r.y, r.z, r.w};
    int in[8], out[8];
#pragma unroll
    for (int x = 0; x < 8; ++x) in[x] = (int16_t)(uint16_t)(rw[x >> 1] >> (16 * (x & 1)));
    idct8(in, out);
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      lo |= clamp255(((out[x] + (1 << 18)) >> 19) + 128) << (8 * x);
      hi |= clamp255(((out[x + 4] + (1 << 18)) >> 19) + 128) << (8 * x);
    }
    *reinterpret_cast<uint2*>(pix + d * 64 + y * 8) = make_uint2(lo, hi);
  }
  __syncwarp();
  if (s420) {  // 16 x 16 texels: lane = (row ty, half h), texels x = 8h .. 8h + 7
    const int ty = lane >> 1, h = lane & 1;
    const uint2 yv = *reinterpret_cast<const uint2*>(pix + ((ty >> 3) * 2 + h) * 64 + (ty & 7) * 8);
    const uint32_t cbv = *reinterpret_cast<const uint32_t*>(pix + 4 * 64 + (ty >> 1) * 8 + 4 * h);
    const uint32_t crv = *reinterpret_cast<const uint32_t*>(pix + 5 * 64 + (ty >> 1) * 8 + 4 * h);
    uint32_t o[8];
#pragma unroll
    for (int c = 0; c < 4; ++c) {  // chroma sample c covers texels 2c, 2c + 1
      int ro, go, bo;
      chroma_offsets((cbv >> (8 * c)) & 255u, (crv >> (8 * c)) & 255u, ro, go, bo);
      const uint32_t yw = c < 2 ? yv.x : yv.y;
      o[2 * c] = ycc_pixel((yw >> (16 * (c & 1))) & 255u, ro, go, bo);
      o[2 * c + 1] = ycc_pixel((yw >> (16 * (c & 1) + 8)) & 255u, ro, go, bo);
    }
    uint4* dst = reinterpret_cast<uint4*>(tile + (ty * 16 + 8 * h) * 4);
    dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
    dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
  } else {  // 8 x 8 texels, Y Cb Cr data units 0 1 2: lane = (row ty, texels x0, x0 + 1)
    const int ty = lane >> 2, x0 = (lane & 3) * 2;
    uint32_t o[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int i = ty * 8 + x0 + e;
      int ro, go, bo;
      chroma_offsets(pix[64 + i], pix[128 + i], ro, go, bo);
      o[e] = ycc_pixel(pix[i], ro, go, bo);
    }
    *reinterpret_cast<uint2*>(tile + (ty * 8 + x0) * 4) = make_uint2(o[0], o[1]);
  }
}

// UNITS: the variant for contexts with data-unit starts. Each MCU of a batch then takes six
// lanes, lane 6m + d decoding data unit d of MCU m from its own start (levels without
// starts are decoded whole by lane 6m); MCUs per batch are at most 4.
// SHORT: the variant that decodes short lists MCU by MCU with whole warps (a separate kernel,
// so that the lane-per-MCU variant is compiled without that code).
template <int M, bool UNITS, bool SHORT>
__global__ void k_decode(const __grid_constant__ DecodeArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  HuffSet* sh = reinterpret_cast<HuffSet*>(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* wbase = smem + sizeof(HuffSet) + 64 + (size_t)warp * warp_smem(M);
  int16_t* coef = reinterpret_cast<int16_t*>(wbase);                    // [6][64][M]
  uint32_t* stage = reinterpret_cast<uint32_t*>(wbase + 6 * 64 * M * 2);  // [M * kStageWords]
  // this lane's MCU slot and data unit (the whole MCU outside the unit variant)
  const int lm = UNITS ? lane / 6 : lane, ld = UNITS ? lane % 6 : 0;
  int16_t* col = coef + (lm < M ? lm : 0);  // this lane's MCU column
  constexpr int kMaxBatch = UNITS ? (M < 4 ? M : 4) : M;

  {  // stage Huffman set 0 (written at upload, so before the wait for the kernel before)
    const uint4* src = reinterpret_cast<const uint4*>(a.huff);
    uint4* dst = reinterpret_cast<uint4*>(sh);
    for (int i = threadIdx.x; i < (int)(sizeof(HuffSet) / 16); i += blockDim.x) dst[i] = __ldg(src + i);
  }
  __syncthreads();
  pdl_wait();  // the work list, slots and counts come from the compaction or the cache update

  const uint32_t count = min(*(volatile uint32_t*)&a.state->count, a.work_cap);
  bool any_bad = false;
  // MCUs per batch: the smallest power of two <= M that covers the list in one batch per
  // warp, so short lists spread one MCU per warp (latency) and long ones fill the lanes
  const uint32_t total_warps = gridDim.x * (blockDim.x >> 5);
  const uint32_t per_warp = (count + total_warps - 1) / total_warps;
  // (up to kWarpMcuMax MCUs per warp they go one at a time, each decoded by the whole warp:
  // a lone lane's chain is several times longer than the warp's)
  int lmeff = 0;
  if (!SHORT || M < 4 || per_warp > (uint32_t)kWarpMcuMax)
    while ((1u << lmeff) < per_warp && (1 << lmeff) < kMaxBatch) ++lmeff;
  const int meff = 1 << lmeff;
  // first batch by rank, interleaved over the CTAs (one warp per SM first), then dynamic
  const uint32_t wrank = (uint32_t)warp * gridDim.x + blockIdx.x;

#pragma unroll 1
  for (uint32_t it = 0;; ++it) {
    uint32_t base = wrank * (uint32_t)meff;
    if (it != 0) {
      uint32_t b = 0;
      if (lane == 0) b = atomicAdd(&a.state->decode_next, (uint32_t)meff);
      base = __shfl_sync(0xFFFFFFFFu, b, 0) + total_warps * (uint32_t)meff;
    }
    if (base >= count) break;

    {  // clear the coefficient buffer (768 M bytes; a warp-decoded MCU needs only its
       // contiguous 768 B: every other byte it reads is written first)
      uint4* z = reinterpret_cast<uint4*>(coef);
      const int nz = (SHORT && M >= 4 && meff == 1) ? 48 : 48 * M;
#pragma unroll 4
      for (int i = lane; i < nz; i += 32) z[i] = make_uint4(0, 0, 0, 0);
    }

    // ---- set-up: lanes of MCU slot m < m_eff take item base + m ----
    const uint32_t item = base + lm;
    bool act = lm < meff && item < count;
    bool unit = false;  // this lane decodes data unit ld only
    const uint32_t gid = act ? __ldg(a.work + item) : 0u;
    const uint32_t di = act ? __ldg(a.desc_of_gid + gid) : 0u;
    int ndu = 0;
    bool s420 = true, store = false;
    uint32_t off = 0, nbits = 0, bitpos = 0, endbit = 0, w0 = 0, want = 0, nwords = 0;
    bool cpt = false;
    int red = 0;  // reduced-resolution level: 1/2^red
    const uint32_t* words = nullptr;
    uint32_t qs = 0;  // the MCU's quantisation table set (zig-zag order, read through L1)
    int16_t pr0 = 0, pr1 = 0, pr2 = 0;
    const HuffTable* hs = sh->t;
    if (act && di < a.ndesc) {
      const DevDesc d = a.descs[di];
      const uint32_t mcu = gid - d.gid_base;
      if (d.sampling == kSamplingCoef || mcu >= d.nmcu) {
        act = false;  // not a JPEG level: nothing to decode
      } else {
        s420 = d.sampling == kSampling420;
        ndu = s420 ? 6 : 3;
        off = __ldg(a.slot + gid);
        store = off + d.units <= a.cap_units;
        cpt = d.compact != 0;
        red = d.reduce;
        if (cpt) {
          // compact form (Sec. 5.1, 5.3): byte offsets from the two-level table, the three
          // stored DCs from the MCU's 36-bit record (at a multiple of 4 bits, so two words)
          const uint32_t ng = (d.nmcu + 8) / 9;
          const uint32_t* ab = reinterpret_cast<const uint32_t*>(d.index);
          const uint16_t* rl = d.index + 2 * (size_t)ng;
          const uint32_t* rec = ab + 5 * (size_t)ng;
          auto start = [&](uint32_t m) {
            const uint32_t j = m / 9, i = m - 9 * j;
            return 8u * (__ldg(ab + j) + (i ? (uint32_t)__ldg(rl + 8 * j + i - 1) : 0u));
          };
          bitpos = start(mcu);
          endbit = mcu + 1 < d.nmcu ? start(mcu + 1) : d.nbits;
          const uint64_t at = 36ull * mcu;
          const uint64_t r = ((uint64_t)__ldg(rec + (at >> 5)) | ((uint64_t)__ldg(rec + (at >> 5) + 1) << 32)) >>
                             (at & 31);
          pr0 = (int16_t)((int32_t)((uint32_t)r << 20) >> 20);  // 12-bit two's complement
          pr1 = (int16_t)((int32_t)((uint32_t)(r >> 12) << 20) >> 20);
          pr2 = (int16_t)((int32_t)((uint32_t)(r >> 24) << 20) >> 20);
        } else {
          const uint16_t* ix = d.index + (size_t)mcu * 5;
          bitpos = (uint32_t)__ldg(ix) | ((uint32_t)__ldg(ix + 1) << 16);
          pr0 = (int16_t)__ldg(ix + 2);
          pr1 = (int16_t)__ldg(ix + 3);
          pr2 = (int16_t)__ldg(ix + 4);
          endbit = mcu + 1 < d.nmcu ? ((uint32_t)__ldg(ix + 5) | ((uint32_t)__ldg(ix + 6) << 16)) : d.nbits;
          if (UNITS && d.du_index != nullptr) {  // this lane's data unit and its bit range
            unit = true;
            const uint16_t* du = d.du_index + (size_t)mcu * (ndu - 1);
            const uint32_t mcu0 = bitpos;
            if (ld >= ndu) act = false;
            if (ld > 0 && ld < ndu) bitpos = mcu0 + __ldg(du + ld - 1);
            if (ld + 1 < ndu) endbit = mcu0 + __ldg(du + ld);
          }
        }
        if (UNITS && !unit && ld != 0) act = false;  // decoded whole by the MCU's first lane
        words = d.stream;
        nwords = d.nwords;
        nbits = d.nbits;
        // the MCU's words: from its first word (16 B aligned) to the next MCU's start plus
        // the window's look-ahead (3 words)
        w0 = (bitpos >> 5) & ~3u;
        want = (max(endbit, bitpos) >> 5) + 3 - w0;
        want = (want + 3) & ~3u;
        if (w0 + want > nwords) want = nwords > w0 ? (nwords - w0) & ~3u : 0u;
        if (d.hset != 0) hs = a.huff[d.hset].t;
        qs = d.qset;
      }
    } else {
      act = false;
    }
    if (!act) want = 0;
    // share the warp's stage pool out by a prefix sum of the lanes' word counts
    uint32_t sbeg = want;
#pragma unroll
    for (int dlt = 1; dlt < 32; dlt <<= 1) {
      const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, sbeg, dlt);
      if (lane >= dlt) sbeg += o;
    }
    sbeg -= want;  // exclusive
    constexpr uint32_t kPool = (uint32_t)kStageWords * M;
    const uint32_t nst = sbeg >= kPool ? 0u : min(want, kPool - sbeg);
    if (act) {
      const uint4* src4 = reinterpret_cast<const uint4*>(words + w0);
      uint4* dst4 = reinterpret_cast<uint4*>(stage + sbeg);
#pragma unroll 1
      for (uint32_t j = 0; j < nst / 4; j += 4) {
        uint4 r[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) r[t] = j + t < nst / 4 ? __ldg(src4 + j + t) : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (j + t < nst / 4) dst4[j + t] = make_uint4(bswap(r[t].x), bswap(r[t].y), bswap(r[t].z), bswap(r[t].w));
      }
    }
    __syncwarp();

    // ---- entropy phase: each active lane decodes all data units of its MCU (or, with
    // data-unit starts, one data unit) ----
    if (act && unit) {
      const Words W{(uint32_t)__cvta_generic_to_shared(stage + sbeg), nst, words + w0,
                    nwords > w0 ? nwords - w0 : 0u};
      const int comp = ld < ndu - 2 ? 0 : 1;
      const uint32_t b0 = bitpos - w0 * 32;
      int16_t* cu = col + ld * 64 * M;
      const uint32_t end = hs == sh->t
                               ? decode_unit<M, true>(W, b0, Tables<true>{hs, (uint32_t)__cvta_generic_to_shared(sh->t)},
                                                      comp, cu)
                               : decode_unit<M, false>(W, b0, Tables<false>{hs, 0u}, comp, cu);
      // a data unit must end at or before the next one's start
      if (end == 0xFFFFFFFFu || (uint64_t)w0 * 32 + end > endbit) any_bad = true;
    }
    bool warp_done = false;  // the MCU's tile was written by the whole warp
    if (SHORT && !UNITS && M >= 4 && meff == 1) {
      // one MCU per warp: the whole warp runs lane 0's chain (coefficients contiguous in
      // the buffer's first 768 B, the window's slots after them); a full-size tile
      // is then transformed and stored by the whole warp, any other is scattered into lane
      // 0's column for the per-lane passes
      if (__shfl_sync(0xFFFFFFFFu, act ? 1 : 0, 0)) {
        const Words W{(uint32_t)__cvta_generic_to_shared(stage), __shfl_sync(0xFFFFFFFFu, nst, 0),
                      reinterpret_cast<const uint32_t*>(
                          __shfl_sync(0xFFFFFFFFu, reinterpret_cast<unsigned long long>(words + w0), 0)),
                      __shfl_sync(0xFFFFFFFFu, nwords > w0 ? nwords - w0 : 0u, 0)};
        const HuffTable* hw = reinterpret_cast<const HuffTable*>(
            __shfl_sync(0xFFFFFFFFu, reinterpret_cast<unsigned long long>(hs), 0));
        const uint32_t b0 = __shfl_sync(0xFFFFFFFFu, bitpos - w0 * 32, 0);
        const int nd = __shfl_sync(0xFFFFFFFFu, ndu, 0);
        const bool cw = __shfl_sync(0xFFFFFFFFu, cpt ? 1 : 0, 0) != 0;
        const int q0 = __shfl_sync(0xFFFFFFFFu, (int)pr0, 0), q1 = __shfl_sync(0xFFFFFFFFu, (int)pr1, 0),
                  q2 = __shfl_sync(0xFFFFFFFFu, (int)pr2, 0);
        const uint32_t tsa = (uint32_t)__cvta_generic_to_shared(coef) + 768u;
        constexpr int kWin = M >= 8 ? kWinBits : kWinBits / 2;  // 16 B slots after the 768 B of coefficients
        static_assert(768 + 16 * kWin <= 768 * M || M < 4, "window slots fit the coefficient buffer");
        const Tables<true> TS{hw, (uint32_t)__cvta_generic_to_shared(sh->t)};
        const Tables<false> TG{hw, 0u};
        // staged whole: every word up to the next MCU's start plus the look-ahead
        const uint32_t nst0 = __shfl_sync(0xFFFFFFFFu, nst, 0);
        const bool whole = nst0 > 0 && nst0 >= __shfl_sync(0xFFFFFFFFu, want, 0);
        const StagedWords SW{W.st, nst0 - 1};
        uint32_t end;
        if (whole && hw == sh->t)
          end = cw ? decode_mcu_warp<true, true, kWin>(SW, b0, TS, nd, q0, q1, q2, coef, tsa, lane)
                   : decode_mcu_warp<true, false, kWin>(SW, b0, TS, nd, q0, q1, q2, coef, tsa, lane);
        else if (whole)
          end = cw ? decode_mcu_warp<false, true, kWin>(SW, b0, TG, nd, q0, q1, q2, coef, tsa, lane)
                   : decode_mcu_warp<false, false, kWin>(SW, b0, TG, nd, q0, q1, q2, coef, tsa, lane);
        else if (hw == sh->t)
          end = cw ? decode_mcu_warp<true, true, kWin>(W, b0, TS, nd, q0, q1, q2, coef, tsa, lane)
                   : decode_mcu_warp<true, false, kWin>(W, b0, TS, nd, q0, q1, q2, coef, tsa, lane);
        else
          end = cw ? decode_mcu_warp<false, true, kWin>(W, b0, TG, nd, q0, q1, q2, coef, tsa, lane)
                   : decode_mcu_warp<false, false, kWin>(W, b0, TG, nd, q0, q1, q2, coef, tsa, lane);
        if (lane == 0 && (end == 0xFFFFFFFFu || (uint64_t)w0 * 32 + end > (cpt ? endbit : nbits))) any_bad = true;
        __syncwarp();
        if (__shfl_sync(0xFFFFFFFFu, (red == 0 && store) ? 1 : 0, 0)) {
          const bool s4 = __shfl_sync(0xFFFFFFFFu, s420 ? 1 : 0, 0) != 0;
          const uint32_t qs0 = __shfl_sync(0xFFFFFFFFu, qs, 0), off0 = __shfl_sync(0xFFFFFFFFu, off, 0);
          mcu_warp_pixels(coef, coef + 384, reinterpret_cast<uint8_t*>(coef) + 1536, nd, s4,
                          a.quant + (size_t)qs0 * 128, a.cache + (size_t)off0 * kUnitBytes, lane);
          warp_done = true;
        } else {
          int16_t v[12];
#pragma unroll
          for (int i = 0; i < 12; ++i) v[i] = coef[lane + 32 * i];
          __syncwarp();
#pragma unroll
          for (int i = 0; i < 12; ++i) coef[(lane + 32 * i) * M] = v[i];
        }
      }
    } else if (act && !unit) {
      const Words W{(uint32_t)__cvta_generic_to_shared(stage + sbeg), nst, words + w0,
                    nwords > w0 ? nwords - w0 : 0u};
      const Tables<true> TS{hs, (uint32_t)__cvta_generic_to_shared(sh->t)};
      const Tables<false> TG{hs, 0u};
      const uint32_t b0 = bitpos - w0 * 32;
      uint32_t end;
      if (hs == sh->t)
        end = cpt ? decode_mcu<M, true, true>(W, b0, TS, ndu, pr0, pr1, pr2, col)
                  : decode_mcu<M, true, false>(W, b0, TS, ndu, pr0, pr1, pr2, col);
      else
        end = cpt ? decode_mcu<M, false, true>(W, b0, TG, ndu, pr0, pr1, pr2, col)
                  : decode_mcu<M, false, false>(W, b0, TG, ndu, pr0, pr1, pr2, col);
      // a compact MCU must also end inside its own bytes
      if (end == 0xFFFFFFFFu || (uint64_t)w0 * 32 + end > (cpt ? endbit : nbits)) any_bad = true;
    }

    if (UNITS) {  // chain the data units' DC differences (first lane of each MCU)
      __syncwarp();
      if (act && unit && ld == 0) {
        int c0 = pr0;
#pragma unroll 1
        for (int du = 0; du < ndu - 2; ++du) {  // luma: each unit's difference to the previous
          int16_t* dcp = col + du * 64 * M;
          c0 = (int16_t)(uint16_t)(c0 + (int)*dcp);  // modulo 2^16
          *dcp = (int16_t)c0;
        }
        int16_t* cb = col + (ndu - 2) * 64 * M;
        int16_t* cr = col + (ndu - 1) * 64 * M;
        *cb = (int16_t)(uint16_t)((int)pr1 + (int)*cb);
        *cr = (int16_t)(uint16_t)((int)pr2 + (int)*cr);
      }
    }

    // ---- IDCT: the batch's data units are shared out over the warp: pair q = (d, m) (data
    // unit d of MCU m) goes to lane q % 32 in round q / 32, which runs the column and the
    // row pass of that data unit. MCU m's set-up values come from its first lane.
    const uint32_t minfo =
        (act ? 1u : 0u) | (s420 ? 2u : 0u) | ((uint32_t)red << 2) | (store ? 16u : 0u) | (qs << 8);
    __syncwarp();  // every lane's coefficients are visible to the warp
#pragma unroll 1
    for (int r0 = 0; r0 < (warp_done ? 0 : 6 * meff); r0 += 32) {
      const int q = r0 + lane;
      const int d = q >> lmeff, m = q & (meff - 1);
      const uint32_t im = __shfl_sync(0xFFFFFFFFu, minfo, UNITS ? 6 * m : m);
      if (q < 6 * meff && (im & 1u) && d < ((im & 2u) ? 6 : 3)) {
        const uint16_t* Qd = a.quant + (size_t)(im >> 8) * 128 + (d < ((im & 2u) ? 4 : 1) ? 0 : 64);
        int16_t* blk = coef + d * 64 * M + m;
        const int rm = (int)((im >> 2) & 3u);
        if (rm == 0)
          idct_full<M>(blk, Qd);
        else if (rm == 1)
          idct_reduced<M, 1>(blk, Qd);
        else if (rm == 2)
          idct_reduced<M, 2>(blk, Qd);
        else
          idct_reduced<M, 3>(blk, Qd);
      }
    }
    __syncwarp();  // every data unit's pixels are visible to the warp

    // ---- colour conversion + tile stores. Full-size 4:2:0 tiles are shared out as pairs
    // (MCU m, column group c2 of 4 texels), 16-byte stores; 4:4:4 and reduced tiles are
    // written by their own lane ----
#pragma unroll 1
    for (int r0 = 0; r0 < (warp_done ? 0 : 4 * meff); r0 += 32) {
      const int q = r0 + lane;
      const int m = (q >> 2) & (meff - 1), c2 = q & 3;
      const uint32_t im = __shfl_sync(0xFFFFFFFFu, minfo, UNITS ? 6 * m : m);
      const uint32_t om = __shfl_sync(0xFFFFFFFFu, off, UNITS ? 6 * m : m);
      if (q < 4 * meff && (im & 0x1Fu) == (1u | 2u | 16u)) {  // active, 4:2:0, full size, stored
        const int16_t* cm = coef + m;
        uint8_t* tile = a.cache + (size_t)om * kUnitBytes;
        // chroma sample (cx, cy) covers texels 2cx..2cx+1, 2cy..2cy+1; texels x = 4 c2 .. 4 c2 + 3
#pragma unroll 1
        for (int cy = 0; cy < 8; ++cy) {
          const uint32_t cb2 = pixel2<M>(cm, 4, cy, c2), cr2 = pixel2<M>(cm, 5, cy, c2);
          int ro[2], go[2], bo[2];
          chroma_offsets(cb2 & 255, cr2 & 255, ro[0], go[0], bo[0]);
          chroma_offsets(cb2 >> 8, cr2 >> 8, ro[1], go[1], bo[1]);
#pragma unroll
          for (int dy = 0; dy < 2; ++dy) {
            const int ty = 2 * cy + dy;
            const int du = (ty >> 3) * 2 + (c2 >> 1), ry = ty & 7, ci = (c2 & 1) * 2;
            const uint32_t ya = pixel2<M>(cm, du, ry, ci), yb = pixel2<M>(cm, du, ry, ci + 1);
            uint4 o;
            o.x = ycc_pixel(ya & 255, ro[0], go[0], bo[0]);
            o.y = ycc_pixel(ya >> 8, ro[0], go[0], bo[0]);
            o.z = ycc_pixel(yb & 255, ro[1], go[1], bo[1]);
            o.w = ycc_pixel(yb >> 8, ro[1], go[1], bo[1]);
            *reinterpret_cast<uint4*>(tile + (ty * 16 + 4 * c2) * 4) = o;
          }
        }
      }
    }
    if (!warp_done && act && ld == 0 && store && red != 0)
      colour_reduced<M>(col, s420, red, reinterpret_cast<uint32_t*>(a.cache + (size_t)off * kUnitBytes));
    if (!warp_done && act && ld == 0 && store && red == 0 && !s420) {  // 4:4:4, 8x8 texels, Y Cb Cr data units 0 1 2
      uint8_t* tile = a.cache + (size_t)off * kUnitBytes;
#pragma unroll 1
      for (int ty = 0; ty < 8; ++ty) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // texels x = 4h .. 4h + 3
          uint32_t o[4];
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const uint32_t y2 = pixel2<M>(col, 0, ty, 2 * h + j), b2 = pixel2<M>(col, 1, ty, 2 * h + j),
                           r2 = pixel2<M>(col, 2, ty, 2 * h + j);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              int ro, go, bo;
              chroma_offsets((b2 >> (8 * e)) & 255, (r2 >> (8 * e)) & 255, ro, go, bo);
              o[2 * j + e] = ycc_pixel((y2 >> (8 * e)) & 255, ro, go, bo);
            }
          }
          *reinterpret_cast<uint4*>(tile + (ty * 8 + 4 * h) * 4) = make_uint4(o[0], o[1], o[2], o[3]);
        }
      }
    }
    __syncwarp();  // the buffers are cleared for the next items
  }
  if (any_bad) atomicOr(&a.state->err, JT_DEVERR_CORRUPT);
}

size_t smem_bytes(int warps, int M) { return sizeof(HuffSet) + 64 + (size_t)warps * warp_smem(M); }

template <int M, bool UNITS, bool SHORT>
int occupancy_of(int warps) {
  const size_t smem = smem_bytes(warps, M);
  if (smem > 227 * 1024) return 0;
  if (cudaFuncSetAttribute(k_decode<M, UNITS, SHORT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_decode<M, UNITS, SHORT>, warps * 32, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// resident CTAs per SM that every variant reaches (the launch picks one per frame)
template <int M>
int occupancy(int warps) {
  return min(min(occupancy_of<M, false, false>(warps), occupancy_of<M, true, false>(warps)),
             occupancy_of<M, false, true>(warps));
}

}  // namespace

size_t decode_smem_bytes(int warps, int mcus_per_warp) { return smem_bytes(warps, mcus_per_warp); }

// The dynamic shared-memory attribute of each variant is set by decode_max_ctas_per_sm(),
// which the context calls for every (warps, M) on its device before the first launch.
void launch_decode(const DecodeArgs& a, int warps, int grid, cudaStream_t s) {
  const size_t smem = smem_bytes(warps, a.mcus_per_warp);
  if (a.unit_mode) {
    switch (a.mcus_per_warp) {
      case 4: launch_pdl(k_decode<4, true, false>, grid, warps * 32, smem, s, a); break;
      case 8: launch_pdl(k_decode<8, true, false>, grid, warps * 32, smem, s, a); break;
      case 16: launch_pdl(k_decode<16, true, false>, grid, warps * 32, smem, s, a); break;
      default: launch_pdl(k_decode<32, true, false>, grid, warps * 32, smem, s, a); break;
    }
    return;
  }
  if (a.short_lists) {
    switch (a.mcus_per_warp) {
      case 4: launch_pdl(k_decode<4, false, true>, grid, warps * 32, smem, s, a); break;
      case 8: launch_pdl(k_decode<8, false, true>, grid, warps * 32, smem, s, a); break;
      case 16: launch_pdl(k_decode<16, false, true>, grid, warps * 32, smem, s, a); break;
      default: launch_pdl(k_decode<32, false, true>, grid, warps * 32, smem, s, a); break;
    }
    return;
  }
  switch (a.mcus_per_warp) {
    case 4: launch_pdl(k_decode<4, false, false>, grid, warps * 32, smem, s, a); break;
    case 8: launch_pdl(k_decode<8, false, false>, grid, warps * 32, smem, s, a); break;
    case 16: launch_pdl(k_decode<16, false, false>, grid, warps * 32, smem, s, a); break;
    default: launch_pdl(k_decode<32, false, false>, grid, warps * 32, smem, s, a); break;
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
