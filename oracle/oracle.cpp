// Oracle for the variable-rate (JPEG) texture path — TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, single-threaded CPU restatement of what the path computes, written
// from the paper and from ITU-T T.81 (baseline JPEG). Only the test-suite, the smoke
// check and the benchmark's CPU-baseline leg call it; the product path never does.
// It shares no code, header, table or constant generator with the CUDA library.
//
// What it computes (section numbers are the paper's):
//   * baseline sequential decode of a JFIF file (Sec. 3.1 pipeline run in reverse):
//     Huffman decode bit by bit with MINCODE/MAXCODE/VALPTR (T.81 F.2.2.3), DC
//     prediction, dequantisation, integer 8x8 IDCT, chroma upsampling, YCbCr->RGB;
//   * the random-access index it implies: the first bit of every MCU in the
//     unstuffed entropy stream plus each component's DC predictor (Sec. 5.1, Sec. 5.3,
//     read as a bit offset with explicit predictors);
//   * random-access decode of one MCU from that index (Sec. 4.3);
//   * Mark: pixel uv -> texel -> MCU id, MCUs keyed by (texture, mip level) (Sec. 4.2,
//     Sec. 4.6); Compact: the sorted unique set (Fig. "pipeline" a);
//   * Resolve / colourise: nearest, bilinear, and bilinear clamped to the nearest texel's
//     MCU (Sec. 4.4);
//   * a float (FP64) forward of the colourise chain from dequantised DCT coefficients,
//     its L2 loss, analytic gradient and central finite differences;
//   * the paper's compact random-access form: byte offsets every ninth MCU with relative
//     offsets between, 12-bit stored DCs (Sec. 5.1, Sec. 5.3);
//   * reduced-resolution levels from the lowest N x N frequencies (Sec. 7);
//   * decode data unit by data unit from recorded unit starts (an index extension);
//   * the fp32 rasteriser of the procedural G-buffer scene (the geometry-pass stand-in).
//
// Readings where the paper is silent (all listed with reasons in the design notes):
//   * integer IDCT: K[x][u] = round(2^14 * c_u * cos((2x+1) u pi / 16)), c_0 = 1/(2 sqrt 2),
//     c_u = 1/2; dequantised inputs clamped to int16; column pass first,
//     t = clamp16(floor((sum + 2^8) / 2^9)) (5 fractional bits); row pass
//     p = clamp(floor((sum + 2^18) / 2^19) + 128, 0, 255). Every sum fits in int32;
//   * colour: JFIF with 16-bit fixed-point constants round(c * 2^16), each channel
//     Y + floor((k1 Cb' + k2 Cr' + 2^15) / 2^16), clamped;
//   * 4:2:0 chroma is replicated inside the MCU (sample (x>>1, y>>1));
//   * DC values wrap modulo 2^16 (int16), so the 16-bit predictors in the index always
//     reproduce the sequential state;
//   * texel addressing: x = floor(fp32(u * w)), floor-mod w; bilinear taps from
//     fp32(fp32(u * w) - 0.5); MCUs per row = ceil(w / 16) (or ceil(w / 8) at 4:4:4).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <unordered_map>
#include <vector>

namespace {

// ---------------------------------------------------------------------------------------
// Arithmetic helpers
// ---------------------------------------------------------------------------------------
int64_t floor_div(int64_t a, int64_t b) {  // b > 0
  int64_t q = a / b;
  if ((a % b) != 0 && a < 0) --q;
  return q;
}
int64_t floor_mod(int64_t a, int64_t b) { return a - floor_div(a, b) * b; }
int64_t clamp64(int64_t v, int64_t lo, int64_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Zig-zag order by walking anti-diagonals s = row + col, alternating direction; the k-th
// coefficient of the scan lands at natural index zigzag()[k].
const int* zigzag() {
  static int zz[64];
  static bool done = false;
  if (!done) {
    int k = 0;
    for (int s = 0; s <= 14; ++s) {
      int rlo = std::max(0, s - 7), rhi = std::min(s, 7);
      if (s & 1)
        for (int r = rlo; r <= rhi; ++r) zz[k++] = r * 8 + (s - r);
      else
        for (int r = rhi; r >= rlo; --r) zz[k++] = r * 8 + (s - r);
    }
    done = true;
  }
  return zz;
}

// ---------------------------------------------------------------------------------------
// Huffman tables (T.81 Annex C and F.2.2.3)
// ---------------------------------------------------------------------------------------
struct HuffTable {
  uint8_t bits[16];
  uint8_t vals[256];
  int nvals = 0;
  // per code length l = 1..16
  int32_t mincode[17], maxcode[17], valptr[17];
  bool ok = false;
};

// Builds HUFFSIZE/HUFFCODE (Annex C.2) and MINCODE/MAXCODE/VALPTR (F.2.2.3).
HuffTable make_table(const uint8_t* bits, const uint8_t* vals) {
  HuffTable t;
  std::memcpy(t.bits, bits, 16);
  int n = 0;
  for (int i = 0; i < 16; ++i) n += bits[i];
  t.nvals = n;
  if (n > 256) return t;
  std::memcpy(t.vals, vals, n);
  std::vector<int> huffsize, huffcode;
  for (int l = 1; l <= 16; ++l)
    for (int i = 0; i < bits[l - 1]; ++i) huffsize.push_back(l);
  int code = 0;
  size_t k = 0;
  int si = huffsize.empty() ? 0 : huffsize[0];
  while (k < huffsize.size()) {
    while (k < huffsize.size() && huffsize[k] == si) {
      huffcode.push_back(code);
      ++code;
      ++k;
    }
    code <<= 1;
    ++si;
  }
  int j = 0;
  for (int l = 1; l <= 16; ++l) {
    if (bits[l - 1] == 0) {
      t.maxcode[l] = -1;
      t.mincode[l] = 0;
      t.valptr[l] = 0;
    } else {
      t.valptr[l] = j;
      t.mincode[l] = huffcode[j];
      j += bits[l - 1];
      t.maxcode[l] = huffcode[j - 1];
    }
  }
  t.ok = true;
  return t;
}

// ---------------------------------------------------------------------------------------
// Bit reader over an unstuffed entropy stream, MSB first
// ---------------------------------------------------------------------------------------
struct BitReader {
  const uint8_t* data;
  uint64_t nbytes;
  uint64_t pos;  // bit position
  bool overrun = false;
  int bit() {
    uint64_t byte = pos >> 3;
    int b = 1;  // reads past the end see 1-bits (the padding value) and set overrun
    if (byte < nbytes)
      b = (data[byte] >> (7 - (pos & 7))) & 1;
    else
      overrun = true;
    ++pos;
    return b;
  }
  int receive(int s) {  // T.81 F.2.2.4 RECEIVE
    int v = 0;
    for (int i = 0; i < s; ++i) v = (v << 1) | bit();
    return v;
  }
};

int extend(int v, int t) {  // T.81 F.2.2.1 EXTEND
  if (t == 0) return 0;
  return v < (1 << (t - 1)) ? v + (-(1 << t)) + 1 : v;
}

// T.81 F.2.2.3 DECODE: read one bit at a time until the code fits a length's range.
int decode_symbol(BitReader& br, const HuffTable& t, bool& err) {
  int code = br.bit();
  for (int l = 1; l <= 16; ++l) {
    if (t.maxcode[l] >= 0 && code <= t.maxcode[l] && code >= t.mincode[l])
      return t.vals[t.valptr[l] + code - t.mincode[l]];
    if (l < 16) code = (code << 1) | br.bit();
  }
  err = true;
  return 0;
}

// Decodes one data unit into quantised coefficients (natural order). Returns false when
// the stream is not a valid coding of a data unit.
// dc_coded = false: the data unit carries no DC difference (the compact form of Sec. 5.3
// stores that DC apart) and its DC is `pred` as given. *dc_bits: the bits the DC took.
bool decode_du(BitReader& br, const HuffTable& dc, const HuffTable& ac, int16_t& pred, int32_t coef[64],
               bool dc_coded = true, int* dc_bits = nullptr) {
  const int* zz = zigzag();
  bool err = false;
  for (int k = 0; k < 64; ++k) coef[k] = 0;
  const uint64_t dc_start = br.pos;
  if (dc_coded) {
    int t = decode_symbol(br, dc, err);
    if (err || t > 11) return false;
    int diff = extend(br.receive(t), t);
    pred = (int16_t)(uint16_t)((int)pred + diff);  // DC wraps modulo 2^16
  }
  if (dc_bits) *dc_bits = (int)(br.pos - dc_start);
  coef[0] = pred;
  int k = 1;
  while (k < 64) {
    int rs = decode_symbol(br, ac, err);
    if (err) return false;
    int s = rs & 15, r = rs >> 4;
    if (s == 0) {
      if (r == 15) {
        k += 16;
        if (k > 63) return false;
        continue;
      }
      break;  // EOB
    }
    k += r;
    if (k > 63 || s > 10) return false;
    coef[zz[k]] = extend(br.receive(s), s);
    ++k;
  }
  return !br.overrun;
}

// ---------------------------------------------------------------------------------------
// Integer IDCT and colour conversion (the decode spec)
// ---------------------------------------------------------------------------------------
// N-point IDCT matrix K_N[x*N+u] = round(2^14 c_u cos((2x+1) u pi / (2N))), c_0 = 1/(2 sqrt 2),
// c_u = 1/2, for N = 8 (the full decode) and N = 4, 2, 1 (the reduced-resolution decode of
// Sec. 7's mip alternative: the N x N lowest frequencies give the block at 1/(8/N) scale;
// the c_u keep their 8-point values because the N-point orthonormal coefficients of a
// block averaged down by 8/N are the 8-point ones times sqrt(N/8) per axis).
const int64_t* idct_matrix(int N = 8) {
  static int64_t K[4][64];
  static bool done = false;
  if (!done) {
    for (int r = 0; r < 4; ++r) {
      const int n = 8 >> r;
      for (int x = 0; x < n; ++x)
        for (int u = 0; u < n; ++u) {
          double cu = u == 0 ? 1.0 / (2.0 * std::sqrt(2.0)) : 0.5;
          K[r][x * n + u] = std::lround(16384.0 * cu * std::cos((2 * x + 1) * u * M_PI / (2.0 * n)));
        }
    }
    done = true;
  }
  return K[N == 8 ? 0 : N == 4 ? 1 : N == 2 ? 2 : 3];
}

// out[y*N+x] = signed spatial value before the +128 level shift, from the N x N lowest
// frequencies d_in[v*8+u], u, v < N (N = 8: the whole block).
void idct_raw(const int32_t d_in[64], int32_t out[64], int N = 8) {
  const int64_t* K = idct_matrix(N);
  int64_t d[64], t[64];
  for (int i = 0; i < 64; ++i) d[i] = clamp64(d_in[i], -32768, 32767);
  for (int u = 0; u < N; ++u)  // column pass: 1-D IDCT down each column (v -> y)
    for (int y = 0; y < N; ++y) {
      int64_t s = 0;
      for (int v = 0; v < N; ++v) s += K[y * N + v] * d[v * 8 + u];
      t[y * 8 + u] = clamp64(floor_div(s + 256, 512), -32768, 32767);
    }
  for (int y = 0; y < N; ++y)  // row pass: 1-D IDCT along each row (u -> x)
    for (int x = 0; x < N; ++x) {
      int64_t s = 0;
      for (int u = 0; u < N; ++u) s += K[x * N + u] * t[y * 8 + u];
      out[y * N + x] = (int32_t)floor_div(s + 262144, 524288);
    }
}

void idct_pixels(const int32_t d[64], uint8_t out[64], int N = 8) {
  int32_t r[64];
  idct_raw(d, r, N);
  for (int i = 0; i < N * N; ++i) out[i] = (uint8_t)clamp64(r[i] + 128, 0, 255);
}

void ycc_to_rgb(int Y, int Cb, int Cr, uint8_t rgb[3]) {
  const int64_t cb = Cb - 128, cr = Cr - 128;
  rgb[0] = (uint8_t)clamp64(Y + floor_div(91881 * cr + 32768, 65536), 0, 255);
  rgb[1] = (uint8_t)clamp64(Y + floor_div(-22554 * cb - 46802 * cr + 32768, 65536), 0, 255);
  rgb[2] = (uint8_t)clamp64(Y + floor_div(116130 * cb + 32768, 65536), 0, 255);
}

// One decoded MCU -> RGBA8 tile, row-major: 16x16 at 4:2:0, 8x8 at 4:4:4, divided by 2^r
// along each axis for the reduced-resolution decode (r = 0..3; each data unit gives
// N x N pixels, N = 8 >> r; 4:2:0 chroma is replicated 2x2 as at full size).
void mcu_to_tile(const int32_t q[6][64], int sampling, const uint16_t qt[2][64], uint8_t* tile, int r = 0) {
  const int ndu = sampling == 420 ? 6 : 3;
  const int N = 8 >> r;
  uint8_t px[6][64];
  for (int d = 0; d < ndu; ++d) {
    int comp = d < ndu - 2 ? 0 : 1;
    int32_t deq[64];
    for (int k = 0; k < 64; ++k) deq[k] = q[d][k] * (int32_t)qt[comp][k];  // dequantise
    idct_pixels(deq, px[d], N);
  }
  const int mw = (sampling == 420 ? 16 : 8) >> r;
  for (int y = 0; y < mw; ++y)
    for (int x = 0; x < mw; ++x) {
      int Y, Cb, Cr;
      if (sampling == 420) {
        Y = px[(y / N) * 2 + (x / N)][(y % N) * N + (x % N)];
        Cb = px[4][(y >> 1) * N + (x >> 1)];
        Cr = px[5][(y >> 1) * N + (x >> 1)];
      } else {
        Y = px[0][y * N + x];
        Cb = px[1][y * N + x];
        Cr = px[2][y * N + x];
      }
      uint8_t* o = tile + (y * mw + x) * 4;
      ycc_to_rgb(Y, Cb, Cr, o);
      o[3] = 255;
    }
}

#pragma pack(push, 2)
struct BlockIndex {
  uint32_t bit_offset;
  int16_t dc_pred[3];
};
#pragma pack(pop)

// ---------------------------------------------------------------------------------------
// JFIF parsing and sequential decode
// ---------------------------------------------------------------------------------------
struct Decoded {
  int status = 0;  // 0 ok, <0 error
  int w = 0, h = 0, sampling = 0, mcus_x = 0, mcus_y = 0;
  uint16_t qt[2][64];  // natural order
  uint8_t hbits[4][16];
  uint8_t hvals[4][256];
  std::vector<uint8_t> scan;  // unstuffed
  uint64_t coded_bits = 0;
  std::vector<BlockIndex> index;
  std::vector<int32_t> qcoef;  // [mcu][du][64] quantised, natural order
  std::vector<uint8_t> rgba;   // [h][w][4]
};

int be16(const uint8_t* p) { return (p[0] << 8) | p[1]; }

Decoded* decode_jfif(const uint8_t* f, size_t n) {
  Decoded* D = new Decoded();
  const int* zz = zigzag();
  if (n < 4 || f[0] != 0xFF || f[1] != 0xD8) {
    D->status = -1;
    return D;
  }
  size_t p = 2;
  int comp_table[3] = {0, 1, 1};
  bool have_sof = false;
  uint8_t tabs_present = 0;
  while (p + 4 <= n) {
    if (f[p] != 0xFF) {
      D->status = -2;
      return D;
    }
    int marker = f[p + 1];
    int len = be16(f + p + 2);
    const uint8_t* seg = f + p + 4;
    if (p + 2 + len > n) {
      D->status = -3;
      return D;
    }
    if (marker == 0xDB) {  // DQT
      int q = 0;
      while (q < len - 2) {
        int pq = seg[q] >> 4, tq = seg[q] & 15;
        if (pq != 0 || tq > 1) {
          D->status = -4;
          return D;
        }
        for (int k = 0; k < 64; ++k) D->qt[tq][zz[k]] = seg[q + 1 + k];
        q += 65;
      }
    } else if (marker == 0xC0) {  // SOF0 baseline
      D->h = be16(seg + 1);
      D->w = be16(seg + 3);
      if (seg[0] != 8 || seg[5] != 3) {
        D->status = -5;
        return D;
      }
      int hv = seg[6 + 1];
      D->sampling = hv == 0x22 ? 420 : (hv == 0x11 ? 444 : 0);
      if (!D->sampling || seg[9 + 1] != 0x11 || seg[12 + 1] != 0x11) {
        D->status = -6;
        return D;
      }
      for (int c = 0; c < 3; ++c) comp_table[c] = seg[6 + 3 * c + 2];
      have_sof = true;
    } else if (marker == 0xC4) {  // DHT
      int q = 0;
      while (q < len - 2) {
        int tc = seg[q] >> 4, th = seg[q] & 15;
        int cnt = 0;
        for (int i = 0; i < 16; ++i) cnt += seg[q + 1 + i];
        int slot = th * 2 + tc;  // DC-Y, AC-Y, DC-C, AC-C
        if (slot > 3 || cnt > 256) {
          D->status = -7;
          return D;
        }
        std::memcpy(D->hbits[slot], seg + q + 1, 16);
        std::memset(D->hvals[slot], 0, 256);
        std::memcpy(D->hvals[slot], seg + q + 17, cnt);
        tabs_present |= (uint8_t)(1 << slot);
        q += 17 + cnt;
      }
    } else if (marker == 0xDA) {  // SOS: entropy-coded data follows the header
      p += 2 + len;
      while (p < n) {
        if (f[p] == 0xFF) {
          if (p + 1 < n && f[p + 1] == 0x00) {
            D->scan.push_back(0xFF);
            p += 2;
            continue;
          }
          break;  // a marker ends the scan (EOI here; restart markers are not used)
        }
        D->scan.push_back(f[p++]);
      }
      break;
    }
    p += 2 + len;
  }
  if (!have_sof || tabs_present != 15 || comp_table[0] != 0 || comp_table[1] != 1 || comp_table[2] != 1) {
    D->status = -8;
    return D;
  }
  HuffTable tab[4];
  for (int t = 0; t < 4; ++t) tab[t] = make_table(D->hbits[t], D->hvals[t]);
  const int mw = D->sampling == 420 ? 16 : 8;
  const int ndu = D->sampling == 420 ? 6 : 3;
  D->mcus_x = (D->w + mw - 1) / mw;
  D->mcus_y = (D->h + mw - 1) / mw;
  const int nmcu = D->mcus_x * D->mcus_y;
  D->qcoef.assign((size_t)nmcu * ndu * 64, 0);
  D->index.resize(nmcu);
  BitReader br{D->scan.data(), D->scan.size(), 0};
  int16_t pred[3] = {0, 0, 0};
  for (int m = 0; m < nmcu; ++m) {
    D->index[m].bit_offset = (uint32_t)br.pos;
    for (int c = 0; c < 3; ++c) D->index[m].dc_pred[c] = pred[c];
    for (int d = 0; d < ndu; ++d) {
      int comp = d < ndu - 2 ? 0 : (d == ndu - 2 ? 1 : 2);
      int tb = comp == 0 ? 0 : 1;
      if (!decode_du(br, tab[tb * 2], tab[tb * 2 + 1], pred[comp], &D->qcoef[((size_t)m * ndu + d) * 64])) {
        D->status = -9;
        return D;
      }
    }
  }
  D->coded_bits = br.pos;
  // pixels
  D->rgba.assign((size_t)D->w * D->h * 4, 0);
  std::vector<uint8_t> tile(mw * mw * 4);
  int32_t q6[6][64];
  for (int m = 0; m < nmcu; ++m) {
    for (int d = 0; d < ndu; ++d) std::memcpy(q6[d], &D->qcoef[((size_t)m * ndu + d) * 64], 64 * sizeof(int32_t));
    mcu_to_tile(q6, D->sampling, D->qt, tile.data());
    int mx = m % D->mcus_x, my = m / D->mcus_x;
    for (int y = 0; y < mw; ++y)
      for (int x = 0; x < mw; ++x) {
        int X = mx * mw + x, Y = my * mw + y;
        if (X < D->w && Y < D->h) std::memcpy(&D->rgba[((size_t)Y * D->w + X) * 4], &tile[(y * mw + x) * 4], 4);
      }
  }
  return D;
}

// ---------------------------------------------------------------------------------------
// Texture set: levels keyed by (texture id, mip level), decoded by random access
// ---------------------------------------------------------------------------------------
struct Level {
  int tex = 0, level = 0, w = 0, h = 0, sampling = 420, mcus_x = 0, mcus_y = 0;
  uint32_t gid_base = 0;
  std::vector<uint8_t> scan;
  uint64_t nbits = 0;
  std::vector<BlockIndex> index;
  // the compact form (Sec. 5.1 indexing table, Sec. 5.3 DC records), when `compact`
  bool compact = false;
  std::vector<uint32_t> c_abs;  // byte offset of MCU 9j
  std::vector<uint16_t> c_rel;  // byte offset of MCU 9j+i (i = 1..8) relative to c_abs[j]
  std::vector<uint32_t> c_dc;   // 12-bit absolute DCs (Y0, Cb, Cr), 36 bits per MCU
  uint16_t qt[2][64];
  HuffTable tab[4];
  std::unordered_map<int, std::vector<uint8_t>> tiles;  // decoded MCUs, by MCU id
  std::vector<uint8_t> full;                            // optional full RGBA decode
  int reduce = 0;  // reduced-resolution decode of a stored level: tiles at 1/2^reduce (Sec. 7)
  int src = -1;    // a reduced level's source level
  // optional data-unit starts [mcu][ndu - 1] (bits from the MCU's first bit): each data unit
  // is then decoded from its own start, its DC difference chained afterwards
  std::vector<uint16_t> du_off;
  int mw() const { return (sampling == 420 ? 16 : 8) >> reduce; }
};

struct TexSet {
  std::map<std::pair<int, int>, Level*> levels;
  std::vector<Level*> order;  // upload order
  uint32_t next_gid = 0;
  int err = 0;
  ~TexSet() {
    for (Level* l : order) delete l;
  }
};

// First bit of MCU m in the compact stream: its byte offset from the two-level table
// (absolute every ninth MCU, the next eight relative to it), times 8.
uint64_t compact_start(const Level& L, int m) {
  if (m >= L.mcus_x * L.mcus_y) return 8ull * L.scan.size();
  const int j = m / 9, i = m % 9;
  return 8ull * ((uint64_t)L.c_abs[j] + (i ? L.c_rel[8 * j + i - 1] : 0u));
}

// Absolute DC c (0 = first Y, 1 = Cb, 2 = Cr) of MCU m: 12-bit two's complement at bit
// 36 m + 12 c of the record array (bit b = bit b % 32 of word b / 32).
int compact_dc(const Level& L, int m, int c) {
  const uint64_t at = 36ull * m + 12ull * c;
  int v = 0;
  for (int i = 0; i < 12; ++i) v |= (int)((L.c_dc[(at + i) / 32] >> ((at + i) % 32)) & 1u) << i;
  return v >= 2048 ? v - 4096 : v;
}

// Random-access decode of one MCU of the compact form: start at the MCU's byte; the first
// luma data unit and the chroma data units take their DCs from the records, the other luma
// units decode their DC differences against the previous luma unit of the MCU. The MCU's
// bits must end inside its own bytes.
int decode_mcu_compact(const Level& L, int mcu, uint8_t* tile) {
  const int ndu = L.sampling == 420 ? 6 : 3;
  BitReader br{L.scan.data(), L.scan.size(), compact_start(L, mcu)};
  int16_t pred[3];
  for (int c = 0; c < 3; ++c) pred[c] = (int16_t)compact_dc(L, mcu, c);
  int32_t q[6][64];
  for (int d = 0; d < ndu; ++d) {
    int comp = d < ndu - 2 ? 0 : (d == ndu - 2 ? 1 : 2);
    int tb = comp == 0 ? 0 : 1;
    const bool stored = d == 0 || comp != 0;
    if (!decode_du(br, L.tab[tb * 2], L.tab[tb * 2 + 1], pred[comp], q[d], !stored)) return -1;
  }
  if (br.pos > compact_start(L, mcu + 1)) return -1;
  mcu_to_tile(q, L.sampling, L.qt, tile, L.reduce);
  return 0;
}

// Random-access decode of one MCU by data units: data unit d starts at the MCU's bit offset
// plus its recorded offset and must end at or before the next one's start (the next MCU's
// for the last). Each DC difference is decoded from a zero predictor, then chained: a
// component's first data unit adds the index's predictor, each further luma unit the
// previous luma DC (modulo 2^16, as in the sequential decode).
int decode_mcu_by_units(const Level& L, int mcu, uint8_t* tile) {
  const int ndu = L.sampling == 420 ? 6 : 3;
  const uint64_t start = L.index[mcu].bit_offset;
  const uint64_t next = mcu + 1 < (int)L.index.size() ? L.index[mcu + 1].bit_offset : L.nbits;
  int32_t q[6][64];
  int16_t prev[3] = {L.index[mcu].dc_pred[0], L.index[mcu].dc_pred[1], L.index[mcu].dc_pred[2]};
  for (int d = 0; d < ndu; ++d) {
    const uint64_t s0 = start + (d ? L.du_off[(size_t)mcu * (ndu - 1) + d - 1] : 0u);
    const uint64_t s1 = d + 1 < ndu ? start + L.du_off[(size_t)mcu * (ndu - 1) + d] : next;
    int comp = d < ndu - 2 ? 0 : (d == ndu - 2 ? 1 : 2);
    int tb = comp == 0 ? 0 : 1;
    BitReader br{L.scan.data(), L.scan.size(), s0};
    int16_t diff = 0;
    if (!decode_du(br, L.tab[tb * 2], L.tab[tb * 2 + 1], diff, q[d])) return -1;
    if (br.pos > s1) return -1;
    prev[comp] = (int16_t)(uint16_t)((int)prev[comp] + (int)diff);
    q[d][0] = prev[comp];
  }
  mcu_to_tile(q, L.sampling, L.qt, tile, L.reduce);
  return 0;
}

// Random-access decode of one MCU (Sec. 4.3 with the index of Sec. 5.1): start at the
// MCU's bit offset with its DC predictors and decode its data units.
int decode_mcu(const Level& L, int mcu, uint8_t* tile) {
  if (L.compact) return decode_mcu_compact(L, mcu, tile);
  if (!L.du_off.empty()) return decode_mcu_by_units(L, mcu, tile);
  const int ndu = L.sampling == 420 ? 6 : 3;
  const BlockIndex& bi = L.index[mcu];
  BitReader br{L.scan.data(), L.scan.size(), bi.bit_offset};
  int16_t pred[3] = {bi.dc_pred[0], bi.dc_pred[1], bi.dc_pred[2]};
  int32_t q[6][64];
  for (int d = 0; d < ndu; ++d) {
    int comp = d < ndu - 2 ? 0 : (d == ndu - 2 ? 1 : 2);
    int tb = comp == 0 ? 0 : 1;
    if (!decode_du(br, L.tab[tb * 2], L.tab[tb * 2 + 1], pred[comp], q[d])) return -1;
  }
  if (br.pos > L.nbits) return -1;
  mcu_to_tile(q, L.sampling, L.qt, tile, L.reduce);
  return 0;
}

const uint8_t* get_tile(Level& L, int mcu) {
  auto it = L.tiles.find(mcu);
  if (it != L.tiles.end()) return it->second.data();
  std::vector<uint8_t> t(L.mw() * L.mw() * 4);
  if (decode_mcu(L, mcu, t.data()) != 0) return nullptr;
  return L.tiles.emplace(mcu, std::move(t)).first->second.data();
}

// Texel addressing for one pixel (Sec. 4.2 / Sec. 4.4).
struct Taps {
  int n;        // 1 (nearest) or 4 (bilinear)
  int x[4], y[4];
  float fx, fy;  // bilinear fractions
};

// filter 0: the nearest texel; 1: the four bilinear taps; 2: the bilinear taps clamped to
// the MCU of the nearest texel (Sec. 4.4, the mode of the linear-interpolation timing in
// Sec. 6.2): along each axis a tap in another MCU (mw texels wide) is replaced by the
// nearest texel's coordinate, so all four fetches fall in one MCU.
Taps pixel_taps(float u, float v, int w, int h, int filter, int mw = 16) {
  Taps t{};
  volatile float uw = u * (float)w;  // one fp32 rounding, no fused multiply-add
  volatile float vh = v * (float)h;
  const int nx = (int)floor_mod((int64_t)std::floor((float)uw), w);
  const int ny = (int)floor_mod((int64_t)std::floor((float)vh), h);
  if (filter == 0) {
    t.n = 1;
    t.x[0] = nx;
    t.y[0] = ny;
  } else {
    volatile float xs = (float)uw - 0.5f;
    volatile float ys = (float)vh - 0.5f;
    float x0f = std::floor((float)xs), y0f = std::floor((float)ys);
    t.fx = (float)xs - x0f;
    t.fy = (float)ys - y0f;
    int64_t x0 = (int64_t)x0f, y0 = (int64_t)y0f;
    int xa = (int)floor_mod(x0, w), xb = (int)floor_mod(x0 + 1, w);
    int ya = (int)floor_mod(y0, h), yb = (int)floor_mod(y0 + 1, h);
    if (filter == 2) {
      if (xa / mw != nx / mw) xa = nx;
      if (xb / mw != nx / mw) xb = nx;
      if (ya / mw != ny / mw) ya = ny;
      if (yb / mw != ny / mw) yb = ny;
    }
    t.n = 4;
    t.x[0] = xa; t.y[0] = ya;
    t.x[1] = xb; t.y[1] = ya;
    t.x[2] = xa; t.y[2] = yb;
    t.x[3] = xb; t.y[3] = yb;
  }
  return t;
}

int mcu_of(const Level& L, int x, int y) { return (x / L.mw()) + (y / L.mw()) * L.mcus_x; }

Level* find_level(TexSet& S, int tex, int level) {
  auto it = S.levels.find({tex, level});
  return it == S.levels.end() ? nullptr : it->second;
}

}  // namespace

// =======================================================================================
// C interface
// =======================================================================================
extern "C" {

void jto_zigzag(int* out) { std::memcpy(out, zigzag(), 64 * sizeof(int)); }

void jto_idct_matrix(int64_t* out) { std::memcpy(out, idct_matrix(), 64 * sizeof(int64_t)); }

void jto_idct_raw(const int32_t* d, int32_t* out, int nblocks) {
  for (int b = 0; b < nblocks; ++b) idct_raw(d + 64 * b, out + 64 * b);
}

// Reduced-size IDCT: N x N pixels (row-major, N*N bytes per block) from the N x N lowest
// frequencies of each dequantised block.
void jto_idct_pixels_n(const int32_t* d, uint8_t* out, int nblocks, int N) {
  for (int b = 0; b < nblocks; ++b) idct_pixels(d + 64 * b, out + N * N * b, N);
}

void jto_idct_pixels(const int32_t* d, uint8_t* out, int nblocks) {
  for (int b = 0; b < nblocks; ++b) idct_pixels(d + 64 * b, out + 64 * b);
}

void jto_ycc_to_rgb(const uint8_t* ycc, uint8_t* rgb, int64_t n) {
  for (int64_t i = 0; i < n; ++i) ycc_to_rgb(ycc[3 * i], ycc[3 * i + 1], ycc[3 * i + 2], rgb + 3 * i);
}

// Canonical decode tables: mincode/maxcode/valptr[17] for one spec; returns 0 if valid.
int jto_huff_tables(const uint8_t* bits, const uint8_t* vals, int32_t* mincode, int32_t* maxcode,
                    int32_t* valptr) {
  HuffTable t = make_table(bits, vals);
  if (!t.ok) return -1;
  std::memcpy(mincode, t.mincode, sizeof t.mincode);
  std::memcpy(maxcode, t.maxcode, sizeof t.maxcode);
  std::memcpy(valptr, t.valptr, sizeof t.valptr);
  return 0;
}

// Decodes one symbol from `nbytes` bytes starting at bit 0; returns the symbol, the number
// of bits consumed in *len, or -1 when no code matches.
int jto_huff_decode_one(const uint8_t* bits, const uint8_t* vals, const uint8_t* data, int nbytes, int* len) {
  HuffTable t = make_table(bits, vals);
  BitReader br{data, (uint64_t)nbytes, 0};
  bool err = false;
  int s = decode_symbol(br, t, err);
  *len = (int)br.pos;
  return err ? -1 : s;
}

// --- full sequential decode of a JFIF file ---
void* jto_decode_jfif(const uint8_t* jfif, size_t n) { return decode_jfif(jfif, n); }

// info: [status, w, h, sampling, mcus_x, mcus_y, scan_bytes, coded_bits]
void jto_decoded_info(void* h, int64_t* info) {
  Decoded* D = static_cast<Decoded*>(h);
  info[0] = D->status;
  info[1] = D->w;
  info[2] = D->h;
  info[3] = D->sampling;
  info[4] = D->mcus_x;
  info[5] = D->mcus_y;
  info[6] = (int64_t)D->scan.size();
  info[7] = (int64_t)D->coded_bits;
}

void jto_decoded_copy(void* h, uint8_t* rgba, int32_t* qcoef, void* index, uint8_t* scan, uint16_t* qt,
                      uint8_t* hbits, uint8_t* hvals) {
  Decoded* D = static_cast<Decoded*>(h);
  if (rgba) std::memcpy(rgba, D->rgba.data(), D->rgba.size());
  if (qcoef) std::memcpy(qcoef, D->qcoef.data(), D->qcoef.size() * sizeof(int32_t));
  if (index) std::memcpy(index, D->index.data(), D->index.size() * sizeof(BlockIndex));
  if (scan) std::memcpy(scan, D->scan.data(), D->scan.size());
  if (qt) std::memcpy(qt, D->qt, sizeof D->qt);
  if (hbits) std::memcpy(hbits, D->hbits, sizeof D->hbits);
  if (hvals) std::memcpy(hvals, D->hvals, sizeof D->hvals);
}

void jto_decoded_free(void* h) { delete static_cast<Decoded*>(h); }

// --- texture set (random access) ---
void* jto_texset_new() { return new TexSet(); }
void jto_texset_free(void* s) { delete static_cast<TexSet*>(s); }

static Level* new_level(int tex, int level, int w, int h, int sampling, uint64_t nindex, const uint16_t* qt,
                        const uint8_t* hbits, const uint8_t* hvals) {
  Level* L = new Level();
  L->tex = tex;
  L->level = level;
  L->w = w;
  L->h = h;
  L->sampling = sampling;
  L->mcus_x = (w + L->mw() - 1) / L->mw();
  L->mcus_y = (h + L->mw() - 1) / L->mw();
  std::memcpy(L->qt, qt, sizeof L->qt);
  bool ok = (uint64_t)L->mcus_x * L->mcus_y == nindex;
  for (int t = 0; t < 4 && ok; ++t) {
    L->tab[t] = make_table(hbits + 16 * t, hvals + 256 * t);
    ok = L->tab[t].ok;
  }
  if (!ok) {
    delete L;
    return nullptr;
  }
  return L;
}

static int64_t register_level(TexSet* S, Level* L) {
  L->gid_base = S->next_gid;
  S->next_gid += (uint32_t)(L->mcus_x * L->mcus_y);
  S->levels[{L->tex, L->level}] = L;
  S->order.push_back(L);
  return L->gid_base;
}

// Registers one (texture, level) with the data the CUDA path receives. Levels receive
// consecutive global MCU ids in registration order. Returns the level's gid base, or -1.
int64_t jto_texset_add(void* s, int tex, int level, int w, int h, int sampling, const uint8_t* scan,
                       uint64_t nbytes, uint64_t nbits, const void* index, uint64_t nindex, const uint16_t* qt,
                       const uint8_t* hbits, const uint8_t* hvals) {
  TexSet* S = static_cast<TexSet*>(s);
  if (S->levels.count({tex, level})) return -1;
  Level* L = new_level(tex, level, w, h, sampling, nindex, qt, hbits, hvals);
  if (!L) return -1;
  L->scan.assign(scan, scan + nbytes);
  L->nbits = nbits;
  const BlockIndex* bi = static_cast<const BlockIndex*>(index);
  L->index.assign(bi, bi + nindex);
  return register_level(S, L);
}

// The same for a level in the compact form: nabs = ceil(n / 9) absolute byte offsets,
// 8 nabs relative ones, ceil(36 n / 32) words of DC records. Returns the gid base, or -1.
int64_t jto_texset_add_compact(void* s, int tex, int level, int w, int h, int sampling, const uint8_t* scan,
                               uint64_t nbytes, const uint32_t* abs_off, uint64_t nabs, const uint16_t* rel_off,
                               uint64_t nrel, const uint32_t* dc, uint64_t ndc, uint64_t nindex,
                               const uint16_t* qt, const uint8_t* hbits, const uint8_t* hvals) {
  TexSet* S = static_cast<TexSet*>(s);
  if (S->levels.count({tex, level})) return -1;
  if (nabs != (nindex + 8) / 9 || nrel != 8 * nabs || ndc != (36 * nindex + 31) / 32) return -1;
  Level* L = new_level(tex, level, w, h, sampling, nindex, qt, hbits, hvals);
  if (!L) return -1;
  L->compact = true;
  L->scan.assign(scan, scan + nbytes);
  L->nbits = 8 * nbytes;
  L->c_abs.assign(abs_off, abs_off + nabs);
  L->c_rel.assign(rel_off, rel_off + nrel);
  L->c_dc.assign(dc, dc + ndc);
  return register_level(S, L);
}

// Registers level `level` of texture `tex` as the reduced-resolution decode of the already
// registered level `src_level` (the mip alternative of Sec. 7): each MCU of the source,
// decoded from its N x N lowest frequencies (N = 8 >> reduce), gives a tile of 1/2^reduce
// the size. The level is max(1, w >> reduce) x max(1, h >> reduce) texels on the source's
// MCU grid and gets its own gid range. Returns the gid base, or -1.
int64_t jto_texset_add_reduced(void* s, int tex, int src_level, int reduce, int level) {
  TexSet* S = static_cast<TexSet*>(s);
  Level* src = find_level(*S, tex, src_level);
  if (!src || src->reduce != 0 || reduce < 1 || reduce > 3 || S->levels.count({tex, level})) return -1;
  Level* L = new Level(*src);
  L->tiles.clear();
  L->full.clear();
  L->level = level;
  L->reduce = reduce;
  L->src = src_level;
  L->w = std::max(1, src->w >> reduce);
  L->h = std::max(1, src->h >> reduce);
  return register_level(S, L);
}

// Records data-unit starts for a standard-form level (and so for the reduced levels made
// from it later): [mcu][ndu - 1] offsets in bits from each MCU's first bit. Returns 0 or -1.
int jto_texset_set_du_offsets(void* s, int tex, int level, const uint16_t* offs, uint64_t n) {
  TexSet* S = static_cast<TexSet*>(s);
  Level* L = find_level(*S, tex, level);
  const int ndu = L && L->sampling == 420 ? 6 : 3;
  if (!L || L->compact || n != (uint64_t)L->mcus_x * L->mcus_y * (ndu - 1)) return -1;
  L->du_off.assign(offs, offs + n);
  for (Level* R : S->order)  // reduced levels share the source's stream
    if (R->tex == tex && R->reduce != 0 && R->src == level) R->du_off = L->du_off;
  return 0;
}

// The data-unit starts a sequential decode of a standard-form level finds:
// [mcu][ndu - 1] offsets from each MCU's first bit. Returns 0, or -1 on a corrupt stream.
int jto_du_starts(void* s, int tex, int level, int64_t* out) {
  TexSet* S = static_cast<TexSet*>(s);
  Level* L = find_level(*S, tex, level);
  if (!L || L->compact) return -1;
  const int ndu = L->sampling == 420 ? 6 : 3;
  BitReader br{L->scan.data(), L->scan.size(), 0};
  int16_t pred[3] = {0, 0, 0};
  int32_t q[64];
  for (int m = 0; m < L->mcus_x * L->mcus_y; ++m) {
    const uint64_t start = br.pos;
    for (int d = 0; d < ndu; ++d) {
      if (d) out[(size_t)m * (ndu - 1) + d - 1] = (int64_t)(br.pos - start);
      int comp = d < ndu - 2 ? 0 : (d == ndu - 2 ? 1 : 2);
      int tb = comp == 0 ? 0 : 1;
      if (!decode_du(br, L->tab[tb * 2], L->tab[tb * 2 + 1], pred[comp], q)) return -1;
    }
  }
  return 0;
}

// For a level in the standard form, per MCU: its coded bits and the bits its first luma DC
// and its chroma DCs take (what the compact form moves out of the stream, Sec. 5.3), from a
// sequential decode. Returns 0, or -1 on a corrupt stream or a compact level.
int jto_mcu_bits(void* s, int tex, int level, int64_t* bits, int64_t* dc_bits) {
  TexSet* S = static_cast<TexSet*>(s);
  Level* L = find_level(*S, tex, level);
  if (!L || L->compact) return -1;
  const int ndu = L->sampling == 420 ? 6 : 3;
  BitReader br{L->scan.data(), L->scan.size(), 0};
  int16_t pred[3] = {0, 0, 0};
  int32_t q[64];
  for (int m = 0; m < L->mcus_x * L->mcus_y; ++m) {
    const uint64_t start = br.pos;
    dc_bits[m] = 0;
    for (int d = 0; d < ndu; ++d) {
      int comp = d < ndu - 2 ? 0 : (d == ndu - 2 ? 1 : 2);
      int tb = comp == 0 ? 0 : 1;
      int db = 0;
      if (!decode_du(br, L->tab[tb * 2], L->tab[tb * 2 + 1], pred[comp], q, true, &db)) return -1;
      if (d == 0 || comp != 0) dc_bits[m] += db;
    }
    bits[m] = (int64_t)(br.pos - start);
  }
  return br.pos == L->nbits ? 0 : -1;
}

// Random-access decode of one MCU into an RGBA8 tile; returns 0 or -1 (corrupt).
int jto_texset_decode_mcu(void* s, int tex, int level, int mcu, uint8_t* tile) {
  TexSet* S = static_cast<TexSet*>(s);
  Level* L = find_level(*S, tex, level);
  if (!L || mcu < 0 || mcu >= L->mcus_x * L->mcus_y) return -1;
  return decode_mcu(*L, mcu, tile);
}

// Mark (Sec. 4.2, Sec. 4.6): flags every global MCU id that a pixel's texel(s) fall in.
// flags has one byte per global MCU id. Returns the number of pixels that name a
// missing (texture, level) pair.
int64_t jto_mark(void* s, const float* uv, const uint16_t* tex, const uint8_t* mip, int64_t npx, int filter,
                 uint8_t* flags) {
  TexSet* S = static_cast<TexSet*>(s);
  int64_t bad = 0;
  for (int64_t p = 0; p < npx; ++p) {
    if (tex[p] == 0xFFFF) continue;
    Level* L = find_level(*S, tex[p], mip[p]);
    if (!L) {
      ++bad;
      continue;
    }
    // the clamped mode needs only the nearest texel's MCU
    Taps t = pixel_taps(uv[2 * p], uv[2 * p + 1], L->w, L->h, filter == 2 ? 0 : filter);
    for (int i = 0; i < t.n; ++i) flags[L->gid_base + mcu_of(*L, t.x[i], t.y[i])] = 1;
  }
  return bad;
}

// Compact: gids with a set flag, ascending. Returns the count.
int64_t jto_compact(const uint8_t* flags, int64_t n, uint32_t* out) {
  int64_t c = 0;
  for (int64_t g = 0; g < n; ++g)
    if (flags[g]) out[c++] = (uint32_t)g;
  return c;
}

// Resolve (Sec. 4.4): RGBA8 per pixel from random-access decoded MCUs. Bilinear blends
// in double precision; output floor(c + 1/2) clamped. Empty pixels are (0,0,0,255).
// Returns the number of pixels whose MCU failed to decode or whose level is missing.
int64_t jto_colorize(void* s, const float* uv, const uint16_t* tex, const uint8_t* mip, int64_t npx, int filter,
                     uint8_t* out) {
  TexSet* S = static_cast<TexSet*>(s);
  int64_t bad = 0;
  for (int64_t p = 0; p < npx; ++p) {
    uint8_t* o = out + 4 * p;
    o[0] = o[1] = o[2] = 0;
    o[3] = 255;
    if (tex[p] == 0xFFFF) continue;
    Level* L = find_level(*S, tex[p], mip[p]);
    if (!L) {
      ++bad;
      continue;
    }
    const int mw = L->mw();
    Taps t = pixel_taps(uv[2 * p], uv[2 * p + 1], L->w, L->h, filter, mw);
    double c[4][3];
    bool ok = true;
    for (int i = 0; i < t.n; ++i) {
      const uint8_t* tile = get_tile(*L, mcu_of(*L, t.x[i], t.y[i]));
      if (!tile) {
        ok = false;
        break;
      }
      const uint8_t* texel = tile + ((t.y[i] % mw) * mw + (t.x[i] % mw)) * 4;
      for (int ch = 0; ch < 3; ++ch) c[i][ch] = texel[ch];
    }
    if (!ok) {
      ++bad;
      continue;
    }
    for (int ch = 0; ch < 3; ++ch) {
      double v;
      if (t.n == 1) {
        v = c[0][ch];
      } else {
        double fx = t.fx, fy = t.fy;
        v = (1 - fy) * ((1 - fx) * c[0][ch] + fx * c[1][ch]) + fy * ((1 - fx) * c[2][ch] + fx * c[3][ch]);
      }
      o[ch] = (uint8_t)clamp64((int64_t)std::floor(v + 0.5), 0, 255);
    }
  }
  return bad;
}

// Number of decoded (cached) MCU tiles, i.e. the distinct MCUs colourise needed.
int64_t jto_texset_cached(void* s) {
  TexSet* S = static_cast<TexSet*>(s);
  int64_t n = 0;
  for (Level* L : S->order) n += (int64_t)L->tiles.size();
  return n;
}

void jto_texset_clear_cache(void* s) {
  TexSet* S = static_cast<TexSet*>(s);
  for (Level* L : S->order) L->tiles.clear();
}

// ---------------------------------------------------------------------------------------
// Float colourise chain (FP64): F = bilinear(RGB(upsample(IDCT_f(c) + 128)))
// c: float32 [T][my][mx][6][64] dequantised DCT coefficients (natural order k = v*8+u),
// 4:2:0, textures of size W x H, level 0; G-buffer uv/tex (no mip); F: [npx][3].
// ---------------------------------------------------------------------------------------
}  // extern "C"

namespace {

struct FloatGeom {
  int T, W, H, mx, my;
  size_t mcu_stride() const { return 6 * 64; }
  size_t coef_index(int t, int mcu, int du, int k) const {
    return (((size_t)t * my * mx + mcu) * 6 + du) * 64 + k;
  }
};

double dct_basis(int x, int u) {  // C(u)/2 * cos((2x+1) u pi / 16)
  double cu = u == 0 ? std::sqrt(0.5) : 1.0;
  return 0.5 * cu * std::cos((2 * x + 1) * u * M_PI / 16.0);
}

// IDCT_f of one DU: f(y,x) = sum_v sum_u [C(u)C(v)/4] c[v*8+u] cos(..x..u) cos(..y..v)
void idct_f(const double c[64], double f[64]) {
  for (int y = 0; y < 8; ++y)
    for (int x = 0; x < 8; ++x) {
      double s = 0;
      for (int v = 0; v < 8; ++v)
        for (int u = 0; u < 8; ++u) s += dct_basis(x, u) * dct_basis(y, v) * c[v * 8 + u];
      f[y * 8 + x] = s;
    }
}

// Adjoint of idct_f (the 2-D forward DCT-II with the same normalisation).
void idct_f_adjoint(const double g[64], double c[64]) {
  for (int v = 0; v < 8; ++v)
    for (int u = 0; u < 8; ++u) {
      double s = 0;
      for (int y = 0; y < 8; ++y)
        for (int x = 0; x < 8; ++x) s += dct_basis(x, u) * dct_basis(y, v) * g[y * 8 + x];
      c[v * 8 + u] = s;
    }
}

const double kCr2R = 1.402, kCb2G = 0.344136, kCr2G = 0.714136, kCb2B = 1.772;

// Float RGB tile of one MCU [16][16][3].
void float_tile(const FloatGeom& G, const float* coef, int t, int mcu, double tile[16][16][3]) {
  double f[6][64];
  for (int d = 0; d < 6; ++d) {
    double c[64];
    for (int k = 0; k < 64; ++k) c[k] = coef[G.coef_index(t, mcu, d, k)];
    idct_f(c, f[d]);
  }
  for (int y = 0; y < 16; ++y)
    for (int x = 0; x < 16; ++x) {
      double Y = f[(y / 8) * 2 + (x / 8)][(y % 8) * 8 + (x % 8)] + 128.0;
      double Cb = f[4][(y >> 1) * 8 + (x >> 1)] + 128.0 - 128.0;
      double Cr = f[5][(y >> 1) * 8 + (x >> 1)] + 128.0 - 128.0;
      tile[y][x][0] = Y + kCr2R * Cr;
      tile[y][x][1] = Y - kCb2G * Cb - kCr2G * Cr;
      tile[y][x][2] = Y + kCb2B * Cb;
    }
}

struct FloatPixel {
  bool valid;
  int t;
  int mcu[4], tx[4], ty[4];
  double w[4];
};

FloatPixel float_pixel(const FloatGeom& G, float u, float v, uint16_t tex) {
  FloatPixel P{};
  if (tex == 0xFFFF || tex >= G.T) return P;
  Taps tp = pixel_taps(u, v, G.W, G.H, 1);
  P.valid = true;
  P.t = tex;
  double fx = tp.fx, fy = tp.fy;
  double w[4] = {(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy};
  for (int i = 0; i < 4; ++i) {
    P.mcu[i] = (tp.x[i] / 16) + (tp.y[i] / 16) * G.mx;
    P.tx[i] = tp.x[i] % 16;
    P.ty[i] = tp.y[i] % 16;
    P.w[i] = w[i];
  }
  return P;
}

struct TileCache {
  const FloatGeom& G;
  const float* coef;
  std::unordered_map<int64_t, std::vector<double>> tiles;
  const double* get(int t, int mcu) {
    int64_t key = (int64_t)t * G.mx * G.my + mcu;
    auto it = tiles.find(key);
    if (it != tiles.end()) return it->second.data();
    std::vector<double> v(16 * 16 * 3);
    float_tile(G, coef, t, mcu, reinterpret_cast<double(*)[16][3]>(v.data()));
    return tiles.emplace(key, std::move(v)).first->second.data();
  }
};

void float_pixel_value(TileCache& C, const FloatPixel& P, double out[3]) {
  out[0] = out[1] = out[2] = 0;
  if (!P.valid) return;
  for (int i = 0; i < 4; ++i) {
    const double* tile = C.get(P.t, P.mcu[i]);
    for (int ch = 0; ch < 3; ++ch) out[ch] += P.w[i] * tile[(P.ty[i] * 16 + P.tx[i]) * 3 + ch];
  }
}

// J^T g for one pixel's RGB gradient, accumulated into per-MCU texel gradients.
void scatter_pixel(const FloatPixel& P, const double g[3], std::unordered_map<int64_t, std::vector<double>>& acc,
                   const FloatGeom& G) {
  if (!P.valid) return;
  for (int i = 0; i < 4; ++i) {
    int64_t key = (int64_t)P.t * G.mx * G.my + P.mcu[i];
    auto& v = acc[key];
    if (v.empty()) v.assign(16 * 16 * 3, 0.0);
    for (int ch = 0; ch < 3; ++ch) v[(P.ty[i] * 16 + P.tx[i]) * 3 + ch] += P.w[i] * g[ch];
  }
}

// Texel RGB gradients of one MCU -> coefficient gradients (colour^T, upsample^T, DCT).
void tile_adjoint(const double* gt /*[16][16][3]*/, double gc[6][64]) {
  double gY[4][64] = {}, gCb[64] = {}, gCr[64] = {};
  for (int y = 0; y < 16; ++y)
    for (int x = 0; x < 16; ++x) {
      const double* g = gt + (y * 16 + x) * 3;
      double gy = g[0] + g[1] + g[2];
      double gcb = -kCb2G * g[1] + kCb2B * g[2];
      double gcr = kCr2R * g[0] - kCr2G * g[1];
      gY[(y / 8) * 2 + (x / 8)][(y % 8) * 8 + (x % 8)] += gy;
      gCb[(y >> 1) * 8 + (x >> 1)] += gcb;
      gCr[(y >> 1) * 8 + (x >> 1)] += gcr;
    }
  for (int d = 0; d < 4; ++d) idct_f_adjoint(gY[d], gc[d]);
  idct_f_adjoint(gCb, gc[4]);
  idct_f_adjoint(gCr, gc[5]);
}

}  // namespace

extern "C" {

void jto_float_forward(const float* coef, int T, int W, int H, const float* uv, const uint16_t* tex, int64_t npx,
                       double* F) {
  FloatGeom G{T, W, H, W / 16, H / 16};
  TileCache C{G, coef, {}};
  for (int64_t p = 0; p < npx; ++p) {
    FloatPixel P = float_pixel(G, uv[2 * p], uv[2 * p + 1], tex[p]);
    float_pixel_value(C, P, F + 3 * p);
  }
}

// J^T g: gradient of sum_p <g_p, F_p> with respect to the coefficients (linear part of
// the chain). out has the coefficient tensor's shape and is overwritten.
void jto_float_vjp(int T, int W, int H, const float* uv, const uint16_t* tex, int64_t npx, const double* g,
                   double* out) {
  FloatGeom G{T, W, H, W / 16, H / 16};
  std::unordered_map<int64_t, std::vector<double>> acc;
  for (int64_t p = 0; p < npx; ++p) {
    FloatPixel P = float_pixel(G, uv[2 * p], uv[2 * p + 1], tex[p]);
    scatter_pixel(P, g + 3 * p, acc, G);
  }
  std::memset(out, 0, (size_t)T * G.mx * G.my * 6 * 64 * sizeof(double));
  for (auto& kv : acc) {
    double gc[6][64];
    tile_adjoint(kv.second.data(), gc);
    int t = (int)(kv.first / ((int64_t)G.mx * G.my)), mcu = (int)(kv.first % ((int64_t)G.mx * G.my));
    for (int d = 0; d < 6; ++d)
      for (int k = 0; k < 64; ++k) out[G.coef_index(t, mcu, d, k)] = gc[d][k];
  }
}

// L = sum_p sum_ch (F - T)^2 and its gradient (= J^T 2 (F - T)).
double jto_float_loss_grad(const float* coef, int T, int W, int H, const float* uv, const uint16_t* tex, int64_t npx,
                           const float* target, double* grad) {
  std::vector<double> F((size_t)npx * 3), g((size_t)npx * 3);
  jto_float_forward(coef, T, W, H, uv, tex, npx, F.data());
  double L = 0;
  for (int64_t i = 0; i < npx * 3; ++i) {
    double r = F[i] - target[i];
    L += r * r;
    g[i] = 2 * r;
  }
  if (grad) jto_float_vjp(T, W, H, uv, tex, npx, g.data(), grad);
  return L;
}

// Central differences (L(c + h e_i) - L(c - h e_i)) / 2h for the listed flat coefficient
// indices. L is a sum over pixels, so each difference only sums the pixels whose taps
// fall in the perturbed MCU (the other terms cancel exactly).
void jto_float_fd(const float* coef, int T, int W, int H, const float* uv, const uint16_t* tex, int64_t npx,
                  const float* target, const int64_t* idx, int nidx, double h, double* out) {
  FloatGeom G{T, W, H, W / 16, H / 16};
  std::unordered_map<int64_t, std::vector<int64_t>> users;  // MCU key -> pixels
  std::vector<FloatPixel> px((size_t)npx);
  for (int64_t p = 0; p < npx; ++p) {
    px[p] = float_pixel(G, uv[2 * p], uv[2 * p + 1], tex[p]);
    if (!px[p].valid) continue;
    std::set<int64_t> keys;
    for (int i = 0; i < 4; ++i) keys.insert((int64_t)px[p].t * G.mx * G.my + px[p].mcu[i]);
    for (int64_t k : keys) users[k].push_back(p);
  }
  const size_t ncoef = (size_t)T * G.mx * G.my * 6 * 64;
  TileCache C{G, coef, {}};  // unperturbed neighbour tiles
  for (int j = 0; j < nidx; ++j) {
    int64_t i = idx[j];
    int64_t key = i / (6 * 64);
    auto it = users.find(key);
    if (i < 0 || (size_t)i >= ncoef || it == users.end()) {
      out[j] = 0.0;
      continue;
    }
    const int du = (int)((i % 384) / 64), kk = (int)(i % 64);
    double Ls[2];
    for (int sgn = 0; sgn < 2; ++sgn) {
      // the perturbed MCU's tile, with the perturbation kept in double precision
      double f[6][64], ftile[16][16][3];
      for (int d = 0; d < 6; ++d) {
        double cc[64];
        for (int k = 0; k < 64; ++k) cc[k] = coef[key * 384 + d * 64 + k];
        if (d == du) cc[kk] += sgn == 0 ? h : -h;
        idct_f(cc, f[d]);
      }
      for (int y = 0; y < 16; ++y)
        for (int x = 0; x < 16; ++x) {
          double Y = f[(y / 8) * 2 + (x / 8)][(y % 8) * 8 + (x % 8)] + 128.0;
          double Cb = f[4][(y >> 1) * 8 + (x >> 1)];
          double Cr = f[5][(y >> 1) * 8 + (x >> 1)];
          ftile[y][x][0] = Y + kCr2R * Cr;
          ftile[y][x][1] = Y - kCb2G * Cb - kCr2G * Cr;
          ftile[y][x][2] = Y + kCb2B * Cb;
        }
      double L = 0;
      for (int64_t p : it->second) {
        const FloatPixel& P = px[p];
        double v[3] = {0, 0, 0};
        for (int q = 0; q < 4; ++q) {
          int64_t k2 = (int64_t)P.t * G.mx * G.my + P.mcu[q];
          const double* tile = k2 == key ? &ftile[0][0][0] : C.get(P.t, P.mcu[q]);
          for (int ch = 0; ch < 3; ++ch) v[ch] += P.w[q] * tile[(P.ty[q] * 16 + P.tx[q]) * 3 + ch];
        }
        for (int ch = 0; ch < 3; ++ch) {
          double r = v[ch] - target[3 * p + ch];
          L += r * r;
        }
      }
      Ls[sgn] = L;
    }
    out[j] = (Ls[0] - Ls[1]) / (2 * h);
  }
}

}  // extern "C"

// =======================================================================================
// Scene rasteriser: the G-buffer of the procedural scene (ground plane + projective quads)
// that the geometry pass of the paper's renderer (Sec. 4, "Geometry Pass") would produce,
// in fp32 with every operation rounded in the order written (no contraction), so that a
// GPU renderer doing the same operations takes the same decisions. The scene's definition
// (double precision) lives in the input generator; this is its fp32 restatement.
// =======================================================================================
namespace {

struct RScene {
  int W, H;
  const float* p;  // cam[3] rot[9] ax ay tan_x tan_y max_t kx ky shift
  uint64_t cell_seed;
  int ntex, use_mips;
  const int32_t *tw, *th, *tl;
};

#pragma pack(push, 4)
struct RQuad {
  float cx[4], cy[4], ex[4], ey[4], h[9], rep, cs, sn, ou, ov;
  int32_t tex, x0, y0, x1, y1;
};
#pragma pack(pop)
static_assert(sizeof(RQuad) == 140, "quad record");

// SplitMix64 (Steele, Lea, Flood 2014), as the generator keys its ground cells
uint64_t splitmix_next(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
uint64_t cell_hash(uint64_t seed, uint64_t a, uint64_t b) {
  uint64_t s = seed ^ (a * 0xD1B54A32D192ED03ull) ^ (b * 0x8CB92BA72F3D8DD7ull);
  splitmix_next(s);
  return splitmix_next(s);
}

// Ground hit of the ray through pixel coordinate (px, py): uv = world (x, z) / 2.
bool r_ground(const RScene& S, float px, float py, float& u, float& v) {
  const float* c = S.p;
  const float* R = S.p + 3;
  const float ax = S.p[12], ay = S.p[13], tx = S.p[14], ty = S.p[15], max_t = S.p[16];
  const float sx = (px * ax - 1.0f) * tx;
  const float sy = (1.0f - py * ay) * ty;
  const float dx = (R[0] * sx + R[1] * sy) - R[2];
  const float dy = (R[3] * sx + R[4] * sy) - R[5];
  const float dz = (R[6] * sx + R[7] * sy) - R[8];
  if (!(dy < -1e-9f)) return false;
  const float t = -c[1] / dy;
  if (t > max_t) return false;
  u = (c[0] + t * dx) * 0.5f;
  v = (c[2] + t * dz) * 0.5f;
  return true;
}

// Level from the squared footprint r2 (texels^2): floor(log2(sqrt(r2)) + 1/2) clamped to
// [0, L-1], i.e. the number of k >= 1 with r2 >= 2^(2k-1).
int r_level(float r2, int L) {
  if (!(r2 > 0.0f)) return 0;
  int m = 0;
  while (m + 1 <= L - 1 && r2 >= std::ldexp(1.0f, 2 * (m + 1) - 1)) ++m;
  return m;
}

float r_footprint(float u0, float v0, float u1, float v1, int w, int h) {
  const float du = (u1 - u0) * (float)w, dv = (v1 - v0) * (float)h;
  return du * du + dv * dv;
}

void r_quad_uv(const RQuad& q, float x, float y, float& u, float& v) {
  float s = (q.h[0] * x + q.h[1] * y) + q.h[2];
  float t = (q.h[3] * x + q.h[4] * y) + q.h[5];
  const float w = (q.h[6] * x + q.h[7] * y) + q.h[8];
  s = s / w;
  t = t / w;
  u = q.ou + q.rep * (q.cs * s - q.sn * t);
  v = q.ov + q.rep * (q.sn * s + q.cs * t);
}

bool r_inside(const RQuad& q, float x, float y) {
  for (int i = 0; i < 4; ++i)
    if (q.ex[i] * (y - q.cy[i]) - q.ey[i] * (x - q.cx[i]) < 0.0f) return false;
  return true;
}

}  // namespace

extern "C" {

// params: cam[3] rot[9] ax ay tan_x tan_y max_t kx ky shift (20 floats); quads: nquads
// records of 140 bytes; outputs uv [H][W][2], tex [H][W], mip [H][W].
void jto_raster_scene(int W, int H, const float* params, uint64_t cell_seed, int ntex, const int32_t* tw,
                      const int32_t* th, const int32_t* tl, int use_mips, const void* quads, int nquads, float* uv,
                      uint16_t* tex, uint8_t* mip) {
  RScene S{W, H, params, cell_seed, ntex, use_mips, tw, th, tl};
  const RQuad* Q = static_cast<const RQuad*>(quads);
  const float kx = params[17], ky = params[18], shift = params[19];
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      const size_t p = (size_t)y * W + x;
      const float fx = (float)x + 0.5f, fy = (float)y + 0.5f;
      int hit = -1;
      const float qx = fx * kx - shift, qy = fy * ky;
      for (int n = nquads - 1; n >= 0 && hit < 0; --n)  // the last quad drawn wins
        if (x >= Q[n].x0 && x <= Q[n].x1 && y >= Q[n].y0 && y <= Q[n].y1 && r_inside(Q[n], qx, qy)) hit = n;
      float u = 0.f, v = 0.f;
      int t = 0xFFFF, lvl = 0;
      if (hit >= 0) {
        const RQuad& q = Q[hit];
        t = q.tex;
        r_quad_uv(q, qx, qy, u, v);
        if (use_mips) {
          const float hx = kx * 0.5f, hy = ky * 0.5f;
          float u0, v0, u1, v1, u2, v2, u3, v3;
          r_quad_uv(q, qx - hx, qy, u0, v0);
          r_quad_uv(q, qx + hx, qy, u1, v1);
          r_quad_uv(q, qx, qy - hy, u2, v2);
          r_quad_uv(q, qx, qy + hy, u3, v3);
          const float rx = r_footprint(u0, v0, u1, v1, tw[t], th[t]);
          const float ry = r_footprint(u2, v2, u3, v3, tw[t], th[t]);
          lvl = r_level(std::max(rx, ry), tl[t]);
        }
      } else if (r_ground(S, fx, fy, u, v)) {
        const int64_t cx = (int64_t)std::floor(u), cz = (int64_t)std::floor(v);  // 2 m cells
        const uint64_t hs = cell_hash(cell_seed, (uint64_t)cx, (uint64_t)cz);
        t = (int)(hs % (uint64_t)ntex);
        u = u + (float)((hs >> 16) & 0xFFFFu) * (1.0f / 65536.0f);  // per-cell uv offset
        v = v + (float)((hs >> 32) & 0xFFFFu) * (1.0f / 65536.0f);
        if (use_mips) {
          float u0, v0, u1, v1, u2, v2, u3, v3;
          const bool ok = r_ground(S, (float)x, fy, u0, v0) && r_ground(S, (float)x + 1.0f, fy, u1, v1) &&
                          r_ground(S, fx, (float)y, u2, v2) && r_ground(S, fx, (float)y + 1.0f, u3, v3);
          if (!ok) {
            lvl = tl[t] - 1;
          } else {
            const float rx = r_footprint(u0, v0, u1, v1, tw[t], th[t]);
            const float ry = r_footprint(u2, v2, u3, v3, tw[t], th[t]);
            lvl = r_level(std::max(rx, ry), tl[t]);
          }
        }
      }
      uv[2 * p] = u;
      uv[2 * p + 1] = v;
      tex[p] = (uint16_t)t;
      mip[p] = (uint8_t)lvl;
    }
}

}  // extern "C"
