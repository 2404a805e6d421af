// Seeded synthetic inputs for the variable-rate (JPEG) texture path.
//
// This module produces everything the path consumes and nothing it computes:
//   * RGB8 textures (1/f value noise + hard-edged rectangles) and 2x2 box mip chains,
//   * a baseline sequential JPEG encoder (the offline step the paper performs with
//     libjpeg-turbo / jpegli, Sec. 6.1) that also emits the unstuffed entropy stream and
//     the per-MCU random-access index (bit offset + DC predictors, Sec. 5.1 / Sec. 5.3),
//   * the same coefficients in the paper's compact form (Sec. 5.1 indexing table and the
//     DC accounting of Sec. 5.3): every MCU starts on a byte; the first luma DC and both
//     chroma DCs leave the entropy stream and are stored as 12-bit absolute values; the
//     byte offset of every ninth MCU is an absolute uint32, the next eight are uint16
//     offsets relative to it,
//   * deferred G-buffers (uv, texture id, mip level; Sec. 4 "Geometry Pass").
//
// It holds none of the decode-side arithmetic: Huffman decoding, dequantisation, the
// inverse DCT, colour conversion back to RGB, MCU marking and texel lookup are written
// independently in the oracle and in the CUDA library. Both of those read what this
// module writes; neither shares code with it.
//
// Every random draw goes through SplitMix64 (Steele, Lea, Flood 2014) keyed by an explicit
// seed, so a given call always produces the same bytes on x86-64 and aarch64.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// ---------------------------------------------------------------------------------------
// Random numbers
// ---------------------------------------------------------------------------------------
struct SplitMix64 {
  uint64_t s;
  explicit SplitMix64(uint64_t seed) : s(seed) {}
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }  // [0,1)
  double uniform(double a, double b) { return a + (b - a) * uniform(); }
  int below(int n) { return (int)(uniform() * n); }
};

uint64_t mix_seed(uint64_t seed, uint64_t a, uint64_t b) {
  SplitMix64 r(seed ^ (a * 0xD1B54A32D192ED03ull) ^ (b * 0x8CB92BA72F3D8DD7ull));
  r.next();
  return r.next();
}

inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// ---------------------------------------------------------------------------------------
// Texture generator: value noise with octaves o = 0..log2(size)-1, lattice spacing
// size/2^(o+1), amplitude 2^-o, smoothstep interpolation, one noise field per channel,
// mixed by a random 3x3 matrix; then 24 axis-aligned solid rectangles.
// ---------------------------------------------------------------------------------------
void value_noise_octave(SplitMix64& rng, int w, int h, double spacing, double amp, float* acc) {
  const int gx = (int)std::ceil(w / spacing) + 2;
  const int gy = (int)std::ceil(h / spacing) + 2;
  std::vector<float> lat((size_t)gx * gy);
  for (auto& v : lat) v = (float)rng.uniform(-1.0, 1.0);
  std::vector<int> ix(w);
  std::vector<float> sx(w);
  for (int x = 0; x < w; ++x) {
    double fx = (x + 0.5) / spacing;
    int i = (int)std::floor(fx);
    double t = fx - i;
    ix[x] = i;
    sx[x] = (float)(t * t * (3.0 - 2.0 * t));
  }
  for (int y = 0; y < h; ++y) {
    double fy = (y + 0.5) / spacing;
    int j = (int)std::floor(fy);
    double t = fy - j;
    float sy = (float)(t * t * (3.0 - 2.0 * t));
    const float* r0 = &lat[(size_t)j * gx];
    const float* r1 = r0 + gx;
    float* out = acc + (size_t)y * w;
    for (int x = 0; x < w; ++x) {
      int i = ix[x];
      float a = r0[i] + (r0[i + 1] - r0[i]) * sx[x];
      float b = r1[i] + (r1[i + 1] - r1[i]) * sx[x];
      out[x] += (float)amp * (a + (b - a) * sy);
    }
  }
}

// Octave amplitude as a function of the lattice spacing in pixels: (spacing/256)^beta,
// capped at 1, so the fine-scale detail per pixel (and so the JPEG bit rate) does not
// depend on the texture size. beta is set so that quality 80 lands near the bit rates
// the paper reports for its textures at Q80 (0.77-0.90 bpp).
const double g_beta = 0.5;
double octave_amplitude(double spacing) { return std::min(1.0, std::pow(spacing / 256.0, g_beta)); }

void gen_texture(uint64_t seed, int w, int h, uint8_t* rgb) {
  const int size = std::max(w, h);
  int noct = 0;
  while ((1 << (noct + 1)) <= size) ++noct;  // floor(log2(size))
  noct = std::max(noct, 1);
  std::vector<float> field[3];
  for (int c = 0; c < 3; ++c) {
    field[c].assign((size_t)w * h, 0.f);
    SplitMix64 rng(mix_seed(seed, 1, (uint64_t)c));
    for (int o = 0; o < noct; ++o) {
      double spacing = std::max(1.0, (double)size / (double)(2 << o));
      value_noise_octave(rng, w, h, spacing, octave_amplitude(spacing), field[c].data());
    }
  }
  SplitMix64 rng(mix_seed(seed, 2, 0));
  double m[3][3];
  for (auto& row : m)
    for (double& v : row) v = rng.uniform(-1.0, 1.0);
  const size_t n = (size_t)w * h;
  for (size_t p = 0; p < n; ++p) {
    double f0 = field[0][p], f1 = field[1][p], f2 = field[2][p];
    for (int c = 0; c < 3; ++c) {
      double v = 128.0 + 64.0 * (m[c][0] * f0 + m[c][1] * f1 + m[c][2] * f2);
      rgb[p * 3 + c] = (uint8_t)clampi((int)std::lround(v), 0, 255);
    }
  }
  const double scale = size / 512.0;
  for (int r = 0; r < 24; ++r) {
    int rw = (int)std::lround(rng.uniform(8.0, 160.0) * scale);
    int rh = (int)std::lround(rng.uniform(8.0, 160.0) * scale);
    int x0 = rng.below(w), y0 = rng.below(h);
    uint8_t col[3] = {(uint8_t)rng.below(256), (uint8_t)rng.below(256), (uint8_t)rng.below(256)};
    for (int y = y0; y < std::min(h, y0 + std::max(rh, 1)); ++y)
      for (int x = x0; x < std::min(w, x0 + std::max(rw, 1)); ++x)
        for (int c = 0; c < 3; ++c) rgb[((size_t)y * w + x) * 3 + c] = col[c];
  }
}

// 2x2 box filter, (a+b+c+d+2)>>2, odd sizes take floor(n/2) with edge clamp.
void mip_down(const uint8_t* src, int w, int h, uint8_t* dst) {
  const int w2 = std::max(1, w / 2), h2 = std::max(1, h / 2);
  for (int y = 0; y < h2; ++y)
    for (int x = 0; x < w2; ++x) {
      int xa = std::min(2 * x, w - 1), xb = std::min(2 * x + 1, w - 1);
      int ya = std::min(2 * y, h - 1), yb = std::min(2 * y + 1, h - 1);
      for (int c = 0; c < 3; ++c) {
        int s = src[((size_t)ya * w + xa) * 3 + c] + src[((size_t)ya * w + xb) * 3 + c] +
                src[((size_t)yb * w + xa) * 3 + c] + src[((size_t)yb * w + xb) * 3 + c];
        dst[((size_t)y * w2 + x) * 3 + c] = (uint8_t)((s + 2) >> 2);
      }
    }
}

// ---------------------------------------------------------------------------------------
// Baseline JPEG encoder (ITU-T T.81, sequential DCT, Huffman, 8-bit, 3 components,
// 4:2:0 or 4:4:4, no restart intervals).
// ---------------------------------------------------------------------------------------

// Zig-zag scan order, generated by walking the anti-diagonals of the 8x8 block and
// alternating direction. zz[k] = natural (row-major) index of the k-th coefficient.
struct ZigZag {
  int zz[64];
  ZigZag() {
    int k = 0;
    for (int s = 0; s < 15; ++s) {
      if (s % 2 == 0) {  // walk up-right: row decreases
        for (int r = std::min(s, 7); r >= 0 && s - r <= 7; --r) zz[k++] = r * 8 + (s - r);
      } else {  // walk down-left: row increases
        for (int r = std::max(0, s - 7); r <= std::min(s, 7); ++r) zz[k++] = r * 8 + (s - r);
      }
    }
  }
};
const ZigZag kZZ;

// Annex K.1 example quantisation tables, natural order (luminance, chrominance).
const uint8_t kQLuma[64] = {16, 11, 10, 16, 24,  40,  51,  61,  12, 12, 14, 19, 26,  58,  60,  55,
                            14, 13, 16, 24, 40,  57,  69,  56,  14, 17, 22, 29, 51,  87,  80,  62,
                            18, 22, 37, 56, 68,  109, 103, 77,  24, 35, 55, 64, 81,  104, 113, 92,
                            49, 64, 78, 87, 103, 121, 120, 101, 72, 92, 95, 98, 112, 100, 103, 99};
const uint8_t kQChromaTop[4][4] = {{17, 18, 24, 47}, {18, 21, 26, 66}, {24, 26, 56, 99}, {47, 66, 99, 99}};

// IJG-style quality scaling, entries clamped to [1,255] (8-bit baseline tables).
void quality_tables(int quality, uint16_t qt[2][64]) {
  quality = clampi(quality, 1, 100);
  int scale = quality < 50 ? 5000 / quality : 200 - 2 * quality;
  for (int i = 0; i < 64; ++i) {
    int r = i / 8, c = i % 8;
    int base_c = (r < 4 && c < 4) ? kQChromaTop[r][c] : 99;
    qt[0][i] = (uint16_t)clampi((kQLuma[i] * scale + 50) / 100, 1, 255);
    qt[1][i] = (uint16_t)clampi((base_c * scale + 50) / 100, 1, 255);
  }
}

struct HuffSpec {
  uint8_t bits[16];
  uint8_t vals[256];
  int nvals;
};

// Annex K.3 typical Huffman tables. The AC tables list the symbols with codes shorter
// than 16 bits explicitly; all remaining valid (run,size) symbols follow in ascending
// order, each with a 16-bit code.
HuffSpec make_ac_spec(const uint8_t bits[16], const uint8_t* head, int nhead) {
  HuffSpec s{};
  std::memcpy(s.bits, bits, 16);
  bool used[256] = {};
  for (int i = 0; i < nhead; ++i) {
    s.vals[i] = head[i];
    used[head[i]] = true;
  }
  int n = nhead;
  for (int sym = 0; sym < 256; ++sym) {
    int r = sym >> 4, sz = sym & 15;
    bool valid = (sz >= 1 && sz <= 10) || sym == 0x00 || sym == 0xF0;
    (void)r;
    if (valid && !used[sym]) s.vals[n++] = (uint8_t)sym;
  }
  s.nvals = n;
  return s;
}

HuffSpec make_dc_spec(const uint8_t bits[16]) {
  HuffSpec s{};
  std::memcpy(s.bits, bits, 16);
  for (int i = 0; i < 12; ++i) s.vals[i] = (uint8_t)i;
  s.nvals = 12;
  return s;
}

void standard_specs(HuffSpec out[4]) {
  static const uint8_t dc_l[16] = {0, 1, 5, 1, 1, 1, 1, 1, 1, 0, 0, 0, 0, 0, 0, 0};
  static const uint8_t dc_c[16] = {0, 3, 1, 1, 1, 1, 1, 1, 1, 1, 1, 0, 0, 0, 0, 0};
  static const uint8_t ac_l[16] = {0, 2, 1, 3, 3, 2, 4, 3, 5, 5, 4, 4, 0, 0, 1, 0x7d};
  static const uint8_t ac_c[16] = {0, 2, 1, 2, 4, 4, 3, 4, 7, 5, 4, 4, 0, 1, 2, 0x77};
  static const uint8_t ac_l_head[37] = {0x01, 0x02, 0x03, 0x00, 0x04, 0x11, 0x05, 0x12, 0x21, 0x31,
                                        0x41, 0x06, 0x13, 0x51, 0x61, 0x07, 0x22, 0x71, 0x14, 0x32,
                                        0x81, 0x91, 0xa1, 0x08, 0x23, 0x42, 0xb1, 0xc1, 0x15, 0x52,
                                        0xd1, 0xf0, 0x24, 0x33, 0x62, 0x72, 0x82};
  static const uint8_t ac_c_head[43] = {0x00, 0x01, 0x02, 0x03, 0x11, 0x04, 0x05, 0x21, 0x31, 0x06, 0x12,
                                        0x41, 0x51, 0x07, 0x61, 0x71, 0x13, 0x22, 0x32, 0x81, 0x08, 0x14,
                                        0x42, 0x91, 0xa1, 0xb1, 0xc1, 0x09, 0x23, 0x33, 0x52, 0xf0, 0x15,
                                        0x62, 0x72, 0xd1, 0x0a, 0x16, 0x24, 0x34, 0xe1, 0x25, 0xf1};
  out[0] = make_dc_spec(dc_l);
  out[1] = make_ac_spec(ac_l, ac_l_head, 37);
  out[2] = make_dc_spec(dc_c);
  out[3] = make_ac_spec(ac_c, ac_c_head, 43);
}

// Encoder-side canonical code assignment (Annex C): codes of each length are
// consecutive integers, and the first code of length l+1 is (last code of length l + 1) << 1.
struct HuffEnc {
  uint16_t code[256];
  uint8_t len[256];
};

HuffEnc encoder_codes(const HuffSpec& s) {
  HuffEnc e{};
  int code = 0, k = 0;
  for (int l = 1; l <= 16; ++l) {
    for (int i = 0; i < s.bits[l - 1]; ++i) {
      e.code[s.vals[k]] = (uint16_t)code;
      e.len[s.vals[k]] = (uint8_t)l;
      ++code;
      ++k;
    }
    code <<= 1;
  }
  return e;
}

#pragma pack(push, 2)
struct BlockIndex {
  uint32_t bit_offset;
  int16_t dc_pred[3];
};
#pragma pack(pop)
static_assert(sizeof(BlockIndex) == 10, "packed 80-bit index entry");

struct BitWriter {
  std::vector<uint8_t>* stuffed;
  std::vector<uint8_t>* plain;
  uint64_t acc = 0;
  int nacc = 0;
  uint64_t nbits = 0;  // bits written to the unstuffed stream
  void put(uint32_t v, int n) {
    if (n == 0) return;
    acc = (acc << n) | (v & ((1u << n) - 1u));
    nacc += n;
    nbits += (uint64_t)n;
    while (nacc >= 8) {
      uint8_t b = (uint8_t)(acc >> (nacc - 8));
      nacc -= 8;
      plain->push_back(b);
      stuffed->push_back(b);
      if (b == 0xFF) stuffed->push_back(0x00);
    }
  }
  void flush_ones() {
    if (nacc > 0) {
      int pad = 8 - nacc;
      // padding bits are ones (T.81 F.1.2.3); they are not counted as coded bits
      uint64_t keep = nbits;
      put((1u << pad) - 1u, pad);
      nbits = keep;
    }
  }
};

int category(int v) {
  int a = v < 0 ? -v : v;
  int s = 0;
  while (a) {
    ++s;
    a >>= 1;
  }
  return s;
}

uint32_t magnitude_bits(int v, int s) { return (uint32_t)(v < 0 ? v - 1 : v) & ((1u << s) - 1u); }

// The compact form (see the header): a byte-aligned stream without the absolute DCs, the
// two-level offset table and the 36-bit DC records, bit i of the record array being bit
// (i mod 32) of word i / 32, MCU m's values (first Y, Cb, Cr; 12-bit two's complement) at
// bits 36 m, 36 m + 12, 36 m + 24.
struct Compact {
  std::vector<uint8_t> scan;
  std::vector<uint32_t> abs;  // [ceil(n / 9)]
  std::vector<uint16_t> rel;  // [8 ceil(n / 9)]; entries past the last MCU are 0
  std::vector<uint32_t> dc;   // [ceil(36 n / 32)]
  uint64_t dc_bits_removed = 0;  // bits the absolute DCs took in the standard stream
  uint64_t pad_bits = 0;         // 1-bits that align each MCU to a byte
  int status = 0;                // nonzero: a DC outside 12 bits, or a relative offset > 65535
};

struct Encoded {
  int w = 0, h = 0, sampling = 420, mcus_x = 0, mcus_y = 0, quality = 0;
  std::vector<uint8_t> jfif, scan;
  uint64_t scan_bits = 0;
  std::vector<BlockIndex> index;
  uint16_t qt[2][64];
  HuffSpec huff[4];
  std::vector<int16_t> qcoef;  // [mcu][du][64] natural order, quantised (optional)
  Compact compact;
  // start bit of data units 1..ndu-1 of each MCU relative to the MCU's first bit
  std::vector<uint16_t> du_offsets;  // [mcu][ndu - 1]
  // Huffman symbols the standard stream codes per MCU: DC categories, AC (run, size)
  // values, ZRL and EOB codes (a property of the input, for issue-rate accounting)
  std::vector<uint16_t> symbols;  // [mcu]
  int status = 0;
};

// Writes one data unit of quantised coefficients (natural order) to the standard stream bw
// and to the compact stream cw, which leaves out the DC difference when dc_absolute.
// Returns the number of Huffman symbols of the standard stream, or -1.
int encode_du(BitWriter& bw, BitWriter& cw, bool dc_absolute, uint64_t& dc_removed, const int16_t* q, int& pred,
              const HuffEnc& dc, const HuffEnc& ac) {
  auto put = [&](uint32_t v, int n) {
    bw.put(v, n);
    cw.put(v, n);
  };
  int diff = q[0] - pred;
  pred = q[0];
  int s = category(diff);
  if (s > 11 || dc.len[s] == 0) return -1;
  bw.put(dc.code[s], dc.len[s]);
  bw.put(magnitude_bits(diff, s), s);
  int nsym = 1;
  if (dc_absolute) {
    dc_removed += (uint64_t)(dc.len[s] + s);
  } else {
    cw.put(dc.code[s], dc.len[s]);
    cw.put(magnitude_bits(diff, s), s);
  }
  int run = 0;
  for (int k = 1; k < 64; ++k) {
    int v = q[kZZ.zz[k]];
    if (v == 0) {
      ++run;
      continue;
    }
    while (run > 15) {
      put(ac.code[0xF0], ac.len[0xF0]);
      run -= 16;
      ++nsym;
    }
    int sz = category(v);
    if (sz > 10) return -1;
    int sym = (run << 4) | sz;
    if (ac.len[sym] == 0) return -1;
    put(ac.code[sym], ac.len[sym]);
    put(magnitude_bits(v, sz), sz);
    run = 0;
    ++nsym;
  }
  if (run > 0) {
    put(ac.code[0x00], ac.len[0x00]);
    ++nsym;
  }
  return nsym;
}

void put_bits(std::vector<uint32_t>& a, uint64_t at, uint32_t v, int n) {
  for (int i = 0; i < n; ++i)
    if ((v >> i) & 1u) a[(at + i) >> 5] |= 1u << ((at + i) & 31);
}

void put16(std::vector<uint8_t>& o, int v) {
  o.push_back((uint8_t)(v >> 8));
  o.push_back((uint8_t)(v & 255));
}

// Entropy-codes quantised coefficient blocks [mcu][du][64] and writes the JFIF container.
void entropy_and_container(Encoded& e, const int16_t* qcoef) {
  const int ndu = e.sampling == 420 ? 6 : 3;
  const int nmcu = e.mcus_x * e.mcus_y;
  HuffEnc enc[4];
  for (int t = 0; t < 4; ++t) enc[t] = encoder_codes(e.huff[t]);
  std::vector<uint8_t> stuffed, cstuffed;
  BitWriter bw{&stuffed, &e.scan};
  Compact& C = e.compact;
  BitWriter cw{&cstuffed, &C.scan};
  const int ngroups = (nmcu + 8) / 9;
  C.abs.assign(ngroups, 0);
  C.rel.assign((size_t)ngroups * 8, 0);
  C.dc.assign(((uint64_t)nmcu * 36 + 31) / 32, 0);
  int pred[3] = {0, 0, 0};
  e.index.resize(nmcu);
  e.du_offsets.assign((size_t)nmcu * (ndu - 1), 0);
  e.symbols.assign((size_t)nmcu, 0);
  for (int m = 0; m < nmcu; ++m) {
    BlockIndex bi;
    bi.bit_offset = (uint32_t)bw.nbits;
    for (int c = 0; c < 3; ++c) bi.dc_pred[c] = (int16_t)pred[c];
    e.index[m] = bi;
    const uint64_t byte = C.scan.size();  // cw is byte aligned here
    if (m % 9 == 0)
      C.abs[m / 9] = (uint32_t)byte;
    else if (byte - C.abs[m / 9] > 65535)
      C.status = -1;
    else
      C.rel[(m / 9) * 8 + m % 9 - 1] = (uint16_t)(byte - C.abs[m / 9]);
    uint32_t nsym = 0;
    for (int d = 0; d < ndu; ++d) {
      int comp = d < ndu - 2 ? 0 : (d == ndu - 2 ? 1 : 2);
      int tab = comp == 0 ? 0 : 1;
      const int16_t* q = qcoef + ((size_t)m * ndu + d) * 64;
      if (d > 0) {
        const uint64_t rel = bw.nbits - bi.bit_offset;
        if (rel > 65535) e.status = -3;
        e.du_offsets[(size_t)m * (ndu - 1) + d - 1] = (uint16_t)rel;
      }
      const bool absolute = d == 0 || comp != 0;  // the first luma DC and the chroma DCs
      if (absolute) {
        if (q[0] < -2048 || q[0] > 2047) C.status = -1;
        put_bits(C.dc, (uint64_t)m * 36 + 12 * comp, (uint32_t)q[0] & 0xFFFu, 12);
      }
      const int ns = encode_du(bw, cw, absolute, C.dc_bits_removed, q, pred[comp], enc[tab * 2], enc[tab * 2 + 1]);
      if (ns < 0) {
        e.status = -2;
        return;
      }
      nsym += (uint32_t)ns;
    }
    e.symbols[m] = (uint16_t)nsym;
    C.pad_bits += cw.nacc ? (uint64_t)(8 - cw.nacc) : 0u;
    cw.flush_ones();
  }
  e.scan_bits = bw.nbits;
  bw.flush_ones();

  std::vector<uint8_t>& o = e.jfif;
  o.clear();
  o.push_back(0xFF); o.push_back(0xD8);  // SOI
  o.push_back(0xFF); o.push_back(0xE0);  // APP0 JFIF
  put16(o, 16);
  const char jf[5] = {'J', 'F', 'I', 'F', 0};
  for (char c : jf) o.push_back((uint8_t)c);
  o.push_back(1); o.push_back(1); o.push_back(0);
  put16(o, 1); put16(o, 1);
  o.push_back(0); o.push_back(0);
  o.push_back(0xFF); o.push_back(0xDB);  // DQT, 8-bit precision, zig-zag order
  put16(o, 2 + 2 * 65);
  for (int t = 0; t < 2; ++t) {
    o.push_back((uint8_t)t);
    for (int k = 0; k < 64; ++k) o.push_back((uint8_t)e.qt[t][kZZ.zz[k]]);
  }
  o.push_back(0xFF); o.push_back(0xC0);  // SOF0
  put16(o, 8 + 3 * 3);
  o.push_back(8);
  put16(o, e.h); put16(o, e.w);
  o.push_back(3);
  o.push_back(1); o.push_back(e.sampling == 420 ? 0x22 : 0x11); o.push_back(0);
  o.push_back(2); o.push_back(0x11); o.push_back(1);
  o.push_back(3); o.push_back(0x11); o.push_back(1);
  const uint8_t tc_th[4] = {0x00, 0x10, 0x01, 0x11};
  for (int t = 0; t < 4; ++t) {  // DHT
    o.push_back(0xFF); o.push_back(0xC4);
    put16(o, 2 + 1 + 16 + e.huff[t].nvals);
    o.push_back(tc_th[t]);
    for (int i = 0; i < 16; ++i) o.push_back(e.huff[t].bits[i]);
    for (int i = 0; i < e.huff[t].nvals; ++i) o.push_back(e.huff[t].vals[i]);
  }
  o.push_back(0xFF); o.push_back(0xDA);  // SOS
  put16(o, 6 + 2 * 3);
  o.push_back(3);
  o.push_back(1); o.push_back(0x00);
  o.push_back(2); o.push_back(0x11);
  o.push_back(3); o.push_back(0x11);
  o.push_back(0); o.push_back(63); o.push_back(0);
  o.insert(o.end(), stuffed.begin(), stuffed.end());
  o.push_back(0xFF); o.push_back(0xD9);  // EOI
}

// Forward DCT of one level-shifted 8x8 block (definition of T.81 A.3.3), double precision.
void fdct8x8(const double* f, double* F) {
  static double cosv[8][8];
  static bool init = false;
  if (!init) {
    for (int x = 0; x < 8; ++x)
      for (int u = 0; u < 8; ++u) cosv[x][u] = std::cos((2 * x + 1) * u * M_PI / 16.0);
    init = true;
  }
  double tmp[64];
  for (int y = 0; y < 8; ++y)
    for (int u = 0; u < 8; ++u) {
      double s = 0;
      for (int x = 0; x < 8; ++x) s += f[y * 8 + x] * cosv[x][u];
      tmp[y * 8 + u] = s;
    }
  for (int v = 0; v < 8; ++v)
    for (int u = 0; u < 8; ++u) {
      double s = 0;
      for (int y = 0; y < 8; ++y) s += tmp[y * 8 + u] * cosv[y][v];
      double cu = u == 0 ? M_SQRT1_2 : 1.0, cv = v == 0 ? M_SQRT1_2 : 1.0;
      F[v * 8 + u] = 0.25 * cu * cv * s;
    }
}

Encoded* encode_rgb(const uint8_t* rgb, int w, int h, int quality, int sampling, bool keep) {
  Encoded* e = new Encoded();
  e->w = w; e->h = h; e->sampling = sampling; e->quality = quality;
  const int mw = sampling == 420 ? 16 : 8;
  e->mcus_x = (w + mw - 1) / mw;
  e->mcus_y = (h + mw - 1) / mw;
  quality_tables(quality, e->qt);
  standard_specs(e->huff);
  const int pw = e->mcus_x * mw, ph = e->mcus_y * mw;
  // Forward colour transform (JFIF), edge-replicated padding to whole MCUs.
  std::vector<uint8_t> Y((size_t)pw * ph), Cb((size_t)pw * ph), Cr((size_t)pw * ph);
  for (int y = 0; y < ph; ++y)
    for (int x = 0; x < pw; ++x) {
      const uint8_t* p = rgb + ((size_t)std::min(y, h - 1) * w + std::min(x, w - 1)) * 3;
      double r = p[0], g = p[1], b = p[2];
      size_t i = (size_t)y * pw + x;
      Y[i] = (uint8_t)clampi((int)std::lround(0.299 * r + 0.587 * g + 0.114 * b), 0, 255);
      Cb[i] = (uint8_t)clampi((int)std::lround(-0.168736 * r - 0.331264 * g + 0.5 * b + 128.0), 0, 255);
      Cr[i] = (uint8_t)clampi((int)std::lround(0.5 * r - 0.418688 * g - 0.081312 * b + 128.0), 0, 255);
    }
  const int ndu = sampling == 420 ? 6 : 3;
  const int nmcu = e->mcus_x * e->mcus_y;
  std::vector<int16_t> q((size_t)nmcu * ndu * 64);
  double f[64], F[64];
  for (int my = 0; my < e->mcus_y; ++my)
    for (int mx = 0; mx < e->mcus_x; ++mx) {
      int m = my * e->mcus_x + mx;
      for (int d = 0; d < ndu; ++d) {
        int comp = d < ndu - 2 ? 0 : (d == ndu - 2 ? 1 : 2);
        for (int yy = 0; yy < 8; ++yy)
          for (int xx = 0; xx < 8; ++xx) {
            double v;
            if (comp == 0) {
              int ox = sampling == 420 ? (d & 1) * 8 : 0, oy = sampling == 420 ? (d >> 1) * 8 : 0;
              v = Y[(size_t)(my * mw + oy + yy) * pw + mx * mw + ox + xx];
            } else {
              const std::vector<uint8_t>& P = comp == 1 ? Cb : Cr;
              if (sampling == 420) {  // 2x2 average of the full-resolution chroma
                int sx = mx * 16 + 2 * xx, sy = my * 16 + 2 * yy;
                int s = P[(size_t)sy * pw + sx] + P[(size_t)sy * pw + sx + 1] + P[(size_t)(sy + 1) * pw + sx] +
                        P[(size_t)(sy + 1) * pw + sx + 1];
                v = (s + 2) >> 2;
              } else {
                v = P[(size_t)(my * 8 + yy) * pw + mx * 8 + xx];
              }
            }
            f[yy * 8 + xx] = v - 128.0;
          }
        fdct8x8(f, F);
        const uint16_t* Q = e->qt[comp == 0 ? 0 : 1];
        int16_t* out = &q[((size_t)m * ndu + d) * 64];
        for (int k = 0; k < 64; ++k) {
          long v = std::lround(F[k] / Q[k]);
          long lim = k == 0 ? 2047 : 1023;
          out[k] = (int16_t)std::max(-lim, std::min(lim, v));
        }
      }
    }
  entropy_and_container(*e, q.data());
  if (keep) e->qcoef.swap(q);
  return e;
}

// ---------------------------------------------------------------------------------------
// G-buffers
// ---------------------------------------------------------------------------------------
struct Vec3 {
  double x, y, z;
};

// Camera ray through pixel centre (px,py) for a camera with yaw/pitch (degrees).
Vec3 camera_ray(double px, double py, int W, int H, double vfov, double yaw, double pitch) {
  double th = std::tan(vfov * M_PI / 360.0);
  double sx = (2.0 * px / W - 1.0) * th * ((double)W / H);
  double sy = (1.0 - 2.0 * py / H) * th;
  Vec3 d{sx, sy, -1.0};
  double cp = std::cos(pitch * M_PI / 180), sp = std::sin(pitch * M_PI / 180);
  Vec3 d1{d.x, d.y * cp - d.z * sp, d.y * sp + d.z * cp};
  double cy = std::cos(yaw * M_PI / 180), sy2 = std::sin(yaw * M_PI / 180);
  return Vec3{d1.x * cy + d1.z * sy2, d1.y, -d1.x * sy2 + d1.z * cy};
}

struct SceneTex {
  int w, h, levels;
};

int mip_from_rho(double rho, int levels) {
  if (!(rho > 0)) return 0;
  int m = (int)std::floor(std::log2(rho) + 0.5);
  return clampi(m, 0, levels - 1);
}

// Gauss-Jordan elimination with partial pivoting on [A | b] (8x8); leaves A diagonal.
bool solve8(double A[8][9]) {
  for (int c = 0; c < 8; ++c) {
    int p = c;
    for (int r = c + 1; r < 8; ++r)
      if (std::fabs(A[r][c]) > std::fabs(A[p][c])) p = r;
    if (std::fabs(A[p][c]) < 1e-12) return false;
    for (int k = 0; k < 9; ++k) std::swap(A[c][k], A[p][k]);
    for (int r = 0; r < 8; ++r)
      if (r != c) {
        double f = A[r][c] / A[c][c];
        for (int k = c; k < 9; ++k) A[r][k] -= f * A[c][k];
      }
  }
  return true;
}

struct Quad {
  double Hinv[9];  // screen (x,y,1) -> unit-square (s,t,w)
  double cx[4], cy[4];
  int tex;
  double rep, cs, sn, ou, ov;
};

bool make_quad(SplitMix64& rng, int W, int H, int ntex, double shift_x, Quad& q) {
  double cx = rng.uniform(0, W), cy = rng.uniform(0, H);
  double size = W * std::exp(rng.uniform(std::log(0.02), std::log(0.40)));
  double a0 = rng.uniform(0, 2 * M_PI);
  for (int i = 0; i < 4; ++i) {
    double a = a0 + i * M_PI / 2 + rng.uniform(-0.12, 0.12);
    double r = 0.5 * size * rng.uniform(0.85, 1.0);
    q.cx[i] = cx + r * std::cos(a) + shift_x;
    q.cy[i] = cy + r * std::sin(a);
  }
  for (int i = 0; i < 4; ++i) {  // strict convexity, counter-clockwise in screen space
    int j = (i + 1) % 4, k = (i + 2) % 4;
    double cr = (q.cx[j] - q.cx[i]) * (q.cy[k] - q.cy[j]) - (q.cy[j] - q.cy[i]) * (q.cx[k] - q.cx[j]);
    if (cr <= 0) return false;
  }
  // Homography from (s,t) in the unit square to the quad corners.
  const double us[4] = {0, 1, 1, 0}, vs[4] = {0, 0, 1, 1};
  double A[8][9];
  for (int i = 0; i < 4; ++i) {
    double s = us[i], t = vs[i], X = q.cx[i], Y = q.cy[i];
    double r0[9] = {s, t, 1, 0, 0, 0, -s * X, -t * X, X};
    double r1[9] = {0, 0, 0, s, t, 1, -s * Y, -t * Y, Y};
    std::memcpy(A[2 * i], r0, sizeof r0);
    std::memcpy(A[2 * i + 1], r1, sizeof r1);
  }
  if (!solve8(A)) return false;
  double Hm[9];
  for (int k = 0; k < 8; ++k) Hm[k] = A[k][8] / A[k][k];  // elimination leaves A diagonal
  Hm[8] = 1.0;
  // inverse by adjugate
  double a = Hm[0], b = Hm[1], c = Hm[2], d = Hm[3], e = Hm[4], f = Hm[5], g = Hm[6], h = Hm[7], i9 = Hm[8];
  double inv[9] = {e * i9 - f * h, c * h - b * i9, b * f - c * e, f * g - d * i9, a * i9 - c * g,
                   c * d - a * f,  d * h - e * g,  b * g - a * h, a * e - b * d};
  std::memcpy(q.Hinv, inv, sizeof inv);
  q.tex = rng.below(ntex);
  q.rep = rng.uniform(0.5, 2.0);
  double phi = rng.uniform(0, 2 * M_PI);
  q.cs = std::cos(phi);
  q.sn = std::sin(phi);
  q.ou = rng.uniform();
  q.ov = rng.uniform();
  return true;
}

void quad_uv(const Quad& q, double x, double y, double& u, double& v) {
  double s = q.Hinv[0] * x + q.Hinv[1] * y + q.Hinv[2];
  double t = q.Hinv[3] * x + q.Hinv[4] * y + q.Hinv[5];
  double w = q.Hinv[6] * x + q.Hinv[7] * y + q.Hinv[8];
  s /= w;
  t /= w;
  u = q.ou + q.rep * (q.cs * s - q.sn * t);
  v = q.ov + q.rep * (q.sn * s + q.cs * t);
}

bool quad_inside(const Quad& q, double x, double y) {
  for (int i = 0; i < 4; ++i) {
    int j = (i + 1) % 4;
    double cr = (q.cx[j] - q.cx[i]) * (y - q.cy[i]) - (q.cy[j] - q.cy[i]) * (x - q.cx[i]);
    if (cr < 0) return false;
  }
  return true;
}

bool ground_uv(double px, double py, int W, int H, double vfov, double yaw, double pitch, const Vec3& cam,
               double& u, double& v, double& wx, double& wz) {
  Vec3 d = camera_ray(px, py, W, H, vfov, yaw, pitch);
  if (d.y >= -1e-9) return false;
  double t = -cam.y / d.y;
  wx = cam.x + t * d.x;
  wz = cam.z + t * d.z;
  if (t > 600.0) return false;
  u = wx / 2.0;
  v = wz / 2.0;
  return true;
}

}  // namespace

// =======================================================================================
// C interface (ctypes)
// =======================================================================================
extern "C" {

uint64_t syn_mix_seed(uint64_t seed, uint64_t a, uint64_t b) { return mix_seed(seed, a, b); }


void syn_texture(uint64_t seed, int w, int h, uint8_t* rgb) { gen_texture(seed, w, h, rgb); }

void syn_mip_down(const uint8_t* src, int w, int h, uint8_t* dst) { mip_down(src, w, h, dst); }

void syn_quality_tables(int quality, uint16_t* qt /*[2][64]*/) {
  quality_tables(quality, reinterpret_cast<uint16_t(*)[64]>(qt));
}

// Standard Huffman specs as bits[4][16], vals[4][256], nvals[4]
// (order: DC luma, AC luma, DC chroma, AC chroma).
void syn_standard_huffman(uint8_t* bits, uint8_t* vals, int* nvals) {
  HuffSpec s[4];
  standard_specs(s);
  for (int t = 0; t < 4; ++t) {
    std::memcpy(bits + 16 * t, s[t].bits, 16);
    std::memset(vals + 256 * t, 0, 256);
    std::memcpy(vals + 256 * t, s[t].vals, s[t].nvals);
    nvals[t] = s[t].nvals;
  }
}

// Encoder-side code table for one spec: code[256], len[256] indexed by symbol.
void syn_huffman_codes(const uint8_t* bits, const uint8_t* vals, uint16_t* code, uint8_t* len) {
  HuffSpec s{};
  std::memcpy(s.bits, bits, 16);
  int n = 0;
  for (int i = 0; i < 16; ++i) n += bits[i];
  std::memcpy(s.vals, vals, n);
  s.nvals = n;
  HuffEnc e = encoder_codes(s);
  std::memcpy(code, e.code, sizeof e.code);
  std::memcpy(len, e.len, sizeof e.len);
}

void syn_zigzag(int* out) { std::memcpy(out, kZZ.zz, sizeof kZZ.zz); }

void* syn_jpeg_encode_rgb(const uint8_t* rgb, int w, int h, int quality, int sampling, int keep_coefs) {
  if (w <= 0 || h <= 0 || (sampling != 420 && sampling != 444)) return nullptr;
  return encode_rgb(rgb, w, h, quality, sampling, keep_coefs != 0);
}

// Entropy-codes given quantised blocks [mcus_y*mcus_x][ndu][64] (natural order) with the
// standard tables, for round-trip tests; width/height are the MCU-aligned sizes.
void* syn_jpeg_encode_coefs(const int16_t* qcoef, int mcus_x, int mcus_y, int sampling, int quality) {
  Encoded* e = new Encoded();
  const int mw = sampling == 420 ? 16 : 8;
  e->sampling = sampling;
  e->mcus_x = mcus_x;
  e->mcus_y = mcus_y;
  e->w = mcus_x * mw;
  e->h = mcus_y * mw;
  e->quality = quality;
  quality_tables(quality, e->qt);
  standard_specs(e->huff);
  entropy_and_container(*e, qcoef);
  return e;
}

// info: [status, w, h, sampling, mcus_x, mcus_y, jfif_bytes, scan_bytes, scan_bits, n_index]
void syn_jpeg_info(void* hnd, int64_t* info) {
  Encoded* e = static_cast<Encoded*>(hnd);
  info[0] = e->status;
  info[1] = e->w;
  info[2] = e->h;
  info[3] = e->sampling;
  info[4] = e->mcus_x;
  info[5] = e->mcus_y;
  info[6] = (int64_t)e->jfif.size();
  info[7] = (int64_t)e->scan.size();
  info[8] = (int64_t)e->scan_bits;
  info[9] = (int64_t)e->index.size();
}

void syn_jpeg_copy(void* hnd, uint8_t* jfif, uint8_t* scan, void* index, uint16_t* qt, uint8_t* bits,
                   uint8_t* vals, int16_t* qcoef) {
  Encoded* e = static_cast<Encoded*>(hnd);
  if (jfif) std::memcpy(jfif, e->jfif.data(), e->jfif.size());
  if (scan) std::memcpy(scan, e->scan.data(), e->scan.size());
  if (index) std::memcpy(index, e->index.data(), e->index.size() * sizeof(BlockIndex));
  if (qt) std::memcpy(qt, e->qt, sizeof e->qt);
  if (bits && vals)
    for (int t = 0; t < 4; ++t) {
      std::memcpy(bits + 16 * t, e->huff[t].bits, 16);
      std::memset(vals + 256 * t, 0, 256);
      std::memcpy(vals + 256 * t, e->huff[t].vals, e->huff[t].nvals);
    }
  if (qcoef && !e->qcoef.empty()) std::memcpy(qcoef, e->qcoef.data(), e->qcoef.size() * sizeof(int16_t));
}

// Compact form sizes: [status, scan_bytes, n_abs, n_rel, n_dc_words, dc_bits_removed, pad_bits]
void syn_jpeg_compact_info(void* hnd, int64_t* info) {
  const Compact& C = static_cast<Encoded*>(hnd)->compact;
  info[0] = C.status;
  info[1] = (int64_t)C.scan.size();
  info[2] = (int64_t)C.abs.size();
  info[3] = (int64_t)C.rel.size();
  info[4] = (int64_t)C.dc.size();
  info[5] = (int64_t)C.dc_bits_removed;
  info[6] = (int64_t)C.pad_bits;
}

void syn_jpeg_compact_copy(void* hnd, uint8_t* scan, uint32_t* abs, uint16_t* rel, uint32_t* dc) {
  const Compact& C = static_cast<Encoded*>(hnd)->compact;
  std::memcpy(scan, C.scan.data(), C.scan.size());
  std::memcpy(abs, C.abs.data(), C.abs.size() * 4);
  std::memcpy(rel, C.rel.data(), C.rel.size() * 2);
  std::memcpy(dc, C.dc.data(), C.dc.size() * 4);
}

// Data-unit start offsets: [mcu][ndu - 1] uint16 (bits from the MCU's first bit).
int64_t syn_jpeg_du_count(void* hnd) { return (int64_t) static_cast<Encoded*>(hnd)->du_offsets.size(); }
void syn_jpeg_symbols_copy(void* hnd, uint16_t* out) {
  const Encoded* e = static_cast<Encoded*>(hnd);
  std::memcpy(out, e->symbols.data(), e->symbols.size() * 2);
}
void syn_jpeg_du_copy(void* hnd, uint16_t* out) {
  const Encoded* e = static_cast<Encoded*>(hnd);
  std::memcpy(out, e->du_offsets.data(), e->du_offsets.size() * 2);
}

void syn_jpeg_free(void* hnd) { delete static_cast<Encoded*>(hnd); }

// Affine G-buffer: uv = 0.5 + R(angle) * scale * ((x+1/2)/W - 1/2, (y+1/2)/H - 1/2),
// one texture id, mip 0.
void syn_gbuffer_affine(int W, int H, double angle_deg, double scale, int tex, float* uv, uint16_t* tex_id,
                        uint8_t* mip) {
  double c = std::cos(angle_deg * M_PI / 180), s = std::sin(angle_deg * M_PI / 180);
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      double a = (x + 0.5) / W - 0.5, b = (y + 0.5) / H - 0.5;
      size_t p = (size_t)y * W + x;
      uv[2 * p] = (float)(0.5 + scale * (c * a - s * b));
      uv[2 * p + 1] = (float)(0.5 + scale * (s * a + c * b));
      tex_id[p] = (uint16_t)tex;
      mip[p] = 0;
    }
}

// Perspective ground plane (y = 0, uv = world (x,z)/2 + a seeded offset per 2 m cell, one
// texture per 2 m cell, so each cell shows one texture period) seen
// from a camera at cam (height cam_y) with yaw/pitch/vfov in degrees, then nquads random
// convex screen-space quads (drawn in order) with projective uv maps. Sky pixels get
// tex_id 0xFFFF. The mip level of each pixel is clamp(floor(log2(rho) + 1/2), 0, L-1) with
// rho the larger texel-space length of the uv derivatives along screen x and y.
// When use_mips is 0 every pixel gets level 0. Quads are drawn in a resolution-independent
// reference frame (1000 units high, 1000*W/H wide), so views of one pose at different
// resolutions see the same quads; quad_shift_frac shifts them by that fraction of the
// width (stereo disparity).
void syn_gbuffer_scene(uint64_t seed, int W, int H, double cam_x, double cam_y, double cam_z, double yaw,
                       double pitch, double vfov, int nquads, uint64_t quad_seed, double quad_shift_frac,
                       int ntex, const int* tex_w, const int* tex_h, const int* tex_levels, int use_mips,
                       float* uv, uint16_t* tex_id, uint8_t* mip) {
  Vec3 cam{cam_x, cam_y, cam_z};
  const uint64_t cell_seed = mix_seed(seed, 7, 0);
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      size_t p = (size_t)py * W + px;
      double u, v, wx, wz;
      if (!ground_uv(px + 0.5, py + 0.5, W, H, vfov, yaw, pitch, cam, u, v, wx, wz)) {
        uv[2 * p] = 0.f;
        uv[2 * p + 1] = 0.f;
        tex_id[p] = 0xFFFF;
        mip[p] = 0;
        continue;
      }
      int64_t cx = (int64_t)std::floor(wx / 2.0), cz = (int64_t)std::floor(wz / 2.0);
      uint64_t hsh = mix_seed(cell_seed, (uint64_t)cx, (uint64_t)cz);
      int t = (int)(hsh % (uint64_t)ntex);
      // per-cell uv offset: cells that share a texture show different parts of it
      double ou = (double)((hsh >> 16) & 0xFFFF) / 65536.0, ov = (double)((hsh >> 32) & 0xFFFF) / 65536.0;
      u += ou;
      v += ov;
      uv[2 * p] = (float)u;
      uv[2 * p + 1] = (float)v;
      tex_id[p] = (uint16_t)t;
      int lvl = 0;
      if (use_mips) {
        double u0, v0, u1, v1, u2, v2, u3, v3, a, b;
        bool ok = ground_uv(px, py + 0.5, W, H, vfov, yaw, pitch, cam, u0, v0, a, b) &&
                  ground_uv(px + 1.0, py + 0.5, W, H, vfov, yaw, pitch, cam, u1, v1, a, b) &&
                  ground_uv(px + 0.5, py, W, H, vfov, yaw, pitch, cam, u2, v2, a, b) &&
                  ground_uv(px + 0.5, py + 1.0, W, H, vfov, yaw, pitch, cam, u3, v3, a, b);
        if (!ok) {
          lvl = tex_levels[t] - 1;
        } else {
          double rx = std::hypot((u1 - u0) * tex_w[t], (v1 - v0) * tex_h[t]);
          double ry = std::hypot((u3 - u2) * tex_w[t], (v3 - v2) * tex_h[t]);
          lvl = mip_from_rho(std::max(rx, ry), tex_levels[t]);
        }
      }
      mip[p] = (uint8_t)lvl;
    }
  const double Hn = 1000.0, Wn = 1000.0 * W / H;
  const double kx = Wn / W, ky = Hn / H;  // reference units per pixel
  const double shift = quad_shift_frac * Wn;
  SplitMix64 rng(quad_seed);
  for (int n = 0; n < nquads; ++n) {
    Quad q;
    int tries = 0;
    while (!make_quad(rng, (int)std::lround(Wn), (int)Hn, ntex, 0.0, q) && ++tries < 100) {
    }
    if (tries >= 100) continue;
    double minx = 1e30, maxx = -1e30, miny = 1e30, maxy = -1e30;
    for (int i = 0; i < 4; ++i) {
      minx = std::min(minx, (q.cx[i] + shift) / kx);
      maxx = std::max(maxx, (q.cx[i] + shift) / kx);
      miny = std::min(miny, q.cy[i] / ky);
      maxy = std::max(maxy, q.cy[i] / ky);
    }
    int x0 = std::max(0, (int)std::floor(minx) - 1), x1 = std::min(W - 1, (int)std::ceil(maxx) + 1);
    int y0 = std::max(0, (int)std::floor(miny) - 1), y1 = std::min(H - 1, (int)std::ceil(maxy) + 1);
    const int t = q.tex;
    for (int py = y0; py <= y1; ++py)
      for (int px = x0; px <= x1; ++px) {
        double qx = (px + 0.5) * kx - shift, qy = (py + 0.5) * ky;
        if (!quad_inside(q, qx, qy)) continue;
        size_t p = (size_t)py * W + px;
        double u, v;
        quad_uv(q, qx, qy, u, v);
        uv[2 * p] = (float)u;
        uv[2 * p + 1] = (float)v;
        tex_id[p] = (uint16_t)t;
        int lvl = 0;
        if (use_mips) {
          double u0, v0, u1, v1, u2, v2, u3, v3;
          quad_uv(q, qx - 0.5 * kx, qy, u0, v0);
          quad_uv(q, qx + 0.5 * kx, qy, u1, v1);
          quad_uv(q, qx, qy - 0.5 * ky, u2, v2);
          quad_uv(q, qx, qy + 0.5 * ky, u3, v3);
          double rx = std::hypot((u1 - u0) * tex_w[t], (v1 - v0) * tex_h[t]);
          double ry = std::hypot((u3 - u2) * tex_w[t], (v3 - v2) * tex_h[t]);
          lvl = mip_from_rho(std::max(rx, ry), tex_levels[t]);
        }
        mip[p] = (uint8_t)lvl;
      }
  }
}

// The quads of syn_gbuffer_scene (same seed, same draws, same order) as its reference frame
// (1000 units high, 1000 * W / H wide) sees them, for renderers of the same scene. Per quad,
// 22 doubles: corners cx[4], cy[4], the inverse homography Hinv[9] (reference (x, y, 1) ->
// unit square (s, t, w)), rep, cos phi, sin phi, ou, ov; and its texture in tex[]. Returns the
// number of quads written (quads that failed 100 draws are skipped, as there).
int syn_scene_quads(int W, int H, int nquads, uint64_t quad_seed, int ntex, double* out, int* tex) {
  const double Hn = 1000.0, Wn = 1000.0 * W / H;
  SplitMix64 rng(quad_seed);
  int k = 0;
  for (int n = 0; n < nquads; ++n) {
    Quad q;
    int tries = 0;
    while (!make_quad(rng, (int)std::lround(Wn), (int)Hn, ntex, 0.0, q) && ++tries < 100) {
    }
    if (tries >= 100) continue;
    double* o = out + 22 * k;
    for (int i = 0; i < 4; ++i) {
      o[i] = q.cx[i];
      o[4 + i] = q.cy[i];
    }
    for (int i = 0; i < 9; ++i) o[8 + i] = q.Hinv[i];
    o[17] = q.rep;
    o[18] = q.cs;
    o[19] = q.sn;
    o[20] = q.ou;
    o[21] = q.ov;
    tex[k] = q.tex;
    ++k;
  }
  return k;
}

// Smooth seeded float image [H][W][3] in [0,255] (value noise), used as a target frame.
void syn_noise_image(uint64_t seed, int W, int H, float* out) {
  std::vector<uint8_t> rgb((size_t)W * H * 3);
  gen_texture(seed, W, H, rgb.data());
  for (size_t i = 0; i < rgb.size(); ++i) out[i] = (float)rgb[i];
}

}  // extern "C"
