"""Oracle pins for the entropy decode and the random-access index.

* lossless round trip: the generator's encoder -> the oracle's decoder returns the
  quantised coefficients exactly, including the extremes of 8-bit baseline;
* brute force: a third decoder (exhaustive prefix match over the code table, written
  here) agrees with the oracle on every MCU of tiny images;
* random access (Sec. 4.3 with the Sec. 5.1 index) equals sequential decode for every
  MCU, and the oracle's own index equals the generator's;
* decoded quality rises with the JPEG quality setting.
"""

import numpy as np
import pytest

import oracle
import synth


def _random_blocks(rng, nmcu, ndu, density):
    q = np.zeros((nmcu, ndu, 64), np.int16)
    mask = rng.random((nmcu, ndu, 64)) < density
    vals = rng.integers(-1023, 1024, (nmcu, ndu, 64))
    q[mask] = vals[mask]
    # DC: keep |diff| <= 2047 along each component's chain
    q[:, :, 0] = rng.integers(-1000, 1001, (nmcu, ndu))
    return q


@pytest.mark.parametrize("sampling", [420, 444])
def test_roundtrip_adversarial_blocks(rng, sampling):
    ndu = 6 if sampling == 420 else 3
    mx, my = 5, 3
    n = mx * my
    q = _random_blocks(rng, n, ndu, 0.3)
    zz = oracle.zigzag()
    q[0, 0, :] = 0                                 # all-zero block
    q[1, 0, zz[63]] = 1023                         # last coefficient, no EOB
    q[1, 0, zz[1:63]] = 0
    q[2, 0, zz[1:]] = 0
    q[2, 0, zz[40]] = -1023                        # a run longer than 16 (ZRL) then a value
    q[3, 0, zz[1:]] = 0
    q[3, 0, zz[17]] = 1
    q[3, 0, zz[34]] = -1                           # two ZRLs in one block
    q[3, 0, zz[63]] = 5
    q[4, :, 1:] = 1023 * np.sign(rng.standard_normal((ndu, 63))).astype(np.int16)  # long 16-bit codes
    q[5, 0, 0] = 1023
    q[6, 0, 0] = -1024                             # DC diff of -2047
    q[7, 0, 0] = 1023                              # and +2047
    enc = synth.encode_coefs(q, mx, my, sampling, quality=75)
    dec = oracle.Decoded(enc.jfif)
    assert dec.coded_bits == enc.scan_bits
    np.testing.assert_array_equal(dec.qcoef, q.astype(np.int32))
    np.testing.assert_array_equal(dec.index, enc.index)


def _bitstring(scan: np.ndarray) -> str:
    return "".join(format(int(b), "08b") for b in scan)


def _brute_force_decode(enc):
    """Exhaustive prefix match: at each symbol try every (code, length) of the table."""
    bits = _bitstring(enc.scan)
    tabs = []
    for t in range(4):
        code, ln = synth.encoder_codes(enc.huff_bits[t], enc.huff_vals[t])
        tabs.append([(format(int(code[s]), f"0{int(ln[s])}b"), s) for s in range(256) if ln[s]])
    zz = oracle.zigzag()
    pos = 0

    def symbol(tab):
        nonlocal pos
        hits = [(c, s) for c, s in tab if bits.startswith(c, pos)]
        assert len(hits) == 1
        pos += len(hits[0][0])
        return hits[0][1]

    def value(s):
        nonlocal pos
        if s == 0:
            return 0
        v = int(bits[pos:pos + s], 2)
        pos += s
        return v if v >= (1 << (s - 1)) else v - (1 << s) + 1

    ndu = enc.ndu
    out = np.zeros((enc.nmcu, ndu, 64), np.int32)
    pred = [0, 0, 0]
    for m in range(enc.nmcu):
        for d in range(ndu):
            comp = 0 if d < ndu - 2 else (1 if d == ndu - 2 else 2)
            tb = 0 if comp == 0 else 1
            pred[comp] += value(symbol(tabs[2 * tb]))
            out[m, d, 0] = pred[comp]
            k = 1
            while k < 64:
                rs = symbol(tabs[2 * tb + 1])
                r, s = rs >> 4, rs & 15
                if s == 0:
                    if r == 15:
                        k += 16
                        continue
                    break
                k += r
                out[m, d, zz[k]] = value(s)
                k += 1
    return out, pos


@pytest.mark.parametrize("size,sampling", [((16, 16), 420), ((24, 40), 420), ((48, 32), 444), ((33, 17), 420)])
def test_brute_force_prefix_decoder_agrees(size, sampling):
    w, h = size
    rgb = synth.texture(synth.mix_seed(7, w, h), w, h)
    enc = synth.encode(rgb, 85, sampling)
    ref, nbits = _brute_force_decode(enc)
    dec = oracle.Decoded(enc.jfif)
    assert dec.coded_bits == nbits == enc.scan_bits
    np.testing.assert_array_equal(dec.qcoef, ref)


def _sequential_tiles(dec, mw):
    """MCU tiles cut from the sequentially decoded RGBA image (padded MCUs are partial)."""
    H, W = dec.height, dec.width
    for m in range(dec.mcus_x * dec.mcus_y):
        mx, my = m % dec.mcus_x, m // dec.mcus_x
        yield m, dec.rgba[my * mw:min(H, my * mw + mw), mx * mw:min(W, mx * mw + mw)]


@pytest.mark.parametrize("size,sampling,q", [((512, 512), 420, 80), ((96, 64), 444, 95), ((37, 23), 420, 50),
                                             ((1, 1), 420, 90), ((9, 1), 444, 70)])
def test_random_access_equals_sequential(size, sampling, q):
    w, h = size
    rgb = synth.texture(synth.mix_seed(11, w, h), w, h)
    enc = synth.encode(rgb, q, sampling)
    dec = oracle.Decoded(enc.jfif)
    np.testing.assert_array_equal(dec.index, enc.index)
    np.testing.assert_array_equal(dec.scan, enc.scan)
    assert dec.coded_bits == enc.scan_bits
    ts = oracle.TexSet()
    ts.add(0, 0, enc)
    mw = 16 if sampling == 420 else 8
    for m, ref in _sequential_tiles(dec, mw):
        tile = ts.decode_mcu(0, 0, m, mw)
        np.testing.assert_array_equal(tile[:ref.shape[0], :ref.shape[1]], ref)


def test_random_access_full_mip_chain():
    rgb = synth.texture(5, 200, 120)
    chain = synth.mip_chain(rgb)
    assert chain[-1].shape[:2] == (1, 1)
    ts = oracle.TexSet()
    for l, lv in enumerate(chain):
        enc = synth.encode(lv, 75, 420)
        ts.add(3, l, enc)
        dec = oracle.Decoded(enc.jfif)
        for m, ref in _sequential_tiles(dec, 16):
            tile = ts.decode_mcu(3, l, m, 16)
            np.testing.assert_array_equal(tile[:ref.shape[0], :ref.shape[1]], ref)


def _psnr(a, b):
    mse = ((a.astype(float) - b.astype(float)) ** 2).mean()
    return 10 * np.log10(255 ** 2 / mse)


def test_quality_monotone():
    rgb = synth.texture(synth.mix_seed(synth.SEED_BASE + 1, 100, 0), 512, 512)
    psnr = [_psnr(oracle.Decoded(synth.encode(rgb, q, 420).jfif).rgba[..., :3], rgb) for q in (30, 50, 80, 95)]
    assert all(a < b for a, b in zip(psnr, psnr[1:])), psnr
    # grey input: Cb = Cr = 128, so only the luma IDCT path is measured; a transposed or
    # mis-scaled IDCT would cost tens of dB here
    g = np.repeat(rgb.mean(axis=2, keepdims=True).round().astype(np.uint8), 3, axis=2)
    grey = {q: _psnr(oracle.Decoded(synth.encode(g, q, 420).jfif).rgba[..., :3], g) for q in (50, 95, 100)}
    assert grey[50] > 40 and grey[95] > 50 and grey[100] > 58, grey


def test_corrupt_stream_is_rejected():
    rgb = synth.texture(3, 64, 64)
    enc = synth.encode(rgb, 80, 420)
    ts = oracle.TexSet()
    bad = synth.Encoded(**{k: getattr(enc, k) for k in enc.__dataclass_fields__})
    bad.scan = np.full_like(enc.scan, 0xFF)  # all-ones matches no code
    ts.add(0, 0, bad)
    with pytest.raises(ValueError):
        ts.decode_mcu(0, 0, 0, 16)
