"""Oracle pins for the reduced-resolution decode (the mip alternative of Sec. 7: a lower
resolution from a subset of the AC coefficients, or from the DC alone).

A data unit decoded at N x N (N = 8, 4, 2, 1) takes its N x N lowest frequencies through the
N-point IDCT, scaled so that the result is the block at 1/(8/N) resolution. Pinned against:
- scipy's orthonormal inverse DCT of the N x N corner times N/8 (within 1 LSB of rounding);
- N = 1: the mean of the full 8 x 8 decode (exact in exact arithmetic);
- whole tiles of a grey texture (chroma flat at 128, so R = G = B = Y) against scipy on the
  sequential decoder's coefficients, which fixes the data-unit placement in the tile;
- DC-only tiles against 8 x 8 box means of the full-resolution image.
"""

import numpy as np
import pytest

import oracle
import synth

idctn = pytest.importorskip("scipy.fft").idctn


def _blocks(seed, n=3000):
    rng = np.random.default_rng(seed)
    d = rng.integers(-200, 200, (n, 64)).astype(np.int32)
    d[:, 0] = rng.integers(-1000, 1000, n)
    d[rng.random((n, 64)) < 0.6] = 0  # mostly sparse, as quantised blocks are
    return d


@pytest.mark.parametrize("n", [8, 4, 2, 1])
def test_reduced_idct_is_the_scaled_orthonormal_idct(n):
    d = _blocks(n)
    got = oracle.idct_pixels_n(d, n).astype(np.float64)
    F = d.reshape(-1, 8, 8)[:, :n, :n].astype(np.float64) * (n / 8)
    ref = np.clip(idctn(F, axes=(1, 2), norm="ortho") + 128, 0, 255).reshape(-1, n * n)
    assert np.abs(got - ref).max() < 1.0
    if n == 8:  # the full-size path is the existing decode spec
        np.testing.assert_array_equal(got, oracle.idct_pixels(d).astype(np.float64))


def test_dc_only_is_the_block_mean():
    d = _blocks(11)
    d[:, 1:] //= 4  # keep the full decode away from 0 and 255, where clamping moves the mean
    full = oracle.idct_pixels(d).astype(np.float64)
    keep = (full.min(axis=1) > 0) & (full.max(axis=1) < 255)
    assert keep.sum() > 1000
    dc = oracle.idct_pixels_n(d, 1)[:, 0].astype(np.float64)
    assert np.abs(dc[keep] - full[keep].mean(axis=1)).max() <= 1.0


def _grey_texture(seed, w, h):
    rgb = synth.texture(seed, w, h)
    g = rgb.mean(axis=2).astype(np.uint8)
    return np.repeat(g[..., None], 3, axis=2)


@pytest.mark.parametrize("sampling", [420, 444])
@pytest.mark.parametrize("r", [1, 2, 3])
def test_grey_tiles_match_scipy(sampling, r):
    w, h = 80, 48
    e = synth.encode(_grey_texture(5 + r, w, h), 85, sampling)
    o = oracle.TexSet()
    o.add(0, 0, e)
    o.add_reduced(0, 0, r, 1)
    dec = oracle.Decoded(e.jfif)
    assert (dec.qcoef[:, -2:, :] == 0).all()  # flat chroma
    n = 8 >> r
    mw = (16 if sampling == 420 else 8) >> r
    ydus = 4 if sampling == 420 else 1
    qt = e.qt[0].astype(np.float64)  # natural order
    for m in range(e.nmcu):
        tile = o.decode_mcu(0, 1, m, mw)
        assert (tile[..., 0] == tile[..., 1]).all() and (tile[..., 0] == tile[..., 2]).all()
        for du in range(ydus):
            F = (dec.qcoef[m, du].astype(np.float64) * qt).reshape(8, 8)[:n, :n] * (n / 8)
            ref = np.clip(idctn(F, norm="ortho") + 128, 0, 255)
            by, bx = (du // 2) * n, (du % 2) * n
            got = tile[by:by + n, bx:bx + n, 0].astype(np.float64)
            assert np.abs(got - ref).max() < 1.0, (m, du)


@pytest.mark.parametrize("sampling", [420, 444])
def test_dc_only_level_is_the_box_downsample(sampling):
    """At 4:4:4 every channel of a 1/8 texel is its 8x8 block's mean. At 4:2:0 the chroma is
    one value per 16x16 MCU, so the check uses a grey texture there."""
    w, h = 96, 64
    rgb = synth.texture(23, w, h) if sampling == 444 else _grey_texture(23, w, h)
    e = synth.encode(rgb, 95, sampling)
    o = oracle.TexSet()
    o.add(0, 0, e)
    o.add_reduced(0, 0, 3, 3)
    full = oracle.Decoded(e.jfif).rgba[..., :3].astype(np.float64)
    box = full.reshape(h // 8, 8, w // 8, 8, 3).mean(axis=(1, 3))
    # one pixel at every texel centre of the 1/8 level
    lw, lh = w // 8, h // 8
    xs, ys = np.meshgrid(np.arange(lw), np.arange(lh))
    uv = np.stack([(xs + 0.5) / lw, (ys + 0.5) / lh], -1).astype(np.float32)
    out = o.colorize(uv, np.zeros((lh, lw), np.uint16), np.full((lh, lw), 3, np.uint8), 0)[..., :3]
    d = np.abs(out.astype(np.float64) - box)
    # colour conversion and 4:2:0 chroma are affine in the means up to rounding and clamping
    assert np.median(d) <= 1.0 and np.percentile(d, 99) <= 4.0


def test_reduced_level_geometry():
    e = synth.encode(synth.texture(3, 33, 17), 70, 420)  # 3 x 2 MCUs
    o = oracle.TexSet()
    o.add(0, 0, e)
    g = o.add_reduced(0, 0, 1, 1)
    assert g == 6 and o.nmcu[(0, 1)] == 6 and o.total == 12
    with pytest.raises(ValueError):
        o.add_reduced(0, 1, 1, 2)  # the source must be a stored level
    with pytest.raises(ValueError):
        o.add_reduced(0, 0, 4, 2)
    # the 16 x 8 level maps texel (x, y) to MCU (x // 8, y // 8) of the source's 3 x 2 grid:
    # MCUs 0 and 1 (the source's third column and second row hold texels past 16 x 8)
    flags = o.mark(synth.GBuffer(16, 8, *_texel_grid(16, 8, 1)), 0)
    assert np.nonzero(flags)[0].tolist() == [6, 7]


def _texel_grid(w, h, level):
    xs, ys = np.meshgrid(np.arange(w), np.arange(h))
    uv = np.stack([(xs + 0.5) / w, (ys + 0.5) / h], -1).astype(np.float32)
    return uv, np.zeros((h, w), np.uint16), np.full((h, w), level, np.uint8)
