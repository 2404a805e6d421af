"""Oracle pins for Mark / Compact / Resolve (Sec. 4.2, Sec. 4.4, Sec. 4.6) and the
paper's closed-form MCU geometry (Sec. 3.1, Sec. 5.2, Sec. 5.3).

* the set of marked MCUs equals a brute-force set computed here with numpy (fp32 index
  arithmetic, the MCU formula of Sec. 4.2 with ceil for partial MCUs);
* compact: ascending, unique, count = popcount(flags);
* nearest colourise equals indexing the sequentially decoded texture (independent of
  the random-access decode and of the needed set);
* bilinear colourise is within 1 of an FP64 bilinear of the full decoded texture.
"""

import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden():
    with open(os.path.join(GOLDEN, "paper_constants.json")) as f:
        return {k: v["value"] for k, v in json.load(f).items() if not k.startswith("_")}


def test_paper_mcu_geometry():
    g = _golden()
    mw = g["mcu_px_420"]
    n = (4096 // mw) * (4096 // mw)
    assert n == g["mcus_4096_420"]
    assert n * g["dus_per_mcu_420"] == g["dus_4096_420"]
    assert g["dus_per_mcu_420"] * 63 == g["acs_per_mcu"]
    # the paper's side-table arithmetic (Sec. 5.3; it prints 160/9 truncated to 17.777)
    trunc3 = lambda x: int(x * 1000) / 1000
    assert trunc3((32 + 16 * 8) / 9) == g["index_bits_per_mcu"]
    assert 3 * 12 == g["dc_bits_per_mcu"]
    assert trunc3((32 + 16 * 8) / 9 + 3 * 12) == g["overhead_bits_per_mcu"]
    assert round(g["overhead_bits_per_mcu"] / 256, 2) == g["overhead_bpp"]
    kb = g["key_bits"]
    assert kb["mcu"] + kb["tex"] + kb["mip"] == 32
    assert (1 << kb["mcu"]) == n  # 16 bits cover one 4k texture's MCUs
    # the generator's encoder agrees with the closed form
    e = synth.encode_coefs(np.zeros((4, 6, 64), np.int16), 2, 2, 420)
    assert e.nmcu == 4 and e.width == 32


def _taps_np(u, v, w, h, filt, mw=16):
    """Texel taps with fp32 index arithmetic, written with numpy. Filter 2 (bilinear clamped
    to one MCU, Sec. 4.4) moves, per axis, a tap outside the nearest texel's MCU onto the
    nearest texel's row or column."""
    w32 = np.float32(w)
    h32 = np.float32(h)
    uw = (u.astype(np.float32) * w32).astype(np.float32)
    vh = (v.astype(np.float32) * h32).astype(np.float32)
    if filt == 0:
        x = np.mod(np.floor(uw).astype(np.int64), w)
        y = np.mod(np.floor(vh).astype(np.int64), h)
        return [(x, y)], None, None
    xs = (uw - np.float32(0.5)).astype(np.float32)
    ys = (vh - np.float32(0.5)).astype(np.float32)
    x0 = np.floor(xs)
    y0 = np.floor(ys)
    fx = (xs - x0).astype(np.float64)
    fy = (ys - y0).astype(np.float64)
    x0 = x0.astype(np.int64)
    y0 = y0.astype(np.int64)
    xa, xb = np.mod(x0, w), np.mod(x0 + 1, w)
    ya, yb = np.mod(y0, h), np.mod(y0 + 1, h)
    if filt == 2:
        (nx, ny), = _taps_np(u, v, w, h, 0)[0]
        xa, xb = [np.where(t // mw == nx // mw, t, nx) for t in (xa, xb)]
        ya, yb = [np.where(t // mw == ny // mw, t, ny) for t in (ya, yb)]
    return [(xa, ya), (xb, ya), (xa, yb), (xb, yb)], fx, fy


def _brute_marks(ts, gb, filt):
    keys = set()
    valid = gb.tex_id != 0xFFFF
    tex = gb.tex_id[valid]
    mip = gb.mip[valid]
    u = gb.uv[..., 0][valid]
    v = gb.uv[..., 1][valid]
    gid = 0
    for t, l, e in ts.uploads():
        sel = (tex == t) & (mip == l)
        if sel.any():
            mw = 16 if e.sampling == 420 else 8
            for x, y in _taps_np(u[sel], v[sel], e.width, e.height, filt, mw)[0]:
                keys |= set((gid + x // mw + (y // mw) * e.mcus_x).tolist())
        gid += e.nmcu
    return keys


def _small_scene(seed=3, W=320, H=180, nq=30):
    sizes = [(64, 64), (128, 128), (256, 256), (96, 48)]
    ts = synth.make_texture_set(seed, sizes, [60, 75, 90, 50], [420, 420, 444, 420])
    gb = synth.gbuffer_scene(seed, W, H, ts.sizes, ts.nlevels, synth.Pose(quad_seed=seed), nquads=nq)
    return ts, gb


@pytest.mark.parametrize("filt", [0, 1, 2])
def test_mark_equals_brute_force_small_scene(filt):
    ts, gb = synth.small_scene()
    o = oracle.texset_from(ts)
    flags = o.mark(gb, filt)
    assert set(np.nonzero(flags)[0].tolist()) == _brute_marks(ts, gb, filt)


@pytest.mark.parametrize("filt", [0, 1, 2])
def test_mark_equals_brute_force_scene(filt):
    ts, gb = _small_scene()
    o = oracle.texset_from(ts)
    flags = o.mark(gb, filt)
    ref = _brute_marks(ts, gb, filt)
    assert len(ref) > 50
    assert set(np.nonzero(flags)[0].tolist()) == ref
    work = o.compact(flags)
    assert work.size == int(flags.sum())
    assert (np.diff(work.astype(np.int64)) > 0).all()


def _full_textures(ts):
    return {(t, l): oracle.Decoded(e.jfif).rgba for t, l, e in ts.uploads()}


@pytest.mark.parametrize("filt", [0, 1, 2])
def test_colorize_equals_full_decode(filt):
    ts, gb = _small_scene(seed=5)
    o = oracle.texset_from(ts)
    out = o.colorize(gb.uv, gb.tex_id, gb.mip, filt)
    full = _full_textures(ts)
    mws = {(t, l): 16 if e.sampling == 420 else 8 for t, l, e in ts.uploads()}
    ref = np.zeros(gb.tex_id.shape + (3,), np.float64)
    valid = gb.tex_id != 0xFFFF
    for (t, l), img in full.items():
        sel = valid & (gb.tex_id == t) & (gb.mip == l)
        if not sel.any():
            continue
        h, w = img.shape[:2]
        mw = mws[(t, l)]
        taps, fx, fy = _taps_np(gb.uv[..., 0][sel], gb.uv[..., 1][sel], w, h, filt, mw)
        c = [img[y, x, :3].astype(np.float64) for x, y in taps]
        if filt == 0:
            ref[sel] = c[0]
        else:
            fx = fx[:, None]
            fy = fy[:, None]
            ref[sel] = (1 - fy) * ((1 - fx) * c[0] + fx * c[1]) + fy * ((1 - fx) * c[2] + fx * c[3])
    ref = np.clip(np.floor(ref + 0.5), 0, 255)
    diff = np.abs(out[..., :3].astype(np.int32) - ref.astype(np.int32))
    if filt == 0:
        assert diff.max() == 0
    else:
        assert diff.max() <= 1
    assert (out[~valid] == [0, 0, 0, 255]).all()
    assert (out[..., 3] == 255).all()
    # exactly the marked MCUs were decoded
    flags = o.mark(gb, filt)
    assert o.cached() == int(flags.sum())


def test_clamp_mode_reduces_to_bilinear_and_nearest():
    """The clamped mode (Sec. 4.4) against the two plain filters: where the four bilinear taps
    lie in the nearest texel's MCU it is the bilinear result; where the taps straddle an MCU
    edge on both axes every tap collapses onto the nearest texel, so it is the nearest
    result; and it marks exactly the nearest filter's MCUs."""
    ts, gb = _small_scene(seed=7)
    o = oracle.texset_from(ts)
    near = o.colorize(gb.uv, gb.tex_id, gb.mip, 0)
    bil = o.colorize(gb.uv, gb.tex_id, gb.mip, 1)
    clamp = o.colorize(gb.uv, gb.tex_id, gb.mip, 2)
    np.testing.assert_array_equal(o.mark(gb, 2), o.mark(gb, 0))
    valid = gb.tex_id != 0xFFFF
    inside = np.zeros(gb.tex_id.shape, bool)
    both = np.zeros(gb.tex_id.shape, bool)
    for t, l, e in ts.uploads():
        sel = valid & (gb.tex_id == t) & (gb.mip == l)
        if not sel.any():
            continue
        mw = 16 if e.sampling == 420 else 8
        u, v = gb.uv[..., 0][sel], gb.uv[..., 1][sel]
        (nx, ny), = _taps_np(u, v, e.width, e.height, 0)[0]
        (xa, ya), (xb, _), (_, yb), _ = _taps_np(u, v, e.width, e.height, 1)[0]
        same_x = (xa // mw == nx // mw) & (xb // mw == nx // mw)
        same_y = (ya // mw == ny // mw) & (yb // mw == ny // mw)
        inside[sel] = same_x & same_y
        both[sel] = ~same_x & ~same_y
    assert inside.sum() > 1000 and (valid & ~inside).sum() > 100 and both.sum() > 10
    np.testing.assert_array_equal(clamp[inside], bil[inside])
    np.testing.assert_array_equal(clamp[both], near[both])
    assert (clamp[valid & ~inside] != bil[valid & ~inside]).any()
