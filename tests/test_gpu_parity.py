"""GPU parity: the CUDA path (through the C ABI) against the oracle.

Bars: decoded tiles bit-exact; work list equal to the oracle's compacted marks (sorted,
unique); nearest pixels exact; bilinear pixels (plain or clamped to the nearest MCU)
within 1 LSB.
"""

import numpy as np
import pytest

import oracle
import synth
from helpers import GidMap, check_tiles, concat_gbuffers, frame, texel_grid_gbuffer

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def jt():
    import paper_2510_08166_gb300 as m
    return m


def _ctx(jt, blocks=1 << 15):
    return jt.Context(0, max_cache_blocks=blocks)


@pytest.mark.parametrize("filt", [0, 1, 2])
def test_affine_view_of_one_texture(jt, filt):
    ts, gb = synth.small_scene()
    ctx = _ctx(jt)
    ctx.upload_set(ts)
    o = oracle.texset_from(ts)
    dgb = jt.DeviceGBuffer.from_host(gb)
    out = frame(ctx, dgb, filt, torch).cpu().numpy()
    st = ctx.stats()
    ref_work = o.compact(o.mark(gb, filt))
    work = ctx.work_list()
    np.testing.assert_array_equal(work, ref_work)
    assert st["needed_blocks"] == ref_work.size and st["cache_units"] == 4 * ref_work.size
    assert check_tiles(ctx, o, GidMap(ts), work) == ref_work.size
    ref = o.colorize(gb.uv, gb.tex_id, gb.mip, filt)
    d = np.abs(out.astype(np.int32) - ref.astype(np.int32))
    assert d.max() <= (0 if filt == 0 else 1)
    ctx.close()


@pytest.mark.parametrize("size,sampling,q", [((16, 16), 420, 80), ((24, 40), 420, 95), ((33, 17), 420, 50),
                                             ((40, 24), 444, 90), ((1, 1), 420, 75), ((9, 3), 444, 60),
                                             ((200, 136), 444, 97), ((256, 128), 420, 30)])
def test_every_mcu_small_textures(jt, size, sampling, q):
    """Texel-centre G-buffer: every MCU of the level is needed; tiles and pixels exact."""
    w, h = size
    rgb = synth.texture(synth.mix_seed(21, w, h), w, h)
    ts = synth.TextureSet([[synth.encode(rgb, q, sampling)]])
    gb = texel_grid_gbuffer(w, h)
    ctx = _ctx(jt)
    ctx.upload_set(ts)
    o = oracle.texset_from(ts)
    out = frame(ctx, jt.DeviceGBuffer.from_host(gb), 0, torch).cpu().numpy()
    ctx.stats()
    work = ctx.work_list()
    assert work.size == ts.levels[0][0].nmcu
    check_tiles(ctx, o, GidMap(ts), work)
    full = oracle.Decoded(ts.levels[0][0].jfif).rgba
    np.testing.assert_array_equal(out, full)
    ctx.close()


def test_mip_chain_and_many_textures(jt):
    sizes = [(64, 64), (100, 60), (128, 128), (37, 91)]
    ts = synth.make_texture_set(31, sizes, [55, 70, 85, 95], [420, 444, 420, 444])
    gbs = []
    for t, l, e in ts.uploads():
        g = texel_grid_gbuffer(e.width, e.height, t, l)
        # pad to a common width of 128 with empty pixels
        W = 128
        uv = np.zeros((g.height, W, 2), np.float32)
        tex = np.full((g.height, W), 0xFFFF, np.uint16)
        mip = np.zeros((g.height, W), np.uint8)
        uv[:, :g.width] = g.uv
        tex[:, :g.width] = g.tex_id
        mip[:, :g.width] = g.mip
        gbs.append(synth.GBuffer(W, g.height, uv, tex, mip))
    gb = concat_gbuffers(gbs)
    ctx = _ctx(jt)
    ctx.upload_set(ts)
    o = oracle.texset_from(ts)
    out = frame(ctx, jt.DeviceGBuffer.from_host(gb), 0, torch).cpu().numpy()
    ctx.stats()
    work = ctx.work_list()
    assert work.size == ts.total_mcus()
    check_tiles(ctx, o, GidMap(ts), work)
    np.testing.assert_array_equal(out, o.colorize(gb.uv, gb.tex_id, gb.mip, 0))
    ctx.close()


@pytest.mark.parametrize("filt", [0, 1, 2])
def test_small_scene(jt, filt):
    sizes = [(64, 64), (128, 128), (256, 256), (96, 48), (512, 512)]
    ts = synth.make_texture_set(3, sizes, [60, 75, 90, 50, 80], [420, 420, 444, 420, 420])
    gb = synth.gbuffer_scene(3, 480, 270, ts.sizes, ts.nlevels, synth.Pose(quad_seed=3), nquads=40)
    ctx = _ctx(jt)
    ctx.upload_set(ts)
    o = oracle.texset_from(ts)
    out = frame(ctx, jt.DeviceGBuffer.from_host(gb), filt, torch).cpu().numpy()
    ctx.stats()
    ref_work = o.compact(o.mark(gb, filt))
    work = ctx.work_list()
    np.testing.assert_array_equal(work, ref_work)
    check_tiles(ctx, o, GidMap(ts), work)
    ref = o.colorize(gb.uv, gb.tex_id, gb.mip, filt)
    d = np.abs(out.astype(np.int32) - ref.astype(np.int32))
    assert d.max() <= (0 if filt == 0 else 1)
    ctx.close()


def test_flags_cleared_between_frames(jt):
    """A second frame with a different G-buffer needs only its own MCUs."""
    ts, gb = synth.small_scene()
    ctx = _ctx(jt)
    ctx.upload_set(ts)
    o = oracle.texset_from(ts)
    frame(ctx, jt.DeviceGBuffer.from_host(gb), 0, torch)
    ctx.stats()
    small = synth.gbuffer_affine(64, 64, 5.0, 0.1, 0)
    out = frame(ctx, jt.DeviceGBuffer.from_host(small), 0, torch).cpu().numpy()
    ctx.stats()
    np.testing.assert_array_equal(ctx.work_list(), o.compact(o.mark(small, 0)))
    np.testing.assert_array_equal(out, o.colorize(small.uv, small.tex_id, small.mip, 0))
    ctx.close()


@pytest.mark.parametrize("filt", [0, 1, 2])
def test_levels_smaller_than_an_mcu_and_odd_sizes(jt, filt):
    """Random uv (repeat wrap) over tiny and non-power-of-two levels: taps wrap inside
    a single MCU and across the last partial MCU."""
    sizes = [(8, 8), (4, 4), (12, 20), (33, 17), (16, 16), (5, 3)]
    ts = synth.make_texture_set(41, sizes, [70] * 6, [420, 444, 420, 444, 420, 420], full_chain=False)
    rng = np.random.default_rng(5)
    H, W = 96, 128
    uv = rng.uniform(-3.0, 3.0, (H, W, 2)).astype(np.float32)
    tex = rng.integers(0, len(sizes), (H, W)).astype(np.uint16)
    tex[rng.random((H, W)) < 0.05] = 0xFFFF
    gb = synth.GBuffer(W, H, uv, tex, np.zeros((H, W), np.uint8))
    ctx = _ctx(jt)
    ctx.upload_set(ts)
    o = oracle.texset_from(ts)
    out = frame(ctx, jt.DeviceGBuffer.from_host(gb), filt, torch).cpu().numpy()
    ctx.stats()
    np.testing.assert_array_equal(ctx.work_list(), o.compact(o.mark(gb, filt)))
    ref = o.colorize(gb.uv, gb.tex_id, gb.mip, filt)
    d = np.abs(out.astype(np.int32) - ref.astype(np.int32))
    assert d.max() <= (0 if filt == 0 else 1)
    ctx.close()


def test_degenerate_g_buffers(jt):
    """A G-buffer with no textured pixel needs no MCU and writes (0, 0, 0, 255) everywhere; a
    1x1 G-buffer needs exactly its pixel's MCU; a 0-pixel G-buffer is an argument error."""
    ts, _ = synth.small_scene()
    ctx = _ctx(jt)
    ctx.upload_set(ts)
    o = oracle.texset_from(ts)
    H, W = 48, 64
    empty = synth.GBuffer(W, H, np.zeros((H, W, 2), np.float32), np.full((H, W), 0xFFFF, np.uint16),
                          np.zeros((H, W), np.uint8))
    for filt in (0, 1, 2):
        out = frame(ctx, jt.DeviceGBuffer.from_host(empty), filt, torch).cpu().numpy()
        st = ctx.stats()
        assert st["needed_blocks"] == 0 and ctx.work_list().size == 0
        assert (out == np.array([0, 0, 0, 255], np.uint8)).all()
    one = synth.GBuffer(1, 1, np.array([[[0.3, 0.7]]], np.float32), np.zeros((1, 1), np.uint16),
                        np.zeros((1, 1), np.uint8))
    out = frame(ctx, jt.DeviceGBuffer.from_host(one), 1, torch).cpu().numpy()
    ctx.stats()
    np.testing.assert_array_equal(ctx.work_list(), o.compact(o.mark(one, 1)))
    assert np.abs(out.astype(int) - o.colorize(one.uv, one.tex_id, one.mip, 1).astype(int)).max() <= 1
    with pytest.raises(jt.JTError):
        ctx.mark(jt.DeviceGBuffer.empty(0, 0), 0)
    ctx.close()
