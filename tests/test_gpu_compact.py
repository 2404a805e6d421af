"""GPU parity for the paper's compact random-access form (Sec. 5.1 indexing table, Sec. 5.3
DC records): levels uploaded with jt_upload_texture_compact decode to the oracle's tiles
bit-exact, mixed with standard-form levels in one context, and a frame gives the same
pixels as the standard form."""

import numpy as np
import pytest

import oracle
import synth
from helpers import GidMap, check_tiles, concat_gbuffers, frame, set_short_lists, texel_grid_gbuffer

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def jt():
    import paper_2510_08166_gb300 as m
    return m


@pytest.mark.parametrize("size,sampling,q", [((16, 16), 420, 80), ((33, 17), 420, 50), ((40, 24), 444, 90),
                                             ((1, 1), 420, 75), ((9, 3), 444, 60), ((200, 136), 444, 100),
                                             ((256, 144), 420, 100), ((256, 128), 420, 30)])
@pytest.mark.parametrize("short", [0, 1])
def test_every_mcu_compact(jt, size, sampling, q, short):
    """Every MCU of the level (144 = 9 x 16 rows of MCUs: whole offset groups and a tail)."""
    w, h = size
    rgb = synth.texture(synth.mix_seed(23, w, h), w, h)
    ts = synth.TextureSet([[synth.encode(rgb, q, sampling, compact=True)]])
    gb = texel_grid_gbuffer(w, h)
    ctx = jt.Context(0, max_cache_blocks=1 << 14)
    set_short_lists(ctx, short)
    ctx.upload_set(ts, compact=True)
    o = oracle.texset_from(ts, compact=True)
    out = frame(ctx, jt.DeviceGBuffer.from_host(gb), 0, torch).cpu().numpy()
    ctx.stats()
    work = ctx.work_list()
    assert work.size == ts.levels[0][0].nmcu
    check_tiles(ctx, o, GidMap(ts), work)
    np.testing.assert_array_equal(out, oracle.Decoded(ts.levels[0][0].jfif).rgba)
    ctx.close()


def test_mixed_forms_in_one_context(jt):
    """Textures alternate between the two forms; every MCU of every level is decoded."""
    sizes = [(64, 64), (100, 60), (128, 128), (37, 91)]
    ts = synth.make_texture_set(33, sizes, [55, 70, 85, 95], [420, 444, 420, 444], compact=True)
    ctx = jt.Context(0, max_cache_blocks=1 << 14)
    o = oracle.TexSet()
    gbs = []
    for t, l, e in ts.uploads():
        if t % 2:
            ctx.upload_compact(t, l, e)
            o.add_compact(t, l, e)
        else:
            ctx.upload(t, l, e)
            o.add(t, l, e)
        g = texel_grid_gbuffer(e.width, e.height, t, l)
        W = 128
        uv = np.zeros((g.height, W, 2), np.float32)
        tex = np.full((g.height, W), 0xFFFF, np.uint16)
        mip = np.zeros((g.height, W), np.uint8)
        uv[:, :g.width] = g.uv
        tex[:, :g.width] = g.tex_id
        mip[:, :g.width] = g.mip
        gbs.append(synth.GBuffer(W, g.height, uv, tex, mip))
    gb = concat_gbuffers(gbs)
    out = frame(ctx, jt.DeviceGBuffer.from_host(gb), 0, torch).cpu().numpy()
    ctx.stats()
    work = ctx.work_list()
    assert work.size == ts.total_mcus()
    check_tiles(ctx, o, GidMap(ts), work)
    np.testing.assert_array_equal(out, o.colorize(gb.uv, gb.tex_id, gb.mip, 0))
    ctx.close()


@pytest.mark.parametrize("filt", [1, 2])
def test_scene_same_pixels_as_standard_form(jt, filt):
    sizes = [(256, 256), (512, 512), (1024, 1024), (128, 128)]
    ts = synth.make_texture_set(35, sizes, [60, 90, 75, 50], [420, 420, 444, 420], compact=True)
    gb = synth.gbuffer_scene(35, 480, 270, ts.sizes, ts.nlevels, synth.Pose(quad_seed=35), nquads=40)
    std = jt.Context(0, max_cache_blocks=1 << 15)
    std.upload_set(ts)
    cpt = jt.Context(0, max_cache_blocks=1 << 15)
    cpt.upload_set(ts, compact=True)
    dgb = jt.DeviceGBuffer.from_host(gb)
    a = frame(std, dgb, filt, torch)
    std.stats()
    b = frame(cpt, dgb, filt, torch)
    cpt.stats()
    assert torch.equal(a, b)
    np.testing.assert_array_equal(cpt.work_list(), std.work_list())
    o = oracle.texset_from(ts, compact=True)
    check_tiles(cpt, o, GidMap(ts), cpt.work_list())
    std.close()
    cpt.close()


def test_bad_offsets_are_rejected(jt):
    e = synth.encode(synth.texture(7, 64, 64), 70, 420, compact=True)
    ctx = jt.Context(0, max_cache_blocks=64)
    e.compact.rel = e.compact.rel.copy()
    e.compact.rel[3] = 0  # MCU 4 would start before MCU 3
    with pytest.raises(jt.JTError):
        ctx.upload_compact(0, 0, e)
    ctx.close()
