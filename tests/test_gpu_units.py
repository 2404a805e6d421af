"""GPU parity for data-unit starts (an index extension: six lanes decode one MCU's data units
at once, each unit's DC difference chained afterwards). Tiles bit-exact against the oracle,
frames identical to the MCU-at-a-time decode, bad offsets reported."""

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


@pytest.mark.parametrize("size,sampling,q", [((16, 16), 420, 80), ((33, 17), 420, 50), ((40, 24), 444, 95),
                                             ((1, 1), 420, 75), ((200, 136), 444, 100), ((256, 144), 420, 100),
                                             ((256, 128), 420, 30)])
@pytest.mark.parametrize("mcus", [4, 32])
def test_every_mcu_by_units(jt, size, sampling, q, mcus):
    w, h = size
    e = synth.encode(synth.texture(synth.mix_seed(29, w, h), w, h), q, sampling)
    ts = synth.TextureSet([[e]])
    ctx = jt.Context(0, max_cache_blocks=1 << 14)
    t = ctx.tuning()
    t.update(decode_mcus_per_warp=mcus, decode_warps=4, decode_ctas_per_sm=1)
    ctx.set_tuning(**t)
    ctx.upload_set(ts, units=True)
    gb = texel_grid_gbuffer(w, h)
    out = frame(ctx, jt.DeviceGBuffer.from_host(gb), 0, torch).cpu().numpy()
    ctx.stats()
    work = ctx.work_list()
    assert work.size == e.nmcu
    check_tiles(ctx, oracle.texset_from(ts), GidMap(ts), work)
    np.testing.assert_array_equal(out, oracle.Decoded(e.jfif).rgba)
    ctx.close()


def test_mixed_levels(jt):
    """Levels with and without starts, compact levels and levels reduced from a level with
    starts, in one context; every MCU of every level decoded."""
    sizes = [(64, 64), (100, 60), (128, 128), (37, 91)]
    ts = synth.make_texture_set(37, sizes, [55, 70, 85, 95], [420, 444, 420, 444], compact=True,
                                full_chain=False)
    ctx = jt.Context(0, max_cache_blocks=1 << 14)
    o = oracle.TexSet()
    gbs = []
    levels = []
    for t, l, e in ts.uploads():
        if t == 1:
            ctx.upload_compact(t, l, e)
            o.add_compact(t, l, e)
        else:
            ctx.upload(t, l, e)
            o.add(t, l, e)
            if t != 3:
                ctx.set_du_offsets(t, l, e.du_offsets)
                o.set_du_offsets(t, l, e.du_offsets)
        levels.append((t, l, e.width, e.height))
    ctx.add_reduced_level(0, 0, 1, 1)
    o.add_reduced(0, 0, 1, 1)
    levels.append((0, 1, 32, 32))
    for t, l, w, h in levels:
        g = texel_grid_gbuffer(w, h, t, l)
        W = 128
        uv = np.zeros((h, W, 2), np.float32)
        tex = np.full((h, W), 0xFFFF, np.uint16)
        mip = np.zeros((h, W), np.uint8)
        uv[:, :w], tex[:, :w], mip[:, :w] = g.uv, g.tex_id, g.mip
        gbs.append(synth.GBuffer(W, h, uv, tex, mip))
    gb = concat_gbuffers(gbs)
    out = frame(ctx, jt.DeviceGBuffer.from_host(gb), 0, torch).cpu().numpy()
    ctx.stats()
    work = ctx.work_list()
    np.testing.assert_array_equal(work, o.compact(o.mark(gb, 0)))
    np.testing.assert_array_equal(out, o.colorize(gb.uv, gb.tex_id, gb.mip, 0))
    ctx.close()


@pytest.mark.parametrize("filt", [1, 2])
def test_scene_same_pixels_as_mcu_decode(jt, filt):
    sizes = [(256, 256), (512, 512), (1024, 1024), (128, 128)]
    ts = synth.make_texture_set(39, sizes, [60, 95, 75, 50], [420, 420, 444, 420])
    gb = synth.gbuffer_scene(39, 480, 270, ts.sizes, ts.nlevels, synth.Pose(quad_seed=39), nquads=40)
    dgb = jt.DeviceGBuffer.from_host(gb)
    outs = []
    for units in (False, True):
        ctx = jt.Context(0, max_cache_blocks=1 << 15)
        ctx.upload_set(ts, units=units)
        outs.append(frame(ctx, dgb, filt, torch))
        ctx.stats()
        if units:
            check_tiles(ctx, oracle.texset_from(ts), GidMap(ts), ctx.work_list())
        ctx.close()
    assert torch.equal(outs[0], outs[1])


def test_bad_offsets(jt):
    e = synth.encode(synth.texture(8, 64, 64), 80, 420)
    ctx = jt.Context(0, max_cache_blocks=256)
    ctx.upload(0, 0, e)
    dec = e.du_offsets.copy()
    dec[0, 1] = dec[0, 0] - 1  # decreasing inside an MCU
    with pytest.raises(jt.JTError):
        ctx.set_du_offsets(0, 0, dec)
    early = e.du_offsets.copy()
    early[:, 0] -= 1  # every second unit starts one bit early: the first unit runs past it
    ctx.set_du_offsets(0, 0, early)
    frame(ctx, jt.DeviceGBuffer.from_host(texel_grid_gbuffer(64, 64)), 0, torch)
    st = ctx.stats(check=False)
    assert st["error_bits"] & jt.DEVERR_CORRUPT
    ctx.close()
