"""GPU: batched frames, CUDA graphs, the per-texture reference form, pass timing,
autotuning and the error paths of the C ABI."""

import ctypes

import numpy as np
import pytest

import oracle
import synth
from helpers import GidMap, check_tiles, frame, set_short_lists

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def jt():
    import paper_2510_08166_gb300 as m
    return m


@pytest.fixture(scope="module")
def scene():
    sizes = [(64, 64), (128, 128), (256, 256), (96, 48), (512, 512), (1024, 1024)]
    ts = synth.make_texture_set(7, sizes, [60, 75, 90, 50, 80, 95], [420, 420, 444, 420, 420, 420])
    views = [synth.gbuffer_scene(7, w, h, ts.sizes, ts.nlevels, synth.Pose((0.3 * i, 1.7, 0.2 * i), 15.0 * i,
                                                                           -25.0, 60.0, 100 + i, 0.0), nquads=30)
             for i, (w, h) in enumerate([(320, 180), (256, 256), (333, 111)])]
    return ts, views


def _outs(views):
    return [torch.zeros((v.height, v.width, 4), dtype=torch.uint8, device="cuda") for v in views]


@pytest.mark.parametrize("filt", [0, 1, 2])
def test_batched_equals_oracle_and_union(jt, scene, filt):
    ts, views = scene
    ctx = jt.Context(0, 1 << 15)
    ctx.upload_set(ts)
    o = oracle.texset_from(ts)
    dv = [jt.DeviceGBuffer.from_host(v) for v in views]
    outs = _outs(views)
    ctx.frame(list(zip(dv, outs)), filt)
    ctx.stats()
    # one work list for the union of the views' marks
    union = np.zeros(o.total, np.uint8)
    for v in views:
        union |= o.mark(v, filt)
    ref_work = o.compact(union)
    work = ctx.work_list()
    np.testing.assert_array_equal(work, ref_work)
    check_tiles(ctx, o, GidMap(ts), work)
    for v, out in zip(views, outs):
        ref = o.colorize(v.uv, v.tex_id, v.mip, filt)
        d = np.abs(out.cpu().numpy().astype(np.int32) - ref.astype(np.int32))
        assert d.max() <= (0 if filt == 0 else 1)
    ctx.close()


def test_graph_plain_and_direct_agree(jt, scene):
    ts, views = scene
    ctx = jt.Context(0, 1 << 15)
    ctx.upload_set(ts)
    dv = [jt.DeviceGBuffer.from_host(v) for v in views]
    a, b, c = _outs(views), _outs(views), _outs(views)
    ctx.frame(list(zip(dv, a)), 1)
    ctx.stats()
    n_direct = ctx.stats()["needed_blocks"]
    g = ctx.frame_graph(list(zip(dv, b)), 1)
    for _ in range(3):  # replays start from cleared flags and status words
        ctx.graph_launch(g)
        st = ctx.stats()
        assert st["needed_blocks"] == n_direct
    ctx.frame_plain(list(zip(dv, c)), 1)
    ctx.stats()
    for x, y, z in zip(a, b, c):
        assert torch.equal(x, y) and torch.equal(x, z)
    # the graph reads the G-buffer contents at launch: change them and replay
    o = oracle.texset_from(ts)
    other = synth.gbuffer_scene(99, views[0].width, views[0].height, ts.sizes, ts.nlevels,
                                synth.Pose(quad_seed=99), nquads=10)
    d0 = jt.DeviceGBuffer.from_host(other)
    dv[0].uv.copy_(d0.uv)
    dv[0].tex_id.copy_(d0.tex_id)
    dv[0].mip.copy_(d0.mip)
    ctx.graph_launch(g)
    ctx.stats()
    ref = o.colorize(other.uv, other.tex_id, other.mip, 1)
    d = np.abs(b[0].cpu().numpy().astype(np.int32) - ref.astype(np.int32))
    assert d.max() <= 1
    ctx.graph_destroy(g)
    ctx.close()


def test_profile_direct_and_graph(jt, scene):
    ts, views = scene
    ctx = jt.Context(0, 1 << 15)
    ctx.upload_set(ts)
    dv = jt.DeviceGBuffer.from_host(views[0])
    out = _outs(views[:1])[0]
    ctx.profile(True)
    ctx.frame([(dv, out)], 1)
    p = ctx.profile_read()
    assert all(v > 0 for v in p.values()), p
    g = ctx.frame_graph([(dv, out)], 1)
    ctx.graph_launch(g)
    p2 = ctx.profile_read()
    assert all(v > 0 for v in p2.values()), p2
    ctx.stats()
    ctx.close()


def test_autotune_keeps_results(jt, scene):
    ts, views = scene
    ctx = jt.Context(0, 1 << 15)
    ctx.upload_set(ts)
    dv = jt.DeviceGBuffer.from_host(views[1])
    ref = frame(ctx, dv, 1, torch)
    ctx.stats()
    out = _outs(views[1:2])[0]
    best, ms = ctx.autotune([(dv, out)], 1, reps=2)
    assert ms > 0 and best == ctx.tuning()
    ctx.frame([(dv, out)], 1)
    ctx.stats()
    assert torch.equal(out, ref)
    ctx.close()


@pytest.mark.parametrize("mcus,warps,per_sm", [(4, 2, 1), (8, 8, 2), (4, 16, 1), (16, 4, 1), (32, 2, 1),
                                               (16, 2, 2), (32, 7, 1), (16, 13, 1), (8, 3, 2)])
@pytest.mark.parametrize("short", [0, 1])
def test_decode_shapes_bit_exact(jt, scene, mcus, warps, per_sm, short):
    ts, views = scene
    ctx = jt.Context(0, 1 << 15)
    ctx.upload_set(ts)
    t = ctx.tuning()
    t.update(decode_mcus_per_warp=mcus, decode_warps=warps, decode_ctas_per_sm=per_sm, pixel_threads=128,
             pixel_ctas_per_sm=2, decode_short_lists=short)
    ctx.set_tuning(**t)
    o = oracle.texset_from(ts)
    dv = jt.DeviceGBuffer.from_host(views[0])
    out = frame(ctx, dv, 0, torch).cpu().numpy()
    ctx.stats()
    check_tiles(ctx, o, GidMap(ts), ctx.work_list())
    np.testing.assert_array_equal(out, o.colorize(views[0].uv, views[0].tex_id, views[0].mip, 0))
    ctx.close()


# ---- errors: returned as statuses, never a trap ----

@pytest.mark.parametrize("short", [0, 1])
def test_corrupt_stream_reports_status(jt, short):
    rgb = synth.texture(3, 64, 64)
    enc = synth.encode(rgb, 80, 420)
    bad = synth.Encoded(**{k: getattr(enc, k) for k in enc.__dataclass_fields__})
    bad.scan = np.full_like(enc.scan, 0xFF)  # sixteen one-bits match no AC/DC code
    ctx = jt.Context(0, 1 << 10)
    set_short_lists(ctx, short)
    ctx.upload(0, 0, bad)
    from helpers import texel_grid_gbuffer
    dv = jt.DeviceGBuffer.from_host(texel_grid_gbuffer(64, 64))
    frame(ctx, dv, 0, torch)
    st = ctx.stats(check=False)
    assert st["status"] == 4 and st["error_bits"] & jt.DEVERR_CORRUPT
    # the word is cleared once read; a good texture in the same context decodes fine
    ctx.upload(1, 0, enc)
    g = texel_grid_gbuffer(64, 64, tex=1)
    out = frame(ctx, jt.DeviceGBuffer.from_host(g), 0, torch).cpu().numpy()
    assert ctx.stats()["status"] == 0
    np.testing.assert_array_equal(out, oracle.Decoded(enc.jfif).rgba)
    ctx.close()


@pytest.mark.parametrize("short", [0, 1])
def test_truncated_stream_reports_status(jt, short):
    rgb = synth.texture(4, 64, 64)
    enc = synth.encode(rgb, 90, 420)
    bad = synth.Encoded(**{k: getattr(enc, k) for k in enc.__dataclass_fields__})
    bad.scan = enc.scan[: len(enc.scan) // 2].copy()
    bad.scan_bits = len(bad.scan) * 8
    ctx = jt.Context(0, 1 << 10)
    set_short_lists(ctx, short)
    ctx.upload(0, 0, bad)
    from helpers import texel_grid_gbuffer
    frame(ctx, jt.DeviceGBuffer.from_host(texel_grid_gbuffer(64, 64)), 0, torch)
    st = ctx.stats(check=False)
    assert st["status"] == 4
    ctx.close()


def test_capacity_overflow_reports_status(jt):
    ts, gb = synth.small_scene()
    ctx = jt.Context(0, max_cache_blocks=100)  # 1024 MCUs are needed
    ctx.upload_set(ts)
    frame(ctx, jt.DeviceGBuffer.from_host(gb), 0, torch)
    st = ctx.stats(check=False)
    assert st["status"] == 5 and st["needed_blocks"] == 1024
    ctx.close()


def test_missing_level_reports_status(jt):
    ts, gb = synth.small_scene()
    ctx = jt.Context(0, 1 << 12)
    ctx.upload_set(ts)
    gb.mip[:4, :] = 3  # level 3 was never uploaded
    frame(ctx, jt.DeviceGBuffer.from_host(gb), 0, torch)
    st = ctx.stats(check=False)
    assert st["status"] == 6
    ctx.close()


def test_state_and_argument_errors(jt):
    ts, gb = synth.small_scene()
    ctx = jt.Context(0, 1 << 12)
    with pytest.raises(jt.JTError) as e:
        ctx.decode()
    assert e.value.status == 7
    ctx.upload_set(ts)
    with pytest.raises(jt.JTError) as e:
        ctx.upload(0, 0, ts.levels[0][0])  # already uploaded
    assert e.value.status == 1
    dv = jt.DeviceGBuffer.from_host(gb)
    out = torch.empty((gb.height, gb.width, 4), dtype=torch.uint8, device="cuda")
    with pytest.raises(jt.JTError):
        ctx.colorize(dv, 0, out)  # before any decode
    bad = jt.jt_gbuffer(dv.uv.data_ptr() + 4, dv.tex_id.data_ptr(), dv.mip.data_ptr(), 4, 4)  # misaligned uv
    assert jt.lib().jt_mark(ctx._h, ctypes.byref(bad), 0, None) == 1
    g = dv.c()
    assert jt.lib().jt_mark(ctx._h, ctypes.byref(g), 7, None) == 1  # bad filter
    ctx.close()
