"""GPU parity at full size, in the launch configuration the benchmark times.

The 4K frame over 64 textures with full mip chains (bilinear) and the float chain over 16
coefficient textures of 2048^2 at 1920x1080. The oracle checks the whole work list and
sampled outputs it can compute one by one:
- decoded tiles of sampled needed MCUs (bit-exact);
- sampled pixels (<= 1 LSB);
- the float forward on sampled pixels;
- the gradient of the whole coefficient tensor against the FP64 adjoint (rel. L2 < 1e-5);
- central differences on 1000 coefficients."""

import numpy as np
import pytest

import oracle
import synth
from helpers import GidMap

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def jt():
    import paper_2510_08166_gb300 as m
    return m


def test_4k_frame_in_benchmark_configuration(jt):
    ts = synth.scene_textures()
    gb = synth.scene_gbuffer(ts)
    ctx = jt.Context(0, max_cache_blocks=1 << 18)  # as the benchmark
    ctx.upload_set(ts)
    dgb = jt.DeviceGBuffer.from_host(gb)
    out = torch.empty((gb.height, gb.width, 4), dtype=torch.uint8, device="cuda")
    ctx.autotune([(dgb, out)], jt.FILTER_BILINEAR, reps=3)  # the benchmark's shapes
    g = ctx.frame_graph([(dgb, out)], jt.FILTER_BILINEAR)
    for _ in range(3):  # replays, as timed
        ctx.graph_launch(g)
    ctx.stats()
    o = oracle.texset_from(ts)
    ref_work = o.compact(o.mark(gb, 1))
    work = ctx.work_list()
    np.testing.assert_array_equal(work, ref_work)
    gm = GidMap(ts)
    rng = np.random.default_rng(2)
    for gid in rng.choice(work, 300, replace=False):
        t, l, e, mcu = gm(int(gid))
        np.testing.assert_array_equal(ctx.tile(int(gid), e.sampling), o.decode_mcu(t, l, mcu, 16))
    idx = rng.choice(gb.width * gb.height, 50000, replace=False)
    ref = o.colorize(gb.uv.reshape(-1, 2)[idx], gb.tex_id.reshape(-1)[idx], gb.mip.reshape(-1)[idx], 1)
    got = out.cpu().numpy().reshape(-1, 4)[idx]
    assert np.abs(got.astype(np.int32) - ref.astype(np.int32)).max() <= 1
    ctx.graph_destroy(g)
    ctx.close()


def test_coefficient_scene_adjoint_full_size(jt):
    ts, coef, gb, target = synth.coefficient_scene()
    T, my, mx = coef.shape[:3]
    ctx = jt.Context(0, max_cache_blocks=T * my * mx)  # as the benchmark
    ctx.register_coeff_textures(0, T, mx * 16, my * 16)
    c = torch.from_numpy(coef).cuda()
    dgb = jt.DeviceGBuffer.from_host(gb)
    F = torch.empty((gb.height, gb.width, 3), dtype=torch.float32, device="cuda")
    ctx.colorize_float(dgb, c, F)
    ctx.stats()
    rng = np.random.default_rng(3)
    idx = rng.choice(gb.width * gb.height, 20000, replace=False)
    sub = synth.GBuffer(idx.size, 1, gb.uv.reshape(-1, 2)[idx].reshape(1, -1, 2),
                        gb.tex_id.reshape(-1)[idx].reshape(1, -1), gb.mip.reshape(-1)[idx].reshape(1, -1))
    F_ref = oracle.float_forward(coef, sub).reshape(-1, 3)
    got = F.cpu().numpy().reshape(-1, 3)[idx].astype(np.float64)
    assert np.linalg.norm(got - F_ref) <= 1e-6 * np.linalg.norm(F_ref)
    # gradient of L = sum (F - T)^2 over the whole tensor
    gF = (2.0 * (F - torch.from_numpy(target).cuda())).contiguous()
    gc = torch.empty_like(c)
    ctx.colorize_backward(dgb, gF, gc)
    ctx.stats()
    L_ref, g_ref = oracle.float_loss_grad(coef, gb, target)
    g = gc.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - g_ref) <= 1e-5 * np.linalg.norm(g_ref)
    zero = np.abs(g_ref).reshape(-1, 384).sum(axis=1) == 0
    assert (np.abs(g).reshape(-1, 384)[zero] == 0).all()
    pick = np.concatenate([rng.choice(np.flatnonzero(g_ref), 900, replace=False),
                           rng.integers(0, g_ref.size, 100)])
    fd = oracle.float_fd(coef, gb, target, pick, h=1.0)
    scale = np.abs(fd).max()
    np.testing.assert_allclose(g.ravel()[pick], fd, rtol=0, atol=2e-5 * scale)
    ctx.close()


def test_full_decode_4096_both_samplings(jt):
    """Full-decode stress shape: 4096^2 textures at quality 90, one 4:4:4 and one 4:2:0;
    every MCU decoded. All tiles, assembled into images, equal the oracle's sequential
    decode of the whole texture."""
    ts = synth.make_texture_set(synth.SEED_BASE + 4, [(4096, 4096)] * 2, [90, 90], [444, 420], full_chain=False)
    from helpers import mcu_grid_gbuffer
    gb = mcu_grid_gbuffer(ts)
    nmcu = ts.total_mcus()
    ctx = jt.Context(0, max_cache_blocks=(262144 + 4 * 65536) // 4 + 1024)
    ctx.upload_set(ts)
    dgb = jt.DeviceGBuffer.from_host(gb)
    ctx.mark(dgb, jt.FILTER_NEAREST)
    ctx.decode()
    st = ctx.stats()
    assert st["needed_blocks"] == nmcu
    work = ctx.work_list()
    np.testing.assert_array_equal(work, np.arange(nmcu, dtype=np.uint32))
    slots = ctx.slots(0, nmcu)
    cache = ctx.cache_units(0, int(st["cache_units"]))
    g0 = 0
    for t, l, e in ts.uploads():
        mw = 16 if e.sampling == 420 else 8
        units = mw * mw * 4 // 256
        mx, my = e.width // mw, e.height // mw
        s = slots[g0:g0 + mx * my].astype(np.int64)
        tiles = np.stack([cache[s + u] for u in range(units)], 1).reshape(my, mx, mw, mw, 4)
        img = tiles.transpose(0, 2, 1, 3, 4).reshape(my * mw, mx * mw, 4)
        np.testing.assert_array_equal(img, oracle.Decoded(e.jfif).rgba)
        g0 += mx * my
    ctx.close()


def _sampled_pixels(o, gb, got, n, seed, filt=1):
    rng = np.random.default_rng(seed)
    idx = rng.choice(gb.width * gb.height, n, replace=False)
    ref = o.colorize(gb.uv.reshape(-1, 2)[idx], gb.tex_id.reshape(-1)[idx], gb.mip.reshape(-1)[idx], filt)
    d = np.abs(got.reshape(-1, 4)[idx].astype(np.int32) - ref.astype(np.int32))
    return d.max()


def test_4k_frame_compact_form(jt):
    """The 4K frame over the same textures in the paper's compact form: identical pixels to
    the standard form, work list and sampled tiles equal to the oracle's compact decode."""
    ts = synth.scene_textures(compact=True)
    gb = synth.scene_gbuffer(ts)
    dgb = jt.DeviceGBuffer.from_host(gb)
    outs = []
    for compact in (False, True):
        ctx = jt.Context(0, max_cache_blocks=1 << 18)
        ctx.upload_set(ts, compact=compact)
        out = torch.empty((gb.height, gb.width, 4), dtype=torch.uint8, device="cuda")
        g = ctx.frame_graph([(dgb, out)], jt.FILTER_BILINEAR)
        ctx.graph_launch(g)
        ctx.stats()
        if compact:
            o = oracle.texset_from(ts, compact=True)
            work = ctx.work_list()
            np.testing.assert_array_equal(work, o.compact(o.mark(gb, 1)))
            gm = GidMap(ts)
            for gid in np.random.default_rng(4).choice(work, 300, replace=False):
                t, l, e, mcu = gm(int(gid))
                np.testing.assert_array_equal(ctx.tile(int(gid), e.sampling), o.decode_mcu(t, l, mcu, 16))
        ctx.graph_destroy(g)
        ctx.close()
        outs.append(out)
    assert torch.equal(outs[0], outs[1])


def test_4k_frame_reduced_mips(jt):
    """The 4K frame with levels 1, 2, 4, 5, ... decoded from levels 0, 3, 6, ... by reduction:
    work list equal to the oracle's, sampled tiles bit-exact, sampled pixels within 1 LSB."""
    ts = synth.scene_textures()
    gb = synth.scene_gbuffer(ts)
    ctx = jt.Context(0, max_cache_blocks=1 << 18)
    o = oracle.TexSet()
    items = []
    for t, lv in enumerate(ts.levels):
        for l, e in enumerate(lv):
            base = 3 * (l // 3)
            if l == base:
                ctx.upload(t, l, e)
                g0 = o.add(t, l, e)
            else:
                ctx.add_reduced_level(t, base, l - base, l)
                g0 = o.add_reduced(t, base, l - base, l)
            items.append((g0, t, l, e.sampling, l - base))
    dgb = jt.DeviceGBuffer.from_host(gb)
    out = torch.empty((gb.height, gb.width, 4), dtype=torch.uint8, device="cuda")
    g = ctx.frame_graph([(dgb, out)], jt.FILTER_BILINEAR)
    ctx.graph_launch(g)
    ctx.stats()
    work = ctx.work_list()
    np.testing.assert_array_equal(work, o.compact(o.mark(gb, 1)))
    bases = [it[0] for it in items]
    import bisect
    for gid in np.random.default_rng(5).choice(work, 300, replace=False):
        i = bisect.bisect_right(bases, int(gid)) - 1
        g0, t, l, sampling, r = items[i]
        mw = (16 if sampling == 420 else 8) >> r
        np.testing.assert_array_equal(ctx.tile(int(gid), sampling, r), o.decode_mcu(t, l, int(gid) - g0, mw))
    assert _sampled_pixels(o, gb, out.cpu().numpy(), 50000, 6) <= 1
    ctx.graph_destroy(g)
    ctx.close()


def test_batched_views_full_size(jt):
    """The 8 batched views (720p looking up, 1080p, 1440p, 4K and two VR stereo pairs) in one
    graph over the scene textures: the work list equals the oracle's union of the views'
    needed sets, and sampled pixels of every view are within 1 LSB of the oracle."""
    ts = synth.scene_textures()
    views = synth.eight_views(ts)
    ctx = jt.Context(0, max_cache_blocks=1 << 18)
    ctx.upload_set(ts)
    dv = [jt.DeviceGBuffer.from_host(v) for v in views]
    outs = [torch.empty((v.height, v.width, 4), dtype=torch.uint8, device="cuda") for v in views]
    g = ctx.frame_graph(list(zip(dv, outs)), jt.FILTER_BILINEAR)
    ctx.graph_launch(g)
    ctx.stats()
    o = oracle.texset_from(ts)
    flags = None
    for v in views:
        f = o.mark(v, 1)
        flags = f if flags is None else np.maximum(flags, f)
    np.testing.assert_array_equal(ctx.work_list(), o.compact(flags))
    for i, (v, out) in enumerate(zip(views, outs)):
        assert _sampled_pixels(o, v, out.cpu().numpy(), 10000, 20 + i) <= 1, f"view {i}"
    ctx.graph_destroy(g)
    ctx.close()
