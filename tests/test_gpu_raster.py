"""GPU parity for the scene rasteriser (the geometry-pass stand-in): the G-buffer written by
jt_raster_scene equals the oracle's fp32 rasteriser bit for bit (uv, texture ids, levels),
and a frame over it equals the frame over the same G-buffer uploaded from the host."""

import numpy as np
import pytest

import oracle
import synth
from helpers import frame

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SIZES = [(1024, 1024), (2048, 2048), (512, 512), (4096, 4096)]
LEVELS = [11, 12, 10, 13]


@pytest.fixture(scope="module")
def jt():
    import paper_2510_08166_gb300 as m
    return m


def _gpu_raster(jt, ctx, d):
    gb = jt.DeviceGBuffer.empty(d.width, d.height)
    ctx.raster_scene(d, gb)
    torch.cuda.synchronize()
    return gb


def _assert_same(gb, uv, tex, mip):
    np.testing.assert_array_equal(gb.tex_id.cpu().numpy().view(np.uint16), tex)
    np.testing.assert_array_equal(gb.mip.cpu().numpy(), mip)
    np.testing.assert_array_equal(gb.uv.cpu().numpy().view(np.uint32), uv.view(np.uint32))


@pytest.mark.parametrize("W,H,pose,nq,mips", [
    (640, 360, synth.Pose(quad_seed=5), 120, True),
    (480, 270, synth.Pose((1.0, 1.7, 2.0), 40.0, -20.0, 60.0, 7, 0.01), 200, True),
    (333, 257, synth.Pose((-3.0, 2.5, 1.0), 200.0, 4.0, 90.0, 9, -0.008), 60, True),  # horizon in view
    (100, 37, synth.Pose(quad_seed=3), 0, True),  # no quads, ragged tiles
    (256, 256, synth.Pose((0.3, 12.0, -0.7), 0.0, -90.0, 40.0, 1, 0.0), 300, False),
])
def test_raster_bit_exact(jt, W, H, pose, nq, mips):
    d = synth.scene_desc(5, W, H, SIZES, LEVELS, pose, nquads=nq, use_mips=mips)
    ctx = jt.Context(0, max_cache_blocks=64)
    gb = _gpu_raster(jt, ctx, d)
    _assert_same(gb, *oracle.raster_scene(d))
    ctx.close()


def test_4k_scene_and_frame(jt):
    """The 4K scene in the benchmark's pose and its frame: the frame over the rastered
    G-buffer equals the frame over the oracle's G-buffer uploaded from the host."""
    ts = synth.scene_textures(ntex=8)
    pose = synth.scene_pose()
    d = synth.scene_desc(synth.SEED_BASE + 2, 3840, 2160, ts.sizes, ts.nlevels, pose, nquads=200)
    ctx = jt.Context(0, max_cache_blocks=1 << 18)
    ctx.upload_set(ts)
    gb = _gpu_raster(jt, ctx, d)
    uv, tex, mip = oracle.raster_scene(d)
    _assert_same(gb, uv, tex, mip)
    a = frame(ctx, gb, jt.FILTER_BILINEAR, torch)
    ctx.stats()
    b = frame(ctx, jt.DeviceGBuffer.from_host(synth.GBuffer(3840, 2160, uv, tex, mip)), jt.FILTER_BILINEAR, torch)
    ctx.stats()
    assert torch.equal(a, b)
    ctx.close()


def test_raster_errors(jt):
    d = synth.scene_desc(5, 64, 32, SIZES, LEVELS, synth.Pose(quad_seed=5), nquads=10)
    ctx = jt.Context(0, max_cache_blocks=64)
    with pytest.raises(jt.JTError):
        ctx.raster_scene(d, jt.DeviceGBuffer.empty(63, 32))  # size mismatch
    d.quads = d.quads.copy()
    d.quads[0]["tex"] = len(SIZES)
    with pytest.raises(jt.JTError):
        ctx.raster_scene(d, jt.DeviceGBuffer.empty(64, 32))
    ctx.close()
