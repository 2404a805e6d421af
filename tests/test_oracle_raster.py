"""Pins for the fp32 scene rasteriser (the G-buffer of the procedural ground plane + quads
scene that stands in for the renderer's geometry pass).

- Against the input generator's double-precision definition of the same scene: texture ids
  equal, mip levels equal but for rounding-boundary pixels, uv within 1/1000 of a texel of
  the selected level.
- Closed form: a camera looking straight down at height h sees the ground at a constant
  footprint of 2 h tan(fov/2) / H metres per pixel, i.e. tw / 2 times that in texels, so
  every ground pixel's level is round(log2(footprint)) (away from the cell offsets).
"""

import numpy as np
import pytest

import oracle
import synth

SIZES = [(1024, 1024), (2048, 2048), (512, 512), (4096, 4096)]
LEVELS = [11, 12, 10, 13]


@pytest.mark.parametrize("W,H,pose,nq", [
    (640, 360, synth.Pose(quad_seed=5), 120),
    (480, 270, synth.Pose((1.0, 1.7, 2.0), 40.0, -20.0, 60.0, 7, 0.01), 200),
    (333, 257, synth.Pose((-3.0, 2.5, 1.0), 200.0, 4.0, 90.0, 9, -0.008), 60),  # horizon in view
])
def test_raster_matches_the_generator(W, H, pose, nq):
    d = synth.scene_desc(5, W, H, SIZES, LEVELS, pose, nquads=nq)
    g = synth.gbuffer_scene(5, W, H, SIZES, LEVELS, pose, nquads=nq)
    uv, tex, mip = oracle.raster_scene(d)
    assert (tex == g.tex_id).mean() >= 0.9999
    assert (mip == g.mip).mean() >= 0.999
    # uv error in texels of the selected level, where that level is at least 8 texels wide
    # (near the horizon the hit point is ill-conditioned, but the level is then a few texels)
    m = (tex == g.tex_id) & (tex != 0xFFFF)
    tw = np.array([s[0] for s in SIZES])[np.where(m, tex, 0)]
    lw = tw >> g.mip.astype(np.int64)
    err = np.abs(uv - g.uv).max(axis=-1) * lw
    sel = m & (lw >= 8)
    assert sel.mean() > 0.5 and err[sel].max() < 1e-3
    assert (uv[tex == 0xFFFF] == 0).all() and (mip[tex == 0xFFFF] == 0).all()
    if pose.pitch > 0:
        assert (tex == 0xFFFF).mean() > 0.1  # sky above the horizon


@pytest.mark.parametrize("h,fov", [(1.7, 60.0), (12.0, 40.0), (100.0, 90.0)])
def test_looking_down_has_the_closed_form_level(h, fov):
    W = H = 256
    pose = synth.Pose((0.3, h, -0.7), 0.0, -90.0, fov, 1, 0.0)
    d = synth.scene_desc(3, W, H, SIZES, LEVELS, pose, nquads=0)
    uv, tex, mip = oracle.raster_scene(d)
    assert (tex != 0xFFFF).all()
    metres = 2 * h * np.tan(np.radians(fov) / 2) / H  # per pixel at the image centre
    c = slice(H // 2 - 4, H // 2 + 4)
    for t in range(len(SIZES)):
        sel = tex[c, c] == t
        if not sel.any():
            continue
        rho = metres / 2 * SIZES[t][0]
        want = int(np.clip(np.floor(np.log2(rho) + 0.5), 0, LEVELS[t] - 1))
        if abs(np.log2(rho) + 0.5 - np.round(np.log2(rho) + 0.5)) > 0.01:  # not at a boundary
            assert (mip[c, c][sel] == want).all()


def test_empty_scene_without_mips():
    pose = synth.Pose(quad_seed=2)
    d = synth.scene_desc(4, 64, 48, SIZES, LEVELS, pose, nquads=30, use_mips=False)
    g = synth.gbuffer_scene(4, 64, 48, SIZES, LEVELS, pose, nquads=30, use_mips=False)
    uv, tex, mip = oracle.raster_scene(d)
    assert (mip == 0).all()
    np.testing.assert_array_equal(tex, g.tex_id)
