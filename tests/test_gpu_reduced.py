"""GPU parity for reduced-resolution levels (the mip alternative of Sec. 7): levels decoded at
1/2, 1/4 or 1/8 from the lowest frequencies of a stored level. Tiles bit-exact against the
oracle, pixels exact (nearest) or within 1 LSB (bilinear), work lists equal."""

import bisect

import numpy as np
import pytest

import oracle
import synth
from helpers import concat_gbuffers, frame, set_short_lists, texel_grid_gbuffer

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def jt():
    import paper_2510_08166_gb300 as m
    return m


class Registry:
    """Registers levels in the same order on the GPU context and the oracle, and maps a gid
    back to (tex, level, mcu, sampling, reduce)."""

    def __init__(self, ctx):
        self.ctx, self.o = ctx, oracle.TexSet()
        self.bases, self.items = [], []

    def upload(self, t, l, e):
        self.ctx.upload(t, l, e)
        self._note(self.o.add(t, l, e), t, l, e.sampling, 0)

    def reduced(self, t, src, r, l, sampling):
        self.ctx.add_reduced_level(t, src, r, l)
        self._note(self.o.add_reduced(t, src, r, l), t, l, sampling, r)

    def _note(self, g, t, l, sampling, r):
        self.bases.append(g)
        self.items.append((t, l, sampling, r))

    def check_tiles(self, gids):
        for gid in gids:
            i = bisect.bisect_right(self.bases, int(gid)) - 1
            t, l, sampling, r = self.items[i]
            mw = (16 if sampling == 420 else 8) >> r
            got = self.ctx.tile(int(gid), sampling, r)
            ref = self.o.decode_mcu(t, l, int(gid) - self.bases[i], mw)
            np.testing.assert_array_equal(got, ref, err_msg=f"gid {gid} tex {t} level {l}")


@pytest.mark.parametrize("size,sampling,q", [((64, 64), 420, 80), ((33, 17), 420, 50), ((40, 24), 444, 95),
                                             ((96, 48), 444, 60), ((256, 128), 420, 100)])
@pytest.mark.parametrize("short", [0, 1])
def test_every_reduced_mcu(jt, size, sampling, q, short):
    w, h = size
    e = synth.encode(synth.texture(synth.mix_seed(41, w, h), w, h), q, sampling)
    ctx = jt.Context(0, max_cache_blocks=1 << 14)
    set_short_lists(ctx, short)
    reg = Registry(ctx)
    reg.upload(0, 0, e)
    gbs = []
    for r in (1, 2, 3):
        reg.reduced(0, 0, r, r, sampling)
        lw, lh = max(1, w >> r), max(1, h >> r)
        g = texel_grid_gbuffer(lw, lh, 0, r)
        W = w  # pad rows to a common width with empty pixels
        uv = np.zeros((lh, W, 2), np.float32)
        tex = np.full((lh, W), 0xFFFF, np.uint16)
        mip = np.zeros((lh, W), np.uint8)
        uv[:, :lw], tex[:, :lw], mip[:, :lw] = g.uv, g.tex_id, g.mip
        gbs.append(synth.GBuffer(W, lh, uv, tex, mip))
    gb = concat_gbuffers(gbs)
    out = frame(ctx, jt.DeviceGBuffer.from_host(gb), 0, torch).cpu().numpy()
    ctx.stats()
    work = ctx.work_list()
    np.testing.assert_array_equal(work, reg.o.compact(reg.o.mark(gb, 0)))
    reg.check_tiles(work)
    np.testing.assert_array_equal(out, reg.o.colorize(gb.uv, gb.tex_id, gb.mip, 0))
    ctx.close()


@pytest.mark.parametrize("filt", [0, 1, 2])
def test_scene_with_mips_from_reduction(jt, filt):
    """Stored levels 0 and 3 of every texture; levels 1, 2 come from level 0 and 4, 5 from
    level 3 by reduction; the rest of the chain is stored."""
    sizes = [(256, 256), (512, 512), (1024, 1024), (128, 128)]
    ts = synth.make_texture_set(43, sizes, [60, 90, 75, 50], [420, 420, 444, 420])
    gb = synth.gbuffer_scene(43, 480, 270, ts.sizes, ts.nlevels, synth.Pose(quad_seed=43), nquads=40)
    ctx = jt.Context(0, max_cache_blocks=1 << 15)
    reg = Registry(ctx)
    for t, lv in enumerate(ts.levels):
        for l, e in enumerate(lv):
            base = 3 * (l // 3)
            if l == base:
                reg.upload(t, l, e)
            else:
                reg.reduced(t, base, l - base, l, e.sampling)
    out = frame(ctx, jt.DeviceGBuffer.from_host(gb), filt, torch).cpu().numpy()
    ctx.stats()
    work = ctx.work_list()
    np.testing.assert_array_equal(work, reg.o.compact(reg.o.mark(gb, filt)))
    reg.check_tiles(work)
    ref = reg.o.colorize(gb.uv, gb.tex_id, gb.mip, filt)
    d = np.abs(out.astype(np.int32) - ref.astype(np.int32))
    assert d.max() <= (0 if filt == 0 else 1)
    ctx.close()


def test_reduced_level_errors(jt):
    e = synth.encode(synth.texture(3, 32, 32), 70, 420)
    ctx = jt.Context(0, max_cache_blocks=64)
    with pytest.raises(jt.JTError):
        ctx.add_reduced_level(0, 0, 1, 1)  # no source
    ctx.upload(0, 0, e)
    for args in [(0, 0, 0, 1), (0, 0, 4, 1), (0, 0, 1, 0)]:
        with pytest.raises(jt.JTError):
            ctx.add_reduced_level(*args)
    ctx.add_reduced_level(0, 0, 1, 1)
    with pytest.raises(jt.JTError):
        ctx.add_reduced_level(0, 1, 1, 2)  # a reduced level is not a source
    ctx.close()
