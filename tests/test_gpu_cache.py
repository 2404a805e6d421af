"""GPU: the cross-frame block cache (decoded MCUs stay resident between frames; a frame
decodes only what is needed and not resident, and evicts what it does not need).

Frames of a turning camera must give exactly the pixels of the per-frame mode (and of the
oracle within 1 LSB). The cache must hold exactly the frame's needed set, decode only the
needed MCUs not already resident, and keep every resident tile bit-exact."""

import numpy as np
import pytest

import oracle
import synth
from helpers import GidMap, check_tiles, frame

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def jt():
    import paper_2510_08166_gb300 as m
    return m


@pytest.fixture(scope="module")
def scene():
    sizes = [(256, 256), (512, 512), (1024, 1024), (128, 128)]
    ts = synth.make_texture_set(17, sizes, [70, 85, 60, 95], [420, 420, 444, 420])
    views = [synth.gbuffer_scene(17, 320, 192, ts.sizes, ts.nlevels,
                                 synth.Pose((0.0, 1.7, 0.0), 6.0 * k, -25.0, 60.0, 5, 0.0), nquads=12)
             for k in range(6)]  # the camera turns 6 degrees per frame
    return ts, views


def test_turning_camera_matches_per_frame_mode(jt, scene):
    ts, views = scene
    o = oracle.texset_from(ts)
    gm = GidMap(ts)
    per = jt.Context(0, 1 << 14)
    per.upload_set(ts)
    cached = jt.Context(0, 1 << 14)
    cached.upload_set(ts)
    cached.set_block_cache(True)
    previous = set()
    for k, v in enumerate(views):
        dv = jt.DeviceGBuffer.from_host(v)
        a = frame(per, dv, 1, torch)
        per.stats()
        b = frame(cached, dv, 1, torch)
        st = cached.stats()
        assert torch.equal(a, b), k
        ref = o.colorize(v.uv, v.tex_id, v.mip, 1)
        assert np.abs(b.cpu().numpy().astype(np.int32) - ref.astype(np.int32)).max() <= 1
        needed = set(o.compact(o.mark(v, 1)).tolist())
        assert st["visible_blocks"] == len(needed)
        assert st["resident_blocks"] == len(needed)  # what the frame does not need is evicted
        assert st["needed_blocks"] == len(needed - previous)  # decoded: needed and not resident
        decoded = cached.work_list()
        assert set(decoded.tolist()) == needed - previous
        check_tiles(cached, o, gm, sorted(needed))  # resident tiles, old and new, bit-exact
        previous = needed
    per.close()
    cached.close()


def test_graph_replay_decodes_nothing_new(jt, scene):
    ts, views = scene
    ctx = jt.Context(0, 1 << 14)
    ctx.upload_set(ts)
    ctx.set_block_cache(True)
    dv = jt.DeviceGBuffer.from_host(views[2])
    out = torch.zeros((views[2].height, views[2].width, 4), dtype=torch.uint8, device="cuda")
    g = ctx.frame_graph([(dv, out)], 1)
    ctx.graph_launch(g)
    st = ctx.stats()
    first = out.clone()
    assert st["needed_blocks"] == st["visible_blocks"] > 0
    for _ in range(3):
        ctx.graph_launch(g)
        st = ctx.stats()
        assert st["needed_blocks"] == 0 and st["evicted_blocks"] == 0
        assert torch.equal(out, first)
    ctx.graph_destroy(g)
    # back to per-frame mode: everything needed is decoded again, same pixels
    ctx.set_block_cache(False)
    again = frame(ctx, dv, 1, torch)
    st = ctx.stats()
    assert st["needed_blocks"] == st["visible_blocks"] and torch.equal(again, first)
    ctx.close()


def test_cache_capacity_is_reported(jt, scene):
    ts, views = scene
    ctx = jt.Context(0, 64)  # 64 blocks; the frame needs more
    ctx.upload_set(ts)
    ctx.set_block_cache(True)
    frame(ctx, jt.DeviceGBuffer.from_host(views[0]), 1, torch)
    st = ctx.stats(check=False)
    assert st["status"] == 5 and st["error_bits"] & jt.DEVERR_CAPACITY
    with pytest.raises(jt.JTError):
        ctx.frame_plain([(jt.DeviceGBuffer.from_host(views[0]),
                          torch.zeros((views[0].height, views[0].width, 4), dtype=torch.uint8, device="cuda"))], 1)
    ctx.close()


def test_tight_cache_reuses_blocks_evicted_by_the_same_frame(jt, scene):
    """A cache exactly the size of the largest needed set: a frame's misses outnumber the
    blocks free when it starts, so some of them must take blocks the same frame evicts."""
    ts, views = scene
    o = oracle.texset_from(ts)
    gm = GidMap(ts)
    needed = [set(o.compact(o.mark(v, 1)).tolist()) for v in views]
    cap = max(len(n) for n in needed)
    order = list(range(len(views))) + list(range(len(views) - 2, -1, -1))  # forward, then back
    assert any(len(needed[a] | needed[b]) > cap for a, b in zip(order, order[1:]))
    per = jt.Context(0, 1 << 14)
    per.upload_set(ts)
    tight = jt.Context(0, cap)
    tight.upload_set(ts)
    tight.set_block_cache(True)
    previous = set()
    for k in order:
        dv = jt.DeviceGBuffer.from_host(views[k])
        a = frame(per, dv, 1, torch)
        per.stats()
        b = frame(tight, dv, 1, torch)
        st = tight.stats()  # raises on a capacity error
        assert torch.equal(a, b), k
        assert st["resident_blocks"] == len(needed[k])
        assert st["needed_blocks"] == len(needed[k] - previous)
        assert st["evicted_blocks"] == len(previous - needed[k])
        check_tiles(tight, o, gm, sorted(needed[k]))
        previous = needed[k]
    per.close()
    tight.close()
