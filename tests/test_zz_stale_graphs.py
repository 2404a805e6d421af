"""GPU: a captured frame graph bakes the context's own tables in (level records, descriptors,
Huffman and quantisation sets, frame buffers, the block cache's arrays). An upload
reallocates them, so jt_graph_launch refuses a graph captured before it (JT_ERR_STATE,
nothing launched); a graph captured again renders the same frame. With the block cache on,
the capture after an upload starts the cache over before it captures."""

import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

JT_ERR_STATE = 7


@pytest.fixture(scope="module")
def jt():
    import paper_2510_08166_gb300 as m
    return m


@pytest.mark.parametrize("persistent", [False, True])
def test_graph_refused_after_an_upload(jt, persistent):
    sizes = [(64, 64), (256, 256), (512, 512)]
    ts = synth.make_texture_set(11, sizes, [60, 85, 75], [420, 444, 420])
    view = synth.gbuffer_scene(11, 320, 180, ts.sizes, ts.nlevels, synth.Pose(quad_seed=11), nquads=20)
    extra = synth.make_texture_set(12, [(64, 64)], [70], [420], full_chain=False)
    ctx = jt.Context(0, 1 << 15)
    ctx.upload_set(ts)
    if persistent:
        ctx.set_block_cache(True)
    dv = jt.DeviceGBuffer.from_host(view)
    out = torch.zeros((view.height, view.width, 4), dtype=torch.uint8, device="cuda")
    g = ctx.frame_graph([(dv, out)], 1)
    ctx.graph_launch(g)
    st = ctx.stats()
    assert st["needed_blocks"] > 0
    first = out.clone()

    ctx.upload(len(ts.levels), 0, extra.levels[0][0])  # a texture the view does not use
    out.zero_()
    with pytest.raises(jt.JTError) as e:
        ctx.graph_launch(g)
    assert e.value.status == JT_ERR_STATE
    torch.cuda.synchronize()
    assert int(out.sum()) == 0  # nothing ran
    ctx.graph_destroy(g)

    g2 = ctx.frame_graph([(dv, out)], 1)
    ctx.graph_launch(g2)
    st = ctx.stats()
    assert st["needed_blocks"] > 0  # the cache, if on, started over
    assert torch.equal(out, first)
    ctx.graph_destroy(g2)
    ctx.close()
