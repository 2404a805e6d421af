"""The batched-view workload (8 views over the 64 scene textures): their needed-block counts
span more than 50x, as the batched-frame measurement requires (a view that looks mostly at
the sky next to 4K and VR views).

The needed set is counted with the mark rule restated in numpy (bilinear taps at texel
centres, repeat wrap, 16 x 16 MCUs of 4:2:0 levels); the sizes come from the texture draws,
so nothing is encoded."""

import numpy as np

import synth


def needed_count(gb: synth.GBuffer, sizes) -> int:
    t = gb.tex_id.reshape(-1).astype(np.int64)
    m = gb.mip.reshape(-1).astype(np.int64)
    uv = gb.uv.reshape(-1, 2)
    ok = t != 0xFFFF
    t, m, u, v = t[ok], m[ok], uv[ok, 0], uv[ok, 1]
    W = np.array([s[0] for s in sizes], np.int64)[t]
    H = np.array([s[1] for s in sizes], np.int64)[t]
    w, h = np.maximum(1, W >> m), np.maximum(1, H >> m)
    xs = (u * w.astype(np.float32)).astype(np.float32) - np.float32(0.5)  # fp32 product, then - 1/2
    ys = (v * h.astype(np.float32)).astype(np.float32) - np.float32(0.5)
    x0 = np.floor(xs).astype(np.int64) % w
    y0 = np.floor(ys).astype(np.int64) % h
    keys = []
    for xx in (x0, (x0 + 1) % w):
        for yy in (y0, (y0 + 1) % h):
            keys.append((((t << 4) | m) << 40) | ((yy >> 4) << 20) | (xx >> 4))
    return int(np.unique(np.concatenate(keys)).size)


def test_eight_views_span_more_than_50x():
    sizes, _ = synth.scene_draws()
    nlevels = [int(np.log2(s[0])) + 1 for s in sizes]  # full chains down to 1 x 1
    views = synth.eight_views_for(sizes, nlevels)
    assert [(v.width, v.height) for v in views] == [(1280, 720), (1920, 1080), (2560, 1440), (3840, 2160)] + \
        [(2064, 2208)] * 4
    counts = [needed_count(v, sizes) for v in views]
    assert min(counts) > 0
    assert max(counts) / min(counts) > 50, counts
