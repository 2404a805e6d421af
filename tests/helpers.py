"""Helpers shared by the GPU parity tests (imported by test modules, not a test itself)."""

from __future__ import annotations

import bisect

import numpy as np

import oracle
import synth


class GidMap:
    """gid -> (tex, level, Encoded, mcu) under the upload-order rule of jt_upload_texture."""

    def __init__(self, ts):
        self.bases, self.items = [], []
        g = 0
        for t, l, e in ts.uploads():
            self.bases.append(g)
            self.items.append((t, l, e))
            g += e.nmcu
        self.total = g

    def __call__(self, gid: int):
        i = bisect.bisect_right(self.bases, gid) - 1
        t, l, e = self.items[i]
        return t, l, e, gid - self.bases[i]


def texel_grid_gbuffer(w: int, h: int, tex: int = 0, level: int = 0) -> synth.GBuffer:
    """One pixel at the centre of every texel of a w x h level: marks every MCU."""
    xs, ys = np.meshgrid(np.arange(w), np.arange(h))
    uv = np.stack([(xs + 0.5) / w, (ys + 0.5) / h], axis=-1).astype(np.float32)
    return synth.GBuffer(w, h, uv, np.full((h, w), tex, np.uint16), np.full((h, w), level, np.uint8))


def concat_gbuffers(gbs) -> synth.GBuffer:
    """Stacks G-buffers of equal width vertically."""
    W = gbs[0].width
    assert all(g.width == W for g in gbs)
    return synth.GBuffer(W, sum(g.height for g in gbs), np.concatenate([g.uv for g in gbs]),
                         np.concatenate([g.tex_id for g in gbs]), np.concatenate([g.mip for g in gbs]))


def check_tiles(ctx, o: oracle.TexSet, gm: GidMap, gids) -> int:
    """Every listed gid's decoded tile equals the oracle's random-access decode."""
    n = 0
    for gid in gids:
        t, l, e, mcu = gm(int(gid))
        mw = 16 if e.sampling == 420 else 8
        got = ctx.tile(int(gid), e.sampling)
        ref = o.decode_mcu(t, l, mcu, mw)
        if not np.array_equal(got, ref):
            diff = np.argwhere(got != ref)
            raise AssertionError(f"gid {gid} (tex {t} level {l} mcu {mcu}) differs at {diff[:5].tolist()}")
        n += 1
    return n


def frame(ctx, dgb, filt, torch):
    out = torch.empty((dgb.height, dgb.width, 4), dtype=torch.uint8, device="cuda")
    ctx.mark(dgb, filt)
    ctx.decode()
    ctx.colorize(dgb, filt, out)
    return out


def mcu_grid_gbuffer(ts, width: int = 2048) -> synth.GBuffer:
    """One pixel at a texel of every MCU of every uploaded level (nearest filtering marks each
    MCU exactly once), packed row-major into a G-buffer `width` pixels wide (tail empty)."""
    uvs, texs, mips = [], [], []
    for t, l, e in ts.uploads():
        mw = 16 if e.sampling == 420 else 8
        mx, my = -(-e.width // mw), -(-e.height // mw)
        gx, gy = np.meshgrid(np.arange(mx), np.arange(my))
        tx = np.minimum(gx * mw + mw // 2, e.width - 1)
        ty = np.minimum(gy * mw + mw // 2, e.height - 1)
        uvs.append(np.stack([(tx + 0.5) / e.width, (ty + 0.5) / e.height], -1).reshape(-1, 2))
        texs.append(np.full(mx * my, t, np.uint16))
        mips.append(np.full(mx * my, l, np.uint8))
    uv = np.concatenate(uvs).astype(np.float32)
    n = uv.shape[0]
    h = -(-n // width)
    U = np.zeros((h * width, 2), np.float32)
    T = np.full(h * width, 0xFFFF, np.uint16)
    M = np.zeros(h * width, np.uint8)
    U[:n], T[:n], M[:n] = uv, np.concatenate(texs), np.concatenate(mips)
    return synth.GBuffer(width, h, U.reshape(h, width, 2), T.reshape(h, width), M.reshape(h, width))


def set_short_lists(ctx, on: int):
    """Short work lists decoded MCU by MCU by whole warps (1) or one MCU per lane (0)."""
    t = ctx.tuning()
    t["decode_short_lists"] = int(on)
    ctx.set_tuning(**t)
