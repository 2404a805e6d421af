"""Seeded synthetic inputs for the variable-rate (JPEG) texture path.

This module is the only code that both the CUDA path and the oracle consume. It makes
textures, mip chains, baseline-JPEG encodings (JFIF file, unstuffed entropy stream,
per-MCU index of bit offset + DC predictors, quantisation and Huffman tables) and
deferred G-buffers (uv, texture id, mip level), all from explicit seeds. It contains
none of the decode-side arithmetic (Huffman decoding, IDCT, colour conversion, MCU
marking, texel lookup).

The native part (``synth.cpp``) is compiled by :func:`build`.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_lib = None

# Config seeds: 0x25100816 + k for workload k (k = 1..5).
SEED_BASE = 0x25100816

INDEX_DTYPE = np.dtype([("bit_offset", "<u4"), ("dc_pred", "<i2", (3,))], align=False)
assert INDEX_DTYPE.itemsize == 10


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "synth.cpp")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(
            ["g++", "-std=c++17", "-O2", "-shared", "-fPIC", "-o", _SO + ".tmp", src]
        )
        os.replace(_SO + ".tmp", _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        L.syn_mix_seed.restype = ctypes.c_uint64
        L.syn_mix_seed.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        L.syn_texture.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, P]
        L.syn_mip_down.argtypes = [P, ctypes.c_int, ctypes.c_int, P]
        L.syn_quality_tables.argtypes = [ctypes.c_int, P]
        L.syn_standard_huffman.argtypes = [P, P, P]
        L.syn_huffman_codes.argtypes = [P, P, P, P]
        L.syn_zigzag.argtypes = [P]
        L.syn_jpeg_encode_rgb.restype = P
        L.syn_jpeg_encode_rgb.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.syn_jpeg_encode_coefs.restype = P
        L.syn_jpeg_encode_coefs.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.syn_jpeg_info.argtypes = [P, P]
        L.syn_jpeg_copy.argtypes = [P, P, P, P, P, P, P, P]
        L.syn_jpeg_free.argtypes = [P]
        L.syn_jpeg_compact_info.argtypes = [P, P]
        L.syn_jpeg_du_count.restype = ctypes.c_int64
        L.syn_jpeg_du_count.argtypes = [P]
        L.syn_jpeg_du_copy.argtypes = [P, P]
        L.syn_jpeg_symbols_copy.argtypes = [P, P]
        L.syn_jpeg_compact_copy.argtypes = [P, P, P, P, P]
        L.syn_gbuffer_affine.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int, P, P, P]
        L.syn_gbuffer_scene.argtypes = [
            ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_uint64,
            ctypes.c_double, ctypes.c_int, P, P, P, ctypes.c_int, P, P, P]
        L.syn_noise_image.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, P]
        L.syn_scene_quads.restype = ctypes.c_int
        L.syn_scene_quads.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, P, P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def mix_seed(seed: int, a: int, b: int) -> int:
    return int(lib().syn_mix_seed(seed & (2**64 - 1), a & (2**64 - 1), b & (2**64 - 1)))


def texture(seed: int, w: int, h: int) -> np.ndarray:
    """RGB8 [h, w, 3]: 1/f value noise mixed by a random 3x3 matrix + 24 solid rectangles."""
    out = np.empty((h, w, 3), np.uint8)
    lib().syn_texture(seed, w, h, _p(out))
    return out


def mip_down(rgb: np.ndarray) -> np.ndarray:
    h, w, _ = rgb.shape
    rgb = np.ascontiguousarray(rgb)
    out = np.empty((max(1, h // 2), max(1, w // 2), 3), np.uint8)
    lib().syn_mip_down(_p(rgb), w, h, _p(out))
    return out


def mip_chain(rgb: np.ndarray, levels: int | None = None) -> list[np.ndarray]:
    """Level 0 = rgb, then 2x2 box downsampling to 1x1 (or `levels` levels)."""
    out = [rgb]
    while (levels is None and (out[-1].shape[0] > 1 or out[-1].shape[1] > 1)) or (
        levels is not None and len(out) < levels
    ):
        out.append(mip_down(out[-1]))
    return out


def quality_tables(q: int) -> np.ndarray:
    out = np.empty((2, 64), np.uint16)
    lib().syn_quality_tables(q, _p(out))
    return out


def standard_huffman():
    """(bits[4,16], vals[4,256], nvals[4]) for DC-Y, AC-Y, DC-C, AC-C."""
    bits = np.zeros((4, 16), np.uint8)
    vals = np.zeros((4, 256), np.uint8)
    nv = np.zeros(4, np.int32)
    lib().syn_standard_huffman(_p(bits), _p(vals), _p(nv))
    return bits, vals, nv


def encoder_codes(bits: np.ndarray, vals: np.ndarray):
    """Encoder's (code[256], len[256]) table for one Huffman spec."""
    bits = np.ascontiguousarray(bits, np.uint8)
    vals = np.ascontiguousarray(vals, np.uint8)
    code = np.zeros(256, np.uint16)
    ln = np.zeros(256, np.uint8)
    lib().syn_huffman_codes(_p(bits), _p(vals), _p(code), _p(ln))
    return code, ln


def zigzag() -> np.ndarray:
    out = np.empty(64, np.int32)
    lib().syn_zigzag(_p(out))
    return out


@dataclass
class Compact:
    """The paper's compact random-access form of one level (Sec. 5.1 indexing table, the DC
    records of Sec. 5.3): every MCU starts on a byte of `scan`; the first luma DC and both
    chroma DCs are not in the stream but in `dc` as 12-bit two's-complement values (bits
    36 m + 12 c of the little-endian bit array, c = Y, Cb, Cr); MCU 9 j starts at byte
    abs[j] and MCU 9 j + i (i = 1..8) at abs[j] + rel[8 j + i - 1]."""

    scan: np.ndarray  # uint8, byte-aligned MCUs padded with 1-bits
    abs: np.ndarray  # uint32 [ceil(n / 9)]
    rel: np.ndarray  # uint16 [8 ceil(n / 9)]
    dc: np.ndarray  # uint32 [ceil(36 n / 32)]
    dc_bits_removed: int  # bits the absolute DCs took in the standard stream
    pad_bits: int  # alignment bits


@dataclass
class Encoded:
    """One encoded texture level (what `jt_upload_texture` takes, plus the JFIF file)."""

    width: int
    height: int
    sampling: int  # 420 or 444
    mcus_x: int
    mcus_y: int
    quality: int
    jfif: np.ndarray  # uint8, complete baseline JPEG file
    scan: np.ndarray  # uint8, unstuffed entropy-coded segment
    scan_bits: int  # number of coded bits in `scan`
    index: np.ndarray  # INDEX_DTYPE [mcus_y*mcus_x]
    qt: np.ndarray  # uint16 [2, 64] natural order
    huff_bits: np.ndarray  # uint8 [4, 16]
    huff_vals: np.ndarray  # uint8 [4, 256]
    qcoef: np.ndarray | None = None  # int16 [nmcu, ndu, 64] natural order
    compact: Compact | None = None  # the paper's compact form (when asked for)
    du_offsets: np.ndarray | None = None  # uint16 [nmcu, ndu - 1]: data-unit starts within each MCU
    symbols: np.ndarray | None = None  # uint16 [nmcu]: Huffman symbols (DC, AC, ZRL, EOB) per MCU

    @property
    def nmcu(self) -> int:
        return self.mcus_x * self.mcus_y

    @property
    def ndu(self) -> int:
        return 6 if self.sampling == 420 else 3


def _collect_compact(h) -> Compact:
    info = np.zeros(7, np.int64)
    lib().syn_jpeg_compact_info(h, _p(info))
    if info[0] != 0:
        raise ValueError("coefficients do not fit the compact form (a DC outside 12 bits)")
    scan = np.empty(int(info[1]), np.uint8)
    a = np.empty(int(info[2]), np.uint32)
    r = np.empty(int(info[3]), np.uint16)
    dc = np.empty(int(info[4]), np.uint32)
    lib().syn_jpeg_compact_copy(h, _p(scan), _p(a), _p(r), _p(dc))
    return Compact(scan, a, r, dc, int(info[5]), int(info[6]))


def _collect(h, quality, keep, compact=False) -> Encoded:
    L = lib()
    info = np.zeros(10, np.int64)
    L.syn_jpeg_info(h, _p(info))
    if info[0] != 0:
        L.syn_jpeg_free(h)
        raise ValueError("encoder rejected the coefficients (category out of range)")
    w, hh, samp, mx, my, nj, ns, nbits, nidx = (int(v) for v in info[1:])
    jfif = np.empty(nj, np.uint8)
    scan = np.empty(ns, np.uint8)
    index = np.empty(nidx, INDEX_DTYPE)
    qt = np.empty((2, 64), np.uint16)
    bits = np.empty((4, 16), np.uint8)
    vals = np.empty((4, 256), np.uint8)
    ndu = 6 if samp == 420 else 3
    qc = np.empty((mx * my, ndu, 64), np.int16) if keep else None
    L.syn_jpeg_copy(h, _p(jfif), _p(scan), _p(index), _p(qt), _p(bits), _p(vals),
                    _p(qc) if keep else None)
    try:
        cp = _collect_compact(h) if compact else None
        du = np.empty(int(L.syn_jpeg_du_count(h)), np.uint16)
        L.syn_jpeg_du_copy(h, _p(du))
        sym = np.empty(mx * my, np.uint16)
        L.syn_jpeg_symbols_copy(h, _p(sym))
    finally:
        L.syn_jpeg_free(h)
    return Encoded(w, hh, samp, mx, my, quality, jfif, scan, nbits, index, qt, bits, vals, qc, cp,
                   du.reshape(mx * my, ndu - 1), sym)


def encode(rgb: np.ndarray, quality: int, sampling: int = 420, keep_coefs: bool = False,
           compact: bool = False) -> Encoded:
    """Baseline JPEG of an RGB8 image; `compact` also returns the paper's compact form."""
    rgb = np.ascontiguousarray(rgb, np.uint8)
    h, w, _ = rgb.shape
    hnd = lib().syn_jpeg_encode_rgb(_p(rgb), w, h, quality, sampling, int(keep_coefs))
    if not hnd:
        raise ValueError("bad encoder arguments")
    return _collect(hnd, quality, keep_coefs, compact)


def encode_coefs(qcoef: np.ndarray, mcus_x: int, mcus_y: int, sampling: int, quality: int = 75,
                 compact: bool = False) -> Encoded:
    """Entropy-codes given quantised blocks [nmcu, ndu, 64] (natural order)."""
    qcoef = np.ascontiguousarray(qcoef, np.int16)
    hnd = lib().syn_jpeg_encode_coefs(_p(qcoef), mcus_x, mcus_y, sampling, quality)
    e = _collect(hnd, quality, False, compact)
    e.qcoef = qcoef.copy()
    return e


@dataclass
class GBuffer:
    width: int
    height: int
    uv: np.ndarray  # float32 [H, W, 2]
    tex_id: np.ndarray  # uint16 [H, W], 0xFFFF = empty
    mip: np.ndarray  # uint8 [H, W]

    @property
    def npx(self) -> int:
        return self.width * self.height


def gbuffer_affine(W: int, H: int, angle_deg: float = 17.0, scale: float = 1.3, tex: int = 0) -> GBuffer:
    uv = np.empty((H, W, 2), np.float32)
    t = np.empty((H, W), np.uint16)
    m = np.empty((H, W), np.uint8)
    lib().syn_gbuffer_affine(W, H, angle_deg, scale, tex, _p(uv), _p(t), _p(m))
    return GBuffer(W, H, uv, t, m)


@dataclass
class Pose:
    cam: tuple = (0.0, 1.7, 0.0)
    yaw: float = 0.0
    pitch: float = -25.0
    vfov: float = 60.0
    quad_seed: int = 1
    quad_shift: float = 0.0


def gbuffer_scene(seed: int, W: int, H: int, sizes, levels, pose: Pose, nquads: int = 200,
                  use_mips: bool = True) -> GBuffer:
    sizes = list(sizes)
    tw = np.array([s[0] for s in sizes], np.int32)
    th = np.array([s[1] for s in sizes], np.int32)
    tl = np.array(levels, np.int32)
    uv = np.empty((H, W, 2), np.float32)
    t = np.empty((H, W), np.uint16)
    m = np.empty((H, W), np.uint8)
    lib().syn_gbuffer_scene(seed, W, H, pose.cam[0], pose.cam[1], pose.cam[2], pose.yaw, pose.pitch,
                            pose.vfov, nquads, pose.quad_seed, pose.quad_shift, len(sizes), _p(tw), _p(th),
                            _p(tl), int(use_mips), _p(uv), _p(t), _p(m))
    return GBuffer(W, H, uv, t, m)


# One quad of the scene as renderers take it (fp32 values rounded from the generator's
# doubles): corners and edge vectors in the reference frame, the inverse homography, the uv
# map, the texture and conservative inclusive pixel bounds.
QUAD_DTYPE = np.dtype([("cx", "<f4", 4), ("cy", "<f4", 4), ("ex", "<f4", 4), ("ey", "<f4", 4), ("h", "<f4", 9),
                       ("rep", "<f4"), ("cs", "<f4"), ("sn", "<f4"), ("ou", "<f4"), ("ov", "<f4"),
                       ("tex", "<i4"), ("x0", "<i4"), ("y0", "<i4"), ("x1", "<i4"), ("y1", "<i4")])


@dataclass
class SceneDesc:
    """The scene of `gbuffer_scene` as fp32 inputs for a renderer: a camera ray through pixel
    coordinate (px, py) is rot @ ((px * ax - 1) * tan_x, (1 - py * ay) * tan_y, -1); the
    ground y = 0 is hit at ray parameter t <= max_t; quads live in a reference frame of kx x ky
    units per pixel, shifted by `shift`; ground cells of 2 m take their texture and uv offset
    from mix_seed(cell_seed, cell x, cell z)."""

    width: int
    height: int
    cam: np.ndarray  # f32 [3]
    rot: np.ndarray  # f32 [9], row-major
    ax: float
    ay: float
    tan_x: float
    tan_y: float
    max_t: float
    kx: float
    ky: float
    shift: float
    cell_seed: int
    tex_w: np.ndarray  # i32 [ntex]
    tex_h: np.ndarray
    tex_levels: np.ndarray
    use_mips: bool
    quads: np.ndarray  # QUAD_DTYPE [nquads]


def scene_desc(seed: int, W: int, H: int, sizes, levels, pose: Pose, nquads: int = 200,
               use_mips: bool = True) -> SceneDesc:
    """The inputs a renderer needs to draw what `gbuffer_scene` draws with the same arguments."""
    f32 = np.float32
    th = np.tan(np.radians(pose.vfov) / 2.0)
    cp, sp = np.cos(np.radians(pose.pitch)), np.sin(np.radians(pose.pitch))
    cy, sy = np.cos(np.radians(pose.yaw)), np.sin(np.radians(pose.yaw))
    rp = np.array([[1, 0, 0], [0, cp, -sp], [0, sp, cp]])
    ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    rot = (ry @ rp).astype(f32).reshape(-1)
    ntex = len(sizes)
    raw = np.zeros((max(nquads, 1), 22), np.float64)
    tex = np.zeros(max(nquads, 1), np.int32)
    n = lib().syn_scene_quads(W, H, nquads, pose.quad_seed, ntex, _p(raw), _p(tex))
    Hn, Wn = 1000.0, 1000.0 * W / H
    kx, ky = Wn / W, Hn / H
    shift = pose.quad_shift * Wn
    q = np.zeros(n, QUAD_DTYPE)
    for k in range(n):
        cxd, cyd = raw[k, 0:4], raw[k, 4:8]
        q[k]["cx"], q[k]["cy"] = cxd.astype(f32), cyd.astype(f32)
        q[k]["ex"] = (np.roll(cxd, -1) - cxd).astype(f32)
        q[k]["ey"] = (np.roll(cyd, -1) - cyd).astype(f32)
        q[k]["h"] = raw[k, 8:17].astype(f32)
        q[k]["rep"], q[k]["cs"], q[k]["sn"], q[k]["ou"], q[k]["ov"] = raw[k, 17:22].astype(f32)
        q[k]["tex"] = tex[k]
        xs, ys = (cxd + shift) / kx, cyd / ky
        q[k]["x0"] = max(0, int(np.floor(xs.min())) - 1)
        q[k]["x1"] = min(W - 1, int(np.ceil(xs.max())) + 1)
        q[k]["y0"] = max(0, int(np.floor(ys.min())) - 1)
        q[k]["y1"] = min(H - 1, int(np.ceil(ys.max())) + 1)
    return SceneDesc(W, H, np.array(pose.cam, f32), rot, float(f32(2.0 / W)), float(f32(2.0 / H)),
                     float(f32(th * W / H)), float(f32(th)), 600.0, float(f32(kx)), float(f32(ky)),
                     float(f32(shift)), mix_seed(seed, 7, 0), np.array([s[0] for s in sizes], np.int32),
                     np.array([s[1] for s in sizes], np.int32), np.array(levels, np.int32), use_mips, q)


def noise_image(seed: int, W: int, H: int) -> np.ndarray:
    out = np.empty((H, W, 3), np.float32)
    lib().syn_noise_image(seed, W, H, _p(out))
    return out


# ---------------------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------------------

@dataclass
class TextureSet:
    """Encoded textures: levels[t][l] is an Encoded for texture t, mip level l."""

    levels: list = field(default_factory=list)

    @property
    def sizes(self):
        return [(lv[0].width, lv[0].height) for lv in self.levels]

    @property
    def nlevels(self):
        return [len(lv) for lv in self.levels]

    def total_mcus(self) -> int:
        return sum(e.nmcu for lv in self.levels for e in lv)

    def uploads(self):
        """(tex_id, level, Encoded) in upload order (texture-major, level-minor)."""
        for t, lv in enumerate(self.levels):
            for l, e in enumerate(lv):
                yield t, l, e


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def make_texture_set(seed: int, sizes, qualities, samplings, full_chain: bool = True,
                     keep_coefs: bool = False, threads: int | None = None, compact: bool = False) -> TextureSet:
    """Generates and encodes textures t (seeded by mix_seed(seed, 100, t)) with mip chains.

    Each mip level is produced from the previous RGB level by the 2x2 box filter and
    encoded separately at the texture's quality and sampling.
    """
    n = len(sizes)

    def one(t):
        w, h = sizes[t]
        rgb = texture(mix_seed(seed, 100, t), w, h)
        chain = mip_chain(rgb) if full_chain else [rgb]
        return [encode(c, int(qualities[t]), int(samplings[t]), keep_coefs, compact) for c in chain]

    with ThreadPoolExecutor(threads or _threads()) as ex:
        levels = list(ex.map(one, range(n)))
    return TextureSet(levels)


def small_scene():
    """512x512 texture, Q80, 4:2:0; 256x256 affine G-buffer (17 deg, x1.3), nearest."""
    seed = SEED_BASE + 1
    ts = make_texture_set(seed, [(512, 512)], [80], [420], full_chain=False)
    gb = gbuffer_affine(256, 256, 17.0, 1.3, 0)
    return ts, gb


def scene_draws(ntex: int = 64):
    """Sizes (uniform in {1024,2048,4096}^2) and qualities (uniform in [50,95]) of the
    64 scene textures, without encoding them."""
    seed = SEED_BASE + 2
    sizes, quals = [], []
    for t in range(ntex):
        s = mix_seed(seed, 200, t)
        sizes.append((1024 << (s % 3),) * 2)
        quals.append(50 + int((s >> 8) % 46))
    return sizes, quals


def scene_textures(ntex: int = 64, threads: int | None = None, compact: bool = False) -> TextureSet:
    """64 textures, sizes uniform in {1024,2048,4096}^2, Q uniform in [50,95], 4:2:0,
    full mip chains each level encoded separately."""
    sizes, quals = scene_draws(ntex)
    return make_texture_set(SEED_BASE + 2, sizes, quals, [420] * ntex, full_chain=True, threads=threads,
                            compact=compact)


def scene_pose() -> Pose:
    return Pose(cam=(0.0, 1.7, 0.0), yaw=20.0, pitch=-25.0, vfov=60.0,
                quad_seed=mix_seed(SEED_BASE + 2, 300, 0))


def scene_gbuffer(ts: TextureSet, W: int = 3840, H: int = 2160) -> GBuffer:
    return gbuffer_scene(SEED_BASE + 2, W, H, ts.sizes, ts.nlevels, scene_pose(), nquads=200)


def eight_views(ts: TextureSet):
    """8 views: 1280x720, 1920x1080, 2560x1440, 3840x2160 and VR stereo 2x(2064x2208) at two
    poses (eye separation 0.064 m). The 720p view pitches up 35 degrees, above the ground, and
    holds six screen quads, so that the views' needed-block counts span more than 50x (the
    tests check the span on the needed sets)."""
    return eight_views_for(ts.sizes, ts.nlevels)


def eight_views_for(sizes, nlevels):
    """eight_views from the textures' sizes and level counts alone."""
    seed = SEED_BASE + 3
    qs = mix_seed(seed, 300, 0)
    views = []
    flat = [((1280, 720), Pose((0.0, 1.7, 0.0), 10.0, 35.0, 60.0, qs, 0.0), 6),
            ((1920, 1080), Pose((3.0, 1.7, 5.0), 40.0, -20.0, 60.0, mix_seed(seed, 300, 1), 0.0), 200),
            ((2560, 1440), Pose((-4.0, 1.7, 2.0), -30.0, -30.0, 60.0, mix_seed(seed, 300, 2), 0.0), 200),
            ((3840, 2160), Pose((1.0, 1.7, -3.0), 75.0, -35.0, 60.0, mix_seed(seed, 300, 3), 0.0), 200)]
    for (w, h), p, nq in flat:
        views.append(gbuffer_scene(seed, w, h, sizes, nlevels, p, nquads=nq))
    for k, (yaw, pitch) in enumerate([(120.0, -30.0), (200.0, -40.0)]):
        base = np.array([2.0 * k, 1.7, -1.0 * k])
        right = np.array([np.cos(np.radians(yaw)), 0.0, -np.sin(np.radians(yaw))])
        qseed = mix_seed(seed, 310, k)
        for eye, sgn in enumerate((-1.0, 1.0)):
            cam = tuple(base + sgn * 0.032 * right)
            p = Pose(cam, yaw, pitch, 90.0, qseed, -sgn * 0.008)
            views.append(gbuffer_scene(seed, 2064, 2208, sizes, nlevels, p, nquads=200))
    return views


def motion_views(ts: TextureSet, W: int = 1920, H: int = 1080, ndir: int = 60, step_deg: float = 6.0,
                 stereo: bool = False, threads: int | None = None):
    """The motion test of the paper's caching evaluation: the camera of the 4K scene turns by
    `step_deg` per frame, `ndir` frames for a full turn. Returns one list of G-buffers per
    direction: one view, or with `stereo` two eyes 0.064 m apart with a 90 degree field of
    view (the VR variant)."""
    p0 = scene_pose()
    seed = SEED_BASE + 2
    jobs = []
    for k in range(ndir):
        yaw = p0.yaw + step_deg * k
        if not stereo:
            jobs.append((k, Pose(p0.cam, yaw, p0.pitch, p0.vfov, p0.quad_seed, 0.0)))
            continue
        right = np.array([np.cos(np.radians(yaw)), 0.0, -np.sin(np.radians(yaw))])
        for sgn in (-1.0, 1.0):
            cam = tuple(np.array(p0.cam) + sgn * 0.032 * right)
            jobs.append((k, Pose(cam, yaw, p0.pitch, 90.0, p0.quad_seed, -sgn * 0.008)))
    with ThreadPoolExecutor(threads or _threads()) as ex:
        gbs = list(ex.map(lambda j: gbuffer_scene(seed, W, H, ts.sizes, ts.nlevels, j[1], nquads=200), jobs))
    out = [[] for _ in range(ndir)]
    for (k, _), g in zip(jobs, gbs):
        out[k].append(g)
    return out


def full_decode_textures(ntex: int = 256, size: int = 4096, threads: int | None = None) -> TextureSet:
    """Full-decode stress: `ntex` textures size^2 at Q90; the first half 4:4:4, the second
    half 4:2:0; level 0 only."""
    seed = SEED_BASE + 4
    samp = [444 if t < ntex // 2 else 420 for t in range(ntex)]
    return make_texture_set(seed, [(size, size)] * ntex, [90] * ntex, samp, full_chain=False, threads=threads)


def coefficient_scene(ntex: int = 16, size: int = 2048, W: int = 1920, H: int = 1080):
    """Differentiable colourise: ntex textures size^2, 4:2:0, Q75, level 0 only, with the
    dequantised DCT coefficients as float32 [ntex, size/16, size/16, 6, 64]; a perspective
    plane G-buffer (no quads, level 0) and a seeded target frame [H, W, 3]."""
    seed = SEED_BASE + 5
    ts = make_texture_set(seed, [(size, size)] * ntex, [75] * ntex, [420] * ntex, full_chain=False,
                          keep_coefs=True)
    m = size // 16
    coef = np.empty((ntex, m, m, 6, 64), np.float32)
    for t, lv in enumerate(ts.levels):
        e = lv[0]
        q = np.empty((6, 64), np.float32)
        q[:4] = e.qt[0]
        q[4:] = e.qt[1]
        coef[t] = (e.qcoef.astype(np.float32) * q[None]).reshape(m, m, 6, 64)
    pose = Pose((0.0, 1.7, 0.0), 15.0, -25.0, 60.0, 0, 0.0)
    gb = gbuffer_scene(seed, W, H, [(size, size)] * ntex, [1] * ntex, pose, nquads=0, use_mips=False)
    target = noise_image(mix_seed(seed, 500, 0), W, H)
    return ts, coef, gb, target
