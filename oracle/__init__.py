"""Oracle for the variable-rate (JPEG) texture path — TEST INFRASTRUCTURE ONLY.

A plain CPU restatement (``oracle.cpp``, single-threaded C++ compiled with
``-ffp-contract=off``) of what the path computes. Only ``tests/``,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline/reference leg may import
it; the CUDA library never calls it and shares no code with it.

Pinned parts (see ``tests/test_oracle_*.py``): zig-zag order, canonical Huffman
tables, entropy decode (round trips and a brute-force prefix decoder), random access
equals sequential decode, IDCT accuracy and DC constancy, colour conversion, mark /
compact / colourise against brute force and the full decode, the FP64 float chain's
gradient against central differences and the adjoint identity, the compact form and the
data-unit starts against the standard decode and a sequential parse, reduced levels
against scipy's orthonormal IDCT and box means, the clamped filter against the plain
filters, and the fp32 rasteriser against the generator's double-precision scene.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

INDEX_DTYPE = np.dtype([("bit_offset", "<u4"), ("dc_pred", "<i2", (3,))], align=False)


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.cpp")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-shared", "-fPIC",
                               "-o", _SO + ".tmp", src])
        os.replace(_SO + ".tmp", _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P, I64, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        L.jto_zigzag.argtypes = [P]
        L.jto_idct_matrix.argtypes = [P]
        L.jto_idct_raw.argtypes = [P, P, I]
        L.jto_idct_pixels.argtypes = [P, P, I]
        L.jto_ycc_to_rgb.argtypes = [P, P, I64]
        L.jto_huff_tables.argtypes = [P, P, P, P, P]
        L.jto_huff_decode_one.argtypes = [P, P, P, I, P]
        L.jto_decode_jfif.restype = P
        L.jto_decode_jfif.argtypes = [P, ctypes.c_size_t]
        L.jto_decoded_info.argtypes = [P, P]
        L.jto_decoded_copy.argtypes = [P, P, P, P, P, P, P, P]
        L.jto_decoded_free.argtypes = [P]
        L.jto_texset_new.restype = P
        L.jto_texset_free.argtypes = [P]
        L.jto_texset_add.restype = I64
        L.jto_texset_add.argtypes = [P, I, I, I, I, I, P, ctypes.c_uint64, ctypes.c_uint64, P, ctypes.c_uint64,
                                     P, P, P]
        L.jto_texset_add_compact.restype = I64
        L.jto_texset_add_compact.argtypes = [P, I, I, I, I, I, P, ctypes.c_uint64, P, ctypes.c_uint64, P,
                                             ctypes.c_uint64, P, ctypes.c_uint64, ctypes.c_uint64, P, P, P]
        L.jto_mcu_bits.argtypes = [P, I, I, P, P]
        L.jto_texset_set_du_offsets.restype = I
        L.jto_texset_set_du_offsets.argtypes = [P, I, I, P, ctypes.c_uint64]
        L.jto_du_starts.restype = I
        L.jto_du_starts.argtypes = [P, I, I, P]
        L.jto_texset_add_reduced.restype = I64
        L.jto_texset_add_reduced.argtypes = [P, I, I, I, I]
        L.jto_idct_pixels_n.argtypes = [P, P, I, I]
        L.jto_raster_scene.argtypes = [I, I, P, ctypes.c_uint64, I, P, P, P, I, P, I, P, P, P]
        L.jto_texset_decode_mcu.argtypes = [P, I, I, I, P]
        L.jto_mark.restype = I64
        L.jto_mark.argtypes = [P, P, P, P, I64, I, P]
        L.jto_compact.restype = I64
        L.jto_compact.argtypes = [P, I64, P]
        L.jto_colorize.restype = I64
        L.jto_colorize.argtypes = [P, P, P, P, I64, I, P]
        L.jto_texset_cached.restype = I64
        L.jto_texset_cached.argtypes = [P]
        L.jto_texset_clear_cache.argtypes = [P]
        L.jto_float_forward.argtypes = [P, I, I, I, P, P, I64, P]
        L.jto_float_vjp.argtypes = [I, I, I, P, P, I64, P, P]
        L.jto_float_loss_grad.restype = ctypes.c_double
        L.jto_float_loss_grad.argtypes = [P, I, I, I, P, P, I64, P, P]
        L.jto_float_fd.argtypes = [P, I, I, I, P, P, I64, P, P, I, ctypes.c_double, P]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def zigzag() -> np.ndarray:
    out = np.empty(64, np.int32)
    lib().jto_zigzag(_p(out))
    return out


def idct_matrix() -> np.ndarray:
    out = np.empty(64, np.int64)
    lib().jto_idct_matrix(_p(out))
    return out.reshape(8, 8)


def idct_raw(d: np.ndarray) -> np.ndarray:
    """Integer IDCT of dequantised blocks [..., 64] -> signed values before the +128 shift."""
    d = np.ascontiguousarray(d, np.int32).reshape(-1, 64)
    out = np.empty_like(d)
    lib().jto_idct_raw(_p(d), _p(out), d.shape[0])
    return out


def idct_pixels(d: np.ndarray) -> np.ndarray:
    d = np.ascontiguousarray(d, np.int32).reshape(-1, 64)
    out = np.empty(d.shape, np.uint8)
    lib().jto_idct_pixels(_p(d), _p(out), d.shape[0])
    return out


def idct_pixels_n(d: np.ndarray, n: int) -> np.ndarray:
    """Reduced-size IDCT: [blocks, n*n] pixels from the n x n lowest frequencies."""
    d = np.ascontiguousarray(d, np.int32).reshape(-1, 64)
    out = np.empty((d.shape[0], n * n), np.uint8)
    lib().jto_idct_pixels_n(_p(d), _p(out), d.shape[0], n)
    return out


def ycc_to_rgb(ycc: np.ndarray) -> np.ndarray:
    ycc = np.ascontiguousarray(ycc, np.uint8).reshape(-1, 3)
    out = np.empty_like(ycc)
    lib().jto_ycc_to_rgb(_p(ycc), _p(out), ycc.shape[0])
    return out


def huff_tables(bits, vals):
    bits = np.ascontiguousarray(bits, np.uint8)
    vals = np.ascontiguousarray(vals, np.uint8)
    mn = np.zeros(17, np.int32)
    mx = np.zeros(17, np.int32)
    vp = np.zeros(17, np.int32)
    rc = lib().jto_huff_tables(_p(bits), _p(vals), _p(mn), _p(mx), _p(vp))
    return rc, mn, mx, vp


def huff_decode_one(bits, vals, data: bytes):
    bits = np.ascontiguousarray(bits, np.uint8)
    vals = np.ascontiguousarray(vals, np.uint8)
    buf = np.frombuffer(bytes(data), np.uint8).copy()
    ln = ctypes.c_int(0)
    s = lib().jto_huff_decode_one(_p(bits), _p(vals), _p(buf), len(buf), ctypes.byref(ln))
    return s, ln.value


class Decoded:
    """Sequential decode of a baseline JFIF file."""

    def __init__(self, jfif: np.ndarray):
        L = lib()
        jfif = np.ascontiguousarray(jfif, np.uint8)
        h = L.jto_decode_jfif(_p(jfif), jfif.size)
        info = np.zeros(8, np.int64)
        L.jto_decoded_info(h, _p(info))
        self.status, self.width, self.height, self.sampling, self.mcus_x, self.mcus_y, nscan, self.coded_bits = (
            int(v) for v in info)
        if self.status != 0:
            L.jto_decoded_free(h)
            raise ValueError(f"oracle JFIF decode failed: {self.status}")
        ndu = 6 if self.sampling == 420 else 3
        n = self.mcus_x * self.mcus_y
        self.rgba = np.empty((self.height, self.width, 4), np.uint8)
        self.qcoef = np.empty((n, ndu, 64), np.int32)
        self.index = np.empty(n, INDEX_DTYPE)
        self.scan = np.empty(nscan, np.uint8)
        self.qt = np.empty((2, 64), np.uint16)
        self.huff_bits = np.empty((4, 16), np.uint8)
        self.huff_vals = np.empty((4, 256), np.uint8)
        L.jto_decoded_copy(h, _p(self.rgba), _p(self.qcoef), _p(self.index), _p(self.scan), _p(self.qt),
                           _p(self.huff_bits), _p(self.huff_vals))
        L.jto_decoded_free(h)


class TexSet:
    """Textures keyed by (texture id, mip level), decoded by random access.

    Levels get consecutive global MCU ids (gids) in registration order, the same rule
    the library states for uploads.
    """

    def __init__(self):
        self._h = lib().jto_texset_new()
        self.gid_base = {}
        self.nmcu = {}
        self.total = 0

    def __del__(self):
        if getattr(self, "_h", None):
            lib().jto_texset_free(self._h)
            self._h = None

    def add(self, tex: int, level: int, enc) -> int:
        """enc: anything with width/height/sampling/scan/scan_bits/index/qt/huff_bits/huff_vals."""
        scan = np.ascontiguousarray(enc.scan, np.uint8)
        idx = np.ascontiguousarray(enc.index)
        qt = np.ascontiguousarray(enc.qt, np.uint16)
        hb = np.ascontiguousarray(enc.huff_bits, np.uint8)
        hv = np.ascontiguousarray(enc.huff_vals, np.uint8)
        g = lib().jto_texset_add(self._h, tex, level, enc.width, enc.height, enc.sampling, _p(scan), scan.size,
                                 int(enc.scan_bits), _p(idx), idx.size, _p(qt), _p(hb), _p(hv))
        if g < 0:
            raise ValueError("oracle rejected texture level")
        self.gid_base[(tex, level)] = int(g)
        self.nmcu[(tex, level)] = int(idx.size)
        self.total = int(g) + int(idx.size)
        return int(g)

    def add_compact(self, tex: int, level: int, enc) -> int:
        """Registers the level's compact form (enc.compact: the paper's byte-aligned stream,
        two-level offset table and 12-bit DC records, Sec. 5.1 / 5.3)."""
        c = enc.compact
        scan = np.ascontiguousarray(c.scan, np.uint8)
        a = np.ascontiguousarray(c.abs, np.uint32)
        r = np.ascontiguousarray(c.rel, np.uint16)
        dc = np.ascontiguousarray(c.dc, np.uint32)
        qt = np.ascontiguousarray(enc.qt, np.uint16)
        hb = np.ascontiguousarray(enc.huff_bits, np.uint8)
        hv = np.ascontiguousarray(enc.huff_vals, np.uint8)
        n = enc.mcus_x * enc.mcus_y
        g = lib().jto_texset_add_compact(self._h, tex, level, enc.width, enc.height, enc.sampling, _p(scan),
                                         scan.size, _p(a), a.size, _p(r), r.size, _p(dc), dc.size, n, _p(qt),
                                         _p(hb), _p(hv))
        if g < 0:
            raise ValueError("oracle rejected compact texture level")
        self.gid_base[(tex, level)] = int(g)
        self.nmcu[(tex, level)] = n
        self.total = int(g) + n
        return int(g)

    def add_reduced(self, tex: int, src_level: int, reduce: int, level: int) -> int:
        """Registers `level` as the reduced-resolution decode (1/2^reduce, reduce 1..3) of
        the registered level `src_level` (the mip alternative of Sec. 7)."""
        g = lib().jto_texset_add_reduced(self._h, tex, src_level, reduce, level)
        if g < 0:
            raise ValueError("oracle rejected reduced level")
        n = self.nmcu[(tex, src_level)]
        self.gid_base[(tex, level)] = int(g)
        self.nmcu[(tex, level)] = n
        self.total = int(g) + n
        return int(g)

    def set_du_offsets(self, tex: int, level: int, offs) -> None:
        """Data-unit starts [mcu][ndu - 1] (bits from each MCU's first bit) for a standard-form
        level: its MCUs are then decoded data unit by data unit."""
        o = np.ascontiguousarray(offs, np.uint16).reshape(-1)
        if lib().jto_texset_set_du_offsets(self._h, tex, level, _p(o), o.size) != 0:
            raise ValueError("oracle rejected data-unit offsets")

    def du_starts(self, tex: int, level: int, ndu: int) -> np.ndarray:
        """The data-unit starts a sequential decode finds, [mcu][ndu - 1]."""
        out = np.empty((self.nmcu[(tex, level)], ndu - 1), np.int64)
        if lib().jto_du_starts(self._h, tex, level, _p(out)) != 0:
            raise ValueError("corrupt stream or compact level")
        return out

    def mcu_bits(self, tex: int, level: int):
        """Per MCU of a standard-form level: (coded bits, bits of its first luma DC and its
        chroma DCs), from a sequential decode."""
        n = self.nmcu[(tex, level)]
        bits = np.empty(n, np.int64)
        dcb = np.empty(n, np.int64)
        if lib().jto_mcu_bits(self._h, tex, level, _p(bits), _p(dcb)) != 0:
            raise ValueError("corrupt stream or compact level")
        return bits, dcb

    def decode_mcu(self, tex: int, level: int, mcu: int, mw: int) -> np.ndarray:
        tile = np.empty((mw, mw, 4), np.uint8)
        rc = lib().jto_texset_decode_mcu(self._h, tex, level, mcu, _p(tile))
        if rc != 0:
            raise ValueError("corrupt MCU")
        return tile

    def mark(self, gb, filter: int) -> np.ndarray:
        flags = np.zeros(self.total, np.uint8)
        uv = np.ascontiguousarray(gb.uv, np.float32)
        t = np.ascontiguousarray(gb.tex_id, np.uint16)
        m = np.ascontiguousarray(gb.mip, np.uint8)
        bad = lib().jto_mark(self._h, _p(uv), _p(t), _p(m), t.size, filter, _p(flags))
        if bad:
            raise ValueError(f"{bad} pixels name missing texture levels")
        return flags

    @staticmethod
    def compact(flags: np.ndarray) -> np.ndarray:
        flags = np.ascontiguousarray(flags, np.uint8)
        out = np.empty(flags.size, np.uint32)
        n = lib().jto_compact(_p(flags), flags.size, _p(out))
        return out[:n].copy()

    def colorize(self, uv, tex, mip, filter: int) -> np.ndarray:
        uv = np.ascontiguousarray(uv, np.float32)
        tex = np.ascontiguousarray(tex, np.uint16)
        mip = np.ascontiguousarray(mip, np.uint8)
        out = np.empty(tex.shape + (4,), np.uint8)
        bad = lib().jto_colorize(self._h, _p(uv), _p(tex), _p(mip), tex.size, filter, _p(out))
        if bad:
            raise ValueError(f"{bad} pixels could not be resolved")
        return out

    def cached(self) -> int:
        return int(lib().jto_texset_cached(self._h))

    def clear_cache(self):
        lib().jto_texset_clear_cache(self._h)


def scene_params(d) -> np.ndarray:
    """The 20 fp32 camera and frame parameters of a scene description, in the order the
    rasterisers take them."""
    return np.concatenate([d.cam, d.rot, np.array([d.ax, d.ay, d.tan_x, d.tan_y, d.max_t, d.kx, d.ky, d.shift],
                                                   np.float32)]).astype(np.float32)


def raster_scene(d):
    """G-buffer (uv, tex_id, mip) of a scene description (fp32, operations in the order the
    scene's renderer takes them)."""
    W, H = d.width, d.height
    uv = np.empty((H, W, 2), np.float32)
    tex = np.empty((H, W), np.uint16)
    mip = np.empty((H, W), np.uint8)
    prm = scene_params(d)
    tw = np.ascontiguousarray(d.tex_w, np.int32)
    th = np.ascontiguousarray(d.tex_h, np.int32)
    tl = np.ascontiguousarray(d.tex_levels, np.int32)
    q = np.ascontiguousarray(d.quads)
    lib().jto_raster_scene(W, H, _p(prm), d.cell_seed, tw.size, _p(tw), _p(th), _p(tl), int(d.use_mips),
                           q.ctypes.data if q.size else None, q.size, _p(uv), _p(tex), _p(mip))
    return uv, tex, mip


def texset_from(ts, compact: bool = False) -> TexSet:
    """Oracle texture set registered in the same (texture-major, level-minor) order, in the
    standard or the compact form."""
    o = TexSet()
    for t, l, e in ts.uploads():
        (o.add_compact if compact else o.add)(t, l, e)
    return o


# ---------------------------------------------------------------------------------------
# FP64 float chain
# ---------------------------------------------------------------------------------------

def float_forward(coef: np.ndarray, gb) -> np.ndarray:
    coef = np.ascontiguousarray(coef, np.float32)
    T, my, mx = coef.shape[:3]
    uv = np.ascontiguousarray(gb.uv, np.float32)
    tex = np.ascontiguousarray(gb.tex_id, np.uint16)
    F = np.empty(tex.shape + (3,), np.float64)
    lib().jto_float_forward(_p(coef), T, mx * 16, my * 16, _p(uv), _p(tex), tex.size, _p(F))
    return F


def float_vjp(shape, gb, g: np.ndarray) -> np.ndarray:
    T, my, mx = shape[:3]
    uv = np.ascontiguousarray(gb.uv, np.float32)
    tex = np.ascontiguousarray(gb.tex_id, np.uint16)
    g = np.ascontiguousarray(g, np.float64)
    out = np.empty(tuple(shape), np.float64)
    lib().jto_float_vjp(T, mx * 16, my * 16, _p(uv), _p(tex), tex.size, _p(g), _p(out))
    return out


def float_loss_grad(coef: np.ndarray, gb, target: np.ndarray, want_grad: bool = True):
    coef = np.ascontiguousarray(coef, np.float32)
    T, my, mx = coef.shape[:3]
    uv = np.ascontiguousarray(gb.uv, np.float32)
    tex = np.ascontiguousarray(gb.tex_id, np.uint16)
    target = np.ascontiguousarray(target, np.float32)
    grad = np.empty(coef.shape, np.float64) if want_grad else None
    L = lib().jto_float_loss_grad(_p(coef), T, mx * 16, my * 16, _p(uv), _p(tex), tex.size, _p(target),
                                  _p(grad))
    return L, grad


def float_fd(coef: np.ndarray, gb, target: np.ndarray, idx: np.ndarray, h: float = 1.0) -> np.ndarray:
    coef = np.ascontiguousarray(coef, np.float32)
    T, my, mx = coef.shape[:3]
    uv = np.ascontiguousarray(gb.uv, np.float32)
    tex = np.ascontiguousarray(gb.tex_id, np.uint16)
    target = np.ascontiguousarray(target, np.float32)
    idx = np.ascontiguousarray(idx, np.int64)
    out = np.empty(idx.size, np.float64)
    lib().jto_float_fd(_p(coef), T, mx * 16, my * 16, _p(uv), _p(tex), tex.size, _p(target), _p(idx), idx.size,
                       h, _p(out))
    return out
