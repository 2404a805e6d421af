"""GB300-native variable-rate (JPEG) texture path — Python binding of libjt.so.

The functions ``jt_*`` mirror the C ABI of ``include/jt.h`` one to one (argument
marshalling only; every step runs in the library's CUDA kernels). :class:`Context` wraps
them for convenience. PyTorch provides device memory and streams.

There is no CPU fallback: if the library cannot be built or loaded, importing the
binding raises.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = ["JTError", "Context", "DeviceGBuffer", "lib", "FILTER_NEAREST", "FILTER_BILINEAR",
           "FILTER_BILINEAR_CLAMP"]

FILTER_NEAREST = 0
FILTER_BILINEAR = 1
FILTER_BILINEAR_CLAMP = 2  # bilinear taps clamped to the nearest texel's MCU (Sec. 4.4)
MAX_VIEWS = 16
EMPTY_TEXTURE = 0xFFFF

STATUS = {0: "JT_OK", 1: "JT_ERR_INVALID_ARG", 2: "JT_ERR_CUDA", 3: "JT_ERR_OOM", 4: "JT_ERR_CORRUPT_STREAM",
          5: "JT_ERR_CAPACITY", 6: "JT_ERR_UNSUPPORTED", 7: "JT_ERR_STATE"}
DEVERR_CORRUPT, DEVERR_CAPACITY, DEVERR_MISSING, DEVERR_TIMEOUT = 1, 2, 4, 8


class JTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class jt_block_index(ctypes.Structure):
    _pack_ = 2
    _fields_ = [("bit_offset", ctypes.c_uint32), ("dc_pred", ctypes.c_int16 * 3)]


class jt_huff_spec(ctypes.Structure):
    _fields_ = [("bits", ctypes.c_uint8 * 16), ("vals", ctypes.c_uint8 * 256)]


class jt_gbuffer(ctypes.Structure):
    _fields_ = [("uv", ctypes.c_void_p), ("tex_id", ctypes.c_void_p), ("mip", ctypes.c_void_p),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class jt_scene(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("cam", ctypes.c_float * 3),
                ("rot", ctypes.c_float * 9), ("ax", ctypes.c_float), ("ay", ctypes.c_float),
                ("tan_x", ctypes.c_float), ("tan_y", ctypes.c_float), ("max_t", ctypes.c_float),
                ("kx", ctypes.c_float), ("ky", ctypes.c_float), ("shift", ctypes.c_float),
                ("cell_seed", ctypes.c_uint64), ("ntex", ctypes.c_int32), ("use_mips", ctypes.c_int32),
                ("tex_w", ctypes.c_void_p), ("tex_h", ctypes.c_void_p), ("tex_levels", ctypes.c_void_p),
                ("quads", ctypes.c_void_p), ("nquads", ctypes.c_int32), ("reserved", ctypes.c_int32)]


assert ctypes.sizeof(jt_scene) == 144


class jt_view(ctypes.Structure):
    _fields_ = [("g", jt_gbuffer), ("out_rgba", ctypes.c_void_p)]


class jt_stats(ctypes.Structure):
    _fields_ = [("needed_blocks", ctypes.c_uint64), ("cache_units", ctypes.c_uint64),
                ("capacity_units", ctypes.c_uint64), ("total_blocks", ctypes.c_uint64),
                ("levels", ctypes.c_uint32), ("error_bits", ctypes.c_uint32),
                ("visible_blocks", ctypes.c_uint64), ("resident_blocks", ctypes.c_uint64),
                ("evicted_blocks", ctypes.c_uint64)]


class jt_tuning(ctypes.Structure):
    _fields_ = [("decode_mcus_per_warp", ctypes.c_int32), ("decode_warps", ctypes.c_int32),
                ("decode_ctas_per_sm", ctypes.c_int32), ("pixel_threads", ctypes.c_int32),
                ("pixel_ctas_per_sm", ctypes.c_int32), ("decode_short_lists", ctypes.c_int32)]


assert ctypes.sizeof(jt_block_index) == 10

_P = ctypes.c_void_p
_U64 = ctypes.c_uint64
_I = ctypes.c_int
_SIGS = {
    "jt_create": [ctypes.POINTER(_P), _I, _U64],
    "jt_destroy": [_P],
    "jt_last_error": [_P],
    "jt_status_string": [_I],
    "jt_upload_texture": [_P, _I, _I, _I, _I, _I, _P, _U64, _U64, _P, _U64, _P, _P],
    "jt_upload_texture_compact": [_P, _I, _I, _I, _I, _I, _P, _U64, _P, _P, _P, _U64, _P, _P],
    "jt_add_reduced_level": [_P, _I, _I, _I, _I],
    "jt_raster_scene": [_P, _P, _P, _P],
    "jt_set_du_offsets": [_P, _I, _I, _P, _U64],
    "jt_mark": [_P, ctypes.POINTER(jt_gbuffer), _I, _P],
    "jt_decode": [_P, _P],
    "jt_colorize": [_P, ctypes.POINTER(jt_gbuffer), _I, _P, _P],
    "jt_get_stats": [_P, ctypes.POINTER(jt_stats)],
    "jt_frame": [_P, ctypes.POINTER(jt_view), _I, _I, _P],
    "jt_frame_graph": [_P, ctypes.POINTER(jt_view), _I, _I, _P, ctypes.POINTER(_P)],
    "jt_graph_launch": [_P, _P],
    "jt_graph_destroy": [_P],
    "jt_frame_plain": [_P, ctypes.POINTER(jt_view), _I, _I, _P],
    "jt_get_tuning": [_P, ctypes.POINTER(jt_tuning)],
    "jt_set_tuning": [_P, ctypes.POINTER(jt_tuning)],
    "jt_autotune": [_P, ctypes.POINTER(jt_view), _I, _I, _P, _I, ctypes.POINTER(jt_tuning),
                    ctypes.POINTER(ctypes.c_float)],
    "jt_profile": [_P, _I],
    "jt_profile_read": [_P, ctypes.POINTER(ctypes.c_float)],
    "jt_read_work_list": [_P, _P, _U64, ctypes.POINTER(_U64)],
    "jt_read_slots": [_P, _U64, _U64, _P],
    "jt_read_cache": [_P, _U64, _U64, _P],
    "jt_register_coeff_textures": [_P, _I, _I, _I, _I],
    "jt_colorize_float": [_P, ctypes.POINTER(jt_gbuffer), _P, _P, _P],
    "jt_colorize_backward": [_P, ctypes.POINTER(jt_gbuffer), _P, _P, _P],
    "jt_compact_static": [_P, ctypes.c_uint32, _P, _P, ctypes.c_uint32, _P, _P],
    "jt_set_block_cache": [_P, _I],
}

STATIC_COMPACT_MAX_FLAGS = 1 << 24  # JT_STATIC_COMPACT_MAX_FLAGS

_lib = None


def lib() -> ctypes.CDLL:
    """Loads (building first if needed) the in-tree libjt.so."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise ImportError(f"libjt.so was not built at {path}")
        L = ctypes.CDLL(path)
        for name, argtypes in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = argtypes
            f.restype = ctypes.c_char_p if name in ("jt_last_error", "jt_status_string") else ctypes.c_int
        _lib = L
    return _lib


def exported_names():
    return list(_SIGS)


# Module-level functions with the C ABI's names.
def _bind(name):
    def f(*args):
        return getattr(lib(), name)(*args)
    f.__name__ = name
    return f


for _n in _SIGS:
    globals()[_n] = _bind(_n)


def _stream(stream=None) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def compact_static(flags, slot, work, totals, stream=None) -> None:
    """jt_compact_static on torch CUDA tensors: flags uint8[n] (zeroed by the call), slot
    int32/uint32[n], work int32/uint32[cap], totals int32/uint32[3] = {count, units, error
    bits}. Asynchronous on `stream`; allocates nothing."""
    n = flags.numel()
    if n > STATIC_COMPACT_MAX_FLAGS:
        raise JTError(5, f"jt_compact_static takes at most {STATIC_COMPACT_MAX_FLAGS} flags, got {n}")
    for name, t, need in (("flags", flags, 1), ("slot", slot, 4), ("work", work, 4), ("totals", totals, 4)):
        if not t.is_cuda or not t.is_contiguous() or t.element_size() != need:
            raise JTError(1, f"{name} must be a contiguous CUDA tensor of {need}-byte elements")
    if slot.numel() < n or totals.numel() < 3:
        raise JTError(1, "slot needs n entries and totals 3")
    s = lib().jt_compact_static(flags.data_ptr(), n, slot.data_ptr(), work.data_ptr(), work.numel(),
                                totals.data_ptr(), _stream(stream))
    if s != 0:
        raise JTError(s, "jt_compact_static: " + lib().jt_status_string(s).decode())


class DeviceGBuffer:
    """A G-buffer resident in device memory (torch tensors), shaped [H, W(, 2)]."""

    def __init__(self, uv, tex_id, mip):
        import torch
        self.uv = uv
        self.tex_id = tex_id
        self.mip = mip
        self.height, self.width = int(tex_id.shape[0]), int(tex_id.shape[1])
        assert uv.dtype == torch.float32 and uv.is_contiguous() and tuple(uv.shape) == (self.height, self.width, 2)
        assert tex_id.dtype == torch.int16 and tex_id.is_contiguous()
        assert mip.dtype == torch.uint8 and mip.is_contiguous()

    @classmethod
    def from_host(cls, gb, device="cuda"):
        """From a host G-buffer with numpy uv float32 [H,W,2], tex_id uint16 [H,W], mip uint8 [H,W]."""
        import torch
        uv = torch.from_numpy(np.ascontiguousarray(gb.uv, np.float32)).to(device)
        tex = torch.from_numpy(np.ascontiguousarray(gb.tex_id, np.uint16).view(np.int16)).to(device)
        mip = torch.from_numpy(np.ascontiguousarray(gb.mip, np.uint8)).to(device)
        return cls(uv, tex, mip)

    @classmethod
    def empty(cls, width: int, height: int, device="cuda"):
        """Uninitialised device G-buffer (e.g. for jt_raster_scene to fill)."""
        import torch
        return cls(torch.empty((height, width, 2), dtype=torch.float32, device=device),
                   torch.empty((height, width), dtype=torch.int16, device=device),
                   torch.empty((height, width), dtype=torch.uint8, device=device))

    def c(self) -> jt_gbuffer:
        return jt_gbuffer(self.uv.data_ptr(), self.tex_id.data_ptr(), self.mip.data_ptr(), self.width, self.height)

    @property
    def npx(self) -> int:
        return self.width * self.height


def _huff_specs(bits: np.ndarray, vals: np.ndarray):
    specs = (jt_huff_spec * 4)()
    for t in range(4):
        ctypes.memmove(specs[t].bits, np.ascontiguousarray(bits[t], np.uint8).ctypes.data, 16)
        ctypes.memmove(specs[t].vals, np.ascontiguousarray(vals[t], np.uint8).ctypes.data, 256)
    return specs


class Context:
    """Owns a jt_ctx: uploaded textures, the block cache and per-frame buffers."""

    def __init__(self, device: int = 0, max_cache_blocks: int = 1 << 16):
        self._h = None
        h = ctypes.c_void_p()
        s = lib().jt_create(ctypes.byref(h), device, max_cache_blocks)
        if s != 0:
            raise JTError(s, "jt_create failed (no CUDA device, bad capacity or out of memory)")
        self._h = h
        self.device = device
        self._graphs = []

    def close(self):
        if self._h:
            for g in self._graphs:
                lib().jt_graph_destroy(g)
            self._graphs = []
            lib().jt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, s: int):
        if s != 0:
            raise JTError(s, lib().jt_last_error(self._h).decode())

    # ---- textures ----
    def upload(self, tex_id: int, level: int, enc) -> None:
        scan = np.ascontiguousarray(enc.scan, np.uint8)
        idx = np.ascontiguousarray(enc.index)
        qt = np.ascontiguousarray(enc.qt, np.uint16)
        self._check(lib().jt_upload_texture(self._h, tex_id, level, enc.width, enc.height, enc.sampling,
                                            scan.ctypes.data, scan.size, int(enc.scan_bits), idx.ctypes.data,
                                            idx.size, qt.ctypes.data, _huff_specs(enc.huff_bits, enc.huff_vals)))

    def upload_compact(self, tex_id: int, level: int, enc) -> None:
        """Uploads enc.compact: the paper's compact form (byte-aligned MCUs, two-level
        offset table, 12-bit DC records; Sec. 5.1, 5.3)."""
        c = enc.compact
        scan = np.ascontiguousarray(c.scan, np.uint8)
        a = np.ascontiguousarray(c.abs, np.uint32)
        r = np.ascontiguousarray(c.rel, np.uint16)
        dc = np.ascontiguousarray(c.dc, np.uint32)
        qt = np.ascontiguousarray(enc.qt, np.uint16)
        n = enc.mcus_x * enc.mcus_y
        if a.size != (n + 8) // 9 or r.size != 8 * a.size or dc.size != (36 * n + 31) // 32:
            raise JTError(1, "compact side-table sizes do not match the level")
        self._check(lib().jt_upload_texture_compact(self._h, tex_id, level, enc.width, enc.height, enc.sampling,
                                                    scan.ctypes.data, scan.size, a.ctypes.data, r.ctypes.data,
                                                    dc.ctypes.data, n, qt.ctypes.data,
                                                    _huff_specs(enc.huff_bits, enc.huff_vals)))

    def add_reduced_level(self, tex_id: int, src_level: int, reduce: int, level: int) -> None:
        """Registers `level` as the 1/2^reduce decode of the stored level `src_level` from its
        lowest frequencies (reduce 1..3; Sec. 7's mip alternative)."""
        self._check(lib().jt_add_reduced_level(self._h, tex_id, src_level, reduce, level))

    def raster_scene(self, d, gb: "DeviceGBuffer", stream=None) -> None:
        """Fills the device G-buffer `gb` with the scene description `d` (fields of
        jt_scene; d.quads a structured array laid out as jt_scene_quad)."""
        tw = np.ascontiguousarray(d.tex_w, np.int32)
        th = np.ascontiguousarray(d.tex_h, np.int32)
        tl = np.ascontiguousarray(d.tex_levels, np.int32)
        q = np.ascontiguousarray(d.quads)
        if q.size and q.dtype.itemsize != 140:
            raise JTError(1, "quads must be 140-byte jt_scene_quad records")
        sc = jt_scene(d.width, d.height, (ctypes.c_float * 3)(*[float(v) for v in d.cam]),
                      (ctypes.c_float * 9)(*[float(v) for v in d.rot]), d.ax, d.ay, d.tan_x, d.tan_y, d.max_t,
                      d.kx, d.ky, d.shift, int(d.cell_seed), tw.size, int(d.use_mips), tw.ctypes.data,
                      th.ctypes.data, tl.ctypes.data, q.ctypes.data if q.size else None, q.size, 0)
        g = gb.c()
        self._check(lib().jt_raster_scene(self._h, ctypes.byref(sc), ctypes.byref(g), _stream(stream)))

    def set_du_offsets(self, tex_id: int, level: int, offs) -> None:
        """Data-unit starts [mcu][ndu - 1] of a standard-form level (an index extension that
        lets six lanes decode one MCU's data units at once)."""
        o = np.ascontiguousarray(offs, np.uint16).reshape(-1)
        self._check(lib().jt_set_du_offsets(self._h, tex_id, level, o.ctypes.data, o.size))

    def upload_set(self, ts, compact: bool = False, units: bool = False) -> None:
        for t, l, e in ts.uploads():
            (self.upload_compact if compact else self.upload)(t, l, e)
            if units and not compact:
                self.set_du_offsets(t, l, e.du_offsets)

    # ---- frame ----
    def mark(self, gb: DeviceGBuffer, filter: int, stream=None):
        g = gb.c()
        self._check(lib().jt_mark(self._h, ctypes.byref(g), filter, _stream(stream)))

    def decode(self, stream=None):
        self._check(lib().jt_decode(self._h, _stream(stream)))

    def colorize(self, gb: DeviceGBuffer, filter: int, out, stream=None):
        g = gb.c()
        self._check(lib().jt_colorize(self._h, ctypes.byref(g), filter, out.data_ptr(), _stream(stream)))

    def stats(self, check: bool = True) -> dict:
        st = jt_stats()
        s = lib().jt_get_stats(self._h, ctypes.byref(st))
        d = {k: getattr(st, k) for k, _ in jt_stats._fields_}
        d["status"] = s
        if check:
            self._check(s)
        return d

    @staticmethod
    def _views(views):
        arr = (jt_view * len(views))()
        for i, (gb, out) in enumerate(views):
            arr[i].g = gb.c()
            arr[i].out_rgba = out.data_ptr()
        return arr

    def frame(self, views, filter: int, stream=None):
        arr = self._views(views)
        self._check(lib().jt_frame(self._h, arr, len(views), filter, _stream(stream)))

    def frame_plain(self, views, filter: int, stream=None):
        arr = self._views(views)
        self._check(lib().jt_frame_plain(self._h, arr, len(views), filter, _stream(stream)))

    def frame_graph(self, views, filter: int, stream=None):
        arr = self._views(views)
        g = ctypes.c_void_p()
        self._check(lib().jt_frame_graph(self._h, arr, len(views), filter, _stream(stream), ctypes.byref(g)))
        self._graphs.append(g)
        return g

    def graph_launch(self, g, stream=None):
        self._check(lib().jt_graph_launch(g, _stream(stream)))

    def graph_destroy(self, g):
        self._graphs = [x for x in self._graphs if x.value != g.value]
        self._check(lib().jt_graph_destroy(g))

    # ---- tuning ----
    def tuning(self) -> dict:
        t = jt_tuning()
        self._check(lib().jt_get_tuning(self._h, ctypes.byref(t)))
        return {k: getattr(t, k) for k, _ in jt_tuning._fields_}

    def set_tuning(self, **kw):
        t = jt_tuning(**{k: int(kw[k]) for k, _ in jt_tuning._fields_})
        self._check(lib().jt_set_tuning(self._h, ctypes.byref(t)))

    def autotune(self, views, filter: int, reps: int = 10, stream=None):
        arr = self._views(views)
        t = jt_tuning()
        ms = ctypes.c_float()
        self._check(lib().jt_autotune(self._h, arr, len(views), filter, _stream(stream), reps, ctypes.byref(t),
                                      ctypes.byref(ms)))
        return {k: getattr(t, k) for k, _ in jt_tuning._fields_}, ms.value

    # ---- pass timing ----
    def profile(self, enable: bool = True):
        self._check(lib().jt_profile(self._h, int(enable)))

    def profile_read(self) -> dict:
        ms = (ctypes.c_float * 4)()
        self._check(lib().jt_profile_read(self._h, ms))
        return {"mark": ms[0], "compact": ms[1], "decode": ms[2], "colorize": ms[3]}

    # ---- inspection ----
    def work_list(self) -> np.ndarray:
        n = ctypes.c_uint64()
        self._check(lib().jt_read_work_list(self._h, None, 0, ctypes.byref(n)))
        out = np.empty(n.value, np.uint32)
        self._check(lib().jt_read_work_list(self._h, out.ctypes.data, out.size, ctypes.byref(n)))
        return out

    def slots(self, gid_begin: int, n: int) -> np.ndarray:
        out = np.empty(n, np.uint32)
        self._check(lib().jt_read_slots(self._h, gid_begin, n, out.ctypes.data))
        return out

    def cache_units(self, unit_begin: int, n: int) -> np.ndarray:
        out = np.empty((n, 256), np.uint8)
        self._check(lib().jt_read_cache(self._h, unit_begin, n, out.ctypes.data))
        return out

    def tile(self, gid: int, sampling: int, reduce: int = 0) -> np.ndarray:
        """RGBA8 tile of a gid from the last decode ([16,16,4] at 4:2:0, [8,8,4] at 4:4:4,
        each side divided by 2^reduce for a reduced-resolution level)."""
        off = int(self.slots(gid, 1)[0])
        mw = (16 if sampling == 420 else 8) >> reduce
        units = 4 if (sampling == 420 and reduce == 0) else 1
        return self.cache_units(off, units).reshape(-1)[:mw * mw * 4].reshape(mw, mw, 4)

    def set_block_cache(self, persistent: bool) -> None:
        """Cross-frame block cache on (decode only MCUs not already resident) or off."""
        self._check(lib().jt_set_block_cache(self._h, 1 if persistent else 0))

    # ---- float chain ----
    def register_coeff_textures(self, first_tex_id: int, count: int, width: int, height: int):
        self._check(lib().jt_register_coeff_textures(self._h, first_tex_id, count, width, height))

    def colorize_float(self, gb: DeviceGBuffer, coef, out, stream=None):
        g = gb.c()
        self._check(lib().jt_colorize_float(self._h, ctypes.byref(g), coef.data_ptr(), out.data_ptr(),
                                            _stream(stream)))

    def colorize_backward(self, gb: DeviceGBuffer, grad_frame, grad_coef, stream=None):
        g = gb.c()
        self._check(lib().jt_colorize_backward(self._h, ctypes.byref(g), grad_frame.data_ptr(),
                                               grad_coef.data_ptr(), _stream(stream)))

    def colorize_float_autograd(self, gb: DeviceGBuffer, coef):
        """F = colorize_float(coef) as a differentiable torch op (backward: jt_colorize_backward)."""
        return _float_function().apply(coef, self, gb)


_FLOAT_FN = None


def _float_function():
    """torch.autograd.Function around jt_colorize_float / jt_colorize_backward (built on first use)."""
    global _FLOAT_FN
    if _FLOAT_FN is None:
        import torch

        class ColorizeFloat(torch.autograd.Function):
            @staticmethod
            def forward(fctx, coef, jctx, gb):
                coef = coef.contiguous()
                out = torch.empty((gb.height, gb.width, 3), dtype=torch.float32, device=coef.device)
                jctx.colorize_float(gb, coef, out)
                fctx.jctx, fctx.gb, fctx.coef_shape = jctx, gb, coef.shape
                return out

            @staticmethod
            def backward(fctx, grad):
                grad = grad.contiguous()
                gc = torch.empty(fctx.coef_shape, dtype=torch.float32, device=grad.device)
                fctx.jctx.colorize_backward(fctx.gb, grad, gc)
                return gc, None, None

        _FLOAT_FN = ColorizeFloat
    return _FLOAT_FN
