#!/usr/bin/env python
"""Throughput of the per-frame JPEG texture path on one GB300 (or N replicas).

Workload (one step = one frame): a 3840x2160 deferred G-buffer (perspective ground plane
+ 200 screen-space quads, per-pixel mip level) over 64 baseline-JPEG textures
(1024-4096^2, quality 50-95, 4:2:0, full mip chains, every level encoded separately);
bilinear colourise. A frame is mark -> compact -> decode -> colourise, captured once as a
CUDA graph and replayed. Inputs are resident in HBM before timing; L2 (129 MB) is flushed
by writing a 256 MB buffer between timed steps (the G-buffer itself is 91 MB).

Metric: needed blocks/s (MCUs decoded per second of frame time). Printed as one JSON line
with ms per frame, per-pass times, the dominant pass's roofline, the same metric end to
end through host buffers, the per-texture "plain" pipeline for comparison, the oracle's
CPU baseline and the SM clocks seen during the timed region.

--impl reference times the oracle (plain C++ on the host cores) on bounded samples of the
same frame and prints the same metric.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "needed blocks/s (4K frame: mark+compact+decode+colourise)"
UNIT = "blocks/s"
WORKLOAD = "4K frame 3840x2160, 64 JPEG textures 1024-4096^2 Q50-95 4:2:0 full mip chains, bilinear"


# DRAM bytes (read + write) per launch of each pass's kernel in an ncu capture of this workload
# with the current kernel code (the summaries under profiles/). A kernel changed since its
# capture must be set back to None.
NCU_TRAFFIC = {"mark": 93.88e6, "compact": 5.45e6, "decode": 2.08e6, "colorize": 133.36e6}
# From one ncu capture of k_decode on the 4K frame in the decode shape the autotuner picks
# (16 MCUs per warp, 12 warps per CTA, 1 CTA per SM): warp instructions executed, issue
# slots busy (% of active cycles) and the frame's symbols; None until captured for the
# current kernel code (see profiles/).
NCU_DECODE = {"warp_instructions": 27327630, "issue_active_pct": 57.77, "symbols": 1257771}


# kernels one frame launches: mark, the compaction's two passes, decode, colourise
LAUNCHES_PER_FRAME = 5


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------------------
# Workload
# ---------------------------------------------------------------------------------------

def workload(compact: bool = False):
    import synth
    ts = synth.scene_textures(compact=compact)
    gb = synth.scene_gbuffer(ts)
    return ts, gb


def frame_symbols(ts, work: np.ndarray) -> int:
    """Huffman symbols (DC, AC, ZRL, EOB) of the listed MCUs, as the encoder coded them."""
    sym = np.concatenate([e.symbols.astype(np.int64) for _, _, e in ts.uploads()])
    return int(sym[work.astype(np.int64)].sum())


def compressed_bytes(ts, work: np.ndarray) -> float:
    """Entropy-coded bytes of the listed MCUs (bit length of each MCU / 8)."""
    bases, ends, lens = [], [], []
    g = 0
    for t, l, e in ts.uploads():
        off = e.index["bit_offset"].astype(np.int64)
        nxt = np.append(off[1:], e.scan_bits)
        bases.append(g)
        lens.append(nxt - off)
        g += e.nmcu
    all_len = np.concatenate(lens)
    return float(all_len[work.astype(np.int64)].sum()) / 8.0


# ---------------------------------------------------------------------------------------
# Clocks during the timed region
# ---------------------------------------------------------------------------------------

class ClockSampler:
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev: int):
        self.dev = dev
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(2)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------
# Oracle (CPU baseline and reference arm)
# ---------------------------------------------------------------------------------------

def oracle_frame_band(o, gb, rows: slice):
    """Oracle mark + bilinear colourise of a band of rows; returns (seconds, blocks)."""
    import synth
    sub = synth.GBuffer(gb.width, rows.stop - rows.start, gb.uv[rows], gb.tex_id[rows], gb.mip[rows])
    o.clear_cache()
    t0 = time.perf_counter()
    o.mark(sub, 1)
    o.colorize(sub.uv, sub.tex_id, sub.mip, 1)
    dt = time.perf_counter() - t0
    return dt, o.cached()


def oracle_baseline(ts, gb, budget_s: float = 10.0):
    """Whole frames (mark + random-access decode + bilinear colourise), repeated with a cold
    tile cache until about budget_s of CPU time has been spent."""
    import oracle
    o = oracle.texset_from(ts)
    secs, blocks, frames = 0.0, 0, 0
    while secs < budget_s or frames == 0:
        dt, nb = oracle_frame_band(o, gb, slice(0, gb.height))
        secs += dt
        blocks += nb
        frames += 1
    return {"value": blocks / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{frames} whole 3840x2160 frames, {blocks // frames} MCUs each, decoded by random "
                      f"access in {secs:.1f} s (single-threaded C++ -O2)"}


# ---------------------------------------------------------------------------------------
# The oracle on all host cores: a pool of worker processes, forked before the first CUDA
# call (the workers inherit the workload and never touch CUDA), each holding its own oracle
# texture set. A frame is split into row bands taken by the workers; every band decodes the
# MCUs its pixels need from a cold tile cache, so MCUs shared by two bands are decoded twice.
# ---------------------------------------------------------------------------------------
_CPU = {}


def _cpu_band(rows):
    if "o" not in _CPU:  # built on a worker's first task, so idle workers cost nothing
        import oracle
        _CPU["o"] = oracle.texset_from(_CPU["ts"])
    return oracle_frame_band(_CPU["o"], _CPU["gb"], slice(rows[0], rows[1]))


def _cpu_full_decode(i):
    """Sequential full decode of full-decode texture i (one 4096^2 level); (seconds, MCUs, bytes)."""
    import oracle
    e = _CPU["ts_full"][i]
    t0 = time.perf_counter()
    d = oracle.Decoded(e.jfif)
    dt = time.perf_counter() - t0
    return dt, e.nmcu, int(d.rgba.size)


class CpuPool:
    def __init__(self, ts, gb, ts_full, n: int):
        import multiprocessing
        _CPU.update(ts=ts, gb=gb, ts_full=ts_full)
        self.n = n
        self.pool = multiprocessing.get_context("fork").Pool(n)

    def frame(self, H: int, needed: int, budget_s: float = 10.0):
        """Whole frames split into 4 n row bands over the n workers, repeated for about
        budget_s of wall time: needed blocks (of the whole frame) per wall second."""
        nb = 4 * self.n
        bands = [(H * i // nb, H * (i + 1) // nb) for i in range(nb)]
        self.pool.map(_cpu_band, bands, chunksize=1)  # warm-up: the workers build their texture sets
        frames, wall, decoded = 0, 0.0, 0
        while wall < budget_s or frames == 0:
            t0 = time.perf_counter()
            res = self.pool.map(_cpu_band, bands, chunksize=1)
            wall += time.perf_counter() - t0
            decoded += sum(r[1] for r in res)
            frames += 1
        return {"value": frames * needed / wall, "frames": frames, "wall_s": wall,
                "decoded_per_frame": decoded / frames}

    def full_decode(self, nt: int):
        """Full decode of 4096^2 textures: the n workers each decode textures round-robin from nt."""
        t0 = time.perf_counter()
        res = self.pool.map(_cpu_full_decode, [i % nt for i in range(self.n)], chunksize=1)
        wall = time.perf_counter() - t0
        mcus = sum(r[1] for r in res)
        out = sum(r[2] for r in res)
        return {"blocks_per_s": mcus / wall, "gbs": out / wall / 1e9, "textures": self.n, "wall_s": wall}

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def full_decode_cpu_textures():
    """One 4096^2 level of each sampling at quality 90 (the full-decode texture shape)."""
    import synth
    ts = synth.full_decode_textures(ntex=2)  # texture 0 at 4:4:4, texture 1 at 4:2:0
    return [lv[0] for lv in ts.levels]


def oracle_all(pool, ts, ts_full, gb, needed):
    """The CPU baseline: the 4K frame on 1 core (the line's value) and on all cores; the
    sequential full decode of 4096^2 Q90 textures on 1 core and on all cores; the FP64 backward
    of the coefficient scene on a band (1 core)."""
    import oracle
    import synth
    one = oracle_baseline(ts, gb)
    fa = pool.frame(gb.height, needed)
    one.update(value_all_cores=fa["value"], cores_all=pool.n, cpu_model=cpu_model(), nproc=os.cpu_count(),
               sample_all_cores=f"{fa['frames']} whole frames, each split into {4 * pool.n} row bands over "
                                f"{pool.n} processes (cold tile cache per band: {fa['decoded_per_frame']:.0f} MCU "
                                f"decodes per frame for {needed} needed)")
    res = {}
    # full decode, one core: both samplings decoded in the main process
    t, mc, ob = 0.0, 0, 0
    for e in ts_full:
        t0 = time.perf_counter()
        d = oracle.Decoded(e.jfif)
        t += time.perf_counter() - t0
        mc += e.nmcu
        ob += int(d.rgba.size)
    res["full_decode_1_core"] = {"blocks_per_s": mc / t, "gbs": ob / t / 1e9,
                                 "sample": "one 4096^2 Q90 texture at 4:4:4 and one at 4:2:0"}
    res["full_decode_all_cores"] = dict(pool.full_decode(len(ts_full)), sample="one 4096^2 Q90 texture per core, "
                                        "alternating 4:4:4 and 4:2:0")
    # coefficient scene, one core: FP64 loss and gradient over a band of 1/16 of the rows
    ts_coef, coef, gb_coef, target = synth.coefficient_scene()
    r = gb_coef.height // 16
    band = synth.GBuffer(gb_coef.width, r, gb_coef.uv[:r], gb_coef.tex_id[:r], gb_coef.mip[:r])
    t0 = time.perf_counter()
    oracle.float_loss_grad(coef, band, target[:r])
    dt = time.perf_counter() - t0
    res["adjoint_fp64_1_core"] = {"band_ms": 1000 * dt, "rows": r, "of_rows": gb_coef.height,
                                  "full_frame_ms_scaled": 1000 * dt * gb_coef.height / r,
                                  "sample": f"FP64 loss and gradient of the 1920x1080 plane's first {r} rows "
                                            f"(the full frame scaled by rows)"}
    return one, res


def run_reference(args, rank, world):
    """The oracle (plain C++, as it stands) on all host cores: each step is one whole 4K frame
    split into row bands over one worker process per core."""
    if rank != 0:
        return 0
    import oracle
    ts, gb = workload()
    o = oracle.texset_from(ts)
    needed = int(o.compact(o.mark(gb, 1)).size)
    del o
    n = len(os.sched_getaffinity(0))
    pool = CpuPool(ts, gb, None, n)
    nb = 4 * n
    bands = [(gb.height * i // nb, gb.height * (i + 1) // nb) for i in range(nb)]
    t_total = 0.0
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        pool.pool.map(_cpu_band, bands, chunksize=1)
        if s >= args.warmup:
            t_total += time.perf_counter() - t0
    pool.close()
    value = args.steps * needed / t_total
    sample = (f"each step: the whole 3840x2160 frame ({needed} needed MCUs), mark + random-access decode + "
              f"bilinear colourise, split into {nb} row bands over {n} processes")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "config": {"workload": WORKLOAD, "l2": "n/a (host)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": n, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------

def max_over_ranks(value: float, world: int, device) -> float:
    """The largest `value` over the replicas (the whole job's time is the slowest rank's)."""
    if world <= 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank: float, world: int, total_ms: float) -> float:
    """Whole-job throughput of `world` replicas that each processed `units_per_rank` units in
    at most `total_ms` (weak scaling)."""
    return world * units_per_rank / (total_ms * 1e-3)


class L2Flush:
    """Evicts every frame's data from L2 (129 MB) between timed steps: a 256 MB write, then a
    read of another 256 MB buffer, so that the dirty lines the write leaves are written back
    before the step begins instead of during it (with `read=False`, the write alone)."""

    def __init__(self, dev, nbytes: int = 256 << 20, read: bool = True):
        import torch
        self.w = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.r = torch.ones(nbytes, dtype=torch.uint8, device=dev) if read else None
        self.sink = None

    def fill_(self, value: int):
        self.w.fill_(value)
        if self.r is not None:
            self.sink = self.r.amax()

    def zero_(self):
        self.fill_(0)


def timed(fn, steps, warmup, stream, flush=None):
    """Mean ms of fn() over `steps` CUDA-event-timed calls after `warmup` untimed ones."""
    import torch
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    ms = []
    for s in range(warmup + steps):
        if flush is not None:
            flush.fill_(s & 255)
        a0.record(stream)
        fn()
        a1.record(stream)
        a1.synchronize()
        if s >= warmup:
            ms.append(a0.elapsed_time(a1))
    return statistics.mean(ms)


def run_views(ctx, ts, jt, dev, flush, stream, steps):
    """Batched views over the same textures: 8 G-buffers (720p .. 4K and two stereo VR
    pairs) in one graph (one mark over all views into one flag array, one compaction, one
    persistent decode of the union, one colourise) against the plain per-view, per-texture
    pipeline."""
    import torch
    import synth
    views = synth.eight_views(ts)
    dv = [jt.DeviceGBuffer.from_host(v, dev) for v in views]
    outs = [torch.empty((v.height, v.width, 4), dtype=torch.uint8, device=dev) for v in views]
    pairs = list(zip(dv, outs))
    g = ctx.frame_graph(pairs, jt.FILTER_BILINEAR)
    ms_graph = timed(lambda: ctx.graph_launch(g), steps, 3, stream, flush)
    st = ctx.stats()
    union = int(st["needed_blocks"])
    ref = [o.clone() for o in outs]
    # the same five launches issued one by one (no graph): the graph's own gain
    ms_eager = timed(lambda: ctx.frame(pairs, jt.FILTER_BILINEAR), steps, 3, stream, flush)
    ctx.stats()
    eager_same = all(bool(torch.equal(a, b)) for a, b in zip(ref, outs))
    per_view = []
    for d, o in pairs:  # needed blocks of each view alone
        ctx.frame([(d, o)], jt.FILTER_BILINEAR)
        per_view.append(int(ctx.stats()["needed_blocks"]))
    ms_plain = timed(lambda: ctx.frame_plain(pairs, jt.FILTER_BILINEAR), max(2, steps // 10), 1, stream, flush)
    ctx.stats()
    same = all(bool(torch.equal(a, b)) for a, b in zip(ref, outs))
    ctx.graph_destroy(g)
    px = sum(v.width * v.height for v in views)
    span = max(per_view) / max(1, min(per_view))
    return {"workload": "8 views 1280x720 (looking up: sky and 6 quads), 1920x1080, 2560x1440, 3840x2160, "
                        "2x2 VR 2064x2208 (two stereo poses), same 64 textures, bilinear", "pixels": px,
            "needed_blocks_union": union, "needed_blocks_per_view": per_view, "span": span,
            "span_over_50": span > 50, "batched_graph_ms": ms_graph, "eager_ms": ms_eager,
            "graph_speedup_over_eager": ms_eager / ms_graph, "plain_ms": ms_plain,
            "speedup": ms_plain / ms_graph, "same_output": same and eager_same,
            "blocks_per_s": union / (ms_graph * 1e-3)}


def run_e2e_pipelined(ctx, jt, host, W, H, dev, frames, render=True):
    """Frames streamed from host buffers with the copies overlapped: two device G-buffers and
    framebuffers (one CUDA graph each); frame k's upload runs on an upload stream while frame
    k - 1 renders, and frame k - 1's download on a download stream while frame k renders.
    Returns ms per frame over `frames` frames (first upload to last download) and whether the
    downloaded frames equal the reference. Every frame's G-buffer is freshly uploaded, and
    the two buffer sets with their framebuffers (250 MB) exceed L2. render=False runs the
    same copies with no frame in between: the copy bound of the loop."""
    import torch
    uv_h, tex_h, mip_h, out_ref = host
    gbs = [jt.DeviceGBuffer.empty(W, H, dev) for _ in range(2)]
    outs = [torch.empty((H, W, 4), dtype=torch.uint8, device=dev) for _ in range(2)]
    outs_h = [torch.empty((H, W, 4), dtype=torch.uint8).pin_memory() for _ in range(2)]
    graphs = [ctx.frame_graph([(gbs[i], outs[i])], jt.FILTER_BILINEAR) for i in range(2)]
    s_gpu = torch.cuda.current_stream(dev)
    s_up, s_dn = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_up = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_dn = [torch.cuda.Event() for _ in range(2)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(s_up)
    for k in range(frames):
        i = k & 1
        if k >= 2:
            s_up.wait_event(ev_done[i])  # frame k - 2 has finished reading this G-buffer
        with torch.cuda.stream(s_up):
            gbs[i].uv.copy_(uv_h, non_blocking=True)
            gbs[i].tex_id.copy_(tex_h, non_blocking=True)
            gbs[i].mip.copy_(mip_h, non_blocking=True)
        ev_up[i].record(s_up)
        s_gpu.wait_event(ev_up[i])
        if k >= 2:
            s_gpu.wait_event(ev_dn[i])  # frame k - 2's framebuffer has been downloaded
        if render:
            ctx.graph_launch(graphs[i], s_gpu)
        ev_done[i].record(s_gpu)
        s_dn.wait_event(ev_done[i])
        with torch.cuda.stream(s_dn):
            outs_h[i].copy_(outs[i], non_blocking=True)
        ev_dn[i].record(s_dn)
    t1.record(s_dn)
    t1.synchronize()
    ms = t0.elapsed_time(t1) / frames
    ctx.stats()
    same = all(bool(torch.equal(o, out_ref)) for o in outs_h)
    for g in graphs:
        ctx.graph_destroy(g)
    return ms, same


def run_clamped(ctx, jt, dgb, out, flush, stream, steps):
    """The 4K frame with bilinear taps clamped to the nearest texel's MCU (Sec. 4.4, the
    linear-interpolation mode of Sec. 6.2): the mark flags one MCU per pixel, so the frame
    decodes the nearest filter's set."""
    g = ctx.frame_graph([(dgb, out)], jt.FILTER_BILINEAR_CLAMP)
    ms = timed(lambda: ctx.graph_launch(g), steps, 3, stream, flush)
    needed = int(ctx.stats()["needed_blocks"])
    ctx.graph_destroy(g)
    return {"workload": "as the headline frame, filter bilinear clamped to one MCU", "ms_per_frame": ms,
            "needed_blocks_per_frame": needed, "blocks_per_s": needed / (ms * 1e-3)}


def run_compact(jt, ts, dgb, ref_out, dev, flush, stream, steps, tuning):
    """The headline frame over the same textures uploaded in the paper's compact form
    (byte-aligned MCUs, two-level offset table, 12-bit DC records; Sec. 5.1, 5.3): frame
    time, identical pixels, and the side-table overhead of both forms per texel."""
    import torch
    ctx = jt.Context(dev.index, max_cache_blocks=1 << 18)
    ctx.upload_set(ts, compact=True)
    ctx.set_tuning(**tuning)
    out = torch.empty_like(ref_out)
    g = ctx.frame_graph([(dgb, out)], jt.FILTER_BILINEAR)
    ms = timed(lambda: ctx.graph_launch(g), steps, 3, stream, flush)
    needed = int(ctx.stats()["needed_blocks"])
    same = bool(torch.equal(out, ref_out))
    ctx.graph_destroy(g)
    ctx.close()
    levels = [e for _, _, e in ts.uploads()]
    n = sum(e.nmcu for e in levels)
    texels = sum(e.nmcu * (256 if e.sampling == 420 else 64) for e in levels)
    table_bits = sum(32 * e.compact.abs.size + 16 * e.compact.rel.size + 36 * e.nmcu for e in levels)
    removed = sum(e.compact.dc_bits_removed for e in levels)
    pad = sum(e.compact.pad_bits for e in levels)
    return {"workload": "as the headline frame, textures in the compact form", "ms_per_frame": ms,
            "needed_blocks_per_frame": needed, "same_output": same,
            "index_bpp_standard": 80.0 * n / texels,
            "side_table_bpp_compact": table_bits / texels,
            "overhead_bpp_compact": (table_bits - removed) / texels,
            "overhead_bpp_compact_with_alignment": (table_bits - removed + pad) / texels,
            "stream_bytes": {"standard": int(sum(e.scan.size for e in levels)),
                             "compact": int(sum(e.compact.scan.size for e in levels))}}


def run_units(jt, ts, dgb, ref_out, dev, flush, stream, steps):
    """The headline frame with data-unit starts recorded for every level (an index extension,
    uint16 per data unit after the first: 80 more bits per 4:2:0 MCU), so six lanes decode an
    MCU's data units at once; autotuned like the headline."""
    import torch
    ctx = jt.Context(dev.index, max_cache_blocks=1 << 18)
    ctx.upload_set(ts, units=True)
    out = torch.empty_like(ref_out)
    tuned, _ = ctx.autotune([(dgb, out)], jt.FILTER_BILINEAR, reps=5)
    g = ctx.frame_graph([(dgb, out)], jt.FILTER_BILINEAR)
    ctx.profile(True)
    pg = ctx.frame_graph([(dgb, out)], jt.FILTER_BILINEAR)  # pass times, replayed apart
    ctx.profile(False)
    ms = [timed(lambda: ctx.graph_launch(g), 1, 0, stream, flush) for _ in range(steps)]
    passes = {"mark": [], "compact": [], "decode": [], "colorize": []}
    for _ in range(steps):
        timed(lambda: ctx.graph_launch(pg), 1, 0, stream, flush)
        for k, v in ctx.profile_read().items():
            passes[k].append(v)
    needed = int(ctx.stats()["needed_blocks"])
    same = bool(torch.equal(out, ref_out))
    ctx.graph_destroy(g)
    ctx.graph_destroy(pg)
    ctx.close()
    return {"workload": "as the headline frame, data-unit starts for every level", "ms_per_frame": statistics.mean(ms),
            "passes_ms": {k: float(np.mean(v)) for k, v in passes.items()}, "needed_blocks_per_frame": needed,
            "same_output": same, "tuning": tuned}


def run_reduced_mips(jt, ts, dgb, ref_out, dev, flush, stream, steps, tuning):
    """The headline frame with mip levels 1, 2, 4, 5, ... not stored but decoded from the
    lowest frequencies of the stored levels 0, 3, 6, ... (the mip alternative of Sec. 7):
    frame time, MCUs decoded, stored stream bytes, and the difference to the stored chain's
    pixels (a DCT-domain reduction is not the box filter that made the stored mips)."""
    import torch
    ctx = jt.Context(dev.index, max_cache_blocks=1 << 18)
    stored = 0
    for t, lv in enumerate(ts.levels):
        for l, e in enumerate(lv):
            base = 3 * (l // 3)
            if l == base:
                ctx.upload(t, l, e)
                stored += e.scan.size
            else:
                ctx.add_reduced_level(t, base, l - base, l)
    ctx.set_tuning(**tuning)
    out = torch.empty_like(ref_out)
    g = ctx.frame_graph([(dgb, out)], jt.FILTER_BILINEAR)
    ms = timed(lambda: ctx.graph_launch(g), steps, 3, stream, flush)
    needed = int(ctx.stats()["needed_blocks"])
    ctx.graph_destroy(g)
    ctx.close()
    d = (out[..., :3].float() - ref_out[..., :3].float())
    mse = float((d * d).mean())
    return {"workload": "as the headline frame; levels 1, 2, 4, 5, ... decoded from levels 0, 3, 6, ...",
            "ms_per_frame": ms, "needed_blocks_per_frame": needed,
            "stream_bytes": {"stored_levels": int(stored),
                             "full_chain": int(sum(e.scan.size for _, _, e in ts.uploads()))},
            "psnr_db_vs_stored_chain": 10.0 * float(np.log10(255.0 ** 2 / max(mse, 1e-12)))}


def run_raster(jt, ctx, ts, gb_host, dev, flush, stream, steps):
    """The geometry-pass stand-in on the GPU: the 4K scene rasterised into a device
    G-buffer (fp32), alone and followed by the frame over it (graph), and how much of the
    rastered G-buffer equals the generator's double-precision one that the headline uses."""
    import torch
    import synth
    d = synth.scene_desc(synth.SEED_BASE + 2, gb_host.width, gb_host.height, ts.sizes, ts.nlevels,
                         synth.scene_pose(), nquads=200)
    gb = jt.DeviceGBuffer.empty(d.width, d.height, dev)
    out = torch.empty((d.height, d.width, 4), dtype=torch.uint8, device=dev)
    ms_raster = timed(lambda: ctx.raster_scene(d, gb), steps, 3, stream, flush)
    g = ctx.frame_graph([(gb, out)], jt.FILTER_BILINEAR)
    ms_both = timed(lambda: (ctx.raster_scene(d, gb), ctx.graph_launch(g)), steps, 3, stream, flush)
    ctx.stats()
    ctx.graph_destroy(g)
    tex = gb.tex_id.cpu().numpy().view(np.uint16)
    mip = gb.mip.cpu().numpy()
    return {"workload": "3840x2160 ground plane + 200 quads (the headline scene), fp32 raster",
            "raster_ms": ms_raster, "raster_plus_frame_ms": ms_both,
            "same_tex_as_generator": float((tex == gb_host.tex_id).mean()),
            "same_mip_as_generator": float((mip == gb_host.mip).mean())}


def mcu_grid(ts, width: int = 2048):
    """G-buffer with one pixel on every MCU of every uploaded level (nearest marks each MCU once)."""
    import synth
    uvs, texs = [], []
    for t, l, e in ts.uploads():
        mw = 16 if e.sampling == 420 else 8
        mx, my = -(-e.width // mw), -(-e.height // mw)
        gx, gy = np.meshgrid(np.arange(mx), np.arange(my))
        tx = np.minimum(gx * mw + mw // 2, e.width - 1)
        ty = np.minimum(gy * mw + mw // 2, e.height - 1)
        uvs.append(np.stack([(tx + 0.5) / e.width, (ty + 0.5) / e.height], -1).reshape(-1, 2))
        texs.append(np.full(mx * my, t, np.uint16))
    uv = np.concatenate(uvs).astype(np.float32)
    n, h = uv.shape[0], -(-uv.shape[0] // width)
    U = np.zeros((h * width, 2), np.float32)
    T = np.full(h * width, 0xFFFF, np.uint16)
    U[:n], T[:n] = uv, np.concatenate(texs)
    return synth.GBuffer(width, h, U.reshape(h, width, 2), T.reshape(h, width), np.zeros((h, width), np.uint8))


def run_full_decode(jt, dev, flush, stream, steps, peak, tuning, ntex=256):
    """Full-decode stress: `ntex` textures of 4096^2 at quality 90, the first half 4:4:4
    (262,144 MCUs each), the second half 4:2:0 (65,536 each), level 0; every MCU is decoded
    into the block cache (17.2 GB of tiles at 256 textures). Timed: mark of an MCU-grid
    G-buffer (one pixel per MCU) + compaction + decode, and compaction + decode alone."""
    import torch
    import synth
    t0 = time.perf_counter()
    ts = synth.full_decode_textures(ntex=ntex)
    encode_s = time.perf_counter() - t0
    units = sum(e.nmcu * (4 if e.sampling == 420 else 1) for _, _, e in ts.uploads())
    ctx = jt.Context(dev.index, max_cache_blocks=units // 4 + 1024)
    ctx.upload_set(ts)
    ctx.set_tuning(**tuning)  # the frame's autotuned launch shapes
    dgb = jt.DeviceGBuffer.from_host(mcu_grid(ts), dev)

    def one():
        ctx.mark(dgb, jt.FILTER_NEAREST)
        ctx.decode()

    ms = timed(one, steps, 2, stream, flush)
    st = ctx.stats()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dec = []
    for s in range(steps):
        ctx.mark(dgb, jt.FILTER_NEAREST)
        flush.fill_(s & 255)
        a0.record(stream)
        ctx.decode()
        a1.record(stream)
        a1.synchronize()
        dec.append(a0.elapsed_time(a1))
    st2 = ctx.stats()
    ctx.close()
    n = int(st["needed_blocks"])
    cbytes = sum(float(e.scan_bits) / 8 for _, _, e in ts.uploads())
    tile_bytes = 256.0 * int(st["cache_units"])
    moved = cbytes + 10.0 * n + 8.0 * n + tile_bytes  # stream + index + slot/work + tiles
    dms = statistics.mean(dec)
    return {"workload": f"{ntex} textures 4096^2 Q90 (half 4:4:4, half 4:2:0), every MCU", "mcus": n,
            "same_count_twice": int(st2["needed_blocks"]) == n,
            "ms_mark_compact_decode": ms, "blocks_per_s": n / (ms * 1e-3),
            "ms_compact_decode": dms, "blocks_per_s_compact_decode": n / (dms * 1e-3),
            "hbm_gbs": moved / (dms * 1e-3) / 1e9, "hbm_frac": moved / (dms * 1e-3) / 1e9 / peak,
            "compressed_mb": cbytes / 1e6, "tiles_mb": tile_bytes / 1e6, "host_encode_s": encode_s}


def run_motion(jt, ts, dev, flush, stream, reps=100, stereo=False):
    """The paper's caching measurement under motion: 60 view directions 6 degrees apart (a
    full turn), the turn repeated `reps` times after one warm-up turn; per direction the
    median frame time over the repetitions, and the maximum of those medians (the worst
    viewpoint). Per-frame mode against the cross-frame block cache, bilinear, each
    direction a graph replay over its own G-buffer(s). With `stereo`, each frame is a VR
    pair (two eyes of 2064x2208 in one batched frame), and the MCUs both eyes share are
    counted per direction."""
    import torch
    import synth
    W, H = (2064, 2208) if stereo else (1920, 1080)
    dirs = synth.motion_views(ts, W, H, stereo=stereo)
    dviews = [[jt.DeviceGBuffer.from_host(g, dev) for g in d] for d in dirs]
    outs = [torch.empty((H, W, 4), dtype=torch.uint8, device=dev) for _ in dirs[0]]
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    res = {}
    modes = ("per_frame", "block_cache") if stereo else ("per_frame", "block_cache", "block_cache_units")
    for mode in modes:
        ctx = jt.Context(dev.index, max_cache_blocks=1 << 18)
        units = mode.endswith("_units")
        ctx.upload_set(ts, units=units)
        if units:  # data units in parallel: small buffers, many warps
            t = ctx.tuning()
            t.update(decode_mcus_per_warp=4, decode_warps=16, decode_ctas_per_sm=4)
            ctx.set_tuning(**t)
        ctx.set_block_cache(mode != "per_frame")
        # timed graphs without event records between their kernels; pass times from a
        # profiled copy of the same turn, replayed once more after the timed turns
        graphs = [ctx.frame_graph(list(zip(dv, outs)), jt.FILTER_BILINEAR) for dv in dviews]
        ctx.profile(True)
        pgraphs = [ctx.frame_graph(list(zip(dv, outs)), jt.FILTER_BILINEAR) for dv in dviews]
        ctx.profile(False)
        ms = np.zeros((reps, len(dirs)))
        dec = np.zeros((reps, len(dirs)))
        passes = {"mark": [], "compact": [], "decode": [], "colorize": []}
        for r in range(reps + 2):
            for k in range(len(dirs)):
                flush.fill_(k & 255)
                a0.record(stream)
                ctx.graph_launch(graphs[k] if r <= reps else pgraphs[k])
                a1.record(stream)
                a1.synchronize()
                if 0 < r <= reps:
                    ms[r - 1, k] = a0.elapsed_time(a1)
                    dec[r - 1, k] = ctx.stats()["needed_blocks"]
                if r > reps:
                    ctx.stats()
                    for name, v in ctx.profile_read().items():
                        passes[name].append(v)
        for g in graphs + pgraphs:
            ctx.graph_destroy(g)
        med = np.median(ms, axis=0)
        res[mode] = {"max_of_medians_ms": float(med.max()), "worst_direction_deg": 6 * int(med.argmax()),
                     "median_ms": float(np.median(ms)), "mean_decoded_blocks": float(dec.mean()),
                     "max_decoded_blocks": int(dec.max()),
                     "passes_median_ms": {k: float(np.median(v)) for k, v in passes.items()}}
        if stereo and mode == "per_frame":  # MCUs shared by the two eyes: |L & R| / |L | R|
            share = []
            for k, dv in enumerate(dviews):
                n = []
                for eye in range(2):
                    ctx.frame([(dv[eye], outs[eye])], jt.FILTER_BILINEAR)
                    n.append(int(ctx.stats()["needed_blocks"]))
                union = dec[0, k]
                share.append((n[0] + n[1] - union) / union)
            res["shared_mcus"] = {"min": float(min(share)), "mean": float(np.mean(share))}
        ctx.close()
    res["workload"] = (f"60 directions x {reps} turns, camera turning 6 deg/frame, "
                       + ("VR pair 2x(2064x2208), 90 deg fov" if stereo else "1920x1080") + ", 64 textures, bilinear")
    res["speedup_max_of_medians"] = res["per_frame"]["max_of_medians_ms"] / res["block_cache"]["max_of_medians_ms"]
    return res


def run_adjoint(jt, dev, flush, stream, steps, peak):
    """Differentiable colourise: 16 coefficient textures 2048^2 (float32 dequantised DCT,
    403 MB), 1920x1080 perspective plane, bilinear; forward F, then the adjoint of
    L = sum (F - T)^2 to the coefficients."""
    import torch
    import synth
    ts, coef, gb, target = synth.coefficient_scene()
    T, my, mx = coef.shape[:3]
    ctx = jt.Context(dev.index, max_cache_blocks=T * my * mx)  # a float tile for every MCU (4 KiB each)
    ctx.register_coeff_textures(0, T, mx * 16, my * 16)
    c = torch.from_numpy(coef).to(dev)
    tgt = torch.from_numpy(target).to(dev)
    dgb = jt.DeviceGBuffer.from_host(gb, dev)
    F = torch.empty((gb.height, gb.width, 3), dtype=torch.float32, device=dev)
    gc = torch.empty_like(c)
    ms_fwd = timed(lambda: ctx.colorize_float(dgb, c, F), steps, 3, stream, flush)
    needed = int(ctx.stats()["needed_blocks"])
    gF = (2.0 * (F - tgt)).contiguous()
    ms_bwd = timed(lambda: ctx.colorize_backward(dgb, gF, gc), steps, 3, stream, flush)
    ctx.stats()
    npx = gb.width * gb.height
    # the method's HBM bytes: the backward writes every coefficient's gradient once (the map
    # is affine, so the coefficients themselves are not read), reads the G-buffer twice (the
    # needed set's mark and the scatter) and the frame gradient once. The forward reads the
    # G-buffer twice, each needed MCU's coefficients once and writes the frame.
    bwd_bytes = 4.0 * c.numel() + 2 * 11.0 * npx + 12.0 * npx
    fwd_bytes = 2 * 11.0 * npx + needed * 1536.0 + 12.0 * npx
    # intermediate traffic, kept out of the method's bytes: both passes' bucket entries (32 B
    # per pixel and needed MCU its taps touch, written and read once; at most four per pixel)
    bucket_bytes_max = 4 * npx * 2 * 32.0
    ctx.close()
    ach = bwd_bytes / (ms_bwd * 1e-3) / 1e9
    return {"workload": "16 coefficient textures 2048^2 4:2:0 (float32 [16,128,128,6,64]), 1920x1080 plane, "
                        "bilinear", "needed_blocks": needed, "forward_ms": ms_fwd, "backward_ms": ms_bwd,
            "backward_roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                                  "algorithmic_bytes": bwd_bytes, "intermediate_bucket_bytes_max": bucket_bytes_max},
            "forward_roofline": {"bound": "hbm", "achieved": fwd_bytes / (ms_fwd * 1e-3) / 1e9, "peak": peak,
                                 "unit": "GB/s", "frac": fwd_bytes / (ms_fwd * 1e-3) / 1e9 / peak,
                                 "algorithmic_bytes": fwd_bytes, "intermediate_bucket_bytes_max": bucket_bytes_max}}


def run_only_motion(args, local_rank):
    """The motion legs alone (also the command the cache-update profile was taken with)."""
    import torch
    import paper_2510_08166_gb300 as jt
    ts, _ = workload()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream(dev)
    out = {"motion": run_motion(jt, ts, dev, flush, stream, reps=args.motion_reps),
           "motion_vr": run_motion(jt, ts, dev, flush, stream, reps=args.motion_reps, stereo=True)}
    print(json.dumps(out), flush=True)
    return 0


def run_gpu(args, rank, world, local_rank):
    import torch
    import paper_2510_08166_gb300 as jt

    if args.only == "motion":
        return run_only_motion(args, local_rank) if rank == 0 else 0
    if args.only == "adjoint":
        if rank == 0:
            torch.cuda.set_device(local_rank)
            dev = torch.device("cuda", local_rank)
            out = run_adjoint(jt, dev, L2Flush(dev), torch.cuda.current_stream(dev), args.steps, peaks()[0])
            print(json.dumps({"adjoint": out}), flush=True)
        return 0
    ts, gb = workload(compact=not args.no_extra)
    pool = ts_full = None
    if rank == 0 and world == 1 and not args.no_cpu and not args.quick:
        # the CPU baseline's workers are forked here, before the first CUDA call
        ts_full = full_decode_cpu_textures()
        pool = CpuPool(ts, gb, ts_full, len(os.sched_getaffinity(0)))
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    ctx = jt.Context(local_rank, max_cache_blocks=1 << 18)
    ctx.upload_set(ts)
    dgb = jt.DeviceGBuffer.from_host(gb, dev)
    out = torch.empty((gb.height, gb.width, 4), dtype=torch.uint8, device=dev)
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream()

    tuned = None
    if args.tuning:
        M, W, C = (int(v) for v in args.tuning.split(","))
        t = ctx.tuning()
        t.update(decode_mcus_per_warp=M, decode_warps=W, decode_ctas_per_sm=C)
        ctx.set_tuning(**t)
        tuned = ctx.tuning()
    elif args.autotune:
        tuned, tuned_ms = ctx.autotune([(dgb, out)], jt.FILTER_BILINEAR, reps=10)
    # the timed graph has no event records between its kernels (they would also cut the
    # programmatic launch edges); pass times come from a profiled copy replayed apart
    graph = ctx.frame_graph([(dgb, out)], jt.FILTER_BILINEAR)
    ctx.profile(True)
    pgraph = ctx.frame_graph([(dgb, out)], jt.FILTER_BILINEAR)
    ctx.profile(False)

    for _ in range(args.warmup):
        flush.zero_()
        ctx.graph_launch(graph)
    st = ctx.stats()
    nblocks = int(st["needed_blocks"])
    work = ctx.work_list()

    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    passes = {"mark": [], "compact": [], "decode": [], "colorize": []}
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for s in range(args.steps):
        flush.fill_(s & 255)  # evict the G-buffer and tiles from L2 between steps
        e0[s].record(stream)
        ctx.graph_launch(graph)
        e1[s].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    for s in range(max(10, min(args.steps, 200))):  # pass times, outside the timed region
        flush.fill_(s & 255)
        ctx.graph_launch(pgraph)
        stream.synchronize()
        for k, v in ctx.profile_read().items():
            passes[k].append(v)
    step_ms = [a.elapsed_time(b) for a, b in zip(e0, e1)]
    total_ms = max_over_ranks(float(sum(step_ms)), world, dev)
    ctx.stats()
    # the same frame after the write alone (L2 full of the flush's dirty lines), for
    # comparison with earlier measurements taken that way
    ms_write_flush = timed(lambda: ctx.graph_launch(graph), max(5, min(args.steps, 50)), 3, stream,
                           L2Flush(dev, read=False))
    ctx.stats()

    if args.quick:  # timed frames only (used under the profiler)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "quick": True, "ms_per_step": total_ms / args.steps,
                              "ms_per_step_write_only_flush": ms_write_flush,
                              "needed_blocks_per_frame": nblocks, "tuning": ctx.tuning(),
                              "passes_ms": {k: float(np.mean(v)) for k, v in passes.items()}}), flush=True)
        ctx.close()
        return 0

    # end to end through host buffers: pinned G-buffer in, framebuffer out, every step
    uv_h = dgb.uv.cpu().pin_memory()
    tex_h = dgb.tex_id.cpu().pin_memory()
    mip_h = dgb.mip.cpu().pin_memory()
    out_h = torch.empty_like(out, device="cpu").pin_memory()
    n_e2e = max(3, min(args.steps, 200))
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    e2e_ms = []
    for s in range(n_e2e + 2):
        flush.fill_(s & 255)
        a0.record(stream)
        dgb.uv.copy_(uv_h, non_blocking=True)
        dgb.tex_id.copy_(tex_h, non_blocking=True)
        dgb.mip.copy_(mip_h, non_blocking=True)
        ctx.graph_launch(graph)
        out_h.copy_(out, non_blocking=True)
        a1.record(stream)
        a1.synchronize()
        if s >= 2:
            e2e_ms.append(a0.elapsed_time(a1))
    h2d = uv_h.numel() * 4 + tex_h.numel() * 2 + mip_h.numel()
    d2h = out_h.numel()
    # the same frames with the copies overlapped with rendering (the serving pattern)
    pipe_ms, pipe_same = run_e2e_pipelined(ctx, jt, (uv_h, tex_h, mip_h, out.cpu()), gb.width, gb.height, dev,
                                           max(10, min(args.steps, 200)))
    copy_ms, _ = run_e2e_pipelined(ctx, jt, (uv_h, tex_h, mip_h, out.cpu()), gb.width, gb.height, dev,
                                   max(10, min(args.steps, 200)), render=False)

    # the per-texture "plain" pipeline for comparison (same output)
    ref_out = out.clone()
    plain_ms = []
    for s in range(4):
        flush.fill_(s & 255)
        a0.record(stream)
        ctx.frame_plain([(dgb, out)], jt.FILTER_BILINEAR)
        a1.record(stream)
        a1.synchronize()
        if s >= 1:
            plain_ms.append(a0.elapsed_time(a1))
    ctx.stats()
    plain_same = bool(torch.equal(ref_out, out))

    mean = {k: float(np.mean(v)) for k, v in passes.items()}
    npx = gb.width * gb.height
    cbytes = compressed_bytes(ts, work)
    symbols = frame_symbols(ts, work)
    dec_ms = mean["decode"]
    decode_roofline = {
        "bound": "issue", "kernel": "decode", "symbols_per_frame": symbols,
        "symbols_per_s": symbols / (dec_ms * 1e-3), "ns_per_symbol_per_gpu": dec_ms * 1e6 / symbols,
        "instructions_per_symbol": (NCU_DECODE["warp_instructions"] * 32.0 / NCU_DECODE["symbols"]
                                    if NCU_DECODE["warp_instructions"] else None),
        "warp_instructions_per_symbol": (NCU_DECODE["warp_instructions"] / NCU_DECODE["symbols"]
                                         if NCU_DECODE["warp_instructions"] else None),
        "issue_active_pct": NCU_DECODE["issue_active_pct"],
        "source": "symbols from the encoder's per-MCU counts over the work list; instructions and issue "
                  "activity from one ncu capture of k_decode (profiles/)"}
    alg = {  # algorithmic HBM bytes per launch
        "mark": 11.0 * npx,
        "compact": float(st["total_blocks"]) + 8.0 * nblocks,
        "decode": nblocks * (10.0 + 8.0 + 1024.0) + cbytes,
        "colorize": 15.0 * npx + 1024.0 * nblocks + 4.0 * nblocks,
    }
    dom = max(mean, key=mean.get)
    peak, peak_kind = peaks()
    achieved = alg[dom] / (mean[dom] * 1e-3) / 1e9
    frame_ms = total_ms / args.steps
    value = replica_value(nblocks * args.steps, world, total_ms)
    e2e_value = world * nblocks / (statistics.mean(e2e_ms) * 1e-3)

    if rank == 0:
        cpu, cpu_legs = oracle_all(pool, ts, ts_full, gb, nblocks) if pool is not None else (None, None)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": frame_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": WORKLOAD, "needed_blocks_per_frame": nblocks, "pixels": npx,
                       "l2": "flushed between timed steps (256 MB write, then 256 MB read of another "
                             "buffer)", "graph": True,
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
            "passes_ms": mean,
            "ms_per_step_write_only_flush": ms_write_flush,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": NCU_TRAFFIC.get(dom), "peak_kind": peak_kind,
                         "algorithmic_bytes": alg[dom]},
            "decode_roofline": decode_roofline,
            "frame_roofline": {"achieved": sum(alg.values()) / (frame_ms * 1e-3) / 1e9, "unit": "GB/s",
                               "frac": sum(alg.values()) / (frame_ms * 1e-3) / 1e9 / peak},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": statistics.mean(e2e_ms),
                    "copies": "pinned host buffers copied by torch around the library's graph launch, "
                              "L2 flushed between steps, one stream (serial)"},
            "e2e_pipelined": {"value": world * nblocks / (pipe_ms * 1e-3), "unit": UNIT, "ms_per_step": pipe_ms,
                              "same_output": pipe_same, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                              "how": "double-buffered G-buffers and framebuffers, uploads and downloads on their "
                                     "own streams overlapped with the previous / next frame's graph",
                              "copy_only_ms": copy_ms, "frame_ms": frame_ms,
                              "over_bound": pipe_ms / max(copy_ms, frame_ms)},
            "plain": {"ms_per_frame": statistics.mean(plain_ms), "same_output": plain_same,
                      "graph_speedup": statistics.mean(plain_ms) / frame_ms},
            "gpu_launches": LAUNCHES_PER_FRAME * args.steps,
            "clocks": clk,
            "wall_s": wall,
            "cpu_baseline": cpu,
            "cpu_legs": cpu_legs,
        }
        if tuned:
            line["tuning"] = tuned
        if not args.no_extra:
            line["clamped_filter"] = run_clamped(ctx, jt, dgb, out, flush, stream, 20)
            line["units"] = run_units(jt, ts, dgb, ref_out, dev, flush, stream, 20)
            line["compact_form"] = run_compact(jt, ts, dgb, ref_out, dev, flush, stream, 20, ctx.tuning())
            line["reduced_mips"] = run_reduced_mips(jt, ts, dgb, ref_out, dev, flush, stream, 20, ctx.tuning())
            line["raster"] = run_raster(jt, ctx, ts, gb, dev, flush, stream, 20)
            line["batched_views"] = run_views(ctx, ts, jt, dev, flush, stream, 20)
            line["adjoint"] = run_adjoint(jt, dev, flush, stream, 20, peak)
            line["full_decode"] = run_full_decode(jt, dev, flush, stream, 5, peak, ctx.tuning(), args.full_decode_textures)
            line["motion"] = run_motion(jt, ts, dev, flush, stream, reps=args.motion_reps)
            line["motion_vr"] = run_motion(jt, ts, dev, flush, stream, reps=args.motion_reps, stereo=True)
        print(json.dumps(line), flush=True)
    if pool is not None:
        pool.close()
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the default launch shapes instead of autotuning them first")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--tuning", default=None,
                    help="fixed decode shape M,W,C (MCUs per warp, warps per CTA, CTAs per SM) instead of autotuning")
    ap.add_argument("--quick", action="store_true", help="timed frames only: no e2e, plain or CPU legs")
    ap.add_argument("--no-extra", action="store_true", help="skip the batched-views and adjoint measurements")
    ap.add_argument("--full-decode-textures", type=int, default=256,
                    help="textures of the full-decode leg (256 is the stated configuration)")
    ap.add_argument("--only", choices=["motion", "adjoint"], default=None,
                    help="run one leg alone and print its JSON (motion: the 1080p and VR motion legs; "
                         "adjoint: the float chain's forward and backward on the coefficient scene)")
    ap.add_argument("--motion-reps", type=int, default=100,
                    help="turns of the motion legs after the warm-up turn (100 is the paper's protocol)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        return run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
