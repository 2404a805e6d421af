"""jt_compact_static (the compaction scan on caller buffers with a fixed scratch array, for
callers that must not allocate) against the context path's compaction, two calls in a row.

Named to be collected last, so that it also runs after every other GPU test in one process
(the fixed scratch must then still start each call from zero)."""

import ctypes

import numpy as np
import pytest

import synth
from helpers import GidMap, frame

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def jt():
    import paper_2510_08166_gb300 as m
    return m


def _units_per_gid(ts) -> np.ndarray:
    units = []
    for _, _, e in ts.uploads():
        units.append(np.full(e.nmcu, 4 if e.sampling == 420 else 1, np.uint8))
    return np.concatenate(units)


@pytest.mark.gpu
def test_compact_static_matches_context_compaction(jt):
    sizes = [(64, 64), (128, 128), (256, 256), (96, 48), (512, 512), (1024, 1024)]
    ts = synth.make_texture_set(7, sizes, [60, 75, 90, 50, 80, 95], [420, 444, 444, 420, 420, 420])
    gm = GidMap(ts)
    units = _units_per_gid(ts)
    views = [synth.gbuffer_scene(11 + i, w, h, ts.sizes, ts.nlevels, synth.Pose(quad_seed=5 + i), nquads=25)
             for i, (w, h) in enumerate([(320, 180), (333, 211)])]
    ctx = jt.Context(0, 1 << 16)
    ctx.upload_set(ts)
    n = gm.total
    # caller-owned buffers, allocated once up front (the call itself allocates nothing)
    flags = torch.zeros(n, dtype=torch.uint8, device="cuda")
    slot = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    work = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    totals = torch.full((3,), -1, dtype=torch.int32, device="cuda")
    for v in views:  # two calls in a row, different needed sets
        frame(ctx, jt.DeviceGBuffer.from_host(v), 1, torch)
        st = ctx.stats()
        ref_work = ctx.work_list()
        ref_slots = ctx.slots(0, n)
        assert ref_work.size == st["needed_blocks"] > 0
        f = np.zeros(n, np.uint8)
        f[ref_work] = units[ref_work]
        flags.copy_(torch.from_numpy(f))
        jt.compact_static(flags, slot, work, totals)
        torch.cuda.synchronize()
        t = totals.cpu().numpy()
        assert t[0] == ref_work.size and t[1] == st["cache_units"] and t[2] == 0, t
        got_work = work.cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(got_work[: ref_work.size], ref_work)
        np.testing.assert_array_equal(slot.cpu().numpy().view(np.uint32)[ref_work], ref_slots[ref_work])
        assert int(flags.count_nonzero()) == 0  # consumed, as the context path leaves its flags
    ctx.close()


@pytest.mark.gpu
def test_compact_static_small_cases_and_work_overflow(jt):
    rng = np.random.default_rng(3)
    for n in (0, 1, 15, 4096, 4097, 3 * 4096 + 5):
        f = (rng.random(n) < 0.3).astype(np.uint8) * rng.integers(1, 5, n).astype(np.uint8)
        flags = torch.from_numpy(f).cuda() if n else torch.zeros(16, dtype=torch.uint8, device="cuda")[:0]
        slot = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
        work = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
        totals = torch.full((3,), -1, dtype=torch.int32, device="cuda")
        jt.compact_static(flags, slot, work, totals)
        torch.cuda.synchronize()
        idx = np.flatnonzero(f)
        exc = np.concatenate([[0], np.cumsum(f.astype(np.int64))])[:-1]
        assert totals.cpu().tolist() == [idx.size, int(f.sum()), 0]
        np.testing.assert_array_equal(work.cpu().numpy()[: idx.size], idx)
        np.testing.assert_array_equal(slot.cpu().numpy()[idx], exc[idx])
    # a work list shorter than the count: the first entries are kept and the error bit set
    f = np.ones(1000, np.uint8)
    flags = torch.from_numpy(f).cuda()
    slot = torch.zeros(1000, dtype=torch.int32, device="cuda")
    work = torch.full((100,), -1, dtype=torch.int32, device="cuda")
    totals = torch.zeros(3, dtype=torch.int32, device="cuda")
    jt.compact_static(flags, slot, work, totals)
    torch.cuda.synchronize()
    t = totals.cpu().tolist()
    assert t[0] == 1000 and t[2] & jt.DEVERR_CAPACITY
    np.testing.assert_array_equal(work.cpu().numpy(), np.arange(100))


@pytest.mark.gpu
def test_compact_static_large_flags_over_many_tiles(jt):
    """Flags of 255 over 1.5 M indices: unit prefixes pass 2^28 within the scan, which must
    carry them in full (checked against the exact cumulative sum)."""
    n = 1_500_000
    f = np.full(n, 255, np.uint8)
    f[::7] = 0  # some gaps, so counts and unit sums differ
    flags = torch.from_numpy(f).cuda()
    slot = torch.zeros(n, dtype=torch.int32, device="cuda")
    work = torch.zeros(n, dtype=torch.int32, device="cuda")
    totals = torch.zeros(3, dtype=torch.int32, device="cuda")
    for _ in range(2):  # twice: the scratch must start each call from zero
        flags.copy_(torch.from_numpy(f))
        jt.compact_static(flags, slot, work, totals)
        torch.cuda.synchronize()
        idx = np.flatnonzero(f)
        exc = np.concatenate([[0], np.cumsum(f.astype(np.int64))])[:-1]
        t = totals.cpu().numpy().view(np.uint32)
        assert int(t[0]) == idx.size and int(t[1]) == int(f.astype(np.int64).sum()) and int(t[2]) == 0
        assert int(f.astype(np.int64).sum()) > (1 << 28)
        np.testing.assert_array_equal(work.cpu().numpy()[: idx.size], idx)
        np.testing.assert_array_equal(slot.cpu().numpy().view(np.uint32)[idx].astype(np.int64), exc[idx])


def test_compact_static_rejects_before_enqueueing(jt):
    """Argument checks return before any CUDA call (no GPU needed)."""
    L = jt.lib()
    buf = ctypes.create_string_buffer(64)
    base = (ctypes.addressof(buf) + 15) & ~15
    big = jt.STATIC_COMPACT_MAX_FLAGS + 1
    assert L.jt_compact_static(base, big, base, base, 1, base, None) == 5  # over the limit
    assert L.jt_compact_static(base + 1, 16, base, base, 1, base, None) == 1  # misaligned flags
    assert L.jt_compact_static(base, 16, base, base, 1, None, None) == 1  # no totals
    assert L.jt_compact_static(None, 16, base, base, 1, base, None) == 1  # no flags
