"""Host-side checks that need no GPU: the C library exports every function include/jt.h
declares, the binding declares each with the header's arity, and the multi-replica timing
logic of the benchmark (max over ranks, whole-job throughput) on two gloo ranks."""

import os
import re
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    h = open(os.path.join(ROOT, "include", "jt.h")).read()
    decls = re.findall(r"^(?:jt_status|const char\*)\s+(jt_\w+)\s*\(([^;]*)\);", h, re.M | re.S)
    return {name: [a for a in args.split(",") if a.strip() and a.strip() != "void"] for name, args in decls}


def test_library_exports_every_declared_function():
    import paper_2510_08166_gb300 as jt
    L = jt.lib()  # builds libjt.so when needed; loading needs no GPU
    fns = _header_functions()
    assert len(fns) >= 26
    for name in fns:
        assert hasattr(L, name), name


def test_binding_matches_header_arity():
    import paper_2510_08166_gb300 as jt
    fns = _header_functions()
    assert set(jt._SIGS) == set(fns)
    for name, args in fns.items():
        assert len(jt._SIGS[name]) == len(args), (name, len(jt._SIGS[name]), len(args))


def test_status_strings():
    import paper_2510_08166_gb300 as jt
    L = jt.lib()
    assert L.jt_status_string(0) == b"ok"
    assert b"capacity" in L.jt_status_string(5)
    assert L.jt_last_error(None) == b"null context"


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, ROOT)
    import bench
    mine = 10.0 + 5.0 * rank  # rank 1 is the slow one
    slowest = bench.max_over_ranks(mine, world, torch.device("cpu"))
    q.put((rank, slowest, bench.replica_value(1000.0, world, slowest)))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    # both ranks see the slower rank's time; the job did 2 x 1000 units in 15 ms
    assert [o[1] for o in out] == [15.0, 15.0]
    assert out[0][2] == pytest.approx(2 * 1000.0 / 0.015)
