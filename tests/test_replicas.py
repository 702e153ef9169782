"""Multi-GPU is replicas only (the sort does not shard without an all-to-all
exchange): every rank sorts its own array and the bench reports all ranks'
keys over the slowest rank's time.  This checks that host logic with two
gloo ranks on the CPU."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [120.0, 200.0][rank]  # the second rank is the slower one
    ms_max, value = bench.replica_result(ms, 1 << 20, 10, world, dist, torch.device("cpu"))
    out[rank] = (ms_max, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        ms_max, value = out[r]
        assert ms_max == 200.0  # both ranks report the slowest time
        assert value == pytest.approx(2 * 10 * (1 << 20) / 0.2 / 1e9)


def test_one_process_needs_no_collective():
    import torch

    sys.path.insert(0, ROOT)
    import bench

    ms_max, value = bench.replica_result(50.0, 1000, 5, 1, None, torch.device("cpu"))
    assert ms_max == 50.0 and value == pytest.approx(5 * 1000 / 0.05 / 1e9)


def test_profiled_traffic_follows_the_kernel_sources(monkeypatch):
    """The roofline's traffic comes from the committed ncu summary only while
    its source hash matches the round kernel's sources and its block size is
    the bench's: scaled by elements (bytes per element x n) when they do, None
    after any change to the sources, at another block size, and for
    configurations the summary does not cover."""
    import bench

    txt = "source_hash: 0123456789abcdef\ntraffic_bytes_per_element: 15.5\nblock_size: 2048\n"
    n = 1 << 28
    monkeypatch.setattr(bench, "round_kernel_hash", lambda files: "0123456789abcdef")
    t = bench.profiled_traffic(n, 4, 8, "grid", 2048, text=txt)
    assert t == round(15.5 * n)
    assert bench.profiled_traffic(n // 2, 4, 8, "grid", 2048, text=txt) == pytest.approx(t / 2, rel=1e-6)
    assert bench.profiled_traffic(n, 4, 8, "grid", 1024, text=txt) is None
    assert bench.profiled_traffic(n, 8, 8, "grid", 2048, text=txt) is None
    assert bench.profiled_traffic(n, 4, 11, "grid", 2048, text=txt) is None
    monkeypatch.setattr(bench, "round_kernel_hash", lambda files: "0" * 16)
    assert bench.profiled_traffic(n, 4, 8, "grid", 2048, text=txt) is None


def test_bench_defines_every_leg():
    """The helpers bench.py's GPU arm calls are defined (a guard for edits
    that drop one: the GPU arm runs only on a GPU)."""
    import ast

    import bench

    tree = ast.parse(open(os.path.join(bench.ROOT, "bench.py")).read())
    called = {n.func.id for n in ast.walk(tree) if isinstance(n, ast.Call) and isinstance(n.func, ast.Name)}
    defined = {n.name for n in ast.walk(tree) if isinstance(n, (ast.FunctionDef, ast.ClassDef))}
    defined |= {n.arg for n in ast.walk(tree) if isinstance(n, ast.arg)}  # callables passed in
    defined |= {n.id for n in ast.walk(tree) if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Store)}
    import builtins
    missing = {c for c in called if c not in defined and not hasattr(builtins, c)}
    assert not missing, missing
