"""GPU parity at the workloads' full sizes, element by element against the
oracle (bit-exact: the stable sort has one result).

  * 2^28 uint32 keys + index payload, 8-bit digits, six distributions
    (uniform, Zipf(1.1) over 2^16 values, all equal, sorted, reverse sorted,
    float32 N(0,1) through the order-preserving transform), in the automatic
    plan (the grid layout the benchmark times), in the chunk layout with
    one chunk per SM and with the MSD split (Sec. 4.3);
  * 2^30 uint32 keys + index, uniform, 8-bit digits (the benchmark's headline
    workload, automatic plan);
  * 2^30 uint64 keys uniform over 64 bits + uint32 index, 8-bit digits
    (n_t = 8) and 11-bit digits (n_t = 6);
  * 20,000 uint32 arrays with lognormal lengths (median 4096, natural-log
    sigma 2, clipped to [16, 2^22]) in one segmented call, against Alg. 1 on
    the composite key (segment, key);
  * requests of the serving loop, each result against the oracle.

The oracle runs on the host (single-threaded C): Radsort with p = 1 (the
paper's sequential algorithm, Alg. 2-7) for the single arrays, Alg. 1 for the
composite segmented key.  Host inputs are the same bytes the device sorts
(uniform keys are made on the device and copied back; the other
distributions are made on the host and uploaded).
"""
import concurrent.futures as cf
import multiprocessing as mp
import os
import tempfile

import numpy as np
import pytest
import torch

import oracle_jobs
from paper_2607_05302_gb300 import radsort as R
from paper_2607_05302_gb300 import serve as S
from paper_2607_05302_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

# oracle jobs, largest first; the 2^28 ones serve both plans
JOBS = [("u64", 8, 30), ("u32", "uniform", 30), ("seg",), ("u64", 11, 30)] + [
    ("u32", d, 28) for d in W.DISTRIBUTIONS]


def _workers():
    """Oracle processes run side by side: up to three, fewer when the host
    has less than ~60 GB of free memory per job (a 2^30 job holds ~50 GB)."""
    try:
        free = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        free = 0
    return max(1, min(3, (os.cpu_count() or 1) // 2, int(free // (60 << 30))))


@pytest.fixture(scope="module")
def expected():
    """Futures of every oracle result, started at once in 'spawn' worker
    processes so that the host work overlaps the GPU tests."""
    d = tempfile.mkdtemp(prefix="radsort_oracle_")
    ex = cf.ProcessPoolExecutor(max_workers=_workers(), mp_context=mp.get_context("spawn"))
    futs = {j: ex.submit(oracle_jobs.run, j, d) for j in JOBS}

    def get(job):
        pk, pv = futs[job].result()
        return np.load(pk, mmap_mode="r"), np.load(pv, mmap_mode="r")

    yield get
    ex.shutdown(wait=True, cancel_futures=True)
    for f in os.listdir(d):
        os.remove(os.path.join(d, f))
    os.rmdir(d)


@pytest.mark.parametrize("plan", ["auto", "chunks", "msd"])
@pytest.mark.parametrize("dist", list(W.DISTRIBUTIONS))
def test_2p28_u32_six_distributions_vs_oracle(dist, plan, expected):
    """The automatic plan (grid layout), the chunk layout with one chunk per
    SM, and the MSD split (Sec. 4.3) on the same inputs."""
    n = 1 << 28
    host = W.make_keys(dist, n)
    kt = torch.from_numpy(host.view(np.int32)).to(DEV)
    vt = torch.arange(n, dtype=torch.int32, device=DEV)
    if plan == "chunks":
        bs, pc = 256, torch.cuda.get_device_properties(0).multi_processor_count
    else:
        bs, pc = 0, 0
    R.sort_tensors(kt, vt, float_keys=dist == "float", block_size=bs, num_chunks=pc,
                   layout="msd" if plan == "msd" else 0)
    R.radsort_device_status()
    ek, ev = expected(("u32", dist, 28))
    assert np.array_equal(kt.cpu().numpy().view(np.uint32), ek)
    assert np.array_equal(vt.cpu().numpy().view(np.uint32), ev)


def test_2p30_u32_uniform_vs_oracle(expected):
    """The benchmark's headline workload in its launch configuration (the
    automatic plan).  Keys are made on the device by the torch form of the
    uniform generator (bit-identical to the host form the oracle sorts)."""
    n = 1 << 30
    r = W.splitmix64_torch(W.SEEDS["uniform"], 0, n, device=DEV)
    kt = ((r >> 32) & 0xFFFFFFFF).to(torch.int32)
    del r
    assert np.array_equal(kt[:4096].cpu().numpy().view(np.uint32), W.uniform_keys(4096))
    vt = torch.arange(n, dtype=torch.int32, device=DEV)
    R.sort_tensors(kt, vt)
    R.radsort_device_status()
    ek, ev = expected(("u32", "uniform", 30))
    assert np.array_equal(kt.cpu().numpy().view(np.uint32), ek)
    assert np.array_equal(vt.cpu().numpy().view(np.uint32), ev)


@pytest.mark.parametrize("db", [8, 11])
def test_2p30_u64_vs_oracle(db, expected):
    """2^30 uint64 keys uniform over 64 bits + uint32 index payloads."""
    n = 1 << 30
    kt = W.splitmix64_torch(W.SEEDS["uniform"], 0, n, device=DEV)
    assert np.array_equal(kt[:4096].cpu().numpy().view(np.uint64), W.uniform_keys(4096, 64))
    vt = torch.arange(n, dtype=torch.int32, device=DEV)
    R.sort_tensors(kt, vt, digit_bits=db)
    R.radsort_device_status()
    ek, ev = expected(("u64", db, 30))
    assert np.array_equal(kt.cpu().numpy().view(np.uint64), ek)
    assert np.array_equal(vt.cpu().numpy().view(np.uint32), ev)


def test_20000_lognormal_segments_vs_oracle(expected):
    """The batched workload: one segmented call over 20,000 arrays, each
    sorted independently and stably, against the oracle's Alg. 1 on the
    composite key segment * 2^32 + key."""
    lens = W.lognormal_lengths(20000)
    off = np.zeros(lens.size + 1, np.uint64)
    np.cumsum(lens.astype(np.uint64), out=off[1:])
    n = int(off[-1])
    r = W.splitmix64_torch(W.SEEDS["uniform"], 0, n, device=DEV)
    kt = ((r >> 32) & 0xFFFFFFFF).to(torch.int32)
    del r
    vt = torch.arange(n, dtype=torch.int32, device=DEV)
    od = torch.from_numpy(off.view(np.int64)).to(DEV)
    need = R.segmented_workspace_size(off, 4, 4)
    ws = torch.empty(need, dtype=torch.uint8, device=DEV)
    R.sort_segmented_tensors(kt, vt, od, off, workspace=ws)
    R.radsort_device_status()
    ek, ev = expected(("seg",))
    assert np.array_equal(kt.cpu().numpy().view(np.uint32), ek)
    assert np.array_equal(vt.cpu().numpy().view(np.uint32), ev)


def test_served_requests_vs_oracle():
    """Requests of the serving loop (32- and 64-bit keys, sizes 2^10 .. 2^21)
    sorted while they overlap on the device; every result equals the
    oracle's sort of that request's keys."""
    reqs = S.make_requests(12, rate=1e6, log2_min=10, log2_max=21)
    assert {q.key_bytes for q in reqs} == {4, 8}
    out = S.serve(reqs, "radsort", cap_bytes=10 ** 10, max_streams=8, keep_results=True)
    R.radsort_device_status()
    assert out["peak_concurrency"] >= 2
    for q in reqs:
        k, v = out["results"][q.rid]
        r = W.splitmix64_np(q.seed, 0, q.n)
        host = (r >> np.uint64(32)).astype(np.uint32) if q.key_bytes == 4 else r
        ek, ev = oracle_jobs._radsort(host, W.index_payload(q.n), 8 * q.key_bytes, 8, b=256)
        gk = k.cpu().numpy().view(np.uint32 if q.key_bytes == 4 else np.uint64)
        assert np.array_equal(gk, ek), q.rid
        assert np.array_equal(v.cpu().numpy().view(np.uint32), ev), q.rid
