"""The seeded generators: the numpy and torch forms of SplitMix64 give the same
bits, the stream matches the published reference value, and the distributions
have the intended shape."""
import numpy as np
import torch

from paper_2607_05302_gb300 import workloads as W


def test_splitmix64_reference_value():
    # SplitMix64 seeded with 0: the first output is 0xE220A8397B1DCDAF
    # (the value printed by the reference implementation of Vigna's splitmix64.c)
    assert int(W.splitmix64_np(0, 0, 1)[0]) == 0xE220A8397B1DCDAF


def test_numpy_and_torch_streams_agree():
    a = W.splitmix64_np(0xC0FFEE01, 12345, 100000)
    b = W.splitmix64_torch(0xC0FFEE01, 12345, 100000).numpy().view(np.uint64)
    assert (a == b).all()


def test_distributions_shape():
    n = 1 << 16
    u = W.make_keys("uniform", n)
    assert u.dtype == np.uint32 and len(np.unique(u)) > n * 0.99
    z = W.make_keys("zipf", n)
    _, cnt = np.unique(z, return_counts=True)
    assert cnt.max() > n * 0.05 and len(cnt) > 1000
    e = W.make_keys("equal", n)
    assert (e == e[0]).all()
    s = W.make_keys("sorted", n)
    assert (np.diff(s.astype(np.int64)) >= 0).all()
    r = W.make_keys("reverse", n)
    assert (np.diff(r.astype(np.int64)) <= 0).all()
    f = W.make_keys("float", n).view(np.float32)
    assert abs(f.mean()) < 0.05 and abs(f.std() - 1) < 0.05
    u64 = W.make_keys("uniform", n, 64)
    assert u64.dtype == np.uint64 and (u64 >> np.uint64(60)).max() == 15
    L = W.lognormal_lengths(20000)
    assert L.min() >= 16 and L.max() <= (1 << 22) and 3000 < np.median(L) < 5500


def test_serving_footprints():
    """Admission inputs of the serving loop, host-only: a Radsort request
    holds its array plus its plan's workspace (within 2-3% from about 2^27
    elements, where the O(sigma b) scratch and the look-back ring no longer
    dominate; at most a quarter more below, where the plan buys larger
    blocks with up to 4 MiB),
    an out-of-place one two arrays plus the comparator's scratch.  Above
    RADSORT_SCRATCH_MAX_N elements Radsort's footprint is the smaller; up to
    it the automatic plan is itself out of place in the workspace, and the two
    are alike."""
    from paper_2607_05302_gb300 import radsort as R
    from paper_2607_05302_gb300 import serve as S

    big = 0
    for req in S.make_requests(400):
        E = req.key_bytes + 4
        r, o = S.footprint(req, "radsort"), S.footprint(req, "oop")
        assert o >= 2 * req.n * E and r >= req.n * E
        if req.n > R.RADSORT_SCRATCH_MAX_N:
            big += 1
            assert r < o
        else:
            assert r <= 1.1 * o
        if req.n >= 1 << 27:
            assert r <= 1.03 * req.n * E
        elif req.n > R.RADSORT_SCRATCH_MAX_N:
            assert r <= 1.25 * req.n * E + (3 << 20)
    assert big > 100


def test_oracle_jobs_match_a_stable_argsort(tmp_path):
    """The worker that computes the full-size parity expectations, run on
    small sizes: its files hold the stable sort of the seeded inputs."""
    import sys
    import os

    sys.path.insert(0, os.path.dirname(__file__))
    import oracle_jobs

    n = 1 << 14
    for job in [("u32", d, 14) for d in W.DISTRIBUTIONS] + [("u64", 8, 14), ("u64", 11, 14)]:
        pk, pv = oracle_jobs.run(job, str(tmp_path))
        k, v = np.load(pk), np.load(pv)
        if job[0] == "u32":
            host = W.make_keys(job[1], n)
            order_keys = host
            if job[1] == "float":  # IEEE total order via the sign-flip transform
                order_keys = np.where(host >> np.uint32(31), ~host, host | np.uint32(1 << 31))
        else:
            host = order_keys = W.make_keys("uniform", n, 64)
        o = np.argsort(order_keys, kind="stable")
        assert np.array_equal(v, o.astype(np.uint32)), job
        assert np.array_equal(k, host[o]), job
