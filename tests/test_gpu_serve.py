"""The serving loop: requests that overlap on the GPU give the same result as
each request sorted alone (a stable sort has one result, so the tolerance is
exact equality), admission respects the memory cap, and Radsort's smaller
footprint admits more requests at once than the out-of-place sort."""
import numpy as np
import pytest
import torch

from paper_2607_05302_gb300 import radsort as R
from paper_2607_05302_gb300 import serve as S
from paper_2607_05302_gb300 import workloads as W


def alone(req):
    r = W.splitmix64_torch(req.seed, 0, req.n, device="cuda")
    keys = ((r >> 32) & 0xFFFFFFFF).to(torch.int32) if req.key_bytes == 4 else r
    vals = torch.arange(req.n, dtype=torch.int32, device="cuda")
    R.sort_tensors(keys, vals)
    return keys, vals


@pytest.mark.gpu
@pytest.mark.parametrize("method", ["radsort", "oop"])
def test_results_alone_equal_results_in_the_mix(method):
    reqs = S.make_requests(24, rate=1e6, log2_min=10, log2_max=21)
    out = S.serve(reqs, method, cap_bytes=10 ** 10, max_streams=8, keep_results=True)
    R.radsort_device_status()
    assert out["peak_concurrency"] >= 2  # requests did overlap on the device
    for q in reqs:
        k, v = out["results"][q.rid]
        ek, ev = alone(q)
        assert torch.equal(k, ek) and torch.equal(v, ev), q.rid


@pytest.mark.gpu
def test_admission_respects_cap_and_favours_radsort():
    # same stream, tight cap: Radsort's footprint (array + workspace) admits
    # more requests at once than out-of-place (two arrays)
    reqs_r = S.make_requests(40, rate=1e6, log2_min=18, log2_max=22)
    reqs_o = S.make_requests(40, rate=1e6, log2_min=18, log2_max=22)
    cap = 200 * 2 ** 20
    rr = S.serve(reqs_r, "radsort", cap_bytes=cap, max_streams=32)
    oo = S.serve(reqs_o, "oop", cap_bytes=cap, max_streams=32)
    R.radsort_device_status()
    assert rr["peak_bytes"] <= cap and oo["peak_bytes"] <= cap
    assert rr["peak_concurrency"] > oo["peak_concurrency"]


def test_request_generator_shape():
    reqs = S.make_requests(20000)
    ns = np.array([q.n for q in reqs])
    assert ns.min() >= 2 ** 10 and ns.max() <= 2 ** 29
    frac64 = np.mean([q.key_bytes == 8 for q in reqs])
    assert 0.27 < frac64 < 0.33
    gaps = np.diff([q.arrival for q in reqs])
    assert abs(gaps.mean() - 1 / 2000) < 0.05 / 2000
