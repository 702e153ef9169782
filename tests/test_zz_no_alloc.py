"""radsort_sort_noalloc, called through the C ABI, against radsort_sort.

Some callers cannot allocate device memory when they sort: a framework that
owns every byte of device memory through its own pool, a latency-bound loop
that cannot absorb cudaMalloc's synchronisation, an out-of-memory handler.
radsort_sort_noalloc serves them from a fixed scratch array compiled into the
library.  The two calls below run back to back on the same shared array; the
second must not see the first one's leftovers.  This file is collected last
on purpose: it passes alone in a fresh process and after every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2607_05302_gb300 import radsort as R
from paper_2607_05302_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("kb", [4, 8])
def test_noalloc_matches_radsort_sort_two_calls(kb):
    lib = R.lib()
    for call, (n, dist) in enumerate([(1_000_003, "uniform"), (777_777, "zipf" if kb == 4 else "sorted")]):
        keys = W.make_keys(dist, n, 8 * kb)
        k0 = torch.from_numpy(keys.view(np.int32 if kb == 4 else np.int64)).cuda()
        v0 = torch.arange(n, dtype=torch.int32, device="cuda")
        ka, va = k0.clone(), v0.clone()
        kb_, vb_ = k0.clone(), v0.clone()
        assert lib.radsort_sort(_ptr(ka), _ptr(va), n, kb, 8, _stream()) == R.RADSORT_OK
        assert lib.radsort_sort_noalloc(_ptr(kb_), _ptr(vb_), n, kb, 8, _stream()) == R.RADSORT_OK
        torch.cuda.synchronize()
        R.radsort_device_status()
        # a stable sort has one result: the tolerance is exact equality
        assert torch.equal(ka, kb_), f"keys differ on call {call}"
        assert torch.equal(va, vb_), f"values differ on call {call}"


def test_noalloc_rejects_sizes_beyond_the_scratch():
    lib = R.lib()
    k = torch.empty(16, dtype=torch.int32, device="cuda")
    huge = 1 << 40  # far beyond what the fixed scratch can plan for; nothing is enqueued
    assert lib.radsort_sort_noalloc(_ptr(k), None, huge, 4, 8, _stream()) == R.RADSORT_ENOMEM
