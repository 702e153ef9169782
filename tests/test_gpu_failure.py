"""Failure detection without a GPU fault: every wait of the library is bounded
(an iteration limit with a sleep per poll); a wait that runs out records a
timeout that radsort_device_status reports as RADSORT_ETIMEOUT, and the
context stays usable.  The wait is made to run out on purpose with a flag that
nothing sets and a short limit (about 2^20 polls)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2607_05302_gb300 import radsort as R  # noqa: E402
from paper_2607_05302_gb300 import workloads as W  # noqa: E402

import oracle  # noqa: E402


def test_wait_that_runs_out_is_reported_and_context_stays_usable():
    dev = torch.device("cuda", 0)
    R.radsort_device_status()  # start clean
    flag = torch.zeros(1, dtype=torch.int32, device=dev)
    R.radsort_debug_wait_probe(flag, 1 << 20)
    with pytest.raises(R.RadsortError) as err:
        R.radsort_device_status()
    assert err.value.status == R.RADSORT_ETIMEOUT
    # the status was read and cleared; a set flag ends the wait at once
    flag.fill_(1)
    R.radsort_debug_wait_probe(flag, 1 << 20)
    R.radsort_device_status()
    # and a sort on the same context still matches the oracle
    n = 100003
    keys = W.make_keys("uniform", n, 32)
    vals = W.index_payload(n)
    kt = torch.from_numpy(keys.view(np.int32)).to(dev)
    vt = torch.from_numpy(vals.view(np.int32)).to(dev)
    R.sort_tensors(kt, vt)
    R.radsort_device_status()
    ek, ev = oracle.lsd_oop(keys, vals, n_t=4, sigma=256, bits=8)
    assert np.array_equal(kt.cpu().numpy().view(np.uint32), ek.astype(np.uint32))
    assert np.array_equal(vt.cpu().numpy().view(np.uint32), ev)
