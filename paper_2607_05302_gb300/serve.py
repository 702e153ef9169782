"""Serving loop: sort requests of different sizes as they arrive, admitted by
device-memory footprint, with work overlapping on the GPU.

Requests arrive as a seeded Poisson process.  The loop admits, in arrival
order, every request that has arrived and whose footprint fits under the
memory cap.  A Radsort request's footprint is its array plus the workspace of
its plan.  An out-of-place request's footprint is twice the array plus its
histograms, since Radsort avoids the n-element second buffer.  Each admitted
request gets its own CUDA stream: its keys are generated on the device, it is
sorted there, and a completion event is recorded.  Requests that arrive while
others run are admitted as soon as memory frees up: continuous batching, not
a queue served one at a time.  Latency is measured from arrival to completion
on the host clock.

All sorting runs in the CUDA library through the C ABI (radsort.py); this
module only schedules.
"""
from __future__ import annotations

import math
import statistics
import time
from dataclasses import dataclass, field

import numpy as np

from . import radsort as R
from . import workloads as W

CAP_BYTES = 150 * 10 ** 9


@dataclass
class Request:
    rid: int
    arrival: float      # seconds since the start of the run
    n: int
    key_bytes: int
    seed: int
    footprint: int = 0
    admit: float = -1.0
    done: float = -1.0
    tensors: list = field(default_factory=list)
    event: object = None


def make_requests(num, rate=2000.0, log2_min=10, log2_max=29, frac_u64=0.3, seed=0xC0FFEE05):
    """Seeded Poisson arrivals (mean `rate` per second), n log-uniform in
    [2^log2_min, 2^log2_max], 30% 64-bit / 70% 32-bit keys."""
    r = W.splitmix64_np(seed, 0, 3 * num)
    u = (r >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    gaps = -np.log1p(-u[0::3]) / rate
    arrivals = np.cumsum(gaps) - gaps[0]
    logn = log2_min + (log2_max - log2_min) * u[1::3]
    ns = np.maximum(2, np.round(2.0 ** logn)).astype(np.int64)
    kbs = np.where(u[2::3] < frac_u64, 8, 4)
    return [Request(i, float(arrivals[i]), int(ns[i]), int(kbs[i]), seed + 1 + i) for i in range(num)]


def footprint(req, method):
    E = req.key_bytes + 4
    if method == "radsort":
        return req.n * E + R.radsort_workspace_size(req.n, req.key_bytes, 4, 8)
    # out of place: the array, the second n-element buffer pair, and the
    # scratch the comparator allocates (histograms, offsets, look-back ring)
    return 2 * req.n * E + R.radsort_lsd_oop_scratch_size(req.n, req.key_bytes, 4, 8)


def _launch(req, method, stream, keep_result):
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    with torch.cuda.stream(stream):
        r = W.splitmix64_torch(req.seed, 0, req.n, device=dev)
        keys = ((r >> 32) & 0xFFFFFFFF).to(torch.int32) if req.key_bytes == 4 else r
        vals = torch.arange(req.n, dtype=torch.int32, device=dev)
        if method == "radsort":
            ws_bytes = R.radsort_workspace_size(req.n, req.key_bytes, 4, 8)
            ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=dev)
            R.sort_tensors(keys, vals, workspace=ws, stream=stream)
            req.tensors = [keys, vals, ws]
        else:
            ka, va = torch.empty_like(keys), torch.empty_like(vals)
            R.lsd_oop_tensors(keys, vals, ka, va, stream=stream)
            req.tensors = [keys, vals, ka, va]
        ev = torch.cuda.Event()
        ev.record(stream)
        req.event = ev
    if not keep_result:
        del r


def serve(reqs, method="radsort", cap_bytes=CAP_BYTES, max_streams=32, keep_results=False,
          time_scale=1.0):
    """Runs the loop over `reqs` (sorted by arrival); returns statistics.
    time_scale stretches arrival times (1.0 = the stated rate)."""
    import torch

    streams = [torch.cuda.Stream() for _ in range(max_streams)]
    free_streams = list(range(max_streams))
    pending = list(reqs)
    for q in pending:
        q.footprint = footprint(q, method)
        if q.footprint > cap_bytes:
            raise ValueError(f"request {q.rid} ({q.footprint} B) exceeds the cap")
    active = {}
    used = peak_used = peak_conc = 0
    results = {}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    head = 0
    while head < len(pending) or active:
        now = time.perf_counter() - t0
        # admit in arrival order while the head fits
        while (head < len(pending) and pending[head].arrival * time_scale <= now and free_streams
               and used + pending[head].footprint <= cap_bytes):
            q = pending[head]
            head += 1
            si = free_streams.pop()
            q.admit = now
            used += q.footprint
            _launch(q, method, streams[si], keep_results)
            active[q.rid] = (q, si)
            peak_conc = max(peak_conc, len(active))
            peak_used = max(peak_used, used)
        # retire completed requests
        for rid in [k for k, (q, si) in active.items() if q.event.query()]:
            q, si = active.pop(rid)
            q.done = time.perf_counter() - t0
            used -= q.footprint
            free_streams.append(si)
            if keep_results:
                results[rid] = (q.tensors[0].clone(), q.tensors[1].clone())
            q.tensors = []
            q.event = None
        if not active and head < len(pending):
            wait = pending[head].arrival * time_scale - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.01))
        elif active:
            time.sleep(20e-6)
    makespan = time.perf_counter() - t0
    lat = [(q.done - q.arrival * time_scale) * 1e3 for q in reqs]
    keys = sum(q.n for q in reqs)
    out = {
        "method": method, "requests": len(reqs), "keys": keys,
        "p50_ms": statistics.median(lat), "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": statistics.fmean(lat), "keys_per_s": keys / makespan, "makespan_s": makespan,
        "peak_concurrency": peak_conc, "peak_bytes": peak_used, "cap_bytes": cap_bytes,
    }
    if keep_results:
        out["results"] = results
    return out


def run_bench(steps=300, cap_bytes=CAP_BYTES, max_streams=512):
    """Both methods on the same seeded request stream; one JSON-ready dict.
    With many streams available, the memory cap is what limits admission."""
    reqs_r = make_requests(steps)
    reqs_o = make_requests(steps)
    rs = serve(reqs_r, "radsort", cap_bytes, max_streams=max_streams)
    oo = serve(reqs_o, "oop", cap_bytes, max_streams=max_streams)
    R.radsort_device_status()
    return {
        "metric": "serve p99 ms (Poisson 2,000 req/s, n log-uniform 2^10..2^29, 150 GB cap)",
        "value": round(rs["p99_ms"], 3), "unit": "ms", "higher_is_better": False, "n_gpus": 1,
        "steps": steps, "data": "synthetic",
        "config": {"workload": "serve_poisson2000_loguniform_2p10_2p29_u32u64_index",
                   "cap_bytes": cap_bytes, "requests": steps, "max_streams": max_streams},
        "radsort": {k: v for k, v in rs.items() if k != "results"},
        "oop": {k: v for k, v in oo.items() if k != "results"},
    }
