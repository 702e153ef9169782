"""Serving loop: sort requests of different sizes as they arrive, admitted by
device-memory footprint, with work overlapping on the GPU.

Requests arrive as a seeded Poisson process.  The loop admits every request
that has arrived and whose footprint fits under the memory cap.  A Radsort
request's footprint is its array plus the workspace of its plan.  An
out-of-place request's footprint is twice the array plus its histograms,
since Radsort avoids the n-element second buffer.  Small requests (up to
2^20 keys) admitted in the same loop turn are sorted together as the
segments of one batched call per key width; large ones run on their own
streams, at most two at once (each sort's round kernels occupy every SM), in
arrival order, and a waiting large request does not hold back small ones.
Keys are generated on the device at admission, and a completion event is
recorded per call.  Requests that arrive while others run are admitted as
soon as memory and slots free up: continuous batching, not a queue served
one at a time.  Latency is measured from arrival to completion on the host
clock.

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


# requests up to SMALL_MAX keys are sorted together, one batched call per
# key width and loop turn; at most LARGE_INFLIGHT larger ones run at once (a
# large sort's round kernels occupy every SM already)
SMALL_MAX = 1 << 20
LARGE_INFLIGHT = 2


def _keys(req, dev):
    import torch

    r = W.splitmix64_torch(req.seed, 0, req.n, device=dev)
    return ((r >> 32) & 0xFFFFFFFF).to(torch.int32) if req.key_bytes == 4 else r


def _launch(req, method, stream, keep_result):
    """One large request on its own stream."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    with torch.cuda.stream(stream):
        keys = _keys(req, dev)
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


def _launch_batch(qs, method, stream):
    """Small requests of one key width as the segments of one batched call
    (radsort_sort_segmented, or its out-of-place comparator); they complete
    together."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    off = np.zeros(len(qs) + 1, np.uint64)
    np.cumsum(np.array([q.n for q in qs], np.uint64), out=off[1:])
    n = int(off[-1])
    kb = qs[0].key_bytes
    with torch.cuda.stream(stream):
        keys = torch.empty(n, dtype=torch.int32 if kb == 4 else torch.int64, device=dev)
        vals = torch.empty(n, dtype=torch.int32, device=dev)
        for q, o in zip(qs, off[:-1]):
            o = int(o)
            keys[o:o + q.n] = _keys(q, dev)
            vals[o:o + q.n] = torch.arange(q.n, dtype=torch.int32, device=dev)
        od = torch.from_numpy(off.view(np.int64)).to(dev, non_blocking=False)
        if method == "radsort":
            ws = torch.empty(max(R.segmented_workspace_size(off, kb, 4), 1), dtype=torch.uint8, device=dev)
            R.sort_segmented_tensors(keys, vals, od, off, workspace=ws, stream=stream)
            held = [keys, vals, od, ws]
        else:
            ka, va = torch.empty_like(keys), torch.empty_like(vals)
            ws = torch.empty(max(R.lsd_oop_segmented_workspace_size(off, kb, 4), 1), dtype=torch.uint8,
                             device=dev)
            R.lsd_oop_segmented_tensors(keys, vals, ka, va, od, off, workspace=ws, stream=stream)
            held = [keys, vals, od, ws, ka, va]
        ev = torch.cuda.Event()
        ev.record(stream)
    for q, o in zip(qs, off[:-1]):
        o = int(o)
        q.tensors = [keys[o:o + q.n], vals[o:o + q.n]] + held
        q.event = ev


def serve(reqs, method="radsort", cap_bytes=CAP_BYTES, max_streams=32, keep_results=False,
          time_scale=1.0, small_max=SMALL_MAX, large_inflight=LARGE_INFLIGHT):
    """Runs the loop over `reqs` (sorted by arrival); returns statistics.
    time_scale stretches arrival times (1.0 = the stated rate).  Requests are
    admitted when they have arrived and their footprint fits under the cap:
    small ones (<= small_max keys) in arrival order, gathered per key width
    into one batched call per loop turn; large ones in arrival order, at most
    large_inflight at once, each on its own stream.  A large request that
    waits does not hold back the small ones behind it."""
    import torch

    streams = [torch.cuda.Stream() for _ in range(max_streams)]
    free_streams = list(range(max_streams))
    for q in reqs:
        q.footprint = footprint(q, method)
        if q.footprint > cap_bytes:
            raise ValueError(f"request {q.rid} ({q.footprint} B) exceeds the cap")
    small = [q for q in reqs if q.n <= small_max]
    large = [q for q in reqs if q.n > small_max]
    hs = hl = 0
    active = {}   # stream index -> requests on it
    used = peak_used = peak_conc = 0
    inflight = 0  # admitted requests not yet retired
    large_active = 0
    results = {}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while hs < len(small) or hl < len(large) or active:
        now = time.perf_counter() - t0
        # large requests, in arrival order, within the in-flight limit
        while (hl < len(large) and large[hl].arrival * time_scale <= now and free_streams
               and large_active < large_inflight and used + large[hl].footprint <= cap_bytes):
            q = large[hl]
            hl += 1
            si = free_streams.pop()
            q.admit = now
            used += q.footprint
            _launch(q, method, streams[si], keep_results)
            active[si] = [q]
            large_active += 1
            inflight += 1
        # small requests that have arrived and fit: one batch per key width
        batch = {4: [], 8: []}
        while hs < len(small) and small[hs].arrival * time_scale <= now and used + small[hs].footprint <= cap_bytes:
            q = small[hs]
            if not batch[q.key_bytes] and len(free_streams) <= sum(1 for k in batch if batch[k]):
                break  # no stream left for a batch of this key width
            hs += 1
            q.admit = now
            used += q.footprint
            batch[q.key_bytes].append(q)
            inflight += 1
        for kb in (4, 8):
            if batch[kb]:
                si = free_streams.pop()
                _launch_batch(batch[kb], method, streams[si])
                active[si] = batch[kb]
        peak_conc = max(peak_conc, inflight)
        peak_used = max(peak_used, used)
        # retire completed work
        for si in [k for k, qs in active.items() if qs[0].event.query()]:
            qs = active.pop(si)
            done = time.perf_counter() - t0
            for q in qs:
                q.done = done
                used -= q.footprint
                inflight -= 1
                if q.n > small_max:
                    large_active -= 1
                if keep_results:
                    results[q.rid] = (q.tensors[0].clone(), q.tensors[1].clone())
                q.tensors = []
                q.event = None
            free_streams.append(si)
        if not active:
            nxt = [x.arrival * time_scale for x in (small[hs:hs + 1] + large[hl:hl + 1])]
            wait = min(nxt) - (time.perf_counter() - t0) if nxt else 0
            if wait > 0:
                time.sleep(min(wait, 0.01))
        else:
            time.sleep(20e-6)
    makespan = time.perf_counter() - t0
    lat = [(q.done - q.arrival * time_scale) * 1e3 for q in reqs]
    keys = sum(q.n for q in reqs)
    out = {
        "method": method, "requests": len(reqs), "keys": keys,
        "p50_ms": statistics.median(lat), "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": statistics.fmean(lat), "keys_per_s": keys / makespan, "makespan_s": makespan,
        "peak_concurrency": peak_conc, "peak_bytes": peak_used, "cap_bytes": cap_bytes,
        "small_max": small_max, "large_inflight": large_inflight,
    }
    if keep_results:
        out["results"] = results
    return out


def run_bench(steps=300, cap_bytes=CAP_BYTES, max_streams=512, tight_cap=None):
    """Both methods on the same seeded request stream with the same policy;
    one JSON-ready dict.  tight_cap (bytes): the same stream again under a
    cap small enough that admission, not the GPU, decides concurrency."""
    # untimed: a short run of each method first (library set-up, stream
    # creation and the allocator's pools would otherwise fall on the first)
    for m in ("radsort", "oop"):
        serve(make_requests(16), m, cap_bytes, max_streams=max_streams)
    reqs_r = make_requests(steps)
    reqs_o = make_requests(steps)
    rs = serve(reqs_r, "radsort", cap_bytes, max_streams=max_streams)
    oo = serve(reqs_o, "oop", cap_bytes, max_streams=max_streams)
    R.radsort_device_status()
    out = {
        "metric": "serve p99 ms (Poisson 2,000 req/s, n log-uniform 2^10..2^29, 150 GB cap)",
        "value": round(rs["p99_ms"], 3), "unit": "ms", "higher_is_better": False, "n_gpus": 1,
        "steps": steps, "data": "synthetic",
        "config": {"workload": "serve_poisson2000_loguniform_2p10_2p29_u32u64_index",
                   "cap_bytes": cap_bytes, "requests": steps, "max_streams": max_streams,
                   "small_max": SMALL_MAX, "large_inflight": LARGE_INFLIGHT},
        "radsort": {k: v for k, v in rs.items() if k != "results"},
        "oop": {k: v for k, v in oo.items() if k != "results"},
    }
    if tight_cap:
        # the largest request must fit either way: an out-of-place 2^29 u64
        # request holds about 12.9 GB
        cap = max(tight_cap, max(footprint(q, "oop") for q in reqs_o))
        t_r = serve(make_requests(steps), "radsort", cap, max_streams=max_streams)
        t_o = serve(make_requests(steps), "oop", cap, max_streams=max_streams)
        R.radsort_device_status()
        out["tight_cap"] = {"cap_bytes": cap,
                            "radsort": {k: v for k, v in t_r.items() if k != "results"},
                            "oop": {k: v for k, v in t_o.items() if k != "results"}}
    return out
