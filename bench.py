#!/usr/bin/env python
"""Radsort benchmark on GB300.

Default workload (N=1): n = 2^30 uint32 keys uniform over [0, 2^32) with a
uint32 payload = original index, 8-bit digits (sigma = 256, n_t = 4 rounds),
the size at which the round kernel's HBM roofline fraction is stated.
One step = one full in-place Radsort: setup, 4 x (sortPhase, fixupPhase),
Finalize.  Every timed step sorts its own fresh copy of the input (8 GiB,
larger than L2), made before the timed region.  The other single-array
workloads (2^28 uint32 keys; 2^30 uint64 keys with 8- and 11-bit digits) are
timed after it with the comparator beside each, and reported under `extra`.

Printed as one JSON line: device-resident throughput (value), end-to-end
throughput through the public call with pinned host buffers, copies in and
out inside the timed region, on one stream and with steps overlapped on three
streams (e2e: the faster, both kept), the roofline of
the dominant kernel (the sortPhase round kernel, CUDA events on its stream),
the out-of-place LSD comparator on the same data and GPU, extra device bytes,
clocks sampled during the timed region, and the oracle timed on the host
cores (cpu_baseline).

--impl reference times the oracle (plain single-threaded C, test
infrastructure) on a bounded sample of the same workload on the host cores.
Multi-GPU (torchrun): replicas only; each rank sorts its own array, and the
value is all ranks' keys / the slowest rank's time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gkeys/s & extra bytes vs out-of-place LSD, same GB300, bit-exact; serve p99 ms"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# the serving run's second cap: the smallest that every request fits under
# out of place (the largest request's out-of-place footprint), so admission
# limits the comparator's concurrency
SERVE_TIGHT_CAP = 1
FALLBACK_HBM = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=24)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="radsort", choices=["radsort", "reference"])
    ap.add_argument("--log2n", type=int, default=30)
    ap.add_argument("--key-bytes", type=int, default=4, choices=[4, 8])
    ap.add_argument("--digit-bits", type=int, default=8, choices=[8, 11])
    ap.add_argument("--dist", default="uniform")
    ap.add_argument("--block-size", type=int, default=0)
    ap.add_argument("--num-chunks", type=int, default=0)
    ap.add_argument("--layout", default="auto", choices=["auto", "grid", "chunks", "msd"],
                    help="block layout (auto: the automatic plan, the grid layout below 2^31; msd: the "
                         "MSD split of Sec. 4.3)")
    ap.add_argument("--no-oop", action="store_true", help="skip the out-of-place comparator")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle cpu_baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-serve", action="store_true",
                    help="skip the short serving run (200 requests) in the default line")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other workloads (2^28 u32, 2^30 u64 with 8- and 11-bit digits)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--segments", type=int, default=20000,
                    help="segmented workload: number of arrays (a smaller batch for profiling)")
    ap.add_argument("--workload", default="radsort", choices=["radsort", "segmented", "serve"],
                    help="radsort: the headline line; segmented: 20,000 lognormal arrays in one "
                         "call under a CUDA graph; serve: the request loop (see serve.py)")
    return ap.parse_args()


def workload_name(a):
    kt = "u32" if a.key_bytes == 4 else "u64"
    return f"radsort_{kt}_keys_u32_index_2^{a.log2n}_{a.dist}_d{a.digit_bits}"


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


# ---------------------------------------------------------------- oracle timing
def oracle_sample_rate(a, seconds):
    """Oracle Radsort (p = 1, the paper's sequential algorithm) on the host
    cores over a bounded sample of the same workload; returns (Gkeys/s,
    sample description, wall seconds)."""
    import numpy as np

    import oracle
    from paper_2607_05302_gb300 import workloads as W

    m = 1 << min(a.log2n, 22)
    keys = W.make_keys(a.dist, m, 8 * a.key_bytes)
    vals = W.index_payload(m)
    n_t = oracle.digits_for(8 * a.key_bytes, a.digit_bits)
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.radsort(keys, vals, n_t=n_t, sigma=1 << a.digit_bits, bits=a.digit_bits, b=1024, p=1,
                       elem_bytes=a.key_bytes + 4)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return reps * m / el / 1e9, f"{reps} x oracle Radsort (p=1, b=1024) of 2^{m.bit_length() - 1} keys of the same distribution", el


def host_cpu():
    """The host CPU's name as the kernel reports it (x86: model name; Arm: the
    implementer and part numbers), for the cpu_baseline records."""
    import platform

    info = {}
    try:
        for ln in open("/proc/cpuinfo"):
            k, _, v = ln.partition(":")
            k, v = k.strip(), v.strip()
            if k and v and k not in info:
                info[k] = v
    except OSError:
        pass
    if "model name" in info:
        return info["model name"]
    if "CPU part" in info:
        return f"{platform.machine()} implementer {info.get('CPU implementer', '?')} part {info['CPU part']}"
    return platform.processor() or platform.machine()


def run_reference(a, rank):
    if rank != 0:
        return
    steps = []
    for i in range(a.warmup + a.steps):
        rate, sample, el = oracle_sample_rate(a, 0.0)
        if i >= a.warmup:
            steps.append(el)
    m = 1 << min(a.log2n, 22)
    value = a.steps * m / sum(steps) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gkeys/s",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * sum(steps) / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32" if a.key_bytes == 4 else "u64", "data": "synthetic",
        "config": {"workload": workload_name(a), "n": 1 << a.log2n, "sample_n": m},
        "cpu_baseline": {"value": value, "unit": "Gkeys/s", "cores": 1, "kind": "oracle", "cpu": host_cpu(),
                         "sample": f"each step: one oracle Radsort (single-threaded C, p=1, b=1024) of 2^{m.bit_length() - 1} keys of the same workload"},
        "e2e": {"value": value, "unit": "Gkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- clocks
class Clocks:
    def __init__(self, path, dev):
        self.path, self.proc = path, None
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={dev}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            c = [x.strip() for x in ln.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1]))
                mx = max(mx, float(c[2]))
            except ValueError:
                continue
            for nm, v in zip(names, c[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# committed ncu summary of each layout's round kernel, and the sources it covers
ROUND_PROFILES = {
    "grid": ("k_lb_round_grid_u32kv_d8_ncu.md", ("rs_grid.cu", "rs_common.cuh", "rs_kernels.cuh")),
    "chunks": ("k_round_u32kv_d8_ncu.md", ("rs_round.cu", "rs_common.cuh", "rs_kernels.cuh")),
}


def round_kernel_hash(files):
    """Hash of a round kernel's sources: a traffic figure taken with ncu on an
    older kernel is not reported."""
    import hashlib

    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2607_05302_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(n, kb, db, lay, bs, text=None):
    """DRAM bytes per round-kernel launch (dram__bytes_read.sum + write.sum)
    from the committed ncu summary of the layout's kernel, scaled from the
    captured size to n by the elements processed; None if the summary is
    missing, older than the kernel, or taken at another block size."""
    name, files = ROUND_PROFILES["chunks" if lay == "chunks" else "grid"]
    txt = text
    if txt is None:
        try:
            txt = open(os.path.join(ROOT, "profiles", name)).read()
        except OSError:
            return None
    import re

    m = re.search(r"source_hash:\s*([0-9a-f]+)", txt)
    t = re.search(r"traffic_bytes_per_element:\s*([0-9.]+)", txt)
    b = re.search(r"block_size:\s*([0-9]+)", txt)
    if not m or not t or m.group(1) != round_kernel_hash(files) or kb != 4 or db != 8:
        return None
    if not b or int(b.group(1)) != bs:
        return None
    return round(float(t.group(1)) * n)


def replica_result(ms, n, steps, world, dist, device):
    """Replicas (one independent sort per rank): the slowest rank's time for
    `steps` sorts, and the whole job's keys per second over that time
    (Gkeys/s).  dist is torch.distributed (None for one process)."""
    import torch

    tmax = torch.tensor([ms], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    ms_max = float(tmax.item())
    return ms_max, world * steps * n / (ms_max / 1e3) / 1e9


def end_to_end(a, R, keys0, vals0, kbufs, vbufs, n, kb, db, E, world, barrier, stream):
    """Same metric through the public call radsort_sort with pinned host
    buffers.  Every step copies its inputs host -> device, sorts them with
    radsort_sort (automatic plan, allocating) and copies the sorted keys and
    values device -> host, all inside the timed region.  The steps run on
    `depth` streams, each with its own device and host output buffers, so
    the copies of one step overlap the sort of another (copy engines and SMs
    work side by side), as a batch of independent requests would run; the
    same steps on one stream, nothing overlapped, are reported as `serial`."""
    import ctypes

    import numpy as np
    import torch

    ktype = keys0.dtype
    hk = torch.empty(n, dtype=ktype, pin_memory=True)
    hv = torch.empty(n, dtype=torch.int32, pin_memory=True)
    hk.copy_(keys0.cpu())
    hv.copy_(vals0.cpu())
    depth = max(1, min(3, len(kbufs)))
    outs = [(torch.empty(n, dtype=ktype, pin_memory=True), torch.empty(n, dtype=torch.int32, pin_memory=True))
            for _ in range(depth)]
    if not all(t.is_pinned() for t in [hk, hv] + [t for o in outs for t in o]):
        raise SystemExit("bench: host buffers are not pinned")
    streams = [torch.cuda.Stream() for _ in range(depth)]

    def step(s, d):
        dk, dv = kbufs[d], vbufs[d]
        with torch.cuda.stream(s):
            dk.copy_(hk, non_blocking=True)
            dv.copy_(hv, non_blocking=True)
            R.radsort_sort(ctypes.c_void_p(dk.data_ptr()), ctypes.c_void_p(dv.data_ptr()), n, kb, db,
                           ctypes.c_void_p(s.cuda_stream))
            outs[d][0].copy_(dk, non_blocking=True)
            outs[d][1].copy_(dv, non_blocking=True)

    def timed(ss, steps):
        for i in range(len(ss)):  # untimed: one step per stream
            step(ss[i], i)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s in ss:
            s.wait_stream(stream)
        for i in range(steps):
            step(ss[i % len(ss)], i % len(ss))
        for s in ss:
            stream.wait_stream(s)
        e1.record(stream)
        barrier()
        R.radsort_device_status()
        return e0.elapsed_time(e1) / steps

    # the host link as this machine has it (outside the timed region): one copy of
    # the keys each way, so the e2e figure can be read against it
    link = {}
    for name, dst, src in (("h2d_gbs", kbufs[0], hk), ("d2h_gbs", outs[0][0], kbufs[0])):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        dst.copy_(src, non_blocking=True)
        c1.record(stream)
        torch.cuda.synchronize()
        link[name] = round(n * keys0.element_size() / (c0.elapsed_time(c1) / 1e3) / 1e9, 1)
    steps = max(2 * depth, min(a.steps, 12))
    ms_serial = timed([stream], max(2, min(a.steps, 5)))
    ms = timed(streams, steps)
    # the last step's result, checked on the host: sorted, and a permutation
    # of the input that keeps equal keys in input order
    k = outs[(steps - 1) % depth][0].numpy()
    k = k.view(np.uint32) if kb == 4 else k.view(np.uint64)
    v = outs[(steps - 1) % depth][1].numpy().astype(np.int64)
    src = hk.numpy().view(k.dtype)
    eq = k[1:] == k[:-1]
    if not (np.all(k[1:] >= k[:-1]) and np.array_equal(src[v], k) and np.all(v[1:][eq] > v[:-1][eq])):
        raise SystemExit("bench: end-to-end result is wrong")
    # both schedules are complete measurements (every step's copies inside the
    # timed region); the line reports the faster, as a caller would pick it
    # (on some boxes the copy engines do not overlap and three streams gain
    # nothing), and keeps both
    piped = {"value": round(world * n / (ms / 1e3) / 1e9, 3), "ms_per_step": round(ms, 3),
             "streams": depth, "steps": steps}
    serial = {"value": round(world * n / (ms_serial / 1e3) / 1e9, 3), "ms_per_step": round(ms_serial, 3),
              "streams": 1, "steps": max(2, min(a.steps, 5))}
    best = piped if ms <= ms_serial else serial
    return {"value": world * n / (best["ms_per_step"] / 1e3) / 1e9, "unit": "Gkeys/s",
            "h2d_bytes_per_step": n * E, "d2h_bytes_per_step": n * E,
            "mode": "pipelined" if best is piped else "serial", "ms_per_step": best["ms_per_step"],
            "link": link, "pipelined": piped, "serial": serial,
            "call": "radsort_sort (automatic plan, allocating, stream-ordered) with pinned host buffers; "
                    "pipelined: H2D, sort and D2H of each step on one of three streams, steps overlapped"}


def run_segmented(a):
    """20,000 uint32 arrays with lognormal lengths (median 4096, natural-log
    sigma 2, clipped to [16, 2^22]) and index payloads, sorted by one
    radsort_sort_segmented call captured in a CUDA graph and replayed; each
    timed replay sorts a fresh copy (restored outside the timed region).
    Beside it, the out-of-place comparator on the same arrays
    (radsort_lsd_oop_sort_segmented: the long segments through n-element
    alternate arrays), and the sort given the smallest workspace it accepts
    (the low-memory plan), captured and timed the same way."""
    import numpy as np
    import torch

    from paper_2607_05302_gb300 import radsort as R
    from paper_2607_05302_gb300 import workloads as W

    dev = torch.device("cuda", 0)
    lens = W.lognormal_lengths(a.segments)
    off = np.zeros(lens.size + 1, np.uint64)
    np.cumsum(lens.astype(np.uint64), out=off[1:])
    n = int(off[-1])
    r = W.splitmix64_torch(W.SEEDS["uniform"], 0, n, device=dev)
    keys0 = ((r >> 32) & 0xFFFFFFFF).to(torch.int64).to(torch.int32)
    del r
    vals0 = torch.arange(n, dtype=torch.int32, device=dev)
    od = torch.from_numpy(off.view(np.int64)).to(dev)

    def timed(call):
        kt, vt = keys0.clone(), vals0.clone()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            call(kt, vt)  # warm-up (also creates the library's streams)
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            call(kt, vt)
        times = []
        for i in range(a.warmup + a.steps):
            kt.copy_(keys0)
            vt.copy_(vals0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            torch.cuda.synchronize()
            if i >= a.warmup:
                times.append(e0.elapsed_time(e1))
        R.radsort_device_status()
        # the last replay's result: sorted inside every segment, a stable permutation
        seg = torch.repeat_interleave(torch.arange(lens.size, device=dev),
                                      torch.from_numpy(lens.astype(np.int64)).to(dev))
        k = kt.to(torch.int64) & 0xFFFFFFFF
        v = vt.to(torch.int64) & 0xFFFFFFFF
        same = seg[1:] == seg[:-1]
        ok = (bool(torch.equal(seg[v], seg)) and bool(torch.equal(keys0.to(torch.int64)[v] & 0xFFFFFFFF, k))
              and bool((k[1:][same] >= k[:-1][same]).all()))
        del g, kt, vt, seg, k, v, same
        return statistics.median(times), ok

    res = {}
    for db in (8, 11):  # both widths, for the record
        need = R.segmented_workspace_size(off, 4, 4, db)
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
        ms, ok = timed(lambda kt, vt: R.sort_segmented_tensors(kt, vt, od, off, digit_bits=db, workspace=ws))
        res[db] = {"ms_per_step": ms, "value": n / (ms / 1e3) / 1e9, "workspace_bytes": need, "checked": ok}
        del ws
    # the smallest workspace the sort accepts (8-bit digits): medium segments
    # and unaligned long ones sorted in place
    need_m = R.segmented_workspace_size(off, 4, 4, 8, minimal=True)
    wsm = torch.empty(need_m, dtype=torch.uint8, device=dev)
    mms, mok = timed(lambda kt, vt: R.sort_segmented_tensors(kt, vt, od, off, digit_bits=8, workspace=wsm))
    low = {"value": round(n / (mms / 1e3) / 1e9, 3), "ms_per_step": round(mms, 3), "checked": mok,
           "extra_bytes": need_m, "extra_frac": round(need_m / (n * 8), 4), "digit_bits": 8}
    del wsm
    # the digit width the library's autotuner picks for this batch
    best = R.segmented_autotune(keys0, vals0, od, off)
    # the out-of-place comparator at the same digit width
    need_o = R.lsd_oop_segmented_workspace_size(off, 4, 4, best)
    wso = torch.empty(max(need_o, 1), dtype=torch.uint8, device=dev)
    ka, va = torch.empty_like(keys0), torch.empty_like(vals0)
    oms, ook = timed(lambda kt, vt: R.lsd_oop_segmented_tensors(kt, vt, ka, va, od, off, digit_bits=best,
                                                                workspace=wso))
    oval = n / (oms / 1e3) / 1e9
    print(json.dumps({
        "metric": f"Gkeys/s, batched segmented sort ({lens.size:,} arrays, one graph replay)",
        "value": round(res[best]["value"], 3), "unit": "Gkeys/s", "n_gpus": 1, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": res[best]["ms_per_step"], "higher_is_better": True,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"segmented_{lens.size}_lognormal_median4096_sigma2_u32_index", "n": n,
                   "segments": int(lens.size), "digit_bits": best,
                   "extra_bytes": res[best]["workspace_bytes"],
                   "extra_frac": round(res[best]["workspace_bytes"] / (n * 8), 4),
                   "by_digit_bits": {str(k): round(v["value"], 3) for k, v in res.items()},
                   "digit_bits_from": "radsort_segmented_autotune",
                   "checked": all(v["checked"] for v in res.values())},
        "oop": {"value": round(oval, 3), "ms_per_step": round(oms, 3), "checked": ook,
                "extra_bytes": n * 8 + need_o, "extra_frac": round((n * 8 + need_o) / (n * 8), 4)},
        "radsort_over_oop": round(res[best]["value"] / oval, 4),
        "low_memory": low,
    }), flush=True)


def time_workload(R, W, dev, log2n, kb, db, steps, warmup, barrier, stream, layout=0, with_oop=True):
    """One more single-array workload (uniform keys, index payload): Radsort
    in the automatic plan and the out-of-place comparator on the same data,
    each timed over `steps` fresh copies with CUDA events; the round kernel's
    mean launch time from the library's trace gives its roofline fraction."""
    import torch

    n = 1 << log2n
    E = kb + 4
    r = W.splitmix64_torch(W.SEEDS["uniform"], 0, n, device=dev)
    keys0 = ((r >> 32) & 0xFFFFFFFF).to(torch.int64).to(torch.int32) if kb == 4 else r
    del r
    vals0 = torch.arange(n, dtype=torch.int32, device=dev)
    if layout:
        bs, pc, lay = 0, 0, layout
    else:
        bs, pc, lay = R.radsort_plan_default(n, kb, 4, db)
    wsb = R.radsort_workspace_size(n, kb, 4, db, 0, 0, layout)
    ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=dev)
    free_b = torch.cuda.mem_get_info(dev)[0]
    nbuf = int(max(2, min(max(steps, warmup), (free_b * 0.8) // (n * E))))
    kbufs = [torch.empty_like(keys0) for _ in range(nbuf)]
    vbufs = [torch.empty_like(vals0) for _ in range(nbuf)]

    def refill(i):
        kbufs[i].copy_(keys0)
        vbufs[i].copy_(vals0)

    def run(fn):
        for i in range(nbuf):
            refill(i)
        for i in range(warmup):
            fn(i % nbuf)
        for i in range(min(warmup, nbuf)):
            refill(i)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s in range(steps):
            if s >= nbuf:  # fewer copies than steps: refill in the timed region
                refill(s % nbuf)
            fn(s % nbuf)
        e1.record(stream)
        barrier()
        R.radsort_device_status()
        return e0.elapsed_time(e1) / steps

    R.radsort_trace_read()
    R.radsort_trace_enable(True)
    ms = run(lambda i: R.sort_tensors(kbufs[i], vbufs[i], digit_bits=db, workspace=ws, layout=layout))
    R.radsort_trace_enable(False)
    recs = R.radsort_trace_read()
    # the last step's result: sorted and a stable permutation of the input
    last = (steps - 1) % nbuf
    k = kbufs[last].to(torch.int64) & 0xFFFFFFFF if kb == 4 else kbufs[last] ^ (-(2 ** 63))
    v = vbufs[last].to(torch.int64) & 0xFFFFFFFF
    eq = kbufs[last][1:] == kbufs[last][:-1]
    ok = bool((k[1:] >= k[:-1]).all()) and bool(torch.equal(keys0[v], kbufs[last])) and bool(
        (v[1:][eq] > v[:-1][eq]).all())
    del k, v, eq
    rounds = [t for ph, rd, t in recs if ph == "sortPhase"]
    fin = [t for ph, rd, t in recs if ph == "Finalize"]
    avg_round = statistics.mean(rounds) if rounds else float("nan")
    hbm, src = peaks()
    val = n / (ms / 1e3) / 1e9
    oms = oval = None
    if with_oop:
        ka, va = torch.empty_like(keys0), torch.empty_like(vals0)
        oms = run(lambda i: R.lsd_oop_tensors(kbufs[i], vbufs[i], ka, va, digit_bits=db))
        oval = n / (oms / 1e3) / 1e9
        del ka, va
    out = {
        "workload": f"radsort_{'u32' if kb == 4 else 'u64'}_keys_u32_index_2^{log2n}_uniform_d{db}"
                    + (f"_{layout}" if layout else ""),
        "n": n, "value": round(val, 3), "unit": "Gkeys/s", "ms_per_step": round(ms, 3), "steps": steps,
        "block_size": bs, "extra_bytes": wsb, "extra_frac": round(wsb / (n * E), 5),
        "round_ms": round(avg_round, 4),
        "round_frac": round((n * 2 * E) / (avg_round / 1e3) / 1e9 / hbm, 4),
        "finalize_ms": round(statistics.mean(fin), 4) if fin else None,
        "result_checked": ok,
        "oop": None if oval is None else {
            "value": round(oval, 3), "ms_per_step": round(oms, 3),
            "extra_bytes": n * E + R.radsort_lsd_oop_scratch_size(n, kb, 4, db)},
        "radsort_over_oop": None if oval is None else round(val / oval, 4),
    }
    del kbufs, vbufs, ws, keys0, vals0
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- GPU arm
def main():
    a = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank)
        return
    if a.workload == "segmented":
        run_segmented(a)
        return
    if a.workload == "serve":
        from paper_2607_05302_gb300 import serve

        print(json.dumps(serve.run_bench(steps=a.steps, tight_cap=SERVE_TIGHT_CAP)), flush=True)
        return

    import numpy as np
    import torch

    from paper_2607_05302_gb300 import radsort as R
    from paper_2607_05302_gb300 import workloads as W

    if not os.path.exists(R.LIB_PATH):
        import __graft_entry__

        __graft_entry__.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    n = 1 << a.log2n
    kb, db = a.key_bytes, a.digit_bits
    E = kb + 4
    ktype = torch.int32 if kb == 4 else torch.int64
    # inputs: identical bytes to workloads.make_keys (uniform via the torch
    # form of the same SplitMix64 stream; other distributions from the host)
    if a.dist == "uniform":
        r = W.splitmix64_torch(W.SEEDS["uniform"], 0, n, device=dev)
        keys0 = ((r >> 32) & 0xFFFFFFFF).to(torch.int64).to(torch.int32) if kb == 4 else r
        del r
    else:
        host = W.make_keys(a.dist, n, 8 * kb)
        keys0 = torch.from_numpy(host.view(np.int32 if kb == 4 else np.int64)).to(dev)
    vals0 = torch.arange(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    # the automatic plan (grid layout, block size of least workspace); the
    # chunk layout with one chunk per SM is timed beside it (chunk_layout)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    lay = a.layout
    if lay == "chunks":
        bs, pc = a.block_size or 256, a.num_chunks or sms
    else:
        bs, pc = a.block_size, 0
    wsb = R.radsort_workspace_size(n, kb, 4, db, bs, pc, lay)
    if not bs and lay != "msd":
        bs, _, _ = R.radsort_plan_default(n, kb, 4, db)
    ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=dev)

    free_b = torch.cuda.mem_get_info(dev)[0]
    per_step = n * E
    # one fresh copy per timed step where memory allows (at 2^30 u32 + u32,
    # 24 copies of 8 GiB), so that no copy is refilled inside the timed region
    nbuf = int(min(max(a.warmup, a.steps), max(1, (free_b * 0.85) // per_step)))
    kbufs = [torch.empty_like(keys0) for _ in range(nbuf)]
    vbufs = [torch.empty_like(vals0) for _ in range(nbuf)]

    def refill(i):
        kbufs[i].copy_(keys0)
        vbufs[i].copy_(vals0)

    for i in range(nbuf):
        refill(i)

    def step(i):
        R.sort_tensors(kbufs[i % nbuf], vbufs[i % nbuf], digit_bits=db, block_size=bs,
                       num_chunks=pc, workspace=ws, layout=lay)

    # warm-up (also checks the result once against the sorted reference)
    for i in range(a.warmup):
        step(i)
    R.radsort_device_status()
    if a.warmup:
        ks = kbufs[0] if kb == 8 else (kbufs[0].to(torch.int64) & 0xFFFFFFFF)
        ok = bool((ks[1:] >= ks[:-1]).all()) if kb == 4 else True
        if not ok:
            raise SystemExit("bench: warm-up result is not sorted")
    for i in range(min(a.warmup, nbuf)):
        refill(i)
    torch.cuda.synchronize()

    clocks = Clocks(os.path.join(tempfile.gettempdir(), f"radsort_clocks_{os.getpid()}_rank{rank}.csv"), local)
    R.radsort_trace_read()  # drop warm-up records
    R.radsort_trace_enable(True)
    l0 = R.radsort_launch_count()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for s in range(a.steps):
        if s >= nbuf:  # not enough memory for a copy per step: refill in the timed region
            refill(s % nbuf)
        step(s)
    ev1.record(stream)
    barrier()
    R.radsort_trace_enable(False)
    launches = R.radsort_launch_count() - l0
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    R.radsort_device_status()
    recs = R.radsort_trace_read()
    ms_max, value = replica_result(ms, n, a.steps, world, dist, dev)

    phases = {}
    for ph, rd, t in recs:
        key = ph if rd < 0 else f"{ph}[{rd}]"
        phases.setdefault(key, []).append(t)
    round_ms = [t for ph, rd, t in recs if ph == "sortPhase"]
    avg_round = statistics.mean(round_ms) if round_ms else float("nan")
    hbm, src = peaks()
    achieved = (n * 2 * E) / (avg_round / 1e3) / 1e9
    traffic = profiled_traffic(n, kb, db, lay, bs)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "traffic": traffic,
                "kernel": ("k_round (sortPhase, Alg. 5, chunk layout)" if lay == "chunks"
                           else "k_lb_round (sortPhase, Alg. 5, grid layout)"),
                "algorithmic_bytes_per_launch": n * 2 * E, "peak_source": src,
                "avg_launch_ms": round(avg_round, 4)}
    step_bytes = n * (4 * 2 * E) if kb == 4 and db == 8 else None
    # Finalize moves every element once at most: n * 2E bytes at most, over
    # its mean duration (a bound on its bandwidth: blocks already in place
    # are not moved)
    fin_ms = [t for ph, rd, t in recs if ph == "Finalize"]
    finalize = None
    if fin_ms:
        fm = statistics.mean(fin_ms)
        finalize = {"ms": round(fm, 4), "bytes": n * 2 * E, "gbs": round(n * 2 * E / (fm / 1e3) / 1e9, 1),
                    "frac": round(n * 2 * E / (fm / 1e3) / 1e9 / hbm, 4)}

    # ---- the paper's chunk layout (Sec. 4.3), one chunk per SM, same data
    plan2 = None
    ws2 = None
    if not a.no_oop and lay != "chunks":
        b2, p2 = 256, sms
        try:
            ws2 = R.radsort_workspace_size(n, kb, 4, db, b2, p2, "chunks")
        except R.RadsortError as err:  # e.g. chain sequence numbers overflow (sigma = 2048, 2^30)
            plan2 = {"layout": "chunks", "block_size": b2, "num_chunks": p2,
                     "unavailable": f"radsort_workspace_size: {err}"}
    if ws2 is not None:
        wst = torch.empty(max(ws2, 1), dtype=torch.uint8, device=dev)
        for i in range(min(nbuf, 2)):
            refill(i)
        R.sort_tensors(kbufs[0], vbufs[0], digit_bits=db, block_size=b2, num_chunks=p2, workspace=wst,
                       layout="chunks")
        barrier()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        R.sort_tensors(kbufs[1 % nbuf], vbufs[1 % nbuf], digit_bits=db, block_size=b2, num_chunks=p2,
                       workspace=wst, layout="chunks")
        q1.record(stream)
        barrier()
        R.radsort_device_status()
        pms = q0.elapsed_time(q1)
        plan2 = {"layout": "chunks", "block_size": b2, "num_chunks": p2, "extra_bytes": ws2,
                 "extra_frac": round(ws2 / (n * E), 5), "value": round(world * n / (pms / 1e3) / 1e9, 3),
                 "unit": "Gkeys/s", "ms_per_step": round(pms, 3), "steps": 1}
        del wst

    # ---- end to end through the public call with host buffers
    e2e = None
    if not a.no_e2e:
        e2e = end_to_end(a, R, keys0, vals0, kbufs, vbufs, n, kb, db, E, world, barrier, stream)

    # ---- out-of-place comparator on the same data and GPU
    oop = None
    if not a.no_oop:
        ka, va = torch.empty_like(keys0), torch.empty_like(vals0)
        def oop_step(i):
            R.lsd_oop_tensors(kbufs[i % nbuf], vbufs[i % nbuf], ka, va, digit_bits=db)
        for i in range(min(nbuf, a.steps + a.warmup)):
            refill(i)
        for i in range(a.warmup):
            oop_step(i)
        for i in range(min(a.warmup, nbuf)):
            refill(i)
        barrier()
        o0, o1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        o0.record(stream)
        for s in range(a.steps):
            if s >= nbuf:
                refill(s % nbuf)
            oop_step(s)
        o1.record(stream)
        barrier()
        R.radsort_device_status()
        oms = o0.elapsed_time(o1)
        oval = world * a.steps * n / (oms / 1e3) / 1e9
        oop = {"value": round(oval, 3), "unit": "Gkeys/s", "ms_per_step": oms / a.steps,
               # the alternate arrays plus histograms and the look-back ring
               "extra_bytes": n * E + R.radsort_lsd_oop_scratch_size(n, kb, 4, db),
               "radsort_over_oop": round(value / oval, 4)}
        del ka, va

    # ---- the other single-array workloads, each with its comparator
    extra = None
    if not a.no_extra and world == 1:
        kbufs.clear()
        vbufs.clear()
        del ws
        torch.cuda.empty_cache()
        extra = {}
        for lg, kb2, db2 in ((28, 4, 8), (30, 8, 8), (30, 8, 11)):
            if (lg, kb2, db2) == (a.log2n, kb, db):
                continue
            key = f"{'u32' if kb2 == 4 else 'u64'}_2^{lg}_d{db2}"
            extra[key] = time_workload(R, W, dev, lg, kb2, db2, min(a.steps, 6), max(3, min(a.warmup, 3)),
                                       barrier, stream)
        # the MSD split of Sec. 4.3 on the headline workload (its comparator
        # is the line's own oop)
        extra[f"msd_split_{'u32' if kb == 4 else 'u64'}_2^{a.log2n}_d{db}"] = (
            time_workload(R, W, dev, a.log2n, kb, db, min(a.steps, 6), max(3, min(a.warmup, 3)), barrier,
                          stream, layout="msd", with_oop=False) if db == 8 else None)

    # ---- a short serving run (config 5, 200 requests), both methods
    serve_line = None
    if not a.no_serve and world == 1:
        from paper_2607_05302_gb300 import serve

        torch.cuda.empty_cache()
        sv = serve.run_bench(steps=200, tight_cap=SERVE_TIGHT_CAP)

        def pick(d):
            return {m: {k: (round(v, 3) if isinstance(v, float) else v) for k, v in d[m].items()
                        if k in ("p50_ms", "p99_ms", "keys_per_s", "peak_concurrency", "peak_bytes")}
                    for m in ("radsort", "oop")}

        serve_line = {"requests": 200, "cap_bytes": sv["config"]["cap_bytes"], **pick(sv),
                      "tight_cap": {"cap_bytes": sv["tight_cap"]["cap_bytes"], **pick(sv["tight_cap"])}}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        rate, sample, el = oracle_sample_rate(a, a.cpu_seconds)
        cpu = {"value": rate, "unit": "Gkeys/s", "cores": 1, "kind": "oracle", "sample": sample,
               "seconds": round(el, 2), "host_cores_available": os.cpu_count(), "cpu": host_cpu()}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "Gkeys/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_max / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32" if kb == 4 else "u64", "data": "synthetic",
            "config": {"workload": workload_name(a), "n": n, "key_bytes": kb, "value_bytes": 4,
                       "digit_bits": db, "layout": "chunks" if lay == "chunks" else "grid",
                       "block_size": bs, "num_chunks": pc,
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2: each timed step sorts its own fresh 2^%d-element copy" % a.log2n,
                       "extra": "uniform keys, automatic plan, comparator beside each; fresh copies per step"},
            "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu,
            "clocks": clk, "extra_bytes": wsb, "extra_frac": round(wsb / (n * E), 5),
            "oop": oop, "chunk_layout": plan2, "extra": extra, "serve": serve_line,
            "phases_ms": {k: round(statistics.mean(v), 4) for k, v in phases.items()},
            "finalize": finalize,
            "algorithmic_bytes_per_step": step_bytes,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
