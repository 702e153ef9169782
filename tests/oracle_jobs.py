"""Oracle results for the full-size parity tests, computed in worker processes.

Each job regenerates its input on the host from the seeded generators (the
same bytes the device sorts), runs the oracle, and writes the expected keys
and values as .npy files; the test maps them back.  The workers are started
with the 'spawn' method, so they never inherit a CUDA context, and they
import numpy and the oracle only.
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _radsort(keys, vals, key_bits, digit_bits, b=4096):
    import oracle

    n_t = oracle.digits_for(key_bits, digit_bits)
    k, v = oracle.radsort(keys, vals, n_t=n_t, sigma=1 << digit_bits, bits=digit_bits, b=b, p=1,
                          elem_bytes=key_bits // 8 + 4)
    return k.astype(keys.dtype), v


def run(job, outdir):
    """job: ("u32", dist, log2n) | ("u64", digit_bits, log2n) | ("seg",).
    Returns the paths of the expected keys and values."""
    import oracle
    from paper_2607_05302_gb300 import workloads as W

    kind = job[0]
    if kind == "u32":
        dist, lg = job[1], job[2]
        n = 1 << lg
        host = W.make_keys(dist, n)
        vals = W.index_payload(n)
        if dist == "float":
            ek, ev = _radsort(oracle.f32_to_ordered(host), vals, 32, 8)
            ek = oracle.ordered_to_f32(ek)
        else:
            ek, ev = _radsort(host, vals, 32, 8)
    elif kind == "u64":
        db, lg = job[1], job[2]
        n = 1 << lg
        ek, ev = _radsort(W.make_keys("uniform", n, 64), W.index_payload(n), 64, db)
    elif kind == "seg":
        # Alg. 1 on the composite key segment * 2^32 + key: segments stay
        # apart, keys sort inside them, equal keys keep their index order
        lens = W.lognormal_lengths(20000)
        n = int(lens.sum())
        host = W.make_keys("uniform", n)
        seg = np.repeat(np.arange(lens.size, dtype=np.uint64), lens)
        comp = (seg << np.uint64(32)) | host.astype(np.uint64)
        del seg, host
        bits = 32 + int(lens.size - 1).bit_length()
        ck, ev = oracle.lsd_oop(comp, W.index_payload(n), n_t=oracle.digits_for(bits, 8), sigma=256,
                                bits=8)
        del comp
        ek = (ck & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    else:
        raise ValueError(job)
    name = "_".join(str(x) for x in job)
    pk, pv = os.path.join(outdir, name + "_k.npy"), os.path.join(outdir, name + "_v.npy")
    np.save(pk, ek)
    np.save(pv, ev)
    return pk, pv
