"""Seeded synthetic inputs for the sort workloads.

This module holds only input generation, none of the sort's arithmetic.  The
same bytes serve the CUDA path, the oracle, the tests and the benchmark.

Uniform keys come from the counter-based SplitMix64 generator (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014; the
finaliser constants are the published ones).  Element i of a stream with seed s
is mix64(s + (i + 1) * 0x9E3779B97F4A7C15).  The generator has a numpy form (host)
and a torch form (any device; bit-identical, checked by the tests), so the
large inputs can be made on the GPU and the small ones on the host.

Zipf keys and float32 N(0,1) keys depend on floating-point library routines.
They are made on the host with numpy only and then uploaded, so both sides
sort identical bytes.

The distributions follow the workloads of the paper's evaluation
(32-bit keys, 32-bit values, uniform keys) and the sort configurations this
package is measured on: Zipf(s=1.1) over 2^16 distinct values, all-equal,
already sorted, reverse sorted, and float32 N(0,1).
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)

SEEDS = {  # fixed per workload
    "uniform": 0xC0FFEE01,
    "zipf": 0xC0FFEE02,
    "equal": 0xC0FFEE03,
    "sorted": 0xC0FFEE04,
    "reverse": 0xC0FFEE05,
    "float": 0xC0FFEE06,
}

DISTRIBUTIONS = ("uniform", "zipf", "equal", "sorted", "reverse", "float")


def _mix64_np(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * M1
    z = (z ^ (z >> np.uint64(27))) * M2
    return z ^ (z >> np.uint64(31))


def splitmix64_np(seed: int, start: int, count: int) -> np.ndarray:
    """uint64 stream elements [start, start+count) of SplitMix64(seed)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        x = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GOLDEN
        return _mix64_np(x)


def _i64(c: int) -> int:
    c &= 0xFFFFFFFFFFFFFFFF
    return c - (1 << 64) if c >= (1 << 63) else c


def splitmix64_torch(seed: int, start: int, count: int, device="cpu"):
    """Same stream as splitmix64_np, as int64 bit patterns (torch has no
    full uint64 arithmetic; two's-complement wraparound gives identical bits)."""
    import torch

    i = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    x = i * _i64(0x9E3779B97F4A7C15) + _i64(seed)

    def lsr(v, k):  # logical right shift of int64 bit patterns
        return (v >> k) & ((1 << (64 - k)) - 1)

    x = (x ^ lsr(x, 30)) * _i64(0xBF58476D1CE4E5B9)
    x = (x ^ lsr(x, 27)) * _i64(0x94D049BB133111EB)
    return x ^ lsr(x, 31)


def fmix32_np(h: np.ndarray) -> np.ndarray:
    """MurmurHash3's 32-bit finaliser (a bijection on uint32)."""
    h = h.astype(np.uint32, copy=True)
    with np.errstate(over="ignore"):
        h ^= h >> np.uint32(16)
        h *= np.uint32(0x85EBCA6B)
        h ^= h >> np.uint32(13)
        h *= np.uint32(0xC2B2AE35)
        h ^= h >> np.uint32(16)
    return h


def _chunks(n, step=1 << 24):
    s = 0
    while s < n:
        yield s, min(step, n - s)
        s += step


def uniform_keys(n: int, key_bits: int = 32, seed: int | None = None) -> np.ndarray:
    """Keys uniform over [0, 2^key_bits) (key_bits 32 or 64), host numpy."""
    seed = SEEDS["uniform"] if seed is None else seed
    out = np.empty(n, np.uint32 if key_bits == 32 else np.uint64)
    for s, c in _chunks(n):
        r = splitmix64_np(seed, s, c)
        out[s:s + c] = (r >> np.uint64(32)).astype(np.uint32) if key_bits == 32 else r
    return out


def zipf_keys(n: int, s: float = 1.1, distinct: int = 1 << 16, seed: int | None = None):
    """Zipf(s) over `distinct` ranks by inverse CDF; rank r maps to the value
    fmix32(r ^ seed32) so every digit position varies."""
    seed = SEEDS["zipf"] if seed is None else seed
    w = np.arange(1, distinct + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    out = np.empty(n, np.uint32)
    for st, c in _chunks(n):
        u = (splitmix64_np(seed, st, c) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        rank = np.minimum(np.searchsorted(cdf, u, side="right"), distinct - 1).astype(np.uint32)
        out[st:st + c] = fmix32_np(rank ^ np.uint32(seed & 0xFFFFFFFF))
    return out


def float_normal_bits(n: int, seed: int | None = None) -> np.ndarray:
    """float32 N(0,1) samples (Box-Muller on SplitMix64 uniforms), as raw bits."""
    seed = SEEDS["float"] if seed is None else seed
    out = np.empty(n, np.float32)
    for st, c in _chunks(n):
        r = splitmix64_np(seed, 2 * st, 2 * c)
        u1 = ((r[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
        u2 = (r[1::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        out[st:st + c] = (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)).astype(np.float32)
    return out.view(np.uint32)


def make_keys(dist: str, n: int, key_bits: int = 32) -> np.ndarray:
    """Host keys for one of DISTRIBUTIONS ('float' gives raw float32 bits)."""
    if dist == "uniform":
        return uniform_keys(n, key_bits)
    if key_bits != 32 and dist in ("zipf", "float"):
        raise ValueError(f"{dist} keys are 32-bit")
    if dist == "zipf":
        return zipf_keys(n)
    if dist == "float":
        return float_normal_bits(n)
    dt = np.uint32 if key_bits == 32 else np.uint64
    if dist == "equal":
        v = splitmix64_np(SEEDS["equal"], 0, 1)[0]
        v = (v >> np.uint64(32)) if key_bits == 32 else v
        return np.full(n, v, dtype=dt)
    if dist in ("sorted", "reverse"):
        k = np.sort(uniform_keys(n, key_bits, seed=SEEDS[dist]))
        return k if dist == "sorted" else k[::-1].copy()
    raise ValueError(dist)


def index_payload(n: int) -> np.ndarray:
    """uint32 payload = original index (the stability check of the configs)."""
    return np.arange(n, dtype=np.uint32)


def lognormal_lengths(num: int, median: float = 4096.0, sigma_ln: float = 2.0,
                      lo: int = 16, hi: int = 1 << 22, seed: int = 0xC0FFEE07):
    """Segment lengths, lognormal (natural-log sigma), clipped to [lo, hi]."""
    r = splitmix64_np(seed, 0, 2 * num)
    u1 = ((r[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
    u2 = (r[1::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    L = np.exp(np.log(median) + sigma_ln * z)
    return np.clip(np.round(L), lo, hi).astype(np.int64)
