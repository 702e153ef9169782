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
