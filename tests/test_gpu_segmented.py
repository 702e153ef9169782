"""GPU parity of the batched segmented sort (many independent arrays in one
call) against the oracle, and the 20,000-segment lognormal workload at full
size by properties that fix a stable sort."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_05302_gb300 import radsort as R
from paper_2607_05302_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def offsets_of(lengths):
    off = np.zeros(len(lengths) + 1, dtype=np.uint64)
    np.cumsum(np.asarray(lengths, dtype=np.uint64), out=off[1:])
    return off


def run_segmented(keys_np, lengths, digit_bits=8, caller_ws=True, minimal=False):
    off = offsets_of(lengths)
    n = int(off[-1])
    kt = torch.from_numpy(keys_np.view(np.int32 if keys_np.dtype == np.uint32 else np.int64)).to(DEV)
    vt = torch.arange(n, dtype=torch.int32, device=DEV)
    od = torch.from_numpy(off.view(np.int64)).to(DEV)
    ws = None
    if caller_ws:
        need = R.segmented_workspace_size(off, keys_np.itemsize, 4, digit_bits, minimal=minimal)
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device=DEV)
    R.sort_segmented_tensors(kt, vt, od, off, digit_bits=digit_bits, workspace=ws)
    R.radsort_device_status()
    return kt, vt, off


def oracle_segmented_u32(keys, lengths, digit_bits=8):
    """The oracle's stable LSD sort on the composite key (segment << 32 | key):
    per-segment stable sort, in one oracle call."""
    seg = np.repeat(np.arange(len(lengths), dtype=np.uint64), lengths)
    comp = (seg << np.uint64(32)) | keys.astype(np.uint64)
    nbits = 32 + max(1, int(len(lengths) - 1).bit_length())
    n_t = oracle.digits_for(nbits, digit_bits)
    k, v = oracle.lsd_oop(comp, np.arange(keys.size, dtype=np.uint32), n_t=n_t, sigma=1 << digit_bits,
                          bits=digit_bits)
    return (k & np.uint64(0xFFFFFFFF)).astype(np.uint32), v


LENGTH_SETS = {
    # every class: tiny, small (<= 4096), medium (<= 2^18), large aligned and misaligned
    "mixed": [1, 0, 2, 17, 4095, 4096, 4097, 70000, 1 << 18, (1 << 18) + 1, 300001, 3, 5000,
              (1 << 18) + 4, 12345],
    "many_small": list(W.lognormal_lengths(3000, median=300.0, sigma_ln=1.5, lo=0, hi=5000)),
}


@pytest.mark.parametrize("lengths", list(LENGTH_SETS), ids=list(LENGTH_SETS))
@pytest.mark.parametrize("digit_bits", [8, 11])
def test_segmented_u32_vs_oracle(lengths, digit_bits):
    lens = [int(x) for x in LENGTH_SETS[lengths]]
    n = sum(lens)
    rng = np.random.default_rng(len(lens) + digit_bits)
    keys = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    keys[::5] = keys[0]  # ties across and within segments
    kt, vt, _ = run_segmented(keys, lens, digit_bits)
    ek, ev = oracle_segmented_u32(keys, lens, digit_bits)
    assert np.array_equal(kt.cpu().numpy().view(np.uint32), ek)
    assert np.array_equal(vt.cpu().numpy().view(np.uint32), ev)


# medium lengths on and off the 32-element block grid, on both sides of the
# in-place threshold (16448 = 514 blocks of 32), and two short ones
MEDIUM_SET = [4097, 4128, 8192, 16448, 16449, 20000, 65536, 65537, 100000, 131071, 262143, 262144, 33, 4099]


@pytest.mark.parametrize("dist", ["uniform", "equal", "sorted", "reverse", "zipf", "few"])
def test_low_memory_plan_medium_segments_vs_oracle(dist):
    """The low-memory plan (a caller workspace of the minimal size): medium
    segments sorted in place by one CTA each, several per CTA, with key
    distributions that give the block maps different shapes (one bucket per
    round, runs in input order or reversed, a few heavy buckets, three
    distinct keys); bit-exact against the oracle's stable sort of each
    segment."""
    lens = MEDIUM_SET * 3
    off = offsets_of(lens)
    assert R.segmented_workspace_size(off, 4, 4, 8, minimal=True) < R.segmented_workspace_size(off, 4, 4, 8)
    n = sum(lens)
    if dist == "few":
        keys = (W.make_keys("uniform", n) % np.uint32(3)) * np.uint32(0x01010101)
    else:
        keys = W.make_keys(dist, n)
    kt, vt, _ = run_segmented(keys, lens, 8, minimal=True)
    ek, ev = oracle_segmented_u32(keys, lens, 8)
    assert np.array_equal(kt.cpu().numpy().view(np.uint32), ek)
    assert np.array_equal(vt.cpu().numpy().view(np.uint32), ev)


def test_low_memory_plan_mixed_and_u64_keys_only():
    """The low-memory plan beside long and short segments, and with 8-byte
    keys and no values."""
    lens = [int(x) for x in LENGTH_SETS["mixed"]] + [40000, 200000]
    n = sum(lens)
    keys = W.make_keys("uniform", n)
    kt, vt, _ = run_segmented(keys, lens, 8, minimal=True)
    ek, ev = oracle_segmented_u32(keys, lens, 8)
    assert np.array_equal(kt.cpu().numpy().view(np.uint32), ek)
    assert np.array_equal(vt.cpu().numpy().view(np.uint32), ev)
    lens = [4097, 70001, 262144, 5000, 131072, 17000]
    n = sum(lens)
    keys = W.make_keys("uniform", n, 64)
    keys[::7] = keys[5]  # ties
    off = offsets_of(lens)
    need = R.segmented_workspace_size(off, 8, 0, 8, minimal=True)
    assert need < R.segmented_workspace_size(off, 8, 0, 8)
    kt = torch.from_numpy(keys.view(np.int64)).to(DEV)
    od = torch.from_numpy(off.view(np.int64)).to(DEV)
    ws = torch.empty(need, dtype=torch.uint8, device=DEV)
    R.sort_segmented_tensors(kt, None, od, off, digit_bits=8, workspace=ws)
    R.radsort_device_status()
    got = kt.cpu().numpy().view(np.uint64)
    for s_ in range(len(lens)):
        a, b = int(off[s_]), int(off[s_ + 1])
        ek, _ = oracle.lsd_oop(keys[a:b], np.arange(b - a, dtype=np.uint32), n_t=8, sigma=256, bits=8)
        assert np.array_equal(got[a:b], ek)


@pytest.mark.parametrize("head", [1, 2, 3])
@pytest.mark.parametrize("kind", ["few", "uniform", "u64"])
def test_low_memory_plan_unaligned_long_segment(head, kind):
    """A long segment whose start is `head` elements short of a 16-byte
    boundary, in the low-memory plan: its first elements are set aside, the
    aligned rest is sorted by Radsort and they are merged back, each before
    the equal keys that followed it.  Three distinct keys make nearly every
    element a tie; bit-exact against the oracle."""
    lens = [4 - head, 300001, 5]
    n = sum(lens)
    off = offsets_of(lens)
    if kind == "u64":
        keys = W.make_keys("uniform", n, 64)
        keys[::3] = keys[4]  # the head's key among the ties
    else:
        keys = W.make_keys("uniform", n)
        if kind == "few":
            keys = (keys % np.uint32(3)) * np.uint32(0x01010101)
    need = R.segmented_workspace_size(off, keys.itemsize, 4, 8, minimal=True)
    assert need < R.segmented_workspace_size(off, keys.itemsize, 4, 8)
    kt, vt, _ = run_segmented(keys, lens, 8, minimal=True)
    if kind == "u64":
        got_k, got_v = kt.cpu().numpy().view(np.uint64), vt.cpu().numpy().view(np.uint32)
        for s_ in range(len(lens)):
            a, b = int(off[s_]), int(off[s_ + 1])
            ek, ev = oracle.lsd_oop(keys[a:b], np.arange(a, b, dtype=np.uint32), n_t=8, sigma=256, bits=8)
            assert np.array_equal(got_k[a:b], ek) and np.array_equal(got_v[a:b], ev)
    else:
        ek, ev = oracle_segmented_u32(keys, lens, 8)
        assert np.array_equal(kt.cpu().numpy().view(np.uint32), ek)
        assert np.array_equal(vt.cpu().numpy().view(np.uint32), ev)


@pytest.mark.parametrize("digit_bits", [8, 11])
def test_segmented_u64_vs_oracle(digit_bits):
    lens = [5, 4096, 2049, 300000, 77777, 1 << 18, (1 << 18) + 2, 1]
    n = sum(lens)
    keys = W.make_keys("uniform", n, 64)
    keys[::3] = keys[1]
    kt, vt, off = run_segmented(keys, lens, digit_bits)
    gk = kt.cpu().numpy().view(np.uint64)
    gv = vt.cpu().numpy().view(np.uint32)
    n_t = oracle.digits_for(64, digit_bits)
    for s in range(len(lens)):
        a, b = int(off[s]), int(off[s + 1])
        ek, ev = oracle.lsd_oop(keys[a:b], np.arange(a, b, dtype=np.uint32), n_t=n_t,
                                sigma=1 << digit_bits, bits=digit_bits)
        assert np.array_equal(gk[a:b], ek) and np.array_equal(gv[a:b], ev), s


def test_segmented_keys_only_and_internal_workspace():
    lens = [100, 5000, 300000, 1, 0, 9999]
    n = sum(lens)
    keys = W.make_keys("uniform", n)
    off = offsets_of(lens)
    kt = torch.from_numpy(keys.view(np.int32)).to(DEV)
    od = torch.from_numpy(off.view(np.int64)).to(DEV)
    R.sort_segmented_tensors(kt, None, od, off)
    R.radsort_device_status()
    got = kt.cpu().numpy().view(np.uint32)
    for s in range(len(lens)):
        a, b = int(off[s]), int(off[s + 1])
        assert np.array_equal(got[a:b], np.sort(keys[a:b]))


def test_config4_20000_lognormal_segments_properties():
    """20,000 uint32 arrays, lengths lognormal (median 4096, natural-log sigma
    2, clipped to [16, 2^22]), index payloads, one call."""
    lens = W.lognormal_lengths(20000)
    off = offsets_of(lens)
    n = int(off[-1])
    r = W.splitmix64_torch(W.SEEDS["uniform"], 0, n, device=DEV)
    keys0 = ((r >> 32) & 0xFFFFFFFF).to(torch.int64)
    del r
    kt = keys0.to(torch.int32)
    vt = torch.arange(n, dtype=torch.int32, device=DEV)
    od = torch.from_numpy(off.view(np.int64)).to(DEV)
    need = R.segmented_workspace_size(off, 4, 4)
    ws = torch.empty(need, dtype=torch.uint8, device=DEV)
    R.sort_segmented_tensors(kt, vt, od, off, workspace=ws)
    R.radsort_device_status()
    seg = torch.repeat_interleave(torch.arange(len(lens), device=DEV),
                                  torch.from_numpy(lens.astype(np.int64)).to(DEV))
    v = vt.to(torch.int64) & 0xFFFFFFFF
    k = kt.to(torch.int64) & 0xFFFFFFFF
    assert torch.equal(torch.sort(v).values, torch.arange(n, device=DEV))  # a permutation
    assert torch.equal(seg[v], seg)  # that stays inside each segment
    assert torch.equal(keys0[v], k)  # carrying each key with its payload
    same = seg[1:] == seg[:-1]
    assert bool((k[1:][same] >= k[:-1][same]).all())  # sorted per segment
    eq = same & (k[1:] == k[:-1])
    assert bool((v[1:][eq] > v[:-1][eq]).all())  # stable


LONG_SET = [300001, 5000, (1 << 18) + 1, 17, 400000, (1 << 20) + 3, 1, 262145, 70000, 600000]


def test_long_segments_on_several_streams_vs_oracle():
    """Six long segments (above 2^18, aligned and misaligned starts) spread
    over the library's streams, between short ones: the same result as the
    oracle's per-segment stable sort."""
    n = sum(LONG_SET)
    rng = np.random.default_rng(77)
    keys = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    keys[::7] = keys[2]
    kt, vt, _ = run_segmented(keys, LONG_SET)
    ek, ev = oracle_segmented_u32(keys, LONG_SET)
    assert np.array_equal(kt.cpu().numpy().view(np.uint32), ek)
    assert np.array_equal(vt.cpu().numpy().view(np.uint32), ev)


@pytest.mark.parametrize("lengths", ["mixed", "long"])
def test_out_of_place_comparator_vs_oracle(lengths):
    """radsort_lsd_oop_sort_segmented: the same arrays through n-element
    alternate arrays give the oracle's result."""
    lens = [int(x) for x in (LENGTH_SETS["mixed"] if lengths == "mixed" else LONG_SET)]
    off = offsets_of(lens)
    n = int(off[-1])
    rng = np.random.default_rng(n)
    keys = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    kt = torch.from_numpy(keys.view(np.int32)).to(DEV)
    vt = torch.arange(n, dtype=torch.int32, device=DEV)
    ka, va = torch.empty_like(kt), torch.empty_like(vt)
    od = torch.from_numpy(off.view(np.int64)).to(DEV)
    ws = torch.empty(max(R.lsd_oop_segmented_workspace_size(off, 4, 4), 1), dtype=torch.uint8, device=DEV)
    R.lsd_oop_segmented_tensors(kt, vt, ka, va, od, off, workspace=ws)
    R.radsort_device_status()
    ek, ev = oracle_segmented_u32(keys, lens)
    assert np.array_equal(kt.cpu().numpy().view(np.uint32), ek)
    assert np.array_equal(vt.cpu().numpy().view(np.uint32), ev)


@pytest.mark.parametrize("minimal", [False, True])
def test_captured_graph_with_long_segments(minimal):
    """The call with long segments captured in a CUDA graph (fork and join
    over the library's streams inside the capture) and replayed twice on
    fresh copies gives the oracle's result each time; with the smallest
    workspace too (medium segments in place, unaligned long ones with their
    first elements merged back)."""
    lens = LONG_SET + ([3, 40000, 70001] if minimal else [])
    off = offsets_of(lens)
    n = int(off[-1])
    keys = W.make_keys("uniform", n)
    k0 = torch.from_numpy(keys.view(np.int32)).to(DEV)
    kt, vt = k0.clone(), torch.arange(n, dtype=torch.int32, device=DEV)
    v0 = vt.clone()
    od = torch.from_numpy(off.view(np.int64)).to(DEV)
    need = R.segmented_workspace_size(off, 4, 4, minimal=minimal)
    if minimal:
        assert need < R.segmented_workspace_size(off, 4, 4)
    ws = torch.empty(need, dtype=torch.uint8, device=DEV)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        R.sort_segmented_tensors(kt, vt, od, off, workspace=ws)  # first call: the streams exist
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        R.sort_segmented_tensors(kt, vt, od, off, workspace=ws)
    ek, ev = oracle_segmented_u32(keys, lens)
    for _ in range(2):
        kt.copy_(k0)
        vt.copy_(v0)
        g.replay()
        torch.cuda.synchronize()
        R.radsort_device_status()
        assert np.array_equal(kt.cpu().numpy().view(np.uint32), ek)
        assert np.array_equal(vt.cpu().numpy().view(np.uint32), ev)


def test_segmented_autotune_leaves_inputs_and_picks_a_width():
    lens = [int(x) for x in LENGTH_SETS["mixed"]]
    off = offsets_of(lens)
    n = int(off[-1])
    keys = W.make_keys("uniform", n)
    kt = torch.from_numpy(keys.view(np.int32)).to(DEV)
    vt = torch.arange(n, dtype=torch.int32, device=DEV)
    od = torch.from_numpy(off.view(np.int64)).to(DEV)
    db = R.segmented_autotune(kt, vt, od, off)
    assert db in (8, 11)
    assert np.array_equal(kt.cpu().numpy().view(np.uint32), keys)
    kt2, vt2, _ = run_segmented(keys, lens, db)
    ek, ev = oracle_segmented_u32(keys, lens, db)
    assert np.array_equal(kt2.cpu().numpy().view(np.uint32), ek)
    assert np.array_equal(vt2.cpu().numpy().view(np.uint32), ev)
