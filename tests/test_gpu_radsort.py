"""GPU parity: the CUDA Radsort (through the C ABI) against the oracle, element
by element, bit-exact (the result of a stable sort is unique, so there is no
tolerance).  Sizes span several tiles and chunks with ragged tails; the
launch configurations include the automatic plan that bench.py uses."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_05302_gb300 import radsort as R
from paper_2607_05302_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def to_dev(a):
    return torch.from_numpy(a.view(np.int32 if a.dtype == np.uint32 else np.int64)).to(DEV)


def from_dev(t, dtype):
    return t.cpu().numpy().view(dtype)


def gpu_sort(keys, vals, digit_bits=8, float_keys=False, block_size=0, num_chunks=0, layout=0, shape=0):
    kt = to_dev(keys)
    vt = None if vals is None else to_dev(vals)
    R.sort_tensors(kt, vt, digit_bits=digit_bits, float_keys=float_keys, block_size=block_size,
                   num_chunks=num_chunks, layout=layout, shape=shape)
    R.radsort_device_status()
    return from_dev(kt, keys.dtype), (None if vt is None else from_dev(vt, np.uint32))


def oracle_sort(keys, vals, key_bits, digit_bits):
    n_t = oracle.digits_for(key_bits, digit_bits)
    k, v = oracle.radsort(keys, vals, n_t=n_t, sigma=1 << digit_bits, bits=digit_bits, b=256, p=1,
                          elem_bytes=key_bits // 8 + 4)
    return k.astype(keys.dtype), v


SIZES = [2, 3, 63, 64, 65, 255, 256, 257, 4095, 4096, 4097, 10000, 65543, 300001]
# (block size, chunks, layout): the chunk layout of Sec. 4.3 and the grid
# layout (one chain per bucket on the output block grid); (0, 0, auto) is the
# automatic plan that bench.py times
PLANS = [(64, 1, "chunks"), (64, 3, "chunks"), (256, 2, "chunks"), (1024, 4, "chunks"),
         (4096, 1, "chunks"), (256, 300, "chunks"), (64, 0, "grid"), (256, 0, "grid"),
         (512, 0, "grid"), (2048, 0, "grid"), (0, 0, "scratch"), (0, 0, "auto")]
PLAN_IDS = [f"{l}-b{b}-p{p}" for b, p, l in PLANS]


@pytest.mark.parametrize("plan", PLANS, ids=PLAN_IDS)
@pytest.mark.parametrize("n", SIZES)
def test_u32_d8_ragged(n, plan):
    rng = np.random.default_rng(n)
    for keys in (rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32),
                 rng.integers(0, 700, n, dtype=np.uint64).astype(np.uint32)):
        vals = W.index_payload(n)
        gk, gv = gpu_sort(keys, vals, block_size=plan[0], num_chunks=plan[1], layout=plan[2])
        ek, ev = oracle_sort(keys, vals, 32, 8)
        assert np.array_equal(gk, ek) and np.array_equal(gv, ev)


@pytest.mark.parametrize("plan", [(64, 3, "chunks"), (256, 5, "chunks"), (1024, 2, "chunks"),
                                  (64, 0, "grid"), (512, 0, "grid")])
def test_logical_sequence_each_round(plan):
    """After r rounds the permuted representation (Sec. 4.1) read in logical
    order equals r rounds of Alg. 1 in the oracle."""
    n = 50001
    keys = W.make_keys("uniform", n)
    keys[::3] = keys[1]  # ties
    vals = W.index_payload(n)
    for r in range(5):
        kt, vt = to_dev(keys), to_dev(vals)
        ok = torch.empty_like(kt)
        ov = torch.empty_like(vt)
        R.sort_rounds_tensors(kt, vt, r, ok, ov, digit_bits=8, block_size=plan[0], num_chunks=plan[1],
                              layout=plan[2])
        R.radsort_device_status()
        lk, lv = oracle.lsd_oop(keys, vals, n_t=4, sigma=256, bits=8, rounds=r)
        assert np.array_equal(from_dev(ok, np.uint32), lk.astype(np.uint32))
        assert np.array_equal(from_dev(ov, np.uint32), lv)


@pytest.mark.parametrize("n", [64 * 11263 + 17, 64 * 11264 + 5])
def test_finalize_small_and_large_pointer_jumping(n):
    """Grid layout, blocks of 64: n_pi = n/64 + 1025 is 12288 (the largest
    map that Finalize pointer-jumps in one CTA in shared memory) or 12289
    (the multi-launch path); both against the oracle, with ties."""
    rng = np.random.default_rng(n)
    keys = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    keys[::9] = keys[4]
    vals = W.index_payload(n)
    gk, gv = gpu_sort(keys, vals, block_size=64, num_chunks=0, layout="grid")
    ek, ev = oracle_sort(keys, vals, 32, 8)
    assert np.array_equal(gk, ek) and np.array_equal(gv, ev)


@pytest.mark.parametrize("layout", ["chunks", "grid", "scratch"])
@pytest.mark.parametrize("dist", W.DISTRIBUTIONS)
def test_config1_distributions(dist, layout):
    """n = 2^20 uint32 keys + index payload, sigma = 256, b = 1024."""
    n = 1 << 20
    keys = W.make_keys(dist, n)
    vals = W.index_payload(n)
    fl = dist == "float"
    gk, gv = gpu_sort(keys, vals, float_keys=fl, block_size=1024,
                      num_chunks=8 if layout == "chunks" else 0, layout=layout)
    ok_keys = oracle.f32_to_ordered(keys) if fl else keys
    ek, ev = oracle_sort(ok_keys, vals, 32, 8)
    if fl:
        ek = oracle.ordered_to_f32(ek)
    assert np.array_equal(gk, ek) and np.array_equal(gv, ev)


@pytest.mark.parametrize("digit_bits", [8, 11])
@pytest.mark.parametrize("with_vals", [True, False])
@pytest.mark.parametrize("plan", [(256, 3, "chunks"), (2048, 2, "chunks"), (256, 0, "grid"),
                                  (2048, 0, "grid"), (0, 0, "auto")])
def test_u64(digit_bits, with_vals, plan):
    n = 200003
    keys = W.make_keys("uniform", n, 64)
    keys[::11] = keys[5]
    vals = W.index_payload(n) if with_vals else None
    gk, gv = gpu_sort(keys, vals, digit_bits=digit_bits, block_size=plan[0], num_chunks=plan[1],
                      layout=plan[2])
    ek, ev = oracle_sort(keys, vals, 64, digit_bits)
    assert np.array_equal(gk, ek)
    if with_vals:
        assert np.array_equal(gv, ev)


@pytest.mark.parametrize("plan", [(256, 4, "chunks"), (512, 1, "chunks"), (256, 0, "grid"),
                                  (1024, 0, "grid")])
def test_u32_d11_and_keys_only(plan):
    n = 123457
    keys = W.make_keys("zipf", n)
    gk, _ = gpu_sort(keys, None, digit_bits=11, block_size=plan[0], num_chunks=plan[1], layout=plan[2])
    assert np.array_equal(gk, np.sort(keys))
    vals = W.index_payload(n)
    gk, gv = gpu_sort(keys, vals, digit_bits=11, block_size=plan[0], num_chunks=plan[1],
                      layout=plan[2])
    ek, ev = oracle_sort(keys, vals, 32, 11)
    assert np.array_equal(gk, ek) and np.array_equal(gv, ev)


@pytest.mark.parametrize("plan", [(512, 3, "chunks"), (512, 0, "grid"), (0, 0, "scratch")])
def test_caller_workspace_and_small_n(plan):
    n = 77777
    keys = W.make_keys("reverse", n)
    vals = W.index_payload(n)
    b, p, lay = plan
    need = R.radsort_workspace_size(n, 4, 4, 8, block_size=b, num_chunks=p, layout=lay)
    assert need >= (n * 8 if lay == "scratch" else 0)
    ws = torch.empty(need, dtype=torch.uint8, device=DEV)
    kt, vt = to_dev(keys), to_dev(vals)
    R.sort_tensors(kt, vt, block_size=b, num_chunks=p, layout=lay, workspace=ws)
    R.radsort_device_status()
    ek, ev = oracle_sort(keys, vals, 32, 8)
    assert np.array_equal(from_dev(kt, np.uint32), ek) and np.array_equal(from_dev(vt, np.uint32), ev)
    small = torch.empty(need - 256, dtype=torch.uint8, device=DEV)
    with pytest.raises(R.RadsortError):
        R.sort_tensors(kt, vt, block_size=b, num_chunks=p, layout=lay, workspace=small)
    for m in (0, 1):
        t = torch.zeros(m, dtype=torch.int32, device=DEV)
        R.sort_tensors(t, None)


@pytest.mark.parametrize("kb,db", [(4, 8), (4, 11), (8, 8), (8, 11)])
def test_lsd_oop_comparator(kb, db):
    n = 300007
    keys = W.make_keys("uniform", n, 8 * kb)
    keys[::7] = keys[2]
    vals = W.index_payload(n)
    kt, vt = to_dev(keys), to_dev(vals)
    ka, va = torch.empty_like(kt), torch.empty_like(vt)
    R.lsd_oop_tensors(kt, vt, ka, va, digit_bits=db)
    R.radsort_device_status()
    lk, lv = oracle.lsd_oop(keys, vals, n_t=oracle.digits_for(8 * kb, db), sigma=1 << db, bits=db)
    assert np.array_equal(from_dev(kt, keys.dtype), lk.astype(keys.dtype))
    assert np.array_equal(from_dev(vt, np.uint32), lv)


def check_sorted_stable_perm(orig_keys_t, keys_t, vals_t, key_bits):
    """Properties that fix the unique stable sort at any size: the payload is a
    permutation, keys[i] = orig[payload[i]], keys ascending, and equal keys
    keep increasing payloads."""
    n = keys_t.numel()
    mask = (1 << key_bits) - 1
    v = vals_t.to(torch.int64) & 0xFFFFFFFF
    assert torch.equal(torch.sort(v).values, torch.arange(n, device=keys_t.device))
    assert torch.equal(orig_keys_t[v], keys_t)
    if key_bits == 32:
        k = keys_t.to(torch.int64) & mask
        assert bool((k[1:] >= k[:-1]).all())
        eq = k[1:] == k[:-1]
    else:  # compare 64-bit unsigned via the sign-flipped signed view
        k = keys_t ^ (-(2 ** 63))
        assert bool((k[1:] >= k[:-1]).all())
        eq = keys_t[1:] == keys_t[:-1]
    assert bool((v[1:][eq] > v[:-1][eq]).all())


def chunk_plan():
    """The chunk layout with one chunk per SM, b = 256 (bench.py times it
    beside the automatic plan)."""
    return 256, torch.cuda.get_device_properties(0).multi_processor_count


@pytest.mark.parametrize("plan", ["auto", "chunks"])
@pytest.mark.parametrize("dist", ["uniform", "zipf", "equal", "sorted", "reverse"])
def test_full_size_2p28_properties(dist, plan):
    """n = 2^28 uint32 keys + index payload, in the automatic plan (the grid
    layout, bench.py's launch configuration) and in the chunk layout with one
    chunk per SM."""
    n = 1 << 28
    keys = torch.from_numpy(W.make_keys(dist, n).view(np.int32)).to(DEV)
    vals = torch.arange(n, dtype=torch.int32, device=DEV)
    kt = keys.clone()
    bs, pc = chunk_plan() if plan == "chunks" else (0, 0)
    R.sort_tensors(kt, vals, block_size=bs, num_chunks=pc)
    R.radsort_device_status()
    check_sorted_stable_perm(keys, kt, vals, 32)
    # sampled outputs the oracle computes one by one: rank of sampled keys
    host = W.make_keys(dist, n)
    for idx in (0, n // 3, n - 1):
        pos = int((vals == idx).nonzero()[0, 0])
        k = host[idx]
        assert pos == int((host < k).sum()) + int((host[:idx] == k).sum())


@pytest.mark.parametrize("plan", ["auto", "chunks"])
def test_full_size_float_2p28(plan):
    """float32 N(0,1) keys at 2^28 through the order-preserving transform."""
    n = 1 << 28
    host = W.make_keys("float", n)
    keys = torch.from_numpy(host.view(np.int32)).to(DEV)
    vals = torch.arange(n, dtype=torch.int32, device=DEV)
    kt = keys.clone()
    bs, pc = chunk_plan() if plan == "chunks" else (0, 0)
    R.sort_tensors(kt, vals, float_keys=True, block_size=bs, num_chunks=pc)
    R.radsort_device_status()
    f = kt.view(torch.float32)
    assert bool((f[1:] >= f[:-1]).all())
    v = vals.to(torch.int64) & 0xFFFFFFFF
    assert torch.equal(keys[v], kt)
    assert torch.equal(torch.sort(v).values, torch.arange(n, device=DEV))


@pytest.mark.parametrize("db", [8, 11])
def test_full_size_2p30_u64_properties(db):
    """n = 2^30 uint64 keys uniform 64-bit + uint32 payloads (8-bit digits:
    n_t = 8; 11-bit digits: n_t = 6), automatic plan."""
    n = 1 << 30
    r = W.splitmix64_torch(W.SEEDS["uniform"], 0, n, device=DEV)
    kt = r.clone()
    vals = torch.arange(n, dtype=torch.int32, device=DEV)
    R.sort_tensors(kt, vals, digit_bits=db)
    R.radsort_device_status()
    check_sorted_stable_perm(r, kt, vals, 64)


@pytest.mark.parametrize("dist", ["uniform", "zipf"])
def test_u32_d11_look_back_ring_reused(dist):
    """11-bit digits at n = 2^26 uint32 keys: 8192 tiles of keys + values and
    4096 of keys alone, more than the look-back ring's 1024 rows, so ring
    slots are reused within every round; with and without payloads."""
    n = 1 << 26
    keys = torch.from_numpy(W.make_keys(dist, n).view(np.int32)).to(DEV)
    vals = torch.arange(n, dtype=torch.int32, device=DEV)
    kt = keys.clone()
    R.sort_tensors(kt, vals, digit_bits=11)
    R.radsort_device_status()
    check_sorted_stable_perm(keys, kt, vals, 32)
    ko = keys.clone()
    R.sort_tensors(ko, None, digit_bits=11)
    R.radsort_device_status()
    assert torch.equal(ko, kt)


def _check_large(orig, kt, vals):
    """Sorted (unsigned), payload a permutation with keys[i] = orig[payload[i]],
    equal keys in payload order: chunked to bound the temporaries."""
    n = kt.numel()
    v = vals.to(torch.int64) & 0xFFFFFFFF
    seen = torch.zeros(n, dtype=torch.bool, device=DEV)
    seen[v] = True
    assert bool(seen.all())
    del seen
    step = 1 << 28
    for s in range(0, n, step):
        e = min(n, s + step + 1)
        k = kt[s:e].to(torch.int64) & 0xFFFFFFFF
        assert bool((k[1:] >= k[:-1]).all())
        assert torch.equal(orig[v[s:e]], kt[s:e])
        eq = k[1:] == k[:-1]
        vv = v[s:e]
        assert bool((vv[1:][eq] > vv[:-1][eq]).all())


@pytest.mark.parametrize("n,plan", [((1 << 31) + 12345, "auto"), ((1 << 31) - 1, "grid")])
def test_largest_sizes(n, plan):
    """The largest arrays each layout takes: past 2^31 elements the automatic
    plan is the chunk layout (64-bit element positions); the grid layout takes
    up to 2^31 - 1 (31-bit look-back prefixes).  uint32 keys + index payload,
    16 GiB of data."""
    r = W.splitmix64_torch(W.SEEDS["uniform"], 0, n, device=DEV)
    keys = ((r >> 32) & 0xFFFFFFFF).to(torch.int64).to(torch.int32)
    del r
    # payload = index as uint32 (int32 bits wrap past 2^31 - 1)
    vals = torch.arange(n, dtype=torch.int64, device=DEV).to(torch.int32)
    kt = keys.clone()
    R.sort_tensors(kt, vals, layout=plan)
    R.radsort_device_status()
    _check_large(keys, kt, vals)


@pytest.mark.parametrize("kb,db", [(4, 8), (8, 11)])
def test_autotune_plan_sorts_and_inputs_untouched(kb, db):
    """radsort_autotune times every candidate plan on copies, leaves the
    arrays as they were, returns a plan of the automatic plan's layout whose
    sort matches the oracle, and answers a second call from its cache."""
    import time

    n = (1 << 21) + 77
    keys = W.make_keys("uniform", n, 8 * kb)
    vals = W.index_payload(n)
    kt, vt = to_dev(keys), to_dev(vals)
    b, p, lay, sh = R.radsort_autotune(kt, vt, digit_bits=db)
    R.radsort_device_status()
    assert np.array_equal(from_dev(kt, keys.dtype), keys)
    assert np.array_equal(from_dev(vt, np.uint32), vals)
    assert lay == R.radsort_plan_default(n, kb, 4, db)[2]
    assert R.radsort_workspace_size(n, kb, 4, db, b, p, lay, sh) > 0
    t0 = time.perf_counter()
    assert R.radsort_autotune(kt, vt, digit_bits=db) == (b, p, lay, sh)
    assert time.perf_counter() - t0 < 0.05
    gk, gv = gpu_sort(keys, vals, digit_bits=db, block_size=b, num_chunks=p, layout=lay, shape=sh)
    ek, ev = oracle_sort(keys, vals, 8 * kb, db)
    assert np.array_equal(gk, ek) and np.array_equal(gv, ev)


@pytest.mark.parametrize("bs", [0, 64, 256])
@pytest.mark.parametrize("n", [2, 63, 4097, 65543, 300001, 1 << 20])
def test_msd_split_layout(n, bs):
    """The MSD split (Sec. 4.3): the sorted result equals the oracle's, and
    the sequence after every round equals the oracle's split-then-bucket
    sequence (round 1 the top digit, then each bucket from its lowest
    digit)."""
    rng = np.random.default_rng(n + bs)
    for keys in (rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32),
                 (rng.integers(0, 40, n, dtype=np.uint64) * np.uint64(0x01010101)).astype(np.uint32)):
        vals = W.index_payload(n)
        gk, gv = gpu_sort(keys, vals, block_size=bs, layout="msd")
        ek, ev = oracle_sort(keys, vals, 32, 8)
        assert np.array_equal(gk, ek) and np.array_equal(gv, ev)
        if n > 300001:
            continue
        for r in range(1, 4):
            kt, vt = to_dev(keys), to_dev(vals)
            ok, ov = torch.empty_like(kt), torch.empty_like(vt)
            R.sort_rounds_tensors(kt, vt, r, ok, ov, digit_bits=8, block_size=bs, layout="msd")
            R.radsort_device_status()
            lk, lv = oracle.msd_split(keys, vals, n_t=4, sigma=256, bits=8, b=256, rounds=r)
            assert np.array_equal(from_dev(ok, np.uint32), lk.astype(np.uint32)), r
            assert np.array_equal(from_dev(ov, np.uint32), lv), r


@pytest.mark.parametrize("with_vals", [True, False])
def test_msd_split_u64(with_vals):
    n = 200003
    keys = W.make_keys("uniform", n, 64)
    keys[::4] = keys[1]
    vals = W.index_payload(n) if with_vals else None
    gk, gv = gpu_sort(keys, vals, layout="msd")
    ek, ev = oracle_sort(keys, W.index_payload(n), 64, 8)
    assert np.array_equal(gk, ek)
    if with_vals:
        assert np.array_equal(gv, ev)


def test_msd_split_rejects_11_bit_digits():
    kt = torch.zeros(1000, dtype=torch.int32, device=DEV)
    with pytest.raises(R.RadsortError):
        R.sort_tensors(kt, None, digit_bits=11, layout="msd")


@pytest.mark.parametrize("kb,with_vals,bs", [(4, True, 256), (4, True, 4096), (4, False, 1024), (8, True, 512),
                                             (8, False, 2048)])
@pytest.mark.parametrize("n", [3, 4097, 65543, 300001, 1 << 20])
def test_tile_shape_two_groups(n, kb, with_vals, bs):
    """The round kernel's second tile shape (two groups of 8 consumer warps
    on smaller tiles): bit-exact against the oracle."""
    rng = np.random.default_rng(n + bs)
    keys = W.make_keys("uniform", n, 8 * kb)
    keys[::4] = keys[n // 2]
    vals = W.index_payload(n)
    gk, gv = gpu_sort(keys, vals if with_vals else None, block_size=bs, layout="grid", shape=2)
    ek, ev = oracle_sort(keys, vals, 8 * kb, 8)
    assert np.array_equal(gk, ek)
    if with_vals:
        assert np.array_equal(gv, ev)


@pytest.mark.parametrize("kb", [4, 8])
def test_autotune_digit_width(kb):
    """radsort_autotune_digits returns a width and a plan whose sort matches
    the oracle; the arrays are left as they were."""
    n = (1 << 21) + 5
    keys = W.make_keys("uniform", n, 8 * kb)
    vals = W.index_payload(n)
    kt, vt = to_dev(keys), to_dev(vals)
    db, b, p, lay, sh = R.radsort_autotune_digits(kt, vt)
    R.radsort_device_status()
    assert db in (8, 11)
    assert np.array_equal(from_dev(kt, keys.dtype), keys)
    gk, gv = gpu_sort(keys, vals, digit_bits=db, block_size=b, num_chunks=p, layout=lay, shape=sh)
    ek, ev = oracle_sort(keys, vals, 8 * kb, db)
    assert np.array_equal(gk, ek) and np.array_equal(gv, ev)
