"""Pins of the oracle (oracle/radsort_oracle.c) to things other than itself.

The sort the paper computes has a plain definition: an LSD radix sort with a
stable per-digit pass yields the unique stable sort by the full key (Sec. 1),
and after r rounds the sequence is the unique stable sort by the r least
significant digits.  So the oracle is pinned to
  * numpy's stable argsort (a library routine) on random inputs,
  * brute-force stable sorting (Python's sorted) over exhaustive tiny inputs,
  * the data invariant of Sec. 2.2 and Lemmas 1-2 (asserted inside the oracle
    after every setup/fixup and at every newBucketBlock),
  * the space and block-copy bounds of Sec. 3,
and planted mistakes (ORACLE_MUTANT) are shown to be caught.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2607_05302_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def stable_ref(keys, mask=None):
    k = keys.astype(np.uint64)
    if mask is not None:
        k = k & np.uint64(mask)
    return np.argsort(k, kind="stable")


def low_digits_mask(r, bits):
    return (1 << (r * bits)) - 1 if r * bits < 64 else 0xFFFFFFFFFFFFFFFF


# ---------------------------------------------------------------- Alg. 1
@pytest.mark.parametrize("key_bits,bits", [(32, 8), (32, 11), (64, 8), (64, 11), (16, 4), (8, 2)])
@pytest.mark.parametrize("n", [0, 1, 2, 37, 1000, 4099])
def test_lsd_oop_is_stable_sort(key_bits, bits, n):
    rng = np.random.default_rng(n * 131 + bits)
    hi = min(2 ** key_bits, 2 ** 63)
    # small value range too, so that equal keys (stability) occur
    for top in (hi, 17):
        keys = rng.integers(0, top, n, dtype=np.uint64)
        vals = np.arange(n, dtype=np.uint32)
        n_t = oracle.digits_for(key_bits, bits)
        k, v = oracle.lsd_oop(keys, vals, n_t=n_t, sigma=1 << bits, bits=bits)
        o = stable_ref(keys)
        assert (k == keys[o]).all() and (v == o).all()


@pytest.mark.parametrize("bits", [8, 11, 3])
def test_lsd_oop_each_round_sorts_by_low_digits(bits):
    rng = np.random.default_rng(7)
    n = 3001
    keys = rng.integers(0, 2 ** 32, n, dtype=np.uint64)
    keys[::5] = keys[0]  # ties
    n_t = oracle.digits_for(32, bits)
    for r in range(n_t + 1):
        k, v = oracle.lsd_oop(keys, np.arange(n, dtype=np.uint32), n_t=n_t, sigma=1 << bits,
                              bits=bits, rounds=r)
        o = stable_ref(keys, low_digits_mask(r, bits))
        assert (v == o).all() and (k == keys[o]).all()


# ---------------------------------------------------------------- Radsort
def brute_force(keys):
    return sorted(range(len(keys)), key=lambda i: keys[i])


@pytest.mark.parametrize("b,p", [(1, 1), (2, 1), (3, 1), (1, 2), (2, 2), (3, 2)])
def test_radsort_exhaustive_tiny_binary_digits(b, p):
    # every array of n <= 6 keys over {0,1,2,3}: 2 digits of 1 bit (sigma = 2)
    for n in range(0, 7):
        for tup in itertools.product(range(4), repeat=n):
            keys = np.array(tup, dtype=np.uint64)
            k, v = oracle.radsort(keys, np.arange(n, dtype=np.uint32), n_t=2, sigma=2, bits=1,
                                  b=b, p=p)
            o = brute_force(list(tup))
            assert list(v) == o and list(k) == [tup[i] for i in o]


@pytest.mark.parametrize("b,p", [(1, 1), (2, 1), (3, 2)])
def test_radsort_exhaustive_tiny_base3(b, p):
    # every array of n <= 4 keys over 2-character strings on {a,b,c} (sigma = 3)
    for n in range(0, 5):
        for tup in itertools.product(range(9), repeat=n):
            keys = np.array(tup, dtype=np.uint64)
            k, v = oracle.radsort(keys, np.arange(n, dtype=np.uint32), n_t=2, sigma=3, bits=0,
                                  b=b, p=p)
            assert list(v) == brute_force(list(tup))


def test_radsort_worked_example_shape():
    """n=26 strings, n_t=4, b=4, alphabet {a,b,c} (Sec. 2, sort-phase figure).
    The figure itself is missing, so the expectation is brute force."""
    with open(os.path.join(HERE, "golden", "worked_example_n26_b4.txt")) as f:
        strs = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(strs) == 26 and all(len(s) == 4 for s in strs)
    code = {"a": 0, "b": 1, "c": 2}
    keys = np.array([sum(code[ch] * 3 ** (3 - j) for j, ch in enumerate(s)) for s in strs],
                    dtype=np.uint64)
    for p in (1, 2):
        for r in range(5):  # logical sequence after r rounds
            (sk, sv) = oracle.radsort(keys, np.arange(26, dtype=np.uint32), n_t=4, sigma=3,
                                      bits=0, b=4, p=p, rounds=r, finalize=False)
            exp = sorted(range(26), key=lambda i: strs[i][4 - r:])
            assert list(sv) == exp
        k, v = oracle.radsort(keys, np.arange(26, dtype=np.uint32), n_t=4, sigma=3, bits=0, b=4, p=p)
        assert [strs[i] for i in v] == sorted(strs)
        assert list(v) == brute_force(strs)


SIZES = [0, 1, 5, 63, 64, 65, 255, 256, 257, 1000, 4095, 4096, 4097, 20000]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("b,p", [(64, 1), (64, 3), (16, 5), (256, 2)])
def test_radsort_matches_numpy_u32_d8(n, b, p):
    rng = np.random.default_rng(n + 17 * b + p)
    for keys in (rng.integers(0, 2 ** 32, n, dtype=np.uint64),
                 rng.integers(0, 300, n, dtype=np.uint64)):
        vals = np.arange(n, dtype=np.uint32)
        k, v = oracle.radsort(keys, vals, n_t=4, sigma=256, bits=8, b=b, p=p)
        o = stable_ref(keys)
        assert (v == o).all() and (k == keys[o]).all()


@pytest.mark.parametrize("bits", [8, 11])
@pytest.mark.parametrize("p", [1, 2])
def test_radsort_matches_numpy_u64(bits, p):
    rng = np.random.default_rng(bits + p)
    n = 5000
    keys = rng.integers(0, 2 ** 63, n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, n, dtype=np.uint64)
    keys[::7] = keys[3]
    n_t = oracle.digits_for(64, bits)
    k, v = oracle.radsort(keys, np.arange(n, dtype=np.uint32), n_t=n_t, sigma=1 << bits, bits=bits,
                          b=128, p=p, elem_bytes=12)
    o = stable_ref(keys)
    assert (v == o).all() and (k == keys[o]).all()


def test_radsort_keys_only():
    rng = np.random.default_rng(3)
    keys = rng.integers(0, 2 ** 32, 3333, dtype=np.uint64)
    k, v = oracle.radsort(keys, None, n_t=4, sigma=256, bits=8, b=32, p=2)
    assert v is None and (k == np.sort(keys)).all()


@pytest.mark.parametrize("dist", W.DISTRIBUTIONS)
def test_radsort_rounds_match_alg1(dist):
    """After r rounds the logical sequence of Radsort equals r rounds of Alg. 1
    and the stable sort by the r low digits (Sec. 2.1: the concatenation of
    the used elements of blocks sigma..f-1 holds the permuted input)."""
    n = 6001
    keys = W.make_keys(dist, n).astype(np.uint64)
    vals = np.arange(n, dtype=np.uint32)
    for r in range(5):
        sk, sv = oracle.radsort(keys, vals, n_t=4, sigma=256, bits=8, b=64, p=3, rounds=r,
                                finalize=False)
        lk, lv = oracle.lsd_oop(keys, vals, n_t=4, sigma=256, bits=8, rounds=r)
        o = stable_ref(keys, low_digits_mask(r, 8))
        assert (sv == lv).all() and (sk == lk).all()
        assert (sv == o).all()


@pytest.mark.parametrize("n,b,p,bits,E", [(100000, 512, 1, 8, 8), (100000, 256, 4, 8, 8),
                                          (30000, 128, 2, 11, 12), (10, 64, 3, 8, 8)])
def test_space_and_copy_bounds(n, b, p, bits, E):
    """Sec. 3: T is 2*sigma*p blocks (2 sigma for p = 1), the bookkeeping is
    O(n/b) entries; Lemma 2 leaves >= H unallocated blocks; Finalize copies
    each of the floor(n/b) A blocks at most twice and every other block once."""
    sigma = 1 << bits
    rng = np.random.default_rng(n)
    keys = rng.integers(0, 2 ** 32, n, dtype=np.uint64)
    n_t = oracle.digits_for(32, bits)
    (_, _), st = oracle.radsort(keys, np.arange(n, dtype=np.uint32), n_t=n_t, sigma=sigma,
                                bits=bits, b=b, p=p, elem_bytes=E, with_stats=True)
    H = sigma * p
    assert st["head"] == H and st["t_blocks"] == 2 * H
    assert st["n_pi"] == n // b + 2 * H
    assert st["min_unallocated"] >= H
    assert st["fin_copies_main"] <= 2 * (n // b)
    assert st["fin_copies_rest"] <= H + 1
    ubytes = 1 if sigma <= 256 else 2
    bound = 2 * H * b * E + st["n_pi"] * (8 + ubytes) + H * 32
    assert st["extra_bytes"] <= bound
    if p == 1 and b == 512 and E == 8:
        # Sec. 4 example: b=512, 8-byte elements -> T = 2 MiB, 9 B/block of input
        assert 2 * H * b * E == 2 * 1024 * 1024
        assert st["extra_bytes"] - 2 * H * b * E - H * 32 == st["n_pi"] * 9


def test_float_transform_order():
    vals = np.array([-np.inf, -3.5, -1.0, -1e-30, -0.0, 0.0, 1e-30, 1.0, 2.5, np.inf],
                    dtype=np.float32)
    rng = np.random.default_rng(0)
    perm = rng.permutation(vals.size)
    bits = vals[perm].view(np.uint32)
    t = oracle.f32_to_ordered(bits)
    back = oracle.ordered_to_f32(np.sort(t))
    got = back.view(np.float32)
    assert [str(x) for x in got] == [str(x) for x in vals]  # -0.0 before 0.0
    r = rng.integers(0, 2 ** 32, 10000, dtype=np.uint64).astype(np.uint32)
    assert (oracle.ordered_to_f32(oracle.f32_to_ordered(r)) == r).all()
    f = W.float_normal_bits(5000)
    t = oracle.f32_to_ordered(f)
    o = np.argsort(t, kind="stable")
    fo = f.view(np.float32)[o]
    assert (np.diff(fo) >= 0).all()


# ---------------------------------------------------------------- mutants
def _battery(mutant):
    """Returns True if every pin passes for the oracle built with `mutant`."""
    rng = np.random.default_rng(11)
    try:
        for n, b, p in [(1000, 4, 1), (1000, 64, 3), (257, 16, 2)]:
            keys = rng.integers(0, 2 ** 12, n, dtype=np.uint64)
            vals = np.arange(n, dtype=np.uint32)
            o = stable_ref(keys)
            k, v = oracle.radsort(keys, vals, n_t=4, sigma=256, bits=8, b=b, p=p, mutant=mutant)
            if not ((v == o).all() and (k == keys[o]).all()):
                return False
            k, v = oracle.lsd_oop(keys, vals, n_t=4, sigma=256, bits=8, mutant=mutant)
            if not ((v == o).all() and (k == keys[o]).all()):
                return False
    except oracle.OracleError:
        return False
    return True


def test_clean_oracle_passes_battery():
    assert _battery(0)


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5, 6])
def test_planted_mistakes_are_caught(mutant):
    lib = oracle._lib(mutant)
    assert lib.ora_mutant_id() == mutant
    assert not _battery(mutant)


# state-only mistakes: each corrupts the algorithm state in one place, and
# the check written for that part of the state must fire with its own code
# (data invariant of Sec. 2.2, Lemmas 1 and 2 of Sec. 2.3, copy bound of Sec. 3)
STATE_MUTANTS = {
    7: -13,   # two P entries exchanged -> invariant 2 (P ascending)
    8: -14,   # f one past the last used block -> invariant 3 (block f-1 partial)
    9: -12,   # a block entered twice in pi' -> invariant 1 (pi a permutation)
    10: -10,  # head start of sigma-1 blocks -> Lemma 1
    11: -11,  # one scratch block fewer -> Lemma 2
    12: -15,  # an open block's fill one short -> invariant 5 (element count)
    13: -17,  # Finalize pulls through a bounce block -> copy bound of Sec. 3
}


def _state_cases():
    """Inputs on which the state mistakes meet their checks: random keys with
    several block sizes and chunk counts, and one bucket that takes every
    element (the tight case of Lemmas 1 and 2)."""
    rng = np.random.default_rng(23)
    out = []
    for n, b, p in [(1000, 4, 1), (1000, 1, 1), (2000, 16, 3)]:
        out.append((rng.integers(0, 2 ** 32, n, dtype=np.uint64), b, p))
    out.append((np.full(1000, 0x12345678, np.uint64), 4, 1))
    return out


@pytest.mark.parametrize("mutant", sorted(STATE_MUTANTS))
def test_state_mistakes_fire_their_own_check(mutant):
    lib = oracle._lib(mutant)
    assert lib.ora_mutant_id() == mutant
    want = STATE_MUTANTS[mutant]
    codes = set()
    for keys, b, p in _state_cases():
        vals = np.arange(keys.size, dtype=np.uint32)
        try:
            oracle.radsort(keys, vals, n_t=4, sigma=256, bits=8, b=b, p=p, mutant=mutant)
            codes.add(0)
        except oracle.OracleError as e:
            codes.add(e.code)
    # the intended check fires, and no other check claims the mistake
    assert want in codes, (mutant, codes)
    assert codes <= {0, want}, (mutant, codes)


def test_clean_oracle_passes_the_state_cases():
    for keys, b, p in _state_cases():
        vals = np.arange(keys.size, dtype=np.uint32)
        k, v = oracle.radsort(keys, vals, n_t=4, sigma=256, bits=8, b=b, p=p)
        o = stable_ref(keys)
        assert (v == o).all() and (k == keys[o]).all()


# ---------------------------------------------------------------- truncate (Alg. 8)
def _perm(keys, vals, b, p, mutant=0):
    return oracle.Perm(keys, vals, n_t=4, sigma=256, bits=8, b=b, p=p, mutant=mutant)


@pytest.mark.parametrize("b,p", [(1, 1), (4, 1), (16, 1), (64, 3), (8, 5)])
def test_truncate_keeps_the_prefix(b, p):
    """After r rounds the logical sequence is r rounds of Alg. 1; truncating
    it to m elements (Alg. 8) leaves exactly its first m elements, and the
    state still satisfies the data invariant (checked inside the oracle)."""
    rng = np.random.default_rng(100 + b + p)
    n = 3000
    keys = rng.integers(0, 2 ** 32, n, dtype=np.uint64)
    vals = np.arange(n, dtype=np.uint32)
    lk, lv = oracle.lsd_oop(keys, vals, n_t=4, sigma=256, bits=8, rounds=2)
    P = _perm(keys, vals, b, p)
    P.rounds(0, 2)
    # cuts inside blocks, at block ends and starts, and the extremes
    for m in sorted({n, n - 1, 2500, 17 * b + 1, 17 * b, 17 * b - 1, 5, 1, 0}, reverse=True):
        P.truncate(m)
        sk, sv = P.sequence()
        assert len(P) == m
        assert np.array_equal(sk, lk[:m]) and np.array_equal(sv, lv[:m]), m


@pytest.mark.parametrize("b,p", [(4, 1), (16, 1), (64, 3), (8, 5)])
def test_sort_after_truncate_and_finalize(b, p):
    """The state after a truncation is a valid Radsort state (Sec. 4.1):
    further rounds sort the truncated sequence stably, and Finalize puts it in
    A; both equal the stable sort of the prefix computed by numpy."""
    rng = np.random.default_rng(7 * b + p)
    for trial in range(6):
        n = int(rng.integers(200, 4000))
        keys = rng.integers(0, 2 ** int(rng.integers(6, 33)), n, dtype=np.uint64)
        vals = np.arange(n, dtype=np.uint32)
        P = _perm(keys, vals, b, p)
        r0 = int(rng.integers(0, 5))
        P.rounds(0, r0)
        m = int(rng.integers(0, n + 1))
        P.truncate(m)
        sk, sv = P.sequence()
        P.rounds(0, 4)
        fk, fv = P.sequence()
        o = np.argsort(sk, kind="stable")
        assert np.array_equal(fk, sk[o]) and np.array_equal(fv, sv[o])
        k, v = P.finalize()
        assert np.array_equal(k, fk) and np.array_equal(v, fv)


def test_truncate_mutants():
    """A stale P entry kept past the new end is caught by invariant 2 at once
    (mutant 14); Finalize without the push of reading G16 writes a wrong
    sequence on some truncated states (mutant 15) while the clean oracle never
    does."""
    keys = np.random.default_rng(3).integers(0, 2 ** 32, 3000, dtype=np.uint64)
    vals = np.arange(3000, dtype=np.uint32)
    P = _perm(keys, vals, 16, 3, mutant=14)
    P.rounds(0, 2)
    with pytest.raises(oracle.OracleError) as e:
        P.truncate(1000)
    assert e.value.code == -13
    # small alphabets give few, long chains, where a remaining block sits in
    # A block floor(n/b) behind other remaining blocks
    rng = np.random.default_rng(9)
    wrong = 0
    for trial in range(400):
        bits = int(rng.integers(1, 5))
        n_t = 8
        n = int(rng.integers(5, 300))
        keys = rng.integers(0, 2 ** (bits * n_t), n, dtype=np.uint64)
        vals = np.arange(n, dtype=np.uint32)
        b, p = int(rng.choice([1, 2, 3, 4, 8])), int(rng.integers(1, 4))
        m, r = int(rng.integers(1, n)), int(rng.integers(0, n_t + 1))
        res = []
        for mut in (0, 15):
            P = oracle.Perm(keys, vals, n_t=n_t, sigma=1 << bits, bits=bits, b=b, p=p, mutant=mut)
            P.rounds(0, r)
            P.truncate(m)
            sk, sv = P.sequence()
            k, v = P.finalize()
            res.append(np.array_equal(k, sk) and np.array_equal(v, sv))
        assert res[0]
        wrong += not res[1]
    assert wrong > 0


# ---------------------------------------------------------------- MSD split (Sec. 4.3)
@pytest.mark.parametrize("n,b", [(1, 4), (37, 1), (1000, 4), (5000, 16)])
def test_msd_split_sequences(n, b):
    """After the split the sequence is the stable sort by the top digit; after
    r rounds the stable sort by (top digit, r-1 lowest digits); after n_t
    rounds the stable sort by the whole key (numpy lexsort / argsort, both
    stable)."""
    rng = np.random.default_rng(n + b)
    keys = rng.integers(0, 2 ** 32, n, dtype=np.uint64)
    keys[::3] = keys[0]  # ties
    vals = np.arange(n, dtype=np.uint32)
    top = keys >> np.uint64(24)
    for r in range(5):
        k, v = oracle.msd_split(keys, vals, n_t=4, sigma=256, bits=8, b=b, rounds=r)
        if r == 0:
            o = np.arange(n)
        else:
            low = keys & np.uint64((1 << (8 * (r - 1))) - 1)
            o = np.lexsort((low, top))
        assert np.array_equal(v, o.astype(np.uint32)), r
        assert np.array_equal(k, keys[o]), r
    assert np.array_equal(v, stable_ref(keys).astype(np.uint32))


def test_msd_split_small_alphabet_brute_force():
    """Every array of n <= 5 two-bit keys of 3 digits (sigma = 4): the split
    then per-bucket rounds give the unique stable sort."""
    for n in range(1, 6):
        for keys in itertools.product(range(8), repeat=n):
            keys = np.array(keys, dtype=np.uint64) * np.uint64(9)  # digits vary at every position
            vals = np.arange(n, dtype=np.uint32)
            k, v = oracle.msd_split(keys, vals, n_t=3, sigma=4, bits=2, b=2)
            o = np.argsort(keys, kind="stable")
            assert np.array_equal(v, o.astype(np.uint32)) and np.array_equal(k, keys[o])
