"""Model of the grid layout's block allocation (host logic, no GPU).

The grid layout keeps one block chain per bucket for the whole array, laid on
the block grid of the round's output: logical block j holds output positions
[j*b, (j+1)*b).  Blocks that contain a bucket start strictly inside are
shared.  Before the round, the shared blocks and the first L non-shared
blocks of every bucket take free-list entries 0 .. nP-1.  Every other block j
of a bucket is taken eagerly (as newBucketBlock in Alg. 5, L blocks ahead) by
the tile that writes the first position of block j-L, so a tile that
continues a block finds it taken long before.  This model replays one round tile by tile with the same
formulas as the CUDA kernel and checks:
  * every output block is taken exactly once, at a distinct free-list index,
    and the indices are exactly 0 .. NB-1;
  * a tile that writes into a block finds it already taken (by the round's
    preparation, an earlier tile, or itself);
  * Lemma 1 with a head start of (L+2)*sigma: the free-list index of every
    block taken by tiles up to t is below (L+2)*sigma + (blocks those tiles
    read);
  * the elements land in stable-sort order (the output sequence equals the
    stable counting sort of the round).
"""
import numpy as np
import pytest


def prep(cnt, b):
    """Bucket starts O, shared blocks, and per bucket (ns0, ns1, fsh, lsh)."""
    sigma = len(cnt)
    n = int(cnt.sum())
    O = np.zeros(sigma + 1, dtype=np.int64)
    O[1:] = np.cumsum(cnt)
    shared = []
    for c in range(sigma):
        if cnt[c] > 0 and O[c] % b != 0:
            j = O[c] // b
            if not shared or shared[-1] != j:
                shared.append(j)
    rank = {j: k for k, j in enumerate(shared)}
    tab = []
    for c in range(sigma):
        if cnt[c] > 0:
            jf, jl = O[c] // b, (O[c] + cnt[c] - 1) // b
            fsh, lsh = rank.get(jf), rank.get(jl)
            ns0 = jf + (fsh is not None)
            ns1 = max(ns0, jl + 1 - (lsh is not None))
        else:
            fsh = lsh = None
            ns0 = ns1 = -(-O[c] // b)
        tab.append((ns0, ns1, fsh, lsh))
    return O, shared, tab, n


def replay(digits, sigma, b, tile, L=2, head=None, log=None):
    n = len(digits)
    cnt = np.bincount(digits, minlength=sigma)
    O, shared, tab, _ = prep(cnt, b)
    H = (L + 2 if head is None else head) * sigma
    NB = -(-n // b)
    M = tile // b
    ntiles = -(-n // tile)
    taken = {}            # block j -> free-list index
    for k, j in enumerate(shared):
        taken[j] = k
    nP = len(shared)
    for c in range(sigma):  # first L non-shared blocks of each bucket
        ns0, ns1 = tab[c][0], tab[c][1]
        for j in range(ns0, min(ns0 + L, ns1)):
            taken[j] = nP
            nP += 1
    assert nP <= (L + 1) * sigma - 1
    out = np.full(n, -1, dtype=np.int64)
    E = np.zeros(sigma, dtype=np.int64)  # elements of each bucket in earlier tiles
    for t in range(ntiles):
        lo, hi = t * tile, min(n, (t + 1) * tile)
        d = digits[lo:hi]
        tc = np.bincount(d, minlength=sigma)
        g = O[:sigma] + E
        # blocks taken eagerly by earlier tiles, and by this one (bucket-major)
        ans = 0
        ks = []
        for c in range(sigma):
            ns0, ns1 = tab[c][0], tab[c][1]
            cs, ce = -(-g[c] // b), -(-(g[c] + tc[c]) // b)
            ans += max(0, min(cs + L, ns1) - (ns0 + L))
            ks.append(max(0, min(ce + L, ns1) - (max(cs, ns0) + L)))
        kofs = np.concatenate([[0], np.cumsum(ks)])[:-1]
        fbase = nP + ans
        fcap = min(H + (t + 1) * M, H + n // b + 1)
        took, touched = [], set()
        for c in range(sigma):
            ns0, ns1, fsh, lsh = tab[c]
            if ks[c]:
                cs = -(-g[c] // b)
                first = max(cs, ns0) + L
                for j in range(first, first + ks[c]):
                    idx = fbase + kofs[c] + (j - first)
                    assert j not in taken, "block taken twice"
                    assert idx < fcap, "Lemma 1"
                    taken[j] = idx
                    took.append(j)
            if tc[c]:
                for j in range(g[c] // b, (g[c] + tc[c] - 1) // b + 1):
                    assert j in taken, "block written before it was taken"
                    touched.add(j)
        # stable placement of this tile's elements
        seen = np.zeros(sigma, dtype=np.int64)
        for i, dd in enumerate(d):
            out[g[dd] + seen[dd]] = lo + i
            seen[dd] += 1
        E += tc
        if log is not None:
            log.append((took, touched))
    assert sorted(taken) == list(range(NB))
    assert sorted(taken.values()) == list(range(NB))
    ref = np.argsort(digits, kind="stable")
    assert np.array_equal(out, ref)
    if log is not None:
        log.append(set(j for j, k in taken.items() if k < nP))  # taken before the round
    return nP


CASES = [
    # (n, sigma, b, tile, digit distribution)
    (5000, 16, 64, 256, "uniform"),
    (4096, 16, 64, 256, "uniform"),
    (777, 16, 64, 128, "skew"),
    (3001, 8, 128, 512, "few"),
    (1, 4, 64, 64, "uniform"),
    (65, 4, 64, 64, "uniform"),
    (20000, 256, 64, 1024, "uniform"),
    (20000, 256, 256, 2048, "skew"),
    (9999, 32, 64, 256, "blocks"),
]


@pytest.mark.parametrize("L", [1, 2, 3])
@pytest.mark.parametrize("n,sigma,b,tile,kind", CASES)
def test_grid_allocation_round(n, sigma, b, tile, kind, L):
    rng = np.random.default_rng(n * 7 + sigma)
    if kind == "uniform":
        d = rng.integers(0, sigma, n)
    elif kind == "skew":   # most elements in one bucket, many tiny buckets
        d = np.where(rng.random(n) < 0.9, 3 % sigma, rng.integers(0, sigma, n))
    elif kind == "few":    # some empty buckets
        d = rng.choice([0, 5, 7], n)
    else:                  # runs of equal digits (sorted-like input)
        d = np.sort(rng.integers(0, sigma, n))[::-1].copy()
    replay(d.astype(np.int64), sigma, b, tile, L=L)


def test_shared_blocks_bounded_by_sigma():
    """At most sigma - 1 shared blocks (bucket 0 starts at position 0)."""
    rng = np.random.default_rng(5)
    for _ in range(50):
        sigma = int(rng.choice([4, 16, 256]))
        cnt = rng.integers(0, 5, sigma)
        O, shared, _, _ = prep(cnt, 64)
        assert len(shared) <= sigma - 1


def front_loaded(sizes, k):
    """Digits of buckets with the given sizes, the first k elements of every
    bucket first (each bucket's start, and the start of its second block,
    fall in the first tiles)."""
    d = np.repeat(np.arange(len(sizes)), sizes)
    late = np.concatenate([np.arange(s) >= k for s in sizes]).astype(int)
    return d[np.argsort(late, kind="stable")].astype(np.int64)


def test_head_start_of_l_plus_two_sigma_is_needed():
    """Shared blocks, the first block of every bucket and one block taken
    ahead per bucket (L = 1): a head start of 2*sigma violates Lemma 1 on this
    input, 3*sigma does not."""
    d = front_loaded([191, 254, 255, 250, 197, 186, 122, 61], 30)
    replay(d, 8, 64, 64, L=1, head=3)
    with pytest.raises(AssertionError, match="Lemma 1"):
        replay(d, 8, 64, 64, L=1, head=2)


def run_concurrent(digits, sigma, b, tile, L, ctas, seed):
    """The same round with tiles on concurrent CTAs: a tile publishes its
    counts, waits until every earlier tile has published (its look-back),
    records the map entries of the blocks it takes, then waits for the map
    entry of every other block it writes, as the kernel does.  Any schedule
    ends (a tile only waits on earlier tiles) and every entry a tile waits for
    is written by the round's preparation, an earlier tile or itself."""
    import random

    log = []
    replay(digits, sigma, b, tile, L=L, log=log)
    pre = log.pop()
    ntiles = len(log)
    rng = random.Random(seed)
    published = [False] * ntiles
    writer = {j: -1 for j in pre}  # block -> tile that recorded its entry
    ticket = [0]

    def cta():
        while True:
            t = ticket[0]
            ticket[0] += 1
            if t >= ntiles:
                return
            published[t] = True
            yield
            while not all(published[:t]):
                yield
            took, touched = log[t]
            for j in took:
                writer[j] = t
                yield
            for j in sorted(touched - set(took)):
                while j not in writer:
                    yield
                assert writer[j] <= t
            yield

    actors = [cta() for _ in range(ctas)]
    live = list(range(ctas))
    steps = 0
    while live:
        i = rng.choice(live)
        for _ in range(rng.choice((1, 3, 20, 100))):
            try:
                next(actors[i])
            except StopIteration:
                live.remove(i)
                break
            steps += 1
        assert steps < 3_000_000, "no progress"
    return writer


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("n,sigma,b,tile,kind", CASES[:4] + CASES[6:])
def test_grid_round_on_concurrent_tiles(n, sigma, b, tile, kind, seed):
    rng = np.random.default_rng(n * 7 + sigma)
    if kind == "uniform":
        d = rng.integers(0, sigma, n)
    elif kind == "skew":
        d = np.where(rng.random(n) < 0.9, 3 % sigma, rng.integers(0, sigma, n))
    elif kind == "few":
        d = rng.choice([0, 5, 7], n)
    else:
        d = np.sort(rng.integers(0, sigma, n))[::-1].copy()
    writer = run_concurrent(d.astype(np.int64), sigma, b, tile, 2, 5, seed)
    assert sorted(writer) == list(range(-(-n // b)))
