"""Model of Finalize's in-place pointer jumping (host logic, no GPU).

Entry x of the jump array is (nxt, val); val = ABS marks an absorbing entry.
Mode 0 starts from (successor, own position) on every moving block and finds
each cycle's minimum; mode 1 starts from (successor, 1) after the cycles are
cut at their minima and finds each block's distance to its chain's end.  The
kernel runs JUMP_STEPS = 3 steps per launch, in place and unsynchronised, so a
read may see a neighbour's entry before or after that neighbour's own update
in the same step; the host issues ceil(log4(n)) + 1 launches.  The model
replays launches under three schedules: entries visited in a random order and
updated in place; every update of a step hidden until the step ends; and the
slowest the kernel allows, where every read of a neighbour sees the entry as
it was when the launch began (its owner runs after the reader), so that a
launch grows windows only fourfold.  It checks the results against the chains
computed directly.
"""
import random

import pytest

ABS = -1
STEPS = 3


def launches_for(n):
    rounds, w = 1, STEPS + 1
    while w < n:
        w *= STEPS + 1
        rounds += 1
    return rounds + 1


def jump(entries, mode, rng, schedule, launches=None):
    n = len(entries)
    for _ in range(launches_for(n) if launches is None else launches):
        launch = list(entries)
        for _ in range(STEPS):
            order = list(range(n))
            rng.shuffle(order)
            step = list(entries)
            for x in order:
                nxt, v = entries[x]
                if v == ABS:
                    continue
                seen = {"inplace": entries, "step": step, "launch": launch}[schedule]
                fn, fv = entries[nxt] if nxt == x else seen[nxt]
                if fv == ABS:
                    continue
                entries[x] = (fn, min(v, fv) if mode == 0 else v + fv)
    return entries


def random_map(n, rng):
    """A partial permutation of n positions: fixed points, cycles, and paths
    that end on a block that does not move."""
    perm = list(range(n))
    rng.shuffle(perm)
    succ = {}
    i = 0
    while i < n:
        kind = rng.random()
        ln = min(n - i, rng.choice((1, 2, 3, 7, 40, 300)))
        group = perm[i:i + ln]
        i += ln
        if kind < 0.2 or ln == 1:
            continue                       # fixed points
        if kind < 0.6:
            for a, b in zip(group, group[1:] + group[:1]):
                succ[a] = b                # a cycle
        else:
            for a, b in zip(group, group[1:]):
                succ[a] = b                # a path ending on group[-1]
    return succ


@pytest.mark.parametrize("schedule", ["inplace", "step", "launch"])
@pytest.mark.parametrize("seed", range(6))
def test_cycle_minima_and_chain_ranks(seed, schedule):
    rng = random.Random(seed)
    n = rng.choice((1000, 3000, 5000))
    succ = random_map(n, rng)
    # mode 0: cycle minima
    e = [(succ[x], x) if x in succ else (x, ABS) for x in range(n)]
    e = jump(e, 0, rng, schedule)
    cyc_min = {}
    for x in succ:
        seen, y = [x], succ[x]
        while y in succ and y != x:
            seen.append(y)
            y = succ[y]
        if y == x:
            cyc_min[x] = min(seen)
    for x, m in cyc_min.items():
        assert e[x][1] == m, (x, e[x], m)
    # mode 1: cycles cut at their minima, distance to the chain's end
    e = [(succ[x], 1) if x in succ and cyc_min.get(x) != x else (x, ABS) for x in range(n)]
    e = jump(e, 1, rng, schedule)
    for x in succ:
        if cyc_min.get(x) == x:
            continue
        d, y = 0, x
        while y in succ and cyc_min.get(y) != y:
            d += 1
            y = succ[y]
        assert e[x] == (y, d), (x, e[x], y, d)


def test_launch_count_covers_a_single_long_cycle():
    """One cycle through every position (the longest window any entry needs)
    under the slowest schedule: the launch count is enough, and without the
    confirming launch and one more it is not (windows grow only fourfold)."""
    rng = random.Random(7)
    for n in (4, 5, 16, 17, 64, 65, 1000, 4097):
        perm = list(range(n))
        rng.shuffle(perm)
        succ = {a: b for a, b in zip(perm, perm[1:] + perm[:1])}
        e = jump([(succ[x], x) for x in range(n)], 0, rng, "launch")
        assert all(v == 0 for _, v in e)
        if n > 4:
            e = jump([(succ[x], x) for x in range(n)], 0, rng, "launch", launches_for(n) - 2)
            assert any(v != 0 for _, v in e)
