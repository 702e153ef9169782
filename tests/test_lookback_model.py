"""Model of the round kernel's decoupled look-back over a reused ring (host
logic, no GPU).

Tiles take tickets in input order and publish, per bucket, first their count
(an aggregate) and then, once their own look-back ends, their inclusive
prefix.  The words live in a ring of R rows: tile t writes row t mod R, each
word tagged with t.  A CTA may hold STAGES tickets ahead; before the tile of a
ticket may be loaded, every tile up to t - R + 1 must have finished its
look-back (the slot's previous owner and its successor).  A reader walks back
from tile t - 1 a window of LBW words at a time: a word with the expected tag
adds its count, an inclusive word ends the walk, an older tag means "not yet
published" (wait), and a newer tag means the slot was reused, so the walk
restarts from t - 1.

The model runs CTAs and their reads as separate actors under a seeded random
schedule: every single word read or write is one step, the words of a window
are read in a random order, and a CTA runs bursts of 1 to 64 steps while the
others stall, so any of them may stall at any point for a long time.  It checks that
every tile's exclusive prefix per bucket equals the sum of the counts of the
tiles before it, that every tile reaches the end (no deadlock under the
kernel's CTA bound), and that the restart path is taken in some runs.
"""
import random

import pytest


def run(seed, ntiles=160, R=8, sigma=3, ctas=3, stages=2, lbw=4):
    rng = random.Random(seed)
    counts = [[rng.randrange(0, 5) for _ in range(sigma)] for _ in range(ntiles)]
    INCL = 1 << 30
    ring = [[(-1, 0)] * sigma for _ in range(R)]  # (tag, value)
    done = [-1] * R                                 # tag of the last tile done in each slot
    ticket = [0]
    result = {}
    stats = {"restarts": 0, "waits": 0}

    def holds_done(z):
        return done[z % R] >= z

    def cta():
        held = []          # tickets whose tiles are loaded, in order
        wm = 0             # tiles below wm are known done
        while True:
            # producer side: keep up to `stages` tiles loaded
            while len(held) < stages:
                t = ticket[0]
                ticket[0] += 1
                if t >= ntiles:
                    held.append(None)
                    break
                if t > R - 1:
                    need = t - R + 2  # tiles below need must be done
                    while wm < need:
                        if holds_done(wm):
                            wm += 1
                        else:
                            stats["waits"] += 1
                            yield "producer-wait"
                held.append(t)
                yield "loaded"
            t = held.pop(0)
            if t is None:
                return
            # publish the aggregates (one word per step)
            for c in range(sigma):
                v = counts[t][c]
                ring[t % R][c] = (t, (INCL | v) if t == 0 else v)
                yield "agg"
            # look-back, bucket by bucket, then publish the inclusive prefix
            ex = []
            for c in range(sigma):
                excl, x = 0, t - 1
                while x >= 0:
                    order = list(range(lbw))
                    rng.shuffle(order)
                    vals = [None] * lbw
                    for k in order:  # the loads of one window land in any order
                        y = x - k
                        vals[k] = ring[y % R][c] if y >= 0 else (-2, INCL)
                        yield "read"
                    k = 0
                    finished = False
                    while k < lbw:
                        y = x - k
                        want = y if y >= 0 else -2
                        tag, val = vals[k]
                        if tag != want:
                            if tag > want:
                                stats["restarts"] += 1
                                excl = 0
                                x = t - 1 + k
                            break
                        if val & INCL:
                            excl += val & ~INCL
                            finished = True
                            break
                        excl += val
                        k += 1
                    if finished:
                        break
                    x -= k
                    if k < lbw:
                        yield "spin"
                ring[t % R][c] = (t, INCL | (excl + counts[t][c]))
                ex.append(excl)
                yield "incl"
            done[t % R] = t
            result[t] = ex
            yield "done"

    actors = [cta() for _ in range(ctas)]
    live = list(range(ctas))
    steps = 0
    while live:
        # one actor runs a burst of 1 .. 64 steps while the others stall
        i = rng.choice(live)
        for _ in range(rng.choice((1, 1, 2, 4, 16, 64))):
            try:
                next(actors[i])
            except StopIteration:
                live.remove(i)
                break
            steps += 1
        assert steps < 5_000_000, "no progress (deadlock)"
    assert sorted(result) == list(range(ntiles))
    run_sum = [0] * sigma
    for t in range(ntiles):
        assert result[t] == run_sum, (t, result[t], run_sum)
        run_sum = [a + b for a, b in zip(run_sum, counts[t])]
    return stats


@pytest.mark.parametrize("seed", range(12))
def test_look_back_prefixes_exact_under_random_schedules(seed):
    # CTAs x stages + 2 <= R: the bound the host keeps (no CTA waits on a
    # ring slot whose tile it holds itself)
    run(seed, R=8, ctas=3, stages=2)


def test_restart_path_is_exercised():
    """Small rings and slow readers: some walks find a reused slot and start
    over, and the prefixes stay exact."""
    total = 0
    for seed in range(60):
        total += run(seed, ntiles=120, R=4, sigma=2, ctas=2, stages=1, lbw=2)["restarts"]
    assert total > 0
