"""Model of Finalize's block permutation F1 (host logic, no GPU).

Logical block q sits at physical block pi[q] and belongs at target(q): A
block q (physical nT + q) for q < nA, scratch block q - nA otherwise.  Every
block that must move is an edge pi[q] -> target(q); the edges form paths
(from a scratch block nothing moves into, to a block whose content is not
needed) and cycles.  Each chain takes a range of an order array, listed from
the block written first: a path from its end, a cycle from its minimum.  Entry
g receives the block at entry g + 1; a cycle's last entry receives the head's
old block.

The move pass takes the order array in strides of K entries, each stride one
ticket, CTAs in any interleaving: all reads of a stride (into its buffer; a
straddling cycle's head also into a slot) come before its writes; after its
reads a stride releases its flag and its slots, then waits for the previous
stride's flag if its first entry continues a chain from there, and for the
slot of any cycle it closes.  Cycles that straddle strides beyond the slot
capacity are deferred and moved afterwards one cycle at a time.

The model replays this under seeded bursty schedules (and with strides that
hold a cycle's head made slow before they save it) and checks that every
block lands at its target, that no CTA waits forever, and that the slot and
deferred paths are taken.  It fails if a stride skips the wait for its
predecessor, if a head is not saved, or if a closing write does not wait for
its slot.
"""
import random

import pytest


def chains(pi, nA, nT, rng):
    """Order array entries (position, first, last, cyc), chain order random
    (the kernel reserves ranges with atomics)."""
    NL = len(pi)
    target = [nT + q if q < nA else q - nA for q in range(NL)]
    nxt = {pi[q]: target[q] for q in range(NL) if pi[q] != target[q]}
    prev = {t: x for x, t in nxt.items()}
    out = []
    seen = set()
    for x in nxt:  # cycles, listed from their minimum
        if x in seen:
            continue
        y, cyc = x, [x]
        while nxt.get(y) is not None and nxt[y] != x:
            y = nxt[y]
            if y not in nxt:
                break
            cyc.append(y)
        if y in nxt and nxt[y] == x:
            seen.update(cyc)
            m = cyc.index(min(cyc))
            ring = cyc[m:] + cyc[:m]
            # entry g receives from entry g+1: order the cycle against the edges
            order = [ring[0]]
            while len(order) < len(ring):
                order.append(prev[order[-1]])
            out.append((order, True))
    for x in nxt:  # paths, listed from their end
        if x in seen or x in prev:
            continue
        path = [x]
        while path[-1] in nxt:
            path.append(nxt[path[-1]])
        seen.update(path)
        out.append((path[::-1], False))
    rng.shuffle(out)
    return out, target


def run(seed, nA=300, extra=20, nT=64, K=4, nslots=2, ctas=3, bursts=(1, 2, 8, 32), head_delay=0):
    rng = random.Random(seed)
    NL = nA + extra
    places = list(range(nT + nA))
    rng.shuffle(places)
    # mostly long cycles and paths, some blocks already in place
    pi = places[:NL]
    for q in rng.sample(range(NL), NL // 10):
        t = nT + q if q < nA else q - nA
        if t in pi and pi.index(t) != q:
            j = pi.index(t)
            pi[q], pi[j] = pi[j], pi[q]
    assert len(set(pi)) == NL
    data = {p: ("blank", p) for p in range(nT + nA)}
    for q in range(NL):
        data[pi[q]] = ("block", q)
    ch, target = chains(pi, nA, nT, rng)
    order, first, last, cyc, defer = [], [], [], [], []
    recs = []  # (base, len, slot or None)
    for seq, c in ch:
        base = len(order)
        straddles = c and base // K != (base + len(seq) - 1) // K
        slot = None
        d = False
        if straddles:
            if len(recs) < nslots:
                slot = len(recs)
            else:
                d = True
            recs.append((base, len(seq), slot))
        for r, x in enumerate(seq):
            order.append(x)
            first.append(r == 0)
            last.append(r == len(seq) - 1)
            cyc.append(c)
            defer.append(d)
    total = len(order)
    nstr = (total + K - 1) // K
    sflag = [False] * nstr
    slot_flag = [False] * nslots
    slots = [None] * nslots
    ticket = [0]
    stats = {"slot_reads": 0, "waits": 0}

    def rec_of(g):
        for base, ln, slot in recs:
            if base <= g < base + ln:
                return base, slot
        return None, None

    def cta():
        while True:
            t = ticket[0]
            ticket[0] += 1
            if t >= nstr:
                return
            g0, g1 = t * K, min(total, t * K + K)
            plan = []  # (dst, kind, src or slot, save slot)
            for g in range(g0, g1):
                dst, kind, src, save = order[g], 0, None, None
                if defer[g]:
                    kind = 0
                elif last[g]:
                    if cyc[g]:
                        base, slot = rec_of(g)
                        if base is not None and base < g0:
                            kind, src = 2, slot
                        else:
                            gh = g
                            while gh > g0 and not first[gh]:
                                gh -= 1
                            kind, src = 1, order[gh]
                else:
                    kind, src = 1, order[g + 1]
                    if first[g] and cyc[g]:
                        base, slot = rec_of(g)
                        if base is not None:
                            save = slot
                plan.append((dst, kind, src, save))
            wait_prev = t > 0 and not first[g0] and not defer[g0]
            # read phase
            buf = {}
            for i, (dst, kind, src, save) in enumerate(plan):
                if kind == 1:
                    buf[i] = data[src]
                    yield
                if save is not None:
                    for _ in range(head_delay):  # a stride holding a head may be slow
                        yield
                    slots[save] = data[dst]
                    yield
            for dst, kind, src, save in plan:
                if save is not None:
                    slot_flag[save] = True
            sflag[t] = True
            yield
            while wait_prev and not sflag[t - 1]:
                stats["waits"] += 1
                yield
            for dst, kind, src, save in plan:
                while kind == 2 and not slot_flag[src]:
                    stats["waits"] += 1
                    yield
            # write phase
            for i, (dst, kind, src, save) in enumerate(plan):
                if kind == 1:
                    data[dst] = buf[i]
                    yield
                elif kind == 2:
                    stats["slot_reads"] += 1
                    data[dst] = slots[src]
                    yield

    actors = [cta() for _ in range(ctas)]
    live = list(range(ctas))
    steps = 0
    while live:
        i = rng.choice(live)
        for _ in range(rng.choice(bursts)):
            try:
                next(actors[i])
            except StopIteration:
                live.remove(i)
                break
            steps += 1
        assert steps < 2_000_000, "a CTA waits forever"
    # deferred cycles, one at a time: save the head, shift, close
    deferred = 0
    for base, ln, slot in recs:
        if slot is not None:
            continue
        deferred += 1
        head = data[order[base]]
        for g in range(base, base + ln - 1):
            data[order[g]] = data[order[g + 1]]
        data[order[base + ln - 1]] = head
    for q in range(len(pi)):
        assert data[target[q]] == ("block", q), (q, target[q], data[target[q]])
    return stats, deferred


@pytest.mark.parametrize("seed", range(16))
def test_every_block_reaches_its_target(seed):
    run(seed)


def test_slots_and_deferred_cycles_are_exercised():
    slot_reads = deferred = 0
    for seed in range(30):
        s, d = run(seed, nA=200, extra=10, nT=32, K=3, nslots=1, ctas=4)
        slot_reads += s["slot_reads"]
        deferred += d
    assert slot_reads > 0 and deferred > 0


@pytest.mark.parametrize("seed", range(12))
def test_cycles_over_many_strides_with_slow_heads(seed):
    """Short strides and many CTAs with long stalls: a cycle spans several
    strides, and the stride that closes it may run before the stride holding
    its head has saved it; the closing write waits for the slot."""
    run(seed, nA=240, extra=8, nT=24, K=2, nslots=4, ctas=8, bursts=(1, 4, 64, 256), head_delay=400)
