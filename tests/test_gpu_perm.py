"""The permuted representation kept between calls (Sec. 4.1) and truncation
(Alg. 8) on the GPU, through the C ABI, against the oracle's persistent
state (oracle.Perm): the logical sequence after rounds, the block list read
in place, the sequence after a truncation, rounds run again on the truncated
or modified sequence, and Finalize.  Bit-exact: every sequence here is a
stable sort (or a prefix of one), which is unique."""
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


def host(t, dtype):
    return t.cpu().numpy().view(dtype)


def sequence(P, n, kdt):
    ok = torch.empty(max(n, 1), dtype=torch.int32 if kdt == np.uint32 else torch.int64, device=DEV)
    ov = torch.empty(max(n, 1), dtype=torch.int32, device=DEV)
    P.gather(ok, ov)
    R.radsort_device_status()
    return host(ok, kdt)[:n], host(ov, np.uint32)[:n]


def element_index(P, keys, ws):
    """For every element of the sequence, where it lives, read from the block
    list alone: (in_scratch flag, element index into keys or into the
    workspace viewed as keys)."""
    lst = P.blocks()
    R.radsort_device_status()
    kb = keys.element_size()
    a0, w0 = keys.data_ptr(), ws.data_ptr()
    addr, lens = lst[:, 0], lst[:, 2] & 0xFFFFFFFF
    in_a = (addr >= a0) & (addr < a0 + keys.numel() * kb)
    base = torch.where(in_a, (addr - a0) // kb, (addr - w0) // kb)
    off = torch.arange(int(lens.sum()), device=DEV) - torch.repeat_interleave(
        torch.cumsum(lens, 0) - lens, lens)
    idx = torch.repeat_interleave(base, lens) + off
    return torch.repeat_interleave(~in_a, lens), idx, lst


def read_blocks(P, keys, vals, ws):
    """The sequence read through the block list (no copy by the library)."""
    t, idx, lst = element_index(P, keys, ws)
    kdt = keys.dtype
    wk = ws.view(kdt)
    k = torch.where(t, wk[idx.clamp(max=wk.numel() - 1)], keys[idx.clamp(max=keys.numel() - 1)])
    # values: the listed value addresses, mapped the same way
    va, v0, w0 = lst[:, 1], vals.data_ptr(), ws.data_ptr()
    lens = lst[:, 2] & 0xFFFFFFFF
    in_a = (va >= v0) & (va < v0 + vals.numel() * 4)
    vb = torch.where(in_a, (va - v0) // 4, (va - w0) // 4)
    off = torch.arange(int(lens.sum()), device=DEV) - torch.repeat_interleave(torch.cumsum(lens, 0) - lens, lens)
    vi = torch.repeat_interleave(vb, lens) + off
    vt = torch.repeat_interleave(~in_a, lens)
    wv = ws.view(torch.int32)
    v = torch.where(vt, wv[vi.clamp(max=wv.numel() - 1)], vals[vi.clamp(max=vals.numel() - 1)])
    return k, v, lst


@pytest.mark.parametrize("kb,db,bs", [(4, 8, 256), (4, 8, 0), (8, 11, 512), (8, 8, 64), (4, 11, 1024)])
def test_rounds_blocks_truncate_resort_finalize(kb, db, bs):
    n = 300007
    kdt = np.uint32 if kb == 4 else np.uint64
    keys = W.make_keys("uniform", n, 8 * kb)
    keys[::5] = keys[3]  # ties: stability shows
    vals = W.index_payload(n)
    n_t = oracle.digits_for(8 * kb, db)
    kt, vt = to_dev(keys), to_dev(vals)
    P = R.Perm(kt, vt, digit_bits=db, block_size=bs)
    ob = bs or 256
    O = oracle.Perm(keys, vals, n_t=n_t, sigma=1 << db, bits=db, b=ob)
    # partial sort: the first two rounds (two least significant digits)
    P.rounds(0, 2)
    O.rounds(0, 2)
    ek, ev = O.sequence()
    gk, gv = sequence(P, n, kdt)
    assert np.array_equal(gk, ek.astype(kdt)) and np.array_equal(gv, ev)
    # the block list reads the same sequence in place, every block full but the last
    k2, v2, lst = read_blocks(P, kt, vt, P.workspace)
    assert np.array_equal(host(k2, kdt), gk) and np.array_equal(host(v2, np.uint32), gv)
    lens = host(lst[:, 2], np.uint64) & 0xFFFFFFFF
    b = int(lens[0])
    assert (lens[:-1] == b).all() and lens[-1] == n % b and P.size() == (n, n // b + 1)
    # truncation keeps the prefix; a cut at a block end leaves an empty final block
    cuts = sorted({n - 1, 200000, 64 * b, 64 * b - 1, 12345}, reverse=True)
    for m in cuts:
        P.truncate(m)
        O.truncate(m)
        gk, gv = sequence(P, m, kdt)
        assert np.array_equal(gk, ek[:m].astype(kdt)) and np.array_equal(gv, ev[:m])
        assert P.size() == (m, m // b + 1)
    # sorting again from the truncated state: all rounds
    P.rounds(0, n_t)
    O.rounds(0, n_t)
    m = cuts[-1]
    fk, fv = O.sequence()
    gk, gv = sequence(P, m, kdt)
    assert np.array_equal(gk, fk.astype(kdt)) and np.array_equal(gv, fv)
    o = np.argsort(ek[:m], kind="stable")
    assert np.array_equal(fv, ev[:m][o])
    # Finalize puts the sequence in keys[0 .. m)
    P.finalize()
    R.radsort_device_status()
    assert np.array_equal(host(kt, kdt)[:m], fk.astype(kdt))
    assert np.array_equal(host(vt, np.uint32)[:m], fv)
    P.close()


def test_keys_modified_in_place_then_sorted_again():
    """Sort, change every key in place through the block list (a new key per
    element), sort again by the new keys: the state needs no Finalize and no
    new setup in between (Sec. 4.1)."""
    n = 200003
    keys = W.make_keys("uniform", n)
    vals = W.index_payload(n)
    kt, vt = to_dev(keys), to_dev(vals)
    P = R.Perm(kt, vt, digit_bits=8, block_size=512)
    P.rounds(0, 4)
    in_t, idx, _ = element_index(P, kt, P.workspace)
    wk = P.workspace.view(torch.int32)
    # new key of each element: a function of its payload (the original index)
    _, sv = sequence(P, n, np.uint32)
    newk = W.fmix32_np(sv ^ np.uint32(0x5BD1E995))
    nk = to_dev(newk)
    kt[idx[~in_t]] = nk[~in_t]
    wk[idx[in_t]] = nk[in_t]
    P.keys_changed()
    P.rounds(0, 4)
    gk, gv = sequence(P, n, np.uint32)
    o = np.argsort(newk, kind="stable")
    assert np.array_equal(gk, newk[o]) and np.array_equal(gv, sv[o])
    P.close()


def test_truncate_to_nothing_and_argument_errors():
    n = 5000
    keys = W.make_keys("uniform", n)
    kt, vt = to_dev(keys), to_dev(W.index_payload(n))
    P = R.Perm(kt, vt, block_size=256)
    with pytest.raises(R.RadsortError):
        P.rounds(0, 5)  # past n_t
    with pytest.raises(R.RadsortError):
        P.truncate(n + 1)
    P.truncate(0)
    assert P.size() == (0, 1)
    P.rounds(0, 4)  # nothing to sort
    P.finalize()
    with pytest.raises(R.RadsortError):
        P.rounds(0, 1)  # finalized
    R.radsort_device_status()
    P.close()
