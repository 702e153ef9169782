"""Radsort oracle -- TEST INFRASTRUCTURE ONLY.

Python marshalling around ``radsort_oracle.c``, the plain single-threaded CPU
restatement of the paper's Alg. 1 (out-of-place LSD round) and of the Radsort
block algorithm (Alg. 2-7, with the parallel-chunk variant of Sec. 4.3).  Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline leg may
import this package; the CUDA library never does, and the two share no code.

Every function is pinned in ``tests/test_oracle_pins.py`` to numpy's stable
argsort, to brute-force stable sorting over exhaustive tiny inputs, and to the
paper's data invariant (Sec. 2.2) and Lemmas 1-2; planted mistakes
(``ORACLE_MUTANT``) show that the pins catch them, and state-only mistakes
show that each invariant, Lemma and copy-bound check fires with its own code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "radsort_oracle.c")
_BUILD = os.path.join(_HERE, "_build")

ERRORS = {
    0: "ok",
    -1: "bad argument",
    -2: "out of memory",
    -10: "Lemma 1 violated (i_out >= i_in at newBucketBlock)",
    -11: "Lemma 2 violated (fewer than H unallocated blocks after sortPhase)",
    -12: "invariant 1 violated (pi is not a permutation)",
    -13: "invariant 2 violated (P not ascending / out of range)",
    -14: "invariant 3 violated (block f-1 is not partial)",
    -15: "invariant 5 violated (element count)",
    -16: "Finalize wrote a wrong element count",
    -17: "Finalize exceeded the block-copy bound of Sec. 3",
}


class OracleError(RuntimeError):
    """A failed check of the oracle; ``code`` is the ORA_* error code."""

    def __init__(self, msg, code=None):
        super().__init__(msg)
        self.code = code


class Stats(ctypes.Structure):
    _fields_ = [
        ("n_pi", ctypes.c_uint64),
        ("head", ctypes.c_uint64),
        ("t_blocks", ctypes.c_uint64),
        ("lemma1_checks", ctypes.c_uint64),
        ("min_unallocated", ctypes.c_uint64),
        ("fin_copies_main", ctypes.c_uint64),
        ("fin_copies_rest", ctypes.c_uint64),
        ("fin_pushes", ctypes.c_uint64),
        ("extra_bytes", ctypes.c_uint64),
        ("fin_copies_trunc", ctypes.c_uint64),
    ]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2); returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    so = os.path.join(_BUILD, f"libradsort_oracle_m{mutant}.so")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(_SRC):
        tmp = so + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", f"-DORACLE_MUTANT={mutant}",
             "-o", tmp, _SRC])
        os.replace(tmp, so)
    return so


_libs: dict[int, ctypes.CDLL] = {}


def _lib(mutant: int = 0) -> ctypes.CDLL:
    if mutant not in _libs:
        lib = ctypes.CDLL(build(mutant))
        P = ctypes.c_void_p
        lib.ora_lsd_oop.argtypes = [P, P, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint32,
                                    ctypes.c_int, ctypes.c_int]
        lib.ora_lsd_oop.restype = ctypes.c_int
        lib.ora_radsort.argtypes = [P, P, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint32,
                                    ctypes.c_int, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_int,
                                    ctypes.c_int, P, P, ctypes.c_uint64, ctypes.POINTER(Stats)]
        lib.ora_radsort.restype = ctypes.c_int
        lib.ora_f32_to_ordered.argtypes = [P, ctypes.c_size_t]
        lib.ora_ordered_to_f32.argtypes = [P, ctypes.c_size_t]
        lib.ora_mutant_id.restype = ctypes.c_int
        lib.ora_perm_new.argtypes = [P, P, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint32, ctypes.c_int,
                                     ctypes.c_size_t, ctypes.c_uint64, ctypes.c_uint64,
                                     ctypes.POINTER(ctypes.c_int)]
        lib.ora_perm_new.restype = ctypes.c_void_p
        lib.ora_perm_free.argtypes = [P]
        lib.ora_perm_rounds.argtypes = [P, ctypes.c_int, ctypes.c_int]
        lib.ora_perm_rounds.restype = ctypes.c_int
        lib.ora_perm_count.argtypes = [P]
        lib.ora_perm_count.restype = ctypes.c_uint64
        lib.ora_perm_gather.argtypes = [P, P, P]
        lib.ora_perm_truncate.argtypes = [P, ctypes.c_uint64]
        lib.ora_perm_truncate.restype = ctypes.c_int
        lib.ora_perm_finalize.argtypes = [P, P, P]
        lib.ora_perm_finalize.restype = ctypes.c_int
        lib.ora_perm_stats.argtypes = [P, ctypes.POINTER(Stats)]
        _libs[mutant] = lib
    return _libs[mutant]


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int):
    if rc != 0:
        raise OracleError(ERRORS.get(rc, f"oracle error {rc}"), rc)


def _prep(keys, vals):
    k = np.ascontiguousarray(keys).astype(np.uint64, copy=True)
    v = None if vals is None else np.ascontiguousarray(vals).astype(np.uint32, copy=True)
    return k, v


def digits_for(key_bits: int, digit_bits: int) -> int:
    """n_t = ceil(key_bits / digit_bits) (reading G8)."""
    return -(-key_bits // digit_bits)


def lsd_oop(keys, vals=None, *, n_t, sigma, bits, rounds=None, mutant=0):
    """Alg. 1 applied for `rounds` rounds (default n_t). Returns (keys, vals)."""
    k, v = _prep(keys, vals)
    _check(_lib(mutant).ora_lsd_oop(_ptr(k), _ptr(v), k.size, n_t, sigma, bits,
                                    n_t if rounds is None else rounds))
    return k, v


def radsort(keys, vals=None, *, n_t, sigma, bits, b, p=1, rounds=None, finalize=True,
            elem_bytes=8, mutant=0, with_stats=False):
    """Alg. 2 with `p` chunks.  finalize=True: the sorted (keys, vals).
    finalize=False: the logical sequence after `rounds` rounds."""
    k, v = _prep(keys, vals)
    st = Stats()
    r = n_t if rounds is None else rounds
    if finalize:
        rc = _lib(mutant).ora_radsort(_ptr(k), _ptr(v), k.size, n_t, sigma, bits, b, p, r, 1,
                                      None, None, elem_bytes, ctypes.byref(st))
        _check(rc)
        out = (k, v)
    else:
        sk = np.zeros(k.size, np.uint64)
        sv = None if v is None else np.zeros(k.size, np.uint32)
        rc = _lib(mutant).ora_radsort(_ptr(k), _ptr(v), k.size, n_t, sigma, bits, b, p, r, 0,
                                      _ptr(sk), _ptr(sv), elem_bytes, ctypes.byref(st))
        _check(rc)
        out = (sk, sv)
    return (out, st.as_dict()) if with_stats else out


def f32_to_ordered(u32):
    a = np.ascontiguousarray(u32).astype(np.uint32, copy=True)
    _lib().ora_f32_to_ordered(_ptr(a), a.size)
    return a


def ordered_to_f32(u32):
    a = np.ascontiguousarray(u32).astype(np.uint32, copy=True)
    _lib().ora_ordered_to_f32(_ptr(a), a.size)
    return a


class Perm:
    """The permuted representation kept between calls (Sec. 4.1): setup
    (Alg. 4) on construction, then rounds (Alg. 5-6), truncate (Alg. 8), the
    logical sequence (Alg. 3 walk) and Finalize (Alg. 7)."""

    def __init__(self, keys, vals=None, *, n_t, sigma, bits, b, p=1, elem_bytes=8, mutant=0):
        k, v = _prep(keys, vals)
        self._lib = _lib(mutant)
        self.has_vals = v is not None
        err = ctypes.c_int(0)
        self._h = self._lib.ora_perm_new(_ptr(k), _ptr(v), k.size, n_t, sigma, bits, b, p, elem_bytes,
                                         ctypes.byref(err))
        if not self._h:
            _check(err.value or -2)

    def close(self):
        if self._h:
            self._lib.ora_perm_free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __len__(self):
        return int(self._lib.ora_perm_count(self._h))

    def rounds(self, first, count):
        """Rounds first .. first+count-1 (round r sorts by digit n_t-1-r)."""
        _check(self._lib.ora_perm_rounds(self._h, first, count))

    def truncate(self, m):
        """Keeps the first m elements of the logical sequence (Alg. 8)."""
        _check(self._lib.ora_perm_truncate(self._h, m))

    def sequence(self):
        n = len(self)
        sk = np.zeros(n, np.uint64)
        sv = np.zeros(n, np.uint32) if self.has_vals else None
        self._lib.ora_perm_gather(self._h, _ptr(sk), _ptr(sv))
        return sk, sv

    def finalize(self):
        n = len(self)
        k = np.zeros(max(n, 1), np.uint64)
        v = np.zeros(max(n, 1), np.uint32)
        _check(self._lib.ora_perm_finalize(self._h, _ptr(k), _ptr(v)))
        return k[:n], (v[:n] if self.has_vals else None)

    def stats(self):
        st = Stats()
        self._lib.ora_perm_stats(self._h, ctypes.byref(st))
        return st.as_dict()


def msd_split(keys, vals=None, *, n_t, sigma, bits, b, rounds=None):
    """The MSD split suggested for parallel operation (Sec. 4.3, last
    paragraph): one round on the most significant digit splits the input into
    sigma buckets, then each bucket is sorted on its own by the remaining
    digits from the least significant one.  Returns the sequence after
    `rounds` rounds (default n_t): round 1 is the split, round r > 1 the
    (r-1)-th least significant digit inside every bucket.  Both steps are this
    oracle's Radsort (Alg. 2-6, p = 1): the split is one round on the keys'
    top digit, each bucket's sort the first rounds-1 rounds on its keys."""
    k, v = _prep(keys, vals)
    r = n_t if rounds is None else rounds
    if r == 0 or k.size == 0:
        return k, v
    shift = np.uint64((n_t - 1) * bits) if bits > 0 else None
    top = (k >> shift) & np.uint64(sigma - 1) if bits > 0 else k // np.uint64(sigma ** (n_t - 1)) % np.uint64(sigma)
    pos = np.arange(k.size, dtype=np.uint32)
    _, order = radsort(top, pos, n_t=1, sigma=sigma, bits=bits, b=b, p=1)
    k, v = k[order], (None if v is None else v[order])
    if r == 1:
        return k, v
    tops = top[order]
    starts = np.flatnonzero(np.r_[True, tops[1:] != tops[:-1]])
    ends = np.r_[starts[1:], k.size]
    out_k, out_v = k.copy(), (None if v is None else v.copy())
    for s0, s1 in zip(starts, ends):
        idx = np.arange(s1 - s0, dtype=np.uint32)
        sk, si = radsort(k[s0:s1], idx, n_t=n_t, sigma=sigma, bits=bits, b=b, p=1, rounds=r - 1,
                         finalize=False)
        out_k[s0:s1] = sk
        if v is not None:
            out_v[s0:s1] = v[s0:s1][si]
    return out_k, out_v
