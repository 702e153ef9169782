"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function include/radsort.h declares; argument errors come back synchronously
(no GPU needed for those)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2607_05302_gb300 import build as B
    from paper_2607_05302_gb300 import radsort as R

    B.build()
    return R.lib()


def header_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(radsort_\w+)\s*\(", txt, re.M)
    return sorted(set(names))


def test_header_declares_expected_calls():
    names = header_functions()
    for must in ("radsort_sort", "radsort_sort_ex", "radsort_workspace_size",
                 "radsort_lsd_oop_sort", "radsort_sort_rounds", "radsort_device_status"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in header_functions():
        assert hasattr(lib, name), name
    from paper_2607_05302_gb300 import radsort as R
    assert set(R.EXPORTS) <= set(header_functions())


def test_synchronous_argument_errors(lib):
    from paper_2607_05302_gb300 import radsort as R

    bad = ctypes.c_void_p(16)
    assert lib.radsort_sort(bad, None, 100, 3, 8, None) == R.RADSORT_EINVAL   # key width
    assert lib.radsort_sort(bad, None, 100, 4, 9, None) == R.RADSORT_EINVAL   # digit width
    assert lib.radsort_sort(ctypes.c_void_p(18), None, 100, 4, 8, None) == R.RADSORT_EINVAL  # alignment
    assert lib.radsort_sort(None, None, 0, 4, 8, None) == R.RADSORT_OK        # n = 0
    assert lib.radsort_sort(None, None, 1, 4, 8, None) == R.RADSORT_OK        # n = 1
    assert lib.radsort_sort_ex(bad, None, 100, 8, 8, R.RADSORT_KEY_FLOAT32, None, None, 0,
                               None) == R.RADSORT_EINVAL  # float flag needs 4-byte keys
    p = R.Plan()
    p.block_size = 100  # not a power of two
    assert lib.radsort_sort_ex(bad, None, 1000, 4, 8, 0, ctypes.byref(p), None, 0,
                               None) == R.RADSORT_EINVAL
    assert R.status_str(R.RADSORT_ETIMEOUT) == "bounded device wait ran out"


def test_workspace_size_matches_space_analysis(lib):
    """Sec. 3: the workspace is the scratch array T plus O(n/b) bookkeeping.
    The automatic plan (grid layout) has T = 4*sigma + 1 blocks and stays
    within 2% of the array at 2^28 and 2^30 8-byte elements; the chunk layout
    (Sec. 4.3) has T = 2*sigma*p blocks."""
    from paper_2607_05302_gb300 import radsort as R

    for n in (1 << 28, 1 << 30):
        b, p, layout = R.radsort_plan_default(n, 4, 4, 8)
        assert layout == R.RADSORT_LAYOUT_GRID
        ws = R.radsort_workspace_size(n, 4, 4, 8)
        T = (4 * 256 + 1) * b * 8
        assert T <= ws <= T + (n // b) * 16 + (n // 8192) * 256 * 4 + (1 << 20)
        assert ws <= 0.02 * n * 8
    ws2 = R.radsort_workspace_size(1 << 20, 4, 4, 8, block_size=1024, num_chunks=2)
    assert ws2 >= 2 * 256 * 2 * 1024 * 8
    # 2^31 elements and more: the chunk layout
    assert R.radsort_plan_default(1 << 31, 4, 4, 8)[2] == R.RADSORT_LAYOUT_CHUNKS


def test_plan_layouts_by_size(lib):
    """Short arrays: out of place with the alternate arrays in the workspace
    (Sec. 5); up to 2^31: the grid layout; beyond: the chunk layout."""
    from paper_2607_05302_gb300 import radsort as R

    n = R.RADSORT_SCRATCH_MAX_N
    assert R.radsort_plan_default(n, 4, 4, 8)[2] == R.RADSORT_LAYOUT_SCRATCH
    assert R.radsort_plan_default(n + 1, 4, 4, 8)[2] == R.RADSORT_LAYOUT_GRID
    # the scratch workspace holds the alternate keys and values
    assert R.radsort_workspace_size(n, 4, 4, 8) >= n * 8
    assert R.radsort_workspace_size(n, 4, 4, 8, layout="grid") < R.radsort_workspace_size(n, 4, 4, 8) + (16 << 20)


def test_comparator_scratch_size(lib):
    """Alg. 1's comparator needs, besides its n-element alternate arrays, the
    histograms and offsets of every digit position (n_t x sigma words each)
    and a look-back ring of at most 4096 (sigma = 256) or 1024 (sigma = 2048)
    rows of sigma 64-bit words: bounded whatever n."""
    from paper_2607_05302_gb300 import radsort as R

    assert R.radsort_lsd_oop_scratch_size(1, 4, 4, 8) == 0
    for kb, db in ((4, 8), (4, 11), (8, 8), (8, 11)):
        sigma, nt = 1 << db, -(-8 * kb // db)
        tables = nt * sigma * 4 + nt * (sigma + 1) * 4
        cap = (4096 if db == 8 else 1024) * (sigma * 8 + 4)
        prev = 0
        for n in (1000, 1 << 20, 1 << 26, 1 << 30):
            s = R.radsort_lsd_oop_scratch_size(n, kb, 4, db)
            assert tables + sigma * 8 <= s <= tables + cap + 4096
            assert s >= prev
            prev = s
        assert s <= 0.02 * (1 << 30) * (kb + 4)
    bad = ctypes.c_size_t(0)
    assert lib.radsort_lsd_oop_scratch_size(100, 4, 2, 8, ctypes.byref(bad)) == R.RADSORT_EINVAL
    assert lib.radsort_lsd_oop_scratch_size(100, 4, 4, 9, ctypes.byref(bad)) == R.RADSORT_EINVAL


def test_wait_probe_argument_errors(lib):
    """The failure-path probe rejects a null flag and iteration counts outside
    1 .. 2^26 (the library's own wait limit) before launching anything."""
    from paper_2607_05302_gb300 import radsort as R

    flag = ctypes.c_void_p(256)
    assert lib.radsort_debug_wait_probe(None, 100, None) == R.RADSORT_EINVAL
    assert lib.radsort_debug_wait_probe(flag, 0, None) == R.RADSORT_EINVAL
    assert lib.radsort_debug_wait_probe(flag, (1 << 26) + 1, None) == R.RADSORT_EINVAL


def test_autotune_without_timing(lib):
    """The autotuner checks its arguments synchronously, and arrays up to
    RADSORT_SCRATCH_MAX_N get the out-of-place plan without any GPU work."""
    from paper_2607_05302_gb300 import radsort as R

    p = R.Plan()
    ptr = ctypes.c_void_p(256)
    assert lib.radsort_autotune(ptr, None, 100, 4, 8, None, None) == R.RADSORT_EINVAL    # no plan
    assert lib.radsort_autotune(ptr, None, 100, 3, 8, None, ctypes.byref(p)) == R.RADSORT_EINVAL
    assert lib.radsort_autotune(ptr, None, 100, 4, 9, None, ctypes.byref(p)) == R.RADSORT_EINVAL
    assert lib.radsort_autotune(ctypes.c_void_p(258), None, 100, 4, 8, None,
                                ctypes.byref(p)) == R.RADSORT_EINVAL                      # alignment
    assert lib.radsort_autotune(ptr, None, 1000, 4, 8, None, ctypes.byref(p)) == R.RADSORT_OK
    assert p.layout == R.RADSORT_LAYOUT_SCRATCH


def test_segmented_workspace_size(lib):
    """Host-side planning of radsort_sort_segmented: decreasing offsets are
    rejected; the per-CTA scratch of the medium segments follows the longest
    medium segment present; each stream of long segments (one per long
    segment, at most four) gets the Radsort workspace of the longest segment
    that takes the full path (above 2^18 elements, in the grid layout at
    these sizes); a long segment whose start is not 16-byte aligned is sorted
    out of place and needs its alternate arrays.  The out-of-place
    comparator needs only its scratch per stream."""
    import numpy as np

    from paper_2607_05302_gb300 import radsort as R

    def ws(lens, db=8):
        off = np.zeros(len(lens) + 1, np.uint64)
        np.cumsum(np.array(lens, np.uint64), out=off[1:])
        return R.segmented_workspace_size(off, 4, 4, db)

    with pytest.raises(R.RadsortError):
        R.segmented_workspace_size(np.array([0, 10, 5], np.uint64), 4, 4, 8)
    base = ws([100])
    assert ws([100] * 1000) - base <= 1000 * 8 + 1024            # index words per segment
    assert ws([5000] * 10) - ws([5000]) <= 10 * 8 + 1024          # medium: the longest decides
    assert ws([5000]) - base < ws([100000]) - base < ws([1 << 18]) - base
    big = (1 << 22) + 4
    assert ws([big]) >= R.radsort_workspace_size(big, 4, 4, 8, layout="grid")
    one = ws([big]) - base                                          # one stream of long segments
    mixed = [big, 1 << 20, 300, 5000]
    medium = max(16 * 5000 * 8, 0.06 * sum(mixed) * 8) + 1024  # medium scratch: 6% of the arrays, >= 16 CTAs
    assert ws(mixed) <= base + 2 * one + medium + 1024
    assert ws([big] * 9) <= base + 4 * one + 9 * 8 + 1024          # at most four streams
    odd = [3, 1 << 20]  # the long segment starts 12 bytes past an aligned address
    assert ws(odd) >= base + (1 << 20) * 8

    def ows(lens):
        off = np.zeros(len(lens) + 1, np.uint64)
        np.cumsum(np.array(lens, np.uint64), out=off[1:])
        return R.lsd_oop_segmented_workspace_size(off, 4, 4, 8)

    assert ows([big]) - ows([100]) < one                             # no block store, only scratch

    # the smallest workspace accepted: the low-memory plan (8-bit digits,
    # medium segments in place, a fixed 514 blocks of 32 elements per CTA,
    # 2 CTAs per SM; no device here: 152 SMs) where it is the smaller
    def mws(lens, db=8):
        off = np.zeros(len(lens) + 1, np.uint64)
        np.cumsum(np.array(lens, np.uint64), out=off[1:])
        return R.segmented_workspace_size(off, 4, 4, db, minimal=True)

    in_place = 2 * 152 * 514 * 32 * 8
    many = [1 << 18] * 2000
    assert abs(mws(many) - ws([100] * 2000) - in_place) <= 1024
    assert mws(many) < ws(many) / 5                                 # the fast plan holds 6% of the arrays
    for lens in ([1 << 18] * 20, mixed, [5000]):                    # never above the fast plan's
        assert mws(lens) <= ws(lens)
    assert abs(mws([1 << 18] * 20) - ws([100] * 20) - 20 * 514 * 32 * 8) <= 1024  # no more CTAs than segments
    assert mws(mixed, 11) == ws(mixed, 11)                          # 11-bit digits: one plan


def test_binding_signatures_match_the_header(lib):
    """Every function include/radsort.h declares is bound in radsort.py with
    as many arguments as the header gives it (a missing or extra argument
    would be read as garbage by the library)."""
    from paper_2607_05302_gb300 import radsort as R

    txt = "\n".join(open(os.path.join(ROOT, "include", h)).read()
                    for h in os.listdir(os.path.join(ROOT, "include")) if h.endswith(".h"))
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    decls = dict(re.findall(r"\b(radsort_\w+)\s*\(([^)]*)\)\s*;", txt))
    assert set(decls) == set(header_functions())
    for name, params in decls.items():
        p = params.strip()
        nargs = 0 if p in ("", "void") else p.count(",") + 1
        fn = getattr(lib, name)
        assert fn.argtypes is not None, name
        assert len(fn.argtypes) == nargs, (name, len(fn.argtypes), nargs)
    assert set(R.EXPORTS) == set(decls)
