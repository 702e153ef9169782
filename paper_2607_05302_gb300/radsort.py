"""Python binding of the C ABI in include/radsort.h (ctypes).

Argument marshalling only: every step of the sort runs in the CUDA library
libradsort_gb300.so built in-tree by paper_2607_05302_gb300/build.py.  If the
library is missing this module raises.  There is no CPU fallback.

The entry points keep the C names and take raw device pointers (ints).  The
`*_tensors` helpers pass torch tensors' data pointers and the current CUDA
stream.  torch supplies memory and streams only.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libradsort_gb300.so")

RADSORT_OK, RADSORT_EINVAL, RADSORT_ENOMEM, RADSORT_ECUDA, RADSORT_ETIMEOUT, RADSORT_EINTERNAL = range(6)
RADSORT_KEY_FLOAT32 = 0x1
RADSORT_LAYOUT_AUTO, RADSORT_LAYOUT_CHUNKS, RADSORT_LAYOUT_GRID, RADSORT_LAYOUT_SCRATCH = 0, 1, 2, 3
RADSORT_LAYOUT_MSD = 4
RADSORT_SCRATCH_MAX_N = 1 << 18
LAYOUTS = {"auto": RADSORT_LAYOUT_AUTO, "chunks": RADSORT_LAYOUT_CHUNKS, "grid": RADSORT_LAYOUT_GRID,
           "scratch": RADSORT_LAYOUT_SCRATCH, "msd": RADSORT_LAYOUT_MSD}


class RadsortError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_str(status)} ({status})")
        self.status = status


class TraceRec(ctypes.Structure):
    _fields_ = [("phase", ctypes.c_int32), ("round", ctypes.c_int32), ("ms", ctypes.c_float)]


PHASES = {0: "setup", 1: "sortPhase", 2: "fixupPhase", 3: "Finalize", 4: "key_transform"}


class Plan(ctypes.Structure):
    _fields_ = [("block_size", ctypes.c_uint32), ("num_chunks", ctypes.c_uint32),
                ("layout", ctypes.c_uint32), ("shape", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 4)]


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"CUDA library {LIB_PATH} is missing: run `python -c 'import __graft_entry__ as g; "
                f"g.build()'` first (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        vp, sz, i, u32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint32
        pplan = ctypes.POINTER(Plan)
        sig = {
            "radsort_status_str": ([i], ctypes.c_char_p),
            "radsort_plan_default": ([sz, i, i, i, pplan], i),
            "radsort_autotune": ([vp, vp, sz, i, i, vp, pplan], i),
            "radsort_autotune_digits": ([vp, vp, sz, i, vp, ctypes.POINTER(i), pplan], i),
            "radsort_segmented_autotune": ([vp, vp, vp, vp, sz, i, vp, ctypes.POINTER(i)], i),
            "radsort_workspace_size": ([sz, i, i, i, pplan, ctypes.POINTER(sz)], i),
            "radsort_sort": ([vp, vp, sz, i, i, vp], i),
            "radsort_sort_noalloc": ([vp, vp, sz, i, i, vp], i),
            "radsort_segmented_workspace_size": ([vp, sz, i, i, i, ctypes.POINTER(sz)], i),
            "radsort_segmented_workspace_size_min": ([vp, sz, i, i, i, ctypes.POINTER(sz)], i),
            "radsort_sort_segmented": ([vp, vp, vp, vp, sz, i, i, vp, sz, vp], i),
            "radsort_lsd_oop_segmented_workspace_size": ([vp, sz, i, i, i, ctypes.POINTER(sz)], i),
            "radsort_lsd_oop_sort_segmented": ([vp, vp, vp, vp, vp, vp, sz, i, i, vp, sz, vp], i),
            "radsort_sort_ex": ([vp, vp, sz, i, i, u32, pplan, vp, sz, vp], i),
            "radsort_sort_rounds": ([vp, vp, sz, i, i, i, pplan, vp, vp, vp], i),
            "radsort_lsd_oop_sort": ([vp, vp, vp, vp, sz, i, i, vp], i),
            "radsort_lsd_oop_scratch_size": ([sz, i, i, i, ctypes.POINTER(sz)], i),
            "radsort_float_keys": ([vp, sz, i, vp], i),
            "radsort_device_status": ([vp], i),
            "radsort_debug_wait_probe": ([vp, ctypes.c_uint, vp], i),
            "radsort_trace_enable": ([i], i),
            "radsort_trace_read": ([ctypes.POINTER(TraceRec), i, ctypes.POINTER(i)], i),
            "radsort_launch_count": ([ctypes.POINTER(ctypes.c_uint64)], i),
            "radsort_perm_workspace_size": ([sz, i, i, i, u32, ctypes.POINTER(sz)], i),
            "radsort_perm_open": ([vp, vp, sz, i, i, u32, vp, sz, vp, ctypes.POINTER(vp)], i),
            "radsort_perm_rounds": ([vp, i, i, vp], i),
            "radsort_perm_keys_changed": ([vp], i),
            "radsort_perm_size": ([vp, ctypes.POINTER(sz), ctypes.POINTER(sz)], i),
            "radsort_perm_blocks": ([vp, vp, sz, vp], i),
            "radsort_perm_gather": ([vp, vp, vp, vp], i),
            "radsort_perm_truncate": ([vp, sz, vp], i),
            "radsort_perm_finalize": ([vp, vp], i),
            "radsort_perm_close": ([vp], i),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


# exported names declared in include/radsort.h
EXPORTS = ("radsort_status_str", "radsort_plan_default", "radsort_autotune", "radsort_autotune_digits",
           "radsort_segmented_autotune", "radsort_workspace_size", "radsort_sort",
           "radsort_sort_noalloc", "radsort_segmented_workspace_size", "radsort_segmented_workspace_size_min",
           "radsort_sort_segmented",
           "radsort_lsd_oop_segmented_workspace_size", "radsort_lsd_oop_sort_segmented",
           "radsort_sort_ex", "radsort_sort_rounds", "radsort_lsd_oop_sort",
           "radsort_lsd_oop_scratch_size", "radsort_float_keys",
           "radsort_device_status", "radsort_debug_wait_probe", "radsort_trace_enable", "radsort_trace_read",
           "radsort_launch_count", "radsort_perm_workspace_size", "radsort_perm_open", "radsort_perm_rounds",
           "radsort_perm_keys_changed", "radsort_perm_size", "radsort_perm_blocks", "radsort_perm_gather",
           "radsort_perm_truncate", "radsort_perm_finalize", "radsort_perm_close")


def status_str(s: int) -> str:
    return lib().radsort_status_str(s).decode()


def _ok(s: int, what: str):
    if s != RADSORT_OK:
        raise RadsortError(s, what)


def _layout(layout):
    return LAYOUTS[layout] if isinstance(layout, str) else int(layout)


def _plan(block_size=0, num_chunks=0, layout=0, shape=0):
    layout = _layout(layout)
    if not block_size and not num_chunks and not layout and not shape:
        return None
    p = Plan()
    p.block_size = block_size
    p.num_chunks = num_chunks
    p.layout = layout
    p.shape = shape
    return ctypes.byref(p)


# ---------------------------------------------------------------- raw C names
def radsort_plan_default(n, key_bytes, value_bytes, digit_bits):
    """(block_size, num_chunks, layout) of the automatic plan."""
    p = Plan()
    _ok(lib().radsort_plan_default(n, key_bytes, value_bytes, digit_bits, ctypes.byref(p)),
        "radsort_plan_default")
    return int(p.block_size), int(p.num_chunks), int(p.layout)


def radsort_autotune(keys, values=None, *, digit_bits=8, stream=None):
    """(block_size, num_chunks, layout, shape) of the fastest plan for sorting
    these CUDA tensors (timed on copies; the tensors are not modified)."""
    p = Plan()
    _ok(lib().radsort_autotune(_ptr(keys), _ptr(values), keys.numel(), _key_bytes(keys), digit_bits,
                               _torch_stream(stream), ctypes.byref(p)), "radsort_autotune")
    return int(p.block_size), int(p.num_chunks), int(p.layout), int(p.shape)


def radsort_autotune_digits(keys, values=None, *, stream=None):
    """(digit_bits, block_size, num_chunks, layout, shape) of the fastest plan
    over both digit widths (timed on copies)."""
    p = Plan()
    d = ctypes.c_int(0)
    _ok(lib().radsort_autotune_digits(_ptr(keys), _ptr(values), keys.numel(), _key_bytes(keys),
                                      _torch_stream(stream), ctypes.byref(d), ctypes.byref(p)),
        "radsort_autotune_digits")
    return int(d.value), int(p.block_size), int(p.num_chunks), int(p.layout), int(p.shape)


def segmented_autotune(keys, values, offsets_dev, offsets_host, *, stream=None):
    """The faster digit width (8 or 11) for this batch, timed on copies."""
    import numpy as np
    oh = np.ascontiguousarray(offsets_host, dtype=np.uint64)
    d = ctypes.c_int(0)
    _ok(lib().radsort_segmented_autotune(_ptr(keys), _ptr(values), _ptr(offsets_dev),
                                         oh.ctypes.data_as(ctypes.c_void_p), oh.size - 1, _key_bytes(keys),
                                         _torch_stream(stream), ctypes.byref(d)), "radsort_segmented_autotune")
    return int(d.value)


def radsort_workspace_size(n, key_bytes, value_bytes, digit_bits, block_size=0, num_chunks=0,
                           layout=0, shape=0):
    out = ctypes.c_size_t(0)
    _ok(lib().radsort_workspace_size(n, key_bytes, value_bytes, digit_bits,
                                     _plan(block_size, num_chunks, layout, shape), ctypes.byref(out)),
        "radsort_workspace_size")
    return int(out.value)


def radsort_sort(keys, values, n, key_bytes, digit_bits, stream):
    _ok(lib().radsort_sort(keys, values, n, key_bytes, digit_bits, stream), "radsort_sort")


def radsort_sort_ex(keys, values, n, key_bytes, digit_bits, flags=0, block_size=0, num_chunks=0,
                    workspace=None, workspace_bytes=0, stream=None, layout=0, shape=0):
    _ok(lib().radsort_sort_ex(keys, values, n, key_bytes, digit_bits, flags,
                              _plan(block_size, num_chunks, layout, shape), workspace, workspace_bytes,
                              stream),
        "radsort_sort_ex")


def radsort_sort_rounds(keys, values, n, key_bytes, digit_bits, rounds, out_keys, out_values,
                        block_size=0, num_chunks=0, stream=None, layout=0):
    _ok(lib().radsort_sort_rounds(keys, values, n, key_bytes, digit_bits, rounds,
                                  _plan(block_size, num_chunks, layout), out_keys, out_values,
                                  stream),
        "radsort_sort_rounds")


def radsort_lsd_oop_scratch_size(n, key_bytes, value_bytes, digit_bits):
    out = ctypes.c_size_t(0)
    _ok(lib().radsort_lsd_oop_scratch_size(n, key_bytes, value_bytes, digit_bits, ctypes.byref(out)),
        "radsort_lsd_oop_scratch_size")
    return out.value


def radsort_lsd_oop_sort(keys, values, keys_alt, values_alt, n, key_bytes, digit_bits, stream):
    _ok(lib().radsort_lsd_oop_sort(keys, values, keys_alt, values_alt, n, key_bytes, digit_bits,
                                   stream), "radsort_lsd_oop_sort")


def radsort_float_keys(keys, n, inverse, stream):
    _ok(lib().radsort_float_keys(keys, n, inverse, stream), "radsort_float_keys")


def radsort_device_status(stream=None):
    _ok(lib().radsort_device_status(stream), "device status")


def radsort_debug_wait_probe(flag, iterations, stream=None):
    """One bounded wait on the device word `flag` (a CUDA int32 tensor); a
    flag that stays 0 makes the next radsort_device_status raise ETIMEOUT."""
    _ok(lib().radsort_debug_wait_probe(_ptr(flag), iterations, _torch_stream(stream)),
        "radsort_debug_wait_probe")


def radsort_trace_enable(on: bool):
    _ok(lib().radsort_trace_enable(1 if on else 0), "radsort_trace_enable")


def radsort_trace_read(cap: int = 1 << 16):
    """[(phase_name, round, ms), ...] in launch order; clears the list."""
    buf = (TraceRec * cap)()
    cnt = ctypes.c_int(0)
    _ok(lib().radsort_trace_read(buf, cap, ctypes.byref(cnt)), "radsort_trace_read")
    return [(PHASES.get(buf[i].phase, "?"), int(buf[i].round), float(buf[i].ms))
            for i in range(min(cnt.value, cap))]


def radsort_launch_count() -> int:
    v = ctypes.c_uint64(0)
    _ok(lib().radsort_launch_count(ctypes.byref(v)), "radsort_launch_count")
    return int(v.value)


# ---------------------------------------------------------------- torch helpers
def _torch_stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _key_bytes(t):
    import torch
    kb = {torch.int32: 4, torch.uint32: 4, torch.float32: 4, torch.int64: 8, torch.uint64: 8}.get(t.dtype)
    if kb is None:
        raise TypeError(f"unsupported key dtype {t.dtype}")
    return kb


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def sort_tensors(keys, values=None, *, digit_bits=8, float_keys=False, block_size=0, num_chunks=0,
                 workspace=None, stream=None, layout=0, shape=0):
    """In-place stable Radsort of CUDA tensors (keys: 32/64-bit, read as
    unsigned; values: optional 32-bit)."""
    assert keys.is_cuda and keys.is_contiguous()
    n = keys.numel()
    if values is not None:
        assert values.is_cuda and values.is_contiguous() and values.numel() == n
        assert values.element_size() == 4
    ws, wsb = (None, 0) if workspace is None else (_ptr(workspace), workspace.numel() * workspace.element_size())
    radsort_sort_ex(_ptr(keys), _ptr(values), n, _key_bytes(keys), digit_bits,
                    RADSORT_KEY_FLOAT32 if float_keys else 0, block_size, num_chunks, ws, wsb,
                    _torch_stream(stream), layout, shape)


def sort_rounds_tensors(keys, values, rounds, out_keys, out_values=None, *, digit_bits=8,
                        block_size=0, num_chunks=0, stream=None, layout=0):
    radsort_sort_rounds(_ptr(keys), _ptr(values), keys.numel(), _key_bytes(keys), digit_bits, rounds,
                        _ptr(out_keys), _ptr(out_values), block_size, num_chunks,
                        _torch_stream(stream), layout)


def lsd_oop_tensors(keys, values, keys_alt, values_alt, *, digit_bits=8, stream=None):
    radsort_lsd_oop_sort(_ptr(keys), _ptr(values), _ptr(keys_alt), _ptr(values_alt), keys.numel(),
                         _key_bytes(keys), digit_bits, _torch_stream(stream))


def segmented_workspace_size(offsets_host, key_bytes, value_bytes, digit_bits=8, *, minimal=False):
    """offsets_host: numpy uint64 array of num_segments + 1 offsets.  minimal:
    the smallest workspace the sort accepts (the low-memory plan: medium
    segments sorted in place, 8-bit digits), else the fast plan's."""
    import numpy as np
    oh = np.ascontiguousarray(offsets_host, dtype=np.uint64)
    out = ctypes.c_size_t(0)
    name = "radsort_segmented_workspace_size_min" if minimal else "radsort_segmented_workspace_size"
    _ok(getattr(lib(), name)(oh.ctypes.data_as(ctypes.c_void_p), oh.size - 1,
                             key_bytes, value_bytes, digit_bits, ctypes.byref(out)), name)
    return int(out.value)


def sort_segmented_tensors(keys, values, offsets_dev, offsets_host, *, digit_bits=8, workspace=None,
                           stream=None):
    """Stable sort of every segment [off[s], off[s+1]) of CUDA tensors in place.
    offsets_dev: int64 CUDA tensor; offsets_host: numpy uint64 array (same values)."""
    import numpy as np
    oh = np.ascontiguousarray(offsets_host, dtype=np.uint64)
    ws, wsb = (None, 0) if workspace is None else (_ptr(workspace), workspace.numel() * workspace.element_size())
    _ok(lib().radsort_sort_segmented(_ptr(keys), _ptr(values), _ptr(offsets_dev),
                                     oh.ctypes.data_as(ctypes.c_void_p), oh.size - 1, _key_bytes(keys),
                                     digit_bits, ws, wsb, _torch_stream(stream)),
        "radsort_sort_segmented")


def lsd_oop_segmented_workspace_size(offsets_host, key_bytes, value_bytes, digit_bits=8):
    import numpy as np
    oh = np.ascontiguousarray(offsets_host, dtype=np.uint64)
    out = ctypes.c_size_t(0)
    _ok(lib().radsort_lsd_oop_segmented_workspace_size(oh.ctypes.data_as(ctypes.c_void_p), oh.size - 1,
                                                       key_bytes, value_bytes, digit_bits, ctypes.byref(out)),
        "radsort_lsd_oop_segmented_workspace_size")
    return int(out.value)


def lsd_oop_segmented_tensors(keys, values, keys_alt, values_alt, offsets_dev, offsets_host, *, digit_bits=8,
                              workspace=None, stream=None):
    """The out-of-place comparator of the batched sort (long segments through
    n-element alternate arrays)."""
    import numpy as np
    oh = np.ascontiguousarray(offsets_host, dtype=np.uint64)
    ws, wsb = (None, 0) if workspace is None else (_ptr(workspace), workspace.numel() * workspace.element_size())
    _ok(lib().radsort_lsd_oop_sort_segmented(_ptr(keys), _ptr(values), _ptr(keys_alt), _ptr(values_alt),
                                             _ptr(offsets_dev), oh.ctypes.data_as(ctypes.c_void_p), oh.size - 1,
                                             _key_bytes(keys), digit_bits, ws, wsb, _torch_stream(stream)),
        "radsort_lsd_oop_sort_segmented")


def float_keys_tensors(keys, inverse=False, stream=None):
    radsort_float_keys(_ptr(keys), keys.numel(), 1 if inverse else 0, _torch_stream(stream))


# ---------------------------------------------------------------- permuted representation
BLOCK_WORDS = 3  # radsort_block as three 64-bit words: keys address, values address, len | reserved << 32


def perm_workspace_size(n, key_bytes, value_bytes, digit_bits=8, block_size=0):
    out = ctypes.c_size_t(0)
    _ok(lib().radsort_perm_workspace_size(n, key_bytes, value_bytes, digit_bits, block_size,
                                          ctypes.byref(out)), "radsort_perm_workspace_size")
    return int(out.value)


class Perm:
    """A Radsort state kept between calls on CUDA tensors (Sec. 4.1): rounds,
    the block list in logical order, truncation (Alg. 8), the gathered
    sequence and Finalize.  Every step runs in the CUDA library; this class
    only marshals arguments."""

    def __init__(self, keys, values=None, *, digit_bits=8, block_size=0, workspace=None, stream=None):
        import torch

        assert keys.is_cuda and keys.is_contiguous()
        self.keys, self.values, self.digit_bits = keys, values, digit_bits
        n = keys.numel()
        need = perm_workspace_size(n, _key_bytes(keys), 4 if values is not None else 0, digit_bits,
                                   block_size)
        self.workspace = workspace if workspace is not None else torch.empty(
            max(need, 1), dtype=torch.uint8, device=keys.device)
        h = ctypes.c_void_p(0)
        _ok(lib().radsort_perm_open(_ptr(keys), _ptr(values), n, _key_bytes(keys), digit_bits, block_size,
                                    _ptr(self.workspace), self.workspace.numel(), _torch_stream(stream),
                                    ctypes.byref(h)), "radsort_perm_open")
        self._h = h

    def close(self):
        if self._h:
            lib().radsort_perm_close(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rounds(self, first, count, stream=None):
        _ok(lib().radsort_perm_rounds(self._h, first, count, _torch_stream(stream)), "radsort_perm_rounds")

    def keys_changed(self):
        _ok(lib().radsort_perm_keys_changed(self._h), "radsort_perm_keys_changed")

    def size(self):
        n, m = ctypes.c_size_t(0), ctypes.c_size_t(0)
        _ok(lib().radsort_perm_size(self._h, ctypes.byref(n), ctypes.byref(m)), "radsort_perm_size")
        return int(n.value), int(m.value)

    def blocks(self, stream=None):
        """The block list as an int64 CUDA tensor of shape (entries, 3):
        key address, value address, used length."""
        import torch

        _, m = self.size()
        out = torch.empty((m, BLOCK_WORDS), dtype=torch.int64, device=self.keys.device)
        _ok(lib().radsort_perm_blocks(self._h, _ptr(out), m, _torch_stream(stream)), "radsort_perm_blocks")
        return out

    def gather(self, out_keys, out_values=None, stream=None):
        _ok(lib().radsort_perm_gather(self._h, _ptr(out_keys), _ptr(out_values), _torch_stream(stream)),
            "radsort_perm_gather")

    def truncate(self, m, stream=None):
        _ok(lib().radsort_perm_truncate(self._h, m, _torch_stream(stream)), "radsort_perm_truncate")

    def finalize(self, stream=None):
        _ok(lib().radsort_perm_finalize(self._h, _torch_stream(stream)), "radsort_perm_finalize")
