"""ctypes loader and multi-threaded driver for the plain C recurrence oracle (swb.c).

TEST INFRASTRUCTURE ONLY (same rule as ``oracle/ranluxpp.py``): only ``tests/``,
``__graft_entry__.smoke()`` and the CPU baseline leg of ``bench.py`` use it.

``build()`` compiles ``swb.c`` with the host C compiler into ``oracle/_build``.  The C
functions release the GIL (ctypes does so for every foreign call), so a thread pool
over stream ranges runs them on all host cores.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "swb.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libswb_oracle.so")
_lib = None

KIND_U24, KIND_F64, KIND_BITS48, KIND_F32 = 0, 1, 2, 3


def build(force=False):
    """Compile the oracle library (plain gcc -O2, no target-specific flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC],
                   check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        vp = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        L.swb_block.argtypes = [vp, vp, i32]
        L.swb_block.restype = None
        L.swb_draw_many.argtypes = [i64, vp, vp, vp, i32, i64, i32, vp]
        L.swb_draw_many.restype = None
        L.swb_sum_hist_many.argtypes = [i64, vp, vp, vp, i32, i64, vp, vp]
        L.swb_sum_hist_many.restype = None
        _lib = L
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def default_threads():
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _ranges(n, parts):
    parts = max(1, min(parts, n))
    edges = np.linspace(0, n, parts + 1).astype(np.int64)
    return [(int(edges[k]), int(edges[k + 1])) for k in range(parts) if edges[k + 1] > edges[k]]


def draw_many(words, carry, pos, p, count, kind, threads=None):
    """Draw ``count`` values from each stream.  ``words``: (n, 24) uint32 windows,
    ``carry``: (n,) uint32, ``pos``: (n,) int32 — all updated in place.  Returns an
    (n, count) array of uint32 (u24), float64 (f64), uint64 (48-bit integers) or
    float32 (f32)."""
    L = lib()
    n = words.shape[0]
    assert words.dtype == np.uint32 and words.shape == (n, 24) and words.flags.c_contiguous
    assert carry.dtype == np.uint32 and pos.dtype == np.int32
    dtype = {KIND_U24: np.uint32, KIND_F64: np.float64, KIND_BITS48: np.uint64, KIND_F32: np.float32}[kind]
    out = np.zeros((n, count), dtype=dtype)
    if n == 0:
        return out

    def work(r):
        a, b = r
        L.swb_draw_many(b - a, _ptr(words[a:b]), _ptr(carry[a:b]), _ptr(pos[a:b]), p,
                        count, kind, _ptr(out[a:b]))

    with ThreadPoolExecutor(threads or default_threads()) as ex:
        list(ex.map(work, _ranges(n, threads or default_threads())))
    return out


def sum_hist_many(words, carry, pos, p, count, threads=None):
    """Fused consumer: per-stream exact sums of ``count`` 48-bit values and the shared
    256-bin histogram of their top 8 bits."""
    L = lib()
    n = words.shape[0]
    sums = np.zeros(n, dtype=np.uint64)
    parts = _ranges(n, threads or default_threads()) if n else []
    hists = np.zeros((max(1, len(parts)), 256), dtype=np.uint64)

    def work(k):
        a, b = parts[k]
        L.swb_sum_hist_many(b - a, _ptr(words[a:b]), _ptr(carry[a:b]), _ptr(pos[a:b]), p,
                            count, _ptr(sums[a:b]), _ptr(hists[k]))

    with ThreadPoolExecutor(threads or default_threads()) as ex:
        list(ex.map(work, range(len(parts))))
    return sums, hists.sum(axis=0, dtype=np.uint64)


def block(window, carry, p):
    """One luxury block on a single window (list of 24 ints); returns (window, carry)."""
    L = lib()
    w = np.array(window, dtype=np.uint32)
    c = np.array([carry], dtype=np.uint32)
    L.swb_block(_ptr(w), _ptr(c), p)
    return [int(x) for x in w], int(c[0])
