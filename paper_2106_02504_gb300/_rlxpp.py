"""ctypes binding of librlxpp.so, one Python function per C entry point of
include/rlxpp.h, with the same names.  Only argument marshalling happens here: integers
and pointers are passed through, torch tensors are passed by ``data_ptr()``, CUDA
streams by their handle.  Every non-OK status raises ``RlxppError``.

There is no fallback: if the CUDA library is missing, importing this module fails.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64
_i64 = ctypes.c_int64
_u32 = ctypes.c_uint32


class RlxppState(ctypes.Structure):
    """struct rlxpp_state (88 bytes)."""
    _fields_ = [("d", ctypes.c_uint64 * 9), ("carry", ctypes.c_uint32), ("pos", ctypes.c_uint32),
                ("p", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


STATE_BYTES = ctypes.sizeof(RlxppState)
assert STATE_BYTES == 88


class RlxppTuning(ctypes.Structure):
    """struct rlxpp_tuning."""
    _fields_ = [("chunk_blocks", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32), ("path", ctypes.c_uint32),
                ("threads_per_block", ctypes.c_uint32)]


RLXPP_KIND_U24, RLXPP_KIND_F64, RLXPP_KIND_F32 = 0, 1, 2
RLXPP_PATH_IMAD, RLXPP_PATH_TENSOR, RLXPP_PATH_WARP = 0, 1, 2
RLXPP_REQ_ADVANCE = 1


def request_dtype():
    """numpy dtype laid out like struct rlxpp_request (40 bytes)."""
    import numpy as np
    return np.dtype([("stream", "<u8"), ("skip", "<u8"), ("pos", "<u4"), ("kind", "<u4"),
                     ("count", "<i8"), ("offset", "<u8")])

def served_dtype():
    """numpy dtype laid out like struct rlxpp_served (80 bytes)."""
    import numpy as np
    return np.dtype([("rid", "<u8"), ("stream", "<u8"), ("skip", "<u8"), ("pos", "<u4"), ("kind", "<u4"),
                     ("count", "<i8"), ("offset", "<u8"), ("nbytes", "<u8"), ("arrival", "<f8"),
                     ("launch", "<f8"), ("done", "<f8")])


RLXPP_SERVER_COPY_TO_HOST, RLXPP_SERVER_KEEP_RESULTS = 1, 2

RLXPP_OK, RLXPP_ERR_INVALID, RLXPP_ERR_NOMEM, RLXPP_ERR_CUDA, RLXPP_ERR_TIMEOUT, \
    RLXPP_ERR_UNSUPPORTED = range(6)
RLXPP_MAX_LEVELS = 16
RLXPP_NOALLOC_MAX_LEVELS = 4


class RlxppError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"rlxpp status {status}: {message}")
        self.status = status


def _load():
    path = _build.LIB_PATH
    if not os.path.exists(path):
        raise ImportError(
            f"librlxpp.so not built ({path}); run paper_2106_02504_gb300.build.build() first")
    L = ctypes.CDLL(path)
    sigs = {
        "rlxpp_create": [_u64, _vp, _u32, _vp, _vp, _vp, ctypes.POINTER(_vp)],
        "rlxpp_seed": [_vp, _vp, _vp],
        "rlxpp_skip": [_vp, _vp, _vp],
        "rlxpp_draw_u24": [_vp, _vp, _vp, _i64, _vp, _vp],
        "rlxpp_draw_f64": [_vp, _vp, _vp, _i64, _vp, _vp],
        "rlxpp_draw_f32": [_vp, _vp, _vp, _i64, _vp, _vp],
        "rlxpp_draw_normal_f64": [_vp, _vp, _vp, _i64, _vp, _vp],
        "rlxpp_draw_exp_f64": [_vp, _vp, _vp, _i64, _vp, _vp],
        "rlxpp_draw_raw_f64": [_vp, _vp, _vp, _i64, _vp, _vp],
        "rlxpp_draw_u24_host_async": [_vp, _i64, _vp, _vp],
        "rlxpp_draw_f64_host_async": [_vp, _i64, _vp, _vp],
        "rlxpp_host_wait": [_vp, _vp],
        "rlxpp_skip_values": [_vp, _vp, _u32, _vp],
        "rlxpp_draw_f64_sum_hist": [_vp, _i64, _vp, _vp, _vp],
        "rlxpp_get_state": [_vp, _vp, _vp],
        "rlxpp_set_state": [_vp, _vp, _vp],
        "rlxpp_sync": [_vp, _vp],
        "rlxpp_test_multiply9x9": [_vp, _vp, _vp, _u64, _vp],
        "rlxpp_test_mod_m": [_vp, _vp, _u64, _vp],
        "rlxpp_test_mul_mod": [_vp, _vp, _vp, _u64, _vp],
        "rlxpp_test_to_ranlux": [_vp, _vp, _vp, _u64, _vp],
        "rlxpp_test_to_lcg": [_vp, _vp, _vp, _u64, _vp],
        "rlxpp_test_f64_from48": [_vp, _vp, _u64, _vp],
        "rlxpp_test_warp_mod_m": [_vp, _vp, _u64, _vp],
        "rlxpp_test_warp_to_ranlux": [_vp, _vp, _vp, _u64, _vp],
        "rlxpp_test_neg_ln48": [_vp, _vp, _u64, _vp],
        "rlxpp_test_fail_alloc": [_i64],
        "rlxpp_test_cos_sin_2pi48": [_vp, _vp, _u64, _vp],
        "rlxpp_test_box_muller48": [_vp, _vp, _u64, _vp],
        "rlxpp_luxury_multiplier": [_u32, _vp],
        "rlxpp_seed_states_noalloc": [_vp, _u32, _vp, _vp, _u64, _vp, _vp],
        "rlxpp_plan_requests": [_vp, _vp, _u64, _u32, _vp, ctypes.POINTER(_vp)],
        "rlxpp_run_plan": [_vp, _vp, _vp, _vp, _vp],
        "rlxpp_draw_requests": [_vp, _vp, _u64, _vp, _vp, _u32, _vp],
        "rlxpp_autotune_requests": [_vp, _vp, _u64, _vp, _vp, _vp, _vp],
        "rlxpp_set_path": [_vp, _u32],
        "rlxpp_test_tc_mulmod": [_u32, _vp, _vp, _u64, _vp],
        "rlxpp_test_tc_timeout": [_vp, _vp],
        "rlxpp_server_create": [_vp, _u64, _u32, _u32, _u64, _u64, _u32, ctypes.POINTER(_vp)],
        "rlxpp_server_submit": [_vp, _u64, _u64, _u32, _i64, ctypes.c_double, ctypes.POINTER(ctypes.c_int)],
        "rlxpp_server_cancel": [_vp, _u64, ctypes.POINTER(ctypes.c_int)],
        "rlxpp_server_pump": [_vp, ctypes.c_int],
        "rlxpp_server_drain": [_vp],
        "rlxpp_server_stats": [_vp, _vp],
        "rlxpp_server_take_done": [_vp, _vp, _u64, ctypes.POINTER(_u64)],
        "rlxpp_server_result": [_vp, _u64, _vp, _u64],
        "rlxpp_server_run_trace": [_vp, _u64, _vp, _vp, _vp, _vp, _vp],
    }
    for name, args in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.rlxpp_num_streams.argtypes = [_vp]
    L.rlxpp_num_streams.restype = _u64
    L.rlxpp_last_error.argtypes = []
    L.rlxpp_last_error.restype = ctypes.c_char_p
    L.rlxpp_destroy.argtypes = [_vp]
    L.rlxpp_destroy.restype = None
    L.rlxpp_plan_items.argtypes = [_vp]
    L.rlxpp_plan_items.restype = _u64
    L.rlxpp_plan_tuning.argtypes = [_vp]
    L.rlxpp_plan_tuning.restype = RlxppTuning
    L.rlxpp_get_path.argtypes = [_vp]
    L.rlxpp_get_path.restype = _u32
    L.rlxpp_destroy_plan.argtypes = [_vp]
    L.rlxpp_destroy_plan.restype = None
    L.rlxpp_server_destroy.argtypes = [_vp]
    L.rlxpp_server_destroy.restype = None
    return L


_lib = _load()
LIB_PATH = _build.LIB_PATH


def _ptr(x):
    """None -> NULL, int -> address, torch tensor / numpy array -> its data pointer."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    if isinstance(x, ctypes.Array) or isinstance(x, ctypes.Structure):
        return ctypes.addressof(x)
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(s):
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:  # pragma: no cover
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(status):
    if status != RLXPP_OK:
        raise RlxppError(status, _lib.rlxpp_last_error().decode(errors="replace"))


# ---- one function per C entry point ------------------------------------------------
def rlxpp_create(n_streams, levels, seeds, level_of_stream=None, stream=None):
    """Returns the handle (an int).  levels: sequence of luxury levels p (host)."""
    arr = (_u32 * len(levels))(*levels)
    h = _vp()
    _check(_lib.rlxpp_create(n_streams, arr, len(levels), _ptr(level_of_stream), _ptr(seeds),
                             _stream(stream), ctypes.byref(h)))
    return h.value


def rlxpp_seed(gen, seeds, stream=None):
    _check(_lib.rlxpp_seed(gen, _ptr(seeds), _stream(stream)))


def rlxpp_skip(gen, n128, stream=None):
    _check(_lib.rlxpp_skip(gen, _ptr(n128), _stream(stream)))


def rlxpp_draw_u24(gen, out, count_each=0, counts=None, offsets=None, stream=None):
    _check(_lib.rlxpp_draw_u24(gen, _ptr(counts), _ptr(offsets), count_each, _ptr(out), _stream(stream)))


def rlxpp_draw_f64(gen, out, count_each=0, counts=None, offsets=None, stream=None):
    _check(_lib.rlxpp_draw_f64(gen, _ptr(counts), _ptr(offsets), count_each, _ptr(out), _stream(stream)))


def rlxpp_draw_f32(gen, out, count_each=0, counts=None, offsets=None, stream=None):
    _check(_lib.rlxpp_draw_f32(gen, _ptr(counts), _ptr(offsets), count_each, _ptr(out), _stream(stream)))


def rlxpp_draw_normal_f64(gen, out, count_each=0, counts=None, offsets=None, stream=None):
    _check(_lib.rlxpp_draw_normal_f64(gen, _ptr(counts), _ptr(offsets), count_each, _ptr(out), _stream(stream)))


def rlxpp_draw_exp_f64(gen, out, count_each=0, counts=None, offsets=None, stream=None):
    _check(_lib.rlxpp_draw_exp_f64(gen, _ptr(counts), _ptr(offsets), count_each, _ptr(out), _stream(stream)))


def rlxpp_draw_raw_f64(gen, out, count_each=0, counts=None, offsets=None, stream=None):
    _check(_lib.rlxpp_draw_raw_f64(gen, _ptr(counts), _ptr(offsets), count_each, _ptr(out), _stream(stream)))


def rlxpp_draw_u24_host_async(gen, out, count_each, stream=None):
    _check(_lib.rlxpp_draw_u24_host_async(gen, count_each, _ptr(out), _stream(stream)))


def rlxpp_draw_f64_host_async(gen, out, count_each, stream=None):
    _check(_lib.rlxpp_draw_f64_host_async(gen, count_each, _ptr(out), _stream(stream)))


def rlxpp_host_wait(gen, stream=None):
    _check(_lib.rlxpp_host_wait(gen, _stream(stream)))


def rlxpp_skip_values(gen, n_values, kind, stream=None):
    _check(_lib.rlxpp_skip_values(gen, _ptr(n_values), kind, _stream(stream)))


def rlxpp_draw_f64_sum_hist(gen, count_each, sums, hist, stream=None):
    _check(_lib.rlxpp_draw_f64_sum_hist(gen, count_each, _ptr(sums), _ptr(hist), _stream(stream)))


def rlxpp_get_state(gen, dst, stream=None):
    _check(_lib.rlxpp_get_state(gen, _ptr(dst), _stream(stream)))


def rlxpp_set_state(gen, src, stream=None):
    _check(_lib.rlxpp_set_state(gen, _ptr(src), _stream(stream)))


def rlxpp_sync(gen, stream=None):
    _check(_lib.rlxpp_sync(gen, _stream(stream)))


def rlxpp_num_streams(gen):
    return int(_lib.rlxpp_num_streams(gen))


def rlxpp_last_error():
    return _lib.rlxpp_last_error().decode(errors="replace")


def rlxpp_destroy(gen):
    _lib.rlxpp_destroy(gen)


def rlxpp_test_multiply9x9(x, y, out, n, stream=None):
    _check(_lib.rlxpp_test_multiply9x9(_ptr(x), _ptr(y), _ptr(out), n, _stream(stream)))


def rlxpp_test_mod_m(inp, out, n, stream=None):
    _check(_lib.rlxpp_test_mod_m(_ptr(inp), _ptr(out), n, _stream(stream)))


def rlxpp_test_mul_mod(x, y, out, n, stream=None):
    _check(_lib.rlxpp_test_mul_mod(_ptr(x), _ptr(y), _ptr(out), n, _stream(stream)))


def rlxpp_test_to_ranlux(x, d, carry, n, stream=None):
    _check(_lib.rlxpp_test_to_ranlux(_ptr(x), _ptr(d), _ptr(carry), n, _stream(stream)))


def rlxpp_test_to_lcg(d, carry, x, n, stream=None):
    _check(_lib.rlxpp_test_to_lcg(_ptr(d), _ptr(carry), _ptr(x), n, _stream(stream)))


def rlxpp_test_f64_from48(v, out, n, stream=None):
    _check(_lib.rlxpp_test_f64_from48(_ptr(v), _ptr(out), n, _stream(stream)))


def rlxpp_test_warp_mod_m(inp, out, n, stream=None):
    _check(_lib.rlxpp_test_warp_mod_m(_ptr(inp), _ptr(out), n, _stream(stream)))


def rlxpp_test_warp_to_ranlux(x, d, carry, n, stream=None):
    _check(_lib.rlxpp_test_warp_to_ranlux(_ptr(x), _ptr(d), _ptr(carry), n, _stream(stream)))


def rlxpp_server_create(gen, pool_bytes, n_cuda_streams=4, max_batch=512, small_bytes=1 << 20,
                        max_queued_bytes=0, flags=RLXPP_SERVER_COPY_TO_HOST):
    h = _vp()
    _check(_lib.rlxpp_server_create(gen, pool_bytes, n_cuda_streams, max_batch, small_bytes, max_queued_bytes,
                                    flags, ctypes.byref(h)))
    return h.value


def rlxpp_server_destroy(server):
    _lib.rlxpp_server_destroy(server)


def rlxpp_server_submit(server, rid, stream, kind, count, arrival=-1.0):
    ok = ctypes.c_int()
    _check(_lib.rlxpp_server_submit(server, rid, stream, kind, count, arrival, ctypes.byref(ok)))
    return bool(ok.value)


def rlxpp_server_cancel(server, rid):
    ok = ctypes.c_int()
    _check(_lib.rlxpp_server_cancel(server, rid, ctypes.byref(ok)))
    return bool(ok.value)


def rlxpp_server_pump(server, wait_for_one=False):
    _check(_lib.rlxpp_server_pump(server, int(bool(wait_for_one))))


def rlxpp_server_drain(server):
    _check(_lib.rlxpp_server_drain(server))


def rlxpp_server_stats(server):
    """dict of the counters of struct rlxpp_server_state."""
    keys = ("waiting", "admitted", "inflight_groups", "arena_used", "queued_bytes", "done", "rejected", "cancelled",
            "max_launch_us", "slow_launches", "batches_timed", "kernel_us_sum", "kernel_us_max", "copy_us_sum",
            "copy_us_max")
    v = (_u64 * len(keys))()
    _check(_lib.rlxpp_server_stats(server, ctypes.addressof(v)))
    return dict(zip(keys, list(v)))


def rlxpp_server_take_done(server, max_records=1 << 16):
    import numpy as np
    out = np.zeros(max_records, dtype=served_dtype())
    n = _u64()
    _check(_lib.rlxpp_server_take_done(server, out.ctypes.data, max_records, ctypes.byref(n)))
    return out[:n.value]


def rlxpp_server_result(server, rid, out):
    """Copies the kept result of request rid into the numpy array out (its size in bytes)."""
    _check(_lib.rlxpp_server_result(server, rid, out.ctypes.data if out.nbytes else None, out.nbytes))


def rlxpp_server_run_trace(server, arrival, stream, count, is_f64):
    """Latencies in seconds (float64 array; -1 for rejected requests)."""
    import numpy as np
    arrival = np.ascontiguousarray(arrival, dtype=np.float64)
    stream = np.ascontiguousarray(stream, dtype=np.uint64)
    count = np.ascontiguousarray(count, dtype=np.int64)
    is_f64 = np.ascontiguousarray(is_f64, dtype=np.uint8)
    n = len(arrival)
    lat = np.zeros(n, dtype=np.float64)
    _check(_lib.rlxpp_server_run_trace(server, n, arrival.ctypes.data, stream.ctypes.data, count.ctypes.data,
                                       is_f64.ctypes.data, lat.ctypes.data))
    return lat


def rlxpp_test_fail_alloc(after):
    _check(_lib.rlxpp_test_fail_alloc(after))


def rlxpp_test_neg_ln48(w, out, n, stream=None):
    _check(_lib.rlxpp_test_neg_ln48(_ptr(w), _ptr(out), n, _stream(stream)))


def rlxpp_test_cos_sin_2pi48(v, out, n, stream=None):
    _check(_lib.rlxpp_test_cos_sin_2pi48(_ptr(v), _ptr(out), n, _stream(stream)))


def rlxpp_test_box_muller48(v, out, n, stream=None):
    _check(_lib.rlxpp_test_box_muller48(_ptr(v), _ptr(out), n, _stream(stream)))


def rlxpp_seed_states_noalloc(levels, seeds, n_streams, out, level_of_stream=None, stream=None):
    """Seeded state records written to caller-owned device memory, without any device
    allocation (the library's fixed scratch array holds the level tables)."""
    arr = (_u32 * max(1, len(levels)))(*levels)
    _check(_lib.rlxpp_seed_states_noalloc(arr if len(levels) else None, len(levels), _ptr(level_of_stream),
                                          _ptr(seeds), n_streams, _ptr(out), _stream(stream)))


def _requests(reqs):
    import numpy as np
    a = np.ascontiguousarray(reqs)
    if a.dtype != request_dtype():
        raise TypeError("requests must use request_dtype()")
    return a, len(a)


def _tuning(t, gen=None):
    """(chunk_blocks, blocks_per_sm[, path[, threads_per_block]]); the path defaults to
    the handle's, the threads per block to the path's default (0)."""
    if t is None:
        return None
    if isinstance(t, RlxppTuning):
        return ctypes.byref(t)
    t = tuple(t)
    if len(t) == 2:  # the handle's path picks the request kernel
        t = t + (rlxpp_get_path(gen) if gen else RLXPP_PATH_TENSOR,)
    if len(t) == 3:
        t = t + (0,)
    return ctypes.byref(RlxppTuning(*t))


def _tuple(t):
    return (t.chunk_blocks, t.blocks_per_sm, t.path, t.threads_per_block)


def rlxpp_plan_requests(gen, reqs, flags=0, tuning=None):
    """Returns a plan handle (int).  reqs: numpy array of request_dtype() (host)."""
    a, n = _requests(reqs)
    h = _vp()
    _check(_lib.rlxpp_plan_requests(gen, a.ctypes.data if n else None, n, flags, _tuning(tuning, gen),
                                    ctypes.byref(h)))
    return h.value


def rlxpp_run_plan(gen, plan, out_u24=None, out_f64=None, stream=None):
    _check(_lib.rlxpp_run_plan(gen, plan, _ptr(out_u24), _ptr(out_f64), _stream(stream)))


def rlxpp_plan_items(plan):
    return int(_lib.rlxpp_plan_items(plan))


def rlxpp_plan_tuning(plan):
    return _tuple(_lib.rlxpp_plan_tuning(plan))


def rlxpp_destroy_plan(plan):
    _lib.rlxpp_destroy_plan(plan)


def rlxpp_draw_requests(gen, reqs, out_u24=None, out_f64=None, flags=0, stream=None):
    a, n = _requests(reqs)
    _check(_lib.rlxpp_draw_requests(gen, a.ctypes.data if n else None, n, _ptr(out_u24), _ptr(out_f64),
                                    flags, _stream(stream)))


def rlxpp_autotune_requests(gen, reqs, out_u24=None, out_f64=None, stream=None):
    """Returns the chosen (chunk_blocks, blocks_per_sm, path, threads_per_block)."""
    a, n = _requests(reqs)
    t = RlxppTuning()
    _check(_lib.rlxpp_autotune_requests(gen, a.ctypes.data if n else None, n, _ptr(out_u24), _ptr(out_f64),
                                        _stream(stream), ctypes.byref(t)))
    return _tuple(t)


def rlxpp_set_path(gen, path):
    _check(_lib.rlxpp_set_path(gen, path))


def rlxpp_get_path(gen):
    return int(_lib.rlxpp_get_path(gen))


def rlxpp_test_tc_mulmod(p, x, out, n, stream=None):
    _check(_lib.rlxpp_test_tc_mulmod(p, _ptr(x), _ptr(out), n, _stream(stream)))


def rlxpp_test_tc_timeout(scratch, stream=None):
    _check(_lib.rlxpp_test_tc_timeout(_ptr(scratch), _stream(stream)))


def rlxpp_luxury_multiplier(p):
    """A = a^p mod m as a Python int (computed on the device)."""
    out = (ctypes.c_uint64 * 9)()
    _check(_lib.rlxpp_luxury_multiplier(p, out))
    return sum(int(out[k]) << (64 * k) for k in range(9))


class Generator:
    """Owns one handle; methods forward to the functions above."""

    def __init__(self, n_streams, levels, seeds, level_of_stream=None, stream=None):
        self.n = n_streams
        self.levels = list(levels)
        self.handle = rlxpp_create(n_streams, self.levels, seeds, level_of_stream, stream)

    def seed(self, seeds, stream=None):
        rlxpp_seed(self.handle, seeds, stream)

    def skip(self, n128, stream=None):
        rlxpp_skip(self.handle, n128, stream)

    def draw_u24(self, out, count_each=0, counts=None, offsets=None, stream=None):
        rlxpp_draw_u24(self.handle, out, count_each, counts, offsets, stream)

    def draw_f64(self, out, count_each=0, counts=None, offsets=None, stream=None):
        rlxpp_draw_f64(self.handle, out, count_each, counts, offsets, stream)

    def set_path(self, path):
        rlxpp_set_path(self.handle, path)

    def draw_requests(self, reqs, out_u24=None, out_f64=None, flags=0, stream=None):
        rlxpp_draw_requests(self.handle, reqs, out_u24, out_f64, flags, stream)

    def draw_f32(self, out, count_each=0, counts=None, offsets=None, stream=None):
        rlxpp_draw_f32(self.handle, out, count_each, counts, offsets, stream)

    def draw_normal_f64(self, out, count_each=0, counts=None, offsets=None, stream=None):
        rlxpp_draw_normal_f64(self.handle, out, count_each, counts, offsets, stream)

    def draw_exp_f64(self, out, count_each=0, counts=None, offsets=None, stream=None):
        rlxpp_draw_exp_f64(self.handle, out, count_each, counts, offsets, stream)

    def draw_raw_f64(self, out, count_each=0, counts=None, offsets=None, stream=None):
        rlxpp_draw_raw_f64(self.handle, out, count_each, counts, offsets, stream)

    def draw_u24_host_async(self, out, count_each, stream=None):
        rlxpp_draw_u24_host_async(self.handle, out, count_each, stream)

    def draw_f64_host_async(self, out, count_each, stream=None):
        rlxpp_draw_f64_host_async(self.handle, out, count_each, stream)

    def host_wait(self, stream=None):
        rlxpp_host_wait(self.handle, stream)

    def skip_values(self, n_values, kind, stream=None):
        rlxpp_skip_values(self.handle, n_values, kind, stream)

    def draw_f64_sum_hist(self, count_each, sums, hist, stream=None):
        rlxpp_draw_f64_sum_hist(self.handle, count_each, sums, hist, stream)

    def get_state(self, dst, stream=None):
        rlxpp_get_state(self.handle, dst, stream)

    def set_state(self, src, stream=None):
        rlxpp_set_state(self.handle, src, stream)

    def sync(self, stream=None):
        rlxpp_sync(self.handle, stream)

    def close(self):
        if self.handle:
            rlxpp_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
