"""The C ABI without a GPU: the library builds for sm_103a, loads, and exports every
entry point include/rlxpp.h declares; the Python binding mirrors them by name and
layout.  No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rlxpp.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rlxpp_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2106_02504_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rlxpp_create", "rlxpp_skip", "rlxpp_draw_u24", "rlxpp_draw_f64",
                     "rlxpp_destroy", "rlxpp_get_state", "rlxpp_set_state", "rlxpp_sync"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_mirrors_header(lib_path):
    from paper_2106_02504_gb300 import _rlxpp as B
    for name in declared_functions():
        assert callable(getattr(B, name, None)), name
    assert B.STATE_BYTES == 88
    text = open(HEADER).read()
    assert int(re.search(r"#define RLXPP_MAX_LEVELS (\d+)", text).group(1)) == B.RLXPP_MAX_LEVELS
    for code, name in enumerate(["RLXPP_OK", "RLXPP_ERR_INVALID", "RLXPP_ERR_NOMEM", "RLXPP_ERR_CUDA",
                                 "RLXPP_ERR_TIMEOUT", "RLXPP_ERR_UNSUPPORTED"]):
        assert re.search(rf"{name} = {code}\b", text), name
        assert getattr(B, name) == code


def test_library_is_built_for_sm_103a(lib_path):
    from paper_2106_02504_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_no_error_before_any_call(lib_path):
    from paper_2106_02504_gb300 import _rlxpp as B
    assert B.rlxpp_last_error() == ""
    assert B.rlxpp_num_streams(None) == 0


def test_argument_errors_need_no_gpu(lib_path):
    """Host-side argument checks return before any CUDA call."""
    from paper_2106_02504_gb300 import _rlxpp as B
    with pytest.raises(B.RlxppError) as e:
        B.rlxpp_create(4, [], None)
    assert e.value.status == B.RLXPP_ERR_INVALID
    with pytest.raises(B.RlxppError):
        B.rlxpp_create(4, [0], None)
    with pytest.raises(B.RlxppError):
        B.rlxpp_create(4, [2048] * 17, None)
    with pytest.raises(B.RlxppError):
        B.rlxpp_create(4, [2048], None)          # seeds missing
    with pytest.raises(B.RlxppError):
        B.rlxpp_draw_f64(None, None, 1)          # null handle
    with pytest.raises(B.RlxppError):
        B.rlxpp_luxury_multiplier(0)


@pytest.mark.parametrize("level", ["0", "1"])
def test_log_level_reports_argument_errors(lib_path, level):
    """RLXPP_LOG=1 writes each failure (here argument errors, which return before any CUDA
    call) with its status to stderr; unset or 0 keeps the library silent."""
    import subprocess
    import sys
    code = (
        "import ctypes, sys\n"
        f"L = ctypes.CDLL({lib_path!r})\n"
        "L.rlxpp_create.argtypes = [ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,\n"
        "                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]\n"
        "h = ctypes.c_void_p()\n"
        "s = L.rlxpp_create(1, None, 0, None, None, None, ctypes.byref(h))\n"
        "L.rlxpp_last_error.restype = ctypes.c_char_p\n"
        "print(s, L.rlxpp_last_error().decode())\n")
    env = dict(os.environ, RLXPP_LOG=level)
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=120)
    assert p.returncode == 0, p.stderr
    status, msg = p.stdout.split(" ", 1)
    assert int(status) == 1 and "luxury levels" in msg           # RLXPP_ERR_INVALID
    if level == "1":
        assert "rlxpp: error 1: " in p.stderr and "luxury levels" in p.stderr
    else:
        assert "rlxpp:" not in p.stderr
