"""The C-ABI library builds for sm_103a, loads on a machine without a GPU,
exports every call include/d2.h declares, and fails cleanly (no crash, a
status code) when no device is usable.  No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "d2.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(d2_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1302_0435_gb300 import build
    try:
        build.build()
    except RuntimeError as e:  # pragma: no cover - no nvcc
        pytest.skip(str(e))
    return ctypes.CDLL(build.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_1302_0435_gb300 import d2
    assert sorted(d2.EXPORTS) == _declared()


def test_strerror_and_version(lib):
    lib.d2_strerror.restype = ctypes.c_char_p
    lib.d2_version.restype = ctypes.c_char_p
    assert lib.d2_strerror(0) == b"ok"
    assert b"invalid" in lib.d2_strerror(-1)
    assert b"sm_103a" in lib.d2_version()


def test_ctx_create_without_gpu_returns_status(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.d2_ctx_create(ctypes.byref(h), 0, None)
    assert rc == -5 and not h.value  # D2_ECUDA


def test_null_arguments_rejected(lib):
    assert lib.d2_sync(None) == -1
    assert lib.d2_ctx_destroy(None) == -1
    assert lib.d2_assign(None, None, None, None, None, None, None) == -1


def test_layout_of_config_structs():
    from paper_1302_0435_gb300 import d2
    assert ctypes.sizeof(d2.D2Bags) == 48
    assert ctypes.sizeof(d2.D2Config) == 56
    assert ctypes.sizeof(d2.D2Flows) == 24


def test_every_called_entry_point_has_a_ctypes_signature():
    """A call without argtypes passes 64-bit pointers and sizes as C int."""
    import re
    from pathlib import Path
    src = (Path(__file__).resolve().parents[1] / "paper_1302_0435_gb300" / "d2.py").read_text()
    called = set(re.findall(r"load\(\)\.(d2_\w+)\(", src))
    declared = set(re.findall(r"lib\.(d2_\w+)\.argtypes", src))
    no_args = {"d2_version"}  # takes no arguments
    assert called - declared - no_args == set()
