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


@pytest.mark.parametrize("field,value", [
    ("group_lanes", 16), ("group_lanes", 8), ("precision", 7), ("precision", -1),
    ("certify", 2), ("start_rule", 3), ("cost_tc", 5), ("segmentation", 2),
    ("centroid_update", 2), ("pivot_budget", -1), ("tile_budget_mib", -4),
    ("no_prune", 2), ("eps_tol", -1.0), ("eps_tol", float("nan")), ("joint_tol", -1e-9)])
def test_ctx_create_rejects_config_outside_documented_values(lib, field, value):
    """A field outside its documented values is rejected (D2_EINVAL) before
    the device is touched, so this holds on a machine without a GPU."""
    from paper_1302_0435_gb300 import d2
    cfg = d2.D2Config()
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    assert lib.d2_ctx_create(ctypes.byref(h), 0, ctypes.byref(cfg)) == -1 and not h.value


def test_null_arguments_rejected(lib):
    assert lib.d2_sync(None) == -1
    assert lib.d2_ctx_destroy(None) == -1
    assert lib.d2_assign(None, None, None, None, None, None, None) == -1


def test_layout_of_config_structs(tmp_path):
    """The ctypes mirrors of the header's structs have the C compiler's
    size and field offsets (compiled from include/d2.h with gcc)."""
    import shutil
    import subprocess
    from pathlib import Path
    from paper_1302_0435_gb300 import d2
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    structs = {"d2_bags": d2.D2Bags, "d2_config": d2.D2Config, "d2_flows": d2.D2Flows,
               "d2_stats": d2.D2Stats}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "d2.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in py._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = Path(__file__).resolve().parents[1] / "include"
    subprocess.run([gcc, "-I", str(inc), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {" ".join(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln.strip()}
    for cname, py in structs.items():
        assert got[cname + " size"] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[cname + " " + fname] == getattr(py, fname).offset, (cname, fname)


def test_every_called_entry_point_has_a_ctypes_signature():
    """A call without argtypes passes 64-bit pointers and sizes as C int."""
    import re
    from pathlib import Path
    src = (Path(__file__).resolve().parents[1] / "paper_1302_0435_gb300" / "d2.py").read_text()
    called = set(re.findall(r"load\(\)\.(d2_\w+)\(", src))
    declared = set(re.findall(r"lib\.(d2_\w+)\.argtypes", src))
    no_args = {"d2_version"}  # takes no arguments
    assert called - declared - no_args == set()
