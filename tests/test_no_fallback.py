"""The product path has no CPU fallback: without a GPU the library still
loads (so its absence is not mistaken for a missing GPU), creating a
context fails with D2_ECUDA, and a missing library raises instead of
degrading.  Host-side marshalling of bag batches is checked too."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1302_0435_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def d2():
    from paper_1302_0435_gb300 import build, d2 as mod
    build.build()
    mod.load()
    return mod


def test_context_fails_loudly_without_a_gpu(d2):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(d2.D2Error) as e:
        d2.Context(0)
    assert e.value.code == d2.D2_ECUDA


def test_missing_library_raises():
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_1302_0435_gb300 import d2\n"
            "try:\n    d2.load('/nonexistent/libd2.so')\nexcept OSError:\n    sys.exit(7)\n"
            "sys.exit(0)\n") % ROOT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 7, r.stderr[-1000:]


def test_host_bag_marshalling(d2):
    objs, _ = synth.image_like(N=12, K=2, seed=3)
    b = d2.bags_from_synth(objs)
    assert b.s.count == objs.count and b.s.dim == objs.dim
    assert b.s.loc == b.loc.ctypes.data and b.s.w == b.w.ctypes.data
    assert b.s.off == b.off.ctypes.data
    assert np.array_equal(np.asarray(b.off), np.asarray(objs.off, dtype=np.int64))
    assert b.loc.flags["C_CONTIGUOUS"] and b.w.flags["C_CONTIGUOUS"]
