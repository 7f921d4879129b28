"""Host sanitizers on the FP64 oracle: the C solver built with
AddressSanitizer + UndefinedBehaviorSanitizer, and with ThreadSanitizer for
its thread pool, runs a driver that certifies every result (feasibility,
dual feasibility, zero gap, thread-count independence)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _run(tmp_path, flags, name):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    exe = str(tmp_path / name)
    cmd = ["gcc", "-O1", "-g", "-std=c11", "-ffp-contract=off", "-fno-omit-frame-pointer"] + flags + [
        os.path.join(ROOT, "oracle", "d2_oracle.c"), os.path.join(HERE, "oracle_sanitize_driver.c"),
        "-o", exe, "-lm", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("sanitizer build unavailable: " + r.stderr.strip().splitlines()[-1][:200])
    env = dict(os.environ, UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1",
               ASAN_OPTIONS="detect_leaks=1", TSAN_OPTIONS="halt_on_error=1")
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "0 failures" in r.stdout


def test_oracle_under_asan_ubsan(tmp_path):
    _run(tmp_path, ["-fsanitize=address,undefined", "-fno-sanitize-recover=undefined"], "asan")


def test_oracle_under_tsan(tmp_path):
    _run(tmp_path, ["-fsanitize=thread"], "tsan")
