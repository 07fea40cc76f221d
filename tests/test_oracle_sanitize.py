"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer (CPU).

A driver (tests/oracle_sanitize_main.cpp) runs the oracle's C interface
through propagation with and without symmetry merging (Z_n, S_n, D_n, torus),
per-gate and per-layer noise, truncation, canonical keys, overlaps, batched
rows, and one- and two-word strings.  Built with both sanitizers and
-fno-sanitize-recover, any invalid access or undefined behaviour ends the
run with a non-zero status; the values it prints must equal those of the
same driver built without instrumentation."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SOURCES = [os.path.join(ROOT, "oracle", "oracle.cpp"), os.path.join(HERE, "oracle_sanitize_main.cpp")]


def build(out, sanitize):
    flags = ["-O1", "-g", "-std=c++17", "-ffp-contract=off"]
    if sanitize:
        flags += ["-fsanitize=address,undefined", "-fno-sanitize-recover=all",
                  "-fno-omit-frame-pointer"]
    r = subprocess.run(["g++", *flags, *SOURCES, "-o", out], capture_output=True, text=True)
    return r.returncode == 0, r.stderr


def test_oracle_is_clean_under_sanitizers(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    san, plain = str(tmp_path / "orc_san"), str(tmp_path / "orc_plain")
    ok, err = build(san, True)
    if not ok:
        pytest.skip("g++ without sanitizer runtimes: " + err.strip()[-200:])
    ok, err = build(plain, False)
    assert ok, err
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1")
    rs = subprocess.run([san], capture_output=True, text=True, env=env, timeout=600)
    assert rs.returncode == 0, rs.stderr[-4000:]
    assert "runtime error" not in rs.stderr and "AddressSanitizer" not in rs.stderr
    rp = subprocess.run([plain], capture_output=True, text=True, timeout=600)
    assert rp.returncode == 0
    got, want = rs.stdout.split(), rp.stdout.split()
    assert len(want) == 9 and got == want
