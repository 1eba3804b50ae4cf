"""The oracle's C code under AddressSanitizer and UndefinedBehaviorSanitizer
(host only): a driver runs its step (both schemes), shift, mass transfer
and reconstruction on small grids with odd, single-cell and periodic or
zero-gradient axes, and must finish without a report."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_under_sanitizers(tmp_path):
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no host compiler")
    exe = tmp_path / "oracle_sanitize"
    build = subprocess.run([cc, "-std=c99", "-O1", "-g", "-fno-omit-frame-pointer",
                            "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-ffp-contract=off",
                            os.path.join(ROOT, "oracle", "vof_oracle.c"),
                            os.path.join(ROOT, "tests", "c", "oracle_sanitize.c"), "-lm", "-o", str(exe)],
                           capture_output=True, text=True)
    if build.returncode != 0 and "sanitize" in build.stderr:
        pytest.skip("sanitizer runtime unavailable: " + build.stderr[:200])
    assert build.returncode == 0, build.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1", UBSAN_OPTIONS="print_stacktrace=1")
    run = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=300)
    assert run.returncode == 0, run.stderr[-3000:]
    assert "sanitize driver ok" in run.stdout
