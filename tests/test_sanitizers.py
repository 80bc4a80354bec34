"""The oracle and the C ABI's host-side paths under AddressSanitizer and
UndefinedBehaviorSanitizer, and the multi-threaded oracle under
ThreadSanitizer (CPU only): tests/sanitize_driver.c is built with the
sanitizers against oracle/vegas_oracle.c (and, for ASan/UBSan, the CUDA
library) and must exit 0 with no sanitizer report."""
import os
import shutil
import subprocess

import pytest

from paper_2002_12921_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_host_code_is_clean_under_asan_and_ubsan(tmp_path):
    lib = build.build()
    exe = str(tmp_path / "sanitize_driver")
    cmd = ["gcc", "-std=c11", "-D_GNU_SOURCE", "-g", "-O1", "-fno-omit-frame-pointer",
           "-ffp-contract=off", "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
           "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "sanitize_driver.c"),
           os.path.join(ROOT, "oracle", "vegas_oracle.c"),
           "-L", os.path.dirname(lib), "-l:" + os.path.basename(lib),
           "-Wl,-rpath," + os.path.dirname(lib), "-lm", "-lpthread", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ)
    # the CUDA runtime maps memory where ASan keeps its shadow gap; leaks of the
    # runtime's process-lifetime allocations are not ours to report
    env["ASAN_OPTIONS"] = "protect_shadow_gap=0:detect_leaks=0:abort_on_error=0"
    env["UBSAN_OPTIONS"] = "print_stacktrace=1:halt_on_error=1"
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "runtime error" not in r.stderr and "AddressSanitizer" not in r.stderr, r.stderr
    assert "sanitized host paths: ok" in r.stdout


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_threaded_oracle_is_race_free_under_tsan(tmp_path):
    exe = str(tmp_path / "sanitize_driver_tsan")
    cmd = ["gcc", "-std=c11", "-D_GNU_SOURCE", "-DORACLE_ONLY", "-g", "-O1",
           "-ffp-contract=off", "-fsanitize=thread", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "sanitize_driver.c"),
           os.path.join(ROOT, "oracle", "vegas_oracle.c"), "-lm", "-lpthread", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, TSAN_OPTIONS="halt_on_error=1")
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "ThreadSanitizer" not in r.stderr, r.stderr
    assert "sanitized host paths: ok" in r.stdout
