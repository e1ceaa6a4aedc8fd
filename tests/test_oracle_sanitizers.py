"""Host sanitizers on the oracle's C routines: oracle/oracle.c built with
AddressSanitizer and UndefinedBehaviorSanitizer together with a driver
(tests/oracle_asan_driver.c) that exercises every exported routine over
periodic and open cells, empty and dense patterns, block sizes 1/4/13, every
op(A)/op(B) combination, upper-only outputs and partial row ranges, and checks
each truncated product against a dense product written independently in the
driver.  A sanitizer report, a failed check or a non-zero exit fails the test.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
FLAGS = ["-std=c11", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
         "-fno-omit-frame-pointer", "-ffp-contract=off"]


def _compile(out, sources):
    return subprocess.run(["gcc", *FLAGS, *sources, "-lm", "-o", out], capture_output=True, text=True)


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    d = tmp_path_factory.mktemp("asan")
    probe = d / "probe.c"
    probe.write_text("int main(void) { return 0; }\n")
    if _compile(str(d / "probe"), [str(probe)]).returncode != 0:
        pytest.skip("this gcc has no AddressSanitizer/UndefinedBehaviorSanitizer runtime")
    exe = d / "oracle_asan_driver"
    r = _compile(str(exe), [os.path.join(ROOT, "oracle", "oracle.c"), os.path.join(HERE, "oracle_asan_driver.c")])
    assert r.returncode == 0, r.stderr
    return str(exe)


def test_oracle_c_is_clean_under_asan_and_ubsan(driver):
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:halt_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    r = subprocess.run([driver], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip() == "ok"
    for marker in ("AddressSanitizer", "LeakSanitizer", "runtime error"):
        assert marker not in r.stderr, r.stderr
