"""The oracle's pins pass against a build of oracle.c with AddressSanitizer and
UndefinedBehaviorSanitizer: no out-of-bounds access, use after free, signed
overflow or other undefined behaviour anywhere the pins reach (any report
aborts the run). The sanitizer runtime is preloaded into a child interpreter."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_MODULES = ["tests/test_oracle_camera.py", "tests/test_oracle_rng.py", "tests/test_oracle_cost.py",
               "tests/test_oracle_patchmatch.py", "tests/test_oracle_filter.py", "tests/test_oracle_warp.py",
               "tests/test_oracle_median.py", "tests/test_oracle_view.py", "tests/test_oracle_fusion.py"]


def test_pins_pass_under_address_and_ub_sanitizers(tmp_path):
    asan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not os.path.isabs(asan) or not os.path.exists(asan):
        pytest.skip("no AddressSanitizer runtime")
    lib = tmp_path / "liboracle_sanitized.so"
    subprocess.check_call(["gcc", "-O1", "-g", "-fopenmp", "-fPIC", "-shared", "-fsanitize=address,undefined",
                           "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", "-o", str(lib),
                           os.path.join(ROOT, "oracle", "oracle.c"), "-lm"])
    env = dict(os.environ, PMSP_ORACLE_LIB=str(lib), LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        *PIN_MODULES], cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
