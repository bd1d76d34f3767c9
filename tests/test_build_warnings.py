"""The library's host-side translation units compile warning-free with the host
compiler's -Wall -Wextra (no GPU needed). A use-after-free on the serving
rejection path was found this way."""
import concurrent.futures as cf
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2211_16266_gb300", "csrc")
HOST_TUS = ("pmsp_api", "serving", "batch_api", "cloud_api", "noalloc", "median", "filter", "warp", "cloud")


def test_host_code_is_warning_free(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")

    def build(tu):
        r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                            "--expt-relaxed-constexpr", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                            "-Xcompiler", "-Wall,-Wextra,-Werror", "-c", os.path.join(CSRC, tu + ".cu"),
                            "-o", str(tmp_path / (tu + ".o"))], capture_output=True, text=True)
        return tu, r.returncode, r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(len(HOST_TUS), os.cpu_count() or 1)) as ex:
        for tu, rc, err in ex.map(build, HOST_TUS):
            assert rc == 0, f"{tu}.cu:\n{err[-3000:]}"
