"""Resource use of the benchmarked kernel instances, as ptxas reports it (no GPU).

The 6-view half-sweep keeps 7 blocks of 128 threads per SM only within 72
registers a thread; a change that needs more would either lower occupancy or
spill more. This builds the 6-view translation unit for sm_103a with
`-Xptxas -v` and checks registers, spills and shared memory of every pixel
kernel instance in it against the budget the measured configuration used.
"""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2211_16266_gb300", "csrc")


def _report(tu, tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                        "--expt-relaxed-constexpr", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-Xptxas", "-v",
                        "-c", os.path.join(CSRC, tu), "-o", str(tmp_path / "k.o")],
                       capture_output=True, text=True, check=True)
    out, cur = {}, None
    for line in r.stderr.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            cur = m.group(1)
            out[cur] = {}
            continue
        if cur is None:
            continue
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m:
            out[cur]["spill"] = int(m.group(1)) + int(m.group(2))
        m = re.search(r"Used (\d+) registers.*?(\d+) bytes smem", line)
        if m:
            out[cur]["regs"], out[cur]["smem"] = int(m.group(1)), int(m.group(2))
    return out


def test_six_view_instances_stay_within_the_measured_budget(tmp_path):
    rep = _report("kernels_s6.cu", tmp_path)
    pixel = {k: v for k, v in rep.items() if "pixel_kernel" in k}
    assert len(pixel) >= 9, sorted(rep)
    for name, v in pixel.items():
        assert v["regs"] <= 72, (name, v)              # 7 blocks x 128 threads per SM
        # at most 292 B of spill stores + loads in the measured build: issuing each view
        # pair's gathers right after its coordinates spills a few more values and
        # measured 1.5 % faster than without
        assert v["spill"] <= 300, (name, v)
        assert v["smem"] * 7 <= 228 * 1024, (name, v)  # 7 blocks fit the SM's shared memory
