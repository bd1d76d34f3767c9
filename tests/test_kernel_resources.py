"""Resource use of the benchmarked kernel instances, as ptxas reports it (no GPU).

The 6- and 8-view half-sweeps run 4 blocks of 128 threads per SM within 128
registers a thread and without spills (measured faster than 5-7 blocks with
spills); the thread-split kernels keep 8 blocks within 64 registers, and the
lane-split kernels (2, 4 or 8 lanes per pixel, every lane holding all views'
sums) the one-thread budget, spill-free. This
builds those translation units for sm_103a with `-Xptxas -v` and checks
registers, spills and shared memory of every pixel kernel instance in them
against the budget the measured configuration used.
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


@pytest.mark.parametrize("tu", ["kernels_s6.cu", "kernels_s8.cu"])
def test_pixel_instances_stay_within_the_measured_budget(tu, tmp_path):
    rep = _report(tu, tmp_path)
    pixel = {k: v for k, v in rep.items() if "pixel_kernel" in k}
    split = {k: v for k, v in rep.items() if "pixel_split_kernel" in k}
    lanes = {k: v for k, v in rep.items() if "pixel_lanes_kernel" in k}
    assert len(pixel) >= 9 and len(split) == 4 and len(lanes) == 6, sorted(rep)
    for name, v in pixel.items():
        assert v["regs"] <= 128, (name, v)             # 4 blocks x 128 threads per SM
        assert v["spill"] == 0, (name, v)
        assert v["smem"] * 4 <= 228 * 1024, (name, v)
    for name, v in split.items():
        assert v["regs"] <= 64, (name, v)              # 8 blocks x 128 threads per SM
        assert v["smem"] * 8 <= 228 * 1024, (name, v)
    for name, v in lanes.items():
        assert v["regs"] <= 128, (name, v)             # 4 blocks x 128 threads per SM
        assert v["spill"] == 0, (name, v)
        assert v["smem"] * 4 <= 228 * 1024, (name, v)
