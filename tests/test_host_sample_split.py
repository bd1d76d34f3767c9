"""The lane split's division of a window among a pixel's lanes
(csrc/sample_split.h), on the CPU: lane `sub` of T takes the row-major samples
sub, sub + T, ..., so every sample of a K x K window lands in exactly one lane,
in ascending order, and the lanes' counts differ by at most one. The header is
built with the host compiler through a small ctypes shim.
"""
import ctypes
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2211_16266_gb300", "csrc")
SHIM = os.path.join(ROOT, "tests", "host", "sample_split_shim.cpp")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("split") / "libsample_split.so")
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-Wall", "-Wextra", "-Werror", "-fPIC", "-shared",
                           "-I", CSRC, "-o", so, SHIM])
    L = ctypes.CDLL(so)
    L.ss_lane_samples.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                  ctypes.c_int]
    L.ss_lane_samples.restype = ctypes.c_int
    return L


def lane_samples(L, sub, T, K):
    buf = (ctypes.c_int * (K * K + 1))()
    n = L.ss_lane_samples(sub, T, K, buf, K * K + 1)
    return list(buf[:n])


@pytest.mark.parametrize("T", [2, 4, 8])
def test_every_sample_in_exactly_one_lane(lib, T):
    # windows of 1 to 21 samples a side (dense 21x21 is the largest patch), K < T included
    for K in range(1, 22):
        lanes = [lane_samples(lib, sub, T, K) for sub in range(T)]
        for sub, ms in enumerate(lanes):
            assert ms == list(range(sub, K * K, T)), (K, sub)
        allm = sorted(m for ms in lanes for m in ms)
        assert allm == list(range(K * K)), K
        counts = [len(ms) for ms in lanes]
        assert max(counts) - min(counts) <= 1, (K, counts)


def test_the_split_of_the_benchmarked_window(lib):
    # 11x11 at stride 2: 6 x 6 samples, the centre (3, 3) = 21 in lane 21 % T
    assert [len(lane_samples(lib, s, 2, 6)) for s in range(2)] == [18, 18]
    assert 21 in lane_samples(lib, 1, 2, 6) and 21 in lane_samples(lib, 1, 4, 6)
    assert [len(lane_samples(lib, s, 8, 6)) for s in range(8)] == [5, 5, 5, 5, 4, 4, 4, 4]
