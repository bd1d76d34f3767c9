// How the lane-split half-sweep divides a window's samples among the T lanes
// of a pixel (pixel_lanes.cuh). Plain C++ without CUDA types, so the host
// tests build and exercise it.
#pragma once

#ifndef PMSP_HD
#ifdef __CUDACC__
#define PMSP_HD __host__ __device__ __forceinline__
#else
#define PMSP_HD inline
#endif
#endif

namespace pmsp {

// Lane `sub` of T takes the samples m = sub, sub + T, sub + 2T, ... of a K x K
// window in row-major order, m = a K + b; the walk ends when a reaches K. Every
// sample belongs to exactly one lane, and the lanes' counts differ by at most
// one. The first sample is (a, b) = divmod(sub, K), and each step adds T to b
// and carries whole rows into a (no division per step).
PMSP_HD void split_first_sample(int sub, int K, int& a, int& b) {
    a = 0;
    b = sub;
    while (b >= K) {
        b -= K;
        ++a;
    }
}

PMSP_HD void split_next_sample(int T, int K, int& a, int& b) {
    b += T;
    while (b >= K) {
        b -= K;
        ++a;
    }
}

}  // namespace pmsp
