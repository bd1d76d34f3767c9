// C entry points over csrc/sample_split.h for the CPU tests (ctypes).
#include "sample_split.h"

extern "C" {

// Writes lane `sub`'s samples (row-major indices a * K + b) into out (at most
// cap of them) and returns how many there are.
int ss_lane_samples(int sub, int T, int K, int* out, int cap) {
    int a, b, n = 0;
    for (pmsp::split_first_sample(sub, K, a, b); a < K; pmsp::split_next_sample(T, K, a, b)) {
        if (n < cap) out[n] = a * K + b;
        ++n;
    }
    return n;
}

}  // extern "C"
