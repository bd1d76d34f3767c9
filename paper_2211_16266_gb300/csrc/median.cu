// Median post-filter of a depth map (paper Sec. III-C, item 2: a median
// filter runs over a copy of the depth image and ranges that deviate from the
// filtered copy by more than a threshold are removed).
//
// For a pixel with range d > 0, the valid ranges (> 0) of its (2R+1)^2
// window (columns wrapped at the seam, rows outside the panorama left out)
// are sorted and the lower median m, the element of rank floor((n-1)/2), is
// taken; d is removed when |d - m| > tau * m in FP32. Every decision reads the
// unfiltered input, so the output buffer must not alias it.
//
// One thread per pixel, a 32x8 tile plus its halo staged in shared memory.
// The window goes into registers with invalid entries as +inf, is sorted by
// Batcher's odd-even merge network (fixed compare-exchange sequence, fully
// unrolled, so the values never leave registers) and the median is picked by
// rank. Selection is exact: the result equals a plain sort bit for bit.
#include "common.cuh"

namespace pmsp {

namespace {

constexpr int MT_W = 32, MT_H = 8;

constexpr int pow2_at_least(int n) {
    int p = 1;
    while (p < n) p <<= 1;
    return p;
}

// Batcher's odd-even merge sort network on N = 2^m keys: the compare-exchange
// pairs in order, built at compile time so every register index is a constant.
template <int N>
struct MergeNetwork {
    static constexpr int size() {
        int c = 0;
        for (int p = 1; p < N; p <<= 1)
            for (int k = p; k >= 1; k >>= 1)
                for (int j = k % p; j + k < N; j += 2 * k)
                    for (int i = 0; i < k && i + j + k < N; ++i)
                        if ((i + j) / (2 * p) == (i + j + k) / (2 * p)) ++c;
        return c;
    }
    int lo[size()], hi[size()];
    constexpr MergeNetwork() : lo(), hi() {
        int c = 0;
        for (int p = 1; p < N; p <<= 1)
            for (int k = p; k >= 1; k >>= 1)
                for (int j = k % p; j + k < N; j += 2 * k)
                    for (int i = 0; i < k && i + j + k < N; ++i)
                        if ((i + j) / (2 * p) == (i + j + k) / (2 * p)) {
                            lo[c] = i + j;
                            hi[c] = i + j + k;
                            ++c;
                        }
    }
};

template <int N>
__device__ __forceinline__ void odd_even_merge_sort(float (&a)[N]) {
    constexpr MergeNetwork<N> net{};
#pragma unroll
    for (int c = 0; c < MergeNetwork<N>::size(); ++c) {
        const float x = a[net.lo[c]], y = a[net.hi[c]];
        a[net.lo[c]] = fminf(x, y);
        a[net.hi[c]] = fmaxf(x, y);
    }
}

template <int R>
__global__ void __launch_bounds__(MT_W * MT_H) median_kernel(const float* __restrict__ in, float* __restrict__ out,
                                                           int W, int H, float tau) {
    constexpr int SW = MT_W + 2 * R, SH = MT_H + 2 * R;
    constexpr int K = (2 * R + 1) * (2 * R + 1);
    constexpr int N = pow2_at_least(K);
    __shared__ float tile[SH * SW];
    const int x0 = blockIdx.x * MT_W, y0 = blockIdx.y * MT_H;
    const int tid = threadIdx.y * MT_W + threadIdx.x;
    for (int k = tid; k < SH * SW; k += MT_W * MT_H) {
        const int sy = k / SW, sx = k - sy * SW;
        const int y = y0 + sy - R;
        int x = (x0 + sx - R) % W;
        if (x < 0) x += W;
        tile[k] = (y >= 0 && y < H) ? in[(size_t)y * W + x] : 0.f;  // rows outside: no value
    }
    __syncthreads();
    const int u = x0 + threadIdx.x, v = y0 + threadIdx.y;
    if (u >= W || v >= H) return;
    const float d = tile[(threadIdx.y + R) * SW + threadIdx.x + R];
    const size_t i = (size_t)v * W + u;
    if (!(d > 0.f)) {
        out[i] = 0.f;
        return;
    }
    float a[N];
    int n = 0;
#pragma unroll
    for (int dy = 0; dy <= 2 * R; ++dy)
#pragma unroll
        for (int dx = 0; dx <= 2 * R; ++dx) {
            const float x = tile[(threadIdx.y + dy) * SW + threadIdx.x + dx];
            const bool ok = x > 0.f;
            a[dy * (2 * R + 1) + dx] = ok ? x : __int_as_float(0x7f800000);
            n += ok;
        }
#pragma unroll
    for (int k = K; k < N; ++k) a[k] = __int_as_float(0x7f800000);
    odd_even_merge_sort<N>(a);
    const int rank = (n - 1) >> 1;
    float m = a[0];
#pragma unroll
    for (int k = 1; k < K; ++k)
        if (k == rank) m = a[k];
    const float diff = fabsf(__fsub_rn(d, m)), lim = __fmul_rn(tau, m);
    out[i] = diff > lim ? 0.f : d;
}

}  // namespace

cudaError_t launch_median_kernel(const float* in, float* out, int W, int H, int radius, float tau,
                                 cudaStream_t stream) {
    const dim3 block(MT_W, MT_H), grid((W + MT_W - 1) / MT_W, (H + MT_H - 1) / MT_H);
    switch (radius) {
        case 1: median_kernel<1><<<grid, block, 0, stream>>>(in, out, W, H, tau); break;
        case 2: median_kernel<2><<<grid, block, 0, stream>>>(in, out, W, H, tau); break;
        case 3: median_kernel<3><<<grid, block, 0, stream>>>(in, out, W, H, tau); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pmsp
