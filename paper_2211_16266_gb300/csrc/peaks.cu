// Measured peaks of the units the densification kernels run on: FP32 FMA
// issue (scalar and packed f32x2), the special-function unit, and texture
// gathers served from L1 and from L2. The cost kernel is bound by plain FP32
// arithmetic and gathers, not by HBM or tensor cores, so its roofline needs
// these figures rather than the copy bandwidth and GEMM throughput.
//
// Each probe is a fixed number of loop iterations per thread (no waits, no
// data-dependent exits), timed with CUDA events on the context's stream after
// one untimed launch; the best of three timed launches is reported.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "pmsp.h"
#include "runtime.h"

namespace pmsp {

namespace {

constexpr int CHAINS = 8;
constexpr int PROBE_THREADS = 256;

// x <- x * a + b on CHAINS independent chains; a < 1 keeps every value finite.
__global__ void __launch_bounds__(PROBE_THREADS) fma_probe(float* sink, float a, float b, int iters) {
    float x[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < CHAINS; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += x[k];
    if (s == 1234.5f) sink[blockIdx.x] = s;  // keeps the chains live; never true for these inputs
}

// The same with packed FP32 (one instruction for two FMAs).
__global__ void __launch_bounds__(PROBE_THREADS) fma2_probe(float* sink, float a, float b, int iters) {
    float2 x[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = make_float2((float)(threadIdx.x + k), (float)(threadIdx.x - k));
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < CHAINS; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += x[k].x + x[k].y;
    if (s == 1234.5f) sink[blockIdx.x] = s;
}

// Special-function unit: reciprocal square roots (rsqrt.approx) on CHAINS
// chains; x -> 1/sqrt(x) stays in (0, inf) and converges to 1.
__global__ void __launch_bounds__(PROBE_THREADS) sfu_probe(float* sink, int iters) {
    float x[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = 1.0f + (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < CHAINS; ++k) asm("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(x[k]));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += x[k];
    if (s == 1234.5f) sink[blockIdx.x] = s;
}

// Texture gathers, four independent fetches per iteration. `scatter` = 0: the
// coordinates walk a small window of the texture (L1-resident); 1: every
// fetch lands on a pseudo-random texel of the whole texture (L1 misses, L2
// hits when the texture fits in L2). Normalised coordinates in [0, 1).
__global__ void __launch_bounds__(PROBE_THREADS) gather_probe(float* sink, cudaTextureObject_t tex, int iters,
                                                             int scatter, float span) {
    unsigned h = blockIdx.x * PROBE_THREADS + threadIdx.x;
    float acc = 0.f;
    float u = (float)(threadIdx.x & 31) * (1.0f / 256.0f), v = (float)(threadIdx.x >> 5) * (1.0f / 256.0f);
    for (int i = 0; i < iters; ++i) {
        float4 g[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float x, y;
            if (scatter) {
                h = h * 1664525u + 1013904223u;  // LCG (Numerical Recipes constants)
                x = (float)(h >> 16) * (1.0f / 65536.0f);
                y = (float)(h & 0xffffu) * (1.0f / 65536.0f);
            } else {
                x = u + (float)k * (1.0f / 1024.0f);
                y = v;
            }
            g[k] = tex2Dgather<float4>(tex, x, y, 0);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) acc += g[k].x + g[k].w;
        if (!scatter) {
            u += span;
            u = u >= 0.25f ? u - 0.25f : u;
        }
    }
    if (acc == -1.0f) sink[blockIdx.x] = acc;
}

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    Timer() {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Timer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// Best of three timed launches (after one untimed), in seconds; < 0 on error.
template <class F>
double best_time(cudaStream_t st, F launch) {
    Timer t;
    launch();
    double best = 1e30;
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(t.a, st);
        launch();
        cudaEventRecord(t.b, st);
        if (cudaEventSynchronize(t.b) != cudaSuccess) return -1.0;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t.a, t.b);
        best = std::min(best, (double)ms * 1e-3);
    }
    return cudaGetLastError() == cudaSuccess ? best : -1.0;
}

int make_u8_texture(int W, int H, cudaArray_t* arr, cudaTextureObject_t* tex) {
    cudaChannelFormatDesc cd = cudaCreateChannelDesc<unsigned char>();
    if (cudaMallocArray(arr, &cd, W, H) != cudaSuccess) return PMSP_ENOMEM;
    std::vector<unsigned char> host((size_t)W * H);  // any contents
    for (size_t i = 0; i < host.size(); ++i) host[i] = (unsigned char)(i * 7 + (i >> 12));
    if (cudaMemcpy2DToArray(*arr, 0, 0, host.data(), W, W, H, cudaMemcpyHostToDevice) != cudaSuccess)
        return PMSP_ECUDA;
    cudaResourceDesc rd;
    memset(&rd, 0, sizeof rd);
    rd.resType = cudaResourceTypeArray;
    rd.res.array.array = *arr;
    cudaTextureDesc td;
    memset(&td, 0, sizeof td);
    td.addressMode[0] = cudaAddressModeWrap;
    td.addressMode[1] = cudaAddressModeClamp;
    td.filterMode = cudaFilterModePoint;
    td.readMode = cudaReadModeNormalizedFloat;
    td.normalizedCoords = 1;
    return cudaCreateTextureObject(tex, &rd, &td, nullptr) == cudaSuccess ? PMSP_OK : PMSP_ECUDA;
}

}  // namespace

}  // namespace pmsp

using namespace pmsp;

extern "C" int pmsp_measure_peaks(pmsp_ctx* c, pmsp_peaks* out) {
    if (!c) return PMSP_EINVAL;
    if (!out) return ctx_fail(c, PMSP_EINVAL, "NULL output");
    if (cudaSetDevice(c->device) != cudaSuccess) return ctx_fail(c, PMSP_ECUDA, "cudaSetDevice failed");
    memset(out, 0, sizeof *out);
    int sms = 0, khz = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, c->device);
    if (sms < 1) return ctx_fail(c, PMSP_ECUDA, "SM count query failed");
    out->sms = sms;
    out->sm_clock_mhz_max = khz / 1000.0;
    const cudaStream_t st = c->stream;
    float* sink = nullptr;
    const int blocks = sms * 8;  // 2048 threads per SM: every FP32 lane has independent work
    if (cudaMalloc(&sink, blocks * sizeof(float)) != cudaSuccess) return ctx_fail(c, PMSP_ENOMEM, "probe sink");
    const double threads = (double)blocks * PROBE_THREADS;

    const int it_fma = 65536;  // x 4 x 8 FMAs per thread
    double t = best_time(st, [&] { fma_probe<<<blocks, PROBE_THREADS, 0, st>>>(sink, 0.999f, 0.001f, it_fma); });
    out->fp32_fma_per_s = t > 0 ? threads * it_fma * 4 * CHAINS / t : 0;
    t = best_time(st, [&] { fma2_probe<<<blocks, PROBE_THREADS, 0, st>>>(sink, 0.999f, 0.001f, it_fma / 2); });
    out->fp32x2_fma_per_s = t > 0 ? threads * (it_fma / 2) * 4 * CHAINS * 2 / t : 0;
    const int it_sfu = 8192;
    t = best_time(st, [&] { sfu_probe<<<blocks, PROBE_THREADS, 0, st>>>(sink, it_sfu); });
    out->sfu_per_s = t > 0 ? threads * it_sfu * 4 * CHAINS / t : 0;

    cudaArray_t small = nullptr, big = nullptr;
    cudaTextureObject_t tsmall = 0, tbig = 0;
    int rc = make_u8_texture(256, 128, &small, &tsmall);
    if (!rc) rc = make_u8_texture(4096, 4096, &big, &tbig);  // 16 MB: L2-resident, far beyond L1
    if (!rc) {
        const int it_g = 16384;  // x 4 gathers per thread
        t = best_time(st, [&] { gather_probe<<<blocks, PROBE_THREADS, 0, st>>>(sink, tsmall, it_g, 0, 1.0f / 512); });
        out->gather_l1_per_s = t > 0 ? threads * it_g * 4 / t : 0;
        t = best_time(st, [&] { gather_probe<<<blocks, PROBE_THREADS, 0, st>>>(sink, tbig, it_g / 4, 1, 0.f); });
        out->gather_l2_per_s = t > 0 ? threads * (it_g / 4) * 4 / t : 0;
    }
    if (tsmall) cudaDestroyTextureObject(tsmall);
    if (tbig) cudaDestroyTextureObject(tbig);
    if (small) cudaFreeArray(small);
    if (big) cudaFreeArray(big);
    cudaStreamSynchronize(st);
    cudaFree(sink);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "peak probes");
    if (rc) return ctx_fail(c, rc, "probe texture");
    if (!(out->fp32_fma_per_s > 0 && out->fp32x2_fma_per_s > 0 && out->sfu_per_s > 0 && out->gather_l1_per_s > 0 &&
          out->gather_l2_per_s > 0))
        return ctx_fail(c, PMSP_ECUDA, "a peak probe failed to run");
    return PMSP_OK;
}
