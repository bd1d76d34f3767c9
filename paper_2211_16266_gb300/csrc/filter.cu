// Geometric-consistency filter kernel and the standalone camera-model kernels
// (bilinear fetch, projection) behind pmsp_sample_bilinear and pmsp_project.
//
// Paper Sec. III: once five depth maps are available the current one is
// checked against its neighbours' depth maps and outliers are removed. A
// reference pixel with range d is lifted to 3-D, projected into neighbour j,
// the range stored at the nearest pixel there is lifted back and reprojected
// into the reference; the view agrees if the reprojection error (longitude
// difference wrapped to half a panorama) is below max_px. The pixel keeps
// its range when at least min_views views agree. FP32, one thread per pixel.
#include "camera.cuh"
#include "common.cuh"

namespace pmsp {

__device__ __forceinline__ float3 apply(const float* R, const float* t, float3 X) {
    return make_float3(fmaf(R[0], X.x, fmaf(R[1], X.y, fmaf(R[2], X.z, t[0]))),
                       fmaf(R[3], X.x, fmaf(R[4], X.y, fmaf(R[5], X.z, t[1]))),
                       fmaf(R[6], X.x, fmaf(R[7], X.y, fmaf(R[8], X.z, t[2]))));
}

__global__ void __launch_bounds__(256) filter_kernel(const __grid_constant__ FilterParams P) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= P.W || y >= P.H) return;
    const size_t i = (size_t)y * P.W + x;
    const float d = P.depth_in[i];
    int cnt = 0;
    if (d > 0.f) {
        const float3 rp = pixel_bearing(x, y, P.W, P.H);
        const float3 X = make_float3(d * rp.x, d * rp.y, d * rp.z);
        const float su = P.W * 0.15915494309189535f, ou = 0.5f * P.W - 0.5f;
        const float sv = -P.H * 0.3183098861837907f, ov = 0.5f * P.H - 0.5f;
        for (int j = 0; j < P.n; ++j) {
            const FilterView& V = P.nb[j];
            const float3 Y = apply(V.Rf, V.tf, X);
            float uc, vc;
            project_dir_fast(Y.x, Y.y, Y.z, V.W * 0.15915494309189535f, 0.5f * V.W - 0.5f,
                        -V.H * 0.3183098861837907f, 0.5f * V.H - 0.5f, uc, vc);
            const int ui = wrap_index((int)floorf(uc + 0.5f), V.W);
            const int vi = clamp_index((int)floorf(vc + 0.5f), V.H - 1);
            const float dj = V.depth[(size_t)vi * V.W + ui];
            if (!(dj > 0.f)) continue;
            const float3 rq = pixel_bearing(ui, vi, V.W, V.H);
            const float3 Z = apply(V.Rb, V.tb, make_float3(dj * rq.x, dj * rq.y, dj * rq.z));
            float u2, v2;
            project_dir_fast(Z.x, Z.y, Z.z, su, ou, sv, ov, u2, v2);
            float du = u2 - (float)x;
            du -= P.W * floorf(du / P.W + 0.5f);
            const float dv = v2 - (float)y;
            if (sqrtf(du * du + dv * dv) < P.max_px) ++cnt;
        }
    }
    P.depth_out[i] = (d > 0.f && cnt >= P.min_views) ? d : 0.f;
    if (P.agree) P.agree[i] = cnt;
}

cudaError_t launch_filter_kernel(const FilterParams& p, cudaStream_t stream) {
    const dim3 grid((p.W + 255) / 256, p.H);
    filter_kernel<<<grid, 256, 0, stream>>>(p);
    return cudaGetLastError();
}

__global__ void sample_kernel(cudaTextureObject_t tex, float inv_w, float inv_h, int n, const float* uc,
                              const float* vc, float* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = sample_bilinear(tex, inv_w, inv_h, uc[i], vc[i]);
}

cudaError_t launch_sample_kernel(cudaTextureObject_t tex, int W, int H, int n, const float* uc,
                                 const float* vc, float* out, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    sample_kernel<<<(n + 255) / 256, 256, 0, stream>>>(tex, 1.0f / W, 1.0f / H, n, uc, vc, out);
    return cudaGetLastError();
}

__global__ void project_kernel(int n, const float* dirs, float su, float ou, float sv, float ov, float* uc,
                               float* vc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) project_dir_fast(dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], su, ou, sv, ov, uc[i], vc[i]);
}

cudaError_t launch_project_kernel(int W, int H, int n, const float* dirs, float* uc, float* vc,
                                  cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    project_kernel<<<(n + 255) / 256, 256, 0, stream>>>(n, dirs, W * 0.15915494309189535f, 0.5f * W - 0.5f,
                                                        -H * 0.3183098861837907f, 0.5f * H - 0.5f, uc, vc);
    return cudaGetLastError();
}

}  // namespace pmsp
