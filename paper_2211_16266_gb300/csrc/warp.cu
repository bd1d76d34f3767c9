// Plane-map warping initialisation (paper Sec. III-B: the optimised plane
// map of the preceding keyframe initialises the current one, after Shen 2013).
//
// Splat: every previous pixel with a range lifts its plane point into the
// current camera and claims the nearest current pixel with a 64-bit atomic
// minimum of (range bits, previous pixel index): the nearest surface wins and
// equal ranges resolve to the smaller index, so the result does not depend on
// thread order. Resolve: a claimed pixel re-intersects the winning plane with
// its own ray; unclaimed pixels, and planes that are grazing, behind or
// outside [d_min, d_max] there, take the ordinary random initial plane. The
// initial costs are then computed by the cost kernel.
#include "pixel_kernel.cuh"

namespace pmsp {

namespace {

__device__ __forceinline__ float3 rigid(const WarpArgs& A, float3 X) {
    return make_float3(fmaf(A.R[0], X.x, fmaf(A.R[1], X.y, fmaf(A.R[2], X.z, A.t[0]))),
                       fmaf(A.R[3], X.x, fmaf(A.R[4], X.y, fmaf(A.R[5], X.z, A.t[1]))),
                       fmaf(A.R[6], X.x, fmaf(A.R[7], X.y, fmaf(A.R[8], X.z, A.t[2]))));
}

__global__ void warp_splat_kernel(const __grid_constant__ WarpArgs A) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y;
    if (u >= A.Wp || v >= A.Hp) return;
    const size_t j = (size_t)v * A.Wp + u;
    const float d = A.prev_depth[j];
    if (!(d > 0.f)) return;
    const float3 r = pixel_bearing(u, v, A.Wp, A.Hp);
    const float3 Y = rigid(A, make_float3(d * r.x, d * r.y, d * r.z));
    float uc, vc;
    project_dir_fast(Y.x, Y.y, Y.z, A.su, A.ou, A.sv, A.ov, uc, vc);
    const int qu = wrap_index((int)floorf(uc + 0.5f), A.W);
    const int qv = clamp_index((int)floorf(vc + 0.5f), A.H - 1);
    const float range = sqrtf(fmaf(Y.x, Y.x, fmaf(Y.y, Y.y, Y.z * Y.z)));
    const unsigned long long key = ((unsigned long long)__float_as_uint(range) << 32) | (unsigned long long)j;
    atomicMin(A.zbuf + (size_t)qv * A.W + qu, key);
}

__global__ void warp_resolve_kernel(const __grid_constant__ PixelParams P, const __grid_constant__ WarpArgs A) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y;
    if (u >= P.W || v >= P.H) return;
    const size_t i = (size_t)v * P.W + u;
    const float3 rp = pixel_bearing(u, v, P.W, P.H);
    const unsigned long long key = A.zbuf[i];
    float d = 0.f;
    float3 n = make_float3(0.f, 0.f, 0.f);
    bool used = false;
    if (key != ~0ull) {
        const size_t j = (size_t)(key & 0xffffffffull);
        const int ju = (int)(j % A.Wp), jv = (int)(j / A.Wp);
        const float dj = A.prev_depth[j];
        const float3 r = pixel_bearing(ju, jv, A.Wp, A.Hp);
        const float3 Y = rigid(A, make_float3(dj * r.x, dj * r.y, dj * r.z));
        const size_t Np = (size_t)A.Wp * A.Hp;
        const float3 nj = make_float3(A.prev_normal[j], A.prev_normal[Np + j], A.prev_normal[2 * Np + j]);
        n = make_float3(fmaf(A.R[0], nj.x, fmaf(A.R[1], nj.y, A.R[2] * nj.z)),
                        fmaf(A.R[3], nj.x, fmaf(A.R[4], nj.y, A.R[5] * nj.z)),
                        fmaf(A.R[6], nj.x, fmaf(A.R[7], nj.y, A.R[8] * nj.z)));
        const float den = n.x * rp.x + n.y * rp.y + n.z * rp.z;
        if (den < -1e-6f) {
            d = (n.x * Y.x + n.y * Y.y + n.z * Y.z) / den;
            used = d >= P.d_min && d <= P.d_max;
        }
    }
    if (!used) random_plane(P, i, rp, d, n);
    P.depth[i] = d;
    P.nx[i] = n.x;
    P.ny[i] = n.y;
    P.nz[i] = n.z;
    if (A.src) A.src[i] = used ? (int)(key & 0xffffffffull) : -1;
}

}  // namespace

cudaError_t launch_warp_init(const PixelParams& p, const WarpArgs& a, cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(a.zbuf, 0xff, (size_t)a.W * a.H * sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
    warp_splat_kernel<<<dim3((a.Wp + 127) / 128, a.Hp), 128, 0, stream>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    warp_resolve_kernel<<<dim3((p.W + 127) / 128, p.H), 128, 0, stream>>>(p, a);
    return cudaGetLastError();
}

}  // namespace pmsp
