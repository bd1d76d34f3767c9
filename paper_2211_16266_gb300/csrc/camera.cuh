// Equirectangular camera model and source fetch on the device (FP32).
//
// Paper Sec. III-C: the patch is rectangular in the reference panorama and
// takes an arbitrary shape in the sources because of the equirectangular
// projection. Convention: pixel (u, v) of a W x H panorama looks along
// lon = 2*pi*(u+0.5)/W - pi, lat = pi/2 - pi*(v+0.5)/H; bearing
// (cos lat sin lon, -sin lat, cos lat cos lon) with x right, y down, z forward.
#pragma once

#include <cuda_runtime.h>

namespace pmsp {

// Unit bearing of pixel centre (u, v). sincospif keeps the angle exact up to
// the rounding of its argument.
__device__ __forceinline__ float3 pixel_bearing(int u, int v, int W, int H) {
    float sl, cl, sn, cn;
    sincospif(0.5f - (2.0f * v + 1.0f) / (2.0f * H), &sl, &cl);
    sincospif((2.0f * u + 1.0f) / W - 1.0f, &sn, &cn);
    return make_float3(cl * sn, -sl, cl * cn);
}

// Continuous pixel coordinates (integers at pixel centres) of direction Y in a
// camera whose scale/offset pair maps longitude and latitude to u_c and v_c.
__device__ __forceinline__ void project_dir(float X, float Y, float Z, float su, float ou, float sv,
                                            float ov, float& uc, float& vc) {
    const float lon = atan2f(X, Z);
    const float lat = atan2f(-Y, sqrtf(fmaf(X, X, Z * Z)));
    uc = fmaf(lon, su, ou);
    vc = fmaf(lat, sv, ov);
}

// Bilinear fetch at (uc, vc): columns floor(uc), floor(uc)+1 wrapped, rows
// floor(vc), floor(vc)+1 clamped, interpolated in FP32 with exact weights.
// One gather returns the 2x2 footprint; the texture addresses it at the
// centre of the footprint, (floor + 1) / size in normalised coordinates,
// so the hardware's reduced coordinate precision never moves the footprint.
// Gather order (component 0 of each texel): x = (i0, j0+1), y = (i0+1, j0+1),
// z = (i0+1, j0), w = (i0, j0).
__device__ __forceinline__ float sample_bilinear(cudaTextureObject_t tex, float inv_w, float inv_h,
                                                 float uc, float vc) {
    const float fi = floorf(uc), fj = floorf(vc);
    const float fx = uc - fi, fy = vc - fj;
    const float4 g = tex2Dgather<float4>(tex, fmaf(fi, inv_w, inv_w), fmaf(fj, inv_h, inv_h), 0);
    const float top = fmaf(fx, g.z - g.w, g.w);
    const float bot = fmaf(fx, g.y - g.x, g.x);
    return fmaf(fy, bot - top, top);
}

__device__ __forceinline__ int wrap_index(int x, int W) {
    x %= W;
    return x < 0 ? x + W : x;
}

__device__ __forceinline__ int clamp_index(int x, int hi) { return x < 0 ? 0 : (x > hi ? hi : x); }

}  // namespace pmsp
