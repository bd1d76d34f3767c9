// Equirectangular camera model and source fetch on the device (FP32).
//
// Paper Sec. III-C: the patch is rectangular in the reference panorama and
// takes an arbitrary shape in the sources because of the equirectangular
// projection. Convention: pixel (u, v) of a W x H panorama looks along
// lon = 2*pi*(u+0.5)/W - pi, lat = pi/2 - pi*(v+0.5)/H; bearing
// (cos lat sin lon, -sin lat, cos lat cos lon) with x right, y down, z forward.
#pragma once

#include <cuda_runtime.h>

#include "atan_coeffs.cuh"

namespace pmsp {

// Unit bearing of pixel centre (u, v). sincospif keeps the angle exact up to
// the rounding of its argument.
__device__ __forceinline__ float3 pixel_bearing(int u, int v, int W, int H) {
    float sl, cl, sn, cn;
    sincospif(0.5f - (2.0f * v + 1.0f) / (2.0f * H), &sl, &cl);
    sincospif((2.0f * u + 1.0f) / W - 1.0f, &sn, &cn);
    return make_float3(cl * sn, -sl, cl * cn);
}

// 2^x for x <= 0 on the special-function unit (relative error ~2^-22).
__device__ __forceinline__ float exp2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// atan(mn / mx) for 0 <= mn <= mx: the Remez-fitted odd polynomial
// r * P(r^2) of atan_coeffs.cuh (|error| below 1.3e-7 rad in FP32). mx = 0
// (the origin) gives 0.
__device__ __forceinline__ float atan_reduced(float mn, float mx) {
    const float r = __fdividef(mn, fmaxf(mx, 1e-30f));
    return r * atan_poly(r * r);
}

// Four-quadrant arctangent by octant reduction and reflection
// (pi/2 - a for |y| > |x|, pi - a for x < 0, sign of y). Matches atan2 on
// the axes, at the origin and for signed zeros.
__device__ __forceinline__ float fast_atan2(float y, float x) {
    const float ax = fabsf(x), ay = fabsf(y);
    float a = atan_reduced(fminf(ax, ay), fmaxf(ax, ay));
    a = ay > ax ? 1.57079632679489662f - a : a;
    a = x < 0.f ? 3.14159265358979324f - a : a;
    return copysignf(a, y);
}

// The same for x >= 0 (half plane: no reflection about the y axis).
__device__ __forceinline__ float fast_atan2_xpos(float y, float x) {
    const float ay = fabsf(y);
    float a = atan_reduced(fminf(x, ay), fmaxf(x, ay));
    a = ay > x ? 1.57079632679489662f - a : a;
    return copysignf(a, y);
}

// Continuous pixel coordinates (integers at pixel centres) of direction
// (X, Y, Z), any length > 0, in a camera whose scale/offset pairs map
// longitude and latitude to u_c and v_c: lon = atan2(X, Z),
// lat = atan2(-Y, hypot(X, Z)); hypot as q * rsqrt(q), exact 0 at the poles.
__device__ __forceinline__ void project_dir_fast(float X, float Y, float Z, float su, float ou, float sv,
                                                 float ov, float& uc, float& vc) {
    const float lon = fast_atan2(X, Z);
    const float q = fmaf(X, X, Z * Z);
    const float rho = q * rsqrtf(fmaxf(q, 1e-30f));
    const float lat = fast_atan2_xpos(-Y, rho);
    uc = fmaf(lon, su, ou);
    vc = fmaf(lat, sv, ov);
}

// 1/x on the special-function unit (rcp.approx: relative error ~2^-23).
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// sqrt(x) on the special-function unit (sqrt.approx), exact 0 at 0.
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The projection of the densification kernels, in half-angle form: both
// arctangent arguments stay in [-1, 1] with no octant logic.
// lon = 2 atan(X / (rho + |Z|)) where Z >= 0 and sign(X) pi minus it where
// Z < 0; -lat = 2 atan(Y / (|Y| + rho)), rho = hypot(X, Z), both square roots
// on the special-function unit. A direction exactly on the source's vertical
// axis (X = Z = 0 in FP32) gives NaN coordinates; the view's NCC then clamps
// to -1 and the view costs 2, as for an invalid sample (no fault: texture
// fetches accept any coordinate).
//
// The pixel coordinates come out split so that their fractions are rounded
// at the scale of a quarter panorama, not of a whole one, and so that the
// whole columns and rows become constant texture offsets (W and H even). With
// al = 2 atan(ql) (|al| <= pi/2): on the front half (front = Z >= 0)
// u_c = su al + W/2 - 0.5 and qu = su al + 0.5 = u_c - (W/2 - 1); on the back
// half u_c = -su al - 0.5 modulo W and qu = -su al + 0.5 = u_c + 1;
// v_c = nsv (-lat) + H/2 - 0.5 and qv = nsv (-lat) + 0.5 = v_c - (H/2 - 1).
// |qu| <= W/4 + 0.5, |qv| <= H/2 + 0.5. The gather footprint centre, the left
// edge of texel floor(u_c) + 1, is then floor(qu) / W + 0.5 (front) or
// floor(qu) / W (back), and floor(qv) / H + 0.5 in v: see
// sample_bilinear_half. nsv = -sv = H / pi. The paired cost path performs
// exactly these operations per lane after its rigid transform.
__device__ __forceinline__ void project_dir_half(float X, float Y, float Z, float su, float nsv, float& qu,
                                                 float& qv, bool& front) {
    const float q = fmaf(X, X, Z * Z);
    const float rho = sqrt_approx(q);
    const float ql = X * rcp_approx(rho + fabsf(Z));
    const float r2 = fmaf(Y, Y, q);
    const float r3 = sqrt_approx(r2);
    const float qt = Y * rcp_approx(r3 + rho);
    const float al = ql * atan2x_poly(ql * ql), nlat = qt * atan2x_poly(qt * qt);
    front = Z >= 0.f;
    qu = fmaf(al, front ? su : -su, 0.5f);
    qv = fmaf(nlat, nsv, 0.5f);
}

// floor(x) for |x| < 2^22 with two FP32 adds: adding 1.5 * 2^23 rounded
// towards -inf leaves floor(x) in the low mantissa bits.
__device__ __forceinline__ float floor_small(float x) {
    const float M = 12582912.0f;
    return __fadd_rd(x, M) - M;
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
    const float fi = floor_small(uc), fj = floor_small(vc);
    const float fx = uc - fi, fy = vc - fj;
    const float4 g = tex2Dgather<float4>(tex, fmaf(fi, inv_w, inv_w), fmaf(fj, inv_h, inv_h), 0);
    const float top = fmaf(fx, g.z - g.w, g.w);
    const float bot = fmaf(fx, g.y - g.x, g.x);
    return fmaf(fy, bot - top, top);
}

// Bilinear fetch at split coordinates (see project_dir_half): the gather
// addresses the 2 x 2 footprint at its centre in normalised coordinates.
__device__ __forceinline__ float sample_bilinear_half(cudaTextureObject_t tex, float inv_w, float inv_h, float qu,
                                                      float qv, bool front) {
    const float fi = floor_small(qu), fj = floor_small(qv);
    const float fx = qu - fi, fy = qv - fj;
    const float4 g = tex2Dgather<float4>(tex, fmaf(fi, inv_w, front ? 0.5f : 0.0f), fmaf(fj, inv_h, 0.5f), 0);
    const float top = fmaf(fx, g.z - g.w, g.w);
    const float bot = fmaf(fx, g.y - g.x, g.x);
    return fmaf(fy, bot - top, top);
}

// ---- Sums of products with their rounding fixed by the source: each
// multiply-add an explicit fmaf and each other product an explicit __fmul_rn,
// which the compiler never fuses. Written as a * b + c * d, the compiler may
// fuse either product depending on the code around it, and on low-variance
// patches the two roundings move the NCC cost by up to 1e-4; with these the
// cost of a plane at a pixel has the same bits in every kernel that
// evaluates it.

// a . b = a.z b.z + (a.y b.y + a.x b.x), fused from the x product outward.
__device__ __forceinline__ float dot3(float3 a, float3 b) { return fmaf(a.z, b.z, fmaf(a.y, b.y, __fmul_rn(a.x, b.x))); }
// a b - c d with a b fused.
__device__ __forceinline__ float mul_sub(float a, float b, float c, float d) { return fmaf(a, b, -__fmul_rn(c, d)); }

// ---- Two views at once: the same arithmetic on float2 pairs with the packed
// FP32 instructions (fma/add/mul .f32x2), which issue once for both lanes.

__device__ __forceinline__ float2 pair(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

__device__ __forceinline__ float2 floor_small2(float2 x) {
    const float M = 12582912.0f;
    return add2(__fadd2_rd(x, pair(M)), pair(-M));
}

__device__ __forceinline__ int wrap_index(int x, int W) {
    x %= W;
    return x < 0 ? x + W : x;
}

__device__ __forceinline__ int clamp_index(int x, int hi) { return x < 0 ? 0 : (x > hi ? hi : x); }

}  // namespace pmsp
