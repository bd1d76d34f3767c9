// Generated by fit_atan.py (Remez minimax fit of atan(r) = r * P(r^2) on [0, 1]).
// Degree 7 in r^2; minimax error 3.748e-08 rad, FP32 Horner error 1.300e-07 rad.
#pragma once

namespace pmsp {

// P(s), s = r^2, by Horner's rule.
__device__ __forceinline__ float atan_poly(float s) {
    float p = -0.00405456218868494f;
    p = fmaf(p, s, 0.02186293713748455f);
    p = fmaf(p, s, -0.05591229349374771f);
    p = fmaf(p, s, 0.09642194211483002f);
    p = fmaf(p, s, -0.1390862762928009f);
    p = fmaf(p, s, 0.19946564733982086f);
    p = fmaf(p, s, -0.33329859375953674f);
    p = fmaf(p, s, 0.9999993443489075f);
    return p;
}

// 2 P(s): 2 atan(q) = q * 2 P(q^2) for |q| <= 1 (coefficients doubled, which is exact).
__device__ __forceinline__ float atan2x_poly(float s) {
    float p = -0.00810912437736988f;
    p = fmaf(p, s, 0.0437258742749691f);
    p = fmaf(p, s, -0.11182458698749542f);
    p = fmaf(p, s, 0.19284388422966003f);
    p = fmaf(p, s, -0.2781725525856018f);
    p = fmaf(p, s, 0.3989312946796417f);
    p = fmaf(p, s, -0.6665971875190735f);
    p = fmaf(p, s, 1.999998688697815f);
    return p;
}

// 2 P(s) for two pairs of lanes at once, packed FP32 FMAs interleaved so each
// coefficient pair serves both: 2 atan(q) = q * 2 P(q^2) for |q| <= 1, the form
// the paired projection uses (coefficients doubled, which is exact).
__device__ __forceinline__ void atan2x_poly2_dual(float2 s1, float2 s2, float2& p1, float2& p2) {
    p1 = make_float2(-0.00810912437736988f, -0.00810912437736988f);
    p2 = p1;
    p1 = __ffma2_rn(p1, s1, make_float2(0.0437258742749691f, 0.0437258742749691f));
    p2 = __ffma2_rn(p2, s2, make_float2(0.0437258742749691f, 0.0437258742749691f));
    p1 = __ffma2_rn(p1, s1, make_float2(-0.11182458698749542f, -0.11182458698749542f));
    p2 = __ffma2_rn(p2, s2, make_float2(-0.11182458698749542f, -0.11182458698749542f));
    p1 = __ffma2_rn(p1, s1, make_float2(0.19284388422966003f, 0.19284388422966003f));
    p2 = __ffma2_rn(p2, s2, make_float2(0.19284388422966003f, 0.19284388422966003f));
    p1 = __ffma2_rn(p1, s1, make_float2(-0.2781725525856018f, -0.2781725525856018f));
    p2 = __ffma2_rn(p2, s2, make_float2(-0.2781725525856018f, -0.2781725525856018f));
    p1 = __ffma2_rn(p1, s1, make_float2(0.3989312946796417f, 0.3989312946796417f));
    p2 = __ffma2_rn(p2, s2, make_float2(0.3989312946796417f, 0.3989312946796417f));
    p1 = __ffma2_rn(p1, s1, make_float2(-0.6665971875190735f, -0.6665971875190735f));
    p2 = __ffma2_rn(p2, s2, make_float2(-0.6665971875190735f, -0.6665971875190735f));
    p1 = __ffma2_rn(p1, s1, make_float2(1.999998688697815f, 1.999998688697815f));
    p2 = __ffma2_rn(p2, s2, make_float2(1.999998688697815f, 1.999998688697815f));
}

}  // namespace pmsp
