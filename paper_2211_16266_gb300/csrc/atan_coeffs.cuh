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

// The same polynomial on two lanes with packed FP32 FMAs.
__device__ __forceinline__ float2 atan_poly2(float2 s) {
    float2 p = make_float2(-0.00405456218868494f, -0.00405456218868494f);
    p = __ffma2_rn(p, s, make_float2(0.02186293713748455f, 0.02186293713748455f));
    p = __ffma2_rn(p, s, make_float2(-0.05591229349374771f, -0.05591229349374771f));
    p = __ffma2_rn(p, s, make_float2(0.09642194211483002f, 0.09642194211483002f));
    p = __ffma2_rn(p, s, make_float2(-0.1390862762928009f, -0.1390862762928009f));
    p = __ffma2_rn(p, s, make_float2(0.19946564733982086f, 0.19946564733982086f));
    p = __ffma2_rn(p, s, make_float2(-0.33329859375953674f, -0.33329859375953674f));
    p = __ffma2_rn(p, s, make_float2(0.9999993443489075f, 0.9999993443489075f));
    return p;
}

}  // namespace pmsp
