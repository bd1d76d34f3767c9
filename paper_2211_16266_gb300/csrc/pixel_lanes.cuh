// Half-sweep with the patch samples of one pixel split over T adjacent lanes
// of a warp (T = 2, 4 or 8), the NCC sums combined by warp shuffles.
//
// Lane `sub` of a pixel group takes the samples m = sub, sub + T, ... of the
// window (row-major order, the centre sample excluded) and accumulates every
// view's four weighted sums over them, exactly as the one-thread kernels do
// over all samples. An xor butterfly of __shfl_xor_sync within the group then
// adds the T partial sums; floating-point addition is commutative, so every
// lane of the group ends with the same bits, evaluates the same view costs
// and best-k mean and takes the same decision, and no shared-memory exchange
// or barrier is needed. The validity of the candidate (every sample ray meets
// the plane in front) is combined the same way.
//
// Every lane still holds the sums of all views (the registers of the
// one-thread kernels), but a block serves 128 / T pixels, so small keyframes
// and the last wave of a launch spread over T times more threads. Each lane
// repeats the centre sample (it centres every view's intensities) and the
// per-candidate set-up; the rest of the work is divided. The split changes
// the order in which a view's sums are added, so the maps agree with the
// one-thread kernels within rounding, not bit for bit.
//
// Unlike the warp split (pixel_split.cuh), every gather instruction of a
// warp still reads one texture: the T lanes of a pixel differ in the sample,
// not in the view.
#pragma once

#include "pixel_kernel.cuh"
#include "sample_split.h"

namespace pmsp {

// The T adjacent lanes (a pixel group) that share this lane's pixel.
template <int T>
__device__ __forceinline__ unsigned lane_group_mask() {
    const unsigned lane = threadIdx.x & 31u;
    return ((1u << T) - 1u) << (lane & ~(unsigned)(T - 1));
}

// Sum of v over the pixel group by an xor butterfly: the same bits in every lane.
template <int T>
__device__ __forceinline__ float group_sum(unsigned mask, float v) {
#pragma unroll
    for (int o = 1; o < T; o <<= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

template <int T>
__device__ __forceinline__ float2 group_sum2(unsigned mask, float2 v) {
    return make_float2(group_sum<T>(mask, v.x), group_sum<T>(mask, v.y));
}

// plane_cost_paired with this lane's share of the samples: the centre sample
// in every lane, then samples m = sub, sub + T, ... (row-major, centre
// skipped), then the group's sums. Returns 2 for an invalid plane, like the
// one-thread cost. Every early return is taken by the whole group (it
// depends on the pixel and the plane only), so the group's shuffles below
// are reached by all T lanes or by none.
template <int NS, int T, int WIN, class SM>
__device__ __forceinline__ float plane_cost_lanes(const PixelParams& P, const SM& sm, int lx, int ly,
                                                  const RefStats& st, float3 rp, float d, float3 n, int sub,
                                                  unsigned mask) {
    constexpr int NP = NS / 2;
    constexpr bool ODD = (NS & 1) != 0;
    const float eps = 1e-8f * st.Sw * st.Sw;
    if (st.varI < eps) return 2.0f;
    const float dn = d * dot3(n, rp);
    const int K = Window<WIN>::K(P), R = Window<WIN>::R(P), stp = Window<WIN>::stride(P);
    const int ac = K >> 1;

    float2 c0[NP], SJ[NP], SJJ[NP], SIJ[NP];
    float c0o = 0.f, SJo = 0.f, SJJo = 0.f, SIJo = 0.f;
    {
        const int o = ac * stp - R;
        const float cl = sm.row_cos[ly + o];
        const float3 rq = make_float3(cl * sm.col_sin[lx + o], -sm.row_sin[ly + o], cl * sm.col_cos[lx + o]);
        const float den = dot3(n, rq);
        if (!(den < -1e-6f)) return 2.0f;
        const float t = __fdividef(dn, den);
        const float X = t * rq.x, Y = t * rq.y, Z = t * rq.z;
        const float alpha = t * cl, beta = -t * sm.row_sin[ly + o];
        pairs_sample<NP, ParamViews, SM::PITCH>(P, alpha, beta, lx + o, c0);
#pragma unroll
        for (int q = 0; q < NP; ++q) SJ[q] = SJJ[q] = SIJ[q] = pair(0.f);
        if (ODD) c0o = view_sample<ParamViews>(P.src[NS - 1], X, Y, Z);
    }
    bool valid = true;
    // this lane's samples: m = sub, sub + T, ... in row-major order (sample_split.h)
    int a, b;
    split_first_sample(sub, K, a, b);
#pragma unroll 1
    for (; a < K; split_next_sample(T, K, a, b)) {
        if (!(a == ac && b == ac)) {
            const int oy = a * stp - R;
            const float cl = sm.row_cos[ly + oy], msl = -sm.row_sin[ly + oy];
            const float Iq = sm.ref[(ly + oy) * SM::PITCH + lx - R + b * stp];
            const float w = bilateral(P, sm, a, b, Iq, st.Ip);
            const float wI = w * (Iq - st.mu);
            const int cx = lx + b * stp - R;
            const float3 rq = make_float3(cl * sm.col_sin[cx], msl, cl * sm.col_cos[cx]);
            const float den = dot3(n, rq);
            valid = valid && (den < -1e-6f);
            const float t = __fdividef(dn, den);
            const float X = t * rq.x, Y = t * rq.y, Z = t * rq.z;
            const float alpha = t * cl, beta = t * msl;
            const float2 w2 = pair(w), wI2 = pair(wI);
            float2 Jall[NP];
            pairs_sample<NP, ParamViews, SM::PITCH>(P, alpha, beta, cx, Jall);
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const float2 Jc = add2(Jall[q], make_float2(-c0[q].x, -c0[q].y));
                const float2 tw = mul2(w2, Jc);
                SJ[q] = add2(SJ[q], tw);
                SJJ[q] = fma2(tw, Jc, SJJ[q]);
                SIJ[q] = fma2(wI2, Jc, SIJ[q]);
            }
            if (ODD) {
                const float Jc = view_sample<ParamViews>(P.src[NS - 1], X, Y, Z) - c0o;
                const float tw = __fmul_rn(w, Jc);
                SJo = __fadd_rn(SJo, tw);
                SJJo = fmaf(tw, Jc, SJJo);
                SIJo = fmaf(wI, Jc, SIJo);
            }
        }
    }
    // the group's sums and validity, identical in all T lanes
    unsigned ok = valid ? 1u : 0u;
#pragma unroll
    for (int o = 1; o < T; o <<= 1) ok &= __shfl_xor_sync(mask, ok, o);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        SJ[q] = group_sum2<T>(mask, SJ[q]);
        SJJ[q] = group_sum2<T>(mask, SJJ[q]);
        SIJ[q] = group_sum2<T>(mask, SIJ[q]);
    }
    if (ODD) {
        SJo = group_sum<T>(mask, SJo);
        SJJo = group_sum<T>(mask, SJJo);
        SIJo = group_sum<T>(mask, SIJo);
    }
    if (!ok) return 2.0f;

    float cs[NS];
    auto view_cost = [&](float sj, float sjj, float sij) {
        const float varJ = mul_sub(st.Sw, sjj, sj, sj);
        const float cov = mul_sub(st.Sw, sij, st.SIc, sj);
        if (varJ < eps) return 2.0f;
        float ncc = cov * rsqrtf(st.varI * varJ);
        ncc = fminf(1.0f, fmaxf(-1.0f, ncc));
        return 1.0f - ncc;
    };
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        cs[2 * q] = view_cost(SJ[q].x, SJJ[q].x, SIJ[q].x);
        cs[2 * q + 1] = view_cost(SJ[q].y, SJJ[q].y, SIJ[q].y);
    }
    if (ODD) cs[NS - 1] = view_cost(SJo, SJJo, SIJo);
#pragma unroll
    for (int pass = 0; pass < NS; ++pass) {
#pragma unroll
        for (int s = (pass & 1); s + 1 < NS; s += 2) {
            const float lo = fminf(cs[s], cs[s + 1]), hi = fmaxf(cs[s], cs[s + 1]);
            cs[s] = lo;
            cs[s + 1] = hi;
        }
    }
    float sum = 0.f;
#pragma unroll
    for (int s = 0; s < NS; ++s)
        if (s < P.best_k) sum += cs[s];
    return sum / (float)P.best_k;
}

// One half-sweep with T lanes per pixel: a 32 x (8 / T) tile, 128 / T pixels
// of one colour per block, lanes 0..T-1 of each group side by side.
template <int NS, int T, int WIN>
__global__ void __launch_bounds__(BLOCK_THREADS, pixel_min_blocks(NS))
    pixel_lanes_kernel(const __grid_constant__ PixelParams P) {
    static_assert(T == 2 || T == 4 || T == 8, "two, four or eight lanes per pixel");
    static_assert(NS >= 2, "view pairs");
    using SM = TileSmemT<32, 8 / T, T, Window<WIN>::HALO>;
    __shared__ SM sm;
    int tx, ty;
    tile_of_block(gridDim.x, gridDim.y, blockIdx.y * gridDim.x + blockIdx.x, tx, ty);
    const int bx = tx * SM::W, by = ty * SM::H;
    stage_tile(P, sm, bx, by);
    __syncthreads();
    {
        constexpr int NP = NS / 2;
        const int cols = SM::W + 2 * P.radius;
        for (int i = threadIdx.x; i < cols * NP; i += BLOCK_THREADS) {
            const int q = i / cols, c = i - q * cols;
            const PixelParams::ViewPair& VP = P.pairs[q];
            const float2 sn = pair(sm.col_sin[c]), cs = pair(sm.col_cos[c]);
            col_table<NP, SM::PITCH>()[q][0][c] = fma2(VP.R[0], sn, mul2(VP.R[2], cs));
            col_table<NP, SM::PITCH>()[q][1][c] = fma2(VP.R[3], sn, mul2(VP.R[5], cs));
            col_table<NP, SM::PITCH>()[q][2][c] = fma2(VP.R[6], sn, mul2(VP.R[8], cs));
        }
        __syncthreads();
    }
    const int pix = threadIdx.x / T, sub = threadIdx.x - pix * T;
    const unsigned mask = lane_group_mask<T>();
    const int px = pix % (SM::W / 2), py = pix / (SM::W / 2);
    const int y = by + py;
    const int x = bx + 2 * px + ((y + P.colour) & 1);
    if (x >= P.W || y >= P.H) return;  // the whole group leaves together
    const int lx = x - bx + P.radius, ly = y - by + P.radius;
    const size_t i = (size_t)y * P.W + x;
    const float3 rp = make_float3(sm.row_cos[ly] * sm.col_sin[lx], -sm.row_sin[ly], sm.row_cos[ly] * sm.col_cos[lx]);
    const RefStats st = ref_stats(P, sm, lx, ly);
    float bd = P.depth[i], bc = P.cost[i];
    float3 bn = make_float3(P.nx[i], P.ny[i], P.nz[i]);
    const float span = P.inv_dmin - P.inv_dmax;
    const int n_cand = 8 + P.n_refine;
#pragma unroll 1
    for (int k = 0; k < n_cand; ++k) {
        float dc = 0.f;
        float3 nc = make_float3(0.f, 0.f, 0.f);
        if (k < 8) {
            if (!neighbour_candidate(P, x, y, rp, k, dc, nc)) continue;
            // the incumbent's own plane has the incumbent's cost: it cannot win
            if (same_plane(dc, nc, bd, bn)) continue;
        } else {
            const int t = k - 8;
            const float s = __int_as_float((126 - t) << 23);  // 2^-(t+1)
            const U4 u = draw_uniform4(i, (uint64_t)P.iter, (uint64_t)(1 + t), P.seed, P.keyframe);
            float inv = fmaf((2.0f * u.x - 1.0f) * s, span, 1.0f / bd);
            inv = fminf(P.inv_dmin, fmaxf(P.inv_dmax, inv));
            dc = 1.0f / inv;
            nc = make_float3(fmaf(s, 2.0f * u.y - 1.0f, bn.x), fmaf(s, 2.0f * u.z - 1.0f, bn.y),
                             fmaf(s, 2.0f * u.w - 1.0f, bn.z));
            const float il = 1.0f / sqrtf(dot3(nc, nc));
            nc = face_camera(make_float3(nc.x * il, nc.y * il, nc.z * il), rp);
        }
        const float c = plane_cost_lanes<NS, T, WIN, SM>(P, sm, lx, ly, st, rp, dc, nc, sub, mask);
        if (c < bc) {
            bc = c;
            bd = dc;
            bn = nc;
        }
    }
    if (sub != 0) return;
    P.depth[i] = bd;
    P.nx[i] = bn.x;
    P.ny[i] = bn.y;
    P.nz[i] = bn.z;
    P.cost[i] = bc;
}

template <int NS, int T>
inline cudaError_t launch_lanes_sweep_t(const PixelParams& p, cudaStream_t stream) {
    const dim3 grid((p.W + 31) / 32, (p.H + 8 / T - 1) / (8 / T));
    if (window_of(p) == 1)
        pixel_lanes_kernel<NS, T, 1><<<grid, BLOCK_THREADS, 0, stream>>>(p);
    else
        pixel_lanes_kernel<NS, T, 0><<<grid, BLOCK_THREADS, 0, stream>>>(p);
    return cudaGetLastError();
}

// PixelParams::tpp = -2, -4 or -8 selects this half-sweep.
template <int NS, bool EXACT>
cudaError_t launch_lanes_sweep(const PixelParams& p, cudaStream_t stream) {
    static_assert(EXACT, "the lane-split half-sweep serves exact view counts");
    if (p.tpp <= -8) return launch_lanes_sweep_t<NS, 8>(p, stream);
    return p.tpp <= -4 ? launch_lanes_sweep_t<NS, 4>(p, stream) : launch_lanes_sweep_t<NS, 2>(p, stream);
}

}  // namespace pmsp
