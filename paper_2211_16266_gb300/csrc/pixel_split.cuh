// Half-sweep with several threads per pixel: the views of one pixel are split
// over T warps (T = 2 or 4). The T warps of a pixel group hold the same 32
// pixels, one per lane; warp `sub` of the group evaluates the view pairs
// q = sub, sub + T, ... (and the odd last view in one of them). Each warp
// writes its views' costs of the current
// candidate to shared memory, the group meets at a named barrier, and every
// warp then reads all view costs of its pixel, sorts them and averages the
// best k itself, so all T warps take the same decision. The split lowers the
// per-thread register footprint (a warp keeps the sums of NS / T views), so
// more warps stay resident, at the price of repeating the per-sample work
// shared by the views (plane intersection, bilateral weight) in each warp.
//
// Splitting by lane instead (the T threads of a pixel side by side in one
// warp) would make one gather instruction fetch from T different textures;
// split by warp, every gather of a warp reads one texture.
//
// Every per-view sum is accumulated in the same sample order as in the
// one-thread-per-pixel kernels and the view costs are sorted in the same
// positions, so the maps are bit-identical to theirs.
#pragma once

#include "pixel_kernel.cuh"

namespace pmsp {

// Resident blocks the split kernels' register budget is sized for: a warp
// keeps about NS / T views' sums, so the budget follows the views per warp
// (8 blocks up to 6, 6 up to 8, 5 beyond).
constexpr int split_min_blocks(int ns, int t) {
    return t == 1 ? pixel_min_blocks(ns) : (ns + t - 1) / t <= 6 ? 8 : (ns + t - 1) / t <= 8 ? 6 : 5;
}

// Barrier of pixel group `group` (its T warps); ids 1 and 2 as constants, so
// the kernel reserves two named barriers besides __syncthreads'.
template <int T>
__device__ __forceinline__ void group_barrier(int group) {
    if (group == 0)
        asm volatile("barrier.sync 1, %0;" ::"n"(32 * T) : "memory");
    else
        asm volatile("barrier.sync 2, %0;" ::"n"(32 * T) : "memory");
}

// pairs_sample for the view pairs q = SUB, SUB + T, ... < NP only (their
// constants in kernel parameters), the same operations per pair.
template <int NP, int T, int SUB, int PITCH, int NPL = (SUB < NP ? (NP - SUB + T - 1) / T : 0)>
__device__ __forceinline__ void pairs_sample_sub(const PixelParams& P, float alpha, float beta, int cx,
                                                 float2 (&J)[NPL > 0 ? NPL : 1]) {
    float2 fx[NPL > 0 ? NPL : 1], fy[NPL > 0 ? NPL : 1], xn[NPL > 0 ? NPL : 1], yn[NPL > 0 ? NPL : 1];
    const float2 av = pair(alpha), bv = pair(beta);
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
        const int q = SUB + j * T;
        const PixelParams::ViewPair& VP = P.pairs[q];
        const float2 Yx = fma2(av, col_table<NP, PITCH>()[q][0][cx], fma2(bv, VP.R[1], VP.t[0]));
        const float2 Yy = fma2(av, col_table<NP, PITCH>()[q][1][cx], fma2(bv, VP.R[4], VP.t[1]));
        const float2 Yz = fma2(av, col_table<NP, PITCH>()[q][2][cx], fma2(bv, VP.R[7], VP.t[2]));
        const float2 q2 = fma2(Yx, Yx, mul2(Yz, Yz));
        const float2 rho = make_float2(sqrt_approx(q2.x), sqrt_approx(q2.y));
        const float2 dl = add2(rho, make_float2(fabsf(Yz.x), fabsf(Yz.y)));
        const float2 ql = mul2(Yx, make_float2(rcp_approx(dl.x), rcp_approx(dl.y)));
        const float2 r2 = fma2(Yy, Yy, q2);
        const float2 r3 = make_float2(sqrt_approx(r2.x), sqrt_approx(r2.y));
        const float2 dt = add2(r3, rho);
        const float2 qt = mul2(Yy, make_float2(rcp_approx(dt.x), rcp_approx(dt.y)));
        float2 pl, pt;
        atan2x_poly2_dual(mul2(ql, ql), mul2(qt, qt), pl, pt);
        const float2 al = mul2(ql, pl), nlat = mul2(qt, pt);
        const bool f0 = Yz.x >= 0.f, f1 = Yz.y >= 0.f;
        const float2 qu = fma2(al, make_float2(f0 ? VP.su.x : -VP.su.x, f1 ? VP.su.y : -VP.su.y), pair(0.5f));
        const float2 qv = fma2(nlat, VP.nsv, pair(0.5f));
        const float2 fi = floor_small2(qu), fj = floor_small2(qv);
        fx[j] = add2(qu, make_float2(-fi.x, -fi.y));
        fy[j] = add2(qv, make_float2(-fj.x, -fj.y));
        xn[j] = fma2(fi, VP.inv_w, make_float2(f0 ? 0.5f : 0.0f, f1 ? 0.5f : 0.0f));
        yn[j] = fma2(fj, VP.inv_h, pair(0.5f));
    }
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
        const int q = SUB + j * T;
        const float4 g0 = tex2Dgather<float4>(P.src[2 * q].tex, xn[j].x, yn[j].x, 0);
        const float4 g1 = tex2Dgather<float4>(P.src[2 * q + 1].tex, xn[j].y, yn[j].y, 0);
        const float top0 = fmaf(fx[j].x, g0.z - g0.w, g0.w), bot0 = fmaf(fx[j].x, g0.y - g0.x, g0.x);
        const float top1 = fmaf(fx[j].y, g1.z - g1.w, g1.w), bot1 = fmaf(fx[j].y, g1.y - g1.x, g1.x);
        J[j] = make_float2(fmaf(fy[j].x, bot0 - top0, top0), fmaf(fy[j].y, bot1 - top1, top1));
    }
}

// Per-view costs of view pairs q = SUB, SUB + T, ... < NP (and the odd last view,
// in warp NP % T) at sample points of plane (d, n), written to xc[s][pix]. The
// arithmetic per view is that of plane_cost_paired.
template <int NS, int T, int SUB, int WIN, class SM>
__device__ __forceinline__ void pair_costs_sub(const PixelParams& P, const SM& sm, int lx, int ly, const RefStats& st,
                                               float3 rp, float d, float3 n, float* xc, int pix, int pix_stride) {
    constexpr int NP = NS / 2;
    constexpr bool ODD = (NS & 1) != 0;
    constexpr bool MY_ODD = ODD && SUB == NP % T;
    constexpr int NPL = SUB < NP ? (NP - SUB + T - 1) / T : 0;
    const float eps = 1e-8f * st.Sw * st.Sw;
    auto store_all = [&](float c) {
#pragma unroll
        for (int j = 0; j < NPL; ++j) {
            const int q = SUB + j * T;
            xc[(2 * q) * pix_stride + pix] = c;
            xc[(2 * q + 1) * pix_stride + pix] = c;
        }
        if (MY_ODD) xc[(NS - 1) * pix_stride + pix] = c;
    };
    if (st.varI < eps) {
        store_all(2.0f);
        return;
    }
    const float dn = d * dot3(n, rp);
    const int K = Window<WIN>::K(P), R = Window<WIN>::R(P), stp = Window<WIN>::stride(P);
    const int ac = K >> 1;

    float2 c0[NPL > 0 ? NPL : 1], SJ[NPL > 0 ? NPL : 1], SJJ[NPL > 0 ? NPL : 1], SIJ[NPL > 0 ? NPL : 1];
    float c0o = 0.f, SJo = 0.f, SJJo = 0.f, SIJo = 0.f;
    {
        const int o = ac * stp - R;
        const float cl = sm.row_cos[ly + o];
        const float3 rq = make_float3(cl * sm.col_sin[lx + o], -sm.row_sin[ly + o], cl * sm.col_cos[lx + o]);
        const float den = dot3(n, rq);
        if (!(den < -1e-6f)) {
            store_all(2.0f);
            return;
        }
        const float t = __fdividef(dn, den);
        const float X = t * rq.x, Y = t * rq.y, Z = t * rq.z;
        const float alpha = t * cl, beta = -t * sm.row_sin[ly + o];
        pairs_sample_sub<NP, T, SUB, SM::PITCH>(P, alpha, beta, lx + o, c0);
#pragma unroll
        for (int j = 0; j < NPL; ++j) SJ[j] = SJJ[j] = SIJ[j] = pair(0.f);
        if (MY_ODD) c0o = view_sample<ParamViews>(P.src[NS - 1], X, Y, Z);
    }
    bool valid = true;
#pragma unroll 1
    for (int a = 0; a < K; ++a) {
        const int oy = a * stp - R;
        const float cl = sm.row_cos[ly + oy], msl = -sm.row_sin[ly + oy];
        const float* ref_row = sm.ref + (ly + oy) * SM::PITCH + lx - R;
#pragma unroll 1
        for (int b = 0; b < K; ++b) {
            if (a == ac && b == ac) continue;
            const float Iq = ref_row[b * stp];
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
            float2 Jall[NPL > 0 ? NPL : 1];
            pairs_sample_sub<NP, T, SUB, SM::PITCH>(P, alpha, beta, cx, Jall);
#pragma unroll
            for (int j = 0; j < NPL; ++j) {
                const float2 Jc = add2(Jall[j], make_float2(-c0[j].x, -c0[j].y));
                const float2 tw = mul2(w2, Jc);
                SJ[j] = add2(SJ[j], tw);
                SJJ[j] = fma2(tw, Jc, SJJ[j]);
                SIJ[j] = fma2(wI2, Jc, SIJ[j]);
            }
            if (MY_ODD) {
                const float Jc = view_sample<ParamViews>(P.src[NS - 1], X, Y, Z) - c0o;
                const float tw = __fmul_rn(w, Jc);
                SJo = __fadd_rn(SJo, tw);
                SJJo = fmaf(tw, Jc, SJJo);
                SIJo = fmaf(wI, Jc, SIJo);
            }
        }
    }
    if (!valid) {
        store_all(2.0f);
        return;
    }
    auto view_cost = [&](float sj, float sjj, float sij) {
        const float varJ = mul_sub(st.Sw, sjj, sj, sj);
        const float cov = mul_sub(st.Sw, sij, st.SIc, sj);
        if (varJ < eps) return 2.0f;
        float ncc = cov * rsqrtf(st.varI * varJ);
        ncc = fminf(1.0f, fmaxf(-1.0f, ncc));
        return 1.0f - ncc;
    };
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
        const int q = SUB + j * T;
        xc[(2 * q) * pix_stride + pix] = view_cost(SJ[j].x, SJJ[j].x, SIJ[j].x);
        xc[(2 * q + 1) * pix_stride + pix] = view_cost(SJ[j].y, SJJ[j].y, SIJ[j].y);
    }
    if (MY_ODD) xc[(NS - 1) * pix_stride + pix] = view_cost(SJo, SJJo, SIJo);
}

// This warp's share of the view costs: a warp-uniform switch over the warp's
// index in its group, so every pair index is a compile-time constant.
template <int NS, int T, int WIN, class SM>
__device__ __forceinline__ void view_costs_split(int sub, const PixelParams& P, const SM& sm, int lx, int ly,
                                                 const RefStats& st, float3 rp, float d, float3 n, float* xc, int pix,
                                                 int pix_stride) {
    switch (sub) {
        case 0: pair_costs_sub<NS, T, 0, WIN>(P, sm, lx, ly, st, rp, d, n, xc, pix, pix_stride); break;
        case 1: pair_costs_sub<NS, T, 1, WIN>(P, sm, lx, ly, st, rp, d, n, xc, pix, pix_stride); break;
        case 2: if constexpr (T > 2) pair_costs_sub<NS, T, 2, WIN>(P, sm, lx, ly, st, rp, d, n, xc, pix, pix_stride); break;
        default: if constexpr (T > 3) pair_costs_sub<NS, T, 3, WIN>(P, sm, lx, ly, st, rp, d, n, xc, pix, pix_stride); break;
    }
}

// Mean of the best_k smallest of the NS view costs of pixel `pix`, with the
// sorting network of the one-thread kernels (same positions, same result).
template <int NS>
__device__ __forceinline__ float best_k_mean(const PixelParams& P, const float* xc, int pix, int pix_stride) {
    float cs[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) cs[s] = xc[s * pix_stride + pix];
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

template <int NS, int T, int WIN>
__global__ void __launch_bounds__(BLOCK_THREADS, split_min_blocks(NS, T))
    pixel_split_kernel(const __grid_constant__ PixelParams P) {
    static_assert(T == 2 || T == 4, "two or four warps per pixel group");
    static_assert(NS >= 2, "view pairs");
    using SM = TileSmemT<32, 8 / T, T, Window<WIN>::HALO>;
    constexpr int PIX = 128 / T;  // pixels of one colour per block
    __shared__ SM sm;
    __shared__ float xc[2][NS * PIX];  // view costs of the current candidate, double-buffered
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
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int group = warp / T, sub = warp - group * T;
    const int pix = group * 32 + lane;
    const int px = pix % (SM::W / 2), py = pix / (SM::W / 2);
    const int y = by + py;
    const int x = bx + 2 * px + ((y + P.colour) & 1);
    // pixels outside the image stay in the loop: the group's barriers need every warp
    const bool active = x < P.W && y < P.H;
    const int lx = x - bx + P.radius, ly = y - by + P.radius;
    const size_t i = active ? (size_t)y * P.W + x : 0;
    float3 rp = make_float3(0.f, 0.f, 1.f);
    RefStats st{};
    float bd = 1.f, bc = 0.f;
    float3 bn = make_float3(0.f, 0.f, -1.f);
    if (active) {
        rp = make_float3(sm.row_cos[ly] * sm.col_sin[lx], -sm.row_sin[ly], sm.row_cos[ly] * sm.col_cos[lx]);
        st = ref_stats(P, sm, lx, ly);
        bd = P.depth[i];
        bn = make_float3(P.nx[i], P.ny[i], P.nz[i]);
        bc = P.cost[i];
    }
    const float span = P.inv_dmin - P.inv_dmax;
    const int n_cand = 8 + P.n_refine;
    int par = 0;
#pragma unroll 1
    for (int k = 0; k < n_cand; ++k) {
        float dc = 0.f;
        float3 nc = make_float3(0.f, 0.f, 0.f);
        bool ok = active;
        if (ok && k < 8) {
            const int qy = y + c_neighbors[P.table][k][1];
            ok = qy >= 0 && qy < P.H;
            if (ok) {
                const int qx = wrap_index(x + c_neighbors[P.table][k][0], P.W);
                const size_t j = (size_t)qy * P.W + qx;
                nc = make_float3(P.nx[j], P.ny[j], P.nz[j]);
                const float den = dot3(nc, rp);
                const float3 rq = pixel_bearing(qx, qy, P.W, P.H);
                dc = P.depth[j] * dot3(nc, rq) / den;
                ok = den < -1e-6f && dc >= P.d_min && dc <= P.d_max;
            }
        } else if (ok) {
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
        if (ok) view_costs_split<NS, T, WIN>(sub, P, sm, lx, ly, st, rp, dc, nc, xc[par], pix, PIX);
        group_barrier<T>(group);
        if (ok) {
            const float c = best_k_mean<NS>(P, xc[par], pix, PIX);
            if (c < bc) {
                bc = c;
                bd = dc;
                bn = nc;
            }
        }
        par ^= 1;
    }
    if (active && sub == 0) {
        P.depth[i] = bd;
        P.nx[i] = bn.x;
        P.ny[i] = bn.y;
        P.nz[i] = bn.z;
        P.cost[i] = bc;
    }
}

template <int NS, int T>
inline cudaError_t launch_split_sweep_t(const PixelParams& p, cudaStream_t stream) {
    const dim3 grid((p.W + 31) / 32, (p.H + 8 / T - 1) / (8 / T));
    if (window_of(p) == 1)
        pixel_split_kernel<NS, T, 1><<<grid, BLOCK_THREADS, 0, stream>>>(p);
    else
        pixel_split_kernel<NS, T, 0><<<grid, BLOCK_THREADS, 0, stream>>>(p);
    return cudaGetLastError();
}

template <int NS, bool EXACT>
cudaError_t launch_split_sweep(const PixelParams& p, cudaStream_t stream) {
    static_assert(EXACT, "the split half-sweep serves exact view counts");
    return p.tpp >= 4 ? launch_split_sweep_t<NS, 4>(p, stream) : launch_split_sweep_t<NS, 2>(p, stream);
}

}  // namespace pmsp
