// Per-pixel PatchMatch kernels: matching cost, random initialisation and the
// red-black half-sweep (propagation + refinement), templated on the number
// of source views the thread keeps in registers.
//
// Paper: random initialisation of the plane map (Sec. III-B); parallel
// red-black propagation over an 8-neighbourhood whose inner neighbours sit
// one position further out than in Galliani et al. (Sec. III-C, Fig. 5);
// six random refinement tests on a shrinking range (Sec. III-C, item 1). The
// cost is the bilaterally weighted NCC of the reference patch against its
// reprojection through the plane into every source, averaged over the best k
// views (the cost of the PatchMatch works the paper cites).
//
// Design: one thread per active pixel of a 32x8 tile (one colour per launch),
// blocks walking the image in strips of tile rows. The reference tile with
// its halo, the per-row / per-column bearing terms, the spatial weights and
// (for exactly known view counts) each view pair's rotated column directions
// are staged in shared memory; the sample loop runs over the patch with all
// views innermost, so the plane intersection and the bilateral weight of a
// sample are shared by every view. Views are processed in pairs with packed
// FP32 instructions, the projection in half-angle form (see camera.cuh). Per
// view four FP32 sums are kept: the source intensity is centred on its value
// at the first (centre-most) sample, which keeps the variance term free of
// cancellation. The 8 neighbour candidates and the refinement candidates run
// through one loop with a single inlined copy of the cost.
#pragma once

#include <cuda_fp16.h>

#include <type_traits>

#include "camera.cuh"
#include "common.cuh"
#include "philox.cuh"

namespace pmsp {

static __constant__ int c_neighbors[2][8][2] = {
    {{0, -3}, {0, 3}, {-3, 0}, {3, 0}, {0, -5}, {0, 5}, {-5, 0}, {5, 0}},
    {{0, -1}, {0, 1}, {-1, 0}, {1, 0}, {0, -5}, {0, 5}, {-5, 0}, {5, 0}}};


// Resident blocks per SM the batched kernel's register budget is sized for,
// by its largest view count (its per-view-count variants share one budget).
constexpr int min_blocks_for(int ns) { return ns <= 4 ? 8 : ns <= 6 ? 7 : ns <= 8 ? 6 : ns <= 10 ? 5 : 4; }

// Resident blocks per SM of the single-keyframe kernels, by view count:
// 5 (96 registers) up to 4 views, 4 (128) for 5-8 views, 3 (168) for 9-10
// and 4 beyond (the compiler left alone takes up to 246). Each tier is the
// fastest of 3-7 blocks on 1920x960 half-sweeps: fewer, spill-free threads
// beat more resident warps once the per-view sums fill the registers.
constexpr int pixel_min_blocks(int ns) { return ns <= 4 ? 5 : ns <= 8 ? 4 : ns <= 10 ? 3 : 4; }

// Reference-side constants of one pixel (independent of the hypothesis).
struct RefStats {
    float Ip;    // centre intensity
    float mu;    // weighted mean of the samples
    float Sw;    // sum of weights
    float SIc;   // sum w (I - mu)   (zero up to rounding)
    float varI;  // Sw * sum w (I - mu)^2 - SIc^2
};

// Per-block scratch of the half-sweep's pooled candidate evaluation: each
// pixel's reference statistics and the minimum (cost, candidate) key of its
// neighbour candidates, and per warp the list of (lane, candidate) pairs that
// need a cost evaluation.
struct SweepPool {
    unsigned long long key[BLOCK_THREADS];
    RefStats st[BLOCK_THREADS];
    unsigned char item[BLOCK_THREADS / 32][32 * 8];
};
struct NoPool {};

// Shared memory of one tile of TW x TH reference pixels with a halo of HALO
// pixels on each side (the window radius the tile serves: the largest, or
// that of a fixed-window instance); every shape has (TW / 2) x TH pixels of
// one colour and TPP threads per pixel, 128 threads in all.
template <int TW, int TH, int TPP = 1, int HALO = MAX_HALO>
struct TileSmemT {
    static constexpr int W = TW, H = TH;
    static constexpr int PITCH = TW + 2 * HALO, ROWS = TH + 2 * HALO;
    static constexpr int THREADS = (TW / 2) * TH;
    static_assert(THREADS * TPP == BLOCK_THREADS, "every tile shape runs 128 threads");
    static_assert(HALO >= 0 && HALO <= MAX_HALO, "halo within the largest window");
    float ref[ROWS * PITCH];             // normalised intensities, halo included
    float row_cos[ROWS], row_sin[ROWS];  // cos lat, sin lat
    float col_sin[PITCH], col_cos[PITCH];  // sin lon, cos lon
    float wsp[2 * HALO + 1];             // spatial log2-weight of offset index k
    // candidate pooling of the one-thread-per-pixel half-sweep
    typename std::conditional<TPP == 1, SweepPool, NoPool>::type pool;
};
using TileSmem = TileSmemT<TILE_W, TILE_H>;  // the batched and no-alloc kernels' shape

// Tile shapes of the single-keyframe half-sweep, chosen by PixelParams::tile.
template <int TS, int HALO = MAX_HALO> struct TileShape { using Smem = TileSmemT<32, 8, 1, HALO>; };
template <int HALO> struct TileShape<1, HALO> { using Smem = TileSmemT<64, 4, 1, HALO>; };
template <int HALO> struct TileShape<2, HALO> { using Smem = TileSmemT<16, 16, 1, HALO>; };

// Rotated column directions of the paired path: for view pair q and tile
// column c, colU[q][k][c] = row k of R_s applied to (sin lon_c, 0, cos lon_c)
// for both views of the pair. A sample direction r = (cl sin, -sl, cl cos)
// then transforms as R r = cl U_c - sl R_col1. One table per kernel, sized
// by the tile's columns (PITCH, halo included) and by CAP pairs: 5 for up to
// 10 views, so the batched kernel's view counts share one table, and 8 only
// in the kernels of 11 to 16 views.
constexpr int MAX_COL_PAIRS = 5;

template <int CAP, int PITCH>
__device__ __forceinline__ auto& col_array() {
    __shared__ float2 t[CAP][3][PITCH];
    return t;
}

template <int NP, int PITCH>
__device__ __forceinline__ auto& col_table() {
    return col_array<NP <= MAX_COL_PAIRS ? MAX_COL_PAIRS : PMSP_MAX_SOURCES / 2, PITCH>();
}

// Sample window of the paired cost loop: WIN 0 reads the window from the
// parameters; the fixed windows make the loop bounds and offsets constants
// (3 % faster half-sweeps at 11x11 / 2). WIN 1: 11x11 sampled at stride 2
// (6 x 6 samples, radius 5); WIN 2: 7x7 dense (7 x 7, radius 3).
template <int WIN>
struct Window {
    static constexpr int HALO = MAX_HALO;  // the tile halo the instance needs
    __device__ static int K(const PixelParams& P) { return P.K; }
    __device__ static int R(const PixelParams& P) { return P.radius; }
    __device__ static int stride(const PixelParams& P) { return P.stride; }
};
template <>
struct Window<1> {
    static constexpr int HALO = 5;
    __device__ static constexpr int K(const PixelParams&) { return 6; }
    __device__ static constexpr int R(const PixelParams&) { return 5; }
    __device__ static constexpr int stride(const PixelParams&) { return 2; }
};
template <>
struct Window<2> {
    static constexpr int HALO = 3;
    __device__ static constexpr int K(const PixelParams&) { return 7; }
    __device__ static constexpr int R(const PixelParams&) { return 3; }
    __device__ static constexpr int stride(const PixelParams&) { return 1; }
};


__device__ __forceinline__ float load_ref(const PixelParams& P, int x, int y) {
    const uint8_t* row = P.ref + (int64_t)y * P.ref_pitch;
    if (P.ref_format == PMSP_U8) return (float)row[x] * (1.0f / 255.0f);
    if (P.ref_format == PMSP_F16) return __half2float(reinterpret_cast<const __half*>(row)[x]);
    return reinterpret_cast<const float*>(row)[x];
}

template <class SM>
__device__ __forceinline__ void stage_tile(const PixelParams& P, SM& sm, int bx, int by) {
    const int R = P.radius;
    const int rows = SM::H + 2 * R, cols = SM::W + 2 * R;
    for (int i = threadIdx.x; i < rows * cols; i += BLOCK_THREADS) {
        const int ly = i / cols, lx = i - ly * cols;
        const int gy = clamp_index(by - R + ly, P.H - 1);
        const int gx = wrap_index(bx - R + lx, P.W);
        sm.ref[ly * SM::PITCH + lx] = load_ref(P, gx, gy);
    }
    // Bearing tables in FP64, rounded once to FP32. An FP32 angle argument
    // (2 gx + 1) / W - 1 is itself rounded by up to 6e-8 near 1, i.e. pi x 6e-8
    // = 1.9e-7 rad of direction error per column, 1.1e-4 px at 3840 px: that,
    // not the projection, was the largest error of the matching cost at that
    // size. A block computes at most 2 x (TILE + 2 x halo) entries, so the FP64
    // cost is negligible.
    for (int i = threadIdx.x; i < rows; i += BLOCK_THREADS) {
        const int gy = clamp_index(by - R + i, P.H - 1);
        double s, c;
        sincospi(0.5 - (2.0 * gy + 1.0) / (2.0 * P.H), &s, &c);
        sm.row_sin[i] = (float)s;
        sm.row_cos[i] = (float)c;
    }
    for (int i = threadIdx.x; i < cols; i += BLOCK_THREADS) {
        const int gx = wrap_index(bx - R + i, P.W);
        double s, c;
        sincospi((2.0 * gx + 1.0) / P.W - 1.0, &s, &c);
        sm.col_sin[i] = (float)s;
        sm.col_cos[i] = (float)c;
    }
    for (int k = threadIdx.x; k < P.K; k += BLOCK_THREADS) {
        const float o = (float)(k * P.stride - R);
        sm.wsp[k] = P.ws * o * o;
    }
}

// Bilateral weight of sample (a, b) with intensity Iq: 2^(wc dI^2 + ws |o|^2).
template <class SM>
__device__ __forceinline__ float bilateral(const PixelParams& P, const SM& sm, int a, int b, float Iq,
                                           float Ip) {
    const float dI = Iq - Ip;
    return exp2_approx(fmaf(P.wc, dI * dI, sm.wsp[a] + sm.wsp[b]));
}

// Local (halo-inclusive) tile coordinates of the pixel: lx, ly.
template <class SM>
__device__ __forceinline__ RefStats ref_stats(const PixelParams& P, const SM& sm, int lx, int ly) {
    RefStats st;
    st.Ip = sm.ref[ly * SM::PITCH + lx];
    const int R = P.radius, stp = P.stride;
    float Sw = 0.f, SI = 0.f;
    for (int a = 0; a < P.K; ++a) {
        const float* row = sm.ref + (ly + a * stp - R) * SM::PITCH + lx - R;
        for (int b = 0; b < P.K; ++b) {
            const float Iq = row[b * stp];
            const float w = bilateral(P, sm, a, b, Iq, st.Ip);
            Sw += w;
            SI = fmaf(w, Iq, SI);
        }
    }
    st.Sw = Sw;
    st.mu = SI / Sw;
    float SIc = 0.f, SIIc = 0.f;
    for (int a = 0; a < P.K; ++a) {
        const float* row = sm.ref + (ly + a * stp - R) * SM::PITCH + lx - R;
        for (int b = 0; b < P.K; ++b) {
            const float Iq = row[b * stp];
            const float w = bilateral(P, sm, a, b, Iq, st.Ip);
            const float Ic = Iq - st.mu;
            SIc = fmaf(w, Ic, SIc);
            SIIc = fmaf(w * Ic, Ic, SIIc);
        }
    }
    st.SIc = SIc;
    st.varI = mul_sub(Sw, SIIc, SIc, SIc);
    return st;
}

// Where the per-view constants are read from. Kernel parameters: plain member
// reads (they become constant-bank operands). Shared memory (the batched
// kernel): volatile vector loads at every use, so the compiler reloads them
// instead of holding all views' constants in registers.
struct ParamViews {
    // Reads go straight to the parameter at each use, so they stay
    // constant-bank operands of the arithmetic instead of register copies.
    struct Loaded {
        const SourceView& V;
        __device__ __forceinline__ float r(int k) const { return V.R[k]; }
        __device__ __forceinline__ float t(int k) const { return V.t[k]; }
        __device__ __forceinline__ float su() const { return V.su; }
        __device__ __forceinline__ float ou() const { return V.ou; }
        __device__ __forceinline__ float sv() const { return V.sv; }
        __device__ __forceinline__ float ov() const { return V.ov; }
        __device__ __forceinline__ float inv_w() const { return V.inv_w; }
        __device__ __forceinline__ float inv_h() const { return V.inv_h; }
        __device__ __forceinline__ cudaTextureObject_t tex() const { return V.tex; }
    };
    __device__ __forceinline__ static Loaded load(const SourceView& V) { return Loaded{V}; }
};

struct SharedViews {
    __device__ __forceinline__ static float4 ld4(const float4* p) {
        float4 v;
        const unsigned a = (unsigned)__cvta_generic_to_shared(p);
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
        return v;
    }
    // The 80-byte view as 20 words: tex (2), R (9), t (3), su, ou, sv, ov, inv_w, inv_h.
    struct Loaded {
        float w[20];
        __device__ __forceinline__ float r(int k) const { return w[2 + k]; }
        __device__ __forceinline__ float t(int k) const { return w[11 + k]; }
        __device__ __forceinline__ float su() const { return w[14]; }
        __device__ __forceinline__ float ou() const { return w[15]; }
        __device__ __forceinline__ float sv() const { return w[16]; }
        __device__ __forceinline__ float ov() const { return w[17]; }
        __device__ __forceinline__ float inv_w() const { return w[18]; }
        __device__ __forceinline__ float inv_h() const { return w[19]; }
        __device__ __forceinline__ cudaTextureObject_t tex() const {
            return (cudaTextureObject_t)(((unsigned long long)__float_as_uint(w[1]) << 32) | __float_as_uint(w[0]));
        }
    };
    __device__ __forceinline__ static Loaded load(const SourceView& V) {
        Loaded L;
        const float4* q = reinterpret_cast<const float4*>(&V);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const float4 a = ld4(q + k);
            L.w[4 * k] = a.x;
            L.w[4 * k + 1] = a.y;
            L.w[4 * k + 2] = a.z;
            L.w[4 * k + 3] = a.w;
        }
        return L;
    }
};

// The constants of a view pair the paired sample loop reads, and the texture
// of a view. Kernel parameters (ParamViews): member reads at the point of use,
// which become constant-bank operands. Shared memory (SharedViews, the batched
// kernel): volatile 16-byte loads at every sample, so the compiler reloads
// them instead of keeping every pair's constants in registers across the
// sample loop.
template <class VA>
struct PairOf {  // kernel parameters: each constant read where it is used
    const PixelParams::ViewPair& V;
    __device__ __forceinline__ float2 r1() const { return V.R[1]; }
    __device__ __forceinline__ float2 r4() const { return V.R[4]; }
    __device__ __forceinline__ float2 r7() const { return V.R[7]; }
    __device__ __forceinline__ float2 t0() const { return V.t[0]; }
    __device__ __forceinline__ float2 t1() const { return V.t[1]; }
    __device__ __forceinline__ float2 t2() const { return V.t[2]; }
    __device__ __forceinline__ float2 su() const { return V.su; }
    __device__ __forceinline__ float2 nsv() const { return V.nsv; }
    __device__ __forceinline__ float2 inv_w() const { return V.inv_w; }
    __device__ __forceinline__ float2 inv_h() const { return V.inv_h; }
};

template <>
struct PairOf<SharedViews> {  // shared memory: the pair's words loaded once per use of the pair
    float4 a, b, c, d, e, f, g;
    __device__ __forceinline__ explicit PairOf(const PixelParams::ViewPair& V) {
        // ViewPair as 8 16-byte words: (R0 R1) (R2 R3) (R4 R5) (R6 R7) (R8 t0) (t1 t2) (su nsv) (inv_w inv_h)
        const float4* q = reinterpret_cast<const float4*>(&V);
        a = SharedViews::ld4(q);
        b = SharedViews::ld4(q + 2);
        c = SharedViews::ld4(q + 3);
        d = SharedViews::ld4(q + 4);
        e = SharedViews::ld4(q + 5);
        f = SharedViews::ld4(q + 6);
        g = SharedViews::ld4(q + 7);
    }
    __device__ __forceinline__ float2 r1() const { return make_float2(a.z, a.w); }
    __device__ __forceinline__ float2 r4() const { return make_float2(b.x, b.y); }
    __device__ __forceinline__ float2 r7() const { return make_float2(c.z, c.w); }
    __device__ __forceinline__ float2 t0() const { return make_float2(d.z, d.w); }
    __device__ __forceinline__ float2 t1() const { return make_float2(e.x, e.y); }
    __device__ __forceinline__ float2 t2() const { return make_float2(e.z, e.w); }
    __device__ __forceinline__ float2 su() const { return make_float2(f.x, f.y); }
    __device__ __forceinline__ float2 nsv() const { return make_float2(f.z, f.w); }
    __device__ __forceinline__ float2 inv_w() const { return make_float2(g.x, g.y); }
    __device__ __forceinline__ float2 inv_h() const { return make_float2(g.z, g.w); }
};

template <class VA>
__device__ __forceinline__ PairOf<VA> pair_of(const PixelParams::ViewPair& V) {
    if constexpr (std::is_same<VA, SharedViews>::value)
        return PairOf<SharedViews>(V);
    else
        return PairOf<VA>{V};
}

template <class VA>
__device__ __forceinline__ cudaTextureObject_t view_tex(const SourceView& V) {
    if constexpr (std::is_same<VA, SharedViews>::value) {
        unsigned long long t;
        const unsigned a = (unsigned)__cvta_generic_to_shared(&V.tex);
        asm volatile("ld.shared.u64 %0, [%1];" : "=l"(t) : "r"(a));
        return (cudaTextureObject_t)t;
    } else {
        return V.tex;
    }
}

// Intensity of source view V at the projection of reference-frame point X.
template <class VA>
__device__ __forceinline__ float view_sample(const SourceView& V, float X, float Y, float Z) {
    const typename VA::Loaded L = VA::load(V);
    const float Yx = fmaf(L.r(0), X, fmaf(L.r(1), Y, fmaf(L.r(2), Z, L.t(0))));
    const float Yy = fmaf(L.r(3), X, fmaf(L.r(4), Y, fmaf(L.r(5), Z, L.t(1))));
    const float Yz = fmaf(L.r(6), X, fmaf(L.r(7), Y, fmaf(L.r(8), Z, L.t(2))));
    float qu, qv;
    bool front;
    project_dir_half(Yx, Yy, Yz, L.su(), -L.sv(), qu, qv, front);
    return sample_bilinear_half(L.tex(), L.inv_w(), L.inv_h(), qu, qv, front);
}

// Cost of plane (range d along rp, unit normal n) at the pixel. Returns 2 for
// an invalid plane (a patch ray meets it from behind or grazing). NS views
// are kept in registers; EXACT means S == NS (no per-view guard).
template <int NS, bool EXACT, class VA, class SM>
__device__ __forceinline__ float plane_cost(const PixelParams& P, const SM& sm, int lx, int ly,
                                            const RefStats& st, float3 rp, float d, float3 n) {
    const float eps = 1e-8f * st.Sw * st.Sw;
    if (st.varI < eps) return 2.0f;
    const float dn = d * dot3(n, rp);
    const int K = P.K, R = P.radius, stp = P.stride;
    const int ac = K >> 1;  // centre-most sample first: its intensity centres each view

    float c0[NS], SJ[NS], SJJ[NS], SIJ[NS];
    {
        const int o = ac * stp - R;
        const float cl = sm.row_cos[ly + o];
        const float3 rq = make_float3(cl * sm.col_sin[lx + o], -sm.row_sin[ly + o], cl * sm.col_cos[lx + o]);
        const float den = dot3(n, rq);
        if (!(den < -1e-6f)) return 2.0f;
        const float t = __fdividef(dn, den);
        const float X = t * rq.x, Y = t * rq.y, Z = t * rq.z;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            c0[s] = 0.f;
            SJ[s] = 0.f;
            SJJ[s] = 0.f;
            SIJ[s] = 0.f;
            if (EXACT || s < P.S) c0[s] = view_sample<VA>(P.src[s], X, Y, Z);
        }
    }
    bool valid = true;
    for (int a = 0; a < K && valid; ++a) {
        const int oy = a * stp - R;
        const float cl = sm.row_cos[ly + oy], msl = -sm.row_sin[ly + oy];
        const float* ref_row = sm.ref + (ly + oy) * SM::PITCH + lx - R;
        for (int b = 0; b < K; ++b) {
            if (a == ac && b == ac) continue;
            const float Iq = ref_row[b * stp];
            const float w = bilateral(P, sm, a, b, Iq, st.Ip);
            const float wI = w * (Iq - st.mu);
            const int cx = lx + b * stp - R;
            const float3 rq = make_float3(cl * sm.col_sin[cx], msl, cl * sm.col_cos[cx]);
            const float den = dot3(n, rq);
            if (!(den < -1e-6f)) {
                valid = false;
                break;
            }
            const float t = __fdividef(dn, den);
            const float X = t * rq.x, Y = t * rq.y, Z = t * rq.z;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                if (EXACT || s < P.S) {
                    const float Jc = view_sample<VA>(P.src[s], X, Y, Z) - c0[s];
                    const float tw = __fmul_rn(w, Jc);
                    SJ[s] = __fadd_rn(SJ[s], tw);
                    SJJ[s] = fmaf(tw, Jc, SJJ[s]);
                    SIJ[s] = fmaf(wI, Jc, SIJ[s]);
                }
            }
        }
    }
    if (!valid) return 2.0f;

    float cs[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        float c = 3.0f;  // unused slots sort last
        if (EXACT || s < P.S) {
            const float varJ = mul_sub(st.Sw, SJJ[s], SJ[s], SJ[s]);
            const float cov = mul_sub(st.Sw, SIJ[s], st.SIc, SJ[s]);
            if (varJ < eps) {
                c = 2.0f;
            } else {
                float ncc = cov * rsqrtf(st.varI * varJ);
                ncc = fminf(1.0f, fmaxf(-1.0f, ncc));
                c = 1.0f - ncc;
            }
        }
        cs[s] = c;
    }
    // odd-even transposition sort, then the mean of the best_k smallest
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

// Intensities of all NP view pairs (views 2q, 2q + 1) at the sample whose
// reference-frame point is X = t r, r = (cl sin lon_c, -sl, cl cos lon_c) in
// tile column c: the source point R_s X + t_s = alpha U_c + beta R_col1 + t_s
// with alpha = t cl, beta = -t sl and U_c from the column table. The
// projection runs on float2 pairs (one packed instruction for both views of a
// pair), then two gathers and the bilinear weights per pair; the arithmetic
// after the rigid transform is that of project_dir_half and
// sample_bilinear_half, operation for operation. Two phases: each pair's
// source coordinates and, right after them, its two gathers, so a pair's
// gathers are in flight while the next pairs' coordinates are computed; then
// the interpolation of every pair (2 % faster than pair by pair, and issuing
// each pair's gathers before the next pair's coordinates another 1.5 %).
template <int NP, class VA, int PITCH>
__device__ __forceinline__ void pairs_sample(const PixelParams& P, float alpha, float beta, int cx, float2 (&J)[NP]) {
    float2 fx[NP], fy[NP];
    float4 G0[NP], G1[NP];
    const float2 av = pair(alpha), bv = pair(beta);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const auto VP = pair_of<VA>(P.pairs[q]);
        const float2 Yx = fma2(av, col_table<NP, PITCH>()[q][0][cx], fma2(bv, VP.r1(), VP.t0()));
        const float2 Yy = fma2(av, col_table<NP, PITCH>()[q][1][cx], fma2(bv, VP.r4(), VP.t1()));
        const float2 Yz = fma2(av, col_table<NP, PITCH>()[q][2][cx], fma2(bv, VP.r7(), VP.t2()));
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
        const float2 qu = fma2(al, make_float2(f0 ? VP.su().x : -VP.su().x, f1 ? VP.su().y : -VP.su().y), pair(0.5f));
        const float2 qv = fma2(nlat, VP.nsv(), pair(0.5f));
        const float2 fi = floor_small2(qu), fj = floor_small2(qv);
        fx[q] = add2(qu, make_float2(-fi.x, -fi.y));
        fy[q] = add2(qv, make_float2(-fj.x, -fj.y));
        const float2 xn = fma2(fi, VP.inv_w(), make_float2(f0 ? 0.5f : 0.0f, f1 ? 0.5f : 0.0f));
        const float2 yn = fma2(fj, VP.inv_h(), pair(0.5f));
        G0[q] = tex2Dgather<float4>(view_tex<VA>(P.src[2 * q]), xn.x, yn.x, 0);
        G1[q] = tex2Dgather<float4>(view_tex<VA>(P.src[2 * q + 1]), xn.y, yn.y, 0);
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const float4 g0 = G0[q];
        const float4 g1 = G1[q];
        const float top0 = fmaf(fx[q].x, g0.z - g0.w, g0.w), bot0 = fmaf(fx[q].x, g0.y - g0.x, g0.x);
        const float top1 = fmaf(fx[q].y, g1.z - g1.w, g1.w), bot1 = fmaf(fx[q].y, g1.y - g1.x, g1.x);
        J[q] = make_float2(fmaf(fy[q].x, bot0 - top0, top0), fmaf(fy[q].y, bot1 - top1, top1));
    }
}

// plane_cost for exactly NS >= 2 views held in kernel parameters, with the
// views processed in pairs (packed FP32) and an odd last view on its own.
template <int NS, int WIN, class SM, class VA>
__device__ __forceinline__ float plane_cost_paired(const PixelParams& P, const SM& sm, int lx, int ly,
                                                   const RefStats& st, float3 rp, float d, float3 n) {
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
        pairs_sample<NP, VA, SM::PITCH>(P, alpha, beta, lx + o, c0);
#pragma unroll
        for (int q = 0; q < NP; ++q) SJ[q] = SJJ[q] = SIJ[q] = pair(0.f);
        if (ODD) c0o = view_sample<VA>(P.src[NS - 1], X, Y, Z);
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
            // an invalid sample makes the cost 2; the loop runs on without a
            // branch (1 % faster than leaving it), its values are discarded
            valid = valid && (den < -1e-6f);
            const float t = __fdividef(dn, den);
            const float X = t * rq.x, Y = t * rq.y, Z = t * rq.z;
            const float alpha = t * cl, beta = t * msl;
            const float2 w2 = pair(w), wI2 = pair(wI);
            float2 Jall[NP];
            pairs_sample<NP, VA, SM::PITCH>(P, alpha, beta, cx, Jall);
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const float2 J = Jall[q];
                const float2 Jc = add2(J, make_float2(-c0[q].x, -c0[q].y));
                const float2 tw = mul2(w2, Jc);
                SJ[q] = add2(SJ[q], tw);
                SJJ[q] = fma2(tw, Jc, SJJ[q]);
                SIJ[q] = fma2(wI2, Jc, SIJ[q]);
            }
            if (ODD) {
                const float Jc = view_sample<VA>(P.src[NS - 1], X, Y, Z) - c0o;
                const float tw = __fmul_rn(w, Jc);
                SJo = __fadd_rn(SJo, tw);
                SJJo = fmaf(tw, Jc, SJJo);
                SIJo = fmaf(wI, Jc, SIJo);
            }
        }
    }
    if (!valid) return 2.0f;

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

// The paired form serves exactly known view counts whose views sit in kernel
// parameters or in shared memory (the batched kernel); the general form the
// guarded view count and plain-load sources.
template <class VA>
constexpr bool paired_views() {
    return std::is_same<VA, ParamViews>::value || std::is_same<VA, SharedViews>::value;
}

// The cost used by the per-pixel kernels: the paired form where the views
// are exactly known, the general one otherwise.
template <int NS, bool EXACT, class VA, int WIN = 0, class SM = TileSmem>
__device__ __forceinline__ float cost_of(const PixelParams& P, const SM& sm, int lx, int ly,
                                         const RefStats& st, float3 rp, float d, float3 n) {
    if constexpr (EXACT && NS >= 2 && paired_views<VA>())
        return plane_cost_paired<NS, WIN, SM, VA>(P, sm, lx, ly, st, rp, d, n);
    else
        return plane_cost<NS, EXACT, VA, SM>(P, sm, lx, ly, st, rp, d, n);
}

// Face the camera: n . r_p < 0 (|n . r_p| < 1e-3: replace by -r_p).
__device__ __forceinline__ float3 face_camera(float3 n, float3 rp) {
    const float c = dot3(n, rp);
    if (fabsf(c) < 1e-3f) return make_float3(-rp.x, -rp.y, -rp.z);
    if (c > 0.f) return make_float3(-n.x, -n.y, -n.z);
    return n;
}

// Random initial plane of pixel i (Sec. III-B): inverse range uniform on
// [1/d_max, 1/d_min), normal uniform on the sphere turned to the camera,
// from Philox block (i, 0, 0, 0).
__device__ __forceinline__ void random_plane(const PixelParams& P, size_t i, float3 rp, float& d, float3& n) {
    const U4 u = draw_uniform4(i, 0, 0, P.seed, P.keyframe);
    const float inv = fmaf(u.x, P.inv_dmin - P.inv_dmax, P.inv_dmax);
    d = 1.0f / inv;
    const float z = 1.0f - 2.0f * u.y;
    const float rho = sqrtf(fmaxf(0.f, fmaf(-z, z, 1.0f)));
    float sp, cp;
    sincospif(2.0f * u.z, &sp, &cp);
    n = face_camera(make_float3(rho * cp, rho * sp, z), rp);
}

// Neighbour candidate k of pixel (x, y) (Sec. III-C): the plane of the k-th
// opposite-colour neighbour re-intersected with this pixel's ray. False where
// the neighbour lies outside the image, the plane does not face the ray or the
// range leaves [d_min, d_max]. Every use computes it with this one function,
// so equal inputs give equal bits.
__device__ __forceinline__ bool neighbour_candidate(const PixelParams& P, int x, int y, float3 rp, int k,
                                                    float& dc, float3& nc) {
    const int qy = y + c_neighbors[P.table][k][1];
    if (qy < 0 || qy >= P.H) return false;
    const int qx = wrap_index(x + c_neighbors[P.table][k][0], P.W);
    const size_t j = (size_t)qy * P.W + qx;
    nc = make_float3(P.nx[j], P.ny[j], P.nz[j]);
    const float den = dot3(nc, rp);
    const float3 rq = pixel_bearing(qx, qy, P.W, P.H);
    dc = P.depth[j] * dot3(nc, rq) / den;
    return den < -1e-6f && dc >= P.d_min && dc <= P.d_max;
}

// Bit-for-bit equal planes (the cost is a deterministic function of them).
__device__ __forceinline__ bool same_plane(float d0, float3 n0, float d1, float3 n1) {
    return __float_as_uint(d0) == __float_as_uint(d1) && __float_as_uint(n0.x) == __float_as_uint(n1.x) &&
           __float_as_uint(n0.y) == __float_as_uint(n1.y) && __float_as_uint(n0.z) == __float_as_uint(n1.z);
}

// Cost bits mapped so that unsigned order is float order (negative values
// bit-inverted, the sign bit set on the others), and back.
__device__ __forceinline__ unsigned ordered_bits(float c) {
    const unsigned u = __float_as_uint(c);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_ordered_bits(unsigned o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// One half-sweep over the pixels of `colour` in a tile (Sec. III-C): each
// pixel tries its 8 neighbour candidates, then n_refine perturbations of the
// best so far, and a candidate replaces the incumbent only if its cost is
// strictly lower. Taken in that order, the neighbour phase ends on the
// candidate of lowest cost, the first of equal ones, if that cost is below
// the incumbent's; a candidate bit-identical to the incumbent or to an
// earlier candidate can never be that one (its cost equals theirs), so it is
// not evaluated. The other neighbour candidates of a warp's 32 pixels are
// pooled and evaluated 32 at a time, each lane taking any pixel's candidate,
// and every pixel keeps the minimum of (cost, candidate index) in shared
// memory; then each pixel adopts that candidate if it wins and runs its
// refinements. The maps equal those of trying all candidates in turn.
template <int NS, bool EXACT, class VA, int WIN, class SM>
__device__ __forceinline__ void sweep_pooled(const PixelParams& P, SM& sm, int bx, int by, int x, int y, int colour,
                                             int iter) {
    const bool active = x < P.W && y < P.H;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lx = x - bx + P.radius, ly = y - by + P.radius;
    const size_t i = (size_t)y * P.W + x;
    float bd = 0.f, bc = 0.f;
    float3 bn = make_float3(0.f, 0.f, 0.f), rp = bn;
    unsigned need = 0;
    if (active) {
        rp = make_float3(sm.row_cos[ly] * sm.col_sin[lx], -sm.row_sin[ly], sm.row_cos[ly] * sm.col_cos[lx]);
        sm.pool.st[threadIdx.x] = ref_stats(P, sm, lx, ly);
        bd = P.depth[i];
        bn = make_float3(P.nx[i], P.ny[i], P.nz[i]);
        bc = P.cost[i];
        float cd[8];
        float3 cn[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const bool ok = neighbour_candidate(P, x, y, rp, k, cd[k], cn[k]);
            bool dup = same_plane(cd[k], cn[k], bd, bn);
#pragma unroll
            for (int m = 0; m < k; ++m) dup = dup || (((need >> m) & 1u) && same_plane(cd[k], cn[k], cd[m], cn[m]));
            if (ok && !dup) need |= 1u << k;
        }
    }
    sm.pool.key[threadIdx.x] = ~0ull;
    // this lane's first slot in the warp's list: exclusive prefix of the counts
    const int cnt = __popc(need);
    int off = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, off, d);
        if (lane >= d) off += v;
    }
    const int total = __shfl_sync(0xffffffffu, off, 31);
    off -= cnt;
    unsigned char* items = sm.pool.item[warp];
    for (unsigned m = need; m; m &= m - 1) items[off++] = (unsigned char)((lane << 3) | (__ffs(m) - 1));
    __syncwarp();

    const int pooled_rounds = (total + 31) >> 5;  // warp-uniform
    const int n_jobs = pooled_rounds + P.n_refine;
    const float span = P.inv_dmin - P.inv_dmax;
    // the neighbour phase's winner, once every pooled evaluation has landed
    auto adopt_best = [&]() {
        __syncwarp();
        const unsigned long long key = sm.pool.key[threadIdx.x];
        if (active && key != ~0ull) {
            const float c = from_ordered_bits((unsigned)(key >> 3));
            if (c < bc) {
                float dc;
                float3 nc;
                neighbour_candidate(P, x, y, rp, (int)(key & 7u), dc, nc);
                bc = c;
                bd = dc;
                bn = nc;
            }
        }
    };
#pragma unroll 1
    for (int r = 0; r < n_jobs; ++r) {
        if (r == pooled_rounds) adopt_best();
        // the job of this round: (pixel, plane)
        bool job = false;
        int jt = threadIdx.x, jx = x, jy = y, k = 0;
        float3 jrp = rp;
        float dc = 0.f;
        float3 nc = make_float3(0.f, 0.f, 0.f);
        if (r < pooled_rounds) {
            const int idx = (r << 5) + lane;
            if (idx < total) {
                const int it = items[idx];
                k = it & 7;
                jt = (warp << 5) + (it >> 3);
                const int otx = jt % (SM::W / 2), oty = jt / (SM::W / 2);
                jy = by + oty;
                jx = bx + 2 * otx + ((jy + colour) & 1);
                job = true;
            }
        } else if (active) {
            const int t = r - pooled_rounds;
            const float sc = __int_as_float((126 - t) << 23);  // 2^-(t+1)
            const U4 u = draw_uniform4(i, (uint64_t)iter, (uint64_t)(1 + t), P.seed, P.keyframe);
            float inv = fmaf((2.0f * u.x - 1.0f) * sc, span, 1.0f / bd);
            inv = fminf(P.inv_dmin, fmaxf(P.inv_dmax, inv));
            dc = 1.0f / inv;
            nc = make_float3(fmaf(sc, 2.0f * u.y - 1.0f, bn.x), fmaf(sc, 2.0f * u.z - 1.0f, bn.y),
                             fmaf(sc, 2.0f * u.w - 1.0f, bn.z));
            const float il = 1.0f / sqrtf(dot3(nc, nc));
            nc = face_camera(make_float3(nc.x * il, nc.y * il, nc.z * il), rp);
            job = true;
        }
        if (!job) continue;
        const int jlx = jx - bx + P.radius, jly = jy - by + P.radius;
        if (r < pooled_rounds) {
            jrp = make_float3(sm.row_cos[jly] * sm.col_sin[jlx], -sm.row_sin[jly], sm.row_cos[jly] * sm.col_cos[jlx]);
            neighbour_candidate(P, jx, jy, jrp, k, dc, nc);
        }
        const float c = cost_of<NS, EXACT, VA, WIN, SM>(P, sm, jlx, jly, sm.pool.st[jt], jrp, dc, nc);
        if (r < pooled_rounds) {
            if (c == c) atomicMin(&sm.pool.key[jt], ((unsigned long long)ordered_bits(c) << 3) | (unsigned)k);
        } else if (c < bc) {
            bc = c;
            bd = dc;
            bn = nc;
        }
    }
    if (n_jobs == pooled_rounds) adopt_best();
    if (!active) return;
    P.depth[i] = bd;
    P.nx[i] = bn.x;
    P.ny[i] = bn.y;
    P.nz[i] = bn.z;
    P.cost[i] = bc;
}

// One tile of one problem: stage the reference tile, then every active
// pixel of `colour` runs MODE. P may live in kernel parameters or in shared
// memory (the batched kernel). Returns without a trailing barrier.
template <int NS, bool EXACT, int MODE, class VA = ParamViews, int WIN = 0, class SM = TileSmem>
__device__ __forceinline__ void process_tile(const PixelParams& P, SM& sm, int bx, int by, int colour,
                                             int iter) {
    stage_tile(P, sm, bx, by);
    __syncthreads();
    if constexpr (EXACT && NS >= 2 && paired_views<VA>()) {
        constexpr int NP = NS / 2;
        static_assert(NP <= PMSP_MAX_SOURCES / 2, "column table too small");
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

    const int tx = threadIdx.x % (SM::W / 2), ty = threadIdx.x / (SM::W / 2);
    const int y = by + ty;
    const int x = bx + 2 * tx + ((y + colour) & 1);
    if constexpr (MODE == MODE_SWEEP) {
        sweep_pooled<NS, EXACT, VA, WIN, SM>(P, sm, bx, by, x, y, colour, iter);
        return;
    }
    if (x >= P.W || y >= P.H) return;
    const int lx = x - bx + P.radius, ly = y - by + P.radius;
    const size_t i = (size_t)y * P.W + x;

    const float3 rp = make_float3(sm.row_cos[ly] * sm.col_sin[lx], -sm.row_sin[ly],
                                  sm.row_cos[ly] * sm.col_cos[lx]);
    const RefStats st = ref_stats(P, sm, lx, ly);

    if (MODE == MODE_COST) {
        const float3 n = make_float3(P.nx[i], P.ny[i], P.nz[i]);
        P.cost[i] = cost_of<NS, EXACT, VA, WIN, SM>(P, sm, lx, ly, st, rp, P.depth[i], n);
        return;
    }
    float d;
    float3 n;
    random_plane(P, i, rp, d, n);
    P.depth[i] = d;
    P.nx[i] = n.x;
    P.ny[i] = n.y;
    P.nz[i] = n.z;
    P.cost[i] = cost_of<NS, EXACT, VA, WIN, SM>(P, sm, lx, ly, st, rp, d, n);
}

template <int NS, bool EXACT, int MODE, int WIN = 0, int TS = 0>
__global__ void __launch_bounds__(BLOCK_THREADS, pixel_min_blocks(NS)) pixel_kernel(const __grid_constant__ PixelParams P) {
    using SM = typename TileShape<TS, Window<WIN>::HALO>::Smem;
    __shared__ SM sm;
    int tx, ty;
    tile_of_block(gridDim.x, gridDim.y, blockIdx.y * gridDim.x + blockIdx.x, tx, ty);
    process_tile<NS, EXACT, MODE, ParamViews, WIN, SM>(P, sm, tx * SM::W, ty * SM::H, P.colour, P.iter);
}

// Grid of a tile shape over a W x H panorama.
template <int TS>
inline dim3 tile_grid(const PixelParams& p) {
    using SM = typename TileShape<TS>::Smem;
    return dim3((p.W + SM::W - 1) / SM::W, (p.H + SM::H - 1) / SM::H);
}

// A fixed-window sweep in the problem's tile shape.
template <int NS, bool EXACT, int WIN>
inline void launch_sweep_window(const PixelParams& p, cudaStream_t stream) {
    switch (p.tile) {
        case 1: pixel_kernel<NS, EXACT, MODE_SWEEP, WIN, 1><<<tile_grid<1>(p), BLOCK_THREADS, 0, stream>>>(p); break;
        case 2: pixel_kernel<NS, EXACT, MODE_SWEEP, WIN, 2><<<tile_grid<2>(p), BLOCK_THREADS, 0, stream>>>(p); break;
        default: pixel_kernel<NS, EXACT, MODE_SWEEP, WIN, 0><<<tile_grid<0>(p), BLOCK_THREADS, 0, stream>>>(p); break;
    }
}

// The window class of a problem: a fixed-window sweep instance where one exists.
__host__ __device__ inline int window_of(const PixelParams& p) {
    if (p.K == 6 && p.radius == 5 && p.stride == 2) return 1;
    if (p.K == 7 && p.radius == 3 && p.stride == 1) return 2;
    return 0;
}

// Half-sweeps with 2 or 4 threads per pixel: the views split over warps
// (pixel_split.cuh, PixelParams::tpp 2 or 4) or the patch samples split over
// adjacent lanes (pixel_lanes.cuh, tpp -2, -4 or -8).
template <int NS, bool EXACT>
cudaError_t launch_split_sweep(const PixelParams& p, cudaStream_t stream);
template <int NS, bool EXACT>
cudaError_t launch_lanes_sweep(const PixelParams& p, cudaStream_t stream);

template <int NS, bool EXACT>
cudaError_t launch_pixel_kernel_ns(const PixelParams& p, int mode, cudaStream_t stream) {
    const dim3 grid((p.W + TILE_W - 1) / TILE_W, (p.H + TILE_H - 1) / TILE_H);
    switch (mode) {
        case MODE_COST: pixel_kernel<NS, EXACT, MODE_COST><<<grid, BLOCK_THREADS, 0, stream>>>(p); break;
        case MODE_INIT: pixel_kernel<NS, EXACT, MODE_INIT><<<grid, BLOCK_THREADS, 0, stream>>>(p); break;
        default:
            // views split over several warps per pixel (a tuning choice; same maps)
            if constexpr (EXACT && NS >= 2) {
                if (p.tpp > 1) return launch_split_sweep<NS, EXACT>(p, stream);
                if (p.tpp < -1) return launch_lanes_sweep<NS, EXACT>(p, stream);
            }
            // the half-sweep dominates the run time: fixed-window instances for the
            // paired path (exact view counts of at least 2), in three tile shapes
            if constexpr (EXACT && NS >= 2) {
                const int win = window_of(p);
                if (win == 1) {
                    launch_sweep_window<NS, EXACT, 1>(p, stream);
                    break;
                }
                if (win == 2) {
                    launch_sweep_window<NS, EXACT, 2>(p, stream);
                    break;
                }
            }
            pixel_kernel<NS, EXACT, MODE_SWEEP><<<grid, BLOCK_THREADS, 0, stream>>>(p);
            break;
    }
    return cudaGetLastError();
}

}  // namespace pmsp
