// Point kernels around the densification path: the View Filter on sparse
// points (paper Sec. III-A, Eq. 1), dense point-cloud fusion with duplicate
// erasure (Sec. III) and keyframe completeness (Sec. IV).
//
// View Filter: one thread per point computes the cosine of the parallax angle
//   between the rays to the two camera centres and tests it against the cosines
//   of the angle bounds; in-range points are counted with a warp ballot and one
//   atomic add per warp.
// Fusion: every valid pixel of every keyframe is lifted to a world point and
//   binned into a cubic voxel; an open-addressing hash table (linear probing,
//   64-bit packed voxel keys) keeps per voxel the smallest (keyframe, pixel)
//   order by an atomic minimum. A second pass marks the pixels that are their
//   voxel's first point, an exclusive scan over the marks gives output slots,
//   and the marked points are written in (keyframe, pixel) order, so the
//   output does not depend on thread timing.
// Completeness: one thread per point projects into a W x H panorama and sets
//   the nearest pixel's flag; a reduction counts the flags.
#include "camera.cuh"
#include "common.cuh"

namespace pmsp {

namespace {

constexpr unsigned long long EMPTY = ~0ull;
constexpr int KEY_BITS = 21;
constexpr long long KEY_HALF = 1ll << (KEY_BITS - 1);

__device__ __forceinline__ float3 lift_world(const CloudView& V, int u, int v, float d) {
    const float3 r = pixel_bearing(u, v, V.W, V.H);
    const float x = fmaf(d, r.x, -V.t[0]), y = fmaf(d, r.y, -V.t[1]), z = fmaf(d, r.z, -V.t[2]);
    // X = R^T (d r - t)
    return make_float3(fmaf(V.R[0], x, fmaf(V.R[3], y, V.R[6] * z)), fmaf(V.R[1], x, fmaf(V.R[4], y, V.R[7] * z)),
                       fmaf(V.R[2], x, fmaf(V.R[5], y, V.R[8] * z)));
}

// Packed voxel key (21 bits per axis, offset binary); false if out of range.
__device__ __forceinline__ bool voxel_key(float3 X, float inv_voxel, unsigned long long& key) {
    const float q[3] = {floorf(X.x * inv_voxel), floorf(X.y * inv_voxel), floorf(X.z * inv_voxel)};
    key = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (!(q[a] >= -(float)KEY_HALF && q[a] < (float)KEY_HALF)) return false;
        key = (key << KEY_BITS) | (unsigned long long)((long long)q[a] + KEY_HALF);
    }
    return true;
}

__device__ __forceinline__ unsigned long long hash_slot(unsigned long long key, unsigned long long mask) {
    key ^= key >> 33;
    key *= 0xff51afd7ed558ccdull;
    key ^= key >> 33;
    key *= 0xc4ceb9fe1a85ec53ull;
    key ^= key >> 33;
    return key & mask;
}

__global__ void fuse_insert_kernel(const __grid_constant__ FuseArgs A, int k) {
    const CloudView& V = A.views[k];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V.W * V.H) return;
    const float d = V.depth[i];
    if (!(d > 0.f)) return;
    const float3 X = lift_world(V, i % V.W, i / V.W, d);
    unsigned long long key;
    if (!voxel_key(X, A.inv_voxel, key)) {
        atomicOr(A.err, ERR_RANGE);
        return;
    }
    const unsigned long long order = ((unsigned long long)k << 32) | (unsigned)i;
    unsigned long long s = hash_slot(key, A.mask);
    for (unsigned long long probe = 0; probe <= A.mask; ++probe) {  // bounded: at most one pass over the table
        const unsigned long long prev = atomicCAS(A.keys + s, EMPTY, key);
        if (prev == EMPTY || prev == key) {
            atomicMin(A.vals + s, order);
            return;
        }
        s = (s + 1) & A.mask;
    }
    atomicOr(A.err, ERR_CAPACITY);
}

__global__ void fuse_mark_kernel(const __grid_constant__ FuseArgs A, int k, unsigned* mark) {
    const CloudView& V = A.views[k];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V.W * V.H) return;
    unsigned m = 0;
    const float d = V.depth[i];
    if (d > 0.f) {
        const float3 X = lift_world(V, i % V.W, i / V.W, d);
        unsigned long long key;
        if (voxel_key(X, A.inv_voxel, key)) {
            const unsigned long long order = ((unsigned long long)k << 32) | (unsigned)i;
            unsigned long long s = hash_slot(key, A.mask);
            for (unsigned long long probe = 0; probe <= A.mask; ++probe) {
                const unsigned long long kk = A.keys[s];
                if (kk == key) {
                    m = A.vals[s] == order;
                    break;
                }
                if (kk == EMPTY) break;
                s = (s + 1) & A.mask;
            }
        }
    }
    mark[A.base[k] + i] = m;
}

// Exclusive scan of n marks in three passes: per-block sums, a single-block
// scan of the block sums, then per-block scans offset by their block's sum.
constexpr int SCAN_BLOCK = 1024;

__device__ __forceinline__ unsigned block_exclusive_scan(unsigned x, unsigned* warp_sums, unsigned& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[w] = incl;
    __syncthreads();
    if (w == 0) {
        unsigned s = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s;  // inclusive prefix of warp sums
    }
    __syncthreads();
    total = warp_sums[(blockDim.x >> 5) - 1];
    const unsigned before = w > 0 ? warp_sums[w - 1] : 0;
    return before + incl - x;
}

__global__ void __launch_bounds__(SCAN_BLOCK) scan_block_sums(const unsigned* mark, long long n, unsigned* sums) {
    __shared__ unsigned ws[32];
    const long long i = (long long)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    const unsigned x = i < n ? mark[i] : 0;
    unsigned total;
    block_exclusive_scan(x, ws, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// One block: exclusive scan of nb block sums in place (chunks of SCAN_BLOCK);
// total written to *count.
__global__ void __launch_bounds__(SCAN_BLOCK) scan_sums(unsigned* sums, int nb, unsigned long long* count) {
    __shared__ unsigned ws[32];
    unsigned carry = 0;
    for (int c = 0; c < nb; c += SCAN_BLOCK) {
        const int i = c + threadIdx.x;
        const unsigned x = i < nb ? sums[i] : 0;
        unsigned total;
        const unsigned ex = block_exclusive_scan(x, ws, total);
        if (i < nb) sums[i] = carry + ex;
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = carry;
}

__global__ void __launch_bounds__(SCAN_BLOCK) scan_apply(unsigned* mark, long long n, const unsigned* sums) {
    __shared__ unsigned ws[32];
    const long long i = (long long)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    const unsigned x = i < n ? mark[i] : 0;
    unsigned total;
    const unsigned ex = block_exclusive_scan(x, ws, total);
    // marks become output positions + 1 (0: not kept)
    if (i < n) mark[i] = x ? sums[blockIdx.x] + ex + 1 : 0;
}

__global__ void fuse_write_kernel(const __grid_constant__ FuseArgs A, int k, const unsigned* pos) {
    const CloudView& V = A.views[k];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V.W * V.H) return;
    const unsigned p = pos[A.base[k] + i];
    if (p == 0 || (long long)(p - 1) >= A.cap) return;
    const float3 X = lift_world(V, i % V.W, i / V.W, V.depth[i]);
    float* o = A.points + 3 * (size_t)(p - 1);
    o[0] = X.x;
    o[1] = X.y;
    o[2] = X.z;
    if (A.src) A.src[p - 1] = (long long)(((unsigned long long)k << 32) | (unsigned)i);
}

__global__ void completeness_kernel(const __grid_constant__ CompletenessArgs A) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    const float* p = A.points + 3 * i;
    const float X = p[0], Y = p[1], Z = p[2];
    const float y0 = fmaf(A.R[0], X, fmaf(A.R[1], Y, fmaf(A.R[2], Z, A.t[0])));
    const float y1 = fmaf(A.R[3], X, fmaf(A.R[4], Y, fmaf(A.R[5], Z, A.t[1])));
    const float y2 = fmaf(A.R[6], X, fmaf(A.R[7], Y, fmaf(A.R[8], Z, A.t[2])));
    if (y0 == 0.f && y1 == 0.f && y2 == 0.f) return;  // at the camera centre: no direction
    float uc, vc;
    project_dir_fast(y0, y1, y2, A.su, A.ou, A.sv, A.ov, uc, vc);
    int u = (int)floorf(uc + 0.5f) % A.W;
    if (u < 0) u += A.W;
    int v = (int)floorf(vc + 0.5f);
    v = v < 0 ? 0 : (v > A.H - 1 ? A.H - 1 : v);
    A.hit[(size_t)v * A.W + u] = 1;
}

__global__ void count_hits_kernel(const unsigned char* hit, long long n, unsigned long long* count) {
    unsigned c = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        c += hit[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
}

__global__ void view_filter_kernel(const __grid_constant__ ViewFilterArgs A) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool ok = false;
    if (i < A.n) {
        const float* p = A.points + 3 * i;
        const float ax = A.ca[0] - p[0], ay = A.ca[1] - p[1], az = A.ca[2] - p[2];
        const float bx = A.cb[0] - p[0], by = A.cb[1] - p[1], bz = A.cb[2] - p[2];
        const float la = fmaf(ax, ax, fmaf(ay, ay, az * az)), lb = fmaf(bx, bx, fmaf(by, by, bz * bz));
        if (la > 0.f && lb > 0.f) {
            const float c = fmaf(ax, bx, fmaf(ay, by, az * bz)) / sqrtf(la * lb);
            ok = c >= A.cos_max && c <= A.cos_min;  // theta in [min, max] <=> cos in [cos max, cos min]
        }
        if (A.flags) A.flags[i] = ok;
    }
    const unsigned votes = __ballot_sync(0xffffffffu, ok);
    if ((threadIdx.x & 31) == 0 && votes) atomicAdd(A.count, (unsigned long long)__popc(votes));
}

}  // namespace

cudaError_t launch_fuse(const FuseArgs& a, int n, unsigned* mark, unsigned* sums, long long total,
                        unsigned long long* count, cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(a.keys, 0xff, (a.mask + 1) * sizeof(unsigned long long), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.vals, 0xff, (a.mask + 1) * sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < n; ++k) {
        const int px = a.views[k].W * a.views[k].H;
        fuse_insert_kernel<<<(px + 255) / 256, 256, 0, stream>>>(a, k);
    }
    for (int k = 0; k < n; ++k) {
        const int px = a.views[k].W * a.views[k].H;
        fuse_mark_kernel<<<(px + 255) / 256, 256, 0, stream>>>(a, k, mark);
    }
    const int nb = (int)((total + SCAN_BLOCK - 1) / SCAN_BLOCK);
    scan_block_sums<<<nb, SCAN_BLOCK, 0, stream>>>(mark, total, sums);
    scan_sums<<<1, SCAN_BLOCK, 0, stream>>>(sums, nb, count);
    scan_apply<<<nb, SCAN_BLOCK, 0, stream>>>(mark, total, sums);
    for (int k = 0; k < n; ++k) {
        const int px = a.views[k].W * a.views[k].H;
        fuse_write_kernel<<<(px + 255) / 256, 256, 0, stream>>>(a, k, mark);
    }
    return cudaGetLastError();
}

cudaError_t launch_completeness(const CompletenessArgs& a, unsigned long long* count, cudaStream_t stream) {
    const size_t px = (size_t)a.W * a.H;
    cudaError_t e = cudaMemsetAsync(a.hit, 0, px, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof *count, stream);
    if (e != cudaSuccess) return e;
    if (a.n > 0) completeness_kernel<<<(unsigned)((a.n + 255) / 256), 256, 0, stream>>>(a);
    count_hits_kernel<<<(unsigned)std::min<size_t>((px + 255) / 256, 4096), 256, 0, stream>>>(a.hit, (long long)px,
                                                                                          count);
    return cudaGetLastError();
}

cudaError_t launch_view_filter(const ViewFilterArgs& a, cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(a.count, 0, sizeof *a.count, stream);
    if (e != cudaSuccess) return e;
    if (a.n > 0) view_filter_kernel<<<(unsigned)((a.n + 255) / 256), 256, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace pmsp
