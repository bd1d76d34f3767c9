// Persistent batched densification kernel: one launch runs one phase
// (initialisation colour 0/1 or a half-sweep) for the tiles of many
// keyframes of different sizes and view counts. Blocks pull work items
// (problem, tile, phase) from a list with an atomic counter until the list
// is exhausted, so the loop is bounded by the list length; there is no
// inter-block waiting. Each problem's parameters are copied into shared
// memory when a block moves to a new problem, and the per-pixel code is the
// same as the single-keyframe kernels', so a keyframe gives bit-identical
// results alone or in a batch.
#pragma once

#include "pixel_kernel.cuh"

namespace pmsp {

static_assert(sizeof(PixelParams) % 16 == 0, "PixelParams must be copied as 16-byte words");

template <int NS, bool EXACT>
__device__ __forceinline__ void run_item(const PixelParams& P, TileSmem& sm, int bx, int by, int phase) {
    const int colour = phase & 1;
    if (phase < 2)
        process_tile<NS, EXACT, MODE_INIT, SharedViews>(P, sm, bx, by, colour, 0);
    else
        process_tile<NS, EXACT, MODE_SWEEP, SharedViews>(P, sm, bx, by, colour, (phase - 2) >> 1);
}

// MAXS bounds the view counts this instance handles: the kernel's register
// budget is the largest of its per-view-count variants, so batches of few
// views use a leaner instance.
template <int MAXS>
__global__ void __launch_bounds__(BLOCK_THREADS, min_blocks_for(MAXS)) batch_kernel(const __grid_constant__ BatchArgs B) {
    __shared__ TileSmem sm;
    __shared__ __align__(16) PixelParams sp;
    __shared__ int s_item, s_prob;
    if (threadIdx.x == 0) s_prob = -1;
    for (;;) {
        __syncthreads();  // the previous item is finished with sm and sp
        if (threadIdx.x == 0) s_item = (int)atomicAdd(B.counter, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= B.n_work) break;
        const int4 w = B.work[it];  // (problem, tile x0, tile y0, phase)
        if (w.x != s_prob) {
            const int4* src = reinterpret_cast<const int4*>(B.problems + w.x);
            int4* dst = reinterpret_cast<int4*>(&sp);
            for (int k = threadIdx.x; k < (int)(sizeof(PixelParams) / 16); k += BLOCK_THREADS) dst[k] = src[k];
            __syncthreads();
            if (threadIdx.x == 0) s_prob = w.x;
        }
        const int phase = B.phase >= 0 ? B.phase : (B.phase == -1 ? w.w : sp.phase);
        const int S = sp.S;
        if (S <= 1) run_item<1, true>(sp, sm, w.y, w.z, phase);
        else if (S == 2) run_item<2, true>(sp, sm, w.y, w.z, phase);
        else if (S == 3) run_item<3, true>(sp, sm, w.y, w.z, phase);
        else if (S == 4) run_item<4, true>(sp, sm, w.y, w.z, phase);
        else if (MAXS >= 6 && S == 5) run_item<(MAXS >= 6 ? 5 : 1), true>(sp, sm, w.y, w.z, phase);
        else if (MAXS >= 6 && S == 6) run_item<(MAXS >= 6 ? 6 : 1), true>(sp, sm, w.y, w.z, phase);
        else if (MAXS >= 8 && S == 7) run_item<(MAXS >= 8 ? 7 : 1), true>(sp, sm, w.y, w.z, phase);
        else if (MAXS >= 8 && S == 8) run_item<(MAXS >= 8 ? 8 : 1), true>(sp, sm, w.y, w.z, phase);
        else if (MAXS >= 10 && S == 9) run_item<(MAXS >= 10 ? 9 : 1), true>(sp, sm, w.y, w.z, phase);
        else if (MAXS >= 10 && S == 10) run_item<(MAXS >= 10 ? 10 : 1), true>(sp, sm, w.y, w.z, phase);
        else if (MAXS > 10) run_item<(MAXS > 10 ? 16 : 1), false>(sp, sm, w.y, w.z, phase);
    }
}

template <int MAXS>
int batch_kernel_blocks_per_sm_t() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<MAXS>, BLOCK_THREADS, 0) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

template <int MAXS>
cudaError_t launch_batch_kernel_t(const BatchArgs& a, int grid, cudaStream_t stream) {
    if (a.n_work <= 0) return cudaSuccess;
    batch_kernel<MAXS><<<grid, BLOCK_THREADS, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace pmsp
