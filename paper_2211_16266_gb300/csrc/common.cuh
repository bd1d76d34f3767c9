// Shared device-side declarations of the densification kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pmsp.h"
#include "tile_order.h"

namespace pmsp {

// Tile of reference pixels handled by one block: TILE_W x TILE_H pixels, of
// which one colour (half of them) is active in a half-sweep; one thread per
// active pixel.
constexpr int TILE_W = 32;
constexpr int TILE_H = 8;
constexpr int BLOCK_THREADS = (TILE_W / 2) * TILE_H;
constexpr int MAX_HALO = (PMSP_MAX_PATCH_W - 1) / 2;

// Error bits written to the device error word.
constexpr unsigned ERR_BAD_INDEX = 1u;
constexpr unsigned ERR_RANGE = 2u;     // a fused point lies outside the voxel key range
constexpr unsigned ERR_CAPACITY = 4u;  // a hash table ran out of slots

// One source view as the kernels see it: its texture, the reference->source
// rotation R (row-major) and translation t, and the projection scales with
// u_c = lon * su + ou, v_c = lat * sv + ov.
// 80 bytes; inside PixelParams every view starts on a 16-byte boundary, so the
// batched kernel can copy it as five 16-byte words. (This field order measured
// 9 % faster in the single-keyframe kernel than rows-with-translation layouts.)
struct SourceView {
    cudaTextureObject_t tex;  // gather-capable texture: x wraps, y clamps, normalised coords
    float R[9];               // reference camera -> source camera rotation, row-major
    float t[3];
    float su, ou;             // u_c = lon * su + ou
    float sv, ov;             // v_c = lat * sv + ov
    float inv_w, inv_h;       // 1/W, 1/H of this source
};
static_assert(sizeof(SourceView) == 80, "SourceView is copied as five 16-byte words");

enum Mode : int { MODE_COST = 0, MODE_INIT = 1, MODE_SWEEP = 2 };

struct alignas(16) PixelParams {
    SourceView src[PMSP_MAX_SOURCES];
    const uint8_t* ref;   // reference image, linear, row pitch ref_pitch bytes
    int64_t ref_pitch;
    int ref_format;       // pmsp_format
    int W, H;
    float* depth;         // state planes, W*H each
    float* nx;
    float* ny;
    float* nz;
    float* cost;
    float d_min, d_max;
    float inv_dmin, inv_dmax;
    int S;                // number of sources
    int K;                // samples per window axis
    int stride;           // sample step (pixels)
    int radius;           // (patch_w - 1) / 2
    int best_k;
    int n_refine;
    int table;            // neighbour table id
    float wc;             // -log2(e) / (2 sigma_c^2), 0 when off
    float ws;             // -log2(e) / (2 sigma_s^2), 0 when off
    unsigned long long seed, keyframe;
    int phase;            // batched serving: 0,1 initialisation colours, 2 + 2 t + c half-sweep (t, c)
    int tile;             // tile shape of the single-keyframe half-sweep: 0 32x8, 1 64x4, 2 16x16
    int tpp;              // threads per pixel of the single-keyframe half-sweep: 1; 2 or 4 warps
                          // (views split); -2, -4 or -8: adjacent lanes (patch samples split)
    int colour;
    int iter;
    unsigned* err;
    // Constants of views (2p, 2p + 1) interleaved, so one packed FP32
    // instruction reads the same constant of both views (an odd last view is
    // paired with itself). 16-byte aligned: the batched kernel reads a pair
    // from shared memory as 16-byte words.
    struct alignas(16) ViewPair {
        float2 R[9];
        float2 t[3];
        float2 su, nsv;    // nsv = -sv: the paired projection computes -lat
        float2 inv_w, inv_h;
    } pairs[PMSP_MAX_SOURCES / 2];
};

struct FilterView {
    const float* depth;  // neighbour range map, W x H
    int W, H;
    float Rf[9], tf[3];  // reference -> neighbour
    float Rb[9], tb[3];  // neighbour -> reference
};

struct FilterParams {
    FilterView nb[PMSP_MAX_SOURCES];
    const float* depth_in;
    float* depth_out;
    int32_t* agree;
    int W, H, n, min_views;
    float max_px;
};

// Plane-map warping from the previous keyframe into the current one.
struct WarpArgs {
    const float* prev_depth;   // Wp x Hp, 0 = no plane
    const float* prev_normal;  // 3 planes of Wp x Hp, previous camera frame
    int Wp, Hp;
    float R[9], t[3];          // previous camera -> current camera
    int W, H;                  // current panorama
    float su, ou, sv, ov;      // current projection scales
    unsigned long long* zbuf;  // W x H claims (range bits << 32 | previous pixel)
    int* src;                  // optional: winning previous pixel or -1
};

// One keyframe's depth map and pose for point-cloud fusion.
struct CloudView {
    const float* depth;  // W x H ranges, <= 0: no point
    int W, H;
    float R[9], t[3];    // world -> camera
};

constexpr int MAX_FUSE_VIEWS = PMSP_MAX_SOURCES;

struct FuseArgs {
    CloudView views[MAX_FUSE_VIEWS];
    long long base[MAX_FUSE_VIEWS];  // offset of each keyframe's pixels in the mark array
    float inv_voxel;
    unsigned long long* keys;        // hash table: packed voxel keys, ~0 = empty
    unsigned long long* vals;        // smallest (keyframe << 32 | pixel) per voxel
    unsigned long long mask;         // table capacity - 1 (capacity a power of two)
    float* points;                   // output: 3 floats per kept point
    long long* src;                  // output (optional): keyframe << 32 | pixel
    long long cap;                   // output capacity in points
    unsigned* err;
};

struct CompletenessArgs {
    const float* points;  // 3 floats per point, world frame
    long long n;
    float R[9], t[3];     // world -> camera
    int W, H;
    float su, ou, sv, ov;
    unsigned char* hit;   // W x H flags
};

struct ViewFilterArgs {
    const float* points;  // 3 floats per point, world frame
    long long n;
    float ca[3], cb[3];   // camera centres
    float cos_min, cos_max;  // cos(min angle), cos(max angle)
    unsigned char* flags;    // optional, n
    unsigned long long* count;
};

// Arguments of one launch of the persistent batched kernel.
struct BatchArgs {
    const PixelParams* problems;  // device array, one per keyframe
    const int4* work;             // (problem, tile x0, tile y0, phase) items
    int n_work;
    int phase;                    // >= 0: phase of every item; -1: each item's own; -2: each problem's own
    unsigned* counter;            // work-item counter, zero before the launch
};

// Launchers. The batched kernel comes in instances for at most
// MAXS in {4, 6, 8, 10, 16} views (batch_s<MAXS>.cu).
template <int MAXS>
int batch_kernel_blocks_per_sm_t();
template <int MAXS>
cudaError_t launch_batch_kernel_t(const BatchArgs& a, int grid, cudaStream_t stream);
cudaError_t launch_pixel_kernel(const PixelParams& p, int mode, cudaStream_t stream);
cudaError_t launch_filter_kernel(const FilterParams& p, cudaStream_t stream);
cudaError_t launch_median_kernel(const float* in, float* out, int W, int H, int radius, float tau,
                                 cudaStream_t stream);
cudaError_t launch_warp_init(const PixelParams& p, const WarpArgs& a, cudaStream_t stream);
cudaError_t launch_fuse(const FuseArgs& a, int n, unsigned* mark, unsigned* sums, long long total,
                        unsigned long long* count, cudaStream_t stream);
cudaError_t launch_completeness(const CompletenessArgs& a, unsigned long long* count, cudaStream_t stream);
cudaError_t launch_view_filter(const ViewFilterArgs& a, cudaStream_t stream);
cudaError_t launch_project_kernel(int W, int H, int n, const float* dirs, float* uc, float* vc,
                                  cudaStream_t stream);
cudaError_t launch_sample_kernel(cudaTextureObject_t tex, int W, int H, int n, const float* uc,
                                 const float* vc, float* out, cudaStream_t stream);

}  // namespace pmsp
