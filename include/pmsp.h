/*
 * pmsp.h - C ABI of the GB300 PatchMatch-Stereo-Panorama densification library.
 *
 * The library computes, for one reference equirectangular keyframe and a small
 * neighbourhood of source keyframes with known poses, a per-pixel plane
 * hypothesis (range along the pixel ray + unit normal) by PatchMatch stereo:
 * random initialisation (paper Sec. III-B), red-black propagation over an
 * 8-neighbourhood (Sec. III-C, Fig. 5), six shrinking random refinement tests
 * (Sec. III-C, item 1), scored by a bilaterally weighted NCC of the reference
 * patch against its reprojection through the plane into every source
 * panorama, averaged over the best k views; and a multi-view geometric
 * consistency filter over neighbouring depth maps (Sec. III). Around that
 * path: initialisation by plane-map warping (Sec. III-B), the median
 * post-filter (Sec. III-C, item 2), the View Filter (Sec. III-A, Eq. 1),
 * point-cloud fusion (Sec. III) and keyframe completeness (Sec. IV); batched
 * and served forms of the densification.
 *
 * Conventions (all calls):
 *  - Panorama W x H, row-major, W and H even for every image the
 *    densification reads (references, sources, ring frames; PMSP_EINVAL
 *    otherwise). Pixel (u, v) looks along longitude
 *    2*pi*(u+0.5)/W - pi and latitude pi/2 - pi*(v+0.5)/H; camera frame x right,
 *    y down, z forward.
 *  - Poses are world->camera, X_c = R X_w + t, R row-major, in double.
 *  - "Depth" is the range along the pixel ray, metres. Normals are unit vectors
 *    in the reference camera frame, stored as three planes nx, ny, nz of W*H
 *    floats each (normal[0..N), normal[N..2N), normal[2N..3N)).
 *  - uint8 images are intensities DN/255; fp16/fp32 images are taken as given,
 *    on the scale of [0, 1] (sigma_color refers to it). Any offset is allowed:
 *    the cost depends on intensity differences and normalised correlations
 *    only, and fp16 images centred on 0 (DN/255 - 0.5) round half as coarsely.
 *  - Ownership: the caller owns every buffer passed in and out; the library
 *    never frees or retains caller memory beyond a call. The context owns its
 *    internal buffers (texture arrays, staging, error flag) and frees them in
 *    pmsp_destroy.
 *  - Errors: every call returns PMSP_OK (0) or a negative code below; the
 *    text of the last failure is available from pmsp_last_error. Nothing is
 *    thrown and nothing aborts across the ABI.
 *  - Streams: work is enqueued on the context's stream. A call whose inputs
 *    and outputs are all device memory returns once the work is enqueued
 *    (asynchronous); a call touching host memory returns after the results
 *    are back on the host, and so do the calls that return counts
 *    (pmsp_view_filter, pmsp_fuse, pmsp_completeness). pmsp_sync waits for
 *    the stream and reports any error the kernels flagged.
 *  - Threads: a context is used by one host thread at a time, except the
 *    serving calls (ring_push/submit/poll/wait/get_serving_stats), which are
 *    internally locked and may be made from different threads at once; the
 *    last-error text then belongs to whichever call failed last.
 */
#ifndef PMSP_H
#define PMSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PMSP_ABI_VERSION 1
#define PMSP_MAX_SOURCES 16
#define PMSP_MAX_PATCH_W 21

/* Status codes. */
#define PMSP_OK 0
#define PMSP_EINVAL (-1)    /* invalid argument or size */
#define PMSP_ENOMEM (-2)    /* device or host allocation failed */
#define PMSP_EADMIT (-3)    /* request exceeds the context's memory cap */
#define PMSP_EBUSY (-4)     /* no free slot, try again later */
#define PMSP_ETIMEDOUT (-5) /* bounded wait expired */
#define PMSP_ECUDA (-6)     /* CUDA runtime error (text in pmsp_last_error) */
#define PMSP_EDEVICE (-7)   /* a kernel flagged an error (bounds/consistency) */
#define PMSP_ENOTFOUND (-8) /* unknown frame id or ticket */

typedef enum { PMSP_U8 = 0, PMSP_F16 = 1, PMSP_F32 = 2 } pmsp_format;
typedef enum { PMSP_HOST = 0, PMSP_DEVICE = 1 } pmsp_memory;

/* A grayscale panorama. pitch_bytes >= w * element size; data is host or
 * device memory according to `memory`. Device images are read in place by
 * element, so their data pointer and pitch_bytes must both be multiples of
 * the element size (2 bytes for F16, 4 for F32); any other device image is
 * refused with PMSP_EINVAL before a launch. Host images may have any pitch. */
typedef struct {
    int32_t w, h;
    int64_t pitch_bytes;
    int32_t format; /* pmsp_format */
    int32_t memory; /* pmsp_memory */
    const void* data;
} pmsp_image;

/* World->camera pose, X_c = R X_w + t (R row-major). */
typedef struct {
    double R[9];
    double t[3];
} pmsp_pose;

/* PatchMatch parameters (see pmsp_default_params for the defaults). */
typedef struct {
    float d_min, d_max;       /* range bounds in metres, 0 < d_min < d_max */
    int32_t patch_w;          /* window extent in pixels, odd, <= PMSP_MAX_PATCH_W */
    int32_t patch_stride;     /* sampling step inside the window, >= 1 */
    int32_t iterations;       /* red-black iterations */
    int32_t best_k;           /* views averaged per cost, 1 <= best_k <= n_src */
    float sigma_color;        /* bilateral colour sigma (normalised units); <= 0: off */
    float sigma_space;        /* bilateral spatial sigma (pixels); <= 0: off */
    int32_t n_refine;         /* random refinement tests per half-sweep (paper: 6) */
    int32_t neighbor_table;   /* 0: axis distances {3, 5}; 1: {1, 5} */
    uint64_t seed;            /* Philox key word 0 */
    uint64_t keyframe_id;     /* Philox key word 1 */
} pmsp_params;

/* Plane map: range, normal (3 planes) and cost, each w*h floats, host or
 * device memory according to `memory`. Any of the pointers may be NULL where
 * a call says so. */
typedef struct {
    int32_t w, h;
    int32_t memory; /* pmsp_memory */
    float* depth;
    float* normal;
    float* cost;
} pmsp_maps;

typedef struct {
    int32_t device;          /* CUDA device ordinal */
    void* stream;            /* cudaStream_t to enqueue on (cudaStreamLegacy, 0x1, for the
                                legacy default stream); NULL: the context creates one */
    uint64_t mem_cap_bytes;  /* serving admission cap (0: 40 GiB) */
    int32_t ring_capacity;   /* frames kept in the device ring (0: 64) */
    int32_t max_active;      /* serving slots (0: 32) */
    int32_t scheduler;       /* pmsp_scheduler of the serving runtime (0: lanes) */
} pmsp_ctx_opts;

/* Serving schedulers (Sec. III: densification in its own thread, fed by a
 * keyframe queue). Both admit FIFO under the same rules (slots, memory cap,
 * resident tiles, depth-map order) and give every request the same maps.
 *   PMSP_SCHED_LANES  each admitted request's whole launch chain starts on a
 *                     stream lane of its own; chains of different requests
 *                     overlap on the device.
 *   PMSP_SCHED_STEPS  iteration-level: each scheduler step is one persistent
 *                     launch running the next phase (initialisation colour or
 *                     half-sweep) of every active request; requests join at
 *                     the next step and leave after their last phase. */
typedef enum { PMSP_SCHED_LANES = 0, PMSP_SCHED_STEPS = 1 } pmsp_scheduler;

typedef struct pmsp_ctx pmsp_ctx;

/* Create a context on opts->device (NULL opts: device 0, own stream). */
int pmsp_create(pmsp_ctx** out, const pmsp_ctx_opts* opts);
/* Wait for outstanding work and free everything the context owns. NULL is a no-op. */
int pmsp_destroy(pmsp_ctx* ctx);
/* Text of the most recent failure on this context ("" if none). Valid until the next call. */
const char* pmsp_last_error(pmsp_ctx* ctx);
/* Block until the context stream is idle; PMSP_EDEVICE if a kernel flagged an error
 * since the last report (the flag is then cleared, so it is reported once). */
int pmsp_sync(pmsp_ctx* ctx);
/* Fill *p with the defaults: d 0.3..10 m, 11x11 window at stride 2, 8
 * iterations, best_k 3, sigma_color 0.2, sigma_space 3 px, 6 refinement
 * tests, table 0, seed 42, keyframe 0. */
void pmsp_default_params(pmsp_params* p);

/*
 * Densify one keyframe (Sec. III-B initialisation, then `iterations` x red and
 * black half-sweeps of Sec. III-C propagation and refinement).
 *   ref, ref_pose        reference panorama and pose
 *   srcs, src_poses      n_src source panoramas (1 <= n_src <= PMSP_MAX_SOURCES),
 *                        any even size each, and their poses
 *   p                    parameters
 *   out                  w x h of the reference; depth, normal, cost all required.
 * Returns PMSP_EINVAL for an odd width or height, best_k outside [1, n_src], a
 * bad window, a bad range, a NULL pointer or an unknown format.
 */
int pmsp_densify(pmsp_ctx* ctx, const pmsp_image* ref, const pmsp_pose* ref_pose,
                 const pmsp_image* srcs, const pmsp_pose* src_poses, int n_src,
                 const pmsp_params* p, pmsp_maps* out);

/*
 * Matching cost (Sec. III-C: rectangular patch in the reference, its
 * reprojection through the plane into every source) of the given planes:
 * planes->depth and planes->normal are read, planes->cost is written.
 */
int pmsp_cost_map(pmsp_ctx* ctx, const pmsp_image* ref, const pmsp_pose* ref_pose,
                  const pmsp_image* srcs, const pmsp_pose* src_poses, int n_src,
                  const pmsp_params* p, pmsp_maps* planes);

/*
 * Initialisation by plane-map warping (Sec. III-B: the optimised plane map of
 * the preceding keyframe is transferred into the current one, after Shen
 * 2013): every previous plane with range > 0 is moved into the current
 * camera and splatted onto the nearest pixel (the nearest surface wins, equal
 * ranges the smaller previous pixel index); a claimed pixel re-intersects the
 * plane with its own ray; unclaimed pixels, and planes grazing, behind or
 * outside [d_min, d_max] there, take the random initial plane of pmsp_init.
 * Then the initial costs.
 *   prev, prev_pose   previous keyframe's maps (depth and normal read; any size,
 *                     host or device) and pose
 *   out               device maps of the reference size
 *   src               optional device array of w*h int32: winning previous pixel
 *                     index (row-major) or -1 where the random plane was used
 */
int pmsp_warp_init(pmsp_ctx* ctx, const pmsp_image* ref, const pmsp_pose* ref_pose,
                   const pmsp_image* srcs, const pmsp_pose* src_poses, int n_src,
                   const pmsp_params* p, const pmsp_maps* prev, const pmsp_pose* prev_pose,
                   pmsp_maps* out, int32_t* src);

/* pmsp_densify with the warping initialisation in place of the random one
 * (the paper's densification with "plane warping" on). */
int pmsp_densify_warped(pmsp_ctx* ctx, const pmsp_image* ref, const pmsp_pose* ref_pose,
                        const pmsp_image* srcs, const pmsp_pose* src_poses, int n_src,
                        const pmsp_params* p, const pmsp_maps* prev, const pmsp_pose* prev_pose,
                        pmsp_maps* out);

/* Random initialisation (Sec. III-B) plus initial cost into out. */
int pmsp_init(pmsp_ctx* ctx, const pmsp_image* ref, const pmsp_pose* ref_pose,
              const pmsp_image* srcs, const pmsp_pose* src_poses, int n_src,
              const pmsp_params* p, pmsp_maps* out);

/*
 * One half-sweep (Sec. III-C) in place on `state`: every pixel with
 * (u + v) % 2 == colour tries its 8 neighbours' planes and p->n_refine random
 * refinements (Philox counter iteration word = `iteration`), keeping a
 * candidate only if its cost is strictly lower.
 */
int pmsp_halfsweep(pmsp_ctx* ctx, const pmsp_image* ref, const pmsp_pose* ref_pose,
                   const pmsp_image* srcs, const pmsp_pose* src_poses, int n_src,
                   const pmsp_params* p, int colour, int iteration, pmsp_maps* state);

/*
 * Geometric consistency filter (Sec. III): a reference pixel keeps its range
 * if, in at least min_views of the n neighbour depth maps, lifting it to 3-D,
 * reading the neighbour's range at the nearest pixel and reprojecting that
 * point lands within max_reproj_px pixels of where it started; otherwise its
 * range becomes 0.
 *   ref        reference depth (ref->depth read)
 *   nbrs       n neighbour maps (depth read; any size each), 1 <= n <= PMSP_MAX_SOURCES
 *   inout      depth written (may alias ref->depth)
 *   agree      optional (NULL) w*h int32 receiving the number of agreeing views,
 *              same memory kind as inout
 */
int pmsp_consistency_filter(pmsp_ctx* ctx, const pmsp_maps* ref, const pmsp_pose* ref_pose,
                            const pmsp_maps* nbrs, const pmsp_pose* nbr_poses, int n,
                            float max_reproj_px, int min_views, pmsp_maps* inout,
                            int32_t* agree);

/*
 * Median post-filter (Sec. III-C, item 2: a median filter over a copy of the
 * depth image; ranges deviating from it by more than a threshold are removed).
 * For a pixel with range d > 0, the valid ranges (> 0) of its
 * (2 radius + 1)^2 window (columns wrapped at the seam, rows outside the
 * panorama left out) give the lower median m (rank floor((n-1)/2)); the
 * output is 0 where |d - m| > tau * m (FP32), else d. Pixels with d <= 0
 * output 0. Selection is exact.
 *   in       depth read (in->depth, w x h)
 *   radius   1, 2 (5 x 5, the default reading) or 3
 *   tau      relative threshold > 0 (0.05 in the default reading)
 *   out      depth written; same size and memory kind as in; must not
 *            alias in->depth (every decision reads the unfiltered map)
 * Errors: PMSP_EINVAL for NULL or mismatched maps, aliasing, radius outside
 * [1, 3] or tau <= 0.
 */
int pmsp_median_filter(pmsp_ctx* ctx, const pmsp_maps* in, int radius, float tau, pmsp_maps* out);

/*
 * View Filter (Sec. III-A, Eq. 1, read as the parallax angle at a point): for
 * each of n sparse points p seen by keyframes a and b,
 * theta_p = arccos((t_a - p).(t_b - p) / (|t_a - p| |t_b - p|)), t_K the camera
 * centre -R_K^T t_K. Keyframe b is accepted when the share of points with
 * theta_p in [min_deg, max_deg] exceeds min_frac (6, 60 and 0.2 in the paper).
 * FP32 on the device; a point at a camera centre counts as out of range.
 *   points     3n floats (x, y, z per point, world frame) in `memory`
 *   in_range   optional (NULL) n bytes, same memory kind, receiving 0/1 per point
 *   accepted   host int32 receiving 1 (accept) or 0
 *   fraction   optional host double receiving the share in range (0 if n = 0)
 * Errors: PMSP_EINVAL for NULL arguments, n < 0, or bounds outside
 * 0 <= min_deg <= max_deg <= 180, 0 <= min_frac <= 1.
 */
int pmsp_view_filter(pmsp_ctx* ctx, const pmsp_pose* a, const pmsp_pose* b, const float* points, int64_t n,
                     int memory, double min_deg, double max_deg, double min_frac, uint8_t* in_range,
                     int32_t* accepted, double* fraction);

/*
 * Dense point-cloud fusion (Sec. III: the point-cloud thread erases duplicate
 * points of the buffered, consistency-filtered keyframes). Every pixel with
 * range d > 0 of keyframe k becomes X = R_k^T (d r_p - t_k) (FP32); points are
 * binned into cubic voxels of edge `voxel` metres (key floor(X / voxel) per
 * axis, at most 2^20 voxels from the origin on each axis) and each occupied
 * voxel keeps its first point in (keyframe, pixel index) order. Kept points
 * are written in that order.
 *   maps     n depth maps (depth read; any sizes), 1 <= n <= PMSP_MAX_SOURCES,
 *            all of one memory kind
 *   poses    n world->camera poses
 *   points   3 * cap floats receiving x, y, z of the first min(count, cap)
 *            kept points, same memory kind as the maps (may be NULL if cap = 0)
 *   src      optional (NULL) cap int64 receiving k << 32 | pixel index
 *   count    host int64 receiving the number of occupied voxels (call with
 *            cap = 0 to size the output)
 * Synchronous. Device memory: a hash table of 16 bytes per slot (a power of
 * two >= twice the input pixels) plus 4 bytes per input pixel, held by the
 * context between calls. Errors: PMSP_EINVAL for NULL or mismatched
 * arguments, voxel <= 0, or a point beyond the key range.
 */
int pmsp_fuse(pmsp_ctx* ctx, const pmsp_maps* maps, const pmsp_pose* poses, int n, float voxel, float* points,
              int64_t* src, int64_t cap, int64_t* count);

/*
 * Keyframe completeness (Sec. IV: the share of pixels of a panorama rendered
 * at a keyframe position onto which some 3-D point projects; 720 x 360 in the
 * paper). Each of the n points is moved into the camera of `pose` and
 * projected onto the nearest pixel of a W x H panorama (u wrapped, v clamped);
 * occlusion plays no part.
 *   points        3n floats in `memory`
 *   hit           optional (NULL) W*H bytes, same memory kind, receiving 0/1
 *   completeness  host double receiving pixels hit / (W * H)
 * Synchronous. Errors: PMSP_EINVAL for NULL arguments, n < 0, W or H < 1.
 */
int pmsp_completeness(pmsp_ctx* ctx, const float* points, int64_t n, int memory, const pmsp_pose* pose, int W,
                      int H, uint8_t* hit, double* completeness);

/*
 * Bilinear sample of img at n continuous pixel coordinates (integers are pixel
 * centres; longitude wrapped, latitude clamped), the source fetch the cost uses.
 * uc, vc, out: n floats each, in the memory kind of img.
 */
int pmsp_sample_bilinear(pmsp_ctx* ctx, const pmsp_image* img, int n, const float* uc,
                         const float* vc, float* out);

/*
 * Equirectangular projection (Sec. III-C camera model) of n directions into a
 * W x H panorama, as the cost and the filter compute it on the device:
 * lon = atan2(x, z), lat = atan2(-y, hypot(x, z)), u_c = W (lon + pi) / 2pi - 0.5,
 * v_c = H (pi/2 - lat) / pi - 0.5.
 *   dirs     3n floats (x, y, z interleaved), any length > 0
 *   uc, vc   n floats each, written
 *   memory   pmsp_memory of all three arrays
 */
int pmsp_project(pmsp_ctx* ctx, int W, int H, int n, const float* dirs, float* uc, float* vc,
                 int memory);

/*
 * Measured peaks of the units the cost kernel is bound by (its roofline; the
 * paper reports no per-unit figures). The cost of one view-sample is plain FP32
 * arithmetic, special-function square roots and reciprocals and one texture
 * gather, so the denominators are these rates, each from a self-terminating
 * probe over every SM (fixed loop counts, independent chains), timed with CUDA
 * events on the context's stream, best of three:
 *   fp32_fma_per_s    scalar FMAs per second, all FP32 lanes
 *   fp32x2_fma_per_s  FMAs per second issued as packed f32x2 instructions
 *   sfu_per_s         rsqrt.approx results per second
 *   gather_l1_per_s   tex2Dgather results per second from an L1-resident texture
 *   gather_l2_per_s   the same at scattered texels of a 16 MB (L2-resident) texture
 *   sm_clock_mhz_max  the device's maximum SM clock (the probes run at the live clock)
 * Allocates a few MB for the probes and frees them; synchronous; about 0.2 s.
 * Errors: PMSP_EINVAL for NULL arguments, PMSP_ECUDA / PMSP_ENOMEM from CUDA.
 */
typedef struct {
    double fp32_fma_per_s;
    double fp32x2_fma_per_s;
    double sfu_per_s;
    double gather_l1_per_s;
    double gather_l2_per_s;
    double sm_clock_mhz_max;
    int32_t sms;
    int32_t reserved;
} pmsp_peaks;

int pmsp_measure_peaks(pmsp_ctx* ctx, pmsp_peaks* out);

/* ------------------------------------------------------------------------
 * Batched densification: many keyframes of different sizes and view counts
 * in one pass. Every phase (initialisation colours, then each half-sweep) is
 * one persistent launch over the tiles of all keyframes; the per-pixel work
 * is the single-keyframe computation, so each keyframe's maps equal what
 * pmsp_densify returns for it alone.
 * ---------------------------------------------------------------------- */
typedef struct {
    pmsp_image ref;
    pmsp_pose ref_pose;
    const pmsp_image* srcs;     /* n_src source panoramas */
    const pmsp_pose* src_poses; /* n_src poses */
    int32_t n_src;
    pmsp_params params;
    pmsp_maps out;              /* depth, normal, cost of the reference size */
} pmsp_batch_item;

/* Launch settings of the batched path (see pmsp_autotune). */
typedef struct {
    int32_t blocks_per_sm; /* persistent grid = SMs x blocks_per_sm; 0: the occupancy maximum */
    int32_t order;         /* work order: 0 largest keyframe first, 1 tiles of all keyframes interleaved */
    int32_t patch_stride;  /* 0: each item's own stride; > 0: use this stride for every item */
    int32_t strategy;      /* 0: one persistent launch per phase over all keyframes' tiles;
                              1: every keyframe's own launch chain, chains run concurrently on
                                 parallel streams (parallel branches of the captured graph) */
    int32_t tile;          /* strategy 1, half-sweeps with an 11x11/2 or 7x7/1 window: tile of
                              reference pixels per 128-thread block, 0: 32x8, 1: 64x4, 2: 16x16
                              (every shape computes the same numbers) */
    int32_t tpp;           /* strategy 1, half-sweeps of keyframes with 2 or more sources:
                              threads per pixel, 0 or 1: one; 2, 4 (or 8 with `lanes` 1):
                              split as `lanes` says (tile 32x4, 32x2 or 32x1, `tile`
                              ignored); 0, 1, 2, 4, or 8 with lanes, else PMSP_EINVAL */
    int32_t lanes;         /* how tpp 2 or more splits a pixel: 0: its view pairs over 2 or 4
                              warps that exchange their view costs through shared memory (the
                              same numbers as one thread, fewer registers per thread); 1: its
                              patch samples over 2, 4 or 8 adjacent lanes of one warp whose
                              NCC sums are added by warp shuffles (the sums in another order:
                              equal within rounding, not bit for bit); 0 or 1, else
                              PMSP_EINVAL */
} pmsp_tuning;

#define PMSP_BATCH_GRAPH 1u /* capture the batch in a CUDA graph and replay it when the identical
                               batch (same buffers, sizes and parameters) is submitted again;
                               applies when every buffer is device memory */

/*
 * Densify n keyframes. tuning may be NULL (defaults). Returns PMSP_EINVAL if
 * any item is invalid (nothing is run). Device-memory batches return once
 * enqueued; a batch with host memory returns with the results on the host.
 * The plan of a strategy-0 batch is staged through pinned host buffers that
 * the context reuses: a call made while the previous call's upload (or graph
 * replay) is still queued waits on the host until that has run. The first
 * capture of a PMSP_BATCH_GRAPH batch waits for the context stream to idle.
 */
int pmsp_densify_batch(pmsp_ctx* ctx, const pmsp_batch_item* items, int n, uint32_t flags,
                       const pmsp_tuning* tuning);

/*
 * Pick pmsp_tuning for a batch by timing candidate settings on it (the items'
 * outputs are overwritten). A coarser patch stride than the items' own is
 * accepted only if the range it produces stays within 1 % of the items'
 * own-stride result on at least (1 - max_changed) of the pixels.
 */
int pmsp_autotune(pmsp_ctx* ctx, const pmsp_batch_item* items, int n, float max_changed,
                  pmsp_tuning* out);

/*
 * pmsp_densify_batch for callers that cannot allocate device memory when they
 * densify. (The paper has no counterpart: this serves integration, not the
 * method.) Such callers include host frameworks that own all device memory
 * and forbid plug-ins to allocate, real-time threads that must not take the
 * allocator's locks or trigger device-wide synchronisation, and code running
 * while a stream is being recorded.
 *
 * The call allocates nothing: no cudaMalloc, cudaFree or allocating library
 * routine. Source images are read with plain loads from the caller's buffers
 * (no texture arrays), and the batch's working state lives in one fixed
 * __device__ array of PMSP_NOALLOC_SCRATCH_BYTES that every GPU loading the
 * library keeps until the process exits. The results are the same
 * computation as pmsp_densify_batch; the uint8 conversion of the plain loads
 * may differ from the texture unit's in the last bit, so maps agree within
 * the parity tolerances rather than bit for bit.
 *   items   n keyframes, 1 <= n <= PMSP_NOALLOC_MAX_ITEMS, every image and map in
 *           device memory; iterations <= 31
 * Work is enqueued on the context's stream (the call returns once enqueued).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Descriptors travel in kernel parameters, so a call recorded into a graph
 * reads no host memory when the graph is replayed.
 * All calls share the one array and each call resets it: calls whose work
 * overlaps on the GPU (different streams or contexts on one device) race, so
 * serialise them. PMSP_EINVAL for a batch above the limits or with host memory.
 */
#define PMSP_NOALLOC_MAX_ITEMS 16
#define PMSP_NOALLOC_SCRATCH_BYTES (64 * 1024)
int pmsp_densify_batch_noalloc(pmsp_ctx* ctx, const pmsp_batch_item* items, int n);

/* ------------------------------------------------------------------------
 * Serving (the densification thread of Sec. III: keyframes arrive from the
 * SLAM front end, each is densified against a small neighbourhood of
 * keyframes, filtered against neighbouring depth maps and handed on).
 * Frames live in a device ring of the last ring_capacity pushes; requests
 * are admitted in arrival order while a slot is free (max_active), their
 * maps fit under mem_cap_bytes and the running requests' tiles stay within
 * about two waves of the GPU's resident blocks (one request is always
 * admitted). An admitted request's launch chain runs on a stream lane of its
 * own, so requests that arrive while others run overlap with them on the
 * device. A request's maps are exactly those pmsp_densify gives for it,
 * whatever else is running.
 * ---------------------------------------------------------------------- */
typedef struct {
    int64_t ref_frame;            /* reference frame id (in the ring) */
    int32_t n_src;
    const int64_t* src_frames;    /* n_src source frame ids */
    pmsp_params params;
    int32_t n_filter;             /* 0: no filter; else neighbour frame ids whose depth maps */
    const int64_t* filter_frames; /*    (from finished requests) filter this result; the request
                                     starts only once no running request has one of them, or its
                                     own reference, as its reference or among its filter frames */
    float max_reproj_px;          /* filter threshold (pixels) */
    int32_t min_views;            /* filter: views that must agree */
} pmsp_request;

typedef struct {
    uint64_t submitted, completed, rejected;
    uint32_t queued, active;
    uint64_t steps;               /* lanes: requests started on a lane; steps: step launches */
    uint64_t bytes_in_use;        /* maps of admitted and unretrieved requests */
} pmsp_serving_stats;

/* Copy a frame into the ring (evicting the oldest frame no queued or active
 * request uses). Re-pushing an id replaces it. PMSP_EBUSY: every slot is in use. */
int pmsp_ring_push(pmsp_ctx* ctx, int64_t frame_id, const pmsp_image* img, const pmsp_pose* pose);

/* Queue a request; *ticket identifies it. PMSP_ENOTFOUND: a frame id is not in
 * the ring; PMSP_EADMIT: its maps alone exceed mem_cap_bytes; PMSP_EINVAL: bad
 * parameters. Returns without waiting for the GPU. */
int pmsp_submit(pmsp_ctx* ctx, const pmsp_request* req, uint64_t* ticket);

/* PMSP_OK once the request has finished: its maps (depth after the filter,
 * normal, cost; the reference frame's size) are copied into *out (NULL:
 * discarded) and the ticket is released. PMSP_EBUSY while it is queued or
 * running; PMSP_ENOTFOUND for an unknown or released ticket. */
int pmsp_poll(pmsp_ctx* ctx, uint64_t ticket, pmsp_maps* out);

/* pmsp_poll, blocking up to timeout_ms (PMSP_ETIMEDOUT when it expires). */
int pmsp_wait(pmsp_ctx* ctx, uint64_t ticket, int timeout_ms, pmsp_maps* out);

/* Counters of the serving runtime. */
int pmsp_get_serving_stats(pmsp_ctx* ctx, pmsp_serving_stats* out);

#ifdef __cplusplus
}
#endif

#endif /* PMSP_H */
