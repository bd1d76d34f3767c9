// pmsp_densify_batch_noalloc: the batched densification for callers that
// cannot allocate device memory.
//
// Some callers are not allowed to allocate at the moment they densify: a
// host framework that owns all device memory and forbids allocation from
// plug-ins, a real-time thread that must not take the allocator's locks or
// device-wide synchronisation, or code that runs while a stream is being
// recorded. This entry point does the work of pmsp_densify_batch without any
// allocation: sources are read with plain loads from the caller's own
// device buffers (no texture arrays), and the batch's working state (work
// counters, per-keyframe descriptors, tile offsets) lives in one file-scope
// __device__ array of fixed size, PMSP_NOALLOC_SCRATCH_BYTES, which every GPU
// that loads the library keeps until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "pixel_kernel.cuh"
#include "pmsp.h"
#include "runtime.h"

namespace pmsp {

namespace {

constexpr int NA_MAX_PHASES = 64;  // 2 + 2 x iterations, iterations <= 31

// Source of one view read with plain loads.
struct LinearSrc {
    const uint8_t* data;
    int64_t pitch;
    int fmt, w, h, pad;
};

// Layout of the scratch array (offsets in bytes).
constexpr size_t NA_OFF_COUNTERS = 0;                                   // uint32 x NA_MAX_PHASES
constexpr size_t NA_OFF_PREFIX = 256;                                   // int x (MAX_ITEMS + 1) tile offsets
constexpr size_t NA_OFF_PHASES = NA_OFF_PREFIX + 128;                   // int x MAX_ITEMS phase counts
constexpr size_t NA_OFF_LINEAR = 512;                                   // LinearSrc x MAX_ITEMS x MAX_SOURCES
constexpr size_t NA_OFF_PARAMS =
    NA_OFF_LINEAR + sizeof(LinearSrc) * PMSP_NOALLOC_MAX_ITEMS * PMSP_MAX_SOURCES;  // PixelParams x MAX_ITEMS
constexpr size_t NA_USED = NA_OFF_PARAMS + sizeof(PixelParams) * PMSP_NOALLOC_MAX_ITEMS;
static_assert(NA_USED <= PMSP_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the stated size");
static_assert((PMSP_NOALLOC_MAX_ITEMS + 1) * sizeof(int) <= 128, "tile offsets overflow their slot");
static_assert(NA_OFF_PARAMS % 16 == 0, "descriptors must be 16-byte aligned");

// The batch state of every call on this device (shared by all calls).
static __device__ __align__(256) unsigned char g_noalloc_scratch[PMSP_NOALLOC_SCRATCH_BYTES];

__shared__ __align__(16) PixelParams na_sp;        // current keyframe's parameters
__shared__ LinearSrc na_lin[PMSP_MAX_SOURCES];     // and its sources

struct LinearViews {};

}  // namespace

// The cost's source fetch for LinearViews: projection as in every other path,
// then bilinear interpolation of the four taps read with plain loads
// (longitude wrapped, latitude clamped).
template <>
__device__ __forceinline__ float view_sample<LinearViews>(const SourceView& V, float X, float Y, float Z) {
    const int s = (int)(&V - na_sp.src);
    const float Yx = fmaf(V.R[0], X, fmaf(V.R[1], Y, fmaf(V.R[2], Z, V.t[0])));
    const float Yy = fmaf(V.R[3], X, fmaf(V.R[4], Y, fmaf(V.R[5], Z, V.t[1])));
    const float Yz = fmaf(V.R[6], X, fmaf(V.R[7], Y, fmaf(V.R[8], Z, V.t[2])));
    float qu, qv;
    bool front;
    project_dir_half(Yx, Yy, Yz, V.su, -V.sv, qu, qv, front);
    const LinearSrc& L = na_lin[s];
    const float fi = floor_small(qu), fj = floor_small(qv);
    const float fx = qu - fi, fy = qv - fj;
    int i0 = ((int)fi + (front ? L.w / 2 - 1 : -1)) % L.w;  // see project_dir_half
    if (i0 < 0) i0 += L.w;
    const int i1 = i0 + 1 == L.w ? 0 : i0 + 1;
    const int jj = (int)fj + L.h / 2 - 1;
    const int j0 = clamp_index(jj, L.h - 1), j1 = clamp_index(jj + 1, L.h - 1);
    const uint8_t* r0 = L.data + (int64_t)j0 * L.pitch;
    const uint8_t* r1 = L.data + (int64_t)j1 * L.pitch;
    float t00, t10, t01, t11;
    if (L.fmt == PMSP_U8) {
        const float k = 1.0f / 255.0f;
        t00 = (float)__ldg(r0 + i0) * k;
        t10 = (float)__ldg(r0 + i1) * k;
        t01 = (float)__ldg(r1 + i0) * k;
        t11 = (float)__ldg(r1 + i1) * k;
    } else if (L.fmt == PMSP_F16) {
        const __half* a = reinterpret_cast<const __half*>(r0);
        const __half* b = reinterpret_cast<const __half*>(r1);
        t00 = __half2float(a[i0]);
        t10 = __half2float(a[i1]);
        t01 = __half2float(b[i0]);
        t11 = __half2float(b[i1]);
    } else {
        const float* a = reinterpret_cast<const float*>(r0);
        const float* b = reinterpret_cast<const float*>(r1);
        t00 = __ldg(a + i0);
        t10 = __ldg(a + i1);
        t01 = __ldg(b + i0);
        t11 = __ldg(b + i1);
    }
    const float top = fmaf(fx, t10 - t00, t00);
    const float bot = fmaf(fx, t11 - t01, t01);
    return fmaf(fy, bot - top, top);
}

namespace {

// One phase of every keyframe of the batch. Work items are numbered across the
// keyframes' tiles (tile offsets in the scratch); blocks take items from the
// phase's counter until the numbering is exhausted, so the loop is bounded.
__global__ void __launch_bounds__(BLOCK_THREADS) noalloc_kernel(unsigned char* scratch, int phase, int n_items) {
    __shared__ TileSmem sm;
    __shared__ int s_item, s_prob;
    unsigned* counter = reinterpret_cast<unsigned*>(scratch + NA_OFF_COUNTERS) + phase;
    const int* prefix = reinterpret_cast<const int*>(scratch + NA_OFF_PREFIX);
    const int* phases = reinterpret_cast<const int*>(scratch + NA_OFF_PHASES);
    const LinearSrc* lin = reinterpret_cast<const LinearSrc*>(scratch + NA_OFF_LINEAR);
    const PixelParams* params = reinterpret_cast<const PixelParams*>(scratch + NA_OFF_PARAMS);
    const int total = prefix[n_items];
    if (threadIdx.x == 0) s_prob = -1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= total) break;
        int p = 0;
        while (p + 1 < n_items && prefix[p + 1] <= it) ++p;
        if (phase >= phases[p]) continue;  // this keyframe has finished its iterations
        if (p != s_prob) {
            const int4* src = reinterpret_cast<const int4*>(params + p);
            int4* dst = reinterpret_cast<int4*>(&na_sp);
            for (int k = threadIdx.x; k < (int)(sizeof(PixelParams) / 16); k += BLOCK_THREADS) dst[k] = src[k];
            if (threadIdx.x < PMSP_MAX_SOURCES) na_lin[threadIdx.x] = lin[p * PMSP_MAX_SOURCES + threadIdx.x];
            __syncthreads();
            if (threadIdx.x == 0) s_prob = p;
        }
        const int tile = it - prefix[p];
        const int tiles_x = (na_sp.W + TILE_W - 1) / TILE_W;
        const int bx = (tile % tiles_x) * TILE_W, by = (tile / tiles_x) * TILE_H;
        const int colour = phase & 1;
        if (phase < 2)
            process_tile<16, false, MODE_INIT, LinearViews>(na_sp, sm, bx, by, colour, 0);
        else
            process_tile<16, false, MODE_SWEEP, LinearViews>(na_sp, sm, bx, by, colour, (phase - 2) >> 1);
    }
}

// Descriptor bytes carried to the device in a kernel's parameters. A call
// recorded into a graph then keeps them in the kernel node; a copy from the
// host image on this function's stack would read that stack at every replay.
constexpr int NA_CHUNK_WORDS = 1000;  // 4000 bytes, within the 4 KB classic parameter limit
struct NaChunk {
    unsigned words[NA_CHUNK_WORDS];
};

__global__ void noalloc_store(unsigned* dst, NaChunk chunk, int n_words) {
    for (int k = threadIdx.x; k < n_words; k += blockDim.x) dst[k] = chunk.words[k];
}

static_assert(sizeof(LinearSrc) % 4 == 0 && sizeof(PixelParams) % 4 == 0, "descriptors are stored as words");
static_assert((NA_OFF_LINEAR - NA_OFF_PREFIX) % 4 == 0, "tile offsets are stored as words");

std::mutex g_setup_mu;
void* g_scratch_addr[128];  // device address of the scratch array, per device ordinal
int g_resident[128];        // SMs x resident blocks of noalloc_kernel, per device ordinal
bool g_scratch_ready[128];

}  // namespace

}  // namespace pmsp

using namespace pmsp;

extern "C" int pmsp_densify_batch_noalloc(pmsp_ctx* c, const pmsp_batch_item* items, int n) {
    if (!c) return PMSP_EINVAL;
    if (cudaSetDevice(c->device) != cudaSuccess) return ctx_fail(c, PMSP_ECUDA, "cudaSetDevice failed");
    if (n < 1 || !items) return ctx_fail(c, PMSP_EINVAL, "empty batch");
    if (n > PMSP_NOALLOC_MAX_ITEMS)
        return ctx_fail(c, PMSP_EINVAL, "batch of %d keyframes exceeds the no-allocation limit of %d", n,
                        PMSP_NOALLOC_MAX_ITEMS);
    if (c->device < 0 || c->device >= 128) return ctx_fail(c, PMSP_EINVAL, "device ordinal %d out of range", c->device);

    // set-up, once per device, with that device current: the device address of
    // the scratch array (its host-side name is only a stand-in) and the number
    // of blocks the persistent kernel keeps resident
    void* scratch = nullptr;
    int resident = 0;
    {
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_scratch_ready[c->device]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return cuda_fail(c, e, "scratch address lookup");
            int sms = 0, occ = 0;
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
            if (e != cudaSuccess) return cuda_fail(c, e, "SM count query");
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, noalloc_kernel, BLOCK_THREADS, 0);
            if (e != cudaSuccess) return cuda_fail(c, e, "occupancy query");
            if (sms < 1 || occ < 1)
                return ctx_fail(c, PMSP_ECUDA, "no-allocation kernel cannot run: %d SMs x %d blocks", sms, occ);
            g_scratch_addr[c->device] = p;
            g_resident[c->device] = sms * occ;
            g_scratch_ready[c->device] = true;
        }
        scratch = g_scratch_addr[c->device];
        resident = g_resident[c->device];
    }

    // host image of the used part of the scratch, on the stack (no allocation)
    alignas(16) unsigned char blob[NA_USED];
    memset(blob, 0, NA_USED);
    int* prefix = reinterpret_cast<int*>(blob + NA_OFF_PREFIX);
    int* phases = reinterpret_cast<int*>(blob + NA_OFF_PHASES);
    LinearSrc* lin = reinterpret_cast<LinearSrc*>(blob + NA_OFF_LINEAR);
    PixelParams* params = reinterpret_cast<PixelParams*>(blob + NA_OFF_PARAMS);
    int max_phases = 0, total = 0;
    for (int i = 0; i < n; ++i) {
        const pmsp_batch_item& it = items[i];
        int rc = check_params(c, &it.params, it.n_src);
        if (rc) return rc;
        if ((rc = check_panorama(c, &it.ref, "no-allocation reference"))) return rc;
        if ((rc = check_maps(c, &it.out, it.ref.w, it.ref.h, true, true, "no-allocation output"))) return rc;
        if (it.ref.w & 1) return ctx_fail(c, PMSP_EINVAL, "reference width %d must be even", it.ref.w);
        if (!it.srcs || !it.src_poses) return ctx_fail(c, PMSP_EINVAL, "item %d without sources", i);
        if (it.params.iterations > (NA_MAX_PHASES - 2) / 2)
            return ctx_fail(c, PMSP_EINVAL, "iterations %d exceed the no-allocation limit of %d", it.params.iterations,
                            (NA_MAX_PHASES - 2) / 2);
        if (it.ref.memory != PMSP_DEVICE || it.out.memory != PMSP_DEVICE)
            return ctx_fail(c, PMSP_EINVAL, "item %d: the no-allocation path takes device memory only", i);
        cudaTextureObject_t none[PMSP_MAX_SOURCES] = {};
        for (int s = 0; s < it.n_src; ++s) {
            const pmsp_image& im = it.srcs[s];
            if ((rc = check_panorama(c, &im, "no-allocation source"))) return rc;
            if (im.memory != PMSP_DEVICE)
                return ctx_fail(c, PMSP_EINVAL, "item %d: the no-allocation path takes device memory only", i);
            LinearSrc& L = lin[i * PMSP_MAX_SOURCES + s];
            L.data = static_cast<const uint8_t*>(im.data);
            L.pitch = im.pitch_bytes;
            L.fmt = im.format;
            L.w = im.w;
            L.h = im.h;
        }
        PixelParams& P = params[i];
        fill_problem(P, &it.ref, it.ref.data, it.ref.pitch_bytes, &it.ref_pose, it.srcs, none, it.src_poses, it.n_src,
                     &it.params);
        const size_t N = (size_t)it.ref.w * it.ref.h;
        P.depth = it.out.depth;
        P.nx = it.out.normal;
        P.ny = it.out.normal + N;
        P.nz = it.out.normal + 2 * N;
        P.cost = it.out.cost;
        P.err = c->d_err;
        prefix[i] = total;
        total += ((it.ref.w + TILE_W - 1) / TILE_W) * ((it.ref.h + TILE_H - 1) / TILE_H);
        phases[i] = 2 + 2 * it.params.iterations;
        if (phases[i] > max_phases) max_phases = phases[i];
    }
    prefix[n] = total;

    // every call starts from zeroed counters and its own descriptors: tile offsets
    // and phase counts, then the n keyframes' sources and parameters
    unsigned char* const dev = static_cast<unsigned char*>(scratch);
    auto store = [&](size_t off, size_t bytes) {
        cudaError_t err = cudaSuccess;
        for (size_t done = 0; done < bytes && err == cudaSuccess; done += sizeof(NaChunk)) {
            const size_t len = std::min(sizeof(NaChunk), bytes - done);
            NaChunk ch;
            memcpy(ch.words, blob + off + done, len);
            noalloc_store<<<1, 256, 0, c->stream>>>(reinterpret_cast<unsigned*>(dev + off + done), ch,
                                                    (int)(len / sizeof(unsigned)));
            err = cudaGetLastError();
        }
        return err;
    };
    cudaError_t e = cudaMemsetAsync(dev + NA_OFF_COUNTERS, 0, NA_MAX_PHASES * sizeof(unsigned), c->stream);
    if (e == cudaSuccess) e = store(NA_OFF_PREFIX, NA_OFF_LINEAR - NA_OFF_PREFIX);
    if (e == cudaSuccess) e = store(NA_OFF_LINEAR, (size_t)n * PMSP_MAX_SOURCES * sizeof(LinearSrc));
    if (e == cudaSuccess) e = store(NA_OFF_PARAMS, (size_t)n * sizeof(PixelParams));
    if (e != cudaSuccess) return cuda_fail(c, e, "no-allocation descriptor upload");
    const int grid = std::max(1, std::min(total, resident));
    for (int ph = 0; ph < max_phases; ++ph) {
        noalloc_kernel<<<grid, BLOCK_THREADS, 0, c->stream>>>(static_cast<unsigned char*>(scratch), ph, n);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(c, e, "no-allocation launch");
    }
    return PMSP_OK;
}
