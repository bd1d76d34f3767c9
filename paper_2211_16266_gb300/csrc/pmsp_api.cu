// C ABI of the densification library (include/pmsp.h): argument checks,
// FP64 pose composition, texture and staging management, kernel launches.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "pmsp.h"
#include "runtime.h"

using namespace pmsp;

namespace pmsp {

template <int NS, bool EXACT>
cudaError_t launch_pixel_kernel_ns(const PixelParams& p, int mode, cudaStream_t stream);

// One instantiation per source count 1..16 (views unrolled without guards,
// in packed pairs from 2 views on).
cudaError_t launch_pixel_kernel(const PixelParams& p, int mode, cudaStream_t stream) {
    switch (p.S) {
        case 1: return launch_pixel_kernel_ns<1, true>(p, mode, stream);
        case 2: return launch_pixel_kernel_ns<2, true>(p, mode, stream);
        case 3: return launch_pixel_kernel_ns<3, true>(p, mode, stream);
        case 4: return launch_pixel_kernel_ns<4, true>(p, mode, stream);
        case 5: return launch_pixel_kernel_ns<5, true>(p, mode, stream);
        case 6: return launch_pixel_kernel_ns<6, true>(p, mode, stream);
        case 7: return launch_pixel_kernel_ns<7, true>(p, mode, stream);
        case 8: return launch_pixel_kernel_ns<8, true>(p, mode, stream);
        case 9: return launch_pixel_kernel_ns<9, true>(p, mode, stream);
        case 10: return launch_pixel_kernel_ns<10, true>(p, mode, stream);
        case 11: return launch_pixel_kernel_ns<11, true>(p, mode, stream);
        case 12: return launch_pixel_kernel_ns<12, true>(p, mode, stream);
        case 13: return launch_pixel_kernel_ns<13, true>(p, mode, stream);
        case 14: return launch_pixel_kernel_ns<14, true>(p, mode, stream);
        case 15: return launch_pixel_kernel_ns<15, true>(p, mode, stream);
        default: return launch_pixel_kernel_ns<16, true>(p, mode, stream);
    }
}

int ctx_fail(pmsp_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) {
        std::lock_guard<std::mutex> lk(c->err_mu);
        memcpy(c->err, buf, sizeof buf);
    }
    return code;
}

int cuda_fail(pmsp_ctx* c, cudaError_t e, const char* what) {
    return ctx_fail(c, PMSP_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t format_bytes(int fmt) {
    switch (fmt) {
        case PMSP_U8: return 1;
        case PMSP_F16: return 2;
        case PMSP_F32: return 4;
        default: return 0;
    }
}

int check_image(pmsp_ctx* c, const pmsp_image* im, const char* what) {
    if (!im || !im->data) return ctx_fail(c, PMSP_EINVAL, "%s: NULL image", what);
    const size_t eb = format_bytes(im->format);
    if (!eb) return ctx_fail(c, PMSP_EINVAL, "%s: unknown format %d", what, im->format);
    if (im->w < 2 || im->h < 1 || im->w > 16384 || im->h > 16384)
        return ctx_fail(c, PMSP_EINVAL, "%s: size %dx%d outside [2..16384]x[1..16384]", what, im->w, im->h);
    if (im->pitch_bytes < (int64_t)(im->w * eb))
        return ctx_fail(c, PMSP_EINVAL, "%s: pitch %lld < row bytes", what, (long long)im->pitch_bytes);
    if (im->memory != PMSP_HOST && im->memory != PMSP_DEVICE)
        return ctx_fail(c, PMSP_EINVAL, "%s: unknown memory kind", what);
    // device images are read in place element by element (the reference tile,
    // the no-alloc source fetch): a misaligned row would fault on the GPU
    if (im->memory == PMSP_DEVICE && (((uintptr_t)im->data % eb) != 0 || (im->pitch_bytes % (int64_t)eb) != 0))
        return ctx_fail(c, PMSP_EINVAL, "%s: device data and pitch must be multiples of %zu bytes", what, eb);
    return PMSP_OK;
}

int check_panorama(pmsp_ctx* c, const pmsp_image* im, const char* what) {
    const int rc = check_image(c, im, what);
    if (rc) return rc;
    if ((im->w | im->h) & 1)  // the projection folds W/2 and H/2 into constant offsets (project_dir_half)
        return ctx_fail(c, PMSP_EINVAL, "%s: size %dx%d must be even in both directions", what, im->w, im->h);
    return PMSP_OK;
}

// Reference->target pose in FP64: R = R_t R_r^T, t = t_t - R t_r.
void compose_rel(const pmsp_pose& r, const pmsp_pose& s, double R[9], double t[3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += s.R[3 * i + k] * r.R[3 * j + k];
            R[3 * i + j] = acc;
        }
    for (int i = 0; i < 3; ++i) {
        double acc = 0.0;
        for (int k = 0; k < 3; ++k) acc += R[3 * i + k] * r.t[k];
        t[i] = s.t[i] - acc;
    }
}

int ensure_buffer(pmsp_ctx* c, DevBuffer& b, size_t bytes) {
    if (b.bytes >= bytes) return PMSP_OK;
    if (b.ptr) {
        cudaStreamSynchronize(c->stream);
        cudaFree(b.ptr);
    }
    b.ptr = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaMalloc(&b.ptr, bytes);
    if (e != cudaSuccess) return ctx_fail(c, PMSP_ENOMEM, "device allocation of %zu bytes: %s", bytes,
                                          cudaGetErrorString(e));
    b.bytes = bytes;
    return PMSP_OK;
}

void free_texture(TexImage& t) {
    if (t.tex) cudaDestroyTextureObject(t.tex);
    if (t.arr) cudaFreeArray(t.arr);
    t = TexImage{};
}

// Copy an image into a gather-capable texture (x wraps, y clamps, normalised
// coordinates; uint8 reads as DN/255).
int upload_texture(pmsp_ctx* c, TexImage& t, const pmsp_image* im, cudaStream_t st) {
    if (t.arr && (t.w != im->w || t.h != im->h || t.fmt != im->format)) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(c, e, "sync before texture resize");
        free_texture(t);
    }
    if (!t.arr) {
        cudaChannelFormatDesc desc;
        if (im->format == PMSP_U8) desc = cudaCreateChannelDesc<unsigned char>();
        else if (im->format == PMSP_F16) desc = cudaCreateChannelDescHalf();
        else desc = cudaCreateChannelDesc<float>();
        cudaError_t e = cudaMallocArray(&t.arr, &desc, im->w, im->h, cudaArrayTextureGather);
        if (e != cudaSuccess) {
            t.arr = nullptr;
            return ctx_fail(c, PMSP_ENOMEM, "texture array %dx%d: %s", im->w, im->h, cudaGetErrorString(e));
        }
        cudaResourceDesc rd;
        memset(&rd, 0, sizeof rd);
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = t.arr;
        cudaTextureDesc td;
        memset(&td, 0, sizeof td);
        td.addressMode[0] = cudaAddressModeWrap;
        td.addressMode[1] = cudaAddressModeClamp;
        td.filterMode = cudaFilterModePoint;
        td.readMode = im->format == PMSP_U8 ? cudaReadModeNormalizedFloat : cudaReadModeElementType;
        td.normalizedCoords = 1;
        e = cudaCreateTextureObject(&t.tex, &rd, &td, nullptr);
        if (e != cudaSuccess) {
            cudaFreeArray(t.arr);
            t = TexImage{};
            return cuda_fail(c, e, "texture object");
        }
        t.w = im->w;
        t.h = im->h;
        t.fmt = im->format;
    }
    const size_t row = (size_t)im->w * format_bytes(im->format);
    cudaError_t e = cudaMemcpy2DToArrayAsync(t.arr, 0, 0, im->data, im->pitch_bytes, row, im->h,
                                             im->memory == PMSP_HOST ? cudaMemcpyHostToDevice
                                                                     : cudaMemcpyDeviceToDevice,
                                             st);
    if (e != cudaSuccess) return cuda_fail(c, e, "texture upload");
    return PMSP_OK;
}

int check_params(pmsp_ctx* c, const pmsp_params* p, int n_src) {
    if (!p) return ctx_fail(c, PMSP_EINVAL, "NULL params");
    if (n_src < 1 || n_src > PMSP_MAX_SOURCES)
        return ctx_fail(c, PMSP_EINVAL, "n_src %d outside [1, %d]", n_src, PMSP_MAX_SOURCES);
    if (p->best_k < 1 || p->best_k > n_src)
        return ctx_fail(c, PMSP_EINVAL, "best_k %d outside [1, n_src=%d]", p->best_k, n_src);
    if (p->patch_w < 1 || p->patch_w > PMSP_MAX_PATCH_W || (p->patch_w & 1) == 0)
        return ctx_fail(c, PMSP_EINVAL, "patch_w %d must be odd in [1, %d]", p->patch_w, PMSP_MAX_PATCH_W);
    if (p->patch_stride < 1) return ctx_fail(c, PMSP_EINVAL, "patch_stride %d < 1", p->patch_stride);
    if (!(p->d_min > 0.f) || !(p->d_max > p->d_min) || !std::isfinite(p->d_max))
        return ctx_fail(c, PMSP_EINVAL, "range bounds must satisfy 0 < d_min < d_max < inf");
    if (p->iterations < 0 || p->n_refine < 0 || p->n_refine > 30)
        return ctx_fail(c, PMSP_EINVAL, "iterations / n_refine out of range");
    if (p->neighbor_table != 0 && p->neighbor_table != 1)
        return ctx_fail(c, PMSP_EINVAL, "neighbor_table %d not in {0, 1}", p->neighbor_table);
    return PMSP_OK;
}

int check_maps(pmsp_ctx* c, const pmsp_maps* m, int W, int H, bool need_normal, bool need_cost,
               const char* what) {
    if (!m) return ctx_fail(c, PMSP_EINVAL, "%s: NULL maps", what);
    if (m->w != W || m->h != H)
        return ctx_fail(c, PMSP_EINVAL, "%s: maps %dx%d do not match %dx%d", what, m->w, m->h, W, H);
    if (m->memory != PMSP_HOST && m->memory != PMSP_DEVICE)
        return ctx_fail(c, PMSP_EINVAL, "%s: unknown memory kind", what);
    if (!m->depth || (need_normal && !m->normal) || (need_cost && !m->cost))
        return ctx_fail(c, PMSP_EINVAL, "%s: NULL map pointer", what);
    return PMSP_OK;
}

// Everything a per-pixel launch needs: checks, textures, reference, poses.
int prepare_problem(pmsp_ctx* c, const pmsp_image* ref, const pmsp_pose* ref_pose, const pmsp_image* srcs,
                    const pmsp_pose* src_poses, int n_src, const pmsp_params* p, PixelParams& P) {
    int rc = check_params(c, p, n_src);
    if (rc) return rc;
    if ((rc = check_panorama(c, ref, "reference"))) return rc;
    if (ref->w & 1) return ctx_fail(c, PMSP_EINVAL, "reference width %d must be even", ref->w);
    if (!ref_pose || !srcs || !src_poses) return ctx_fail(c, PMSP_EINVAL, "NULL pose or source array");
    for (int s = 0; s < n_src; ++s)
        if ((rc = check_panorama(c, &srcs[s], "source"))) return rc;

    if ((int)c->src_tex.size() < n_src) c->src_tex.resize(n_src);
    cudaTextureObject_t tex[PMSP_MAX_SOURCES];
    for (int s = 0; s < n_src; ++s) {
        if ((rc = upload_texture(c, c->src_tex[s], &srcs[s], c->stream))) return rc;
        tex[s] = c->src_tex[s].tex;
    }
    const void* ref_dev = ref->data;
    int64_t ref_pitch = ref->pitch_bytes;
    if (ref->memory != PMSP_DEVICE) {
        const size_t row = (size_t)ref->w * format_bytes(ref->format);
        if ((rc = ensure_buffer(c, c->ref_stage, row * ref->h))) return rc;
        cudaError_t e = cudaMemcpy2DAsync(c->ref_stage.ptr, row, ref->data, ref->pitch_bytes, row, ref->h,
                                          cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "reference upload");
        ref_dev = c->ref_stage.ptr;
        ref_pitch = (int64_t)row;
    }
    fill_problem(P, ref, ref_dev, ref_pitch, ref_pose, srcs, tex, src_poses, n_src, p);
    P.err = c->d_err;
    return PMSP_OK;
}

// Kernel parameters of one problem from validated arguments: FP64 pose
// composition cast to FP32, projection scales, window and weight constants.
void fill_problem(PixelParams& P, const pmsp_image* ref, const void* ref_dev, int64_t ref_pitch,
                  const pmsp_pose* ref_pose, const pmsp_image* srcs, const cudaTextureObject_t* tex,
                  const pmsp_pose* src_poses, int n_src, const pmsp_params* p) {
    memset(&P, 0, sizeof P);
    for (int s = 0; s < n_src; ++s) {
        double R[9], t[3];
        compose_rel(*ref_pose, src_poses[s], R, t);
        SourceView& V = P.src[s];
        V.tex = tex[s];
        for (int k = 0; k < 9; ++k) V.R[k] = (float)R[k];
        for (int k = 0; k < 3; ++k) V.t[k] = (float)t[k];
        const double Ws = srcs[s].w, Hs = srcs[s].h;
        V.su = (float)(Ws / (2.0 * M_PI));
        V.ou = (float)(0.5 * Ws - 0.5);
        V.sv = (float)(-Hs / M_PI);
        V.ov = (float)(0.5 * Hs - 0.5);
        V.inv_w = (float)(1.0 / Ws);
        V.inv_h = (float)(1.0 / Hs);
    }
    for (int q = 0; 2 * q < n_src; ++q) {
        const SourceView& A = P.src[2 * q];
        const SourceView& B = P.src[2 * q + 1 < n_src ? 2 * q + 1 : 2 * q];
        PixelParams::ViewPair& VP = P.pairs[q];
        for (int k = 0; k < 9; ++k) VP.R[k] = make_float2(A.R[k], B.R[k]);
        for (int k = 0; k < 3; ++k) VP.t[k] = make_float2(A.t[k], B.t[k]);
        VP.su = make_float2(A.su, B.su);
        VP.nsv = make_float2(-A.sv, -B.sv);
        VP.inv_w = make_float2(A.inv_w, B.inv_w);
        VP.inv_h = make_float2(A.inv_h, B.inv_h);
    }
    P.ref = static_cast<const uint8_t*>(ref_dev);
    P.ref_pitch = ref_pitch;
    P.ref_format = ref->format;
    P.W = ref->w;
    P.H = ref->h;
    P.d_min = p->d_min;
    P.d_max = p->d_max;
    P.inv_dmin = 1.0f / p->d_min;
    P.inv_dmax = 1.0f / p->d_max;
    P.S = n_src;
    P.radius = (p->patch_w - 1) / 2;
    P.stride = p->patch_stride;
    P.K = (2 * P.radius) / P.stride + 1;
    P.best_k = p->best_k;
    P.n_refine = p->n_refine;
    P.table = p->neighbor_table;
    const double log2e = 1.4426950408889634;
    P.wc = p->sigma_color > 0 ? (float)(-log2e / (2.0 * (double)p->sigma_color * p->sigma_color)) : 0.f;
    P.ws = p->sigma_space > 0 ? (float)(-log2e / (2.0 * (double)p->sigma_space * p->sigma_space)) : 0.f;
    P.seed = p->seed;
    P.keyframe = p->keyframe_id;
}

// Bind state planes: device maps directly, host maps through staging.
int bind_maps(pmsp_ctx* c, pmsp_maps* m, PixelParams& P, bool copy_in) {
    const size_t N = (size_t)P.W * P.H;
    if (m->memory == PMSP_DEVICE) {
        P.depth = m->depth;
        P.nx = m->normal;
        P.ny = m->normal ? m->normal + N : nullptr;
        P.nz = m->normal ? m->normal + 2 * N : nullptr;
        P.cost = m->cost;
        return PMSP_OK;
    }
    int rc = ensure_buffer(c, c->map_stage, 5 * N * sizeof(float));
    if (rc) return rc;
    float* base = static_cast<float*>(c->map_stage.ptr);
    P.depth = base;
    P.nx = base + N;
    P.ny = base + 2 * N;
    P.nz = base + 3 * N;
    P.cost = base + 4 * N;
    if (copy_in) {
        cudaError_t e = cudaMemcpyAsync(P.depth, m->depth, N * sizeof(float), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess && m->normal)
            e = cudaMemcpyAsync(P.nx, m->normal, 3 * N * sizeof(float), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess && m->cost)
            e = cudaMemcpyAsync(P.cost, m->cost, N * sizeof(float), cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "map upload");
    }
    return PMSP_OK;
}

int finish_maps(pmsp_ctx* c, pmsp_maps* m, const PixelParams& P, bool depth_normal_out) {
    if (m->memory == PMSP_DEVICE) return PMSP_OK;
    const size_t N = (size_t)P.W * P.H;
    cudaError_t e = cudaSuccess;
    if (depth_normal_out) {
        e = cudaMemcpyAsync(m->depth, P.depth, N * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(m->normal, P.nx, 3 * N * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->cost, P.cost, N * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "map download");
    return pmsp_sync(c);
}

int launch(pmsp_ctx* c, const PixelParams& P, int mode) {
    cudaError_t e = launch_pixel_kernel(P, mode, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
    return PMSP_OK;
}

}  // namespace pmsp

extern "C" {

void pmsp_default_params(pmsp_params* p) {
    if (!p) return;
    p->d_min = 0.3f;
    p->d_max = 10.0f;
    p->patch_w = 11;
    p->patch_stride = 2;
    p->iterations = 8;
    p->best_k = 3;
    p->sigma_color = 0.2f;
    p->sigma_space = 3.0f;
    p->n_refine = 6;
    p->neighbor_table = 0;
    p->seed = 42;
    p->keyframe_id = 0;
}

int pmsp_create(pmsp_ctx** out, const pmsp_ctx_opts* opts) {
    if (!out) return PMSP_EINVAL;
    *out = nullptr;
    if (opts && opts->scheduler != PMSP_SCHED_LANES && opts->scheduler != PMSP_SCHED_STEPS) return PMSP_EINVAL;
    pmsp_ctx* c = new (std::nothrow) pmsp_ctx();
    if (!c) return PMSP_ENOMEM;
    c->device = opts ? opts->device : 0;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) {
        delete c;
        return PMSP_ECUDA;
    }
    if (opts && opts->stream) {
        c->stream = static_cast<cudaStream_t>(opts->stream);
        c->own_stream = false;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return PMSP_ECUDA;
        }
        c->own_stream = true;
    }
    c->mem_cap = (opts && opts->mem_cap_bytes) ? opts->mem_cap_bytes : (40ull << 30);
    c->ring_capacity = (opts && opts->ring_capacity > 0) ? opts->ring_capacity : 64;
    c->max_active = (opts && opts->max_active > 0) ? opts->max_active : 32;
    c->scheduler = opts ? opts->scheduler : PMSP_SCHED_LANES;
    e = cudaMalloc(&c->d_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(unsigned));
    if (e != cudaSuccess) {
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return PMSP_ENOMEM;
    }
    *out = c;
    return PMSP_OK;
}

int pmsp_destroy(pmsp_ctx* c) {
    if (!c) return PMSP_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    runtime_shutdown(c);
    for (auto& t : c->src_tex) free_texture(t);
    free_texture(c->sample_tex);
    for (DevBuffer* b : {&c->ref_stage, &c->map_stage, &c->filter_stage, &c->sample_stage, &c->median_stage,
                         &c->warp_zbuf, &c->warp_prev, &c->cloud_table, &c->cloud_stage})
        if (b->ptr) cudaFree(b->ptr);
    if (c->d_err) cudaFree(c->d_err);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return PMSP_OK;
}

const char* pmsp_last_error(pmsp_ctx* c) { return c ? c->err : "NULL context"; }

int pmsp_sync(pmsp_ctx* c) {
    if (!c) return PMSP_EINVAL;
    cudaSetDevice(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronise");
    unsigned flag = 0;
    e = cudaMemcpy(&flag, c->d_err, sizeof flag, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "error flag read");
    if (flag) {
        // report once: the flag is cleared so later calls on the context start clean
        e = cudaMemset(c->d_err, 0, sizeof(unsigned));
        if (e != cudaSuccess) return cuda_fail(c, e, "error flag reset");
        return ctx_fail(c, PMSP_EDEVICE, "kernel error flag 0x%x", flag);
    }
    return PMSP_OK;
}

int pmsp_densify(pmsp_ctx* c, const pmsp_image* ref, const pmsp_pose* ref_pose, const pmsp_image* srcs,
                 const pmsp_pose* src_poses, int n_src, const pmsp_params* p, pmsp_maps* out) {
    if (!c) return PMSP_EINVAL;
    cudaSetDevice(c->device);
    PixelParams P;
    int rc = prepare_problem(c, ref, ref_pose, srcs, src_poses, n_src, p, P);
    if (rc) return rc;
    if ((rc = check_maps(c, out, ref->w, ref->h, true, true, "output"))) return rc;
    if ((rc = bind_maps(c, out, P, false))) return rc;
    for (int colour = 0; colour < 2; ++colour) {
        P.colour = colour;
        if ((rc = launch(c, P, MODE_INIT))) return rc;
    }
    for (int it = 0; it < p->iterations; ++it)
        for (int colour = 0; colour < 2; ++colour) {
            P.colour = colour;
            P.iter = it;
            if ((rc = launch(c, P, MODE_SWEEP))) return rc;
        }
    return finish_maps(c, out, P, true);
}

}  // extern "C"

namespace pmsp {

// Warping initialisation into P's planes, then the initial costs.
static int warp_init_into(pmsp_ctx* c, PixelParams& P, const pmsp_maps* prev, const pmsp_pose* prev_pose,
                          const pmsp_pose* ref_pose, int32_t* src) {
    if (!prev || !prev->depth || !prev->normal || !prev_pose)
        return ctx_fail(c, PMSP_EINVAL, "previous keyframe: depth, normal and pose are required");
    if (prev->w < 2 || prev->h < 1 || (prev->memory != PMSP_HOST && prev->memory != PMSP_DEVICE))
        return ctx_fail(c, PMSP_EINVAL, "previous keyframe: bad maps");
    WarpArgs A;
    memset(&A, 0, sizeof A);
    A.Wp = prev->w;
    A.Hp = prev->h;
    const size_t Np = (size_t)A.Wp * A.Hp;
    int rc;
    if (prev->memory == PMSP_DEVICE) {
        A.prev_depth = prev->depth;
        A.prev_normal = prev->normal;
    } else {
        if ((rc = ensure_buffer(c, c->warp_prev, 4 * Np * sizeof(float)))) return rc;
        float* base = static_cast<float*>(c->warp_prev.ptr);
        cudaError_t e = cudaMemcpyAsync(base, prev->depth, Np * 4, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(base + Np, prev->normal, 3 * Np * 4, cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "previous maps upload");
        A.prev_depth = base;
        A.prev_normal = base + Np;
    }
    double R[9], t[3];
    compose_rel(*prev_pose, *ref_pose, R, t);  // previous camera -> current camera
    for (int k = 0; k < 9; ++k) A.R[k] = (float)R[k];
    for (int k = 0; k < 3; ++k) A.t[k] = (float)t[k];
    A.W = P.W;
    A.H = P.H;
    A.su = (float)(P.W / (2.0 * M_PI));
    A.ou = (float)(0.5 * P.W - 0.5);
    A.sv = (float)(-P.H / M_PI);
    A.ov = (float)(0.5 * P.H - 0.5);
    if ((rc = ensure_buffer(c, c->warp_zbuf, (size_t)P.W * P.H * sizeof(unsigned long long)))) return rc;
    A.zbuf = static_cast<unsigned long long*>(c->warp_zbuf.ptr);
    A.src = src;
    cudaError_t e = launch_warp_init(P, A, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "warp launch");
    for (int colour = 0; colour < 2; ++colour) {
        P.colour = colour;
        if ((rc = launch(c, P, MODE_COST))) return rc;
    }
    return PMSP_OK;
}

}  // namespace pmsp

extern "C" {

int pmsp_warp_init(pmsp_ctx* c, const pmsp_image* ref, const pmsp_pose* ref_pose, const pmsp_image* srcs,
                   const pmsp_pose* src_poses, int n_src, const pmsp_params* p, const pmsp_maps* prev,
                   const pmsp_pose* prev_pose, pmsp_maps* out, int32_t* src) {
    if (!c) return PMSP_EINVAL;
    cudaSetDevice(c->device);
    PixelParams P;
    int rc = prepare_problem(c, ref, ref_pose, srcs, src_poses, n_src, p, P);
    if (rc) return rc;
    if ((rc = check_maps(c, out, ref->w, ref->h, true, true, "output"))) return rc;
    if (out->memory != PMSP_DEVICE) return ctx_fail(c, PMSP_EINVAL, "pmsp_warp_init writes device maps only");
    if ((rc = bind_maps(c, out, P, false))) return rc;
    return warp_init_into(c, P, prev, prev_pose, ref_pose, src);
}

int pmsp_densify_warped(pmsp_ctx* c, const pmsp_image* ref, const pmsp_pose* ref_pose, const pmsp_image* srcs,
                        const pmsp_pose* src_poses, int n_src, const pmsp_params* p, const pmsp_maps* prev,
                        const pmsp_pose* prev_pose, pmsp_maps* out) {
    if (!c) return PMSP_EINVAL;
    cudaSetDevice(c->device);
    PixelParams P;
    int rc = prepare_problem(c, ref, ref_pose, srcs, src_poses, n_src, p, P);
    if (rc) return rc;
    if ((rc = check_maps(c, out, ref->w, ref->h, true, true, "output"))) return rc;
    if ((rc = bind_maps(c, out, P, false))) return rc;
    if ((rc = warp_init_into(c, P, prev, prev_pose, ref_pose, nullptr))) return rc;
    for (int it = 0; it < p->iterations; ++it)
        for (int colour = 0; colour < 2; ++colour) {
            P.colour = colour;
            P.iter = it;
            if ((rc = launch(c, P, MODE_SWEEP))) return rc;
        }
    return finish_maps(c, out, P, true);
}

int pmsp_cost_map(pmsp_ctx* c, const pmsp_image* ref, const pmsp_pose* ref_pose, const pmsp_image* srcs,
                  const pmsp_pose* src_poses, int n_src, const pmsp_params* p, pmsp_maps* planes) {
    if (!c) return PMSP_EINVAL;
    cudaSetDevice(c->device);
    PixelParams P;
    int rc = prepare_problem(c, ref, ref_pose, srcs, src_poses, n_src, p, P);
    if (rc) return rc;
    if ((rc = check_maps(c, planes, ref->w, ref->h, true, true, "planes"))) return rc;
    if ((rc = bind_maps(c, planes, P, true))) return rc;
    for (int colour = 0; colour < 2; ++colour) {
        P.colour = colour;
        if ((rc = launch(c, P, MODE_COST))) return rc;
    }
    return finish_maps(c, planes, P, false);
}

int pmsp_init(pmsp_ctx* c, const pmsp_image* ref, const pmsp_pose* ref_pose, const pmsp_image* srcs,
              const pmsp_pose* src_poses, int n_src, const pmsp_params* p, pmsp_maps* out) {
    if (!c) return PMSP_EINVAL;
    cudaSetDevice(c->device);
    PixelParams P;
    int rc = prepare_problem(c, ref, ref_pose, srcs, src_poses, n_src, p, P);
    if (rc) return rc;
    if ((rc = check_maps(c, out, ref->w, ref->h, true, true, "output"))) return rc;
    if ((rc = bind_maps(c, out, P, false))) return rc;
    for (int colour = 0; colour < 2; ++colour) {
        P.colour = colour;
        if ((rc = launch(c, P, MODE_INIT))) return rc;
    }
    return finish_maps(c, out, P, true);
}

int pmsp_halfsweep(pmsp_ctx* c, const pmsp_image* ref, const pmsp_pose* ref_pose, const pmsp_image* srcs,
                   const pmsp_pose* src_poses, int n_src, const pmsp_params* p, int colour, int iteration,
                   pmsp_maps* state) {
    if (!c) return PMSP_EINVAL;
    cudaSetDevice(c->device);
    if (colour != 0 && colour != 1) return ctx_fail(c, PMSP_EINVAL, "colour %d not in {0, 1}", colour);
    if (iteration < 0) return ctx_fail(c, PMSP_EINVAL, "iteration %d < 0", iteration);
    PixelParams P;
    int rc = prepare_problem(c, ref, ref_pose, srcs, src_poses, n_src, p, P);
    if (rc) return rc;
    if ((rc = check_maps(c, state, ref->w, ref->h, true, true, "state"))) return rc;
    if ((rc = bind_maps(c, state, P, true))) return rc;
    P.colour = colour;
    P.iter = iteration;
    if ((rc = launch(c, P, MODE_SWEEP))) return rc;
    return finish_maps(c, state, P, true);
}

int pmsp_consistency_filter(pmsp_ctx* c, const pmsp_maps* ref, const pmsp_pose* ref_pose, const pmsp_maps* nbrs,
                            const pmsp_pose* nbr_poses, int n, float max_reproj_px, int min_views,
                            pmsp_maps* inout, int32_t* agree) {
    if (!c) return PMSP_EINVAL;
    cudaSetDevice(c->device);
    if (!ref || !ref->depth || !ref_pose || !inout || !inout->depth)
        return ctx_fail(c, PMSP_EINVAL, "NULL reference or output");
    if (n < 1 || n > PMSP_MAX_SOURCES || !nbrs || !nbr_poses)
        return ctx_fail(c, PMSP_EINVAL, "neighbour count %d outside [1, %d]", n, PMSP_MAX_SOURCES);
    if (!(max_reproj_px > 0.f) || min_views < 0)
        return ctx_fail(c, PMSP_EINVAL, "max_reproj_px must be > 0 and min_views >= 0");
    const int W = ref->w, H = ref->h;
    if (W < 2 || H < 1 || inout->w != W || inout->h != H || inout->memory != ref->memory)
        return ctx_fail(c, PMSP_EINVAL, "output must match the reference size and memory kind");
    for (int j = 0; j < n; ++j)
        if (!nbrs[j].depth || nbrs[j].w < 2 || nbrs[j].h < 1 || nbrs[j].memory != ref->memory)
            return ctx_fail(c, PMSP_EINVAL, "neighbour %d: bad depth map", j);

    FilterParams F;
    memset(&F, 0, sizeof F);
    F.W = W;
    F.H = H;
    F.n = n;
    F.min_views = min_views;
    F.max_px = max_reproj_px;
    const bool host = ref->memory == PMSP_HOST;
    const size_t N = (size_t)W * H;
    auto rounded = [](size_t bytes) { return (bytes + 255) & ~size_t(255); };
    int rc;
    char* stage = nullptr;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* q = stage + off;
        off += rounded(bytes);
        return q;
    };
    if (host) {
        size_t need = 3 * rounded(N * 4);
        for (int j = 0; j < n; ++j) need += rounded((size_t)nbrs[j].w * nbrs[j].h * 4);
        if ((rc = ensure_buffer(c, c->filter_stage, need))) return rc;
        stage = static_cast<char*>(c->filter_stage.ptr);
        float* din = reinterpret_cast<float*>(take(N * 4));
        cudaError_t e = cudaMemcpyAsync(din, ref->depth, N * 4, cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "filter upload");
        F.depth_in = din;
        F.depth_out = reinterpret_cast<float*>(take(N * 4));
        F.agree = agree ? reinterpret_cast<int32_t*>(take(N * 4)) : nullptr;
    } else {
        F.depth_in = ref->depth;
        F.depth_out = inout->depth;
        F.agree = agree;
    }
    for (int j = 0; j < n; ++j) {
        FilterView& V = F.nb[j];
        V.W = nbrs[j].w;
        V.H = nbrs[j].h;
        if (host) {
            const size_t bytes = (size_t)V.W * V.H * 4;
            float* d = reinterpret_cast<float*>(take(bytes));
            cudaError_t e = cudaMemcpyAsync(d, nbrs[j].depth, bytes, cudaMemcpyHostToDevice, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "filter upload");
            V.depth = d;
        } else {
            V.depth = nbrs[j].depth;
        }
        double R[9], t[3];
        compose_rel(*ref_pose, nbr_poses[j], R, t);
        for (int k = 0; k < 9; ++k) V.Rf[k] = (float)R[k];
        for (int k = 0; k < 3; ++k) V.tf[k] = (float)t[k];
        compose_rel(nbr_poses[j], *ref_pose, R, t);
        for (int k = 0; k < 9; ++k) V.Rb[k] = (float)R[k];
        for (int k = 0; k < 3; ++k) V.tb[k] = (float)t[k];
    }
    cudaError_t e = launch_filter_kernel(F, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "filter launch");
    if (host) {
        e = cudaMemcpyAsync(inout->depth, F.depth_out, N * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess && agree)
            e = cudaMemcpyAsync(agree, F.agree, N * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "filter download");
        return pmsp_sync(c);
    }
    return PMSP_OK;
}

int pmsp_median_filter(pmsp_ctx* c, const pmsp_maps* in, int radius, float tau, pmsp_maps* out) {
    if (!c) return PMSP_EINVAL;
    cudaSetDevice(c->device);
    if (!in || !in->depth || !out || !out->depth) return ctx_fail(c, PMSP_EINVAL, "NULL input or output depth");
    const int W = in->w, H = in->h;
    if (W < 1 || H < 1 || out->w != W || out->h != H || out->memory != in->memory)
        return ctx_fail(c, PMSP_EINVAL, "output must match the input size and memory kind");
    if (in->memory != PMSP_HOST && in->memory != PMSP_DEVICE) return ctx_fail(c, PMSP_EINVAL, "bad memory kind");
    if (out->depth == in->depth) return ctx_fail(c, PMSP_EINVAL, "output must not alias the input");
    if (radius < 1 || radius > 3) return ctx_fail(c, PMSP_EINVAL, "radius %d outside [1, 3]", radius);
    if (!(tau > 0.f)) return ctx_fail(c, PMSP_EINVAL, "tau must be > 0");
    const size_t bytes = (size_t)W * H * sizeof(float);
    const float* din = in->depth;
    float* dout = out->depth;
    int rc;
    const bool host = in->memory == PMSP_HOST;
    if (host) {
        const size_t half = (bytes + 255) & ~size_t(255);
        if ((rc = ensure_buffer(c, c->median_stage, 2 * half))) return rc;
        float* a = static_cast<float*>(c->median_stage.ptr);
        float* b = reinterpret_cast<float*>(static_cast<char*>(c->median_stage.ptr) + half);
        cudaError_t e = cudaMemcpyAsync(a, in->depth, bytes, cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "median upload");
        din = a;
        dout = b;
    }
    cudaError_t e = launch_median_kernel(din, dout, W, H, radius, tau, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "median launch");
    if (host) {
        e = cudaMemcpyAsync(out->depth, dout, bytes, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "median download");
        return pmsp_sync(c);
    }
    return PMSP_OK;
}

int pmsp_sample_bilinear(pmsp_ctx* c, const pmsp_image* img, int n, const float* uc, const float* vc,
                         float* out) {
    if (!c) return PMSP_EINVAL;
    cudaSetDevice(c->device);
    int rc = check_image(c, img, "image");
    if (rc) return rc;
    if (n < 0 || (n > 0 && (!uc || !vc || !out))) return ctx_fail(c, PMSP_EINVAL, "bad sample arrays");
    if (n == 0) return PMSP_OK;
    if ((rc = upload_texture(c, c->sample_tex, img, c->stream))) return rc;
    const float *du = uc, *dv = vc;
    float* dout = out;
    if (img->memory == PMSP_HOST) {
        if ((rc = ensure_buffer(c, c->sample_stage, 3 * (size_t)n * sizeof(float)))) return rc;
        float* base = static_cast<float*>(c->sample_stage.ptr);
        cudaError_t e = cudaMemcpyAsync(base, uc, n * 4, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(base + n, vc, n * 4, cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "sample upload");
        du = base;
        dv = base + n;
        dout = base + 2 * n;
    }
    cudaError_t e = launch_sample_kernel(c->sample_tex.tex, img->w, img->h, n, du, dv, dout, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "sample launch");
    if (img->memory == PMSP_HOST) {
        e = cudaMemcpyAsync(out, dout, n * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "sample download");
        return pmsp_sync(c);
    }
    return PMSP_OK;
}

int pmsp_project(pmsp_ctx* c, int W, int H, int n, const float* dirs, float* uc, float* vc, int memory) {
    if (!c) return PMSP_EINVAL;
    cudaSetDevice(c->device);
    if (W < 1 || H < 1 || n < 0 || (n > 0 && (!dirs || !uc || !vc)))
        return ctx_fail(c, PMSP_EINVAL, "bad projection arguments");
    if (memory != PMSP_HOST && memory != PMSP_DEVICE) return ctx_fail(c, PMSP_EINVAL, "unknown memory kind");
    if (n == 0) return PMSP_OK;
    const float* dd = dirs;
    float *du = uc, *dv = vc;
    int rc;
    if (memory == PMSP_HOST) {
        if ((rc = ensure_buffer(c, c->sample_stage, 5 * (size_t)n * sizeof(float)))) return rc;
        float* base = static_cast<float*>(c->sample_stage.ptr);
        cudaError_t e = cudaMemcpyAsync(base, dirs, 3 * (size_t)n * 4, cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "projection upload");
        dd = base;
        du = base + 3 * (size_t)n;
        dv = base + 4 * (size_t)n;
    }
    cudaError_t e = launch_project_kernel(W, H, n, dd, du, dv, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "projection launch");
    if (memory == PMSP_HOST) {
        e = cudaMemcpyAsync(uc, du, (size_t)n * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(vc, dv, (size_t)n * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "projection download");
        return pmsp_sync(c);
    }
    return PMSP_OK;
}

}  // extern "C"
