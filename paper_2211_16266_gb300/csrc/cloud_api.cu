// C entry points of the point kernels (cloud.cu): View Filter, point-cloud
// fusion and keyframe completeness. Host buffers are staged through context
// buffers; every call returns after its results are on the host side of the
// caller (counts are always read back).
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "runtime.h"

using namespace pmsp;

namespace {

size_t rounded(size_t bytes) { return (bytes + 255) & ~size_t(255); }

bool valid_memory(int m) { return m == PMSP_HOST || m == PMSP_DEVICE; }

void centre_of(const pmsp_pose& P, float c[3]) {
    for (int k = 0; k < 3; ++k) c[k] = (float)-(P.R[k] * P.t[0] + P.R[3 + k] * P.t[1] + P.R[6 + k] * P.t[2]);
}

// Upload n floats to a staging area when the caller's buffer is on the host.
int stage_in(pmsp_ctx* c, const float* src, size_t n, float* dst) {
    cudaError_t e = cudaMemcpyAsync(dst, src, n * sizeof(float), cudaMemcpyHostToDevice, c->stream);
    return e == cudaSuccess ? PMSP_OK : cuda_fail(c, e, "upload");
}

int read_count(pmsp_ctx* c, const unsigned long long* d_count, unsigned long long& out) {
    cudaError_t e = cudaMemcpyAsync(&out, d_count, sizeof out, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? PMSP_OK : cuda_fail(c, e, "count read-back");
}

}  // namespace

int pmsp_view_filter(pmsp_ctx* c, const pmsp_pose* a, const pmsp_pose* b, const float* points, int64_t n,
                     int memory, double min_deg, double max_deg, double min_frac, uint8_t* in_range,
                     int32_t* accepted, double* fraction) {
    if (!c) return PMSP_EINVAL;
    cudaSetDevice(c->device);
    if (!a || !b || !accepted) return ctx_fail(c, PMSP_EINVAL, "NULL pose or result");
    if (n < 0 || (n > 0 && !points) || !valid_memory(memory)) return ctx_fail(c, PMSP_EINVAL, "bad point array");
    if (!(min_deg >= 0 && min_deg <= max_deg && max_deg <= 180) || !(min_frac >= 0 && min_frac <= 1))
        return ctx_fail(c, PMSP_EINVAL, "need 0 <= min_deg <= max_deg <= 180 and 0 <= min_frac <= 1");
    const bool host = memory == PMSP_HOST;
    const size_t np = (size_t)n;
    size_t need = rounded(sizeof(unsigned long long));
    if (host) need += rounded(np * 3 * sizeof(float)) + (in_range ? rounded(np) : 0);
    int rc;
    if ((rc = ensure_buffer(c, c->cloud_stage, need))) return rc;
    char* base = static_cast<char*>(c->cloud_stage.ptr);
    ViewFilterArgs A;
    memset(&A, 0, sizeof A);
    A.count = reinterpret_cast<unsigned long long*>(base);
    A.n = n;
    A.points = points;
    A.flags = in_range;
    if (host) {
        float* p = reinterpret_cast<float*>(base + rounded(sizeof(unsigned long long)));
        if (n > 0 && (rc = stage_in(c, points, np * 3, p))) return rc;
        A.points = p;
        A.flags = in_range ? reinterpret_cast<unsigned char*>(base + rounded(sizeof(unsigned long long)) +
                                                              rounded(np * 3 * sizeof(float)))
                           : nullptr;
    }
    centre_of(*a, A.ca);
    centre_of(*b, A.cb);
    A.cos_min = (float)std::cos(min_deg * M_PI / 180.0);
    A.cos_max = (float)std::cos(max_deg * M_PI / 180.0);
    cudaError_t e = launch_view_filter(A, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "view filter launch");
    if (host && in_range && n > 0) {
        e = cudaMemcpyAsync(in_range, A.flags, np, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "view filter download");
    }
    unsigned long long cnt = 0;
    if ((rc = read_count(c, A.count, cnt))) return rc;
    const double f = n > 0 ? (double)cnt / (double)n : 0.0;
    if (fraction) *fraction = f;
    *accepted = f > min_frac ? 1 : 0;
    return PMSP_OK;
}

int pmsp_fuse(pmsp_ctx* c, const pmsp_maps* maps, const pmsp_pose* poses, int n, float voxel, float* points,
              int64_t* src, int64_t cap, int64_t* count) {
    if (!c) return PMSP_EINVAL;
    cudaSetDevice(c->device);
    if (!maps || !poses || !count) return ctx_fail(c, PMSP_EINVAL, "NULL maps, poses or count");
    if (n < 1 || n > MAX_FUSE_VIEWS) return ctx_fail(c, PMSP_EINVAL, "keyframe count %d outside [1, %d]", n,
                                                     MAX_FUSE_VIEWS);
    if (!(voxel > 0.f)) return ctx_fail(c, PMSP_EINVAL, "voxel must be > 0");
    if (cap < 0 || (cap > 0 && !points)) return ctx_fail(c, PMSP_EINVAL, "bad output capacity");
    const int memory = maps[0].memory;
    if (!valid_memory(memory)) return ctx_fail(c, PMSP_EINVAL, "bad memory kind");
    long long total = 0;
    for (int k = 0; k < n; ++k) {
        if (!maps[k].depth || maps[k].w < 1 || maps[k].h < 1 || maps[k].memory != memory)
            return ctx_fail(c, PMSP_EINVAL, "keyframe %d: bad depth map", k);
        total += (long long)maps[k].w * maps[k].h;
    }
    if (total >= (1ll << 31)) return ctx_fail(c, PMSP_EINVAL, "too many pixels to fuse in one call");
    unsigned long long slots = 1024;
    while (slots < 2ull * (unsigned long long)total) slots <<= 1;
    const int nb = (int)((total + 1023) / 1024);
    const bool host = memory == PMSP_HOST;
    const long long kept_max = cap < total ? cap : total;
    // context buffers: hash table | marks | block sums | count + error | host staging
    const size_t t_bytes = rounded(2 * slots * sizeof(unsigned long long));
    const size_t m_bytes = rounded((size_t)total * sizeof(unsigned)), s_bytes = rounded((size_t)nb * sizeof(unsigned));
    const size_t c_bytes = rounded(2 * sizeof(unsigned long long));
    size_t h_bytes = 0;
    if (host)
        h_bytes = rounded((size_t)total * sizeof(float)) + rounded((size_t)kept_max * 3 * sizeof(float)) +
                  rounded((size_t)kept_max * sizeof(long long));
    int rc;
    if ((rc = ensure_buffer(c, c->cloud_table, t_bytes + m_bytes + s_bytes + c_bytes + h_bytes))) return rc;
    char* base = static_cast<char*>(c->cloud_table.ptr);
    FuseArgs A;
    memset(&A, 0, sizeof A);
    A.keys = reinterpret_cast<unsigned long long*>(base);
    A.vals = A.keys + slots;
    A.mask = slots - 1;
    unsigned* mark = reinterpret_cast<unsigned*>(base + t_bytes);
    unsigned* sums = reinterpret_cast<unsigned*>(base + t_bytes + m_bytes);
    unsigned long long* d_count = reinterpret_cast<unsigned long long*>(base + t_bytes + m_bytes + s_bytes);
    A.err = reinterpret_cast<unsigned*>(d_count + 1);
    char* hs = base + t_bytes + m_bytes + s_bytes + c_bytes;
    A.inv_voxel = 1.0f / voxel;
    A.cap = cap;
    A.points = points;
    A.src = reinterpret_cast<long long*>(src);
    if (host) {
        A.points = reinterpret_cast<float*>(hs + rounded((size_t)total * sizeof(float)));
        A.src = src ? reinterpret_cast<long long*>(hs + rounded((size_t)total * sizeof(float)) +
                                                   rounded((size_t)kept_max * 3 * sizeof(float)))
                    : nullptr;
        A.cap = kept_max;
    }
    cudaError_t e = cudaMemsetAsync(A.err, 0, sizeof(unsigned), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "fuse setup");
    long long off = 0;
    for (int k = 0; k < n; ++k) {
        CloudView& V = A.views[k];
        V.W = maps[k].w;
        V.H = maps[k].h;
        V.depth = maps[k].depth;
        const size_t px = (size_t)V.W * V.H;
        if (host) {
            float* d = reinterpret_cast<float*>(hs) + off;
            if ((rc = stage_in(c, maps[k].depth, px, d))) return rc;
            V.depth = d;
        }
        for (int j = 0; j < 9; ++j) V.R[j] = (float)poses[k].R[j];
        for (int j = 0; j < 3; ++j) V.t[j] = (float)poses[k].t[j];
        A.base[k] = off;
        off += (long long)px;
    }
    e = launch_fuse(A, n, mark, sums, total, d_count, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "fuse launch");
    unsigned long long res[2] = {0, 0};
    e = cudaMemcpyAsync(res, d_count, sizeof res, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "fuse read-back");
    const unsigned err = (unsigned)res[1];
    if (err & ERR_RANGE) return ctx_fail(c, PMSP_EINVAL, "a point lies more than 2^20 voxels from the origin");
    if (err) return ctx_fail(c, PMSP_EDEVICE, "fuse error flag 0x%x", err);
    *count = (int64_t)res[0];
    if (host) {
        const long long kept = (long long)res[0] < kept_max ? (long long)res[0] : kept_max;
        if (kept > 0) {
            e = cudaMemcpyAsync(points, A.points, (size_t)kept * 3 * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess && src)
                e = cudaMemcpyAsync(src, A.src, (size_t)kept * sizeof(long long), cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "fuse download");
        }
    }
    return PMSP_OK;
}

int pmsp_completeness(pmsp_ctx* c, const float* points, int64_t n, int memory, const pmsp_pose* pose, int W,
                      int H, uint8_t* hit, double* completeness) {
    if (!c) return PMSP_EINVAL;
    cudaSetDevice(c->device);
    if (!pose || !completeness) return ctx_fail(c, PMSP_EINVAL, "NULL pose or result");
    if (n < 0 || (n > 0 && !points) || !valid_memory(memory)) return ctx_fail(c, PMSP_EINVAL, "bad point array");
    if (W < 1 || H < 1) return ctx_fail(c, PMSP_EINVAL, "panorama must be at least 1 x 1");
    const bool host = memory == PMSP_HOST;
    const size_t px = (size_t)W * H, np = (size_t)n;
    const bool own_hit = host || !hit;
    size_t need = rounded(sizeof(unsigned long long)) + (own_hit ? rounded(px) : 0) +
                  (host ? rounded(np * 3 * sizeof(float)) : 0);
    int rc;
    if ((rc = ensure_buffer(c, c->cloud_stage, need))) return rc;
    char* base = static_cast<char*>(c->cloud_stage.ptr);
    unsigned long long* d_count = reinterpret_cast<unsigned long long*>(base);
    CompletenessArgs A;
    memset(&A, 0, sizeof A);
    A.n = n;
    A.W = W;
    A.H = H;
    A.points = points;
    A.hit = own_hit ? reinterpret_cast<unsigned char*>(base + rounded(sizeof(unsigned long long))) : hit;
    if (host) {
        float* p = reinterpret_cast<float*>(base + rounded(sizeof(unsigned long long)) + rounded(px));
        if (n > 0 && (rc = stage_in(c, points, np * 3, p))) return rc;
        A.points = p;
    }
    for (int j = 0; j < 9; ++j) A.R[j] = (float)pose->R[j];
    for (int j = 0; j < 3; ++j) A.t[j] = (float)pose->t[j];
    A.su = (float)(W / (2.0 * M_PI));
    A.ou = (float)(0.5 * W - 0.5);
    A.sv = (float)(-H / M_PI);
    A.ov = (float)(0.5 * H - 0.5);
    cudaError_t e = launch_completeness(A, d_count, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "completeness launch");
    if (host && hit) {
        e = cudaMemcpyAsync(hit, A.hit, px, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "completeness download");
    }
    unsigned long long cnt = 0;
    if ((rc = read_count(c, d_count, cnt))) return rc;
    *completeness = (double)cnt / (double)px;
    return PMSP_OK;
}
