// Host-side context of the densification library.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "pmsp.h"

namespace pmsp {

struct DevBuffer {
    void* ptr = nullptr;
    size_t bytes = 0;
};

// A source image held as a gather-capable 2-D texture.
struct TexImage {
    cudaArray_t arr = nullptr;
    cudaTextureObject_t tex = 0;
    int w = 0, h = 0, fmt = -1;
};

struct Serving;  // continuous-batching runtime (serving calls)

struct PixelParams;
struct BatchEngine;

int ctx_fail(pmsp_ctx* c, int code, const char* fmt, ...);
int cuda_fail(pmsp_ctx* c, cudaError_t e, const char* what);
void runtime_shutdown(pmsp_ctx* c);
size_t format_bytes(int fmt);
int check_image(pmsp_ctx* c, const pmsp_image* im, const char* what);
// check_image plus even width and height: every image the densification reads.
int check_panorama(pmsp_ctx* c, const pmsp_image* im, const char* what);
int check_params(pmsp_ctx* c, const pmsp_params* p, int n_src);
int check_maps(pmsp_ctx* c, const pmsp_maps* m, int W, int H, bool need_normal, bool need_cost, const char* what);
int ensure_buffer(pmsp_ctx* c, DevBuffer& b, size_t bytes);
int upload_texture(pmsp_ctx* c, TexImage& t, const pmsp_image* im, cudaStream_t st);
void free_texture(TexImage& t);
void compose_rel(const pmsp_pose& r, const pmsp_pose& s, double R[9], double t[3]);
void fill_problem(PixelParams& P, const pmsp_image* ref, const void* ref_dev, int64_t ref_pitch,
                  const pmsp_pose* ref_pose, const pmsp_image* srcs, const cudaTextureObject_t* tex,
                  const pmsp_pose* src_poses, int n_src, const pmsp_params* p);
void batch_shutdown(pmsp_ctx* c);
struct BatchArgs;
int batch_bucket(int max_s);
int batch_blocks_per_sm(int bucket);
cudaError_t batch_launch(int bucket, const BatchArgs& a, int grid, cudaStream_t st);

}  // namespace pmsp

struct pmsp_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // last error text: fixed storage (the pointer pmsp_last_error returns stays
    // valid), written under err_mu because the serving calls may fail on
    // different threads at once
    char err[512] = {0};
    std::mutex err_mu;
    unsigned* d_err = nullptr;  // device error word written by kernels
    uint64_t mem_cap = 0;
    int ring_capacity = 0;
    int max_active = 0;
    int scheduler = 0;  // pmsp_scheduler of the serving runtime
    std::vector<pmsp::TexImage> src_tex;  // one texture per source slot
    pmsp::TexImage sample_tex;
    pmsp::DevBuffer ref_stage, map_stage, filter_stage, sample_stage, median_stage;
    pmsp::DevBuffer cloud_table, cloud_stage;  // fusion (hash table, marks, staging); view filter, completeness
    pmsp::DevBuffer warp_zbuf, warp_prev;  // plane-map warping: claims, staged previous maps
    pmsp::Serving* serving = nullptr;
    pmsp::BatchEngine* batch = nullptr;
};
