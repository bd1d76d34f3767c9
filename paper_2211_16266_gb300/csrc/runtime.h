// Host-side context of the densification library.
#pragma once

#include <cuda_runtime.h>

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

int ctx_fail(pmsp_ctx* c, int code, const char* fmt, ...);
int cuda_fail(pmsp_ctx* c, cudaError_t e, const char* what);
void runtime_shutdown(pmsp_ctx* c);

}  // namespace pmsp

struct pmsp_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    unsigned* d_err = nullptr;  // device error word written by kernels
    uint64_t mem_cap = 0;
    int ring_capacity = 0;
    int max_active = 0;
    std::vector<pmsp::TexImage> src_tex;  // one texture per source slot
    pmsp::TexImage sample_tex;
    pmsp::DevBuffer ref_stage, map_stage, filter_stage, sample_stage;
    pmsp::Serving* serving = nullptr;
};
