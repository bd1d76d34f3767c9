// Batched densification (pmsp_densify_batch) and its autotuner.
//
// A batch of keyframes runs phase by phase: the two initialisation colours,
// then red/black half-sweeps. Each phase is one launch of the persistent
// batched kernel over a work list of (keyframe, tile) items of every keyframe
// still in that phase. Source images are kept as gather-capable textures in
// a cache keyed by the caller's buffer, so a frame shared by several
// keyframes is uploaded once per call. With PMSP_BATCH_GRAPH the whole
// sequence (uploads, counters, launches) is captured in a CUDA graph and
// replayed while the caller submits the identical batch again.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "pmsp.h"
#include "runtime.h"

namespace pmsp {

using TexKey = std::tuple<const void*, int, int, int, int, int64_t>;

struct BatchPlan {
    std::vector<PixelParams> problems;
    std::vector<int4> work;        // all phases, concatenated
    std::vector<int> phase_off;    // phase p: work[phase_off[p], phase_off[p + 1])
    std::vector<int> n_phases;     // per keyframe
    std::vector<int64_t> pixels;   // per keyframe
    int max_s = 0;
    std::vector<std::pair<int, DevBuffer*>> host_out;  // items whose outputs are on the host
};

struct BatchEngine {
    std::map<TexKey, TexImage> tex;
    std::vector<DevBuffer> ref_stage, out_stage;
    DevBuffer d_problems, d_work, d_counters;
    void* h_problems = nullptr;  // pinned copies read by the captured graph
    void* h_work = nullptr;
    size_t h_problems_bytes = 0, h_work_bytes = 0;
    cudaEvent_t staged_ev = nullptr;  // recorded after the last eager read of the pinned copies
    cudaStream_t capture = nullptr;
    std::vector<cudaStream_t> branch;  // per-keyframe launch chains (strategy 1)
    std::vector<cudaEvent_t> join_ev;
    cudaEvent_t fork_ev = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<uint8_t> signature;
    int sms = 0;
};

// Kernel instance for the largest view count of a batch (register budget).
int batch_bucket(int max_s) { return max_s <= 4 ? 0 : max_s <= 6 ? 1 : max_s <= 8 ? 2 : max_s <= 10 ? 3 : 4; }

int batch_blocks_per_sm(int bucket) {
    static int occ[5] = {0, 0, 0, 0, 0};
    if (!occ[bucket]) {
        switch (bucket) {
            case 0: occ[0] = batch_kernel_blocks_per_sm_t<4>(); break;
            case 1: occ[1] = batch_kernel_blocks_per_sm_t<6>(); break;
            case 2: occ[2] = batch_kernel_blocks_per_sm_t<8>(); break;
            case 3: occ[3] = batch_kernel_blocks_per_sm_t<10>(); break;
            default: occ[4] = batch_kernel_blocks_per_sm_t<16>(); break;
        }
    }
    return occ[bucket];
}

cudaError_t batch_launch(int bucket, const BatchArgs& a, int grid, cudaStream_t st) {
    switch (bucket) {
        case 0: return launch_batch_kernel_t<4>(a, grid, st);
        case 1: return launch_batch_kernel_t<6>(a, grid, st);
        case 2: return launch_batch_kernel_t<8>(a, grid, st);
        case 3: return launch_batch_kernel_t<10>(a, grid, st);
        default: return launch_batch_kernel_t<16>(a, grid, st);
    }
}

static BatchEngine& engine(pmsp_ctx* c) {
    if (!c->batch) {
        c->batch = new BatchEngine();
        cudaDeviceGetAttribute(&c->batch->sms, cudaDevAttrMultiProcessorCount, c->device);
    }
    return *c->batch;
}

static void drop_graph(BatchEngine& b) {
    if (b.exec) cudaGraphExecDestroy(b.exec);
    b.exec = nullptr;
    b.signature.clear();
}

void batch_shutdown(pmsp_ctx* c) {
    if (!c->batch) return;
    BatchEngine& b = *c->batch;
    drop_graph(b);
    for (auto& kv : b.tex) free_texture(kv.second);
    for (auto* v : {&b.ref_stage, &b.out_stage})
        for (auto& d : *v)
            if (d.ptr) cudaFree(d.ptr);
    for (DevBuffer* d : {&b.d_problems, &b.d_work, &b.d_counters})
        if (d->ptr) cudaFree(d->ptr);
    if (b.h_problems) cudaFreeHost(b.h_problems);
    if (b.h_work) cudaFreeHost(b.h_work);
    if (b.capture) cudaStreamDestroy(b.capture);
    for (cudaStream_t x : b.branch) cudaStreamDestroy(x);
    for (cudaEvent_t x : b.join_ev) cudaEventDestroy(x);
    if (b.fork_ev) cudaEventDestroy(b.fork_ev);
    if (b.staged_ev) cudaEventDestroy(b.staged_ev);
    delete c->batch;
    c->batch = nullptr;
}

static int check_item(pmsp_ctx* c, const pmsp_batch_item& it) {
    int rc = check_params(c, &it.params, it.n_src);
    if (rc) return rc;
    if ((rc = check_panorama(c, &it.ref, "batch reference"))) return rc;
    if (it.ref.w & 1) return ctx_fail(c, PMSP_EINVAL, "batch reference width %d must be even", it.ref.w);
    if (!it.srcs || !it.src_poses) return ctx_fail(c, PMSP_EINVAL, "batch item without sources");
    for (int s = 0; s < it.n_src; ++s)
        if ((rc = check_panorama(c, &it.srcs[s], "batch source"))) return rc;
    return check_maps(c, &it.out, it.ref.w, it.ref.h, true, true, "batch output");
}

static void append_bytes(std::vector<uint8_t>& v, const void* p, size_t n) {
    const uint8_t* b = static_cast<const uint8_t*>(p);
    v.insert(v.end(), b, b + n);
}

static std::vector<uint8_t> batch_signature(const pmsp_batch_item* items, int n, const pmsp_tuning& t) {
    std::vector<uint8_t> sig;
    append_bytes(sig, &t, sizeof t);
    for (int i = 0; i < n; ++i) {
        append_bytes(sig, &items[i], sizeof(pmsp_batch_item));
        append_bytes(sig, items[i].srcs, sizeof(pmsp_image) * items[i].n_src);
        append_bytes(sig, items[i].src_poses, sizeof(pmsp_pose) * items[i].n_src);
    }
    return sig;
}

// Uploads (textures, host references) and the plan; enqueued on `st`.
static int build_plan(pmsp_ctx* c, BatchEngine& b, const pmsp_batch_item* items, int n, const pmsp_tuning& t,
                      cudaStream_t st, BatchPlan& plan) {
    const cudaStream_t saved = c->stream;
    c->stream = st;  // texture and staging copies go on the build stream
    int rc = PMSP_OK;
    plan.problems.resize(n);
    if ((int)b.ref_stage.size() < n) b.ref_stage.resize(n);
    if ((int)b.out_stage.size() < n) b.out_stage.resize(n);
    int max_phases = 0;
    for (int i = 0; i < n && !rc; ++i) {
        const pmsp_batch_item& it = items[i];
        pmsp_params p = it.params;
        if (t.patch_stride > 0) p.patch_stride = t.patch_stride;
        cudaTextureObject_t tex[PMSP_MAX_SOURCES];
        for (int s = 0; s < it.n_src && !rc; ++s) {
            const pmsp_image& im = it.srcs[s];
            TexImage& ti = b.tex[TexKey(im.data, im.w, im.h, im.format, im.memory, im.pitch_bytes)];
            rc = upload_texture(c, ti, &im, c->stream);
            tex[s] = ti.tex;
        }
        if (rc) break;
        const void* ref_dev = it.ref.data;
        int64_t pitch = it.ref.pitch_bytes;
        if (it.ref.memory != PMSP_DEVICE) {
            const size_t row = (size_t)it.ref.w * format_bytes(it.ref.format);
            if ((rc = ensure_buffer(c, b.ref_stage[i], row * it.ref.h))) break;
            cudaError_t e = cudaMemcpy2DAsync(b.ref_stage[i].ptr, row, it.ref.data, it.ref.pitch_bytes, row,
                                              it.ref.h, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) {
                rc = cuda_fail(c, e, "batch reference upload");
                break;
            }
            ref_dev = b.ref_stage[i].ptr;
            pitch = (int64_t)row;
        }
        PixelParams& P = plan.problems[i];
        fill_problem(P, &it.ref, ref_dev, pitch, &it.ref_pose, it.srcs, tex, it.src_poses, it.n_src, &p);
        P.err = c->d_err;
        P.tile = t.strategy == 1 ? t.tile : 0;
        P.tpp = t.strategy == 1 && t.tpp > 1 ? (t.lanes ? -t.tpp : t.tpp) : 1;
        const size_t N = (size_t)it.ref.w * it.ref.h;
        if (it.out.memory == PMSP_DEVICE) {
            P.depth = it.out.depth;
            P.nx = it.out.normal;
            P.ny = it.out.normal + N;
            P.nz = it.out.normal + 2 * N;
            P.cost = it.out.cost;
        } else {
            if ((rc = ensure_buffer(c, b.out_stage[i], 5 * N * sizeof(float)))) break;
            float* base = static_cast<float*>(b.out_stage[i].ptr);
            P.depth = base;
            P.nx = base + N;
            P.ny = base + 2 * N;
            P.nz = base + 3 * N;
            P.cost = base + 4 * N;
            plan.host_out.emplace_back(i, &b.out_stage[i]);
        }
        plan.max_s = std::max(plan.max_s, it.n_src);
        plan.n_phases.push_back(2 + 2 * it.params.iterations);
        plan.pixels.push_back((int64_t)N);
        max_phases = std::max(max_phases, 2 + 2 * it.params.iterations);
    }
    c->stream = saved;
    if (rc) return rc;

    // work lists: per phase, the tiles of every keyframe that has that phase
    std::vector<int> ids(n);
    for (int i = 0; i < n; ++i) ids[i] = i;
    std::stable_sort(ids.begin(), ids.end(), [&](int a, int bb) {
        return (int64_t)items[a].ref.w * items[a].ref.h > (int64_t)items[bb].ref.w * items[bb].ref.h;
    });
    plan.work.clear();
    plan.phase_off.assign(1, 0);
    for (int ph = 0; ph < max_phases; ++ph) {
        std::vector<std::vector<int4>> per(n);
        for (int i : ids) {
            if (ph >= 2 + 2 * items[i].params.iterations) continue;
            const int tw = (items[i].ref.w + TILE_W - 1) / TILE_W, th = (items[i].ref.h + TILE_H - 1) / TILE_H;
            for (int L = 0; L < tw * th; ++L) {  // strips of tile rows, as the single-keyframe launches walk them
                int tx, ty;
                tile_of_block(tw, th, L, tx, ty);
                per[i].push_back(make_int4(i, tx * TILE_W, ty * TILE_H, ph));
            }
        }
        if (t.order == 1) {
            bool more = true;
            for (size_t k = 0; more; ++k) {
                more = false;
                for (int i : ids)
                    if (k < per[i].size()) {
                        plan.work.push_back(per[i][k]);
                        more = true;
                    }
            }
        } else {
            for (int i : ids) plan.work.insert(plan.work.end(), per[i].begin(), per[i].end());
        }
        plan.phase_off.push_back((int)plan.work.size());
    }
    return PMSP_OK;
}

// Wait until the last eager read of the pinned plan copies has run (the event is
// created on first use; an event never recorded counts as complete).
static int wait_staged(pmsp_ctx* c, BatchEngine& b) {
    const cudaError_t e = b.staged_ev ? cudaEventSynchronize(b.staged_ev)
                                      : cudaEventCreateWithFlags(&b.staged_ev, cudaEventDisableTiming);
    return e == cudaSuccess ? PMSP_OK : cuda_fail(c, e, "batch staging wait");
}

static int ensure_pinned(pmsp_ctx* c, BatchEngine& b, void*& p, size_t& have, size_t need) {
    if (have >= need) return PMSP_OK;
    int rc;
    if (p && (rc = wait_staged(c, b))) return rc;  // a queued copy may still read the old buffer
    if (p) cudaFreeHost(p);
    p = nullptr;
    have = 0;
    if (cudaMallocHost(&p, need) != cudaSuccess) return ctx_fail(c, PMSP_ENOMEM, "pinned host buffer of %zu bytes", need);
    have = need;
    return PMSP_OK;
}

// Copies of the plan, counters and all phase launches, enqueued on `st`.
// Strategy 1: each keyframe's own launch chain (the single-keyframe kernels),
// chains spread over parallel streams that fork from and join back into `st`.
static int enqueue_branches(pmsp_ctx* c, BatchEngine& b, const BatchPlan& plan, cudaStream_t st) {
    const int n = (int)plan.problems.size();
    const int nb = std::min(n, 8);
    cudaError_t e = cudaSuccess;
    if (!b.fork_ev) e = cudaEventCreateWithFlags(&b.fork_ev, cudaEventDisableTiming);
    while (e == cudaSuccess && (int)b.branch.size() < nb) {
        cudaStream_t x;
        cudaEvent_t ev;
        e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) {
            b.branch.push_back(x);
            b.join_ev.push_back(ev);
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(b.fork_ev, st);
    for (int k = 0; k < nb && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b.branch[k], b.fork_ev, 0);
    if (e != cudaSuccess) return cuda_fail(c, e, "batch branches");
    // largest keyframes first, each onto the least loaded chain
    std::vector<int> ids(n);
    for (int i = 0; i < n; ++i) ids[i] = i;
    std::stable_sort(ids.begin(), ids.end(), [&](int x, int y) { return plan.pixels[x] > plan.pixels[y]; });
    std::vector<int64_t> load(nb, 0);
    for (int i : ids) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[k] += plan.pixels[i] * plan.n_phases[i];
        PixelParams P = plan.problems[i];
        for (int ph = 0; ph < plan.n_phases[i] && e == cudaSuccess; ++ph) {
            P.colour = ph & 1;
            P.iter = ph < 2 ? 0 : (ph - 2) >> 1;
            e = launch_pixel_kernel(P, ph < 2 ? MODE_INIT : MODE_SWEEP, b.branch[k]);
        }
    }
    for (int k = 0; k < nb && e == cudaSuccess; ++k) {
        e = cudaEventRecord(b.join_ev[k], b.branch[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b.join_ev[k], 0);
    }
    return e == cudaSuccess ? PMSP_OK : cuda_fail(c, e, "batch branch launch");
}

static int enqueue_plan(pmsp_ctx* c, BatchEngine& b, const BatchPlan& plan, const pmsp_tuning& t, cudaStream_t st) {
    if (t.strategy == 1) return enqueue_branches(c, b, plan, st);
    const size_t pb = plan.problems.size() * sizeof(PixelParams), wb = plan.work.size() * sizeof(int4);
    const int phases = (int)plan.phase_off.size() - 1;
    int rc;
    if ((rc = ensure_buffer(c, b.d_problems, pb)) || (rc = ensure_buffer(c, b.d_work, wb)) ||
        (rc = ensure_buffer(c, b.d_counters, (size_t)std::max(phases, 1) * sizeof(unsigned))))
        return rc;
    if ((rc = ensure_pinned(c, b, b.h_problems, b.h_problems_bytes, pb)) ||
        (rc = ensure_pinned(c, b, b.h_work, b.h_work_bytes, wb)))
        return rc;
    // The pinned copies are rewritten below, and stream order does not cover host
    // writes: outside a capture, wait until the last eager read of them (an earlier
    // call's upload or graph replay, possibly still queued) has run. A capture only
    // records the read; its replays are followed by that wait in the next eager call.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const bool eager = cudaStreamIsCapturing(st, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone;
    if (eager && (rc = wait_staged(c, b))) return rc;
    memcpy(b.h_problems, plan.problems.data(), pb);
    memcpy(b.h_work, plan.work.data(), wb);
    cudaError_t e = cudaMemcpyAsync(b.d_problems.ptr, b.h_problems, pb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.d_work.ptr, b.h_work, wb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && eager) e = cudaEventRecord(b.staged_ev, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.d_counters.ptr, 0, (size_t)phases * sizeof(unsigned), st);
    if (e != cudaSuccess) return cuda_fail(c, e, "batch plan upload");
    const int bucket = batch_bucket(plan.max_s);
    const int occ = batch_blocks_per_sm(bucket);
    const int bps = t.blocks_per_sm > 0 ? std::min(t.blocks_per_sm, occ) : occ;
    for (int ph = 0; ph < phases; ++ph) {
        BatchArgs a;
        a.problems = static_cast<const PixelParams*>(b.d_problems.ptr);
        a.work = static_cast<const int4*>(b.d_work.ptr) + plan.phase_off[ph];
        a.n_work = plan.phase_off[ph + 1] - plan.phase_off[ph];
        a.phase = ph;
        a.counter = static_cast<unsigned*>(b.d_counters.ptr) + ph;
        const int grid = std::max(1, std::min(a.n_work, b.sms * bps));
        e = batch_launch(bucket, a, grid, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "batch launch");
    }
    return PMSP_OK;
}

static int copy_host_outputs(pmsp_ctx* c, const pmsp_batch_item* items, const BatchPlan& plan) {
    for (auto& ho : plan.host_out) {
        const pmsp_batch_item& it = items[ho.first];
        const size_t N = (size_t)it.ref.w * it.ref.h;
        const float* base = static_cast<const float*>(ho.second->ptr);
        cudaError_t e = cudaMemcpyAsync(it.out.depth, base, N * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(it.out.normal, base + N, 3 * N * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(it.out.cost, base + 4 * N, N * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "batch output download");
    }
    return plan.host_out.empty() ? PMSP_OK : pmsp_sync(c);
}

}  // namespace pmsp

using namespace pmsp;

extern "C" {

int pmsp_densify_batch(pmsp_ctx* c, const pmsp_batch_item* items, int n, uint32_t flags, const pmsp_tuning* tuning) {
    if (!c) return PMSP_EINVAL;
    cudaSetDevice(c->device);
    if (n < 1 || !items) return ctx_fail(c, PMSP_EINVAL, "empty batch");
    int rc;
    bool all_device = true;
    for (int i = 0; i < n; ++i) {
        if ((rc = check_item(c, items[i]))) return rc;
        all_device = all_device && items[i].ref.memory == PMSP_DEVICE && items[i].out.memory == PMSP_DEVICE;
        for (int s = 0; s < items[i].n_src; ++s) all_device = all_device && items[i].srcs[s].memory == PMSP_DEVICE;
    }
    pmsp_tuning t{0, 0, 0, 0, 0, 0, 0};
    if (tuning) t = *tuning;
    if (t.tile < 0 || t.tile > 2) return ctx_fail(c, PMSP_EINVAL, "tuning: tile %d outside [0, 2]", t.tile);
    if (t.lanes != 0 && t.lanes != 1) return ctx_fail(c, PMSP_EINVAL, "tuning: lanes %d not 0 or 1", t.lanes);
    if (t.tpp != 0 && t.tpp != 1 && t.tpp != 2 && t.tpp != 4 && !(t.tpp == 8 && t.lanes == 1))
        return ctx_fail(c, PMSP_EINVAL, "tuning: tpp %d not 1, 2 or 4 (or 8 with lanes)", t.tpp);
    BatchEngine& b = engine(c);
    if (b.tex.size() > 1024) {  // bound the texture cache: start over
        cudaStreamSynchronize(c->stream);
        drop_graph(b);
        for (auto& kv : b.tex) free_texture(kv.second);
        b.tex.clear();
    }
    const bool graph = (flags & PMSP_BATCH_GRAPH) && all_device;
    if (graph) {
        std::vector<uint8_t> sig = batch_signature(items, n, t);
        if (b.exec && sig == b.signature) {
            cudaError_t e = cudaGraphLaunch(b.exec, c->stream);
            // the replay reads the pinned copies: mark it, unless the caller is recording
            // the stream (an event recorded there could not be waited on afterwards)
            cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
            if (e == cudaSuccess && cudaStreamIsCapturing(c->stream, &cap) == cudaSuccess &&
                cap == cudaStreamCaptureStatusNone) {
                if (!b.staged_ev) e = cudaEventCreateWithFlags(&b.staged_ev, cudaEventDisableTiming);
                if (e == cudaSuccess) e = cudaEventRecord(b.staged_ev, c->stream);
            }
            return e == cudaSuccess ? PMSP_OK : cuda_fail(c, e, "graph launch");
        }
        drop_graph(b);
        cudaError_t e = cudaStreamSynchronize(c->stream);  // buffers of a replaced graph are reused below
        if (e != cudaSuccess) return cuda_fail(c, e, "sync before capture");
        if (!b.capture && (e = cudaStreamCreateWithFlags(&b.capture, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(c, e, "capture stream");
        // allocations and texture creation happen outside the capture: build once eagerly
        BatchPlan plan;
        if ((rc = build_plan(c, b, items, n, t, c->stream, plan))) return rc;
        if ((rc = enqueue_plan(c, b, plan, t, c->stream))) return rc;
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "batch run before capture");
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(b.capture, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(c, e, "begin capture");
        BatchPlan plan2;
        int rc2 = build_plan(c, b, items, n, t, b.capture, plan2);
        if (!rc2) rc2 = enqueue_plan(c, b, plan2, t, b.capture);
        e = cudaStreamEndCapture(b.capture, &g);
        if (rc2) {
            if (g) cudaGraphDestroy(g);
            return rc2;
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
        e = cudaGraphInstantiate(&b.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b.exec = nullptr;
            return cuda_fail(c, e, "graph instantiate");
        }
        b.signature = std::move(sig);
        return PMSP_OK;  // the eager run already produced this call's results
    }
    // an eager batch reuses the buffers a captured graph reads: forget the graph
    drop_graph(b);
    BatchPlan plan;
    if ((rc = build_plan(c, b, items, n, t, c->stream, plan))) return rc;
    if ((rc = enqueue_plan(c, b, plan, t, c->stream))) return rc;
    return copy_host_outputs(c, items, plan);
}

int pmsp_autotune(pmsp_ctx* c, const pmsp_batch_item* items, int n, float max_changed, pmsp_tuning* out) {
    if (!c || !out) return PMSP_EINVAL;
    cudaSetDevice(c->device);
    if (n < 1 || !items) return ctx_fail(c, PMSP_EINVAL, "empty batch");
    int rc;
    for (int i = 0; i < n; ++i)
        if ((rc = check_item(c, items[i]))) return rc;
    BatchEngine& b = engine(c);
    int max_s = 0;
    for (int i = 0; i < n; ++i) max_s = std::max(max_s, items[i].n_src);
    const int occ = batch_blocks_per_sm(batch_bucket(max_s));

    auto time_run = [&](const pmsp_tuning& t, double& ms) -> int {
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, c->stream);
        int r = pmsp_densify_batch(c, items, n, 0, &t);
        cudaEventRecord(e1, c->stream);
        if (!r) r = pmsp_sync(c);
        float f = 0.f;
        cudaEventElapsedTime(&f, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        ms = f;
        return r;
    };
    pmsp_tuning best{0, 0, 0, 0, 0, 0, 0};
    double best_ms = 1e30;
    std::vector<int> bps_list;
    for (int k = occ; k >= 1 && (int)bps_list.size() < 4; --k) bps_list.push_back(k);
    for (int tile = 0; tile < 3; ++tile) {
        pmsp_tuning t{0, 0, 0, 1, tile, 1, 0};  // concurrent per-keyframe chains, each tile shape
        double ms;
        if ((rc = time_run(t, ms)) || (rc = time_run(t, ms))) return rc;
        if (ms < best_ms) {
            best_ms = ms;
            best = t;
        }
    }
    // per-keyframe chains with 2 or 4 threads per pixel: the views split over
    // warps, or the patch samples over adjacent lanes
    for (int lanes = 0; lanes < 2; ++lanes)
        for (int tpp : {2, 4, 8}) {
            if (tpp == 8 && !lanes) continue;  // the warp split serves 2 or 4 warps
            pmsp_tuning t{0, 0, 0, 1, 0, tpp, lanes};
            double ms;
            if ((rc = time_run(t, ms)) || (rc = time_run(t, ms))) return rc;
            if (ms < best_ms) {
                best_ms = ms;
                best = t;
            }
        }
    for (int order = 0; order < 2; ++order)
        for (int bps : bps_list) {
            pmsp_tuning t{bps, order, 0, 0, 0, 0, 0};
            double ms;
            if ((rc = time_run(t, ms))) return rc;  // first run of each setting also warms caches
            if ((rc = time_run(t, ms))) return rc;
            if (ms < best_ms) {
                best_ms = ms;
                best = t;
            }
        }
    // coarser patch stride: accepted only if the ranges stay within 1 % of the own-stride result
    bool all_device = true;
    for (int i = 0; i < n; ++i) all_device = all_device && items[i].out.memory == PMSP_DEVICE;
    int own = items[0].params.patch_stride;
    bool same = true;
    for (int i = 0; i < n; ++i) same = same && items[i].params.patch_stride == own;
    if (all_device && same && own == 1 && max_changed > 0.f) {
        std::vector<std::vector<float>> ref_depth(n);
        if ((rc = pmsp_densify_batch(c, items, n, 0, &best))) return rc;
        if ((rc = pmsp_sync(c))) return rc;
        for (int i = 0; i < n; ++i) {
            ref_depth[i].resize((size_t)items[i].ref.w * items[i].ref.h);
            cudaMemcpy(ref_depth[i].data(), items[i].out.depth, ref_depth[i].size() * 4, cudaMemcpyDeviceToHost);
        }
        pmsp_tuning t2 = best;
        t2.patch_stride = 2;
        double ms2;
        if ((rc = time_run(t2, ms2))) return rc;
        if ((rc = time_run(t2, ms2))) return rc;
        size_t changed = 0, total = 0;
        for (int i = 0; i < n; ++i) {
            std::vector<float> d(ref_depth[i].size());
            cudaMemcpy(d.data(), items[i].out.depth, d.size() * 4, cudaMemcpyDeviceToHost);
            for (size_t k = 0; k < d.size(); ++k) {
                const float r = ref_depth[i][k];
                changed += (std::fabs(d[k] - r) > 0.01f * r);
            }
            total += d.size();
        }
        if (ms2 < best_ms && (double)changed <= (double)max_changed * (double)total) best = t2;
    }
    *out = best;
    return PMSP_OK;
}

}  // extern "C"
