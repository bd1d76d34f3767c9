// Serving runtime: device frame ring, admission by slots, memory and resident
// work, and a scheduler thread with two policies. Lanes: every admitted
// request's whole launch chain starts on a stream lane of its own, so requests
// that arrive while others run are admitted as soon as a lane and memory free
// up and their kernels overlap on the device. Steps (iteration-level
// continuous batching): each scheduler step is one persistent launch that runs
// the next phase (initialisation colour or half-sweep) of every active
// request; requests join at the next step and leave after their last phase.
// Paper Sec. III runs densification in its own thread fed by a keyframe queue;
// this is that thread, reshaped for many concurrent keyframes on one GPU.
//
// Host waits are bounded: the scheduler polls CUDA events and fails a request
// with PMSP_ETIMEDOUT when it has not finished within a deadline; pmsp_wait
// blocks on a condition variable up to the caller's timeout.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"
#include "pmsp.h"
#include "runtime.h"
#include "serving_policy.h"

namespace pmsp {

namespace {

using Clock = std::chrono::steady_clock;

struct RingFrame {
    int64_t id = -1;
    bool used = false;
    uint64_t seq = 0;      // push order, for eviction
    int pins = 0;          // queued or active requests using the frame
    int w = 0, h = 0, fmt = 0;
    pmsp_pose pose{};
    TexImage tex;          // as a source
    DevBuffer lin;         // as a reference (row-major, unpadded)
    DevBuffer depth;       // depth of the last finished request with this reference
    bool has_depth = false;
    bool loading = false;  // being rewritten by pmsp_ring_push
};

using TexKey = std::tuple<int, int, int>;  // w, h, format

enum Status { QUEUED, ACTIVE, FINISHING, DONE, FAILED };

struct Request {
    uint64_t ticket = 0;
    int status = QUEUED;
    int fail_code = PMSP_OK;
    int ref = -1;
    std::vector<int> srcs, filters;
    pmsp_params params{};
    float max_px = 1.f;
    int min_views = 2;
    int W = 0, H = 0;
    int n_phases = 0;
    size_t bytes = 0, tiles = 0;
    int lane = -1;
    cudaStream_t stream = nullptr;  // the stream its work runs on (maps are freed in its order)
    int phase = 0;                  // steps: next phase to launch
    int slot = -1;                  // steps: its parameter slot on the device
    Clock::time_point admitted;
    DevBuffer maps;        // depth, nx, ny, nz, cost, filtered depth
    cudaEvent_t done = nullptr;
    PixelParams prob;
};

}  // namespace

struct Serving {
    pmsp_ctx* ctx = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread th;
    bool stop = false;
    std::vector<cudaStream_t> lanes;  // one running request per lane
    std::vector<Request*> lane_req;
    size_t running_tiles = 0;
    cudaStream_t upload = nullptr;   // ring uploads
    cudaEvent_t upload_ev = nullptr;
    std::multimap<TexKey, TexImage> tex_pool;  // texture arrays kept for frames of their size
    std::vector<RingFrame> ring;
    uint64_t push_seq = 0;
    std::deque<Request*> queue;
    std::vector<Request*> running;
    std::vector<Request*> zombies;  // overran the deadline and were given up on
    std::map<uint64_t, Request*> tickets;
    uint64_t next_ticket = 1;
    uint64_t bytes_in_use = 0;
    pmsp_serving_stats stats{};
    int sms = 0;
    std::string err;
    // step scheduler (PMSP_SCHED_STEPS): one stream, per-request parameter slots
    // on the device, a work list per step staged through two pinned buffers
    cudaStream_t step_stream = nullptr;
    PixelParams* d_slots = nullptr;
    PixelParams* h_slots = nullptr;     // pinned host copies, one per slot
    std::vector<cudaEvent_t> slot_ev;   // last upload from each host copy
    std::vector<int> free_slots;
    DevBuffer d_work;
    unsigned* d_counter = nullptr;
    int4* h_work[2] = {nullptr, nullptr};
    size_t h_work_cap[2] = {0, 0};
    cudaEvent_t work_ev[2] = {nullptr, nullptr};
    int work_next = 0;
    std::deque<cudaEvent_t> inflight;   // completion events of launched steps
    std::vector<cudaEvent_t> ev_pool;
};

namespace {

constexpr double STEP_DEADLINE_S = 60.0;     // bound on a ring upload
constexpr double REQUEST_DEADLINE_S = 600.0; // bound on one request's GPU work

int find_frame(Serving& s, int64_t id) {
    for (int i = 0; i < (int)s.ring.size(); ++i)
        if (s.ring[i].used && s.ring[i].id == id) return i;
    return -1;
}

// Poll an event until it completes or the deadline passes (no unbounded wait).
bool wait_event(cudaEvent_t ev, double seconds) {
    const auto until = Clock::now() + std::chrono::duration<double>(seconds);
    for (;;) {
        const cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return true;
        if (e != cudaErrorNotReady) return false;
        if (Clock::now() > until) return false;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

// Grow-only buffer, allocated and freed in stream order on `st` (no
// device-wide synchronisation while other work runs).
int dev_alloc(DevBuffer& b, size_t bytes, cudaStream_t st) {
    if (b.bytes >= bytes) return PMSP_OK;
    if (b.ptr) cudaFreeAsync(b.ptr, st);
    b.ptr = nullptr;
    b.bytes = 0;
    if (cudaMallocAsync(&b.ptr, bytes, st) != cudaSuccess) {
        b.ptr = nullptr;
        return PMSP_ENOMEM;
    }
    b.bytes = bytes;
    return PMSP_OK;
}

// Give back a request's frames and maps (stream-ordered free: no device-wide sync).
void release_request(Serving& s, Request* r) {
    for (int f : r->srcs) s.ring[f].pins--;
    for (int f : r->filters) s.ring[f].pins--;
    s.ring[r->ref].pins--;
    // freed in the order of the stream the request's work ran on, so a request
    // whose launch chain failed part-way cannot have its maps reused under it
    if (r->maps.ptr) cudaFreeAsync(r->maps.ptr, r->stream ? r->stream : s.upload);
    if (r->done) cudaEventDestroy(r->done);
    if (r->maps.ptr) s.bytes_in_use -= r->bytes;
    delete r;
}

// Build one request's kernel parameters; called at admission (maps allocated).
void fill_request(Serving& s, Request* r) {
    RingFrame& ref = s.ring[r->ref];
    pmsp_image ri{ref.w, ref.h, (int64_t)ref.w * (int64_t)format_bytes(ref.fmt), ref.fmt, PMSP_DEVICE, ref.lin.ptr};
    pmsp_image si[PMSP_MAX_SOURCES];
    pmsp_pose sp[PMSP_MAX_SOURCES];
    cudaTextureObject_t tex[PMSP_MAX_SOURCES];
    for (size_t k = 0; k < r->srcs.size(); ++k) {
        const RingFrame& f = s.ring[r->srcs[k]];
        si[k] = pmsp_image{f.w, f.h, (int64_t)f.w * (int64_t)format_bytes(f.fmt), f.fmt, PMSP_DEVICE, f.lin.ptr};
        sp[k] = f.pose;
        tex[k] = f.tex.tex;
    }
    fill_problem(r->prob, &ri, ref.lin.ptr, ri.pitch_bytes, &ref.pose, si, tex, sp, (int)r->srcs.size(), &r->params);
    const size_t N = (size_t)r->W * r->H;
    float* base = static_cast<float*>(r->maps.ptr);
    r->prob.depth = base;
    r->prob.nx = base + N;
    r->prob.ny = base + 2 * N;
    r->prob.nz = base + 3 * N;
    r->prob.cost = base + 4 * N;
    r->prob.err = s.ctx->d_err;
}

// What follows a request's last phase: the consistency filter against the
// named neighbours whose depth maps exist, the copy of its depth into the
// ring, the completion event.
int enqueue_tail(Serving& s, Request* r, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    const size_t N = (size_t)r->W * r->H;
    float* base = static_cast<float*>(r->maps.ptr);
    float* filtered = base + 5 * N;
    FilterParams F;
    memset(&F, 0, sizeof F);
    int n = 0;
    for (int f : r->filters) {
        RingFrame& fr = s.ring[f];
        if (!fr.has_depth) continue;
        FilterView& V = F.nb[n++];
        V.depth = static_cast<const float*>(fr.depth.ptr);
        V.W = fr.w;
        V.H = fr.h;
        double R[9], t[3];
        const pmsp_pose& rp = s.ring[r->ref].pose;
        compose_rel(rp, fr.pose, R, t);
        for (int k = 0; k < 9; ++k) V.Rf[k] = (float)R[k];
        for (int k = 0; k < 3; ++k) V.tf[k] = (float)t[k];
        compose_rel(fr.pose, rp, R, t);
        for (int k = 0; k < 9; ++k) V.Rb[k] = (float)R[k];
        for (int k = 0; k < 3; ++k) V.tb[k] = (float)t[k];
    }
    if (e == cudaSuccess && n > 0) {
        F.depth_in = base;
        F.depth_out = filtered;
        F.agree = nullptr;
        F.W = r->W;
        F.H = r->H;
        F.n = n;
        F.min_views = r->min_views;
        F.max_px = r->max_px;
        e = launch_filter_kernel(F, st);
    } else if (e == cudaSuccess) {
        e = cudaMemcpyAsync(filtered, base, N * 4, cudaMemcpyDeviceToDevice, st);
    }
    // the ring's depth buffer was sized when the frame was pushed; it counts as the
    // frame's depth map once the scheduler has seen this chain finish
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.ring[r->ref].depth.ptr, base, N * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(r->done, st);
    return e == cudaSuccess ? PMSP_OK : PMSP_ECUDA;
}

// A request's whole launch chain on its lane: initialisation, the red/black
// half-sweeps, then the tail.
int enqueue_request(Serving& s, Request* r, cudaStream_t st) {
    PixelParams P = r->prob;
    cudaError_t e = cudaSuccess;
    for (int ph = 0; ph < r->n_phases && e == cudaSuccess; ++ph) {
        P.colour = ph & 1;
        P.iter = ph < 2 ? 0 : (ph - 2) >> 1;
        e = launch_pixel_kernel(P, ph < 2 ? MODE_INIT : MODE_SWEEP, st);
    }
    if (e != cudaSuccess) return PMSP_ECUDA;
    return enqueue_tail(s, r, st);
}

DepthUse depth_use(const Request* r) { return DepthUse{r->ref, r->filters.data(), (int)r->filters.size()}; }

// Whether starting r now would let two running chains touch one frame's depth
// map at once (serving_policy.h).
bool conflicts_with_running(const Serving& s, const Request* r) {
    std::vector<DepthUse> running;
    running.reserve(s.running.size());
    for (const Request* q : s.running) running.push_back(depth_use(q));
    return depth_conflict(depth_use(r), running.data(), (int)running.size());
}

// Retire requests whose completion event has fired (or that overran the
// deadline). `finished` says whether a request's last work is enqueued.
template <class Finished>
void retire(Serving& s, Finished finished) {
    for (size_t k = 0; k < s.running.size();) {
        Request* r = s.running[k];
        if (!finished(r)) {
            ++k;
            continue;
        }
        // a request whose work could not be enqueued has fail_code set and no
        // completion event recorded (an unrecorded event would read as complete)
        const bool broken = r->fail_code != PMSP_OK;
        const cudaError_t q = broken ? cudaErrorLaunchFailure : cudaEventQuery(r->done);
        const bool late = q == cudaErrorNotReady &&
                          Clock::now() - r->admitted > std::chrono::duration<double>(REQUEST_DEADLINE_S);
        if (q == cudaErrorNotReady && !late) {
            ++k;
            continue;
        }
        r->status = q == cudaSuccess ? DONE : FAILED;
        if (q == cudaSuccess) s.ring[r->ref].has_depth = true;  // later filters may read it
        if (q != cudaSuccess && !broken) {
            r->fail_code = late ? PMSP_ETIMEDOUT : PMSP_ECUDA;
            s.err = late ? "request did not finish within the deadline" : cudaGetErrorString(q);
        }
        s.stats.completed += q == cudaSuccess;
        s.running_tiles -= r->tiles;
        if (!late) {  // a late request keeps its lane or slot blocked
            if (r->lane >= 0) s.lane_req[r->lane] = nullptr;
            if (r->slot >= 0) s.free_slots.push_back(r->slot);
        }
        s.running.erase(s.running.begin() + k);
        s.cv_done.notify_all();
    }
}

void scheduler(Serving* sp) {
    Serving& s = *sp;
    cudaSetDevice(s.ctx->device);
    std::unique_lock<std::mutex> lk(s.mu);
    for (;;) {
        retire(s, [](const Request*) { return true; });
        // admission: FIFO while a lane is free, the maps fit, the resident work allows
        // and no running chain writes or reads a depth map that this one reads or writes
        while (!s.queue.empty()) {
            Request* r = s.queue.front();
            const AdmitState now{(int)s.running.size(), s.ctx->max_active, s.bytes_in_use, s.ctx->mem_cap,
                                 s.running_tiles, serving_tile_budget(s.sms)};
            if (admit_block(now, r->bytes, r->tiles, conflicts_with_running(s, r)) != ADMIT_OK) break;
            int lane = -1;
            for (int i = 0; i < (int)s.lanes.size() && lane < 0; ++i)
                if (!s.lane_req[i]) lane = i;
            if (lane < 0 && (int)s.lanes.size() < s.ctx->max_active) {
                cudaStream_t st;
                if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) break;
                s.lanes.push_back(st);
                s.lane_req.push_back(nullptr);
                lane = (int)s.lanes.size() - 1;
            }
            if (lane < 0) break;
            const cudaStream_t st = s.lanes[lane];
            if (cudaMallocAsync(&r->maps.ptr, r->bytes, st) != cudaSuccess) {
                r->maps.ptr = nullptr;
                break;  // retried on the next pass
            }
            r->maps.bytes = r->bytes;
            if (!r->done && cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming) != cudaSuccess) break;
            s.queue.pop_front();
            s.bytes_in_use += r->bytes;
            fill_request(s, r);
            r->lane = lane;
            r->stream = st;
            r->admitted = Clock::now();
            if (enqueue_request(s, r, st) != PMSP_OK) {
                r->status = FAILED;
                r->fail_code = PMSP_ECUDA;
                s.err = "launch failed";
                s.cv_done.notify_all();
                continue;
            }
            r->status = ACTIVE;
            s.lane_req[lane] = r;
            s.running.push_back(r);
            s.running_tiles += r->tiles;
            s.stats.steps++;
        }
        s.stats.queued = (uint32_t)s.queue.size();
        s.stats.active = (uint32_t)s.running.size();
        s.stats.bytes_in_use = s.bytes_in_use;
        if (s.stop) break;
        if (s.running.empty())
            s.cv_work.wait_for(lk, std::chrono::milliseconds(20));
        else
            s.cv_work.wait_for(lk, std::chrono::microseconds(200));
    }
}

// Wait (bounded) until an event has completed, releasing the lock meanwhile.
bool wait_event_unlocked(Serving& s, std::unique_lock<std::mutex>& lk, cudaEvent_t ev, double seconds) {
    const auto until = Clock::now() + std::chrono::duration<double>(seconds);
    for (;;) {
        const cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return true;
        if (e != cudaErrorNotReady || Clock::now() > until) return false;
        s.cv_work.wait_for(lk, std::chrono::microseconds(50));
    }
}

// One step: the next phase of every active request in one persistent launch
// over all their tiles (largest request first, strips of tile rows), then the tail
// of each request whose last phase this was. Returns PMSP_OK or PMSP_ECUDA.
int launch_step(Serving& s, std::unique_lock<std::mutex>& lk) {
    const cudaStream_t st = s.step_stream;
    std::vector<Request*> act;
    for (Request* r : s.running)
        if (r->phase < r->n_phases) act.push_back(r);
    if (act.empty()) return PMSP_OK;
    std::stable_sort(act.begin(), act.end(), [](const Request* a, const Request* b) { return a->W * a->H > b->W * b->H; });
    size_t n_work = 0;
    int max_s = 0;
    for (Request* r : act) {
        n_work += r->tiles;
        max_s = std::max(max_s, (int)r->srcs.size());
    }
    // the pinned buffer is rewritten only after its previous copy has been read
    const int b = s.work_next;
    s.work_next ^= 1;
    if (s.work_ev[b] && !wait_event_unlocked(s, lk, s.work_ev[b], STEP_DEADLINE_S)) return PMSP_ECUDA;
    if (s.h_work_cap[b] < n_work) {
        if (s.h_work[b]) cudaFreeHost(s.h_work[b]);
        s.h_work[b] = nullptr;
        s.h_work_cap[b] = 0;
        if (cudaMallocHost(&s.h_work[b], n_work * sizeof(int4)) != cudaSuccess) return PMSP_ECUDA;
        s.h_work_cap[b] = n_work;
    }
    int4* w = s.h_work[b];
    for (Request* r : act) {
        const int tw = (r->W + TILE_W - 1) / TILE_W, th = (r->H + TILE_H - 1) / TILE_H;
        for (int L = 0; L < tw * th; ++L) {  // strips of tile rows (texture-cache locality)
            int tx, ty;
            tile_of_block(tw, th, L, tx, ty);
            *w++ = make_int4(r->slot, tx * TILE_W, ty * TILE_H, r->phase);
        }
    }
    if (dev_alloc(s.d_work, n_work * sizeof(int4), st) != PMSP_OK) return PMSP_ECUDA;
    cudaError_t e = cudaMemcpyAsync(s.d_work.ptr, s.h_work[b], n_work * sizeof(int4), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(s.work_ev[b], st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.d_counter, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return PMSP_ECUDA;
    BatchArgs a;
    a.problems = s.d_slots;
    a.work = static_cast<const int4*>(s.d_work.ptr);
    a.n_work = (int)n_work;
    a.phase = -1;  // each item's own phase
    a.counter = s.d_counter;
    const int bucket = batch_bucket(max_s);
    const int grid = (int)std::min<size_t>(n_work, (size_t)s.sms * batch_blocks_per_sm(bucket));
    if (batch_launch(bucket, a, grid, st) != cudaSuccess) return PMSP_ECUDA;
    for (Request* r : act)
        if (++r->phase == r->n_phases && enqueue_tail(s, r, st) != PMSP_OK) {
            r->fail_code = PMSP_ECUDA;
            return PMSP_ECUDA;
        }
    cudaEvent_t ev;
    if (!s.ev_pool.empty()) {
        ev = s.ev_pool.back();
        s.ev_pool.pop_back();
    } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        return PMSP_ECUDA;
    }
    if (cudaEventRecord(ev, st) != cudaSuccess) return PMSP_ECUDA;
    s.inflight.push_back(ev);
    s.stats.steps++;
    return PMSP_OK;
}

// Iteration-level scheduler: admission at step boundaries into parameter
// slots, at most two steps in flight (phase progress is known on the host, so
// the next step is enqueued while the current one runs).
void scheduler_steps(Serving* sp) {
    Serving& s = *sp;
    cudaSetDevice(s.ctx->device);
    std::unique_lock<std::mutex> lk(s.mu);
    const cudaStream_t st = s.step_stream;
    for (;;) {
        while (!s.inflight.empty() && cudaEventQuery(s.inflight.front()) != cudaErrorNotReady) {
            s.ev_pool.push_back(s.inflight.front());
            s.inflight.pop_front();
        }
        retire(s, [](const Request* r) { return r->phase >= r->n_phases; });
        // admission: FIFO under the same rules as the lanes (slots, memory cap,
        // resident tiles, depth-map order), into a free parameter slot
        while (!s.queue.empty() && !s.free_slots.empty()) {
            Request* r = s.queue.front();
            const AdmitState now{(int)s.running.size(), s.ctx->max_active, s.bytes_in_use, s.ctx->mem_cap,
                                 s.running_tiles, serving_tile_budget(s.sms)};
            if (admit_block(now, r->bytes, r->tiles, conflicts_with_running(s, r)) != ADMIT_OK) break;
            if (cudaMallocAsync(&r->maps.ptr, r->bytes, st) != cudaSuccess) {
                r->maps.ptr = nullptr;
                break;  // retried on the next pass
            }
            r->maps.bytes = r->bytes;
            if (!r->done && cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming) != cudaSuccess) break;
            const int slot = s.free_slots.back();
            // the slot's host copy is rewritten only after its last upload has been read
            if (!wait_event_unlocked(s, lk, s.slot_ev[slot], STEP_DEADLINE_S)) break;
            s.free_slots.pop_back();
            s.queue.pop_front();
            s.bytes_in_use += r->bytes;
            fill_request(s, r);
            r->slot = slot;
            r->stream = st;
            r->phase = 0;
            r->admitted = Clock::now();
            s.h_slots[slot] = r->prob;
            cudaError_t e = cudaMemcpyAsync(s.d_slots + slot, s.h_slots + slot, sizeof(PixelParams),
                                            cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaEventRecord(s.slot_ev[slot], st);
            r->status = ACTIVE;
            s.running.push_back(r);
            s.running_tiles += r->tiles;
            if (e != cudaSuccess) {
                r->phase = r->n_phases;  // nothing more is launched for it
                r->fail_code = PMSP_ECUDA;
                s.err = "parameter upload failed";
            }
        }
        if (s.inflight.size() < 2 && launch_step(s, lk) != PMSP_OK) {
            // a failed launch fails every request still in its phases
            s.err = "step launch failed";
            for (Request* r : s.running)
                if (r->phase < r->n_phases) {
                    r->phase = r->n_phases;
                    r->fail_code = PMSP_ECUDA;
                }
        }
        s.stats.queued = (uint32_t)s.queue.size();
        s.stats.active = (uint32_t)s.running.size();
        s.stats.bytes_in_use = s.bytes_in_use;
        if (s.stop) break;
        if (s.running.empty())
            s.cv_work.wait_for(lk, std::chrono::milliseconds(20));
        else
            s.cv_work.wait_for(lk, std::chrono::microseconds(100));
    }
}

Serving& serving(pmsp_ctx* c) {
    if (!c->serving) {
        Serving* s = new Serving();
        s->ctx = c;
        s->ring.resize(c->ring_capacity);
        cudaStreamCreateWithFlags(&s->upload, cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&s->upload_ev, cudaEventDisableTiming);
        cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, c->device);
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;  // keep freed request maps in the pool for the next admission
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        if (c->scheduler == PMSP_SCHED_STEPS) {
            cudaStreamCreateWithFlags(&s->step_stream, cudaStreamNonBlocking);
            cudaMalloc(&s->d_slots, (size_t)c->max_active * sizeof(PixelParams));
            cudaMallocHost(&s->h_slots, (size_t)c->max_active * sizeof(PixelParams));
            cudaMalloc(&s->d_counter, sizeof(unsigned));
            s->slot_ev.resize(c->max_active);
            for (int k = 0; k < c->max_active; ++k) {
                cudaEventCreateWithFlags(&s->slot_ev[k], cudaEventDisableTiming);
                s->free_slots.push_back(c->max_active - 1 - k);
            }
            for (auto& ev : s->work_ev) cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            s->th = std::thread(scheduler_steps, s);
        } else {
            s->th = std::thread(scheduler, s);
        }
        c->serving = s;
    }
    return *c->serving;
}

int take(Serving& s, uint64_t ticket, pmsp_maps* out, pmsp_ctx* c) {
    auto it = s.tickets.find(ticket);
    if (it == s.tickets.end()) return ctx_fail(c, PMSP_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Request* r = it->second;
    if (r->status == FAILED) {
        const int code = r->fail_code ? r->fail_code : PMSP_ECUDA;
        s.tickets.erase(it);
        if (code == PMSP_ETIMEDOUT)
            s.zombies.push_back(r);  // its kernels may still run: keep its maps and frames until shutdown
        else
            release_request(s, r);
        return ctx_fail(c, code, "request failed: %s", s.err.c_str());
    }
    if (r->status != DONE) return PMSP_EBUSY;
    int rc = PMSP_OK;
    if (out) {
        const size_t N = (size_t)r->W * r->H;
        if (out->w != r->W || out->h != r->H || !out->depth)
            return ctx_fail(c, PMSP_EINVAL, "output maps must be %dx%d", r->W, r->H);
        const float* base = static_cast<const float*>(r->maps.ptr);
        const cudaMemcpyKind k = out->memory == PMSP_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
        cudaError_t e = cudaMemcpy(out->depth, base + 5 * N, N * 4, k);
        if (e == cudaSuccess && out->normal) e = cudaMemcpy(out->normal, base + N, 3 * N * 4, k);
        if (e == cudaSuccess && out->cost) e = cudaMemcpy(out->cost, base + 4 * N, N * 4, k);
        if (e != cudaSuccess) rc = cuda_fail(c, e, "result copy");
    }
    s.tickets.erase(it);
    release_request(s, r);
    return rc;
}

}  // namespace

void runtime_shutdown(pmsp_ctx* c) {
    if (c->serving) {
        Serving& s = *c->serving;
        {
            std::lock_guard<std::mutex> lk(s.mu);
            s.stop = true;
        }
        s.cv_work.notify_all();
        if (s.th.joinable()) s.th.join();
        for (cudaStream_t st : s.lanes) cudaStreamSynchronize(st);
        if (s.step_stream) cudaStreamSynchronize(s.step_stream);
        cudaStreamSynchronize(s.upload);
        for (auto& kv : s.tickets) s.zombies.push_back(kv.second);
        for (Request* r : s.zombies) {
            if (r->maps.ptr) cudaFree(r->maps.ptr);
            if (r->done) cudaEventDestroy(r->done);
            delete r;
        }
        for (auto& kv : s.tex_pool) free_texture(kv.second);
        for (auto& f : s.ring) {
            free_texture(f.tex);
            if (f.lin.ptr) cudaFree(f.lin.ptr);
            if (f.depth.ptr) cudaFree(f.depth.ptr);
        }
        for (cudaStream_t st : s.lanes) cudaStreamDestroy(st);
        if (s.step_stream) {
            for (cudaEvent_t ev : s.slot_ev) cudaEventDestroy(ev);
            for (cudaEvent_t ev : s.work_ev) cudaEventDestroy(ev);
            for (cudaEvent_t ev : s.inflight) cudaEventDestroy(ev);
            for (cudaEvent_t ev : s.ev_pool) cudaEventDestroy(ev);
            for (int4* h : s.h_work)
                if (h) cudaFreeHost(h);
            if (s.d_work.ptr) cudaFree(s.d_work.ptr);
            cudaFree(s.d_slots);
            cudaFreeHost(s.h_slots);
            cudaFree(s.d_counter);
            cudaStreamDestroy(s.step_stream);
        }
        cudaStreamDestroy(s.upload);
        cudaEventDestroy(s.upload_ev);
        delete c->serving;
        c->serving = nullptr;
    }
    batch_shutdown(c);
}

}  // namespace pmsp

using namespace pmsp;

extern "C" {

int pmsp_ring_push(pmsp_ctx* c, int64_t id, const pmsp_image* img, const pmsp_pose* pose) {
    if (!c) return PMSP_EINVAL;
    cudaSetDevice(c->device);
    int rc = check_panorama(c, img, "ring frame");
    if (rc) return rc;
    if (!pose) return ctx_fail(c, PMSP_EINVAL, "NULL pose");
    Serving& s = serving(c);
    std::unique_lock<std::mutex> lk(s.mu);
    int slot = find_frame(s, id);
    if (slot >= 0 && s.ring[slot].pins > 0) return ctx_fail(c, PMSP_EBUSY, "frame %lld is in use", (long long)id);
    if (slot < 0) {  // a free slot, else evict the oldest frame no request holds
        std::vector<SlotView> view(s.ring.size());
        for (size_t i = 0; i < s.ring.size(); ++i)
            view[i] = SlotView{s.ring[i].used, s.ring[i].loading, s.ring[i].pins, s.ring[i].seq};
        slot = ring_pick_slot(view.data(), (int)view.size());
        if (slot < 0) return ctx_fail(c, PMSP_EBUSY, "every ring frame is used by a request");
    }
    // Claim the slot: nothing uses an unpinned frame, so it is rewritten while
    // the scheduler keeps running; the copies go on the upload stream so they
    // do not queue behind the scheduler's launches.
    RingFrame& f = s.ring[slot];
    f.used = false;
    f.loading = true;
    f.pins = 1;
    const TexKey want(img->w, img->h, img->format);
    if (f.tex.arr && TexKey(f.tex.w, f.tex.h, f.tex.fmt) != want) {  // keep arrays of other sizes for reuse
        s.tex_pool.emplace(TexKey(f.tex.w, f.tex.h, f.tex.fmt), f.tex);
        f.tex = TexImage{};
    }
    if (!f.tex.arr) {
        auto it = s.tex_pool.find(want);
        if (it != s.tex_pool.end()) {
            f.tex = it->second;
            s.tex_pool.erase(it);
        }
    }
    lk.unlock();
    const size_t row = (size_t)img->w * format_bytes(img->format);
    cudaError_t e = cudaSuccess;
    if (f.lin.bytes < row * img->h) {  // grow only, stream-ordered (no device-wide synchronisation)
        if (f.lin.ptr) cudaFreeAsync(f.lin.ptr, s.upload);
        f.lin.ptr = nullptr;
        f.lin.bytes = 0;
        e = cudaMallocAsync(&f.lin.ptr, row * img->h, s.upload);
        if (e == cudaSuccess) f.lin.bytes = row * img->h;
    }
    // the depth map a finished request leaves for later filters: sized here, while
    // nothing reads the slot, so finishing requests only copy into it
    if (e == cudaSuccess && dev_alloc(f.depth, (size_t)img->w * img->h * sizeof(float), s.upload) != PMSP_OK)
        e = cudaErrorMemoryAllocation;
    const cudaMemcpyKind k = img->memory == PMSP_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (e == cudaSuccess) e = cudaMemcpy2DAsync(f.lin.ptr, row, img->data, img->pitch_bytes, row, img->h, k, s.upload);
    if (e == cudaSuccess) rc = upload_texture(c, f.tex, img, s.upload);
    if (e == cudaSuccess && !rc) e = cudaEventRecord(s.upload_ev, s.upload);
    const bool ok = e == cudaSuccess && !rc && wait_event(s.upload_ev, STEP_DEADLINE_S);
    lk.lock();
    f.loading = false;
    f.pins = 0;
    if (!ok) {
        if (rc) return rc;
        return e != cudaSuccess ? cuda_fail(c, e, "ring upload") : ctx_fail(c, PMSP_ETIMEDOUT, "ring upload timed out");
    }
    f.id = id;
    f.used = true;
    f.seq = ++s.push_seq;
    f.w = img->w;
    f.h = img->h;
    f.fmt = img->format;
    f.pose = *pose;
    f.has_depth = false;
    return PMSP_OK;
}

int pmsp_submit(pmsp_ctx* c, const pmsp_request* q, uint64_t* ticket) {
    if (!c) return PMSP_EINVAL;
    cudaSetDevice(c->device);
    if (!q || !ticket) return ctx_fail(c, PMSP_EINVAL, "NULL request or ticket");
    int rc = check_params(c, &q->params, q->n_src);
    if (rc) return rc;
    if (q->n_filter < 0 || q->n_filter > PMSP_MAX_SOURCES || (q->n_filter > 0 && !q->filter_frames) ||
        !q->src_frames)
        return ctx_fail(c, PMSP_EINVAL, "bad frame lists");
    if (q->n_filter > 0 && (!(q->max_reproj_px > 0.f) || q->min_views < 0))
        return ctx_fail(c, PMSP_EINVAL, "bad filter parameters");
    Serving& s = serving(c);
    std::lock_guard<std::mutex> lk(s.mu);
    Request tmp;
    tmp.ref = find_frame(s, q->ref_frame);
    if (tmp.ref < 0) return ctx_fail(c, PMSP_ENOTFOUND, "reference frame %lld not in the ring", (long long)q->ref_frame);
    for (int k = 0; k < q->n_src; ++k) {
        const int f = find_frame(s, q->src_frames[k]);
        if (f < 0) return ctx_fail(c, PMSP_ENOTFOUND, "source frame %lld not in the ring", (long long)q->src_frames[k]);
        tmp.srcs.push_back(f);
    }
    for (int k = 0; k < q->n_filter; ++k) {
        const int f = find_frame(s, q->filter_frames[k]);
        if (f < 0) return ctx_fail(c, PMSP_ENOTFOUND, "filter frame %lld not in the ring", (long long)q->filter_frames[k]);
        tmp.filters.push_back(f);
    }
    const RingFrame& ref = s.ring[tmp.ref];
    if (ref.w & 1) return ctx_fail(c, PMSP_EINVAL, "reference width %d must be even", ref.w);
    Request* r = new Request(std::move(tmp));
    r->params = q->params;
    r->max_px = q->max_reproj_px;
    r->min_views = q->min_views;
    r->W = ref.w;
    r->H = ref.h;
    r->n_phases = 2 + 2 * q->params.iterations;
    r->bytes = (size_t)r->W * r->H * 6 * sizeof(float);
    r->tiles = (size_t)((r->W + TILE_W - 1) / TILE_W) * ((r->H + TILE_H - 1) / TILE_H);
    if (r->bytes > c->mem_cap) {
        const size_t need = r->bytes;
        delete r;
        s.stats.rejected++;
        return ctx_fail(c, PMSP_EADMIT, "request needs %zu bytes, above the cap", need);
    }
    for (int f : r->srcs) s.ring[f].pins++;
    for (int f : r->filters) s.ring[f].pins++;
    s.ring[r->ref].pins++;
    r->ticket = s.next_ticket++;
    s.tickets[r->ticket] = r;
    s.queue.push_back(r);
    s.stats.submitted++;
    *ticket = r->ticket;
    s.cv_work.notify_all();
    return PMSP_OK;
}

int pmsp_poll(pmsp_ctx* c, uint64_t ticket, pmsp_maps* out) {
    if (!c) return PMSP_EINVAL;
    cudaSetDevice(c->device);
    Serving& s = serving(c);
    std::lock_guard<std::mutex> lk(s.mu);
    return take(s, ticket, out, c);
}

int pmsp_wait(pmsp_ctx* c, uint64_t ticket, int timeout_ms, pmsp_maps* out) {
    if (!c) return PMSP_EINVAL;
    cudaSetDevice(c->device);
    Serving& s = serving(c);
    std::unique_lock<std::mutex> lk(s.mu);
    const auto until = Clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
    for (;;) {
        const int rc = take(s, ticket, out, c);
        if (rc != PMSP_EBUSY) return rc;
        if (s.cv_done.wait_until(lk, until) == std::cv_status::timeout) {
            const int rc2 = take(s, ticket, out, c);
            if (rc2 != PMSP_EBUSY) return rc2;
            return ctx_fail(c, PMSP_ETIMEDOUT, "ticket %llu not finished after %d ms", (unsigned long long)ticket,
                            timeout_ms);
        }
    }
}

int pmsp_get_serving_stats(pmsp_ctx* c, pmsp_serving_stats* out) {
    if (!c || !out) return PMSP_EINVAL;
    Serving& s = serving(c);
    std::lock_guard<std::mutex> lk(s.mu);
    *out = s.stats;
    return PMSP_OK;
}

}  // extern "C"
