// Decisions of the serving runtime (serving.cu) that need no GPU: when the
// request at the head of the queue may start, which ring slot a new frame
// takes, and how much resident work admission aims for. Plain C++ without
// CUDA types, so the host tests build and exercise it on any machine.
#pragma once

#include <cstddef>
#include <cstdint>

namespace pmsp {

// Tiles of resident work admission aims for: about two waves of six resident
// 128-thread blocks per SM (the sweep kernels keep 4 to 7). More would only
// stretch every running request's latency; a request that alone exceeds it
// still runs.
inline size_t serving_tile_budget(int sms) { return (size_t)(sms > 0 ? sms : 1) * 6 * 2; }

// The depth maps a request touches: it writes its reference's map at the end
// of its chain and its consistency filter reads its neighbours' maps.
struct DepthUse {
    int ref;
    const int* filters;
    int n_filters;
};

inline bool depth_uses_frame(const int* frames, int n, int f) {
    for (int k = 0; k < n; ++k)
        if (frames[k] == f) return true;
    return false;
}

// Whether r shares a depth map with a running request in a way that needs
// ordering: both write the same one, or one writes what the other reads.
// Running chains sit on stream lanes that are not ordered with each other.
inline bool depth_conflict(const DepthUse& r, const DepthUse* running, int n_running) {
    for (int k = 0; k < n_running; ++k) {
        const DepthUse& q = running[k];
        if (q.ref == r.ref || depth_uses_frame(r.filters, r.n_filters, q.ref) ||
            depth_uses_frame(q.filters, q.n_filters, r.ref))
            return true;
    }
    return false;
}

// What keeps the head of the queue from starting now (admission is FIFO:
// nothing behind it starts either).
enum AdmitBlock { ADMIT_OK = 0, ADMIT_SLOTS, ADMIT_MEMORY, ADMIT_TILES, ADMIT_DEPTH };

struct AdmitState {
    int running;            // requests on the GPU
    int max_active;         // lanes
    uint64_t bytes_in_use;  // maps of the running (and timed-out) requests
    uint64_t mem_cap;
    size_t running_tiles;   // tiles of the running requests
    size_t tile_budget;
};

inline int admit_block(const AdmitState& s, uint64_t bytes, size_t tiles, bool conflict) {
    if (s.running >= s.max_active) return ADMIT_SLOTS;
    if (s.bytes_in_use + bytes > s.mem_cap) return ADMIT_MEMORY;
    if (s.running_tiles > 0 && s.running_tiles + tiles > s.tile_budget) return ADMIT_TILES;
    if (conflict) return ADMIT_DEPTH;
    return ADMIT_OK;
}

// One ring slot as the push policy sees it.
struct SlotView {
    bool used;      // holds a frame
    bool loading;   // being rewritten by a push
    int pins;       // queued or running requests holding it (a loading slot holds one)
    uint64_t seq;   // push order
};

// Slot for a new frame: the first slot that holds nothing and is not being
// loaded, else the frame pushed longest ago that no request holds; -1 when
// every slot is held.
inline int ring_pick_slot(const SlotView* slots, int n) {
    for (int i = 0; i < n; ++i)
        if (!slots[i].used && !slots[i].loading) return i;
    int slot = -1;
    uint64_t oldest = UINT64_MAX;
    for (int i = 0; i < n; ++i)
        if (slots[i].pins == 0 && slots[i].seq < oldest) oldest = slots[i].seq, slot = i;
    return slot;
}

}  // namespace pmsp
