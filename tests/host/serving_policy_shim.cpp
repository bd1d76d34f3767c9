// C entry points over the serving runtime's GPU-free decisions
// (paper_2211_16266_gb300/csrc/serving_policy.h) and the tile order of the
// launches and work lists (tile_order.h), built by tests/test_host_policy.py
// with the host compiler and called through ctypes.
#include <vector>

#include "serving_policy.h"
#include "tile_order.h"

using namespace pmsp;

extern "C" {

unsigned long long sp_tile_budget(int sms) { return serving_tile_budget(sms); }

// Running request k reads run_filters[off_k, off_k + run_nf[k]) (offsets are
// the running sum of run_nf).
int sp_depth_conflict(int ref, const int* filters, int nf, const int* run_refs, const int* run_filters,
                      const int* run_nf, int n_running) {
    std::vector<DepthUse> running;
    int off = 0;
    for (int k = 0; k < n_running; ++k) {
        running.push_back(DepthUse{run_refs[k], run_filters + off, run_nf[k]});
        off += run_nf[k];
    }
    return depth_conflict(DepthUse{ref, filters, nf}, running.data(), n_running) ? 1 : 0;
}

int sp_admit_block(int running, int max_active, unsigned long long bytes_in_use, unsigned long long mem_cap,
                   unsigned long long running_tiles, unsigned long long tile_budget, unsigned long long bytes,
                   unsigned long long tiles, int conflict) {
    const AdmitState s{running, max_active, bytes_in_use, mem_cap, (size_t)running_tiles, (size_t)tile_budget};
    return admit_block(s, bytes, (size_t)tiles, conflict != 0);
}

int sp_ring_pick_slot(const int* used, const int* loading, const int* pins, const unsigned long long* seq, int n) {
    std::vector<SlotView> v(n);
    for (int i = 0; i < n; ++i) v[i] = SlotView{used[i] != 0, loading[i] != 0, pins[i], seq[i]};
    return ring_pick_slot(v.data(), n);
}

void sp_tile_of_block(int gx, int gy, int L, int* tx, int* ty) { tile_of_block(gx, gy, L, *tx, *ty); }

}  // extern "C"
