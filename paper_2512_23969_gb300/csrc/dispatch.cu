// dispatch.cu -- routes each launch to the parameter set's table with the
// tuned launch shape (see hs_tune_set in include/hs.h).
#include <algorithm>
#include <atomic>
#include "hs_launch.h"

namespace hs {

const SetOps* set_ops(int pset) {
    switch (pset) {
    case 0: return &kOps_128F;
    case 1: return &kOps_192F;
    case 2: return &kOps_256F;
    case 3: return &kOps_Toy;
    case 4: return &kOps_128S;
    case 5: return &kOps_192S;
    case 6: return &kOps_256S;
    case 7: return &kOps_K128F;
    case 8: return &kOps_K192F;
    case 9: return &kOps_K256F;
    case 10: return &kOps_K128S;
    case 11: return &kOps_K192S;
    case 12: return &kOps_K256S;
    case 13: return &kOps_R128F;
    case 14: return &kOps_R192F;
    case 15: return &kOps_R256F;
    }
    return nullptr;
}

namespace {
// -1 = not set: use the table's default (knob 5: the process-wide stride).
struct TuneSlots {
    std::atomic<int> v[kNumSets][kNumKnobs];
    TuneSlots() {
        for (auto& row : v)
            for (auto& x : row) x.store(-1);
    }
};
TuneSlots g_slots;
auto& g_tune = g_slots.v;
std::atomic<int> g_ck_default{2};
// Default batch size below which TREE_Sign runs chain-parallel, per set.
constexpr int kSplitDefault[kNumSets] = {8192, 2048, 4096, 0, 64, 64, 64, 8192, 2048, 4096, 64, 64, 64,
                                         8192, 2048, 4096};
constexpr int kStrides[] = {0, 1, 2, 4, 8};
// Default batch size below which the message stage runs a warp per message
// (SHA-2 sets; the SHAKE sets always run a thread per message).
constexpr int kMsgWarpDefault[kNumSets] = {512, 512, 512, 512, 512, 512, 512, 0, 0, 0, 0, 0, 0, 512, 512, 512};
bool is_shake(int pset) { return pset >= 7 && pset <= 12; }
}

int tune_get(int pset, int knob) {
    const SetOps* o = set_ops(pset);
    if (!o || knob < 0 || knob >= kNumKnobs) return -1;
    const int v = g_tune[pset][knob].load();
    if (v >= 0) return v;
    switch (knob) {
    case 0: return o->fors_lpt_default;
    case 1: return o->tree_minb_default;
    case 2: return kSplitDefault[pset];
    case 3: return o->tree_pol_default;
    case 4: return 1;
    case 5: return g_ck_default.load();
    case 8: return kMsgWarpDefault[pset];
    default: return 0;                  // 6, 7: no cost model
    }
}

uint32_t chain_checkpoint_stride(int pset) {
    const int v = tune_get(pset, 5);
    return v < 0 ? (uint32_t)g_ck_default.load() : (uint32_t)v;
}

void set_default_checkpoint(uint32_t stride) {
    g_ck_default.store((int)stride);
    for (auto& row : g_tune) row[5].store(-1);       // one stride for every set again
}

int tune_options(int pset, int knob, int32_t* values, int max) {
    const SetOps* o = set_ops(pset);
    if (!o || knob < 0 || knob >= kNumKnobs) return -1;
    int32_t buf[16];
    int n = 0;
    switch (knob) {
    case 0: for (int i = 0; i < o->n_fors_lpt; i++) buf[n++] = o->fors_lpt[i]; break;
    case 1: for (int i = 0; i < o->n_tree_minb; i++) buf[n++] = o->tree_minb[i]; break;
    case 2: for (int v : {0, 256, 512, 1024, 2048, 4096, 8192}) buf[n++] = v; break;   // suggestions: any value works
    case 3: for (int v : {7, 15}) if (o->tree_has(0, v, 1)) buf[n++] = v; break;
    case 4: for (int v : {1, 2}) if (o->tree_has(0, o->tree_pol_default, v)) buf[n++] = v; break;
    case 5: for (int v : kStrides) buf[n++] = v; break;
    case 8:                             // suggestions: any value works (SHAKE sets: 0 only)
        if (is_shake(pset)) buf[n++] = 0;
        else for (int v : {0, 64, 256, 512, 1024, 4096}) buf[n++] = v;
        break;
    default: buf[n++] = 0; break;       // 6, 7: measured coefficients, any value >= 0
    }
    for (int i = 0; i < n && i < max; i++)
        if (values) values[i] = buf[i];
    return n;
}

bool tree_split(int pset, uint32_t count) {
    const int below = tune_get(pset, 2);
    if (below > 0 && count < (uint32_t)below) return true;
    // Above the threshold, the per-leaf form's time is a staircase: one
    // warp per SM sub-partition already keeps the ALU pipe busy, so it
    // takes about step_us x ceil(warps / sub-partitions), while the
    // chain-parallel form's time grows with the batch (split_ns per
    // message).  Within the first few steps, where a batch just past a step
    // wastes most of its last one, take the form predicted faster.
    const int step_us = tune_get(pset, 6), split_ns = tune_get(pset, 7);
    SetShape sh{};
    if (step_us <= 0 || split_ns <= 0 || !set_shape(pset, &sh)) return false;
    const uint64_t warps = ((uint64_t)count * sh.d * sh.leaves + 31) / 32, smsp = 4ull * (uint64_t)sm_count();
    const uint64_t steps = (warps + smsp - 1) / smsp;
    if (steps > 4) return false;
    return (uint64_t)split_ns * count < (uint64_t)step_us * 1000ull * steps;
}

bool msg_warp(int pset, uint32_t count) {
    return !is_shake(pset) && count < (uint32_t)std::max(0, tune_get(pset, 8));
}

// SM count of the current device (looked up once per device).
int sm_count() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 152;
    }
    int v = cache[dev].load();
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
        cudaGetLastError();
        return 152;
    }
    cache[dev].store(v);
    return v;
}

int fors_lanes(int pset, uint32_t count) {
    const SetOps* o = set_ops(pset);
    SetShape sh{};
    if (!o || !set_shape(pset, &sh)) return -1;
    int lpt = tune_get(pset, 0);
    const uint64_t want = (uint64_t)sm_count() * 1024;
    while ((uint64_t)count * sh.k * lpt < want) {
        int wider = 0;                    // smallest compiled value above lpt
        for (int i = 0; i < o->n_fors_lpt; i++)
            if (o->fors_lpt[i] > lpt && (wider == 0 || o->fors_lpt[i] < wider)) wider = o->fors_lpt[i];
        if (wider == 0) break;
        lpt = wider;
    }
    return lpt;
}

bool tune_set(int pset, int knob, int value) {
    const SetOps* o = set_ops(pset);
    if (!o || knob < 0 || knob >= kNumKnobs) return false;
    if (knob == 2 || knob == 6 || knob == 7 || knob == 8) {   // batch-size thresholds, cost coefficients
        if (value < 0 || (knob == 8 && value > 0 && is_shake(pset))) return false;
        g_tune[pset][knob].store(value);
        return true;
    }
    if (knob == 1 || knob == 3 || knob == 4) {   // a compiled TREE_Sign combination
        int t[3] = {tune_get(pset, 1), tune_get(pset, 3), tune_get(pset, 4)};
        t[knob == 1 ? 0 : (knob == 3 ? 1 : 2)] = value;
        if (!o->tree_has(t[0], t[1], t[2])) return false;
        g_tune[pset][knob].store(value);
        return true;
    }
    int32_t opts[16];
    const int n = tune_options(pset, knob, opts, 16);
    for (int i = 0; i < n; i++)
        if (opts[i] == value) {
            g_tune[pset][knob].store(value);
            return true;
        }
    return false;
}

cudaError_t launch_keyprep(const Batch& b, bool from_pk, cudaStream_t s) {
    const SetOps* o = set_ops(b.pset);
    return o ? o->keyprep(b, from_pk, s) : cudaErrorInvalidValue;
}
cudaError_t launch_message(const Batch& b, bool verify, cudaStream_t s) {
    const SetOps* o = set_ops(b.pset);
    return o ? o->message(b, verify, s) : cudaErrorInvalidValue;
}
cudaError_t launch_fors(const Batch& b, cudaStream_t s) {
    const SetOps* o = set_ops(b.pset);
    return o ? o->fors(b, fors_lanes(b.pset, b.count), s) : cudaErrorInvalidValue;
}
cudaError_t launch_fors_pk(const Batch& b, cudaStream_t s) {
    const SetOps* o = set_ops(b.pset);
    return o ? o->fors_pk(b, s) : cudaErrorInvalidValue;
}
cudaError_t launch_tree(const Batch& b, cudaStream_t s) {
    const SetOps* o = set_ops(b.pset);
    if (!o) return cudaErrorInvalidValue;
    if (b.cached) {                       // prebuilt upper layers of a keyset
        cudaError_t e = o->tree_cached(b, s);
        if (e != cudaSuccess) return e;
    } else if (b.dedup_layer) {           // shared upper layers first
        cudaError_t e = cudaMemsetAsync(b.table, 0, sizeof(unsigned long long) << b.cap_log2, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(b.nuniq, 0, sizeof(uint32_t), s);
        if (e == cudaSuccess) e = o->tree_dedup(b, s);
        if (e != cudaSuccess) return e;
    }
    return b.split ? o->tree_split(b, s)
                   : o->tree(b, tune_get(b.pset, 1), tune_get(b.pset, 3), tune_get(b.pset, 4), s);
}
cudaError_t launch_wots(const Batch& b, cudaStream_t s) {
    const SetOps* o = set_ops(b.pset);
    return o ? o->wots(b, s) : cudaErrorInvalidValue;
}
cudaError_t launch_verify(const Batch& b, cudaStream_t s) {
    const SetOps* o = set_ops(b.pset);
    return o ? o->verify(b, s) : cudaErrorInvalidValue;
}
cudaError_t launch_keygen(int pset, const uint8_t* seeds, uint32_t count, uint8_t* pk, uint8_t* sk,
                          cudaStream_t s) {
    const SetOps* o = set_ops(pset);
    return o ? o->keygen(seeds, count, pk, sk, s) : cudaErrorInvalidValue;
}

}  // namespace hs
