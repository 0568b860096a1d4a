// hs_server.cu -- continuous-batching signing server (include/hs.h, hs_server_*).
//
// Requests (parameter set, key index, message) arrive at any time through
// hs_server_submit.  A scheduler thread keeps up to 'max_inflight' batches
// on the GPU, each on its own stream: whenever a slot frees up and memory
// is available, it takes the oldest pending requests of one parameter set
// (up to 'max_batch') as the next batch, stages them through pinned host
// memory, launches message stage -> FORS_Sign || TREE_Sign -> WOTS+_Sign,
// and copies the signatures back.  Batches of different sets and different
// arrival times therefore overlap on the device, and a request that arrives
// while others are running is admitted as soon as a slot and memory free
// up -- not after the running batches drain.
//
// Admission is bounded by a device-memory budget: one device arena of
// 'mem_budget_bytes' is reserved at creation and every batch's messages,
// signatures and scratch are carved from it (first-fit, coalescing); a batch
// that does not fit waits for running batches to return memory.  Keys and
// their SHA-2 midstates are made resident once, at creation.
// Completion: each batch records an event after its signature copy; the
// scheduler polls the events (cudaEventQuery) between bounded sleeps.  No
// CUDA host function is used: a host function that waited for the
// scheduler's mutex while the scheduler, holding it, made CUDA calls could
// deadlock the two.  No thread spins on the GPU, and every wait is bounded.
#include <cuda_runtime.h>
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>
#include "hs_launch.h"
#include "../../include/hs.h"

#define HS_API extern "C" __attribute__((visibility("default")))

namespace hs {
namespace {

using Clock = std::chrono::steady_clock;
inline uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}
inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// First-fit allocator over [0, cap) with coalescing of freed ranges.
class Arena {
public:
    explicit Arena(size_t cap = 0) { reset(cap); }
    void reset(size_t cap) {
        free_.clear();
        cap_ = cap;
        used_ = 0;
        if (cap) free_[0] = cap;
    }
    // returns offset or SIZE_MAX
    size_t alloc(size_t n) {
        n = al256(n ? n : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > n) free_[off + n] = len - n;
                used_ += n;
                return off;
            }
        }
        return SIZE_MAX;
    }
    void release(size_t off, size_t n) {
        n = al256(n ? n : 1);
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t cap() const { return cap_; }

private:
    std::map<size_t, size_t> free_;
    size_t cap_ = 0, used_ = 0;
};

struct Request {
    int pset;
    uint32_t key;
    std::vector<uint8_t> msg;
    uint8_t* out;          // caller's signature buffer (host)
    uint64_t t_arrive;     // ns (submit time, or scheduled arrival in replay)
    uint64_t t_done = 0;
    int status = -1;       // -1 pending, else hs_status
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    bool failed = false;
    int pset = 0;
    std::vector<uint64_t> ids;
    size_t dev_off = 0, dev_len = 0, host_off = 0, host_len = 0;
    size_t sig_host = 0;   // offset of the signatures inside the host region
};

}  // namespace

struct ServerImpl {
    hs_server_config cfg;
    int device = 0;
    // per set: resident keys and midstates
    hs_keyset* ks[kNumSets] = {};     // resident keys (with the cached top layers)
    uint32_t nkeys[kNumSets] = {};
    // arenas
    uint8_t* dev_base = nullptr;
    uint8_t* host_base = nullptr;
    Arena dev_arena, host_arena;
    std::vector<Slot> slots;
    // requests
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::unordered_map<uint64_t, Request> reqs;
    std::deque<uint64_t> pending[kNumSets];
    std::deque<uint64_t> completed;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread th;
    // stats
    uint64_t n_done = 0, n_batches = 0, n_batched_reqs = 0, max_dev_used = 0, n_failed = 0, n_cancelled = 0;
    uint32_t max_inflight_seen = 0;
    hs_status fatal = HS_OK;
    uint32_t inject_failures = 0;   // test hook: batches to fail without launching
};

namespace {

int sig_bytes_of(int p) {
    SetShape sh;
    return set_shape(p, &sh) ? sh.sig : 0;
}

// Bytes a batch needs from each arena.
struct Need { size_t dev, host; };
Need batch_need(int pset, size_t count, size_t msg_bytes, const hs_keyset* ks) {
    const size_t sig = (size_t)count * sig_bytes_of(pset);
    Need n;
    n.host = al256(msg_bytes) + al256(count * 8) + al256(count * 4) + al256(sig);
    n.dev = n.host + al256(scratch_bytes(pset, 0, (uint32_t)count, ks->ck, tree_split(pset, (uint32_t)count),
                                         ks->layers ? ks->first_layer : 0));
    return n;
}

// Retire finished batches (lock held).
void retire(ServerImpl& sv) {
    for (auto& s : sv.slots) {
        if (!s.busy) continue;
        cudaError_t e = cudaSuccess;
        if (!s.failed) {
            e = cudaEventQuery(s.done);            // recorded after the signature copy
            if (e == cudaErrorNotReady) continue;
        } else {
            cudaStreamSynchronize(s.stream);       // whatever was queued before the failure
        }
        const int S = sig_bytes_of(s.pset);
        const uint64_t t = now_ns();
        for (size_t i = 0; i < s.ids.size(); i++) {
            auto it = sv.reqs.find(s.ids[i]);
            if (it == sv.reqs.end()) continue;
            Request& r = it->second;
            if (!s.failed && e == cudaSuccess) {
                if (r.out) memcpy(r.out, sv.host_base + s.host_off + s.sig_host + (size_t)i * S, S);
                r.status = HS_OK;
            } else {
                r.status = HS_ECUDA;
                sv.n_failed++;
            }
            r.t_done = t;
            sv.completed.push_back(s.ids[i]);
            sv.n_done++;
        }
        sv.dev_arena.release(s.dev_off, s.dev_len);
        sv.host_arena.release(s.host_off, s.host_len);
        s.ids.clear();
        s.busy = false;
        s.failed = false;
        if (e != cudaSuccess) cudaGetLastError();
        sv.cv_done.notify_all();
    }
}

constexpr size_t kMinShare = 256;

// Form and launch one batch on a free slot (lock held).  Returns false if
// nothing could be launched (no pending request, or no memory for even one).
bool admit(ServerImpl& sv, Slot& slot) {
    int best = -1;
    uint64_t oldest = UINT64_MAX;
    for (int p = 0; p < kNumSets; p++)
        if (!sv.pending[p].empty()) {
            const uint64_t t = sv.reqs[sv.pending[p].front()].t_arrive;
            if (t < oldest) { oldest = t; best = p; }
        }
    if (best < 0) return false;
    const int p = best;
    const hs_keyset* ks = sv.ks[p];
    // Batch size: up to max_batch, but no more than the backlog's share of
    // one slot (pending / max_inflight, at least kMinShare): a saturating
    // backlog still forms full batches, while a transient backlog near
    // capacity is spread over the slots instead of becoming one long batch
    // that every request in it waits for.
    size_t pending_all = 0;
    for (int q = 0; q < kNumSets; q++) pending_all += sv.pending[q].size();
    const size_t share = std::max<size_t>(kMinShare, pending_all / sv.cfg.max_inflight);
    // The message stage's warp form (a warp per message) only for a batch
    // that has the GPU to itself: it shortens a small batch's serial message
    // hashing when the GPU is otherwise idle, but in a server whose batches
    // overlap it measured worse at high load (the serving mix at 85k
    // requests/s: p99 17.5-18.0 ms with it, 11.6-12.2 ms without; at 75k
    // 4.3 vs 4.6 ms).
    bool alone = true;
    for (const Slot& o : sv.slots) alone = alone && (&o == &slot || !o.busy);
    // take requests while the cumulative need fits what the arenas could give
    size_t count = 0, msg_bytes = 0;
    const size_t limit = std::min<size_t>(std::min<size_t>(sv.cfg.max_batch, share), sv.pending[p].size());
    const size_t dev_free = sv.dev_arena.cap() - sv.dev_arena.used();
    const size_t host_free = sv.host_arena.cap() - sv.host_arena.used();
    while (count < limit) {
        const Request& r = sv.reqs[sv.pending[p][count]];
        const Need n = batch_need(p, count + 1, msg_bytes + r.msg.size(), ks);
        if (n.dev > dev_free || n.host > host_free) break;
        msg_bytes += r.msg.size();
        count++;
    }
    if (count == 0) return false;
    Need need = batch_need(p, count, msg_bytes, ks);
    size_t doff = sv.dev_arena.alloc(need.dev);
    size_t hoff = doff == SIZE_MAX ? SIZE_MAX : sv.host_arena.alloc(need.host);
    while ((doff == SIZE_MAX || hoff == SIZE_MAX) && count > 1) {   // fragmentation: shrink
        if (doff != SIZE_MAX) sv.dev_arena.release(doff, need.dev);
        count = (count + 1) / 2;
        msg_bytes = 0;
        for (size_t i = 0; i < count; i++) msg_bytes += sv.reqs[sv.pending[p][i]].msg.size();
        need = batch_need(p, count, msg_bytes, ks);
        doff = sv.dev_arena.alloc(need.dev);
        hoff = doff == SIZE_MAX ? SIZE_MAX : sv.host_arena.alloc(need.host);
    }
    if (doff == SIZE_MAX || hoff == SIZE_MAX) {
        if (doff != SIZE_MAX) sv.dev_arena.release(doff, need.dev);
        return false;
    }
    // host staging layout: msgs | lens | key_idx | sigs  (device: same, then scratch)
    uint8_t* h = sv.host_base + hoff;
    uint8_t* d = sv.dev_base + doff;
    const size_t o_lens = al256(msg_bytes), o_kidx = o_lens + al256(count * 8),
                 o_sigs = o_kidx + al256(count * 4), o_scr = o_sigs + al256(count * (size_t)sig_bytes_of(p));
    slot.ids.clear();
    size_t mo = 0;
    for (size_t i = 0; i < count; i++) {
        const uint64_t id = sv.pending[p].front();
        sv.pending[p].pop_front();
        Request& r = sv.reqs[id];
        if (!r.msg.empty()) memcpy(h + mo, r.msg.data(), r.msg.size());
        mo += r.msg.size();
        reinterpret_cast<uint64_t*>(h + o_lens)[i] = r.msg.size();
        reinterpret_cast<uint32_t*>(h + o_kidx)[i] = r.key;
        std::vector<uint8_t>().swap(r.msg);       // staged: the copy is no longer needed
        slot.ids.push_back(id);
    }
    Batch b{};
    b.pset = p;
    b.keys_in = ks->sk;
    b.num_keys = 0;                               // scratch holds no key blocks (see below)
    b.key_idx = reinterpret_cast<const uint32_t*>(d + o_kidx);
    b.msgs = msg_bytes ? d : d + o_lens;          // never read when all lengths are 0
    b.lens = reinterpret_cast<const uint64_t*>(d + o_lens);
    b.count = (uint32_t)count;
    b.sigs = d + o_sigs;
    b.ck = ks->ck;
    if (ks->layers) {                             // top layers from the keyset's cache
        b.dedup_layer = ks->first_layer;
        b.cached = true;
        b.cache_tpk = ks->tpk;
    }
    b.split = tree_split(p, (uint32_t)count);
    b.msg_warp = alone && msg_warp(p, (uint32_t)count);
    b.status = device_status_word();
    carve_scratch(b, d + o_scr);
    b.keys = ks->kb;                              // resident midstates, not scratch
    b.num_keys = ks->num_keys;
    b.nodes_u = ks->nodes;
    b.chk_u = ks->chk;
    cudaStream_t s = slot.stream;
    cudaError_t e = cudaSuccess;
    const bool injected = sv.inject_failures > 0;   // a fake failed launch: nothing reaches the GPU
    if (injected) {
        sv.inject_failures--;
        e = cudaErrorLaunchFailure;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(d, h, o_sigs, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_offsets(b, s);
    if (e == cudaSuccess) e = launch_message(b, false, s);
    if (e == cudaSuccess) e = launch_fors(b, s);
    if (e == cudaSuccess) e = launch_fors_pk(b, s);
    if (e == cudaSuccess) e = launch_tree(b, s);
    if (e == cudaSuccess) e = launch_wots(b, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h + o_sigs, d + o_sigs, count * (size_t)sig_bytes_of(p), cudaMemcpyDeviceToHost, s);
    slot.pset = p;
    slot.dev_off = doff;
    slot.dev_len = need.dev;
    slot.host_off = hoff;
    slot.host_len = need.host;
    slot.sig_host = o_sigs;
    slot.busy = true;
    slot.failed = false;
    if (e == cudaSuccess) e = cudaEventRecord(slot.done, s);
    if (e != cudaSuccess) {
        slot.failed = true;             // retire() marks the requests failed
        if (!injected) {                // a real CUDA error: the server stops taking work
            sv.fatal = HS_ECUDA;
            cudaGetLastError();
        }
    }
    sv.n_batches++;
    sv.n_batched_reqs += count;
    sv.max_dev_used = std::max<uint64_t>(sv.max_dev_used, sv.dev_arena.used());
    return true;
}

void scheduler(ServerImpl* sv) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (!sv->stop) {
        retire(*sv);
        bool launched = true;
        while (launched) {
            launched = false;
            for (auto& s : sv->slots)
                if (!s.busy && admit(*sv, s)) { launched = true; break; }
        }
        uint32_t busy = 0;
        for (auto& s : sv->slots) busy += s.busy ? 1 : 0;
        sv->max_inflight_seen = std::max(sv->max_inflight_seen, busy);
        // sleep until a submit or a short timeout (batch completions are polled)
        if (busy) sv->cv_sched.wait_for(lk, std::chrono::microseconds(100));
        else sv->cv_sched.wait_for(lk, std::chrono::milliseconds(50));
    }
    retire(*sv);
}

}  // namespace
}  // namespace hs

using namespace hs;

struct hs_server { ServerImpl impl; };

static hs_status sv_fail(hs_status st, const char* msg) {
    set_last_error(msg);
    return st;
}

HS_API hs_status hs_server_create(const hs_server_config* cfg, const uint8_t* const sks[HS_NUM_PARAMS],
                                  const uint32_t nkeys[HS_NUM_PARAMS], hs_server** out) {
    if (!cfg || !sks || !nkeys || !out) return sv_fail(HS_EINVAL, "hs_server_create: NULL argument");
    if (cfg->max_inflight < 1 || cfg->max_inflight > 16 || cfg->max_batch < 1 || cfg->mem_budget_bytes < (1u << 20))
        return sv_fail(HS_EINVAL, "hs_server_create: max_inflight 1..16, max_batch >= 1, budget >= 1 MiB");
    hs_server* s = new hs_server();
    ServerImpl& sv = s->impl;
    sv.cfg = *cfg;
    cudaGetDevice(&sv.device);
    bool ok = true;
    for (int p = 0; p < kNumSets && ok; p++) {
        sv.nkeys[p] = nkeys[p];
        if (!nkeys[p]) continue;
        if (!sks[p]) { ok = false; break; }
        SetShape sh;
        set_shape(p, &sh);
        const uint32_t layers = std::min<uint32_t>(cfg->cache_layers, (uint32_t)sh.d - 1);
        ok = hs_keyset_create((hs_params)p, sks[p], nkeys[p], layers, nullptr, &sv.ks[p]) == HS_OK;
    }
    const size_t host_bytes = cfg->pinned_bytes ? cfg->pinned_bytes : cfg->mem_budget_bytes / 2;
    ok = ok && cudaMalloc(&sv.dev_base, cfg->mem_budget_bytes) == cudaSuccess &&
         cudaHostAlloc(&sv.host_base, host_bytes, cudaHostAllocDefault) == cudaSuccess;
    if (ok) {
        sv.dev_arena.reset(cfg->mem_budget_bytes);
        sv.host_arena.reset(host_bytes);
        sv.slots = std::vector<Slot>(cfg->max_inflight);
        for (auto& sl : sv.slots)
            ok = ok && cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok || !device_status_word()) {
        cudaGetLastError();
        hs_server_destroy(s);
        return sv_fail(HS_ENOMEM, "hs_server_create: could not reserve keys, arenas or streams");
    }
    sv.th = std::thread(scheduler, &sv);
    *out = s;
    return HS_OK;
}

static hs_status submit_at(hs_server* s, hs_params p, uint32_t key, const uint8_t* msg, uint64_t len,
                           uint8_t* sig_out, uint64_t* id, uint64_t t_arrive) {
    if (!s || (int)p < 0 || (int)p >= kNumSets || (len && !msg))
        return sv_fail(HS_EINVAL, "hs_server_submit: bad argument");
    ServerImpl& sv = s->impl;
    if (key >= sv.nkeys[p]) return sv_fail(HS_EKEY, "hs_server_submit: key index out of range");
    Request r;
    r.pset = p;
    r.key = key;
    r.msg.assign(msg, msg + len);
    r.out = sig_out;
    r.t_arrive = t_arrive;
    const Need one = batch_need(p, 1, len, sv.ks[p]);
    if (one.dev > sv.dev_arena.cap() || one.host > sv.host_arena.cap())
        return sv_fail(HS_EBUDGET, "hs_server_submit: request larger than the memory budget");
    uint64_t rid;
    {
        std::lock_guard<std::mutex> lk(sv.mu);
        rid = sv.next_id++;
        sv.reqs.emplace(rid, std::move(r));
        sv.pending[p].push_back(rid);
    }
    sv.cv_sched.notify_one();
    if (id) *id = rid;
    return HS_OK;
}

HS_API hs_status hs_server_submit(hs_server* s, hs_params p, uint32_t key, const uint8_t* msg, uint64_t len,
                                  uint8_t* sig_out, uint64_t* id) {
    return submit_at(s, p, key, msg, len, sig_out, id, now_ns());
}

HS_API hs_status hs_server_wait(hs_server* s, uint64_t id, uint32_t timeout_ms) {
    if (!s) return sv_fail(HS_EINVAL, "hs_server_wait: NULL server");
    ServerImpl& sv = s->impl;
    std::unique_lock<std::mutex> lk(sv.mu);
    auto it = sv.reqs.find(id);
    if (it == sv.reqs.end()) return sv_fail(HS_EINVAL, "hs_server_wait: unknown request id");
    const bool done = sv.cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
        auto f = sv.reqs.find(id);
        return f == sv.reqs.end() || f->second.status >= 0;
    });
    if (!done) return sv_fail(HS_ETIMEOUT, "hs_server_wait: timed out");
    auto f = sv.reqs.find(id);
    return f == sv.reqs.end() ? HS_OK : (hs_status)f->second.status;   // collected by a poll: it completed
}

HS_API int hs_server_poll(hs_server* s, uint64_t* ids, uint64_t* latency_ns, int32_t* status, int max) {
    if (!s || max < 0) return -1;
    ServerImpl& sv = s->impl;
    std::lock_guard<std::mutex> lk(sv.mu);
    int n = 0;
    while (n < max && !sv.completed.empty()) {
        const uint64_t id = sv.completed.front();
        sv.completed.pop_front();
        auto it = sv.reqs.find(id);
        if (it == sv.reqs.end()) continue;
        if (ids) ids[n] = id;
        if (latency_ns) latency_ns[n] = it->second.t_done - it->second.t_arrive;
        if (status) status[n] = it->second.status;
        sv.reqs.erase(it);
        n++;
    }
    return n;
}

HS_API hs_status hs_server_get_stats(hs_server* s, hs_server_stats* st) {
    if (!s || !st) return sv_fail(HS_EINVAL, "hs_server_get_stats: NULL argument");
    ServerImpl& sv = s->impl;
    std::lock_guard<std::mutex> lk(sv.mu);
    st->completed = sv.n_done;
    st->batches = sv.n_batches;
    st->batched_requests = sv.n_batched_reqs;
    st->max_device_bytes_in_use = sv.max_dev_used;
    st->max_inflight_batches = sv.max_inflight_seen;
    st->failed = sv.n_failed;
    st->cancelled = sv.n_cancelled;
    uint64_t pend = 0;
    for (int p = 0; p < kNumSets; p++) pend += sv.pending[p].size();
    st->pending = pend;
    return sv.fatal;
}

HS_API hs_status hs_server_replay(hs_server* s, uint32_t count, const uint8_t* params, const uint32_t* keys,
                                  const uint32_t* pool_idx, const uint8_t* pool_msgs, const uint64_t* pool_lens,
                                  uint32_t pool_count, const uint64_t* arrival_ns, uint8_t* sigs,
                                  const uint64_t* sig_offsets, uint64_t* latency_ns, uint32_t timeout_ms) {
    if (!s || (count && (!params || !keys || !pool_idx || !pool_lens || !pool_count || !arrival_ns || !latency_ns)) ||
        (sigs && !sig_offsets))
        return sv_fail(HS_EINVAL, "hs_server_replay: NULL argument");
    ServerImpl& sv = s->impl;
    std::vector<uint64_t> pool_off(pool_count + 1, 0);
    for (uint32_t i = 0; i < pool_count; i++) pool_off[i + 1] = pool_off[i] + pool_lens[i];
    for (uint32_t i = 0; i < count; i++)
        if (pool_idx[i] >= pool_count) return sv_fail(HS_EINVAL, "hs_server_replay: pool index out of range");
    std::vector<uint64_t> ids(count);
    std::unordered_map<uint64_t, uint32_t> index;
    index.reserve(count * 2 + 16);
    uint32_t got = 0;
    std::vector<uint64_t> cid(4096), lat(4096);
    std::vector<int32_t> cst(4096);
    hs_status worst = HS_OK;
    // collect finished requests as they come, so the server's request table
    // stays small during a long run (it is a hash map guarded by the
    // scheduler's mutex)
    auto drain = [&]() {
        const int n = hs_server_poll(s, cid.data(), lat.data(), cst.data(), (int)cid.size());
        for (int k = 0; k < n; k++) {
            auto it = index.find(cid[k]);
            if (it != index.end()) {
                latency_ns[it->second] = lat[k];
                got++;
                if (cst[k] != HS_OK && worst == HS_OK) worst = (hs_status)cst[k];
            }
        }
        return n;
    };
    const uint64_t t0 = now_ns();
    uint64_t last_drain = t0;
    for (uint32_t i = 0; i < count; i++) {
        const uint64_t due = t0 + arrival_ns[i];
        for (uint64_t t = now_ns(); t < due; t = now_ns()) {
            if (due - t > 200000) {
                drain();
                last_drain = now_ns();
                if (due > last_drain + 100000) std::this_thread::sleep_for(std::chrono::nanoseconds(due - last_drain - 100000));
            }
        }
        const uint32_t q = pool_idx[i];
        // latency is measured from the scheduled arrival, not from the submit
        hs_status st = submit_at(s, (hs_params)params[i], keys[i], pool_msgs ? pool_msgs + pool_off[q] : nullptr,
                                 pool_lens[q], sigs ? sigs + sig_offsets[i] : nullptr, &ids[i], due);
        if (st != HS_OK) return st;
        index[ids[i]] = i;
        if (now_ns() - last_drain > 1000000) {      // at least once a millisecond while submitting
            drain();
            last_drain = now_ns();
        }
    }
    const uint64_t deadline = now_ns() + (uint64_t)timeout_ms * 1000000ull;
    while (got < count) {
        drain();
        if (got >= count) break;
        if (now_ns() > deadline) return sv_fail(HS_ETIMEOUT, "hs_server_replay: requests still pending at the timeout");
        std::unique_lock<std::mutex> lk(sv.mu);
        sv.cv_done.wait_for(lk, std::chrono::milliseconds(5));
    }
    if (worst == HS_OK) return sv.fatal;
    set_last_error("hs_server_replay: some requests failed");
    return worst;
}

HS_API hs_status hs_server_cancel(hs_server* s, uint64_t id) {
    if (!s) return sv_fail(HS_EINVAL, "hs_server_cancel: NULL server");
    ServerImpl& sv = s->impl;
    std::lock_guard<std::mutex> lk(sv.mu);
    auto it = sv.reqs.find(id);
    if (it == sv.reqs.end() || it->second.status >= 0)
        return sv_fail(HS_EINVAL, "hs_server_cancel: unknown or finished request");
    auto& q = sv.pending[it->second.pset];
    auto pos = std::find(q.begin(), q.end(), id);
    if (pos == q.end()) return sv_fail(HS_EINVAL, "hs_server_cancel: request is already running");
    q.erase(pos);
    it->second.status = HS_ECANCELED;
    it->second.t_done = now_ns();
    sv.completed.push_back(id);
    sv.n_done++;
    sv.n_cancelled++;
    sv.cv_done.notify_all();
    return HS_OK;
}

HS_API hs_status hs_server_inject_launch_failures(hs_server* s, uint32_t n) {
    if (!s) return sv_fail(HS_EINVAL, "hs_server_inject_launch_failures: NULL server");
    std::lock_guard<std::mutex> lk(s->impl.mu);
    s->impl.inject_failures = n;
    return HS_OK;
}

HS_API hs_status hs_server_destroy(hs_server* s) {
    if (!s) return HS_OK;
    ServerImpl& sv = s->impl;
    if (sv.th.joinable()) {
        {
            std::lock_guard<std::mutex> lk(sv.mu);
            sv.stop = true;
        }
        sv.cv_sched.notify_all();
        sv.th.join();
    }
    for (auto& sl : sv.slots) {
        if (sl.stream) {
            cudaStreamSynchronize(sl.stream);
            cudaStreamDestroy(sl.stream);
        }
        if (sl.done) cudaEventDestroy(sl.done);
    }
    for (int p = 0; p < kNumSets; p++) hs_keyset_destroy(sv.ks[p]);
    if (sv.dev_base) cudaFree(sv.dev_base);
    if (sv.host_base) cudaFreeHost(sv.host_base);
    delete s;
    return HS_OK;
}
