// hs_mixed.cu -- hs_sign_mixed: one call signing several batches, possibly
// under different parameter sets, as one CUDA graph launch.
//
// Per job the stage DAG of the paper (Sec. III-F: FORS_Sign and TREE_Sign
// are independent given the digest; WOTS+_Sign needs both) is laid out on
// two forked streams:
//   A: keyprep -> offsets -> message -> [fork] -> TREE_Sign -> [join] -> WOTS+_Sign
//   B:                                   [fork] -> FORS_Sign -> FORS pk -> [join]
// and all jobs fork from, and join back into, the caller's stream.  With
// use_graph the whole fork/join sequence is stream-captured into one graph
// and launched once; without it the same launches go out directly (the
// "plain" per-stage form that the graph form is measured against).  The
// instantiated graph is kept per device, with its scratch at a fixed device
// address: a later call with the same batches and launch choices relaunches
// it unchanged (no capture: one cudaGraphLaunch), and one whose DAG has the
// same shape (same sets, batch-size class and options; only pointers and
// counts differ) updates its kernel arguments in place
// (cudaGraphExecUpdate) instead of instantiating anew.
#include <cuda_runtime.h>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>
#include "hs_launch.h"
#include "../../include/hs.h"

#define HS_API extern "C" __attribute__((visibility("default")))

namespace hs {
namespace {

constexpr int kMaxJobs = 16;

struct MixedDev {
    bool init = false;
    std::mutex mu;                      // one call at a time per device: shared streams and graph
    cudaGraphExec_t exec = nullptr;     // last instantiated graph, reused when the DAG shape matches
    uint64_t instantiations = 0, updates = 0, replays = 0;
    // Graph form: its scratch is one device buffer at a fixed address, so
    // that the instantiated graph stays valid from call to call; a call
    // whose batches and launch choices equal the last graph's relaunches it
    // as it is.  Every graph launch waits for the previous one (gdone):
    // they share the buffer.
    void* gscratch = nullptr;
    size_t gcap = 0;
    cudaEvent_t gdone = nullptr;
    cudaEvent_t gin = nullptr;          // the caller's stream up to the call
    cudaStream_t glaunch = nullptr;     // graph launches (idle between calls)
    bool gdone_valid = false;
    std::vector<Batch> last_bs;
    std::vector<int> last_choice;
    cudaStream_t capture;               // graphs are captured here, launched on the caller's stream
    cudaStream_t side[2 * kMaxJobs];
    cudaEvent_t fork, msg[kMaxJobs], fors[kMaxJobs], done[kMaxJobs];
};
std::mutex g_mx_mu;
MixedDev g_mx[64];

hs_status mx_fail(hs_status st, const char* msg) {
    set_last_error(msg);
    return st;
}

hs_status mixed_dev(MixedDev** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return mx_fail(HS_ECUDA, "hs_sign_mixed: no usable current device");
    }
    std::lock_guard<std::mutex> lk(g_mx_mu);
    MixedDev& d = g_mx[dev];
    if (!d.init) {
        bool ok = cudaStreamCreateWithFlags(&d.capture, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&d.glaunch, cudaStreamNonBlocking) == cudaSuccess;
        for (int i = 0; i < 2 * kMaxJobs && ok; i++)
            ok = cudaStreamCreateWithFlags(&d.side[i], cudaStreamNonBlocking) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&d.fork, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&d.gdone, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&d.gin, cudaEventDisableTiming) == cudaSuccess;
        for (int i = 0; i < kMaxJobs && ok; i++)
            ok = cudaEventCreateWithFlags(&d.msg[i], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&d.fors[i], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&d.done[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            return mx_fail(HS_ECUDA, "hs_sign_mixed: stream/event creation failed");
        }
        d.init = true;
    }
    *out = &d;
    return HS_OK;
}

// Device memory of the current device 'dev' (or managed memory); memory of
// another GPU is refused, since the kernels would reach it without peer access.
bool is_dev(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

// The choices the launchers make at launch time from the tuning state (FORS
// lanes, TREE_Sign variant), per batch: a graph captured under other
// choices must be captured again.
std::vector<int> launch_choices(const std::vector<Batch>& bs) {
    std::vector<int> c;
    for (const Batch& b : bs) {
        c.push_back(fors_lanes(b.pset, b.count));
        c.push_back(tune_get(b.pset, 1));
        c.push_back(tune_get(b.pset, 3));
        c.push_back(tune_get(b.pset, 4));
    }
    return c;
}

bool same_batches(const std::vector<Batch>& a, const std::vector<Batch>& b) {
    return a.size() == b.size() && (a.empty() || memcmp(a.data(), b.data(), a.size() * sizeof(Batch)) == 0);
}

// Launch the kept graph after the work queued on 'origin', and make origin
// wait for it.  The graph goes to a library stream of its own (idle
// between calls; it runs the graph launches in order, so each follows the
// previous one's use of the scratch), fenced by events, rather than into
// 'origin' itself: a graph launched behind other work in a busy stream
// started ~0.14 ms later (96-message mixed batch after a 256 MB fill, 5.59
// vs 5.44 ms for the same launches on plain streams).
cudaError_t launch_graph(MixedDev& d, cudaStream_t origin) {
    cudaError_t e = cudaEventRecord(d.gin, origin);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(d.glaunch, d.gin, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(d.exec, d.glaunch);
    if (e == cudaSuccess) e = cudaEventRecord(d.gdone, d.glaunch);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, d.gdone, 0);
    return e;
}

// Enqueue every job's stage DAG (fork from / join into 'origin').
cudaError_t enqueue_jobs(MixedDev& d, std::vector<Batch>& bs, cudaStream_t origin) {
    cudaError_t e = cudaEventRecord(d.fork, origin);
    for (size_t j = 0; j < bs.size() && e == cudaSuccess; j++) {
        const Batch& b = bs[j];
        cudaStream_t A = d.side[2 * j], B = d.side[2 * j + 1];
        e = cudaStreamWaitEvent(A, d.fork, 0);
        if (e == cudaSuccess) e = launch_keyprep(b, false, A);
        if (e == cudaSuccess) e = launch_offsets(b, A);
        if (e == cudaSuccess) e = launch_message(b, false, A);
        if (e == cudaSuccess) e = cudaEventRecord(d.msg[j], A);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(B, d.msg[j], 0);
        if (e == cudaSuccess) e = launch_fors(b, B);
        if (e == cudaSuccess) e = launch_fors_pk(b, B);
        if (e == cudaSuccess) e = cudaEventRecord(d.fors[j], B);
        if (e == cudaSuccess) e = launch_tree(b, A);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(A, d.fors[j], 0);
        if (e == cudaSuccess) e = launch_wots(b, A);
        if (e == cudaSuccess) e = cudaEventRecord(d.done[j], A);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, d.done[j], 0);
    }
    return e;
}

}  // namespace
}  // namespace hs

using namespace hs;

HS_API hs_status hs_sign_mixed(const hs_sign_job* jobs, uint32_t njobs, int use_graph, void* stream) {
    if (njobs == 0) return HS_OK;
    if (!jobs) return mx_fail(HS_EINVAL, "hs_sign_mixed: NULL job array");
    if (njobs > (uint32_t)kMaxJobs) return mx_fail(HS_EINVAL, "hs_sign_mixed: at most 16 jobs per call");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<Batch> bs;
    std::vector<size_t> off;
    size_t total = 0;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return mx_fail(HS_ECUDA, "hs_sign_mixed: no usable current device");
    }
    for (uint32_t j = 0; j < njobs; j++) {
        const hs_sign_job& jb = jobs[j];
        if ((int)jb.params < 0 || (int)jb.params >= kNumSets) return mx_fail(HS_EINVAL, "hs_sign_mixed: invalid parameter set");
        if (jb.count == 0) continue;
        if (!jb.sk || !jb.msgs || !jb.lens || !jb.sigs || jb.num_keys == 0)
            return mx_fail(HS_EINVAL, "hs_sign_mixed: NULL buffer or num_keys == 0");
        if (!is_dev(jb.sk, dev) || !is_dev(jb.msgs, dev) || !is_dev(jb.lens, dev) || !is_dev(jb.sigs, dev) ||
            (jb.key_idx && !is_dev(jb.key_idx, dev)))
            return mx_fail(HS_EINVAL, "hs_sign_mixed: every buffer must be memory of the current device");
        Batch b{};
        b.pset = jb.params;
        b.keys_in = jb.sk;
        b.num_keys = jb.num_keys;
        b.key_idx = jb.key_idx;
        b.msgs = jb.msgs;
        b.lens = jb.lens;
        b.count = jb.count;
        b.sigs = jb.sigs;
        b.ck = chain_checkpoint_stride(b.pset);
        b.split = tree_split(b.pset, b.count);
        b.msg_warp = msg_warp(b.pset, b.count);
        plan_dedup(b);
        bs.push_back(b);
        off.push_back(total);
        total += scratch_bytes(b);
    }
    if (bs.empty()) return HS_OK;
    MixedDev* d = nullptr;
    hs_status st = mixed_dev(&d);
    if (st != HS_OK) return st;
    uint32_t* status = device_status_word();
    if (!status) return mx_fail(HS_ECUDA, "hs_sign_mixed: device state unavailable");
    std::lock_guard<std::mutex> lk(d->mu);
    void* base = nullptr;
    cudaError_t e = cudaSuccess;
    if (use_graph && total > d->gcap) {       // grow the graph's fixed scratch
        if (d->gdone_valid) cudaEventSynchronize(d->gdone);
        cudaFree(d->gscratch);
        d->gscratch = nullptr;
        d->gcap = 0;
        d->last_bs.clear();                   // the old graph points into the old buffer
        e = cudaMalloc(&d->gscratch, total);
        if (e == cudaSuccess) d->gcap = total;
    } else if (!use_graph) {
        e = pool_alloc(&base, total, s);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();                  // consumed here: reported by the status below
        char buf[200];
        snprintf(buf, sizeof(buf), "hs_sign_mixed: scratch of %zu bytes: %s", total, cudaGetErrorString(e));
        return mx_fail(e == cudaErrorMemoryAllocation ? HS_ENOMEM : HS_ECUDA, buf);
    }
    if (use_graph) base = d->gscratch;
    for (size_t j = 0; j < bs.size(); j++) {
        bs[j].status = status;
        carve_scratch(bs[j], static_cast<char*>(base) + off[j]);
    }
    {
    if (use_graph) {
        const std::vector<int> choice = launch_choices(bs);
        if (d->exec && same_batches(bs, d->last_bs) && choice == d->last_choice) {
            // the same batches as the last graph: relaunch it as it is
            e = launch_graph(*d, s);
            d->gdone_valid = e == cudaSuccess;
            if (e == cudaSuccess) {
                d->replays++;
                return HS_OK;
            }
            char buf[200];
            snprintf(buf, sizeof(buf), "hs_sign_mixed: %s", cudaGetErrorString(e));
            cudaGetLastError();
            return mx_fail(HS_ECUDA, buf);
        }
        cudaGraph_t g = nullptr;
        // Capture on a library stream (the caller's may be the legacy default
        // stream, which cannot be captured); the graph is launched on 'stream'.
        e = cudaStreamBeginCapture(d->capture, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = enqueue_jobs(*d, bs, d->capture);
            e = cudaStreamEndCapture(d->capture, &g);
            if (e2 != cudaSuccess) e = e2;
        }
        if (e == cudaSuccess && d->exec) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(d->exec, g, &info) == cudaSuccess) {
                d->updates++;
            } else {                    // another DAG shape: instantiate below
                cudaGetLastError();
                cudaGraphExecDestroy(d->exec);
                d->exec = nullptr;
            }
        }
        if (e == cudaSuccess && !d->exec) {
            e = cudaGraphInstantiate(&d->exec, g, 0);
            if (e == cudaSuccess) d->instantiations++;
            else d->exec = nullptr;
        }
        if (e == cudaSuccess) e = launch_graph(*d, s);
        d->gdone_valid = e == cudaSuccess;
        if (e == cudaSuccess) {
            d->last_bs = bs;
            d->last_choice = choice;
        } else {
            d->last_bs.clear();
        }
        if (g) cudaGraphDestroy(g);
    } else {
        e = enqueue_jobs(*d, bs, s);
        // A failed launch leaves that job's side streams unjoined: wait for
        // them here so the scratch freed below is not reused under them.
        if (e != cudaSuccess)
            for (size_t i = 0; i < 2 * bs.size(); i++) cudaStreamSynchronize(d->side[i]);
    }
    }
    if (!use_graph) {
        cudaError_t ef = cudaFreeAsync(base, s);
        if (e == cudaSuccess) e = ef;
    }
    if (e != cudaSuccess) {
        char buf[200];
        snprintf(buf, sizeof(buf), "hs_sign_mixed: %s", cudaGetErrorString(e));
        cudaGetLastError();
        return mx_fail(HS_ECUDA, buf);
    }
    return HS_OK;
}
