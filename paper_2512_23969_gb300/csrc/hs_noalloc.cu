// hs_noalloc.cu -- hs_sign_batch_noalloc: signing without any device
// allocation, for callers that reserve their memory up front or embed the
// library and forbid it its own allocations (see include/hs.h).
//
// The scratch of a batch (key blocks, message offsets, digest fields, FORS
// roots, PK_FORS, layer roots, the chain ends of the chain-parallel
// TREE_Sign form, the leaves of wide trees) lives in one file-scope device
// array.  Host code cannot use the array's name as a device address,
// so the first call on each device looks the address up with
// cudaGetSymbolAddress (that device current) and caches it per device.  The
// kernels are the same ones hs_sign_batch launches, in the same order, with
// chain checkpoints off so that the scratch stays small.  The cached address
// belongs to the device's current context: it does not survive
// cudaDeviceReset (nor does the rest of the library's per-device state).
#include <cuda_runtime.h>
#include <cstdio>
#include <mutex>
#include "hs_launch.h"
#include "../../include/hs.h"

#define HS_API extern "C" __attribute__((visibility("default")))

namespace hs {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[HS_NOALLOC_SCRATCH_BYTES];

constexpr size_t kStatusBytes = 256;   // status word at the start of the array

std::mutex g_na_mu;
void* g_na_ptr[64];                    // device address of the array, per device ordinal

hs_status na_fail(hs_status st, const char* msg) {
    set_last_error(msg);
    return st;
}

// Device memory of the current device 'dev' (or managed memory).  Memory of
// another GPU is refused: the kernels would reach it without peer access.
bool is_device_ptr(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

// Device address of the array on the current device (looked up once).
hs_status scratch_ptr(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return na_fail(HS_ECUDA, "hs_sign_batch_noalloc: no usable current device");
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (g_na_ptr[dev] == nullptr) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            char buf[256];
            snprintf(buf, sizeof(buf), "hs_sign_batch_noalloc: cudaGetSymbolAddress failed: %s",
                     cudaGetErrorString(e));
            cudaGetLastError();
            return na_fail(HS_ECUDA, buf);
        }
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return HS_OK;
}

}  // namespace
}  // namespace hs

using namespace hs;

HS_API hs_status hs_sign_batch_noalloc(hs_params p, const uint8_t* sk, uint32_t num_keys,
                                       const uint32_t* key_idx, const uint8_t* msgs, const uint64_t* lens,
                                       uint32_t count, uint8_t* sigs, void* stream) {
    if ((int)p < 0 || (int)p >= kNumSets) return na_fail(HS_EINVAL, "hs_sign_batch_noalloc: invalid parameter set");
    if (count == 0) return HS_OK;
    if (!sk || !msgs || !lens || !sigs) return na_fail(HS_EINVAL, "hs_sign_batch_noalloc: NULL buffer");
    if (num_keys == 0) return na_fail(HS_EINVAL, "hs_sign_batch_noalloc: num_keys must be > 0");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return na_fail(HS_ECUDA, "hs_sign_batch_noalloc: no usable current device");
    }
    if (!is_device_ptr(sk, dev) || !is_device_ptr(msgs, dev) || !is_device_ptr(lens, dev) ||
        !is_device_ptr(sigs, dev) || (key_idx && !is_device_ptr(key_idx, dev)))
        return na_fail(HS_EINVAL, "hs_sign_batch_noalloc: every buffer must be memory of the current device");
    // TREE_Sign's form: chain-parallel where hs_sign_batch would use it and
    // its chain-end region fits the array, otherwise one thread per leaf
    // (the same bytes either way).
    bool split = tree_split(p, count);
    size_t need = kStatusBytes + scratch_bytes(p, num_keys, count, 0, split);
    if (split && need > HS_NOALLOC_SCRATCH_BYTES) {
        split = false;
        need = kStatusBytes + scratch_bytes(p, num_keys, count, 0, false);
    }
    if (need > HS_NOALLOC_SCRATCH_BYTES) {
        char buf[256];
        snprintf(buf, sizeof(buf),
                 "hs_sign_batch_noalloc: batch needs %zu bytes of scratch, the static buffer holds %zu",
                 need, (size_t)HS_NOALLOC_SCRATCH_BYTES);
        return na_fail(HS_EINVAL, buf);
    }
    void* base = nullptr;
    hs_status st = scratch_ptr(&base);
    if (st != HS_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    Batch b{};
    b.pset = p;
    b.keys_in = sk;
    b.num_keys = num_keys;
    b.key_idx = key_idx;
    b.msgs = msgs;
    b.lens = lens;
    b.count = count;
    b.sigs = sigs;
    b.ck = 0;
    b.split = split;
    b.msg_warp = msg_warp(p, count);
    // Key-index errors go to the status word hs_check_status reads when the
    // library has already set it up on this device (by any earlier call);
    // otherwise to a word at the start of the array, which nothing reads.
    uint32_t* shared_status = device_status_word_if_ready();
    b.status = shared_status ? shared_status : static_cast<uint32_t*>(base);
    carve_scratch(b, static_cast<char*>(base) + kStatusBytes);

    cudaError_t e = shared_status ? cudaSuccess : cudaMemsetAsync(b.status, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) e = launch_keyprep(b, false, s);
    if (e == cudaSuccess) e = launch_offsets(b, s);
    if (e == cudaSuccess) e = launch_message(b, false, s);
    if (e == cudaSuccess) e = launch_fors(b, s);
    if (e == cudaSuccess) e = launch_fors_pk(b, s);
    if (e == cudaSuccess) e = launch_tree(b, s);
    if (e == cudaSuccess) e = launch_wots(b, s);
    if (e != cudaSuccess) {
        char buf[256];
        snprintf(buf, sizeof(buf), "hs_sign_batch_noalloc: launch failed: %s", cudaGetErrorString(e));
        cudaGetLastError();            // consumed here: reported by the status below
        return na_fail(HS_ECUDA, buf);
    }
    return HS_OK;
}
