// hs_api.cu -- the C ABI of include/hs.h: argument checks, host-buffer
// staging, stream-ordered scratch, and the per-call kernel sequence
//   keyprep -> offsets -> message -> FORS_Sign -> FORS pk -> TREE_Sign -> WOTS+_Sign
// (the paper's decomposition, Sec. III and Fig. 2; FORS_Sign and TREE_Sign
// are independent given the digest, WOTS+_Sign consumes both).
#include <cuda_runtime.h>
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include "hs_launch.h"
#include "../../include/hs.h"

#define HS_API extern "C" __attribute__((visibility("default")))

namespace hs {

static thread_local std::string g_err;


static hs_status fail(hs_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
static hs_status fail(hs_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

void set_last_error(const char* msg) { g_err = msg; }

// Reports a CUDA error and consumes it: a non-sticky error (an allocation
// that failed, a bad launch configuration) must not surface again in the
// next call's launch checks.
static hs_status cuda_fail(cudaError_t e, const char* what) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? HS_ENOMEM : HS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

struct SetInfo { int n, d, k, len, sig, leaves, hp, tree_bits; };
static bool set_info(int p, SetInfo* s) {
#define HS_SETINFO(P) {P::N, P::D, P::K, P::LEN, P::SIG_BYTES, P::LEAVES, P::HP, P::TREE_BITS}
    switch (p) {
    case 0: *s = HS_SETINFO(P128f); return true;
    case 1: *s = HS_SETINFO(P192f); return true;
    case 2: *s = HS_SETINFO(P256f); return true;
    case 3: *s = HS_SETINFO(PToy); return true;
    case 4: *s = HS_SETINFO(P128s); return true;
    case 5: *s = HS_SETINFO(P192s); return true;
    case 6: *s = HS_SETINFO(P256s); return true;
    case 7: *s = HS_SETINFO(PK128f); return true;
    case 8: *s = HS_SETINFO(PK192f); return true;
    case 9: *s = HS_SETINFO(PK256f); return true;
    case 10: *s = HS_SETINFO(PK128s); return true;
    case 11: *s = HS_SETINFO(PK192s); return true;
    case 12: *s = HS_SETINFO(PK256s); return true;
    case 13: *s = HS_SETINFO(PR128f); return true;
    case 14: *s = HS_SETINFO(PR192f); return true;
    case 15: *s = HS_SETINFO(PR256f); return true;
    }
#undef HS_SETINFO
    return false;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool set_shape(int pset, SetShape* out) {
    SetInfo s{};
    if (!set_info(pset, &s)) return false;
    out->n = s.n;
    out->d = s.d;
    out->sig = s.sig;
    out->leaves = s.leaves;
    out->k = s.k;
    return true;
}

// Tree sharing within a batch (process-wide switch, off by default).
static bool g_share = false;

void plan_dedup(Batch& b) {
    b.dedup_layer = 0;
    b.cap_log2 = 0;
    b.max_uniq = 0;
    SetInfo s{};
    if (!g_share || !set_info(b.pset, &s) || b.num_keys > (1u << 20) || b.count == 0) return;
    // Share layers from the top down while the number of distinct trees a
    // layer can hold (keys x 2^bits of its tree index, at most one per
    // message) is at most half the messages, and the tree index fits the
    // 27 bits of the table key.
    uint32_t L = (uint32_t)s.d;
    uint64_t total = 0;
    for (int j = s.d - 1; j >= 1; j--) {
        const int bits = s.tree_bits - j * s.hp > 0 ? s.tree_bits - j * s.hp : 0;
        if (bits > 27) break;
        const uint64_t u = std::min<uint64_t>(b.count, (uint64_t)b.num_keys << bits);
        if (2 * u > b.count) break;
        L = (uint32_t)j;
        total += u;
    }
    if (L == (uint32_t)s.d) return;
    const uint64_t entries = (uint64_t)b.count * (s.d - L);
    uint32_t lg = 4;
    while ((1ull << lg) < 2 * entries) lg++;
    b.dedup_layer = L;
    b.cap_log2 = lg;
    b.max_uniq = (uint32_t)total;
}

// Every scratch region of a batch, in carve order (256-byte aligned each).
static constexpr int kRegions = 18;
static void scratch_layout(const Batch& b, const SetInfo& s, size_t sz[kRegions], int* n) {
    const size_t nw = (size_t)s.n / 4, cnt = b.count;
    int i = 0;
    sz[i++] = sizeof(uint32_t);                                      // reserved
    sz[i++] = (size_t)b.num_keys * sizeof(KeyBlock);                 // keys
    sz[i++] = (cnt + 1) * sizeof(uint64_t);                          // offsets
    sz[i++] = cnt * sizeof(MsgInfo);                                 // infos
    sz[i++] = cnt * s.k * nw * 4;                                    // fors_roots
    sz[i++] = cnt * nw * 4;                                          // pk_fors
    sz[i++] = cnt * s.d * nw * 4;                                    // roots
    sz[i++] = b.ck ? cnt * s.d * s.len * (16 / b.ck) * nw * 4 : 0;   // chk
    sz[i++] = b.verify ? cnt * s.len * nw * 4                        // ends (one layer when verifying)
                       : (b.split ? cnt * s.d * s.leaves * s.len * nw * 4 : 0);
    const bool sh = b.dedup_layer != 0 && !b.cached;                 // in-batch sharing
    const size_t mj = b.dedup_layer ? cnt * (s.d - b.dedup_layer) : 0;
    const size_t cap = sh ? ((size_t)1 << b.cap_log2) : 0;
    sz[i++] = cap * sizeof(unsigned long long);                      // table
    sz[i++] = sh ? mj * 4 : 0;                                       // mj_slot
    sz[i++] = mj * 4;                                                // mj_id
    sz[i++] = cap * 4;                                               // slot_id
    sz[i++] = sh ? sizeof(uint32_t) : 0;                             // nuniq
    const size_t mu = sh ? b.max_uniq : 0;
    sz[i++] = mu * sizeof(DedupDesc);                                // desc
    sz[i++] = mu * 2 * s.leaves * nw * 4 +                           // nodes_u, then chk_u
              (b.ck ? mu * s.leaves * s.len * (16 / b.ck) * nw * 4 : 0);
    sz[i++] = s.leaves > 32 ? cnt * s.d * s.leaves * nw * 4 : 0;     // leafv
    sz[i++] = b.verify ? 16 * (size_t)s.d * 4 + 2 * cnt * s.len * 4 : 0;   // vcnt, vsitem, vorder
    *n = i;
}

size_t scratch_bytes(const Batch& b) {
    SetInfo s{};
    if (!set_info(b.pset, &s)) return 0;
    size_t sz[kRegions], t = 0;
    int n;
    scratch_layout(b, s, sz, &n);
    for (int i = 0; i < n; i++) t += align256(sz[i]);
    return t;
}

size_t scratch_bytes(int pset, uint32_t num_keys, uint32_t count, uint32_t ck, bool split, uint32_t cached_from) {
    Batch b{};
    b.pset = pset;
    b.num_keys = num_keys;
    b.count = count;
    b.ck = ck;
    b.split = split;
    b.dedup_layer = cached_from;
    b.cached = cached_from != 0;
    return scratch_bytes(b);
}

void carve_scratch(Batch& b, void* base) {
    SetInfo s{};
    set_info(b.pset, &s);
    size_t sz[kRegions];
    int n;
    scratch_layout(b, s, sz, &n);
    char* p = static_cast<char*>(base);
    char* r[kRegions];
    for (int i = 0; i < n; i++) { r[i] = p; p += align256(sz[i]); }
    b.keys = reinterpret_cast<KeyBlock*>(r[1]);
    b.offsets = reinterpret_cast<uint64_t*>(r[2]);
    b.infos = reinterpret_cast<MsgInfo*>(r[3]);
    b.fors_roots = reinterpret_cast<uint32_t*>(r[4]);
    b.pk_fors = reinterpret_cast<uint32_t*>(r[5]);
    b.roots = reinterpret_cast<uint32_t*>(r[6]);
    b.chk = b.ck ? reinterpret_cast<uint32_t*>(r[7]) : nullptr;
    b.ends = (b.split || b.verify) ? reinterpret_cast<uint32_t*>(r[8]) : nullptr;
    b.leafv = s.leaves > 32 ? reinterpret_cast<uint32_t*>(r[16]) : nullptr;
    b.vcnt = b.verify ? reinterpret_cast<uint32_t*>(r[17]) : nullptr;
    b.vsitem = b.verify ? b.vcnt + 16 * s.d : nullptr;
    b.vorder = b.verify ? b.vsitem + (size_t)b.count * s.len : nullptr;
    const bool sh = b.dedup_layer != 0 && !b.cached;
    b.table = sh ? reinterpret_cast<unsigned long long*>(r[9]) : nullptr;
    b.mj_slot = sh ? reinterpret_cast<uint32_t*>(r[10]) : nullptr;
    b.mj_id = b.dedup_layer ? reinterpret_cast<uint32_t*>(r[11]) : nullptr;
    b.slot_id = sh ? reinterpret_cast<uint32_t*>(r[12]) : nullptr;
    b.nuniq = sh ? reinterpret_cast<uint32_t*>(r[13]) : nullptr;
    b.desc = sh ? reinterpret_cast<DedupDesc*>(r[14]) : nullptr;
    if (b.cached) return;             // nodes_u / chk_u belong to the keyset
    b.nodes_u = sh ? reinterpret_cast<uint32_t*>(r[15]) : nullptr;
    b.chk_u = (sh && b.ck) ? b.nodes_u + (size_t)b.max_uniq * 2 * s.leaves * (s.n / 4) : nullptr;
}

// ----------------------------------------------------------- device state
struct DevState {
    bool init = false;
    cudaMemPool_t pool = nullptr;
    uint32_t* status = nullptr;
};
static std::mutex g_mu;
static DevState g_dev[64];

static hs_status dev_state(DevState** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(HS_EINVAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    DevState& d = g_dev[dev];
    if (!d.init) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        e = cudaMemPoolCreate(&d.pool, &props);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemPoolCreate");
        uint64_t thr = UINT64_MAX;   // keep freed blocks cached for the next call
        e = cudaMemPoolSetAttribute(d.pool, cudaMemPoolAttrReleaseThreshold, &thr);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemPoolSetAttribute");
        e = cudaMalloc(&d.status, 256);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(status)");
        e = cudaMemset(d.status, 0, 256);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(status)");
        d.init = true;
    }
    *out = &d;
    return HS_OK;
}

uint32_t* device_status_word() {
    DevState* d = nullptr;
    return dev_state(&d) == HS_OK ? d->status : nullptr;
}

uint32_t* device_status_word_if_ready() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    return g_dev[dev].init ? g_dev[dev].status : nullptr;
}

cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s) {
    DevState* d = nullptr;
    if (dev_state(&d) != HS_OK) return cudaErrorUnknown;
    return cudaMallocFromPoolAsync(p, bytes, d->pool, s);
}


// 1 if p is host memory (pageable or pinned), 0 if device or managed.
// Device-side address of page-locked, mapped host memory (nullptr if p is
// not such memory).  The kernels can write signatures straight into it:
// on Grace + GB300 the stores cross NVLink-C2C coherently, so no staging
// buffer and no device-to-host copy is needed.
static bool g_direct = true;
static void* mapped_host_ptr(const void* p) {
    if (!p || !g_direct) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

static int is_host_ptr(const void* p) {
    if (!p) return 0;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) { cudaGetLastError(); return 1; }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? 0 : 1;
}

// ----------------------------------------------------------- profiling
static const char* kStageNames[7] = {"keyprep", "offsets", "message", "fors", "fors_pk", "tree", "wots"};
static bool g_prof = false;
static bool g_prof_valid = false;
static cudaEvent_t g_ev[8];
static bool g_ev_init = false;

static void prof_mark(int k, cudaStream_t s) {
    if (!g_prof) return;
    if (!g_ev_init) {
        for (int i = 0; i < 8; i++) cudaEventCreate(&g_ev[i]);
        g_ev_init = true;
    }
    cudaEventRecord(g_ev[k], s);
}

// ----------------------------------------------------------- staging
struct Staging {
    void* base = nullptr;
    size_t off = 0;
    size_t cap = 0;
    char* take(size_t n) {
        char* p = static_cast<char*>(base) + off;
        off += align256(n);
        return p;
    }
};

}  // namespace hs

using namespace hs;

HS_API size_t hs_sig_bytes(hs_params p) { SetInfo s; return set_info(p, &s) ? (size_t)s.sig : 0; }
HS_API size_t hs_pk_bytes(hs_params p) { SetInfo s; return set_info(p, &s) ? (size_t)2 * s.n : 0; }
HS_API size_t hs_sk_bytes(hs_params p) { SetInfo s; return set_info(p, &s) ? (size_t)4 * s.n : 0; }
HS_API size_t hs_seed_bytes(hs_params p) { SetInfo s; return set_info(p, &s) ? (size_t)3 * s.n : 0; }
HS_API const char* hs_last_error(void) { return g_err.c_str(); }
HS_API hs_status hs_last_error_copy(char* buf, size_t len) {
    if (!buf || len == 0) return HS_EINVAL;      // the error text itself is kept
    const size_t n = std::min(len - 1, g_err.size());
    memcpy(buf, g_err.data(), n);
    buf[n] = '\0';
    return HS_OK;
}
HS_API int hs_sign_kernel_count(void) { return 7; }

HS_API int hs_tune_options(hs_params p, int knob, int32_t* values, int max) {
    return tune_options(p, knob, values, max);
}

HS_API hs_status hs_tune_set(hs_params p, int knob, int32_t value) {
    if (!tune_set(p, knob, value))
        return fail(HS_EINVAL, "tuning value %d is not available for set %d, knob %d", value, (int)p, knob);
    return HS_OK;
}

HS_API int32_t hs_tune_get(hs_params p, int knob) { return tune_get(p, knob); }

HS_API hs_status hs_set_host_direct(int on) {
    g_direct = on != 0;
    return HS_OK;
}

HS_API hs_status hs_set_tree_sharing(int on) {
    g_share = on != 0;
    return HS_OK;
}

HS_API hs_status hs_set_chain_checkpoint(uint32_t stride) {
    if (stride != 0 && stride != 1 && stride != 2 && stride != 4 && stride != 8)
        return fail(HS_EINVAL, "checkpoint stride must be 0, 1, 2, 4 or 8 (got %u)", stride);
    set_default_checkpoint(stride);
    return HS_OK;
}
HS_API void hs_profile_enable(int on) { g_prof = on != 0; g_prof_valid = false; }

HS_API int hs_profile_read(float* ms, const char** names, int max) {
    if (!g_prof_valid) return -1;
    int n = 0;
    for (int k = 0; k < 7 && n < max; k++, n++) {
        float t = 0.f;
        if (cudaEventSynchronize(g_ev[k + 1]) != cudaSuccess ||
            cudaEventElapsedTime(&t, g_ev[k], g_ev[k + 1]) != cudaSuccess) {
            cudaGetLastError();
            t = -1.f;
        }
        if (ms) ms[n] = t;
        if (names) names[n] = kStageNames[k];
    }
    return n;
}

HS_API hs_status hs_check_status(void* stream, uint32_t* flags) {
    DevState* d = nullptr;
    hs_status st = dev_state(&d);
    if (st != HS_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    uint32_t v = 0;
    e = cudaMemcpy(&v, d->status, sizeof(v), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(status)");
    e = cudaMemset(d->status, 0, sizeof(uint32_t));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(status)");
    if (flags) *flags = v;
    if (v & (1u << HS_EKEY)) return fail(HS_EKEY, "a key index was out of range");
    return HS_OK;
}

HS_API hs_status hs_keygen(hs_params p, const uint8_t* seeds, uint32_t count, uint8_t* pk, uint8_t* sk,
                           void* stream) {
    SetInfo si{};
    if (!set_info(p, &si)) return fail(HS_EINVAL, "invalid parameter set %d", (int)p);
    if (count == 0) return HS_OK;
    if (!seeds || !pk || !sk) return fail(HS_EINVAL, "NULL buffer");
    DevState* d = nullptr;
    hs_status st = dev_state(&d);
    if (st != HS_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t nseed = (size_t)count * 3 * si.n, npk = (size_t)count * 2 * si.n, nsk = (size_t)count * 4 * si.n;
    const int hs_ = is_host_ptr(seeds), hp = is_host_ptr(pk), hk = is_host_ptr(sk);
    Staging sg;
    const size_t need = (hs_ ? align256(nseed) : 0) + (hp ? align256(npk) : 0) + (hk ? align256(nsk) : 0);
    cudaError_t e;
    if (need) {
        e = cudaMallocFromPoolAsync(&sg.base, need, d->pool, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocFromPoolAsync(keygen staging)");
    }
    const uint8_t* dseeds = seeds;
    uint8_t* dpk = pk;
    uint8_t* dsk = sk;
    if (hs_) {
        uint8_t* t = reinterpret_cast<uint8_t*>(sg.take(nseed));
        e = cudaMemcpyAsync(t, seeds, nseed, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(seeds)");
        dseeds = t;
    }
    if (hp) dpk = reinterpret_cast<uint8_t*>(sg.take(npk));
    if (hk) dsk = reinterpret_cast<uint8_t*>(sg.take(nsk));
    e = launch_keygen(p, dseeds, count, dpk, dsk, s);
    if (e != cudaSuccess) return cuda_fail(e, "keygen launch");
    if (hp && (e = cudaMemcpyAsync(pk, dpk, npk, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(pk)");
    if (hk && (e = cudaMemcpyAsync(sk, dsk, nsk, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(sk)");
    if (need) {
        e = cudaFreeAsync(sg.base, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFreeAsync");
    }
    if (hs_ || hp || hk) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    }
    return HS_OK;
}

// Shared driver for sign (verify = false) and verify (verify = true); ks =
// a keyset whose resident keys (and cached top layers) replace keys_in.
// fips: FIPS 205 index order, and prefix (host, plen <= 257 bytes) hashed
// before every message.
static hs_status run_batch(const hs_keyset* ks, bool verify, hs_params p, const uint8_t* keys_in,
                           uint32_t num_keys, const uint32_t* key_idx, const uint8_t* msgs, const uint64_t* lens,
                           const uint8_t* sigs_in, uint8_t* sigs_out, uint32_t count, uint8_t* ok, void* stream,
                           bool fips = false, const uint8_t* prefix = nullptr, uint32_t plen = 0) {
    SetInfo si{};
    if (!set_info(p, &si)) return fail(HS_EINVAL, "invalid parameter set %d", (int)p);
    if (count == 0) return HS_OK;
    if (!keys_in || !lens || (!verify && !sigs_out) || (verify && (!sigs_in || !ok)))
        return fail(HS_EINVAL, "NULL buffer");
    if (num_keys == 0) return fail(HS_EINVAL, "num_keys must be > 0");
    if (verify && (uint64_t)count * si.len >= (1ull << 28))
        return fail(HS_EINVAL, "verify: at most %llu signatures per call", (unsigned long long)((1ull << 28) / si.len - 1));
    DevState* d = nullptr;
    hs_status st = dev_state(&d);
    if (st != HS_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;

    const size_t key_bytes = (size_t)num_keys * (verify ? 2 : 4) * si.n;
    const size_t sig_total = (size_t)count * si.sig;
    const int h_keys = is_host_ptr(keys_in), h_idx = is_host_ptr(key_idx), h_lens = is_host_ptr(lens);
    const int h_msgs = is_host_ptr(msgs);
    // signatures into mapped host memory: written in place by the kernels
    void* sig_direct = (!verify && is_host_ptr(sigs_out)) ? mapped_host_ptr(sigs_out) : nullptr;
    const int h_sig = verify ? is_host_ptr(sigs_in) : (is_host_ptr(sigs_out) && !sig_direct);
    const int h_ok = verify ? is_host_ptr(ok) : 0;
    uint64_t msg_total = 0;
    if (h_msgs) {
        if (!h_lens) return fail(HS_EINVAL, "msgs is host memory but lens is device memory");
        for (uint32_t i = 0; i < count; i++) {
            if (lens[i] > (1ull << 60) || msg_total + lens[i] < msg_total)
                return fail(HS_EINVAL, "message length overflow at %u", i);
            msg_total += lens[i];
        }
    }
    if (!msgs) {
        // a NULL message buffer is only valid when every length is zero,
        // which can only be checked when the lengths are host memory
        if (!h_lens) return fail(HS_EINVAL, "msgs is NULL and lens is device memory");
        for (uint32_t i = 0; i < count; i++)
            if (lens[i]) return fail(HS_EINVAL, "msgs is NULL but lens[%u] = %llu", i, (unsigned long long)lens[i]);
    }

    Batch b;
    memset(&b, 0, sizeof(b));
    b.pset = p;
    b.num_keys = num_keys;
    b.count = count;
    b.status = d->status;
    b.ck = verify ? 0u : (ks ? ks->ck : chain_checkpoint_stride(p));
    b.split = !verify && tree_split(p, count);
    b.msg_warp = msg_warp(p, count);
    b.verify = verify;
    if (ks && ks->layers) {
        b.dedup_layer = ks->first_layer;
        b.cached = true;
        b.cache_tpk = ks->tpk;
    } else if (!verify) {
        plan_dedup(b);
    }
    if (ks) b.num_keys = 0;                       // no key blocks in scratch: they are resident
    const size_t scratch = scratch_bytes(b);
    b.num_keys = num_keys;
    const size_t stage = (h_keys ? align256(key_bytes) : 0) + (h_idx ? align256((size_t)count * 4) : 0) +
                         (h_lens ? align256((size_t)count * 8) : 0) + (h_msgs ? align256(msg_total) : 0) +
                         (h_sig ? align256(sig_total) : 0) + (h_ok ? align256(count) : 0) + align256(plen);
    void* base = nullptr;
    e = cudaMallocFromPoolAsync(&base, scratch + stage, d->pool, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocFromPoolAsync(scratch)");
    carve_scratch(b, base);
    if (ks) {
        b.keys = ks->kb;
        b.nodes_u = ks->nodes;
        b.chk_u = ks->chk;
    }
    Staging sg;
    sg.base = static_cast<char*>(base) + scratch;

    auto h2d = [&](const void* src, size_t n, const char* what) -> const void* {
        void* t = sg.take(n);
        if (n) {
            cudaError_t ee = cudaMemcpyAsync(t, src, n, cudaMemcpyHostToDevice, s);
            if (ee != cudaSuccess) { cuda_fail(ee, what); return nullptr; }
        }
        return t;
    };
    b.keys_in = h_keys ? static_cast<const uint8_t*>(h2d(keys_in, key_bytes, "copy keys")) : keys_in;
    b.key_idx = (key_idx && h_idx) ? static_cast<const uint32_t*>(h2d(key_idx, (size_t)count * 4, "copy key_idx")) : key_idx;
    b.lens = h_lens ? static_cast<const uint64_t*>(h2d(lens, (size_t)count * 8, "copy lens")) : lens;
    b.msgs = h_msgs ? static_cast<const uint8_t*>(h2d(msgs, msg_total, "copy msgs")) : msgs;
    if (verify) {
        b.sigs = h_sig ? const_cast<uint8_t*>(static_cast<const uint8_t*>(h2d(sigs_in, sig_total, "copy sigs")))
                       : const_cast<uint8_t*>(sigs_in);
        b.ok = h_ok ? reinterpret_cast<uint8_t*>(sg.take(count)) : ok;
    } else {
        b.sigs = h_sig ? reinterpret_cast<uint8_t*>(sg.take(sig_total))
                       : (sig_direct ? static_cast<uint8_t*>(sig_direct) : sigs_out);
    }
    b.fips = fips;
    b.prefix_len = plen;
    b.prefix = plen ? static_cast<const uint8_t*>(h2d(prefix, plen, "copy prefix")) : nullptr;
    if (!b.keys_in || !b.lens || (h_msgs && !b.msgs) || !b.sigs || (plen && !b.prefix)) {
        cudaFreeAsync(base, s);
        return HS_ECUDA;
    }
    if (!b.msgs) b.msgs = reinterpret_cast<const uint8_t*>(b.offsets);   // never read: all lengths 0

    const bool prof = g_prof && !verify;
    if (prof) prof_mark(0, s);
    e = ks ? cudaSuccess : launch_keyprep(b, verify, s);
    if (prof) prof_mark(1, s);
    if (e == cudaSuccess) e = launch_offsets(b, s);
    if (prof) prof_mark(2, s);
    if (e == cudaSuccess) e = launch_message(b, verify, s);
    if (prof) prof_mark(3, s);
    if (!verify) {
        if (e == cudaSuccess) e = launch_fors(b, s);
        if (prof) prof_mark(4, s);
        if (e == cudaSuccess) e = launch_fors_pk(b, s);
        if (prof) prof_mark(5, s);
        if (e == cudaSuccess) e = launch_tree(b, s);
        if (prof) prof_mark(6, s);
        if (e == cudaSuccess) e = launch_wots(b, s);
        if (prof) prof_mark(7, s);
    } else {
        if (e == cudaSuccess) e = launch_verify(b, s);
    }
    if (e != cudaSuccess) {
        cudaFreeAsync(base, s);
        return cuda_fail(e, "kernel launch");
    }
    if (prof) g_prof_valid = true;
    if (!verify && h_sig) {
        e = cudaMemcpyAsync(sigs_out, b.sigs, sig_total, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "copy sigs back");
    }
    if (verify && h_ok) {
        e = cudaMemcpyAsync(ok, b.ok, count, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "copy ok back");
    }
    e = cudaFreeAsync(base, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFreeAsync");
    if (h_keys || h_idx || h_lens || h_msgs || h_sig || h_ok || sig_direct) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    }
    return HS_OK;
}

HS_API hs_status hs_sign_batch(hs_params p, const uint8_t* sk, uint32_t num_keys, const uint32_t* key_idx,
                               const uint8_t* msgs, const uint64_t* lens, uint32_t count, uint8_t* sigs,
                               void* stream) {
    return run_batch(nullptr, false, p, sk, num_keys, key_idx, msgs, lens, nullptr, sigs, count, nullptr, stream);
}

HS_API hs_status hs_verify_batch(hs_params p, const uint8_t* pk, uint32_t num_keys, const uint32_t* key_idx,
                                 const uint8_t* msgs, const uint64_t* lens, const uint8_t* sigs, uint32_t count,
                                 uint8_t* ok, void* stream) {
    return run_batch(nullptr, true, p, pk, num_keys, key_idx, msgs, lens, sigs, nullptr, count, ok, stream);
}

// ----------------------------------------------------------- FIPS 205
// The pure-signing prefix 0x00 || len(ctx) || ctx, or none for the
// internal functions (ctx_len == HS_SLH_INTERNAL).
// FIPS 205 defines no robust sets.
static bool robust_set(hs_params p) { return (int)p >= HS_ROBUST_128F && (int)p <= HS_ROBUST_256F; }

static hs_status slh_prefix(const uint8_t* ctx, uint32_t ctx_len, uint8_t* out, uint32_t* plen) {
    if (ctx_len == HS_SLH_INTERNAL) { *plen = 0; return HS_OK; }
    if (ctx_len > 255) return fail(HS_EINVAL, "context string of %u bytes (at most 255)", ctx_len);
    if (ctx_len && !ctx) return fail(HS_EINVAL, "NULL context string");
    out[0] = 0;
    out[1] = (uint8_t)ctx_len;
    if (ctx_len) memcpy(out + 2, ctx, ctx_len);
    *plen = 2 + ctx_len;
    return HS_OK;
}

HS_API hs_status hs_slh_sign_batch(hs_params p, const uint8_t* sk, uint32_t num_keys, const uint32_t* key_idx,
                                   const uint8_t* ctx, uint32_t ctx_len, const uint8_t* msgs, const uint64_t* lens,
                                   uint32_t count, uint8_t* sigs, void* stream) {
    if (robust_set(p)) return fail(HS_EINVAL, "FIPS 205 has no robust parameter sets");
    uint8_t pre[258];
    uint32_t plen = 0;
    const hs_status st = slh_prefix(ctx, ctx_len, pre, &plen);
    if (st != HS_OK) return st;
    return run_batch(nullptr, false, p, sk, num_keys, key_idx, msgs, lens, nullptr, sigs, count, nullptr, stream,
                     true, pre, plen);
}

HS_API hs_status hs_slh_verify_batch(hs_params p, const uint8_t* pk, uint32_t num_keys, const uint32_t* key_idx,
                                     const uint8_t* ctx, uint32_t ctx_len, const uint8_t* msgs, const uint64_t* lens,
                                     const uint8_t* sigs, uint32_t count, uint8_t* ok, void* stream) {
    if (robust_set(p)) return fail(HS_EINVAL, "FIPS 205 has no robust parameter sets");
    uint8_t pre[258];
    uint32_t plen = 0;
    const hs_status st = slh_prefix(ctx, ctx_len, pre, &plen);
    if (st != HS_OK) return st;
    return run_batch(nullptr, true, p, pk, num_keys, key_idx, msgs, lens, sigs, nullptr, count, ok, stream, true,
                     pre, plen);
}

// ----------------------------------------------------------- keysets
static void keyset_free(hs_keyset* ks) {
    if (!ks) return;
    cudaFree(ks->sk);
    cudaFree(ks->kb);
    cudaFree(ks->nodes);
    cudaFree(ks->chk);
    delete ks;
}

HS_API hs_status hs_keyset_create(hs_params p, const uint8_t* sk, uint32_t num_keys, uint32_t cache_layers,
                                  void* stream, hs_keyset** out) {
    SetInfo si{};
    if (!set_info(p, &si)) return fail(HS_EINVAL, "invalid parameter set %d", (int)p);
    if (!sk || !out || num_keys == 0) return fail(HS_EINVAL, "hs_keyset_create: NULL buffer or no keys");
    if (cache_layers > (uint32_t)si.d - 1)
        return fail(HS_EINVAL, "cache_layers %u: at most d - 1 = %d", cache_layers, si.d - 1);
    if (cache_layers && (uint64_t)(cache_layers - 1) * si.hp > 24)
        return fail(HS_EINVAL, "cache_layers %u: more than 2^24 trees per key", cache_layers);
    uint64_t tpk = 0;
    for (uint32_t u = 0; u < cache_layers; u++) tpk += 1ull << (u * si.hp);
    const uint64_t trees = tpk * num_keys;
    if (trees >= (1ull << 32)) return fail(HS_EINVAL, "hs_keyset_create: more than 2^32 cached trees");
    DevState* d = nullptr;
    hs_status st = dev_state(&d);
    if (st != HS_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    hs_keyset* ks = new hs_keyset();
    cudaGetDevice(&ks->device);
    ks->pset = p;
    ks->num_keys = num_keys;
    ks->layers = cache_layers;
    ks->first_layer = (uint32_t)si.d - cache_layers;
    ks->tpk = (uint32_t)tpk;
    ks->ck = chain_checkpoint_stride(p);
    const size_t nw = (size_t)si.n / 4, sk_bytes = (size_t)num_keys * 4 * si.n;
    const size_t node_bytes = (size_t)trees * 2 * si.leaves * nw * 4;
    const size_t chk_bytes = ks->ck ? (size_t)trees * si.leaves * si.len * (16 / ks->ck) * nw * 4 : 0;
    ks->bytes = sk_bytes + (size_t)num_keys * sizeof(KeyBlock) + node_bytes + chk_bytes;
    cudaError_t e = cudaMalloc(&ks->sk, sk_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&ks->kb, (size_t)num_keys * sizeof(KeyBlock));
    if (e == cudaSuccess && node_bytes) e = cudaMalloc(&ks->nodes, node_bytes);
    if (e == cudaSuccess && chk_bytes) e = cudaMalloc(&ks->chk, chk_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        keyset_free(ks);
        return cuda_fail(e, "hs_keyset_create: cudaMalloc");
    }
    e = cudaMemcpyAsync(ks->sk, sk, sk_bytes, cudaMemcpyDefault, s);
    Batch b;
    memset(&b, 0, sizeof(b));
    b.pset = p;
    b.keys_in = ks->sk;
    b.num_keys = num_keys;
    b.keys = ks->kb;
    if (e == cudaSuccess) e = launch_keyprep(b, false, s);
    void* desc = nullptr;
    if (e == cudaSuccess && trees) {
        e = cudaMallocFromPoolAsync(&desc, (size_t)trees * sizeof(DedupDesc), d->pool, s);
        if (e == cudaSuccess)
            e = set_ops(p)->cache_build(ks->kb, num_keys, ks->first_layer, ks->tpk, static_cast<DedupDesc*>(desc),
                                        ks->nodes, ks->chk, ks->ck, s);
        if (desc) {
            const cudaError_t f = cudaFreeAsync(desc, s);
            if (e == cudaSuccess) e = f;
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(s);
        keyset_free(ks);
        return cuda_fail(e, "hs_keyset_create: build");
    }
    *out = ks;
    return HS_OK;
}

HS_API size_t hs_keyset_bytes(const hs_keyset* ks) { return ks ? ks->bytes : 0; }

HS_API hs_status hs_sign_keyset(const hs_keyset* ks, const uint32_t* key_idx, const uint8_t* msgs,
                                const uint64_t* lens, uint32_t count, uint8_t* sigs, void* stream) {
    if (!ks) return fail(HS_EINVAL, "hs_sign_keyset: NULL keyset");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != ks->device) return fail(HS_EINVAL, "hs_sign_keyset: keyset of device %d used on %d", ks->device, dev);
    return run_batch(ks, false, (hs_params)ks->pset, ks->sk, ks->num_keys, key_idx, msgs, lens, nullptr, sigs, count,
                     nullptr, stream);
}

HS_API hs_status hs_keyset_destroy(hs_keyset* ks) {
    if (!ks) return HS_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ks->device);
    keyset_free(ks);
    cudaSetDevice(prev);
    return HS_OK;
}
