// kern_verify.cuh -- batched signature verification on the GPU.
//
// The scheme's verification (the paper signs only; this is the definition's
// inverse of Fig. 2): PK_FORS from the FORS signature (leaf from the
// revealed secret, a climbs with the auth path, T_k over the roots), then
// for each layer j the WOTS+ public key from the signature of msg_j (chain i
// advanced from digit_i to w-1), T_len, and h' climbs with the auth path to
// root_j = msg_{j+1}.  Valid iff root_{d-1} equals PK.root.
//
// GB300 mapping: verification is serial across layers (layer j's digits
// come from root_{j-1}), but a batch has count x len independent chains in
// every layer.  So: one thread per (message, FORS tree) for the FORS roots
// (then the signer's T_k kernel for PK_FORS); then for each layer one
// thread per (message, chain) advancing its chain to the end, and one
// thread per message for T_len and the h' climbs, which leaves root_j in
// scratch for the next layer; finally a comparison with PK.root.
// A chain needs w - 1 - digit steps (0 .. 15), so a warp of chains in
// message order waits for its longest.  The chains of a layer are
// therefore bucketed by their step count (the thread that produced msg_j
// counts its message's digits and takes ranks with 16 atomics), scattered
// longest first, and the chain kernel runs them in that order: the chains
// of a warp then have the same length.
#pragma once
#include <cuda_runtime.h>
#include "hs_common.cuh"
#include "hs_launch.h"
#include "sha256_chain.cuh"

namespace hs {

// FORS root i of message m from the signature: leaf from the revealed
// secret, a climbs with the auth path.
template <class P>
__global__ void __launch_bounds__(128) vfors_kernel(const KeyBlock* __restrict__ keys,
                                                    const MsgInfo* __restrict__ infos, uint32_t count,
                                                    const uint8_t* __restrict__ sigs,
                                                    uint32_t* __restrict__ fors_roots) {
    constexpr int NW = P::NW, A = P::A, K = P::K;
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t m = gid / K;
    const uint32_t i = (uint32_t)(gid % K);
    if (m >= count) return;
    const MsgInfo& info = infos[m];
    if (info.key == KEY_INVALID) return;
    const KeyBlock& kb = keys[info.key];
    uint32_t ms256[8], msT[P::BIG ? 16 : 8];
#pragma unroll
    for (int w = 0; w < 8; w++) ms256[w] = kb.ms256[w];
#pragma unroll
    for (int w = 0; w < (P::BIG ? 16 : 8); w++) msT[w] = P::BIG ? kb.ms512[w] : kb.ms256[w];
    const uint8_t* s = sigs + (size_t)m * P::SIG_BYTES + P::N + (size_t)i * (A + 1) * P::N;
    const uint32_t g = (i << A) + info.fors_idx[i];
    uint32_t sk[NW], node[NW];
    load_be<NW>(s, sk);
    hashF<P, false>(ms256, make_adrs(0, info.idx_tree, T_FORS_TREE, info.idx_leaf, 0, g), sk, node, kb.pk_seed);
#pragma unroll 1
    for (int z = 0; z < A; z++) {
        const uint32_t gz = g >> z;
        uint32_t au[NW], lr[2 * NW];
        load_be<NW>(s + (size_t)(1 + z) * P::N, au);
#pragma unroll
        for (int w = 0; w < NW; w++) {
            lr[w] = (gz & 1) ? au[w] : node[w];
            lr[NW + w] = (gz & 1) ? node[w] : au[w];
        }
        hashH_ms<P>(ms256, msT, make_adrs(0, info.idx_tree, T_FORS_TREE, info.idx_leaf, z + 1, gz >> 1), lr, node,
                    kb.pk_seed);
    }
    uint32_t* r = fors_roots + ((size_t)m * K + i) * NW;
#pragma unroll
    for (int w = 0; w < NW; w++) r[w] = node[w];
}

// The len base-w digits of an n-byte value (message nibbles, high first,
// then the 3 checksum digits).
template <class P>
__device__ __forceinline__ uint32_t wots_digit(const uint32_t* msg, uint32_t i) {
    constexpr int NW = P::NW;
    if (i < (uint32_t)P::LEN1) return (msg[i >> 3] >> (28 - 4 * (i & 7))) & 15u;
    uint32_t csum = 0;
#pragma unroll
    for (int w = 0; w < NW; w++)
#pragma unroll
        for (int b = 0; b < 8; b++) csum += 15u - ((msg[w] >> (28 - 4 * b)) & 15u);
    return ((csum << 4) >> (12 - 4 * (i - P::LEN1))) & 15u;
}

constexpr uint32_t kRankBits = 28;        // sitem = steps << 28 | rank within the steps bucket

// For message m's layer: each chain's step count, counted into the layer's
// 16 buckets, with the chain's rank inside its bucket recorded in sitem.
// Called by all 32 lanes of a warp, converged (inactive lanes count
// nothing): per bucket the warp scans its lanes' counts with shuffles and
// one lane adds the warp's total with a single atomic, so the 16 counters
// see one atomic per warp instead of one per thread.  Messages with an
// invalid key count as 0 steps.
template <class P>
__device__ __forceinline__ void count_steps(const uint32_t* msg, bool active, bool valid, uint64_t m,
                                            uint32_t* __restrict__ cnt, uint32_t* __restrict__ sitem) {
    constexpr int LEN = P::LEN;
    const uint32_t lane = threadIdx.x & 31;
    uint32_t hist[16];
#pragma unroll
    for (int b = 0; b < 16; b++) hist[b] = 0;
    if (active) {
#pragma unroll 1
        for (uint32_t i = 0; i < (uint32_t)LEN; i++) {
            const uint32_t st = valid ? 15u - wots_digit<P>(msg, i) : 0u;
#pragma unroll
            for (int b = 0; b < 16; b++) hist[b] += (st == (uint32_t)b) ? 1u : 0u;
        }
    }
    uint32_t base[16];
#pragma unroll
    for (int b = 0; b < 16; b++) {
        uint32_t x = hist[b];                       // inclusive scan over the lanes
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
            if (lane >= (uint32_t)off) x += y;
        }
        const uint32_t total = __shfl_sync(0xFFFFFFFFu, x, 31);
        uint32_t wbase = 0;
        if (lane == 31 && total) wbase = atomicAdd(&cnt[b], total);
        wbase = __shfl_sync(0xFFFFFFFFu, wbase, 31);
        base[b] = wbase + x - hist[b];
    }
    if (!active) return;
#pragma unroll 1
    for (uint32_t i = 0; i < (uint32_t)LEN; i++) {
        const uint32_t st = valid ? 15u - wots_digit<P>(msg, i) : 0u;
        uint32_t r = 0;
#pragma unroll
        for (int b = 0; b < 16; b++)
            if (st == (uint32_t)b) r = base[b]++;
        sitem[m * LEN + i] = (st << kRankBits) | r;
    }
}

// Layer 0: count from PK_FORS (every lane of every warp takes part).
template <class P>
__global__ void __launch_bounds__(128) vcount0_kernel(const MsgInfo* __restrict__ infos, uint32_t count,
                                                      const uint32_t* __restrict__ pk_fors, uint32_t* __restrict__ cnt,
                                                      uint32_t* __restrict__ sitem) {
    const uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = m < count;
    const bool valid = active && infos[m].key != KEY_INVALID;
    uint32_t msg[P::NW];
#pragma unroll
    for (int w = 0; w < P::NW; w++) msg[w] = active ? pk_fors[(size_t)m * P::NW + w] : 0u;
    count_steps<P>(msg, active, valid, m, cnt, sitem);
}

// Place every chain of the layer at its sorted position (longest first).
template <class P>
__global__ void __launch_bounds__(256) vscatter_kernel(uint32_t count, const uint32_t* __restrict__ cnt,
                                                       const uint32_t* __restrict__ sitem, uint32_t* __restrict__ order) {
    const uint64_t it = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= (uint64_t)count * P::LEN) return;
    const uint32_t v = sitem[it];
    const uint32_t st = v >> kRankBits, r = v & ((1u << kRankBits) - 1u);
    uint32_t base = 0;
#pragma unroll
    for (int b = 15; b >= 0; b--) base += ((uint32_t)b > st) ? cnt[b] : 0u;
    order[base + r] = (uint32_t)it;
}

// Layer j, chain i of message m: its digit from msg_j (PK_FORS for j = 0,
// else root_{j-1} in vroot), then F from the signed position to w - 1.
template <class P, int POL>
__global__ void __launch_bounds__(128) vchain_kernel(const KeyBlock* __restrict__ keys,
                                                     const MsgInfo* __restrict__ infos, uint32_t count,
                                                     const uint8_t* __restrict__ sigs,
                                                     const uint32_t* __restrict__ order,
                                                     const uint32_t* __restrict__ sitem,
                                                     uint32_t* __restrict__ ends, uint32_t j, uint32_t one) {
    constexpr int NW = P::NW, LEN = P::LEN;
    const uint64_t pos = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= (uint64_t)count * LEN) return;
    const uint64_t gid = order[pos];             // chains in order of decreasing length
    const uint64_t m = gid / LEN;
    const uint32_t i = (uint32_t)(gid % LEN);
    const MsgInfo& info = infos[m];
    if (info.key == KEY_INVALID) return;
    const KeyBlock& kb = keys[info.key];
    const uint32_t digit = 15u - (sitem[gid] >> kRankBits);
    const uint64_t tree = layer_tree<P>(info.idx_tree, (int)j);
    const uint32_t kp = layer_leaf<P>(info.idx_tree, info.idx_leaf, (int)j);
    uint32_t ms256[8], x[NW];
#pragma unroll
    for (int w = 0; w < 8; w++) ms256[w] = kb.ms256[w];
    load_be<NW>(sigs + (size_t)m * P::SIG_BYTES + P::N + P::FORS_BYTES + (size_t)j * P::LAYER_BYTES +
                    (size_t)i * P::N, x);
    const Pipes<POL> pp(one);
    if (digit < 15u) {
        if constexpr (P::SHAKE) {
#pragma unroll 1
            for (uint32_t q = digit; q < 15u; q++)
                hashF_p<P, POL>(ms256, make_adrs(j, tree, T_WOTS_HASH, kp, i, q), x, x, pp);
        } else if constexpr (P::ROBUST) {
            ChainCtx cx;
            MaskCtx<NW> mk;
            const Adrs ah = make_adrs(j, tree, T_WOTS_HASH, kp, i, 0);
            chain_ctx<POL>(ms256, ah, cx, pp);
            mask_ctx<POL, NW>(kb.pk_seed, ah, mk, pp);
#pragma unroll 1
            for (uint32_t q = digit; q < 15u; q++) chain_step_p<P, POL>(cx, mk, ms256, q, x, x, pp);
        } else {
            ChainCtx cx;
            chain_ctx<POL>(ms256, make_adrs(j, tree, T_WOTS_HASH, kp, i, 0), cx, pp);
#pragma unroll 1
            for (uint32_t q = digit; q < 15u; q++) chain_step<POL, NW>(cx, ms256, q, x, x, pp);
        }
    }
    uint32_t* e = ends + gid * NW;
#pragma unroll
    for (int w = 0; w < NW; w++) e[w] = x[w];
}

// root_j of message m: T_len over its chain ends, h' climbs with the auth path.
template <class P>
__device__ __forceinline__ void layer_root(const KeyBlock* __restrict__ keys, const MsgInfo& info,
                                           const uint8_t* __restrict__ sigs, const uint32_t* __restrict__ ends,
                                           uint32_t m, uint32_t j, uint32_t* node, uint32_t* __restrict__ vroot) {
    constexpr int NW = P::NW, LEN = P::LEN, HP = P::HP;
    const KeyBlock& kb = keys[info.key];
    uint32_t ms256[8], msT[P::BIG ? 16 : 8];
#pragma unroll
    for (int w = 0; w < 8; w++) ms256[w] = kb.ms256[w];
#pragma unroll
    for (int w = 0; w < (P::BIG ? 16 : 8); w++) msT[w] = P::BIG ? kb.ms512[w] : kb.ms256[w];
    const uint64_t tree = layer_tree<P>(info.idx_tree, (int)j);
    const uint32_t kp = layer_leaf<P>(info.idx_tree, info.idx_leaf, (int)j);
    const uint32_t* e = ends + (size_t)m * LEN * NW;
    if constexpr (P::SHAKE) {
        TStreamP<P> ts;
        ts.init(msT, make_adrs(j, tree, T_WOTS_PK, kp, 0, 0));
#pragma unroll 1
        for (int i = 0; i < LEN; i++) ts.template push_n<NW>(e + i * NW);
        ts.template finish<NW>(LEN * P::N, node);
    } else {
        const Adrs apk = make_adrs(j, tree, T_WOTS_PK, kp, 0, 0);
        // robust: mask this message's chain ends of the layer in place (scratch, read once)
        if constexpr (P::ROBUST) mask_mem<P::BIG, NW, LEN * NW>(kb.pk_seed, apk, const_cast<uint32_t*>(e));
        tl_from_mem<P::BIG, LEN * NW, NW>(msT, apk, e, node);
    }
    const uint8_t* auth = sigs + (size_t)m * P::SIG_BYTES + P::N + P::FORS_BYTES + (size_t)j * P::LAYER_BYTES +
                          (size_t)LEN * P::N;
#pragma unroll 1
    for (int z = 0; z < HP; z++) {
        const uint32_t iz = kp >> z;
        uint32_t au[NW], lr[2 * NW];
        load_be<NW>(auth + (size_t)z * P::N, au);
#pragma unroll
        for (int w = 0; w < NW; w++) {
            lr[w] = (iz & 1) ? au[w] : node[w];
            lr[NW + w] = (iz & 1) ? node[w] : au[w];
        }
        hashH_ms<P>(ms256, msT, make_adrs(j, tree, T_TREE, 0, z + 1, iz >> 1), lr, node, kb.pk_seed);
    }
#pragma unroll
    for (int w = 0; w < NW; w++) vroot[(size_t)m * NW + w] = node[w];
}

// Layer j of message m: T_len over the chain ends, then h' climbs with the
// auth path; root_j replaces msg_j in vroot.
template <class P>
__global__ void __launch_bounds__(128) vleaf_kernel(const KeyBlock* __restrict__ keys,
                                                    const MsgInfo* __restrict__ infos, uint32_t count,
                                                    const uint8_t* __restrict__ sigs, const uint32_t* __restrict__ ends,
                                                    uint32_t* __restrict__ vroot, uint32_t j,
                                                    uint32_t* __restrict__ cnt_next, uint32_t* __restrict__ sitem) {
    constexpr int NW = P::NW;
    const uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = m < count;
    const bool valid = active && infos[m].key != KEY_INVALID;
    uint32_t node[NW];
#pragma unroll
    for (int w = 0; w < NW; w++) node[w] = 0;
    if (valid) layer_root<P>(keys, infos[m], sigs, ends, m, j, node, vroot);
    __syncwarp();
    if (cnt_next) count_steps<P>(node, active, valid, m, cnt_next, sitem);   // the next layer's chains
}

// ok[m] = 1 iff the top root equals PK.root.
template <class P>
__global__ void vfinal_kernel(const KeyBlock* __restrict__ keys, const MsgInfo* __restrict__ infos, uint32_t count,
                              const uint32_t* __restrict__ vroot, uint8_t* __restrict__ ok) {
    const uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= count) return;
    const MsgInfo& info = infos[m];
    if (info.key == KEY_INVALID) { ok[m] = 0; return; }
    const KeyBlock& kb = keys[info.key];
    uint32_t diff = 0;
#pragma unroll
    for (int w = 0; w < P::NW; w++) diff |= vroot[(size_t)m * P::NW + w] ^ kb.pk_root[w];
    ok[m] = diff == 0 ? 1 : 0;
}

}  // namespace hs
