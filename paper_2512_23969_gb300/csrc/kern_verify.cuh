// kern_verify.cuh -- batched signature verification on the GPU.
//
// The scheme's verification (the paper signs only; this is the definition's
// inverse of Fig. 2): PK_FORS from the FORS signature (leaf from the
// revealed secret, a climbs with the auth path, T_k over the roots), then
// for each layer j the WOTS+ public key from the signature of msg_j (chain i
// advanced from digit_i to w-1), T_len, and h' climbs with the auth path to
// root_j = msg_{j+1}.  Valid iff root_{d-1} equals PK.root.
//
// GB300 mapping: one warp per message.  Lanes share the k FORS trees and the
// len chains of a layer; lane 0 runs the short serial parts (T_k, T_len and
// the climbs) from a per-warp shared-memory slice.  The layers are serial
// by definition, so a warp walks them in order.
#pragma once
#include <cuda_runtime.h>
#include "hs_common.cuh"
#include "hs_launch.h"

namespace hs {

template <class P>
__global__ void __launch_bounds__(128) verify_kernel(const KeyBlock* __restrict__ keys,
                                                     const MsgInfo* __restrict__ infos, uint32_t count,
                                                     const uint8_t* __restrict__ sigs, uint8_t* __restrict__ ok) {
    constexpr int NW = P::NW, A = P::A, K = P::K, LEN = P::LEN, HP = P::HP;
    constexpr int SLOTS = (LEN > K ? LEN : K) + 1;
    __shared__ uint32_t sh[4][SLOTS * NW];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t m = blockIdx.x * 4 + warp;
    if (m >= count) return;                         // warp-uniform
    uint32_t* buf = sh[warp];
    uint32_t* bmsg = buf + (SLOTS - 1) * NW;
    const MsgInfo& info = infos[m];
    if (info.key == KEY_INVALID) {
        if (lane == 0) ok[m] = 0;
        return;
    }
    const KeyBlock& kb = keys[info.key];
    uint32_t ms256[8], msT[P::BIG ? 16 : 8];
#pragma unroll
    for (int w = 0; w < 8; w++) ms256[w] = kb.ms256[w];
#pragma unroll
    for (int w = 0; w < (P::BIG ? 16 : 8); w++) msT[w] = P::BIG ? kb.ms512[w] : kb.ms256[w];
    const uint8_t* sig = sigs + (size_t)m * P::SIG_BYTES;

    // FORS roots from the signature
    for (uint32_t i = lane; i < (uint32_t)K; i += 32) {
        const uint8_t* s = sig + P::N + (size_t)i * (A + 1) * P::N;
        const uint32_t g = (i << A) + info.fors_idx[i];
        uint32_t sk[NW], node[NW];
        load_be<NW>(s, sk);
        hashF<P, false>(ms256, make_adrs(0, info.idx_tree, T_FORS_TREE, info.idx_leaf, 0, g), sk, node);
        for (int z = 0; z < A; z++) {
            const uint32_t gz = g >> z;
            uint32_t au[NW], lr[2 * NW];
            load_be<NW>(s + (size_t)(1 + z) * P::N, au);
#pragma unroll
            for (int w = 0; w < NW; w++) {
                lr[w] = (gz & 1) ? au[w] : node[w];
                lr[NW + w] = (gz & 1) ? node[w] : au[w];
            }
            hashH_ms<P>(ms256, msT, make_adrs(0, info.idx_tree, T_FORS_TREE, info.idx_leaf, z + 1, gz >> 1), lr, node);
        }
#pragma unroll
        for (int w = 0; w < NW; w++) buf[i * NW + w] = node[w];
    }
    __syncwarp();
    if (lane == 0) {
        TStreamP<P> ts;
        ts.init(msT, make_adrs(0, info.idx_tree, T_FORS_ROOTS, info.idx_leaf, 0, 0));
        for (int i = 0; i < K; i++) ts.template push_n<NW>(buf + i * NW);
        uint32_t pkf[NW];
        ts.template finish<NW>(K * P::N, pkf);
#pragma unroll
        for (int w = 0; w < NW; w++) bmsg[w] = pkf[w];
    }
    __syncwarp();

    for (int j = 0; j < P::D; j++) {
        const uint64_t tree = layer_tree<P>(info.idx_tree, j);
        const uint32_t kp = layer_leaf<P>(info.idx_tree, info.idx_leaf, j);
        const uint8_t* ls = sig + P::N + P::FORS_BYTES + (size_t)j * P::LAYER_BYTES;
        uint32_t msg[NW];
#pragma unroll
        for (int w = 0; w < NW; w++) msg[w] = bmsg[w];
        uint32_t csum = 0;
#pragma unroll
        for (int w = 0; w < NW; w++)
#pragma unroll
            for (int b = 0; b < 8; b++) csum += 15u - ((msg[w] >> (28 - 4 * b)) & 15u);
        __syncwarp();
        for (uint32_t i = lane; i < (uint32_t)LEN; i += 32) {
            uint32_t digit;
            if (i < (uint32_t)P::LEN1) digit = (msg[i >> 3] >> (28 - 4 * (i & 7))) & 15u;
            else digit = ((csum << 4) >> (12 - 4 * (i - P::LEN1))) & 15u;
            uint32_t x[NW];
            load_be<NW>(ls + (size_t)i * P::N, x);
            Adrs a = make_adrs(j, tree, T_WOTS_HASH, kp, i, 0);
            for (uint32_t q = digit; q < 15u; q++) {
                a.half = q;
                hashF<P, false>(ms256, a, x, x);
            }
#pragma unroll
            for (int w = 0; w < NW; w++) buf[i * NW + w] = x[w];
        }
        __syncwarp();
        if (lane == 0) {
            TStreamP<P> ts;
            ts.init(msT, make_adrs(j, tree, T_WOTS_PK, kp, 0, 0));
            for (int i = 0; i < LEN; i++) ts.template push_n<NW>(buf + i * NW);
            uint32_t node[NW];
            ts.template finish<NW>(LEN * P::N, node);
            for (int z = 0; z < HP; z++) {
                const uint32_t iz = kp >> z;
                uint32_t au[NW], lr[2 * NW];
                load_be<NW>(ls + (size_t)(LEN + z) * P::N, au);
#pragma unroll
                for (int w = 0; w < NW; w++) {
                    lr[w] = (iz & 1) ? au[w] : node[w];
                    lr[NW + w] = (iz & 1) ? node[w] : au[w];
                }
                hashH_ms<P>(ms256, msT, make_adrs(j, tree, T_TREE, 0, z + 1, iz >> 1), lr, node);
            }
#pragma unroll
            for (int w = 0; w < NW; w++) bmsg[w] = node[w];
        }
        __syncwarp();
    }
    if (lane == 0) {
        uint32_t diff = 0;
#pragma unroll
        for (int w = 0; w < NW; w++) diff |= bmsg[w] ^ kb.pk_root[w];
        ok[m] = diff == 0 ? 1 : 0;
    }
}

}  // namespace hs
