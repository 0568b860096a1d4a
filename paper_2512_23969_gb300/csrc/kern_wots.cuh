// kern_wots.cuh -- WOTS+_Sign (paper Sec. III, after FORS_Sign and TREE_Sign).
//
// What it computes (Sec. II-A-1): layer j signs the n-byte value
// msg_j = PK_FORS (j = 0) or root_{j-1} (j >= 1).  Its base-16 digits (high
// nibble first) are followed by the 3 digits of the checksum
// sum(15 - d_i) << 4; chain i of the signing keypair is advanced from its
// secret PRF(WOTS_PRF) by digit_i applications of F(WOTS_HASH).
//
// GB300 mapping: one thread per (message, layer, chain); each thread
// recomputes the checksum from msg_j (2n nibble reads, negligible next to
// its chain) so no cross-thread exchange is needed.  TREE_Sign already ran
// every chain of the signing keypair to its end; when it stored every
// ck-th chain position (ck = 1, 2 or 4), a chain's signature value is the
// stored position floor(d / ck) ck advanced by d mod ck < ck steps, instead
// of PRF plus d steps (the same value: chain composition).
#pragma once
#include <cuda_runtime.h>
#include "hs_common.cuh"
#include "hs_launch.h"
#include "sha256_chain.cuh"

namespace hs {

template <class P, int POL>
__global__ void __launch_bounds__(256) wots_kernel(const KeyBlock* __restrict__ keys,
                                                   const MsgInfo* __restrict__ infos, uint32_t count,
                                                   const uint32_t* __restrict__ pk_fors,
                                                   const uint32_t* __restrict__ roots, uint8_t* __restrict__ sigs,
                                                   const uint32_t* __restrict__ chk, uint32_t ck, uint32_t L,
                                                   const uint32_t* __restrict__ mj_id,
                                                   const uint32_t* __restrict__ chk_u, uint32_t one) {
    constexpr int NW = P::NW, LEN = P::LEN;
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t per_msg = (uint32_t)P::D * LEN;
    const uint64_t m = gid / per_msg;
    const uint32_t r = (uint32_t)(gid % per_msg);
    const uint32_t j = r / LEN;
    const uint32_t i = r % LEN;
    if (m >= count) return;
    const MsgInfo& info = infos[m];
    if (info.key == KEY_INVALID) return;
    const KeyBlock& kb = keys[info.key];

    const uint32_t* mj = (j == 0) ? pk_fors + m * NW : roots + (m * P::D + (j - 1)) * NW;
    uint32_t msg[NW];
#pragma unroll
    for (int w = 0; w < NW; w++) msg[w] = mj[w];
    uint32_t csum = 0;
#pragma unroll
    for (int w = 0; w < NW; w++)
#pragma unroll
        for (int b = 0; b < 8; b++) csum += 15u - ((msg[w] >> (28 - 4 * b)) & 15u);
    uint32_t digit;
    if (i < (uint32_t)P::LEN1) {
        digit = (msg[i >> 3] >> (28 - 4 * (i & 7))) & 15u;
    } else {
        const uint32_t c = csum << 4;                 // (8 - (len2 * 4) % 8) % 8 = 4
        digit = (c >> (12 - 4 * (i - P::LEN1))) & 15u;
    }

    const uint64_t tree = layer_tree<P>(info.idx_tree, (int)j);
    const uint32_t kp = layer_leaf<P>(info.idx_tree, info.idx_leaf, (int)j);
    uint32_t ms256[8];
#pragma unroll
    for (int w = 0; w < 8; w++) ms256[w] = kb.ms256[w];
    const Pipes<POL> pp(one);
    uint32_t x[NW];
    if (ck != 0) {
        const uint32_t per_chain = 16u / ck;
        const uint32_t base = (digit / ck) * ck;
        // checkpoints of the message's own tree, or of the shared tree of
        // its (key, layer, tree) when layer j is shared within the batch
        const uint32_t* c =
            (j >= L) ? chk_u + ((((size_t)mj_id[m * (P::D - L) + (j - L)] * P::LEAVES + kp) * LEN + i) * per_chain +
                                digit / ck) * NW
                     : chk + (((m * P::D + j) * (size_t)LEN + i) * per_chain + digit / ck) * NW;
#pragma unroll
        for (int w = 0; w < NW; w++) x[w] = c[w];
        Adrs a = make_adrs(j, tree, T_WOTS_HASH, kp, i, 0);
#pragma unroll 1
        for (uint32_t q = base; q < digit; q++) {
            a.half = q;
            hashF_p<P, POL>(ms256, a, x, x, pp, kb.pk_seed);
        }
    } else {
#pragma unroll
        for (int w = 0; w < NW; w++) x[w] = kb.sk_seed[w];
        if constexpr (P::SHAKE) {
            hashF_p<P, POL>(ms256, make_adrs(j, tree, T_WOTS_PRF, kp, i, 0), x, x, pp);
#pragma unroll 1
            for (uint32_t q = 0; q < digit; q++) hashF_p<P, POL>(ms256, make_adrs(j, tree, T_WOTS_HASH, kp, i, q), x, x, pp);
        } else if constexpr (P::ROBUST) {
        ChainCtx cx;
        MaskCtx<NW> mk;
        chain_ctx<POL>(ms256, make_adrs(j, tree, T_WOTS_PRF, kp, i, 0), cx, pp);
        chain_step<POL, NW>(cx, ms256, 0u, x, x, pp);           // PRF: not masked
        if (digit > 0) {
            const Adrs ah = make_adrs(j, tree, T_WOTS_HASH, kp, i, 0);
            chain_ctx<POL>(ms256, ah, cx, pp);
            mask_ctx<POL, NW>(kb.pk_seed, ah, mk, pp);
        }
#pragma unroll 1
        for (uint32_t q = 0; q < digit; q++) chain_step_p<P, POL>(cx, mk, ms256, q, x, x, pp);
        } else {
        ChainCtx cx;
        chain_ctx<POL>(ms256, make_adrs(j, tree, T_WOTS_PRF, kp, i, 0), cx, pp);
        chain_step<POL, NW>(cx, ms256, 0u, x, x, pp);
        if (digit > 0) chain_ctx<POL>(ms256, make_adrs(j, tree, T_WOTS_HASH, kp, i, 0), cx, pp);
#pragma unroll 1
        for (uint32_t q = 0; q < digit; q++) chain_step<POL, NW>(cx, ms256, q, x, x, pp);
        }
    }
    store_be<NW>(sigs + m * P::SIG_BYTES + P::N + P::FORS_BYTES + (size_t)j * P::LAYER_BYTES + (size_t)i * P::N, x);
}

}  // namespace hs
