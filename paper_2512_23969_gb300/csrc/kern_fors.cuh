// kern_fors.cuh -- FORS_Sign (paper Sec. III-B) and the FORS public key.
//
// What it computes (Sec. II-A-2): for each of the k trees of height a, the
// leaves F(FORS_TREE(0, g), PRF(FORS_PRF(g))) with g = i 2^a + j, the
// Merkle root by H up a levels, the secret of the selected leaf idx_i and
// its a auth nodes.  PK_FORS = T_k(FORS_ROOTS, root_0 .. root_{k-1}).
//
// GB300 mapping (ours, not the paper's Tree Fusion): a tree is owned by an
// aligned group of LPT lanes of one warp.  Each lane builds a subtree of
// height R = a - log2(LPT) over 2^R consecutive leaves with a register
// treehash (one H call site, left siblings in a small stack, SibStack),
// then the top log2(LPT) levels are merged across the group with
// warp shuffles.  Lane subtrees taller than 7 levels (a = 12-14 of the s
// sets) are built as 2^(R-7) consecutive height-7 subtrees whose roots are
// merged through a second stack of at most 3 nodes.  No shared memory and no block barriers; the grid is flat
// over (message, tree, lane), so every message's k trees run in parallel.
#pragma once
#include <cuda_runtime.h>
#include "hs_common.cuh"
#include "hs_launch.h"
#include "sha256_chain.cuh"

namespace hs {

template <int L> struct Log2 { static constexpr int v = 1 + Log2<L / 2>::v; };
template <> struct Log2<1> { static constexpr int v = 0; };

// Left siblings of a lane's treehash: levels 0..RI-1 (inner subtrees) and
// RI..R-1 (outer merges).  LOCAL: one per-thread array at run-time indices
// (local memory) -- no registers, no select chains; measured faster for
// lane subtrees of up to 7 levels.  Otherwise registers read through
// select chains (faster for the 9-10 level subtrees of the s sets).
template <int R, int RI, int NW, bool LOCAL>
struct SibStack;

template <int R, int RI, int NW>
struct SibStack<R, RI, NW, true> {
    uint32_t v[R * NW];
    __device__ __forceinline__ void load(uint32_t z, uint32_t* o) const {
#pragma unroll
        for (int w = 0; w < NW; w++) o[w] = v[z * NW + w];
    }
    __device__ __forceinline__ void store(uint32_t z, const uint32_t* x) {
#pragma unroll
        for (int w = 0; w < NW; w++) v[z * NW + w] = x[w];
    }
    __device__ __forceinline__ void load_outer(uint32_t z, uint32_t* o) const { load(z, o); }
    __device__ __forceinline__ void store_outer(uint32_t z, const uint32_t* x) { store(z, x); }
};

template <int R, int RI, int NW>
struct SibStack<R, RI, NW, false> {
    static constexpr int RO = R - RI;
    uint32_t in[RI][NW];
    uint32_t out[RO > 0 ? RO : 1][NW];
    __device__ __forceinline__ void load(uint32_t z, uint32_t* o) const {
#pragma unroll
        for (int w = 0; w < NW; w++) {
            uint32_t v = in[0][w];
#pragma unroll
            for (int zz = 1; zz < RI; zz++) v = (z == (uint32_t)zz) ? in[zz][w] : v;
            o[w] = v;
        }
    }
    __device__ __forceinline__ void store(uint32_t z, const uint32_t* x) {
#pragma unroll
        for (int zz = 0; zz < RI; zz++)
            if (z == (uint32_t)zz) {
#pragma unroll
                for (int w = 0; w < NW; w++) in[zz][w] = x[w];
            }
    }
    __device__ __forceinline__ void load_outer(uint32_t z, uint32_t* o) const {
#pragma unroll
        for (int w = 0; w < NW; w++) {
            uint32_t v = out[0][w];
#pragma unroll
            for (int zz = 1; zz < RO; zz++) v = (z - RI == (uint32_t)zz) ? out[zz][w] : v;
            o[w] = v;
        }
    }
    __device__ __forceinline__ void store_outer(uint32_t z, const uint32_t* x) {
#pragma unroll
        for (int zz = 0; zz < RO; zz++)
            if (z - RI == (uint32_t)zz) {
#pragma unroll
                for (int w = 0; w < NW; w++) out[zz][w] = x[w];
            }
    }
};

template <class P, int POL, int LPT>
__global__ void __launch_bounds__(256) fors_kernel(const KeyBlock* __restrict__ keys,
                                                   const MsgInfo* __restrict__ infos, uint32_t count,
                                                   uint8_t* __restrict__ sigs, uint32_t* __restrict__ fors_roots,
                                                   uint32_t one) {
    constexpr int NW = P::NW, A = P::A, K = P::K;
    constexpr int R = A - Log2<LPT>::v;           // height built inside one lane
    constexpr int RI = R < 7 ? R : 7;             // inner treehash height
    constexpr int RO = R - RI;                    // levels merged by the outer stack
    static_assert(R >= 1 && RO <= 3, "lane subtree height");
    const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t L = gid % LPT;                  // lane within the tree group
    const uint32_t grp = gid / LPT;                // (message, tree)
    const uint32_t m = grp / K;
    const uint32_t i = grp % K;
    if (m >= count) return;                        // whole groups exit together
    const MsgInfo& info = infos[m];
    if (info.key == KEY_INVALID) return;
    const unsigned gmask = (LPT == 32) ? 0xFFFFFFFFu : (((1u << LPT) - 1u) << (lane & ~(uint32_t)(LPT - 1)));

    const KeyBlock& kb = keys[info.key];
    uint32_t ms256[8], ms512[P::BIG ? 16 : 1], skseed[NW];
#pragma unroll
    for (int w = 0; w < 8; w++) ms256[w] = kb.ms256[w];
    if constexpr (P::BIG) {
#pragma unroll
        for (int w = 0; w < 16; w++) ms512[w] = kb.ms512[w];
    }
#pragma unroll
    for (int w = 0; w < NW; w++) skseed[w] = kb.sk_seed[w];

    const uint64_t tree = info.idx_tree;
    const uint32_t kp = info.idx_leaf;
    const uint32_t gs = info.fors_idx[i];          // selected leaf in tree i
    uint8_t* sf = sigs + (size_t)m * P::SIG_BYTES + P::N + (size_t)i * (A + 1) * P::N;

    const Pipes<POL> pp(one);
    // Leaf hashes with a chain context: PRF and F of every leaf of this
    // message share address words 0..4 (layer, tree, type, key pair, height
    // 0 and the top half of the leaf index, which is 0 while k * 2^a <=
    // 2^16), so rounds 0..4 of each (and round 5 up to its message word)
    // are computed once here and a leaf hash runs rounds 6..63 -- the same
    // compression as the chain steps of TREE_Sign, bit for bit.  The two
    // contexts are read at a run-time
    // index (local memory): 60 registers instead of 79 for a register
    // select, and as fast or faster (FORS 128f 6.39 -> 6.19 ms, 256f 45.2
    // -> 43.6 ms per 16384 / 8192 signatures).
    constexpr bool kCtx = !P::SHAKE && ((uint64_t)K << A) <= 65536u;
    ChainCtx cxs[kCtx ? 2 : 1];
    MaskCtx<NW> mk;                                // robust sets: the leaf F masks
    if constexpr (kCtx) {
        chain_ctx<POL>(ms256, make_adrs(0, tree, T_FORS_PRF, kp, 0, 0), cxs[0], pp);
        chain_ctx<POL>(ms256, make_adrs(0, tree, T_FORS_TREE, kp, 0, 0), cxs[1], pp);
        if constexpr (P::ROBUST) mask_ctx<POL, NW>(kb.pk_seed, make_adrs(0, tree, T_FORS_TREE, kp, 0, 0), mk, pp);
    }
    SibStack<R, RI, NW, (R <= 7)> stk;                 // left siblings, levels 0..R-1
    uint32_t node[NW];
    const uint32_t base = L << R;                  // first leaf of this lane (within tree)
#pragma unroll 1
    for (uint32_t ob = 0; ob < (1u << RO); ob++) {
#pragma unroll 1
        for (uint32_t p = 0; p < (1u << RI); p++) {
            const uint32_t t = base + (ob << RI) + p;  // leaf index within tree
            const uint32_t g = (i << A) + t;           // global leaf index
            // leaf g: sk = PRF(FORS_PRF(g)), then F(FORS_TREE(height 0, g), sk);
            // both through one call site of the compression
#pragma unroll
            for (int w = 0; w < NW; w++) node[w] = skseed[w];
#pragma unroll 1
            for (int s = 0; s < 2; s++) {
                if constexpr (kCtx && P::ROBUST) {
                    // the leaf F (s = 1) hashes sk masked with its own address; PRF does not
                    uint32_t xm[NW];
#pragma unroll
                    for (int w = 0; w < NW; w++) xm[w] = node[w];
                    if (s == 1) {
                        uint32_t m[NW];
                        mask_step<POL, NW>(mk, g, m, pp);
#pragma unroll
                        for (int w = 0; w < NW; w++) xm[w] ^= m[w];
                    }
                    chain_step<POL, NW>(cxs[s], ms256, g, xm, node, pp);
                } else if constexpr (kCtx) {
                    chain_step<POL, NW>(cxs[s], ms256, g, node, node, pp);
                } else {
                    hashF_p<P, POL>(ms256, make_adrs(0, tree, s == 0 ? T_FORS_PRF : T_FORS_TREE, kp, 0, g), node,
                                    node, pp, s == 0 ? nullptr : kb.pk_seed);
                }
                if (s == 0 && t == gs) store_be<NW>(sf, node);
            }
            if (t == (gs ^ 1u)) store_be<NW>(sf + P::N, node);
            // merge with stacked left siblings while this node is a right child
            uint32_t z = 0, idx = t;
#pragma unroll 1
            while ((idx & 1u) && z < (uint32_t)RI) {
                uint32_t lr[2 * NW];
                stk.load(z, lr);
#pragma unroll
                for (int w = 0; w < NW; w++) lr[NW + w] = node[w];
                z++;
                idx >>= 1;
                hashH_p<P, POL>(ms256, ms512,
                                make_adrs(0, tree, T_FORS_TREE, kp, z, (i << (A - z)) + idx), lr, node, pp, kb.pk_seed);
                if (z < (uint32_t)A && idx == ((gs >> z) ^ 1u)) store_be<NW>(sf + (size_t)(1 + z) * P::N, node);
            }
            if (z < (uint32_t)RI) stk.store(z, node);
        }
        if constexpr (RO > 0) {
            // node = root of inner subtree ob (level RI); merge with the outer stack
            uint32_t z = RI, idx = (base >> RI) + ob;
#pragma unroll 1
            while ((idx & 1u) && z < (uint32_t)R) {
                uint32_t lr[2 * NW];
                stk.load_outer(z, lr);
#pragma unroll
                for (int w = 0; w < NW; w++) lr[NW + w] = node[w];
                z++;
                idx >>= 1;
                hashH_p<P, POL>(ms256, ms512,
                                make_adrs(0, tree, T_FORS_TREE, kp, z, (i << (A - z)) + idx), lr, node, pp, kb.pk_seed);
                if (z < (uint32_t)A && idx == ((gs >> z) ^ 1u)) store_be<NW>(sf + (size_t)(1 + z) * P::N, node);
            }
            if (z < (uint32_t)R) stk.store_outer(z, node);
        }
    }
    // node = lane subtree root, level R, index L within the tree
#pragma unroll
    for (int z = R + 1; z <= A; z++) {
        const int step = 1 << (z - R - 1);
        uint32_t other[NW];
#pragma unroll
        for (int w = 0; w < NW; w++) other[w] = __shfl_xor_sync(gmask, node[w], step);
        if ((L & (2 * step - 1)) == 0) {
            uint32_t lr[2 * NW];
#pragma unroll
            for (int w = 0; w < NW; w++) { lr[w] = node[w]; lr[NW + w] = other[w]; }
            const uint32_t idx = L >> (z - R);
            hashH_p<P, POL>(ms256, ms512, make_adrs(0, tree, T_FORS_TREE, kp, z, (i << (A - z)) + idx), lr, node, pp, kb.pk_seed);
            if (z < A && idx == ((gs >> z) ^ 1u)) store_be<NW>(sf + (size_t)(1 + z) * P::N, node);
        }
    }
    if (L == 0) {
        uint32_t* r = fors_roots + ((size_t)m * K + i) * NW;
#pragma unroll
        for (int w = 0; w < NW; w++) r[w] = node[w];
    }
}

// PK_FORS = T_k(FORS_ROOTS(layer 0, idx_tree, keypair idx_leaf), roots).
template <class P>
__global__ void fors_pk_kernel(const KeyBlock* __restrict__ keys, const MsgInfo* __restrict__ infos,
                               uint32_t count, const uint32_t* __restrict__ fors_roots,
                               uint32_t* __restrict__ pk_fors) {
    const uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= count) return;
    const MsgInfo& info = infos[m];
    if (info.key == KEY_INVALID) return;
    const KeyBlock& kb = keys[info.key];
    constexpr int NW = P::NW;
    const uint32_t* r = fors_roots + (size_t)m * P::K * NW;
    const Adrs a = make_adrs(0, info.idx_tree, T_FORS_ROOTS, info.idx_leaf, 0, 0);
    uint32_t out[NW];
    if constexpr (P::SHAKE) {
        TStreamP<P> ts;
        ts.init(kb.ms256, a);
        for (int i = 0; i < P::K; i++) ts.template push_n<NW>(r + i * NW);
        ts.template finish<NW>(P::K * P::N, out);
    } else {
        // robust: mask this message's roots in place (scratch, read once)
        if constexpr (P::ROBUST) mask_mem<P::BIG, NW, P::K * NW>(kb.pk_seed, a, const_cast<uint32_t*>(r));
        tl_from_mem<P::BIG, P::K * NW, NW>(P::BIG ? kb.ms512 : kb.ms256, a, r, out);
    }
#pragma unroll
    for (int w = 0; w < NW; w++) pk_fors[(size_t)m * NW + w] = out[w];
}

}  // namespace hs
