// kern_stree.cuh -- TREE_Sign and key generation for XMSS trees wider than a
// warp (2^h' = 256 or 512 leaves: the s parameter sets).
//
// Same computation as kern_tree.cuh (paper Sec. II-A-1, II-A-3/4): every
// leaf of tree t_j at layer j is the WOTS+ public key of its keypair, the
// leaves are merged by H(TREE) into root_j, and the signing leaf's h' auth
// nodes go to the signature.  A tree no longer fits one lane group, so the
// work is two launches: the leaves (one thread per leaf, or the
// chain-parallel form followed by one thread per leaf for T_len) are
// written to scratch, then one 256-thread block per tree merges its 2^h'
// leaves level by level in shared memory (at most 512 x 32 B = 16 KB).
// The merge is a few hundred H calls against the leaves' 2^h' x 16 len
// SHA-256 calls, so its lower parallelism costs nothing measurable.
#pragma once
#include <cuda_runtime.h>
#include "hs_common.cuh"
#include "hs_launch.h"
#include "sha256_chain.cuh"
#include "kern_tree.cuh"

namespace hs {

constexpr int kMergeThreads = 256;

// Leaves of layers 0 .. layers-1 of every message: one thread per leaf.
template <class P, int POL, int MINB, int ILP = 1>
__global__ void __launch_bounds__(128, MINB) bleaf_kernel(const KeyBlock* __restrict__ keys,
                                                          const MsgInfo* __restrict__ infos, uint32_t count,
                                                          uint32_t* __restrict__ leafv, uint32_t* __restrict__ chk,
                                                          uint32_t ck, uint32_t layers, uint32_t one) {
    constexpr int NW = P::NW, LV = P::LEAVES;
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t per_msg = layers * LV;
    const uint64_t m = gid / per_msg;
    const uint32_t r = (uint32_t)(gid % per_msg);
    const uint32_t j = r / LV;
    const uint32_t l = r % LV;
    if (m >= count) return;
    const MsgInfo& info = infos[m];
    if (info.key == KEY_INVALID) return;
    const KeyBlock& kb = keys[info.key];
    uint32_t ms256[8], msT[P::BIG ? 16 : 8], skseed[NW];
#pragma unroll
    for (int w = 0; w < 8; w++) ms256[w] = kb.ms256[w];
#pragma unroll
    for (int w = 0; w < (P::BIG ? 16 : 8); w++) msT[w] = P::BIG ? kb.ms512[w] : kb.ms256[w];
#pragma unroll
    for (int w = 0; w < NW; w++) skseed[w] = kb.sk_seed[w];
    const uint64_t tree = layer_tree<P>(info.idx_tree, (int)j);
    const uint32_t sl = layer_leaf<P>(info.idx_tree, info.idx_leaf, (int)j);
    const Pipes<POL> pp(one);
    uint32_t* mychk = (ck != 0 && l == sl)
                          ? chk + ((size_t)m * P::D + j) * (size_t)P::LEN * (16u / ck) * NW : nullptr;
    uint32_t node[NW];
    wots_leaf<P, POL, ILP>(ms256, msT, skseed, j, tree, l, node, mychk, ck, pp, kb.pk_seed);
    uint32_t* out = leafv + (((size_t)m * P::D + j) * LV + l) * NW;
#pragma unroll
    for (int w = 0; w < NW; w++) out[w] = node[w];
}

// Chain-parallel form, second half: T_len over the len chain ends that
// chains_kernel wrote for each leaf.
template <class P>
__global__ void __launch_bounds__(128) bleaf_from_ends_kernel(const KeyBlock* __restrict__ keys,
                                                              const MsgInfo* __restrict__ infos, uint32_t count,
                                                              const uint32_t* __restrict__ ends,
                                                              uint32_t* __restrict__ leafv, uint32_t layers) {
    constexpr int NW = P::NW, LV = P::LEAVES, LEN = P::LEN;
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t per_msg = layers * LV;
    const uint64_t m = gid / per_msg;
    const uint32_t r = (uint32_t)(gid % per_msg);
    const uint32_t j = r / LV;
    const uint32_t l = r % LV;
    if (m >= count) return;
    const MsgInfo& info = infos[m];
    if (info.key == KEY_INVALID) return;
    const KeyBlock& kb = keys[info.key];
    const uint64_t tree = layer_tree<P>(info.idx_tree, (int)j);
    const uint32_t* e = ends + (size_t)gid * LEN * NW;
    uint32_t node[NW];
    if constexpr (P::SHAKE) {
        TStreamP<P> ts;
        ts.init(kb.ms256, make_adrs(j, tree, T_WOTS_PK, l, 0, 0));
#pragma unroll 1
        for (int i = 0; i < LEN; i++) ts.template push_n<NW>(e + i * NW);
        ts.template finish<NW>(LEN * P::N, node);
    } else {
        tl_from_mem<P::BIG, LEN * NW, NW>(P::BIG ? kb.ms512 : kb.ms256, make_adrs(j, tree, T_WOTS_PK, l, 0, 0), e,
                                          node);
    }
    uint32_t* out = leafv + (((size_t)m * P::D + j) * LV + l) * NW;
#pragma unroll
    for (int w = 0; w < NW; w++) out[w] = node[w];
}

// Merge the 2^h' nodes in sh (level 0) up to the root, left in sh[0 .. NW).
// auth (may be null): the h' auth nodes of leaf sl are stored there.  Every
// thread of the block calls it.
// heap (may be null): every node is also stored there, heap-ordered (node
// (z, i) at (2^h' >> z) + i, NW words each).
template <class P>
__device__ __forceinline__ void block_merkle(const uint32_t* ms256, const uint32_t* msT, uint32_t layer,
                                             uint64_t tree, uint32_t* sh, uint32_t sl, uint8_t* auth,
                                             uint32_t* heap = nullptr) {
    constexpr int NW = P::NW, HP = P::HP, LV = P::LEAVES;
    static_assert(LV <= 2 * kMergeThreads, "one node per thread from the first level up");
    const uint32_t t = threadIdx.x;
#pragma unroll 1
    for (int z = 1; z <= HP; z++) {
        if (auth != nullptr && t == 0) store_be<NW>(auth + (size_t)(z - 1) * P::N, sh + ((sl >> (z - 1)) ^ 1u) * NW);
        const uint32_t cnt = (uint32_t)LV >> z;
        uint32_t out[NW];
        if (t < cnt) {
            uint32_t lr[2 * NW];
#pragma unroll
            for (int w = 0; w < 2 * NW; w++) lr[w] = sh[2 * t * NW + w];
            hashH_ms<P>(ms256, msT, make_adrs(layer, tree, T_TREE, 0, z, t), lr, out);
        }
        __syncthreads();
        if (t < cnt) {
#pragma unroll
            for (int w = 0; w < NW; w++) sh[t * NW + w] = out[w];
            if (heap != nullptr) {
#pragma unroll
                for (int w = 0; w < NW; w++) heap[((size_t)(LV >> z) + t) * NW + w] = out[w];
            }
        }
        __syncthreads();
    }
}

// One block per (message, layer): auth nodes into the signature, root_j.
template <class P>
__global__ void __launch_bounds__(kMergeThreads) bmerkle_kernel(const KeyBlock* __restrict__ keys,
                                                                const MsgInfo* __restrict__ infos, uint32_t count,
                                                                const uint32_t* __restrict__ leafv,
                                                                uint8_t* __restrict__ sigs,
                                                                uint32_t* __restrict__ roots, uint32_t layers) {
    constexpr int NW = P::NW, LV = P::LEAVES;
    __shared__ uint32_t sh[LV * NW];
    const uint32_t m = blockIdx.x / layers;
    const uint32_t j = blockIdx.x % layers;
    if (m >= count) return;                         // block-uniform
    const MsgInfo& info = infos[m];
    if (info.key == KEY_INVALID) return;            // block-uniform
    const KeyBlock& kb = keys[info.key];
    uint32_t ms256[8], msT[P::BIG ? 16 : 8];
#pragma unroll
    for (int w = 0; w < 8; w++) ms256[w] = kb.ms256[w];
#pragma unroll
    for (int w = 0; w < (P::BIG ? 16 : 8); w++) msT[w] = P::BIG ? kb.ms512[w] : kb.ms256[w];
    const uint64_t tree = layer_tree<P>(info.idx_tree, (int)j);
    const uint32_t sl = layer_leaf<P>(info.idx_tree, info.idx_leaf, (int)j);
    const uint32_t* lv = leafv + ((size_t)m * P::D + j) * LV * NW;
    for (uint32_t i = threadIdx.x; i < (uint32_t)(LV * NW); i += blockDim.x) sh[i] = lv[i];
    __syncthreads();
    uint8_t* auth = sigs + (size_t)m * P::SIG_BYTES + P::N + P::FORS_BYTES + (size_t)j * P::LAYER_BYTES +
                    (size_t)P::LEN * P::N;
    block_merkle<P>(ms256, msT, j, tree, sh, sl, auth);
    if (threadIdx.x == 0) {
        uint32_t* rt = roots + ((size_t)m * P::D + j) * NW;
#pragma unroll
        for (int w = 0; w < NW; w++) rt[w] = sh[w];
    }
}

// ---------------------------------------------------------------- shared / cached trees
// Distinct trees (tree sharing within a batch, keyset caches) for wide
// trees: one thread per (tree, leaf) for the leaves, with the chain
// checkpoints of every leaf, stored heap-ordered; then one block per tree
// for the internal nodes.  nuniq (may be null) bounds the live trees.
template <class P, int POL>
__global__ void __launch_bounds__(128) wtree_leaf_kernel(const KeyBlock* __restrict__ keys,
                                                         const DedupDesc* __restrict__ desc,
                                                         const uint32_t* __restrict__ nuniq, uint32_t max_uniq,
                                                         uint32_t* __restrict__ nodes, uint32_t* __restrict__ chk_u,
                                                         uint32_t ck, uint32_t one) {
    constexpr int NW = P::NW, LV = P::LEAVES;
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t id = gid / LV;
    const uint32_t l = (uint32_t)(gid % LV);
    if (id >= max_uniq || (nuniq && id >= *nuniq)) return;
    const DedupDesc d = desc[id];
    const KeyBlock& kb = keys[d.key];
    uint32_t ms256[8], msT[P::BIG ? 16 : 8], skseed[NW];
#pragma unroll
    for (int w = 0; w < 8; w++) ms256[w] = kb.ms256[w];
#pragma unroll
    for (int w = 0; w < (P::BIG ? 16 : 8); w++) msT[w] = P::BIG ? kb.ms512[w] : kb.ms256[w];
#pragma unroll
    for (int w = 0; w < NW; w++) skseed[w] = kb.sk_seed[w];
    const Pipes<POL> pp(one);
    uint32_t* mychk = ck ? chk_u + ((size_t)id * LV + l) * (size_t)P::LEN * (16u / ck) * NW : nullptr;
    uint32_t node[NW];
    wots_leaf<P, POL>(ms256, msT, skseed, d.layer, d.tree, l, node, mychk, ck, pp, kb.pk_seed);
    uint32_t* tn = nodes + (size_t)id * 2 * LV * NW;
#pragma unroll
    for (int w = 0; w < NW; w++) tn[((size_t)LV + l) * NW + w] = node[w];
}

template <class P>
__global__ void __launch_bounds__(kMergeThreads) wtree_merge_kernel(const KeyBlock* __restrict__ keys,
                                                                    const DedupDesc* __restrict__ desc,
                                                                    const uint32_t* __restrict__ nuniq,
                                                                    uint32_t max_uniq, uint32_t* __restrict__ nodes) {
    constexpr int NW = P::NW, LV = P::LEAVES;
    __shared__ uint32_t sh[LV * NW];
    const uint32_t id = blockIdx.x;
    if (id >= max_uniq || (nuniq && id >= *nuniq)) return;      // block-uniform
    const DedupDesc d = desc[id];
    const KeyBlock& kb = keys[d.key];
    uint32_t ms256[8], msT[P::BIG ? 16 : 8];
#pragma unroll
    for (int w = 0; w < 8; w++) ms256[w] = kb.ms256[w];
#pragma unroll
    for (int w = 0; w < (P::BIG ? 16 : 8); w++) msT[w] = P::BIG ? kb.ms512[w] : kb.ms256[w];
    uint32_t* tn = nodes + (size_t)id * 2 * LV * NW;
    for (uint32_t i = threadIdx.x; i < (uint32_t)(LV * NW); i += blockDim.x) sh[i] = tn[LV * NW + i];
    __syncthreads();
    block_merkle<P>(ms256, msT, d.layer, d.tree, sh, 0u, nullptr, tn);
}

// ---------------------------------------------------------------- keygen
// Key blocks straight from the 3n-byte seeds (SK.seed || SK.prf || PK.seed).
template <class P>
__global__ void seed_keys_kernel(const uint8_t* __restrict__ seeds, uint32_t count, KeyBlock* __restrict__ out) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    constexpr int NW = P::NW;
    KeyBlock kb;
    for (int i = 0; i < 64; i++) reinterpret_cast<uint32_t*>(&kb)[i] = 0;
    const uint8_t* sd = seeds + (size_t)k * 3 * P::N;
    load_be_unaligned<NW>(sd, kb.sk_seed);
    load_be_unaligned<NW>(sd + P::N, kb.sk_prf);
    load_be_unaligned<NW>(sd + 2 * P::N, kb.pk_seed);
    if constexpr (P::SHAKE) {         // the SHAKE hashes take PK.seed itself
        for (int i = 0; i < 8; i++) kb.ms256[i] = (i < NW) ? kb.pk_seed[i] : 0u;
    } else {
        uint32_t W[16];
        for (int i = 0; i < 16; i++) W[i] = (i < NW) ? kb.pk_seed[i] : 0u;
        sha256_iv(kb.ms256);
        sha256_compress_rolled(kb.ms256, W);
    }
    if constexpr (P::BIG) {
        uint32_t blk[32];
        for (int i = 0; i < 32; i++) blk[i] = (i < NW) ? kb.pk_seed[i] : 0u;
        uint64_t s[8];
        sha512_iv(s);
        sha512_compress_w32(s, blk);
        for (int i = 0; i < 8; i++) { kb.ms512[2 * i] = (uint32_t)(s[i] >> 32); kb.ms512[2 * i + 1] = (uint32_t)s[i]; }
    }
    out[k] = kb;
}

// Leaves of the top tree (layer d-1, tree 0) of every key.
template <class P, int POL>
__global__ void __launch_bounds__(128) bkeygen_leaf_kernel(const KeyBlock* __restrict__ kbs, uint32_t count,
                                                           uint32_t* __restrict__ leafv, uint32_t one) {
    constexpr int NW = P::NW, LV = P::LEAVES;
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t key = gid / LV;
    const uint32_t l = (uint32_t)(gid % LV);
    if (key >= count) return;
    const KeyBlock& kb = kbs[key];
    uint32_t ms256[8], msT[P::BIG ? 16 : 8], skseed[NW];
#pragma unroll
    for (int w = 0; w < 8; w++) ms256[w] = kb.ms256[w];
#pragma unroll
    for (int w = 0; w < (P::BIG ? 16 : 8); w++) msT[w] = P::BIG ? kb.ms512[w] : kb.ms256[w];
#pragma unroll
    for (int w = 0; w < NW; w++) skseed[w] = kb.sk_seed[w];
    const Pipes<POL> pp(one);
    uint32_t node[NW];
    wots_leaf<P, POL>(ms256, msT, skseed, (uint32_t)P::D - 1, 0ull, l, node, nullptr, 0u, pp, kb.pk_seed);
#pragma unroll
    for (int w = 0; w < NW; w++) leafv[((size_t)key * LV + l) * NW + w] = node[w];
}

// One block per key: PK.root, then pk = PK.seed || PK.root and
// sk = SK.seed || SK.prf || PK.seed || PK.root.
template <class P>
__global__ void __launch_bounds__(kMergeThreads) bkeygen_root_kernel(const KeyBlock* __restrict__ kbs,
                                                                     const uint8_t* __restrict__ seeds,
                                                                     uint32_t count,
                                                                     const uint32_t* __restrict__ leafv,
                                                                     uint8_t* __restrict__ pk,
                                                                     uint8_t* __restrict__ sk) {
    constexpr int NW = P::NW, LV = P::LEAVES, N = P::N;
    __shared__ uint32_t sh[LV * NW];
    const uint32_t key = blockIdx.x;
    if (key >= count) return;
    const KeyBlock& kb = kbs[key];
    uint32_t ms256[8], msT[P::BIG ? 16 : 8];
#pragma unroll
    for (int w = 0; w < 8; w++) ms256[w] = kb.ms256[w];
#pragma unroll
    for (int w = 0; w < (P::BIG ? 16 : 8); w++) msT[w] = P::BIG ? kb.ms512[w] : kb.ms256[w];
    const uint32_t* lv = leafv + (size_t)key * LV * NW;
    for (uint32_t i = threadIdx.x; i < (uint32_t)(LV * NW); i += blockDim.x) sh[i] = lv[i];
    __syncthreads();
    block_merkle<P>(ms256, msT, (uint32_t)P::D - 1, 0ull, sh, 0u, nullptr);
    if (threadIdx.x == 0) {
        const uint8_t* sd = seeds + (size_t)key * 3 * N;
        uint8_t* p = pk + (size_t)key * 2 * N;
        uint8_t* s = sk + (size_t)key * 4 * N;
        for (int b = 0; b < 3 * N; b++) s[b] = sd[b];
        for (int b = 0; b < N; b++) {
            const uint8_t v = (uint8_t)(sh[b >> 2] >> (24 - 8 * (b & 3)));
            s[3 * N + b] = v;
            p[N + b] = v;
            p[b] = sd[2 * N + b];
        }
    }
}

}  // namespace hs
