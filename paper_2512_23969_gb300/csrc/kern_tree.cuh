// kern_tree.cuh -- TREE_Sign (paper Sec. III-A, III-C) and key generation.
//
// What it computes (Sec. II-A-1, II-A-3/4): for every layer j of the
// hypertree, tree t_j = idx_tree >> (j h'), all 2^h' leaves.  A leaf is the
// WOTS+ public key of keypair l: len chains, each PRF(WOTS_PRF) followed by
// w-1 = 15 applications of F(WOTS_HASH), compressed by T_len(WOTS_PK)
// (560 / 816 / 1072 SHA-256 calls per leaf).  Leaves are merged by H(TREE)
// into the tree root; the h' auth nodes of the signing leaf go to the
// signature and the root to scratch (it is what layer j+1 signs).
//
// GB300 mapping: one thread per leaf, the 2^h' leaves of a tree in an
// aligned lane group of one warp, so the Merkle levels are merged with warp
// shuffles (no shared memory, no barriers).  Each thread runs its len
// chains back to back and stores every chain end in a per-thread array
// (len * n bytes, local memory); T_len then runs over that array block by
// block, so no T_len hash state is live across the chain loop.  The PRF and
// the 15 F steps of a chain share one call site of the fully unrolled
// SHA-256 compression (all known-zero message words folded).
// All d layers of all messages form one flat grid: the layers of a
// signature are independent given the digest (paper Fig. 2).
#pragma once
#include <cuda_runtime.h>
#include "hs_common.cuh"
#include "hs_launch.h"
#include "sha256_chain.cuh"

namespace hs {

// Store n bytes of a chain checkpoint with the evict-first (streaming) hint:
// WOTS+_Sign reads them in a later kernel, long after they have left L2,
// and without the hint this 1.6 GB stream (16384 signatures at 128f)
// pushes the threads' chain-end arrays (local memory, reused by the next
// thread on the same SM slot) out of L2 and so out to DRAM.  'd' is
// 4 * NW-byte aligned (checkpoints are NW-word records from a 256-byte
// aligned base).
template <int NW>
__device__ __forceinline__ void store_checkpoint(uint32_t* d, const uint32_t* x) {
    if constexpr (NW % 4 == 0) {
#pragma unroll
        for (int w = 0; w < NW; w += 4)
            __stcs(reinterpret_cast<uint4*>(d + w), make_uint4(x[w], x[w + 1], x[w + 2], x[w + 3]));
    } else if constexpr (NW % 2 == 0) {
#pragma unroll
        for (int w = 0; w < NW; w += 2) __stcs(reinterpret_cast<uint2*>(d + w), make_uint2(x[w], x[w + 1]));
    } else {
#pragma unroll
        for (int w = 0; w < NW; w++) __stcs(d + w, x[w]);
    }
}

// Hypertree leaf = WOTS+ public key of keypair kp in tree (layer, tree).
// If chk is not null (the thread owns the signing leaf of its tree), every
// ck-th chain position (0, ck, 2ck, ...) of every chain is stored there,
// [chain][position / ck][NW words], so that WOTS+_Sign only has to finish
// at most ck - 1 steps of each chain instead of recomputing it.
// ILP = 2 (SHA-2 only): the thread runs its chains two at a time, the two
// chains' compressions interleaved (more independent work per thread, more
// registers); the last chain of an odd len runs alone.  Same bytes.
// pks: PK.seed words (the robust sets' masks; unused by the others).
template <class P, int POL, int ILP = 1>
__device__ __forceinline__ void wots_leaf(const uint32_t* ms256, const uint32_t* msT, const uint32_t* skseed,
                                          uint32_t layer, uint64_t tree, uint32_t kp, uint32_t* out,
                                          uint32_t* chk, uint32_t ck, const Pipes<POL>& pp, const uint32_t* pks) {
    constexpr int NW = P::NW;
    static_assert(ILP == 1 || (ILP == 2 && !P::SHAKE && !P::ROBUST),
                  "two chains per thread: simple SHA-2 sets only");
    // SHA-2: chain ends go to a per-thread array (local memory) and T_len
    // runs over it afterwards, so no hash state is live across the chain
    // loop; SHAKE streams them into its own buffer.
    uint32_t ends[P::SHAKE ? 1 : P::LEN * NW];
    TStreamP<P> ts;
    if constexpr (P::SHAKE) ts.init(msT, make_adrs(layer, tree, T_WOTS_PK, kp, 0, 0));
    const Adrs aprf = make_adrs(layer, tree, T_WOTS_PRF, kp, 0, 0);
    const Adrs ahash = make_adrs(layer, tree, T_WOTS_HASH, kp, 0, 0);
    // ck is a power of two (1, 2, 4 or 8 when chk is set): test and index
    // positions with a mask and a shift, not a run-time division per step
    const uint32_t per_chain = ck ? 16u >> (__ffs(ck) - 1) : 0u;
    const uint32_t ck_mask = ck ? ck - 1u : 0u, ck_shift = ck ? (uint32_t)(__ffs(ck) - 1) : 0u;
    auto keep = [&](uint32_t i, uint32_t s, const uint32_t* x) {
        if (chk != nullptr && (s & ck_mask) == 0) {
            store_checkpoint<NW>(chk + ((size_t)i * per_chain + (s >> ck_shift)) * NW, x);
        }
    };
    uint32_t i0 = 0;
    if constexpr (ILP == 2) {
#pragma unroll 1
        for (; i0 + 1 < (uint32_t)P::LEN; i0 += 2) {
            uint32_t x0[NW], x1[NW];
#pragma unroll
            for (int w = 0; w < NW; w++) x0[w] = x1[w] = skseed[w];
            ChainCtx c0, c1;
#pragma unroll 1
            for (uint32_t s = 0; s < 16; s++) {
                if (s <= 1) {
                    Adrs a = (s == 0) ? aprf : ahash;
                    a.w4 = i0 << 16;
                    chain_ctx<POL>(ms256, a, c0, pp);
                    a.w4 = (i0 + 1) << 16;
                    chain_ctx<POL>(ms256, a, c1, pp);
                }
                const uint32_t half = s == 0 ? 0u : s - 1u;
                chain_step<POL, NW>(c0, ms256, half, x0, x0, pp);
                chain_step<POL, NW>(c1, ms256, half, x1, x1, pp);
                keep(i0, s, x0);
                keep(i0 + 1, s, x1);
            }
#pragma unroll
            for (int w = 0; w < NW; w++) {
                ends[i0 * NW + w] = x0[w];
                ends[(i0 + 1) * NW + w] = x1[w];
            }
        }
    }
#pragma unroll 1
    for (uint32_t i = i0; i < (uint32_t)P::LEN; i++) {
        uint32_t x[NW];
#pragma unroll
        for (int w = 0; w < NW; w++) x[w] = skseed[w];
        ChainCtx cx;
        MaskCtx<NW> mk;                          // robust sets: the chain's F masks
        // step 0: PRF(WOTS_PRF(kp, chain i, hash 0)) = chain position 0;
        // step s >= 1: F(WOTS_HASH(kp, chain i, hash s-1)) = position s.
#pragma unroll 1
        for (uint32_t s = 0; s < 16; s++) {
            if constexpr (P::SHAKE) {
                Adrs a = (s == 0) ? aprf : ahash;
                a.w4 = i << 16;
                a.half = s == 0 ? 0u : s - 1u;
                hashF_p<P, POL>(ms256, a, x, x, pp);
            } else if constexpr (P::ROBUST) {
                if (s <= 1) {
                    Adrs a = (s == 0) ? aprf : ahash;
                    a.w4 = i << 16;
                    chain_ctx<POL>(ms256, a, cx, pp);
                    if (s == 1) mask_ctx<POL, NW>(pks, a, mk, pp);
                }
                // F steps hash x masked with their own address; PRF (s = 0) does not
                uint32_t xm[NW];
#pragma unroll
                for (int w = 0; w < NW; w++) xm[w] = x[w];
                if (s > 0) {
                    uint32_t m[NW];
                    mask_step<POL, NW>(mk, s - 1u, m, pp);
#pragma unroll
                    for (int w = 0; w < NW; w++) xm[w] ^= m[w];
                }
                chain_step<POL, NW>(cx, ms256, s == 0 ? 0u : s - 1u, xm, x, pp);
            } else {
                if (s <= 1) {
                    Adrs a = (s == 0) ? aprf : ahash;
                    a.w4 = i << 16;              // chain i (< 2^16) | hash >> 16 (= 0)
                    chain_ctx<POL>(ms256, a, cx, pp);
                }
                chain_step<POL, NW>(cx, ms256, s == 0 ? 0u : s - 1u, x, x, pp);
            }
            keep(i, s, x);
        }
        if constexpr (P::SHAKE) {
            ts.template push_n<NW>(x);
        } else {
#pragma unroll
            for (int w = 0; w < NW; w++) ends[i * NW + w] = x[w];
        }
    }
    if constexpr (P::SHAKE) {
        ts.template finish<NW>(P::LEN * P::N, out);
    } else {
        const Adrs apk = make_adrs(layer, tree, T_WOTS_PK, kp, 0, 0);
        if constexpr (P::ROBUST) mask_mem<P::BIG, NW, P::LEN * NW>(pks, apk, ends);
        tl_from_mem_p<P::BIG, P::LEN * NW, NW, POL>(msT, apk, ends, out, pp);
    }
}

// Merkle levels of one XMSS tree held by an aligned lane group (one leaf
// node per lane): H(TREE) up h' levels by shuffles, the signing leaf's auth
// nodes into the signature, root_j to scratch.
template <class P>
__device__ __forceinline__ void merkle_finish(const uint32_t* ms256, const uint32_t* msT, unsigned gmask,
                                              uint32_t m, uint32_t j, uint32_t l, uint32_t sl, uint64_t tree,
                                              uint32_t* node, uint8_t* __restrict__ sigs,
                                              uint32_t* __restrict__ roots, const uint32_t* pks) {
    constexpr int NW = P::NW, HP = P::HP;
    uint8_t* auth = sigs + (size_t)m * P::SIG_BYTES + P::N + P::FORS_BYTES + (size_t)j * P::LAYER_BYTES +
                    (size_t)P::LEN * P::N;
    if (l == (sl ^ 1u)) store_be<NW>(auth, node);
#pragma unroll
    for (int z = 1; z <= HP; z++) {
        const int step = 1 << (z - 1);
        uint32_t other[NW];
#pragma unroll
        for (int w = 0; w < NW; w++) other[w] = __shfl_xor_sync(gmask, node[w], step);
        if ((l & (2 * step - 1)) == 0) {
            uint32_t lr[2 * NW];
#pragma unroll
            for (int w = 0; w < NW; w++) { lr[w] = node[w]; lr[NW + w] = other[w]; }
            const uint32_t idx = l >> z;
            hashH_ms<P>(ms256, msT, make_adrs(j, tree, T_TREE, 0, z, idx), lr, node, pks);
            if (z < HP && idx == ((sl >> z) ^ 1u)) store_be<NW>(auth + (size_t)z * P::N, node);
        }
    }
    if (l == 0) {
        uint32_t* rt = roots + ((size_t)m * P::D + j) * NW;
#pragma unroll
        for (int w = 0; w < NW; w++) rt[w] = node[w];
    }
}


template <class P, int POL, int MINB, int ILP = 1>
__global__ void __launch_bounds__(128, MINB) tree_kernel(const KeyBlock* __restrict__ keys,
                                                   const MsgInfo* __restrict__ infos, uint32_t count,
                                                   uint8_t* __restrict__ sigs, uint32_t* __restrict__ roots,
                                                   uint32_t* __restrict__ chk, uint32_t ck, uint32_t layers,
                                                   uint32_t one) {
    constexpr int NW = P::NW, LV = P::LEAVES;
    const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t per_msg = layers * LV;           // layers 0 .. layers-1 of every message
    const uint32_t m = gid / per_msg;
    const uint32_t r = gid % per_msg;
    const uint32_t j = r / LV;                      // layer
    const uint32_t l = r % LV;                      // leaf (keypair) in the tree
    if (m >= count) return;                         // whole trees exit together
    const MsgInfo& info = infos[m];
    if (info.key == KEY_INVALID) return;
    const unsigned gmask = ((LV == 32) ? 0xFFFFFFFFu : ((1u << LV) - 1u)) << (lane & ~(uint32_t)(LV - 1));

    const KeyBlock& kb = keys[info.key];
    uint32_t ms256[8], msT[P::BIG ? 16 : 8], skseed[NW];
#pragma unroll
    for (int w = 0; w < 8; w++) ms256[w] = kb.ms256[w];
#pragma unroll
    for (int w = 0; w < (P::BIG ? 16 : 8); w++) msT[w] = P::BIG ? kb.ms512[w] : kb.ms256[w];
#pragma unroll
    for (int w = 0; w < NW; w++) skseed[w] = kb.sk_seed[w];
    uint32_t pks[P::ROBUST ? NW : 1];
#pragma unroll
    for (int w = 0; w < (P::ROBUST ? NW : 1); w++) pks[w] = P::ROBUST ? kb.pk_seed[w] : 0u;

    const uint64_t tree = layer_tree<P>(info.idx_tree, (int)j);
    const uint32_t sl = layer_leaf<P>(info.idx_tree, info.idx_leaf, (int)j);

    const Pipes<POL> pp(one);
    uint32_t* mychk = (ck != 0 && l == sl)
                          ? chk + ((size_t)m * P::D + j) * (size_t)P::LEN * (16u / ck) * NW : nullptr;
    uint32_t node[NW];
    wots_leaf<P, POL, ILP>(ms256, msT, skseed, j, tree, l, node, mychk, ck, pp, pks);

    merkle_finish<P>(ms256, msT, gmask, m, j, l, sl, tree, node, sigs, roots, pks);
}

// TREE_Sign, chain-parallel form for batches too small to fill the GPU with
// one thread per leaf: first one thread per WOTS+ chain of every leaf of
// every layer (d 2^h' len threads per message) writes its chain end to
// scratch [m][j][l][i], then one thread per leaf absorbs its len chain ends
// into T_len and the lane groups merge the Merkle levels as above.  Same
// results; ~len times more parallelism per message.
template <class P, int POL>
__global__ void __launch_bounds__(128) chains_kernel(const KeyBlock* __restrict__ keys,
                                                     const MsgInfo* __restrict__ infos, uint32_t count,
                                                     uint32_t* __restrict__ ends, uint32_t* __restrict__ chk,
                                                     uint32_t ck, uint32_t layers, uint32_t one) {
    constexpr int NW = P::NW, LV = P::LEAVES, LEN = P::LEN;
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t per_msg = layers * LV * LEN;
    const uint64_t m = gid / per_msg;
    const uint32_t r = (uint32_t)(gid % per_msg);
    const uint32_t j = r / (LV * LEN);
    const uint32_t l = (r / LEN) % LV;
    const uint32_t i = r % LEN;
    if (m >= count) return;
    const MsgInfo& info = infos[m];
    if (info.key == KEY_INVALID) return;
    const KeyBlock& kb = keys[info.key];
    uint32_t ms256[8], x[NW];
#pragma unroll
    for (int w = 0; w < 8; w++) ms256[w] = kb.ms256[w];
#pragma unroll
    for (int w = 0; w < NW; w++) x[w] = kb.sk_seed[w];
    const uint64_t tree = layer_tree<P>(info.idx_tree, (int)j);
    const uint32_t sl = layer_leaf<P>(info.idx_tree, info.idx_leaf, (int)j);
    const Pipes<POL> pp(one);
    uint32_t* mychk = nullptr;
    const uint32_t per_chain = ck ? 16u >> (__ffs(ck) - 1) : 0u;      // ck: a power of two
    const uint32_t ck_mask = ck ? ck - 1u : 0u, ck_shift = ck ? (uint32_t)(__ffs(ck) - 1) : 0u;
    if (ck != 0 && l == sl) mychk = chk + (((size_t)m * P::D + j) * (size_t)LEN + i) * per_chain * NW;
    ChainCtx cx;
    MaskCtx<NW> mk;                              // robust sets: the chain's F masks
#pragma unroll 1
    for (uint32_t s = 0; s < 16; s++) {
        if constexpr (P::SHAKE) {
            hashF_p<P, POL>(ms256, make_adrs(j, tree, s == 0 ? T_WOTS_PRF : T_WOTS_HASH, l, i, s == 0 ? 0u : s - 1u),
                            x, x, pp);
        } else if constexpr (P::ROBUST) {
            if (s <= 1) {
                Adrs a = make_adrs(j, tree, s == 0 ? T_WOTS_PRF : T_WOTS_HASH, l, i, 0);
                chain_ctx<POL>(ms256, a, cx, pp);
                if (s == 1) mask_ctx<POL, NW>(kb.pk_seed, a, mk, pp);
            }
            uint32_t xm[NW];
#pragma unroll
            for (int w = 0; w < NW; w++) xm[w] = x[w];
            if (s > 0) {
                uint32_t mm[NW];
                mask_step<POL, NW>(mk, s - 1u, mm, pp);
#pragma unroll
                for (int w = 0; w < NW; w++) xm[w] ^= mm[w];
            }
            chain_step<POL, NW>(cx, ms256, s == 0 ? 0u : s - 1u, xm, x, pp);
        } else {
            if (s <= 1) {
                Adrs a = make_adrs(j, tree, s == 0 ? T_WOTS_PRF : T_WOTS_HASH, l, i, 0);
                chain_ctx<POL>(ms256, a, cx, pp);
            }
            chain_step<POL, NW>(cx, ms256, s == 0 ? 0u : s - 1u, x, x, pp);
        }
        if (mychk != nullptr && (s & ck_mask) == 0) store_checkpoint<NW>(mychk + (s >> ck_shift) * NW, x);
    }
    uint32_t* e = ends + gid * NW;
#pragma unroll
    for (int w = 0; w < NW; w++) e[w] = x[w];
}

template <class P>
__global__ void __launch_bounds__(128) leaves_kernel(const KeyBlock* __restrict__ keys,
                                                     const MsgInfo* __restrict__ infos, uint32_t count,
                                                     const uint32_t* __restrict__ ends, uint8_t* __restrict__ sigs,
                                                     uint32_t* __restrict__ roots, uint32_t layers) {
    constexpr int NW = P::NW, LV = P::LEAVES, LEN = P::LEN;
    const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t per_msg = layers * LV;
    const uint32_t m = gid / per_msg;
    const uint32_t r = gid % per_msg;
    const uint32_t j = r / LV;
    const uint32_t l = r % LV;
    if (m >= count) return;                         // whole trees exit together
    const MsgInfo& info = infos[m];
    if (info.key == KEY_INVALID) return;
    const unsigned gmask = ((LV == 32) ? 0xFFFFFFFFu : ((1u << LV) - 1u)) << (lane & ~(uint32_t)(LV - 1));
    const KeyBlock& kb = keys[info.key];
    uint32_t ms256[8], msT[P::BIG ? 16 : 8];
#pragma unroll
    for (int w = 0; w < 8; w++) ms256[w] = kb.ms256[w];
#pragma unroll
    for (int w = 0; w < (P::BIG ? 16 : 8); w++) msT[w] = P::BIG ? kb.ms512[w] : kb.ms256[w];
    const uint64_t tree = layer_tree<P>(info.idx_tree, (int)j);
    const uint32_t sl = layer_leaf<P>(info.idx_tree, info.idx_leaf, (int)j);
    const uint32_t* e = ends + (size_t)gid * LEN * NW;
    uint32_t node[NW];
    if constexpr (P::SHAKE) {
        TStreamP<P> ts;
        ts.init(msT, make_adrs(j, tree, T_WOTS_PK, l, 0, 0));
#pragma unroll 1
        for (int i = 0; i < LEN; i++) ts.template push_n<NW>(e + i * NW);
        ts.template finish<NW>(LEN * P::N, node);
    } else {
        const Adrs apk = make_adrs(j, tree, T_WOTS_PK, l, 0, 0);
        // robust: mask this leaf's own chain ends in place (scratch, read once)
        if constexpr (P::ROBUST) mask_mem<P::BIG, NW, LEN * NW>(kb.pk_seed, apk, const_cast<uint32_t*>(e));
        tl_from_mem<P::BIG, LEN * NW, NW>(msT, apk, e, node);
    }
    merkle_finish<P>(ms256, msT, gmask, m, j, l, sl, tree, node, sigs, roots, kb.pk_seed);
}

// Key generation: PK.root = root of tree 0 of the top layer d-1.  One lane
// group per key; the midstates are derived from the seed in-thread.
template <class P>
__global__ void __launch_bounds__(128) keygen_kernel(const uint8_t* __restrict__ seeds, uint32_t count,
                                                     uint8_t* __restrict__ pk, uint8_t* __restrict__ sk,
                                                     uint32_t one) {
    constexpr int NW = P::NW, HP = P::HP, LV = P::LEAVES, N = P::N;
    const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t key = gid / LV;
    const uint32_t l = gid % LV;
    if (key >= count) return;
    const unsigned gmask = ((LV == 32) ? 0xFFFFFFFFu : ((1u << LV) - 1u)) << (lane & ~(uint32_t)(LV - 1));
    const uint8_t* sd = seeds + (size_t)key * 3 * N;
    uint32_t skseed[NW], pkseed[NW];
    load_be_unaligned<NW>(sd, skseed);
    load_be_unaligned<NW>(sd + 2 * N, pkseed);
    uint32_t ms256[8], msT[P::BIG ? 16 : 8];
    if constexpr (P::SHAKE) {         // the SHAKE hashes take PK.seed itself
#pragma unroll
        for (int i = 0; i < 8; i++) ms256[i] = (i < NW) ? pkseed[i] : 0u;
    } else {
        uint32_t W[16];
#pragma unroll
        for (int i = 0; i < 16; i++) W[i] = (i < NW) ? pkseed[i] : 0u;
        sha256_iv(ms256);
        sha256_compress_rolled(ms256, W);
    }
    if constexpr (P::BIG) {
        uint32_t blk[32];
#pragma unroll
        for (int i = 0; i < 32; i++) blk[i] = (i < NW) ? pkseed[i] : 0u;
        uint64_t s[8];
        sha512_iv(s);
        sha512_compress_w32(s, blk);
#pragma unroll
        for (int i = 0; i < 8; i++) { msT[2 * i] = (uint32_t)(s[i] >> 32); msT[2 * i + 1] = (uint32_t)s[i]; }
    } else {
#pragma unroll
        for (int i = 0; i < 8; i++) msT[i] = ms256[i];
    }
    const uint32_t top = (uint32_t)P::D - 1;
    uint32_t node[NW];
    const Pipes<kChainPol> pp(one);
    wots_leaf<P, kChainPol>(ms256, msT, skseed, top, 0ull, l, node, nullptr, 0u, pp, pkseed);
#pragma unroll
    for (int z = 1; z <= HP; z++) {
        const int step = 1 << (z - 1);
        uint32_t other[NW];
#pragma unroll
        for (int w = 0; w < NW; w++) other[w] = __shfl_xor_sync(gmask, node[w], step);
        if ((l & (2 * step - 1)) == 0) {
            uint32_t lr[2 * NW];
#pragma unroll
            for (int w = 0; w < NW; w++) { lr[w] = node[w]; lr[NW + w] = other[w]; }
            hashH_ms<P>(ms256, msT, make_adrs(top, 0ull, T_TREE, 0, z, l >> z), lr, node, pkseed);
        }
    }
    if (l == 0) {
        uint8_t* p = pk + (size_t)key * 2 * N;
        uint8_t* s = sk + (size_t)key * 4 * N;
        for (int b = 0; b < 3 * N; b++) s[b] = sd[b];
        for (int b = 0; b < N; b++) {
            const uint8_t v = (uint8_t)(node[b >> 2] >> (24 - 8 * (b & 3)));
            s[3 * N + b] = v;
            p[N + b] = v;
            p[b] = sd[2 * N + b];
        }
    }
}

}  // namespace hs
