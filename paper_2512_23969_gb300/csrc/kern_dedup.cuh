// kern_dedup.cuh -- bit-exact sharing of XMSS trees within a batch.
//
// The tree of layer j that message m signs with is fixed by (key, j,
// t_j = idx_tree >> (j h')) alone (paper Fig. 2: every layer's tree and leaf
// come from the digest).  In a batch where many messages share a key, the
// upper layers repeat the same trees -- e.g. the top layer is tree 0 for all
// of them.  For the layers the host marks shareable (j >= L), the batch's
// (key, j, t_j) triples are entered into a device hash table, each distinct
// tree is built once with all its Merkle nodes and, when chain checkpoints
// are on, the checkpoints of every one of its leaves; each message then
// copies its own auth path and root from its tree.  Every signature byte is
// the same as without sharing; only repeated work is skipped.
#pragma once
#include <cuda_runtime.h>
#include "hs_common.cuh"
#include "hs_launch.h"
#include "sha256_chain.cuh"
#include "kern_tree.cuh"

namespace hs {

constexpr uint32_t kNoSlot = 0xFFFFFFFFu;

// Packed table key: key index (32 bits) | layer (5 bits) | tree (27 bits), +1
// so that 0 marks an empty slot.  The host only shares layers whose trees
// have at most 27 bits.
__device__ __forceinline__ uint64_t dedup_key(uint32_t key, uint32_t j, uint64_t tree) {
    return (((uint64_t)key << 32) | ((uint64_t)j << 27) | tree) + 1ull;
}

// One thread per (message, shared layer): find or insert its triple.
template <class P>
__global__ void dedup_insert_kernel(const MsgInfo* __restrict__ infos, uint32_t count, uint32_t L,
                                    unsigned long long* __restrict__ table, uint32_t cap_log2,
                                    uint32_t* __restrict__ mj_slot, uint32_t* __restrict__ status) {
    const uint32_t per_msg = (uint32_t)P::D - L;
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (uint64_t)count * per_msg) return;
    const uint32_t m = (uint32_t)(gid / per_msg);
    const uint32_t j = L + (uint32_t)(gid % per_msg);
    const MsgInfo& info = infos[m];
    if (info.key == KEY_INVALID) { mj_slot[gid] = kNoSlot; return; }
    const uint64_t key = dedup_key(info.key, j, layer_tree<P>(info.idx_tree, (int)j));
    const uint32_t cap = 1u << cap_log2;
    uint32_t h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> (64 - cap_log2));
    for (uint32_t probe = 0; probe < cap; probe++) {     // the table is at most half full
        const unsigned long long prev = atomicCAS(&table[h], 0ull, (unsigned long long)key);
        if (prev == 0ull || prev == key) { mj_slot[gid] = h; return; }
        h = (h + 1) & (cap - 1);
    }
    mj_slot[gid] = kNoSlot;
    atomicOr(status, 1u << HS_ECUDA);
}

// One thread per table slot: occupied slots get dense tree ids.
static __global__ void dedup_compact_kernel(const unsigned long long* __restrict__ table, uint32_t cap,
                                            uint32_t* __restrict__ slot_id, DedupDesc* __restrict__ desc,
                                            uint32_t* __restrict__ nuniq, uint32_t max_uniq,
                                            uint32_t* __restrict__ status) {
    const uint32_t slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= cap) return;
    const unsigned long long k = table[slot];
    if (k == 0ull) return;
    const uint32_t id = atomicAdd(nuniq, 1u);
    if (id >= max_uniq) {               // cannot happen: max_uniq bounds the distinct trees
        slot_id[slot] = 0;
        atomicOr(status, 1u << HS_ECUDA);
        return;
    }
    slot_id[slot] = id;
    const uint64_t v = (uint64_t)k - 1ull;
    DedupDesc d;
    d.tree = v & ((1ull << 27) - 1ull);
    d.layer = (uint32_t)(v >> 27) & 31u;
    d.key = (uint32_t)(v >> 32);
    desc[id] = d;
}

// One lane group per distinct tree: every leaf (with all its checkpoints)
// and every Merkle node, stored heap-ordered (node (z, i) at (2^h' >> z) + i;
// root at 1).
template <class P, int POL>
__global__ void __launch_bounds__(128) utree_kernel(const KeyBlock* __restrict__ keys,
                                                    const DedupDesc* __restrict__ desc,
                                                    const uint32_t* __restrict__ nuniq, uint32_t max_uniq,
                                                    uint32_t* __restrict__ nodes, uint32_t* __restrict__ chk_u,
                                                    uint32_t ck, uint32_t one) {
    constexpr int NW = P::NW, HP = P::HP, LV = P::LEAVES;
    const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t id = gid / LV, l = gid % LV;
    if (id >= max_uniq || (nuniq && id >= *nuniq)) return;   // whole trees exit together
    const unsigned gmask = ((LV == 32) ? 0xFFFFFFFFu : ((1u << LV) - 1u)) << (lane & ~(uint32_t)(LV - 1));
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
    for (int w = 0; w < NW; w++) tn[(LV + l) * NW + w] = node[w];
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
            hashH_ms<P>(ms256, msT, make_adrs(d.layer, d.tree, T_TREE, 0, z, l >> z), lr, node, kb.pk_seed);
#pragma unroll
            for (int w = 0; w < NW; w++) tn[((LV >> z) + (l >> z)) * NW + w] = node[w];
        }
    }
}

// One thread per (message, shared layer): its auth path and root from its tree.
template <class P>
__global__ void dedup_scatter_kernel(const MsgInfo* __restrict__ infos, uint32_t count, uint32_t L,
                                     const uint32_t* __restrict__ mj_slot, const uint32_t* __restrict__ slot_id,
                                     const uint32_t* __restrict__ nodes, uint8_t* __restrict__ sigs,
                                     uint32_t* __restrict__ roots, uint32_t* __restrict__ mj_id) {
    constexpr int NW = P::NW, HP = P::HP, LV = P::LEAVES;
    const uint32_t per_msg = (uint32_t)P::D - L;
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (uint64_t)count * per_msg) return;
    const uint32_t m = (uint32_t)(gid / per_msg);
    const uint32_t j = L + (uint32_t)(gid % per_msg);
    const MsgInfo& info = infos[m];
    const uint32_t slot = mj_slot[gid];
    if (info.key == KEY_INVALID || slot == kNoSlot) { mj_id[gid] = kNoSlot; return; }
    const uint32_t id = slot_id[slot];
    mj_id[gid] = id;
    const uint32_t sl = layer_leaf<P>(info.idx_tree, info.idx_leaf, (int)j);
    const uint32_t* tn = nodes + (size_t)id * 2 * LV * NW;
    uint8_t* auth = sigs + (size_t)m * P::SIG_BYTES + P::N + P::FORS_BYTES + (size_t)j * P::LAYER_BYTES +
                    (size_t)P::LEN * P::N;
#pragma unroll
    for (int z = 0; z < HP; z++) store_be<NW>(auth + (size_t)z * P::N, tn + ((LV >> z) + ((sl >> z) ^ 1u)) * NW);
    uint32_t* rt = roots + ((size_t)m * P::D + j) * NW;
#pragma unroll
    for (int w = 0; w < NW; w++) rt[w] = tn[1 * NW + w];
}

// ---------------------------------------------------------------- key cache
// A keyset keeps, per key, every tree of its top layers L..D-1 built once:
// layer j holds 2^((D-1-j) h') trees (the possible values of
// idx_tree >> (j h')).  Trees of one key are stored top layer first, so the
// tree t of layer j has id  key * tpk + cache_off(j) + t.

// Trees of the layers above j: sum over u < D-1-j of 2^(u h').
template <class P>
__host__ __device__ __forceinline__ uint64_t cache_off(uint32_t j) {
    uint64_t off = 0;
    for (uint32_t u = 0; u + 1 + j < (uint32_t)P::D; u++) off += 1ull << (u * P::HP);
    return off;
}

// One thread per cached tree: its (key, layer, tree) description.
template <class P>
__global__ void cache_desc_kernel(uint32_t num_keys, uint32_t L, uint32_t tpk, DedupDesc* __restrict__ desc) {
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (uint64_t)num_keys * tpk) return;
    const uint32_t key = (uint32_t)(gid / tpk);
    uint64_t r = gid % tpk;
    uint32_t j = (uint32_t)P::D - 1;
    while (j > L && r >= (1ull << ((P::D - 1 - j) * P::HP))) {
        r -= 1ull << ((P::D - 1 - j) * P::HP);
        j--;
    }
    DedupDesc d;
    d.tree = r;
    d.layer = j;
    d.key = key;
    desc[gid] = d;
}

// One thread per (message, cached layer): auth path and root from the cache.
template <class P>
__global__ void cache_scatter_kernel(const MsgInfo* __restrict__ infos, uint32_t count, uint32_t L, uint32_t tpk,
                                     const uint32_t* __restrict__ nodes, uint8_t* __restrict__ sigs,
                                     uint32_t* __restrict__ roots, uint32_t* __restrict__ mj_id) {
    constexpr int NW = P::NW, HP = P::HP, LV = P::LEAVES;
    const uint32_t per_msg = (uint32_t)P::D - L;
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (uint64_t)count * per_msg) return;
    const uint32_t m = (uint32_t)(gid / per_msg);
    const uint32_t j = L + (uint32_t)(gid % per_msg);
    const MsgInfo& info = infos[m];
    if (info.key == KEY_INVALID) { mj_id[gid] = kNoSlot; return; }
    const uint64_t id = (uint64_t)info.key * tpk + cache_off<P>(j) + layer_tree<P>(info.idx_tree, (int)j);
    mj_id[gid] = (uint32_t)id;
    const uint32_t sl = layer_leaf<P>(info.idx_tree, info.idx_leaf, (int)j);
    const uint32_t* tn = nodes + id * 2 * LV * NW;
    uint8_t* auth = sigs + (size_t)m * P::SIG_BYTES + P::N + P::FORS_BYTES + (size_t)j * P::LAYER_BYTES +
                    (size_t)P::LEN * P::N;
#pragma unroll
    for (int z = 0; z < HP; z++) store_be<NW>(auth + (size_t)z * P::N, tn + ((LV >> z) + ((sl >> z) ^ 1u)) * NW);
    uint32_t* rt = roots + ((size_t)m * P::D + j) * NW;
#pragma unroll
    for (int w = 0; w < NW; w++) rt[w] = tn[1 * NW + w];
}

}  // namespace hs
