// set_impl.cuh -- host launchers of every kernel for one parameter set P.
// Each set_<name>.cu instantiates SetImpl<P> and the launch-shape variants
// the tuner may choose from, and exports them as one SetOps table.
#pragma once
#include <cuda_runtime.h>
#include "hs_launch.h"
#include "kern_msg.cuh"
#include "kern_fors.cuh"
#include "kern_tree.cuh"
#include "kern_wots.cuh"
#include "kern_verify.cuh"
#include "kern_dedup.cuh"
#include "kern_stree.cuh"

namespace hs {

template <class P>
struct SetImpl {
    // XMSS trees wider than a warp (s sets) take the two-launch form of
    // kern_stree.cuh, also for the shared and cached trees.
    static constexpr bool kWide = P::LEAVES > 32;

    // layers each message builds itself: all of them unless the upper
    // layers are shared within the batch (dedup_layer = first shared layer)
    static uint32_t own_layers(const Batch& b) { return b.dedup_layer ? b.dedup_layer : (uint32_t)P::D; }

    static cudaError_t keyprep(const Batch& b, bool from_pk, cudaStream_t s) {
        const uint32_t T = 128, G = (b.num_keys + T - 1) / T;
        keyprep_kernel<P><<<G, T, 0, s>>>(b.keys_in, b.num_keys, from_pk ? 1 : 0, b.keys);
        return cudaGetLastError();
    }
    static cudaError_t message(const Batch& b, bool verify, cudaStream_t s) {
        if constexpr (!P::SHAKE) {
            if (b.msg_warp) {                               // a warp per message
                const uint32_t T = 32 * kMsgWarpsPerBlock, G = (b.count + kMsgWarpsPerBlock - 1) / kMsgWarpsPerBlock;
                message_warp_kernel<P><<<G, T, 0, s>>>(b.keys, b.num_keys, b.key_idx, b.msgs, b.offsets, b.count,
                                                       b.sigs, b.infos, b.status, verify ? 1 : 0, b.prefix,
                                                       b.prefix_len, b.fips ? 1 : 0);
                return cudaGetLastError();
            }
        }
        const uint32_t T = 64, G = (b.count + T - 1) / T;
        message_kernel<P><<<G, T, 0, s>>>(b.keys, b.num_keys, b.key_idx, b.msgs, b.offsets, b.count, b.sigs,
                                          b.infos, b.status, verify ? 1 : 0, b.prefix, b.prefix_len,
                                          b.fips ? 1 : 0);
        return cudaGetLastError();
    }
    template <int LPT>
    static cudaError_t fors(const Batch& b, cudaStream_t s) {
        const uint64_t threads = (uint64_t)b.count * P::K * LPT;
        const uint32_t T = 256;
        const uint32_t G = (uint32_t)((threads + T - 1) / T);
        fors_kernel<P, fors_pol<P>(), LPT><<<G, T, 0, s>>>(b.keys, b.infos, b.count, b.sigs, b.fors_roots, 1u);
        return cudaGetLastError();
    }
    static cudaError_t fors_pk(const Batch& b, cudaStream_t s) {
        const uint32_t T = 128, G = (b.count + T - 1) / T;
        fors_pk_kernel<P><<<G, T, 0, s>>>(b.keys, b.infos, b.count, b.fors_roots, b.pk_fors);
        return cudaGetLastError();
    }
    template <int MINB, int POL = tree_pol<P>(), int ILP = 1>
    static cudaError_t tree(const Batch& b, cudaStream_t s) {
        const uint32_t L = own_layers(b);
        const uint64_t threads = (uint64_t)b.count * L * P::LEAVES;
        const uint32_t T = 128;
        const uint32_t G = (uint32_t)((threads + T - 1) / T);
        if (threads == 0) return cudaSuccess;
        if constexpr (kWide) {
            bleaf_kernel<P, POL, MINB, ILP><<<G, T, 0, s>>>(b.keys, b.infos, b.count, b.leafv, b.chk, b.ck, L, 1u);
            cudaError_t e = cudaGetLastError();
            return e == cudaSuccess ? merge(b, s) : e;
        } else {
            tree_kernel<P, POL, MINB, ILP><<<G, T, 0, s>>>(b.keys, b.infos, b.count, b.sigs, b.roots, b.chk, b.ck,
                                                        L, 1u);
            return cudaGetLastError();
        }
    }
    // Wide trees: one block per (message, layer) merges the stored leaves.
    static cudaError_t merge(const Batch& b, cudaStream_t s) {
        const uint32_t L = own_layers(b);
        const uint64_t blocks = (uint64_t)b.count * L;
        if (blocks == 0) return cudaSuccess;
        bmerkle_kernel<P><<<(uint32_t)blocks, kMergeThreads, 0, s>>>(b.keys, b.infos, b.count, b.leafv, b.sigs,
                                                                     b.roots, L);
        return cudaGetLastError();
    }
    // The distinct trees of the shared / cached layers, all nodes and the
    // checkpoints of every leaf (desc: their (key, layer, tree)).
    static cudaError_t build_trees(const KeyBlock* keys, const DedupDesc* desc, const uint32_t* nuniq,
                                   uint32_t max_uniq, uint32_t* nodes, uint32_t* chk, uint32_t ck, cudaStream_t s) {
        const uint32_t T = 128;
        const uint64_t th = (uint64_t)max_uniq * P::LEAVES;
        if (th == 0) return cudaSuccess;
        if constexpr (kWide) {
            wtree_leaf_kernel<P, tree_pol<P>()><<<(uint32_t)((th + T - 1) / T), T, 0, s>>>(keys, desc, nuniq, max_uniq,
                                                                                      nodes, chk, ck, 1u);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            wtree_merge_kernel<P><<<max_uniq, kMergeThreads, 0, s>>>(keys, desc, nuniq, max_uniq, nodes);
        } else {
            utree_kernel<P, tree_pol<P>()><<<(uint32_t)((th + T - 1) / T), T, 0, s>>>(keys, desc, nuniq, max_uniq, nodes,
                                                                                  chk, ck, 1u);
        }
        return cudaGetLastError();
    }
    static cudaError_t tree_dedup(const Batch& b, cudaStream_t s) {
        const uint32_t T = 128, L = own_layers(b);
        const uint64_t mj = (uint64_t)b.count * (P::D - L);
        dedup_insert_kernel<P><<<(uint32_t)((mj + T - 1) / T), T, 0, s>>>(b.infos, b.count, L, b.table, b.cap_log2,
                                                                          b.mj_slot, b.status);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const uint32_t cap = 1u << b.cap_log2;
        dedup_compact_kernel<<<(cap + T - 1) / T, T, 0, s>>>(b.table, cap, b.slot_id, b.desc, b.nuniq, b.max_uniq,
                                                             b.status);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = build_trees(b.keys, b.desc, b.nuniq, b.max_uniq, b.nodes_u, b.chk_u, b.ck, s)) != cudaSuccess)
            return e;
        dedup_scatter_kernel<P><<<(uint32_t)((mj + T - 1) / T), T, 0, s>>>(b.infos, b.count, L, b.mj_slot, b.slot_id,
                                                                           b.nodes_u, b.sigs, b.roots, b.mj_id);
        return cudaGetLastError();
    }
    // Cached top layers (keyset): auth paths, roots and tree ids from the cache.
    static cudaError_t tree_cached(const Batch& b, cudaStream_t s) {
        const uint32_t T = 128, L = own_layers(b);
        const uint64_t mj = (uint64_t)b.count * (P::D - L);
        if (mj == 0) return cudaSuccess;
        cache_scatter_kernel<P><<<(uint32_t)((mj + T - 1) / T), T, 0, s>>>(b.infos, b.count, L, b.cache_tpk,
                                                                           b.nodes_u, b.sigs, b.roots, b.mj_id);
        return cudaGetLastError();
    }
    // Build every tree of layers L..D-1 of num_keys resident keys.
    static cudaError_t cache_build(const KeyBlock* keys, uint32_t num_keys, uint32_t L, uint32_t tpk,
                                   DedupDesc* desc, uint32_t* nodes, uint32_t* chk, uint32_t ck, cudaStream_t s) {
        const uint32_t T = 128;
        const uint64_t trees = (uint64_t)num_keys * tpk;
        if (trees == 0) return cudaSuccess;
        cache_desc_kernel<P><<<(uint32_t)((trees + T - 1) / T), T, 0, s>>>(num_keys, L, tpk, desc);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return build_trees(keys, desc, nullptr, (uint32_t)trees, nodes, chk, ck, s);
    }
    static cudaError_t tree_split(const Batch& b, cudaStream_t s) {
        const uint32_t T = 128;
        const uint32_t L = own_layers(b);
        const uint64_t chains = (uint64_t)b.count * L * P::LEAVES * P::LEN;
        if (chains == 0) return cudaSuccess;
        chains_kernel<P, tree_pol<P>()><<<(uint32_t)((chains + T - 1) / T), T, 0, s>>>(b.keys, b.infos, b.count, b.ends,
                                                                                  b.chk, b.ck, L, 1u);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const uint64_t leaves = (uint64_t)b.count * L * P::LEAVES;
        if constexpr (kWide) {
            bleaf_from_ends_kernel<P><<<(uint32_t)((leaves + T - 1) / T), T, 0, s>>>(b.keys, b.infos, b.count,
                                                                                    b.ends, b.leafv, L);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            return merge(b, s);
        } else {
            leaves_kernel<P><<<(uint32_t)((leaves + T - 1) / T), T, 0, s>>>(b.keys, b.infos, b.count, b.ends,
                                                                            b.sigs, b.roots, L);
            return cudaGetLastError();
        }
    }
    static cudaError_t wots(const Batch& b, cudaStream_t s) {
        const uint64_t threads = (uint64_t)b.count * P::D * P::LEN;
        const uint32_t T = 256;
        const uint32_t G = (uint32_t)((threads + T - 1) / T);
        wots_kernel<P, kChainPol><<<G, T, 0, s>>>(b.keys, b.infos, b.count, b.pk_fors, b.roots, b.sigs, b.chk,
                                                   b.ck, own_layers(b), b.mj_id, b.chk_u, 1u);
        return cudaGetLastError();
    }
    // Verification: FORS roots, PK_FORS, then per layer chains and T_len +
    // climbs (layers are serial), then the comparison with PK.root.  The
    // layer messages live in pk_fors (layer 0) and roots (layers >= 1).
    // Scratch: fors_roots, pk_fors, roots (root_j of the current layer),
    // ends (chain ends of one layer), vcnt (16 step buckets per layer),
    // vsitem / vorder (one word per chain of a layer).
    static cudaError_t verify(const Batch& b, cudaStream_t s) {
        const uint32_t T = 128;
        cudaError_t e = cudaMemsetAsync(b.vcnt, 0, sizeof(uint32_t) * 16 * P::D, s);
        const uint64_t ft = (uint64_t)b.count * P::K;
        if (e == cudaSuccess) {
            vfors_kernel<P><<<(uint32_t)((ft + T - 1) / T), T, 0, s>>>(b.keys, b.infos, b.count, b.sigs,
                                                                       b.fors_roots);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = fors_pk(b, s);
        const uint64_t ct = (uint64_t)b.count * P::LEN;
        const uint32_t G1 = (b.count + T - 1) / T;
        if (e == cudaSuccess) {
            vcount0_kernel<P><<<G1, T, 0, s>>>(b.infos, b.count, b.pk_fors, b.vcnt, b.vsitem);
            e = cudaGetLastError();
        }
        for (uint32_t j = 0; j < (uint32_t)P::D && e == cudaSuccess; j++) {
            vscatter_kernel<P><<<(uint32_t)((ct + 255) / 256), 256, 0, s>>>(b.count, b.vcnt + 16 * j, b.vsitem,
                                                                            b.vorder);
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            vchain_kernel<P, kChainPol><<<(uint32_t)((ct + T - 1) / T), T, 0, s>>>(
                b.keys, b.infos, b.count, b.sigs, b.vorder, b.vsitem, b.ends, j, 1u);
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            vleaf_kernel<P><<<G1, T, 0, s>>>(b.keys, b.infos, b.count, b.sigs, b.ends, b.roots, j,
                                             j + 1 < (uint32_t)P::D ? b.vcnt + 16 * (j + 1) : nullptr, b.vsitem);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return e;
        vfinal_kernel<P><<<G1, T, 0, s>>>(b.keys, b.infos, b.count, b.roots, b.ok);
        return cudaGetLastError();
    }
    static cudaError_t keygen(const uint8_t* seeds, uint32_t count, uint8_t* pk, uint8_t* sk, cudaStream_t s) {
        const uint64_t threads = (uint64_t)count * P::LEAVES;
        const uint32_t T = 128;
        const uint32_t G = (uint32_t)((threads + T - 1) / T);
        if constexpr (kWide) {
            // key blocks, top-tree leaves, then one block per key for the root
            const size_t kb_bytes = ((size_t)count * sizeof(KeyBlock) + 255) & ~(size_t)255;
            void* scratch = nullptr;
            cudaError_t e = pool_alloc(&scratch, kb_bytes + threads * P::NW * 4, s);
            if (e != cudaSuccess) return e;
            KeyBlock* kbs = static_cast<KeyBlock*>(scratch);
            uint32_t* leafv = reinterpret_cast<uint32_t*>(static_cast<char*>(scratch) + kb_bytes);
            seed_keys_kernel<P><<<(count + T - 1) / T, T, 0, s>>>(seeds, count, kbs);
            e = cudaGetLastError();
            if (e == cudaSuccess) {
                bkeygen_leaf_kernel<P, kChainPol><<<G, T, 0, s>>>(kbs, count, leafv, 1u);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) {
                bkeygen_root_kernel<P><<<count, kMergeThreads, 0, s>>>(kbs, seeds, count, leafv, pk, sk);
                e = cudaGetLastError();
            }
            const cudaError_t f = cudaFreeAsync(scratch, s);
            return e == cudaSuccess ? f : e;
        } else {
            keygen_kernel<P><<<G, T, 0, s>>>(seeds, count, pk, sk, 1u);
            return cudaGetLastError();
        }
    }
};

// The compiled variants of TREE_Sign's per-leaf kernel for one set, as
// (min blocks per SM, addition policy, chains per thread): the default
// (0, tree_pol<P>(), 1); the other addition policy and two interleaved
// chains per thread (simple SHA-2 sets other than toy); and MB_ALT min blocks
// (0 = none) -- each alternative with the other two at their defaults.
template <class P, int MB_ALT>
struct TreeVariants {
    static constexpr int PD = tree_pol<P>();
    static constexpr bool kAlts = !P::SHAKE && !P::ROBUST && P::LEAVES >= 8;   // simple SHA-2, not toy
    static constexpr int PA = PD == 7 ? 15 : 7;
    static bool has(int minb, int pol, int ilp) {
        if (minb == 0 && pol == PD && ilp == 1) return true;
        if (MB_ALT != 0 && minb == MB_ALT && pol == PD && ilp == 1) return true;
        return kAlts && minb == 0 && ((pol == PA && ilp == 1) || (pol == PD && ilp == 2));
    }
    static cudaError_t run(const Batch& b, int minb, int pol, int ilp, cudaStream_t s) {
        if (minb == 0 && pol == PD && ilp == 1) return SetImpl<P>::template tree<1, PD, 1>(b, s);
        if constexpr (MB_ALT != 0)
            if (minb == MB_ALT && pol == PD && ilp == 1) return SetImpl<P>::template tree<MB_ALT, PD, 1>(b, s);
        if constexpr (kAlts) {
            if (minb == 0 && pol == PA && ilp == 1) return SetImpl<P>::template tree<1, PA, 1>(b, s);
            if (minb == 0 && pol == PD && ilp == 2) return SetImpl<P>::template tree<1, PD, 2>(b, s);
        }
        return cudaErrorInvalidValue;
    }
};

}  // namespace hs
