// kern_msg.cuh -- per-key preparation and the message stage (kernel templates).
//
// Message stage (the paper's hash_message + message_to_indices, Fig. 2):
//   R      = Trunc_n(HMAC-SHA-x(SK.prf, PK.seed || M))          (PRF_msg)
//   digest = MGF1-SHA-x(R || PK.seed || SHA-x(R || PK.seed || PK.root || M), m)
//   digest = md || tree bytes || leaf bytes -> k FORS indices, idx_tree, idx_leaf
// FIPS 205 mode: M is preceded by a per-call prefix (0x00 || len(ctx) || ctx
// for pure SLH-DSA) in both hashes, and the FORS indices are read from md
// most significant bit first (FIPS 205 base_2b).
// One thread per message; the work is serial in the message length (two
// passes over M), which is the only length-dependent part of signing.
#pragma once
#include <cuda_runtime.h>
#include "hs_common.cuh"
#include "hs_launch.h"
#include "../../include/hs.h"

namespace hs {

// ------------------------------------------------------------- byte SHA-x
// Streaming SHA-256 / SHA-512 over bytes and big-endian words.  Only the
// message stage uses it: key words, pads and digests are appended a word at
// a time from registers; message bytes arrive through aligned word loads,
// whole blocks with the next block's loads in flight (blocks()), the partial
// blocks at either end through one batch of loads each (append()).
template <bool BIG>
struct ByteSha {
    static constexpr int B = BIG ? 128 : 64;   // block bytes
    static constexpr int BW = B / 4;
    uint32_t st[BIG ? 16 : 8];
    uint32_t blk[BW];
    uint32_t fill;      // bytes in blk
    uint64_t total;     // message bytes so far

    __device__ void init() {
        if constexpr (BIG) {
            uint64_t s[8];
            sha512_iv(s);
            for (int i = 0; i < 8; i++) { st[2 * i] = (uint32_t)(s[i] >> 32); st[2 * i + 1] = (uint32_t)s[i]; }
        } else {
            sha256_iv(st);
        }
        for (int i = 0; i < BW; i++) blk[i] = 0;
        fill = 0;
        total = 0;
    }
    __device__ void compress() {
        if constexpr (BIG) {
            uint64_t s[8];
            for (int i = 0; i < 8; i++) s[i] = ((uint64_t)st[2 * i] << 32) | st[2 * i + 1];
            sha512_compress_w32(s, blk);
            for (int i = 0; i < 8; i++) { st[2 * i] = (uint32_t)(s[i] >> 32); st[2 * i + 1] = (uint32_t)s[i]; }
        } else {
            uint32_t W[16];
            for (int i = 0; i < 16; i++) W[i] = blk[i];
            sha256_compress_rolled(st, W);
        }
        for (int i = 0; i < BW; i++) blk[i] = 0;
        fill = 0;
    }
    __device__ void byte(uint32_t b) {
        blk[fill >> 2] |= (b & 0xFFu) << (24 - 8 * (fill & 3));
        fill++;
        total++;
        if (fill == B) compress();
    }
    // Append the top nb (1..4) bytes of the big-endian word w at any byte
    // offset; the caller keeps fill + nb <= B and compresses a full block.
    __device__ __forceinline__ void put(uint32_t w, uint32_t nb) {
        if (nb < 4) w &= 0xFFFFFFFFu << (32 - 8 * nb);
        const uint32_t s = 8 * (fill & 3), j = fill >> 2;
        if (s == 0) {
            blk[j] = w;
        } else {
            blk[j] |= w >> s;
            if (s + 8 * nb > 32) blk[j + 1] |= w << (32 - s);
        }
        fill += nb;
        total += nb;
    }
    // nbytes of a big-endian word array (register data: keys, pads, digests)
    __device__ void words(const uint32_t* w, int nbytes) {
#pragma unroll 1
        for (int i = 0; i < nbytes; i += 4) {
            const uint32_t avail = nbytes - i < 4 ? (uint32_t)(nbytes - i) : 4u;
            const uint32_t room = (uint32_t)B - fill;
            if (avail <= room) {
                put(w[i >> 2], avail);
            } else {                                  // the word straddles the block end
                put(w[i >> 2], room);
                compress();
                put(w[i >> 2] << (8 * room), avail - room);
            }
            if (fill == (uint32_t)B) compress();
        }
    }
    // The message word selector: big-endian word k of bytes q[4k .. 4k+3]
    // from the aligned little-endian words around it (q & 3 = sh).
    static __device__ __forceinline__ uint32_t be_sel(uint32_t sh) {
        return (sh << 12) | ((sh + 1) << 8) | ((sh + 2) << 4) | (sh + 3);
    }
    __device__ __forceinline__ void compress_words(const uint32_t w[BW]) {
        if constexpr (BIG) {
            uint64_t s[8], W[16];
#pragma unroll
            for (int i = 0; i < 8; i++) s[i] = ((uint64_t)st[2 * i] << 32) | st[2 * i + 1];
#pragma unroll
            for (int i = 0; i < 16; i++) W[i] = ((uint64_t)w[2 * i] << 32) | w[2 * i + 1];
            sha512_compress(s, W);
#pragma unroll
            for (int i = 0; i < 8; i++) { st[2 * i] = (uint32_t)(s[i] >> 32); st[2 * i + 1] = (uint32_t)s[i]; }
        } else {
            uint32_t W[16];
#pragma unroll
            for (int i = 0; i < 16; i++) W[i] = w[i];
            sha256_compress_full(st, W);
        }
    }
    // Append r < B message bytes at q (any alignment) without crossing the
    // end of the open block.  The bytes arrive through aligned 32-bit loads
    // issued together, each holding at least one byte of q[0, r), so nothing
    // outside the message is read.
    __device__ void append(const uint8_t* q, uint32_t r) {
        if (r == 0) return;
        const uintptr_t addr = reinterpret_cast<uintptr_t>(q);
        const uint32_t* a = reinterpret_cast<const uint32_t*>(addr & ~(uintptr_t)3);
        const uint32_t sh = (uint32_t)(addr & 3), sel = be_sel(sh);
        const uint32_t nl = (sh + r + 3) >> 2;
        uint32_t raw[BW + 1];
#pragma unroll
        for (int k = 0; k < BW + 1; k++) raw[k] = ((uint32_t)k < nl) ? __ldg(a + k) : 0u;
#pragma unroll
        for (int k = 0; k < BW; k++)
            if ((uint32_t)(4 * k) < r) put(__byte_perm(raw[k], raw[k + 1], sel), min(4u, r - 4u * k));
        if (fill == (uint32_t)B) compress();
    }
    // nb whole blocks from q at any alignment: aligned 32-bit loads (every
    // word holds at least one byte of the blocks), one prmt per big-endian
    // word, and the next block's loads in flight during this compression.
    __device__ void blocks(const uint8_t* q, uint64_t nb) {
        const uintptr_t addr = reinterpret_cast<uintptr_t>(q);
        const uint32_t* a = reinterpret_cast<const uint32_t*>(addr & ~(uintptr_t)3);
        const uint32_t sh = (uint32_t)(addr & 3), sel = be_sel(sh);
        uint32_t raw[BW + 1];
#pragma unroll
        for (int k = 0; k < BW; k++) raw[k] = __ldg(a + k);
        raw[BW] = sh ? __ldg(a + BW) : 0u;
        for (uint64_t b = 0; b < nb; b++) {
            uint32_t w[BW];
#pragma unroll
            for (int k = 0; k < BW; k++) w[k] = __byte_perm(raw[k], raw[k + 1], sel);
            if (b + 1 < nb) {
                const uint32_t* an = a + (b + 1) * BW;
#pragma unroll
                for (int k = 0; k < BW; k++) raw[k] = __ldg(an + k);
                raw[BW] = sh ? __ldg(an + BW) : 0u;
            }
            compress_words(w);
        }
        total += nb * B;
    }
    // raw bytes from global memory at any alignment: the rest of the open
    // block, whole blocks, then the tail
    __device__ void mem(const uint8_t* p, uint64_t len) {
        uint64_t i = 0;
        if (fill != 0 && len != 0) {
            i = ((uint64_t)B - fill < len) ? (uint64_t)B - fill : len;
            append(p, (uint32_t)i);
        }
        const uint64_t nb = (len - i) / B;
        if (nb) {
            blocks(p + i, nb);
            i += nb * B;
        }
        if (i < len) append(p + i, (uint32_t)(len - i));
    }
    // Pad (0x80, zeros, bit length) and return the digest words (8 or 16).
    __device__ void finish(uint32_t* out) {
        const uint64_t bits = total * 8;
        blk[fill >> 2] |= 0x80u << (24 - 8 * (fill & 3));
        fill++;
        if (fill > (uint32_t)(B - (BIG ? 16 : 8))) compress();
        blk[BW - 1] = (uint32_t)bits;
        blk[BW - 2] = (uint32_t)(bits >> 32);
        compress();
        for (int i = 0; i < (BIG ? 16 : 8); i++) out[i] = st[i];
    }
};

// ------------------------------------------------------------- keyprep
// KeyBlock from a key buffer: sign keys are SK.seed||SK.prf||PK.seed||PK.root
// (4n); verify keys are PK.seed||PK.root (2n).  The midstates are the SHA-2
// state after the first block BlockPad(PK.seed).
template <class P>
__global__ void keyprep_kernel(const uint8_t* __restrict__ in, uint32_t num_keys, int from_pk,
                               KeyBlock* __restrict__ out) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= num_keys) return;
    KeyBlock kb;
    for (int i = 0; i < 64; i++) reinterpret_cast<uint32_t*>(&kb)[i] = 0;
    constexpr int NW = P::NW;
    if (from_pk) {
        const uint8_t* p = in + (size_t)k * 2 * P::N;
        load_be_unaligned<NW>(p, kb.pk_seed);
        load_be_unaligned<NW>(p + P::N, kb.pk_root);
    } else {
        const uint8_t* p = in + (size_t)k * 4 * P::N;
        load_be_unaligned<NW>(p, kb.sk_seed);
        load_be_unaligned<NW>(p + P::N, kb.sk_prf);
        load_be_unaligned<NW>(p + 2 * P::N, kb.pk_seed);
        load_be_unaligned<NW>(p + 3 * P::N, kb.pk_root);
    }
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

// ------------------------------------------------------------- message stage
template <class P>
__device__ __forceinline__ uint32_t digest_byte(const uint32_t* dw, int i) {
    return (dw[i >> 2] >> (24 - 8 * (i & 3))) & 0xFFu;
}

// verify = 0: compute R (PRF_msg) and write it to sig[0:n].
// verify = 1: R is read from the signature.
template <class P>
__global__ void message_kernel(const KeyBlock* __restrict__ keys, uint32_t num_keys,
                               const uint32_t* __restrict__ key_idx, const uint8_t* __restrict__ msgs,
                               const uint64_t* __restrict__ off, uint32_t count, uint8_t* __restrict__ sigs,
                               MsgInfo* __restrict__ infos, uint32_t* __restrict__ status, int verify,
                               const uint8_t* __restrict__ prefix, uint32_t plen, int msb_first) {
    const uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= count) return;
    constexpr int NW = P::NW;
    constexpr int DW = P::BIG ? 16 : 8;            // digest words of SHA-x
    uint8_t* sig = sigs + (size_t)m * P::SIG_BYTES;
    MsgInfo info;
    info.pad[0] = info.pad[1] = 0;
    const uint32_t key = key_idx ? key_idx[m] : 0u;
    if (key >= num_keys) {
        atomicOr(status, 1u << HS_EKEY);
        info.key = KEY_INVALID;
        info.idx_tree = 0;
        info.idx_leaf = 0;
        for (int i = 0; i < 36; i++) info.fors_idx[i] = 0;
        infos[m] = info;
        if (!verify) {
            uint4* s4 = reinterpret_cast<uint4*>(sig);
            for (int i = 0; i < P::SIG_BYTES / 16; i++) s4[i] = make_uint4(0, 0, 0, 0);
        }
        return;
    }
    const KeyBlock& kb = keys[key];
    const uint8_t* M = msgs + off[m];
    const uint64_t mlen = off[m + 1] - off[m];

    uint32_t R[8];
    uint32_t dg[16];                     // digest words, >= m bytes (m <= 49)
    if constexpr (P::SHAKE) {
        // PRF_msg = SHAKE256(SK.prf || opt_rand || M, 8n), H_msg =
        // SHAKE256(R || PK.seed || PK.root || M, 8m); M may carry a prefix
        ByteShake k;
        if (!verify) {
            k.init();
            k.words(kb.sk_prf, P::N);
            k.words(kb.pk_seed, P::N);
            if (plen) k.mem(prefix, plen);
            k.mem(M, mlen);
            k.finish(R, P::N);
            store_be<NW>(sig, R);
        } else {
            load_be<NW>(sig, R);
        }
        k.init();
        k.words(R, P::N);
        k.words(kb.pk_seed, P::N);
        k.words(kb.pk_root, P::N);
        if (plen) k.mem(prefix, plen);
        k.mem(M, mlen);
        k.finish(dg, P::M);
    } else {
    ByteSha<P::BIG> h;
    if (!verify) {
        // PRF_msg = HMAC-SHA-x(SK.prf, opt_rand || M), opt_rand = PK.seed
        uint32_t kw[ByteSha<P::BIG>::BW];
        for (int i = 0; i < ByteSha<P::BIG>::BW; i++) kw[i] = (i < NW) ? kb.sk_prf[i] : 0u;
        uint32_t inner[DW];
        h.init();
        for (int i = 0; i < ByteSha<P::BIG>::BW; i++) {
            uint32_t x = kw[i] ^ 0x36363636u;
            h.words(&x, 4);
        }
        h.words(kb.pk_seed, P::N);
        if (plen) h.mem(prefix, plen);
        h.mem(M, mlen);
        h.finish(inner);
        h.init();
        for (int i = 0; i < ByteSha<P::BIG>::BW; i++) {
            uint32_t x = kw[i] ^ 0x5c5c5c5cu;
            h.words(&x, 4);
        }
        h.words(inner, 4 * DW);
        uint32_t mac[DW];
        h.finish(mac);
        for (int i = 0; i < NW; i++) R[i] = mac[i];
        store_be<NW>(sig, R);
    } else {
        load_be<NW>(sig, R);
    }
    // H_msg
    uint32_t inner[DW];
    h.init();
    h.words(R, P::N);
    h.words(kb.pk_seed, P::N);
    h.words(kb.pk_root, P::N);
    if (plen) h.mem(prefix, plen);
    h.mem(M, mlen);
    h.finish(inner);
    int got = 0;
    for (uint32_t c = 0; got < P::M; c++) {
        h.init();
        h.words(R, P::N);
        h.words(kb.pk_seed, P::N);
        h.words(inner, 4 * DW);
        h.words(&c, 4);
        uint32_t blockd[DW];
        h.finish(blockd);
        for (int i = 0; i < DW && got < P::M; i++, got += 4) dg[got >> 2] = blockd[i];
    }
    }
    // md -> FORS indices: md read as a little-endian bit stream, index i from
    // stream bits i*a .. i*a+a-1, first bit least significant; in FIPS 205
    // mode bit q is bit 7 - q mod 8 of byte q/8 and the first bit read is the
    // most significant.
    for (int i = 0; i < P::K; i++) {
        uint32_t v = 0;
        for (int j = 0; j < P::A; j++) {
            const int q = i * P::A + j;
            if (msb_first) v |= ((digest_byte<P>(dg, q >> 3) >> (7 - (q & 7))) & 1u) << (P::A - 1 - j);
            else v |= ((digest_byte<P>(dg, q >> 3) >> (q & 7)) & 1u) << j;
        }
        info.fors_idx[i] = (uint16_t)v;
    }
    for (int i = P::K; i < 36; i++) info.fors_idx[i] = 0;
    uint64_t t = 0;
    for (int b = 0; b < P::TREE_BYTES; b++) t = (t << 8) | digest_byte<P>(dg, P::MD_BYTES + b);
    if (P::TREE_BITS < 64) t &= (1ull << (P::TREE_BITS & 63)) - 1ull;
    uint32_t l = 0;
    for (int b = 0; b < P::LEAF_BYTES; b++) l = (l << 8) | digest_byte<P>(dg, P::MD_BYTES + P::TREE_BYTES + b);
    l &= (uint32_t)(P::LEAVES - 1);
    info.idx_tree = t;
    info.idx_leaf = l;
    info.key = key;
    infos[m] = info;
}

}  // namespace hs
