// hs_common.cuh -- tweakable hashes of SPHINCS+ SHA2-simple on device (the
// SHAKE instantiation branches to keccak.cuh where a set asks for it).
//
// All n-byte values live in registers as n/4 big-endian 32-bit words (the
// natural SHA-2 word order, so digests chain into the next message block
// without byte swaps).  Every tweakable hash is
//   Trunc_n(SHA-x(BlockPad_x(PK.seed) || ADRSc || payload)),
// and the first block BlockPad_x(PK.seed) is the same for every call of a
// key, so each call starts from the key's precomputed midstate (the
// "state_seed" the paper keeps in fast memory, Sec. III-D) and compresses
// only the blocks after it.  ADRSc is 22 bytes, so every payload starts at a
// 2-byte offset inside a word; mid16() builds the straddling words.
#pragma once
#include <cstdint>
#include <type_traits>
#include "hs_params.cuh"
#include "sha2.cuh"
#include "adrs.cuh"
#include "keccak.cuh"
#include "robust.cuh"

namespace hs {

// Fill the words of one message block after the midstate: ADRSc, payload of
// PW words, 0x80 pad byte; zero the rest (length added by the caller).
template <int BW, int PW>
__device__ __forceinline__ void fill_block(uint32_t blk[BW], const Adrs& a, const uint32_t* x) {
    static_assert(5 + PW + 1 <= BW - (BW == 16 ? 2 : 4), "payload fits one block");
    blk[0] = a.w0; blk[1] = a.w1; blk[2] = a.w2; blk[3] = a.w3; blk[4] = a.w4;
    blk[5] = mid16(a.half, x[0]);
#pragma unroll
    for (int k = 1; k < PW; k++) blk[5 + k] = mid16(x[k - 1], x[k]);
    blk[5 + PW] = (x[PW - 1] << 16) | 0x8000u;
#pragma unroll
    for (int k = 6 + PW; k < BW; k++) blk[k] = 0;
}

// One-block SHA-256 tweakable hash: payload PW words, output NW words.
// FULL selects the fully unrolled compression (hot chain steps).
template <int PW, int NW, bool FULL>
__device__ __forceinline__ void thash256(const uint32_t ms[8], const Adrs& a, const uint32_t* x, uint32_t* out) {
    uint32_t W[16];
    fill_block<16, PW>(W, a, x);
    W[15] = (64 + 22 + 4 * PW) * 8;
    uint32_t st[8];
#pragma unroll
    for (int i = 0; i < 8; i++) st[i] = ms[i];
    if (FULL) sha256_compress_full(st, W); else sha256_compress_rolled(st, W);
#pragma unroll
    for (int i = 0; i < NW; i++) out[i] = st[i];
}

// One-block SHA-512 tweakable hash (ms as 16 words: hi, lo pairs).
template <int PW, int NW>
__device__ __forceinline__ void thash512(const uint32_t ms[16], const Adrs& a, const uint32_t* x, uint32_t* out) {
    uint32_t blk[32];
    fill_block<32, PW>(blk, a, x);
    blk[31] = (128 + 22 + 4 * PW) * 8;
    uint64_t st[8];
#pragma unroll
    for (int i = 0; i < 8; i++) st[i] = ((uint64_t)ms[2 * i] << 32) | ms[2 * i + 1];
    sha512_compress_w32(st, blk);
#pragma unroll
    for (int i = 0; i < NW; i++) out[i] = (i & 1) ? (uint32_t)st[i / 2] : (uint32_t)(st[i / 2] >> 32);
}

// F / PRF: always SHA-256 over an n-byte payload (chain steps use FULL).
// (SHAKE sets: ms256 holds PK.seed and the hash is SHAKE256, keccak.cuh.)
// Robust sets: F hashes x masked (pks = PK.seed words); PRF passes
// pks = nullptr, as PRF is never masked.
template <class P, bool FULL = true>
__device__ __forceinline__ void hashF(const uint32_t ms256[8], const Adrs& a, const uint32_t* x, uint32_t* out,
                                      const uint32_t* pks = nullptr) {
    if constexpr (P::SHAKE) {
        shake_thash1<P::NW, P::NW>(ms256, a, x, out);
    } else if constexpr (P::ROBUST) {
        uint32_t xm[P::NW];
#pragma unroll
        for (int i = 0; i < P::NW; i++) xm[i] = x[i];
        if (pks) mask_regs<false, P::NW, P::NW>(pks, a, xm);
        thash256<P::NW, P::NW, FULL>(ms256, a, xm, out);
    } else {
        thash256<P::NW, P::NW, FULL>(ms256, a, x, out);
    }
}

// H: two n-byte children; SHA-512 for n > 16.  Robust sets: the children
// masked first (pks = PK.seed words).
template <class P>
__device__ __forceinline__ void hashH_ms(const uint32_t* ms256, const uint32_t* ms512, const Adrs& a,
                                         const uint32_t* lr, uint32_t* out, const uint32_t* pks = nullptr);
template <class P>
__device__ __forceinline__ void hashH(const KeyBlock& kb, const Adrs& a, const uint32_t* lr, uint32_t* out) {
    hashH_ms<P>(kb.ms256, kb.ms512, a, lr, out, kb.pk_seed);
}
// Same, with the midstates passed separately (kernels that keep them in registers).
template <class P>
__device__ __forceinline__ void hashH_ms(const uint32_t* ms256, const uint32_t* ms512, const Adrs& a,
                                         const uint32_t* lr, uint32_t* out, const uint32_t* pks) {
    if constexpr (P::SHAKE) {
        shake_thash1<P::NW, 2 * P::NW>(ms256, a, lr, out);
    } else if constexpr (P::ROBUST) {
        uint32_t m[2 * P::NW];
#pragma unroll
        for (int i = 0; i < 2 * P::NW; i++) m[i] = lr[i];
        mask_regs<P::BIG, P::NW, 2 * P::NW>(pks, a, m);
        if constexpr (P::BIG) thash512<2 * P::NW, P::NW>(ms512, a, m, out);
        else thash256<2 * P::NW, P::NW, false>(ms256, a, m, out);
    } else if constexpr (P::BIG) {
        thash512<2 * P::NW, P::NW>(ms512, a, lr, out);
    } else {
        thash256<2 * P::NW, P::NW, false>(ms256, a, lr, out);
    }
}

// Streaming T_l: SHA-x over ADRSc || v_0 || ... || v_{l-1} after the
// midstate, fed one n-byte value at a time.  The block buffer is a small
// per-thread array; the 2-byte misalignment is carried in 'carry'.
template <bool BIG>
struct TStream {
    static constexpr int BW = BIG ? 32 : 16;   // 32-bit words per block
    static constexpr int LW = BIG ? 4 : 2;     // words of the length field
    uint32_t st[BIG ? 16 : 8];
    uint32_t buf[BW];
    int pos;
    uint32_t carry;

    __device__ __forceinline__ void compress() {
        if constexpr (BIG) {
            uint64_t s[8];
#pragma unroll
            for (int i = 0; i < 8; i++) s[i] = ((uint64_t)st[2 * i] << 32) | st[2 * i + 1];
            sha512_compress_w32(s, buf);
#pragma unroll
            for (int i = 0; i < 8; i++) { st[2 * i] = (uint32_t)(s[i] >> 32); st[2 * i + 1] = (uint32_t)s[i]; }
        } else {
            uint32_t W[16];
#pragma unroll
            for (int i = 0; i < 16; i++) W[i] = buf[i];
            sha256_compress_rolled(st, W);
        }
    }
    __device__ __forceinline__ void init(const uint32_t* ms, const Adrs& a) {
#pragma unroll
        for (int i = 0; i < (BIG ? 16 : 8); i++) st[i] = ms[i];
        buf[0] = a.w0; buf[1] = a.w1; buf[2] = a.w2; buf[3] = a.w3; buf[4] = a.w4;
        pos = 5;
        carry = a.half;
    }
    __device__ __forceinline__ void push(uint32_t v) {
        buf[pos++] = (carry << 16) | (v >> 16);
        carry = v & 0xFFFFu;
        if (pos == BW) { compress(); pos = 0; }
    }
    template <int NW>
    __device__ __forceinline__ void push_n(const uint32_t* v) {
#pragma unroll
        for (int i = 0; i < NW; i++) push(v[i]);
    }
    // payload_bytes: total bytes pushed (l * n); writes NW output words.
    template <int NW>
    __device__ __forceinline__ void finish(uint32_t payload_bytes, uint32_t* out) {
        buf[pos++] = (carry << 16) | 0x8000u;
        if (pos > BW - LW) {
            while (pos < BW) buf[pos++] = 0;
            compress();
            pos = 0;
        }
        while (pos < BW - 1) buf[pos++] = 0;
        buf[BW - 1] = ((BIG ? 128u : 64u) + 22u + payload_bytes) * 8u;
        compress();
#pragma unroll
        for (int i = 0; i < NW; i++) out[i] = st[i];
    }
};

// Block b of a T_l call over PW payload words in memory (chain ends, FORS
// roots): ADRSc || payload || pad || bit length after the midstate.  Word
// positions inside a block are compile-time constants and b is a loop
// counter, so nothing is buffered in registers with run-time indices (which
// would live in local memory).
template <bool BIG, int PW>
__device__ __forceinline__ void tl_block(const Adrs& a, const uint32_t* p, int b, uint32_t* W) {
    constexpr int BW = BIG ? 32 : 16;            // words per block
    constexpr int LW = BIG ? 4 : 2;              // length words
    constexpr int TW = 5 + PW + 1;               // ADRSc words, payload at a 2-byte offset, pad word
    constexpr int NB = (TW + LW + BW - 1) / BW;
    constexpr uint32_t BITS = ((BIG ? 128u : 64u) + 22u + 4u * PW) * 8u;
#pragma unroll
    for (int k = 0; k < BW; k++) {
        const int j = b * BW + k;
        uint32_t v;
        if (j < 5) v = j == 0 ? a.w0 : j == 1 ? a.w1 : j == 2 ? a.w2 : j == 3 ? a.w3 : a.w4;
        else if (j == 5) v = mid16(a.half, p[0]);
        else if (j < 5 + PW) v = mid16(p[j - 6], p[j - 5]);
        else if (j == 5 + PW) v = (p[PW - 1] << 16) | 0x8000u;
        else v = 0u;
        if (b == NB - 1 && k == BW - 1) v = BITS;
        W[k] = v;
    }
}
template <bool BIG, int PW>
__host__ __device__ constexpr int tl_blocks() {
    return (5 + PW + 1 + (BIG ? 4 : 2) + (BIG ? 32 : 16) - 1) / (BIG ? 32 : 16);
}

// T_l over PW payload words in memory: Trunc_n(SHA-x(midstate; ADRSc ||
// payload)), block by block as above.  Same value as the streaming form.
template <bool BIG, int PW, int NW>
__device__ __forceinline__ void tl_from_mem(const uint32_t* ms, const Adrs& a, const uint32_t* p, uint32_t* out) {
    uint32_t st[BIG ? 16 : 8];
#pragma unroll
    for (int i = 0; i < (BIG ? 16 : 8); i++) st[i] = ms[i];
#pragma unroll 1
    for (int b = 0; b < tl_blocks<BIG, PW>(); b++) {
        uint32_t W[BIG ? 32 : 16];
        tl_block<BIG, PW>(a, p, b, W);
        if constexpr (BIG) {
            uint64_t s64[8];
#pragma unroll
            for (int i = 0; i < 8; i++) s64[i] = ((uint64_t)st[2 * i] << 32) | st[2 * i + 1];
            sha512_compress_w32(s64, W);
#pragma unroll
            for (int i = 0; i < 8; i++) { st[2 * i] = (uint32_t)(s64[i] >> 32); st[2 * i + 1] = (uint32_t)s64[i]; }
        } else {
            sha256_compress_rolled(st, W);
        }
    }
#pragma unroll
    for (int i = 0; i < NW; i++) out[i] = st[i];
}

// T_l stream of a parameter set: SHA-2 as above, or SHAKE256 (whose init
// takes PK.seed where the SHA-2 stream takes the midstate).
template <class P>
using TStreamP = std::conditional_t<P::SHAKE, ShakeStream<P::NW, (P::LEN > P::K ? P::LEN : P::K) * P::NW>,
                                    TStream<P::BIG>>;

// ------------------------------------------------------------ byte I/O

// Store / load an n-byte value (NW big-endian words) at a byte address that
// is at least 8-byte aligned (every node offset inside a signature is a
// multiple of n from a 16-byte aligned signature start).
template <int NW>
__device__ __forceinline__ void store_be(uint8_t* p, const uint32_t* v) {
    if constexpr (NW % 4 == 0) {
        if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
#pragma unroll
            for (int i = 0; i < NW; i += 4)
                *reinterpret_cast<uint4*>(p + 4 * i) =
                    make_uint4(bswap32(v[i]), bswap32(v[i + 1]), bswap32(v[i + 2]), bswap32(v[i + 3]));
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < NW; i += 2)
        *reinterpret_cast<uint2*>(p + 4 * i) = make_uint2(bswap32(v[i]), bswap32(v[i + 1]));
}

template <int NW>
__device__ __forceinline__ void load_be(const uint8_t* p, uint32_t* v) {
#pragma unroll
    for (int i = 0; i < NW; i += 2) {
        uint2 t = *reinterpret_cast<const uint2*>(p + 4 * i);
        v[i] = bswap32(t.x);
        v[i + 1] = bswap32(t.y);
    }
}

// Byte-granular load of NW big-endian words from any address (key material).
template <int NW>
__device__ __forceinline__ void load_be_unaligned(const uint8_t* p, uint32_t* v) {
#pragma unroll
    for (int i = 0; i < NW; i++)
        v[i] = ((uint32_t)p[4 * i] << 24) | ((uint32_t)p[4 * i + 1] << 16) |
               ((uint32_t)p[4 * i + 2] << 8) | (uint32_t)p[4 * i + 3];
}

// Tree at layer j of the hypertree: idx_tree >> (j h'); shifts of 64 or more
// give 0 (at 256f, h - h' = 64 and layer 16 would shift by 64).
template <class P>
__device__ __forceinline__ uint64_t layer_tree(uint64_t idx_tree, int j) {
    const int s = j * P::HP;
    return s >= 64 ? 0ull : (idx_tree >> s);
}
// Signing leaf at layer j: idx_leaf at j = 0, else the h' bits of idx_tree
// just below layer j's tree bits.
template <class P>
__device__ __forceinline__ uint32_t layer_leaf(uint64_t idx_tree, uint32_t idx_leaf, int j) {
    if (j == 0) return idx_leaf;
    const int s = (j - 1) * P::HP;
    return (uint32_t)((s >= 64 ? 0ull : (idx_tree >> s)) & (uint64_t)(P::LEAVES - 1));
}

}  // namespace hs
