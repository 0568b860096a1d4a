// robust.cuh -- the masks of the robust SHA2 tweakable hashes (SPHINCS+
// round 3.1; a variant beside the paper's simple instantiation).
//
// Robust F, H and T_l hash M xor MGF1-SHA-x(PK.seed || ADRSc, |M|) in place
// of M, with SHA-x the hash the tweakable hash itself uses (SHA-256 for F;
// SHA-512 for H and T_l at n = 24 / 32) and PK.seed unpadded; PRF, PRF_msg
// and H_msg are as in the simple instantiation.  MGF1 block c is
// SHA-x(PK.seed || ADRSc || BE32(c)): 4 n + 26 bytes, one compression from
// the IV (two for SHA-256 at n = 32, where the length no longer fits the
// first block).  The mask does not depend on the hashed value, only on the
// key and the address.
#pragma once
#include <cstdint>
#include "sha2.cuh"
#include "adrs.cuh"

namespace hs {

// Message words of MGF1 block c: PK.seed (NW words) || ADRSc (5 words and
// the half word) || BE32(c), then the 0x80 pad byte; the rest zero.
template <int NW, int BW>
__device__ __forceinline__ void mgf1_seed_words(const uint32_t* pks, const Adrs& a, uint32_t c, uint32_t* W) {
#pragma unroll
    for (int i = 0; i < BW; i++) W[i] = 0u;
#pragma unroll
    for (int i = 0; i < NW; i++) W[i] = pks[i];
    W[NW] = a.w0; W[NW + 1] = a.w1; W[NW + 2] = a.w2; W[NW + 3] = a.w3; W[NW + 4] = a.w4;
    W[NW + 5] = (a.half << 16) | (c >> 16);
    W[NW + 6] = (c << 16) | 0x8000u;
}

// SHA-256 MGF1 block c (8 words).
template <int NW>
__device__ __forceinline__ void mgf1_256_block(const uint32_t* pks, const Adrs& a, uint32_t c, uint32_t out[8]) {
    constexpr uint32_t L = 4 * NW + 26;          // seed || counter bytes
    uint32_t W[16];
    mgf1_seed_words<NW, 16>(pks, a, c, W);
    sha256_iv(out);
    if constexpr (L + 9 <= 64) {
        W[15] = L * 8;
        sha256_compress_rolled(out, W);
    } else {                                      // n = 32: the length goes to a second block
        sha256_compress_rolled(out, W);
#pragma unroll
        for (int i = 0; i < 15; i++) W[i] = 0u;
        W[15] = L * 8;
        sha256_compress_rolled(out, W);
    }
}

// SHA-512 MGF1 block c (16 words, big-endian 32-bit halves).
template <int NW>
__device__ __forceinline__ void mgf1_512_block(const uint32_t* pks, const Adrs& a, uint32_t c, uint32_t out[16]) {
    constexpr uint32_t L = 4 * NW + 26;
    static_assert(L + 17 <= 128, "one SHA-512 block");
    uint32_t W[32];
    mgf1_seed_words<NW, 32>(pks, a, c, W);
    W[31] = L * 8;
    uint64_t s[8];
    sha512_iv(s);
    sha512_compress_w32(s, W);
#pragma unroll
    for (int i = 0; i < 8; i++) { out[2 * i] = (uint32_t)(s[i] >> 32); out[2 * i + 1] = (uint32_t)s[i]; }
}

// x[0 .. PW) ^= the first PW words of the mask (PW a compile-time count:
// register payloads of F and H).  BIG selects SHA-512 blocks.
template <bool BIG, int NW, int PW>
__device__ __forceinline__ void mask_regs(const uint32_t* pks, const Adrs& a, uint32_t* x) {
    constexpr int DW = BIG ? 16 : 8;             // mask words per MGF1 block
#pragma unroll
    for (int c = 0; c * DW < PW; c++) {
        uint32_t m[DW];
        if constexpr (BIG) mgf1_512_block<NW>(pks, a, (uint32_t)c, m);
        else mgf1_256_block<NW>(pks, a, (uint32_t)c, m);
#pragma unroll
        for (int i = 0; i < DW; i++)
            if (c * DW + i < PW) x[c * DW + i] ^= m[i];
    }
}

// The same over PW words in memory (T_l payloads: chain ends, FORS roots),
// in place, one MGF1 block at a time.
template <bool BIG, int NW, int PW>
__device__ __forceinline__ void mask_mem(const uint32_t* pks, const Adrs& a, uint32_t* p) {
    constexpr int DW = BIG ? 16 : 8;
#pragma unroll 1
    for (int c = 0; c * DW < PW; c++) {
        uint32_t m[DW];
        if constexpr (BIG) mgf1_512_block<NW>(pks, a, (uint32_t)c, m);
        else mgf1_256_block<NW>(pks, a, (uint32_t)c, m);
#pragma unroll
        for (int i = 0; i < DW; i++)
            if (c * DW + i < PW) p[c * DW + i] ^= m[i];
    }
}

}  // namespace hs
