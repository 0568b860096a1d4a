// keccak.cuh -- Keccak-f[1600] and the SHAKE256 tweakable hashes of the
// SHAKE instantiation (a variant; the paper signs with SHA-2).
//
// SHAKE-simple (SPHINCS+ round 3.1, FIPS 205 Sec. 11.1): every tweakable
// hash is SHAKE256(PK.seed || ADRS || payload, 8n) with the full 32-byte
// ADRS.  Values stay n/4 big-endian 32-bit words in registers, as in the
// SHA-2 path; a Keccak lane is 8 bytes little-endian, so lane i takes
// bswap(word 2i) as its low half and bswap(word 2i+1) as its high half.
//
// GB300 mapping: the 25 lanes are 50 32-bit registers; every 64-bit XOR,
// AND-NOT and rotation is two 32-bit LOP3 / funnel shifts on the ALU pipe
// (~190 ALU ops per round).  The 24 rounds run in a rolled loop (the round
// body is the same each time; only the round constant changes), keeping the
// code of each call site small.  The rotation offsets, the lane permutation
// and the round constants are derived at compile time from FIPS 202's
// definitions (Sec. 3.2.2 - 3.2.5), not written out.
#pragma once
#include <cstdint>
#include "sha2.cuh"
#include "adrs.cuh"

namespace hs {
namespace kk {

// rho offset of lane x + 5y: walk (x, y) <- (y, 2x + 3y) from (1, 0); the
// t-th lane visited is rotated by (t + 1)(t + 2) / 2 mod 64.
__host__ __device__ constexpr int rho_offset(int lane) {
    int x = 1, y = 0;
    for (int t = 0; t < 24; t++) {
        if (x + 5 * y == lane) return ((t + 1) * (t + 2) / 2) % 64;
        const int nx = y, ny = (2 * x + 3 * y) % 5;
        x = nx;
        y = ny;
    }
    return 0;   // lane 0
}
// pi: the lane that lands at x + 5y comes from ((x + 3y) mod 5) + 5x.
__host__ __device__ constexpr int pi_source(int lane) {
    const int x = lane % 5, y = lane / 5;
    return (x + 3 * y) % 5 + 5 * x;
}
// rc(t): output bit of the LFSR x^8 + x^6 + x^5 + x^4 + 1 after t steps.
__host__ __device__ constexpr uint32_t lfsr_bit(int t) {
    uint32_t r = 1;
    for (int i = 0; i < t % 255; i++) {
        r <<= 1;
        if (r & 0x100u) r ^= 0x171u;   // x^8 = x^6 + x^5 + x^4 + 1
    }
    return r & 1u;
}
__host__ __device__ constexpr uint64_t round_constant(int ir) {
    uint64_t rc = 0;
    for (int j = 0; j <= 6; j++) rc |= (uint64_t)lfsr_bit(j + 7 * ir) << ((1 << j) - 1);
    return rc;
}
struct RC {
    uint32_t lo[24], hi[24];
    __host__ __device__ constexpr RC() : lo(), hi() {
        for (int i = 0; i < 24; i++) {
            lo[i] = (uint32_t)round_constant(i);
            hi[i] = (uint32_t)(round_constant(i) >> 32);
        }
    }
};
static __constant__ RC kRC = RC();

// 64-bit rotation left by R of (hi:lo) as two funnel shifts.
template <int R>
__device__ __forceinline__ void rotl(uint32_t lo, uint32_t hi, uint32_t& olo, uint32_t& ohi) {
    if constexpr (R == 0) {
        olo = lo; ohi = hi;
    } else if constexpr (R == 32) {
        olo = hi; ohi = lo;
    } else if constexpr (R < 32) {
        ohi = __funnelshift_l(lo, hi, R);
        olo = __funnelshift_l(hi, lo, R);
    } else {
        ohi = __funnelshift_l(hi, lo, R - 32);
        olo = __funnelshift_l(lo, hi, R - 32);
    }
}

template <int L>
__device__ __forceinline__ void rho_pi_lane(const uint32_t* alo, const uint32_t* ahi, const uint32_t* dlo,
                                            const uint32_t* dhi, uint32_t* blo, uint32_t* bhi) {
    constexpr int S = pi_source(L);
    rotl<rho_offset(S)>(alo[S] ^ dlo[S % 5], ahi[S] ^ dhi[S % 5], blo[L], bhi[L]);
    if constexpr (L + 1 < 25) rho_pi_lane<L + 1>(alo, ahi, dlo, dhi, blo, bhi);
}

}  // namespace kk

// Keccak-f[1600] on lanes A[x + 5y] = (hi[i]:lo[i]).
__device__ __forceinline__ void keccak_f1600(uint32_t lo[25], uint32_t hi[25]) {
#pragma unroll 1
    for (int ir = 0; ir < 24; ir++) {
        uint32_t clo[5], chi[5], dlo[5], dhi[5];
#pragma unroll
        for (int x = 0; x < 5; x++) {
            clo[x] = lo[x] ^ lo[x + 5] ^ lo[x + 10] ^ lo[x + 15] ^ lo[x + 20];
            chi[x] = hi[x] ^ hi[x + 5] ^ hi[x + 10] ^ hi[x + 15] ^ hi[x + 20];
        }
#pragma unroll
        for (int x = 0; x < 5; x++) {
            uint32_t rlo, rhi;
            kk::rotl<1>(clo[(x + 1) % 5], chi[(x + 1) % 5], rlo, rhi);
            dlo[x] = clo[(x + 4) % 5] ^ rlo;
            dhi[x] = chi[(x + 4) % 5] ^ rhi;
        }
        uint32_t blo[25], bhi[25];
        kk::rho_pi_lane<0>(lo, hi, dlo, dhi, blo, bhi);
#pragma unroll
        for (int y = 0; y < 5; y++)
#pragma unroll
            for (int x = 0; x < 5; x++) {
                lo[x + 5 * y] = blo[x + 5 * y] ^ (~blo[(x + 1) % 5 + 5 * y] & blo[(x + 2) % 5 + 5 * y]);
                hi[x + 5 * y] = bhi[x + 5 * y] ^ (~bhi[(x + 1) % 5 + 5 * y] & bhi[(x + 2) % 5 + 5 * y]);
            }
        lo[0] ^= kk::kRC.lo[ir];
        hi[0] ^= kk::kRC.hi[ir];
    }
}

// The full 32-byte ADRS (eight big-endian words) from the compressed form
// (layer and type are below 256, the tree below 2^64).
__device__ __forceinline__ void adrs_words(const Adrs& a, uint32_t w[8]) {
    w[0] = a.w0 >> 24;
    w[1] = 0;
    w[2] = ((a.w0 & 0xFFFFFFu) << 8) | (a.w1 >> 24);
    w[3] = (a.w1 << 8) | (a.w2 >> 24);
    w[4] = (a.w2 >> 16) & 0xFFu;
    w[5] = (a.w2 << 16) | (a.w3 >> 16);
    w[6] = (a.w3 << 16) | (a.w4 >> 16);
    w[7] = (a.w4 << 16) | a.half;
}

constexpr int kRateWords = 34;     // 136-byte rate in 32-bit words

// SHAKE256(seed || ADRS || x, 8 * 4 NW) for payloads that fit one block
// (4 (NW + 8 + PW) + 1 <= 136 bytes): everything in registers.
template <int NW, int PW>
__device__ __forceinline__ void shake_thash1(const uint32_t* seed, const Adrs& a, const uint32_t* x, uint32_t* out) {
    constexpr int T = NW + 8 + PW;
    static_assert(T % 2 == 0 && 4 * T + 1 <= 136, "one SHAKE256 block");
    uint32_t w[T], ad[8];
    adrs_words(a, ad);
#pragma unroll
    for (int i = 0; i < NW; i++) w[i] = seed[i];
#pragma unroll
    for (int i = 0; i < 8; i++) w[NW + i] = ad[i];
#pragma unroll
    for (int i = 0; i < PW; i++) w[NW + 8 + i] = x[i];
    uint32_t lo[25], hi[25];
#pragma unroll
    for (int i = 0; i < 25; i++) {
        lo[i] = (2 * i < T) ? bswap32(w[2 * i]) : 0u;
        hi[i] = (2 * i + 1 < T) ? bswap32(w[2 * i + 1]) : 0u;
    }
    lo[T / 2] ^= 0x1Fu;            // domain bits 1111 and the first pad bit
    hi[16] ^= 0x80000000u;         // last pad bit: byte 135
    keccak_f1600(lo, hi);
#pragma unroll
    for (int i = 0; i < NW; i += 2) {
        out[i] = bswap32(lo[i / 2]);
        out[i + 1] = bswap32(hi[i / 2]);
    }
}

// Streaming SHAKE256(seed || ADRS || v_0 || ... || v_{l-1}, 8n) for T_l:
// the words are collected in a per-thread buffer (local memory; a few
// hundred bytes to 2.3 KB), then absorbed block by block through one
// permutation call site.  MAXW bounds the payload words.
template <int NW, int MAXW>
struct ShakeStream {
    static constexpr int CAP = ((NW + 8 + MAXW) * 4 + 1 + 135) / 136 * kRateWords;
    uint32_t buf[CAP];
    const uint32_t* seed;
    int pos;

    __device__ __forceinline__ void init(const uint32_t* sd, const Adrs& a) {
        seed = sd;
        uint32_t ad[8];
        adrs_words(a, ad);
#pragma unroll
        for (int i = 0; i < NW; i++) buf[i] = sd[i];
#pragma unroll
        for (int i = 0; i < 8; i++) buf[NW + i] = ad[i];
        pos = NW + 8;
    }
    template <int K>
    __device__ __forceinline__ void push_n(const uint32_t* v) {
#pragma unroll
        for (int i = 0; i < K; i++) buf[pos + i] = v[i];
        pos += K;
    }
    template <int K>
    __device__ __forceinline__ void finish(uint32_t /*payload_bytes*/, uint32_t* out) {
        const int total = pos;                        // words; a whole number of n-byte values
        const int nblk = (4 * total + 1 + 135) / 136;
        for (int i = total; i < nblk * kRateWords; i++) buf[i] = 0;
        buf[total] = 0x1F000000u;                     // byte 4 total (big-endian word order)
        buf[nblk * kRateWords - 1] |= 0x00000080u;    // byte 136 nblk - 1
        uint32_t lo[25], hi[25];
#pragma unroll
        for (int i = 0; i < 25; i++) lo[i] = hi[i] = 0;
#pragma unroll 1
        for (int b = 0; b < nblk; b++) {
            const uint32_t* p = buf + b * kRateWords;
#pragma unroll
            for (int i = 0; i < kRateWords / 2; i++) {
                lo[i] ^= bswap32(p[2 * i]);
                hi[i] ^= bswap32(p[2 * i + 1]);
            }
            keccak_f1600(lo, hi);
        }
#pragma unroll
        for (int i = 0; i < K; i += 2) {
            out[i] = bswap32(lo[i / 2]);
            out[i + 1] = bswap32(hi[i / 2]);
        }
    }
};

// Byte-granular SHAKE256 for the message stage: absorbs bytes (and whole
// 136-byte blocks straight from memory), squeezes up to 136 bytes.
struct ByteShake {
    uint32_t lo[25], hi[25];
    uint32_t blk[kRateWords];      // little-endian words of the open block
    uint32_t fill;

    __device__ void init() {
        for (int i = 0; i < 25; i++) lo[i] = hi[i] = 0;
        for (int i = 0; i < kRateWords; i++) blk[i] = 0;
        fill = 0;
    }
    __device__ void absorb_block(const uint32_t* w) {
#pragma unroll
        for (int i = 0; i < kRateWords / 2; i++) {
            lo[i] ^= w[2 * i];
            hi[i] ^= w[2 * i + 1];
        }
        keccak_f1600(lo, hi);
    }
    __device__ void byte(uint32_t b) {
        blk[fill >> 2] |= (b & 0xFFu) << (8 * (fill & 3));
        if (++fill == 136) {
            absorb_block(blk);
            for (int i = 0; i < kRateWords; i++) blk[i] = 0;
            fill = 0;
        }
    }
    // Append the low nb (1..4) bytes of the little-endian word w at any byte
    // offset; the caller keeps fill + nb <= 136 and absorbs a full block.
    __device__ __forceinline__ void put(uint32_t w, uint32_t nb) {
        if (nb < 4) w &= (1u << (8 * nb)) - 1u;
        const uint32_t s = 8 * (fill & 3), j = fill >> 2;
        blk[j] |= w << s;
        if (s + 8 * nb > 32) blk[j + 1] |= w >> (32 - s);
        fill += nb;
    }
    __device__ void flush_if_full() {
        if (fill == 136) {
            absorb_block(blk);
            for (int i = 0; i < kRateWords; i++) blk[i] = 0;
            fill = 0;
        }
    }
    __device__ void words(const uint32_t* w, int nbytes) {   // big-endian words
#pragma unroll 1
        for (int i = 0; i < nbytes; i += 4) {
            const uint32_t avail = nbytes - i < 4 ? (uint32_t)(nbytes - i) : 4u;
            const uint32_t room = 136u - fill;
            const uint32_t le = bswap32(w[i >> 2]);
            if (avail <= room) {
                put(le, avail);
            } else {                                  // the word straddles the block end
                put(le, room);
                flush_if_full();
                put(le >> (8 * room), avail - room);
            }
            flush_if_full();
        }
    }
    // r < 136 message bytes at q without crossing the end of the open block,
    // through aligned word loads issued together (each holds at least one
    // byte of q[0, r)).
    __device__ void append(const uint8_t* q, uint32_t r) {
        if (r == 0) return;
        const uintptr_t addr = reinterpret_cast<uintptr_t>(q);
        const uint32_t* a = reinterpret_cast<const uint32_t*>(addr & ~(uintptr_t)3);
        const uint32_t sh = (uint32_t)(addr & 3);
        const uint32_t nl = (sh + r + 3) >> 2;
        uint32_t raw[kRateWords + 1];
#pragma unroll
        for (int k = 0; k < kRateWords + 1; k++) raw[k] = ((uint32_t)k < nl) ? __ldg(a + k) : 0u;
#pragma unroll
        for (int k = 0; k < kRateWords; k++)
            if ((uint32_t)(4 * k) < r) put(__funnelshift_r(raw[k], raw[k + 1], 8 * sh), min(4u, r - 4u * k));
        flush_if_full();
    }
    // Whole blocks at any alignment, the next block's loads in flight during
    // this permutation.
    __device__ void blocks(const uint8_t* q, uint64_t nb) {
        const uintptr_t addr = reinterpret_cast<uintptr_t>(q);
        const uint32_t* a = reinterpret_cast<const uint32_t*>(addr & ~(uintptr_t)3);
        const uint32_t sh = (uint32_t)(addr & 3);
        uint32_t raw[kRateWords + 1];
#pragma unroll
        for (int k = 0; k < kRateWords; k++) raw[k] = __ldg(a + k);
        raw[kRateWords] = sh ? __ldg(a + kRateWords) : 0u;
        for (uint64_t b = 0; b < nb; b++) {
            uint32_t w[kRateWords];
#pragma unroll
            for (int k = 0; k < kRateWords; k++) w[k] = __funnelshift_r(raw[k], raw[k + 1], 8 * sh);
            if (b + 1 < nb) {
                const uint32_t* an = a + (b + 1) * kRateWords;
#pragma unroll
                for (int k = 0; k < kRateWords; k++) raw[k] = __ldg(an + k);
                raw[kRateWords] = sh ? __ldg(an + kRateWords) : 0u;
            }
            absorb_block(w);
        }
    }
    __device__ void mem(const uint8_t* p, uint64_t len) {
        uint64_t i = 0;
        if (fill != 0 && len != 0) {
            i = (136u - fill < len) ? 136u - fill : len;
            append(p, (uint32_t)i);
        }
        const uint64_t nb = (len - i) / 136;
        if (nb) {
            blocks(p + i, nb);
            i += nb * 136;
        }
        if (i < len) append(p + i, (uint32_t)(len - i));
    }
    // Pad and squeeze nbytes (<= 136) as big-endian words into out.
    __device__ void finish(uint32_t* out, int nbytes) {
        blk[fill >> 2] ^= 0x1Fu << (8 * (fill & 3));
        blk[kRateWords - 1] ^= 0x80000000u;
        absorb_block(blk);
        for (int i = 0; i < (nbytes + 3) / 4; i++) {
            const uint32_t v = (i & 1) ? hi[i / 2] : lo[i / 2];
            out[i] = bswap32(v);
        }
    }
};

}  // namespace hs
