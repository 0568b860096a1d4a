// sha2.cuh -- register-resident SHA-256 / SHA-512 compression for sm_103a.
//
// FIPS 180-4 compression functions, written for the 32-bit integer pipes:
//  * rotations are funnel shifts (__funnelshift_r -> SHF with both sources
//    equal), 64-bit rotations are pairs of 32-bit funnel shifts;
//  * byte swaps of big-endian words use prmt (__byte_perm), the same
//    instruction choice the paper makes for its SHA-2 loads (Sec. III-C);
//  * the message schedule lives in a 16-word ring, so with the rounds
//    unrolled every index is static and everything stays in registers.
// sha256_compress_full unrolls all 64 rounds (constant-folds known-zero
// message words; used for the hot F / PRF calls).  The *_rolled variants
// unroll 16 rounds and loop, keeping code size small for the rarer calls.
#pragma once
#include <cstdint>

namespace hs {

__device__ __forceinline__ uint32_t rotr32(uint32_t x, int r) { return __funnelshift_r(x, x, r); }
__device__ __forceinline__ uint32_t bswap32(uint32_t x) { return __byte_perm(x, 0, 0x0123); }
// (hi << 16) | (lo >> 16): the word straddling two big-endian words at a
// 2-byte offset (every payload of a 22-byte compressed address).
__device__ __forceinline__ uint32_t mid16(uint32_t hi, uint32_t lo) { return __byte_perm(lo, hi, 0x5432); }

#define HS_K256_LIST                                                                          \
    0x428a2f98u, 0x71374491u, 0xb5c0fbcfu, 0xe9b5dba5u, 0x3956c25bu, 0x59f111f1u, 0x923f82a4u, \
    0xab1c5ed5u, 0xd807aa98u, 0x12835b01u, 0x243185beu, 0x550c7dc3u, 0x72be5d74u, 0x80deb1feu, \
    0x9bdc06a7u, 0xc19bf174u, 0xe49b69c1u, 0xefbe4786u, 0x0fc19dc6u, 0x240ca1ccu, 0x2de92c6fu, \
    0x4a7484aau, 0x5cb0a9dcu, 0x76f988dau, 0x983e5152u, 0xa831c66du, 0xb00327c8u, 0xbf597fc7u, \
    0xc6e00bf3u, 0xd5a79147u, 0x06ca6351u, 0x14292967u, 0x27b70a85u, 0x2e1b2138u, 0x4d2c6dfcu, \
    0x53380d13u, 0x650a7354u, 0x766a0abbu, 0x81c2c92eu, 0x92722c85u, 0xa2bfe8a1u, 0xa81a664bu, \
    0xc24b8b70u, 0xc76c51a3u, 0xd192e819u, 0xd6990624u, 0xf40e3585u, 0x106aa070u, 0x19a4c116u, \
    0x1e376c08u, 0x2748774cu, 0x34b0bcb5u, 0x391c0cb3u, 0x4ed8aa4au, 0x5b9cca4fu, 0x682e6ff3u, \
    0x748f82eeu, 0x78a5636fu, 0x84c87814u, 0x8cc70208u, 0x90befffau, 0xa4506cebu, 0xbef9a3f7u, \
    0xc67178f2u

static __constant__ uint32_t c_K256[64] = {HS_K256_LIST};

static __constant__ uint64_t c_K512[80] = {
    0x428a2f98d728ae22ull, 0x7137449123ef65cdull, 0xb5c0fbcfec4d3b2full, 0xe9b5dba58189dbbcull,
    0x3956c25bf348b538ull, 0x59f111f1b605d019ull, 0x923f82a4af194f9bull, 0xab1c5ed5da6d8118ull,
    0xd807aa98a3030242ull, 0x12835b0145706fbeull, 0x243185be4ee4b28cull, 0x550c7dc3d5ffb4e2ull,
    0x72be5d74f27b896full, 0x80deb1fe3b1696b1ull, 0x9bdc06a725c71235ull, 0xc19bf174cf692694ull,
    0xe49b69c19ef14ad2ull, 0xefbe4786384f25e3ull, 0x0fc19dc68b8cd5b5ull, 0x240ca1cc77ac9c65ull,
    0x2de92c6f592b0275ull, 0x4a7484aa6ea6e483ull, 0x5cb0a9dcbd41fbd4ull, 0x76f988da831153b5ull,
    0x983e5152ee66dfabull, 0xa831c66d2db43210ull, 0xb00327c898fb213full, 0xbf597fc7beef0ee4ull,
    0xc6e00bf33da88fc2ull, 0xd5a79147930aa725ull, 0x06ca6351e003826full, 0x142929670a0e6e70ull,
    0x27b70a8546d22ffcull, 0x2e1b21385c26c926ull, 0x4d2c6dfc5ac42aedull, 0x53380d139d95b3dfull,
    0x650a73548baf63deull, 0x766a0abb3c77b2a8ull, 0x81c2c92e47edaee6ull, 0x92722c851482353bull,
    0xa2bfe8a14cf10364ull, 0xa81a664bbc423001ull, 0xc24b8b70d0f89791ull, 0xc76c51a30654be30ull,
    0xd192e819d6ef5218ull, 0xd69906245565a910ull, 0xf40e35855771202aull, 0x106aa07032bbd1b8ull,
    0x19a4c116b8d2d0c8ull, 0x1e376c085141ab53ull, 0x2748774cdf8eeb99ull, 0x34b0bcb5e19b48a8ull,
    0x391c0cb3c5c95a63ull, 0x4ed8aa4ae3418acbull, 0x5b9cca4f7763e373ull, 0x682e6ff3d6b2b8a3ull,
    0x748f82ee5defb2fcull, 0x78a5636f43172f60ull, 0x84c87814a1f0ab72ull, 0x8cc702081a6439ecull,
    0x90befffa23631e28ull, 0xa4506cebde82bde9ull, 0xbef9a3f7b2c67915ull, 0xc67178f2e372532bull,
    0xca273eceea26619cull, 0xd186b8c721c0c207ull, 0xeada7dd6cde0eb1eull, 0xf57d4f7fee6ed178ull,
    0x06f067aa72176fbaull, 0x0a637dc5a2c898a6ull, 0x113f9804bef90daeull, 0x1b710b35131c471bull,
    0x28db77f523047d84ull, 0x32caab7b40c72493ull, 0x3c9ebe0a15c9bebcull, 0x431d67c49c100d4cull,
    0x4cc5d4becb3e42b6ull, 0x597f299cfc657e2aull, 0x5fcb6fab3ad6faecull, 0x6c44198c4a475817ull};

__device__ __forceinline__ void sha256_iv(uint32_t s[8]) {
    s[0] = 0x6a09e667u; s[1] = 0xbb67ae85u; s[2] = 0x3c6ef372u; s[3] = 0xa54ff53au;
    s[4] = 0x510e527fu; s[5] = 0x9b05688cu; s[6] = 0x1f83d9abu; s[7] = 0x5be0cd19u;
}
__device__ __forceinline__ void sha512_iv(uint64_t s[8]) {
    s[0] = 0x6a09e667f3bcc908ull; s[1] = 0xbb67ae8584caa73bull; s[2] = 0x3c6ef372fe94f82bull;
    s[3] = 0xa54ff53a5f1d36f1ull; s[4] = 0x510e527fade682d1ull; s[5] = 0x9b05688c2b3e6c1full;
    s[6] = 0x1f83d9abfb41bd6bull; s[7] = 0x5be0cd19137e2179ull;
}

// ---------------------------------------------------------------- SHA-256

__device__ __forceinline__ uint32_t S0_256(uint32_t a) { return rotr32(a, 2) ^ rotr32(a, 13) ^ rotr32(a, 22); }
__device__ __forceinline__ uint32_t S1_256(uint32_t e) { return rotr32(e, 6) ^ rotr32(e, 11) ^ rotr32(e, 25); }
__device__ __forceinline__ uint32_t s0_256(uint32_t w) { return rotr32(w, 7) ^ rotr32(w, 18) ^ (w >> 3); }
__device__ __forceinline__ uint32_t s1_256(uint32_t w) { return rotr32(w, 17) ^ rotr32(w, 19) ^ (w >> 10); }
__device__ __forceinline__ uint32_t ch32(uint32_t e, uint32_t f, uint32_t g) { return (e & f) ^ (~e & g); }
__device__ __forceinline__ uint32_t maj32(uint32_t a, uint32_t b, uint32_t c) { return (a & b) | (c & (a | b)); }

// One round; the state rotation is renaming, free once unrolled.
#define HS_R256(a, b, c, d, e, f, g, h, k, w)                  \
    do {                                                       \
        uint32_t t1_ = h + S1_256(e) + ch32(e, f, g) + (k) + (w); \
        uint32_t t2_ = S0_256(a) + maj32(a, b, c);             \
        d += t1_;                                              \
        h = t1_ + t2_;                                         \
    } while (0)

// Full compression, all 64 rounds unrolled; W is consumed (ring-extended).
// st += compress(st, W) (feed-forward included).
__device__ __forceinline__ void sha256_compress_full(uint32_t st[8], uint32_t W[16]) {
    constexpr uint32_t K[64] = {HS_K256_LIST};
    uint32_t a = st[0], b = st[1], c = st[2], d = st[3], e = st[4], f = st[5], g = st[6], h = st[7];
#pragma unroll
    for (int t = 0; t < 64; t += 8) {
        if (t >= 16) {
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int i = t + j;
                W[i & 15] += s1_256(W[(i - 2) & 15]) + W[(i - 7) & 15] + s0_256(W[(i - 15) & 15]);
            }
        }
        HS_R256(a, b, c, d, e, f, g, h, K[t + 0], W[(t + 0) & 15]);
        HS_R256(h, a, b, c, d, e, f, g, K[t + 1], W[(t + 1) & 15]);
        HS_R256(g, h, a, b, c, d, e, f, K[t + 2], W[(t + 2) & 15]);
        HS_R256(f, g, h, a, b, c, d, e, K[t + 3], W[(t + 3) & 15]);
        HS_R256(e, f, g, h, a, b, c, d, K[t + 4], W[(t + 4) & 15]);
        HS_R256(d, e, f, g, h, a, b, c, K[t + 5], W[(t + 5) & 15]);
        HS_R256(c, d, e, f, g, h, a, b, K[t + 6], W[(t + 6) & 15]);
        HS_R256(b, c, d, e, f, g, h, a, K[t + 7], W[(t + 7) & 15]);
    }
    st[0] += a; st[1] += b; st[2] += c; st[3] += d; st[4] += e; st[5] += f; st[6] += g; st[7] += h;
}

// Same function, 16 rounds unrolled inside a loop of 4 (K from constant memory).
__device__ __forceinline__ void sha256_compress_rolled(uint32_t st[8], uint32_t W[16]) {
    uint32_t a = st[0], b = st[1], c = st[2], d = st[3], e = st[4], f = st[5], g = st[6], h = st[7];
#pragma unroll 1
    for (int t = 0; t < 64; t += 16) {
        if (t > 0) {
#pragma unroll
            for (int i = 0; i < 16; i++)
                W[i] += s1_256(W[(i + 14) & 15]) + W[(i + 9) & 15] + s0_256(W[(i + 1) & 15]);
        }
#pragma unroll
        for (int j = 0; j < 16; j += 8) {
            HS_R256(a, b, c, d, e, f, g, h, c_K256[t + j + 0], W[j + 0]);
            HS_R256(h, a, b, c, d, e, f, g, c_K256[t + j + 1], W[j + 1]);
            HS_R256(g, h, a, b, c, d, e, f, c_K256[t + j + 2], W[j + 2]);
            HS_R256(f, g, h, a, b, c, d, e, c_K256[t + j + 3], W[j + 3]);
            HS_R256(e, f, g, h, a, b, c, d, c_K256[t + j + 4], W[j + 4]);
            HS_R256(d, e, f, g, h, a, b, c, c_K256[t + j + 5], W[j + 5]);
            HS_R256(c, d, e, f, g, h, a, b, c_K256[t + j + 6], W[j + 6]);
            HS_R256(b, c, d, e, f, g, h, a, c_K256[t + j + 7], W[j + 7]);
        }
    }
    st[0] += a; st[1] += b; st[2] += c; st[3] += d; st[4] += e; st[5] += f; st[6] += g; st[7] += h;
}
#undef HS_R256

// ---------------------------------------------------------------- SHA-512

// 64-bit rotate right by a compile-time r as two 32-bit funnel shifts.
__device__ __forceinline__ uint64_t rotr64(uint64_t x, int r) {
    const uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
    uint32_t nlo, nhi;
    if (r < 32) { nlo = __funnelshift_r(lo, hi, r); nhi = __funnelshift_r(hi, lo, r); }
    else        { nlo = __funnelshift_r(hi, lo, r - 32); nhi = __funnelshift_r(lo, hi, r - 32); }
    return ((uint64_t)nhi << 32) | nlo;
}
__device__ __forceinline__ uint64_t shr64(uint64_t x, int s) {   // s < 32
    const uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
    return ((uint64_t)(hi >> s) << 32) | __funnelshift_r(lo, hi, s);
}
__device__ __forceinline__ uint64_t S0_512(uint64_t a) { return rotr64(a, 28) ^ rotr64(a, 34) ^ rotr64(a, 39); }
__device__ __forceinline__ uint64_t S1_512(uint64_t e) { return rotr64(e, 14) ^ rotr64(e, 18) ^ rotr64(e, 41); }
__device__ __forceinline__ uint64_t s0_512(uint64_t w) { return rotr64(w, 1) ^ rotr64(w, 8) ^ shr64(w, 7); }
__device__ __forceinline__ uint64_t s1_512(uint64_t w) { return rotr64(w, 19) ^ rotr64(w, 61) ^ shr64(w, 6); }

#define HS_R512(a, b, c, d, e, f, g, h, k, w)                                  \
    do {                                                                       \
        uint64_t t1_ = h + S1_512(e) + ((e & f) ^ (~e & g)) + (k) + (w);       \
        uint64_t t2_ = S0_512(a) + ((a & b) | (c & (a | b)));                  \
        d += t1_;                                                              \
        h = t1_ + t2_;                                                         \
    } while (0)

// st += compress(st, W); W (16 x 64-bit) is consumed.  16 rounds unrolled
// inside a loop of 5 (K from constant memory).
__device__ __forceinline__ void sha512_compress(uint64_t st[8], uint64_t W[16]) {
    uint64_t a = st[0], b = st[1], c = st[2], d = st[3], e = st[4], f = st[5], g = st[6], h = st[7];
#pragma unroll 1
    for (int t = 0; t < 80; t += 16) {
        if (t > 0) {
#pragma unroll
            for (int i = 0; i < 16; i++)
                W[i] += s1_512(W[(i + 14) & 15]) + W[(i + 9) & 15] + s0_512(W[(i + 1) & 15]);
        }
#pragma unroll
        for (int j = 0; j < 16; j += 8) {
            HS_R512(a, b, c, d, e, f, g, h, c_K512[t + j + 0], W[j + 0]);
            HS_R512(h, a, b, c, d, e, f, g, c_K512[t + j + 1], W[j + 1]);
            HS_R512(g, h, a, b, c, d, e, f, c_K512[t + j + 2], W[j + 2]);
            HS_R512(f, g, h, a, b, c, d, e, c_K512[t + j + 3], W[j + 3]);
            HS_R512(e, f, g, h, a, b, c, d, c_K512[t + j + 4], W[j + 4]);
            HS_R512(d, e, f, g, h, a, b, c, c_K512[t + j + 5], W[j + 5]);
            HS_R512(c, d, e, f, g, h, a, b, c_K512[t + j + 6], W[j + 6]);
            HS_R512(b, c, d, e, f, g, h, a, c_K512[t + j + 7], W[j + 7]);
        }
    }
    st[0] += a; st[1] += b; st[2] += c; st[3] += d; st[4] += e; st[5] += f; st[6] += g; st[7] += h;
}
#undef HS_R512

// SHA-512 block given as 32 big-endian 32-bit words (hi, lo per 64-bit word).
__device__ __forceinline__ void sha512_compress_w32(uint64_t st[8], const uint32_t blk[32]) {
    uint64_t W[16];
#pragma unroll
    for (int i = 0; i < 16; i++) W[i] = ((uint64_t)blk[2 * i] << 32) | blk[2 * i + 1];
    sha512_compress(st, W);
}

}  // namespace hs
