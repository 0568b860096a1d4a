/*
 * spx_oracle.c -- plain, slow, obviously-correct CPU SPHINCS+ (SHA2-simple).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness oracle for the GPU
 * signer.  Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline
 * leg (and its --impl reference arm) may load or call it.  It shares no
 * source with the CUDA path under paper_2512_23969_gb300/csrc and never
 * includes any of its headers.
 *
 * What it computes.  HERO-Sign (arxiv 2512.23969) signs with SPHINCS+ at the
 * -f parameter sets of its Table 1 (128f/192f/256f) and paraphrases the scheme
 * in Sec. II-A (WOTS+, FORS, MSS, hypertree) and in the signing listing of
 * Fig. 2 (hash_message -> message_to_indices -> fors_sign -> d x merkle_sign,
 * with leaf_idx = tree & (2^h' - 1); tree >>= h').  The paper cites, but does
 * not restate, the byte-level scheme; it is taken here from the SPHINCS+
 * round-3.1 specification with the SHA2 "simple" tweakable hashes:
 *   F, PRF               : SHA-256 always
 *   H, T_l, H_msg, PRF_msg: SHA-256 at n = 16, SHA-512 at n = 24 / 32
 *   deterministic signing: opt_rand = PK.seed
 * Each point the paper leaves open is decided where it is used, in a comment
 * marked "READING" that states the reading taken.
 *
 * Style.  Every function follows its definition directly: whole SHA-2 over a
 * fully assembled input (no midstates), recursive Merkle node() with no
 * caching, and separately written verify climbs.  Nothing here is tuned.
 *
 * SHAKE instantiation (parameter id + 32; a variant): every tweakable hash
 * is SHAKE256(PK.seed || ADRS || payload, 8n) with the full 32-byte ADRS,
 * PRF_msg = SHAKE256(SK.prf || opt_rand || M, 8n) and
 * H_msg = SHAKE256(R || PK.seed || PK.root || M, 8m) (SPHINCS+ round 3.1
 * SHAKE-simple; FIPS 205 Sec. 11.1).  Keccak-f[1600] is written from
 * FIPS 202 Sec. 3: round constants come from its LFSR (Algorithm 5) and the
 * rotation offsets from its (x, y) walk (Algorithm 2), not from tables.
 *
 * Robust instantiation (parameter id + 64; a variant): SPHINCS+ round 3.1's
 * robust SHA2 tweakable hashes, which mask the inputs of F, H and T_l with
 * MGF1 output seeded by PK.seed and the address (thash_masked).
 *
 * FIPS 205 mode (parameter id + 16): SLH-DSA's two departures from the
 * round-3.1 scheme, stated in FIPS 205 -- the FORS indices are the base-2^a
 * digits of md read most significant bit first (its base_2b), and the pure
 * signing interface signs M' = 0x00 || len(ctx) || ctx || M (oracle_slh_*).
 * Keys, hashes, addresses and sizes are the same at these three sets.
 *
 * Parity status: every exported function is pinned by tests/test_oracle_*.py
 * (hashlib/hmac for SHA-2, hand-derived byte layouts and digits, closed-form
 * sizes and call counts from the paper, sign/verify/tamper invariants and a
 * brute-force toy hypertree).  External bit-level parity against published
 * SPHINCS+ known-answer files is NOT pinned: none are available here.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <stdlib.h>

#define SPX_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* Parameter sets (paper Table 1; len, m and sizes derived from the scheme)  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n;      /* hash output bytes                                 */
    int h;      /* hypertree height                                  */
    int d;      /* hypertree layers                                  */
    int hp;     /* h' = h / d, XMSS tree height                       */
    int a;      /* FORS tree height log(t)                            */
    int k;      /* FORS trees                                         */
    int w;      /* Winternitz parameter (16)                          */
    int big;    /* 1: H, T_l, H_msg, PRF_msg use SHA-512              */
    int len1, len2, len;
    int md_bytes, tree_bytes, leaf_bytes, m;
    int tree_bits, leaf_bits;
    int fips;   /* 1: FORS indices in FIPS 205 order (MSB first)        */
    int shake;  /* 1: SHAKE256 tweakable hashes instead of SHA-2         */
    int robust; /* 1: robust SHA2 tweakable hashes (inputs masked)       */
    size_t fors_bytes, sig_bytes;
} spx_params;

/* ids: 0 = 128f, 1 = 192f, 2 = 256f, 3 = toy (n=16,h=4,d=2,h'=2,a=3,k=4),
 * 4 = 128s, 5 = 192s, 6 = 256s (the scheme's small-signature sets, a
 * variant the paper does not use); + 16 = the same set in FIPS 205 mode,
 * + 32 = its SHAKE instantiation, + 64 = its robust SHA2 instantiation
 * (round 3.1 only: not with FIPS 205 mode or SHAKE) */
static int params_init(int id, spx_params *p)
{
    memset(p, 0, sizeof(*p));
    if (id < 0 || id > 127) return -1;
    p->fips = (id >> 4) & 1;
    p->shake = (id >> 5) & 1;
    p->robust = (id >> 6) & 1;
    if (p->robust && (p->fips || p->shake)) return -1;
    switch (id & 15) {
    case 0: p->n = 16; p->h = 66; p->d = 22; p->a = 6; p->k = 33; break;
    case 1: p->n = 24; p->h = 66; p->d = 22; p->a = 8; p->k = 33; break;
    case 2: p->n = 32; p->h = 68; p->d = 17; p->a = 9; p->k = 35; break;
    case 3: p->n = 16; p->h = 4;  p->d = 2;  p->a = 3; p->k = 4;  break;
    case 4: p->n = 16; p->h = 63; p->d = 7;  p->a = 12; p->k = 14; break;
    case 5: p->n = 24; p->h = 63; p->d = 7;  p->a = 14; p->k = 17; break;
    case 6: p->n = 32; p->h = 64; p->d = 8;  p->a = 14; p->k = 22; break;
    default: return -1;
    }
    p->w = 16;
    p->hp = p->h / p->d;
    p->big = (p->n > 16);
    /* len1 = ceil(8n / log2 w); len2 = floor(log2(len1 (w-1)) / log2 w) + 1 */
    p->len1 = (8 * p->n) / 4;
    {
        int v = p->len1 * (p->w - 1), lg = 0;
        while ((1 << (lg + 1)) <= v) lg++;          /* floor(log2 v) */
        p->len2 = lg / 4 + 1;
    }
    p->len = p->len1 + p->len2;
    p->tree_bits = p->h - p->hp;
    p->leaf_bits = p->hp;
    p->md_bytes = (p->k * p->a + 7) / 8;
    p->tree_bytes = (p->tree_bits + 7) / 8;
    p->leaf_bytes = (p->leaf_bits + 7) / 8;
    p->m = p->md_bytes + p->tree_bytes + p->leaf_bytes;
    p->fors_bytes = (size_t)p->k * (p->a + 1) * p->n;
    p->sig_bytes = (size_t)p->n + p->fors_bytes
                 + (size_t)(p->h + p->d * p->len) * p->n;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* SHA-256 / SHA-512 (FIPS 180-4), whole-message, byte oriented              */
/* ------------------------------------------------------------------------ */

static const uint32_t K256[64] = {
    0x428a2f98u, 0x71374491u, 0xb5c0fbcfu, 0xe9b5dba5u, 0x3956c25bu, 0x59f111f1u, 0x923f82a4u, 0xab1c5ed5u,
    0xd807aa98u, 0x12835b01u, 0x243185beu, 0x550c7dc3u, 0x72be5d74u, 0x80deb1feu, 0x9bdc06a7u, 0xc19bf174u,
    0xe49b69c1u, 0xefbe4786u, 0x0fc19dc6u, 0x240ca1ccu, 0x2de92c6fu, 0x4a7484aau, 0x5cb0a9dcu, 0x76f988dau,
    0x983e5152u, 0xa831c66du, 0xb00327c8u, 0xbf597fc7u, 0xc6e00bf3u, 0xd5a79147u, 0x06ca6351u, 0x14292967u,
    0x27b70a85u, 0x2e1b2138u, 0x4d2c6dfcu, 0x53380d13u, 0x650a7354u, 0x766a0abbu, 0x81c2c92eu, 0x92722c85u,
    0xa2bfe8a1u, 0xa81a664bu, 0xc24b8b70u, 0xc76c51a3u, 0xd192e819u, 0xd6990624u, 0xf40e3585u, 0x106aa070u,
    0x19a4c116u, 0x1e376c08u, 0x2748774cu, 0x34b0bcb5u, 0x391c0cb3u, 0x4ed8aa4au, 0x5b9cca4fu, 0x682e6ff3u,
    0x748f82eeu, 0x78a5636fu, 0x84c87814u, 0x8cc70208u, 0x90befffau, 0xa4506cebu, 0xbef9a3f7u, 0xc67178f2u
};
static const uint32_t IV256[8] = {
    0x6a09e667u, 0xbb67ae85u, 0x3c6ef372u, 0xa54ff53au, 0x510e527fu, 0x9b05688cu, 0x1f83d9abu, 0x5be0cd19u
};
static const uint64_t K512[80] = {
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
    0x4cc5d4becb3e42b6ull, 0x597f299cfc657e2aull, 0x5fcb6fab3ad6faecull, 0x6c44198c4a475817ull
};
static const uint64_t IV512[8] = {
    0x6a09e667f3bcc908ull, 0xbb67ae8584caa73bull, 0x3c6ef372fe94f82bull, 0xa54ff53a5f1d36f1ull,
    0x510e527fade682d1ull, 0x9b05688c2b3e6c1full, 0x1f83d9abfb41bd6bull, 0x5be0cd19137e2179ull
};

static uint32_t ror32(uint32_t x, int r) { return (x >> r) | (x << (32 - r)); }
static uint64_t ror64(uint64_t x, int r) { return (x >> r) | (x << (64 - r)); }

/* FIPS 180-4 Sec. 6.2.2: one SHA-256 block, schedule then 64 rounds. */
static void sha256_block(uint32_t H[8], const uint8_t blk[64])
{
    uint32_t W[64], a, b, c, d, e, f, g, h;
    int t;
    for (t = 0; t < 16; t++)
        W[t] = ((uint32_t)blk[4 * t] << 24) | ((uint32_t)blk[4 * t + 1] << 16)
             | ((uint32_t)blk[4 * t + 2] << 8) | (uint32_t)blk[4 * t + 3];
    for (t = 16; t < 64; t++) {
        uint32_t s0 = ror32(W[t - 15], 7) ^ ror32(W[t - 15], 18) ^ (W[t - 15] >> 3);
        uint32_t s1 = ror32(W[t - 2], 17) ^ ror32(W[t - 2], 19) ^ (W[t - 2] >> 10);
        W[t] = s1 + W[t - 7] + s0 + W[t - 16];
    }
    a = H[0]; b = H[1]; c = H[2]; d = H[3]; e = H[4]; f = H[5]; g = H[6]; h = H[7];
    for (t = 0; t < 64; t++) {
        uint32_t S1 = ror32(e, 6) ^ ror32(e, 11) ^ ror32(e, 25);
        uint32_t ch = (e & f) ^ (~e & g);
        uint32_t T1 = h + S1 + ch + K256[t] + W[t];
        uint32_t S0 = ror32(a, 2) ^ ror32(a, 13) ^ ror32(a, 22);
        uint32_t mj = (a & b) ^ (a & c) ^ (b & c);
        uint32_t T2 = S0 + mj;
        h = g; g = f; f = e; e = d + T1; d = c; c = b; b = a; a = T1 + T2;
    }
    H[0] += a; H[1] += b; H[2] += c; H[3] += d; H[4] += e; H[5] += f; H[6] += g; H[7] += h;
}

/* FIPS 180-4 Sec. 6.4.2: one SHA-512 block, schedule then 80 rounds. */
static void sha512_block(uint64_t H[8], const uint8_t blk[128])
{
    uint64_t W[80], a, b, c, d, e, f, g, h;
    int t, i;
    for (t = 0; t < 16; t++) {
        W[t] = 0;
        for (i = 0; i < 8; i++) W[t] = (W[t] << 8) | blk[8 * t + i];
    }
    for (t = 16; t < 80; t++) {
        uint64_t s0 = ror64(W[t - 15], 1) ^ ror64(W[t - 15], 8) ^ (W[t - 15] >> 7);
        uint64_t s1 = ror64(W[t - 2], 19) ^ ror64(W[t - 2], 61) ^ (W[t - 2] >> 6);
        W[t] = s1 + W[t - 7] + s0 + W[t - 16];
    }
    a = H[0]; b = H[1]; c = H[2]; d = H[3]; e = H[4]; f = H[5]; g = H[6]; h = H[7];
    for (t = 0; t < 80; t++) {
        uint64_t S1 = ror64(e, 14) ^ ror64(e, 18) ^ ror64(e, 41);
        uint64_t ch = (e & f) ^ (~e & g);
        uint64_t T1 = h + S1 + ch + K512[t] + W[t];
        uint64_t S0 = ror64(a, 28) ^ ror64(a, 34) ^ ror64(a, 39);
        uint64_t mj = (a & b) ^ (a & c) ^ (b & c);
        uint64_t T2 = S0 + mj;
        h = g; g = f; f = e; e = d + T1; d = c; c = b; b = a; a = T1 + T2;
    }
    H[0] += a; H[1] += b; H[2] += c; H[3] += d; H[4] += e; H[5] += f; H[6] += g; H[7] += h;
}

/* Per-thread call counters (instrumentation for structure-count tests). */
static _Thread_local uint64_t g_c256_blocks, g_c512_blocks, g_calls_f, g_calls_prf,
                              g_calls_h, g_calls_t, g_keccak_perms;

/* SHA-256 of a whole message: full blocks straight from the input, then the
 * padded tail (0x80, zeros, 64-bit big-endian bit length; FIPS 180-4 5.1.1). */
static void sha256(const uint8_t *msg, size_t len, uint8_t out[32])
{
    uint32_t H[8];
    uint8_t tail[128];
    size_t full = len / 64, rem = len % 64, tl, i;
    uint64_t bits = (uint64_t)len * 8;
    memcpy(H, IV256, sizeof(H));
    for (i = 0; i < full; i++) { sha256_block(H, msg + 64 * i); g_c256_blocks++; }
    memset(tail, 0, sizeof(tail));
    memcpy(tail, msg + 64 * full, rem);
    tail[rem] = 0x80;
    tl = (rem + 1 + 8 <= 64) ? 64 : 128;
    for (i = 0; i < 8; i++) tail[tl - 1 - i] = (uint8_t)(bits >> (8 * i));
    for (i = 0; i < tl; i += 64) { sha256_block(H, tail + i); g_c256_blocks++; }
    for (i = 0; i < 8; i++) {
        out[4 * i] = (uint8_t)(H[i] >> 24); out[4 * i + 1] = (uint8_t)(H[i] >> 16);
        out[4 * i + 2] = (uint8_t)(H[i] >> 8); out[4 * i + 3] = (uint8_t)H[i];
    }
}

/* SHA-512 of a whole message (FIPS 180-4 5.1.2: 128-bit length field). */
static void sha512(const uint8_t *msg, size_t len, uint8_t out[64])
{
    uint64_t H[8];
    uint8_t tail[256];
    size_t full = len / 128, rem = len % 128, tl, i;
    uint64_t bits = (uint64_t)len * 8;
    int j;
    memcpy(H, IV512, sizeof(H));
    for (i = 0; i < full; i++) { sha512_block(H, msg + 128 * i); g_c512_blocks++; }
    memset(tail, 0, sizeof(tail));
    memcpy(tail, msg + 128 * full, rem);
    tail[rem] = 0x80;
    tl = (rem + 1 + 16 <= 128) ? 128 : 256;
    /* high 64 bits of the 128-bit length are zero for any size_t length < 2^61 */
    for (i = 0; i < 8; i++) tail[tl - 1 - i] = (uint8_t)(bits >> (8 * i));
    for (i = 0; i < tl; i += 128) { sha512_block(H, tail + i); g_c512_blocks++; }
    for (i = 0; i < 8; i++)
        for (j = 0; j < 8; j++) out[8 * i + j] = (uint8_t)(H[i] >> (56 - 8 * j));
}

/* SHA-x selected by 'big' (0: SHA-256, 32-byte out; 1: SHA-512, 64-byte out). */
static void shax(int big, const uint8_t *msg, size_t len, uint8_t *out)
{
    if (big) sha512(msg, len, out); else sha256(msg, len, out);
}

/* Concatenate up to four byte strings into 'buf' (cap bytes), return length. */
static size_t cat4(uint8_t *buf, size_t cap,
                   const uint8_t *p0, size_t l0, const uint8_t *p1, size_t l1,
                   const uint8_t *p2, size_t l2, const uint8_t *p3, size_t l3)
{
    size_t off = 0;
    if (l0 + l1 + l2 + l3 > cap) return (size_t)-1;
    if (l0) { memcpy(buf + off, p0, l0); off += l0; }
    if (l1) { memcpy(buf + off, p1, l1); off += l1; }
    if (l2) { memcpy(buf + off, p2, l2); off += l2; }
    if (l3) { memcpy(buf + off, p3, l3); off += l3; }
    return off;
}

/* HMAC (RFC 2104) with SHA-x; key shorter than the block, as n <= 32 here.
 * 'text' is the concatenation t0 || t1 (so messages need not be copied). */
static void hmac_shax(int big, const uint8_t *key, size_t keylen,
                      const uint8_t *t0, size_t l0, const uint8_t *t1, size_t l1,
                      uint8_t *out)
{
    size_t B = big ? 128 : 64, D = big ? 64 : 32, i;
    uint8_t kpad[128], inner[64];
    uint8_t *buf = (uint8_t *)malloc(B + l0 + l1 + 1);
    uint8_t obuf[128 + 64];
    memset(kpad, 0, sizeof(kpad));
    memcpy(kpad, key, keylen);
    for (i = 0; i < B; i++) buf[i] = kpad[i] ^ 0x36;
    if (l0) memcpy(buf + B, t0, l0);
    if (l1) memcpy(buf + B + l0, t1, l1);
    shax(big, buf, B + l0 + l1, inner);
    free(buf);
    for (i = 0; i < B; i++) obuf[i] = kpad[i] ^ 0x5c;
    memcpy(obuf + B, inner, D);
    shax(big, obuf, B + D, out);
}

/* MGF1 (RFC 8017 B.2.1) with SHA-x: T = H(seed||BE32(0)) || H(seed||BE32(1)) ... */
static void mgf1_shax(int big, const uint8_t *seed, size_t seedlen, uint8_t *out, size_t outlen)
{
    size_t D = big ? 64 : 32, done = 0;
    uint32_t c = 0;
    uint8_t buf[256], dig[64];
    while (done < outlen) {
        size_t take;
        memcpy(buf, seed, seedlen);
        buf[seedlen] = (uint8_t)(c >> 24); buf[seedlen + 1] = (uint8_t)(c >> 16);
        buf[seedlen + 2] = (uint8_t)(c >> 8); buf[seedlen + 3] = (uint8_t)c;
        shax(big, buf, seedlen + 4, dig);
        take = (outlen - done < D) ? outlen - done : D;
        memcpy(out + done, dig, take);
        done += take;
        c++;
    }
}

/* ------------------------------------------------------------------------ */
/* Keccak-f[1600] and SHAKE256 (FIPS 202)                                    */
/* ------------------------------------------------------------------------ */

static uint64_t rotl64(uint64_t x, int r)
{
    r &= 63;
    return r ? (x << r) | (x >> (64 - r)) : x;
}

/* rc(t) of FIPS 202 Algorithm 5: the output bit of an 8-bit LFSR. */
static int keccak_rc(int t)
{
    uint32_t R = 1;   /* R = 10000000 with bit 0 first */
    int i;
    if (t % 255 == 0) return 1;
    for (i = 1; i <= t % 255; i++) {
        uint32_t b8;
        R <<= 1;                              /* R = 0 || R */
        b8 = (R >> 8) & 1;
        R ^= b8 | (b8 << 4) | (b8 << 5) | (b8 << 6);   /* R[0,4,5,6] ^= R[8] */
        R &= 0xFF;
    }
    return (int)(R & 1);
}

/* Round constants and rotation offsets, derived once per thread by the
 * definitions above (not typed in). */
static _Thread_local int g_keccak_ready;
static _Thread_local uint64_t g_keccak_rc[24];
static _Thread_local int g_keccak_off[25];

static void keccak_tables(void)
{
    int x, y, t, ir, j;
    /* rho offsets: (x, y) walks from (1, 0); lane t is rotated by (t+1)(t+2)/2 */
    g_keccak_off[0] = 0;
    x = 1; y = 0;
    for (t = 0; t < 24; t++) {
        int nx = y, ny = (2 * x + 3 * y) % 5;
        g_keccak_off[x + 5 * y] = ((t + 1) * (t + 2) / 2) % 64;
        x = nx; y = ny;
    }
    /* iota: bit 2^j - 1 of RC[ir] is rc(j + 7 ir) */
    for (ir = 0; ir < 24; ir++) {
        g_keccak_rc[ir] = 0;
        for (j = 0; j <= 6; j++)
            if (keccak_rc(j + 7 * ir)) g_keccak_rc[ir] |= (uint64_t)1 << ((1 << j) - 1);
    }
    g_keccak_ready = 1;
}

/* A[x + 5 y], lanes as little-endian 64-bit integers. */
static void keccak_f1600(uint64_t A[25])
{
    int x, y, ir;
    const int *off = g_keccak_off;
    if (!g_keccak_ready) keccak_tables();
    for (ir = 0; ir < 24; ir++) {
        uint64_t C[5], D[5], B[25];
        for (x = 0; x < 5; x++) C[x] = A[x] ^ A[x + 5] ^ A[x + 10] ^ A[x + 15] ^ A[x + 20];
        for (x = 0; x < 5; x++) D[x] = C[(x + 4) % 5] ^ rotl64(C[(x + 1) % 5], 1);
        for (x = 0; x < 5; x++)
            for (y = 0; y < 5; y++) A[x + 5 * y] ^= D[x];
        /* rho then pi: B[x, y] = rot(A[(x + 3y) mod 5, x]) */
        for (x = 0; x < 5; x++)
            for (y = 0; y < 5; y++) {
                int sx = (x + 3 * y) % 5, sy = x;
                B[x + 5 * y] = rotl64(A[sx + 5 * sy], off[sx + 5 * sy]);
            }
        /* chi */
        for (x = 0; x < 5; x++)
            for (y = 0; y < 5; y++)
                A[x + 5 * y] = B[x + 5 * y] ^ (~B[(x + 1) % 5 + 5 * y] & B[(x + 2) % 5 + 5 * y]);
        A[0] ^= g_keccak_rc[ir];   /* iota */
    }
    g_keccak_perms++;
}

/* SHAKE256(M, 8 outlen): rate 136 bytes, domain bits 1111 then pad10*1. */
static void shake256(const uint8_t *in, size_t inlen, uint8_t *out, size_t outlen)
{
    uint64_t A[25];
    const size_t rate = 136;
    size_t i, off = 0;
    memset(A, 0, sizeof(A));
    for (;;) {
        size_t take = inlen - off < rate ? inlen - off : rate;
        for (i = 0; i < take; i++) A[i / 8] ^= (uint64_t)in[off + i] << (8 * (i % 8));
        off += take;
        if (take < rate) {
            A[take / 8] ^= (uint64_t)0x1F << (8 * (take % 8));
            A[(rate - 1) / 8] ^= (uint64_t)0x80 << (8 * ((rate - 1) % 8));
            keccak_f1600(A);
            break;
        }
        keccak_f1600(A);
    }
    for (off = 0;;) {
        size_t take = outlen - off < rate ? outlen - off : rate;
        for (i = 0; i < take; i++) out[off + i] = (uint8_t)(A[i / 8] >> (8 * (i % 8)));
        off += take;
        if (off == outlen) break;
        keccak_f1600(A);
    }
}

/* ------------------------------------------------------------------------ */
/* ADRS (32-byte address) and its 22-byte compressed form ADRSc             */
/* ------------------------------------------------------------------------ */

enum { ADDR_WOTS_HASH = 0, ADDR_WOTS_PK = 1, ADDR_TREE = 2, ADDR_FORS_TREE = 3,
       ADDR_FORS_ROOTS = 4, ADDR_WOTS_PRF = 5, ADDR_FORS_PRF = 6 };

/* Words: 0 layer | 1..3 tree (96-bit, word 1 always 0) | 4 type | 5,6,7.
 * Word 5 = keypair, word 6 = chain or tree height, word 7 = hash or tree index. */
typedef struct { uint32_t w[8]; } adrs_t;

static void adrs_zero(adrs_t *A) { memset(A, 0, sizeof(*A)); }
static void adrs_set_layer(adrs_t *A, uint32_t l) { A->w[0] = l; }
static void adrs_set_tree(adrs_t *A, uint64_t t)
{ A->w[1] = 0; A->w[2] = (uint32_t)(t >> 32); A->w[3] = (uint32_t)t; }
/* Changing the type clears the three type-specific words. */
static void adrs_set_type(adrs_t *A, uint32_t ty) { A->w[4] = ty; A->w[5] = A->w[6] = A->w[7] = 0; }
static void adrs_set_keypair(adrs_t *A, uint32_t kp) { A->w[5] = kp; }
static void adrs_set_chain(adrs_t *A, uint32_t c) { A->w[6] = c; }
static void adrs_set_hash(adrs_t *A, uint32_t q) { A->w[7] = q; }
static void adrs_set_height(adrs_t *A, uint32_t z) { A->w[6] = z; }
static void adrs_set_index(adrs_t *A, uint32_t i) { A->w[7] = i; }

static void put_be32(uint8_t *p, uint32_t v)
{ p[0] = (uint8_t)(v >> 24); p[1] = (uint8_t)(v >> 16); p[2] = (uint8_t)(v >> 8); p[3] = (uint8_t)v; }

/* ADRSc = low byte of layer || low 8 bytes of tree || low byte of type ||
 *         word 5 || word 6 || word 7   (all big-endian; 1+8+1+12 = 22 bytes) */
static void adrs_compress(const adrs_t *A, uint8_t out[22])
{
    out[0] = (uint8_t)A->w[0];
    put_be32(out + 1, A->w[2]);
    put_be32(out + 5, A->w[3]);
    out[9] = (uint8_t)A->w[4];
    put_be32(out + 10, A->w[5]);
    put_be32(out + 14, A->w[6]);
    put_be32(out + 18, A->w[7]);
}

/* The full 32-byte ADRS: the eight words big-endian. */
static void adrs_full(const adrs_t *A, uint8_t out[32])
{
    int i;
    for (i = 0; i < 8; i++) put_be32(out + 4 * i, A->w[i]);
}

/* ------------------------------------------------------------------------ */
/* Keys and tweakable hashes                                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    spx_params p;
    uint8_t sk_seed[32], sk_prf[32], pk_seed[32], pk_root[32];
} spx_ctx;

/* Tweakable hash, SHA2-simple: Trunc_n(SHA-x(BlockPad_x(PK.seed) || ADRSc || in)),
 * BlockPad_x = PK.seed followed by zero bytes up to the SHA-x block size. */
static void thash(const spx_ctx *c, int big, const adrs_t *A,
                  const uint8_t *in, size_t inlen, uint8_t *out)
{
    size_t B = big ? 128 : 64;
    if (c->p.shake) {
        /* SHAKE-simple: SHAKE256(PK.seed || ADRS || in, 8n) */
        size_t n = (size_t)c->p.n;
        uint8_t *sb = (uint8_t *)malloc(n + 32 + inlen);
        memcpy(sb, c->pk_seed, n);
        adrs_full(A, sb + n);
        memcpy(sb + n + 32, in, inlen);
        shake256(sb, n + 32 + inlen, out, n);
        free(sb);
        return;
    }
    uint8_t *buf = (uint8_t *)malloc(B + 22 + inlen);
    uint8_t dig[64];
    memset(buf, 0, B);
    memcpy(buf, c->pk_seed, c->p.n);
    adrs_compress(A, buf + B);
    memcpy(buf + B + 22, in, inlen);
    shax(big, buf, B + 22 + inlen, dig);
    free(buf);
    memcpy(out, dig, c->p.n);
}

/* READING (robust instantiation, a variant; the paper signs with the
 * simple one): SPHINCS+ round 3.1's robust SHA2 tweakable hashes F, H and
 * T_l hash M xor MGF1-SHA-x(PK.seed || ADRSc, |M|) in place of M, where
 * SHA-x is the hash that tweakable hash itself uses (SHA-256 for F; SHA-512
 * for H and T_l at n = 24 / 32) and the mask seed is PK.seed unpadded,
 * followed by the 22-byte compressed address.  PRF, PRF_msg and H_msg are
 * the same as in the simple instantiation. */
static void thash_masked(const spx_ctx *c, int big, const adrs_t *A,
                         const uint8_t *in, size_t inlen, uint8_t *out)
{
    uint8_t *x, seed[32 + 22];
    size_t i, n = (size_t)c->p.n;
    if (!c->p.robust) {
        thash(c, big, A, in, inlen, out);
        return;
    }
    x = (uint8_t *)malloc(inlen);
    memcpy(seed, c->pk_seed, n);
    adrs_compress(A, seed + n);
    mgf1_shax(big, seed, n + 22, x, inlen);     /* the mask */
    for (i = 0; i < inlen; i++) x[i] ^= in[i];
    thash(c, big, A, x, inlen, out);
    free(x);
}

/* F: chain step / FORS leaf; always SHA-256, one n-byte block. */
static void hash_F(const spx_ctx *c, const adrs_t *A, const uint8_t *in, uint8_t *out)
{ g_calls_f++; thash_masked(c, 0, A, in, c->p.n, out); }

/* H: Merkle parent of two n-byte children; SHA-512 when n > 16. */
static void hash_H(const spx_ctx *c, const adrs_t *A, const uint8_t *l, const uint8_t *r, uint8_t *out)
{
    uint8_t buf[64];
    g_calls_h++;
    memcpy(buf, l, c->p.n);
    memcpy(buf + c->p.n, r, c->p.n);
    thash_masked(c, c->p.big, A, buf, 2 * (size_t)c->p.n, out);
}

/* T_l: compress l n-byte values (WOTS public key, FORS roots). */
static void hash_T(const spx_ctx *c, const adrs_t *A, const uint8_t *in, int l, uint8_t *out)
{ g_calls_t++; thash_masked(c, c->p.big, A, in, (size_t)l * c->p.n, out); }

/* PRF: secret value for an address; SHA-256 over SK.seed. */
static void prf_addr(const spx_ctx *c, const adrs_t *A, uint8_t *out)
{ g_calls_prf++; thash(c, 0, A, c->sk_seed, c->p.n, out); }

/* PRF_msg(SK.prf, opt_rand, M) = Trunc_n(HMAC-SHA-x(SK.prf, opt_rand || M)). */
static void prf_msg(const spx_ctx *c, const uint8_t *opt, const uint8_t *m, size_t mlen, uint8_t *R)
{
    uint8_t mac[64];
    if (c->p.shake) {   /* SHAKE256(SK.prf || opt_rand || M, 8n) */
        size_t n = (size_t)c->p.n;
        uint8_t *sb = (uint8_t *)malloc(2 * n + mlen + 1);
        memcpy(sb, c->sk_prf, n);
        memcpy(sb + n, opt, n);
        if (mlen) memcpy(sb + 2 * n, m, mlen);
        shake256(sb, 2 * n + mlen, R, n);
        free(sb);
        return;
    }
    hmac_shax(c->p.big, c->sk_prf, c->p.n, opt, c->p.n, m, mlen, mac);
    memcpy(R, mac, c->p.n);
}

/* H_msg(R, PK.seed, PK.root, M)
 *   = MGF1-SHA-x(R || PK.seed || SHA-x(R || PK.seed || PK.root || M), m bytes). */
static void hash_msg(const spx_ctx *c, const uint8_t *R, const uint8_t *m, size_t mlen, uint8_t *digest)
{
    int n = c->p.n, big = c->p.big;
    size_t D = big ? 64 : 32;
    uint8_t *buf = (uint8_t *)malloc(3 * (size_t)n + mlen + 1);
    uint8_t inner[64], seed[32 + 32 + 64];
    size_t off = cat4(buf, 3 * (size_t)n + mlen + 1, R, n, c->pk_seed, n, c->pk_root, n, m, mlen);
    if (c->p.shake) {   /* SHAKE256(R || PK.seed || PK.root || M, 8m) */
        shake256(buf, off, digest, (size_t)c->p.m);
        free(buf);
        return;
    }
    shax(big, buf, off, inner);
    free(buf);
    off = cat4(seed, sizeof(seed), R, n, c->pk_seed, n, inner, D, NULL, 0);
    mgf1_shax(big, seed, off, digest, c->p.m);
}

/* ------------------------------------------------------------------------ */
/* Digest split and base-w (paper Fig. 2: message_to_indices, leaf/tree idx)  */
/* ------------------------------------------------------------------------ */

/* READING (FORS index bit order): the md bytes are read as one little-endian
 * bit stream -- stream bit q is bit (q mod 8) of byte q/8 -- and FORS index i
 * is built from stream bits i*a .. i*a+a-1, the first bit read becoming the
 * least significant bit (the SPHINCS+ round-3 lineage the paper's identifiers
 * come from).  The paper names the step only. */
static void message_to_indices(const spx_params *p, const uint8_t *md, uint32_t *idx)
{
    int i, j, q = 0;
    if (p->fips) {
        /* FIPS 205 base_2b(md, a, k): bytes enter an accumulator from the
         * left; each digit is the top a bits not yet used. */
        uint64_t acc = 0;
        int have = 0, in = 0;
        for (i = 0; i < p->k; i++) {
            while (have < p->a) {
                acc = (acc << 8) | md[in++];
                have += 8;
            }
            have -= p->a;
            idx[i] = (uint32_t)((acc >> have) & (((uint64_t)1 << p->a) - 1));
        }
        return;
    }
    for (i = 0; i < p->k; i++) {
        idx[i] = 0;
        for (j = 0; j < p->a; j++, q++)
            idx[i] |= (uint32_t)((md[q / 8] >> (q % 8)) & 1) << j;
    }
}

static uint64_t be_bytes_to_u64(const uint8_t *b, int nbytes)
{
    uint64_t v = 0;
    int i;
    for (i = 0; i < nbytes; i++) v = (v << 8) | b[i];
    return v;
}

/* digest = md || tree bytes || leaf bytes; idx_tree keeps h - h' low bits,
 * idx_leaf keeps h' low bits (big-endian integers). */
static void split_digest(const spx_params *p, const uint8_t *digest,
                         uint32_t *fors_idx, uint64_t *idx_tree, uint32_t *idx_leaf)
{
    uint64_t t = be_bytes_to_u64(digest + p->md_bytes, p->tree_bytes);
    uint64_t l = be_bytes_to_u64(digest + p->md_bytes + p->tree_bytes, p->leaf_bytes);
    if (p->tree_bits < 64) t &= ((uint64_t)1 << p->tree_bits) - 1;
    l &= ((uint64_t)1 << p->leaf_bits) - 1;
    *idx_tree = t;
    *idx_leaf = (uint32_t)l;
    message_to_indices(p, digest, fors_idx);
}

/* base_w (w = 16): each byte gives its high nibble, then its low nibble. */
static void base_w16(const uint8_t *x, int outlen, int *digits)
{
    int i;
    for (i = 0; i < outlen; i++)
        digits[i] = (i % 2 == 0) ? (x[i / 2] >> 4) : (x[i / 2] & 15);
}

/* WOTS+ digits of an n-byte message: len1 message digits followed by len2
 * checksum digits.  csum = sum(w-1-d_i), shifted left by (8 - (len2*4) % 8) % 8
 * bits, written as ceil(len2*4/8) big-endian bytes and split with base_w. */
static void wots_digits(const spx_params *p, const uint8_t *msg, int *digits)
{
    uint32_t csum = 0;
    uint8_t cb[4];
    int i, nbytes = (p->len2 * 4 + 7) / 8;
    base_w16(msg, p->len1, digits);
    for (i = 0; i < p->len1; i++) csum += (uint32_t)(p->w - 1 - digits[i]);
    csum <<= (8 - (p->len2 * 4) % 8) % 8;
    for (i = 0; i < nbytes; i++) cb[i] = (uint8_t)(csum >> (8 * (nbytes - 1 - i)));
    base_w16(cb, p->len2, digits + p->len1);
}

/* ------------------------------------------------------------------------ */
/* WOTS+ (paper Sec. II-A-1)                                                 */
/* ------------------------------------------------------------------------ */

/* chain(X, s, t): t applications of F, step q using WOTS_HASH with hash = q.
 * 'A' carries layer, tree, keypair and chain already. */
static void wots_chain(const spx_ctx *c, adrs_t *A, const uint8_t *in, int start, int steps, uint8_t *out)
{
    int q;
    uint8_t tmp[32];
    memcpy(tmp, in, c->p.n);
    for (q = start; q < start + steps; q++) {
        adrs_set_hash(A, (uint32_t)q);
        hash_F(c, A, tmp, tmp);
    }
    memcpy(out, tmp, c->p.n);
}

/* Secret start of chain i of keypair kp: PRF(WOTS_PRF(layer,tree,kp,chain=i,hash=0)). */
static void wots_sk(const spx_ctx *c, uint32_t layer, uint64_t tree, uint32_t kp, int i, uint8_t *out)
{
    adrs_t A;
    adrs_zero(&A);
    adrs_set_layer(&A, layer);
    adrs_set_tree(&A, tree);
    adrs_set_type(&A, ADDR_WOTS_PRF);
    adrs_set_keypair(&A, kp);
    adrs_set_chain(&A, (uint32_t)i);
    adrs_set_hash(&A, 0);
    prf_addr(c, &A, out);
}

static void wots_hash_adrs(adrs_t *A, uint32_t layer, uint64_t tree, uint32_t kp, int i)
{
    adrs_zero(A);
    adrs_set_layer(A, layer);
    adrs_set_tree(A, tree);
    adrs_set_type(A, ADDR_WOTS_HASH);
    adrs_set_keypair(A, kp);
    adrs_set_chain(A, (uint32_t)i);
}

/* Compress the len chain ends with T_len under WOTS_PK(layer,tree,kp). */
static void wots_pk_compress(const spx_ctx *c, uint32_t layer, uint64_t tree, uint32_t kp,
                             const uint8_t *ends, uint8_t *pk)
{
    adrs_t A;
    adrs_zero(&A);
    adrs_set_layer(&A, layer);
    adrs_set_tree(&A, tree);
    adrs_set_type(&A, ADDR_WOTS_PK);
    adrs_set_keypair(&A, kp);
    hash_T(c, &A, ends, c->p.len, pk);
}

/* WOTS public key of keypair kp = the hypertree leaf value: every chain from
 * its secret start to position w-1, then T_len. */
static void wots_pkgen(const spx_ctx *c, uint32_t layer, uint64_t tree, uint32_t kp, uint8_t *pk)
{
    int i, n = c->p.n;
    uint8_t *ends = (uint8_t *)malloc((size_t)c->p.len * n), sk[32];
    adrs_t A;
    for (i = 0; i < c->p.len; i++) {
        wots_sk(c, layer, tree, kp, i, sk);
        wots_hash_adrs(&A, layer, tree, kp, i);
        wots_chain(c, &A, sk, 0, c->p.w - 1, ends + (size_t)i * n);
    }
    wots_pk_compress(c, layer, tree, kp, ends, pk);
    free(ends);
}

/* WOTS signature of an n-byte message: chain i advanced to its digit. */
static void wots_sign(const spx_ctx *c, const uint8_t *msg, uint32_t layer, uint64_t tree,
                      uint32_t kp, uint8_t *sig)
{
    int digits[80], i, n = c->p.n;
    uint8_t sk[32];
    adrs_t A;
    wots_digits(&c->p, msg, digits);
    for (i = 0; i < c->p.len; i++) {
        wots_sk(c, layer, tree, kp, i, sk);
        wots_hash_adrs(&A, layer, tree, kp, i);
        wots_chain(c, &A, sk, 0, digits[i], sig + (size_t)i * n);
    }
}

/* Public key recomputed from a signature: chain i from digit to w-1. */
static void wots_pk_from_sig(const spx_ctx *c, const uint8_t *sig, const uint8_t *msg,
                             uint32_t layer, uint64_t tree, uint32_t kp, uint8_t *pk)
{
    int digits[80], i, n = c->p.n;
    uint8_t *ends = (uint8_t *)malloc((size_t)c->p.len * n);
    adrs_t A;
    wots_digits(&c->p, msg, digits);
    for (i = 0; i < c->p.len; i++) {
        wots_hash_adrs(&A, layer, tree, kp, i);
        wots_chain(c, &A, sig + (size_t)i * n, digits[i], c->p.w - 1 - digits[i], ends + (size_t)i * n);
    }
    wots_pk_compress(c, layer, tree, kp, ends, pk);
    free(ends);
}

/* ------------------------------------------------------------------------ */
/* XMSS / MSS trees of the hypertree (paper Sec. II-A-3, II-A-4)             */
/* ------------------------------------------------------------------------ */

/* node(i, z) of tree 'tree' at layer 'layer', by its recursive definition:
 * height 0 is the WOTS public key of keypair i; above, H under
 * TREE(height z, index i) of the two children. */
static void xmss_node(const spx_ctx *c, uint32_t layer, uint64_t tree, uint32_t i, int z, uint8_t *out)
{
    uint8_t l[32], r[32];
    adrs_t A;
    if (z == 0) { wots_pkgen(c, layer, tree, i, out); return; }
    xmss_node(c, layer, tree, 2 * i, z - 1, l);
    xmss_node(c, layer, tree, 2 * i + 1, z - 1, r);
    adrs_zero(&A);
    adrs_set_layer(&A, layer);
    adrs_set_tree(&A, tree);
    adrs_set_type(&A, ADDR_TREE);
    adrs_set_height(&A, (uint32_t)z);
    adrs_set_index(&A, i);
    hash_H(c, &A, l, r, out);
}

/* XMSS signature: WOTS signature of msg under keypair 'leaf', then the auth
 * path auth_z = node((leaf >> z) xor 1, z), z = 0..h'-1.  Also returns the
 * tree root node(0, h'). */
static void xmss_sign(const spx_ctx *c, const uint8_t *msg, uint32_t layer, uint64_t tree,
                      uint32_t leaf, uint8_t *sig, uint8_t *root)
{
    int z, n = c->p.n;
    uint8_t *auth = sig + (size_t)c->p.len * n;
    wots_sign(c, msg, layer, tree, leaf, sig);
    for (z = 0; z < c->p.hp; z++)
        xmss_node(c, layer, tree, (leaf >> z) ^ 1u, z, auth + (size_t)z * n);
    xmss_node(c, layer, tree, 0, c->p.hp, root);
}

/* Root from an XMSS signature: leaf = WOTS pk from sig, then climb: at step
 * z the node index is leaf >> z; an even index is a left child. */
static void xmss_root_from_sig(const spx_ctx *c, const uint8_t *sig, const uint8_t *msg,
                               uint32_t layer, uint64_t tree, uint32_t leaf, uint8_t *root)
{
    int z, n = c->p.n;
    const uint8_t *auth = sig + (size_t)c->p.len * n;
    uint8_t node[32];
    adrs_t A;
    wots_pk_from_sig(c, sig, msg, layer, tree, leaf, node);
    for (z = 0; z < c->p.hp; z++) {
        uint32_t idx = leaf >> z;
        adrs_zero(&A);
        adrs_set_layer(&A, layer);
        adrs_set_tree(&A, tree);
        adrs_set_type(&A, ADDR_TREE);
        adrs_set_height(&A, (uint32_t)z + 1);
        adrs_set_index(&A, idx >> 1);
        if ((idx & 1) == 0) hash_H(c, &A, node, auth + (size_t)z * n, node);
        else                hash_H(c, &A, auth + (size_t)z * n, node, node);
    }
    memcpy(root, node, n);
}

/* ------------------------------------------------------------------------ */
/* FORS (paper Sec. II-A-2)                                                  */
/* ------------------------------------------------------------------------ */

/* FORS addresses live at layer 0, tree idx_tree, keypair idx_leaf. */
static void fors_base_adrs(adrs_t *A, uint64_t idx_tree, uint32_t idx_leaf, uint32_t type)
{
    adrs_zero(A);
    adrs_set_layer(A, 0);
    adrs_set_tree(A, idx_tree);
    adrs_set_type(A, type);
    adrs_set_keypair(A, idx_leaf);
}

/* FORS secret of global leaf index g = i*2^a + j: PRF(FORS_PRF(index g)). */
static void fors_sk(const spx_ctx *c, uint64_t idx_tree, uint32_t idx_leaf, uint32_t g, uint8_t *out)
{
    adrs_t A;
    fors_base_adrs(&A, idx_tree, idx_leaf, ADDR_FORS_PRF);
    adrs_set_height(&A, 0);
    adrs_set_index(&A, g);
    prf_addr(c, &A, out);
}

/* FORS node at height z with global index g (= i*2^(a-z) + j): leaves are
 * F(FORS_TREE(height 0, index g), sk_g); above, H of the two children under
 * FORS_TREE(height z, index g). */
static void fors_node(const spx_ctx *c, uint64_t idx_tree, uint32_t idx_leaf, uint32_t g, int z, uint8_t *out)
{
    adrs_t A;
    uint8_t l[32], r[32];
    if (z == 0) {
        uint8_t sk[32];
        fors_sk(c, idx_tree, idx_leaf, g, sk);
        fors_base_adrs(&A, idx_tree, idx_leaf, ADDR_FORS_TREE);
        adrs_set_height(&A, 0);
        adrs_set_index(&A, g);
        hash_F(c, &A, sk, out);
        return;
    }
    fors_node(c, idx_tree, idx_leaf, 2 * g, z - 1, l);
    fors_node(c, idx_tree, idx_leaf, 2 * g + 1, z - 1, r);
    fors_base_adrs(&A, idx_tree, idx_leaf, ADDR_FORS_TREE);
    adrs_set_height(&A, (uint32_t)z);
    adrs_set_index(&A, g);
    hash_H(c, &A, l, r, out);
}

/* FORS signature: for tree i, sk of leaf idx_i then the a auth nodes
 * node(((i*2^a + idx_i) >> z) xor 1, z).  PK_FORS = T_k(FORS_ROOTS, roots). */
static void fors_sign(const spx_ctx *c, const uint32_t *fidx, uint64_t idx_tree, uint32_t idx_leaf,
                      uint8_t *sig, uint8_t *pk_fors)
{
    int i, z, n = c->p.n, a = c->p.a;
    uint8_t *roots = (uint8_t *)malloc((size_t)c->p.k * n);
    adrs_t A;
    for (i = 0; i < c->p.k; i++) {
        uint32_t g = ((uint32_t)i << a) + fidx[i];
        uint8_t *s = sig + (size_t)i * (a + 1) * n;
        fors_sk(c, idx_tree, idx_leaf, g, s);
        for (z = 0; z < a; z++)
            fors_node(c, idx_tree, idx_leaf, (g >> z) ^ 1u, z, s + (size_t)(z + 1) * n);
        fors_node(c, idx_tree, idx_leaf, (uint32_t)i, a, roots + (size_t)i * n);
    }
    fors_base_adrs(&A, idx_tree, idx_leaf, ADDR_FORS_ROOTS);
    hash_T(c, &A, roots, c->p.k, pk_fors);
    free(roots);
}

/* PK_FORS from a FORS signature: per tree, leaf from sk, climb with auth. */
static void fors_pk_from_sig(const spx_ctx *c, const uint8_t *sig, const uint32_t *fidx,
                             uint64_t idx_tree, uint32_t idx_leaf, uint8_t *pk_fors)
{
    int i, z, n = c->p.n, a = c->p.a;
    uint8_t *roots = (uint8_t *)malloc((size_t)c->p.k * n), node[32];
    adrs_t A;
    for (i = 0; i < c->p.k; i++) {
        const uint8_t *s = sig + (size_t)i * (a + 1) * n;
        uint32_t g = ((uint32_t)i << a) + fidx[i];
        fors_base_adrs(&A, idx_tree, idx_leaf, ADDR_FORS_TREE);
        adrs_set_height(&A, 0);
        adrs_set_index(&A, g);
        hash_F(c, &A, s, node);
        for (z = 0; z < a; z++) {
            uint32_t gz = g >> z;
            const uint8_t *au = s + (size_t)(z + 1) * n;
            fors_base_adrs(&A, idx_tree, idx_leaf, ADDR_FORS_TREE);
            adrs_set_height(&A, (uint32_t)z + 1);
            adrs_set_index(&A, gz >> 1);
            if ((gz & 1) == 0) hash_H(c, &A, node, au, node);
            else               hash_H(c, &A, au, node, node);
        }
        memcpy(roots + (size_t)i * n, node, n);
    }
    fors_base_adrs(&A, idx_tree, idx_leaf, ADDR_FORS_ROOTS);
    hash_T(c, &A, roots, c->p.k, pk_fors);
    free(roots);
}

/* ------------------------------------------------------------------------ */
/* Key generation, signing, verification                                     */
/* ------------------------------------------------------------------------ */

static int ctx_from_sk(int pid, const uint8_t *sk, spx_ctx *c)
{
    int n;
    if (params_init(pid, &c->p)) return -1;
    n = c->p.n;
    memcpy(c->sk_seed, sk, n);
    memcpy(c->sk_prf, sk + n, n);
    memcpy(c->pk_seed, sk + 2 * n, n);
    memcpy(c->pk_root, sk + 3 * n, n);
    return 0;
}

/* Hypertree signing given the digest fields (the loop of paper Fig. 2):
 * layer j signs the previous root with keypair leaf of tree 'tree', then
 * leaf = tree mod 2^h', tree >>= h'. */
static void ht_sign(const spx_ctx *c, const uint8_t *pk_fors, uint64_t idx_tree, uint32_t idx_leaf, uint8_t *sig)
{
    int j, n = c->p.n;
    uint8_t root[32];
    uint64_t tree = idx_tree;
    uint32_t leaf = idx_leaf;
    memcpy(root, pk_fors, n);
    for (j = 0; j < c->p.d; j++) {
        uint8_t next[32];
        xmss_sign(c, root, (uint32_t)j, tree, leaf, sig, next);
        memcpy(root, next, n);
        sig += (size_t)(c->p.len + c->p.hp) * n;
        leaf = (uint32_t)(tree & (((uint64_t)1 << c->p.hp) - 1));
        tree >>= c->p.hp;
    }
}

/* Signing from explicit digest fields (R given); used by sign() and by the
 * brute-force tests that enumerate every (idx_tree, idx_leaf). */
static void sign_fields(const spx_ctx *c, const uint8_t *R, const uint32_t *fidx,
                        uint64_t idx_tree, uint32_t idx_leaf, uint8_t *sig)
{
    uint8_t pk_fors[32];
    memcpy(sig, R, c->p.n);
    fors_sign(c, fidx, idx_tree, idx_leaf, sig + c->p.n, pk_fors);
    ht_sign(c, pk_fors, idx_tree, idx_leaf, sig + c->p.n + c->p.fors_bytes);
}

/* ------------------------------------------------------------------------ */
/* Exported C ABI (ctypes)                                                   */
/* ------------------------------------------------------------------------ */

/* info[0..15] = n,h,d,hp,a,k,w,big,len1,len2,len,md_bytes,tree_bytes,leaf_bytes,m,sig_bytes */
SPX_EXPORT int oracle_params(int pid, int64_t *info)
{
    spx_params p;
    if (params_init(pid, &p)) return -1;
    info[0] = p.n; info[1] = p.h; info[2] = p.d; info[3] = p.hp; info[4] = p.a; info[5] = p.k;
    info[6] = p.w; info[7] = p.big; info[8] = p.len1; info[9] = p.len2; info[10] = p.len;
    info[11] = p.md_bytes; info[12] = p.tree_bytes; info[13] = p.leaf_bytes; info[14] = p.m;
    info[15] = (int64_t)p.sig_bytes;
    return 0;
}

SPX_EXPORT void oracle_sha256(const uint8_t *m, size_t len, uint8_t *out) { sha256(m, len, out); }
SPX_EXPORT void oracle_sha512(const uint8_t *m, size_t len, uint8_t *out) { sha512(m, len, out); }
SPX_EXPORT void oracle_shake256(const uint8_t *m, size_t len, uint8_t *out, size_t outlen)
{ shake256(m, len, out, outlen); }
SPX_EXPORT void oracle_keccak_f1600(uint64_t *state25) { keccak_f1600(state25); }
SPX_EXPORT void oracle_hmac(int big, const uint8_t *key, size_t keylen, const uint8_t *m, size_t len, uint8_t *out)
{ hmac_shax(big, key, keylen, m, len, NULL, 0, out); }
SPX_EXPORT void oracle_mgf1(int big, const uint8_t *seed, size_t seedlen, uint8_t *out, size_t outlen)
{ mgf1_shax(big, seed, seedlen, out, outlen); }
SPX_EXPORT void oracle_sha_tables(uint32_t *k256, uint32_t *iv256, uint64_t *k512, uint64_t *iv512)
{ memcpy(k256, K256, sizeof(K256)); memcpy(iv256, IV256, sizeof(IV256));
  memcpy(k512, K512, sizeof(K512)); memcpy(iv512, IV512, sizeof(IV512)); }

SPX_EXPORT void oracle_adrs_compress(const uint32_t *words8, uint8_t *out22)
{ adrs_t A; memcpy(A.w, words8, sizeof(A.w)); adrs_compress(&A, out22); }

/* which: 0 = F, 1 = H (in = 2n bytes), 2 = T_l (in = l*n bytes), 3 = PRF (in = SK.seed) */
SPX_EXPORT int oracle_thash(int pid, int which, const uint8_t *pk_seed, const uint8_t *sk_seed,
                            const uint32_t *words8, const uint8_t *in, int l, uint8_t *out)
{
    spx_ctx c;
    adrs_t A;
    memset(&c, 0, sizeof(c));
    if (params_init(pid, &c.p)) return -1;
    memcpy(c.pk_seed, pk_seed, c.p.n);
    if (sk_seed) memcpy(c.sk_seed, sk_seed, c.p.n);
    memcpy(A.w, words8, sizeof(A.w));
    switch (which) {
    case 0: hash_F(&c, &A, in, out); break;
    case 1: hash_H(&c, &A, in, in + c.p.n, out); break;
    case 2: hash_T(&c, &A, in, l, out); break;
    case 3: prf_addr(&c, &A, out); break;
    default: return -1;
    }
    return 0;
}

SPX_EXPORT int oracle_wots_digits(int pid, const uint8_t *msg, int32_t *digits)
{
    spx_params p;
    int d[80], i;
    if (params_init(pid, &p)) return -1;
    wots_digits(&p, msg, d);
    for (i = 0; i < p.len; i++) digits[i] = d[i];
    return 0;
}

/* Digest fields of a message under sk: R, digest, FORS indices, idx_tree, idx_leaf. */
SPX_EXPORT int oracle_hash_message(int pid, const uint8_t *sk, const uint8_t *m, size_t mlen,
                                   uint8_t *R, uint8_t *digest, uint32_t *fidx,
                                   uint64_t *idx_tree, uint32_t *idx_leaf)
{
    spx_ctx c;
    if (ctx_from_sk(pid, sk, &c)) return -1;
    prf_msg(&c, c.pk_seed, m, mlen, R);
    hash_msg(&c, R, m, mlen, digest);
    split_digest(&c.p, digest, fidx, idx_tree, idx_leaf);
    return 0;
}

SPX_EXPORT int oracle_split_digest(int pid, const uint8_t *digest, uint32_t *fidx,
                                   uint64_t *idx_tree, uint32_t *idx_leaf)
{
    spx_params p;
    if (params_init(pid, &p)) return -1;
    split_digest(&p, digest, fidx, idx_tree, idx_leaf);
    return 0;
}

SPX_EXPORT int oracle_wots_chain(int pid, const uint8_t *sk, uint32_t layer, uint64_t tree, uint32_t kp,
                                 int chain, const uint8_t *in, int start, int steps, uint8_t *out)
{
    spx_ctx c;
    adrs_t A;
    if (ctx_from_sk(pid, sk, &c)) return -1;
    wots_hash_adrs(&A, layer, tree, kp, chain);
    wots_chain(&c, &A, in, start, steps, out);
    return 0;
}

SPX_EXPORT int oracle_wots_sk(int pid, const uint8_t *sk, uint32_t layer, uint64_t tree, uint32_t kp,
                              int chain, uint8_t *out)
{
    spx_ctx c;
    if (ctx_from_sk(pid, sk, &c)) return -1;
    wots_sk(&c, layer, tree, kp, chain, out);
    return 0;
}

SPX_EXPORT int oracle_wots_pkgen(int pid, const uint8_t *sk, uint32_t layer, uint64_t tree, uint32_t kp, uint8_t *pk)
{
    spx_ctx c;
    if (ctx_from_sk(pid, sk, &c)) return -1;
    wots_pkgen(&c, layer, tree, kp, pk);
    return 0;
}

SPX_EXPORT int oracle_wots_sign(int pid, const uint8_t *sk, const uint8_t *msg, uint32_t layer,
                                uint64_t tree, uint32_t kp, uint8_t *sig)
{
    spx_ctx c;
    if (ctx_from_sk(pid, sk, &c)) return -1;
    wots_sign(&c, msg, layer, tree, kp, sig);
    return 0;
}

SPX_EXPORT int oracle_wots_pk_from_sig(int pid, const uint8_t *sk, const uint8_t *sig, const uint8_t *msg,
                                       uint32_t layer, uint64_t tree, uint32_t kp, uint8_t *pk)
{
    spx_ctx c;
    if (ctx_from_sk(pid, sk, &c)) return -1;
    wots_pk_from_sig(&c, sig, msg, layer, tree, kp, pk);
    return 0;
}

SPX_EXPORT int oracle_xmss_node(int pid, const uint8_t *sk, uint32_t layer, uint64_t tree,
                                uint32_t idx, int z, uint8_t *out)
{
    spx_ctx c;
    if (ctx_from_sk(pid, sk, &c)) return -1;
    xmss_node(&c, layer, tree, idx, z, out);
    return 0;
}

SPX_EXPORT int oracle_xmss_root_from_sig(int pid, const uint8_t *sk, const uint8_t *sig, const uint8_t *msg,
                                         uint32_t layer, uint64_t tree, uint32_t leaf, uint8_t *root)
{
    spx_ctx c;
    if (ctx_from_sk(pid, sk, &c)) return -1;
    xmss_root_from_sig(&c, sig, msg, layer, tree, leaf, root);
    return 0;
}

SPX_EXPORT int oracle_fors_node(int pid, const uint8_t *sk, uint64_t idx_tree, uint32_t idx_leaf,
                                uint32_t g, int z, uint8_t *out)
{
    spx_ctx c;
    if (ctx_from_sk(pid, sk, &c)) return -1;
    fors_node(&c, idx_tree, idx_leaf, g, z, out);
    return 0;
}

SPX_EXPORT int oracle_fors_sk(int pid, const uint8_t *sk, uint64_t idx_tree, uint32_t idx_leaf,
                              uint32_t g, uint8_t *out)
{
    spx_ctx c;
    if (ctx_from_sk(pid, sk, &c)) return -1;
    fors_sk(&c, idx_tree, idx_leaf, g, out);
    return 0;
}

SPX_EXPORT int oracle_fors_pk_from_sig(int pid, const uint8_t *sk, const uint8_t *sig, const uint32_t *fidx,
                                       uint64_t idx_tree, uint32_t idx_leaf, uint8_t *pk_fors)
{
    spx_ctx c;
    if (ctx_from_sk(pid, sk, &c)) return -1;
    fors_pk_from_sig(&c, sig, fidx, idx_tree, idx_leaf, pk_fors);
    return 0;
}

/* Key generation from a 3n-byte seed SK.seed || SK.prf || PK.seed:
 * PK.root = node(0, h') of tree 0 at the top layer d-1.
 * pk = PK.seed || PK.root (2n); sk = SK.seed || SK.prf || PK.seed || PK.root (4n). */
SPX_EXPORT int oracle_keygen(int pid, const uint8_t *seed, uint8_t *pk, uint8_t *sk)
{
    spx_ctx c;
    int n;
    memset(&c, 0, sizeof(c));
    if (params_init(pid, &c.p)) return -1;
    n = c.p.n;
    memcpy(c.sk_seed, seed, n);
    memcpy(c.sk_prf, seed + n, n);
    memcpy(c.pk_seed, seed + 2 * n, n);
    xmss_node(&c, (uint32_t)(c.p.d - 1), 0, 0, c.p.hp, c.pk_root);
    memcpy(pk, c.pk_seed, n);
    memcpy(pk + n, c.pk_root, n);
    memcpy(sk, c.sk_seed, n);
    memcpy(sk + n, c.sk_prf, n);
    memcpy(sk + 2 * n, c.pk_seed, n);
    memcpy(sk + 3 * n, c.pk_root, n);
    return 0;
}

/* Deterministic signing: R = PRF_msg(SK.prf, PK.seed, M); digest = H_msg;
 * SIG = R || SIG_FORS || (WOTS sig_j || auth_j) for j = 0..d-1. */
SPX_EXPORT int oracle_sign(int pid, const uint8_t *sk, const uint8_t *m, size_t mlen, uint8_t *sig)
{
    spx_ctx c;
    uint8_t R[32], digest[64];
    uint32_t fidx[64], idx_leaf;
    uint64_t idx_tree;
    if (ctx_from_sk(pid, sk, &c)) return -1;
    prf_msg(&c, c.pk_seed, m, mlen, R);
    hash_msg(&c, R, m, mlen, digest);
    split_digest(&c.p, digest, fidx, &idx_tree, &idx_leaf);
    sign_fields(&c, R, fidx, idx_tree, idx_leaf, sig);
    return 0;
}

/* Signing with the digest fields given (brute-force enumeration in tests). */
SPX_EXPORT int oracle_sign_fields(int pid, const uint8_t *sk, const uint8_t *R, const uint32_t *fidx,
                                  uint64_t idx_tree, uint32_t idx_leaf, uint8_t *sig)
{
    spx_ctx c;
    if (ctx_from_sk(pid, sk, &c)) return -1;
    sign_fields(&c, R, fidx, idx_tree, idx_leaf, sig);
    return 0;
}

/* Verification by the inverse climbs; returns 1 = accept, 0 = reject, -1 = bad params. */
SPX_EXPORT int oracle_verify(int pid, const uint8_t *pk, const uint8_t *m, size_t mlen, const uint8_t *sig)
{
    spx_ctx c;
    uint8_t digest[64], root[32];
    uint32_t fidx[64], leaf;
    uint64_t tree;
    const uint8_t *s;
    int j, n;
    memset(&c, 0, sizeof(c));
    if (params_init(pid, &c.p)) return -1;
    n = c.p.n;
    memcpy(c.pk_seed, pk, n);
    memcpy(c.pk_root, pk + n, n);
    hash_msg(&c, sig, m, mlen, digest);
    split_digest(&c.p, digest, fidx, &tree, &leaf);
    fors_pk_from_sig(&c, sig + n, fidx, tree, leaf, root);
    s = sig + n + c.p.fors_bytes;
    for (j = 0; j < c.p.d; j++) {
        uint8_t next[32];
        xmss_root_from_sig(&c, s, root, (uint32_t)j, tree, leaf, next);
        memcpy(root, next, n);
        s += (size_t)(c.p.len + c.p.hp) * n;
        leaf = (uint32_t)(tree & (((uint64_t)1 << c.p.hp) - 1));
        tree >>= c.p.hp;
    }
    return memcmp(root, c.pk_root, n) == 0 ? 1 : 0;
}

/* FIPS 205 pure SLH-DSA (deterministic): sign / verify M' = 0x00 ||
 * len(ctx) || ctx || M with the FIPS 205 index order; ctxlen <= 255. */
static uint8_t *slh_wrap(const uint8_t *ctx, size_t ctxlen, const uint8_t *m, size_t mlen, size_t *outlen)
{
    uint8_t *w = (uint8_t *)malloc(2 + ctxlen + mlen + 1);
    if (!w) return NULL;
    w[0] = 0;
    w[1] = (uint8_t)ctxlen;
    if (ctxlen) memcpy(w + 2, ctx, ctxlen);
    if (mlen) memcpy(w + 2 + ctxlen, m, mlen);
    *outlen = 2 + ctxlen + mlen;
    return w;
}

SPX_EXPORT int oracle_slh_sign(int pid, const uint8_t *sk, const uint8_t *ctx, size_t ctxlen,
                               const uint8_t *m, size_t mlen, uint8_t *sig)
{
    size_t wl;
    uint8_t *w;
    int rc;
    if (pid < 0 || pid > 47 || (pid & 16) || ctxlen > 255) return -1;   /* a base set, SHA2 or SHAKE */
    w = slh_wrap(ctx, ctxlen, m, mlen, &wl);
    if (!w) return -1;
    rc = oracle_sign(pid + 16, sk, w, wl, sig);
    free(w);
    return rc;
}

SPX_EXPORT int oracle_slh_verify(int pid, const uint8_t *pk, const uint8_t *ctx, size_t ctxlen,
                                 const uint8_t *m, size_t mlen, const uint8_t *sig)
{
    size_t wl;
    uint8_t *w;
    int rc;
    if (pid < 0 || pid > 47 || (pid & 16) || ctxlen > 255) return -1;
    w = slh_wrap(ctx, ctxlen, m, mlen, &wl);
    if (!w) return -1;
    rc = oracle_verify(pid + 16, pk, w, wl, sig);
    free(w);
    return rc;
}

/* Counters: [0] SHA-256 blocks, [1] SHA-512 blocks, [2] F, [3] PRF, [4] H, [5] T,
 * [6] Keccak-f[1600] permutations. */
SPX_EXPORT void oracle_counters(uint64_t *out, int reset)
{
    out[0] = g_c256_blocks; out[1] = g_c512_blocks; out[2] = g_calls_f;
    out[3] = g_calls_prf; out[4] = g_calls_h; out[5] = g_calls_t; out[6] = g_keccak_perms;
    if (reset)
        g_c256_blocks = g_c512_blocks = g_calls_f = g_calls_prf = g_calls_h = g_calls_t = g_keccak_perms = 0;
}
