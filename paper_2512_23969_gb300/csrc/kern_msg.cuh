// kern_msg.cuh -- per-key preparation and the message stage (kernel templates).
//
// Message stage (the paper's hash_message + message_to_indices, Fig. 2):
//   R      = Trunc_n(HMAC-SHA-x(SK.prf, PK.seed || M))          (PRF_msg)
//   digest = MGF1-SHA-x(R || PK.seed || SHA-x(R || PK.seed || PK.root || M), m)
//   digest = md || tree bytes || leaf bytes -> k FORS indices, idx_tree, idx_leaf
// FIPS 205 mode: M is preceded by a per-call prefix (0x00 || len(ctx) || ctx
// for pure SLH-DSA) in both hashes, and the FORS indices are read from md
// most significant bit first (FIPS 205 base_2b).
// The work is serial in the message length (two passes over M), the only
// length-dependent part of signing.  Large batches run a thread per message;
// small ones (SHA-2 sets) a warp per message, which takes the message
// schedule of a long message's blocks off its serial path (blocks_coop).
#pragma once
#include <cuda_runtime.h>
#include "hs_common.cuh"
#include "hs_launch.h"
#include "../../include/hs.h"

namespace hs {

// ------------------------------------------------------------- warp-cooperative blocks
// A message's hash is one serial chain of compressions (FIPS 180-4 Sec.
// 6.2.2 / 6.4.2: each block starts from the previous block's state), so a
// thread hashing a long message runs at one warp's latency: about 46 cycles
// per SHA-256 round and 105 per SHA-512 round, with the message schedule's
// instructions on the same serial path.  The schedule W_0..W_{63|79} of a
// block depends on the block alone, so in the cooperative form a warp
// computes the schedules of up to CH blocks at once, one block per lane,
// and keeps W_t + K_t in shared memory; every lane then runs the same rounds
// over them (one instruction stream, the same state in every lane), which
// leaves only the rounds on the serial path.
template <bool BIG> struct CoopShape;
// rows of W_t + K_t, padded by 4 words so that the lanes' rows start in
// different banks (each lane stores its own row)
template <> struct CoopShape<false> { static constexpr int CH = 32, WKW = 64 + 4; };
template <> struct CoopShape<true> { static constexpr int CH = 32, WKW = 2 * 80 + 4; };

// W_t + K_t (t = 0..63) of one SHA-256 block (16 big-endian words) into o.
__device__ __forceinline__ void wk256_store(const uint32_t w[16], uint32_t* o) {
    constexpr uint32_t K[64] = {HS_K256_LIST};
    uint32_t W[16];
#pragma unroll
    for (int i = 0; i < 16; i++) W[i] = w[i];
#pragma unroll
    for (int t = 0; t < 64; t += 4) {
        uint32_t v[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int i = t + j;
            if (i >= 16) W[i & 15] += s1_256(W[(i - 2) & 15]) + W[(i - 7) & 15] + s0_256(W[(i - 15) & 15]);
            v[j] = W[i & 15] + K[i];
        }
        *reinterpret_cast<uint4*>(o + t) = make_uint4(v[0], v[1], v[2], v[3]);
    }
}

// The 64 SHA-256 rounds and the feed-forward, W_t + K_t read from wk.
// Latency form: the new e is d + T1 = (d + h + W_t + K_t) + Sigma1(e) +
// Ch(e, f, g), with the first sum formed before Sigma1 is ready (h and d
// are known rounds ahead), so only one three-input addition follows
// Sigma1 on the serial path; the empty asm keeps the compiler from folding
// that sum back into d + T1.  Measured 13 % faster than d + T1 in the warp
// form; the same restructuring made the SHA-512 rounds 8 % slower.
__device__ __forceinline__ void rounds256_wk(uint32_t st[8], const uint32_t* wk) {
    uint32_t a = st[0], b = st[1], c = st[2], d = st[3], e = st[4], f = st[5], g = st[6], h = st[7];
#define HS_RW256(a, b, c, d, e, f, g, h, x)                         \
    do {                                                            \
        const uint32_t hx_ = h + (x);                               \
        uint32_t dhx_ = d + hx_;                                    \
        asm("" : "+r"(dhx_));                                       \
        const uint32_t s1_ = S1_256(e), ch_ = ch32(e, f, g);        \
        d = dhx_ + s1_ + ch_;                                       \
        h = (hx_ + s1_ + ch_) + S0_256(a) + maj32(a, b, c);         \
    } while (0)
#pragma unroll
    for (int t = 0; t < 64; t += 8) {
        const uint4 u = *reinterpret_cast<const uint4*>(wk + t);
        const uint4 v = *reinterpret_cast<const uint4*>(wk + t + 4);
        HS_RW256(a, b, c, d, e, f, g, h, u.x);
        HS_RW256(h, a, b, c, d, e, f, g, u.y);
        HS_RW256(g, h, a, b, c, d, e, f, u.z);
        HS_RW256(f, g, h, a, b, c, d, e, u.w);
        HS_RW256(e, f, g, h, a, b, c, d, v.x);
        HS_RW256(d, e, f, g, h, a, b, c, v.y);
        HS_RW256(c, d, e, f, g, h, a, b, v.z);
        HS_RW256(b, c, d, e, f, g, h, a, v.w);
    }
#undef HS_RW256
    st[0] += a; st[1] += b; st[2] += c; st[3] += d; st[4] += e; st[5] += f; st[6] += g; st[7] += h;
}

// W_t + K_t (t = 0..79) of one SHA-512 block (32 big-endian 32-bit words)
// into o as (hi, lo) word pairs.
__device__ __forceinline__ void wk512_store(const uint32_t w[32], uint32_t* o) {
    uint64_t W[16];
#pragma unroll
    for (int i = 0; i < 16; i++) W[i] = ((uint64_t)w[2 * i] << 32) | w[2 * i + 1];
#pragma unroll 1
    for (int t = 0; t < 80; t += 16) {
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
            uint64_t v[2];
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const int i = j + q;
                if (t > 0) W[i] += s1_512(W[(i + 14) & 15]) + W[(i + 9) & 15] + s0_512(W[(i + 1) & 15]);
                v[q] = W[i] + c_K512[t + i];
            }
            *reinterpret_cast<uint4*>(o + 2 * (t + j)) =
                make_uint4((uint32_t)(v[0] >> 32), (uint32_t)v[0], (uint32_t)(v[1] >> 32), (uint32_t)v[1]);
        }
    }
}

// The 80 SHA-512 rounds and the feed-forward on a state of 16 big-endian
// words (hi, lo pairs), W_t + K_t read from wk.
__device__ __forceinline__ void rounds512_wk(uint32_t st32[16], const uint32_t* wk) {
    uint64_t s[8];
#pragma unroll
    for (int i = 0; i < 8; i++) s[i] = ((uint64_t)st32[2 * i] << 32) | st32[2 * i + 1];
    uint64_t a = s[0], b = s[1], c = s[2], d = s[3], e = s[4], f = s[5], g = s[6], h = s[7];
#define HS_RW512(a, b, c, d, e, f, g, h, x)                                        \
    do {                                                                           \
        const uint64_t t1_ = h + S1_512(e) + ((e & f) ^ (~e & g)) + (x);           \
        const uint64_t t2_ = S0_512(a) + ((a & b) | (c & (a | b)));                \
        d += t1_;                                                                  \
        h = t1_ + t2_;                                                             \
    } while (0)
#pragma unroll 1
    for (int t = 0; t < 80; t += 16) {
        const uint32_t* r = wk + 2 * t;
#pragma unroll
        for (int j = 0; j < 16; j += 8) {
            uint64_t x[8];
#pragma unroll
            for (int q = 0; q < 8; q += 2) {
                const uint4 u = *reinterpret_cast<const uint4*>(r + 2 * (j + q));
                x[q] = ((uint64_t)u.x << 32) | u.y;
                x[q + 1] = ((uint64_t)u.z << 32) | u.w;
            }
            HS_RW512(a, b, c, d, e, f, g, h, x[0]);
            HS_RW512(h, a, b, c, d, e, f, g, x[1]);
            HS_RW512(g, h, a, b, c, d, e, f, x[2]);
            HS_RW512(f, g, h, a, b, c, d, e, x[3]);
            HS_RW512(e, f, g, h, a, b, c, d, x[4]);
            HS_RW512(d, e, f, g, h, a, b, c, x[5]);
            HS_RW512(c, d, e, f, g, h, a, b, x[6]);
            HS_RW512(b, c, d, e, f, g, h, a, x[7]);
        }
    }
#undef HS_RW512
    s[0] += a; s[1] += b; s[2] += c; s[3] += d; s[4] += e; s[5] += f; s[6] += g; s[7] += h;
#pragma unroll
    for (int i = 0; i < 8; i++) { st32[2 * i] = (uint32_t)(s[i] >> 32); st32[2 * i + 1] = (uint32_t)s[i]; }
}

// ------------------------------------------------------------- byte SHA-x
// Streaming SHA-256 / SHA-512 over bytes and big-endian words.  Only the
// message stage uses it: key words, pads and digests are appended a word at
// a time from registers; message bytes arrive through aligned word loads,
// whole blocks with the next block's loads in flight (blocks()), the partial
// blocks at either end through one batch of loads each (append()).
// COOP: every lane of a warp runs the same instance on the same bytes, and
// whole blocks of message bytes go through the warp-cooperative schedule
// (wk: this warp's CH x WKW words of shared memory).
template <bool BIG, bool COOP = false>
struct ByteSha {
    static constexpr int B = BIG ? 128 : 64;   // block bytes
    static constexpr int BW = B / 4;
    uint32_t st[BIG ? 16 : 8];
    uint32_t blk[BW];
    uint32_t fill;      // bytes in blk
    uint64_t total;     // message bytes so far
    uint32_t* wk;       // COOP only

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
        if constexpr (COOP) {
            blocks_coop(q, nb);
            return;
        }
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
    // The same nb blocks with the whole warp: lane j loads block b0 + j of
    // each chunk (the aligned words around it, as blocks() does) and stores
    // its W_t + K_t row; then every lane runs the rounds of the chunk's
    // blocks in order.  Called by all 32 lanes with the same arguments.
    __device__ void blocks_coop(const uint8_t* q, uint64_t nb) {
        constexpr int CH = CoopShape<BIG>::CH, WKW = CoopShape<BIG>::WKW;
        const uint32_t lane = threadIdx.x & 31;
        const uintptr_t addr = reinterpret_cast<uintptr_t>(q);
        const uint32_t* a = reinterpret_cast<const uint32_t*>(addr & ~(uintptr_t)3);
        const uint32_t sh = (uint32_t)(addr & 3), sel = be_sel(sh);
        for (uint64_t b0 = 0; b0 < nb; b0 += CH) {
            const uint32_t c = (nb - b0 < (uint64_t)CH) ? (uint32_t)(nb - b0) : (uint32_t)CH;
            if (lane < c) {
                const uint32_t* ab = a + (b0 + lane) * BW;
                uint32_t raw[BW + 1];
#pragma unroll
                for (int k = 0; k < BW; k++) raw[k] = __ldg(ab + k);
                raw[BW] = sh ? __ldg(ab + BW) : 0u;
                uint32_t w[BW];
#pragma unroll
                for (int k = 0; k < BW; k++) w[k] = __byte_perm(raw[k], raw[k + 1], sel);
                if constexpr (BIG) wk512_store(w, wk + lane * WKW);
                else wk256_store(w, wk + lane * WKW);
            }
            __syncwarp();
#pragma unroll 1
            for (uint32_t j = 0; j < c; j++) {
                if constexpr (BIG) rounds512_wk(st, wk + j * WKW);
                else rounds256_wk(st, wk + j * WKW);
            }
            __syncwarp();
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

// One message's stage.  verify = 0: compute R (PRF_msg) and write it to
// sig[0:n]; verify = 1: R is read from the signature.  COOP: called by all
// 32 lanes of a warp for the same message (whole blocks of M through the
// warp-cooperative schedule in wk); lane 0 writes the results.
template <class P, bool COOP>
__device__ __forceinline__ void message_one(uint32_t m, uint32_t* wk, const KeyBlock* __restrict__ keys,
                                            uint32_t num_keys, const uint32_t* __restrict__ key_idx,
                                            const uint8_t* __restrict__ msgs, const uint64_t* __restrict__ off,
                                            uint8_t* __restrict__ sigs, MsgInfo* __restrict__ infos,
                                            uint32_t* __restrict__ status, int verify,
                                            const uint8_t* __restrict__ prefix, uint32_t plen, int msb_first) {
    constexpr int NW = P::NW;
    constexpr int DW = P::BIG ? 16 : 8;            // digest words of SHA-x
    const uint32_t lane = COOP ? (threadIdx.x & 31) : 0u;
    const bool lead = lane == 0;                   // the lane that writes
    uint8_t* sig = sigs + (size_t)m * P::SIG_BYTES;
    MsgInfo info;
    info.pad[0] = info.pad[1] = 0;
    const uint32_t key = key_idx ? key_idx[m] : 0u;
    if (key >= num_keys) {
        if (lead) atomicOr(status, 1u << HS_EKEY);
        info.key = KEY_INVALID;
        info.idx_tree = 0;
        info.idx_leaf = 0;
        for (int i = 0; i < 36; i++) info.fors_idx[i] = 0;
        if (lead) infos[m] = info;
        if (!verify) {
            uint4* s4 = reinterpret_cast<uint4*>(sig);
            for (uint32_t i = lane; i < (uint32_t)(P::SIG_BYTES / 16); i += (COOP ? 32u : 1u))
                s4[i] = make_uint4(0, 0, 0, 0);
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
        static_assert(!COOP, "the SHAKE message stage runs a thread per message");
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
    using Sha = ByteSha<P::BIG, COOP>;
    Sha h;
    h.wk = wk;
    if (!verify) {
        // PRF_msg = HMAC-SHA-x(SK.prf, opt_rand || M), opt_rand = PK.seed
        uint32_t kw[Sha::BW];
        for (int i = 0; i < Sha::BW; i++) kw[i] = (i < NW) ? kb.sk_prf[i] : 0u;
        uint32_t inner[DW];
        h.init();
        for (int i = 0; i < Sha::BW; i++) {
            uint32_t x = kw[i] ^ 0x36363636u;
            h.words(&x, 4);
        }
        h.words(kb.pk_seed, P::N);
        if (plen) h.mem(prefix, plen);
        h.mem(M, mlen);
        h.finish(inner);
        h.init();
        for (int i = 0; i < Sha::BW; i++) {
            uint32_t x = kw[i] ^ 0x5c5c5c5cu;
            h.words(&x, 4);
        }
        h.words(inner, 4 * DW);
        uint32_t mac[DW];
        h.finish(mac);
        for (int i = 0; i < NW; i++) R[i] = mac[i];
        if (lead) store_be<NW>(sig, R);
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
    if (lead) infos[m] = info;
}

// One thread per message: the throughput form for large batches.
template <class P>
__global__ void message_kernel(const KeyBlock* __restrict__ keys, uint32_t num_keys,
                               const uint32_t* __restrict__ key_idx, const uint8_t* __restrict__ msgs,
                               const uint64_t* __restrict__ off, uint32_t count, uint8_t* __restrict__ sigs,
                               MsgInfo* __restrict__ infos, uint32_t* __restrict__ status, int verify,
                               const uint8_t* __restrict__ prefix, uint32_t plen, int msb_first) {
    const uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= count) return;
    message_one<P, false>(m, nullptr, keys, num_keys, key_idx, msgs, off, sigs, infos, status, verify, prefix,
                          plen, msb_first);
}

// One warp per message (SHA-2 sets): the latency form for small batches,
// where a long message's serial hash is the batch's critical path.  Two
// warps per block, each with its own schedule buffer.
constexpr int kMsgWarpsPerBlock = 2;
template <class P>
__global__ void __launch_bounds__(32 * kMsgWarpsPerBlock)
    message_warp_kernel(const KeyBlock* __restrict__ keys, uint32_t num_keys, const uint32_t* __restrict__ key_idx,
                        const uint8_t* __restrict__ msgs, const uint64_t* __restrict__ off, uint32_t count,
                        uint8_t* __restrict__ sigs, MsgInfo* __restrict__ infos, uint32_t* __restrict__ status,
                        int verify, const uint8_t* __restrict__ prefix, uint32_t plen, int msb_first) {
    constexpr int PER_WARP = CoopShape<P::BIG>::CH * CoopShape<P::BIG>::WKW;
    __shared__ __align__(16) uint32_t wk[kMsgWarpsPerBlock * PER_WARP];
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t m = blockIdx.x * kMsgWarpsPerBlock + warp;
    if (m >= count) return;                        // the whole warp
    message_one<P, true>(m, wk + warp * PER_WARP, keys, num_keys, key_idx, msgs, off, sigs, infos, status, verify,
                         prefix, plen, msb_first);
}

}  // namespace hs
