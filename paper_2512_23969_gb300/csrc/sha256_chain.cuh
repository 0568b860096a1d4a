// sha256_chain.cuh -- the SHA-256 compression specialised for WOTS+ chains
// and other one-block tweakable hashes, balanced across GB300's pipes.
//
// Measured on this GB300 (sm_103a): LOP3, SHF and PRMT issue on the ALU pipe
// at 64 lanes/clk/SM; IMAD issues on the FMA-heavy pipe at 64 lanes/clk/SM;
// IADD3 can go to either; warp issue is 128 lanes/clk/SM.  SHA-256 is
// dominated by rotations and 3-input logic that only the ALU pipe executes,
// so the additions of each round are written as IMAD (a * one + b with a
// kernel-argument 'one' the compiler cannot fold) to keep them off the ALU
// pipe -- the same instruction re-selection the paper applies with its
// mad.lo listing (Sec. III-C), chosen here by measurement on sm_103a.
//
// WOTS+ chains: within one chain every F call has the same first 5 message
// words (the compressed address up to the hash index), so the state after
// rounds 0..4, round 5 up to its message word, and the address-only parts
// of message words 16..20 are computed once per chain (ChainCtx); each of
// the chain's F steps adds W_5 into round 5's two sums and runs rounds
// 6..63.  The result is the same compression, bit for bit.
#pragma once
#include <cstdint>
#include "hs_common.cuh"

namespace hs {

__device__ __forceinline__ uint32_t mad_add(uint32_t a, uint32_t b, uint32_t one) {
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(one), "r"(b));
    return r;
}
template <uint32_t IMM>
__device__ __forceinline__ uint32_t mad_addi(uint32_t a, uint32_t one) {
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(one), "n"(IMM));
    return r;
}

// Addition policy: bit 0 = T1 sums on IMAD, bit 1 = e update on IMAD,
// bit 2 = a update on IMAD, bit 3 = message-schedule sums on IMAD.
// Measured on GB300: POL 7 for the chains at n = 16 (POL 15: TREE_Sign
// 88.4 -> 97.8 ms at 128f), POL 15 for the tree-building chains at n = 24 /
// 32, whose kernels also run SHA-512 T_len and H (TREE_Sign 1.5-2.8 %
// faster at 192f / 256f / 192s / 256s).
template <int POL>
struct Pipes {
    uint32_t one;
    __device__ __forceinline__ explicit Pipes(uint32_t o) : one(o) {}
};

// Policy used by the signing kernels (all round additions on IMAD).
constexpr int kChainPol = 7;
// Policy of the kernels that build XMSS trees (TREE_Sign, the split and
// wide-tree leaf kernels, shared trees) for a parameter set.
template <class P>
constexpr int tree_pol() { return P::BIG ? 15 : kChainPol; }
// Policy of FORS_Sign: 15 only where its leaves run full compressions
// (no per-message chain context: k * 2^a > 2^16) at n = 24 / 32; with the
// context POL 7 measured faster (256f FORS 43.7 vs 44.8 ms).
template <class P>
constexpr int fors_pol() { return (P::BIG && ((uint64_t)P::K << P::A) > 65536u) ? 15 : kChainPol; }

namespace detail {
constexpr uint32_t kK256[64] = {HS_K256_LIST};
}

// Round t on a rotating state array: a = v[(-t) & 7], ..., h = v[(7 - t) & 7].
template <int POL, int t>
__device__ __forceinline__ void round256(uint32_t v[8], uint32_t w, const Pipes<POL>& p) {
    constexpr uint32_t K = detail::kK256[t];
    uint32_t& a = v[(8 - (t & 7)) & 7];
    uint32_t& b = v[(9 - (t & 7)) & 7];
    uint32_t& c = v[(10 - (t & 7)) & 7];
    uint32_t& d = v[(11 - (t & 7)) & 7];
    uint32_t& e = v[(12 - (t & 7)) & 7];
    uint32_t& f = v[(13 - (t & 7)) & 7];
    uint32_t& g = v[(14 - (t & 7)) & 7];
    uint32_t& h = v[(15 - (t & 7)) & 7];
    const uint32_t ch = (e & f) ^ (~e & g);
    const uint32_t mj = (a & b) | (c & (a | b));
    uint32_t t1;
    if constexpr (POL & 1) t1 = mad_add(mad_add(mad_add(mad_addi<K>(h, p.one), w, p.one), S1_256(e), p.one), ch, p.one);
    else t1 = h + S1_256(e) + ch + K + w;
    if constexpr (POL & 2) d = mad_add(d, t1, p.one);
    else d = d + t1;
    if constexpr (POL & 4) h = mad_add(mad_add(t1, S0_256(a), p.one), mj, p.one);
    else h = t1 + S0_256(a) + mj;
}

// Rounds [t0, t1) with the message schedule extended in the 16-word ring W.
// PRE: words 0..4 are replaced by the chain constants c[] in words 16..20.
// K16 (PRE, one-block calls at n = 16, whose words 10..14 are zero and 15
// the constant length): words 17 and 19 and sigma1(W_19) depend on the
// chain's address alone and come from k[0..2].
template <int POL, bool PRE, int t0, int t1, bool K16 = false>
struct Rounds256 {
    __device__ static __forceinline__ void run(uint32_t v[8], uint32_t W[16], const uint32_t* c, const Pipes<POL>& p,
                                               const uint32_t* k = nullptr) {
        constexpr int t = t0;
        if constexpr (K16 && (t == 17 || t == 19)) {
            W[t & 15] = k[(t - 17) / 2];
        } else if constexpr (K16 && t == 21) {   // sigma1(W19) + W14 (= 0) + sigma0(W6) + W5
            if constexpr (POL & 8) W[t & 15] = mad_add(mad_add(k[2], s0_256(W[6]), p.one), W[5], p.one);
            else W[t & 15] = k[2] + s0_256(W[6]) + W[5];
        } else if constexpr (t >= 16 && (POL & 8)) {
            const uint32_t a = mad_add(s1_256(W[(t - 2) & 15]), W[(t - 7) & 15], p.one);
            if constexpr (PRE && t <= 19) {
                W[t & 15] = mad_add(a, c[t - 16], p.one);
            } else if constexpr (PRE && t == 20) {
                W[t & 15] = mad_add(mad_add(a, s0_256(W[5]), p.one), c[4], p.one);
            } else {
                W[t & 15] = mad_add(mad_add(a, s0_256(W[(t - 15) & 15]), p.one), W[t & 15], p.one);
            }
        } else if constexpr (t >= 16) {
            if constexpr (PRE && t <= 19) {
                W[t & 15] = s1_256(W[(t - 2) & 15]) + W[(t - 7) & 15] + c[t - 16];
            } else if constexpr (PRE && t == 20) {
                W[t & 15] = s1_256(W[(t - 2) & 15]) + W[(t - 7) & 15] + s0_256(W[5]) + c[4];
            } else {
                W[t & 15] = s1_256(W[(t - 2) & 15]) + W[(t - 7) & 15] + s0_256(W[(t - 15) & 15]) + W[t & 15];
            }
        }
        round256<POL, t>(v, W[t & 15], p);
        if constexpr (t0 + 1 < t1) Rounds256<POL, PRE, t0 + 1, t1, K16>::run(v, W, c, p, k);
    }
};

// Chain-invariant part of an F call: the state after rounds 0..4 (from the
// key midstate, message words 0..4 = the address words) with round 5
// applied except for its message word -- in the rotating layout of round 5,
// s[6] = d + T1' and s[2] = T1' + T2 with T1' = h + Sigma1(e) + Ch(e, f, g)
// + K_5, so that adding W_5 to both gives the new e and a -- and the
// address-only terms of message words 16..20; and for the n = 16 block
// (words 10..14 zero, word 15 the length 816) the address-only words 17
// and 19 and sigma1(W_19) in k[].
struct ChainCtx {
    uint32_t s[8];
    uint32_t c[5];
    uint32_t k[3];
};

template <int POL>
__device__ __forceinline__ void chain_ctx(const uint32_t ms[8], const Adrs& a, ChainCtx& x, const Pipes<POL>& p) {
    uint32_t W[16];
    W[0] = a.w0; W[1] = a.w1; W[2] = a.w2; W[3] = a.w3; W[4] = a.w4;
#pragma unroll
    for (int i = 0; i < 8; i++) x.s[i] = ms[i];
    round256<POL, 0>(x.s, W[0], p);
    round256<POL, 1>(x.s, W[1], p);
    round256<POL, 2>(x.s, W[2], p);
    round256<POL, 3>(x.s, W[3], p);
    round256<POL, 4>(x.s, W[4], p);
    {   // round 5 without W_5 (a = s[3], b = s[4], c = s[5], d = s[6], e = s[7], f = s[0], g = s[1], h = s[2])
        const uint32_t e = x.s[7], f = x.s[0], g = x.s[1], a = x.s[3], b = x.s[4], c = x.s[5];
        const uint32_t t1 = x.s[2] + S1_256(e) + ((e & f) ^ (~e & g)) + detail::kK256[5];
        const uint32_t t2 = S0_256(a) + ((a & b) | (c & (a | b)));
        x.s[6] += t1;
        x.s[2] = t1 + t2;
    }
    x.c[0] = s0_256(W[1]) + W[0];
    x.c[1] = s0_256(W[2]) + W[1];
    x.c[2] = s0_256(W[3]) + W[2];
    x.c[3] = s0_256(W[4]) + W[3];
    x.c[4] = W[4];
    // n = 16: W17 = sigma1(W15) + W10 + c[1], W19 = sigma1(W17) + W12 + c[3]
    // (unused, and removed by the compiler, at the other widths)
    constexpr uint32_t kLen16 = (64 + 22 + 16) * 8;
    x.k[0] = s1_256(kLen16) + x.c[1];
    x.k[1] = s1_256(x.k[0]) + x.c[3];
    x.k[2] = s1_256(x.k[1]);
}

// ---- robust F masks with a per-chain context --------------------------
// The mask of a chain's F step q is MGF1-SHA-256(PK.seed || ADRSc(q), n)
// block 0: message words 0 .. K-1 (K = NW + 5: PK.seed and the chain's
// address up to the hash index) are the same for every step of the chain,
// word K holds q, then the counter's low half and the pad, zeros, the
// length.  So the state after rounds 0 .. K-1 and the fixed-word terms of
// schedule words 16 .. 16 + K - 1 are computed once per chain, and a step
// runs rounds K .. 63 (at n = 32 the length does not fit the block: a
// second block of zeros and the length follows, whose whole schedule is a
// compile-time constant).  Same bytes as mgf1_256_block.
template <int NW>
struct MaskCtx {
    uint32_t s[8];
    uint32_t c[NW + 5];
};

// Rounds [t0, t1) of a compression whose message words 0 .. K-1 are not
// in W but folded into c[]: schedule word 16 + j takes its terms W[j],
// sigma0(W[j + 1]) and W[j + 9] from c[j] wherever their index is below K.
template <int POL, int K, int t0, int t1>
struct RoundsPre {
    __device__ static __forceinline__ void run(uint32_t v[8], uint32_t W[16], const uint32_t* c, const Pipes<POL>& p) {
        constexpr int t = t0;
        if constexpr (t >= 16 && t < 16 + K) {
            constexpr int j = t - 16;
            uint32_t w = s1_256(W[(t - 2) & 15]) + c[j];
            if constexpr (j + 1 >= K) w += s0_256(W[(t - 15) & 15]);
            if constexpr (j + 9 >= K) w += W[(t - 7) & 15];
            W[t & 15] = w;
        } else if constexpr (t >= 16) {
            W[t & 15] = s1_256(W[(t - 2) & 15]) + W[(t - 7) & 15] + s0_256(W[(t - 15) & 15]) + W[t & 15];
        }
        round256<POL, t>(v, W[t & 15], p);
        if constexpr (t0 + 1 < t1) RoundsPre<POL, K, t0 + 1, t1>::run(v, W, c, p);
    }
};

template <int POL, int NW, int t>
__device__ __forceinline__ void mask_ctx_rounds(uint32_t s[8], const uint32_t* W, const Pipes<POL>& p) {
    round256<POL, t>(s, W[t], p);
    if constexpr (t + 1 < NW + 5) mask_ctx_rounds<POL, NW, t + 1>(s, W, p);
}

// Context of the masks of one chain (a: its WOTS_HASH / FORS_TREE address;
// only the half word varies between its steps).
template <int POL, int NW>
__device__ __forceinline__ void mask_ctx(const uint32_t* pks, const Adrs& a, MaskCtx<NW>& m, const Pipes<POL>& p) {
    constexpr int K = NW + 5;
    uint32_t W[K];
#pragma unroll
    for (int i = 0; i < NW; i++) W[i] = pks[i];
    W[NW] = a.w0; W[NW + 1] = a.w1; W[NW + 2] = a.w2; W[NW + 3] = a.w3; W[NW + 4] = a.w4;
    sha256_iv(m.s);
    mask_ctx_rounds<POL, NW, 0>(m.s, W, p);
#pragma unroll
    for (int j = 0; j < K; j++) {
        uint32_t c = W[j];
        if (j + 1 < K) c += s0_256(W[j + 1]);
        if (j + 9 < K) c += W[j + 9];
        m.c[j] = c;
    }
}

// The first NW words of the mask of the step whose half word is 'half'.
template <int POL, int NW>
__device__ __forceinline__ void mask_step(const MaskCtx<NW>& m, uint32_t half, uint32_t* out, const Pipes<POL>& p) {
    constexpr int K = NW + 5;
    constexpr uint32_t L = 4 * NW + 26;            // PK.seed || ADRSc || counter bytes
    uint32_t W[16];
#pragma unroll
    for (int i = 0; i < 16; i++) W[i] = 0u;
    W[K] = half << 16;                             // counter 0: its high half is 0
    W[K + 1] = 0x8000u;                            // counter low half 0, then the pad byte
    if constexpr (L + 9 <= 64) W[15] = L * 8;
    uint32_t v[8];
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = m.s[i];
    RoundsPre<POL, K, K, 64>::run(v, W, m.c, p);
    uint32_t st[8];
    sha256_iv(st);
#pragma unroll
    for (int i = 0; i < 8; i++) st[i] += v[i];
    if constexpr (L + 9 > 64) {                    // n = 32: zeros and the length
        uint32_t W2[16];
#pragma unroll
        for (int i = 0; i < 15; i++) W2[i] = 0u;
        W2[15] = L * 8;
        sha256_compress_full(st, W2);
    }
#pragma unroll
    for (int i = 0; i < NW; i++) out[i] = st[i];
}

// Message words 5..15 of a one-block call: low half of the last address word,
// NW payload words at a 2-byte offset, 0x80 pad, zeros, bit length.
template <int NW>
__device__ __forceinline__ void tail_words(uint32_t W[16], uint32_t half, const uint32_t* x) {
    W[5] = mid16(half, x[0]);
#pragma unroll
    for (int k = 1; k < NW; k++) W[5 + k] = mid16(x[k - 1], x[k]);
    W[5 + NW] = (x[NW - 1] << 16) | 0x8000u;
#pragma unroll
    for (int k = 6 + NW; k < 15; k++) W[k] = 0;
    W[15] = (64 + 22 + 4 * NW) * 8;
}

// One chain step with a precomputed context: out = Trunc_n(compress(ms, block)),
// where the block's hash address is 'half' and its payload is x (NW words).
template <int POL, int NW>
__device__ __forceinline__ void chain_step(const ChainCtx& cx, const uint32_t ms[8], uint32_t half,
                                           const uint32_t* x, uint32_t* out, const Pipes<POL>& p) {
    uint32_t W[16];
    tail_words<NW>(W, half, x);
    uint32_t v[8];
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = cx.s[i];
    v[6] = mad_add(v[6], W[5], p.one);            // round 5: its message word
    v[2] = mad_add(v[2], W[5], p.one);
    Rounds256<POL, true, 6, 64, NW == 4>::run(v, W, cx.c, p, cx.k);
#pragma unroll
    for (int i = 0; i < NW; i++) out[i] = v[i] + ms[i];
}

// Plain one-block F / PRF (no reusable context), same round code.
template <int POL, int NW>
__device__ __forceinline__ void hashF_fast(const uint32_t ms[8], const Adrs& a, const uint32_t* x, uint32_t* out,
                                           const Pipes<POL>& p) {
    uint32_t W[16];
    W[0] = a.w0; W[1] = a.w1; W[2] = a.w2; W[3] = a.w3; W[4] = a.w4;
    tail_words<NW>(W, a.half, x);
    uint32_t v[8];
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = ms[i];
    Rounds256<POL, false, 0, 64>::run(v, W, nullptr, p);
#pragma unroll
    for (int i = 0; i < NW; i++) out[i] = v[i] + ms[i];
}

// F / PRF of a parameter set: the chain-specialised SHA-256 call above, or
// one SHAKE256 block for the SHAKE sets (ms256 then holds PK.seed).
// Robust sets: pks = PK.seed words masks the payload (F); nullptr = PRF.
template <class P, int POL>
__device__ __forceinline__ void hashF_p(const uint32_t ms256[8], const Adrs& a, const uint32_t* x, uint32_t* out,
                                        const Pipes<POL>& pp, const uint32_t* pks = nullptr) {
    if constexpr (P::SHAKE) {
        shake_thash1<P::NW, P::NW>(ms256, a, x, out);
    } else if constexpr (P::ROBUST) {
        uint32_t xm[P::NW];
#pragma unroll
        for (int i = 0; i < P::NW; i++) xm[i] = x[i];
        if (pks) mask_regs<false, P::NW, P::NW>(pks, a, xm);
        hashF_fast<POL, P::NW>(ms256, a, xm, out, pp);
    } else {
        hashF_fast<POL, P::NW>(ms256, a, x, out, pp);
    }
}

// One chain step F(WOTS_HASH(.., hash q), x) with the chain's context; the
// robust sets mask x first with the step's mask (mk: the chain's mask
// context; unused by the other sets).
template <class P, int POL>
__device__ __forceinline__ void chain_step_p(const ChainCtx& cx, const MaskCtx<P::NW>& mk, const uint32_t ms256[8],
                                             uint32_t q, const uint32_t* x, uint32_t* out, const Pipes<POL>& pp) {
    if constexpr (P::ROBUST) {
        uint32_t m[P::NW];
        mask_step<POL, P::NW>(mk, q, m, pp);
#pragma unroll
        for (int i = 0; i < P::NW; i++) m[i] ^= x[i];
        chain_step<POL, P::NW>(cx, ms256, q, m, out, pp);
    } else {
        chain_step<POL, P::NW>(cx, ms256, q, x, out, pp);
    }
}

// The same compression as sha256_compress_rolled (16 rounds unrolled in a
// loop of 4, K from constant memory: a small code footprint for call sites
// outside the chain loops) with the round additions on IMAD as in round256.
template <int POL>
__device__ __forceinline__ void compress256_rolled_p(uint32_t st[8], uint32_t W[16], const Pipes<POL>& p) {
    uint32_t v[8];
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = st[i];
#pragma unroll 1
    for (int t0 = 0; t0 < 64; t0 += 16) {
        if (t0 > 0) {
#pragma unroll
            for (int i = 0; i < 16; i++)
                W[i] += s1_256(W[(i + 14) & 15]) + W[(i + 9) & 15] + s0_256(W[(i + 1) & 15]);
        }
#pragma unroll
        for (int j = 0; j < 16; j++) {
            uint32_t& a = v[(8 - (j & 7)) & 7];
            uint32_t& b = v[(9 - (j & 7)) & 7];
            uint32_t& c = v[(10 - (j & 7)) & 7];
            uint32_t& d = v[(11 - (j & 7)) & 7];
            uint32_t& e = v[(12 - (j & 7)) & 7];
            uint32_t& f = v[(13 - (j & 7)) & 7];
            uint32_t& g = v[(14 - (j & 7)) & 7];
            uint32_t& h = v[(15 - (j & 7)) & 7];
            const uint32_t ch = (e & f) ^ (~e & g);
            const uint32_t mj = (a & b) | (c & (a | b));
            const uint32_t t1 =
                mad_add(mad_add(mad_add(mad_add(h, c_K256[t0 + j], p.one), W[j], p.one), S1_256(e), p.one), ch, p.one);
            d = mad_add(d, t1, p.one);
            h = mad_add(mad_add(t1, S0_256(a), p.one), mj, p.one);
        }
    }
#pragma unroll
    for (int i = 0; i < 8; i++) st[i] += v[i];
}

// T_l over PW payload words in memory through the rolled IMAD-addition
// compression (SHA-256); the SHA-512 form is tl_from_mem's.
template <bool BIG, int PW, int NW, int POL>
__device__ __forceinline__ void tl_from_mem_p(const uint32_t* ms, const Adrs& a, const uint32_t* p, uint32_t* out,
                                              const Pipes<POL>& pp) {
    if constexpr (BIG) {
        tl_from_mem<BIG, PW, NW>(ms, a, p, out);
    } else {
        uint32_t st[8];
#pragma unroll
        for (int i = 0; i < 8; i++) st[i] = ms[i];
#pragma unroll 1
        for (int b = 0; b < tl_blocks<false, PW>(); b++) {
            uint32_t W[16];
            tl_block<false, PW>(a, p, b, W);
            compress256_rolled_p<POL>(st, W, pp);
        }
#pragma unroll
        for (int i = 0; i < NW; i++) out[i] = st[i];
    }
}

// H of a parameter set through the rolled IMAD-addition compression where
// it is one SHA-256 block (n = 16); SHA-512 (n > 16) and SHAKE as hashH_ms.
template <class P, int POL>
__device__ __forceinline__ void hashH_p(const uint32_t* ms256, const uint32_t* ms512, const Adrs& a,
                                        const uint32_t* lr, uint32_t* out, const Pipes<POL>& pp,
                                        const uint32_t* pks = nullptr) {
    if constexpr (P::SHAKE || P::BIG) {
        hashH_ms<P>(ms256, ms512, a, lr, out, pks);
    } else {
        uint32_t W[16], st[8], m[2 * P::NW];
#pragma unroll
        for (int i = 0; i < 2 * P::NW; i++) m[i] = lr[i];
        if constexpr (P::ROBUST) mask_regs<false, P::NW, 2 * P::NW>(pks, a, m);
        fill_block<16, 2 * P::NW>(W, a, m);
        W[15] = (64 + 22 + 8 * P::NW) * 8;
#pragma unroll
        for (int i = 0; i < 8; i++) st[i] = ms256[i];
        compress256_rolled_p<POL>(st, W, pp);
#pragma unroll
        for (int i = 0; i < P::NW; i++) out[i] = st[i];
    }
}

}  // namespace hs
