// hs_params.cuh -- compile-time parameter sets (paper Table 1, and the s and
// SHAKE variants) and the sizes derived from them.  Every kernel is
// instantiated once per set.
#pragma once
#include <cstdint>

namespace hs {

// N: hash bytes, H: hypertree height, D: layers, A: FORS height, K: FORS trees.
// BIG: H, T_l, H_msg, PRF_msg use SHA-512 (n = 24 / 32).
// SHAKE_: the SHAKE256 instantiation (a variant; the paper uses SHA-2).
// ROBUST_: the robust SHA2 instantiation (a variant): F, H and T_l hash
// their input masked by MGF1 of PK.seed and the address (robust.cuh).
template <int N_, int H_, int D_, int A_, int K_, bool SHAKE_ = false, bool ROBUST_ = false>
struct Params {
    static_assert(!(SHAKE_ && ROBUST_), "robust: SHA2 sets only");
    static constexpr bool SHAKE = SHAKE_;
    static constexpr bool ROBUST = ROBUST_;
    static constexpr int N = N_;
    static constexpr int H = H_;
    static constexpr int D = D_;
    static constexpr int HP = H_ / D_;             // XMSS tree height h'
    static constexpr int A = A_;
    static constexpr int K = K_;
    static constexpr int W = 16;
    static constexpr bool BIG = !SHAKE_ && (N_ > 16);
    static constexpr int NW = N_ / 4;              // n in 32-bit words
    static constexpr int LEN1 = 2 * N_;            // 8n / log2(w)
    static constexpr int LEN2 = 3;                 // every set here (and toy): n = 16 .. 32 at w = 16
    static constexpr int LEN = LEN1 + LEN2;
    static constexpr int TREE_BITS = H_ - HP;
    static constexpr int MD_BYTES = (K_ * A_ + 7) / 8;
    static constexpr int TREE_BYTES = (TREE_BITS + 7) / 8;
    static constexpr int LEAF_BYTES = (HP + 7) / 8;
    static constexpr int M = MD_BYTES + TREE_BYTES + LEAF_BYTES;
    static constexpr int FORS_BYTES = K_ * (A_ + 1) * N_;
    static constexpr int LAYER_BYTES = (LEN + HP) * N_;   // WOTS sig + auth
    static constexpr int SIG_BYTES = N_ + FORS_BYTES + D_ * LAYER_BYTES;
    static constexpr int LEAVES = 1 << HP;         // leaves per XMSS tree
};

using P128f = Params<16, 66, 22, 6, 33>;
using P192f = Params<24, 66, 22, 8, 33>;
using P256f = Params<32, 68, 17, 9, 35>;
using PToy  = Params<16, 4, 2, 3, 4>;
// The small-signature sets of the same scheme (a variant; the paper uses
// the f sets only): h' = 9 / 9 / 8, FORS height 12 / 14 / 14.
using P128s = Params<16, 63, 7, 12, 14>;
using P192s = Params<24, 63, 7, 14, 17>;
using P256s = Params<32, 64, 8, 14, 22>;
// The SHAKE instantiation of each of them.
using PK128f = Params<16, 66, 22, 6, 33, true>;
using PK192f = Params<24, 66, 22, 8, 33, true>;
using PK256f = Params<32, 68, 17, 9, 35, true>;
using PK128s = Params<16, 63, 7, 12, 14, true>;
using PK192s = Params<24, 63, 7, 14, 17, true>;
using PK256s = Params<32, 64, 8, 14, 22, true>;

// The robust SHA2 instantiation of the f sets.
using PR128f = Params<16, 66, 22, 6, 33, false, true>;
using PR192f = Params<24, 66, 22, 8, 33, false, true>;
using PR256f = Params<32, 68, 17, 9, 35, false, true>;

static_assert(P128f::SIG_BYTES == 17088, "128f signature size");
static_assert(P192f::SIG_BYTES == 35664, "192f signature size");
static_assert(P256f::SIG_BYTES == 49856, "256f signature size");
static_assert(PToy::SIG_BYTES == 1456, "toy signature size");
static_assert(P128s::SIG_BYTES == 7856 && P192s::SIG_BYTES == 16224 && P256s::SIG_BYTES == 29792,
              "s signature sizes");
static_assert(P128s::M == 30 && P192s::M == 39 && P256s::M == 47, "s digest bytes");
static_assert(P128f::LEN == 35 && P192f::LEN == 51 && P256f::LEN == 67, "WOTS len");
static_assert(P128f::M == 34 && P192f::M == 42 && P256f::M == 49, "digest bytes");
// every signature starts 16-byte aligned when the buffer does
static_assert(P128f::SIG_BYTES % 16 == 0 && P192f::SIG_BYTES % 16 == 0 &&
              P256f::SIG_BYTES % 16 == 0 && PToy::SIG_BYTES % 16 == 0 && P128s::SIG_BYTES % 16 == 0 &&
              P192s::SIG_BYTES % 16 == 0 && P256s::SIG_BYTES % 16 == 0, "sig alignment");

// Address types of the scheme's ADRS.
enum : uint32_t { T_WOTS_HASH = 0, T_WOTS_PK = 1, T_TREE = 2, T_FORS_TREE = 3,
                  T_FORS_ROOTS = 4, T_WOTS_PRF = 5, T_FORS_PRF = 6 };

// Per-key block derived once per call (256 bytes): midstates after the
// padded PK.seed block, and the key's n-byte values as big-endian words.
struct KeyBlock {
    uint32_t ms256[8];     // SHA-256 state after BlockPad_256(PK.seed)
    uint32_t ms512[16];    // SHA-512 state after BlockPad_512(PK.seed), (hi,lo) pairs
    uint32_t sk_seed[8];
    uint32_t sk_prf[8];
    uint32_t pk_seed[8];
    uint32_t pk_root[8];
    uint32_t pad[8];
};
static_assert(sizeof(KeyBlock) == 256, "KeyBlock is 256 bytes");

// Per-message digest fields produced by the message stage.
struct MsgInfo {
    uint64_t idx_tree;
    uint32_t idx_leaf;
    uint32_t key;          // validated key index; KEY_INVALID if out of range
    uint16_t fors_idx[36]; // k <= 35
    uint32_t pad[2];
};
static_assert(sizeof(MsgInfo) == 96, "MsgInfo is 96 bytes");
constexpr uint32_t KEY_INVALID = 0xFFFFFFFFu;

}  // namespace hs
