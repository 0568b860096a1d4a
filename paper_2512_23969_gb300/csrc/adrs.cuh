// adrs.cuh -- the scheme's hash address in the compressed 22-byte form the
// SHA2 instantiation hashes (ADRSc).  The SHAKE instantiation rebuilds the
// full 32-byte address from the same fields (keccak.cuh).
#pragma once
#include <cstdint>

namespace hs {

// Compressed address ADRSc as five full message words plus the 16-bit half
// word that precedes the payload: layer(1) tree(8) type(1) w5(4) w6(4) w7(4).
struct Adrs {
    uint32_t w0, w1, w2, w3, w4, half;
};

__device__ __forceinline__ Adrs make_adrs(uint32_t layer, uint64_t tree, uint32_t type,
                                          uint32_t kp, uint32_t w6, uint32_t w7) {
    Adrs a;
    a.w0 = (layer << 24) | (uint32_t)(tree >> 40);
    a.w1 = (uint32_t)(tree >> 8);
    a.w2 = ((uint32_t)tree << 24) | (type << 16) | (kp >> 16);
    a.w3 = (kp << 16) | (w6 >> 16);
    a.w4 = (w6 << 16) | (w7 >> 16);
    a.half = w7 & 0xFFFFu;
    return a;
}

}  // namespace hs
