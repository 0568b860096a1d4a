// set_robust_128f.cu -- every kernel instantiated for SPHINCS+-SHA2-128f-robust
// (the robust SHA2 instantiation: a variant beside the paper's simple one),
// with the launch-shape variants the tuner may pick from.
#include "set_impl.cuh"

namespace hs {
namespace {
using P = PR128f;
const int kForsLpt[] = {2, 4, 8, 16, 32};
const int kTreeMinb[] = {0};

cudaError_t fors_variant(const Batch& b, int lpt, cudaStream_t s) {
    switch (lpt) {
    case 2: return SetImpl<P>::fors<2>(b, s);
    case 4: return SetImpl<P>::fors<4>(b, s);
    case 8: return SetImpl<P>::fors<8>(b, s);
    case 16: return SetImpl<P>::fors<16>(b, s);
    case 32: return SetImpl<P>::fors<32>(b, s);
    }
    return cudaErrorInvalidValue;
}
}  // namespace

extern const SetOps kOps_R128F = {
    SetImpl<P>::keyprep, SetImpl<P>::message, fors_variant, SetImpl<P>::fors_pk,
    TreeVariants<P, 0>::run, TreeVariants<P, 0>::has,
    SetImpl<P>::tree_split, SetImpl<P>::tree_dedup, SetImpl<P>::tree_cached, SetImpl<P>::cache_build,
    SetImpl<P>::wots,       SetImpl<P>::verify,     SetImpl<P>::keygen,
    kForsLpt, 5, 2, kTreeMinb, 1, 0, tree_pol<P>()};

}  // namespace hs
