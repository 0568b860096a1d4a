// set_256s.cu -- every kernel instantiated for SPHINCS+-SHA2-256s (a
// small-signature set: 2^h' = 256 leaves per XMSS tree, FORS height 14), with
// the launch-shape variants the tuner may pick from.
#include "set_impl.cuh"

namespace hs {
namespace {
using P = P256s;
const int kForsLpt[] = {16, 32};
const int kTreeMinb[] = {0};

cudaError_t fors_variant(const Batch& b, int lpt, cudaStream_t s) {
    switch (lpt) {
    case 16: return SetImpl<P>::fors<16>(b, s);
    case 32: return SetImpl<P>::fors<32>(b, s);
    }
    return cudaErrorInvalidValue;
}
}  // namespace

extern const SetOps kOps_256S = {
    SetImpl<P>::keyprep, SetImpl<P>::message, fors_variant, SetImpl<P>::fors_pk,
    TreeVariants<P, 0>::run, TreeVariants<P, 0>::has,
    SetImpl<P>::tree_split, SetImpl<P>::tree_dedup, SetImpl<P>::tree_cached, SetImpl<P>::cache_build,
    SetImpl<P>::wots,       SetImpl<P>::verify,     SetImpl<P>::keygen,
    kForsLpt, 2, 32, kTreeMinb, 1, 0, tree_pol<P>()};

}  // namespace hs
