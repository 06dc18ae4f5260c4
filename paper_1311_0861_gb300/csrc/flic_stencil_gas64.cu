// Candidate launch shapes of the float64 gas kernel (Sec. 2.1, 2.4).  Entry 0
// is the default: 32 x 8 tiles, 256 threads, two blocks per SM, z chunks.
#include "flic_stencil_launch.cuh"

namespace flic {
namespace {
using P = GasPhys<double>;
using C0 = TileCfg<32, 8, 2, false, false, 0>;
using C1 = TileCfg<32, 4, 3, false, false, 0>;
const StencilCand<double> kCands[] = {
    FLIC_STENCIL_CAND(P, double, C0, "32x8 tile, 256 threads, 2 blocks/SM", SPLIT_CHUNK),
    FLIC_STENCIL_CAND(P, double, C0, "32x8 tile, 256 threads, 2 blocks/SM", SPLIT_BALANCED),
    FLIC_STENCIL_CAND(P, double, C0, "32x8 tile, 256 threads, 2 blocks/SM", SPLIT_BALANCED_WHOLE),
    FLIC_STENCIL_CAND(P, double, C1, "32x4 tile, 128 threads, 3 blocks/SM", SPLIT_CHUNK),
};
}  // namespace

template <> const StencilCand<double>* gas_cands<double>(int* count) {
    *count = int(sizeof(kCands) / sizeof(kCands[0]));
    return kCands;
}

}  // namespace flic
