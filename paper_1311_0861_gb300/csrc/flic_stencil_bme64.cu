// Candidate launch shapes of the float64 Boltzmann-moment kernel (Sec. 2.2,
// 2.4).  Entry 0 is the default: 32 x 4 tiles with one thread per updated cell
// and the energy tensor staged in shared memory, one block per SM, z chunks.
#include "flic_stencil_launch.cuh"

namespace flic {
namespace {
using P = BmePhys<double>;
using C0 = TileCfg<32, 4, 1, true, true, 4>;
using C1 = TileCfg<16, 8, 1, true, true, 4>;
const StencilCand<double> kCands[] = {
    FLIC_STENCIL_CAND(P, double, C0, "32x4 tile, 224 threads (one per updated cell), staged energy tensor",
                      SPLIT_CHUNK),
    FLIC_STENCIL_CAND(P, double, C0,
                      "32x4 tile, 224 threads (one per updated cell), staged energy tensor",
                      SPLIT_BALANCED),
    FLIC_STENCIL_CAND(P, double, C1, "16x8 tile, 192 threads (one per updated cell), staged energy tensor",
                      SPLIT_CHUNK),
};
}  // namespace

template <> const StencilCand<double>* bme_cands<double>(int* count) {
    *count = int(sizeof(kCands) / sizeof(kCands[0]));
    return kCands;
}

}  // namespace flic
