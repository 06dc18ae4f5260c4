// Candidate launch shapes of the float32 gas kernel (Sec. 2.1, 2.4).  Entry 0
// is the default: 32 x 12 tiles, one thread per tile cell (border cells in a
// second round), two blocks per SM, balanced split in lockstep half columns
// (measured at 256^3: 0.452 ms, vs 0.464 with whole columns, 0.474 in z chunks
// and 0.473 for 32 x 8 with three blocks per SM).
#include "flic_stencil_launch.cuh"

namespace flic {
namespace {
using P = GasPhys<float>;
using C0 = TileCfg<32, 12, 2, false, false, 0>;
using C1 = TileCfg<32, 8, 3, false, false, 0>;
using C2 = TileCfg<32, 8, 2, false, true, 4>;
using C3 = TileCfg<32, 16, 1, false, false, 0>;
using C4 = TileCfg<64, 4, 3, false, false, 0>;
const StencilCand<float> kCands[] = {
    FLIC_STENCIL_CAND(P, float, C0, "32x12 tile, 384 threads, 2 blocks/SM", SPLIT_BALANCED),
    FLIC_STENCIL_CAND(P, float, C0, "32x12 tile, 384 threads, 2 blocks/SM", SPLIT_BALANCED_WHOLE),
    FLIC_STENCIL_CAND(P, float, C0, "32x12 tile, 384 threads, 2 blocks/SM", SPLIT_CHUNK),
    FLIC_STENCIL_CAND(P, float, C1, "32x8 tile, 256 threads, 3 blocks/SM", SPLIT_CHUNK),
    FLIC_STENCIL_CAND(P, float, C1, "32x8 tile, 256 threads, 3 blocks/SM", SPLIT_BALANCED),
    FLIC_STENCIL_CAND(P, float, C1, "32x8 tile, 256 threads, 3 blocks/SM", SPLIT_BALANCED_WHOLE),
    FLIC_STENCIL_CAND(P, float, C2, "32x8 tile, 352 threads (one per updated cell), 2 blocks/SM",
                      SPLIT_CHUNK),
    FLIC_STENCIL_CAND(P, float, C3, "32x16 tile, 512 threads, 1 block/SM", SPLIT_CHUNK),
    FLIC_STENCIL_CAND(P, float, C4, "64x4 tile, 256 threads, 3 blocks/SM", SPLIT_CHUNK),
};
}  // namespace

template <> const StencilCand<float>* gas_cands<float>(int* count) {
    *count = int(sizeof(kCands) / sizeof(kCands[0]));
    return kCands;
}

}  // namespace flic
