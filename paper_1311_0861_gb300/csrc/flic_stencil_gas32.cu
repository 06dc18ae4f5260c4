// Candidate launch shapes of the float32 gas kernel (Sec. 2.1, 2.4).  Entry 0
// is the default: 32 x 16 tiles with one thread per updated cell (512 tile + 96
// border cells, 608 threads; the 96 threads without a tile column take 2 x/y
// faces each first), one block per SM (95 registers); with fewer tiles than
// blocks (128 tiles at 256^3) one block per tile column marches the lower planes
// in lockstep and the other blocks share the tops.  Measured at 256^3 (ms per
// launch): 0.424 default, 0.426 over whole tile columns, 0.430 with 4 helper
// faces, 0.456 for the 32 x 12 tile with one thread per tile cell and two blocks
// per SM.
#include "flic_stencil_launch.cuh"

namespace flic {
namespace {
using P = GasPhys<float>;
using C0 = TileCfg<32, 16, 1, false, true, 2>;
using C1 = TileCfg<32, 16, 1, false, true, 4>;
using C2 = TileCfg<32, 12, 2, false, false, 0>;
using C3 = TileCfg<32, 8, 3, false, false, 0>;
using C4 = TileCfg<32, 8, 2, false, true, 4>;
#define FLIC_GAS_32X16 "32x16 tile, 608 threads (one per updated cell), 1 block/SM"
const StencilCand<float> kCands[] = {
    FLIC_STENCIL_CAND(P, float, C0, FLIC_GAS_32X16 ", 2 x/y faces per helper thread", SPLIT_TOPS),
    FLIC_STENCIL_CAND(P, float, C0, FLIC_GAS_32X16 ", 2 x/y faces per helper thread", SPLIT_BALANCED_WHOLE),
    FLIC_STENCIL_CAND(P, float, C1, FLIC_GAS_32X16 ", 4 x/y faces per helper thread", SPLIT_TOPS),
    FLIC_STENCIL_CAND(P, float, C1, FLIC_GAS_32X16 ", 4 x/y faces per helper thread", SPLIT_BALANCED_WHOLE),
    FLIC_STENCIL_CAND(P, float, C1, FLIC_GAS_32X16 ", 4 x/y faces per helper thread", SPLIT_BALANCED),
    FLIC_STENCIL_CAND(P, float, C2, "32x12 tile, 384 threads, 2 blocks/SM", SPLIT_BALANCED),
    FLIC_STENCIL_CAND(P, float, C2, "32x12 tile, 384 threads, 2 blocks/SM", SPLIT_BALANCED_WHOLE),
    FLIC_STENCIL_CAND(P, float, C2, "32x12 tile, 384 threads, 2 blocks/SM", SPLIT_CHUNK),
    FLIC_STENCIL_CAND(P, float, C3, "32x8 tile, 256 threads, 3 blocks/SM", SPLIT_CHUNK),
    FLIC_STENCIL_CAND(P, float, C3, "32x8 tile, 256 threads, 3 blocks/SM", SPLIT_BALANCED),
    FLIC_STENCIL_CAND(P, float, C4, "32x8 tile, 352 threads (one per updated cell), 2 blocks/SM", SPLIT_CHUNK),
};
#undef FLIC_GAS_32X16
}  // namespace

template <> const StencilCand<float>* gas_cands<float>(int* count) {
    *count = int(sizeof(kCands) / sizeof(kCands[0]));
    return kCands;
}

}  // namespace flic
