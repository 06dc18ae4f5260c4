// Candidate launch shapes of the float32 Boltzmann-moment kernel (Sec. 2.2,
// 2.4).  Entry 0 is the default: 32 x 12 tiles with one thread per updated cell
// (384 tile + 88 border cells, 480 threads; the 96 threads without a tile
// column take 4 x/y faces each first -- measured at 256^3: 2 / 3 / 4 / 5 faces
// 1.059 / 1.052 / 1.047 / 1.062 ms), one block per SM with no register cap,
// balanced split over the resident blocks.
#include "flic_stencil_launch.cuh"

namespace flic {
namespace {
using P = BmePhys<float>;
using C0 = TileCfg<32, 12, 1, false, true, 4>;   // 4 x/y faces per helper thread first
using C1 = TileCfg<32, 8, 1, false, true, 4>;
using C2 = TileCfg<32, 16, 1, false, true, 6>;
using C3 = TileCfg<16, 16, 1, false, true, 4>;
using C4 = TileCfg<32, 8, 1, false, true, 4, true>;
using C5 = TileCfg<32, 8, 1, false, true, 4, true, 1>;
using C6 = TileCfg<32, 12, 1, false, true, 5>;
using C7 = TileCfg<32, 12, 1, false, true, 3>;
const StencilCand<float> kCands[] = {
    FLIC_STENCIL_CAND(P, float, C0, "32x12 tile, 480 threads (one per updated cell), 1 block/SM",
                      SPLIT_BALANCED),
    FLIC_STENCIL_CAND(P, float, C0, "32x12 tile, 480 threads (one per updated cell), 1 block/SM",
                      SPLIT_CHUNK),
    FLIC_STENCIL_CAND(P, float, C1, "32x8 tile, 352 threads (one per updated cell), 1 block/SM",
                      SPLIT_BALANCED),
    FLIC_STENCIL_CAND(P, float, C1, "32x8 tile, 352 threads (one per updated cell), 1 block/SM",
                      SPLIT_BALANCED_WHOLE),
    FLIC_STENCIL_CAND(P, float, C2, "32x16 tile, 608 threads (one per updated cell), 1 block/SM",
                      SPLIT_BALANCED),
    FLIC_STENCIL_CAND(P, float, C3, "16x16 tile, 320 threads (one per updated cell), 1 block/SM",
                      SPLIT_BALANCED),
    FLIC_STENCIL_CAND(P, float, C4,
                      "32x8 tile, 352 threads (one per updated cell), 1 block/SM, one barrier per plane",
                      SPLIT_BALANCED),
    FLIC_STENCIL_CAND(P, float, C5,
                      "32x8 tile, 352 threads (one per updated cell), 1 block/SM, one barrier per plane, "
                      "f' as field pairs",
                      SPLIT_BALANCED),
    FLIC_STENCIL_CAND(P, float, C5,
                      "32x8 tile, 352 threads (one per updated cell), 1 block/SM, one barrier per plane, "
                      "f' as field pairs",
                      SPLIT_BALANCED_WHOLE),
    FLIC_STENCIL_CAND(P, float, C6,
                      "32x12 tile, 480 threads (one per updated cell), 1 block/SM, 5 x/y faces per helper thread",
                      SPLIT_BALANCED),
    FLIC_STENCIL_CAND(P, float, C7,
                      "32x12 tile, 480 threads (one per updated cell), 1 block/SM, 3 x/y faces per helper thread",
                      SPLIT_BALANCED),
};
}  // namespace

template <> const StencilCand<float>* bme_cands<float>(int* count) {
    *count = int(sizeof(kCands) / sizeof(kCands[0]));
    return kCands;
}

}  // namespace flic
