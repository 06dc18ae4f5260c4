// Candidate launch shapes of the float32 Boltzmann-moment kernel (Sec. 2.2,
// 2.4).  Entry 0 is the default: 32 x 12 tiles with one thread per updated cell
// (384 tile + 88 border cells, 480 threads; the 96 threads without a tile
// column take 4 x/y faces each first), the transported state f' as field pairs,
// one block per SM with no register cap, balanced split over the resident
// blocks.  Measured at 256^3 (ms per launch): 0.926 default, 0.935 with 3 helper
// faces, 0.951 with 5, 0.961 with f' as scalar rows.
#include "flic_stencil_launch.cuh"

namespace flic {
namespace {
using P = BmePhys<float>;
using C0 = TileCfg<32, 12, 1, false, true, 4, false, 1>;
using C1 = TileCfg<32, 12, 1, false, true, 3, false, 1>;
using C2 = TileCfg<32, 12, 1, false, true, 4, false, 0>;
using C3 = TileCfg<32, 8, 1, false, true, 4, false, 1>;
using C4 = TileCfg<32, 8, 1, false, true, 4, true, 1>;
using C5 = TileCfg<32, 8, 1, false, true, 4, false, 0>;
using C6 = TileCfg<16, 16, 1, false, true, 4, false, 1>;
#define FLIC_BME_32X12 "32x12 tile, 480 threads (one per updated cell), 1 block/SM"
#define FLIC_BME_32X8 "32x8 tile, 352 threads (one per updated cell), 1 block/SM"
const StencilCand<float> kCands[] = {
    FLIC_STENCIL_CAND(P, float, C0, FLIC_BME_32X12 ", f' as field pairs", SPLIT_BALANCED),
    FLIC_STENCIL_CAND(P, float, C0, FLIC_BME_32X12 ", f' as field pairs", SPLIT_BALANCED_WHOLE),
    FLIC_STENCIL_CAND(P, float, C0, FLIC_BME_32X12 ", f' as field pairs", SPLIT_CHUNK),
    FLIC_STENCIL_CAND(P, float, C1, FLIC_BME_32X12 ", f' as field pairs, 3 x/y faces per helper thread",
                      SPLIT_BALANCED),
    FLIC_STENCIL_CAND(P, float, C2, FLIC_BME_32X12 ", f' as scalar rows", SPLIT_BALANCED),
    FLIC_STENCIL_CAND(P, float, C3, FLIC_BME_32X8 ", f' as field pairs", SPLIT_BALANCED),
    FLIC_STENCIL_CAND(P, float, C4, FLIC_BME_32X8 ", one barrier per plane, f' as field pairs", SPLIT_BALANCED),
    FLIC_STENCIL_CAND(P, float, C4, FLIC_BME_32X8 ", one barrier per plane, f' as field pairs",
                      SPLIT_BALANCED_WHOLE),
    FLIC_STENCIL_CAND(P, float, C5, FLIC_BME_32X8 ", f' as scalar rows", SPLIT_BALANCED_WHOLE),
    FLIC_STENCIL_CAND(P, float, C6, "16x16 tile, 320 threads (one per updated cell), 1 block/SM, f' as field pairs",
                      SPLIT_BALANCED),    FLIC_STENCIL_CAND(P, float, C0, FLIC_BME_32X12 ", f' as field pairs", SPLIT_TOPS),
    FLIC_STENCIL_CAND(P, float, C4, FLIC_BME_32X8 ", one barrier per plane, f' as field pairs", SPLIT_TOPS),
};
#undef FLIC_BME_32X12
#undef FLIC_BME_32X8
}  // namespace

template <> const StencilCand<float>* bme_cands<float>(int* count) {
    *count = int(sizeof(kCands) / sizeof(kCands[0]));
    return kCands;
}

}  // namespace flic
