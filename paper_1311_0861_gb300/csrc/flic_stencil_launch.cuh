// Host-side launchers of one compiled launch shape of a fused fluid kernel, and
// the table entry through which the launch-shape tuner and the step reach it.
// Included by the translation units that instantiate the candidate shapes.
#pragma once

#include <algorithm>

#include "flic_internal.h"

namespace flic {

template <class P, typename T, class C>
struct StencilOps {
    // Launch geometry.  tz > 0 (batched ensembles): a (tile, z chunk) grid of
    // that chunk height.  tz <= 0 (single grid): SPLIT_BALANCED -- one block per
    // resident slot (the kernel's occupancy times the SM count), whole units in
    // lockstep rounds, then an equal share of the remaining (unit, plane)
    // updates, so no wave is partly empty (at least 8 planes a block); a unit is
    // a tile column, or with fewer tiles than blocks 1/K of one (K = 2, 4, 8,
    // at least 16 planes; SPLIT_BALANCED_WHOLE keeps whole columns);
    // SPLIT_TOPS -- with fewer tiles than blocks, one block per tile column over
    // planes [0, H) in lockstep and the remaining blocks sharing the tops;
    // SPLIT_CHUNK -- a (tile, chunk) grid whose chunk height minimises
    // waves x (chunk + 4).
    static StepCfg cfg(int N, int tz, int split) {
        StepCfg c;
        c.tx = C::TX;
        c.ty = C::TY;
        c.tiles_x = (N + C::TX - 1) / C::TX;
        c.tiles_y = (N + C::TY - 1) / C::TY;
        c.threads = Geom<P, T, C>::NTH;
        c.smem = Geom<P, T, C>::smem_bytes;
        if (tz <= 0) {
            int dev = 0, sms = 152, per_sm = 1;
            if (cudaGetDevice(&dev) == cudaSuccess)
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fluid_step_kernel<P, T, C, false>, c.threads,
                                                          c.smem);
            if (per_sm < 1) per_sm = 1;
            const long slots = long(sms) * per_sm;
            const long tiles = long(c.tiles_x) * c.tiles_y;
            if (split == SPLIT_BALANCED || split == SPLIT_BALANCED_WHOLE || split == SPLIT_TOPS) {
                long b = slots;
                if (b > tiles * N / 8) b = tiles * N / 8;
                if (b < 1) b = 1;
                c.tz = 0;
                c.blocks_z = 1;
                c.balanced = int(b);
                // fewer tiles than blocks: cut each tile column into K equal parts
                // (at least 16 planes) so that whole units still fill a round
                c.zparts = 1;
                for (int K = 2; split == SPLIT_BALANCED && K <= 8 && tiles * c.zparts < b; K *= 2)
                    if (N % K == 0 && N / K >= 16) c.zparts = K;
                // tops: the height H of the lockstep part that balances its blocks
                // (H planes + 2 warm-up) against the tops' blocks (their share of
                // T (N - H) planes, + 2 warm-up planes per segment)
                if (split == SPLIT_TOPS && tiles < b) {
                    double best = -1.0;
                    for (int H = 8; H < N; ++H) {
                        const double share = double(tiles) * (N - H) / double(b - tiles);
                        const double segs = share / (N - H) + 1.0;
                        const double cost = std::max(double(H + 2), share + 2.0 * segs);
                        if (best < 0.0 || cost < best) { best = cost; c.ztop = H; }
                    }
                }
                return c;
            }
            long best = -1;
            for (int bz = 1; bz <= N / 8 || bz == 1; ++bz) {
                const int t = (N + bz - 1) / bz;
                const long blocks = tiles * ((N + t - 1) / t);
                const long waves = (blocks + slots - 1) / slots;
                const long cost = waves * (t + 4);
                if (best < 0 || cost < best) { best = cost; tz = t; }
            }
        }
        if (tz > N) tz = N;
        c.tz = tz;
        c.blocks_z = (N + tz - 1) / tz;
        return c;
    }

    template <bool OUT, bool COOL>
    static cudaError_t set_smem() {
        return cudaFuncSetAttribute(fluid_step_kernel<P, T, C, OUT, COOL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)Geom<P, T, C>::smem_bytes);
    }

    static cudaError_t prepare() {
        cudaError_t e = set_smem<false, false>();
        if (e == cudaSuccess) e = set_smem<true, false>();
        if constexpr (P::COOLS) {
            if (e == cudaSuccess) e = set_smem<false, true>();
            if (e == cudaSuccess) e = set_smem<true, true>();
        }
        return e;
    }

    // the instance for the boundary kind and the cooling switch
    static cudaError_t go(bool out, bool cool, dim3 grid, int nth, size_t smem, cudaStream_t st,
                          const StencilArgs<T>& a, BatchArgs<T> b) {
        if constexpr (P::COOLS) {
            if (cool) {
                if (out)
                    fluid_step_kernel<P, T, C, true, true><<<grid, nth, smem, st>>>(a, b);
                else
                    fluid_step_kernel<P, T, C, false, true><<<grid, nth, smem, st>>>(a, b);
                return cudaGetLastError();
            }
        }
        if (out)
            fluid_step_kernel<P, T, C, true, false><<<grid, nth, smem, st>>>(a, b);
        else
            fluid_step_kernel<P, T, C, false, false><<<grid, nth, smem, st>>>(a, b);
        return cudaGetLastError();
    }

    static cudaError_t launch(const StencilArgs<T>& a, const StepCfg& c, cudaStream_t st) {
        const dim3 grid = c.balanced > 0 ? dim3(c.balanced) : dim3(c.tiles_x * c.tiles_y, c.blocks_z);
        return go(a.outflow != 0, a.cool != T(0), grid, c.threads, c.smem, st, a, BatchArgs<T>{nullptr, nullptr});
    }

    static cudaError_t launch_batch(const StencilArgs<T>* table, const WorkItem* work, int nwork, bool outflow,
                                    bool cool, cudaStream_t st) {
        StencilArgs<T> unused{};
        return go(outflow, cool, dim3(nwork), Geom<P, T, C>::NTH, Geom<P, T, C>::smem_bytes, st, unused,
                  BatchArgs<T>{table, work});
    }
};

// Table entry of candidate shape C with z split `split` for single grids.
#define FLIC_STENCIL_CAND(P, T, C, NAME, SPLIT)                                                       \
    StencilCand<T> {                                                                                  \
        NAME, SPLIT, &StencilOps<P, T, C>::cfg, &StencilOps<P, T, C>::prepare, &StencilOps<P, T, C>::launch, \
            &StencilOps<P, T, C>::launch_batch                                                        \
    }

}  // namespace flic
