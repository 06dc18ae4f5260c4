// Host-side launchers of one compiled launch shape of a fused fluid kernel, and
// the table entry through which the launch-shape tuner and the step reach it.
// Included by the translation units that instantiate the candidate shapes.
#pragma once

#include "flic_internal.h"

namespace flic {

template <class P, typename T, class C>
struct StencilOps {
    // Launch geometry.  tz > 0 (batched ensembles): a (tile, z chunk) grid of
    // that chunk height.  tz <= 0 (single grid): SPLIT_BALANCED -- one block per
    // resident slot (the kernel's occupancy times the SM count), whole tile
    // columns in lockstep rounds, then an equal share of the remaining (tile,
    // plane) updates, so no wave is partly empty (at least 8 planes a block);
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
            if (split == SPLIT_BALANCED) {
                long b = slots;
                if (b > tiles * N / 8) b = tiles * N / 8;
                if (b < 1) b = 1;
                c.tz = 0;
                c.blocks_z = 1;
                c.balanced = int(b);
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

    static cudaError_t prepare() {
        cudaError_t e = cudaFuncSetAttribute(fluid_step_kernel<P, T, C, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Geom<P, T, C>::smem_bytes);
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(fluid_step_kernel<P, T, C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)Geom<P, T, C>::smem_bytes);
    }

    static cudaError_t launch(const StencilArgs<T>& a, const StepCfg& c, cudaStream_t st) {
        BatchArgs<T> none{nullptr, nullptr};
        const dim3 grid = c.balanced > 0 ? dim3(c.balanced) : dim3(c.tiles_x * c.tiles_y, c.blocks_z);
        if (a.outflow)
            fluid_step_kernel<P, T, C, true><<<grid, c.threads, c.smem, st>>>(a, none);
        else
            fluid_step_kernel<P, T, C, false><<<grid, c.threads, c.smem, st>>>(a, none);
        return cudaGetLastError();
    }

    static cudaError_t launch_batch(const StencilArgs<T>* table, const WorkItem* work, int nwork, bool outflow,
                                    cudaStream_t st) {
        StencilArgs<T> unused{};
        BatchArgs<T> b{table, work};
        constexpr int nth = Geom<P, T, C>::NTH;
        constexpr size_t smem = Geom<P, T, C>::smem_bytes;
        if (outflow)
            fluid_step_kernel<P, T, C, true><<<nwork, nth, smem, st>>>(unused, b);
        else
            fluid_step_kernel<P, T, C, false><<<nwork, nth, smem, st>>>(unused, b);
        return cudaGetLastError();
    }
};

// Table entry of candidate shape C with z split `split` for single grids.
#define FLIC_STENCIL_CAND(P, T, C, NAME, SPLIT)                                                       \
    StencilCand<T> {                                                                                  \
        NAME, SPLIT, &StencilOps<P, T, C>::cfg, &StencilOps<P, T, C>::prepare, &StencilOps<P, T, C>::launch, \
            &StencilOps<P, T, C>::launch_batch                                                        \
    }

}  // namespace flic
