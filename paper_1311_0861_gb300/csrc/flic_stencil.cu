// Launchers of the fused fluid-step kernels (instantiations for float64 and float32).
#include "flic_internal.h"

namespace flic {

namespace {

template <typename T> struct Tiles;
// Launch shapes (TileCfg: tile, min blocks per SM, staged energy tensor, one
// thread per updated cell, helper face rounds), chosen by measurement at 256^3.
// float32 gas: 32 x 8, one thread per tile cell, three blocks per SM.
// float32 moments: 32 x 12 with 480 threads (384 tile + 96 helpers taking 5 faces
// each first), one block per SM and no register cap -- faster than 256-thread
// blocks two per SM, whose 128-register cap spills and whose border cells take
// a second phase-1 round (helper rounds 5 / 6 / 7: 1.153 / 1.164 / 1.175 ms);
// the balanced split over its 152 resident blocks (whole tile columns in
// lockstep rounds, then an even share of the rest) beats the chunked grid
// (1.083 vs 1.154 ms; DRAM traffic 1.18x the compulsory bytes, vs 2.46x for a
// plain tile-major share, whose concurrent blocks no longer share halos in
// L2), while the gas kernel keeps the chunked grid (0.473 vs 0.492 ms).
template <> struct Tiles<float> {
    using Gas = TileCfg<32, 8, 3, false, false, 0>;
    using Bme = TileCfg<32, 12, 1, false, true, 5, true>;
};
template <> struct Tiles<double> {
    using Gas = TileCfg<32, 8, 2, false, false, 0>;
    using Bme = TileCfg<32, 4, 1, true, true, 4>;
};

// Launch geometry.  tz > 0 (batched ensembles): a (tile, z chunk) grid of that
// chunk height.  tz <= 0 (single grid): with C::BAL a balanced split -- one
// block per resident slot (the kernel's occupancy times the SM count), each
// taking an equal share of the tile-major (tile, plane) sequence, so no wave is
// partly empty (at least 8 planes a block); else a (tile, chunk) grid whose
// chunk height minimises waves x (chunk + 4).
template <class P, typename T, class C>
StepCfg make_cfg(int N, int tz) {
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
        if (C::BAL) {
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

template <class P, typename T, class C>
cudaError_t prepare() {
    cudaError_t e = cudaFuncSetAttribute(fluid_step_kernel<P, T, C, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Geom<P, T, C>::smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fluid_step_kernel<P, T, C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Geom<P, T, C>::smem_bytes);
}

template <class P, typename T, class C>
cudaError_t launch(const StencilArgs<T>& a, const StepCfg& c, cudaStream_t st) {
    BatchArgs<T> none{nullptr, nullptr};
    const dim3 grid = c.balanced > 0 ? dim3(c.balanced) : dim3(c.tiles_x * c.tiles_y, c.blocks_z);
    if (a.outflow)
        fluid_step_kernel<P, T, C, true><<<grid, c.threads, c.smem, st>>>(a, none);
    else
        fluid_step_kernel<P, T, C, false><<<grid, c.threads, c.smem, st>>>(a, none);
    return cudaGetLastError();
}

template <class P, typename T, class C>
cudaError_t launch_batch(const StencilArgs<T>* table, const WorkItem* work, int nwork, bool outflow,
                         cudaStream_t st) {
    StencilArgs<T> unused{};
    BatchArgs<T> b{table, work};
    if (outflow)
        fluid_step_kernel<P, T, C, true><<<nwork, Geom<P, T, C>::NTH, Geom<P, T, C>::smem_bytes, st>>>(unused, b);
    else
        fluid_step_kernel<P, T, C, false><<<nwork, Geom<P, T, C>::NTH, Geom<P, T, C>::smem_bytes, st>>>(unused, b);
    return cudaGetLastError();
}

}  // namespace

template <typename T> StepCfg gas_cfg(int N, int tz) {
    return make_cfg<GasPhys<T>, T, typename Tiles<T>::Gas>(N, tz);
}
template <typename T> StepCfg bme_cfg(int N, int tz) {
    return make_cfg<BmePhys<T>, T, typename Tiles<T>::Bme>(N, tz);
}
template <typename T> cudaError_t launch_gas(const StencilArgs<T>& a, const StepCfg& c, cudaStream_t st) {
    return launch<GasPhys<T>, T, typename Tiles<T>::Gas>(a, c, st);
}
template <typename T> cudaError_t launch_bme(const StencilArgs<T>& a, const StepCfg& c, cudaStream_t st) {
    return launch<BmePhys<T>, T, typename Tiles<T>::Bme>(a, c, st);
}

template <typename T>
cudaError_t launch_gas_batch(const StencilArgs<T>* table, const WorkItem* work, int nwork, bool outflow,
                             cudaStream_t st) {
    return launch_batch<GasPhys<T>, T, typename Tiles<T>::Gas>(table, work, nwork, outflow, st);
}
template <typename T>
cudaError_t launch_bme_batch(const StencilArgs<T>* table, const WorkItem* work, int nwork, bool outflow,
                             cudaStream_t st) {
    return launch_batch<BmePhys<T>, T, typename Tiles<T>::Bme>(table, work, nwork, outflow, st);
}
template cudaError_t launch_gas_batch<float>(const StencilArgs<float>*, const WorkItem*, int, bool, cudaStream_t);
template cudaError_t launch_gas_batch<double>(const StencilArgs<double>*, const WorkItem*, int, bool, cudaStream_t);
template cudaError_t launch_bme_batch<float>(const StencilArgs<float>*, const WorkItem*, int, bool, cudaStream_t);
template cudaError_t launch_bme_batch<double>(const StencilArgs<double>*, const WorkItem*, int, bool, cudaStream_t);

template <typename T> cudaError_t stencil_prepare() {
    cudaError_t e = prepare<GasPhys<T>, T, typename Tiles<T>::Gas>();
    if (e != cudaSuccess) return e;
    return prepare<BmePhys<T>, T, typename Tiles<T>::Bme>();
}
template cudaError_t stencil_prepare<float>();
template cudaError_t stencil_prepare<double>();

template StepCfg gas_cfg<float>(int, int);
template StepCfg gas_cfg<double>(int, int);
template StepCfg bme_cfg<float>(int, int);
template StepCfg bme_cfg<double>(int, int);
template cudaError_t launch_gas<float>(const StencilArgs<float>&, const StepCfg&, cudaStream_t);
template cudaError_t launch_gas<double>(const StencilArgs<double>&, const StepCfg&, cudaStream_t);
template cudaError_t launch_bme<float>(const StencilArgs<float>&, const StepCfg&, cudaStream_t);
template cudaError_t launch_bme<double>(const StencilArgs<double>&, const StepCfg&, cudaStream_t);

}  // namespace flic
