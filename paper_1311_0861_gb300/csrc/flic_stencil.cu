// Launchers of the fused fluid-step kernels (instantiations for float64 and float32).
#include "flic_internal.h"

namespace flic {

namespace {

template <typename T> struct Tiles;
// Column tiles, minimum resident blocks per SM (register budget) and whether
// the moment energy tensor is staged in shared memory (BS) or read directly.
// float32 moments: 32 x 8 tiles, two blocks per SM (measured faster than one
// 32 x 16 block with staging, whose single 16-warp barrier group issues worse).
template <> struct Tiles<float> {
    static constexpr int GX = 32, GY = 8, GB = 3, BX = 32, BY = 8, BB = 2;
    static constexpr bool BS = false;
};
template <> struct Tiles<double> {
    static constexpr int GX = 32, GY = 8, GB = 2, BX = 32, BY = 4, BB = 1;
    static constexpr bool BS = true;
};

// Launch geometry: the z-chunk height minimises (waves of resident blocks) x
// (planes a block marches, including its 4-plane warm-up), using the kernel's
// measured occupancy and the device's SM count.
template <class P, typename T, int TX, int TY, int MB, bool SX>
StepCfg make_cfg(int N, int tz) {
    StepCfg c;
    c.tx = TX;
    c.ty = TY;
    c.tiles_x = (N + TX - 1) / TX;
    c.tiles_y = (N + TY - 1) / TY;
    c.threads = TX * TY;
    c.smem = Geom<P, T, TX, TY, SX>::smem_bytes;
    if (tz <= 0) {
        int dev = 0, sms = 152, per_sm = 1;
        if (cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fluid_step_kernel<P, T, TX, TY, MB, SX>,
                                                      c.threads, c.smem);
        if (per_sm < 1) per_sm = 1;
        const long slots = long(sms) * per_sm;
        const long tiles = long(c.tiles_x) * c.tiles_y;
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

template <class P, typename T, int TX, int TY, int MB, bool SX>
cudaError_t prepare() {
    return cudaFuncSetAttribute(fluid_step_kernel<P, T, TX, TY, MB, SX>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Geom<P, T, TX, TY, SX>::smem_bytes);
}

template <class P, typename T, int TX, int TY, int MB, bool SX>
cudaError_t launch(const StencilArgs<T>& a, const StepCfg& c, cudaStream_t st) {
    BatchArgs<T> none{nullptr, nullptr};
    fluid_step_kernel<P, T, TX, TY, MB, SX>
        <<<dim3(c.tiles_x * c.tiles_y, c.blocks_z), c.threads, c.smem, st>>>(a, none);
    return cudaGetLastError();
}

template <class P, typename T, int TX, int TY, int MB, bool SX>
cudaError_t launch_batch(const StencilArgs<T>* table, const WorkItem* work, int nwork, cudaStream_t st) {
    StencilArgs<T> unused{};
    BatchArgs<T> b{table, work};
    fluid_step_kernel<P, T, TX, TY, MB, SX>
        <<<nwork, TX * TY, Geom<P, T, TX, TY, SX>::smem_bytes, st>>>(unused, b);
    return cudaGetLastError();
}

}  // namespace

template <typename T> StepCfg gas_cfg(int N, int tz) {
    return make_cfg<GasPhys<T>, T, Tiles<T>::GX, Tiles<T>::GY, Tiles<T>::GB, false>(N, tz);
}
template <typename T> StepCfg bme_cfg(int N, int tz) {
    return make_cfg<BmePhys<T>, T, Tiles<T>::BX, Tiles<T>::BY, Tiles<T>::BB, Tiles<T>::BS>(N, tz);
}
template <typename T> cudaError_t launch_gas(const StencilArgs<T>& a, const StepCfg& c, cudaStream_t st) {
    return launch<GasPhys<T>, T, Tiles<T>::GX, Tiles<T>::GY, Tiles<T>::GB, false>(a, c, st);
}
template <typename T> cudaError_t launch_bme(const StencilArgs<T>& a, const StepCfg& c, cudaStream_t st) {
    return launch<BmePhys<T>, T, Tiles<T>::BX, Tiles<T>::BY, Tiles<T>::BB, Tiles<T>::BS>(a, c, st);
}

template <typename T>
cudaError_t launch_gas_batch(const StencilArgs<T>* table, const WorkItem* work, int nwork, cudaStream_t st) {
    return launch_batch<GasPhys<T>, T, Tiles<T>::GX, Tiles<T>::GY, Tiles<T>::GB, false>(table, work, nwork, st);
}
template <typename T>
cudaError_t launch_bme_batch(const StencilArgs<T>* table, const WorkItem* work, int nwork, cudaStream_t st) {
    return launch_batch<BmePhys<T>, T, Tiles<T>::BX, Tiles<T>::BY, Tiles<T>::BB, Tiles<T>::BS>(table, work, nwork,
                                                                                              st);
}
template cudaError_t launch_gas_batch<float>(const StencilArgs<float>*, const WorkItem*, int, cudaStream_t);
template cudaError_t launch_gas_batch<double>(const StencilArgs<double>*, const WorkItem*, int, cudaStream_t);
template cudaError_t launch_bme_batch<float>(const StencilArgs<float>*, const WorkItem*, int, cudaStream_t);
template cudaError_t launch_bme_batch<double>(const StencilArgs<double>*, const WorkItem*, int, cudaStream_t);

template <typename T> cudaError_t stencil_prepare() {
    cudaError_t e = prepare<GasPhys<T>, T, Tiles<T>::GX, Tiles<T>::GY, Tiles<T>::GB, false>();
    if (e != cudaSuccess) return e;
    return prepare<BmePhys<T>, T, Tiles<T>::BX, Tiles<T>::BY, Tiles<T>::BB, Tiles<T>::BS>();
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
