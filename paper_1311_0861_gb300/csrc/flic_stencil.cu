// Launchers of the fused fluid-step kernels (instantiations for float64 and float32).
#include "flic_internal.h"

namespace flic {

namespace {

template <typename T> struct Tiles;
// 32 x 8 column tiles; minimum resident blocks per SM for the register budget
// (float32: 3 gas / 2 moment blocks; float64: 2 gas / 1 moment block, whose
// shared memory takes most of the SM).
template <> struct Tiles<float> {
    static constexpr int GX = 32, GY = 8, GB = 3, BX = 32, BY = 8, BB = 2;
};
template <> struct Tiles<double> {
    static constexpr int GX = 32, GY = 8, GB = 2, BX = 32, BY = 8, BB = 1;
};

template <class P, typename T, int TX, int TY>
StepCfg make_cfg(int N, int tz) {
    StepCfg c;
    c.tx = TX;
    c.ty = TY;
    c.tiles_x = (N + TX - 1) / TX;
    c.tiles_y = (N + TY - 1) / TY;
    if (tz <= 0) {
        // enough blocks for several waves on 152 SMs, chunks of >= 16 planes
        const int tiles = c.tiles_x * c.tiles_y;
        int chunks = (4 * 152 * 2 + tiles - 1) / tiles;
        tz = (N + chunks - 1) / chunks;
        if (tz < 16) tz = 16;
    }
    if (tz > N) tz = N;
    c.tz = tz;
    c.blocks_z = (N + tz - 1) / tz;
    c.threads = TX * TY;
    c.smem = Geom<P, T, TX, TY>::smem_bytes;
    return c;
}

template <class P, typename T, int TX, int TY, int MB>
cudaError_t prepare() {
    return cudaFuncSetAttribute(fluid_step_kernel<P, T, TX, TY, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Geom<P, T, TX, TY>::smem_bytes);
}

template <class P, typename T, int TX, int TY, int MB>
cudaError_t launch(const StencilArgs<T>& a, const StepCfg& c, cudaStream_t st) {
    fluid_step_kernel<P, T, TX, TY, MB><<<dim3(c.tiles_x * c.tiles_y, c.blocks_z), c.threads, c.smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

template <typename T> StepCfg gas_cfg(int N, int tz) {
    return make_cfg<GasPhys<T>, T, Tiles<T>::GX, Tiles<T>::GY>(N, tz);
}
template <typename T> StepCfg bme_cfg(int N, int tz) {
    return make_cfg<BmePhys<T>, T, Tiles<T>::BX, Tiles<T>::BY>(N, tz);
}
template <typename T> cudaError_t launch_gas(const StencilArgs<T>& a, const StepCfg& c, cudaStream_t st) {
    return launch<GasPhys<T>, T, Tiles<T>::GX, Tiles<T>::GY, Tiles<T>::GB>(a, c, st);
}
template <typename T> cudaError_t launch_bme(const StencilArgs<T>& a, const StepCfg& c, cudaStream_t st) {
    return launch<BmePhys<T>, T, Tiles<T>::BX, Tiles<T>::BY, Tiles<T>::BB>(a, c, st);
}

template <typename T> cudaError_t stencil_prepare() {
    cudaError_t e = prepare<GasPhys<T>, T, Tiles<T>::GX, Tiles<T>::GY, Tiles<T>::GB>();
    if (e != cudaSuccess) return e;
    return prepare<BmePhys<T>, T, Tiles<T>::BX, Tiles<T>::BY, Tiles<T>::BB>();
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
