// Shared device helpers of libflic (CUDA, sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace flic {

// Field indices of the 22-field state (structure of arrays, x fastest).
enum Field {
    F_RHO = 0, F_MX, F_MY, F_MZ, F_E, F_EINT,
    F_N = 6, F_QX, F_QY, F_QZ,
    F_NEXX = 10, F_NEYY, F_NEZZ, F_NEXY, F_NEXZ, F_NEYZ,
    F_PXX = 16, F_PYY, F_PZZ, F_PXY, F_PXZ, F_PYZ,
    F_COUNT = 22
};

// Quantities summed per block by the step kernels (double partials).
enum DiagQ {
    Q_MASS_GAS = 0, Q_MASS_BME, Q_MOMX, Q_MOMY, Q_MOMZ,
    Q_EKIN_GAS, Q_EINT_GAS, Q_EKIN_BME, Q_ETHERM_BME, Q_EPOT,
    Q_KAPPA_GAS, Q_KAPPA_BME,
    Q_COUNT = 12
};

// Status bits set by kernels (atomicOr).
enum StatusBits { ST_NONPHYSICAL = 1u };

// Reciprocal, reciprocal square root, square root.  float64 keeps IEEE division
// and sqrt; float32 uses the hardware approximations (the float32 path is
// gated at 1e-4 relative L1 against the float64 oracle).
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rsq(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double sqr_root(double x) { return sqrt(x); }
__device__ __forceinline__ float sqr_root(float x) { return x * rsqrtf(x); }

__host__ __device__ __forceinline__ int wrap_mod(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

template <typename T>
__device__ __forceinline__ bool finite_val(T x) { return isfinite(x); }

// Warp-level reductions.
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Non-negative doubles order like their bit patterns, so a max over them is an
// integer atomicMax on the 64-bit representation.
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
    atomicMax(reinterpret_cast<unsigned long long*>(addr),
              static_cast<unsigned long long>(__double_as_longlong(v)));
}

}  // namespace flic
