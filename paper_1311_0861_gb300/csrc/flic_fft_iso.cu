// Isolated (zero-padded) Poisson solve: the potential of s = rho + n on an N^3
// grid with vacuum boundaries, as the linear convolution of s with the
// point-mass Green's function g(r) = -G h^3 / |r| (cell centres r != 0) and
// g(0) = -G h^2 (3 ln(2 + sqrt 3) - pi/2) (the potential of a uniform unit cube
// at its centre), computed by FFTs of length L = 2N with s zero-padded
// (Hockney-Eastwood).  The paper's Poisson symbol (Sec. 2.3) is periodic; this
// mode serves the isolated collision runs.
//
// The transform of g is computed once per grid (green_init) on the full (2N)^3
// array and kept compressed by its even symmetry as (N+1)^3 reals, with the
// 1/((L/2) L L) scale of the unnormalised inverse folded in.  Per solve, the
// padding is never stored: the x pass reads N^2 rows, the y pass extends N to L
// rows, the z pass reads and writes only the N physical planes, and the inverse
// passes keep the physical octant.
#include <cmath>

#include "flic_fft.h"
#include "flic_fft_kernels.cuh"

namespace flic {

#define FLIC_ISO_SIZES(X) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(256) X(512)

// g on the (L)^3 padded grid with wrapped (minimum-image) cell distances
template <typename T>
__global__ void green_real_kernel(T* __restrict__ g, int L, T gh2, T self) {
    const size_t total = size_t(L) * L * L;
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total;
         i += size_t(gridDim.x) * blockDim.x) {
        const int x = int(i % L), y = int((i / L) % L), z = int(i / (size_t(L) * L));
        const int dx = min(x, L - x), dy = min(y, L - y), dz = min(z, L - z);
        const double r = sqrt(double(dx) * dx + double(dy) * dy + double(dz) * dz);
        g[i] = (r == 0.0) ? T(gh2 * self) : T(double(gh2) / r);
    }
}

// z forward transform of the y-transformed Green's function; keeps Re (the
// transform of an even real function is real) for kz, ky <= L/2, scaled
template <typename T, int L>
__global__ void __launch_bounds__(FftGeom<T, L>::NTC) fft_z_green(const typename C2<T>::t* __restrict__ spec,
                                                                  const typename C2<T>::t* __restrict__ tw,
                                                                  T scale, T* __restrict__ gtab) {
    typedef typename C2<T>::t C;
    typedef FftGeom<T, L> Gm;
    constexpr int MH = Gm::MH, KB = Gm::KB, NTC = Gm::NTC;
    extern __shared__ __align__(16) unsigned char sm[];
    C* A = reinterpret_cast<C*>(sm);
    C* tws = A + L * KB;
    stage_twiddles<C, L>(tws, tw);
    const int k0 = blockIdx.x * KB;
    const int y = blockIdx.y;   // 0 .. L/2
    constexpr size_t zs = size_t(L) * MH;
    for (int t = threadIdx.x; t < L * KB; t += NTC) {
        const int c = t % KB, z = t / KB;
        C v;
        if (k0 + c < MH) v = spec[size_t(y) * MH + size_t(z) * zs + k0 + c];
        else { v.x = T(0); v.y = T(0); }
        A[z * KB + c] = v;
    }
    __syncthreads();
    StockhamIP<C, false, L, KB, KB, 1, true, 1, L, L, NTC>::run(A, tws);
    // layout of the solve's reads: [ky'][kx block][kz'][kx within the block]
    constexpr int NKB = (MH + KB - 1) / KB;
    T* out = gtab + (size_t(y) * NKB + blockIdx.x) * (L / 2 + 1) * KB;
    for (int t = threadIdx.x; t < (L / 2 + 1) * KB; t += NTC) out[t] = A[t].x * scale;   // t = z * KB + c
}

template <typename T, int N>
static cudaError_t prepare_iso_n() {
    constexpr int L = 2 * N;
    typedef FftGeom<T, L> Gm;
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(fft_x_forward<T, L, N>, A, (int)Gm::smem_x))) return e;
    if ((e = cudaFuncSetAttribute(fft_x_forward<T, L, L>, A, (int)Gm::smem_x))) return e;
    if ((e = cudaFuncSetAttribute(fft_x_inverse<T, L, N>, A, (int)Gm::smem_x))) return e;
    if ((e = cudaFuncSetAttribute(fft_y<T, L, N, false>, A, (int)Gm::smem_c))) return e;
    if ((e = cudaFuncSetAttribute(fft_y<T, L, N, true>, A, (int)Gm::smem_c))) return e;
    if ((e = cudaFuncSetAttribute(fft_y<T, L, L, false>, A, (int)Gm::smem_c))) return e;
    if ((e = cudaFuncSetAttribute(fft_z_solve<T, L, N, true>, A, (int)Gm::smem_c))) return e;
    return cudaFuncSetAttribute(fft_z_green<T, L>, A, (int)Gm::smem_c);
}

template <typename T, int N>
static cudaError_t green_init_n(double h, double G, T* gtab, T* greal, void* tmp_spec, const void* tw_v,
                                cudaStream_t st) {
    constexpr int L = 2 * N;
    typedef typename C2<T>::t C;
    typedef FftGeom<T, L> Gm;
    C* spec = reinterpret_cast<C*>(tmp_spec);
    const C* tw = reinterpret_cast<const C*>(tw_v);
    const double self = 3.0 * std::log(2.0 + std::sqrt(3.0)) - 0.5 * 3.14159265358979323846;
    green_real_kernel<T><<<152 * 8, 256, 0, st>>>(greal, L, T(-G * h * h), T(self));
    const int nrows = L * L;
    const int gx = (nrows + Gm::RB - 1) / Gm::RB;
    const int gk = (Gm::MH + Gm::KB - 1) / Gm::KB;
    fft_x_forward<T, L, L><<<gx, Gm::NTX, Gm::smem_x, st>>>(greal, nullptr, spec, nrows, tw, 0, 0);
    fft_y<T, L, L, false><<<dim3(gk, L), Gm::NTC, Gm::smem_c, st>>>(spec, tw, 0);
    const double scale = 1.0 / (double(L / 2) * L * L);
    fft_z_green<T, L><<<dim3(gk, L / 2 + 1), Gm::NTC, Gm::smem_c, st>>>(spec, tw, T(scale), gtab);
    return cudaGetLastError();
}

template <typename T, int N>
static cudaError_t solve_iso_n(const T* rho, const T* nd, T* phi, void* spec_v, const void* tw_v, const T* gtab,
                               cudaStream_t st, int nb, size_t bs_in, size_t bs_phi, size_t bs_spec) {
    constexpr int L = 2 * N;
    typedef typename C2<T>::t C;
    typedef FftGeom<T, L> Gm;
    C* spec = reinterpret_cast<C*>(spec_v);
    const C* tw = reinterpret_cast<const C*>(tw_v);
    const int nrows = N * N;
    const int gx = (nrows + Gm::RB - 1) / Gm::RB;
    const int gk = (Gm::MH + Gm::KB - 1) / Gm::KB;
    fft_x_forward<T, L, N><<<dim3(gx, nb), Gm::NTX, Gm::smem_x, st>>>(rho, nd, spec, nrows, tw, bs_in, bs_spec);
    fft_y<T, L, N, false><<<dim3(gk, N, nb), Gm::NTC, Gm::smem_c, st>>>(spec, tw, bs_spec);
    fft_z_solve<T, L, N, true><<<dim3(gk, L, nb), Gm::NTC, Gm::smem_c, st>>>(spec, tw, nullptr, T(0), gtab, bs_spec);
    fft_y<T, L, N, true><<<dim3(gk, N, nb), Gm::NTC, Gm::smem_c, st>>>(spec, tw, bs_spec);
    fft_x_inverse<T, L, N><<<dim3(gx, nb), Gm::NTX, Gm::smem_x, st>>>(spec, phi, nrows, tw, bs_spec, bs_phi);
    return cudaGetLastError();
}

template <typename T, int N>
static size_t green_elems_n() {
    typedef FftGeom<T, 2 * N> Gm;
    constexpr size_t NKB = (Gm::MH + Gm::KB - 1) / Gm::KB;
    return size_t(N + 1) * (N + 1) * NKB * Gm::KB;
}

template <typename T>
size_t green_table_elems(int N) {
    switch (N) {
#define FLIC_CASE(n) case n: return green_elems_n<T, n>();
        FLIC_ISO_SIZES(FLIC_CASE)
#undef FLIC_CASE
        default: return 0;
    }
}
template size_t green_table_elems<float>(int);
template size_t green_table_elems<double>(int);

int fft_iso_supported(int N) {
    switch (N) {
#define FLIC_CASE(n) case n:
        FLIC_ISO_SIZES(FLIC_CASE)
#undef FLIC_CASE
        return 1;
        default:
            return 0;
    }
}

template <typename T>
cudaError_t fft_prepare_iso(int N) {
    switch (N) {
#define FLIC_CASE(n) case n: return prepare_iso_n<T, n>();
        FLIC_ISO_SIZES(FLIC_CASE)
#undef FLIC_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t green_init(int N, double h, double G, T* gtab, T* greal, void* tmp_spec, const void* tw,
                       cudaStream_t st) {
    switch (N) {
#define FLIC_CASE(n) case n: return green_init_n<T, n>(h, G, gtab, greal, tmp_spec, tw, st);
        FLIC_ISO_SIZES(FLIC_CASE)
#undef FLIC_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t poisson_isolated(const T* rho, const T* nd, T* phi, void* spec, int N, const void* tw, const T* gtab,
                             cudaStream_t st, int nbatch, size_t bs_in, size_t bs_phi, size_t bs_spec) {
    if (nbatch < 1) return cudaErrorInvalidValue;
    switch (N) {
#define FLIC_CASE(n) case n: return solve_iso_n<T, n>(rho, nd, phi, spec, tw, gtab, st, nbatch, bs_in, bs_phi, bs_spec);
        FLIC_ISO_SIZES(FLIC_CASE)
#undef FLIC_CASE
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t fft_prepare_iso<float>(int);
template cudaError_t fft_prepare_iso<double>(int);
template cudaError_t green_init<float>(int, double, double, float*, float*, void*, const void*, cudaStream_t);
template cudaError_t green_init<double>(int, double, double, double*, double*, void*, const void*, cudaStream_t);
template cudaError_t poisson_isolated<float>(const float*, const float*, float*, void*, int, const void*,
                                             const float*, cudaStream_t, int, size_t, size_t, size_t);
template cudaError_t poisson_isolated<double>(const double*, const double*, double*, void*, int, const void*,
                                              const double*, cudaStream_t, int, size_t, size_t, size_t);

}  // namespace flic
