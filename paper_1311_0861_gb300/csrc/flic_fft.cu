// Periodic Poisson solve of Sec. 2.3 (transform length = physical extent = N):
//   Phi_hat(k) = -4 pi G h^2 s_hat(k) / (6 (1 - prod_d (1 - 2/3 sin^2(pi k_d / N)))),
//   Phi_hat(0) = 0,  s = rho + n.
// (The printed symbol has no minus sign; Laplace(Phi) = 4 pi rho of Sec. 2 fixes it.)
// Five launches, each one read and one write of the data:
//   X  real-to-complex along x (s = rho + n summed while loading);
//   Y  complex along y (forward);
//   Z  complex along z forward, multiply by the symbol and the 1/N^3 scale, inverse;
//   Y  complex along y (inverse);
//   X  complex-to-real along x, writes Phi.
// The symbol is evaluated as 6 (a_x + f_x (a_y + f_y a_z)), a_d = 2/3 sin^2 and
// f = 1 - a, which has no cancellation at low k in float32.
#include "flic_fft.h"
#include "flic_fft_kernels.cuh"

namespace flic {

#define FLIC_FFT_SIZES(X) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512)

int fft_plan_init(int N, FftPlans* p) {
    (void)p;
    switch (N) {
#define FLIC_CASE(n) case n:
        FLIC_FFT_SIZES(FLIC_CASE)
#undef FLIC_CASE
        return 0;
        default:
            return -1;
    }
}

template <typename T, int N>
static cudaError_t prepare_n() {
    typedef FftGeom<T, N> Gm;
    cudaError_t e;
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if ((e = cudaFuncSetAttribute(fft_x_forward<T, N, N>, A, (int)Gm::smem_x))) return e;
    if ((e = cudaFuncSetAttribute(fft_x_inverse<T, N, N>, A, (int)Gm::smem_x))) return e;
    if ((e = cudaFuncSetAttribute(fft_y<T, N, N, false>, A, (int)Gm::smem_c))) return e;
    if ((e = cudaFuncSetAttribute(fft_y<T, N, N, true>, A, (int)Gm::smem_c))) return e;
    return cudaFuncSetAttribute(fft_z_solve<T, N, N, false>, A, (int)Gm::smem_c);
}

template <typename T, int N>
static cudaError_t solve_n(const T* rho, const T* nd, T* phi, void* spec_v, const void* tw_v, const T* asin2,
                           double coef_G_h2, cudaStream_t st, int nb, size_t bs_in, size_t bs_phi,
                           size_t bs_spec) {
    typedef typename C2<T>::t C;
    typedef FftGeom<T, N> Gm;
    C* spec = reinterpret_cast<C*>(spec_v);
    const C* tw = reinterpret_cast<const C*>(tw_v);
    const int nrows = N * N;
    const int gx = (nrows + Gm::RB - 1) / Gm::RB;
    const int gk = (Gm::MH + Gm::KB - 1) / Gm::KB;
    // total scale of the unnormalised inverse: 1 / ((N/2) N N)
    const double coef = -4.0 * 3.14159265358979323846 * coef_G_h2 / (double(Gm::M) * N * N);
    fft_x_forward<T, N, N><<<dim3(gx, nb), Gm::NTX, Gm::smem_x, st>>>(rho, nd, spec, nrows, tw, bs_in, bs_spec);
    fft_y<T, N, N, false><<<dim3(gk, N, nb), Gm::NTC, Gm::smem_c, st>>>(spec, tw, bs_spec);
    fft_z_solve<T, N, N, false><<<dim3(gk, N, nb), Gm::NTC, Gm::smem_c, st>>>(spec, tw, asin2, T(coef), nullptr,
                                                                          bs_spec);
    fft_y<T, N, N, true><<<dim3(gk, N, nb), Gm::NTC, Gm::smem_c, st>>>(spec, tw, bs_spec);
    fft_x_inverse<T, N, N><<<dim3(gx, nb), Gm::NTX, Gm::smem_x, st>>>(spec, phi, nrows, tw, bs_spec, bs_phi);
    return cudaGetLastError();
}

template <typename T>
cudaError_t fft_prepare(int N) {
    switch (N) {
#define FLIC_CASE(n) case n: return prepare_n<T, n>();
        FLIC_FFT_SIZES(FLIC_CASE)
#undef FLIC_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t poisson_periodic(const T* rho, const T* nd, T* phi, void* spec, int N, const FftPlans&,
                             const void* tw, int tw_len, const T* asin2, double coef_G_h2, cudaStream_t st,
                             int nbatch, size_t bs_in, size_t bs_phi, size_t bs_spec) {
    if (tw_len != N || nbatch < 1) return cudaErrorInvalidValue;
    switch (N) {
#define FLIC_CASE(n) \
    case n: return solve_n<T, n>(rho, nd, phi, spec, tw, asin2, coef_G_h2, st, nbatch, bs_in, bs_phi, bs_spec);
        FLIC_FFT_SIZES(FLIC_CASE)
#undef FLIC_CASE
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t fft_prepare<float>(int);
template cudaError_t fft_prepare<double>(int);
template cudaError_t poisson_periodic<float>(const float*, const float*, float*, void*, int, const FftPlans&,
                                             const void*, int, const float*, double, cudaStream_t, int, size_t,
                                             size_t, size_t);
template cudaError_t poisson_periodic<double>(const double*, const double*, double*, void*, int,
                                              const FftPlans&, const void*, int, const double*, double,
                                              cudaStream_t, int, size_t, size_t, size_t);

}  // namespace flic
