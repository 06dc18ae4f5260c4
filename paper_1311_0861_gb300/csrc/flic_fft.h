// FFT Poisson solver interface (internal to libflic).
#pragma once

#include <cuda_runtime.h>

namespace flic {

constexpr int FFT_MAX_RADIX = 16;

// Radix sequence of one transform length (4s, then a 2, then 3s).
struct FftPlan {
    int nrad;
    int radix[FFT_MAX_RADIX];
};

struct FftPlans {
    FftPlan full;   // length N (y, z passes)
    FftPlan half;   // length N/2 (packed real x pass)
};

int fft_plan_init(int N, FftPlans* p);

// Sets the dynamic shared-memory limits of the FFT kernels for size N (call
// once per size before launching or capturing).
template <typename T>
cudaError_t fft_prepare(int N);

// Periodic solve of Sec. 2.3: phi = potential of s = rho + n.
//   spec: (N/2+1) N N complex workspace; tw: table exp(-2 pi i j / tw_len),
//   j < tw_len (tw_len a multiple of N); asin2[k] = 2/3 sin^2(pi k / N), k < N;
//   coef_G_h2 = G h^2.
//   nbatch independent runs of the same N in one set of launches: run r reads
//   rho + r*bs_in, nd + r*bs_in, writes phi + r*bs_phi, uses spec + r*bs_spec
//   (complex elements).
template <typename T>
cudaError_t poisson_periodic(const T* rho, const T* nd, T* phi, void* spec, int N, const FftPlans& pl,
                             const void* tw, int tw_len, const T* asin2, double coef_G_h2,
                             cudaStream_t st, int nbatch = 1, size_t bs_in = 0, size_t bs_phi = 0,
                             size_t bs_spec = 0);

// Elements of the isolated solve's Green's function table (about (N+1)^3).
template <typename T> size_t green_table_elems(int N);

// Isolated (zero-padded, L = 2N) solve.  gtab: green_table_elems reals (the scaled
// transform of the Green's function, from green_init); spec: N * 2N * (N+1)
// complex workspace; tw: table of length 2N.  green_init needs (2N)^3 reals
// (greal) and (2N)^2 (N+1) complex (tmp_spec) of temporary workspace.
int fft_iso_supported(int N);
template <typename T>
cudaError_t fft_prepare_iso(int N);
template <typename T>
cudaError_t green_init(int N, double h, double G, T* gtab, T* greal, void* tmp_spec, const void* tw,
                       cudaStream_t st);
template <typename T>
cudaError_t poisson_isolated(const T* rho, const T* nd, T* phi, void* spec, int N, const void* tw, const T* gtab,
                             cudaStream_t st, int nbatch = 1, size_t bs_in = 0, size_t bs_phi = 0,
                             size_t bs_spec = 0);

}  // namespace flic
