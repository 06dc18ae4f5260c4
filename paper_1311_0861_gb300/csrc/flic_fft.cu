// Poisson equation of Sec. 2.3 by FFT on the periodic N^3 grid:
//   Phi_hat(k) = -4 pi G h^2 s_hat(k) / (6 (1 - prod_d (1 - 2/3 sin^2(pi k_d / N)))),
//   Phi_hat(0) = 0,  s = rho + n.
// (The printed symbol has no minus sign; Laplace(Phi) = 4 pi rho of Sec. 2 fixes it.)
//
// Five passes over HBM, each a hand-written shared-memory FFT (Stockham
// autosort; radix-4, then 2, then 3 butterflies; the radix sequence, strides
// and index arithmetic are compile-time for each supported N; twiddles are read
// from a table staged in shared memory):
//   X  real-to-complex along x: s = rho + n is summed while loading, packed as
//      N/2 complex values, transformed, and unpacked to N/2 + 1 modes;
//   Y  complex along y (forward);
//   Z  complex along z forward, multiply by the symbol (and the 1/N^3 scale),
//      inverse -- one read and one write of the spectrum;
//   Y  complex along y (inverse);
//   X  complex-to-real along x (inverse of the packing), writes Phi.
// The spectrum is [z][y][kx] with N/2 + 1 modes per row (kx fastest).  The
// symbol uses 1 - f_x f_y f_z = a_x + f_x (a_y + f_y a_z) with a_d = 2/3 sin^2,
// which has no cancellation at low k in float32.
#include <cuda_runtime.h>

#include "flic_common.cuh"
#include "flic_fft.h"

namespace flic {

template <typename T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C>
__device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }

// ---------------------------------------------------------------------------
// r-point DFTs (forward: exp(-2 pi i / r); inverse: conjugate)
// ---------------------------------------------------------------------------
template <typename C, bool INV, int R> struct Butterfly;
template <typename C, bool INV> struct Butterfly<C, INV, 2> {
    static __device__ __forceinline__ void run(C* x) {
        C a = x[0];
        x[0] = cadd(a, x[1]);
        x[1] = csub(a, x[1]);
    }
};
template <typename C, bool INV> struct Butterfly<C, INV, 4> {
    static __device__ __forceinline__ void run(C* x) {
        C a = cadd(x[0], x[2]), b = csub(x[0], x[2]);
        C c = cadd(x[1], x[3]), d0 = csub(x[1], x[3]);
        C d;   // (x1 - x3) * (-i) forward, * (+i) inverse
        if (INV) { d.x = -d0.y; d.y = d0.x; } else { d.x = d0.y; d.y = -d0.x; }
        x[0] = cadd(a, c);
        x[1] = cadd(b, d);
        x[2] = csub(a, c);
        x[3] = csub(b, d);
    }
};
template <typename C, bool INV> struct Butterfly<C, INV, 3> {
    static __device__ __forceinline__ void run(C* x) {
        typedef decltype(C().x) R;
        const R h = R(0.86602540378443864676372317075294);   // sqrt(3)/2
        C sum = cadd(x[1], x[2]);
        C dif = csub(x[1], x[2]);
        C t1;
        t1.x = x[0].x - R(0.5) * sum.x;
        t1.y = x[0].y - R(0.5) * sum.y;
        C t2;   // -i h dif forward, +i h dif inverse
        if (INV) { t2.x = -h * dif.y; t2.y = h * dif.x; } else { t2.x = h * dif.y; t2.y = -h * dif.x; }
        x[0] = cadd(x[0], sum);
        x[1] = cadd(t1, t2);
        x[2] = csub(t1, t2);
    }
};

template <int L> struct FirstRadix {
    static constexpr int value = (L % 4 == 0) ? 4 : (L % 2 == 0) ? 2 : (L % 3 == 0) ? 3 : 1;
};

// One Stockham pass of radix R at span NS over NL lines of length L held in
// shared memory; element (line l, index j) at buf[j * SJ + l * SL].  Twiddle
// exp(-2 pi i m / TWL) is tw[m] (TWL a multiple of L).
template <typename C, bool INV, int L, int NL, int SJ, int SL, bool LFAST, int NS, int R, int TWL>
__device__ __forceinline__ void stockham_pass(const C* __restrict__ A, C* __restrict__ B, const C* tw) {
    constexpr int NB = L / R;
    constexpr int TOTAL = NB * NL;
    constexpr int TSC = (TWL / L) * (L / (NS * R));
    for (int t = threadIdx.x; t < TOTAL; t += blockDim.x) {
        const int l = LFAST ? t % NL : t / NB;
        const int j = LFAST ? t / NL : t % NB;
        const int k = j % NS;
        C x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = A[(j + q * NB) * SJ + l * SL];
        if (NS > 1) {
#pragma unroll
            for (int q = 1; q < R; ++q) {
                C w = tw[q * k * TSC];
                if (INV) w.y = -w.y;
                x[q] = cmul(x[q], w);
            }
        }
        Butterfly<C, INV, R>::run(x);
        const int idx = (j / NS) * NS * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) B[(idx + q * NS) * SJ + l * SL] = x[q];
    }
}

template <typename C, bool INV, int L, int NL, int SJ, int SL, bool LFAST, int NS, int REM, int TWL>
struct Stockham {
    static __device__ __forceinline__ C* run(C* A, C* B, const C* tw) {
        constexpr int R = FirstRadix<REM>::value;
        static_assert(R > 1, "transform length must be 2^a 3^b");
        stockham_pass<C, INV, L, NL, SJ, SL, LFAST, NS, R, TWL>(A, B, tw);
        __syncthreads();
        return Stockham<C, INV, L, NL, SJ, SL, LFAST, NS * R, REM / R, TWL>::run(B, A, tw);
    }
};
template <typename C, bool INV, int L, int NL, int SJ, int SL, bool LFAST, int NS, int TWL>
struct Stockham<C, INV, L, NL, SJ, SL, LFAST, NS, 1, TWL> {
    static __device__ __forceinline__ C* run(C* A, C*, const C*) { return A; }
};

// Sizes of the blocks: rows per block of the x passes (~16 KB of complex data
// per buffer), columns per block of the y/z passes (two N x KB buffers in 96 KB).
template <typename T, int N> struct FftGeom {
    typedef typename C2<T>::t C;
    static constexpr int M = N / 2, MH = M + 1;
    static constexpr int RB0 = int(16384 / (sizeof(C) * M));
    static constexpr int RB = RB0 < 1 ? 1 : (RB0 > 64 ? 64 : RB0);
    static constexpr int KLIM = int(98304 / (2 * sizeof(C) * N));
    static constexpr int KB = KLIM >= 16 ? 16 : KLIM >= 8 ? 8 : KLIM >= 4 ? 4 : KLIM >= 2 ? 2 : 1;
    static constexpr size_t smem_x = (size_t(2) * RB * M + N) * sizeof(C);
    static constexpr size_t smem_c = (size_t(2) * N * KB + N) * sizeof(C);
};

template <typename C, int N>
__device__ __forceinline__ void stage_twiddles(C* tws, const C* __restrict__ tw) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) tws[i] = tw[i];
}

// ---------------------------------------------------------------------------
// X pass, forward: rows of s = rho + n -> N/2 + 1 modes per row
// ---------------------------------------------------------------------------
template <typename T, int N>
__global__ void __launch_bounds__(256) fft_x_forward(const T* __restrict__ rho, const T* __restrict__ nd,
                                                     typename C2<T>::t* __restrict__ spec, int nrows,
                                                     const typename C2<T>::t* __restrict__ tw) {
    typedef typename C2<T>::t C;
    typedef FftGeom<T, N> Gm;
    constexpr int M = Gm::M, MH = Gm::MH, RB = Gm::RB;
    extern __shared__ __align__(16) unsigned char sm[];
    C* A = reinterpret_cast<C*>(sm);
    C* B = A + RB * M;
    C* tws = B + RB * M;
    stage_twiddles<C, N>(tws, tw);
    const int row0 = blockIdx.x * RB;
    for (int t = threadIdx.x; t < RB * M; t += blockDim.x) {
        const int l = t / M, j = t % M;
        const int row = row0 + l;
        C z;
        if (row < nrows) {
            const size_t g = size_t(row) * N + 2 * j;
            z.x = rho[g] + nd[g];
            z.y = rho[g + 1] + nd[g + 1];
        } else {
            z.x = T(0); z.y = T(0);
        }
        A[l * M + j] = z;
    }
    __syncthreads();
    C* Z = Stockham<C, false, M, RB, 1, M, false, 1, M, N>::run(A, B, tws);
    for (int t = threadIdx.x; t < RB * MH; t += blockDim.x) {
        const int l = t / MH, k = t % MH;
        const int row = row0 + l;
        if (row >= nrows) continue;
        C zk = Z[l * M + (k == M ? 0 : k)];
        C zm = cconj(Z[l * M + (k == 0 ? 0 : M - k)]);
        C Ek, Ok;
        Ek.x = T(0.5) * (zk.x + zm.x);
        Ek.y = T(0.5) * (zk.y + zm.y);
        Ok.x = T(0.5) * (zk.y - zm.y);     // (zk - zm) / (2 i)
        Ok.y = -T(0.5) * (zk.x - zm.x);
        spec[size_t(row) * MH + k] = cadd(Ek, cmul(tws[k], Ok));
    }
}

// ---------------------------------------------------------------------------
// X pass, inverse: N/2 + 1 modes per row -> N reals (Phi)
// ---------------------------------------------------------------------------
template <typename T, int N>
__global__ void __launch_bounds__(256) fft_x_inverse(const typename C2<T>::t* __restrict__ spec,
                                                     T* __restrict__ phi, int nrows,
                                                     const typename C2<T>::t* __restrict__ tw) {
    typedef typename C2<T>::t C;
    typedef FftGeom<T, N> Gm;
    constexpr int M = Gm::M, MH = Gm::MH, RB = Gm::RB;
    extern __shared__ __align__(16) unsigned char sm[];
    C* A = reinterpret_cast<C*>(sm);
    C* B = A + RB * M;
    C* tws = B + RB * M;
    stage_twiddles<C, N>(tws, tw);
    __syncthreads();
    const int row0 = blockIdx.x * RB;
    for (int t = threadIdx.x; t < RB * M; t += blockDim.x) {
        const int l = t / M, k = t % M;
        const int row = row0 + l;
        C z;
        if (row < nrows) {
            C xk = spec[size_t(row) * MH + k];
            C xm = cconj(spec[size_t(row) * MH + (M - k)]);
            C Ek, D;
            Ek.x = T(0.5) * (xk.x + xm.x);
            Ek.y = T(0.5) * (xk.y + xm.y);
            D.x = T(0.5) * (xk.x - xm.x);
            D.y = T(0.5) * (xk.y - xm.y);
            C Ok = cmul(D, cconj(tws[k]));
            z.x = Ek.x - Ok.y;   // E + i O
            z.y = Ek.y + Ok.x;
        } else {
            z.x = T(0); z.y = T(0);
        }
        A[l * M + k] = z;
    }
    __syncthreads();
    C* Z = Stockham<C, true, M, RB, 1, M, false, 1, M, N>::run(A, B, tws);
    for (int t = threadIdx.x; t < RB * M; t += blockDim.x) {
        const int l = t / M, j = t % M;
        const int row = row0 + l;
        if (row >= nrows) continue;
        C z = Z[l * M + j];
        const size_t g = size_t(row) * N + 2 * j;
        phi[g] = z.x;
        phi[g + 1] = z.y;
    }
}

// ---------------------------------------------------------------------------
// Y pass: columns of the spectrum along y for a fixed z
// ---------------------------------------------------------------------------
template <typename T, int N, bool INV>
__global__ void __launch_bounds__(256) fft_y(typename C2<T>::t* __restrict__ spec,
                                             const typename C2<T>::t* __restrict__ tw) {
    typedef typename C2<T>::t C;
    typedef FftGeom<T, N> Gm;
    constexpr int MH = Gm::MH, KB = Gm::KB;
    extern __shared__ __align__(16) unsigned char sm[];
    C* A = reinterpret_cast<C*>(sm);
    C* B = A + N * KB;
    C* tws = B + N * KB;
    stage_twiddles<C, N>(tws, tw);
    const int k0 = blockIdx.x * KB;
    const size_t base = size_t(blockIdx.y) * N * MH;
    for (int t = threadIdx.x; t < N * KB; t += blockDim.x) {
        const int c = t % KB, y = t / KB;
        C v;
        if (k0 + c < MH) v = spec[base + size_t(y) * MH + k0 + c];
        else { v.x = T(0); v.y = T(0); }
        A[y * KB + c] = v;
    }
    __syncthreads();
    C* R = Stockham<C, INV, N, KB, KB, 1, true, 1, N, N>::run(A, B, tws);
    for (int t = threadIdx.x; t < N * KB; t += blockDim.x) {
        const int c = t % KB, y = t / KB;
        if (k0 + c < MH) spec[base + size_t(y) * MH + k0 + c] = R[y * KB + c];
    }
}

// ---------------------------------------------------------------------------
// Z pass with the symbol: forward along z, multiply, inverse along z
// ---------------------------------------------------------------------------
template <typename T, int N>
__global__ void __launch_bounds__(256) fft_z_solve(typename C2<T>::t* __restrict__ spec,
                                                   const typename C2<T>::t* __restrict__ tw,
                                                   const T* __restrict__ asin2, T coef) {
    typedef typename C2<T>::t C;
    typedef FftGeom<T, N> Gm;
    constexpr int MH = Gm::MH, KB = Gm::KB;
    extern __shared__ __align__(16) unsigned char sm[];
    C* A = reinterpret_cast<C*>(sm);
    C* B = A + N * KB;
    C* tws = B + N * KB;
    stage_twiddles<C, N>(tws, tw);
    const int k0 = blockIdx.x * KB;
    const int y = blockIdx.y;
    constexpr size_t zs = size_t(N) * MH;
    const size_t base = size_t(y) * MH;
    for (int t = threadIdx.x; t < N * KB; t += blockDim.x) {
        const int c = t % KB, z = t / KB;
        C v;
        if (k0 + c < MH) v = spec[base + size_t(z) * zs + k0 + c];
        else { v.x = T(0); v.y = T(0); }
        A[z * KB + c] = v;
    }
    __syncthreads();
    C* R = Stockham<C, false, N, KB, KB, 1, true, 1, N, N>::run(A, B, tws);
    C* S = (R == A) ? B : A;
    const T ay = asin2[y];
    for (int t = threadIdx.x; t < N * KB; t += blockDim.x) {
        const int c = t % KB, z = t / KB;
        const int kx = k0 + c;
        C v = R[z * KB + c];
        if (kx < MH) {
            const T ax = asin2[kx], az = asin2[z];
            // 1 - f_x f_y f_z without cancellation, f = 1 - a
            const T D = T(6) * (ax + (T(1) - ax) * (ay + (T(1) - ay) * az));
            const T g = (kx == 0 && y == 0 && z == 0) ? T(0) : coef / D;
            v.x *= g;
            v.y *= g;
        }
        S[z * KB + c] = v;
    }
    __syncthreads();
    C* Q = Stockham<C, true, N, KB, KB, 1, true, 1, N, N>::run(S, R, tws);
    for (int t = threadIdx.x; t < N * KB; t += blockDim.x) {
        const int c = t % KB, z = t / KB;
        if (k0 + c < MH) spec[base + size_t(z) * zs + k0 + c] = Q[z * KB + c];
    }
}

// ---------------------------------------------------------------------------
// host side: one instantiation set per supported N
// ---------------------------------------------------------------------------
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
    if ((e = cudaFuncSetAttribute(fft_x_forward<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::smem_x))) return e;
    if ((e = cudaFuncSetAttribute(fft_x_inverse<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::smem_x))) return e;
    if ((e = cudaFuncSetAttribute(fft_y<T, N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::smem_c))) return e;
    if ((e = cudaFuncSetAttribute(fft_y<T, N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::smem_c))) return e;
    return cudaFuncSetAttribute(fft_z_solve<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::smem_c);
}

template <typename T, int N>
static cudaError_t solve_n(const T* rho, const T* nd, T* phi, void* spec_v, const void* tw_v, const T* asin2,
                           double coef_G_h2, cudaStream_t st) {
    typedef typename C2<T>::t C;
    typedef FftGeom<T, N> Gm;
    C* spec = reinterpret_cast<C*>(spec_v);
    const C* tw = reinterpret_cast<const C*>(tw_v);
    const int nrows = N * N;
    const int gx = (nrows + Gm::RB - 1) / Gm::RB;
    const int gk = (Gm::MH + Gm::KB - 1) / Gm::KB;
    // total scale of the unnormalised inverse: 1 / (M N N)
    const double coef = -4.0 * 3.14159265358979323846 * coef_G_h2 / (double(Gm::M) * N * N);
    fft_x_forward<T, N><<<gx, 256, Gm::smem_x, st>>>(rho, nd, spec, nrows, tw);
    fft_y<T, N, false><<<dim3(gk, N), 256, Gm::smem_c, st>>>(spec, tw);
    fft_z_solve<T, N><<<dim3(gk, N), 256, Gm::smem_c, st>>>(spec, tw, asin2, T(coef));
    fft_y<T, N, true><<<dim3(gk, N), 256, Gm::smem_c, st>>>(spec, tw);
    fft_x_inverse<T, N><<<gx, 256, Gm::smem_x, st>>>(spec, phi, nrows, tw);
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
                             const void* tw, int tw_len, const T* asin2, double coef_G_h2, cudaStream_t st) {
    if (tw_len != N) return cudaErrorInvalidValue;
    switch (N) {
#define FLIC_CASE(n) case n: return solve_n<T, n>(rho, nd, phi, spec, tw, asin2, coef_G_h2, st);
        FLIC_FFT_SIZES(FLIC_CASE)
#undef FLIC_CASE
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t fft_prepare<float>(int);
template cudaError_t fft_prepare<double>(int);
template cudaError_t poisson_periodic<float>(const float*, const float*, float*, void*, int, const FftPlans&,
                                             const void*, int, const float*, double, cudaStream_t);
template cudaError_t poisson_periodic<double>(const double*, const double*, double*, void*, int,
                                              const FftPlans&, const void*, int, const double*, double,
                                              cudaStream_t);

}  // namespace flic
