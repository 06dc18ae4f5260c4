// Poisson equation of Sec. 2.3 by FFT on the periodic N^3 grid:
//   Phi_hat(k) = -4 pi G h^2 s_hat(k) / (6 (1 - prod_d (1 - 2/3 sin^2(pi k_d / N)))),
//   Phi_hat(0) = 0,  s = rho + n.
// (The printed symbol has no minus sign; Laplace(Phi) = 4 pi rho of Sec. 2 fixes it.)
//
// Five passes over HBM, each a hand-written shared-memory FFT (Stockham
// autosort, radix 4/2/3 butterflies, twiddles from a table):
//   X  real-to-complex along x: s = rho + n is summed while loading, packed as
//      N/2 complex values, transformed, and unpacked to N/2 + 1 modes;
//   Y  complex along y (forward);
//   Z  complex along z forward, multiply by the symbol (and 1/N^3), inverse;
//   Y  complex along y (inverse);
//   X  complex-to-real along x (inverse of the packing), writes Phi.
// The spectrum is [z][y][kx] with N/2 + 1 modes per row (kx fastest).  The
// symbol uses 1 - f_x f_y f_z = a_x + f_x (a_y + f_y a_z) with a_d = 2/3 sin^2,
// which has no cancellation at low k in float32.
#include <cuda_runtime.h>

#include "flic_fft.h"
#include "flic_common.cuh"

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

// Twiddle exp(-+2 pi i m / L) from the table of length Ltab (entries
// exp(-2 pi i j / Ltab)); tstride = Ltab / L.
template <typename C, bool INV>
__device__ __forceinline__ C twiddle(const C* __restrict__ tw, int m, int tstride) {
    C w = tw[m * tstride];
    if (INV) w.y = -w.y;
    return w;
}

// In-block FFT of `nl` lines of length L held in shared memory; element (line l,
// index j) at buf[j * sj + l * sl].  Stockham passes alternate between A and B;
// the return value is the buffer that holds the result.  LFAST selects the
// thread-to-element map (line index fastest for sl == 1 layouts).
template <typename C, bool INV, bool LFAST>
__device__ C* block_fft(C* A, C* B, int L, int nl, int sj, int sl, const FftPlan& pl,
                        const C* __restrict__ tw, int tstride) {
    typedef decltype(C().x) R;
    const int tid = threadIdx.x, nt = blockDim.x;
    int ns = 1;
    for (int s = 0; s < pl.nrad; ++s) {
        const int r = pl.radix[s];
        const int nb = L / r;
        const int total = nb * nl;
        const int tsc = L / (ns * r);
        for (int t = tid; t < total; t += nt) {
            int l, j;
            if (LFAST) { l = t % nl; j = t / nl; } else { j = t % nb; l = t / nb; }
            const int k = j % ns;
            C x[4];
            for (int q = 0; q < r; ++q) x[q] = A[(j + q * nb) * sj + l * sl];
            for (int q = 1; q < r; ++q) x[q] = cmul(x[q], twiddle<C, INV>(tw, q * k * tsc, tstride));
            C y[4];
            if (r == 4) {
                C a = cadd(x[0], x[2]), b = csub(x[0], x[2]);
                C c = cadd(x[1], x[3]), d0 = csub(x[1], x[3]);
                C d;   // (x1 - x3) * (-i) forward, * (+i) inverse
                if (INV) { d.x = -d0.y; d.y = d0.x; } else { d.x = d0.y; d.y = -d0.x; }
                y[0] = cadd(a, c);
                y[1] = cadd(b, d);
                y[2] = csub(a, c);
                y[3] = csub(b, d);
            } else if (r == 2) {
                y[0] = cadd(x[0], x[1]);
                y[1] = csub(x[0], x[1]);
            } else {   // r == 3
                const R h = R(0.86602540378443864676372317075294);   // sqrt(3)/2
                C sum = cadd(x[1], x[2]);
                C dif = csub(x[1], x[2]);
                C t1;
                t1.x = x[0].x - R(0.5) * sum.x;
                t1.y = x[0].y - R(0.5) * sum.y;
                C t2;   // -i h dif forward, +i h dif inverse
                if (INV) { t2.x = -h * dif.y; t2.y = h * dif.x; } else { t2.x = h * dif.y; t2.y = -h * dif.x; }
                y[0] = cadd(x[0], sum);
                y[1] = cadd(t1, t2);
                y[2] = csub(t1, t2);
            }
            const int idx = (j / ns) * ns * r + k;
            for (int q = 0; q < r; ++q) B[(idx + q * ns) * sj + l * sl] = y[q];
        }
        __syncthreads();
        C* t = A; A = B; B = t;
        ns *= r;
    }
    return A;
}

// ---------------------------------------------------------------------------
// X pass, forward: rows of s = rho + n -> N/2 + 1 modes per row
// ---------------------------------------------------------------------------
template <typename T>
__global__ void fft_x_forward(const T* __restrict__ rho, const T* __restrict__ nd,
                              typename C2<T>::t* __restrict__ spec, int N, int nrows, int rows_per_block,
                              FftPlan pl, const typename C2<T>::t* __restrict__ tw, int tw_len) {
    typedef typename C2<T>::t C;
    extern __shared__ __align__(16) unsigned char sm[];
    const int M = N / 2;
    const int RB = rows_per_block;
    C* A = reinterpret_cast<C*>(sm);
    C* B = A + RB * M;
    const int row0 = blockIdx.x * RB;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int t = tid; t < RB * M; t += nt) {
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
    C* Z = block_fft<C, false, false>(A, B, M, RB, 1, M, pl, tw, (tw_len / M));
    const int MH = M + 1;
    for (int t = tid; t < RB * MH; t += nt) {
        const int l = t / MH, k = t % MH;
        const int row = row0 + l;
        if (row >= nrows) continue;
        C zk = Z[l * M + (k == M ? 0 : k)];
        C zm = cconj(Z[l * M + (k == 0 ? 0 : M - k)]);
        C Ek, Ok;
        Ek.x = T(0.5) * (zk.x + zm.x);
        Ek.y = T(0.5) * (zk.y + zm.y);
        // O = (zk - zm) / (2 i)
        Ok.x = T(0.5) * (zk.y - zm.y);
        Ok.y = -T(0.5) * (zk.x - zm.x);
        C w = tw[k * (tw_len / N)];
        spec[size_t(row) * MH + k] = cadd(Ek, cmul(w, Ok));
    }
}

// ---------------------------------------------------------------------------
// X pass, inverse: N/2 + 1 modes per row -> N reals (Phi)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void fft_x_inverse(const typename C2<T>::t* __restrict__ spec, T* __restrict__ phi, int N,
                              int nrows, int rows_per_block, FftPlan pl,
                              const typename C2<T>::t* __restrict__ tw, int tw_len) {
    typedef typename C2<T>::t C;
    extern __shared__ __align__(16) unsigned char sm[];
    const int M = N / 2, MH = M + 1;
    const int RB = rows_per_block;
    C* A = reinterpret_cast<C*>(sm);
    C* B = A + RB * M;
    const int row0 = blockIdx.x * RB;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int t = tid; t < RB * M; t += nt) {
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
            C Ok = cmul(D, cconj(tw[k * (tw_len / N)]));
            z.x = Ek.x - Ok.y;   // E + i O
            z.y = Ek.y + Ok.x;
        } else {
            z.x = T(0); z.y = T(0);
        }
        A[l * M + k] = z;
    }
    __syncthreads();
    C* Z = block_fft<C, true, false>(A, B, M, RB, 1, M, pl, tw, (tw_len / M));
    for (int t = tid; t < RB * M; t += nt) {
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
template <typename T, bool INV>
__global__ void fft_y(typename C2<T>::t* __restrict__ spec, int N, int KB, FftPlan pl,
                      const typename C2<T>::t* __restrict__ tw, int tw_len) {
    typedef typename C2<T>::t C;
    extern __shared__ __align__(16) unsigned char sm[];
    const int MH = N / 2 + 1;
    C* A = reinterpret_cast<C*>(sm);
    C* B = A + N * KB;
    const int k0 = blockIdx.x * KB;
    const int z = blockIdx.y;
    const int tid = threadIdx.x, nt = blockDim.x;
    const size_t base = size_t(z) * N * MH;
    for (int t = tid; t < N * KB; t += nt) {
        const int c = t % KB, y = t / KB;
        C v;
        if (k0 + c < MH) v = spec[base + size_t(y) * MH + k0 + c];
        else { v.x = T(0); v.y = T(0); }
        A[y * KB + c] = v;
    }
    __syncthreads();
    C* R = block_fft<C, INV, true>(A, B, N, KB, KB, 1, pl, tw, tw_len / N);
    for (int t = tid; t < N * KB; t += nt) {
        const int c = t % KB, y = t / KB;
        if (k0 + c < MH) spec[base + size_t(y) * MH + k0 + c] = R[y * KB + c];
    }
}

// ---------------------------------------------------------------------------
// Z pass with the symbol: forward along z, multiply, inverse along z
// ---------------------------------------------------------------------------
template <typename T>
__global__ void fft_z_solve(typename C2<T>::t* __restrict__ spec, int N, int KB, FftPlan pl,
                            const typename C2<T>::t* __restrict__ tw, int tw_len,
                            const T* __restrict__ asin2, T coef) {
    typedef typename C2<T>::t C;
    extern __shared__ __align__(16) unsigned char sm[];
    const int MH = N / 2 + 1;
    C* A = reinterpret_cast<C*>(sm);
    C* B = A + N * KB;
    const int k0 = blockIdx.x * KB;
    const int y = blockIdx.y;
    const int tid = threadIdx.x, nt = blockDim.x;
    const size_t zs = size_t(N) * MH;
    const size_t base = size_t(y) * MH;
    for (int t = tid; t < N * KB; t += nt) {
        const int c = t % KB, z = t / KB;
        C v;
        if (k0 + c < MH) v = spec[base + size_t(z) * zs + k0 + c];
        else { v.x = T(0); v.y = T(0); }
        A[z * KB + c] = v;
    }
    __syncthreads();
    C* R = block_fft<C, false, true>(A, B, N, KB, KB, 1, pl, tw, tw_len / N);
    C* S = (R == A) ? B : A;
    const T ay = asin2[y];
    for (int t = tid; t < N * KB; t += nt) {
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
    C* Q = block_fft<C, true, true>(S, R, N, KB, KB, 1, pl, tw, tw_len / N);
    for (int t = tid; t < N * KB; t += nt) {
        const int c = t % KB, z = t / KB;
        if (k0 + c < MH) spec[base + size_t(z) * zs + k0 + c] = Q[z * KB + c];
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int make_plan(int L, FftPlan* pl) {
    pl->nrad = 0;
    int m = L;
    while (m % 4 == 0) { pl->radix[pl->nrad++] = 4; m /= 4; }
    while (m % 2 == 0) { pl->radix[pl->nrad++] = 2; m /= 2; }
    while (m % 3 == 0) { pl->radix[pl->nrad++] = 3; m /= 3; }
    if (m != 1 || pl->nrad > FFT_MAX_RADIX) return -1;
    return 0;
}

int fft_plan_init(int N, FftPlans* p) {
    if (N < 4 || N % 2) return -1;
    if (make_plan(N, &p->full) || make_plan(N / 2, &p->half)) return -1;
    return 0;
}

// Rows per block of the x passes (~16 KB of complex data per buffer) and
// columns per block of the y/z passes (two N x KB buffers within 96 KB).
static void pick(int N, size_t elem, int* rows_per_block, int* kb) {
    const int M = N / 2;
    int rb = (int)(16384 / (elem * M));
    *rows_per_block = rb < 1 ? 1 : (rb > 64 ? 64 : rb);
    int lim = (int)(98304 / (2 * size_t(N) * elem));
    int k = 1;
    while (k * 2 <= lim && k * 2 <= 16) k *= 2;
    *kb = k;
}

template <typename T>
cudaError_t fft_prepare(int N) {
    typedef typename C2<T>::t C;
    int rb, kb;
    pick(N, sizeof(C), &rb, &kb);
    const int smx = (int)(size_t(2) * rb * (N / 2) * sizeof(C));
    const int smc = (int)(size_t(2) * N * kb * sizeof(C));
    cudaError_t e = cudaSuccess;
    if ((e = cudaFuncSetAttribute(fft_x_forward<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smx))) return e;
    if ((e = cudaFuncSetAttribute(fft_x_inverse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smx))) return e;
    if ((e = cudaFuncSetAttribute(fft_y<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smc))) return e;
    if ((e = cudaFuncSetAttribute(fft_y<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smc))) return e;
    return cudaFuncSetAttribute(fft_z_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smc);
}
template cudaError_t fft_prepare<float>(int);
template cudaError_t fft_prepare<double>(int);

template <typename T>
cudaError_t poisson_periodic(const T* rho, const T* nd, T* phi, void* spec_v, int N, const FftPlans& pl,
                             const void* tw_v, int tw_len, const T* asin2, double coef_G_h2,
                             cudaStream_t st) {
    typedef typename C2<T>::t C;
    C* spec = reinterpret_cast<C*>(spec_v);
    const C* tw = reinterpret_cast<const C*>(tw_v);
    int rb, kb;
    pick(N, sizeof(C), &rb, &kb);
    const int M = N / 2, MH = M + 1;
    const int nrows = N * N;
    const int threads = 256;
    const size_t smx = size_t(2) * rb * M * sizeof(C);
    const size_t smc = size_t(2) * N * kb * sizeof(C);
    const int gx = (nrows + rb - 1) / rb;
    const int gk = (MH + kb - 1) / kb;
    // total scale of the unnormalised inverse: 1 / (M N N)
    const double coef = -4.0 * 3.14159265358979323846 * coef_G_h2 / (double(M) * N * N);
    fft_x_forward<T><<<gx, threads, smx, st>>>(rho, nd, spec, N, nrows, rb, pl.half, tw, tw_len);
    fft_y<T, false><<<dim3(gk, N), threads, smc, st>>>(spec, N, kb, pl.full, tw, tw_len);
    fft_z_solve<T><<<dim3(gk, N), threads, smc, st>>>(spec, N, kb, pl.full, tw, tw_len, asin2, T(coef));
    fft_y<T, true><<<dim3(gk, N), threads, smc, st>>>(spec, N, kb, pl.full, tw, tw_len);
    fft_x_inverse<T><<<gx, threads, smx, st>>>(spec, phi, N, nrows, rb, pl.half, tw, tw_len);
    return cudaGetLastError();
}

template cudaError_t poisson_periodic<float>(const float*, const float*, float*, void*, int, const FftPlans&,
                                             const void*, int, const float*, double, cudaStream_t);
template cudaError_t poisson_periodic<double>(const double*, const double*, double*, void*, int,
                                              const FftPlans&, const void*, int, const double*, double,
                                              cudaStream_t);

}  // namespace flic
