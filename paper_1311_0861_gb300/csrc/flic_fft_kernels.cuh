// Shared-memory FFT kernels of the Poisson solve (Sec. 2.3), generic in the
// transform length L and the physical extent P of each axis:
//   periodic solve: P = L = N;
//   isolated solve: L = 2N, P = N -- the source is zero-padded to (2N)^3; the
//   padding is never stored (rows and planes beyond P load as zeros and are
//   never written back).
//
// Each pass is one HBM read and one write of the spectrum.  In-block transforms
// are Stockham autosort, in place in one shared buffer (each thread holds its
// butterflies' 16 elements in registers across a barrier), with radix 16 first,
// then 8, 4, 2 and 3; the radix sequence, strides and index arithmetic are
// compile-time; twiddles are staged in shared memory from a table
// exp(-2 pi i j / L), j < L.
//
// Spectrum layout: S[z][y][kx], z < P (only physical z planes are ever held),
// y < L, kx < L/2 + 1 (kx fastest).
#pragma once

#include <cuda_runtime.h>

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

// 8- and 16-point DFTs as two layers of 4-point DFTs (and a 2-point layer for
// 8): with n = 4 n1 + n2 (n = 2 n1 + n2 for 8) and k = k1 + 4 k2,
//   X[k1 + 4 k2] = sum_n2 W4^(n2 k2) [ W_R^(n2 k1) sum_n1 x[n] W4^(n1 k1) ],
// W_R = exp(-2 pi i / R) (conjugate for the inverse).
template <typename C, bool INV>
__device__ __forceinline__ C rot(C v, double c, double s) {   // v * (c - i s) forward, (c + i s) inverse
    typedef decltype(C().x) R;
    const R cr = R(c), sr = INV ? R(-s) : R(s);
    C r;
    r.x = v.x * cr + v.y * sr;
    r.y = v.y * cr - v.x * sr;
    return r;
}
template <typename C, bool INV> struct Butterfly<C, INV, 8> {
    static __device__ __forceinline__ void run(C* x) {
        constexpr double h = 0.70710678118654752440;   // cos(pi/4) = sin(pi/4)
        C z[2][4];
#pragma unroll
        for (int n2 = 0; n2 < 2; ++n2) {
            C t[4] = {x[n2], x[2 + n2], x[4 + n2], x[6 + n2]};
            Butterfly<C, INV, 4>::run(t);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) z[n2][k1] = t[k1];
        }
        // W8^(k1) for n2 = 1: k1 = 1: (h, h); 2: (0, 1); 3: (-h, h) as (cos, sin)
        z[1][1] = rot<C, INV>(z[1][1], h, h);
        z[1][2] = rot<C, INV>(z[1][2], 0.0, 1.0);
        z[1][3] = rot<C, INV>(z[1][3], -h, h);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            x[k1] = cadd(z[0][k1], z[1][k1]);
            x[k1 + 4] = csub(z[0][k1], z[1][k1]);
        }
    }
};
template <typename C, bool INV> struct Butterfly<C, INV, 16> {
    static __device__ __forceinline__ void run(C* x) {
        // cos and sin of 2 pi m / 16, m = 0..9
        constexpr double c1 = 0.92387953251128675613, s1 = 0.38268343236508977173;
        constexpr double h = 0.70710678118654752440;
        const double cs[10][2] = {{1.0, 0.0}, {c1, s1}, {h, h}, {s1, c1}, {0.0, 1.0},
                                  {-s1, c1}, {-h, h}, {-c1, s1}, {-1.0, 0.0}, {-c1, -s1}};
        C z[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            C t[4] = {x[n2], x[4 + n2], x[8 + n2], x[12 + n2]};
            Butterfly<C, INV, 4>::run(t);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) {
                const int m = n2 * k1;   // twiddle W16^(n2 k1), 0 <= m <= 9
                z[n2][k1] = (m == 0) ? t[k1] : rot<C, INV>(t[k1], cs[m][0], cs[m][1]);
            }
        }
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            C t[4] = {z[0][k1], z[1][k1], z[2][k1], z[3][k1]};
            Butterfly<C, INV, 4>::run(t);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) x[k1 + 4 * k2] = t[k2];
        }
    }
};

template <int L> struct FirstRadix {
    static constexpr int value = (L % 4 == 0) ? 4 : (L % 2 == 0) ? 2 : (L % 3 == 0) ? 3 : 1;
};
// Radix sequence of the in-place column passes: 16 first (fewest passes
// through shared memory), then 8, 4, 2, 3.
template <int L> struct RadixIP {
    static constexpr int value = (L % 16 == 0) ? 16 : (L % 8 == 0) ? 8 : FirstRadix<L>::value;
};

// One Stockham pass of radix R at span NS over NL lines of length L held in
// shared memory, element (line l, index j) at A[j * SJ + l * SL], twiddle
// exp(-2 pi i m / TWL) at tw[m] (TWL a multiple of L); in place, for a block of
// exactly NTHR threads: every thread reads the inputs of its butterflies into
// registers, the block synchronises, then the outputs overwrite the same
// buffer (one buffer instead of two, so twice the lines fit in shared memory).
// HALF bit 0: the line's second half is zero (zero-padded input), so the first
// pass (span 1) skips loading it; bit 1: only the first half of the result is
// wanted, so the last pass (span L/R) stores only its first R/2 outputs.
template <typename C, bool INV, int L, int NL, int SJ, int SL, bool LFAST, int NS, int R, int TWL, int NTHR,
          int HALF = 0>
__device__ __forceinline__ void stockham_pass_ip(C* A, const C* tw) {
    constexpr int NB = L / R;
    constexpr int TOTAL = NB * NL;
    constexpr int PER = (TOTAL + NTHR - 1) / NTHR;
    constexpr int TSC = (TWL / L) * (L / (NS * R));
    constexpr bool ZIN = (HALF & 1) && NS == 1 && R % 2 == 0;
    constexpr bool HOUT = (HALF & 2) && NS * R == L && R % 2 == 0;
    C x[PER][R];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int t = threadIdx.x + p * NTHR;
        if (TOTAL % NTHR == 0 || t < TOTAL) {
            const int l = LFAST ? t % NL : t / NB;
            const int j = LFAST ? t / NL : t % NB;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                if (ZIN && q >= R / 2) {   // index j + q L/R >= L/2
                    x[p][q].x = 0;
                    x[p][q].y = 0;
                } else {
                    x[p][q] = A[(j + q * NB) * SJ + l * SL];
                }
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int t = threadIdx.x + p * NTHR;
        if (TOTAL % NTHR == 0 || t < TOTAL) {
            const int l = LFAST ? t % NL : t / NB;
            const int j = LFAST ? t / NL : t % NB;
            const int k = j % NS;
            if (NS > 1) {
#pragma unroll
                for (int q = 1; q < R; ++q) {
                    C w = tw[q * k * TSC];
                    if (INV) w.y = -w.y;
                    x[p][q] = cmul(x[p][q], w);
                }
            }
            Butterfly<C, INV, R>::run(x[p]);
            const int idx = (j / NS) * NS * R + k;
#pragma unroll
            for (int q = 0; q < (HOUT ? R / 2 : R); ++q) A[(idx + q * NS) * SJ + l * SL] = x[p][q];
        }
    }
    __syncthreads();
}

template <typename C, bool INV, int L, int NL, int SJ, int SL, bool LFAST, int NS, int REM, int TWL, int NTHR,
          int HALF = 0>
struct StockhamIP {
    static __device__ __forceinline__ void run(C* A, const C* tw) {
        constexpr int R = RadixIP<REM>::value;
        static_assert(R > 1, "transform length must be 2^a 3^b");
        stockham_pass_ip<C, INV, L, NL, SJ, SL, LFAST, NS, R, TWL, NTHR, HALF>(A, tw);
        StockhamIP<C, INV, L, NL, SJ, SL, LFAST, NS * R, REM / R, TWL, NTHR, HALF>::run(A, tw);
    }
};
template <typename C, bool INV, int L, int NL, int SJ, int SL, bool LFAST, int NS, int TWL, int NTHR, int HALF>
struct StockhamIP<C, INV, L, NL, SJ, SL, LFAST, NS, 1, TWL, NTHR, HALF> {
    static __device__ __forceinline__ void run(C*, const C*) {}
};

// Block sizes: rows per block of the x passes (at least 8, at least 1024
// elements; one in-place buffer, NTX threads of 16 elements each); columns per block of the y/z passes: KB
// columns (up to 16, i.e. 128-byte row segments in float32) of length L in one
// in-place buffer of at most 64 KB (three blocks per SM), NTC threads (16
// elements each).
template <typename T, int L> struct FftGeom {
    typedef typename C2<T>::t C;
    static constexpr int M = L / 2, MH = M + 1;
    static constexpr int RB0 = 1024 / M;   // 8 rows from M = 128 up (measured best at M = 128 and 512)
    static constexpr int RB = RB0 < 8 ? 8 : (RB0 > 64 ? 64 : RB0);
    static constexpr int NTX0 = (RB * M / 16 + 31) / 32 * 32;
    static constexpr int NTX = NTX0 < 32 ? 32 : (NTX0 > 1024 ? 1024 : NTX0);
    static constexpr int KLIM = int(65536 / (sizeof(C) * L));
    static constexpr int KB = KLIM >= 16 ? 16 : KLIM >= 8 ? 8 : KLIM >= 4 ? 4 : KLIM >= 2 ? 2 : 1;
    static constexpr int NTC0 = (L * KB / 16 + 31) / 32 * 32;
    static constexpr int NTC = NTC0 < 64 ? 64 : (NTC0 > 1024 ? 1024 : NTC0);
    static constexpr size_t smem_x = (size_t(RB) * M + L) * sizeof(C);
    static constexpr size_t smem_c = (size_t(L) * KB + L) * sizeof(C);
};

template <typename C, int L>
__device__ __forceinline__ void stage_twiddles(C* tws, const C* __restrict__ tw) {
    for (int i = threadIdx.x; i < L; i += blockDim.x) tws[i] = tw[i];
}

// ---------------------------------------------------------------------------
// X pass, forward: physical rows (y, z < P) of s = a + b (b may be null),
// zero-padded to L, packed as L/2 complex values, transformed, unpacked to
// L/2 + 1 modes.
// ---------------------------------------------------------------------------
template <typename T, int L, int P>
__global__ void __launch_bounds__(FftGeom<T, L>::NTX) fft_x_forward(const T* __restrict__ a, const T* __restrict__ b,
                                                                    typename C2<T>::t* __restrict__ spec, int nrows,
                                                                    const typename C2<T>::t* __restrict__ tw,
                                                                    size_t bs_in, size_t bs_spec) {
    typedef typename C2<T>::t C;
    typedef FftGeom<T, L> Gm;
    constexpr int M = Gm::M, MH = Gm::MH, RB = Gm::RB, NTX = Gm::NTX;
    static_assert(P % 2 == 0 && P <= L, "physical extent");
    // batch of independent runs along grid y
    a += blockIdx.y * bs_in;
    if (b) b += blockIdx.y * bs_in;
    spec += blockIdx.y * bs_spec;
    extern __shared__ __align__(16) unsigned char sm[];
    C* A = reinterpret_cast<C*>(sm);
    C* tws = A + RB * M;
    stage_twiddles<C, L>(tws, tw);
    const int row0 = blockIdx.x * RB;
    // pairs of reals load as one complex (row starts and P are even)
#pragma unroll 4
    for (int t = threadIdx.x; t < RB * M; t += NTX) {
        const int l = t / M, j = t % M;
        const int row = row0 + l;
        C z;
        z.x = T(0);
        z.y = T(0);
        if (row < nrows && 2 * j < P) {
            const size_t g = size_t(row) * P + 2 * j;
            z = *reinterpret_cast<const C*>(a + g);
            if (b) {
                const C w = *reinterpret_cast<const C*>(b + g);
                z.x += w.x;
                z.y += w.y;
            }
        }
        A[l * M + j] = z;
    }
    __syncthreads();
    StockhamIP<C, false, M, RB, 1, M, false, 1, M, L, NTX, (2 * P <= L) ? 1 : 0>::run(A, tws);
    // unpack row by row (modes k = threadIdx.x, + NTX, ... of each row: no
    // division by the odd mode count per element)
#pragma unroll
    for (int l = 0; l < RB; ++l) {
        const int row = row0 + l;
        if (row >= nrows) break;
        const C* Z = A + l * M;
        C* dst = spec + (size_t(row / P) * L + row % P) * MH;
        for (int k = threadIdx.x; k < MH; k += NTX) {
            C zk = Z[k == M ? 0 : k];
            C zm = cconj(Z[k == 0 ? 0 : M - k]);
            C Ek, Ok;
            Ek.x = T(0.5) * (zk.x + zm.x);
            Ek.y = T(0.5) * (zk.y + zm.y);
            Ok.x = T(0.5) * (zk.y - zm.y);     // (zk - zm) / (2 i)
            Ok.y = -T(0.5) * (zk.x - zm.x);
            dst[k] = cadd(Ek, cmul(tws[k], Ok));
        }
    }
}

// ---------------------------------------------------------------------------
// X pass, inverse: L/2 + 1 modes per physical row -> the first P reals
// ---------------------------------------------------------------------------
template <typename T, int L, int P>
__global__ void __launch_bounds__(FftGeom<T, L>::NTX) fft_x_inverse(const typename C2<T>::t* __restrict__ spec,
                                                                    T* __restrict__ phi, int nrows,
                                                                    const typename C2<T>::t* __restrict__ tw,
                                                                    size_t bs_spec, size_t bs_phi) {
    typedef typename C2<T>::t C;
    typedef FftGeom<T, L> Gm;
    constexpr int M = Gm::M, MH = Gm::MH, RB = Gm::RB, NTX = Gm::NTX;
    spec += blockIdx.y * bs_spec;
    phi += blockIdx.y * bs_phi;
    extern __shared__ __align__(16) unsigned char sm[];
    C* A = reinterpret_cast<C*>(sm);
    C* tws = A + RB * M;
    stage_twiddles<C, L>(tws, tw);
    __syncthreads();
    const int row0 = blockIdx.x * RB;
    for (int t = threadIdx.x; t < RB * M; t += NTX) {
        const int l = t / M, k = t % M;
        const int row = row0 + l;
        C z;
        if (row < nrows) {
            const size_t srow = size_t(row / P) * L + row % P;
            C xk = spec[srow * MH + k];
            C xm = cconj(spec[srow * MH + (M - k)]);
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
    StockhamIP<C, true, M, RB, 1, M, false, 1, M, L, NTX, (2 * P <= L) ? 2 : 0>::run(A, tws);
    for (int t = threadIdx.x; t < RB * M; t += NTX) {
        const int l = t / M, j = t % M;
        const int row = row0 + l;
        if (row >= nrows || 2 * j >= P) continue;
        const size_t g = size_t(row) * P + 2 * j;
        *reinterpret_cast<C*>(phi + g) = A[l * M + j];   // two reals as one complex
    }
}

// ---------------------------------------------------------------------------
// Y pass: columns along y for a fixed z < P (forward: P inputs, L outputs;
// inverse: L inputs, P outputs)
// ---------------------------------------------------------------------------
template <typename T, int L, int P, bool INV>
__global__ void __launch_bounds__(FftGeom<T, L>::NTC) fft_y(typename C2<T>::t* __restrict__ spec,
                                                            const typename C2<T>::t* __restrict__ tw,
                                                            size_t bs_spec) {
    typedef typename C2<T>::t C;
    typedef FftGeom<T, L> Gm;
    constexpr int MH = Gm::MH, KB = Gm::KB, NTC = Gm::NTC;
    constexpr int NIN = INV ? L : P, NOUT = INV ? P : L;
    spec += blockIdx.z * bs_spec;
    extern __shared__ __align__(16) unsigned char sm[];
    C* A = reinterpret_cast<C*>(sm);
    C* tws = A + L * KB;
    stage_twiddles<C, L>(tws, tw);
    const int k0 = blockIdx.x * KB;
    const size_t base = size_t(blockIdx.y) * L * MH;
#pragma unroll 4
    for (int t = threadIdx.x; t < L * KB; t += NTC) {
        const int c = t % KB, y = t / KB;
        C v;
        if (k0 + c < MH && y < NIN) v = spec[base + size_t(y) * MH + k0 + c];
        else { v.x = T(0); v.y = T(0); }
        A[y * KB + c] = v;
    }
    __syncthreads();
    // forward: the rows beyond NIN are zero; inverse: only the first NOUT rows are kept
    StockhamIP<C, INV, L, KB, KB, 1, true, 1, L, L, NTC,
               (!INV && 2 * NIN <= L) ? 1 : ((INV && 2 * NOUT <= L) ? 2 : 0)>::run(A, tws);
    for (int t = threadIdx.x; t < NOUT * KB; t += NTC) {
        const int c = t % KB, y = t / KB;
        if (k0 + c < MH) spec[base + size_t(y) * MH + k0 + c] = A[y * KB + c];
    }
}

// ---------------------------------------------------------------------------
// Z pass with the kernel of the solve: forward along z (P inputs), multiply,
// inverse (P outputs).  ISO = false: the 27-point symbol of Sec. 2.3 with
// asin2[k] = 2/3 sin^2(pi k / L) and coef = -4 pi G h^2 * scale; ISO = true:
// the precomputed transform of the isolated Green's function, stored by its
// even symmetry for ky' = min(ky, L - ky), kz' likewise, in the order these
// blocks read it: gtab[ky'][kx block][kz'][kx within the block] (KB columns per
// block, kx padded to whole blocks), so a block reads one contiguous run.
// ---------------------------------------------------------------------------
template <typename T, int L, int P, bool ISO>
__global__ void __launch_bounds__(FftGeom<T, L>::NTC) fft_z_solve(typename C2<T>::t* __restrict__ spec,
                                                                  const typename C2<T>::t* __restrict__ tw,
                                                                  const T* __restrict__ asin2, T coef,
                                                                  const T* __restrict__ gtab, size_t bs_spec) {
    typedef typename C2<T>::t C;
    typedef FftGeom<T, L> Gm;
    constexpr int MH = Gm::MH, KB = Gm::KB, NTC = Gm::NTC;
    spec += blockIdx.z * bs_spec;
    extern __shared__ __align__(16) unsigned char sm[];
    C* A = reinterpret_cast<C*>(sm);
    C* tws = A + L * KB;
    stage_twiddles<C, L>(tws, tw);
    const int k0 = blockIdx.x * KB;
    const int y = blockIdx.y;
    constexpr size_t zs = size_t(L) * MH;
    const size_t base = size_t(y) * MH;
#pragma unroll 4
    for (int t = threadIdx.x; t < L * KB; t += NTC) {
        const int c = t % KB, z = t / KB;
        C v;
        if (k0 + c < MH && z < P) v = spec[base + size_t(z) * zs + k0 + c];
        else { v.x = T(0); v.y = T(0); }
        A[z * KB + c] = v;
    }
    __syncthreads();
    StockhamIP<C, false, L, KB, KB, 1, true, 1, L, L, NTC, (2 * P <= L) ? 1 : 0>::run(A, tws);
    const int ys = y <= L / 2 ? y : L - y;
    for (int t = threadIdx.x; t < L * KB; t += NTC) {
        const int c = t % KB, z = t / KB;
        const int kx = k0 + c;
        C v = A[z * KB + c];
        if (kx < MH) {
            T g;
            if (ISO) {
                const int zz = z <= L / 2 ? z : L - z;
                constexpr int NKB = (MH + KB - 1) / KB;
                g = gtab[((size_t(ys) * NKB + blockIdx.x) * (L / 2 + 1) + zz) * KB + c];
            } else {
                const T ax = asin2[kx], ay = asin2[y], az = asin2[z];
                // 1 - f_x f_y f_z without cancellation, f = 1 - a
                const T D = T(6) * (ax + (T(1) - ax) * (ay + (T(1) - ay) * az));
                g = (kx == 0 && y == 0 && z == 0) ? T(0) : coef / D;
            }
            v.x *= g;
            v.y *= g;
        }
        A[z * KB + c] = v;   // each element is read and written by the same thread
    }
    __syncthreads();
    StockhamIP<C, true, L, KB, KB, 1, true, 1, L, L, NTC, (2 * P <= L) ? 2 : 0>::run(A, tws);
    for (int t = threadIdx.x; t < P * KB; t += NTC) {
        const int c = t % KB, z = t / KB;
        if (k0 + c < MH) spec[base + size_t(z) * zs + k0 + c] = A[z * KB + c];
    }
}

}  // namespace flic
