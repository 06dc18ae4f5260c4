// Fused FlIC/Godunov step of one fluid: Eulerian stage (face solutions, pressure /
// stress and gravity sources), Lagrangian stage (upwind face fluxes), kappa check,
// energy balance, CFL signal speed and conserved sums -- one kernel per fluid.
//
// Kulikov 2013 (GPUPEGAS): Sec. 2.1 (gas), Sec. 2.2 (Boltzmann moments),
// Sec. 2.4 (kappa, energy balance).  Readings where the paper is silent:
//   * Lagrangian flux F_{i+1/2} = W_{i+1/2} f_upwind with W the Eulerian face
//     velocity of that face at time n (gas: V; moments: u_n*);
//   * gravity by central differences of Phi^n with the time-n state;
//   * after kappa is measured the dual variables are synchronised: gas takes
//     e = E - |m|^2/(2 rho) when that is >= eta E, else resets E = e + |m|^2/(2 rho);
//     moments take Pi = nE - q q^T/n when its trace is >= eta tr(nE) and its
//     diagonal is positive, else reset nE = Pi + q q^T/n.
//
// Structure (2.5D z-march).  A block owns a TX x TY column tile and a range of
// z planes (a chunk of a (tile, chunk) grid, or the segments of a balanced
// split, see the kernel).  It walks up the range with a ring of input planes in
// shared memory over the tile plus a 2-cell halo (R2).  Thread i < TX*TY owns
// tile column i; with WIDE the block has one thread per cell of the tile and
// its four 1-cell edge strips (rounded up to whole warps), so the Eulerian
// update of a plane is one item per thread.  Per plane e (two barriers):
//   S0  asynchronous 16-byte copies of plane e+2 into a three-slot ring (the
//       fields the faces need, + Phi), one full iteration ahead of its use;
//   S2  z-face e+1/2, then the Eulerian update of plane e over R1 (f' to smem);
//   S3  upwind fluxes of f' for the tile cells; plane e-1 completes (its +z flux
//       needs f'_e), gets the energy balance and is written out;
//   S1  (same phase as S3) x- and y-face solutions of plane e+1 over the tile
//       plus a 1-cell halo (R1), for the next S2; the threads without a tile
//       column start on them while the others run S3.
// The transported state f' of the tile cell, its partial sum and the last z-flux
// live in registers of the thread that owns the column.
#pragma once

#include <type_traits>

#include "flic_common.cuh"

namespace flic {

// Work item of a batched launch: (run, tile, z chunk, partial-sum row of the run).
struct WorkItem {
    int run, tile, chunk, prow;
};

template <typename T>
struct StencilArgs {
    const T* in;              // input state, field f at in + f * fs (fluid-local field order)
    T* out;                   // output state, same layout
    const T* phi;             // potential of the input state, N^3
    size_t fs;                // field stride in elements
    int n;                    // cells per axis
    int tz;                   // z planes per block; 0: balanced split (below)
    int tiles_x;              // tiles along x (ceil(n / TX))
    int tiles_y;              // tiles along y (ceil(n / TY))
    int zparts;               // balanced split: parts each tile column is cut into (n % zparts == 0)
    int ztop;                 // > 0: tops split (fewer tiles than blocks), lockstep height H < n
    int outflow;              // hydro boundaries: 0 periodic wrap, 1 zero-gradient ghost cells
    const double* tau;        // step size (device scalar)
    double inv_h;             // 1 / h
    T gamma, eta;
    T cool;                   // Lambda of the gas cooling placeholder (0: adiabatic)
    double* partials;         // [num_blocks][Q_COUNT] per-block sums (unscaled by h^3); float32
                              // kernels store (sum, compensation) float32 pairs in the 8-byte slots
    double* vmax;             // signal speed of the output state (atomic max)
    unsigned int* status;     // ST_* bits
};

// Batched launch: block b processes work[b] with the arguments of table[work[b].run].
// Both null for a single run (block (x, y) = (tile, chunk) with the kernel argument).
template <typename T>
struct BatchArgs {
    const StencilArgs<T>* table;
    const WorkItem* work;
};

// ---------------------------------------------------------------------------
// compensated accumulator: float pairs (two-sum) or plain double
// ---------------------------------------------------------------------------
template <typename T> struct Acc;
template <> struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct Acc<float> {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {   // Knuth two-sum
        float t = s + x;
        float bb = t - s;
        c += (s - (t - bb)) + (x - bb);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// The warp's total of float32 two-sum pairs (s, c), as a pair (valid on lane 0):
// combined lane to lane with the two-sum in float32 arithmetic.  The block
// reductions at the end of the float32 fluid kernels stay in float32 until one
// conversion per quantity: float64 arithmetic runs on a unit of this GPU that is
// far slower than the float32 pipes (float64 warp sums had cost the gas kernel
// 1.2 % at 256^3, and 5 % at 128^3).
__device__ __forceinline__ void warp_pair_sum(float& s, float& c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
        const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
        const float t = s + s2;
        const float bb = t - s;
        c += c2 + ((s - (t - bb)) + (s2 - bb));
        s = t;
    }
}

// Two accumulators advanced together: packed float32 two-sum (one instruction
// per operation for both), plain adds in float64.
__device__ __forceinline__ void acc_add2(Acc<double>& qa, Acc<double>& qb, double xa, double xb) {
    qa.add(xa);
    qb.add(xb);
}
__device__ __forceinline__ void acc_add2(Acc<float>& qa, Acc<float>& qb, float xa, float xb) {
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 S = make_float2(qa.s, qb.s), X = make_float2(xa, xb);
    const float2 t = __fadd2_rn(S, X);
    const float2 bb = __ffma2_rn(m1, S, t);                                  // t - s
    const float2 e = __fadd2_rn(__ffma2_rn(m1, __ffma2_rn(m1, bb, t), S),    // s - (t - bb)
                                __ffma2_rn(m1, bb, X));                       // x - bb
    const float2 c = __fadd2_rn(make_float2(qa.c, qb.c), e);
    qa.s = t.x; qb.s = t.y;
    qa.c = c.x; qb.c = c.y;
}

// ---------------------------------------------------------------------------
// physics policies
// ---------------------------------------------------------------------------
// Ring layout: ring[slot][ring field][R2 cell]; the last ring field is Phi.
// Face layout: face[value][...].  Reciprocal densities are formed at use.

template <typename T>
struct GasPhys {
    static constexpr int NF = 6;      // rho, mx, my, mz, E, e
    static constexpr int NR = 7;      // ring: the 6 conserved fields + Phi
    static constexpr int NEX = 0;     // fields read directly (not staged) by the Eulerian update
    static constexpr int NFACE = 2;   // V, P
    static constexpr int R_PHI = 6;
    static constexpr int NQ = 8;      // accumulated quantities
    static constexpr bool COOLS = true;   // has the cooling term (instances with and without it)
    static __device__ __forceinline__ int ring_field(int r) { return r; }
    static __device__ __forceinline__ int extra_field(int) { return 0; }

    // Eulerian face solution (Sec. 2.1) between ring cells a (left) and b (right)
    // along axis d (the stress scale is used by the moment policy only).
    static __device__ __forceinline__ void face(const T* ra, int a, const T* rb, int b, int R2,
                                                int d, T gamma, T, T* outv) {
        T rL = ra[0 * R2 + a], rR = rb[0 * R2 + b];
        T vL = ra[(1 + d) * R2 + a] * rcp(rL);
        T vR = rb[(1 + d) * R2 + b] * rcp(rR);
        T pL = (gamma - T(1)) * ra[5 * R2 + a];
        T pR = (gamma - T(1)) * rb[5 * R2 + b];
        T z2 = rL * rR * gamma * (pL + pR) * rcp(rL + rR);   // squared acoustic impedance
        T iz = rsq(z2);
        T Z = z2 * iz;
        outv[0] = T(0.5) * (vL + vR) + T(0.5) * (pL - pR) * iz;   // V
        outv[1] = T(0.5) * (pL + pR) + T(0.5) * (vL - vR) * Z;    // P
    }

    // Eulerian update of one cell.  fm[d], fpv[d]: face values on the -d and +d
    // faces; g[d]: central-difference gradient of Phi.
    static __device__ __forceinline__ void euler(const T* r, int c, int R2, const T fm[3][NFACE],
                                                 const T fpv[3][NFACE], const T g[3], T tau,
                                                 T rat, T gamma, T cool, const T*, T* f1) {
        T rho = r[0 * R2 + c];
        T m[3] = {r[1 * R2 + c], r[2 * R2 + c], r[3 * R2 + c]};
        T E = r[4 * R2 + c], e = r[5 * R2 + c];
        T dPV = T(0), dV = T(0), mg = T(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            dPV += fpv[d][1] * fpv[d][0] - fm[d][1] * fm[d][0];
            dV += fpv[d][0] - fm[d][0];
            mg += m[d] * g[d];
        }
        f1[0] = rho;
#pragma unroll
        for (int d = 0; d < 3; ++d) f1[1 + d] = m[d] - rat * (fpv[d][1] - fm[d][1]) - tau * rho * g[d];
        f1[4] = E - rat * dPV - tau * mg;
        f1[5] = e - rat * (gamma - T(1)) * e * dV;
        if (cool != T(0)) {
            // cooling placeholder q = Lambda rho^2 sqrt(e / rho) of both energy equations
            const T qc = cool * rho * sqr_root(rho * e);
            f1[4] -= tau * qc;
            f1[5] -= tau * qc;
        }
    }

    static __device__ __forceinline__ T normal_velocity(const T* facev, int) { return facev[0]; }

    // Conserved sums of the time-n state (tile cells).
    static __device__ __forceinline__ void accumulate_input(const T* r, int c, int R2, Acc<T>* q) {
        T rho = r[0 * R2 + c];
        T mx = r[1 * R2 + c], my = r[2 * R2 + c], mz = r[3 * R2 + c];
        acc_add2(q[0], q[1], rho, mx);
        acc_add2(q[2], q[3], my, mz);
        acc_add2(q[4], q[5], T(0.5) * (mx * mx + my * my + mz * mz) * rcp(rho), r[5 * R2 + c]);
        q[6].add(T(0.5) * rho * r[R_PHI * R2 + c]);
    }

    // kappa, energy balance, signal speed and validity of an output cell.
    static __device__ __forceinline__ void finish(T* f, T gamma, T eta, Acc<T>* q, T& vmax, bool& bad) {
        T ir = rcp(f[0]);
        T K = T(0.5) * (f[1] * f[1] + f[2] * f[2] + f[3] * f[3]) * ir;
        T E = f[4], e = f[5];
        const T kap = fabs(E - e - K);
        q[7].add(kap);
        T epsE = E - K;
        if (epsE >= eta * E) e = epsE; else E = e + K;
        f[4] = E;
        f[5] = e;
        T cs = sqr_root(gamma * (gamma - T(1)) * e * ir);
        T vm = fmax(fabs(f[1]), fmax(fabs(f[2]), fabs(f[3]))) * ir + cs;
        vmax = fmax(vmax, vm);
        // kappa takes every output but rho through rho > 0 (1/rho, K), so with rho
        // finite the outputs are all finite iff kappa is (no overflow at these
        // magnitudes)
        bool ok = (f[0] > T(0)) && finite_val(f[0]) && (e > T(0)) && finite_val(kap);
        bad = bad || !ok;
    }

    // Map of accumulated quantities to DiagQ slots.
    static __device__ __forceinline__ int qslot(int i) {
        const int s[NQ] = {Q_MASS_GAS, Q_MOMX, Q_MOMY, Q_MOMZ, Q_EKIN_GAS, Q_EINT_GAS, Q_EPOT, Q_KAPPA_GAS};
        return s[i];
    }
};

template <typename T>
struct BmePhys {
    // transported fields: n, qx, qy, qz, nExx, nEyy, nEzz, nExy, nExz, nEyz, Pxx, Pyy, Pzz, Pxy, Pxz, Pyz
    static constexpr int NF = 16;
    // ring: n, qx, qy, qz, Pxx, Pyy, Pzz, Pxy, Pxz, Pyz, Phi (what the faces need);
    // the energy tensor nE is read directly by the Eulerian update
    static constexpr int NR = 11;
    static constexpr int NEX = 6;
    static constexpr int NFACE = 6;   // u*_x, u*_y, u*_z, Pi*_xd, Pi*_yd, Pi*_zd
    static constexpr int R_P = 4, R_PHI = 10;
    static constexpr int NQ = 8;
    static constexpr bool COOLS = false;
    static __device__ __forceinline__ int ring_field(int r) { return r < 4 ? r : r + 6; }
    static __device__ __forceinline__ int extra_field(int k) { return 4 + k; }

    // index of tensor component (i, j) among (xx, yy, zz, xy, xz, yz)
    static __device__ __forceinline__ int tc(int i, int j) {
        return (i == j) ? i : (i + j + 2);   // (0,1)->3, (0,2)->4, (1,2)->5
    }

    // Eulerian face solution (Sec. 2.2), normal d with tangents t1 < t2.  The
    // stresses Pi*_{.d} are returned multiplied by rs (= tau / h in the step), the
    // factor they carry in every use by the Eulerian update.
    static __device__ __forceinline__ void face(const T* ra, int a, const T* rb, int b, int R2,
                                                int d, T, T rs, T* outv) {
        const int t1 = (d == 0) ? 1 : 0;
        const int t2 = (d == 2) ? 1 : 2;
        T nL = ra[0 * R2 + a], nR = rb[0 * R2 + b];
        T inL = rcp(nL), inR = rcp(nR);
        T unL = ra[(1 + d) * R2 + a] * inL, unR = rb[(1 + d) * R2 + b] * inR;
        T u1L = ra[(1 + t1) * R2 + a] * inL, u1R = rb[(1 + t1) * R2 + b] * inR;
        T u2L = ra[(1 + t2) * R2 + a] * inL, u2R = rb[(1 + t2) * R2 + b] * inR;
        const int pnn = R_P + tc(d, d), pn1 = R_P + tc(d, t1), pn2 = R_P + tc(d, t2);
        T PnnL = ra[pnn * R2 + a], PnnR = rb[pnn * R2 + b];
        T P1L = ra[pn1 * R2 + a], P1R = rb[pn1 * R2 + b];
        T P2L = ra[pn2 * R2 + a], P2R = rb[pn2 * R2 + b];
        const T s3 = T(1.7320508075688772935274463);
        T rho = T(0.5) * (nL + nR);
        T A = T(0.5) * (PnnL + PnnR);
        T iz2 = rsq(rho * A);            // 1/sqrt(rho Pi_nn)
        T Z2 = rho * A * iz2;            // sqrt(rho Pi_nn)
        T Z1 = s3 * Z2;                  // sqrt(3 rho Pi_nn)
        T iz1 = iz2 * (T(1) / s3);
        T iA = rho * iz2 * iz2;          // 1 / Pi_nn
        T dPnn = T(0.5) * (PnnL - PnnR);
        T dun = T(0.5) * (unL - unR);
        T cu = dPnn * (T(1) - s3) * iA * iz1;   // multiplies b_k in u_t
        T cp = dun * rho * (s3 - T(1)) * iz2;   // multiplies b_k in Pi_nt
        outv[d] = T(0.5) * (unL + unR) + dPnn * iz1;
        outv[3 + d] = rs * (A + dun * Z1);
        if constexpr (std::is_same<T, float>::value) {
            // the two tangents share every coefficient: one packed instruction
            // per operation on (t1, t2)
            const float2 h = make_float2(0.5f, 0.5f);
            const float2 uL = make_float2(u1L, u2L), uR = make_float2(u1R, u2R);
            const float2 PL = make_float2(P1L, P2L), PR = make_float2(P1R, P2R);
            const float2 b = __fmul2_rn(h, __fadd2_rn(PL, PR));
            const float2 hiz2 = make_float2(T(0.5) * iz2, T(0.5) * iz2), hZ2 = make_float2(T(0.5) * Z2, T(0.5) * Z2);
            const float2 m1 = make_float2(-1.0f, -1.0f);
            const float2 ut = __ffma2_rn(b, make_float2(cu, cu),
                                         __ffma2_rn(__ffma2_rn(m1, PR, PL), hiz2, __fmul2_rn(h, __fadd2_rn(uL, uR))));
            const float2 pt = __fmul2_rn(make_float2(rs, rs),
                                         __ffma2_rn(b, make_float2(cp, cp), __ffma2_rn(__ffma2_rn(m1, uR, uL), hZ2, b)));
            outv[t1] = ut.x;
            outv[t2] = ut.y;
            outv[3 + t1] = pt.x;
            outv[3 + t2] = pt.y;
        } else {
            T b1 = T(0.5) * (P1L + P1R);
            T b2 = T(0.5) * (P2L + P2R);
            outv[t1] = T(0.5) * (u1L + u1R) + T(0.5) * (P1L - P1R) * iz2 + b1 * cu;
            outv[t2] = T(0.5) * (u2L + u2R) + T(0.5) * (P2L - P2R) * iz2 + b2 * cu;
            outv[3 + t1] = rs * (b1 + T(0.5) * (u1L - u1R) * Z2 + b1 * cp);
            outv[3 + t2] = rs * (b2 + T(0.5) * (u2L - u2R) * Z2 + b2 * cp);
        }
    }

    // nE: the cell's energy tensor (6 components, read directly from global memory).
    // The face stresses fm/fpv[d][3 + i] arrive multiplied by rat = tau / h, so
    // each tensor component is one chain of fused multiply-adds.
    static __device__ __forceinline__ void euler(const T* r, int c, int R2, const T fm[3][NFACE],
                                                 const T fpv[3][NFACE], const T g[3], T tau,
                                                 T rat, T, T, const T* nE, T* f1) {
        T n = r[0 * R2 + c];
        T q[3] = {r[1 * R2 + c], r[2 * R2 + c], r[3 * R2 + c]};
        T Pi[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) Pi[k] = r[(R_P + k) * R2 + c];
        f1[0] = n;
        // momentum: q_i -= sum_d delta_d (rat Pi*_{id}) + tau n dPhi/dx_i
        const T tn = tau * n;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            T acc = q[i] - tn * g[i];
#pragma unroll
            for (int d = 0; d < 3; ++d) acc = (acc - fpv[d][3 + i]) + fm[d][3 + i];
            f1[1 + i] = acc;
        }
        // velocity jumps delta_d u*_i
        T du[3][3];
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int i = 0; i < 3; ++i) du[d][i] = fpv[d][i] - fm[d][i];
        T tq[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) tq[i] = tau * q[i];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int i = (k < 3) ? k : (k == 5 ? 1 : 0);
            const int j = (k < 3) ? k : (k == 3 ? 1 : 2);
            // nE_ij -= sum_d delta_d (rat Pi*_{jd} u*_i + rat Pi*_{id} u*_j) + tau (q_i g_j + q_j g_i)
            T acc = nE[k] - tq[i] * g[j];
            acc = acc - tq[j] * g[i];
            T sP = T(0);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                acc = acc - fpv[d][3 + j] * fpv[d][i];
                acc = acc - fpv[d][3 + i] * fpv[d][j];
                acc = acc + fm[d][3 + j] * fm[d][i];
                acc = acc + fm[d][3 + i] * fm[d][j];
                sP += Pi[tc(j, d)] * du[d][i] + Pi[tc(i, d)] * du[d][j];
            }
            f1[4 + k] = acc;
            f1[10 + k] = Pi[k] - rat * sP;
        }
    }

    static __device__ __forceinline__ T normal_velocity(const T* facev, int d) { return facev[d]; }

    static __device__ __forceinline__ void accumulate_input(const T* r, int c, int R2, Acc<T>* q) {
        T n = r[0 * R2 + c];
        T qx = r[1 * R2 + c], qy = r[2 * R2 + c], qz = r[3 * R2 + c];
        // (scalar adds: pairing these measured slower in this kernel)
        q[0].add(n);
        q[1].add(qx);
        q[2].add(qy);
        q[3].add(qz);
        q[4].add(T(0.5) * (qx * qx + qy * qy + qz * qz) * rcp(n));
        q[5].add(T(0.5) * (r[(R_P + 0) * R2 + c] + r[(R_P + 1) * R2 + c] + r[(R_P + 2) * R2 + c]));
        q[6].add(T(0.5) * n * r[R_PHI * R2 + c]);
    }

    static __device__ __forceinline__ void finish(T* f, T, T eta, Acc<T>* q, T& vmax, bool& bad) {
        T in = rcp(f[0]);
        T qq[6], PE[6];
        T kap = T(0);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int i = (k < 3) ? k : (k == 5 ? 1 : 0);
            const int j = (k < 3) ? k : (k == 3 ? 1 : 2);
            qq[k] = f[1 + i] * f[1 + j] * in;
            PE[k] = f[4 + k] - qq[k];
            kap += fabs(PE[k] - f[10 + k]);
        }
        q[7].add(kap);
        T trE = PE[0] + PE[1] + PE[2];
        T trN = f[4] + f[5] + f[6];
        bool take = (trE >= eta * trN) && (PE[0] > T(0)) && (PE[1] > T(0)) && (PE[2] > T(0));
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            if (take) f[10 + k] = PE[k]; else f[4 + k] = f[10 + k] + qq[k];
        }
        T vm = T(0);
#pragma unroll
        for (int d = 0; d < 3; ++d)
            vm = fmax(vm, fabs(f[1 + d]) * in + sqr_root(T(3) * f[10 + d] * in));
        vmax = fmax(vmax, vm);
        // kappa takes every input of the balance (n through 1/n, q through q q^T / n,
        // nE and Pi directly) and the balance maps finite values to finite values,
        // so with n finite and positive every output is finite iff kappa is (no
        // overflow at these magnitudes)
        bool ok = (f[0] > T(0)) && finite_val(f[0]) && (f[10] > T(0)) && (f[11] > T(0)) && (f[12] > T(0)) &&
                  finite_val(kap);
        bad = bad || !ok;
    }

    static __device__ __forceinline__ int qslot(int i) {
        const int s[NQ] = {Q_MASS_BME, Q_MOMX, Q_MOMY, Q_MOMZ, Q_EKIN_BME, Q_ETHERM_BME, Q_EPOT, Q_KAPPA_BME};
        return s[i];
    }
};

// ---------------------------------------------------------------------------
// shared-memory geometry of a tile
// ---------------------------------------------------------------------------
constexpr int RING_SLOTS = 3;   // planes e, e+1 in use, e+2 in flight

// Launch shape of a fluid kernel: TX x TY column tile, minimum resident blocks
// per SM (register budget), whether the moment energy tensor is staged in
// shared memory (SEX), whether the block has one thread per updated cell (WIDE;
// else one per tile cell, looping over the border cells) and how many x/y faces
// each thread without a tile cell takes first (HR).  How the z planes of a grid
// are split over blocks is chosen at launch (StepCfg).
// With DB the transported state f' and the x/y face buffers are double-buffered
// by plane parity, which lets one barrier per plane separate the stages (see
// the kernel).  PAIRS: float32 f' stored as field pairs (8-byte shared loads and
// stores) -- 1 on, 0 off, -1 for the fluid's default (on for the gas).
template <int TX_, int TY_, int MINB_, bool SEX_, bool WIDE_, int HR_, bool DB_ = false, int PAIRS_ = -1>
struct TileCfg {
    static constexpr int TX = TX_, TY = TY_, MINB = MINB_, HR = HR_, PAIRS = PAIRS_;
    static constexpr bool SEX = SEX_, WIDE = WIDE_, DB = DB_;
};

template <class P, typename T, class C>
struct Geom {
    static constexpr int TX = C::TX, TY = C::TY;
    static constexpr bool SEX = C::SEX;
    static constexpr int NT = TX * TY;                               // tile (own) cells
    // The ring holds the tile + 2-cell halo, filled by 16-byte asynchronous
    // copies of CH elements.  Its rows start XO = CH - 2 columns before the halo
    // (x0 - CH), so that every copy starts on a 16-byte boundary, and are padded
    // to whole copies: logical column ix (global x0 - 2 + ix) sits at ix + XO.
    static constexpr int CH = 16 / sizeof(T);                        // elements per 16-byte copy
    static constexpr int XO = CH - 2;
    static constexpr int W2 = (TX + 4 + XO + CH - 1) / CH * CH, H2 = TY + 4, R2 = W2 * H2;
    static constexpr int W1 = TX + 2, H1 = TY + 2, R1 = W1 * H1;   // tile + 1 halo
    // cells updated by the Eulerian stage: the tile and its four edge strips
    // (the corners of the 1-cell border feed no tile cell's flux)
    static constexpr int NU = NT + 2 * TX + 2 * TY;
    // threads: WIDE -- one updated cell each in phase 1, and the NTH - NT
    // threads without a tile cell (helpers) take x/y faces while the tile
    // threads run S3; else one per tile cell
    static constexpr int NTH = C::WIDE ? (NU + 31) / 32 * 32 : NT;
    static_assert(NTH <= 1024, "tile too large for one block");
    static constexpr int XFW = TX + 3;                               // x faces per R1 row
    static constexpr int YFH = TY + 3;                               // y-face rows
    static constexpr int CPR = W2 / CH;                              // copies per ring row
    static_assert(W2 % CH == 0, "ring rows must split into 16-byte copies");
    static constexpr int NBUF = C::DB ? 2 : 1;                      // copies of f' and the x/y faces
    static_assert(!(C::DB && SEX), "the staged energy tensor has no slot for the one-barrier schedule");
    static constexpr size_t ring_elems = size_t(RING_SLOTS) * P::NR * R2;
    static constexpr size_t xf_one = size_t(P::NFACE) * H1 * XFW;
    static constexpr size_t yf_one = size_t(P::NFACE) * YFH * W1;
    static constexpr size_t fp_one = size_t(P::NF) * R1;
    static constexpr size_t xf_elems = NBUF * xf_one;
    static constexpr size_t yf_elems = NBUF * yf_one;
    // with one updated cell per thread (NTH >= NU) the z face below a cell and the
    // potential of the plane below stay in that thread's registers
    static constexpr bool ZREG = NTH >= NU;
    static constexpr size_t zc_elems = ZREG ? 0 : size_t(P::NFACE) * R1;
    static constexpr size_t fp_elems = NBUF * fp_one;
    static constexpr size_t phim_elems = ZREG ? 0 : R1;
    // fields read only by the Eulerian update (moment energy tensor), staged
    // over the R1 rows in two slots when SEX
    static constexpr size_t ex_slot = size_t(P::NEX) * H1 * W2;
    static constexpr size_t ex_elems = SEX ? 2 * ex_slot : 0;
    // the double-precision reduction scratch starts on a 16-byte boundary,
    // followed by the coordinate tables (CPR + H2 ints, then CPR more used by
    // the outflow kernels)
    static constexpr size_t red_offset =
        ((ring_elems + xf_elems + yf_elems + zc_elems + fp_elems + phim_elems + ex_elems) * sizeof(T) + 15) /
        16 * 16;
    static constexpr size_t tab_offset = red_offset + sizeof(double) * 32 * (P::NQ + 1);
    static constexpr size_t smem_bytes = tab_offset + sizeof(int) * (2 * CPR + H2);

    // Alignment of the 16-byte asynchronous copies (and of the 8-byte float2
    // field pairs and double partials).  The copies land at ring + slot * NR * R2
    // + r * R2 + row * W2 + chunk * CH and exb + (slot * NEX + k) * H1 * W2 + row *
    // W2 + chunk * CH; all terms are multiples of CH when W2 is, and the region
    // bases must be too.  Global sources are x0 - CH + CH * i (x0 a multiple of
    // TX) plus multiples of N (a multiple of 4) and of the field stride (a
    // multiple of 64) from 16-byte aligned field bases, so TX must be a multiple
    // of CH.
    static_assert(TX % CH == 0, "tile columns must start on a 16-byte boundary");
    static_assert(XO + TX + 4 <= W2, "ring rows hold the tile and its halo");
    static_assert((size_t(RING_SLOTS) * P::NR * R2) % CH == 0 && R2 % CH == 0, "ring slots and fields 16-byte aligned");
    static_assert(!SEX || ((ring_elems + xf_elems + yf_elems + zc_elems + fp_elems + phim_elems) * sizeof(T)) % 16 == 0,
                  "staged energy-tensor rows must start on a 16-byte boundary");
    static_assert(!SEX || (size_t(Geom::H1) * W2) % CH == 0, "staged energy-tensor fields 16-byte aligned");
    static_assert(red_offset % 16 == 0 && tab_offset % 8 == 0, "reduction scratch and tables aligned");
    static_assert(smem_bytes <= 227 * 1024, "shared memory of one block");
};

// Updated cell i -> R1 coordinates (jx, jy): tile cells first (so that thread i
// owns the column of tile cell i), then the four edge strips of the border.
template <int TX, int TY>
__device__ __forceinline__ void r1_coords(int i, int& jx, int& jy) {
    if (i < TX * TY) {
        jx = 1 + i % TX;
        jy = 1 + i / TX;
        return;
    }
    int h = i - TX * TY;
    if (h < TX) { jx = 1 + h; jy = 0; return; }
    h -= TX;
    if (h < TX) { jx = 1 + h; jy = TY + 1; return; }
    h -= TX;
    if (h < TY) { jx = 0; jy = 1 + h; return; }
    h -= TY;
    jx = TX + 1;
    jy = 1 + h;
}

// Asynchronous 16-byte global -> shared copy through L2 only (no register
// staging, no L1 allocation) and group bookkeeping.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Ring slot of plane p (p >= -2: the march starts two planes below its range).
__device__ __forceinline__ int ring_slot(int p) { return int(unsigned(p + RING_SLOTS) % unsigned(RING_SLOTS)); }

// OUT: outflow hydro boundaries -- indices clamp to the edge instead of
// wrapping, so the ring holds two layers of ghost copies of the edge cells
// (zero gradient) and the step acts as on the grid extended by them.
// COOL: the gas cooling placeholder is applied (a separate instance, so the
// adiabatic kernels carry none of its code).
template <class P, typename T, class C, bool OUT, bool COOL = false>
__global__ void __launch_bounds__(Geom<P, T, C>::NTH, C::MINB)
fluid_step_kernel(StencilArgs<T> a1, BatchArgs<T> batch) {
    using Gm = Geom<P, T, C>;
    constexpr int TX = C::TX, TY = C::TY;
    constexpr bool SEX = C::SEX;
    constexpr int NT = Gm::NT, R2 = Gm::R2, W2 = Gm::W2, H2 = Gm::H2, R1 = Gm::R1, W1 = Gm::W1;
    constexpr int NTH = Gm::NTH, NU = Gm::NU;
    // float32: the transport runs on field pairs with packed arithmetic (PK);
    // f' may also be stored as field pairs (float2 per pair of fields,
    // pair-major), loaded and stored 8 bytes at a time (FP2): the default for the
    // gas, chosen per launch shape for the moments (their 32 x 12 shape fits it
    // in 128 registers since the z-face carry moved from shared memory to
    // registers, and is 2-4 % faster with it).
    constexpr bool PK = std::is_same<T, float>::value && P::NF % 2 == 0;
    constexpr bool FP2 = PK && (C::PAIRS < 0 ? P::NF < 16 : C::PAIRS > 0);
    static_assert(!FP2 || ((Gm::ring_elems + Gm::xf_elems + Gm::yf_elems + Gm::zc_elems) % 2 == 0 &&
                           Gm::fp_one % 2 == 0),
                  "the f' buffers must start on an 8-byte boundary");
    constexpr int NF = P::NF, NR = P::NR, NFACE = P::NFACE, NEX = P::NEX;
    // float32 x/y face solutions stored as value pairs (one 8-byte shared store
    // or load per two values)
    constexpr bool FC2 = std::is_same<T, float>::value && NFACE % 2 == 0;
    static_assert(!FC2 || (Gm::ring_elems % 2 == 0 && Gm::xf_one % 2 == 0 && Gm::yf_one % 2 == 0),
                  "the face buffers must start on an 8-byte boundary");
    constexpr int NXF = Gm::H1 * Gm::XFW;
    constexpr int NYF = Gm::YFH * W1;
    constexpr int CH = Gm::CH, CPR = Gm::CPR, XO = Gm::XO;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* ring = reinterpret_cast<T*>(smem_raw);
    T* xf = ring + Gm::ring_elems;
    T* yf = xf + Gm::xf_elems;
    T* zc = yf + Gm::yf_elems;
    T* fpb = zc + Gm::zc_elems;
    T* phim = fpb + Gm::fp_elems;
    T* exb = phim + Gm::phim_elems;
    double* red = reinterpret_cast<double*>(smem_raw + Gm::red_offset);
    int* xoff = reinterpret_cast<int*>(smem_raw + Gm::tab_offset);   // wrapped x of each 16-byte column chunk
    int* yoff = xoff + CPR;                                            // wrapped y * N of R2 rows
    int* xlast = yoff + H2;   // outflow: x of the last element of each chunk (ghost chunks repeat the edge)

    const int tid = threadIdx.x;
    // Work of this block: one (tile, z chunk) of a batched work list or of the
    // (tile, chunk) grid; or, with tz = 0, a balanced split over B blocks (one
    // per resident slot).  The work is cut into units -- each tile column in K
    // equal parts along z (K > 1 only when there are fewer tiles than blocks),
    // unit v = tile (v mod T) of part (v / T) -- and the blocks take F = K T / B
    // rounds of whole units (block b takes units b, b + B, ...; concurrent blocks
    // march the same planes of neighbouring tiles, which share their halos in
    // L2), then an equal share of the unit-major (unit, plane) sequence of the
    // remaining K T - F B units, walked as segments that each lie in one unit.
    // With ztop = H > 0 (fewer tiles than blocks) block b < T marches tile b over
    // planes [0, H) -- neighbouring tiles in lockstep -- and the other blocks
    // take equal shares of the tile-major sequence of the tops [H, n).
    int tile = 0, prow, z0 = 0, z1 = 0;
    long long u = 0, u_end = 0;   // remainder range, in plane updates
    int round = 0, full_rounds = 0;
    int ntiles = 1, Lp = 1;       // tiles; planes per unit
    int zbase = 0;                // first plane of the units (tops: H)
    StencilArgs<T> a;
    // unit v from plane offset off, at most `left` planes
    auto unit_seg = [&](int v, int off, long long left) {
        tile = v % ntiles;
        const int zb = zbase + (v / ntiles) * Lp;
        z0 = zb + off;
        z1 = (left < Lp - off) ? z0 + int(left) : zb + Lp;
    };
    if (batch.work) {
        const WorkItem w = batch.work[blockIdx.x];
        a = batch.table[w.run];
        tile = w.tile;
        prow = w.prow;
        z0 = w.chunk * a.tz;
        z1 = min(z0 + a.tz, a.n);
    } else {
        a = a1;
        if (a.tz > 0) {
            tile = blockIdx.x;
            prow = blockIdx.y * gridDim.x + blockIdx.x;
            z0 = blockIdx.y * a.tz;
            z1 = min(z0 + a.tz, a.n);
        } else if (a.ztop > 0) {
            ntiles = a.tiles_x * a.tiles_y;
            prow = blockIdx.x;
            if (int(blockIdx.x) < ntiles) {   // lockstep part: one segment, u = u_end = 0
                tile = blockIdx.x;
                z0 = 0;
                z1 = a.ztop;
            } else {                           // a share of the tops
                zbase = a.ztop;
                Lp = a.n - a.ztop;
                const int nb = int(gridDim.x) - ntiles, j = int(blockIdx.x) - ntiles;
                const long long U = (long long)ntiles * Lp;
                u = U * j / nb;
                u_end = U * (j + 1) / nb;
                const int ur = int(u / Lp);
                unit_seg(ur, int(u - (long long)ur * Lp), u_end - u);
            }
        } else {
            ntiles = a.tiles_x * a.tiles_y;
            const int K = a.zparts > 0 ? a.zparts : 1;
            Lp = a.n / K;
            const int units = ntiles * K;
            full_rounds = units / int(gridDim.x);
            const long long U = (long long)(units - full_rounds * int(gridDim.x)) * Lp;
            u = U * blockIdx.x / gridDim.x;
            u_end = U * (blockIdx.x + 1) / gridDim.x;
            prow = blockIdx.x;
            if (full_rounds > 0) {
                unit_seg(blockIdx.x, 0, Lp);
                round = 1;
            } else {
                const int ur = int(u / Lp);
                unit_seg(ur, int(u - (long long)ur * Lp), u_end - u);
            }
        }
    }
    const bool balanced = !batch.work && a.tz <= 0;
    const int N = a.n;
    const size_t plane = size_t(N) * N;
    // the step's scalars in the storage precision, formed once per block and
    // kept in shared memory (a re-read is a shared load, not a float64 load,
    // multiply and conversion)
    __shared__ T cst[3];
    if (tid == 0) {
        cst[0] = T(*a.tau);
        cst[1] = T(*a.tau * a.inv_h);
        cst[2] = T(0.5 * a.inv_h);
    }
    __syncthreads();
    const T tau = cst[0];
    const T rat = cst[1];
    const T half_ih = cst[2];
    const T gamma = a.gamma, eta = a.eta;
    const T cool = COOL ? a.cool : T(0);
    Acc<T> q[P::NQ];
    T vmax = T(0);
    bool bad = false;

    while (z1 > z0) {   // one segment: a column of planes [z0, z1) of one tile
        const int x0 = (tile % a.tiles_x) * TX;
        const int y0 = (tile / a.tiles_x) * TY;

        // x0 - 2 - XO = x0 - CH and N are multiples of CH, so no chunk straddles the periodic wrap
        // or the domain edge: with outflow a chunk lies inside the grid or wholly
        // in the ghost layers (all its elements then copy one edge cell)
        if constexpr (OUT) {
            for (int i = tid; i < CPR; i += NTH) {
                xoff[i] = min(max(x0 - 2 - XO + CH * i, 0), N - 1);
                xlast[i] = min(max(x0 - 2 - XO + CH * i + CH - 1, 0), N - 1);
            }
            for (int i = tid; i < H2; i += NTH) yoff[i] = min(max(y0 + i - 2, 0), N - 1) * N;
        } else {
            for (int i = tid; i < CPR; i += NTH) xoff[i] = wrap_mod(x0 - 2 - XO + CH * i, N);
            for (int i = tid; i < H2; i += NTH) yoff[i] = wrap_mod(y0 + i - 2, N) * N;
        }
        __syncthreads();

        // own tile cell (threads tid < NT)
        const bool own_tile = tid < NT;
        const int own_tx = own_tile ? tid % TX : 0, own_ty = own_tile ? tid / TX : 0;
        const bool own_valid = own_tile && (x0 + own_tx < N) && (y0 + own_ty < N);
        const int own_c1 = (own_ty + 1) * W1 + (own_tx + 1);

        // S0 of plane pz: asynchronous 16-byte copies of the ring fields of the plane
        // (tile + 2-cell halo) into its ring slot, committed as one group.  Each
        // thread owns fixed (row, chunk) positions and walks the fields.
        constexpr int NPOS = H2 * CPR;
        auto plane_of = [&](int pz) {
            if constexpr (OUT) return min(max(pz, 0), N - 1);
            return pz < 0 ? pz + N : (pz >= N ? pz - N : pz);
        };
        // a ghost chunk at an outflow edge (its elements all copy one edge cell)
        auto ghost_chunk = [&](int c) { return OUT && CH > 1 && xlast[c] != xoff[c] + CH - 1; };
        auto issue_plane = [&](int pz) {
            T* dst = ring + ring_slot(pz) * NR * R2;
            const size_t zoff = size_t(plane_of(pz)) * plane;
            for (int pos = tid; pos < NPOS; pos += NTH) {
                const int iy = pos / CPR, c = pos % CPR;
                T* d = dst + iy * W2 + c * CH;
                const size_t goff = zoff + size_t(yoff[iy]) + xoff[c];
                const T* src = a.in + goff;
                if (ghost_chunk(c)) {
                    // plain loads (visible after the barrier that precedes this
                    // slot's first use, like the asynchronous copies)
#pragma unroll
                    for (int r = 0; r < NR - 1; ++r) {
                        const T v = __ldg(src + size_t(P::ring_field(r)) * a.fs);
#pragma unroll
                        for (int k = 0; k < CH; ++k) d[r * R2 + k] = v;
                    }
                    const T v = __ldg(a.phi + goff);
#pragma unroll
                    for (int k = 0; k < CH; ++k) d[(NR - 1) * R2 + k] = v;
                    continue;
                }
#pragma unroll
                for (int r = 0; r < NR - 1; ++r) cp_async16(d + r * R2, src + size_t(P::ring_field(r)) * a.fs);
                cp_async16(d + (NR - 1) * R2, a.phi + goff);
            }
            cp_async_commit();
        };
        // extra fields of plane pz over the R1 rows into slot pz & 1 (same group as
        // the ring copy issued in the same iteration)
        constexpr int NPOS1 = Gm::H1 * CPR;
        auto issue_extra = [&](int pz) {
            T* dst = exb + (pz & 1) * Gm::ex_slot;
            const size_t zoff = size_t(plane_of(pz)) * plane;
            for (int pos = tid; pos < NPOS1; pos += NTH) {
                const int jy = pos / CPR, c = pos % CPR;
                T* d = dst + jy * W2 + c * CH;
                const T* src = a.in + zoff + size_t(yoff[jy + 1]) + xoff[c];
                if (ghost_chunk(c)) {
#pragma unroll
                    for (int k = 0; k < NEX; ++k) {
                        const T v = __ldg(src + size_t(P::extra_field(k)) * a.fs);
#pragma unroll
                        for (int j = 0; j < CH; ++j) d[k * Gm::H1 * W2 + j] = v;
                    }
                    continue;
                }
#pragma unroll
                for (int k = 0; k < NEX; ++k)
                    cp_async16(d + k * Gm::H1 * W2, src + size_t(P::extra_field(k)) * a.fs);
            }
        };
        // global x of logical R2 column ix (chunks never straddle the wrap or the edge)
        auto gx = [&](int ix) {
            const int px = ix + XO;
            if constexpr (OUT) return ghost_chunk(px / CH) ? xoff[px / CH] : xoff[px / CH] + px % CH;
            return xoff[px / CH] + px % CH;
        };

        const size_t own_g = size_t(yoff[own_ty + 2]) + gx(own_tx + 2);
        T fprev[NF], acc[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) { fprev[f] = T(0); acc[f] = T(0); }
        T wz_prev = T(0);

        // Fields the Eulerian update reads straight from global memory (SEX false):
        // with one updated cell per thread (NTH >= NU) each thread keeps its cell
        // for the whole march, so the next plane's values are loaded into
        // registers one iteration ahead and their latency hides behind a plane.
        constexpr bool PREF = !SEX && NEX > 0 && NTH >= NU;
        T exn[NEX > 0 ? NEX : 1];
        size_t my_g = 0;
        if constexpr (PREF) {
            if (tid < NU) {
                int jx, jy;
                r1_coords<TX, TY>(tid, jx, jy);
                my_g = size_t(yoff[jy + 1]) + gx(jx + 1);
            }
        }
        auto load_ex = [&](int pz) {
            const size_t g = size_t(plane_of(pz)) * plane + my_g;
#pragma unroll
            for (int k = 0; k < NEX; ++k) exn[k] = __ldg(a.in + size_t(P::extra_field(k)) * a.fs + g);
        };
        if constexpr (PREF) {
            if (tid < NU) load_ex(z0 - 1);   // the first plane whose update is needed
        }

        // x / y face solutions of plane pe over the tile + 1-cell halo (S1).  The
        // helpers take the first NH * HR faces (they have no S3 work); the rest go
        // round-robin over all threads.
        constexpr int NH = NTH - NT;
        constexpr int HF = (NH * C::HR < NXF + NYF) ? NH * C::HR : NXF + NYF;
        auto face_item = [&](const T* rpe, T* xfo, T* yfo, int i) {
            T v[NFACE];
            if (i < NXF) {
                const int fx = i % Gm::XFW, jy = i / Gm::XFW;
                const int a2 = (jy + 1) * W2 + fx + XO;
                P::face(rpe, a2, rpe, a2 + 1, R2, 0, gamma, rat, v);
                if constexpr (FC2) {
#pragma unroll
                    for (int k = 0; k < NFACE; k += 2)
                        reinterpret_cast<float2*>(xfo)[(k / 2) * NXF + i] = make_float2(v[k], v[k + 1]);
                } else {
#pragma unroll
                    for (int k = 0; k < NFACE; ++k) xfo[k * NXF + i] = v[k];
                }
            } else {
                const int j = i - NXF;
                const int jx = j % W1, fy = j / W1;
                const int a2 = fy * W2 + jx + 1 + XO;
                P::face(rpe, a2, rpe, a2 + W2, R2, 1, gamma, rat, v);
                if constexpr (FC2) {
#pragma unroll
                    for (int k = 0; k < NFACE; k += 2)
                        reinterpret_cast<float2*>(yfo)[(k / 2) * NYF + j] = make_float2(v[k], v[k + 1]);
                } else {
#pragma unroll
                    for (int k = 0; k < NFACE; ++k) yfo[k * NYF + j] = v[k];
                }
            }
        };
        // face buffers and f' buffer of plane p (by parity with DB)
        auto xf_of = [&](int p) { return xf + (C::DB ? (p & 1) * Gm::xf_one : 0); };
        auto yf_of = [&](int p) { return yf + (C::DB ? (p & 1) * Gm::yf_one : 0); };
        auto fp_of = [&](int p) { return fpb + (C::DB ? (p & 1) * Gm::fp_one : 0); };
        auto xy_faces = [&](const T* rpe, int pe) {
            T* xfo = xf_of(pe);
            T* yfo = yf_of(pe);
            if constexpr (NH > 0) {
                if (!own_tile)
                    for (int i = tid - NT; i < HF; i += NH) face_item(rpe, xfo, yfo, i);
            }
            for (int i = HF + tid; i < NXF + NYF; i += NTH) face_item(rpe, xfo, yfo, i);
        };

        T Wxm = T(0), Wxp = T(0), Wym = T(0), Wyp = T(0);
        // z face e-1/2 of the thread's updated cell and Phi of plane e-1 there,
        // carried from phase 1 of plane e-1 (one updated cell per thread)
        constexpr bool ZREG = Gm::ZREG;
        T zreg[ZREG ? NFACE : 1], phreg = T(0);
#pragma unroll
        for (int k = 0; k < (ZREG ? NFACE : 1); ++k) zreg[k] = T(0);

        // Phase 1 of plane e: the z face e+1/2 and the Eulerian update of plane e
        // over R1 (S2), f' into the plane's buffer; the own tile cell keeps its
        // face normal velocities for its Lagrangian fluxes.
        auto phase1 = [&](int e) {
            const T* re = ring + ring_slot(e) * NR * R2;       // plane e
            const T* rp = ring + ring_slot(e + 1) * NR * R2;   // plane e + 1
            const bool active = (e >= z0 - 1);                // f' of plane e is needed
            const T* xfe = xf_of(e);
            const T* yfe = yf_of(e);
            T* fpo = fp_of(e);
            const size_t zoff_e = size_t(plane_of(e)) * plane;
            for (int i = tid; i < NU; i += NTH) {
                int jx, jy;
                r1_coords<TX, TY>(i, jx, jy);
                const int c1 = jy * W1 + jx;
                const int c2 = (jy + 1) * W2 + jx + 1 + XO;
                T ex[NEX > 0 ? NEX : 1];
                if (active) {
                    if constexpr (PREF) {
#pragma unroll
                        for (int k = 0; k < NEX; ++k) ex[k] = exn[k];
                        if (e + 1 <= z1) load_ex(e + 1);
                    } else if (SEX) {
                        const T* eb = exb + (e & 1) * Gm::ex_slot + jy * W2 + jx + 1 + XO;
#pragma unroll
                        for (int k = 0; k < NEX; ++k) ex[k] = eb[k * Gm::H1 * W2];
                    } else {
                        const size_t g = zoff_e + size_t(yoff[jy + 1]) + gx(jx + 1);
#pragma unroll
                        for (int k = 0; k < NEX; ++k) ex[k] = __ldg(a.in + size_t(P::extra_field(k)) * a.fs + g);
                    }
                }
                T zn[NFACE];
                // conserved sums of the own tile cell at time n (before any shared
                // store of this phase, so its ring reads are shared with the face and
                // the update below)
                if (i < NT && e >= z0 && e < z1 && own_valid) P::accumulate_input(re, c2, R2, q);
                P::face(re, c2, rp, c2, R2, 2, gamma, rat, zn);
                if (active) {
                    T fm[3][NFACE], fpv[3][NFACE];
                    if constexpr (FC2) {
                        const float2* x2 = reinterpret_cast<const float2*>(xfe) + jy * Gm::XFW + jx;
                        const float2* y2 = reinterpret_cast<const float2*>(yfe) + jy * W1 + jx;
#pragma unroll
                        for (int k = 0; k < NFACE; k += 2) {
                            const float2 xm = x2[(k / 2) * NXF], xp = x2[(k / 2) * NXF + 1];
                            const float2 ym = y2[(k / 2) * NYF], yp = y2[(k / 2) * NYF + W1];
                            fm[0][k] = xm.x; fm[0][k + 1] = xm.y;
                            fpv[0][k] = xp.x; fpv[0][k + 1] = xp.y;
                            fm[1][k] = ym.x; fm[1][k + 1] = ym.y;
                            fpv[1][k] = yp.x; fpv[1][k + 1] = yp.y;
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < NFACE; ++k) {
                            fm[0][k] = xfe[k * NXF + jy * Gm::XFW + jx];
                            fpv[0][k] = xfe[k * NXF + jy * Gm::XFW + jx + 1];
                            fm[1][k] = yfe[k * NYF + jy * W1 + jx];
                            fpv[1][k] = yfe[k * NYF + (jy + 1) * W1 + jx];
                        }
                    }
#pragma unroll
                    for (int k = 0; k < NFACE; ++k) {
                        fm[2][k] = ZREG ? zreg[k] : zc[k * R1 + c1];
                        fpv[2][k] = zn[k];
                    }
                    T g[3];
                    g[0] = (re[P::R_PHI * R2 + c2 + 1] - re[P::R_PHI * R2 + c2 - 1]) * half_ih;
                    g[1] = (re[P::R_PHI * R2 + c2 + W2] - re[P::R_PHI * R2 + c2 - W2]) * half_ih;
                    g[2] = (rp[P::R_PHI * R2 + c2] - (ZREG ? phreg : phim[c1])) * half_ih;
                    T f1[NF];
                    P::euler(re, c2, R2, fm, fpv, g, tau, rat, gamma, cool, ex, f1);
                    if constexpr (FP2) {
                        // field pairs side by side: one 8-byte store per pair
#pragma unroll
                        for (int f = 0; f < NF; f += 2)
                            reinterpret_cast<float2*>(fpo)[(f / 2) * R1 + c1] = make_float2(f1[f], f1[f + 1]);
                    } else {
#pragma unroll
                        for (int f = 0; f < NF; ++f) fpo[f * R1 + c1] = f1[f];
                    }
                    if (i < NT) {
                        // own tile cell (i == tid): keep its face normal velocities for S3
                        // (gas: V first on every axis; moments: u*_d is value d)
                        wz_prev = P::normal_velocity(fm[2], 2);
                        Wxm = P::normal_velocity(fm[0], 0);
                        Wxp = P::normal_velocity(fpv[0], 0);
                        Wym = P::normal_velocity(fm[1], 1);
                        Wyp = P::normal_velocity(fpv[1], 1);
                    }
                }
                if constexpr (ZREG) {
#pragma unroll
                    for (int k = 0; k < NFACE; ++k) zreg[k] = zn[k];
                    phreg = re[P::R_PHI * R2 + c2];
                } else {
#pragma unroll
                    for (int k = 0; k < NFACE; ++k) zc[k * R1 + c1] = zn[k];
                    phim[c1] = re[P::R_PHI * R2 + c2];
                }
            }
        };

        // S3 of plane e for the own tile cell: Lagrangian fluxes of f'_e (its own
        // column and four lateral neighbours) with the face velocities kept by
        // phase 1 of plane e; completes plane e - 1 (energy balance, store).
        auto s3 = [&](int e) {
            const T* fpi = fp_of(e);
            const T Wzm = wz_prev;
            // upwind cell of each lateral face (the own cell where the face
            // velocity points away from it)
            const int cxm = own_c1 - (Wxm > T(0) ? 1 : 0);
            const int cxp = own_c1 + (Wxp > T(0) ? 0 : 1);
            const int cym = own_c1 - (Wym > T(0) ? W1 : 0);
            const int cyp = own_c1 + (Wyp > T(0) ? 0 : W1);
            T out[NF];
            if constexpr (PK) {
                // fields in pairs with packed float32 arithmetic (one instruction
                // for two fields); the same operations as the scalar form below
                const float2 wz = make_float2(Wzm, Wzm), nr = make_float2(-rat, -rat), pr = make_float2(rat, rat);
                const float2 wxp = make_float2(Wxp, Wxp), nwxm = make_float2(-Wxm, -Wxm);
                const float2 wyp = make_float2(Wyp, Wyp), nwym = make_float2(-Wym, -Wym);
                const bool zup = Wzm > T(0);
#pragma unroll
                for (int f = 0; f < NF; f += 2) {
                    float2 fc, uxm, uxp, uym, uyp;
                    if constexpr (FP2) {
                        const float2* F2 = reinterpret_cast<const float2*>(fpi) + (f / 2) * R1;
                        fc = F2[own_c1];
                        uxm = F2[cxm];
                        uxp = F2[cxp];
                        uym = F2[cym];
                        uyp = F2[cyp];
                    } else {
                        const T* F0 = fpi + f * R1;
                        const T* F1 = F0 + R1;
                        fc = make_float2(F0[own_c1], F1[own_c1]);
                        uxm = make_float2(F0[cxm], F1[cxm]);
                        uxp = make_float2(F0[cxp], F1[cxp]);
                        uym = make_float2(F0[cym], F1[cym]);
                        uyp = make_float2(F0[cyp], F1[cyp]);
                    }
                    const float2 Fzm = __fmul2_rn(wz, zup ? make_float2(fprev[f], fprev[f + 1]) : fc);
                    const float2 o = __ffma2_rn(nr, Fzm, make_float2(acc[f], acc[f + 1]));   // completes plane e-1
                    float2 t = __fadd2_rn(__ffma2_rn(nwxm, uxm, __fmul2_rn(wxp, uxp)),
                                          __ffma2_rn(nwym, uym, __fmul2_rn(wyp, uyp)));
                    const float2 n2 = __ffma2_rn(pr, Fzm, __ffma2_rn(nr, t, fc));
                    out[f] = o.x;
                    out[f + 1] = o.y;
                    acc[f] = n2.x;
                    acc[f + 1] = n2.y;
                    fprev[f] = fc.x;
                    fprev[f + 1] = fc.y;
                }
            } else {
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    const T* F = fpi + f * R1;
                    const T fc = F[own_c1];
                    const T uxm = F[cxm], uxp = F[cxp], uym = F[cym], uyp = F[cyp];
                    const T Fzm = Wzm * (Wzm > T(0) ? fprev[f] : fc);
                    out[f] = acc[f] - rat * Fzm;                           // completes plane e-1
                    acc[f] = fc - rat * ((Wxp * uxp - Wxm * uxm) + (Wyp * uyp - Wym * uym)) + rat * Fzm;
                    fprev[f] = fc;
                }
            }
            const int l = e - 1;
            if (l >= z0 && l < z1 && own_valid) {
                P::finish(out, gamma, eta, q, vmax, bad);
                const size_t g = size_t(l) * plane + own_g;
#pragma unroll
                for (int f = 0; f < NF; ++f) __stcs(a.out + f * a.fs + g, out[f]);   // streaming global store
            }
        };

        issue_plane(z0 - 2);
        issue_plane(z0 - 1);
        if constexpr (!C::DB) {
            // Two barriers per plane.  Iteration e:
            //   [copies of planes e, e+1 landed; barrier]
            //   phase 1: z faces e+1/2 and the Eulerian update of plane e over R1 (S2)
            //   [barrier]
            //   phase 2: Lagrangian fluxes of the own cell at plane e (S3), then the x/y
            //            faces of plane e+1 (S1) -- the own cell's face velocities were
            //            kept in registers in phase 1, so the face buffers can be reused
            for (int e = z0 - 2; e <= z1; ++e) {
                // plane e + 2 goes into the slot of plane e - 1 (last read in phase 1
                // of the previous iteration); the staged extra fields of plane e + 1
                // (read in phase 1 of the next iteration) travel in the same group
                if (e + 2 <= z1 + 1) {
                    if (SEX && NEX > 0 && e + 1 >= z0 - 1) issue_extra(e + 1);
                    issue_plane(e + 2);
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
                __syncthreads();
                phase1(e);
                __syncthreads();
                if (e >= z0 - 1 && own_tile) s3(e);
                if (e + 1 <= z1) xy_faces(ring + ring_slot(e + 1) * NR * R2, e + 1);
            }
        } else {
            // One barrier per plane (f' and the x/y faces double-buffered by plane
            // parity).  Iteration e, after the barrier that follows the landing of
            // planes e and e+1:
            //   copies of plane e+2 into the slot of plane e-1 (last read before it);
            //   S3 of plane e-1 from f'_{e-1} (complete at the barrier), with the
            //   face velocities phase 1 of plane e-1 left in registers;
            //   phase 1 of plane e: f'_e into the other buffer, reading the x/y
            //   faces of plane e (written in the previous iteration);
            //   x/y faces of plane e+1 into the buffer last read by phase 1 of
            //   plane e-1.
            for (int e = z0 - 2; e <= z1 + 1; ++e) {
                cp_async_wait<0>();
                __syncthreads();
                if (e + 2 <= z1 + 1) issue_plane(e + 2);
                if (e - 1 >= z0 - 1 && own_tile) s3(e - 1);
                if (e <= z1) phase1(e);
                if (e + 1 <= z1) xy_faces(ring + ring_slot(e + 1) * NR * R2, e + 1);
            }
        }
        cp_async_wait<0>();
        // next segment (balanced split only)
        if (!balanced) break;
        if (round > 0 && round < full_rounds) {           // next whole unit
            unit_seg(blockIdx.x + round * int(gridDim.x), 0, Lp);
            ++round;
        } else {
            if (round > 0) {                               // whole units done: the remainder share
                round = 0;
                if (u >= u_end) break;
                const int ur = int(u / Lp);
                unit_seg(full_rounds * int(gridDim.x) + ur, int(u - (long long)ur * Lp), u_end - u);
            } else {                                       // within the remainder share
                u += z1 - z0;
                if (u >= u_end) break;
                unit_seg(full_rounds * int(gridDim.x) + int(u / Lp), 0, u_end - u);
            }
        }
        __syncthreads();   // the ring and the coordinate tables are reused
    }

    // ---- block reduction of the conserved sums, kappa and the signal speed ----
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int NW = NTH / 32;
    const unsigned int badw = __any_sync(0xffffffffu, bad) ? 1u : 0u;
    if constexpr (std::is_same<T, float>::value) {
        // float32 pairs per warp into the scratch, then warp 0 combines them and
        // writes the block's partial row as float32 (sum, compensation) pairs
        float* redf = reinterpret_cast<float*>(red);
#pragma unroll
        for (int k = 0; k < P::NQ; ++k) {
            float s = q[k].s, c = q[k].c;
            warp_pair_sum(s, c);
            if (lane == 0) {
                redf[2 * (warp * (P::NQ + 1) + k)] = s;
                redf[2 * (warp * (P::NQ + 1) + k) + 1] = c;
            }
        }
        const float vm = warp_max(vmax);
        if (lane == 0) redf[2 * (warp * (P::NQ + 1) + P::NQ)] = vm;
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int k = 0; k < P::NQ; ++k) {
                float s = (lane < NW) ? redf[2 * (lane * (P::NQ + 1) + k)] : 0.0f;
                float c = (lane < NW) ? redf[2 * (lane * (P::NQ + 1) + k) + 1] : 0.0f;
                warp_pair_sum(s, c);
                if (lane == 0)
                    reinterpret_cast<float2*>(a.partials)[size_t(prow) * Q_COUNT + P::qslot(k)] = make_float2(s, c);
            }
            const float v = warp_max((lane < NW) ? redf[2 * (lane * (P::NQ + 1) + P::NQ)] : 0.0f);
            if (lane == 0) atomic_max_nonneg(a.vmax, (double)v);
        }
    } else {
#pragma unroll
        for (int k = 0; k < P::NQ; ++k) {
            const double v = warp_sum(q[k].value());
            if (lane == 0) red[warp * (P::NQ + 1) + k] = v;
        }
        const double vm = warp_max((double)vmax);
        if (lane == 0) red[warp * (P::NQ + 1) + P::NQ] = vm;
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int k = 0; k < P::NQ + 1; ++k) {
                double v = (lane < NW) ? red[lane * (P::NQ + 1) + k] : 0.0;
                if (k < P::NQ) {
                    v = warp_sum(v);
                    if (lane == 0) a.partials[size_t(prow) * Q_COUNT + P::qslot(k)] = v;
                } else {
                    v = warp_max(v);
                    if (lane == 0) atomic_max_nonneg(a.vmax, v);
                }
            }
        }
    }
    if (badw && lane == 0) atomicOr(a.status, ST_NONPHYSICAL);
}

}  // namespace flic
