// Reading B of the Lagrangian flux (Sec. 2.1): the transport velocity of a face
// is the mean of the face velocities of the same orientation at the four
// transverse diagonal neighbours of the face (the printed 4-term form taken
// literally), and the upwind side follows the sign of that mean.  Reading A
// (the fused kernels) uses the face's own velocity.
//
// Two plain kernels per fluid, periodic grids only: the Eulerian stage writes
// the post-Eulerian state f' and the normal face velocities of every cell's
// +x, +y, +z faces to scratch; the transport kernel averages the velocities,
// moves f' through the six faces of each cell, and applies the kappa check,
// the energy balance and the signal speed exactly as the fused kernels do
// (the same physics routines of flic_stencil.cuh, here reading one cell's
// fields from registers instead of a shared-memory ring).  This path is a
// reading switch for experiments, not a tuned kernel.
#include "flic_internal.h"

namespace flic {
namespace {

constexpr int FB_THREADS = 256;

// periodic neighbour of cell (i, j, k) by s along axis d
__device__ __forceinline__ size_t nbr(int i, int j, int k, int d, int s, int N) {
    if (d == 0) i = (i + s + N) % N;
    else if (d == 1) j = (j + s + N) % N;
    else k = (k + s + N) % N;
    return size_t(i) + size_t(N) * (size_t(j) + size_t(N) * size_t(k));
}

// the ring fields of a cell (the order the face and Eulerian routines read, Phi last)
template <class P, typename T>
__device__ __forceinline__ void load_cell(const FluxBArgs<T>& a, size_t c, T* v) {
#pragma unroll
    for (int r = 0; r < P::NR - 1; ++r) v[r] = a.in[size_t(P::ring_field(r)) * a.fs + c];
    v[P::NR - 1] = a.phi[c];
}

// block sum of the first `count` accumulators into the partial row of the block
// (slots from P::qslot, starting at `first`; float32: (sum, compensation) pairs
// as in the fused kernels), the maximum signal speed and the validity bit
template <class P, typename T>
__device__ void block_finish(const FluxBArgs<T>& a, Acc<T>* q, int first, int count, T vmax, bool bad) {
    __shared__ double red[32][P::NQ + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = FB_THREADS / 32;
    if constexpr (std::is_same<T, float>::value) {
        float* redf = reinterpret_cast<float*>(&red[0][0]);
        for (int k = 0; k < count; ++k) {
            float s = q[first + k].s, c = q[first + k].c;
            warp_pair_sum(s, c);
            if (lane == 0) {
                redf[2 * (warp * (P::NQ + 1) + k)] = s;
                redf[2 * (warp * (P::NQ + 1) + k) + 1] = c;
            }
        }
        const float vmw = warp_max(vmax);
        if (lane == 0) redf[2 * (warp * (P::NQ + 1) + P::NQ)] = vmw;
        const bool badw = __any_sync(0xffffffffu, bad);
        __syncthreads();
        if (warp == 0) {
            for (int k = 0; k < count; ++k) {
                float s = lane < NW ? redf[2 * (lane * (P::NQ + 1) + k)] : 0.0f;
                float c = lane < NW ? redf[2 * (lane * (P::NQ + 1) + k) + 1] : 0.0f;
                warp_pair_sum(s, c);
                if (lane == 0)
                    reinterpret_cast<float2*>(a.partials)[size_t(blockIdx.x) * Q_COUNT + P::qslot(first + k)] =
                        make_float2(s, c);
            }
            const float v = warp_max(lane < NW ? redf[2 * (lane * (P::NQ + 1) + P::NQ)] : 0.0f);
            if (lane == 0 && v > 0.0f) atomic_max_nonneg(a.vmax, (double)v);
        }
        if (badw && lane == 0) atomicOr(a.status, ST_NONPHYSICAL);
        return;
    }
    for (int k = 0; k < count; ++k) {
        const double v = warp_sum(q[first + k].value());
        if (lane == 0) red[warp][k] = v;
    }
    const double vm = warp_max((double)vmax);
    if (lane == 0) red[warp][P::NQ] = vm;
    const bool badw = __any_sync(0xffffffffu, bad);
    __syncthreads();
    if (warp == 0) {
        for (int k = 0; k < count; ++k) {
            double v = lane < NW ? red[lane][k] : 0.0;
            v = warp_sum(v);
            if (lane == 0) a.partials[size_t(blockIdx.x) * Q_COUNT + P::qslot(first + k)] = v;
        }
        double v = lane < NW ? red[lane][P::NQ] : 0.0;
        v = warp_max(v);
        if (lane == 0 && v > 0.0) atomic_max_nonneg(a.vmax, v);
    }
    if (badw && lane == 0) atomicOr(a.status, ST_NONPHYSICAL);
}

// Eulerian stage (Sec. 2.1 / 2.2) of every cell: f' and the velocities of its
// +x, +y, +z faces; conserved sums of the time-n state.
template <class P, typename T>
__global__ void __launch_bounds__(FB_THREADS) euler_b_kernel(FluxBArgs<T> a) {
    constexpr int NF = P::NF, NR = P::NR, NFACE = P::NFACE, NEX = P::NEX;
    const int N = a.n;
    const size_t cells = size_t(N) * N * N;
    const T tau = T(*a.tau), rat = T(*a.tau * a.inv_h), half_ih = T(0.5 * a.inv_h);
    Acc<T> q[P::NQ];
    for (size_t c = blockIdx.x * size_t(blockDim.x) + threadIdx.x; c < cells; c += size_t(gridDim.x) * blockDim.x) {
        const int i = int(c % N), j = int((c / N) % N), k = int(c / (size_t(N) * N));
        T ctr[NR];
        load_cell<P, T>(a, c, ctr);
        T fm[3][NFACE], fpv[3][NFACE], g[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            T lo[NR], hi[NR];
            load_cell<P, T>(a, nbr(i, j, k, d, -1, N), lo);
            load_cell<P, T>(a, nbr(i, j, k, d, +1, N), hi);
            P::face(lo, 0, ctr, 0, 1, d, a.gamma, rat, fm[d]);
            P::face(ctr, 0, hi, 0, 1, d, a.gamma, rat, fpv[d]);
            g[d] = (hi[NR - 1] - lo[NR - 1]) * half_ih;
        }
        T ex[NEX > 0 ? NEX : 1];
#pragma unroll
        for (int e = 0; e < NEX; ++e) ex[e] = a.in[size_t(P::extra_field(e)) * a.fs + c];
        T f1[NF];
        P::euler(ctr, 0, 1, fm, fpv, g, tau, rat, a.gamma, a.cool, ex, f1);
#pragma unroll
        for (int f = 0; f < NF; ++f) a.fp[size_t(f) * a.fs + c] = f1[f];
#pragma unroll
        for (int d = 0; d < 3; ++d) a.w[size_t(d) * a.fs + c] = P::normal_velocity(fpv[d], d);
        P::accumulate_input(ctr, 0, 1, q);
    }
    block_finish<P, T>(a, q, 0, P::NQ - 1, T(0), false);
}

// Lagrangian stage with the reading-B velocity, then kappa, the energy balance
// (Sec. 2.4) and the signal speed of every cell.
template <class P, typename T>
__global__ void __launch_bounds__(FB_THREADS) transport_b_kernel(FluxBArgs<T> a) {
    constexpr int NF = P::NF;
    const int N = a.n;
    const size_t cells = size_t(N) * N * N;
    const T rat = T(*a.tau * a.inv_h);
    Acc<T> q[P::NQ];
    T vmax = T(0);
    bool bad = false;
    for (size_t c = blockIdx.x * size_t(blockDim.x) + threadIdx.x; c < cells; c += size_t(gridDim.x) * blockDim.x) {
        const int i = int(c % N), j = int((c / N) % N), k = int(c / (size_t(N) * N));
        // mean face velocity over the four transverse diagonal neighbours of the
        // +d face of cell (ii, jj, kk)
        auto wbar = [&](int d, int ii, int jj, int kk) {
            const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
            const T* W = a.w + size_t(d) * a.fs;
            T acc = T(0);
#pragma unroll
            for (int s1 = 1; s1 >= -1; s1 -= 2)
#pragma unroll
                for (int s2 = 1; s2 >= -1; s2 -= 2) {
                    int c3[3] = {ii, jj, kk};
                    c3[t1] = (c3[t1] + s1 + N) % N;
                    c3[t2] = (c3[t2] + s2 + N) % N;
                    acc = acc + W[size_t(c3[0]) + size_t(N) * (size_t(c3[1]) + size_t(N) * size_t(c3[2]))];
                }
            return T(0.25) * acc;
        };
        T Wp[3], Wm[3];
        size_t cp[3], cm[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            cp[d] = nbr(i, j, k, d, +1, N);
            cm[d] = nbr(i, j, k, d, -1, N);
            Wp[d] = wbar(d, i, j, k);
            Wm[d] = wbar(d, d == 0 ? (i - 1 + N) % N : i, d == 1 ? (j - 1 + N) % N : j, d == 2 ? (k - 1 + N) % N : k);
        }
        T o[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const T* F = a.fp + size_t(f) * a.fs;
            const T fc = F[c];
            T out = fc;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const T Fp = Wp[d] * (Wp[d] > T(0) ? fc : F[cp[d]]);
                const T Fm = Wm[d] * (Wm[d] > T(0) ? F[cm[d]] : fc);
                out = out - rat * (Fp - Fm);
            }
            o[f] = out;
        }
        P::finish(o, a.gamma, a.eta, q, vmax, bad);
#pragma unroll
        for (int f = 0; f < NF; ++f) a.out[size_t(f) * a.fs + c] = o[f];
    }
    block_finish<P, T>(a, q, P::NQ - 1, 1, vmax, bad);
}

}  // namespace

template <typename T>
cudaError_t launch_flux_b(int fluid, const FluxBArgs<T>& a, int blocks, cudaStream_t st) {
    if (fluid == FLUID_GAS) {
        euler_b_kernel<GasPhys<T>, T><<<blocks, FB_THREADS, 0, st>>>(a);
        transport_b_kernel<GasPhys<T>, T><<<blocks, FB_THREADS, 0, st>>>(a);
    } else {
        euler_b_kernel<BmePhys<T>, T><<<blocks, FB_THREADS, 0, st>>>(a);
        transport_b_kernel<BmePhys<T>, T><<<blocks, FB_THREADS, 0, st>>>(a);
    }
    return cudaGetLastError();
}

template cudaError_t launch_flux_b<float>(int, const FluxBArgs<float>&, int, cudaStream_t);
template cudaError_t launch_flux_b<double>(int, const FluxBArgs<double>&, int, cudaStream_t);

}  // namespace flic
