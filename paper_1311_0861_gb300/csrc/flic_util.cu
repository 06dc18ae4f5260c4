// Conversion, whole-state reduction and per-step bookkeeping kernels of libflic.
#include "flic_internal.h"

namespace flic {

template <typename T>
__global__ void convert_in_kernel(const double* __restrict__ src, T* __restrict__ dst, size_t n) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        dst[i] = T(src[i]);
}
template <typename T>
__global__ void convert_out_kernel(const T* __restrict__ src, double* __restrict__ dst, size_t n) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        dst[i] = double(src[i]);
}

// Pairs of elements per access (16-byte float64 loads or stores), four pairs in
// flight per thread: the host side of these copies may be page-locked memory
// read or written across the CPU-GPU link, where bytes in flight set the rate.
template <typename T> struct Pair;
template <> struct Pair<float> { typedef float2 t; };
template <> struct Pair<double> { typedef double2 t; };

template <typename T>
__global__ void convert_in_pairs(const double2* __restrict__ src, typename Pair<T>::t* __restrict__ dst, size_t npair) {
    const size_t stride = size_t(gridDim.x) * blockDim.x;
    size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x;
    for (; i + 3 * stride < npair; i += 4 * stride) {
        double2 v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = src[i + k * stride];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            typename Pair<T>::t w;
            w.x = T(v[k].x);
            w.y = T(v[k].y);
            dst[i + k * stride] = w;
        }
    }
    for (; i < npair; i += stride) {
        const double2 v = src[i];
        typename Pair<T>::t w;
        w.x = T(v.x);
        w.y = T(v.y);
        dst[i] = w;
    }
}
template <typename T>
__global__ void convert_out_pairs(const typename Pair<T>::t* __restrict__ src, double2* __restrict__ dst, size_t npair) {
    const size_t stride = size_t(gridDim.x) * blockDim.x;
    size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x;
    for (; i + 3 * stride < npair; i += 4 * stride) {
        typename Pair<T>::t v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = src[i + k * stride];
#pragma unroll
        for (int k = 0; k < 4; ++k) dst[i + k * stride] = make_double2(double(v[k].x), double(v[k].y));
    }
    for (; i < npair; i += stride) {
        const typename Pair<T>::t v = src[i];
        dst[i] = make_double2(double(v.x), double(v.y));
    }
}

static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

template <typename T> cudaError_t convert_in(const double* src, T* dst, size_t n, cudaStream_t st) {
    if (n % 2 == 0 && aligned(src, 16) && aligned(dst, 2 * sizeof(T))) {
        convert_in_pairs<T><<<152 * 8, 256, 0, st>>>(reinterpret_cast<const double2*>(src),
                                                      reinterpret_cast<typename Pair<T>::t*>(dst), n / 2);
    } else {
        convert_in_kernel<T><<<152 * 8, 256, 0, st>>>(src, dst, n);
    }
    return cudaGetLastError();
}
template <typename T> cudaError_t convert_out(const T* src, double* dst, size_t n, cudaStream_t st) {
    if (n % 2 == 0 && aligned(dst, 16) && aligned(src, 2 * sizeof(T))) {
        convert_out_pairs<T><<<152 * 8, 256, 0, st>>>(reinterpret_cast<const typename Pair<T>::t*>(src),
                                                       reinterpret_cast<double2*>(dst), n / 2);
    } else {
        convert_out_kernel<T><<<152 * 8, 256, 0, st>>>(src, dst, n);
    }
    return cudaGetLastError();
}
// Device address of a host buffer the GPU reads and writes directly (page-locked
// and mapped into the device address space, e.g. cudaHostAlloc'd), or null for
// pageable memory, which goes through a staging copy instead.
const void* mapped_device_view(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return (at.type == cudaMemoryTypeHost && at.devicePointer) ? at.devicePointer : nullptr;
}

template cudaError_t convert_in<float>(const double*, float*, size_t, cudaStream_t);
template cudaError_t convert_in<double>(const double*, double*, size_t, cudaStream_t);
template cudaError_t convert_out<float>(const float*, double*, size_t, cudaStream_t);
template cudaError_t convert_out<double>(const double*, double*, size_t, cudaStream_t);

// Conserved sums, kappa (Sec. 2.4) and signal speed of a whole state; one row of
// Q_COUNT partial sums per block, plus an atomic max and the validity bit.
template <typename T>
__global__ void state_reduce_kernel(FieldPtrs<T> s, const T* __restrict__ phi, size_t cells, T gamma,
                                    double* partials, double* vmax, unsigned int* status) {
    __shared__ double red[32][Q_COUNT + 1];
    Acc<T> q[Q_COUNT];
    T vm = T(0);
    bool bad = false;
    for (size_t c = blockIdx.x * size_t(blockDim.x) + threadIdx.x; c < cells;
         c += size_t(gridDim.x) * blockDim.x) {
        T f[F_COUNT];
#pragma unroll
        for (int k = 0; k < F_COUNT; ++k) f[k] = s.f[k][c];
        const T ir = rcp(f[F_RHO]), in = rcp(f[F_N]);
        const T K = T(0.5) * (f[F_MX] * f[F_MX] + f[F_MY] * f[F_MY] + f[F_MZ] * f[F_MZ]) * ir;
        const T Kb = T(0.5) * (f[F_QX] * f[F_QX] + f[F_QY] * f[F_QY] + f[F_QZ] * f[F_QZ]) * in;
        q[Q_MASS_GAS].add(f[F_RHO]);
        q[Q_MASS_BME].add(f[F_N]);
        q[Q_MOMX].add(f[F_MX] + f[F_QX]);
        q[Q_MOMY].add(f[F_MY] + f[F_QY]);
        q[Q_MOMZ].add(f[F_MZ] + f[F_QZ]);
        q[Q_EKIN_GAS].add(K);
        q[Q_EINT_GAS].add(f[F_EINT]);
        q[Q_EKIN_BME].add(Kb);
        q[Q_ETHERM_BME].add(T(0.5) * (f[F_PXX] + f[F_PYY] + f[F_PZZ]));
        if (phi) q[Q_EPOT].add(T(0.5) * (f[F_RHO] + f[F_N]) * phi[c]);
        q[Q_KAPPA_GAS].add(fabs(f[F_E] - f[F_EINT] - K));
        T kb = T(0);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int i = (k < 3) ? k : (k == 5 ? 1 : 0);
            const int j = (k < 3) ? k : (k == 3 ? 1 : 2);
            kb += fabs(f[F_NEXX + k] - f[F_PXX + k] - f[F_QX + i] * f[F_QX + j] * in);
        }
        q[Q_KAPPA_BME].add(kb);
        const T cs = sqr_root(gamma * (gamma - T(1)) * f[F_EINT] * ir);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            vm = fmax(vm, fabs(f[F_MX + d]) * ir + cs);
            vm = fmax(vm, fabs(f[F_QX + d]) * in + sqr_root(T(3) * f[F_PXX + d] * in));
        }
        bool ok = f[F_RHO] > T(0) && f[F_N] > T(0) && f[F_EINT] > T(0) && f[F_PXX] > T(0) &&
                  f[F_PYY] > T(0) && f[F_PZZ] > T(0);
#pragma unroll
        for (int k = 0; k < F_COUNT; ++k) ok = ok && finite_val(f[k]);
        bad = bad || !ok;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < Q_COUNT; ++k) {
        double v = warp_sum(q[k].value());
        if (lane == 0) red[warp][k] = v;
    }
    double m = warp_max((double)vm);
    if (lane == 0) red[warp][Q_COUNT] = m;
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, ST_NONPHYSICAL);
    __syncthreads();
    if (warp == 0) {
        for (int k = 0; k <= Q_COUNT; ++k) {
            double v = (lane < nw) ? red[lane][k] : 0.0;
            if (k < Q_COUNT) {
                v = warp_sum(v);
                if (lane == 0) partials[size_t(blockIdx.x) * Q_COUNT + k] = v;
            } else {
                v = warp_max(v);
                if (lane == 0) atomic_max_nonneg(vmax, v);
            }
        }
    }
}

template <typename T>
cudaError_t state_reduce(const FieldPtrs<T>& fields, const T* phi, size_t cells, double gamma, double* partials,
                         int nb, double* vmax, unsigned int* status, cudaStream_t st) {
    state_reduce_kernel<T><<<nb, 256, 0, st>>>(fields, phi, cells, T(gamma), partials, vmax, status);
    return cudaGetLastError();
}

template <typename T>
cudaError_t state_reduce(const T* state, size_t fs, const T* phi, size_t cells, double gamma,
                         double* partials, int nb, double* vmax, unsigned int* status, cudaStream_t st) {
    FieldPtrs<T> f;
    for (int k = 0; k < F_COUNT; ++k) f.f[k] = state + size_t(k) * fs;
    return state_reduce<T>(f, phi, cells, gamma, partials, nb, vmax, status, st);
}
template cudaError_t state_reduce<float>(const float*, size_t, const float*, size_t, double, double*, int,
                                         double*, unsigned int*, cudaStream_t);
template cudaError_t state_reduce<double>(const double*, size_t, const double*, size_t, double, double*, int,
                                          double*, unsigned int*, cudaStream_t);
template cudaError_t state_reduce<double>(const FieldPtrs<double>&, const double*, size_t, double, double*, int,
                                          double*, unsigned int*, cudaStream_t);

__global__ void step_prep_kernel(double* scal, unsigned int* status, double dt, double courant_h) {
    const double v = scal[S_VMAX_CUR];
    scal[S_TAU] = (dt > 0.0) ? dt : courant_h / v;
    scal[S_VMAX_NEXT] = 0.0;
    *status = 0u;
}

cudaError_t step_prep(double* scal, unsigned int* status, double dt, double courant_h, cudaStream_t st) {
    step_prep_kernel<<<1, 1, 0, st>>>(scal, status, dt, courant_h);
    return cudaGetLastError();
}

__global__ void step_prep_batch_kernel(const RunScalars* __restrict__ runs, int nruns, double dt) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nruns) return;
    const RunScalars a = runs[r];
    a.scal[S_TAU] = (dt > 0.0) ? dt : a.courant_h / a.scal[S_VMAX_CUR];
    a.scal[S_VMAX_NEXT] = 0.0;
    *a.status = 0u;
}

cudaError_t step_prep_batch(const RunScalars* runs, int nruns, double dt, cudaStream_t st) {
    step_prep_batch_kernel<<<(nruns + 127) / 128, 128, 0, st>>>(runs, nruns, dt);
    return cudaGetLastError();
}

// Deterministic two-level sum of the per-block partials.  Level 1: FIN_BLOCKS
// blocks each sum a fixed contiguous range of rows (Neumaier compensation) and
// reduce in a fixed order -- float64 throughput per SM is low on this part, so
// the float64 work is spread over many SMs.  Level 2: one block sums the
// FIN_BLOCKS rows in a fixed order and writes the record.
constexpr int FIN_BLOCKS = FINALIZE_ROWS;

template <int NTH>
__device__ __forceinline__ void block_sum_rows(const double* __restrict__ pa, int na, const double* __restrict__ pb,
                                               int nb, int r0, int r1, double* out /* [Q_COUNT] smem */) {
    __shared__ double part[NTH / 32][Q_COUNT];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double s[Q_COUNT], c[Q_COUNT];
#pragma unroll
    for (int k = 0; k < Q_COUNT; ++k) { s[k] = 0.0; c[k] = 0.0; }
    for (int r = r0 + threadIdx.x; r < r1; r += NTH) {
        const double* p = (r < na) ? pa + size_t(r) * Q_COUNT : pb + size_t(r - na) * Q_COUNT;
#pragma unroll
        for (int k = 0; k < Q_COUNT; ++k) {
            const double x = p[k];
            const double t = s[k] + x;
            c[k] += (fabs(s[k]) >= fabs(x)) ? (s[k] - t) + x : (x - t) + s[k];
            s[k] = t;
        }
    }
#pragma unroll
    for (int k = 0; k < Q_COUNT; ++k) {
        const double v = warp_sum(s[k] + c[k]);
        if (lane == 0) part[warp][k] = v;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < Q_COUNT; ++k) {
            const double v = warp_sum(lane < NTH / 32 ? part[lane][k] : 0.0);
            if (lane == 0) out[k] = v;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void finalize_level1_body(const FinalizeArgs& f, int blk, int nblk) {
    __shared__ double res[Q_COUNT];
    const int nb = f.pb ? f.nb : 0;
    const int rows = f.na + nb;
    const int per = (rows + nblk - 1) / nblk;
    const int r0 = min(rows, blk * per), r1 = min(rows, r0 + per);
    block_sum_rows<256>(f.pa, f.na, f.pb, nb, r0, r1, res);
    if (threadIdx.x < Q_COUNT) f.level1[size_t(blk) * Q_COUNT + threadIdx.x] = res[threadIdx.x];
}

// The record of the sums res (already scaled by h^3); thread 0 only.
__device__ __forceinline__ void write_record(const FinalizeArgs& f, const double* res, int count_step) {
    {
        flic_diag* d = f.diag;
        double* scal = f.scal;
        d->mass_gas = res[Q_MASS_GAS];
        d->mass_bme = res[Q_MASS_BME];
        d->mom[0] = res[Q_MOMX];
        d->mom[1] = res[Q_MOMY];
        d->mom[2] = res[Q_MOMZ];
        d->ekin_gas = res[Q_EKIN_GAS];
        d->eint_gas = res[Q_EINT_GAS];
        d->ekin_bme = res[Q_EKIN_BME];
        d->etherm_bme = res[Q_ETHERM_BME];
        d->epot = res[Q_EPOT];
        d->kappa_gas = res[Q_KAPPA_GAS];
        d->kappa_bme = res[Q_KAPPA_BME];
        d->status = (*f.status & ST_NONPHYSICAL) ? FLIC_ERR_NONPHYSICAL : FLIC_OK;
        if (count_step) {
            d->vmax = scal[S_VMAX_NEXT];
            d->dt = scal[S_TAU];
            scal[S_TIME] += scal[S_TAU];
            d->time = scal[S_TIME];
            d->step += 1;
            scal[S_VMAX_CUR] = scal[S_VMAX_NEXT];
        } else {
            d->vmax = scal[S_VMAX_NEXT];
            d->dt = 0.0;
            d->time = scal[S_TIME];
        }
    }
}

__device__ __forceinline__ void finalize_level2_body(const FinalizeArgs& f, int count_step) {
    __shared__ double res[Q_COUNT];
    block_sum_rows<64>(f.level1, FIN_BLOCKS, nullptr, 0, 0, FIN_BLOCKS, res);
    if (threadIdx.x < Q_COUNT) res[threadIdx.x] *= f.h3;
    __syncthreads();
    if (threadIdx.x == 0) write_record(f, res, count_step);
}

// Rows of float32 (sum, compensation) pairs: each thread folds a fixed set of
// rows into per-quantity pairs with the two-sum, the warps and then warp 0
// combine them lane to lane (the same float32 two-sum), and lane k converts
// quantity k once -- no float64 arithmetic in the reduction itself (the
// float64 unit of this GPU is far slower than the float32 pipes).
constexpr int FIN_PAIR_THREADS = 256;
__device__ __forceinline__ void finalize_pairs_body(const FinalizeArgs& f, int count_step) {
    constexpr int NW = FIN_PAIR_THREADS / 32;
    __shared__ float part[NW][Q_COUNT][2];
    __shared__ double res[Q_COUNT];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nb = f.pb ? f.nb : 0;
    const int rows = f.na + nb;
    float s[Q_COUNT], c[Q_COUNT];
#pragma unroll
    for (int k = 0; k < Q_COUNT; ++k) { s[k] = 0.0f; c[k] = 0.0f; }
    for (int r = threadIdx.x; r < rows; r += FIN_PAIR_THREADS) {
        const float2* p = reinterpret_cast<const float2*>(r < f.na ? f.pa + size_t(r) * Q_COUNT
                                                                   : f.pb + size_t(r - f.na) * Q_COUNT);
#pragma unroll
        for (int k = 0; k < Q_COUNT; ++k) {
            const float2 x = p[k];
            const float t = s[k] + x.x;
            const float bb = t - s[k];
            c[k] += x.y + ((s[k] - (t - bb)) + (x.x - bb));
            s[k] = t;
        }
    }
#pragma unroll
    for (int k = 0; k < Q_COUNT; ++k) {
        warp_pair_sum(s[k], c[k]);
        if (lane == 0) {
            part[warp][k][0] = s[k];
            part[warp][k][1] = c[k];
        }
    }
    __syncthreads();
    if (warp == 0) {
        float ms = 0.0f, mc = 0.0f;   // quantity `lane` (lanes < Q_COUNT)
#pragma unroll
        for (int k = 0; k < Q_COUNT; ++k) {
            float ss = lane < NW ? part[lane][k][0] : 0.0f;
            float cc = lane < NW ? part[lane][k][1] : 0.0f;
            warp_pair_sum(ss, cc);
            if (lane == k) { ms = ss; mc = cc; }
        }
        if (lane < Q_COUNT) res[lane] = ((double)ms + (double)mc) * f.h3;
    }
    __syncthreads();
    if (threadIdx.x == 0) write_record(f, res, count_step);
}

__global__ void __launch_bounds__(256) finalize_level1(FinalizeArgs f) {
    finalize_level1_body(f, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(64) step_finalize_kernel(FinalizeArgs f, int count_step) {
    finalize_level2_body(f, count_step);
}
__global__ void __launch_bounds__(FIN_PAIR_THREADS) step_finalize_pairs_kernel(FinalizeArgs f, int count_step) {
    finalize_pairs_body(f, count_step);
}
__global__ void __launch_bounds__(FIN_PAIR_THREADS) step_finalize_pairs_batch_kernel(
    const FinalizeArgs* __restrict__ table, int count_step) {
    const FinalizeArgs f = table[blockIdx.x];
    finalize_pairs_body(f, count_step);
}
// batched: one run per grid row (level 1) / per block (level 2)
__global__ void __launch_bounds__(256) finalize_level1_batch(const FinalizeArgs* __restrict__ table) {
    const FinalizeArgs f = table[blockIdx.y];
    finalize_level1_body(f, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(64) step_finalize_batch_kernel(const FinalizeArgs* __restrict__ table,
                                                                int count_step) {
    const FinalizeArgs f = table[blockIdx.x];
    finalize_level2_body(f, count_step);
}

cudaError_t step_finalize(const double* pa, int na, const double* pb, int nb, double h3, double* scal,
                          unsigned int* status, flic_diag* diag, int count_step, double* level1, int pairs,
                          cudaStream_t st) {
    FinalizeArgs f{pa, na, pb, nb, h3, scal, status, diag, level1, pairs};
    if (pairs) {
        step_finalize_pairs_kernel<<<1, FIN_PAIR_THREADS, 0, st>>>(f, count_step);
        return cudaGetLastError();
    }
    finalize_level1<<<FIN_BLOCKS, 256, 0, st>>>(f);
    step_finalize_kernel<<<1, 64, 0, st>>>(f, count_step);
    return cudaGetLastError();
}

cudaError_t step_finalize_batch(const FinalizeArgs* table, int nruns, int count_step, int pairs, cudaStream_t st) {
    if (pairs) {
        step_finalize_pairs_batch_kernel<<<nruns, FIN_PAIR_THREADS, 0, st>>>(table, count_step);
        return cudaGetLastError();
    }
    finalize_level1_batch<<<dim3(FIN_BLOCKS, nruns), 256, 0, st>>>(table);
    step_finalize_batch_kernel<<<nruns, 64, 0, st>>>(table, count_step);
    return cudaGetLastError();
}

}  // namespace flic
