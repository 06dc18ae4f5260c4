// C ABI of libflic: handle, device memory, one step as a launch sequence or a
// CUDA-graph replay, state transfer and diagnostics.  See include/flic.h.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "flic_fft.h"
#include "flic_internal.h"

using namespace flic;

struct flic_handle {
    flic_grid_desc d;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int N = 0;
    size_t cells = 0, fs = 0;
    double h = 0.0;
    bool fp64 = true;
    size_t esz = 8;
    void* state[2] = {nullptr, nullptr};
    int cur = 0;
    void* phi = nullptr;
    void* spec = nullptr;
    void* tw = nullptr;
    int tw_len = 0;
    void* asin2 = nullptr;
    void* gtab = nullptr;             // isolated mode: scaled transform of the Green's function, ~(N+1)^3
    bool iso = false;
    FftPlans plans;
    double* scal = nullptr;
    unsigned int* status = nullptr;
    double* part_gas = nullptr;
    double* part_bme = nullptr;
    double* part_diag = nullptr;
    double* level1 = nullptr;         // second-level partial sums
    int nb_diag = 0;
    StepCfg gcfg, bcfg;
    int rows_gas = 0, rows_bme = 0;   // partial rows allocated per fluid kernel
    bool flux_b = false;              // reading B of the transport velocity (flic_flux_b.cu)
    void* fb_fp = nullptr;            // reading B: f' of both fluids (22 fields)
    void* fb_w = nullptr;             // reading B: +x/+y/+z face velocities of both fluids (6 fields)
    flic_diag* diag_dev = nullptr;    // [0] last step, [1] current-state diagnostics
    flic_diag* diag_host = nullptr;   // pinned
    double* staging = nullptr;        // one float64 field
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    double graph_dt[2] = {0.0, 0.0};
    std::string err;
};

static std::string g_init_err;

namespace flic {
void set_global_error(const char* msg) { g_init_err = msg; }
}  // namespace flic

#define FLIC_CK(h, call)                                                                     \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            (h)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                   \
            return (e_ == cudaErrorMemoryAllocation) ? FLIC_ERR_OOM : FLIC_ERR_CUDA;         \
        }                                                                                    \
    } while (0)

static bool valid_n(int n) {
    if (n < 8 || n > 1024) return false;
    int m = n;
    while (m % 2 == 0) m /= 2;
    while (m % 3 == 0) m /= 3;
    return m == 1 && n % 4 == 0;
}

template <typename T>
static T* field_ptr(void* base, size_t fs, int f) {
    return reinterpret_cast<T*>(base) + size_t(f) * fs;
}

template <typename T>
static int enqueue_poisson(flic_handle* h) {
    if (h->d.G == 0.0) return FLIC_OK;   // phi stays zero
    const T* s = reinterpret_cast<const T*>(h->state[h->cur]);
    if (h->iso) {
        FLIC_CK(h, poisson_isolated<T>(s + F_RHO * h->fs, s + F_N * h->fs, reinterpret_cast<T*>(h->phi), h->spec,
                                       h->N, h->tw, reinterpret_cast<const T*>(h->gtab), h->st));
    } else {
        FLIC_CK(h, poisson_periodic<T>(s + F_RHO * h->fs, s + F_N * h->fs, reinterpret_cast<T*>(h->phi), h->spec,
                                       h->N, h->plans, h->tw, h->tw_len, reinterpret_cast<const T*>(h->asin2),
                                       h->d.G * h->h * h->h, h->st));
    }
    return FLIC_OK;
}

// Arguments of one fluid kernel of the current step (state[cur] -> state[1 - cur])
// launched with geometry c.
template <typename T>
static StencilArgs<T> fluid_args(const flic_handle* h, int fluid, const StepCfg& c) {
    StencilArgs<T> a;
    a.phi = reinterpret_cast<const T*>(h->phi);
    a.fs = h->fs;
    a.n = h->N;
    a.outflow = h->d.hydro_bc == FLIC_HYDRO_OUTFLOW;
    a.tau = h->scal + S_TAU;
    a.inv_h = 1.0 / h->h;
    a.gamma = T(h->d.gamma);
    a.eta = T(h->d.eta);
    a.cool = T(h->d.cooling);
    a.vmax = h->scal + S_VMAX_NEXT;
    a.status = h->status;
    const int f0 = fluid == FLUID_GAS ? F_RHO : F_N;   // gas: fields 0..5; moments: 6..21
    a.in = field_ptr<T>(h->state[h->cur], h->fs, f0);
    a.out = field_ptr<T>(h->state[1 - h->cur], h->fs, f0);
    a.tz = c.tz;
    a.tiles_x = c.tiles_x;
    a.tiles_y = c.tiles_y;
    a.zparts = c.zparts;
    a.ztop = c.ztop;
    a.partials = fluid == FLUID_GAS ? h->part_gas : h->part_bme;
    return a;
}

// Arguments of the reading-B kernels of one fluid (state[cur] -> state[1 - cur]).
template <typename T>
static FluxBArgs<T> flux_b_args(const flic_handle* h, int fluid) {
    FluxBArgs<T> a;
    const int f0 = fluid == FLUID_GAS ? F_RHO : F_N;
    a.in = field_ptr<T>(h->state[h->cur], h->fs, f0);
    a.out = field_ptr<T>(h->state[1 - h->cur], h->fs, f0);
    a.phi = reinterpret_cast<const T*>(h->phi);
    a.fp = field_ptr<T>(h->fb_fp, h->fs, f0);
    a.w = field_ptr<T>(h->fb_w, h->fs, fluid == FLUID_GAS ? 0 : 3);
    a.fs = h->fs;
    a.n = h->N;
    a.tau = h->scal + S_TAU;
    a.inv_h = 1.0 / h->h;
    a.gamma = T(h->d.gamma);
    a.eta = T(h->d.eta);
    a.cool = fluid == FLUID_GAS ? T(h->d.cooling) : T(0);
    a.partials = fluid == FLUID_GAS ? h->part_gas : h->part_bme;
    a.vmax = h->scal + S_VMAX_NEXT;
    a.status = h->status;
    return a;
}

// One full step on the handle's stream; flips the state buffers.  With `ev`
// (5 events) the stage boundaries are recorded: start, after the Poisson solve,
// after the gas kernel, after the moment kernel, after the final reduction.
template <typename T>
static int enqueue_step(flic_handle* h, double dt, cudaEvent_t* ev = nullptr) {
    if (ev) FLIC_CK(h, cudaEventRecord(ev[0], h->st));
    FLIC_CK(h, step_prep(h->scal, h->status, dt, h->d.courant * h->h, h->st));
    int rc = enqueue_poisson<T>(h);
    if (rc) return rc;
    if (ev) FLIC_CK(h, cudaEventRecord(ev[1], h->st));
    if (h->flux_b) {
        for (int fluid = 0; fluid < 2; ++fluid) {
            FLIC_CK(h, launch_flux_b<T>(fluid, flux_b_args<T>(h, fluid), FLUX_B_BLOCKS, h->st));
            if (ev) FLIC_CK(h, cudaEventRecord(ev[2 + fluid], h->st));
        }
        FLIC_CK(h, step_finalize(h->part_gas, FLUX_B_BLOCKS, h->part_bme, FLUX_B_BLOCKS, h->h * h->h * h->h,
                                 h->scal, h->status, h->diag_dev, 1, h->level1, !h->fp64, h->st));
    } else {
        const StencilArgs<T> ag = fluid_args<T>(h, FLUID_GAS, h->gcfg);
        FLIC_CK(h, stencil_launch<T>(FLUID_GAS, ag, h->gcfg, h->st));
        if (ev) FLIC_CK(h, cudaEventRecord(ev[2], h->st));
        const StencilArgs<T> ab = fluid_args<T>(h, FLUID_BME, h->bcfg);
        FLIC_CK(h, stencil_launch<T>(FLUID_BME, ab, h->bcfg, h->st));
        if (ev) FLIC_CK(h, cudaEventRecord(ev[3], h->st));
        FLIC_CK(h, step_finalize(h->part_gas, h->gcfg.num_blocks(), h->part_bme, h->bcfg.num_blocks(),
                                 h->h * h->h * h->h, h->scal, h->status, h->diag_dev, 1, h->level1, !h->fp64,
                                 h->st));
    }
    if (ev) FLIC_CK(h, cudaEventRecord(ev[4], h->st));
    h->cur = 1 - h->cur;
    return FLIC_OK;
}

static int do_step(flic_handle* h, double dt, cudaEvent_t* ev = nullptr) {
    return h->fp64 ? enqueue_step<double>(h, dt, ev) : enqueue_step<float>(h, dt, ev);
}

// signal speed and validity of the current state -> vmax_cur, status
template <typename T>
static int enqueue_state_check(flic_handle* h, double* vmax_dst) {
    FLIC_CK(h, cudaMemsetAsync(vmax_dst, 0, sizeof(double), h->st));
    FLIC_CK(h, cudaMemsetAsync(h->status, 0, sizeof(unsigned int), h->st));
    FLIC_CK(h, state_reduce<T>(reinterpret_cast<const T*>(h->state[h->cur]), h->fs,
                               reinterpret_cast<const T*>(h->phi), h->cells, h->d.gamma, h->part_diag,
                               h->nb_diag, vmax_dst, h->status, h->st));
    return FLIC_OK;
}

static int check_status(flic_handle* h) {
    unsigned int s = 0;
    FLIC_CK(h, cudaMemcpyAsync(&s, h->status, sizeof(s), cudaMemcpyDeviceToHost, h->st));
    FLIC_CK(h, cudaStreamSynchronize(h->st));
    if (s & ST_NONPHYSICAL) {
        h->err = "state has a non-positive density, internal energy or diagonal stress, or a non-finite value";
        return FLIC_ERR_NONPHYSICAL;
    }
    return FLIC_OK;
}

template <typename T>
static int set_state_impl(flic_handle* h, const double* const* fields, bool device) {
    for (int f = 0; f < F_COUNT; ++f) {
        if (!fields[f]) { h->err = "null field pointer"; return FLIC_ERR_INVALID_ARG; }
        const double* src = fields[f];
        if (!device) {
            // page-locked host arrays are read in place by the conversion kernel
            src = static_cast<const double*>(mapped_device_view(fields[f]));
            if (!src) {
                FLIC_CK(h, cudaMemcpyAsync(h->staging, fields[f], h->cells * sizeof(double),
                                           cudaMemcpyHostToDevice, h->st));
                src = h->staging;
            }
        }
        FLIC_CK(h, convert_in<T>(src, field_ptr<T>(h->state[h->cur], h->fs, f), h->cells, h->st));
    }
    int rc = enqueue_state_check<T>(h, h->scal + S_VMAX_CUR);
    if (rc) return rc;
    return check_status(h);
}

template <typename T>
static int get_state_impl(flic_handle* h, double* const* fields, bool device) {
    for (int f = 0; f < F_COUNT; ++f) {
        if (!fields[f]) { h->err = "null field pointer"; return FLIC_ERR_INVALID_ARG; }
        const T* src = field_ptr<T>(h->state[h->cur], h->fs, f);
        double* view = device ? fields[f] : static_cast<double*>(const_cast<void*>(mapped_device_view(fields[f])));
        if (view) {
            // device arrays, or page-locked host arrays written in place
            FLIC_CK(h, convert_out<T>(src, view, h->cells, h->st));
        } else {
            FLIC_CK(h, convert_out<T>(src, h->staging, h->cells, h->st));
            FLIC_CK(h, cudaMemcpyAsync(fields[f], h->staging, h->cells * sizeof(double), cudaMemcpyDeviceToHost,
                                       h->st));
        }
    }
    FLIC_CK(h, cudaStreamSynchronize(h->st));
    return FLIC_OK;
}

static void free_all(flic_handle* h) {
    for (int i = 0; i < 2; ++i) {
        if (h->graph[i]) cudaGraphExecDestroy(h->graph[i]);
        if (h->state[i]) cudaFree(h->state[i]);
    }
    void* bufs[] = {h->phi, h->spec, h->tw, h->asin2, h->gtab, h->scal, h->status, h->part_gas, h->part_bme,
                    h->part_diag, h->level1, h->diag_dev, h->staging, h->fb_fp, h->fb_w};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (h->diag_host) cudaFreeHost(h->diag_host);
    if (h->own_stream && h->st) cudaStreamDestroy(h->st);
}

template <typename T>
static int init_impl(flic_handle* h) {
    typedef typename std::conditional<sizeof(T) == 8, double2, float2>::type C;
    const int N = h->N;
    h->cells = size_t(N) * N * N;
    h->fs = (h->cells + 63) / 64 * 64;
    h->esz = sizeof(T);
    if (fft_plan_init(N, &h->plans)) { h->err = "unsupported FFT length"; return FLIC_ERR_INVALID_ARG; }
    if (h->iso && !fft_iso_supported(N)) { h->err = "unsupported size for the isolated solve"; return FLIC_ERR_INVALID_ARG; }
    FLIC_CK(h, stencil_prepare<T>());
    FLIC_CK(h, fft_prepare<T>(N));
    if (h->iso) FLIC_CK(h, fft_prepare_iso<T>(N));
    h->gcfg = stencil_cfg<T>(FLUID_GAS, 0, N, 0);
    h->bcfg = stencil_cfg<T>(FLUID_BME, 0, N, 0);
    // partial rows for the largest grid of any candidate shape (the tuner may switch)
    // and for the reading-B kernels
    h->rows_gas = h->rows_bme = FLUX_B_BLOCKS;
    for (int fluid = 0; fluid < 2; ++fluid) {
        int nc = 0;
        stencil_cands<T>(fluid, &nc);
        for (int c = 0; c < nc; ++c) {
            const int nb = stencil_cfg<T>(fluid, c, N, 0).num_blocks();
            int& m = fluid == FLUID_GAS ? h->rows_gas : h->rows_bme;
            if (nb > m) m = nb;
        }
    }
    h->nb_diag = 152 * 4;
    for (int i = 0; i < 2; ++i) {
        FLIC_CK(h, cudaMalloc(&h->state[i], F_COUNT * h->fs * sizeof(T)));
        FLIC_CK(h, cudaMemsetAsync(h->state[i], 0, F_COUNT * h->fs * sizeof(T), h->st));
    }
    FLIC_CK(h, cudaMalloc(&h->phi, h->fs * sizeof(T)));
    FLIC_CK(h, cudaMemsetAsync(h->phi, 0, h->fs * sizeof(T), h->st));
    const int L = h->iso ? 2 * N : N;   // transform length
    FLIC_CK(h, cudaMalloc(&h->spec, size_t(N) * L * (L / 2 + 1) * sizeof(C)));
    h->tw_len = L;
    {
        C* tw = new C[L];
        for (int j = 0; j < L; ++j) {
            const long double ang = 2.0L * 3.141592653589793238462643383279502884L * j / L;
            tw[j].x = T(std::cos(ang));
            tw[j].y = T(-std::sin(ang));
        }
        cudaError_t e = cudaMalloc(&h->tw, L * sizeof(C));
        if (e == cudaSuccess) e = cudaMemcpy(h->tw, tw, L * sizeof(C), cudaMemcpyHostToDevice);
        delete[] tw;
        FLIC_CK(h, e);
        T* a2 = new T[N];
        for (int k = 0; k < N; ++k) {
            const long double s = std::sin(3.141592653589793238462643383279502884L * k / N);
            a2[k] = T((2.0L / 3.0L) * s * s);
        }
        e = cudaMalloc(&h->asin2, N * sizeof(T));
        if (e == cudaSuccess) e = cudaMemcpy(h->asin2, a2, N * sizeof(T), cudaMemcpyHostToDevice);
        delete[] a2;
        FLIC_CK(h, e);
    }
    if (h->iso) {
        // transform of the Green's function, computed once with temporary workspace
        FLIC_CK(h, cudaMalloc(&h->gtab, green_table_elems<T>(N) * sizeof(T)));
        void* greal = nullptr;
        void* gspec = nullptr;
        cudaError_t e = cudaMalloc(&greal, size_t(L) * L * L * sizeof(T));
        if (e == cudaSuccess) e = cudaMalloc(&gspec, size_t(L) * L * (L / 2 + 1) * sizeof(C));
        if (e == cudaSuccess)
            e = green_init<T>(N, h->h, h->d.G, reinterpret_cast<T*>(h->gtab), reinterpret_cast<T*>(greal), gspec,
                              h->tw, h->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
        if (greal) cudaFree(greal);
        if (gspec) cudaFree(gspec);
        FLIC_CK(h, e);
    }
    FLIC_CK(h, cudaMalloc(&h->scal, S_COUNT * sizeof(double)));
    FLIC_CK(h, cudaMemsetAsync(h->scal, 0, S_COUNT * sizeof(double), h->st));
    FLIC_CK(h, cudaMalloc(&h->status, sizeof(unsigned int)));
    FLIC_CK(h, cudaMemsetAsync(h->status, 0, sizeof(unsigned int), h->st));
    const size_t pg = size_t(h->rows_gas) * Q_COUNT, pb = size_t(h->rows_bme) * Q_COUNT;
    FLIC_CK(h, cudaMalloc(&h->part_gas, pg * sizeof(double)));
    FLIC_CK(h, cudaMalloc(&h->part_bme, pb * sizeof(double)));
    FLIC_CK(h, cudaMalloc(&h->part_diag, size_t(h->nb_diag) * Q_COUNT * sizeof(double)));
    FLIC_CK(h, cudaMalloc(&h->level1, size_t(FINALIZE_ROWS) * Q_COUNT * sizeof(double)));
    FLIC_CK(h, cudaMemsetAsync(h->part_gas, 0, pg * sizeof(double), h->st));
    FLIC_CK(h, cudaMemsetAsync(h->part_bme, 0, pb * sizeof(double), h->st));
    FLIC_CK(h, cudaMalloc(&h->diag_dev, 2 * sizeof(flic_diag)));
    FLIC_CK(h, cudaMemsetAsync(h->diag_dev, 0, 2 * sizeof(flic_diag), h->st));
    FLIC_CK(h, cudaMallocHost(&h->diag_host, 2 * sizeof(flic_diag)));
    FLIC_CK(h, cudaMalloc(&h->staging, h->cells * sizeof(double)));
    if (h->flux_b) {
        FLIC_CK(h, cudaMalloc(&h->fb_fp, F_COUNT * h->fs * sizeof(T)));
        FLIC_CK(h, cudaMalloc(&h->fb_w, 6 * h->fs * sizeof(T)));
    }
    FLIC_CK(h, cudaStreamSynchronize(h->st));
    return FLIC_OK;
}

// ---- launch-shape tuner ------------------------------------------------------
// Choices made in this process, per (device name and SM count, n, precision,
// hydro boundary): (gas candidate, moment candidate).
typedef std::tuple<std::string, int, int, int> TuneKey;
static std::mutex g_tune_mu;
static std::map<TuneKey, std::pair<int, int>> g_tune_cache;

static TuneKey tune_key(const flic_handle* h) {
    int dev = 0;
    cudaDeviceProp p;
    std::string name = "unknown";
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&p, dev) == cudaSuccess)
        name = std::string(p.name) + "/" + std::to_string(p.multiProcessorCount);
    return TuneKey(name, h->N, h->d.precision, h->d.hydro_bc);
}

static void drop_graphs(flic_handle* h) {
    for (int i = 0; i < 2; ++i)
        if (h->graph[i]) {
            cudaGraphExecDestroy(h->graph[i]);
            h->graph[i] = nullptr;
        }
}

template <typename T>
static int apply_tile_config(flic_handle* h, int gas, int bme) {
    int ng = 0, nb = 0;
    stencil_cands<T>(FLUID_GAS, &ng);
    stencil_cands<T>(FLUID_BME, &nb);
    if (gas >= ng || bme >= nb || gas < -1 || bme < -1) {
        h->err = "launch shape index out of range";
        return FLIC_ERR_INVALID_ARG;
    }
    FLIC_CK(h, cudaStreamSynchronize(h->st));
    if (gas >= 0) h->gcfg = stencil_cfg<T>(FLUID_GAS, gas, h->N, 0);
    if (bme >= 0) h->bcfg = stencil_cfg<T>(FLUID_BME, bme, h->N, 0);
    drop_graphs(h);
    return FLIC_OK;
}

// Times every candidate shape of both fluid kernels on the current state (one
// untimed launch, then `reps` launches between two events) and applies the
// fastest.  The launches write the spare state buffer only, so the current
// state, the step count and the CFL signal speed are unchanged.
template <typename T>
static int tune_impl(flic_handle* h, int reps, double* ms) {
    FLIC_CK(h, step_prep(h->scal, h->status, 0.0, h->d.courant * h->h, h->st));
    int rc = enqueue_poisson<T>(h);
    if (rc) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    FLIC_CK(h, cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        FLIC_CK(h, ce);
    }
    int best[2] = {0, 0};
    int k = 0;
    for (int fluid = 0; fluid < 2 && rc == FLIC_OK; ++fluid) {
        int nc = 0;
        stencil_cands<T>(fluid, &nc);
        double best_ms = -1.0;
        for (int c = 0; c < nc; ++c, ++k) {
            const StepCfg cfg = stencil_cfg<T>(fluid, c, h->N, 0);
            const StencilArgs<T> a = fluid_args<T>(h, fluid, cfg);
            double t = -1.0;
            if (cfg.num_blocks() <= (fluid == FLUID_GAS ? h->rows_gas : h->rows_bme)) {
                cudaError_t e = stencil_launch<T>(fluid, a, cfg, h->st);
                if (e == cudaSuccess) e = cudaEventRecord(e0, h->st);
                for (int r = 0; r < reps && e == cudaSuccess; ++r) e = stencil_launch<T>(fluid, a, cfg, h->st);
                if (e == cudaSuccess) e = cudaEventRecord(e1, h->st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float el = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&el, e0, e1);
                if (e == cudaSuccess) {
                    t = double(el) / reps;
                } else if (e == cudaErrorInvalidConfiguration || e == cudaErrorLaunchOutOfResources ||
                           e == cudaErrorInvalidValue) {
                    cudaGetLastError();   // a shape this device cannot launch: skipped
                } else {
                    h->err = std::string("launch-shape tuning: ") + cudaGetErrorString(e);
                    rc = FLIC_ERR_CUDA;
                    break;
                }
            }
            if (ms) ms[k] = t;
            if (t >= 0.0 && (best_ms < 0.0 || t < best_ms * (1.0 - TUNE_MARGIN))) {
                best_ms = t;
                best[fluid] = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    return apply_tile_config<T>(h, best[0], best[1]);
}

extern "C" {

int flic_init_grid(const flic_grid_desc* desc, void* stream, flic_handle** out) {
    if (!desc || !out) { g_init_err = "null argument"; return FLIC_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!valid_n(desc->n)) { g_init_err = "n must be 2^a 3^b, a multiple of 4, 8 <= n <= 1024"; return FLIC_ERR_INVALID_ARG; }
    if (!(desc->box_max > desc->box_min) || !(desc->gamma > 1.0) || !(desc->courant > 0.0) ||
        !(desc->eta >= 0.0) || !(desc->G >= 0.0) || !(desc->cooling >= 0.0)) {
        g_init_err = "invalid physical constants";
        return FLIC_ERR_INVALID_ARG;
    }
    if (desc->precision != FLIC_FP64 && desc->precision != FLIC_MIXED) { g_init_err = "unknown precision"; return FLIC_ERR_INVALID_ARG; }
    if (desc->poisson_bc != FLIC_PERIODIC && desc->poisson_bc != FLIC_ISOLATED) { g_init_err = "unknown Poisson boundary"; return FLIC_ERR_INVALID_ARG; }
    if (desc->hydro_bc != FLIC_HYDRO_PERIODIC && desc->hydro_bc != FLIC_HYDRO_OUTFLOW) { g_init_err = "unknown hydro boundary"; return FLIC_ERR_INVALID_ARG; }
    if (desc->flux_reading != FLIC_FLUX_A && desc->flux_reading != FLIC_FLUX_B) { g_init_err = "unknown flux reading"; return FLIC_ERR_INVALID_ARG; }
    if (desc->flux_reading == FLIC_FLUX_B && desc->hydro_bc != FLIC_HYDRO_PERIODIC) {
        g_init_err = "flux reading B is built for periodic hydro boundaries only";
        return FLIC_ERR_INVALID_ARG;
    }
    flic_handle* h = new flic_handle();
    h->d = *desc;
    h->N = desc->n;
    h->h = (desc->box_max - desc->box_min) / desc->n;
    h->fp64 = desc->precision == FLIC_FP64;
    h->iso = desc->poisson_bc == FLIC_ISOLATED;
    h->flux_b = desc->flux_reading == FLIC_FLUX_B;
    if (stream) {
        h->st = reinterpret_cast<cudaStream_t>(stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking);
        if (e != cudaSuccess) { g_init_err = cudaGetErrorString(e); delete h; return FLIC_ERR_CUDA; }
        h->own_stream = true;
    }
    int rc = h->fp64 ? init_impl<double>(h) : init_impl<float>(h);
    if (rc) {
        g_init_err = h->err;
        free_all(h);
        delete h;
        return rc;
    }
    *out = h;
    return FLIC_OK;
}

int flic_set_state(flic_handle* h, const double* const fields[FLIC_NFIELDS]) {
    if (!h || !fields) return FLIC_ERR_INVALID_ARG;
    return h->fp64 ? set_state_impl<double>(h, fields, false) : set_state_impl<float>(h, fields, false);
}

int flic_set_state_device(flic_handle* h, const double* const fields[FLIC_NFIELDS]) {
    if (!h || !fields) return FLIC_ERR_INVALID_ARG;
    return h->fp64 ? set_state_impl<double>(h, fields, true) : set_state_impl<float>(h, fields, true);
}

int flic_get_state(flic_handle* h, double* const fields[FLIC_NFIELDS]) {
    if (!h || !fields) return FLIC_ERR_INVALID_ARG;
    return h->fp64 ? get_state_impl<double>(h, fields, false) : get_state_impl<float>(h, fields, false);
}

int flic_get_state_device(flic_handle* h, double* const fields[FLIC_NFIELDS]) {
    if (!h || !fields) return FLIC_ERR_INVALID_ARG;
    return h->fp64 ? get_state_impl<double>(h, fields, true) : get_state_impl<float>(h, fields, true);
}

int flic_step(flic_handle* h, double dt, double* dt_used) {
    if (!h) return FLIC_ERR_INVALID_ARG;
    int rc = do_step(h, dt);
    if (rc) return rc;
    if (dt_used) {
        FLIC_CK(h, cudaMemcpyAsync(h->diag_host, h->diag_dev, sizeof(flic_diag), cudaMemcpyDeviceToHost, h->st));
        FLIC_CK(h, cudaStreamSynchronize(h->st));
        *dt_used = h->diag_host[0].dt;
        if (h->diag_host[0].status != FLIC_OK) {
            h->err = "step produced a non-physical state";
            return FLIC_ERR_NONPHYSICAL;
        }
    }
    return FLIC_OK;
}

int flic_run(flic_handle* h, int nsteps, double dt, int sync) {
    if (!h || nsteps < 0) return FLIC_ERR_INVALID_ARG;
    for (int s = 0; s < nsteps; ++s) {
        const int c = h->cur;
        if (!h->graph[c] || h->graph_dt[c] != dt) {
            if (h->graph[c]) { cudaGraphExecDestroy(h->graph[c]); h->graph[c] = nullptr; }
            cudaGraph_t g = nullptr;
            FLIC_CK(h, cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
            int rc = do_step(h, dt);
            cudaError_t e = cudaStreamEndCapture(h->st, &g);
            h->cur = c;   // capture does not run the step
            if (rc) { if (g) cudaGraphDestroy(g); return rc; }
            if (e != cudaSuccess) { h->err = std::string("graph capture: ") + cudaGetErrorString(e); return FLIC_ERR_CUDA; }
            e = cudaGraphInstantiate(&h->graph[c], g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) { h->err = std::string("graph instantiate: ") + cudaGetErrorString(e); return FLIC_ERR_CUDA; }
            h->graph_dt[c] = dt;
        }
        FLIC_CK(h, cudaGraphLaunch(h->graph[c], h->st));
        h->cur = 1 - c;
    }
    if (sync) {
        FLIC_CK(h, cudaMemcpyAsync(h->diag_host, h->diag_dev, sizeof(flic_diag), cudaMemcpyDeviceToHost, h->st));
        FLIC_CK(h, cudaStreamSynchronize(h->st));
        if (nsteps > 0 && h->diag_host[0].status != FLIC_OK) {
            h->err = "step produced a non-physical state";
            return FLIC_ERR_NONPHYSICAL;
        }
    }
    return FLIC_OK;
}

int flic_profile(flic_handle* h, int nsteps, double dt, double stage_ms[FLIC_NSTAGES], double* total_ms) {
    if (!h || nsteps <= 0 || !stage_ms) return FLIC_ERR_INVALID_ARG;
    const int ne = 5 * nsteps;
    cudaEvent_t* ev = new cudaEvent_t[ne];
    int made = 0, rc = FLIC_OK;
    for (; made < ne; ++made) {
        cudaError_t e = cudaEventCreate(&ev[made]);
        if (e != cudaSuccess) { h->err = cudaGetErrorString(e); rc = FLIC_ERR_CUDA; break; }
    }
    for (int s = 0; rc == FLIC_OK && s < nsteps; ++s) rc = do_step(h, dt, ev + 5 * s);
    if (rc == FLIC_OK) {
        cudaError_t e = cudaEventSynchronize(ev[ne - 1]);
        if (e != cudaSuccess) { h->err = cudaGetErrorString(e); rc = FLIC_ERR_CUDA; }
    }
    if (rc == FLIC_OK) {
        for (int k = 0; k < FLIC_NSTAGES; ++k) stage_ms[k] = 0.0;
        for (int s = 0; s < nsteps; ++s)
            for (int k = 0; k < FLIC_NSTAGES; ++k) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[5 * s + k], ev[5 * s + k + 1]);
                stage_ms[k] += ms;
            }
        if (total_ms) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[0], ev[ne - 1]);
            *total_ms = ms;
        }
    }
    for (int i = 0; i < made; ++i) cudaEventDestroy(ev[i]);
    delete[] ev;
    return rc;
}

int flic_launches_per_step(flic_handle* h) {
    if (!h) return FLIC_ERR_INVALID_ARG;
    // step setup, five FFT passes (none without gravity), two fluid kernels (four with
    // reading B), the reduction (one launch over float32 pairs; two levels in float64)
    return 1 + (h->d.G != 0.0 ? 5 : 0) + (h->flux_b ? 4 : 2) + (h->fp64 ? 2 : 1);
}

int flic_solve_poisson(flic_handle* h, double* phi_out) {
    if (!h) return FLIC_ERR_INVALID_ARG;
    int rc = h->fp64 ? enqueue_poisson<double>(h) : enqueue_poisson<float>(h);
    if (rc) return rc;
    if (phi_out) {
        if (h->fp64) {
            FLIC_CK(h, cudaMemcpyAsync(phi_out, h->phi, h->cells * sizeof(double), cudaMemcpyDeviceToHost, h->st));
        } else {
            FLIC_CK(h, convert_out<float>(reinterpret_cast<const float*>(h->phi), h->staging, h->cells, h->st));
            FLIC_CK(h, cudaMemcpyAsync(phi_out, h->staging, h->cells * sizeof(double), cudaMemcpyDeviceToHost, h->st));
        }
    }
    FLIC_CK(h, cudaStreamSynchronize(h->st));
    return FLIC_OK;
}

int flic_step_diagnostics(flic_handle* h, flic_diag* out) {
    if (!h || !out) return FLIC_ERR_INVALID_ARG;
    FLIC_CK(h, cudaMemcpyAsync(h->diag_host, h->diag_dev, sizeof(flic_diag), cudaMemcpyDeviceToHost, h->st));
    FLIC_CK(h, cudaStreamSynchronize(h->st));
    *out = h->diag_host[0];
    return FLIC_OK;
}

int flic_diagnostics(flic_handle* h, flic_diag* out) {
    if (!h || !out) return FLIC_ERR_INVALID_ARG;
    int rc = h->fp64 ? enqueue_poisson<double>(h) : enqueue_poisson<float>(h);
    if (rc) return rc;
    rc = h->fp64 ? enqueue_state_check<double>(h, h->scal + S_VMAX_NEXT)
                 : enqueue_state_check<float>(h, h->scal + S_VMAX_NEXT);
    if (rc) return rc;
    FLIC_CK(h, step_finalize(h->part_diag, h->nb_diag, nullptr, 0, h->h * h->h * h->h, h->scal, h->status,
                             h->diag_dev + 1, 0, h->level1, 0, h->st));
    FLIC_CK(h, cudaMemcpyAsync(h->diag_host, h->diag_dev, 2 * sizeof(flic_diag), cudaMemcpyDeviceToHost, h->st));
    FLIC_CK(h, cudaStreamSynchronize(h->st));
    *out = h->diag_host[1];
    out->step = h->diag_host[0].step;
    return FLIC_OK;
}

int flic_num_tile_configs(flic_handle* h, int* n_gas, int* n_bme) {
    if (!h || !n_gas || !n_bme) return FLIC_ERR_INVALID_ARG;
    if (h->fp64) {
        stencil_cands<double>(FLUID_GAS, n_gas);
        stencil_cands<double>(FLUID_BME, n_bme);
    } else {
        stencil_cands<float>(FLUID_GAS, n_gas);
        stencil_cands<float>(FLUID_BME, n_bme);
    }
    return FLIC_OK;
}

int flic_set_tile_config(flic_handle* h, int gas, int bme) {
    if (!h) return FLIC_ERR_INVALID_ARG;
    return h->fp64 ? apply_tile_config<double>(h, gas, bme) : apply_tile_config<float>(h, gas, bme);
}

int flic_tile_config(flic_handle* h, int* gas, int* bme, char* text, int len) {
    if (!h) return FLIC_ERR_INVALID_ARG;
    if (gas) *gas = h->gcfg.cand;
    if (bme) *bme = h->bcfg.cand;
    if (text && len > 0) {
        int ng = 0, nb = 0;
        const char* gn = h->fp64 ? stencil_cands<double>(FLUID_GAS, &ng)[h->gcfg.cand].name
                                 : stencil_cands<float>(FLUID_GAS, &ng)[h->gcfg.cand].name;
        const char* bn = h->fp64 ? stencil_cands<double>(FLUID_BME, &nb)[h->bcfg.cand].name
                                 : stencil_cands<float>(FLUID_BME, &nb)[h->bcfg.cand].name;
        char gs[128], bs[128];
        auto split_text = [](char* out, size_t n, const StepCfg& c) {
            if (c.balanced > 0 && c.ztop > 0)
                snprintf(out, n, "balanced split over %d blocks (planes 0-%d of each tile column in lockstep, "
                         "the tops shared)", c.balanced, c.ztop - 1);
            else if (c.balanced > 0)
                snprintf(out, n, "balanced split over %d blocks (%d part%s per tile column)", c.balanced, c.zparts,
                         c.zparts > 1 ? "s" : "");
            else snprintf(out, n, "z chunks of %d planes", c.tz);
        };
        split_text(gs, sizeof gs, h->gcfg);
        split_text(bs, sizeof bs, h->bcfg);
        snprintf(text, size_t(len), "gas: %s, %s; moments: %s, %s", gn, gs, bn, bs);
    }
    return FLIC_OK;
}

int flic_autotune(flic_handle* h, int reps, int use_cache, double* ms) {
    if (!h || reps < 1) return FLIC_ERR_INVALID_ARG;
    const TuneKey key = tune_key(h);
    if (use_cache) {
        std::pair<int, int> hit(-1, -1);
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) hit = it->second;
        }
        if (hit.first >= 0) {
            const int rc = flic_set_tile_config(h, hit.first, hit.second);
            return rc ? rc : 1;
        }
    }
    const int rc = h->fp64 ? tune_impl<double>(h, reps, ms) : tune_impl<float>(h, reps, ms);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = std::make_pair(h->gcfg.cand, h->bcfg.cand);
    return 0;
}

int flic_sync(flic_handle* h) {
    if (!h) return FLIC_ERR_INVALID_ARG;
    FLIC_CK(h, cudaStreamSynchronize(h->st));
    return FLIC_OK;
}

int flic_destroy(flic_handle* h) {
    if (!h) return FLIC_ERR_INVALID_ARG;
    cudaStreamSynchronize(h->st);
    free_all(h);
    delete h;
    return FLIC_OK;
}

const char* flic_last_error(flic_handle* h) {
    return h ? h->err.c_str() : g_init_err.c_str();
}

const char* flic_version(void) {
    return "libflic 0.2 (sm_103a; two-fluid FlIC/Godunov step, FFT Poisson, launch-shape tuner)";
}

}  // extern "C"
