// C ABI of libflic: handle, device memory, one step as a launch sequence or a
// CUDA-graph replay, state transfer and diagnostics.  See include/flic.h.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

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
    StencilArgs<T> a;
    a.phi = reinterpret_cast<const T*>(h->phi);
    a.fs = h->fs;
    a.n = h->N;
    a.outflow = h->d.hydro_bc == FLIC_HYDRO_OUTFLOW;
    a.tau = h->scal + S_TAU;
    a.inv_h = 1.0 / h->h;
    a.gamma = T(h->d.gamma);
    a.eta = T(h->d.eta);
    a.vmax = h->scal + S_VMAX_NEXT;
    a.status = h->status;
    // gas: fields 0..5
    a.in = field_ptr<T>(h->state[h->cur], h->fs, F_RHO);
    a.out = field_ptr<T>(h->state[1 - h->cur], h->fs, F_RHO);
    a.tz = h->gcfg.tz;
    a.tiles_x = h->gcfg.tiles_x;
    a.tiles_y = h->gcfg.tiles_y;
    a.partials = h->part_gas;
    FLIC_CK(h, launch_gas<T>(a, h->gcfg, h->st));
    if (ev) FLIC_CK(h, cudaEventRecord(ev[2], h->st));
    // moments: fields 6..21
    a.in = field_ptr<T>(h->state[h->cur], h->fs, F_N);
    a.out = field_ptr<T>(h->state[1 - h->cur], h->fs, F_N);
    a.tz = h->bcfg.tz;
    a.tiles_x = h->bcfg.tiles_x;
    a.tiles_y = h->bcfg.tiles_y;
    a.partials = h->part_bme;
    FLIC_CK(h, launch_bme<T>(a, h->bcfg, h->st));
    if (ev) FLIC_CK(h, cudaEventRecord(ev[3], h->st));
    FLIC_CK(h, step_finalize(h->part_gas, h->gcfg.num_blocks(), h->part_bme, h->bcfg.num_blocks(),
                             h->h * h->h * h->h, h->scal, h->status, h->diag_dev, 1, h->level1, h->st));
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
                    h->part_diag, h->level1, h->diag_dev, h->staging};
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
    h->gcfg = gas_cfg<T>(N, 0);
    h->bcfg = bme_cfg<T>(N, 0);
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
    const size_t pg = size_t(h->gcfg.num_blocks()) * Q_COUNT, pb = size_t(h->bcfg.num_blocks()) * Q_COUNT;
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
    FLIC_CK(h, cudaStreamSynchronize(h->st));
    return FLIC_OK;
}

extern "C" {

int flic_init_grid(const flic_grid_desc* desc, void* stream, flic_handle** out) {
    if (!desc || !out) { g_init_err = "null argument"; return FLIC_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!valid_n(desc->n)) { g_init_err = "n must be 2^a 3^b, a multiple of 4, 8 <= n <= 1024"; return FLIC_ERR_INVALID_ARG; }
    if (!(desc->box_max > desc->box_min) || !(desc->gamma > 1.0) || !(desc->courant > 0.0) ||
        !(desc->eta >= 0.0) || !(desc->G >= 0.0)) {
        g_init_err = "invalid physical constants";
        return FLIC_ERR_INVALID_ARG;
    }
    if (desc->precision != FLIC_FP64 && desc->precision != FLIC_MIXED) { g_init_err = "unknown precision"; return FLIC_ERR_INVALID_ARG; }
    if (desc->poisson_bc != FLIC_PERIODIC && desc->poisson_bc != FLIC_ISOLATED) { g_init_err = "unknown Poisson boundary"; return FLIC_ERR_INVALID_ARG; }
    if (desc->hydro_bc != FLIC_HYDRO_PERIODIC && desc->hydro_bc != FLIC_HYDRO_OUTFLOW) { g_init_err = "unknown hydro boundary"; return FLIC_ERR_INVALID_ARG; }
    flic_handle* h = new flic_handle();
    h->d = *desc;
    h->N = desc->n;
    h->h = (desc->box_max - desc->box_min) / desc->n;
    h->fp64 = desc->precision == FLIC_FP64;
    h->iso = desc->poisson_bc == FLIC_ISOLATED;
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
    // step setup, five FFT passes (none without gravity), two fluid kernels, two-level reduction
    return 1 + (h->d.G != 0.0 ? 5 : 0) + 2 + 2;
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
                             h->diag_dev + 1, 0, h->level1, h->st));
    FLIC_CK(h, cudaMemcpyAsync(h->diag_host, h->diag_dev, 2 * sizeof(flic_diag), cudaMemcpyDeviceToHost, h->st));
    FLIC_CK(h, cudaStreamSynchronize(h->st));
    *out = h->diag_host[1];
    out->step = h->diag_host[0].step;
    return FLIC_OK;
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
    return "libflic 0.1 (sm_103a; two-fluid FlIC/Godunov step, FFT Poisson)";
}

}  // extern "C"
