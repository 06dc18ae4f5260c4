// Batched ensemble of independent runs (uneven grid sizes) advanced together.
//
// Runs of equal N form a size class whose states, potentials and spectra are
// contiguous (one run stride), so each FFT pass of a class is one launch over
// all its runs.  Each fluid stage is ONE launch over a work list spanning every
// run's (tile, z chunk) items, the per-run arguments coming from a device table;
// step setup and the two-level reduction are one launch each for all runs.  A
// step is captured once per state parity as a CUDA graph and replayed.
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "flic_fft.h"
#include "flic_internal.h"

using namespace flic;

namespace {

struct EnsClass {
    int N = 0;
    double h = 0.0;
    std::vector<int> runs;        // run ids in slot order
    size_t fs = 0;                // field stride
    size_t run_stride = 0;        // elements between runs' states (22 fields)
    size_t spec_stride = 0;       // complex elements between runs' spectra
    void* state[2] = {nullptr, nullptr};
    void* phi = nullptr;
    void* spec = nullptr;
    void* tw = nullptr;
    int tw_len = 0;
    void* asin2 = nullptr;
    void* gtab = nullptr;
    FftPlans plans;
    StepCfg gcfg, bcfg;
};

}  // namespace

struct flic_ensemble {
    flic_grid_desc d;             // shared constants (n unused)
    bool fp64 = true, iso = false;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int nruns = 0;
    std::vector<int> run_n, run_class, run_slot;
    std::vector<EnsClass> classes;
    // per-run device records
    double* scal = nullptr;              // [nruns][S_COUNT]
    unsigned int* status = nullptr;      // [nruns]
    flic_diag* diag = nullptr;           // [nruns]
    flic_diag* diag_host = nullptr;      // pinned [nruns]
    double* level1 = nullptr;            // [nruns][FINALIZE_ROWS][Q_COUNT]
    double* part_gas = nullptr;
    double* part_bme = nullptr;
    double* part_diag = nullptr;
    int nb_diag = 0;
    // device tables
    void* tab_gas[2] = {nullptr, nullptr};   // StencilArgs<T>[nruns], per parity
    void* tab_bme[2] = {nullptr, nullptr};
    WorkItem* work_gas = nullptr;
    WorkItem* work_bme = nullptr;
    int nwork_gas = 0, nwork_bme = 0;
    RunScalars* prep_tab = nullptr;
    FinalizeArgs* fin_tab = nullptr;
    // launch shapes of the fluid kernels (candidate index, z-chunk height cap)
    int cand[2] = {0, 0};
    int tz[2] = {32, 32};
    double* staging = nullptr;
    int cur = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    double graph_dt[2] = {0.0, 0.0};
    std::string err;
};

#define ENS_CK(e, call)                                                                      \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            (e)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                  \
            return (e_ == cudaErrorMemoryAllocation) ? FLIC_ERR_OOM : FLIC_ERR_CUDA;         \
        }                                                                                    \
    } while (0)

namespace {

// Potentials of every run's current state (one set of FFT passes per size class).
template <typename T>
int ens_enqueue_poisson(flic_ensemble* e) {
    if (e->d.G != 0.0) {
        for (auto& c : e->classes) {
            const T* s = reinterpret_cast<const T*>(c.state[e->cur]);
            const int nb = int(c.runs.size());
            if (e->iso) {
                ENS_CK(e, poisson_isolated<T>(s + F_RHO * c.fs, s + F_N * c.fs, reinterpret_cast<T*>(c.phi), c.spec,
                                              c.N, c.tw, reinterpret_cast<const T*>(c.gtab), e->st, nb,
                                              c.run_stride, c.fs, c.spec_stride));
            } else {
                ENS_CK(e, poisson_periodic<T>(s + F_RHO * c.fs, s + F_N * c.fs, reinterpret_cast<T*>(c.phi), c.spec,
                                              c.N, c.plans, c.tw, c.tw_len, reinterpret_cast<const T*>(c.asin2),
                                              e->d.G * c.h * c.h, e->st, nb, c.run_stride, c.fs, c.spec_stride));
            }
        }
    }
    return FLIC_OK;
}

template <typename T>
int ens_enqueue_step(flic_ensemble* e, double dt, cudaEvent_t* ev = nullptr) {
    if (ev) ENS_CK(e, cudaEventRecord(ev[0], e->st));
    ENS_CK(e, step_prep_batch(e->prep_tab, e->nruns, dt, e->st));
    const int prc = ens_enqueue_poisson<T>(e);
    if (prc) return prc;
    if (ev) ENS_CK(e, cudaEventRecord(ev[1], e->st));
    ENS_CK(e, stencil_launch_batch<T>(FLUID_GAS, e->cand[FLUID_GAS],
                                      reinterpret_cast<const StencilArgs<T>*>(e->tab_gas[e->cur]), e->work_gas,
                                      e->nwork_gas, e->d.hydro_bc == FLIC_HYDRO_OUTFLOW, e->d.cooling != 0.0,
                                      e->st));
    if (ev) ENS_CK(e, cudaEventRecord(ev[2], e->st));
    ENS_CK(e, stencil_launch_batch<T>(FLUID_BME, e->cand[FLUID_BME],
                                      reinterpret_cast<const StencilArgs<T>*>(e->tab_bme[e->cur]), e->work_bme,
                                      e->nwork_bme, e->d.hydro_bc == FLIC_HYDRO_OUTFLOW, false, e->st));
    if (ev) ENS_CK(e, cudaEventRecord(ev[3], e->st));
    ENS_CK(e, step_finalize_batch(e->fin_tab, e->nruns, 1, e->fp64 ? 0 : 1, e->st));
    if (ev) ENS_CK(e, cudaEventRecord(ev[4], e->st));
    e->cur = 1 - e->cur;
    return FLIC_OK;
}

int ens_step(flic_ensemble* e, double dt, cudaEvent_t* ev = nullptr) {
    return e->fp64 ? ens_enqueue_step<double>(e, dt, ev) : ens_enqueue_step<float>(e, dt, ev);
}

void ens_free(flic_ensemble* e) {
    for (int i = 0; i < 2; ++i) {
        if (e->graph[i]) cudaGraphExecDestroy(e->graph[i]);
        if (e->tab_gas[i]) cudaFree(e->tab_gas[i]);
        if (e->tab_bme[i]) cudaFree(e->tab_bme[i]);
    }
    for (auto& c : e->classes) {
        void* bufs[] = {c.state[0], c.state[1], c.phi, c.spec, c.tw, c.asin2, c.gtab};
        for (void* b : bufs)
            if (b) cudaFree(b);
    }
    void* bufs[] = {e->scal, e->status, e->diag, e->level1, e->part_gas, e->part_bme, e->part_diag,
                    e->work_gas, e->work_bme, e->prep_tab, e->fin_tab, e->staging};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (e->diag_host) cudaFreeHost(e->diag_host);
    if (e->own_stream && e->st) cudaStreamDestroy(e->st);
}

// (Re)builds what depends on the fluid kernels' launch shapes: each size
// class's geometry, the work lists spanning all runs, the per-run partial rows
// and the argument tables (the graphs are dropped).
template <typename T>
int ens_build_work(flic_ensemble* e) {
    for (int i = 0; i < 2; ++i) {
        if (e->graph[i]) { cudaGraphExecDestroy(e->graph[i]); e->graph[i] = nullptr; }
        if (e->tab_gas[i]) { cudaFree(e->tab_gas[i]); e->tab_gas[i] = nullptr; }
        if (e->tab_bme[i]) { cudaFree(e->tab_bme[i]); e->tab_bme[i] = nullptr; }
    }
    void* old[] = {e->work_gas, e->work_bme, e->part_gas, e->part_bme, e->prep_tab, e->fin_tab};
    for (void* b : old)
        if (b) cudaFree(b);
    e->work_gas = e->work_bme = nullptr;
    e->part_gas = e->part_bme = nullptr;
    e->prep_tab = nullptr;
    e->fin_tab = nullptr;
    // (tile, z chunk) items: chunks of at most tz planes, so the work list of all
    // runs fills the GPU
    for (auto& c : e->classes) {
        c.gcfg = stencil_cfg<T>(FLUID_GAS, e->cand[FLUID_GAS], c.N, c.N < e->tz[FLUID_GAS] ? c.N : e->tz[FLUID_GAS]);
        c.bcfg = stencil_cfg<T>(FLUID_BME, e->cand[FLUID_BME], c.N, c.N < e->tz[FLUID_BME] ? c.N : e->tz[FLUID_BME]);
    }
    std::vector<int> goff(e->nruns), boff(e->nruns);
    std::vector<WorkItem> wg, wb;
    // work lists and partial rows
    int pg = 0, pb = 0;
    for (int r = 0; r < e->nruns; ++r) {
        const EnsClass& c = e->classes[e->run_class[r]];
        goff[r] = pg;
        boff[r] = pb;
        const int gt = c.gcfg.tiles_x * c.gcfg.tiles_y, bt = c.bcfg.tiles_x * c.bcfg.tiles_y;
        for (int ch = 0; ch < c.gcfg.blocks_z; ++ch)
            for (int t = 0; t < gt; ++t) wg.push_back(WorkItem{r, t, ch, ch * gt + t});
        for (int ch = 0; ch < c.bcfg.blocks_z; ++ch)
            for (int t = 0; t < bt; ++t) wb.push_back(WorkItem{r, t, ch, ch * bt + t});
        pg += c.gcfg.num_blocks();
        pb += c.bcfg.num_blocks();
    }
    e->nwork_gas = int(wg.size());
    e->nwork_bme = int(wb.size());
    ENS_CK(e, cudaMalloc(&e->work_gas, wg.size() * sizeof(WorkItem)));
    ENS_CK(e, cudaMalloc(&e->work_bme, wb.size() * sizeof(WorkItem)));
    ENS_CK(e, cudaMemcpy(e->work_gas, wg.data(), wg.size() * sizeof(WorkItem), cudaMemcpyHostToDevice));
    ENS_CK(e, cudaMemcpy(e->work_bme, wb.data(), wb.size() * sizeof(WorkItem), cudaMemcpyHostToDevice));
    ENS_CK(e, cudaMalloc(&e->part_gas, size_t(pg) * Q_COUNT * sizeof(double)));
    ENS_CK(e, cudaMalloc(&e->part_bme, size_t(pb) * Q_COUNT * sizeof(double)));
    ENS_CK(e, cudaMemsetAsync(e->part_gas, 0, size_t(pg) * Q_COUNT * sizeof(double), e->st));
    ENS_CK(e, cudaMemsetAsync(e->part_bme, 0, size_t(pb) * Q_COUNT * sizeof(double), e->st));
    // per-run argument tables
    std::vector<RunScalars> prep(e->nruns);
    std::vector<FinalizeArgs> fin(e->nruns);
    std::vector<StencilArgs<T>> tg[2], tb[2];
    for (int p = 0; p < 2; ++p) {
        tg[p].resize(e->nruns);
        tb[p].resize(e->nruns);
    }
    for (int r = 0; r < e->nruns; ++r) {
        const EnsClass& c = e->classes[e->run_class[r]];
        const int s = e->run_slot[r];
        double* sc = e->scal + size_t(r) * S_COUNT;
        prep[r] = RunScalars{sc, e->status + r, e->d.courant * c.h};
        fin[r] = FinalizeArgs{e->part_gas + size_t(goff[r]) * Q_COUNT, c.gcfg.num_blocks(),
                              e->part_bme + size_t(boff[r]) * Q_COUNT, c.bcfg.num_blocks(), c.h * c.h * c.h, sc,
                              e->status + r, e->diag + r, e->level1 + size_t(r) * FINALIZE_ROWS * Q_COUNT,
                              std::is_same<T, float>::value ? 1 : 0};
        for (int p = 0; p < 2; ++p) {
            const T* in = reinterpret_cast<const T*>(c.state[p]) + size_t(s) * c.run_stride;
            T* out = reinterpret_cast<T*>(c.state[1 - p]) + size_t(s) * c.run_stride;
            StencilArgs<T> a;
            a.phi = reinterpret_cast<const T*>(c.phi) + size_t(s) * c.fs;
            a.fs = c.fs;
            a.n = c.N;
            a.outflow = e->d.hydro_bc == FLIC_HYDRO_OUTFLOW;
            a.tau = sc + S_TAU;
            a.inv_h = 1.0 / c.h;
            a.gamma = T(e->d.gamma);
            a.eta = T(e->d.eta);
            a.cool = T(e->d.cooling);
            a.vmax = sc + S_VMAX_NEXT;
            a.status = e->status + r;
            a.zparts = 1;
            a.ztop = 0;
            StencilArgs<T> g = a, b = a;
            g.in = in + F_RHO * c.fs;
            g.out = out + F_RHO * c.fs;
            g.tz = c.gcfg.tz;
            g.tiles_x = c.gcfg.tiles_x;
            g.tiles_y = c.gcfg.tiles_y;
            g.partials = e->part_gas + size_t(goff[r]) * Q_COUNT;
            b.in = in + F_N * c.fs;
            b.out = out + F_N * c.fs;
            b.tz = c.bcfg.tz;
            b.tiles_x = c.bcfg.tiles_x;
            b.tiles_y = c.bcfg.tiles_y;
            b.partials = e->part_bme + size_t(boff[r]) * Q_COUNT;
            tg[p][r] = g;
            tb[p][r] = b;
        }
    }
    for (int p = 0; p < 2; ++p) {
        ENS_CK(e, cudaMalloc(&e->tab_gas[p], e->nruns * sizeof(StencilArgs<T>)));
        ENS_CK(e, cudaMalloc(&e->tab_bme[p], e->nruns * sizeof(StencilArgs<T>)));
        ENS_CK(e, cudaMemcpy(e->tab_gas[p], tg[p].data(), e->nruns * sizeof(StencilArgs<T>), cudaMemcpyHostToDevice));
        ENS_CK(e, cudaMemcpy(e->tab_bme[p], tb[p].data(), e->nruns * sizeof(StencilArgs<T>), cudaMemcpyHostToDevice));
    }
    ENS_CK(e, cudaMalloc(&e->prep_tab, e->nruns * sizeof(RunScalars)));
    ENS_CK(e, cudaMalloc(&e->fin_tab, e->nruns * sizeof(FinalizeArgs)));
    ENS_CK(e, cudaMemcpy(e->prep_tab, prep.data(), e->nruns * sizeof(RunScalars), cudaMemcpyHostToDevice));
    ENS_CK(e, cudaMemcpy(e->fin_tab, fin.data(), e->nruns * sizeof(FinalizeArgs), cudaMemcpyHostToDevice));
    ENS_CK(e, cudaStreamSynchronize(e->st));
    return FLIC_OK;
}

template <typename T>
int ens_init(flic_ensemble* e) {
    typedef typename std::conditional<sizeof(T) == 8, double2, float2>::type C;
    ENS_CK(e, stencil_prepare<T>());
    // size classes in order of first appearance
    for (int r = 0; r < e->nruns; ++r) {
        int ci = -1;
        for (size_t k = 0; k < e->classes.size(); ++k)
            if (e->classes[k].N == e->run_n[r]) ci = int(k);
        if (ci < 0) {
            EnsClass c;
            c.N = e->run_n[r];
            e->classes.push_back(c);
            ci = int(e->classes.size()) - 1;
        }
        e->run_class[r] = ci;
        e->run_slot[r] = int(e->classes[ci].runs.size());
        e->classes[ci].runs.push_back(r);
    }
    size_t max_cells = 0;
    // per-run partial-row offsets
    std::vector<int> goff(e->nruns), boff(e->nruns);
    std::vector<WorkItem> wg, wb;
    for (auto& c : e->classes) {
        const int N = c.N;
        if (fft_plan_init(N, &c.plans)) { e->err = "unsupported FFT length"; return FLIC_ERR_INVALID_ARG; }
        if (e->iso && !fft_iso_supported(N)) { e->err = "unsupported size for the isolated solve"; return FLIC_ERR_INVALID_ARG; }
        ENS_CK(e, fft_prepare<T>(N));
        if (e->iso) ENS_CK(e, fft_prepare_iso<T>(N));
        c.h = (e->d.box_max - e->d.box_min) / N;
        const size_t cells = size_t(N) * N * N;
        if (cells > max_cells) max_cells = cells;
        c.fs = (cells + 63) / 64 * 64;
        c.run_stride = F_COUNT * c.fs;
        const int nb = int(c.runs.size());
        const int L = e->iso ? 2 * N : N;
        c.spec_stride = size_t(N) * L * (L / 2 + 1);
        for (int i = 0; i < 2; ++i) {
            ENS_CK(e, cudaMalloc(&c.state[i], c.run_stride * nb * sizeof(T)));
            ENS_CK(e, cudaMemsetAsync(c.state[i], 0, c.run_stride * nb * sizeof(T), e->st));
        }
        ENS_CK(e, cudaMalloc(&c.phi, c.fs * nb * sizeof(T)));
        ENS_CK(e, cudaMemsetAsync(c.phi, 0, c.fs * nb * sizeof(T), e->st));
        ENS_CK(e, cudaMalloc(&c.spec, c.spec_stride * nb * sizeof(C)));
        c.tw_len = L;
        std::vector<C> tw(L);
        for (int j = 0; j < L; ++j) {
            const long double ang = 2.0L * 3.141592653589793238462643383279502884L * j / L;
            tw[j].x = T(std::cos(ang));
            tw[j].y = T(-std::sin(ang));
        }
        ENS_CK(e, cudaMalloc(&c.tw, L * sizeof(C)));
        ENS_CK(e, cudaMemcpy(c.tw, tw.data(), L * sizeof(C), cudaMemcpyHostToDevice));
        std::vector<T> a2(N);
        for (int k = 0; k < N; ++k) {
            const long double s = std::sin(3.141592653589793238462643383279502884L * k / N);
            a2[k] = T((2.0L / 3.0L) * s * s);
        }
        ENS_CK(e, cudaMalloc(&c.asin2, N * sizeof(T)));
        ENS_CK(e, cudaMemcpy(c.asin2, a2.data(), N * sizeof(T), cudaMemcpyHostToDevice));
        if (e->iso) {
            ENS_CK(e, cudaMalloc(&c.gtab, green_table_elems<T>(N) * sizeof(T)));
            void* greal = nullptr;
            void* gspec = nullptr;
            cudaError_t er = cudaMalloc(&greal, size_t(L) * L * L * sizeof(T));
            if (er == cudaSuccess) er = cudaMalloc(&gspec, size_t(L) * L * (L / 2 + 1) * sizeof(C));
            if (er == cudaSuccess)
                er = green_init<T>(N, c.h, e->d.G, reinterpret_cast<T*>(c.gtab), reinterpret_cast<T*>(greal), gspec,
                                   c.tw, e->st);
            if (er == cudaSuccess) er = cudaStreamSynchronize(e->st);
            if (greal) cudaFree(greal);
            if (gspec) cudaFree(gspec);
            ENS_CK(e, er);
        }
    }
    ENS_CK(e, cudaMalloc(&e->staging, max_cells * sizeof(double)));
    e->nb_diag = 152 * 4;
    ENS_CK(e, cudaMalloc(&e->part_diag, size_t(e->nb_diag) * Q_COUNT * sizeof(double)));
    ENS_CK(e, cudaMalloc(&e->scal, size_t(e->nruns) * S_COUNT * sizeof(double)));
    ENS_CK(e, cudaMemsetAsync(e->scal, 0, size_t(e->nruns) * S_COUNT * sizeof(double), e->st));
    ENS_CK(e, cudaMalloc(&e->status, size_t(e->nruns) * sizeof(unsigned int)));
    ENS_CK(e, cudaMemsetAsync(e->status, 0, size_t(e->nruns) * sizeof(unsigned int), e->st));
    ENS_CK(e, cudaMalloc(&e->diag, size_t(e->nruns) * sizeof(flic_diag)));
    ENS_CK(e, cudaMemsetAsync(e->diag, 0, size_t(e->nruns) * sizeof(flic_diag), e->st));
    ENS_CK(e, cudaMallocHost(&e->diag_host, size_t(e->nruns) * sizeof(flic_diag)));
    ENS_CK(e, cudaMalloc(&e->level1, size_t(e->nruns) * FINALIZE_ROWS * Q_COUNT * sizeof(double)));
    const int rc = ens_build_work<T>(e);
    if (rc) return rc;
    ENS_CK(e, cudaStreamSynchronize(e->st));
    return FLIC_OK;
}

// z-chunk height caps the ensemble tuner tries with every candidate shape
constexpr int ENS_TZ_OPTIONS[3] = {16, 32, 64};

// Times every (candidate shape, chunk cap) of both fluid kernels over the whole
// work list on the current states and keeps the fastest of each kernel.  The
// launches write the spare state buffers only.
template <typename T>
int ens_tune(flic_ensemble* e, int reps, double* ms) {
    ENS_CK(e, step_prep_batch(e->prep_tab, e->nruns, 0.0, e->st));
    int rc = ens_enqueue_poisson<T>(e);
    if (rc) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ENS_CK(e, cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        ENS_CK(e, ce);
    }
    int k = 0;
    int best_c[2] = {e->cand[0], e->cand[1]}, best_t[2] = {e->tz[0], e->tz[1]};
    for (int fluid = 0; fluid < 2 && rc == FLIC_OK; ++fluid) {
        int nc = 0;
        stencil_cands<T>(fluid, &nc);
        double best_ms = -1.0;
        const StencilCand<T>* cands = stencil_cands<T>(fluid, &nc);
        for (int c = 0; c < nc && rc == FLIC_OK; ++c) {
            // entries that differ only in the single-grid split are one compiled shape here
            bool seen = false;
            for (int c2 = 0; c2 < c; ++c2) seen = seen || cands[c2].launch_batch == cands[c].launch_batch;
            if (seen) {
                for (int t = 0; t < 3; ++t, ++k)
                    if (ms) ms[k] = -1.0;
                continue;
            }
            for (int t = 0; t < 3; ++t, ++k) {
                e->cand[fluid] = c;
                e->tz[fluid] = ENS_TZ_OPTIONS[t];
                rc = ens_build_work<T>(e);
                if (rc) break;
                const bool gas = fluid == FLUID_GAS;
                const StencilArgs<T>* tab = reinterpret_cast<const StencilArgs<T>*>(gas ? e->tab_gas[e->cur]
                                                                                          : e->tab_bme[e->cur]);
                const WorkItem* work = gas ? e->work_gas : e->work_bme;
                const int nwork = gas ? e->nwork_gas : e->nwork_bme;
                const bool out = e->d.hydro_bc == FLIC_HYDRO_OUTFLOW;
                const bool cool = gas && e->d.cooling != 0.0;
                cudaError_t er = stencil_launch_batch<T>(fluid, c, tab, work, nwork, out, cool, e->st);
                if (er == cudaSuccess) er = cudaEventRecord(e0, e->st);
                for (int r = 0; r < reps && er == cudaSuccess; ++r)
                    er = stencil_launch_batch<T>(fluid, c, tab, work, nwork, out, cool, e->st);
                if (er == cudaSuccess) er = cudaEventRecord(e1, e->st);
                if (er == cudaSuccess) er = cudaEventSynchronize(e1);
                float el = 0.f;
                if (er == cudaSuccess) er = cudaEventElapsedTime(&el, e0, e1);
                double tm = -1.0;
                if (er == cudaSuccess) {
                    tm = double(el) / reps;
                } else if (er == cudaErrorInvalidConfiguration || er == cudaErrorLaunchOutOfResources ||
                           er == cudaErrorInvalidValue) {
                    cudaGetLastError();   // a shape this device cannot launch: skipped
                } else {
                    e->err = std::string("launch-shape tuning: ") + cudaGetErrorString(er);
                    rc = FLIC_ERR_CUDA;
                    break;
                }
                if (ms) ms[k] = tm;
                if (tm >= 0.0 && (best_ms < 0.0 || tm < best_ms * (1.0 - TUNE_MARGIN))) {
                    best_ms = tm;
                    best_c[fluid] = c;
                    best_t[fluid] = ENS_TZ_OPTIONS[t];
                }
            }
        }
        e->cand[fluid] = best_c[fluid];
        e->tz[fluid] = best_t[fluid];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    return ens_build_work<T>(e);
}

template <typename T>
int ens_set_state(flic_ensemble* e, int r, const double* const* fields) {
    EnsClass& c = e->classes[e->run_class[r]];
    const size_t cells = size_t(c.N) * c.N * c.N;
    T* base = reinterpret_cast<T*>(c.state[e->cur]) + size_t(e->run_slot[r]) * c.run_stride;
    for (int f = 0; f < F_COUNT; ++f) {
        if (!fields[f]) { e->err = "null field pointer"; return FLIC_ERR_INVALID_ARG; }
        const double* src = static_cast<const double*>(mapped_device_view(fields[f]));
        if (!src) {
            ENS_CK(e, cudaMemcpyAsync(e->staging, fields[f], cells * sizeof(double), cudaMemcpyHostToDevice, e->st));
            src = e->staging;
        }
        ENS_CK(e, convert_in<T>(src, base + size_t(f) * c.fs, cells, e->st));
    }
    double* sc = e->scal + size_t(r) * S_COUNT;
    ENS_CK(e, cudaMemsetAsync(sc, 0, S_COUNT * sizeof(double), e->st));
    ENS_CK(e, cudaMemsetAsync(e->status + r, 0, sizeof(unsigned int), e->st));
    ENS_CK(e, cudaMemsetAsync(e->diag + r, 0, sizeof(flic_diag), e->st));
    ENS_CK(e, state_reduce<T>(base, c.fs, reinterpret_cast<const T*>(c.phi) + size_t(e->run_slot[r]) * c.fs, cells,
                              e->d.gamma, e->part_diag, e->nb_diag, sc + S_VMAX_CUR, e->status + r, e->st));
    unsigned int s = 0;
    ENS_CK(e, cudaMemcpyAsync(&s, e->status + r, sizeof(s), cudaMemcpyDeviceToHost, e->st));
    ENS_CK(e, cudaStreamSynchronize(e->st));
    if (s & ST_NONPHYSICAL) {
        e->err = "state has a non-positive density, internal energy or diagonal stress, or a non-finite value";
        return FLIC_ERR_NONPHYSICAL;
    }
    return FLIC_OK;
}

template <typename T>
int ens_get_state(flic_ensemble* e, int r, double* const* fields) {
    EnsClass& c = e->classes[e->run_class[r]];
    const size_t cells = size_t(c.N) * c.N * c.N;
    const T* base = reinterpret_cast<const T*>(c.state[e->cur]) + size_t(e->run_slot[r]) * c.run_stride;
    for (int f = 0; f < F_COUNT; ++f) {
        if (!fields[f]) { e->err = "null field pointer"; return FLIC_ERR_INVALID_ARG; }
        double* view = static_cast<double*>(const_cast<void*>(mapped_device_view(fields[f])));
        if (view) {
            ENS_CK(e, convert_out<T>(base + size_t(f) * c.fs, view, cells, e->st));
        } else {
            ENS_CK(e, convert_out<T>(base + size_t(f) * c.fs, e->staging, cells, e->st));
            ENS_CK(e, cudaMemcpyAsync(fields[f], e->staging, cells * sizeof(double), cudaMemcpyDeviceToHost,
                                      e->st));
        }
    }
    ENS_CK(e, cudaStreamSynchronize(e->st));
    return FLIC_OK;
}

}  // namespace

extern "C" {

int flic_ensemble_create(const flic_grid_desc* descs, int nruns, void* stream, flic_ensemble** out) {
    if (!descs || !out || nruns < 1) { set_global_error("null argument or nruns < 1"); return FLIC_ERR_INVALID_ARG; }
    *out = nullptr;
    const flic_grid_desc& d0 = descs[0];
    for (int r = 0; r < nruns; ++r) {
        const flic_grid_desc& d = descs[r];
        if (d.precision != d0.precision || d.poisson_bc != d0.poisson_bc || d.hydro_bc != d0.hydro_bc ||
            d.gamma != d0.gamma || d.G != d0.G ||
            d.courant != d0.courant || d.eta != d0.eta || d.box_min != d0.box_min || d.box_max != d0.box_max ||
            d.cooling != d0.cooling || d.flux_reading != d0.flux_reading) {
            set_global_error("ensemble runs must share every constant except n");
            return FLIC_ERR_INVALID_ARG;
        }
        int m = d.n;
        while (m % 2 == 0 && m > 0) m /= 2;
        while (m % 3 == 0 && m > 0) m /= 3;
        if (d.n < 8 || d.n > 512 || m != 1 || d.n % 4) {
            set_global_error("ensemble run sizes must be 2^a 3^b, multiples of 4, 8..512");
            return FLIC_ERR_INVALID_ARG;
        }
    }
    if (!(d0.box_max > d0.box_min) || !(d0.gamma > 1.0) || !(d0.courant > 0.0) || !(d0.G >= 0.0) ||
        !(d0.cooling >= 0.0) || d0.flux_reading != FLIC_FLUX_A ||
        (d0.precision != FLIC_FP64 && d0.precision != FLIC_MIXED) ||
        (d0.poisson_bc != FLIC_PERIODIC && d0.poisson_bc != FLIC_ISOLATED) ||
        (d0.hydro_bc != FLIC_HYDRO_PERIODIC && d0.hydro_bc != FLIC_HYDRO_OUTFLOW)) {
        set_global_error("invalid ensemble constants");
        return FLIC_ERR_INVALID_ARG;
    }
    flic_ensemble* e = new flic_ensemble();
    e->d = d0;
    e->fp64 = d0.precision == FLIC_FP64;
    e->iso = d0.poisson_bc == FLIC_ISOLATED;
    e->nruns = nruns;
    e->run_n.resize(nruns);
    e->run_class.resize(nruns);
    e->run_slot.resize(nruns);
    for (int r = 0; r < nruns; ++r) e->run_n[r] = descs[r].n;
    if (stream) {
        e->st = reinterpret_cast<cudaStream_t>(stream);
    } else {
        cudaError_t er = cudaStreamCreateWithFlags(&e->st, cudaStreamNonBlocking);
        if (er != cudaSuccess) { set_global_error(cudaGetErrorString(er)); delete e; return FLIC_ERR_CUDA; }
        e->own_stream = true;
    }
    int rc = e->fp64 ? ens_init<double>(e) : ens_init<float>(e);
    if (rc) {
        set_global_error(e->err.c_str());
        ens_free(e);
        delete e;
        return rc;
    }
    *out = e;
    return FLIC_OK;
}

int flic_ensemble_set_state(flic_ensemble* e, int run, const double* const fields[FLIC_NFIELDS]) {
    if (!e || !fields || run < 0 || run >= e->nruns) return FLIC_ERR_INVALID_ARG;
    return e->fp64 ? ens_set_state<double>(e, run, fields) : ens_set_state<float>(e, run, fields);
}

int flic_ensemble_get_state(flic_ensemble* e, int run, double* const fields[FLIC_NFIELDS]) {
    if (!e || !fields || run < 0 || run >= e->nruns) return FLIC_ERR_INVALID_ARG;
    return e->fp64 ? ens_get_state<double>(e, run, fields) : ens_get_state<float>(e, run, fields);
}

int flic_ensemble_step(flic_ensemble* e, int nsteps, double dt, int sync) {
    if (!e || nsteps < 0) return FLIC_ERR_INVALID_ARG;
    for (int s = 0; s < nsteps; ++s) {
        const int c = e->cur;
        if (!e->graph[c] || e->graph_dt[c] != dt) {
            if (e->graph[c]) { cudaGraphExecDestroy(e->graph[c]); e->graph[c] = nullptr; }
            cudaGraph_t g = nullptr;
            ENS_CK(e, cudaStreamBeginCapture(e->st, cudaStreamCaptureModeThreadLocal));
            int rc = ens_step(e, dt);
            cudaError_t er = cudaStreamEndCapture(e->st, &g);
            e->cur = c;
            if (rc) { if (g) cudaGraphDestroy(g); return rc; }
            if (er != cudaSuccess) { e->err = std::string("graph capture: ") + cudaGetErrorString(er); return FLIC_ERR_CUDA; }
            er = cudaGraphInstantiate(&e->graph[c], g, 0);
            cudaGraphDestroy(g);
            if (er != cudaSuccess) { e->err = std::string("graph instantiate: ") + cudaGetErrorString(er); return FLIC_ERR_CUDA; }
            e->graph_dt[c] = dt;
        }
        ENS_CK(e, cudaGraphLaunch(e->graph[c], e->st));
        e->cur = 1 - c;
    }
    if (sync) {
        ENS_CK(e, cudaMemcpyAsync(e->diag_host, e->diag, size_t(e->nruns) * sizeof(flic_diag), cudaMemcpyDeviceToHost,
                                  e->st));
        ENS_CK(e, cudaStreamSynchronize(e->st));
        for (int r = 0; r < e->nruns && nsteps > 0; ++r)
            if (e->diag_host[r].status != FLIC_OK) {
                e->err = "a run produced a non-physical state";
                return FLIC_ERR_NONPHYSICAL;
            }
    }
    return FLIC_OK;
}

int flic_ensemble_diagnostics(flic_ensemble* e, int run, flic_diag* out) {
    if (!e || !out || run < 0 || run >= e->nruns) return FLIC_ERR_INVALID_ARG;
    ENS_CK(e, cudaMemcpyAsync(out, e->diag + run, sizeof(flic_diag), cudaMemcpyDeviceToHost, e->st));
    ENS_CK(e, cudaStreamSynchronize(e->st));
    return FLIC_OK;
}

int flic_ensemble_profile(flic_ensemble* e, int nsteps, double dt, double stage_ms[FLIC_NSTAGES],
                          double* total_ms) {
    if (!e || nsteps <= 0 || !stage_ms) return FLIC_ERR_INVALID_ARG;
    const int ne = 5 * nsteps;
    std::vector<cudaEvent_t> ev(ne);
    int made = 0, rc = FLIC_OK;
    for (; made < ne; ++made) {
        cudaError_t er = cudaEventCreate(&ev[made]);
        if (er != cudaSuccess) { e->err = cudaGetErrorString(er); rc = FLIC_ERR_CUDA; break; }
    }
    for (int s = 0; rc == FLIC_OK && s < nsteps; ++s) rc = ens_step(e, dt, ev.data() + 5 * s);
    if (rc == FLIC_OK) {
        cudaError_t er = cudaEventSynchronize(ev[ne - 1]);
        if (er != cudaSuccess) { e->err = cudaGetErrorString(er); rc = FLIC_ERR_CUDA; }
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
    return rc;
}

int flic_ensemble_launches_per_step(flic_ensemble* e) {
    if (!e) return FLIC_ERR_INVALID_ARG;
    // setup, five FFT passes per size class, two fluid launches, the reduction (one
    // launch over float32 pairs; two levels in float64)
    return 1 + (e->d.G != 0.0 ? 5 * int(e->classes.size()) : 0) + 2 + (e->fp64 ? 2 : 1);
}

int flic_ensemble_autotune(flic_ensemble* e, int reps, double* ms) {
    if (!e || reps < 1) return FLIC_ERR_INVALID_ARG;
    return e->fp64 ? ens_tune<double>(e, reps, ms) : ens_tune<float>(e, reps, ms);
}

int flic_ensemble_num_tile_configs(flic_ensemble* e, int* n_gas, int* n_bme) {
    if (!e || !n_gas || !n_bme) return FLIC_ERR_INVALID_ARG;
    if (e->fp64) {
        stencil_cands<double>(FLUID_GAS, n_gas);
        stencil_cands<double>(FLUID_BME, n_bme);
    } else {
        stencil_cands<float>(FLUID_GAS, n_gas);
        stencil_cands<float>(FLUID_BME, n_bme);
    }
    return FLIC_OK;
}

int flic_ensemble_set_tile_config(flic_ensemble* e, int gas, int bme, int tz_gas, int tz_bme) {
    if (!e) return FLIC_ERR_INVALID_ARG;
    int ng = 0, nb = 0;
    if (e->fp64) {
        stencil_cands<double>(FLUID_GAS, &ng);
        stencil_cands<double>(FLUID_BME, &nb);
    } else {
        stencil_cands<float>(FLUID_GAS, &ng);
        stencil_cands<float>(FLUID_BME, &nb);
    }
    if (gas < -1 || gas >= ng || bme < -1 || bme >= nb || tz_gas == 0 || tz_bme == 0 || tz_gas < -1 ||
        tz_bme < -1) {
        e->err = "launch shape index or chunk height out of range";
        return FLIC_ERR_INVALID_ARG;
    }
    if (gas >= 0) e->cand[FLUID_GAS] = gas;
    if (bme >= 0) e->cand[FLUID_BME] = bme;
    if (tz_gas > 0) e->tz[FLUID_GAS] = tz_gas;
    if (tz_bme > 0) e->tz[FLUID_BME] = tz_bme;
    ENS_CK(e, cudaStreamSynchronize(e->st));
    return e->fp64 ? ens_build_work<double>(e) : ens_build_work<float>(e);
}

int flic_ensemble_tile_config(flic_ensemble* e, int* gas, int* bme, int* tz_gas, int* tz_bme, char* text, int len) {
    if (!e) return FLIC_ERR_INVALID_ARG;
    if (gas) *gas = e->cand[FLUID_GAS];
    if (bme) *bme = e->cand[FLUID_BME];
    if (tz_gas) *tz_gas = e->tz[FLUID_GAS];
    if (tz_bme) *tz_bme = e->tz[FLUID_BME];
    if (text && len > 0) {
        int n = 0;
        const char* gn = e->fp64 ? stencil_cands<double>(FLUID_GAS, &n)[e->cand[FLUID_GAS]].name
                                 : stencil_cands<float>(FLUID_GAS, &n)[e->cand[FLUID_GAS]].name;
        const char* bn = e->fp64 ? stencil_cands<double>(FLUID_BME, &n)[e->cand[FLUID_BME]].name
                                 : stencil_cands<float>(FLUID_BME, &n)[e->cand[FLUID_BME]].name;
        snprintf(text, size_t(len), "gas: %s, work items of at most %d planes; moments: %s, work items of at most %d planes",
                 gn, e->tz[FLUID_GAS], bn, e->tz[FLUID_BME]);
    }
    return FLIC_OK;
}

int flic_ensemble_destroy(flic_ensemble* e) {
    if (!e) return FLIC_ERR_INVALID_ARG;
    cudaStreamSynchronize(e->st);
    ens_free(e);
    delete e;
    return FLIC_OK;
}

const char* flic_ensemble_last_error(flic_ensemble* e) { return e ? e->err.c_str() : "null ensemble"; }

}  // extern "C"
