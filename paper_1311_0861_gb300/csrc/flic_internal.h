// Declarations shared by the translation units of libflic.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "flic.h"
#include "flic_stencil.cuh"

namespace flic {

// Launch geometry of one fluid kernel: the compiled launch shape (index into
// the fluid's candidate table), tiles of TX x TY columns, z chunks of tz planes.
struct StepCfg {
    int cand = 0;
    int tx = 0, ty = 0;   // tile shape
    int tiles_x = 0, tiles_y = 0;
    int tz = 0, blocks_z = 0;   // tz = 0: balanced split over `balanced` blocks
    int balanced = 0;
    int zparts = 1;       // balanced split: parts per tile column
    int ztop = 0;         // balanced split with tops: height of the lockstep part (0: off)
    int threads = 0;
    size_t smem = 0;
    int num_blocks() const { return balanced > 0 ? balanced : tiles_x * tiles_y * blocks_z; }
};

enum Fluid { FLUID_GAS = 0, FLUID_BME = 1 };
// The tuners keep an earlier (lower-index) candidate unless a later one is faster
// by more than this fraction: shapes that launch identically or time the same
// within noise resolve to the same, reproducible choice (entry 0 the default).
constexpr double TUNE_MARGIN = 0.005;
// How a single grid's z planes are split over blocks (a batched ensemble always
// uses (tile, chunk) work items): a (tile, z chunk) grid; a balanced split over
// one block per resident slot whose units are tile columns cut into parts when
// there are fewer tiles than blocks; the same with whole tile columns only; with
// fewer tiles than blocks, one block per tile column marching planes [0, H) in
// lockstep and the other blocks sharing the tops [H, N) of all columns.
enum Split { SPLIT_CHUNK = 0, SPLIT_BALANCED = 1, SPLIT_BALANCED_WHOLE = 2, SPLIT_TOPS = 3 };

// One compiled launch shape of a fluid kernel (tile, threads, occupancy, staging)
// together with the z split it is used with on a single grid: an entry of the
// candidate table that the launch-shape tuner times.  Entry 0 of each table is
// the default.
template <typename T>
struct StencilCand {
    const char* name;
    int split;
    StepCfg (*cfg)(int N, int tz, int split);
    cudaError_t (*prepare)();
    cudaError_t (*launch)(const StencilArgs<T>& a, const StepCfg& c, cudaStream_t st);
    cudaError_t (*launch_batch)(const StencilArgs<T>* table, const WorkItem* work, int nwork, bool outflow,
                                bool cool, cudaStream_t st);
};
template <typename T> const StencilCand<T>* gas_cands(int* count);
template <typename T> const StencilCand<T>* bme_cands(int* count);
template <typename T> const StencilCand<T>* stencil_cands(int fluid, int* count) {
    return fluid == FLUID_GAS ? gas_cands<T>(count) : bme_cands<T>(count);
}

template <typename T> cudaError_t stencil_prepare();   // shared-memory limits of every candidate, once
// Geometry of candidate `cand` on an N^3 grid; tz > 0 forces (tile, chunk) work
// of that height (batched ensembles), tz <= 0 uses the candidate's split.
template <typename T> StepCfg stencil_cfg(int fluid, int cand, int N, int tz);
template <typename T> cudaError_t stencil_launch(int fluid, const StencilArgs<T>& a, const StepCfg& c, cudaStream_t st);
// One launch over a work list spanning several runs (table and work in device memory).
template <typename T>
cudaError_t stencil_launch_batch(int fluid, int cand, const StencilArgs<T>* table, const WorkItem* work, int nwork,
                                 bool outflow, bool cool, cudaStream_t st);

// Reading B of the Lagrangian flux (flic_flux_b.cu): arguments of the Eulerian
// and transport kernels of one fluid (fluid-local field order as StencilArgs;
// fp: NF fields of f', w: 3 fields of +x/+y/+z face velocities, stride fs).
template <typename T>
struct FluxBArgs {
    const T* in;
    T* out;
    const T* phi;
    T* fp;
    T* w;
    size_t fs;
    int n;
    const double* tau;
    double inv_h;
    T gamma, eta, cool;
    double* partials;     // float32: (sum, compensation) float32 pairs in the 8-byte slots
    double* vmax;
    unsigned int* status;
};
// Both kernels of one fluid over `blocks` blocks (partial rows 0..blocks-1).
template <typename T> cudaError_t launch_flux_b(int fluid, const FluxBArgs<T>& a, int blocks, cudaStream_t st);
constexpr int FLUX_B_BLOCKS = 152 * 4;

// float64 <-> storage precision conversion of one field.
template <typename T> cudaError_t convert_in(const double* src, T* dst, size_t n, cudaStream_t st);
const void* mapped_device_view(const void* host_ptr);
template <typename T> cudaError_t convert_out(const T* src, double* dst, size_t n, cudaStream_t st);

// The 22 field arrays of a state.
template <typename T>
struct FieldPtrs {
    const T* f[F_COUNT];
};

// Conserved sums, kappa and signal speed of a whole state (partials[nb][Q_COUNT];
// phi may be null, E_pot then sums to zero).
template <typename T>
cudaError_t state_reduce(const T* state, size_t fs, const T* phi, size_t cells, double gamma,
                         double* partials, int nb, double* vmax, unsigned int* status, cudaStream_t st);
template <typename T>
cudaError_t state_reduce(const FieldPtrs<T>& fields, const T* phi, size_t cells, double gamma, double* partials,
                         int nb, double* vmax, unsigned int* status, cudaStream_t st);

// Message returned by flic_last_error(NULL).
void set_global_error(const char* msg);

// Device scalars of a handle.
enum Scalar { S_VMAX_CUR = 0, S_TAU, S_VMAX_NEXT, S_TIME, S_COUNT = 8 };

// tau = dt (dt > 0) or courant*h / vmax_cur; clears vmax_next and the status word.
cudaError_t step_prep(double* scal, unsigned int* status, double dt, double courant_h, cudaStream_t st);

// Per-run scalars of a batched step.
struct RunScalars {
    double* scal;
    unsigned int* status;
    double courant_h;
};
cudaError_t step_prep_batch(const RunScalars* runs, int nruns, double dt, cudaStream_t st);

// Arguments of the reduction of one run's partial rows (a: gas, b: moments).
// Each row holds Q_COUNT 8-byte slots: float64 sums, or (pairs = 1, written by
// the float32 kernels) float32 (sum, compensation) pairs.
struct FinalizeArgs {
    const double* pa;
    int na;
    const double* pb;
    int nb;
    double h3;
    double* scal;
    unsigned int* status;
    flic_diag* diag;
    double* level1;
    int pairs;
};
// one reduction per run of the device table (all runs of one kind of row)
cudaError_t step_finalize_batch(const FinalizeArgs* table, int nruns, int count_step, int pairs, cudaStream_t st);

// Sums the per-block partials (fixed order, compensated), writes the record and
// advances vmax_cur, time and the step counter.  count_step = 0 for a
// diagnostics-only reduction.  float64 rows: two levels (FINALIZE_ROWS blocks,
// then one; level1: FINALIZE_ROWS x Q_COUNT doubles of scratch); float32 pair
// rows: one block in float32 two-sum arithmetic, one conversion per quantity.
constexpr int FINALIZE_ROWS = 64;
cudaError_t step_finalize(const double* pa, int na, const double* pb, int nb, double h3, double* scal,
                          unsigned int* status, flic_diag* diag, int count_step, double* level1, int pairs,
                          cudaStream_t st);

}  // namespace flic
