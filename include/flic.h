/*
 * flic.h -- C ABI of the GB300 two-fluid FlIC/Godunov step library (libflic.so).
 *
 * The library advances a self-gravitating adiabatic gas and a collisionless
 * "Boltzmann-moment" fluid (density, momentum, full symmetric energy and
 * velocity-dispersion tensors) on a uniform N^3 grid (periodic or outflow) by the scheme of
 * Kulikov 2013 (GPUPEGAS):
 *   Sec. 2.3  Poisson equation for the total potential, Laplace(Phi) = 4 pi G (rho + n),
 *             solved by FFT with the 27-point stencil symbol;
 *   Sec. 2.1  gas Eulerian stage (face pressure/velocity from the linearised
 *             Riemann solution), then the Lagrangian stage (face-flux transport);
 *   Sec. 2.2  Boltzmann-moment Eulerian stage (closed-form face solution of the
 *             6x6 linear system), then the Lagrangian stage;
 *   Sec. 2.4  correctness checks kappa_gas, kappa_bme and the energy balance;
 *   Sec. 2    an optional analytic stand-in for the gas cooling function q.
 * Every stage runs in hand-written CUDA kernels for sm_103a; there is no CPU
 * fallback.
 *
 * State layout (host arrays given to or taken from the library): 22 float64
 * arrays of N^3 values each, structure of arrays, x fastest
 * (index = i + N*(j + N*k)), in this field order:
 *    0 rho   1 mx   2 my   3 mz   4 E (total gas energy density)   5 e (internal)
 *    6 n     7 qx   8 qy   9 qz
 *   10 nExx 11 nEyy 12 nEzz 13 nExy 14 nExz 15 nEyz   (n E_ij = Pi_ij + n u_i u_j)
 *   16 Pxx  17 Pyy  18 Pzz  19 Pxy  20 Pxz  21 Pyz    (velocity-dispersion tensor)
 * The grid covers [box_min, box_max]^3 with cell width h = (box_max - box_min)/N.
 *
 * Ownership: the library owns every device buffer it allocates (state, potential,
 * FFT and reduction workspace).  Host pointers passed in are only read or written
 * during the call.  "_device" entry points take device pointers owned by the
 * caller and only read/write them during the call (stream-ordered).
 *
 * Errors: every call returns FLIC_OK (0) or a negative code; no exception or
 * trap crosses the boundary.  flic_last_error() gives a message for the last
 * failing call on a handle.
 */
#ifndef FLIC_H
#define FLIC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FLIC_NFIELDS 22

enum flic_status {
    FLIC_OK = 0,
    FLIC_ERR_INVALID_ARG = -1,   /* bad size, null pointer, unsupported option */
    FLIC_ERR_CUDA = -2,          /* a CUDA runtime call failed (message in last_error) */
    FLIC_ERR_NONPHYSICAL = -3,   /* step finished but produced rho, n, e or Pi_dd <= 0 or a non-finite value */
    FLIC_ERR_TIMEOUT = -4,       /* a bounded device wait expired (reserved) */
    FLIC_ERR_OOM = -5            /* device allocation failed */
};

enum flic_precision {
    FLIC_FP64 = 0,   /* all storage and arithmetic in float64 */
    FLIC_MIXED = 1   /* float32 storage and arithmetic; float64 for tau, diagnostics sums */
};

enum flic_poisson_bc {
    FLIC_PERIODIC = 0,   /* periodic potential, 27-point symbol (Sec. 2.3) */
    FLIC_ISOLATED = 1    /* vacuum boundaries: zero-padded (2N)^3 convolution with the point-mass
                            Green's function -G h^3/|r|, -G h^2 (3 ln(2+sqrt 3) - pi/2) at r = 0
                            (n = 8..128, 256, 512) */
};

/* Hydrodynamic boundaries.  The paper states none; periodic is the default
 * reading.  Outflow (zero gradient): two layers of ghost cells along each axis
 * copy the nearest edge cell of the time-n state and potential, and the step is
 * computed as on the grid extended by them (ghost cells take the Eulerian stage
 * from their own ghost neighbours); mass and momentum then change by the
 * boundary fluxes. */
enum flic_hydro_bc {
    FLIC_HYDRO_PERIODIC = 0,
    FLIC_HYDRO_OUTFLOW = 1
};

/* Transport velocity of the Lagrangian stage (Sec. 2.1, whose printed flux averages
 * four transverse face velocities in a garbled form).  A: the face's own Eulerian
 * velocity (default, the fused kernels).  B: the mean of the face velocities of
 * the same orientation at the face's four transverse diagonal neighbours, the
 * printed form taken literally (periodic hydro boundaries only; two plain kernels
 * per fluid, for experiments). */
enum flic_flux_reading {
    FLIC_FLUX_A = 0,
    FLIC_FLUX_B = 1
};

typedef struct flic_grid_desc {
    int n;               /* cells per axis (cube); N = 2^a 3^b, 8 <= N <= 1024 */
    double box_min;      /* domain [box_min, box_max]^3 */
    double box_max;
    double gamma;        /* adiabatic index of the gas */
    double G;            /* gravitational constant (0 disables gravity) */
    double courant;      /* Courant number of the CFL step */
    double eta;          /* energy-balance switch (1e-3) */
    int precision;       /* enum flic_precision */
    int poisson_bc;      /* enum flic_poisson_bc */
    int hydro_bc;        /* enum flic_hydro_bc (0: periodic) */
    double cooling;      /* Lambda >= 0 of the gas cooling function q of Sec. 2, whose tabulated form the
                            paper takes from Sutherland & Dopita; here an analytic placeholder
                            q = Lambda rho^2 sqrt(eps), subtracted (times tau, time-n state) from E and e
                            in the Eulerian stage; 0 = adiabatic */
    int flux_reading;    /* enum flic_flux_reading (0: A); ensembles take A only */
} flic_grid_desc;

/* Per-step record.  Conserved sums describe the state at the START of the step
 * (with the potential solved in that step); kappa_* are measured on the
 * post-Lagrangian state before the energy balance; vmax is the signal speed of
 * the state at the END of the step (it sets the next CFL step). */
typedef struct flic_diag {
    double mass_gas, mass_bme;        /* sum rho h^3, sum n h^3 */
    double mom[3];                    /* sum (m + q) h^3 */
    double ekin_gas, eint_gas;        /* sum |m|^2/(2 rho) h^3, sum e h^3 */
    double ekin_bme, etherm_bme;      /* sum |q|^2/(2 n) h^3, sum tr(Pi)/2 h^3 */
    double epot;                      /* 1/2 sum (rho + n) Phi h^3 */
    double kappa_gas, kappa_bme;      /* Sec. 2.4 integrals (h^3 sum of |.|) */
    double vmax;                      /* max |v_d| + c_s, |u_d| + sqrt(3 Pi_dd / n) */
    double dt;                        /* step size used */
    double time;                      /* simulated time after the step */
    long long step;                   /* steps taken */
    int status;                       /* FLIC_OK or FLIC_ERR_NONPHYSICAL */
} flic_diag;

typedef struct flic_handle flic_handle;

/* The grid and constants of Sec. 2: a uniform cubic grid of n^3 cells of width
 * h = (box_max - box_min)/n, the adiabatic index gamma and the gravitational
 * constant G of the equations of Sec. 2, the Courant number of the step size
 * (Sec. 2 states no CFL formula; the library takes tau = courant * h / vmax with
 * vmax as in flic_diag), the energy-balance switch eta of Sec. 2.4, and the
 * Poisson boundary of Sec. 2.3 (periodic, as its discrete Fourier indices imply,
 * or isolated).
 * Allocates device state for one grid; *out receives the handle.  `stream` is a
 * cudaStream_t on which every launch of this handle is issued; NULL makes the
 * library create (and later destroy) a non-blocking stream of its own.  The
 * state starts as zeros; call flic_set_state first.  Errors: INVALID_ARG for an
 * unsupported n or constants, OOM / CUDA on allocation failures (nothing leaks). */
int flic_init_grid(const flic_grid_desc* desc, void* stream, flic_handle** out);

/* The state of Sec. 2: the gas's conserved density, momentum, total and
 * internal energy and the Boltzmann moments (density, momentum, energy tensor)
 * with the velocity-dispersion tensor Pi of Sec. 2.2.
 * Copies 22 host float64 arrays (field order above, N^3 each) to the device,
 * converting to the storage precision on the device, and computes the initial
 * signal speed.  Page-locked, device-mapped arrays (cudaHostAlloc) are read in
 * place by the conversion kernel; pageable arrays go through a staging copy.
 * Returns FLIC_ERR_NONPHYSICAL if the state has rho, n, e or Pi_dd <= 0 or a
 * non-finite value (the state is still stored). */
int flic_set_state(flic_handle* h, const double* const fields[FLIC_NFIELDS]);

/* Same, from 22 device float64 arrays owned by the caller. */
int flic_set_state_device(flic_handle* h, const double* const fields[FLIC_NFIELDS]);

/* Copies the state to 22 host float64 arrays (N^3 each); page-locked mapped
 * arrays are written in place by the conversion kernel. */
int flic_get_state(flic_handle* h, double* const fields[FLIC_NFIELDS]);

/* Same, into 22 device float64 arrays owned by the caller. */
int flic_get_state_device(flic_handle* h, double* const fields[FLIC_NFIELDS]);

/* One full time step of the method, Sec. 2.1-2.4: the potential of the total
 * density (Sec. 2.3), the step size, the gas Eulerian stage with the face
 * velocity and pressure of the linearised Riemann problem and the Lagrangian
 * stage (Sec. 2.1), the Boltzmann-moment Eulerian stage with the closed-form face
 * solution of its 6x6 system and the same Lagrangian stage (Sec. 2.2), then the
 * kappa checks and the energy balance (Sec. 2.4), and the conserved sums.
 * (Poisson, tau, both fluids, kappa, energy balance, diagnostics.)
 * dt > 0: fixed step; dt <= 0: CFL step tau = courant * h / vmax computed on the
 * device.  If dt_used is non-NULL the call waits for the step and stores tau;
 * otherwise it returns after enqueueing (stream-ordered). */
int flic_step(flic_handle* h, double dt, double* dt_used);

/* nsteps consecutive steps of Sec. 2.1-2.4 (as flic_step) with no host synchronisation (CUDA-graph replay after
 * the first call for a given dt mode).  Waits for completion only if `sync`. */
int flic_run(flic_handle* h, int nsteps, double dt, int sync);

/* Profiling: runs nsteps steps as plain launches (no graph), recording CUDA
 * events on the handle's stream around each stage; stage_ms[k] receives the
 * summed device time of stage k over the steps and *total_ms (nullable) the
 * elapsed time from the first to the last event.  Stages: 0 step setup and
 * Poisson solve (Sec. 2.3), 1 gas kernel (Sec. 2.1, 2.4), 2 Boltzmann-moment
 * kernel (Sec. 2.2, 2.4), 3 final reduction of the diagnostics. */
#define FLIC_NSTAGES 4
int flic_profile(flic_handle* h, int nsteps, double dt, double stage_ms[FLIC_NSTAGES], double* total_ms);

/* Number of kernels one step launches (for launch accounting). */
int flic_launches_per_step(flic_handle* h);

/* ---- launch-shape tuner (no counterpart in the paper) ----
 *
 * Each fluid kernel (gas: Sec. 2.1, 2.4; moments: Sec. 2.2, 2.4) is compiled in
 * several launch shapes -- tile of columns, threads per block, blocks per SM --
 * each used with a z split over blocks (a balanced split over one block per
 * resident slot -- whole tile columns, equal parts of them, or, with fewer tiles
 * than blocks, the lower part of every column in lockstep and the tops shared --
 * or z chunks); which is fastest depends on the GPU and the grid size, not on
 * the method.  The shapes compute the same cell updates; only the
 * partial sums of the diagnostics are grouped differently.
 *
 * flic_autotune times every shape of both kernels on the handle's CURRENT state
 * (call it after flic_set_state): one untimed launch, then `reps` launches
 * between two CUDA events on the handle's stream, and keeps the fastest shape of
 * each kernel (shapes are taken in index order, and a later one replaces the one
 * kept only when it is more than 0.5 % faster, so that shapes timing the same
 * within noise resolve to the lower index).  The launches write only the library's spare state buffer: the
 * current state, time, step count and CFL signal speed are unchanged.  With
 * use_cache != 0 a choice made earlier in this process for the same device model,
 * n, precision and hydro boundary is applied without timing (return value 1);
 * otherwise the shapes are timed and the choice is cached (return value 0).
 * ms (nullable) receives, when timing, the mean milliseconds per launch of every
 * shape (gas shapes first, then moment shapes; -1 for a shape the device cannot
 * launch).  Errors: INVALID_ARG (reps < 1), CUDA. */
int flic_autotune(flic_handle* h, int reps, int use_cache, double* ms);

/* Number of compiled shapes of the gas and moment kernels for this handle's precision. */
int flic_num_tile_configs(flic_handle* h, int* n_gas, int* n_bme);

/* Selects shape `gas` / `bme` (indices below flic_num_tile_configs; -1 keeps the
 * current one).  Shape 0 of each kernel is the default of a new handle. */
int flic_set_tile_config(flic_handle* h, int gas, int bme);

/* The shapes in use: their indices (nullable pointers) and, when text is not
 * NULL, a description of at most len - 1 characters. */
int flic_tile_config(flic_handle* h, int* gas, int* bme, char* text, int len);

/* Solves Sec. 2.3 for the current state; phi_out (host, N^3 float64) may be NULL
 * to keep the potential on the device only. */
int flic_solve_poisson(flic_handle* h, double* phi_out);

/* Record of the last completed step (waits for the stream): the kappa_gas and
 * kappa_bme checks of Sec. 2.4 and the quantities whose conservation the paper
 * reports for its cloud-collision test (Sec. 4.5: mass and total momentum kept
 * by the scheme, the kinetic, internal and potential energies traced). */
int flic_step_diagnostics(flic_handle* h, flic_diag* out);

/* The same quantities (Sec. 2.4; Sec. 4.5) for the CURRENT state (solves the
 * Poisson equation of Sec. 2.3 for E_pot; kappa of the current state; dt = 0). */
int flic_diagnostics(flic_handle* h, flic_diag* out);

/* Diagnostics of a caller-owned float64 state with NO device allocation (no
 * counterpart in the paper: this is a deployment entry point).
 *
 * For callers that cannot call cudaMalloc -- code running while another owner
 * has reserved the device memory (an in-situ analysis hook inside a simulation
 * that pre-allocates the GPU), or a latency-critical path that cannot take an
 * allocation's implicit device synchronisation.  It computes what
 * flic_diagnostics computes (conserved sums, kappa_gas, kappa_bme, signal speed,
 * validity) for 22 device float64 arrays of n^3 cells (field order and layout
 * above) and, when phi (device, n^3 float64) is not NULL, E_pot; dt = 0,
 * step = 0, time = 0.  The result is written to the host record *out.
 *
 * Scratch: the per-block partial sums live in one file-scope device array of
 * about 102 KiB (1024 partial rows) that every GPU loading the library keeps
 * until exit; n must be between 1 and 1024, larger grids are rejected with
 * FLIC_ERR_INVALID_ARG.  The array belongs to the library's device code, which
 * the CUDA runtime loads onto a device at the first call of this library there
 * (this call or any other), so that first call needs the device memory for it.
 * The first call of this entry point on a device looks up the array's device
 * address (with that device current) and keeps it for the process; make that
 * first call before any stream capture, and do not reset the device
 * (cudaDeviceReset) while the library is in use.  Every call shares the array
 * and leaves the last call's contents in it; the scalars that must start at
 * zero are cleared on entry.  Calls that overlap on the GPU (different streams
 * or threads) race on it.  The call is synchronous: it runs on `stream`
 * (cudaStream_t, NULL = legacy default stream), waits for that stream and copies
 * the record to *out before it returns.  Errors: INVALID_ARG, CUDA (message in
 * flic_last_error(NULL)), NONPHYSICAL (record still written). */
int flic_state_diagnostics_noalloc(const double* const fields[FLIC_NFIELDS], const double* phi, int n, double h,
                                   double gamma, void* stream, flic_diag* out);

/* ---- batched ensembles (independent runs, uneven sizes, advanced together) ----
 *
 * A deployment form of the step of Sec. 2.1-2.4 with no counterpart in the
 * paper: each run takes exactly the steps flic_step would take on its own grid.
 *
 * nruns grids, descs[r] for run r; every constant except n must be equal across
 * runs (n = 2^a 3^b, multiple of 4, 8..512).  Each step solves every run's
 * Poisson equation (one set of FFT launches per grid size, batched over the runs
 * of that size), then runs each fluid stage as ONE launch over a work list that
 * spans all runs' tiles, and the setup / reduction as one launch each; steps are
 * replayed as CUDA graphs.  Each run keeps its own CFL step (tau from its own
 * signal speed), diagnostics record and status.  Errors of create: message in
 * flic_last_error(NULL); afterwards flic_ensemble_last_error(e). */
typedef struct flic_ensemble flic_ensemble;
int flic_ensemble_create(const flic_grid_desc* descs, int nruns, void* stream, flic_ensemble** out);
int flic_ensemble_set_state(flic_ensemble* e, int run, const double* const fields[FLIC_NFIELDS]);  /* host */
int flic_ensemble_get_state(flic_ensemble* e, int run, double* const fields[FLIC_NFIELDS]);        /* host */
/* nsteps steps of every run (dt > 0: fixed step for all; dt <= 0: each run's CFL
 * step); waits and checks every run's status only if `sync`. */
int flic_ensemble_step(flic_ensemble* e, int nsteps, double dt, int sync);
/* Last step record of one run (same fields as flic_step_diagnostics). */
int flic_ensemble_diagnostics(flic_ensemble* e, int run, flic_diag* out);
/* nsteps steps as plain launches with CUDA events on the ensemble's stream
 * between stages (the stages of flic_profile); stage_ms[k] summed over steps,
 * *total_ms (nullable) first to last event. */
int flic_ensemble_profile(flic_ensemble* e, int nsteps, double dt, double stage_ms[FLIC_NSTAGES],
                          double* total_ms);
int flic_ensemble_launches_per_step(flic_ensemble* e);
/* Launch-shape tuner of an ensemble (see flic_autotune): every compiled shape of
 * each fluid kernel is timed over the whole work list with work items of at most
 * 16, 32 and 64 z planes (`reps` launches after one untimed launch, on the
 * current states; only the spare state buffers are written), and the fastest
 * (shape, chunk height) of each kernel is kept.  ms (nullable) receives 3 values
 * per shape (gas shapes first; -1 for a shape that is skipped, i.e. one that
 * differs from an earlier entry only in its single-grid split, or that the
 * device cannot launch).  No caching. */
int flic_ensemble_autotune(flic_ensemble* e, int reps, double* ms);
/* Number of compiled shapes of the gas and moment kernels for this ensemble's precision. */
int flic_ensemble_num_tile_configs(flic_ensemble* e, int* n_gas, int* n_bme);
/* Selects the shapes and the z-chunk caps of the work items (-1 keeps the current value). */
int flic_ensemble_set_tile_config(flic_ensemble* e, int gas, int bme, int tz_gas, int tz_bme);
/* The shapes and chunk caps in use (nullable pointers) and their description. */
int flic_ensemble_tile_config(flic_ensemble* e, int* gas, int* bme, int* tz_gas, int* tz_bme, char* text, int len);
int flic_ensemble_destroy(flic_ensemble* e);
const char* flic_ensemble_last_error(flic_ensemble* e);

/* Waits for all work of the handle (no counterpart in the paper). */
int flic_sync(flic_handle* h);

int flic_destroy(flic_handle* h);

/* Message of the last failing call on h (or of the last failing flic_init_grid
 * when h is NULL).  The pointer stays valid until the next call on h. */
const char* flic_last_error(flic_handle* h);

/* Library build information (compile flags, architecture). */
const char* flic_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FLIC_H */
