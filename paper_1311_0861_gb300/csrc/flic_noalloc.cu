// Diagnostics of a caller-owned state without any device allocation.
//
// For callers that cannot call cudaMalloc: code that runs while another owner
// has reserved the device memory (an in-situ analysis hook inside a simulation
// that pre-allocates the GPU), or a latency-critical path where an allocation's
// implicit device synchronisation is not acceptable.  The per-block partial
// sums, the second-level sums, the scalars and the result record live in one
// file-scope __device__ array instead of handle-owned buffers.
#include <mutex>
#include <string>

#include "flic_internal.h"

namespace flic {
namespace {

constexpr int NOALLOC_ROWS = 1024;     // per-block partial rows the scratch holds
constexpr int NOALLOC_MAX_N = 1024;    // largest grid accepted (cells per axis)
constexpr size_t CELLS_PER_ROW = 4096; // cells summed per block before the block count saturates

struct NoallocScratch {
    double partials[NOALLOC_ROWS * Q_COUNT];
    double level1[FINALIZE_ROWS * Q_COUNT];
    double scal[S_COUNT];
    unsigned int status[4];
    flic_diag diag;
};

// About 102 KiB; every GPU that loads the library keeps it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

// Device address of the scratch array per device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up once per
// device with that device current.
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_scratch_addr[MAX_DEVICES] = {};

int scratch_of_current_device(NoallocScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_global_error(cudaGetErrorString(e));
        return FLIC_ERR_CUDA;
    }
    if (dev < 0 || dev >= MAX_DEVICES) {
        set_global_error("device index beyond the scratch table");
        return FLIC_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_global_error(e != cudaSuccess ? cudaGetErrorString(e) : "null scratch address");
            return FLIC_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = reinterpret_cast<NoallocScratch*>(g_scratch_addr[dev]);
    return FLIC_OK;
}

}  // namespace
}  // namespace flic

using namespace flic;

#define NOALLOC_CK(call)                                                         \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            set_global_error((std::string(#call) + ": " + cudaGetErrorString(e_)).c_str()); \
            return FLIC_ERR_CUDA;                                                \
        }                                                                        \
    } while (0)

extern "C" int flic_state_diagnostics_noalloc(const double* const fields[FLIC_NFIELDS], const double* phi, int n,
                                              double h, double gamma, void* stream, flic_diag* out) {
    if (!fields || !out) {
        set_global_error("null argument");
        return FLIC_ERR_INVALID_ARG;
    }
    for (int k = 0; k < FLIC_NFIELDS; ++k)
        if (!fields[k]) {
            set_global_error("null field pointer");
            return FLIC_ERR_INVALID_ARG;
        }
    if (n < 1 || n > NOALLOC_MAX_N) {
        set_global_error("n must be between 1 and 1024 (the size the no-allocation scratch is built for)");
        return FLIC_ERR_INVALID_ARG;
    }
    if (!(h > 0.0) || !(gamma > 1.0)) {
        set_global_error("invalid h or gamma");
        return FLIC_ERR_INVALID_ARG;
    }
    NoallocScratch* sc = nullptr;
    int rc = scratch_of_current_device(&sc);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t cells = size_t(n) * n * n;
    size_t rows = (cells + CELLS_PER_ROW - 1) / CELLS_PER_ROW;
    if (rows > size_t(NOALLOC_ROWS)) rows = NOALLOC_ROWS;
    // the scalars start at zero (vmax is an atomic max, status an atomic or);
    // partial rows are overwritten by every call
    NOALLOC_CK(cudaMemsetAsync(sc->scal, 0, sizeof(sc->scal) + sizeof(sc->status), st));
    FieldPtrs<double> f;
    for (int k = 0; k < F_COUNT; ++k) f.f[k] = fields[k];
    NOALLOC_CK(state_reduce<double>(f, phi, cells, gamma, sc->partials, int(rows), sc->scal + S_VMAX_NEXT,
                                    sc->status, st));
    NOALLOC_CK(step_finalize(sc->partials, int(rows), nullptr, 0, h * h * h, sc->scal, sc->status, &sc->diag, 0,
                             sc->level1, 0, st));
    NOALLOC_CK(cudaMemcpyAsync(out, &sc->diag, sizeof(flic_diag), cudaMemcpyDeviceToHost, st));
    NOALLOC_CK(cudaStreamSynchronize(st));
    out->step = 0;
    return out->status == FLIC_OK ? FLIC_OK : FLIC_ERR_NONPHYSICAL;
}
