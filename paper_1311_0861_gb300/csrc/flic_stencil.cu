// Dispatch of the fused fluid-step kernels through their candidate tables (the
// compiled launch shapes, one translation unit per fluid and precision).
#include "flic_internal.h"

namespace flic {

template <typename T> cudaError_t stencil_prepare() {
    for (int fluid = 0; fluid < 2; ++fluid) {
        int n = 0;
        const StencilCand<T>* c = stencil_cands<T>(fluid, &n);
        for (int i = 0; i < n; ++i) {
            cudaError_t e = c[i].prepare();
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

template <typename T> StepCfg stencil_cfg(int fluid, int cand, int N, int tz) {
    int n = 0;
    const StencilCand<T>* c = stencil_cands<T>(fluid, &n);
    if (cand < 0 || cand >= n) cand = 0;
    StepCfg s = c[cand].cfg(N, tz, c[cand].split);
    s.cand = cand;
    return s;
}

template <typename T>
cudaError_t stencil_launch(int fluid, const StencilArgs<T>& a, const StepCfg& c, cudaStream_t st) {
    int n = 0;
    const StencilCand<T>* t = stencil_cands<T>(fluid, &n);
    if (c.cand < 0 || c.cand >= n) return cudaErrorInvalidValue;
    return t[c.cand].launch(a, c, st);
}

template <typename T>
cudaError_t stencil_launch_batch(int fluid, int cand, const StencilArgs<T>* table, const WorkItem* work, int nwork,
                                 bool outflow, bool cool, cudaStream_t st) {
    int n = 0;
    const StencilCand<T>* t = stencil_cands<T>(fluid, &n);
    if (cand < 0 || cand >= n) return cudaErrorInvalidValue;
    return t[cand].launch_batch(table, work, nwork, outflow, cool, st);
}

template cudaError_t stencil_prepare<float>();
template cudaError_t stencil_prepare<double>();
template StepCfg stencil_cfg<float>(int, int, int, int);
template StepCfg stencil_cfg<double>(int, int, int, int);
template cudaError_t stencil_launch<float>(int, const StencilArgs<float>&, const StepCfg&, cudaStream_t);
template cudaError_t stencil_launch<double>(int, const StencilArgs<double>&, const StepCfg&, cudaStream_t);
template cudaError_t stencil_launch_batch<float>(int, int, const StencilArgs<float>*, const WorkItem*, int, bool,
                                                 bool, cudaStream_t);
template cudaError_t stencil_launch_batch<double>(int, int, const StencilArgs<double>*, const WorkItem*, int, bool,
                                                  bool, cudaStream_t);

}  // namespace flic
