// kern_capture.cu -- kernel instantiations for the pursuit-evasion capture
// model of Section 4.2 (relative Dubins cars), including its per-stage alpha.
#include "hj_kernels.cuh"

namespace odp {

cudaError_t launch_stage_capture(const GridDesc &g, const DynDesc &dy, SolveState *st, const float *l,
                                 const float *gob, int order, int stage, int brt, cudaStream_t s)
{
    return launch_stage_t<3, DYN_CAPTURE>(g, dy, st, l, gob, order, stage, brt, s);
}

cudaError_t configure_stage_capture() { return configure_stage_t<3, DYN_CAPTURE>(); }

cudaError_t launch_alpha_static_capture(const GridDesc &g, const DynDesc &dy, SolveState *st, cudaStream_t s)
{
    return launch_alpha_static_t<3, DYN_CAPTURE>(g, dy, st, s);
}

cudaError_t launch_alpha_dynamic_capture(const GridDesc &g, const DynDesc &dy, SolveState *st, int order, int slot,
                                         cudaStream_t s)
{
    const int blocks = blocks_for(g.nthreads, 256);
    if (order == 1)
        k_alpha_capture<1><<<blocks, 256, 0, s>>>(g, dy, st, slot);
    else
        k_alpha_capture<2><<<blocks, 256, 0, s>>>(g, dy, st, slot);
    return cudaGetLastError();
}

}  // namespace odp
