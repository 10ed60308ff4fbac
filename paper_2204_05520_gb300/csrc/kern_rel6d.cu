// kern_rel6d.cu -- kernel instantiations for the 6-D relative
// pursuit-evasion model, including its per-stage heading-rate alpha.
#include "hj_kernels.cuh"

namespace odp {

cudaError_t launch_stage_rel6d(const GridDesc &g, const DynDesc &dy, SolveState *st,
                               const float *l, const float *gob, int order, int stage, int brt, cudaStream_t s)
{
    return launch_stage_t<6, DYN_REL6D>(g, dy, st, l, gob, order, stage, brt, s);
}

cudaError_t configure_stage_rel6d() { return configure_stage_t<6, DYN_REL6D>(); }

cudaError_t occupancy_stage_bulk_rel6d(int order, int threads, int smem, int *per_sm)
{
    return occupancy_stage_bulk_nd<6, DYN_REL6D>(order, threads, smem, per_sm);
}

cudaError_t launch_alpha_static_rel6d(const GridDesc &g, const DynDesc &dy, SolveState *st,
                                      cudaStream_t s)
{
    return launch_alpha_static_t<6, DYN_REL6D>(g, dy, st, s);
}

cudaError_t launch_alpha_dynamic_rel6d(const GridDesc &g, const DynDesc &dy, SolveState *st,
                                       int order, int slot, cudaStream_t s)
{
    const int blocks = blocks_for(alpha_rel6d_threads(g), 256);
    if (order == 1)
        k_alpha_rel6d<1><<<blocks, 256, 0, s>>>(g, dy, st, slot);
    else
        k_alpha_rel6d<2><<<blocks, 256, 0, s>>>(g, dy, st, slot);
    return cudaGetLastError();
}

}  // namespace odp
