// kern_dubins.cu -- kernel instantiations for the 3D Dubins car and the 4D
// Dubins car (Appendix models).
#include "hj_kernels.cuh"

namespace odp {

cudaError_t launch_stage_dubins(int nd, const GridDesc &g, const DynDesc &dy, SolveState *st,
                                const float *l, const float *gob, int order, int stage, int brt, cudaStream_t s)
{
    if (nd == 3) return launch_stage_t<3, DYN_DUBINS3D>(g, dy, st, l, gob, order, stage, brt, s);
    return launch_stage_t<4, DYN_DUBINSCAR4D>(g, dy, st, l, gob, order, stage, brt, s);
}

cudaError_t configure_stage_dubins(int nd)
{
    if (nd == 3) return configure_stage_t<3, DYN_DUBINS3D>();
    return configure_stage_t<4, DYN_DUBINSCAR4D>();
}

cudaError_t occupancy_stage_bulk_dubins(int nd, int order, int threads, int smem, int *per_sm)
{
    if (nd == 3) return occupancy_stage_bulk_nd<3, DYN_DUBINS3D>(order, threads, smem, per_sm);
    return occupancy_stage_bulk_nd<4, DYN_DUBINSCAR4D>(order, threads, smem, per_sm);
}

cudaError_t launch_alpha_static_dubins(int nd, const GridDesc &g, const DynDesc &dy,
                                       SolveState *st, cudaStream_t s)
{
    if (nd == 3) return launch_alpha_static_t<3, DYN_DUBINS3D>(g, dy, st, s);
    return launch_alpha_static_t<4, DYN_DUBINSCAR4D>(g, dy, st, s);
}

}  // namespace odp
