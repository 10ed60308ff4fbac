// kern_si.cu -- kernel instantiations for the single integrator and the
// constant-velocity advection model, 1 to 6 dimensions.
#include "hj_kernels.cuh"

namespace odp {

#define ODP_ND_SWITCH(nd, CALL)                                                  \
    switch (nd) {                                                                \
    case 1: { constexpr int ND = 1; return CALL; }                               \
    case 2: { constexpr int ND = 2; return CALL; }                               \
    case 3: { constexpr int ND = 3; return CALL; }                               \
    case 4: { constexpr int ND = 4; return CALL; }                               \
    case 5: { constexpr int ND = 5; return CALL; }                               \
    case 6: { constexpr int ND = 6; return CALL; }                               \
    default: return cudaErrorInvalidValue;                                       \
    }

cudaError_t launch_stage_si(int nd, const GridDesc &g, const DynDesc &dy, SolveState *st,
                            const float *l, int order, int stage, int brt, cudaStream_t s)
{
    if (dy.kind == DYN_SINGLE_INT) {
        ODP_ND_SWITCH(nd, (launch_stage_t<ND, DYN_SINGLE_INT>(g, dy, st, l, order, stage, brt, s)))
    }
    ODP_ND_SWITCH(nd, (launch_stage_t<ND, DYN_ADVECTION>(g, dy, st, l, order, stage, brt, s)))
}

cudaError_t configure_stage_si(int nd, int kind)
{
    if (kind == DYN_SINGLE_INT) {
        ODP_ND_SWITCH(nd, (configure_stage_t<ND, DYN_SINGLE_INT>()))
    }
    ODP_ND_SWITCH(nd, (configure_stage_t<ND, DYN_ADVECTION>()))
}

cudaError_t launch_alpha_static_si(int nd, const GridDesc &g, const DynDesc &dy, SolveState *st,
                                   cudaStream_t s)
{
    if (dy.kind == DYN_SINGLE_INT) {
        ODP_ND_SWITCH(nd, (launch_alpha_static_t<ND, DYN_SINGLE_INT>(g, dy, st, s)))
    }
    ODP_ND_SWITCH(nd, (launch_alpha_static_t<ND, DYN_ADVECTION>(g, dy, st, s)))
}

}  // namespace odp
