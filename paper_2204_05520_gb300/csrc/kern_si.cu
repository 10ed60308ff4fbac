// kern_si.cu -- kernel instantiations for the single integrator and the
// constant-velocity advection model: 1 to 3 dimensions here, 4, 5 and 6 in
// kern_si4.cu, kern_si5.cu and kern_si6.cu; the launchers dispatch on the
// dimension count.
#include "kern_si_nd.cuh"

namespace odp {

ODP_SI_INSTANTIATE(1)
ODP_SI_INSTANTIATE(2)
ODP_SI_INSTANTIATE(3)
ODP_SI_EXTERN(4)
ODP_SI_EXTERN(5)
ODP_SI_EXTERN(6)

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
                            const float *l, const float *gob, int order, int stage, int brt, cudaStream_t s)
{
    ODP_ND_SWITCH(nd, (launch_stage_si_nd<ND>(g, dy, st, l, gob, order, stage, brt, s)))
}

cudaError_t configure_stage_si(int nd, int kind)
{
    ODP_ND_SWITCH(nd, (configure_stage_si_nd<ND>(kind)))
}

cudaError_t launch_alpha_static_si(int nd, const GridDesc &g, const DynDesc &dy, SolveState *st,
                                   cudaStream_t s)
{
    ODP_ND_SWITCH(nd, (launch_alpha_static_si_nd<ND>(g, dy, st, s)))
}

}  // namespace odp
