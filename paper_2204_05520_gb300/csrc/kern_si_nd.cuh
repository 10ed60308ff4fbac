// kern_si_nd.cuh -- single integrator and constant-velocity advection
// kernels of one dimension count.  kern_si.cu instantiates 1 to 3 dimensions
// and kern_si4/5/6.cu one count each, so the translation units compile in
// parallel.
#pragma once

#include "hj_kernels.cuh"

namespace odp {

template <int ND>
cudaError_t launch_stage_si_nd(const GridDesc &g, const DynDesc &dy, SolveState *st, const float *l,
                               const float *gob, int order, int stage, int brt, cudaStream_t s)
{
    if (dy.kind == DYN_SINGLE_INT) return launch_stage_t<ND, DYN_SINGLE_INT>(g, dy, st, l, gob, order, stage, brt, s);
    return launch_stage_t<ND, DYN_ADVECTION>(g, dy, st, l, gob, order, stage, brt, s);
}

template <int ND>
cudaError_t configure_stage_si_nd(int kind)
{
    if (kind == DYN_SINGLE_INT) return configure_stage_t<ND, DYN_SINGLE_INT>();
    return configure_stage_t<ND, DYN_ADVECTION>();
}

template <int ND>
cudaError_t launch_alpha_static_si_nd(const GridDesc &g, const DynDesc &dy, SolveState *st, cudaStream_t s)
{
    if (dy.kind == DYN_SINGLE_INT) return launch_alpha_static_t<ND, DYN_SINGLE_INT>(g, dy, st, s);
    return launch_alpha_static_t<ND, DYN_ADVECTION>(g, dy, st, s);
}

#define ODP_SI_INSTANTIATE(ND)                                                                               \
    template cudaError_t launch_stage_si_nd<ND>(const GridDesc &, const DynDesc &, SolveState *, const float *, \
                                                const float *, int, int, int, cudaStream_t);                  \
    template cudaError_t configure_stage_si_nd<ND>(int);                                                      \
    template cudaError_t launch_alpha_static_si_nd<ND>(const GridDesc &, const DynDesc &, SolveState *,       \
                                                       cudaStream_t);

#define ODP_SI_EXTERN(ND)                                                                                     \
    extern template cudaError_t launch_stage_si_nd<ND>(const GridDesc &, const DynDesc &, SolveState *,       \
                                                       const float *, const float *, int, int, int,           \
                                                       cudaStream_t);                                         \
    extern template cudaError_t configure_stage_si_nd<ND>(int);                                               \
    extern template cudaError_t launch_alpha_static_si_nd<ND>(const GridDesc &, const DynDesc &, SolveState *, \
                                                              cudaStream_t);

}  // namespace odp
