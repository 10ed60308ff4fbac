// odp_time.cuh -- the CFL step of Algorithm 1 in float64 on the device,
// shared by the single-solve graph and the batched solve so that both take
// bit-identical step sequences.
#pragma once

#include "odp_common.cuh"

namespace odp {

// dt_cfl = cfl / sum_d (alpha_d / h_d) (Algorithm 1's CFL step with the
// global alpha; infinity when every alpha is 0).
__device__ __forceinline__ double cfl_dt(const unsigned *alpha_bits, const double *dz, int ndim, double cfl)
{
    double s = 0.0;
    for (int d = 0; d < ndim; ++d) s = __dadd_rn(s, __ddiv_rn(double(__uint_as_float(alpha_bits[d])), dz[d]));
    return (s > 0.0) ? __ddiv_rn(cfl, s) : INFINITY;
}

// The step taken at look-back time t towards the segment end t_end: the CFL
// step, or the remainder when it reaches the end (then *last = 1).
__device__ __forceinline__ double clipped_step(double dt_cfl, double t, double t_end, int *last)
{
    const double rem = __dsub_rn(t_end, t);
    *last = !(dt_cfl < rem);
    return *last ? rem : dt_cfl;
}

// Time after a step, and whether the segment is finished (its remainder is at
// most 1e-12 of its end).
__device__ __forceinline__ double after_step(double t, double dt, double t_end, int last)
{
    return last ? t_end : __dadd_rn(t, dt);
}

__device__ __forceinline__ bool segment_done(double t, double t_end)
{
    return !(__dsub_rn(t_end, t) > __dmul_rn(1e-12, t_end));
}

}  // namespace odp
