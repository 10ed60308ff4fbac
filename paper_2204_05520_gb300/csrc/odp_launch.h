// odp_launch.h -- host-side launchers of the per-model kernel instantiations.
#pragma once

#include <cuda_runtime.h>

#include "odp_common.cuh"

namespace odp {

// One fused stage pass (K2) over the whole grid; gob is the reach-avoid
// obstacle (nullptr: none).
cudaError_t launch_stage_si(int nd, const GridDesc &g, const DynDesc &dy, SolveState *st,
                            const float *l, const float *gob, int order, int stage, int brt, cudaStream_t s);
cudaError_t launch_stage_dubins(int nd, const GridDesc &g, const DynDesc &dy, SolveState *st,
                                const float *l, const float *gob, int order, int stage, int brt, cudaStream_t s);
cudaError_t launch_stage_rel6d(const GridDesc &g, const DynDesc &dy, SolveState *st,
                               const float *l, const float *gob, int order, int stage, int brt, cudaStream_t s);

// Shared-memory limits of the plane-streaming kernels of a model (call before
// launching or capturing them on the current device).
cudaError_t configure_stage_si(int nd, int kind);
cudaError_t configure_stage_dubins(int nd);
cudaError_t configure_stage_rel6d();

// Resident CTAs per SM of the bulk-staged pass (radius `order`, `threads`
// threads and `smem` shared bytes a CTA), after configure_stage_*.
cudaError_t occupancy_stage_bulk_dubins(int nd, int order, int threads, int smem, int *per_sm);
cudaError_t occupancy_stage_bulk_rel6d(int order, int threads, int smem, int *per_sm);

// Grid-wide max of the phi-independent alpha components (K1, once per solve).
cudaError_t launch_alpha_static_si(int nd, const GridDesc &g, const DynDesc &dy, SolveState *st,
                                   cudaStream_t s);
cudaError_t launch_alpha_static_dubins(int nd, const GridDesc &g, const DynDesc &dy,
                                       SolveState *st, cudaStream_t s);
cudaError_t launch_alpha_static_rel6d(const GridDesc &g, const DynDesc &dy, SolveState *st,
                                      cudaStream_t s);

// The pursuit-evasion capture model (Section 4.2): stage pass, shared-memory
// limits, static alpha (zero: every component is per stage) and the
// per-stage alpha of cur (slot 0) or nxt (slot 1).
cudaError_t launch_stage_capture(const GridDesc &g, const DynDesc &dy, SolveState *st, const float *l,
                                 const float *gob, int order, int stage, int brt, cudaStream_t s);
cudaError_t configure_stage_capture();
cudaError_t launch_alpha_static_capture(const GridDesc &g, const DynDesc &dy, SolveState *st, cudaStream_t s);
cudaError_t launch_alpha_dynamic_capture(const GridDesc &g, const DynDesc &dy, SolveState *st, int order, int slot,
                                         cudaStream_t s);

// Grid-wide max of the Rel6D heading-rate alpha of cur (slot 0) or nxt (slot 1).
cudaError_t launch_alpha_dynamic_rel6d(const GridDesc &g, const DynDesc &dy, SolveState *st,
                                       int order, int slot, cudaStream_t s);

}  // namespace odp
