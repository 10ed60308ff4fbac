// odp_internal.h -- the grid object shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/odp.h"
#include "odp_common.cuh"

namespace odp {
// Record a message for odp_last_error() and return code.
odp_status fail(odp_status code, const char *fmt, ...);
}  // namespace odp

struct odp_grid;
namespace odp {
// Free the time-to-reach plan of a grid (tile lists, state, graph).
void ttr_release(odp_grid *g);
// Geometry of the plane-streaming pass of a grid (D.pg; pg.use = 0 when the
// pass does not apply), aiming at about twelve CTAs per SM on `sms` SMs.
void plane_geometry(GridDesc &D, int sms);
// The same geometry for a grid advanced together with many others: stream
// chunks of up to 16 planes (the parallelism comes from the many grids).
void plane_geometry_many(GridDesc &D);
// Geometry of the bulk-staged pass of a single solve (D.bk; bk.use = 0 when
// the pass does not apply): bands of about `threads` compute threads, and
// stream-axis chunks for an estimated occupancy on `sms` SMs.
void bulk_geometry(GridDesc &D, int sms, int threads);
// Ceiling of the Rel6D heading-rate dissipation bound over a grid whose w_p
// axis has n nodes on [lo, hi] (periodic or not), b the evader's turn bound:
// no node's bound exceeds it, and a node whose one-sided differences
// straddle zero at the largest |w_p| reaches it (the alpha pass stops there).
float rel6d_heading_ceiling(float b, double lo, double hi, int n, int periodic);
// Stream-axis chunking of the bulk-staged pass for stencil radius o, with
// per_sm CTAs resident per SM on `sms` SMs (bk.chunk, nchunks, items).
void bulk_chunking(GridDesc &D, int o, int per_sm, int sms);
}  // namespace odp

// Kernel arguments (grid and dynamics descriptors) are frozen into the graph
// when it is captured, so any change of scheme or dynamics rebuilds it.
struct GraphKey {
    int order = 0, time_order = 0, brt = 0, keep = 0, obstacle = 0;
    long long dyn_version = -1;
    long long sched_version = -1;     // time-varying target / obstacle schedules
    bool operator==(const GraphKey &o) const
    {
        return order == o.order && time_order == o.time_order && brt == o.brt && keep == o.keep &&
               obstacle == o.obstacle && dyn_version == o.dyn_version && sched_version == o.sched_version;
    }
};

struct odp_grid {
    int ndim = 0;
    int n[ODP_MAXD] = {0};
    double lo[ODP_MAXD] = {0}, hi[ODP_MAXD] = {0};
    int periodic[ODP_MAXD] = {0};
    int64_t total = 0;                // nodes
    int64_t total_pad = 0;            // stored floats (last axis padded to n_pad)
    int n_last = 0, n_pad = 0;
    int64_t rows = 0;
    cudaStream_t stream = nullptr;
    int device = 0;

    float *phi_a = nullptr, *phi_b = nullptr, *l = nullptr;
    float *obst = nullptr;            // reach-avoid obstacle g (allocated on first use)
    float *cdn = nullptr;             // per-node dissipation coefficients of the capture model
    bool has_obst = false;
    int local_diss = 0;               // per-node dissipation (odp_set_dissipation)
    float *tables = nullptr;          // all node-coordinate and trig tables
    odp::SolveState *state = nullptr;
    double *tau = nullptr;
    int tau_cap = 0;
    float *snapshots = nullptr;
    int snap_cap = 0;

    odp::GridDesc desc{};
    odp::DynDesc dyn{};
    bool has_dyn = false, has_target = false, solved = false;
    long long dyn_version = 0;
    int64_t max_steps = 10000000;
    int n_tau = 0, keep = 0, time_order = 1, order = 1, brt = 0;
    bool timed = false;

    cudaStream_t capture_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    GraphKey key;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int64_t launches_per_step = 0;
    int host_loop = 0;                // 1: the time loop is stepped from the host
    int bulk_ok = 0;                  // the bulk-staged pass applies to this grid's shape
    int stage_pass = 0;               // odp_set_stage_pass: 0 automatic, 1 plane-streaming, 2 bulk-staged
    void *ttr = nullptr;              // time-to-reach plan (ttr.cu), built on first use
    // time-varying sets (odp_set_target_schedule / odp_set_obstacle_schedule):
    // n sets of total_pad floats each; during a solve l and obst hold the
    // current segment's sets
    float *l_seq = nullptr, *g_seq = nullptr;
    int l_seq_n = 0, g_seq_n = 0;
    int l_seq_cap = 0, g_seq_cap = 0;
    long long sched_version = 0;
};

