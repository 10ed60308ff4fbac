// batch.cu -- many independent solves advanced together in one persistent
// cooperative launch (odp_batch_solve).
//
// Every grid keeps its own arrays, dynamics, alpha and dt.  A prepare kernel
// (one CTA per grid) reduces each grid's static alpha and precomputes its
// whole step schedule in float64 with the same functions the single-solve
// graph uses (odp_time.cuh), so every grid takes exactly the steps it would
// take alone.  The persistent kernel then runs lockstep rounds: in round r
// every grid with more than r steps takes its step r (Euler: one pass; TVD-RK2:
// stage 1 in phase A, stage 2 in phase B), its work split into items of 256
// threads of the row-blocked stage pass.  Grids are sorted by step count, so
// the active items of a round are a prefix of the item list.  CTAs take items
// round robin and meet at a grid-wide barrier between phases; the barrier
// spin is bounded and reports a failure instead of hanging.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "hj_kernels.cuh"
#include "odp_internal.h"
#include "odp_time.cuh"

namespace odp {

struct BatchGrid {
    GridDesc g;
    DynDesc dy;
    float *a, *b;             // value buffers (the grid's phi_a, phi_b)
    const float *l;           // target
    SolveState *state;        // the grid's solve state (written at the end)
    double T, dt_cfl, dt_last;
    int n_steps;
    int kind, time_order, brt, items;
    unsigned alpha_bits[8];
    float cD[ODP_MAXD];
};

struct BatchBarrier {
    unsigned arrive;
    unsigned gen;
    int flags;                // 1: a barrier wait gave up
};

// ---------------------------------------------------------------------------
// prepare: static alpha and the step schedule of each grid
// ---------------------------------------------------------------------------
template <int DYN, int ND>
__device__ void batch_alpha(const GridDesc &g, const DynDesc &dy, float *a)
{
    for (int d = 0; d < ND; ++d) a[d] = 0.0f;
    for (uint32_t i = threadIdx.x; i < uint32_t(g.total); i += blockDim.x) {
        int idx[ND];
        unflatten(g, ND, i, idx);
        float la[ND];
        static_alpha<DYN, ND>(g, dy, idx, la);
        for (int d = 0; d < ND; ++d) a[d] = fmaxf(a[d], la[d]);
    }
}

__global__ void __launch_bounds__(256) k_batch_prepare(BatchGrid *bg, double cfl)
{
    __shared__ float red[8][ODP_MAXD];
    BatchGrid &B = bg[blockIdx.x];
    float a[ODP_MAXD];
    for (int d = 0; d < ODP_MAXD; ++d) a[d] = 0.0f;
    switch (B.kind) {
    case DYN_DUBINS3D: batch_alpha<DYN_DUBINS3D, 3>(B.g, B.dy, a); break;
    case DYN_DUBINSCAR4D: batch_alpha<DYN_DUBINSCAR4D, 4>(B.g, B.dy, a); break;
    case DYN_SINGLE_INT:
        if (B.g.ndim == 2) batch_alpha<DYN_SINGLE_INT, 2>(B.g, B.dy, a);
        else batch_alpha<DYN_SINGLE_INT, 3>(B.g, B.dy, a);
        break;
    default: break;
    }
    const int nd = B.g.ndim;
    for (int d = 0; d < nd; ++d) {
        const float m = warp_max(a[d]);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][d] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int d = 0; d < 8; ++d) B.alpha_bits[d] = 0u;
        for (int d = 0; d < nd; ++d) {
            float m = 0.0f;
            for (int w = 0; w < (blockDim.x >> 5); ++w) m = fmaxf(m, red[w][d]);
            B.alpha_bits[d] = __float_as_uint(m);
            B.cD[d] = 0.5f * m * B.g.inv_dz[d];
        }
        // the step schedule of a solve over [0, T] (as k_dt / k_advance take it)
        const double dt_cfl = cfl_dt(B.alpha_bits, B.g.dz, nd, cfl);
        double t = 0.0, dt = 0.0;
        int steps = 0, last = 0;
        do {
            dt = clipped_step(dt_cfl, t, B.T, &last);
            t = after_step(t, dt, B.T, last);
            ++steps;
        } while (!segment_done(t, B.T) && steps < (1 << 30));
        B.n_steps = steps;
        B.dt_cfl = dt_cfl;
        B.dt_last = dt;
        B.state->flags = 0;
    }
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  The
// arrival counter only grows: generation k ends when it reaches
// nblocks * (k + 1).  The wait gives up after a bounded number of polls.
__device__ bool grid_barrier(BatchBarrier *bar, unsigned &gen)
{
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        const unsigned target = gen + 1;
        __threadfence();
        const unsigned prev = atomicAdd(&bar->arrive, 1u);
        if (prev == gridDim.x * target - 1) {
            atomicExch(&bar->gen, target);
        } else {
            unsigned it = 0;
            while (ld_acquire(&bar->gen) < target) {
                if (++it > (1u << 22)) {
                    ok = 0;
                    atomicOr(&bar->flags, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    gen += 1;
    return __syncthreads_and(ok) != 0;
}

template <int ORDER, int R>
__device__ bool batch_item(const BatchGrid &B, int blk, int round, int phase)
{
    const uint32_t t = uint32_t(blk) * blockDim.x + threadIdx.x;
    if (t >= uint32_t(B.g.nthreads_rb)) return false;
    StageArgs A;
    const bool first = (round == 0);
    if (B.time_order == 1) {
        A.stage = 0;
        A.src = first ? B.l : ((round & 1) ? B.b : B.a);
        A.dst = (round & 1) ? B.a : B.b;
        A.prev = A.src;
    } else if (phase == 0) {
        A.stage = 1;
        A.src = first ? B.l : B.a;
        A.dst = B.b;
        A.prev = A.src;
    } else {
        A.stage = 2;
        A.src = B.b;
        A.prev = first ? B.l : B.a;
        A.dst = B.a;
    }
    A.l = B.l;
    A.gob = nullptr;
    A.brt = B.brt;
    A.dt = float(round == B.n_steps - 1 ? B.dt_last : B.dt_cfl);
    for (int d = 0; d < ODP_MAXD; ++d) A.cD[d] = B.cD[d];
    switch (B.kind) {
    case DYN_DUBINS3D: return stage_tile<3, ORDER, DYN_DUBINS3D, R>(B.g, B.dy, A, t);
    case DYN_DUBINSCAR4D: return stage_tile<4, ORDER, DYN_DUBINSCAR4D, R>(B.g, B.dy, A, t);
    case DYN_SINGLE_INT:
        if (B.g.ndim == 2) return stage_tile<2, ORDER, DYN_SINGLE_INT, R>(B.g, B.dy, A, t);
        return stage_tile<3, ORDER, DYN_SINGLE_INT, R>(B.g, B.dy, A, t);
    default: return false;
    }
}

// Rounds [round0, round1) of the batch.  sorted: grid ids by step count
// (descending); item_start: first item of each sorted grid (n + 1 entries);
// active: active items of every round.
// The upwind instantiations are held to 3 CTAs of 8 warps per SM (at most 85
// registers: each SM sub-partition holds 16384 registers for its warps).
template <int ORDER, int R>
__global__ void __launch_bounds__(256, ORDER == 1 ? 3 : 2) k_batch_run(const BatchGrid *__restrict__ bg, const int *__restrict__ sorted,
                                                   const int *__restrict__ item_start, int n,
                                                   const int *__restrict__ active, const int *__restrict__ active_rk2,
                                                   int round0, int round1, BatchBarrier *bar)
{
    __shared__ BatchGrid sB;
    unsigned gen = 0;
    for (int r = round0; r < round1; ++r) {
        for (int phase = 0; phase < 2; ++phase) {
            const int items = phase == 0 ? active[r] : active_rk2[r];
            if (phase == 1 && items == 0) break;
            for (int i = blockIdx.x; i < items; i += gridDim.x) {
                // sorted grid holding item i: last k with item_start[k] <= i
                int lo = 0, hi = n - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (item_start[mid] <= i) lo = mid; else hi = mid - 1;
                }
                const int gid = sorted[lo];
                {
                    const int words = int(sizeof(BatchGrid) / 4);
                    const unsigned *srcw = reinterpret_cast<const unsigned *>(bg + gid);
                    unsigned *dstw = reinterpret_cast<unsigned *>(&sB);
                    for (int w = threadIdx.x; w < words; w += blockDim.x) dstw[w] = srcw[w];
                }
                __syncthreads();
                if (!(phase == 1 && sB.time_order != 2)) {
                    if (batch_item<ORDER, R>(sB, i - item_start[lo], r, phase))
                        atomicOr(&sB.state->flags, FLAG_NONFINITE);
                }
                __syncthreads();
            }
            if (!grid_barrier(bar, gen)) return;
        }
    }
}

__global__ void k_batch_finish(const BatchGrid *bg, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const BatchGrid &B = bg[i];
    SolveState *st = B.state;
    const bool in_b = (B.time_order == 1) && (B.n_steps & 1);
    st->cur = in_b ? B.b : B.a;
    st->nxt = in_b ? B.a : B.b;
    st->t = B.T;
    st->t_end = B.T;
    st->dt = B.dt_last;
    st->steps = B.n_steps;
    st->seg = 1;
    st->n_seg = 1;
    for (int d = 0; d < 8; ++d) st->alpha_last[d] = B.alpha_bits[d];
}

// ---------------------------------------------------------------------------
// plane-streaming rounds (Dubins3D and DubinsCar4D batches)
// ---------------------------------------------------------------------------
// One launch per round and RK phase covers the plane items of the grids still
// active (a prefix of the item list, grids sorted by step count).  CTA i finds
// its grid, copies the grid's record into shared memory and runs one item of
// the plane pass with the grid's buffers, step and alpha of that round: the
// same per-node arithmetic as the solo solve.
// The 3-D upwind instantiation is held to 80 registers: 3 CTAs of 8 warps
// per SM (12,400 vs 11,640 solves/s on 512 Dubins3D grids).
template <int ND, int ORDER, int DYN>
__global__ void __launch_bounds__(512) __maxnreg__(((ND == 3 && ORDER == 1) ? 80 : plane_max_regs<ND, ORDER, DYN>()))
    k_batch_plane(const BatchGrid *__restrict__ bg, const int *__restrict__ sorted,
                  const int *__restrict__ item_start, int n, int round, int phase)
{
    __shared__ BatchGrid sB;
    const int i = blockIdx.x;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (item_start[mid] <= i) lo = mid; else hi = mid - 1;
    }
    {
        const int words = int(sizeof(BatchGrid) / 4);
        const unsigned *srcw = reinterpret_cast<const unsigned *>(bg + sorted[lo]);
        unsigned *dstw = reinterpret_cast<unsigned *>(&sB);
        for (int w = threadIdx.x; w < words; w += blockDim.x) dstw[w] = srcw[w];
    }
    __syncthreads();
    const BatchGrid &B = sB;
    PlaneArgs pa;
    const bool first = (round == 0);
    if (B.time_order == 1) {
        pa.stage = 0;
        pa.src = first ? B.l : ((round & 1) ? B.b : B.a);
        pa.dst = (round & 1) ? B.a : B.b;
        pa.prev = pa.src;
    } else if (phase == 0) {
        pa.stage = 1;
        pa.src = first ? B.l : B.a;
        pa.dst = B.b;
        pa.prev = pa.src;
    } else {
        pa.stage = 2;
        pa.src = B.b;
        pa.prev = first ? B.l : B.a;
        pa.dst = B.a;
    }
    pa.l = B.l;
    pa.gob = nullptr;
    pa.alpha_bits = B.alpha_bits;
    pa.dt = float(round == B.n_steps - 1 ? B.dt_last : B.dt_cfl);
    pa.brt = B.brt;
    pa.flags = &B.state->flags;
    plane_pass<ND, ORDER, DYN, false, -1, 0>(B.g, B.dy, pa, uint32_t(i - item_start[lo]));
}

template <int ND, int DYN>
static cudaError_t launch_plane_round(int order, int ctas, int threads, int smem, const BatchGrid *bg,
                                      const int *sorted, const int *item_start, int n, int round, int phase,
                                      cudaStream_t s)
{
    if (order == 1)
        k_batch_plane<ND, 1, DYN><<<ctas, threads, smem, s>>>(bg, sorted, item_start, n, round, phase);
    else
        k_batch_plane<ND, 2, DYN><<<ctas, threads, smem, s>>>(bg, sorted, item_start, n, round, phase);
    return cudaGetLastError();
}

// The dynamic shared memory the round launches need (set before capturing
// them: it is not a stream operation).
template <int ND, int DYN>
static cudaError_t set_plane_smem(int order, int smem)
{
    if (order == 1)
        return cudaFuncSetAttribute(k_batch_plane<ND, 1, DYN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return cudaFuncSetAttribute(k_batch_plane<ND, 2, DYN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

// Stream-axis chunks of up to `cap` planes (the parallelism of a batch comes
// from its many grids, so the single-solve geometry, which cuts finer, is
// recut).
static void plane_geometry_chunk(GridDesc &D, int cap)
{
    PlaneGeom &pg = D.pg;
    if (!pg.use) return;
    const int pencils = pg.items / (pg.nbands * pg.nchunks);
    pg.chunk = pg.ns < cap ? pg.ns : cap;
    pg.nchunks = (pg.ns + pg.chunk - 1) / pg.chunk;
    pg.items = pencils * pg.nbands * pg.nchunks;
    pg.div_nchunks = make_fastdiv(uint32_t(pg.nchunks));
}

void plane_geometry_many(GridDesc &D) { plane_geometry_chunk(D, 16); }

// The CUDA graph of a plane-path batch's per-round launches, kept for the
// batch signature it was captured for (the launch shapes and the workspace
// pointers its kernel arguments hold).
struct PlaneGraphKey {
    int kind = -1, order = 0, time_order = 0, n = 0, rounds = 0, chunk = 0, threads = 0, smem = 0;
    const void *bg = nullptr, *ints = nullptr;
    std::vector<int> active;   // CTAs of every launch
    bool operator==(const PlaneGraphKey &o) const
    {
        return kind == o.kind && order == o.order && time_order == o.time_order && n == o.n && rounds == o.rounds &&
               chunk == o.chunk && threads == o.threads && smem == o.smem && bg == o.bg && ints == o.ints &&
               active == o.active;
    }
};

struct BatchWorkspace {
    std::mutex mu;
    int device = -1;
    BatchGrid *bg = nullptr;
    int *ints = nullptr;
    BatchBarrier *bar = nullptr;
    size_t cap_grids = 0, cap_ints = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    PlaneGraphKey graph_key;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t cap_stream = nullptr;   // private stream the batch graph is captured on
    int cap_device = -1;
};

static BatchWorkspace &workspace()
{
    static BatchWorkspace w;
    return w;
}

template <int ORDER, int R>
static cudaError_t launch_run(int ctas, const BatchGrid *bg, const int *sorted, const int *item_start, int n,
                              const int *active, const int *active_rk2, int r0, int r1, BatchBarrier *bar,
                              cudaStream_t s)
{
    void *args[] = {(void *)&bg, (void *)&sorted, (void *)&item_start, (void *)&n, (void *)&active,
                    (void *)&active_rk2, (void *)&r0, (void *)&r1, (void *)&bar};
    return cudaLaunchCooperativeKernel((const void *)k_batch_run<ORDER, R>, dim3(ctas), dim3(256), args, 0, s);
}

template <int ORDER, int R>
static int max_ctas_per_sm()
{
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_run<ORDER, R>, 256, 0);
    return nb;
}

// Autotuned launch shape, cached per batch signature (scheme, rows per
// thread, total items): CTAs per SM from 1 to the occupancy limit, timed on
// the first rounds of the real batch.
struct TuneKey {
    int order, R, sms;
    long long items0;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(order, R, sms, items0) < std::tie(o.order, o.R, o.sms, o.items0);
    }
};

}  // namespace odp

#include <map>
#include <tuple>

using namespace odp;

#define ODP_TRY_CUDA(call)                                                                          \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return fail(e_ == cudaErrorMemoryAllocation ? ODP_ENOMEM : ODP_ECUDA, "%s: %s", #call, \
                        cudaGetErrorString(e_));                                                    \
    } while (0)

static std::map<TuneKey, int> g_tuned;
// plane-path batches: the tuned stream-chunk cap per batch signature
struct PlaneTuneKey {
    int kind, order, time_order, n, rounds;
    double nodes;
    bool operator<(const PlaneTuneKey &o) const
    {
        return std::tie(kind, order, time_order, n, rounds, nodes) <
               std::tie(o.kind, o.order, o.time_order, o.n, o.rounds, o.nodes);
    }
};
static std::map<PlaneTuneKey, int> g_plane_tuned;
static std::mutex g_tuned_mu;
static int g_tune_enabled = 1;

extern "C" odp_status odp_batch_set_autotune(int enabled)
{
    g_tune_enabled = enabled ? 1 : 0;
    return ODP_OK;
}

extern "C" odp_status odp_batch_solve(odp_grid *const *grids, int n, const double *T, odp_set set,
                                      int space_order, int time_order, double cfl, odp_batch_stats *stats)
{
    if (!grids || !T || n < 1) return fail(ODP_EINVAL, "need n >= 1 grids and horizons");
    if (set != ODP_BRS && set != ODP_BRT) return fail(ODP_EINVAL, "set must be ODP_BRS or ODP_BRT");
    if (space_order != 1 && space_order != 2) return fail(ODP_EINVAL, "space_order must be 1 or 2");
    if (time_order != 1 && time_order != 2) return fail(ODP_EINVAL, "time_order must be 1 or 2");
    if (!(cfl > 0.0 && cfl <= 1.0)) return fail(ODP_EINVAL, "cfl must lie in (0, 1]");
    const int device = grids[0] ? grids[0]->device : 0;
    int all_r4 = 1;
    for (int i = 0; i < n; ++i) {
        const odp_grid *g = grids[i];
        if (!g) return fail(ODP_EINVAL, "grid %d is NULL", i);
        if (!g->has_dyn || !g->has_target) return fail(ODP_ESTATE, "grid %d lacks dynamics or target", i);
        if (g->has_obst) return fail(ODP_EINVAL, "grid %d has an obstacle: the batched solve has no reach-avoid", i);
        if (g->l_seq_n) return fail(ODP_EINVAL, "grid %d has a target schedule: the batched solve takes one target", i);
        if (g->local_diss)
            return fail(ODP_EINVAL, "grid %d uses per-node dissipation: the batched solve uses the grid alpha", i);
        if (g->device != device) return fail(ODP_EINVAL, "grid %d is on another device", i);
        if (!(T[i] > 0.0) || !std::isfinite(T[i])) return fail(ODP_EINVAL, "horizon %d must be finite and > 0", i);
        const int k = g->dyn.kind;
        const bool ok = k == DYN_DUBINS3D || k == DYN_DUBINSCAR4D ||
                        (k == DYN_SINGLE_INT && (g->ndim == 2 || g->ndim == 3));
        if (!ok) return fail(ODP_EINVAL, "grid %d: the batched solve supports Dubins3D, DubinsCar4D and 2-3D "
                                         "single integrators", i);
        if (g->desc.R != 4) all_r4 = 0;
    }
    const int R = all_r4 ? 4 : 1;
    // Dubins3D or DubinsCar4D batches whose grids all take the plane pass run
    // it round by round; the others run the persistent row-blocked kernel
    const int kind0 = grids[0]->dyn.kind;
    bool plane = kind0 == DYN_DUBINS3D || kind0 == DYN_DUBINSCAR4D;
    for (int i = 0; i < n && plane; ++i)
        if (grids[i]->dyn.kind != kind0 || !grids[i]->desc.pg.use) plane = false;
    cudaStream_t s = grids[0]->stream;
    BatchWorkspace &W = workspace();
    std::lock_guard<std::mutex> lock(W.mu);
    ODP_TRY_CUDA(cudaSetDevice(device));

    // per-grid records
    std::vector<BatchGrid> hb(static_cast<size_t>(n));
    for (int i = 0; i < n; ++i) {
        odp_grid *g = grids[i];
        BatchGrid &B = hb[size_t(i)];
        memset(&B, 0, sizeof(B));
        B.g = g->desc;
        if (R == 1) {   // row-blocked geometry with one row per thread
            B.g.R = 1;
            B.g.row_groups = B.g.nr;
            B.g.nthreads_rb = B.g.segs * B.g.row_groups * B.g.planes;
            B.g.div_row_groups = make_fastdiv(uint32_t(B.g.row_groups));
        }
        B.dy = g->dyn;
        B.a = g->phi_a;
        B.b = g->phi_b;
        B.l = g->l;
        B.state = g->state;
        B.T = T[i];
        B.kind = g->dyn.kind;
        B.time_order = time_order;
        B.brt = set == ODP_BRT ? 1 : 0;
        B.items = (B.g.nthreads_rb + 255) / 256;
        if (plane) {
            plane_geometry_many(B.g);
            B.items = B.g.pg.items;
        }
    }
    if (size_t(n) > W.cap_grids || W.device != device) {
        cudaFree(W.bg);
        W.bg = nullptr;
        W.cap_grids = 0;
        ODP_TRY_CUDA(cudaMalloc(&W.bg, sizeof(BatchGrid) * size_t(n)));
        W.cap_grids = size_t(n);
    }
    if (!W.bar || W.device != device) {
        cudaFree(W.bar);
        W.bar = nullptr;
        ODP_TRY_CUDA(cudaMalloc(&W.bar, sizeof(BatchBarrier)));
        if (!W.ev0) cudaEventCreate(&W.ev0);
        if (!W.ev1) cudaEventCreate(&W.ev1);
    }
    W.device = device;
    ODP_TRY_CUDA(cudaMemcpyAsync(W.bg, hb.data(), sizeof(BatchGrid) * size_t(n), cudaMemcpyHostToDevice, s));
    k_batch_prepare<<<n, 256, 0, s>>>(W.bg, cfl);
    ODP_TRY_CUDA(cudaGetLastError());
    ODP_TRY_CUDA(cudaMemcpyAsync(hb.data(), W.bg, sizeof(BatchGrid) * size_t(n), cudaMemcpyDeviceToHost, s));
    ODP_TRY_CUDA(cudaStreamSynchronize(s));

    // items sorted by step count, active prefixes per round
    std::vector<int> sorted(static_cast<size_t>(n));
    std::iota(sorted.begin(), sorted.end(), 0);
    std::stable_sort(sorted.begin(), sorted.end(),
                     [&](int x, int y) { return hb[size_t(x)].n_steps > hb[size_t(y)].n_steps; });
    const int rounds = hb[size_t(sorted[0])].n_steps;
    std::vector<int> item_start(static_cast<size_t>(n) + 1, 0), active(static_cast<size_t>(rounds), 0),
        active_rk2(static_cast<size_t>(rounds), 0);
    for (int k = 0; k < n; ++k) item_start[size_t(k) + 1] = item_start[size_t(k)] + hb[size_t(sorted[size_t(k)])].items;
    {
        int k = n;
        for (int r = 0; r < rounds; ++r) {
            while (k > 0 && hb[size_t(sorted[size_t(k) - 1])].n_steps <= r) --k;
            active[size_t(r)] = item_start[size_t(k)];
            active_rk2[size_t(r)] = time_order == 2 ? active[size_t(r)] : 0;
        }
    }
    const size_t nints = size_t(n) + size_t(n) + 1 + 2 * size_t(rounds);
    if (nints > W.cap_ints) {
        cudaFree(W.ints);
        W.ints = nullptr;
        W.cap_ints = 0;
        ODP_TRY_CUDA(cudaMalloc(&W.ints, sizeof(int) * nints));
        W.cap_ints = nints;
    }
    std::vector<int> packed;
    packed.reserve(nints);
    packed.insert(packed.end(), sorted.begin(), sorted.end());
    packed.insert(packed.end(), item_start.begin(), item_start.end());
    packed.insert(packed.end(), active.begin(), active.end());
    packed.insert(packed.end(), active_rk2.begin(), active_rk2.end());
    ODP_TRY_CUDA(cudaMemcpyAsync(W.ints, packed.data(), sizeof(int) * nints, cudaMemcpyHostToDevice, s));
    const int *d_sorted = W.ints, *d_start = W.ints + n, *d_active = W.ints + 2 * n + 1;
    const int *d_active_rk2 = d_active + rounds;

    if (plane) {
        // The plane layout of the batch for a stream-chunk cap: every grid's
        // items, the item list, the active prefix of every launch; uploaded.
        int threads = 32, smem = 0, chunk = 16;
        std::vector<int> launch_ctas;
        auto apply = [&](int cap) -> cudaError_t {
            chunk = cap;
            threads = 32;
            smem = 0;
            for (int i = 0; i < n; ++i) {
                BatchGrid &B = hb[size_t(i)];
                B.g.pg = grids[i]->desc.pg;
                plane_geometry_chunk(B.g, cap);
                B.items = B.g.pg.items;
                threads = std::max(threads, B.g.pg.threads);
                smem = std::max(smem, B.g.pg.smem[space_order - 1]);
            }
            for (int k = 0; k < n; ++k)
                item_start[size_t(k) + 1] = item_start[size_t(k)] + hb[size_t(sorted[size_t(k)])].items;
            int k = n;
            launch_ctas.clear();
            for (int r = 0; r < rounds; ++r) {
                while (k > 0 && hb[size_t(sorted[size_t(k) - 1])].n_steps <= r) --k;
                active[size_t(r)] = item_start[size_t(k)];
                active_rk2[size_t(r)] = time_order == 2 ? active[size_t(r)] : 0;
                launch_ctas.push_back(active[size_t(r)]);
                if (time_order == 2) launch_ctas.push_back(active_rk2[size_t(r)]);
            }
            packed.clear();
            packed.insert(packed.end(), sorted.begin(), sorted.end());
            packed.insert(packed.end(), item_start.begin(), item_start.end());
            packed.insert(packed.end(), active.begin(), active.end());
            packed.insert(packed.end(), active_rk2.begin(), active_rk2.end());
            cudaError_t e = cudaMemcpyAsync(W.bg, hb.data(), sizeof(BatchGrid) * size_t(n), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(W.ints, packed.data(), sizeof(int) * nints, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = kind0 == DYN_DUBINS3D ? set_plane_smem<3, DYN_DUBINS3D>(space_order, smem)
                                                            : set_plane_smem<4, DYN_DUBINSCAR4D>(space_order, smem);
            return e;
        };
        auto launch_rounds = [&](int r1) -> cudaError_t {
            for (int r = 0; r < r1; ++r) {
                for (int phase = 0; phase < time_order; ++phase) {
                    const int ctas = phase == 0 ? active[size_t(r)] : active_rk2[size_t(r)];
                    if (ctas == 0) continue;
                    cudaError_t e = kind0 == DYN_DUBINS3D
                                        ? launch_plane_round<3, DYN_DUBINS3D>(space_order, ctas, threads, smem, W.bg,
                                                                              d_sorted, d_start, n, r, phase, s)
                                        : launch_plane_round<4, DYN_DUBINSCAR4D>(space_order, ctas, threads, smem,
                                                                                 W.bg, d_sorted, d_start, n, r, phase, s);
                    if (e != cudaSuccess) return e;
                }
            }
            return cudaSuccess;
        };

        // Autotuner: the stream-chunk cap (planes per CTA, which sets the
        // items per grid and so the CTAs of every launch), timed on the first
        // rounds of this batch and cached per batch signature.  Every probe
        // restarts from round 0, which reads the targets, so the probes
        // leave no trace in the solve.
        double nodes_all = 0.0;
        for (int i = 0; i < n; ++i) nodes_all += double(grids[i]->total);
        const PlaneTuneKey tkey{kind0, space_order, time_order, n, rounds, nodes_all};
        int best_cap = 16;
        bool have = false;
        {
            std::lock_guard<std::mutex> lk(g_tuned_mu);
            auto it = g_plane_tuned.find(tkey);
            if (it != g_plane_tuned.end()) {
                best_cap = it->second;
                have = true;
            }
        }
        bool tuned_now = false;
        if (!have && g_tune_enabled && rounds >= 2) {
            const int probe = std::min(rounds, 6);
            const int caps[4] = {8, 16, 32, 64};
            float best = 1e30f;
            for (int c = 0; c < 4; ++c) {
                ODP_TRY_CUDA(apply(caps[c]));
                if (c == 0) ODP_TRY_CUDA(launch_rounds(probe));   // warm the caches once
                for (int rep = 0; rep < 2; ++rep) {
                    ODP_TRY_CUDA(cudaEventRecord(W.ev0, s));
                    ODP_TRY_CUDA(launch_rounds(probe));
                    ODP_TRY_CUDA(cudaEventRecord(W.ev1, s));
                    ODP_TRY_CUDA(cudaEventSynchronize(W.ev1));
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, W.ev0, W.ev1);
                    if (ms < best) {
                        best = ms;
                        best_cap = caps[c];
                    }
                }
            }
            std::lock_guard<std::mutex> lk(g_tuned_mu);
            g_plane_tuned[tkey] = best_cap;
            tuned_now = true;
        }
        ODP_TRY_CUDA(apply(best_cap));

        // the whole batch as one CUDA graph of its per-round launches,
        // captured once per signature and replayed
        PlaneGraphKey gkey;
        gkey.kind = kind0;
        gkey.order = space_order;
        gkey.time_order = time_order;
        gkey.n = n;
        gkey.rounds = rounds;
        gkey.chunk = chunk;
        gkey.threads = threads;
        gkey.smem = smem;
        gkey.bg = W.bg;
        gkey.ints = W.ints;
        gkey.active = launch_ctas;
        bool captured_now = false;
        if (!W.graph_exec || !(W.graph_key == gkey)) {
            if (W.graph_exec) cudaGraphExecDestroy(W.graph_exec);
            W.graph_exec = nullptr;
            // captured on a private stream (the caller's may be the legacy
            // default stream, which cannot be captured), launched on the
            // caller's; the uploads above are ordered before the launch by s
            if (!W.cap_stream || W.cap_device != device) {
                if (W.cap_stream) cudaStreamDestroy(W.cap_stream);
                W.cap_stream = nullptr;
                ODP_TRY_CUDA(cudaStreamCreateWithFlags(&W.cap_stream, cudaStreamNonBlocking));
                W.cap_device = device;
            }
            cudaStream_t cs = W.cap_stream;
            std::swap(s, cs);   // launch_rounds issues on s
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) e = launch_rounds(rounds);
            cudaError_t e2 = cudaStreamEndCapture(s, &graph);
            std::swap(s, cs);
            if (e == cudaSuccess && e2 != cudaSuccess) e = e2;
            if (e != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();
                return fail(ODP_ECUDA, "capturing the batch's launches: %s", cudaGetErrorString(e));
            }
            e = cudaGraphInstantiate(&W.graph_exec, graph, 0);

            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                W.graph_exec = nullptr;
                return fail(ODP_ECUDA, "instantiating the batch graph: %s", cudaGetErrorString(e));
            }
            W.graph_key = gkey;
            captured_now = true;
        }
        ODP_TRY_CUDA(cudaEventRecord(W.ev0, s));
        ODP_TRY_CUDA(cudaGraphLaunch(W.graph_exec, s));
        ODP_TRY_CUDA(cudaEventRecord(W.ev1, s));
        k_batch_finish<<<(n + 127) / 128, 128, 0, s>>>(W.bg, n);
        ODP_TRY_CUDA(cudaGetLastError());
        ODP_TRY_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < n; ++i) {
            odp_grid *g = grids[i];
            g->solved = true;
            g->n_tau = 2;
            g->keep = 0;
            g->time_order = time_order;
            g->order = space_order;
            g->brt = set == ODP_BRT ? 1 : 0;
            g->timed = false;
        }
        if (stats) {
            memset(stats, 0, sizeof(*stats));
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, W.ev0, W.ev1);
            stats->device_ms = ms;
            stats->rounds = rounds;
            stats->ctas_per_sm = 0;       // one launch per round, occupancy by the hardware
            stats->rows_per_thread = 0;   // plane pass
            stats->plane_chunk = chunk;
            stats->launches = int64_t(launch_ctas.size());
            stats->graph = captured_now ? 1 : 2;
            stats->tuned = tuned_now ? 1 : 0;
            double updates = 0.0, bytes = 0.0;
            for (int i = 0; i < n; ++i) {
                const double nodes = double(grids[i]->total) * double(hb[size_t(i)].n_steps);
                updates += nodes;
                const double per = (time_order == 1 ? 8.0 : 20.0) + (set == ODP_BRT ? 4.0 : 0.0);
                bytes += per * nodes;
            }
            stats->point_updates = updates;
            stats->bytes = bytes;
        }
        return ODP_OK;
    }

    int sms = 0;
    ODP_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const int max_per_sm = space_order == 1 ? (R == 4 ? max_ctas_per_sm<1, 4>() : max_ctas_per_sm<1, 1>())
                                            : (R == 4 ? max_ctas_per_sm<2, 4>() : max_ctas_per_sm<2, 1>());
    if (max_per_sm < 1) return fail(ODP_ECUDA, "the batched kernel cannot be resident");
    auto run = [&](int per_sm, int r0, int r1) -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(W.bar, 0, sizeof(BatchBarrier), s);
        if (e != cudaSuccess) return e;
        const int ctas = per_sm * sms;
        if (space_order == 1)
            return R == 4 ? launch_run<1, 4>(ctas, W.bg, d_sorted, d_start, n, d_active, d_active_rk2, r0, r1, W.bar, s)
                          : launch_run<1, 1>(ctas, W.bg, d_sorted, d_start, n, d_active, d_active_rk2, r0, r1, W.bar, s);
        return R == 4 ? launch_run<2, 4>(ctas, W.bg, d_sorted, d_start, n, d_active, d_active_rk2, r0, r1, W.bar, s)
                      : launch_run<2, 1>(ctas, W.bg, d_sorted, d_start, n, d_active, d_active_rk2, r0, r1, W.bar, s);
    };

    // autotune the CTAs per SM on the first rounds of this batch
    TuneKey key{space_order, R, sms, item_start[size_t(n)]};
    int per_sm = max_per_sm;
    bool tuned = false;
    {
        std::lock_guard<std::mutex> lk(g_tuned_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            per_sm = std::min(it->second, max_per_sm);
            tuned = true;
        }
    }
    if (!tuned && g_tune_enabled && rounds >= 2) {
        // the first rounds (every grid active) once untimed to warm the
        // caches, then each occupancy twice; the faster of the two counts.
        // Every probe restarts from round 0, which reads the targets, so the
        // probes leave no trace in the solve.
        const int probe = std::min(rounds, 6);
        ODP_TRY_CUDA(run(max_per_sm, 0, probe));
        float best = 1e30f;
        for (int c = 1; c <= max_per_sm; ++c) {
            for (int rep = 0; rep < 2; ++rep) {
                ODP_TRY_CUDA(cudaEventRecord(W.ev0, s));
                ODP_TRY_CUDA(run(c, 0, probe));
                ODP_TRY_CUDA(cudaEventRecord(W.ev1, s));
                ODP_TRY_CUDA(cudaEventSynchronize(W.ev1));
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, W.ev0, W.ev1);
                if (ms < best) {
                    best = ms;
                    per_sm = c;
                }
            }
        }
        std::lock_guard<std::mutex> lk(g_tuned_mu);
        g_tuned[key] = per_sm;
    }

    ODP_TRY_CUDA(cudaEventRecord(W.ev0, s));
    ODP_TRY_CUDA(run(per_sm, 0, rounds));
    ODP_TRY_CUDA(cudaEventRecord(W.ev1, s));
    k_batch_finish<<<(n + 127) / 128, 128, 0, s>>>(W.bg, n);
    ODP_TRY_CUDA(cudaGetLastError());
    BatchBarrier hbar{};
    ODP_TRY_CUDA(cudaMemcpyAsync(&hbar, W.bar, sizeof(hbar), cudaMemcpyDeviceToHost, s));
    ODP_TRY_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < n; ++i) {
        odp_grid *g = grids[i];
        g->solved = true;
        g->n_tau = 2;
        g->keep = 0;
        g->time_order = time_order;
        g->order = space_order;
        g->brt = set == ODP_BRT ? 1 : 0;
        g->timed = false;
    }
    if (hbar.flags) return fail(ODP_ECUDA, "a grid-wide barrier of the batched solve gave up waiting");
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, W.ev0, W.ev1);
        stats->device_ms = ms;
        stats->rounds = rounds;
        stats->ctas_per_sm = per_sm;
        stats->rows_per_thread = R;
        double updates = 0.0, bytes = 0.0;
        for (int i = 0; i < n; ++i) {
            const double nodes = double(grids[i]->total) * double(hb[size_t(i)].n_steps);
            updates += nodes;
            const double per = (time_order == 1 ? 8.0 : 20.0) + (set == ODP_BRT ? 4.0 : 0.0);
            bytes += per * nodes;
        }
        stats->point_updates = updates;
        stats->bytes = bytes;
    }
    return ODP_OK;
}

// ===========================================================================
// Allocation-free single solve (odp_solve_noalloc)
//
// Some callers cannot allocate device memory at the point where they need a
// solve: code that runs inside a memory pool or arena it does not own (a
// framework's caching allocator, a serving process whose HBM is partitioned
// up front), or code that must not call cudaMalloc/cudaFree because those
// calls synchronise the whole device.  This entry point serves them: the
// caller passes the target and the output as device buffers, and everything
// else the solve needs (the two value buffers, the target copy, node tables,
// the batch record, the barrier, the solve state) lives in one file-scope
// device array of fixed size.  It runs the same persistent batched kernel as
// odp_batch_solve on a single grid, so its result equals odp_solve_hjb's.
//
// The array is held by every GPU that loads the library until the process
// exits.  All calls share it and it keeps the last call's contents: each call
// clears what must start at zero (barrier, flags, target padding), and calls
// whose GPU work overlaps (for example on two streams) race on it.
// ===========================================================================

namespace odp {

constexpr size_t kNoallocBytes = size_t(16) << 20;   // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// One grid's rounds from the solve's own step count (read on the device).
template <int ORDER, int R>
__global__ void __launch_bounds__(256) k_noalloc_run(BatchGrid *bg, BatchBarrier *bar)
{
    __shared__ BatchGrid sB;
    {
        const int words = int(sizeof(BatchGrid) / 4);
        const unsigned *srcw = reinterpret_cast<const unsigned *>(bg);
        unsigned *dstw = reinterpret_cast<unsigned *>(&sB);
        for (int w = threadIdx.x; w < words; w += blockDim.x) dstw[w] = srcw[w];
    }
    __syncthreads();
    unsigned gen = 0;
    const int phases = sB.time_order == 2 ? 2 : 1;
    for (int r = 0; r < sB.n_steps; ++r) {
        for (int phase = 0; phase < phases; ++phase) {
            for (int i = blockIdx.x; i < sB.items; i += gridDim.x)
                if (batch_item<ORDER, R>(sB, i, r, phase)) atomicOr(&sB.state->flags, FLAG_NONFINITE);
            if (!grid_barrier(bar, gen)) return;
        }
    }
}

// Copy the final value (a or b by step parity) into the caller's dense output.
__global__ void k_noalloc_out(const BatchGrid *bg, float *out)
{
    const BatchGrid &B = *bg;
    const float *src = ((B.time_order == 1) && (B.n_steps & 1)) ? B.b : B.a;
    const int nl = B.g.n[B.g.ndim - 1], npad = B.g.n_pad;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B.g.total; i += gridDim.x * blockDim.x) {
        const int row = i / nl, c = i - row * nl;
        out[i] = src[row * npad + c];
    }
}

constexpr int kNoallocMaxDevices = 64;

// Per device: the array's device address (looked up on the first call) and
// a lock held for the whole call, so calls on one device run one after
// another and calls on different devices do not wait for each other.
struct NoallocDevice {
    std::mutex mu[kNoallocMaxDevices];
    unsigned char *base[kNoallocMaxDevices] = {nullptr};
};

static NoallocDevice &noalloc_devices()
{
    static NoallocDevice d;
    return d;
}

}  // namespace odp

extern "C" odp_status odp_solve_noalloc(int ndim, const int32_t *n, const double *lo, const double *hi,
                                        const uint8_t *periodic, odp_dyn kind, const double *params, int n_params,
                                        odp_mode u_mode, odp_mode d_mode, const float *l, double T, odp_set set,
                                        int space_order, int time_order, double cfl, float *out, void *cuda_stream)
{
    if (ndim < 2 || ndim > 4 || !n || !lo || !hi || !periodic || !l || !out)
        return fail(ODP_EINVAL, "odp_solve_noalloc: bad arguments (2 to 4 dimensions, device l and out)");
    if (!(T > 0.0) || !std::isfinite(T)) return fail(ODP_EINVAL, "odp_solve_noalloc: T must be finite and > 0");
    if (set != ODP_BRS && set != ODP_BRT) return fail(ODP_EINVAL, "odp_solve_noalloc: set must be BRS or BRT");
    if ((space_order != 1 && space_order != 2) || (time_order != 1 && time_order != 2))
        return fail(ODP_EINVAL, "odp_solve_noalloc: orders must be 1 or 2");
    if (!(cfl > 0.0 && cfl <= 1.0)) return fail(ODP_EINVAL, "odp_solve_noalloc: cfl must lie in (0, 1]");
    if ((u_mode != ODP_MIN && u_mode != ODP_MAX) || (d_mode != ODP_MIN && d_mode != ODP_MAX))
        return fail(ODP_EINVAL, "odp_solve_noalloc: modes must be ODP_MIN or ODP_MAX");
    int need = 0, angle = -1;
    if (kind == ODP_DYN_DUBINS3D && ndim == 3) {
        need = 2;
        angle = 2;
    } else if (kind == ODP_DYN_DUBINSCAR4D && ndim == 4) {
        need = 2;
        angle = 3;
    } else if (kind == ODP_DYN_SINGLE_INT && (ndim == 2 || ndim == 3)) {
        need = 1;
    } else {
        return fail(ODP_EINVAL, "odp_solve_noalloc: supports Dubins3D, DubinsCar4D and the 2-3D single integrator");
    }
    if (!params || n_params < need || n_params > 8) return fail(ODP_EINVAL, "odp_solve_noalloc: missing parameters");
    for (int k = 0; k < n_params; ++k)
        if (!std::isfinite(params[k]) || params[k] < 0.0)
            return fail(ODP_EINVAL, "odp_solve_noalloc: parameter %d must be finite and >= 0", k);
    if (angle >= 0 && !periodic[angle]) return fail(ODP_EINVAL, "odp_solve_noalloc: the angle axis must be periodic");

    // grid description (row-blocked pass; same rules as odp_grid_create)
    GridDesc D{};
    D.ndim = ndim;
    int64_t total = 1;
    for (int d = 0; d < ndim; ++d) {
        if (n[d] < (periodic[d] ? 1 : 2) || !(hi[d] > lo[d]) || !std::isfinite(lo[d]) || !std::isfinite(hi[d]))
            return fail(ODP_EINVAL, "odp_solve_noalloc: bad axis %d", d);
        total *= n[d];
        if (total >= (int64_t(1) << 31)) return fail(ODP_EINVAL, "odp_solve_noalloc: grid has 2^31 nodes or more");
    }
    if (total / n[ndim - 1] * ((n[ndim - 1] + 3) / 4 * 4) >= (int64_t(1) << 31))
        return fail(ODP_EINVAL, "odp_solve_noalloc: padded grid storage has 2^31 floats or more");
    const int nl = n[ndim - 1], npad = (nl + 3) / 4 * 4;
    const int64_t rows = total / nl, total_pad = rows * npad;
    int64_t tab_len = 0;
    for (int d = 0; d < ndim; ++d) tab_len += 3 * int64_t((n[d] + 3) / 4 * 4);
    const size_t rec = (sizeof(BatchGrid) + 255) / 256 * 256;
    const size_t barb = 256, stb = (sizeof(SolveState) + 255) / 256 * 256;
    const size_t tabb = (size_t(tab_len) * 4 + 255) / 256 * 256;
    const size_t arrb = (size_t(total_pad) * 4 + 255) / 256 * 256;
    const size_t bytes = rec + barb + stb + tabb + 3 * arrb;
    if (bytes > kNoallocBytes)
        return fail(ODP_EINVAL, "odp_solve_noalloc: the grid needs %zu bytes of scratch, the fixed limit is %zu "
                                "(about %lld nodes)", bytes, kNoallocBytes, (long long)(kNoallocBytes / 12));

    int device = 0, caller_device = 0;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the call copies from host memory and synchronises its stream, so it
    // cannot be recorded into a CUDA graph: checked before any other CUDA
    // call, so that a refused call leaves the caller's capture intact
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    ODP_TRY_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone)
        return fail(ODP_EINVAL, "odp_solve_noalloc: the stream is capturing; this call cannot be captured");
    ODP_TRY_CUDA(cudaGetDevice(&caller_device));
    if (s) ODP_TRY_CUDA(cudaStreamGetDevice(s, &device));
    else device = caller_device;
    if (device < 0 || device >= kNoallocMaxDevices)
        return fail(ODP_EINVAL, "odp_solve_noalloc: device %d out of range", device);
    // the caller's current device is restored on every return
    struct DeviceRestore {
        int dev;
        ~DeviceRestore() { cudaSetDevice(dev); }
    } restore{caller_device};
    ODP_TRY_CUDA(cudaSetDevice(device));
    NoallocDevice &ND = noalloc_devices();
    std::lock_guard<std::mutex> lock(ND.mu[device]);
    if (!ND.base[device]) {
        // set-up, once per device, with that device current: the array's
        // device address (its host-side name is not a device address)
        void *ptr = nullptr;
        ODP_TRY_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
        ND.base[device] = static_cast<unsigned char *>(ptr);
    }
    unsigned char *base = ND.base[device];
    BatchGrid *d_rec = reinterpret_cast<BatchGrid *>(base);
    BatchBarrier *d_bar = reinterpret_cast<BatchBarrier *>(base + rec);
    SolveState *d_state = reinterpret_cast<SolveState *>(base + rec + barb);
    float *d_tab = reinterpret_cast<float *>(base + rec + barb + stb);
    float *d_l = reinterpret_cast<float *>(base + rec + barb + stb + tabb);
    float *d_a = reinterpret_cast<float *>(base + rec + barb + stb + tabb + arrb);
    float *d_b = reinterpret_cast<float *>(base + rec + barb + stb + tabb + 2 * arrb);

    // tables: node coordinates, cos and sin per axis (float64 rounded once)
    std::vector<float> tab(static_cast<size_t>(tab_len), 0.0f);
    int64_t off = 0;
    for (int d = 0; d < ndim; ++d) {
        const double h = periodic[d] ? (hi[d] - lo[d]) / double(n[d]) : (hi[d] - lo[d]) / double(n[d] - 1);
        const int64_t np = (n[d] + 3) / 4 * 4;
        D.n[d] = n[d];
        D.periodic[d] = periodic[d] ? 1 : 0;
        D.dz[d] = h;
        D.inv_dz[d] = float(1.0 / h);
        D.div[d] = make_fastdiv(uint32_t(n[d]));
        D.coord[d] = d_tab + off;
        for (int i = 0; i < n[d]; ++i) {
            const double z = lo[d] + double(i) * h;
            tab[size_t(off + i)] = float(z);
            tab[size_t(off + np + i)] = float(std::cos(z));
            tab[size_t(off + 2 * np + i)] = float(std::sin(z));
        }
        if (d == angle) {
            D.cos_tab = d_tab + off + np;
            D.sin_tab = d_tab + off + 2 * np;
        }
        off += 3 * np;
    }
    D.total = int(total);
    D.n_pad = npad;
    D.rows = int(rows);
    D.segs = npad / 4;
    D.nthreads = int(rows * D.segs);
    D.div_segs = make_fastdiv(uint32_t(D.segs));
    int64_t st = 1;
    for (int d = ndim - 1; d >= 0; --d) {
        D.stride[d] = int(st);
        st *= (d == ndim - 1) ? npad : n[d];
    }
    D.nr = n[ndim - 2];
    D.R = D.nr >= 4 ? 4 : 1;
    D.row_groups = (D.nr + D.R - 1) / D.R;
    D.planes = int(rows / D.nr);
    D.nthreads_rb = D.segs * D.row_groups * D.planes;
    D.div_row_groups = make_fastdiv(uint32_t(D.row_groups));

    BatchGrid hb;
    memset(&hb, 0, sizeof(hb));
    hb.g = D;
    hb.dy.kind = int(kind);
    hb.dy.umode = int(u_mode);
    hb.dy.dmode = int(d_mode);
    hb.dy.angle_axis = angle;
    for (int k = 0; k < n_params; ++k) hb.dy.prm[k] = float(params[k]);
    hb.a = d_a;
    hb.b = d_b;
    hb.l = d_l;
    hb.state = d_state;
    hb.T = T;
    hb.kind = int(kind);
    hb.time_order = time_order;
    hb.brt = set == ODP_BRT ? 1 : 0;
    hb.items = (D.nthreads_rb + 255) / 256;

    // upload (pageable sources are staged at once) and clear what starts at zero
    ODP_TRY_CUDA(cudaMemcpyAsync(d_rec, &hb, sizeof(hb), cudaMemcpyHostToDevice, s));
    ODP_TRY_CUDA(cudaMemcpyAsync(d_tab, tab.data(), size_t(tab_len) * 4, cudaMemcpyHostToDevice, s));
    ODP_TRY_CUDA(cudaMemsetAsync(d_bar, 0, sizeof(BatchBarrier), s));
    ODP_TRY_CUDA(cudaMemsetAsync(d_state, 0, sizeof(SolveState), s));
    ODP_TRY_CUDA(cudaMemsetAsync(d_l, 0, size_t(total_pad) * 4, s));
    ODP_TRY_CUDA(cudaMemcpy2DAsync(d_l, size_t(npad) * 4, l, size_t(nl) * 4, size_t(nl) * 4, size_t(rows),
                                   cudaMemcpyDeviceToDevice, s));
    k_batch_prepare<<<1, 256, 0, s>>>(d_rec, cfl);
    ODP_TRY_CUDA(cudaGetLastError());

    int sms = 0, per_sm = 0;
    ODP_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const void *fn = space_order == 1 ? (D.R == 4 ? (const void *)k_noalloc_run<1, 4> : (const void *)k_noalloc_run<1, 1>)
                                      : (D.R == 4 ? (const void *)k_noalloc_run<2, 4> : (const void *)k_noalloc_run<2, 1>);
    ODP_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0));
    if (per_sm < 1) return fail(ODP_ECUDA, "odp_solve_noalloc: the kernel cannot be resident");
    int ctas = per_sm * sms;
    if (ctas > hb.items) ctas = hb.items;
    void *args[] = {(void *)&d_rec, (void *)&d_bar};
    ODP_TRY_CUDA(cudaLaunchCooperativeKernel(fn, dim3(ctas), dim3(256), args, 0, s));
    k_noalloc_out<<<int(std::min<int64_t>((total + 255) / 256, 1024)), 256, 0, s>>>(d_rec, out);
    ODP_TRY_CUDA(cudaGetLastError());
    int flags[2] = {0, 0};
    ODP_TRY_CUDA(cudaMemcpyAsync(&flags[0], &d_state->flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    ODP_TRY_CUDA(cudaMemcpyAsync(&flags[1], &d_bar->flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    ODP_TRY_CUDA(cudaStreamSynchronize(s));
    if (flags[1]) return fail(ODP_ECUDA, "odp_solve_noalloc: a grid-wide barrier gave up waiting");
    if (flags[0] & FLAG_NONFINITE) return fail(ODP_ENUMERIC, "odp_solve_noalloc: a non-finite value appeared");
    return ODP_OK;
}
