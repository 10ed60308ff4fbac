// server.cu -- the serving loop: continuous batching of reachability solves
// under an HBM budget (odp_server_*).
//
// Requests of different grid shapes and dynamics are queued by
// odp_server_submit.  Every call of odp_server_step
//   1. admits queued requests in arrival order while their arrays fit in the
//      HBM budget (one arena allocated once at creation, first-fit blocks),
//      uploads their targets and computes their alpha and step schedules,
//   2. advances every resident solve by up to `rounds` of its own time steps
//      in one persistent cooperative launch (the batched kernel of batch.cu,
//      with per-solve step offsets and per-item scheme), and
//   3. retires the solves that reached their horizon: their values stay in
//      HBM until the client reads them back and releases them.
// Solves admitted while others are on the GPU join the next launch, so the
// batch composition changes between launches (continuous batching).  Each
// solve takes exactly the steps and per-node arithmetic of a single
// odp_solve_hjb over tau = {0, T}.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "hj_kernels.cuh"
#include "odp_internal.h"
#include "odp_time.cuh"

namespace odp {

// One resident solve as the persistent kernel sees it.
struct ServeGrid {
    GridDesc g;
    DynDesc dy;
    float *a, *b;
    const float *l;
    int *flags;
    double T, dt_cfl, dt_last;
    int n_steps, step0;       // total steps, steps taken before this launch
    int kind, order, time_order, brt, items;
    unsigned alpha_bits[8];
    float cD[ODP_MAXD];
};

struct ServeBarrier {
    unsigned arrive;
    unsigned gen;
    int flags;
};

// static alpha and step schedule of the newly admitted solves (one CTA each)
template <int DYN, int ND>
__device__ void serve_alpha(const GridDesc &g, const DynDesc &dy, float *a)
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

__global__ void __launch_bounds__(256) k_serve_prepare(ServeGrid *sg, const int *which, double *cfl)
{
    __shared__ float red[8][ODP_MAXD];
    ServeGrid &B = sg[which[blockIdx.x]];
    float a[ODP_MAXD];
    for (int d = 0; d < ODP_MAXD; ++d) a[d] = 0.0f;
    switch (B.kind) {
    case DYN_DUBINS3D: serve_alpha<DYN_DUBINS3D, 3>(B.g, B.dy, a); break;
    case DYN_DUBINSCAR4D: serve_alpha<DYN_DUBINSCAR4D, 4>(B.g, B.dy, a); break;
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
        const double dt_cfl = cfl_dt(B.alpha_bits, B.g.dz, nd, cfl[which[blockIdx.x]]);
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
        *B.flags = 0;
    }
}

__device__ __forceinline__ unsigned serve_ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ bool serve_barrier(ServeBarrier *bar, unsigned &gen)
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
            while (serve_ld_acquire(&bar->gen) < target) {
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
__device__ bool serve_item_t(const ServeGrid &B, const StageArgs &A, uint32_t t)
{
    switch (B.kind) {
    case DYN_DUBINS3D: return stage_tile<3, ORDER, DYN_DUBINS3D, R>(B.g, B.dy, A, t);
    case DYN_DUBINSCAR4D: return stage_tile<4, ORDER, DYN_DUBINSCAR4D, R>(B.g, B.dy, A, t);
    default: return false;
    }
}

template <int R>
__device__ bool serve_item(const ServeGrid &B, int blk, int step, int phase)
{
    const uint32_t t = uint32_t(blk) * blockDim.x + threadIdx.x;
    if (t >= uint32_t(B.g.nthreads_rb)) return false;
    StageArgs A;
    const bool first = (step == 0);
    if (B.time_order == 1) {
        A.stage = 0;
        A.src = first ? B.l : ((step & 1) ? B.b : B.a);
        A.dst = (step & 1) ? B.a : B.b;
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
    A.dt = float(step == B.n_steps - 1 ? B.dt_last : B.dt_cfl);
    for (int d = 0; d < ODP_MAXD; ++d) A.cD[d] = B.cD[d];
    return B.order == 1 ? serve_item_t<1, R>(B, A, t) : serve_item_t<2, R>(B, A, t);
}

// Rounds 0 .. rounds-1 of this launch: solve g takes its step step0 + r while
// it has steps left.  Solves are sorted by remaining steps, so round r's
// items are a prefix of the item list.  Phase 1 (TVD-RK2 stage 2) walks the
// same prefix and skips the items of Euler solves.
template <int R>
__global__ void __launch_bounds__(256) k_serve_run(const ServeGrid *__restrict__ sg, const int *__restrict__ sorted,
                                                   const int *__restrict__ item_start, int n,
                                                   const int *__restrict__ active, int any_rk2, int rounds,
                                                   ServeBarrier *bar)
{
    __shared__ ServeGrid sB;
    unsigned gen = 0;
    for (int r = 0; r < rounds; ++r) {
        for (int phase = 0; phase < (any_rk2 ? 2 : 1); ++phase) {
            const int items = active[r];
            for (int i = blockIdx.x; i < items; i += gridDim.x) {
                int lo = 0, hi = n - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (item_start[mid] <= i) lo = mid; else hi = mid - 1;
                }
                {
                    const int words = int(sizeof(ServeGrid) / 4);
                    const unsigned *srcw = reinterpret_cast<const unsigned *>(sg + sorted[lo]);
                    unsigned *dstw = reinterpret_cast<unsigned *>(&sB);
                    for (int w = threadIdx.x; w < words; w += blockDim.x) dstw[w] = srcw[w];
                }
                __syncthreads();
                if (!(phase == 1 && sB.time_order != 2)) {
                    if (serve_item<R>(sB, i - item_start[lo], sB.step0 + r, phase)) atomicOr(sB.flags, FLAG_NONFINITE);
                }
                __syncthreads();
            }
            if (!serve_barrier(bar, gen)) return;
        }
    }
}

// The plane-streaming pass over the active solves of one class (model, space
// order, time order) in round `round` of a serving step: solve g takes its
// step step0 + round.  The same per-node arithmetic as the single solve.
template <int ND, int ORDER, int DYN>
__global__ void __launch_bounds__(512) __maxnreg__(((ND == 3 && ORDER == 1) ? 80 : plane_max_regs<ND, ORDER, DYN>()))
    k_serve_plane(const ServeGrid *__restrict__ sg, const int *__restrict__ members,
                  const int *__restrict__ item_start, int n, int round, int phase)
{
    __shared__ ServeGrid sB;
    const int i = blockIdx.x;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (item_start[mid] <= i) lo = mid; else hi = mid - 1;
    }
    {
        const int words = int(sizeof(ServeGrid) / 4);
        const unsigned *srcw = reinterpret_cast<const unsigned *>(sg + members[lo]);
        unsigned *dstw = reinterpret_cast<unsigned *>(&sB);
        for (int w = threadIdx.x; w < words; w += blockDim.x) dstw[w] = srcw[w];
    }
    __syncthreads();
    const ServeGrid &B = sB;
    const int step = B.step0 + round;
    const bool first = (step == 0);
    PlaneArgs pa;
    if (B.time_order == 1) {
        pa.stage = 0;
        pa.src = first ? B.l : ((step & 1) ? B.b : B.a);
        pa.dst = (step & 1) ? B.a : B.b;
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
    pa.dt = float(step == B.n_steps - 1 ? B.dt_last : B.dt_cfl);
    pa.brt = B.brt;
    pa.flags = B.flags;
    plane_pass<ND, ORDER, DYN, false, -1, 0>(B.g, B.dy, pa, uint32_t(i - item_start[lo]));
}

template <int ND, int DYN>
static cudaError_t launch_serve_plane(int order, int ctas, int threads, int smem, const ServeGrid *sg,
                                      const int *members, const int *item_start, int n, int round, int phase,
                                      cudaStream_t s)
{
    if (order == 1) {
        cudaError_t e = cudaFuncSetAttribute(k_serve_plane<ND, 1, DYN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smem);
        if (e != cudaSuccess) return e;
        k_serve_plane<ND, 1, DYN><<<ctas, threads, smem, s>>>(sg, members, item_start, n, round, phase);
    } else {
        cudaError_t e = cudaFuncSetAttribute(k_serve_plane<ND, 2, DYN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smem);
        if (e != cudaSuccess) return e;
        k_serve_plane<ND, 2, DYN><<<ctas, threads, smem, s>>>(sg, members, item_start, n, round, phase);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// device arena: first-fit blocks inside one allocation made at creation
// ---------------------------------------------------------------------------
class Arena {
  public:
    explicit Arena(size_t bytes) : size_(bytes) { free_[0] = bytes; }
    // offset of a block of `bytes` (256-byte aligned), or SIZE_MAX
    size_t take(size_t bytes)
    {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                used_ += bytes;
                return off;
            }
        }
        return SIZE_MAX;
    }
    void give(size_t off, size_t bytes)
    {
        bytes = (bytes + 255) / 256 * 256;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t size() const { return size_; }

  private:
    size_t size_, used_ = 0;
    std::map<size_t, size_t> free_;
};

}  // namespace odp

using namespace odp;

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t id = 0;
    int state = 0;            // ODP_REQ_*
    odp_status error = ODP_OK;
    // description
    int ndim = 0;
    int32_t n[ODP_MAXD] = {0};
    double lo[ODP_MAXD] = {0}, hi[ODP_MAXD] = {0};
    uint8_t periodic[ODP_MAXD] = {0};
    int kind = 0, umode = 0, dmode = 0, n_params = 0;
    double params[8] = {0};
    double T = 0, cfl = 0.8;
    int set = 1, order = 1, time_order = 1;
    std::vector<float> target;
    // resident
    size_t off = SIZE_MAX, bytes = 0;
    ServeGrid rec{};
    int n_steps = 0, done_steps = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
};

}  // namespace

struct odp_server {
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t budget = 0;
    unsigned char *base = nullptr;   // the arena's allocation
    Arena *arena = nullptr;
    uint64_t next_id = 1;
    std::map<uint64_t, Request> reqs;
    std::deque<uint64_t> queue;
    std::vector<uint64_t> resident;   // admitted and not finished
    // device work tables
    ServeGrid *d_rec = nullptr;
    int *d_ints = nullptr;
    double *d_cfl = nullptr;
    ServeBarrier *d_bar = nullptr;
    int *d_flags = nullptr;            // one flag word per record slot
    size_t cap_rec = 0, cap_ints = 0;
    int per_sm = 0, sms = 0;
    int64_t launches = 0;
    int64_t max_nodes = 0;             // resident-node cap (0: none)
    std::mutex mu;
};

#define ODP_SRV_CUDA(call)                                                                          \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return fail(e_ == cudaErrorMemoryAllocation ? ODP_ENOMEM : ODP_ECUDA, "%s: %s", #call, \
                        cudaGetErrorString(e_));                                                    \
    } while (0)

static size_t request_bytes(const Request &r, size_t *tab_floats, size_t *arr_floats)
{
    int64_t total = 1;
    for (int d = 0; d < r.ndim; ++d) total *= r.n[d];
    const int nl = r.n[r.ndim - 1], npad = (nl + 3) / 4 * 4;
    const int64_t total_pad = total / nl * npad;
    size_t tab = 0;
    for (int d = 0; d < r.ndim; ++d) tab += 3 * size_t((r.n[d] + 3) / 4 * 4);
    *tab_floats = (tab + 63) / 64 * 64;
    *arr_floats = (size_t(total_pad) + 63) / 64 * 64;
    return (*tab_floats + 3 * *arr_floats) * 4;
}

// Row-blocked geometry and node tables of a request (the rules of
// odp_grid_create), its arrays placed at `block` in the arena.
static void describe(Request &r, float *block, size_t tab_floats, size_t arr_floats, std::vector<float> &tab)
{
    GridDesc &D = r.rec.g;
    D = GridDesc{};
    const int ndim = r.ndim;
    D.ndim = ndim;
    int64_t total = 1;
    for (int d = 0; d < ndim; ++d) total *= r.n[d];
    const int nl = r.n[ndim - 1], npad = (nl + 3) / 4 * 4;
    const int64_t rows = total / nl;
    float *d_tab = block;
    tab.assign(tab_floats, 0.0f);
    int64_t off = 0;
    const int angle = r.kind == ODP_DYN_DUBINS3D ? 2 : (r.kind == ODP_DYN_DUBINSCAR4D ? 3 : -1);
    for (int d = 0; d < ndim; ++d) {
        const int nd = r.n[d];
        const double h = r.periodic[d] ? (r.hi[d] - r.lo[d]) / double(nd) : (r.hi[d] - r.lo[d]) / double(nd - 1);
        const int64_t np = (nd + 3) / 4 * 4;
        D.n[d] = nd;
        D.periodic[d] = r.periodic[d] ? 1 : 0;
        D.dz[d] = h;
        D.inv_dz[d] = float(1.0 / h);
        D.div[d] = make_fastdiv(uint32_t(nd));
        D.coord[d] = d_tab + off;
        for (int i = 0; i < nd; ++i) {
            const double z = r.lo[d] + double(i) * h;
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
        st *= (d == ndim - 1) ? npad : r.n[d];
    }
    D.nr = r.n[ndim - 2];
    D.R = 4;
    D.row_groups = (D.nr + 3) / 4;
    D.planes = int(rows / D.nr);
    D.nthreads_rb = D.segs * D.row_groups * D.planes;
    D.div_row_groups = make_fastdiv(uint32_t(D.row_groups));
    plane_geometry(D, 152);
    plane_geometry_many(D);
    DynDesc &dy = r.rec.dy;
    dy = DynDesc{};
    dy.kind = r.kind;
    dy.umode = r.umode;
    dy.dmode = r.dmode;
    dy.angle_axis = angle;
    for (int k = 0; k < r.n_params; ++k) dy.prm[k] = float(r.params[k]);
    r.rec.l = block + tab_floats;
    r.rec.a = block + tab_floats + arr_floats;
    r.rec.b = block + tab_floats + 2 * arr_floats;
    r.rec.T = r.T;
    r.rec.kind = r.kind;
    r.rec.order = r.order;
    r.rec.time_order = r.time_order;
    r.rec.brt = r.set == ODP_BRT ? 1 : 0;
    r.rec.items = (D.nthreads_rb + 255) / 256;
}

extern "C" odp_status odp_server_create(size_t hbm_budget_bytes, void *cuda_stream, odp_server **out)
{
    if (!out) return fail(ODP_EINVAL, "out is NULL");
    *out = nullptr;
    if (hbm_budget_bytes < 4096) return fail(ODP_EINVAL, "the HBM budget must be at least 4 KiB");
    odp_server *s = new (std::nothrow) odp_server();
    if (!s) return fail(ODP_ENOMEM, "host allocation failed");
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = s->stream ? cudaStreamGetDevice(s->stream, &s->device) : cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaSetDevice(s->device);
    if (e == cudaSuccess) e = cudaMalloc(&s->base, hbm_budget_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_bar, sizeof(ServeBarrier));
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s->per_sm, k_serve_run<4>, 256, 0);
    if (e != cudaSuccess) {
        cudaFree(s->base);
        cudaFree(s->d_bar);
        delete s;
        return fail(e == cudaErrorMemoryAllocation ? ODP_ENOMEM : ODP_ECUDA, "creating the server: %s",
                    cudaGetErrorString(e));
    }
    s->budget = hbm_budget_bytes;
    s->arena = new Arena(hbm_budget_bytes);
    *out = s;
    return ODP_OK;
}

extern "C" odp_status odp_server_destroy(odp_server *s)
{
    if (!s) return ODP_OK;
    cudaSetDevice(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    else cudaDeviceSynchronize();
    cudaFree(s->base);
    cudaFree(s->d_rec);
    cudaFree(s->d_ints);
    cudaFree(s->d_cfl);
    cudaFree(s->d_bar);
    cudaFree(s->d_flags);
    delete s->arena;
    delete s;
    return ODP_OK;
}

extern "C" odp_status odp_server_submit(odp_server *s, const odp_request *q, uint64_t *req_id)
{
    if (!s || !q || !req_id) return fail(ODP_EINVAL, "NULL argument");
    const int nd = q->ndim;
    const bool d3 = q->kind == ODP_DYN_DUBINS3D && nd == 3, d4 = q->kind == ODP_DYN_DUBINSCAR4D && nd == 4;
    if (!d3 && !d4) return fail(ODP_EINVAL, "the server runs Dubins3D (3-D) and DubinsCar4D (4-D) requests");
    if (!q->target) return fail(ODP_EINVAL, "the request has no target");
    if (!(q->T > 0.0) || !std::isfinite(q->T)) return fail(ODP_EINVAL, "T must be finite and > 0");
    if (!(q->cfl > 0.0 && q->cfl <= 1.0)) return fail(ODP_EINVAL, "cfl must lie in (0, 1]");
    if ((q->space_order != 1 && q->space_order != 2) || (q->time_order != 1 && q->time_order != 2))
        return fail(ODP_EINVAL, "orders must be 1 or 2");
    if (q->n_params < 2 || q->n_params > 8) return fail(ODP_EINVAL, "the model needs 2 parameters");
    int64_t total = 1;
    for (int d = 0; d < nd; ++d) {
        if (q->n[d] < (q->periodic[d] ? 1 : 2) || !(q->hi[d] > q->lo[d])) return fail(ODP_EINVAL, "bad axis %d", d);
        total *= q->n[d];
    }
    if (q->n[nd - 2] < 4) return fail(ODP_EINVAL, "the second-last axis needs at least 4 nodes");
    if (!q->periodic[nd - 1]) return fail(ODP_EINVAL, "the angle axis must be periodic");
    for (int k = 0; k < q->n_params; ++k)
        if (!(q->params[k] >= 0.0) || !std::isfinite(q->params[k])) return fail(ODP_EINVAL, "bad parameter %d", k);
    Request r;
    r.ndim = nd;
    for (int d = 0; d < nd; ++d) {
        r.n[d] = q->n[d];
        r.lo[d] = q->lo[d];
        r.hi[d] = q->hi[d];
        r.periodic[d] = q->periodic[d];
    }
    r.kind = q->kind;
    r.umode = q->u_mode;
    r.dmode = q->d_mode;
    r.n_params = q->n_params;
    for (int k = 0; k < q->n_params; ++k) r.params[k] = q->params[k];
    r.T = q->T;
    r.cfl = q->cfl;
    r.set = q->set;
    r.order = q->space_order;
    r.time_order = q->time_order;
    r.target.assign(q->target, q->target + total);
    size_t tf, af;
    if (request_bytes(r, &tf, &af) > s->budget) return fail(ODP_ENOMEM, "the request alone exceeds the HBM budget");
    std::lock_guard<std::mutex> lock(s->mu);
    r.id = s->next_id++;
    r.state = ODP_REQ_QUEUED;
    r.t_submit = now_s();
    *req_id = r.id;
    s->queue.push_back(r.id);
    s->reqs.emplace(r.id, std::move(r));
    return ODP_OK;
}

extern "C" odp_status odp_server_set_max_resident(odp_server *s, int64_t max_nodes)
{
    if (!s || max_nodes < 0) return fail(ODP_EINVAL, "need a server and a cap >= 0");
    std::lock_guard<std::mutex> lock(s->mu);
    s->max_nodes = max_nodes;
    return ODP_OK;
}

extern "C" odp_status odp_server_step(odp_server *s, int rounds, int *n_done)
{
    if (!s || rounds < 1) return fail(ODP_EINVAL, "need a server and rounds >= 1");
    std::lock_guard<std::mutex> lock(s->mu);
    ODP_SRV_CUDA(cudaSetDevice(s->device));
    cudaStream_t st = s->stream;
    if (n_done) *n_done = 0;

    // 1. admission in arrival order while the arrays fit the budget and the
    // resident nodes stay within the cap
    std::vector<uint64_t> fresh;
    auto nodes_of = [](const Request &r) {
        int64_t v = 1;
        for (int d = 0; d < r.ndim; ++d) v *= r.n[d];
        return v;
    };
    int64_t in_flight = 0;
    for (uint64_t id : s->resident) in_flight += nodes_of(s->reqs.at(id));
    while (!s->queue.empty()) {
        Request &r = s->reqs.at(s->queue.front());
        if (s->max_nodes > 0 && !s->resident.empty() && in_flight + nodes_of(r) > s->max_nodes) break;
        size_t tf, af;
        const size_t need = request_bytes(r, &tf, &af);
        const size_t off = s->arena->take(need);
        if (off == SIZE_MAX) break;
        s->queue.pop_front();
        r.off = off;
        r.bytes = need;
        std::vector<float> tab;
        float *block = reinterpret_cast<float *>(s->base + off);
        describe(r, block, tf, af, tab);
        ODP_SRV_CUDA(cudaMemcpyAsync(block, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, st));
        const int nl = r.n[r.ndim - 1], npad = r.rec.g.n_pad;
        ODP_SRV_CUDA(cudaMemsetAsync(const_cast<float *>(r.rec.l), 0, af * 4, st));
        ODP_SRV_CUDA(cudaMemcpy2DAsync(const_cast<float *>(r.rec.l), size_t(npad) * 4, r.target.data(),
                                       size_t(nl) * 4, size_t(nl) * 4, size_t(r.rec.g.rows), cudaMemcpyHostToDevice,
                                       st));
        r.state = ODP_REQ_RESIDENT;
        in_flight += nodes_of(r);
        r.t_admit = now_s();
        r.done_steps = 0;
        s->resident.push_back(r.id);
        fresh.push_back(r.id);
    }
    const int n = int(s->resident.size());
    if (n == 0) return ODP_OK;

    // device record table: one slot per resident solve, rebuilt every step
    if (size_t(n) > s->cap_rec) {
        cudaFree(s->d_rec);
        cudaFree(s->d_cfl);
        cudaFree(s->d_flags);
        s->d_rec = nullptr;
        s->d_cfl = nullptr;
        s->d_flags = nullptr;
        s->cap_rec = 0;
        const size_t cap = size_t(n) * 2;
        ODP_SRV_CUDA(cudaMalloc(&s->d_rec, sizeof(ServeGrid) * cap));
        ODP_SRV_CUDA(cudaMalloc(&s->d_cfl, sizeof(double) * cap));
        ODP_SRV_CUDA(cudaMalloc(&s->d_flags, sizeof(int) * cap));
        s->cap_rec = cap;
    }
    std::vector<ServeGrid> recs(static_cast<size_t>(n));
    std::vector<double> cfls(static_cast<size_t>(n));
    std::vector<int> fresh_slots;
    for (int i = 0; i < n; ++i) {
        Request &r = s->reqs.at(s->resident[size_t(i)]);
        r.rec.flags = s->d_flags + i;
        r.rec.step0 = r.done_steps;
        recs[size_t(i)] = r.rec;
        cfls[size_t(i)] = r.cfl;
        if (std::find(fresh.begin(), fresh.end(), r.id) != fresh.end()) fresh_slots.push_back(i);
    }
    ODP_SRV_CUDA(cudaMemcpyAsync(s->d_rec, recs.data(), sizeof(ServeGrid) * size_t(n), cudaMemcpyHostToDevice, st));
    ODP_SRV_CUDA(cudaMemcpyAsync(s->d_cfl, cfls.data(), sizeof(double) * size_t(n), cudaMemcpyHostToDevice, st));
    const size_t need_ints = size_t(n) * 2 + 1 + size_t(rounds) + fresh_slots.size();
    if (need_ints > s->cap_ints) {
        cudaFree(s->d_ints);
        s->d_ints = nullptr;
        s->cap_ints = 0;
        ODP_SRV_CUDA(cudaMalloc(&s->d_ints, sizeof(int) * need_ints * 2));
        s->cap_ints = need_ints * 2;
    }
    if (!fresh_slots.empty()) {
        // flags of the fresh slots are cleared by the prepare kernel
        ODP_SRV_CUDA(cudaMemcpyAsync(s->d_ints, fresh_slots.data(), sizeof(int) * fresh_slots.size(),
                                     cudaMemcpyHostToDevice, st));
        k_serve_prepare<<<int(fresh_slots.size()), 256, 0, st>>>(s->d_rec, s->d_ints, s->d_cfl);
        ODP_SRV_CUDA(cudaGetLastError());
        ODP_SRV_CUDA(cudaMemcpyAsync(recs.data(), s->d_rec, sizeof(ServeGrid) * size_t(n), cudaMemcpyDeviceToHost, st));
        ODP_SRV_CUDA(cudaStreamSynchronize(st));
        for (int i : fresh_slots) {
            Request &r = s->reqs.at(s->resident[size_t(i)]);
            const ServeGrid &g = recs[size_t(i)];
            memcpy(r.rec.alpha_bits, g.alpha_bits, sizeof(g.alpha_bits));
            memcpy(r.rec.cD, g.cD, sizeof(g.cD));
            r.rec.n_steps = g.n_steps;
            r.rec.dt_cfl = g.dt_cfl;
            r.rec.dt_last = g.dt_last;
            r.n_steps = g.n_steps;
        }
    }

    // 2. one persistent launch: every resident solve takes up to `rounds` steps
    std::vector<int> sorted(static_cast<size_t>(n));
    std::iota(sorted.begin(), sorted.end(), 0);
    auto remaining = [&](int i) {
        const Request &r = s->reqs.at(s->resident[size_t(i)]);
        return r.n_steps - r.done_steps;
    };
    std::stable_sort(sorted.begin(), sorted.end(), [&](int x, int y) { return remaining(x) > remaining(y); });
    const int launch_rounds = std::min(rounds, remaining(sorted[0]));
    // the step offsets and schedules of every record
    for (int i = 0; i < n; ++i) {
        const Request &r = s->reqs.at(s->resident[size_t(i)]);
        recs[size_t(i)] = r.rec;
        recs[size_t(i)].flags = s->d_flags + i;
        recs[size_t(i)].step0 = r.done_steps;
    }
    ODP_SRV_CUDA(cudaMemcpyAsync(s->d_rec, recs.data(), sizeof(ServeGrid) * size_t(n), cudaMemcpyHostToDevice, st));
    ODP_SRV_CUDA(cudaMemsetAsync(s->d_bar, 0, sizeof(ServeBarrier), st));
    // flags are per launch slot: cleared before every launch (a failure is
    // kept in the request's host state once read back)
    ODP_SRV_CUDA(cudaMemsetAsync(s->d_flags, 0, sizeof(int) * size_t(n), st));

    // When every resident grid takes the plane-streaming pass, each round
    // (and RK phase) is one launch per class of solves (model, space order,
    // time order); otherwise one persistent cooperative launch of the
    // row-blocked pass runs all rounds.
    bool plane = true;
    for (int i = 0; i < n && plane; ++i)
        if (!s->reqs.at(s->resident[size_t(i)]).rec.g.pg.use) plane = false;
    if (plane) {
        struct Cls {
            int kind, order, time_order, threads = 32, smem = 0;
            std::vector<int> members, start, active;
        };
        std::vector<Cls> cls;
        for (int k = 0; k < n; ++k) {
            const int i = sorted[size_t(k)];
            const Request &r = s->reqs.at(s->resident[size_t(i)]);
            size_t c = 0;
            while (c < cls.size() &&
                   !(cls[c].kind == r.kind && cls[c].order == r.order && cls[c].time_order == r.time_order))
                ++c;
            if (c == cls.size()) {
                Cls nc;
                nc.kind = r.kind;
                nc.order = r.order;
                nc.time_order = r.time_order;
                nc.start.push_back(0);
                cls.push_back(nc);
            }
            Cls &C = cls[c];
            C.members.push_back(i);
            C.start.push_back(C.start.back() + r.rec.g.pg.items);
            C.threads = std::max(C.threads, r.rec.g.pg.threads);
            C.smem = std::max(C.smem, r.rec.g.pg.smem[r.order - 1]);
        }
        std::vector<int> packed;
        std::vector<size_t> off(cls.size());
        for (size_t c = 0; c < cls.size(); ++c) {
            Cls &C = cls[c];
            off[c] = packed.size();
            packed.insert(packed.end(), C.members.begin(), C.members.end());
            packed.insert(packed.end(), C.start.begin(), C.start.end());
            // members are in order of remaining steps: round rr's active
            // items are a prefix
            C.active.assign(size_t(launch_rounds), 0);
            int k = int(C.members.size());
            for (int rr = 0; rr < launch_rounds; ++rr) {
                while (k > 0 && remaining(C.members[size_t(k) - 1]) <= rr) --k;
                C.active[size_t(rr)] = C.start[size_t(k)];
            }
        }
        if (packed.size() > s->cap_ints) {
            cudaFree(s->d_ints);
            s->d_ints = nullptr;
            s->cap_ints = 0;
            ODP_SRV_CUDA(cudaMalloc(&s->d_ints, sizeof(int) * packed.size() * 2));
            s->cap_ints = packed.size() * 2;
        }
        ODP_SRV_CUDA(cudaMemcpyAsync(s->d_ints, packed.data(), sizeof(int) * packed.size(), cudaMemcpyHostToDevice, st));
        for (int rr = 0; rr < launch_rounds; ++rr) {
            for (int phase = 0; phase < 2; ++phase) {
                for (size_t c = 0; c < cls.size(); ++c) {
                    const Cls &C = cls[c];
                    if (phase == 1 && C.time_order != 2) continue;
                    const int ctas = C.active[size_t(rr)];
                    if (ctas == 0) continue;
                    const int nc = int(C.members.size());
                    const int *d_members = s->d_ints + off[c], *d_start = d_members + nc;
                    cudaError_t e = C.kind == ODP_DYN_DUBINS3D
                                        ? launch_serve_plane<3, DYN_DUBINS3D>(C.order, ctas, C.threads, C.smem,
                                                                              s->d_rec, d_members, d_start, nc, rr,
                                                                              phase, st)
                                        : launch_serve_plane<4, DYN_DUBINSCAR4D>(C.order, ctas, C.threads, C.smem,
                                                                                 s->d_rec, d_members, d_start, nc, rr,
                                                                                 phase, st);
                    ODP_SRV_CUDA(e);
                    s->launches += 1;
                }
            }
        }
    } else {
        std::vector<int> packed;
        packed.reserve(size_t(n) * 2 + 1 + size_t(launch_rounds));
        packed.insert(packed.end(), sorted.begin(), sorted.end());
        int acc = 0, any_rk2 = 0;
        packed.push_back(0);
        for (int k = 0; k < n; ++k) {
            const Request &r = s->reqs.at(s->resident[size_t(sorted[size_t(k)])]);
            acc += r.rec.items;
            packed.push_back(acc);
            any_rk2 |= r.time_order == 2;
        }
        {
            int k = n;
            for (int rr = 0; rr < launch_rounds; ++rr) {
                while (k > 0 && remaining(sorted[size_t(k) - 1]) <= rr) --k;
                packed.push_back(packed[size_t(n) + size_t(k)]);
            }
        }
        ODP_SRV_CUDA(cudaMemcpyAsync(s->d_ints, packed.data(), sizeof(int) * packed.size(), cudaMemcpyHostToDevice, st));
        const int *d_sorted = s->d_ints, *d_start = s->d_ints + n, *d_active = s->d_ints + 2 * n + 1;
        int ctas = s->per_sm * s->sms;
        if (ctas > acc) ctas = std::max(1, acc);
        const ServeGrid *rec_arg = s->d_rec;
        ServeBarrier *bar_arg = s->d_bar;
        int n_arg = n, rk2_arg = any_rk2, rounds_arg = launch_rounds;
        void *args[] = {(void *)&rec_arg, (void *)&d_sorted, (void *)&d_start, (void *)&n_arg, (void *)&d_active,
                        (void *)&rk2_arg, (void *)&rounds_arg, (void *)&bar_arg};
        ODP_SRV_CUDA(cudaLaunchCooperativeKernel((const void *)k_serve_run<4>, dim3(ctas), dim3(256), args, 0, st));
        s->launches += 1;
    }
    std::vector<int> flags(static_cast<size_t>(n));
    ServeBarrier hbar{};
    ODP_SRV_CUDA(cudaMemcpyAsync(flags.data(), s->d_flags, sizeof(int) * size_t(n), cudaMemcpyDeviceToHost, st));
    ODP_SRV_CUDA(cudaMemcpyAsync(&hbar, s->d_bar, sizeof(hbar), cudaMemcpyDeviceToHost, st));
    ODP_SRV_CUDA(cudaStreamSynchronize(st));
    if (hbar.flags) return fail(ODP_ECUDA, "a grid-wide barrier of the serving launch gave up waiting");

    // 3. retire the solves that reached their horizon
    const double t = now_s();
    std::vector<uint64_t> still;
    for (int i = 0; i < n; ++i) {
        Request &r = s->reqs.at(s->resident[size_t(i)]);
        r.done_steps += std::min(launch_rounds, r.n_steps - r.done_steps);
        if (flags[size_t(i)] & FLAG_NONFINITE) {
            r.state = ODP_REQ_FAILED;
            r.error = ODP_ENUMERIC;
            r.t_done = t;
            if (n_done) ++*n_done;
        } else if (r.done_steps >= r.n_steps) {
            r.state = ODP_REQ_DONE;
            r.t_done = t;
            if (n_done) ++*n_done;
        } else {
            still.push_back(r.id);
        }
    }
    s->resident.swap(still);
    return ODP_OK;
}

extern "C" odp_status odp_server_poll(odp_server *s, uint64_t req_id, odp_request_stats *out)
{
    if (!s || !out) return fail(ODP_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return fail(ODP_EINVAL, "unknown request %llu", (unsigned long long)req_id);
    const Request &r = it->second;
    memset(out, 0, sizeof(*out));
    out->state = r.state;
    out->steps = r.n_steps;
    out->steps_done = r.done_steps;
    out->queue_s = (r.state == ODP_REQ_QUEUED) ? 0.0 : r.t_admit - r.t_submit;
    out->latency_s = (r.state == ODP_REQ_DONE || r.state == ODP_REQ_FAILED) ? r.t_done - r.t_submit : 0.0;
    out->t_submit = r.t_submit;
    out->t_done = r.t_done;
    out->bytes = double(r.bytes);
    return r.state == ODP_REQ_FAILED ? fail(r.error, "request %llu failed", (unsigned long long)req_id) : ODP_OK;
}

extern "C" odp_status odp_server_readback(odp_server *s, uint64_t req_id, float *dst, int64_t n_elems, int on_device)
{
    if (!s || !dst) return fail(ODP_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return fail(ODP_EINVAL, "unknown request");
    Request &r = it->second;
    if (r.state != ODP_REQ_DONE) return fail(ODP_ESTATE, "request %llu is not done", (unsigned long long)req_id);
    if (n_elems != int64_t(r.rec.g.total)) return fail(ODP_EINVAL, "destination size mismatch");
    ODP_SRV_CUDA(cudaSetDevice(s->device));
    const float *src = (r.time_order == 1 && (r.n_steps & 1)) ? r.rec.b : r.rec.a;
    const int nl = r.n[r.ndim - 1], npad = r.rec.g.n_pad;
    ODP_SRV_CUDA(cudaMemcpy2DAsync(dst, size_t(nl) * 4, src, size_t(npad) * 4, size_t(nl) * 4, size_t(r.rec.g.rows),
                                   on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream));
    ODP_SRV_CUDA(cudaStreamSynchronize(s->stream));
    return ODP_OK;
}

extern "C" odp_status odp_server_release(odp_server *s, uint64_t req_id)
{
    if (!s) return fail(ODP_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return fail(ODP_EINVAL, "unknown request");
    Request &r = it->second;
    if (r.state == ODP_REQ_RESIDENT) return fail(ODP_EBUSY, "request %llu is still running", (unsigned long long)req_id);
    if (r.state == ODP_REQ_QUEUED) {
        s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), req_id), s->queue.end());
    } else if (r.off != SIZE_MAX) {
        s->arena->give(r.off, r.bytes);
    }
    s->reqs.erase(it);
    return ODP_OK;
}

extern "C" odp_status odp_server_info(odp_server *s, odp_server_stats *out)
{
    if (!s || !out) return fail(ODP_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    memset(out, 0, sizeof(*out));
    out->budget_bytes = double(s->budget);
    out->used_bytes = double(s->arena->used());
    out->queued = int64_t(s->queue.size());
    out->resident = int64_t(s->resident.size());
    out->launches = s->launches;
    return ODP_OK;
}
