// ttr.cu -- time-to-reach function by Lax-Friedrichs sweeping (Section 2.2,
// the static HJ equation of the time-to-reach function, Algorithm 2; sweep
// directions of Section 5.3).
//
// What one sweep computes (the paper's Gauss-Seidel order, kept exactly):
//   for every interior node, in nested C-order loops with axis d visited in
//   descending order when bit d of (sweep mod 2^ndim) is set,
//     pbar_d  = (phi(i+e_d) - phi(i-e_d)) / (2 h_d)      (current values)
//     u*, d*  = argmin_u, argmax_d pbar . f(z, u, d)
//     sigma_d = |f_d(z, u*, d*)|
//     phi_i   = min(phi_i, (1 + pbar . f(z, u*, d*)
//                           + sum_d sigma_d (phi(i+e_d) + phi(i-e_d)) / (2 h_d))
//                          / sum_d(sigma_d / h_d))
//   (the update of Algorithm 2 with the static Hamiltonian -pbar.f - 1; the
//   kernel evaluates it in the equal cancellation-free form given above
//   ttr_node_terms), then
//   each non-periodic axis in turn sets its first and last nodes to
//   min(max(2 phi_1 - phi_2, phi_2), phi_b) along that axis.  Sweeps repeat
//   while the largest change of a sweep exceeds eps.
//
// GPU order.  A node's neighbours differ from it by one along one axis, so in
// the direction-mapped coordinates y (y_d = x_d, or n_d - 1 - x_d on a
// descending axis) every neighbour that the sequential sweep has already
// updated lies on the hyperplane sum(y) - 1 and every one it has not on
// sum(y) + 1 (a periodic wrap pair is ordered the same way by both).  The
// sweep therefore runs hyperplane by hyperplane and every node reads exactly
// the values the sequential order gives it.  The grid is cut into tiles in
// y-space; tiles with the same tile-coordinate sum never touch, so one launch
// takes one tile hyperplane, and inside a CTA the tile's own hyperplanes are
// walked with a barrier between them, on a copy of the tile and its face halo
// in shared memory.  Boundary faces follow, one launch per non-periodic axis,
// then a one-thread kernel closes the sweep and sets the device-side loop
// condition of the CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hj_device.cuh"
#include "odp_internal.h"

namespace odp {

constexpr int TTR_MAXD = 4;
constexpr int TTR_MAX_THREADS = 512;

// Tiling of the sweep (y-space, last axis fastest).
struct TtrGeom {
    int T[TTR_MAXD];    // tile extent per axis
    int NT[TTR_MAXD];   // tiles per axis
    int hs[TTR_MAXD];   // strides of the shared copy, extents T + 2
    int tvol;           // nodes per tile = threads per CTA
    int hvol;           // floats of the shared copy
    int depth;          // hyperplanes inside a tile: sum(T - 1) + 1
};

struct TtrState {
    long long sweeps;       // sweeps finished
    long long max_sweeps;
    double eps;
    unsigned change_bits;   // largest change of the running sweep (float bits)
    unsigned last_bits;     // largest change of the last finished sweep
    int flags;              // FLAG_NONFINITE, FLAG_TIMEOUT
    int go;                 // the loop continues (host-stepped loop)
};

// The plan of one grid: tile lists, state, graph.
struct TtrPlan {
    TtrGeom tg{};
    int planes = 0;
    std::vector<int> plane_off, plane_cnt;
    int *tiles = nullptr;       // tile ids ordered by tile hyperplane (device)
    TtrState *st = nullptr;     // device
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long dyn_version = -1;
    int64_t launches_per_sweep = 0;
};

// ---------------------------------------------------------------------------
// per-node model terms
//
// With sigma_d = |f_d(z, u*, d*)|, each axis's part of the update is
//   sigma_d (phi(i+e_d) + phi(i-e_d)) / (2 h_d) + pbar_d f_d
//     = (|f_d| / h_d) * phi(i + sign(f_d) e_d),
// so the update equals (1 + sum_d w_d phi_nb(d)) / sum_d w_d with
// w_d = |f_d| / h_d and phi_nb(d) the neighbour the flow points to.  For an
// input axis, u* = -bound when pbar_d >= 0 (u_mode min), so phi_nb(d) is the
// smaller of the two neighbours; for a drift axis it is fixed by the sign of
// f_d(z).  This form is what the kernel evaluates: the printed one subtracts
// terms of size big * sigma / h that cancel, which in float32 leaves errors
// of a few 1e-4 that the min keeps for good; this one adds non-negative terms
// only.
// ---------------------------------------------------------------------------

// Per node: weights w_d = |f_d| / h_d, the side of each drift axis (1: the
// neighbour at i + e_d), and sum_d w_d.
template <int DYN, int ND>
__device__ __forceinline__ void ttr_node_terms(const GridDesc &g, const DynDesc &dy, const int *x, float *w,
                                               bool *fwd, float &den)
{
#pragma unroll
    for (int d = 0; d < ND; ++d) fwd[d] = false;
    if (DYN == DYN_SINGLE_INT) {
#pragma unroll
        for (int d = 0; d < ND; ++d) w[d] = dy.prm[0] * g.inv_dz[d];
    } else if (DYN == DYN_DUBINS3D) {
        const float fx = dy.prm[0] * ldgf(g.cos_tab + x[2]), fy = dy.prm[0] * ldgf(g.sin_tab + x[2]);
        w[0] = fabsf(fx) * g.inv_dz[0];
        w[1] = fabsf(fy) * g.inv_dz[1];
        w[2] = dy.prm[1] * g.inv_dz[2];
        fwd[0] = fx >= 0.0f;
        fwd[1] = fy >= 0.0f;
    } else {   // DubinsCar4D (x, y, v, th)
        const float v = ldgf(g.coord[2] + x[2]);
        const float fx = v * ldgf(g.cos_tab + x[3]), fy = v * ldgf(g.sin_tab + x[3]);
        w[0] = fabsf(fx) * g.inv_dz[0];
        w[1] = fabsf(fy) * g.inv_dz[1];
        w[2] = dy.prm[0] * g.inv_dz[2];
        w[3] = dy.prm[1] * g.inv_dz[3];
        fwd[0] = fx >= 0.0f;
        fwd[1] = fy >= 0.0f;
    }
    den = 0.0f;
#pragma unroll
    for (int d = 0; d < ND; ++d) den += w[d];
}

// Whether axis d of the model is driven by a bounded input (its neighbour is
// the smaller one) rather than a drift.
template <int DYN>
__device__ __forceinline__ constexpr bool ttr_input_axis(int d)
{
    return DYN == DYN_SINGLE_INT ? true : DYN == DYN_DUBINS3D ? d == 2 : d >= 2;
}

__device__ __forceinline__ void block_max_change(float v, TtrState *st)
{
    __shared__ float red[TTR_MAX_THREADS / 32];
    v = warp_max(v);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        float m = lane < nw ? red[lane] : 0.0f;
        m = warp_max(m);
        if (lane == 0 && m > 0.0f) atomicMax(&st->change_bits, __float_as_uint(m));
    }
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// One tile hyperplane of a sweep: CTA b takes tile tiles[b].
template <int ND, int DYN>
__global__ void __launch_bounds__(TTR_MAX_THREADS) k_ttr_tiles(GridDesc g, DynDesc dy, TtrGeom tg,
                                                               const int *__restrict__ tiles, TtrState *st,
                                                               float *phi)
{
    extern __shared__ float sh[];
    const unsigned dirs = unsigned(st->sweeps) & ((1u << ND) - 1u);
    int t[ND];
    {
        int r = tiles[blockIdx.x];
#pragma unroll
        for (int d = ND - 1; d >= 0; --d) {
            t[d] = r % tg.NT[d];
            r /= tg.NT[d];
        }
    }
    // this thread's slot of the tile
    int a[ND], y[ND], x[ND], pos = 0, level = 0, addr = 0;
    const bool inside = threadIdx.x < unsigned(tg.tvol);
    bool mine = inside;
    {
        int r = threadIdx.x;
#pragma unroll
        for (int d = ND - 1; d >= 0; --d) {
            a[d] = r % tg.T[d];
            r /= tg.T[d];
        }
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            y[d] = t[d] * tg.T[d] + a[d];
            const int n = g.n[d];
            if (y[d] >= n) mine = false;
            x[d] = ((dirs >> d) & 1u) ? n - 1 - y[d] : y[d];
            if (!g.periodic[d] && (x[d] <= 0 || x[d] >= n - 1)) mine = false;
            pos += (a[d] + 1) * tg.hs[d];
            level += a[d];
            addr += x[d] * g.stride[d];
        }
    }
    // The shared copy: every thread loads its own slot (a slot past the end
    // of a periodic axis holds the wrapped node) and, on a tile face, the
    // face halo slot beyond it; slots outside a non-periodic axis are never
    // read and stay unloaded.
    if (inside) {
#pragma unroll
        for (int k = -1; k < ND; ++k) {
            // k = -1: the own slot; k = 0 .. ND-1: the halo below (a = 0) or
            // above (a = T - 1) along axis k
            int off = 0, shift = 0;
            if (k >= 0) {
                if (a[k] == 0) {
                    off = -tg.hs[k];
                    shift = -1;
                } else if (a[k] == tg.T[k] - 1) {
                    off = tg.hs[k];
                    shift = 1;
                } else {
                    continue;
                }
            }
            bool ok = true;
            int src = 0;
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                int yy = y[d] + (d == k ? shift : 0);
                const int n = g.n[d];
                if (yy < 0 || yy >= n) {
                    if (!g.periodic[d]) {
                        ok = false;
                        break;
                    }
                    yy = yy < 0 ? yy + n : yy - n;
                    if (yy < 0 || yy >= n) {
                        ok = false;
                        break;
                    }
                }
                src += (((dirs >> d) & 1u) ? n - 1 - yy : yy) * g.stride[d];
            }
            if (ok) sh[pos + off] = phi[src];
        }
    }
    float w[ND], inv_den = 0.0f;
    bool fwd[ND];
    if (mine) {
        float den;
        ttr_node_terms<DYN, ND>(g, dy, x, w, fwd, den);
        if (den > 0.0f) inv_den = 1.0f / den;
        else mine = false;   // sum_d sigma_d / h_d = 0: the node keeps its value
    }
    // offset of phi(x + e_d) in the shared copy
    int o[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) o[d] = ((dirs >> d) & 1u) ? -tg.hs[d] : tg.hs[d];
    __syncthreads();

    float change = 0.0f;
    for (int s = 0; s < tg.depth; ++s) {
        if (mine && level == s) {
            float num = 1.0f;
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                const float up = sh[pos + o[d]], dn = sh[pos - o[d]];
                const float nb = ttr_input_axis<DYN>(d) ? fminf(up, dn) : (fwd[d] ? up : dn);
                num = fmaf(w[d], nb, num);
            }
            const float old = sh[pos];
            const float v = fminf(num * inv_den, old);
            sh[pos] = v;
            change = old - v;
        }
        __syncthreads();
    }
    if (mine) phi[addr] = sh[pos];
    block_max_change(change, st);
}

// The boundary rule of one non-periodic axis d on both faces.  start holds
// the value a node had before the first face pass that touched it, for the
// change of nodes on several faces.
template <int ND>
__global__ void __launch_bounds__(256) k_ttr_face(GridDesc g, int d, TtrState *st, float *phi, float *start)
{
    const int n = g.n[d];
    const int per_face = g.total / n;
    float change = 0.0f;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < 2 * per_face; j += gridDim.x * blockDim.x) {
        const int side = j >= per_face ? 1 : 0;
        int r = side ? j - per_face : j;
        int x[ND], addr = 0;
#pragma unroll
        for (int e = ND - 1; e >= 0; --e) {
            if (e == d) {
                x[e] = side ? n - 1 : 0;
            } else {
                x[e] = r % g.n[e];
                r /= g.n[e];
            }
            addr += x[e] * g.stride[e];
        }
        int first = -1, last = -1;
#pragma unroll
        for (int e = 0; e < ND; ++e) {
            if (!g.periodic[e] && (x[e] == 0 || x[e] == g.n[e] - 1)) {
                if (first < 0) first = e;
                last = e;
            }
        }
        const int step = side ? -g.stride[d] : g.stride[d];
        const float old = phi[addr];
        const float p1 = phi[addr + step], p2 = phi[addr + 2 * step];
        const float v = fminf(fmaxf(2.0f * p1 - p2, p2), old);
        const float before = (d == first) ? old : start[addr];
        if (d == last) change = fmaxf(change, before - v);
        else if (d == first) start[addr] = old;
        phi[addr] = v;
    }
    block_max_change(change, st);
}

// Closes a sweep: counts it, keeps its change and decides whether the loop
// continues (change > eps and sweeps left).
__global__ void k_ttr_check(TtrState *st, cudaGraphConditionalHandle h, int in_graph)
{
    st->sweeps += 1;
    const unsigned bits = st->change_bits;
    st->last_bits = bits;
    st->change_bits = 0u;
    const float ch = __uint_as_float(bits);
    int go = 1;
    if (!isfinite(ch)) {
        st->flags |= FLAG_NONFINITE;
        go = 0;
    } else if (!(double(ch) > st->eps)) {
        go = 0;
    } else if (st->sweeps >= st->max_sweeps) {
        st->flags |= FLAG_TIMEOUT;
        go = 0;
    }
    st->go = go;
    if (in_graph) cudaGraphSetConditional(h, go);
}

// phi = 0 on the target set {l <= 0}, big elsewhere (Section 2.2).
__global__ void k_ttr_init(GridDesc g, int n_last, const float *__restrict__ l, float *phi, float big)
{
    const int total = g.rows * g.n_pad;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int c = i % g.n_pad;
        if (c < n_last) phi[i] = (l[i] <= 0.0f) ? 0.0f : big;
    }
}

// Hands the result to the grid's readback path.
__global__ void k_ttr_finish(SolveState *ss, const TtrState *st, float *phi)
{
    ss->cur = phi;
    ss->flags = st->flags;
    ss->steps = st->sweeps;
    ss->max_steps = st->max_sweeps;
    ss->t = 0.0;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static bool ttr_model(int kind) { return kind == DYN_SINGLE_INT || kind == DYN_DUBINS3D || kind == DYN_DUBINSCAR4D; }

// Tile extents: cube-like tiles of at most 512 nodes, the last axis widest;
// a periodic axis keeps at least two tiles so that its wrap neighbour is
// never inside the same tile.
static TtrGeom ttr_geometry(const odp_grid *g)
{
    static const int base[TTR_MAXD + 1][TTR_MAXD] = {
        {0, 0, 0, 0}, {512, 0, 0, 0}, {16, 32, 0, 0}, {8, 8, 8, 0}, {4, 4, 4, 8}};
    TtrGeom tg{};
    const int nd = g->ndim;
    tg.tvol = 1;
    tg.hvol = 1;
    tg.depth = 1;
    for (int d = 0; d < nd; ++d) {
        int T = std::min(base[nd][d], g->n[d]);
        if (g->periodic[d]) T = std::min(T, g->n[d] / 2);
        T = std::max(T, 1);
        tg.T[d] = T;
        tg.NT[d] = (g->n[d] + T - 1) / T;
        tg.tvol *= T;
        tg.depth += T - 1;
    }
    for (int d = nd - 1; d >= 0; --d) {
        tg.hs[d] = tg.hvol;
        tg.hvol *= tg.T[d] + 2;
    }
    return tg;
}

#define TTR_CUDA(call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? ODP_ENOMEM : ODP_ECUDA,         \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                        \
    } while (0)

template <int ND, int DYN>
static cudaError_t launch_tiles(odp_grid *g, TtrPlan *P, int plane, cudaStream_t s)
{
    const int cnt = P->plane_cnt[size_t(plane)];
    k_ttr_tiles<ND, DYN><<<cnt, P->tg.tvol, size_t(P->tg.hvol) * sizeof(float), s>>>(
        g->desc, g->dyn, P->tg, P->tiles + P->plane_off[size_t(plane)], P->st, g->phi_a);
    return cudaGetLastError();
}

static cudaError_t launch_plane(odp_grid *g, TtrPlan *P, int plane, cudaStream_t s)
{
    const int kind = g->dyn.kind;
    switch (g->ndim) {
    case 1: return launch_tiles<1, DYN_SINGLE_INT>(g, P, plane, s);
    case 2: return launch_tiles<2, DYN_SINGLE_INT>(g, P, plane, s);
    case 3: return kind == DYN_DUBINS3D ? launch_tiles<3, DYN_DUBINS3D>(g, P, plane, s)
                                        : launch_tiles<3, DYN_SINGLE_INT>(g, P, plane, s);
    default: return kind == DYN_DUBINSCAR4D ? launch_tiles<4, DYN_DUBINSCAR4D>(g, P, plane, s)
                                            : launch_tiles<4, DYN_SINGLE_INT>(g, P, plane, s);
    }
}

static cudaError_t launch_face(odp_grid *g, TtrPlan *P, int d, cudaStream_t s)
{
    const int per = int(g->total / g->n[d]);
    const int blocks = std::max(1, std::min((2 * per + 255) / 256, 152 * 8));
    switch (g->ndim) {
    case 1: k_ttr_face<1><<<blocks, 256, 0, s>>>(g->desc, d, P->st, g->phi_a, g->phi_b); break;
    case 2: k_ttr_face<2><<<blocks, 256, 0, s>>>(g->desc, d, P->st, g->phi_a, g->phi_b); break;
    case 3: k_ttr_face<3><<<blocks, 256, 0, s>>>(g->desc, d, P->st, g->phi_a, g->phi_b); break;
    default: k_ttr_face<4><<<blocks, 256, 0, s>>>(g->desc, d, P->st, g->phi_a, g->phi_b); break;
    }
    return cudaGetLastError();
}

// The kernels of one sweep, in order.
static cudaError_t launch_sweep(odp_grid *g, TtrPlan *P, cudaStream_t s, cudaGraphConditionalHandle h, int in_graph,
                                int64_t *launches)
{
    int64_t n = 0;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < P->planes && e == cudaSuccess; ++k, ++n) e = launch_plane(g, P, k, s);
    for (int d = 0; d < g->ndim && e == cudaSuccess; ++d) {
        if (g->periodic[d]) continue;
        e = launch_face(g, P, d, s);
        ++n;
    }
    if (e == cudaSuccess) {
        k_ttr_check<<<1, 1, 0, s>>>(P->st, h, in_graph);
        e = cudaGetLastError();
        ++n;
    }
    if (launches) *launches = n;
    return e;
}

static odp_status ttr_plan(odp_grid *g, TtrPlan **out)
{
    TtrPlan *P = static_cast<TtrPlan *>(g->ttr);
    if (!P) {
        P = new TtrPlan();
        g->ttr = P;
        P->tg = ttr_geometry(g);
        const TtrGeom &tg = P->tg;
        int ntiles = 1;
        P->planes = 1;
        for (int d = 0; d < g->ndim; ++d) {
            ntiles *= tg.NT[d];
            P->planes += tg.NT[d] - 1;
        }
        // tile ids grouped by tile hyperplane (counting sort on sum of tile coordinates)
        std::vector<int> plane_of(static_cast<size_t>(ntiles));
        P->plane_cnt.assign(size_t(P->planes), 0);
        for (int id = 0; id < ntiles; ++id) {
            int r = id, sum = 0;
            for (int d = g->ndim - 1; d >= 0; --d) {
                sum += r % tg.NT[d];
                r /= tg.NT[d];
            }
            plane_of[size_t(id)] = sum;
            P->plane_cnt[size_t(sum)] += 1;
        }
        P->plane_off.assign(size_t(P->planes), 0);
        for (int k = 1; k < P->planes; ++k) P->plane_off[size_t(k)] = P->plane_off[size_t(k) - 1] + P->plane_cnt[size_t(k) - 1];
        std::vector<int> fill(P->plane_off), order(static_cast<size_t>(ntiles));
        for (int id = 0; id < ntiles; ++id) order[size_t(fill[size_t(plane_of[size_t(id)])]++)] = id;
        TTR_CUDA(cudaMalloc(&P->tiles, sizeof(int) * size_t(ntiles)));
        TTR_CUDA(cudaMalloc(&P->st, sizeof(TtrState)));
        TTR_CUDA(cudaMemcpyAsync(P->tiles, order.data(), sizeof(int) * size_t(ntiles), cudaMemcpyHostToDevice,
                                 g->stream));
        TTR_CUDA(cudaStreamSynchronize(g->stream));
    }
    *out = P;
    return ODP_OK;
}

static odp_status ttr_build_graph(odp_grid *g, TtrPlan *P)
{
    if (P->exec && P->dyn_version == g->dyn_version) return ODP_OK;
    if (P->exec) {
        TTR_CUDA(cudaStreamSynchronize(g->stream));
        cudaGraphExecDestroy(P->exec);
        P->exec = nullptr;
    }
    if (P->graph) {
        cudaGraphDestroy(P->graph);
        P->graph = nullptr;
    }
    TTR_CUDA(cudaGraphCreate(&P->graph, 0));
    cudaGraphConditionalHandle h;
    TTR_CUDA(cudaGraphConditionalHandleCreate(&h, P->graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams wp{};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = h;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t loop_node;
    TTR_CUDA(cudaGraphAddNode(&loop_node, P->graph, nullptr, nullptr, 0, &wp));
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    cudaStream_t s = g->capture_stream;
    TTR_CUDA(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    int64_t launches = 0;
    cudaError_t e = launch_sweep(g, P, s, h, 1, &launches);
    cudaGraph_t captured = body;
    cudaError_t e2 = cudaStreamEndCapture(s, &captured);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        cudaGetLastError();
        P->graph = nullptr;
        return fail(ODP_ECUDA, "capturing the sweep loop: %s / %s", cudaGetErrorString(e), cudaGetErrorString(e2));
    }
    cudaError_t ei = cudaGraphInstantiate(&P->exec, P->graph, 0);
    if (ei != cudaSuccess) {
        P->exec = nullptr;
        cudaGraphDestroy(P->graph);
        P->graph = nullptr;
        return fail(ODP_ECUDA, "instantiating the sweep loop: %s", cudaGetErrorString(ei));
    }
    P->launches_per_sweep = launches;
    P->dyn_version = g->dyn_version;
    return ODP_OK;
}

void ttr_release(odp_grid *g)
{
    TtrPlan *P = static_cast<TtrPlan *>(g->ttr);
    if (!P) return;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    cudaFree(P->tiles);
    cudaFree(P->st);
    delete P;
    g->ttr = nullptr;
}

}  // namespace odp

using namespace odp;

extern "C" odp_status odp_solve_ttr(odp_grid *g, double eps, double big, int64_t max_sweeps, odp_ttr_stats *stats)
{
    if (!g) return fail(ODP_EINVAL, "grid is NULL");
    if (!g->has_dyn || !g->has_target) return fail(ODP_ESTATE, "dynamics and target must be set first");
    if (g->l_seq_n) return fail(ODP_EINVAL, "the time-to-reach sweep takes one target set, not a schedule");
    if (!ttr_model(g->dyn.kind))
        return fail(ODP_EINVAL, "the time-to-reach sweep supports the single integrator, Dubins3D and DubinsCar4D");
    if (g->dyn.umode != MODE_MIN || g->dyn.dmode != MODE_MAX)
        return fail(ODP_EINVAL, "the time-to-reach function needs u_mode min and d_mode max");
    if (g->ndim > TTR_MAXD) return fail(ODP_EINVAL, "the time-to-reach sweep supports at most %d dimensions", TTR_MAXD);
    for (int d = 0; d < g->ndim; ++d)
        if (g->n[d] < 4) return fail(ODP_EINVAL, "axis %d has %d nodes; the sweep needs at least 4", d, g->n[d]);
    if (!(eps >= 0.0) || !std::isfinite(eps)) return fail(ODP_EINVAL, "eps must be finite and >= 0");
    if (!(big > 0.0) || !(big <= 3.0e38)) return fail(ODP_EINVAL, "big must be positive and a finite float");
    if (max_sweeps < 1) return fail(ODP_EINVAL, "max_sweeps must be >= 1");
    TTR_CUDA(cudaSetDevice(g->device));

    TtrPlan *P = nullptr;
    odp_status rc = ttr_plan(g, &P);
    if (rc != ODP_OK) return rc;
    if (!g->host_loop) {
        rc = ttr_build_graph(g, P);
        if (rc != ODP_OK) return rc;
    }
    cudaStream_t s = g->stream;
    TtrState h{};
    h.max_sweeps = max_sweeps;
    h.eps = eps;
    TTR_CUDA(cudaMemcpyAsync(P->st, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    {
        const int blocks = int(std::min<int64_t>((g->total_pad + 255) / 256, 152 * 8));
        k_ttr_init<<<blocks, 256, 0, s>>>(g->desc, g->n_last, g->l, g->phi_a, float(big));
        TTR_CUDA(cudaGetLastError());
    }
    TTR_CUDA(cudaEventRecord(g->ev0, s));
    int64_t launches = 0;
    if (!g->host_loop) {
        TTR_CUDA(cudaGraphLaunch(P->exec, s));
    } else {
        // the same kernels one sweep at a time, the loop condition read back
        for (;;) {
            int64_t n = 0;
            cudaError_t e = launch_sweep(g, P, s, 0, 0, &n);
            if (e != cudaSuccess) return fail(ODP_ECUDA, "sweep launch: %s", cudaGetErrorString(e));
            launches += n;
            int go = 0;
            TTR_CUDA(cudaMemcpyAsync(&go, &P->st->go, sizeof(int), cudaMemcpyDeviceToHost, s));
            TTR_CUDA(cudaStreamSynchronize(s));
            if (!go) break;
        }
    }
    TTR_CUDA(cudaEventRecord(g->ev1, s));
    k_ttr_finish<<<1, 1, 0, s>>>(g->state, P->st, g->phi_a);
    TTR_CUDA(cudaGetLastError());
    g->solved = true;
    g->n_tau = 1;
    g->keep = 0;
    if (!stats) return ODP_OK;

    TTR_CUDA(cudaStreamSynchronize(s));
    TTR_CUDA(cudaMemcpy(&h, P->st, sizeof(h), cudaMemcpyDeviceToHost));
    float ms = 0.0f;
    TTR_CUDA(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
    stats->sweeps = h.sweeps;
    float ch;
    std::memcpy(&ch, &h.last_bits, sizeof(ch));
    stats->change = double(ch);
    stats->device_ms = double(ms);
    // one read and one write of every node per sweep
    stats->bytes = 8.0 * double(g->total) * double(h.sweeps);
    stats->launches = g->host_loop ? launches : P->launches_per_sweep * h.sweeps;
    stats->tile_planes = P->planes;
    if (h.flags & FLAG_NONFINITE) return fail(ODP_ENUMERIC, "a non-finite change appeared in the sweep");
    if (h.flags & FLAG_TIMEOUT)
        return fail(ODP_ETIMEOUT, "sweep limit %lld reached with change %g", (long long)h.max_sweeps, double(ch));
    return ODP_OK;
}
