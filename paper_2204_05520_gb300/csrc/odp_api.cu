// odp_api.cu -- the C ABI of libodp (include/odp.h): grid objects, the host
// scheduler of one solve and the CUDA graph that runs its time loop.
//
// One solve (Algorithm 1 with the tau schedule of HJSolver, Section 4.3):
//   host, once per solve:  phi <- l, state upload, static alpha reduction
//   one CUDA graph:        WHILE (device flag) {
//                            [Rel6D: heading alpha of phi]    K1
//                            dt from alpha (float64)          K3
//                            stage pass(es)                   K2
//                            [Rel6D: heading alpha of phi1]   K1
//                            advance t, segment, flags        K3
//                            IF (segment ended) snapshot copy
//                          }
// t, dt and the tau schedule stay in float64 on the device; the loop never
// returns to the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/odp.h"
#include "odp_common.cuh"
#include "odp_internal.h"
#include "odp_launch.h"
#include "odp_time.cuh"

using namespace odp;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

odp_status odp::fail(odp_status code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define ODP_CUDA(call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? ODP_ENOMEM : ODP_ECUDA,         \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                        \
    } while (0)

// ---------------------------------------------------------------------------
// graph-control kernels (single thread)
// ---------------------------------------------------------------------------

// CFL step of Algorithm 1 from the stage-1 alpha, clipped to the segment end.
__global__ void k_dt(SolveState *st, GridDesc g)
{
    const double dt_cfl = cfl_dt(st->alpha_bits[0], g.dz, g.ndim, st->cfl);
    int last = 0;
    st->dt = clipped_step(dt_cfl, st->t, st->t_end, &last);
    st->last = last;
}

// Close a full step: advance t, count it, swap the Euler ping-pong buffers,
// clear the phi-dependent alpha components, move to the next tau segment
// when this one is done, and set the loop and snapshot conditions.  With
// next_dt (models whose alpha does not depend on phi) it also takes the next
// step's CFL step, which k_dt would otherwise compute at the top of the step.
__global__ void k_advance(SolveState *st, GridDesc g, int swap, unsigned dyn_mask, int next_dt,
                          cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_snap, int keep,
                          cudaGraphConditionalHandle h_seq, int seq, int in_graph)
{
    for (int d = 0; d < 8; ++d) st->alpha_last[d] = st->alpha_bits[swap ? 0 : 1][d];
    st->t = after_step(st->t, st->dt, st->t_end, st->last);
    st->steps += 1;
    if (swap) {
        float *tmp = st->cur;
        st->cur = st->nxt;
        st->nxt = tmp;
    }
    for (int d = 0; d < 8; ++d)
        if (dyn_mask & (1u << d)) {
            st->alpha_bits[0][d] = 0u;
            st->alpha_bits[1][d] = 0u;
        }
    int go = 1, snap = 0, next_sets = 0;
    if (segment_done(st->t, st->t_end)) {
        snap = keep;
        st->snap_index = st->seg + 1;
        st->seg += 1;
        if (st->seg >= st->n_seg) {
            go = 0;
        } else {
            st->t_end = st->tau[st->seg + 1];
            next_sets = seq;   // time-varying sets: load the new segment's
        }
    }
    if (st->flags) go = 0;
    if (go && st->steps >= st->max_steps) {
        st->flags |= FLAG_TIMEOUT;
        go = 0;
    }
    if (!go) next_sets = 0;
    st->go = go;
    st->snap_now = snap;
    if (next_dt && go) {
        const double dt_cfl = cfl_dt(st->alpha_bits[0], g.dz, g.ndim, st->cfl);
        int last = 0;
        st->dt = clipped_step(dt_cfl, st->t, st->t_end, &last);
        st->last = last;
    }
    if (in_graph) {
        cudaGraphSetConditional(h_loop, go);
        if (keep) cudaGraphSetConditional(h_snap, snap);
        if (seq) cudaGraphSetConditional(h_seq, next_sets);
    }
}

// Time-varying sets: the target and obstacle of segment seg (the sets at its
// end, tau[seg + 1]) into the buffers the stage kernels read.
__global__ void k_seq_sets(const SolveState *st, float *l, const float *l_seq, float *obst, const float *g_seq,
                           int total_pad)
{
    const long long k = st->seg + 1;
    const float *ls = l_seq ? l_seq + k * total_pad : nullptr;
    const float *gs = g_seq ? g_seq + k * total_pad : nullptr;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total_pad; i += gridDim.x * blockDim.x) {
        if (ls) l[i] = ls[i];
        if (gs) obst[i] = gs[i];
    }
}

__global__ void k_snapshot(SolveState *st, int total)
{
    const float *src = st->cur;
    float *dst = st->snapshots + (long long)st->snap_index * total;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// ---------------------------------------------------------------------------
// grid object
// ---------------------------------------------------------------------------
// Make the grid's device current on the calling thread.
static odp_status bind(const odp_grid *g)
{
    ODP_CUDA(cudaSetDevice(g->device));
    return ODP_OK;
}

#define ODP_BIND(g)                      \
    do {                                 \
        odp_status b_ = bind(g);         \
        if (b_ != ODP_OK) return b_;     \
    } while (0)

// Geometry of the plane-streaming pass (hj_plane.cuh): planes are the last
// two axes; a CTA streams a chunk of axis ndim-3 for fixed outer indices.  The
// chunk length is chosen so that a launch has about four CTAs per SM.  Grids
// whose planes do not fit in shared memory use the row-blocked pass instead.
void odp::plane_geometry(GridDesc &D, int sms)
{
    PlaneGeom &pg = D.pg;
    pg = PlaneGeom{};
    const int nr = D.nr, segs = D.segs;
    if (D.ndim < 3 || nr < 4 || segs > 128) return;
    // bands of about 256 threads, at least 4 rows each (radius-2 halos come
    // from one thread per row)
    int rb = 256 / segs;
    if (rb < 4) rb = 4;
    int nb = 1;
    if (rb >= nr) {
        rb = nr;
    } else {
        nb = (nr + rb - 1) / rb;
        rb = (nr + nb - 1) / nb;
        while (nb > 1 && nr - (nb - 1) * rb < 4) {
            --nb;
            rb = (nr + nb - 1) / nb;
        }
    }
    const int threads = (rb * segs + 31) / 32 * 32;
    if (threads > 512) return;
    pg.rb = rb;
    pg.nbands = nb;
    pg.threads = threads;
    pg.plane = nr * D.n_pad;
    pg.cp = D.n_pad + 4;
    // two tiles, then 32 bytes per thread for the drift rows of the
    // register-capped passes
    for (int o = 1; o <= 2; ++o) pg.smem[o - 1] = 2 * (4 + (rb + 2 * o) * pg.cp) * 4 + threads * 32;
    if (pg.smem[1] > 48 * 1024) {   // beyond the default dynamic shared memory of a CTA
        pg = PlaneGeom{};
        return;
    }
    pg.ns = D.n[D.ndim - 3];
    long long pencils = 1;
    for (int d = 0; d < D.ndim - 3; ++d) pencils *= D.n[d];
    // chunks of the stream axis: about twelve CTAs per SM per launch
    const long long base = pencils * nb;
    const long long target = 12LL * sms;
    long long chunk = (base * pg.ns + target - 1) / target;
    const int cmin = pg.ns < 4 ? pg.ns : 4;
    if (chunk < cmin) chunk = cmin;
    if (chunk > pg.ns) chunk = pg.ns;
    pg.chunk = int(chunk);
    pg.nchunks = (pg.ns + pg.chunk - 1) / pg.chunk;
    pg.items = int(base * pg.nchunks);
    pg.div_nchunks = make_fastdiv(uint32_t(pg.nchunks));
    pg.div_nbands = make_fastdiv(uint32_t(pg.nbands));
    // blocks of outer pencils: per outer axis the largest divisor of its
    // length up to ODP_PB0, ODP_PB1, ODP_PB2 (8 each)
#ifndef ODP_PB0
#define ODP_PB0 8
#endif
#ifndef ODP_PB1
#define ODP_PB1 8
#endif
#ifndef ODP_PB2
#define ODP_PB2 8
#endif
    const int bmax[3] = {ODP_PB0, ODP_PB1, ODP_PB2};
    pg.bvol = 1;
    for (int d = 0; d < 3; ++d) {
        int b = 1;
        if (d < D.ndim - 3)
            for (int c = bmax[d]; c >= 1; --c)
                if (D.n[d] % c == 0) {
                    b = c;
                    break;
                }
        pg.bdim[d] = b;
        pg.nblk[d] = d < D.ndim - 3 ? D.n[d] / b : 1;
        pg.bvol *= b;
        pg.div_bdim[d] = make_fastdiv(uint32_t(b));
        pg.div_nblk[d] = make_fastdiv(uint32_t(pg.nblk[d]));
    }
    pg.div_bvol = make_fastdiv(uint32_t(pg.bvol));
    pg.use = 1;
}

#ifndef ODP_BULK_THREADS
#define ODP_BULK_THREADS 256   // compute threads a band aims at
#endif
#ifndef ODP_BULK_THREADS4
#define ODP_BULK_THREADS4 128  // ... on the DubinsCar4D grids
#endif
#ifndef ODP_BULK_RC
#define ODP_BULK_RC 5
#endif
#ifndef ODP_BULK_RX
#define ODP_BULK_RX 3
#endif

// Stream-axis chunking of the bulk-staged pass for stencil radius o with
// per_sm resident CTAs per SM: the chunk count that minimises a makespan
// model.  A launch runs items / (per_sm x sms) waves; in a partial last wave
// an SM holds c <= per_sm CTAs and takes 0.4 + 0.6 c / per_sm of a full
// wave's time; each item costs its planes plus about 2o + 1 planes of window
// fill and setup.  Launches of fewer than 1.5 waves are avoided where the
// stream axis allows (measured slow: SMs stay part-empty throughout).
void odp::bulk_chunking(GridDesc &D, int o, int per_sm, int sms)
{
    BulkGeom &bk = D.bk;
    const int nd = D.ndim, ns = D.n[nd - 3];
    per_sm = std::max(per_sm, 1);
    sms = std::max(sms, 1);
    long long pencils = 1;
    for (int d = 0; d < nd - 3; ++d) pencils *= D.n[d];
    const long long base = pencils * bk.nbands;
    const long long res = (long long)per_sm * sms;
    double best = 0.0;
    int best_chunk = 0;
    bool best_deep = false;
    for (int nch = 1; nch <= std::max(1, ns / 4); ++nch) {   // at least four planes per chunk
        int chunk = (ns + nch - 1) / nch;
        // every chunk holds at least two planes (the window fill reads two ahead)
        while (ns % chunk != 0 && ns % chunk < 2) ++chunk;
        const long long items = base * ((ns + chunk - 1) / chunk);
        const long long full = items / res, last = items - full * res;
        const long long c = (last + sms - 1) / sms;
        const double waves = double(full) + (last > 0 ? 0.4 + 0.6 * double(c) / double(per_sm) : 0.0);
        const double cost = waves * double(chunk + 2 * o + 1);
        const bool deep = 2 * items >= 3 * res;
        if (best_chunk == 0 || (deep && !best_deep) || (deep == best_deep && cost < best)) {
            best = cost;
            best_chunk = chunk;
            best_deep = deep;
        }
    }
#ifdef ODP_BULK_NCH
    best_chunk = (ns + ODP_BULK_NCH - 1) / ODP_BULK_NCH;
    while (ns % best_chunk != 0 && ns % best_chunk < 2) ++best_chunk;
#endif
    bk.chunk[o - 1] = best_chunk;
    bk.nchunks[o - 1] = (ns + best_chunk - 1) / best_chunk;
    bk.items[o - 1] = int(base * bk.nchunks[o - 1]);
    bk.div_nchunks[o - 1] = make_fastdiv(uint32_t(bk.nchunks[o - 1]));
}

float odp::rel6d_heading_ceiling(float b, double lo, double hi, int n, int periodic)
{
    // the straddling case max(|b - w_p|, |-b - w_p|) at every w_p node, in
    // float as the kernel evaluates it, at the float node coordinates of the
    // grid's table (the same spacing and rounding as odp_grid_create's)
    const double h = periodic ? (hi - lo) / double(n) : (hi - lo) / double(n - 1);
    float cap = 0.0f;
    for (int i = 0; i < n; ++i) {
        const float wp = float(lo + double(i) * h);
        cap = std::max(cap, std::max(std::fabs(b - wp), std::fabs(-b - wp)));
    }
    return cap;
}

void odp::bulk_geometry(GridDesc &D, int sms, int threads)
{
    BulkGeom &bk = D.bk;
    bk = BulkGeom{};
    const int nd = D.ndim;
    // the pass numbers its outer pencils with the plane pass's blocks
    if (nd < 3 || D.n[nd - 1] % 4 != 0 || !D.pg.use) return;
    const int nr = D.nr, segs = D.segs, ns = D.n[nd - 3];
    if (nr < 4 || ns < 4 || segs > 128) return;
    // every model here has non-periodic stream and row axes; the pass
    // takes only those
    if (D.periodic[nd - 2] || D.periodic[nd - 3]) return;
    // bands of about `threads` compute threads (balanced band heights)
    int rb = std::max(threads, 32) / segs;
    if (rb < 1) rb = 1;
    int nb = 1;
    if (rb >= nr) {
        rb = nr;
    } else {
        nb = (nr + rb - 1) / rb;
        rb = (nr + nb - 1) / nb;
    }
    const int cwarps = (rb * segs + 31) / 32;
    if (cwarps + 1 > 16) return;
    bk.rb = rb;
    bk.nbands = nb;
    bk.cwarps = cwarps;
    bk.rc = ODP_BULK_RC;
    bk.rx = ODP_BULK_RX;
    // (ODP_BULK_RC <= 8 and ODP_BULK_RX <= 6: the barrier area holds that many)
    for (int o = 1; o <= 2; ++o) {
        const long long bytes = bulk_smem_bytes(bk, D.n_pad, nd, o, 3);
        bk.smem[o - 1] = bytes <= 200 * 1024 ? int(bytes) : 0;
    }
    if (bk.smem[0] == 0 && bk.smem[1] == 0) return;
    // resident CTAs per SM estimated from shared memory and threads (about
    // 96 registers a thread); odp_set_dynamics replaces the estimate with
    // the kernels' own occupancy
    for (int o = 1; o <= 2; ++o) {
        const int sm_bytes = bk.smem[o - 1] ? bk.smem[o - 1] : bk.smem[2 - o];
        int per_sm = (228 * 1024) / (sm_bytes + 1024);
        per_sm = std::min(per_sm, 65536 / (96 * 32 * (cwarps + 1)));
        bulk_chunking(D, o, std::max(per_sm, 1), sms);
    }
    bk.div_nbands = make_fastdiv(uint32_t(bk.nbands));
    bk.use = 1;
}

static void release(odp_grid *g)
{
    if (!g) return;
    cudaSetDevice(g->device);
    if (g->stream) cudaStreamSynchronize(g->stream);
    ttr_release(g);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->capture_stream) cudaStreamDestroy(g->capture_stream);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    cudaFree(g->phi_a);
    cudaFree(g->phi_b);
    cudaFree(g->l);
    cudaFree(g->obst);
    cudaFree(g->cdn);
    cudaFree(g->l_seq);
    cudaFree(g->g_seq);
    cudaFree(g->tables);
    cudaFree(g->state);
    cudaFree(g->tau);
    cudaFree(g->snapshots);
    delete g;
}

extern "C" const char *odp_last_error(void) { return g_last_error.c_str(); }

extern "C" const char *odp_version(void) { return "libodp 0.1 (sm_103a)"; }

extern "C" int64_t odp_grid_points(const odp_grid *g) { return g ? g->total : 0; }

extern "C" odp_status odp_plan_geometry(int ndim, const int32_t *n, int64_t *out, int n_out)
{
    if (ndim < 1 || ndim > ODP_MAXD || !n || !out || n_out < 14) return fail(ODP_EINVAL, "bad arguments");
    GridDesc D{};
    D.ndim = ndim;
    int64_t total = 1;
    for (int d = 0; d < ndim; ++d) {
        if (n[d] < 1) return fail(ODP_EINVAL, "axis %d has no nodes", d);
        total *= n[d];
        D.n[d] = n[d];
    }
    const int nl = n[ndim - 1];
    D.n_pad = (nl + 3) / 4 * 4;
    D.segs = D.n_pad / 4;
    D.nr = ndim >= 2 ? n[ndim - 2] : 1;
    D.R = D.nr >= 4 ? 4 : 1;
    D.row_groups = (D.nr + D.R - 1) / D.R;
    D.planes = int(total / nl / D.nr);
    D.nthreads_rb = D.segs * D.row_groups * D.planes;
    plane_geometry(D, 152);
    const PlaneGeom &pg = D.pg;
    const int64_t v[14] = {D.n_pad, D.R, D.row_groups, D.planes, D.nthreads_rb, pg.use, pg.ns,
                           pg.chunk, pg.items, pg.threads, pg.smem[0], pg.smem[1], pg.rb, pg.nbands};
    for (int k = 0; k < 14; ++k) out[k] = v[k];
    return ODP_OK;
}

extern "C" odp_status odp_grid_create(int ndim, const int32_t *n, const double *lo, const double *hi,
                                      const uint8_t *periodic, void *cuda_stream, odp_grid **out)
{
    if (!out) return fail(ODP_EINVAL, "out is NULL");
    *out = nullptr;
    if (ndim < 1 || ndim > ODP_MAXD) return fail(ODP_EINVAL, "ndim %d outside [1, %d]", ndim, ODP_MAXD);
    if (!n || !lo || !hi || !periodic) return fail(ODP_EINVAL, "NULL grid description");
    int64_t total = 1;
    for (int d = 0; d < ndim; ++d) {
        const int need = periodic[d] ? 1 : 2;
        if (n[d] < need) return fail(ODP_EINVAL, "axis %d: n = %d < %d", d, n[d], need);
        if (!(hi[d] > lo[d]) || !std::isfinite(lo[d]) || !std::isfinite(hi[d]))
            return fail(ODP_EINVAL, "axis %d: need finite lo < hi", d);
        total *= n[d];
        if (total >= (int64_t(1) << 31)) return fail(ODP_EINVAL, "grid has 2^31 nodes or more");
    }
    // the kernels index the padded storage (last axis rounded up to a
    // multiple of 4) with 32-bit offsets
    if (total / n[ndim - 1] * ((n[ndim - 1] + 3) / 4 * 4) >= (int64_t(1) << 31))
        return fail(ODP_EINVAL, "padded grid storage has 2^31 floats or more");
    odp_grid *g = new (std::nothrow) odp_grid();
    if (!g) return fail(ODP_ENOMEM, "host allocation failed");
    g->ndim = ndim;
    g->total = total;
    g->stream = static_cast<cudaStream_t>(cuda_stream);
    for (int d = 0; d < ndim; ++d) {
        g->n[d] = n[d];
        g->lo[d] = lo[d];
        g->hi[d] = hi[d];
        g->periodic[d] = periodic[d] ? 1 : 0;
    }
    auto bail = [&](odp_status rc) {
        release(g);
        return rc;
    };
    odp_status rc;
#define ODP_TRY(call)                    \
    do {                                 \
        cudaError_t e_ = (call);         \
        if (e_ != cudaSuccess) {         \
            rc = fail(e_ == cudaErrorMemoryAllocation ? ODP_ENOMEM : ODP_ECUDA, "%s: %s", #call, \
                      cudaGetErrorString(e_)); \
            return bail(rc);             \
        }                                \
    } while (0)
    // work runs on the device of the given stream (or the current device)
    if (g->stream) {
        int dev = -1;
        ODP_TRY(cudaStreamGetDevice(g->stream, &dev));
        ODP_TRY(cudaSetDevice(dev));
    }
    ODP_TRY(cudaGetDevice(&g->device));
    g->n_last = n[ndim - 1];
    g->n_pad = (g->n_last + 3) / 4 * 4;
    g->rows = total / g->n_last;
    g->total_pad = g->rows * g->n_pad;
    const size_t bytes = size_t(g->total_pad) * sizeof(float);
    ODP_TRY(cudaMalloc(&g->phi_a, bytes));
    ODP_TRY(cudaMalloc(&g->phi_b, bytes));
    ODP_TRY(cudaMalloc(&g->l, bytes));
    ODP_TRY(cudaMemset(g->phi_a, 0, bytes));
    ODP_TRY(cudaMemset(g->phi_b, 0, bytes));
    ODP_TRY(cudaMemset(g->l, 0, bytes));
    ODP_TRY(cudaMalloc(&g->state, sizeof(SolveState)));
    ODP_TRY(cudaStreamCreateWithFlags(&g->capture_stream, cudaStreamNonBlocking));
    ODP_TRY(cudaEventCreate(&g->ev0));
    ODP_TRY(cudaEventCreate(&g->ev1));

    // node tables: per axis, coordinates then cos and sin of the coordinates
    // (only an angle axis uses the trig tables), each table padded to a
    // multiple of 4 entries so that four-node segments load them as one
    // vector; float64 on the host, rounded once.
    int64_t tab_len = 0;
    for (int d = 0; d < ndim; ++d) tab_len += 3 * int64_t((n[d] + 3) / 4 * 4);
    std::vector<float> tab(static_cast<size_t>(tab_len), 0.0f);
    GridDesc &D = g->desc;
    D.ndim = ndim;
    D.total = int(total);
    D.n_pad = g->n_pad;
    D.rows = int(g->rows);
    D.segs = g->n_pad / 4;
    D.nthreads = int(g->rows * (g->n_pad / 4));
    D.div_segs = make_fastdiv(uint32_t(D.segs));
    D.nr = ndim >= 2 ? n[ndim - 2] : 1;
    D.R = D.nr >= 4 ? 4 : 1;
    D.row_groups = (D.nr + D.R - 1) / D.R;
    D.planes = int(g->rows / D.nr);
    D.nthreads_rb = D.segs * D.row_groups * D.planes;
    D.div_row_groups = make_fastdiv(uint32_t(D.row_groups));
    int64_t off = 0;
    std::vector<int64_t> coord_off(ndim);
    for (int d = 0; d < ndim; ++d) {
        const double h = periodic[d] ? (hi[d] - lo[d]) / double(n[d]) : (hi[d] - lo[d]) / double(n[d] - 1);
        const int64_t np = (n[d] + 3) / 4 * 4;
        D.n[d] = n[d];
        D.periodic[d] = periodic[d] ? 1 : 0;
        D.dz[d] = h;
        D.inv_dz[d] = float(1.0 / h);
        D.div[d] = make_fastdiv(uint32_t(n[d]));
        coord_off[d] = off;
        for (int i = 0; i < n[d]; ++i) {
            const double z = lo[d] + double(i) * h;
            tab[size_t(off + i)] = float(z);
            tab[size_t(off + np + i)] = float(std::cos(z));
            tab[size_t(off + 2 * np + i)] = float(std::sin(z));
        }
        off += 3 * np;
    }
    int64_t s = 1;
    for (int d = ndim - 1; d >= 0; --d) {
        D.stride[d] = int(s);
        s *= (d == ndim - 1) ? g->n_pad : n[d];
    }
    plane_geometry(D, 152);   // needs the axis sizes above
    bulk_geometry(D, 152, ODP_BULK_THREADS);
    g->bulk_ok = D.bk.use;
    ODP_TRY(cudaMalloc(&g->tables, size_t(tab_len) * sizeof(float)));
    ODP_TRY(cudaMemcpy(g->tables, tab.data(), size_t(tab_len) * sizeof(float), cudaMemcpyHostToDevice));
    for (int d = 0; d < ndim; ++d) D.coord[d] = g->tables + coord_off[d];
    // the trig tables of the angle axis are bound by odp_set_dynamics
    D.cos_tab = nullptr;
    D.sin_tab = nullptr;
    g->dyn.angle_axis = -1;
#undef ODP_TRY
    *out = g;
    return ODP_OK;
}

extern "C" odp_status odp_grid_destroy(odp_grid *g)
{
    release(g);
    return ODP_OK;
}

static int64_t padded4(int n) { return (int64_t(n) + 3) / 4 * 4; }

static int64_t trig_offset(const odp_grid *g, int axis)
{
    int64_t off = 0;
    for (int d = 0; d < axis; ++d) off += 3 * padded4(g->n[d]);
    return off + padded4(g->n[axis]);
}

extern "C" odp_status odp_set_dynamics(odp_grid *g, odp_dyn kind, const double *params, int n_params,
                                       odp_mode u_mode, odp_mode d_mode)
{
    if (!g) return fail(ODP_EINVAL, "grid is NULL");
    if ((u_mode != ODP_MIN && u_mode != ODP_MAX) || (d_mode != ODP_MIN && d_mode != ODP_MAX))
        return fail(ODP_EINVAL, "input modes must be ODP_MIN or ODP_MAX");
    int need = 0, angle = -1, nd_req = -1;
    switch (kind) {
    case ODP_DYN_SINGLE_INT: need = 1; break;
    case ODP_DYN_ADVECTION: need = g->ndim; break;
    case ODP_DYN_DUBINS3D: need = 2; angle = 2; nd_req = 3; break;
    case ODP_DYN_DUBINSCAR4D: need = 2; angle = 3; nd_req = 4; break;
    case ODP_DYN_REL6D: need = 4; angle = 2; nd_req = 6; break;
    case ODP_DYN_DUBINS_CAPTURE: need = 3; angle = 2; nd_req = 3; break;
    default: return fail(ODP_EINVAL, "unknown dynamics %d", int(kind));
    }
    if (nd_req > 0 && g->ndim != nd_req)
        return fail(ODP_EINVAL, "dynamics %d needs %d dimensions, grid has %d", int(kind), nd_req, g->ndim);
    if (n_params < need || n_params > 8 || (need > 0 && !params))
        return fail(ODP_EINVAL, "dynamics %d needs %d parameters, got %d", int(kind), need, n_params);
    for (int k = 0; k < n_params; ++k) {
        if (!std::isfinite(params[k])) return fail(ODP_EINVAL, "parameter %d is not finite", k);
        if (kind != ODP_DYN_ADVECTION && params[k] < 0.0)
            return fail(ODP_EINVAL, "parameter %d (a bound or speed) is negative", k);
    }
    if (angle >= 0 && !g->periodic[angle])
        return fail(ODP_EINVAL, "axis %d holds an angle and must be periodic", angle);
    DynDesc dy{};
    dy.kind = int(kind);
    dy.umode = int(u_mode);
    dy.dmode = int(d_mode);
    dy.angle_axis = angle;
    dy.local_diss = g->local_diss;
    for (int k = 0; k < n_params; ++k) dy.prm[k] = float(params[k]);
    if (kind == ODP_DYN_REL6D) dy.acap = rel6d_heading_ceiling(dy.prm[3], g->lo[4], g->hi[4], g->n[4], g->periodic[4]);
    g->dyn = dy;
    g->dyn_version += 1;
    if (angle >= 0) {
        const int64_t off = trig_offset(g, angle);
        g->desc.cos_tab = g->tables + off;
        g->desc.sin_tab = g->tables + off + padded4(g->n[angle]);
    }
    cudaError_t ce = cudaSuccess;
    ODP_BIND(g);
    switch (dy.kind) {
    case DYN_SINGLE_INT:
    case DYN_ADVECTION: ce = configure_stage_si(g->ndim, dy.kind); break;
    case DYN_DUBINS3D:
    case DYN_DUBINSCAR4D: ce = configure_stage_dubins(g->ndim); break;
    case DYN_CAPTURE: ce = configure_stage_capture(); break;
    default: ce = configure_stage_rel6d(); break;
    }
    if (ce != cudaSuccess) return fail(ODP_ECUDA, "configuring the stage kernels: %s", cudaGetErrorString(ce));
    // the bulk-staged pass: bands sized for the model, stream chunks for the
    // kernels' own occupancy on this device
    if (g->bulk_ok && (dy.kind == DYN_DUBINS3D || dy.kind == DYN_DUBINSCAR4D || dy.kind == DYN_REL6D)) {
        GridDesc &D = g->desc;
        const int use = D.bk.use;
        int sms = 0;
        ODP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device));
        bulk_geometry(D, sms, dy.kind == DYN_DUBINSCAR4D ? ODP_BULK_THREADS4 : ODP_BULK_THREADS);
        if (!D.bk.use) bulk_geometry(D, sms, ODP_BULK_THREADS);   // the shape checked at creation
        D.bk.use = use;
        for (int o = 1; o <= 2 && D.bk.rb > 0; ++o) {
            if (!D.bk.smem[o - 1]) continue;
            // the occupancy of a BRT stage 2 (l and phi^n staged beside the neighbours)
            const int threads = 32 * (D.bk.cwarps + 1);
            const int bytes = int(bulk_smem_bytes(D.bk, D.n_pad, g->ndim, o, 2));
            int per_sm = 0;
            ce = dy.kind == DYN_REL6D ? occupancy_stage_bulk_rel6d(o, threads, bytes, &per_sm)
                                      : occupancy_stage_bulk_dubins(g->ndim, o, threads, bytes, &per_sm);
            if (ce != cudaSuccess)
                return fail(ODP_ECUDA, "occupancy of the bulk-staged pass: %s", cudaGetErrorString(ce));
            if (per_sm > 0) bulk_chunking(D, o, per_sm, sms);
        }
    }
    g->has_dyn = true;
    return ODP_OK;
}

extern "C" odp_status odp_set_target(odp_grid *g, const float *l, int64_t n_elems, int on_device)
{
    if (!g || !l) return fail(ODP_EINVAL, "NULL argument");
    ODP_BIND(g);
    if (n_elems != g->total) return fail(ODP_EINVAL, "target has %lld values, grid has %lld",
                                         (long long)n_elems, (long long)g->total);
    ODP_CUDA(cudaMemcpy2DAsync(g->l, size_t(g->n_pad) * sizeof(float), l, size_t(g->n_last) * sizeof(float),
                               size_t(g->n_last) * sizeof(float), size_t(g->rows),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->stream));
    g->has_target = true;
    if (g->l_seq_n) {   // a time-invariant target replaces a schedule
        g->l_seq_n = 0;
        g->sched_version += 1;
    }
    return ODP_OK;
}

// n_sets dense arrays of n_elems floats into the padded layout at *dst
// (grown to hold them; padding lanes zero).
static odp_status copy_sets(odp_grid *g, float **dst, int *cap, const float *src, int n_sets, int64_t n_elems,
                            int on_device, const char *what)
{
    if (n_sets < 2) return fail(ODP_EINVAL, "a %s schedule needs a set per tau (at least 2)", what);
    if (n_elems != g->total) return fail(ODP_EINVAL, "%s sets have %lld values, grid has %lld", what,
                                         (long long)n_elems, (long long)g->total);
    const size_t per = size_t(g->total_pad);
    if (n_sets > *cap) {
        ODP_CUDA(cudaStreamSynchronize(g->stream));
        cudaFree(*dst);
        *dst = nullptr;
        *cap = 0;
        if (cudaMalloc(dst, sizeof(float) * per * size_t(n_sets)) != cudaSuccess) {
            cudaGetLastError();
            *dst = nullptr;
            return fail(ODP_ENOMEM, "%s schedule of %d sets", what, n_sets);
        }
        *cap = n_sets;
        ODP_CUDA(cudaMemsetAsync(*dst, 0, sizeof(float) * per * size_t(n_sets), g->stream));
    }
    for (int k = 0; k < n_sets; ++k)
        ODP_CUDA(cudaMemcpy2DAsync(*dst + size_t(k) * per, size_t(g->n_pad) * sizeof(float),
                                   src + k * n_elems, size_t(g->n_last) * sizeof(float),
                                   size_t(g->n_last) * sizeof(float), size_t(g->rows),
                                   on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->stream));
    return ODP_OK;
}

extern "C" odp_status odp_set_target_schedule(odp_grid *g, const float *l_seq, int n_sets, int64_t n_elems,
                                              int on_device)
{
    if (!g) return fail(ODP_EINVAL, "grid is NULL");
    if (!l_seq) {
        if (g->l_seq_n) g->sched_version += 1;
        g->l_seq_n = 0;
        return ODP_OK;
    }
    ODP_BIND(g);
    odp_status rc = copy_sets(g, &g->l_seq, &g->l_seq_cap, l_seq, n_sets, n_elems, on_device, "target");
    if (rc != ODP_OK) return rc;
    g->l_seq_n = n_sets;
    g->has_target = true;
    g->sched_version += 1;
    return ODP_OK;
}

extern "C" odp_status odp_set_obstacle_schedule(odp_grid *g, const float *g_seq, int n_sets, int64_t n_elems,
                                                int on_device)
{
    if (!g) return fail(ODP_EINVAL, "grid is NULL");
    if (!g_seq) {
        if (g->g_seq_n) {
            g->sched_version += 1;
            g->has_obst = false;
        }
        g->g_seq_n = 0;
        return ODP_OK;
    }
    ODP_BIND(g);
    const size_t bytes = size_t(g->total_pad) * sizeof(float);
    if (!g->obst) {
        if (cudaMalloc(&g->obst, bytes) != cudaSuccess) {
            cudaGetLastError();
            g->obst = nullptr;
            return fail(ODP_ENOMEM, "obstacle array of %zu bytes", bytes);
        }
        ODP_CUDA(cudaMemsetAsync(g->obst, 0, bytes, g->stream));
    }
    odp_status rc = copy_sets(g, &g->g_seq, &g->g_seq_cap, g_seq, n_sets, n_elems, on_device, "obstacle");
    if (rc != ODP_OK) return rc;
    g->g_seq_n = n_sets;
    g->has_obst = true;
    g->sched_version += 1;
    return ODP_OK;
}

extern "C" odp_status odp_set_obstacle(odp_grid *g, const float *gv, int64_t n_elems, int on_device)
{
    if (!g) return fail(ODP_EINVAL, "grid is NULL");
    if (g->g_seq_n) {   // a time-invariant obstacle (or none) replaces a schedule
        g->g_seq_n = 0;
        g->sched_version += 1;
    }
    if (!gv) {
        g->has_obst = false;
        return ODP_OK;
    }
    ODP_BIND(g);
    if (n_elems != g->total) return fail(ODP_EINVAL, "obstacle has %lld values, grid has %lld",
                                         (long long)n_elems, (long long)g->total);
    if (!g->obst) {
        const size_t bytes = size_t(g->total_pad) * sizeof(float);
        if (cudaMalloc(&g->obst, bytes) != cudaSuccess) {
            cudaGetLastError();
            g->obst = nullptr;
            return fail(ODP_ENOMEM, "obstacle array of %zu bytes", bytes);
        }
        ODP_CUDA(cudaMemsetAsync(g->obst, 0, bytes, g->stream));
    }
    ODP_CUDA(cudaMemcpy2DAsync(g->obst, size_t(g->n_pad) * sizeof(float), gv, size_t(g->n_last) * sizeof(float),
                               size_t(g->n_last) * sizeof(float), size_t(g->rows),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->stream));
    g->has_obst = true;
    return ODP_OK;
}

extern "C" odp_status odp_set_dissipation(odp_grid *g, int per_node)
{
    if (!g) return fail(ODP_EINVAL, "grid is NULL");
    if (per_node != 0 && per_node != 1) return fail(ODP_EINVAL, "per_node must be 0 or 1");
    if (g->local_diss != per_node) {
        g->local_diss = per_node;
        g->dyn.local_diss = per_node;
        g->dyn_version += 1;   // the captured loop holds the old flag
    }
    return ODP_OK;
}

extern "C" odp_status odp_set_step_limit(odp_grid *g, int64_t max_steps)
{
    if (!g || max_steps < 1) return fail(ODP_EINVAL, "need a grid and max_steps >= 1");
    g->max_steps = max_steps;
    return ODP_OK;
}

// ---------------------------------------------------------------------------
// the time-loop graph
// ---------------------------------------------------------------------------
// alpha components that depend on phi and are reduced again every stage
static unsigned dynamic_alpha_mask(const odp_grid *g)
{
    return g->dyn.kind == DYN_REL6D ? (1u << 2) : (g->dyn.kind == DYN_CAPTURE ? 7u : 0u);
}

static cudaError_t launch_alpha_dynamic(const odp_grid *g, int slot, cudaStream_t s)
{
    if (g->dyn.kind == DYN_CAPTURE) return launch_alpha_dynamic_capture(g->desc, g->dyn, g->state, g->order, slot, s);
    return launch_alpha_dynamic_rel6d(g->desc, g->dyn, g->state, g->order, slot, s);
}

static cudaError_t launch_stage_any(odp_grid *g, int stage, cudaStream_t s)
{
    const GridDesc &D = g->desc;
    const float *gob = g->has_obst ? g->obst : nullptr;
    switch (g->dyn.kind) {
    case DYN_SINGLE_INT:
    case DYN_ADVECTION:
        return launch_stage_si(g->ndim, D, g->dyn, g->state, g->l, gob, g->order, stage, g->brt, s);
    case DYN_DUBINS3D:
    case DYN_DUBINSCAR4D:
        return launch_stage_dubins(g->ndim, D, g->dyn, g->state, g->l, gob, g->order, stage, g->brt, s);
    case DYN_CAPTURE:
        return launch_stage_capture(D, g->dyn, g->state, g->l, gob, g->order, stage, g->brt, s);
    default:
        return launch_stage_rel6d(D, g->dyn, g->state, g->l, gob, g->order, stage, g->brt, s);
    }
}

// The kernels of one full time step, in order, on stream s: the per-stage alpha
// pass, the CFL step, the stage pass(es) and the closing k_advance.  Used for
// the captured graph body (in_graph = 1) and for the host-stepped loop.
static int seq_active(const odp_grid *g) { return (g->l_seq_n > 0 || g->g_seq_n > 0) ? 1 : 0; }

static cudaError_t launch_seq_sets(odp_grid *g, cudaStream_t s)
{
    const int blocks = int(std::min<int64_t>((g->total_pad + 255) / 256, 152 * 8));
    k_seq_sets<<<blocks, 256, 0, s>>>(g->state, g->l, g->l_seq_n ? g->l_seq : nullptr, g->obst,
                                      g->g_seq_n ? g->g_seq : nullptr, int(g->total_pad));
    return cudaGetLastError();
}

static cudaError_t launch_step(odp_grid *g, cudaStream_t s, cudaGraphConditionalHandle h_loop,
                               cudaGraphConditionalHandle h_snap, cudaGraphConditionalHandle h_seq, int in_graph,
                               int64_t *launches)
{
    const bool dyn_alpha = dynamic_alpha_mask(g) != 0;
    int64_t n = 0;
    cudaError_t e = cudaSuccess;
    if (dyn_alpha) {
        e = launch_alpha_dynamic(g, 0, s);
        ++n;
    }
    // phi-independent alpha: the step's dt comes from the previous step's
    // k_advance (or, for the first step, the k_dt launched before the loop)
    if (e == cudaSuccess && dyn_alpha) {
        k_dt<<<1, 1, 0, s>>>(g->state, g->desc);
        ++n;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        if (g->time_order == 1) {
            e = launch_stage_any(g, 0, s);
            ++n;
        } else {
            e = launch_stage_any(g, 1, s);
            ++n;
            if (e == cudaSuccess && dyn_alpha) {
                e = launch_alpha_dynamic(g, 1, s);
                ++n;
            }
            if (e == cudaSuccess) {
                e = launch_stage_any(g, 2, s);
                ++n;
            }
        }
    }
    if (e == cudaSuccess) {
        k_advance<<<1, 1, 0, s>>>(g->state, g->desc, g->time_order == 1 ? 1 : 0, dynamic_alpha_mask(g),
                                  dyn_alpha ? 0 : 1, h_loop, h_snap, g->keep, h_seq, seq_active(g), in_graph);
        ++n;
        e = cudaGetLastError();
    }
    if (launches) *launches = n;
    return e;
}

static cudaError_t launch_alpha_static_any(odp_grid *g, cudaStream_t s)
{
    switch (g->dyn.kind) {
    case DYN_SINGLE_INT:
    case DYN_ADVECTION: return launch_alpha_static_si(g->ndim, g->desc, g->dyn, g->state, s);
    case DYN_DUBINS3D:
    case DYN_DUBINSCAR4D: return launch_alpha_static_dubins(g->ndim, g->desc, g->dyn, g->state, s);
    case DYN_CAPTURE: return launch_alpha_static_capture(g->desc, g->dyn, g->state, s);
    default: return launch_alpha_static_rel6d(g->desc, g->dyn, g->state, s);
    }
}


// Capture the body of the time loop into `body` and add the snapshot IF node.
static odp_status build_graph(odp_grid *g)
{
    if (g->exec) {
        ODP_CUDA(cudaStreamSynchronize(g->stream));
        cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
    }
    if (g->graph) {
        cudaGraphDestroy(g->graph);
        g->graph = nullptr;
    }
    ODP_CUDA(cudaGraphCreate(&g->graph, 0));
    cudaGraphConditionalHandle h_loop;
    ODP_CUDA(cudaGraphConditionalHandleCreate(&h_loop, g->graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams wp{};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = h_loop;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t loop_node;
    ODP_CUDA(cudaGraphAddNode(&loop_node, g->graph, nullptr, nullptr, 0, &wp));
    cudaGraph_t body = wp.conditional.phGraph_out[0];

    cudaGraphConditionalHandle h_snap = 0, h_seq = 0;
    if (g->keep) ODP_CUDA(cudaGraphConditionalHandleCreate(&h_snap, body, 0, 0));
    if (seq_active(g)) ODP_CUDA(cudaGraphConditionalHandleCreate(&h_seq, body, 0, 0));

    cudaStream_t s = g->capture_stream;
    ODP_CUDA(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    int64_t launches = 0;
    cudaError_t e = launch_step(g, s, h_loop, h_snap, h_seq, 1, &launches);
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    std::vector<cudaGraphNode_t> leaf;
    if (e == cudaSuccess) {
        e = cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &deps, nullptr, &ndeps);
        if (e == cudaSuccess) leaf.assign(deps, deps + ndeps);
    }
    cudaGraph_t captured = body;
    cudaError_t e2 = cudaStreamEndCapture(s, &captured);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        // the graph of a failed capture is dropped, not destroyed
        cudaGetLastError();
        g->graph = nullptr;
        if (e != cudaSuccess) return fail(ODP_ECUDA, "capturing the time loop: %s", cudaGetErrorString(e));
        return fail(ODP_ECUDA, "ending the capture: %s", cudaGetErrorString(e2));
    }

    if (g->keep) {
        cudaGraphNodeParams ip{};
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = h_snap;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        cudaGraphNode_t if_node;
        ODP_CUDA(cudaGraphAddNode(&if_node, body, leaf.data(), nullptr, leaf.size(), &ip));
        cudaGraph_t snap_body = ip.conditional.phGraph_out[0];
        ODP_CUDA(cudaStreamBeginCaptureToGraph(s, snap_body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        const int blocks = int(std::min<int64_t>((g->total_pad + 255) / 256, 152 * 8));
        k_snapshot<<<blocks, 256, 0, s>>>(g->state, int(g->total_pad));
        e = cudaGetLastError();
        cudaGraph_t cap2 = snap_body;
        e2 = cudaStreamEndCapture(s, &cap2);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            cudaGetLastError();
            g->graph = nullptr;
            return fail(ODP_ECUDA, "capturing the snapshot copy: %s / %s", cudaGetErrorString(e),
                        cudaGetErrorString(e2));
        }
    }
    if (seq_active(g)) {
        cudaGraphNodeParams ip{};
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = h_seq;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        cudaGraphNode_t if_node;
        ODP_CUDA(cudaGraphAddNode(&if_node, body, leaf.data(), nullptr, leaf.size(), &ip));
        cudaGraph_t seq_body = ip.conditional.phGraph_out[0];
        ODP_CUDA(cudaStreamBeginCaptureToGraph(s, seq_body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        e = launch_seq_sets(g, s);
        cudaGraph_t cap3 = seq_body;
        e2 = cudaStreamEndCapture(s, &cap3);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            cudaGetLastError();
            g->graph = nullptr;
            return fail(ODP_ECUDA, "capturing the set copy: %s / %s", cudaGetErrorString(e), cudaGetErrorString(e2));
        }
    }
    cudaError_t ei = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (ei != cudaSuccess) {
        g->exec = nullptr;
        cudaGraphDestroy(g->graph);
        g->graph = nullptr;
        return fail(ODP_ECUDA, "instantiating the time loop: %s", cudaGetErrorString(ei));
    }
    g->launches_per_step = launches;
    return ODP_OK;
}

// The time loop stepped from the host: the kernels of the graph body launched
// one step at a time, the loop and snapshot conditions read back after each
// step (one synchronisation per step).
static odp_status run_host_loop(odp_grid *g)
{
    cudaStream_t s = g->stream;
    SolveState *h = nullptr;
    ODP_CUDA(cudaMallocHost(&h, sizeof(SolveState)));
    odp_status rc = ODP_OK;
    int seg_before = 0;
    for (;;) {
        cudaError_t e = launch_step(g, s, 0, 0, 0, 0, nullptr);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, g->state, sizeof(SolveState), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && h->snap_now) {
            const int blocks = int(std::min<int64_t>((g->total_pad + 255) / 256, 152 * 8));
            k_snapshot<<<blocks, 256, 0, s>>>(g->state, int(g->total_pad));
            e = cudaGetLastError();
        }
        // a new segment started: its time-varying sets (the graph's IF node)
        if (e == cudaSuccess && seq_active(g) && h->go && h->seg != seg_before) e = launch_seq_sets(g, s);
        seg_before = h->seg;
        if (e != cudaSuccess) {
            rc = fail(ODP_ECUDA, "host-stepped time loop: %s", cudaGetErrorString(e));
            break;
        }
        if (!h->go) break;
    }
    cudaFreeHost(h);
    return rc;
}

extern "C" odp_status odp_set_loop_mode(odp_grid *g, int host_stepped)
{
    if (!g) return fail(ODP_EINVAL, "grid is NULL");
    if (host_stepped != 0 && host_stepped != 1) return fail(ODP_EINVAL, "host_stepped must be 0 or 1");
    g->host_loop = host_stepped;
    return ODP_OK;
}

extern "C" odp_status odp_set_stage_pass(odp_grid *g, int pass)
{
    if (!g) return fail(ODP_EINVAL, "grid is NULL");
    if (pass < 0 || pass > 2) return fail(ODP_EINVAL, "pass must be 0, 1 or 2");
    if (pass == 2 && !g->bulk_ok)
        return fail(ODP_EINVAL, "the bulk-staged pass does not apply to this grid's shape");
    const int use = g->bulk_ok ? (pass == 0 ? 1 : pass == 2 ? 2 : 0) : 0;
    g->stage_pass = pass;
    if (g->desc.bk.use != use) {
        g->desc.bk.use = use;
        g->dyn_version += 1;   // the captured loop holds the old kernels
    }
    return ODP_OK;
}

extern "C" odp_status odp_solve_hjb(odp_grid *g, const double *tau, int n_tau, odp_set set,
                                    int space_order, int time_order, double cfl, int keep_snapshots,
                                    odp_solve_stats *stats)
{
    if (!g) return fail(ODP_EINVAL, "grid is NULL");
    if (!g->has_dyn) return fail(ODP_ESTATE, "odp_set_dynamics was not called");
    if (!g->has_target) return fail(ODP_ESTATE, "odp_set_target was not called");
    if (!tau || n_tau < 2) return fail(ODP_EINVAL, "need n_tau >= 2");
    if (g->l_seq_n && g->l_seq_n != n_tau)
        return fail(ODP_EINVAL, "the target schedule holds %d sets, the solve has %d taus", g->l_seq_n, n_tau);
    if (g->g_seq_n && g->g_seq_n != n_tau)
        return fail(ODP_EINVAL, "the obstacle schedule holds %d sets, the solve has %d taus", g->g_seq_n, n_tau);
    if (tau[0] != 0.0) return fail(ODP_EINVAL, "tau[0] must be 0");
    for (int k = 1; k < n_tau; ++k)
        if (!(tau[k] > tau[k - 1]) || !std::isfinite(tau[k]))
            return fail(ODP_EINVAL, "tau must be finite and strictly increasing");
    if (set != ODP_BRS && set != ODP_BRT) return fail(ODP_EINVAL, "set must be ODP_BRS or ODP_BRT");
    if (space_order != 1 && space_order != 2) return fail(ODP_EINVAL, "space_order must be 1 or 2");
    if (time_order != 1 && time_order != 2) return fail(ODP_EINVAL, "time_order must be 1 or 2");
    if (!(cfl > 0.0 && cfl <= 1.0)) return fail(ODP_EINVAL, "cfl must lie in (0, 1]");
    ODP_BIND(g);

    cudaStream_t st = g->stream;
    if (n_tau > g->tau_cap) {
        cudaFree(g->tau);
        g->tau = nullptr;
        ODP_CUDA(cudaMalloc(&g->tau, sizeof(double) * size_t(n_tau)));
        g->tau_cap = n_tau;
    }
    if (keep_snapshots && n_tau > g->snap_cap) {
        cudaStreamSynchronize(st);
        cudaFree(g->snapshots);
        g->snapshots = nullptr;
        g->snap_cap = 0;
        ODP_CUDA(cudaMalloc(&g->snapshots, sizeof(float) * size_t(n_tau) * size_t(g->total_pad)));
        g->snap_cap = n_tau;
    }
    g->order = space_order;
    g->time_order = time_order;
    g->brt = (set == ODP_BRT) ? 1 : 0;
    g->keep = keep_snapshots ? 1 : 0;
    g->n_tau = n_tau;
    // per-node dissipation of the capture model: the alpha pass writes each
    // node's coefficients into a buffer the stage pass reads (allocated on
    // first use, 3 arrays of total_pad floats)
    float *cdn = nullptr;
    if (g->dyn.kind == DYN_CAPTURE && g->local_diss) {
        if (!g->cdn) {
            const size_t bytes = 3 * size_t(g->total_pad) * sizeof(float);
            if (cudaMalloc(&g->cdn, bytes) != cudaSuccess) {
                cudaGetLastError();
                g->cdn = nullptr;
                return fail(ODP_ENOMEM, "per-node dissipation buffer of %zu bytes", bytes);
            }
        }
        cdn = g->cdn;
    }
    if (g->desc.cdn != cdn) {
        g->desc.cdn = cdn;
        g->desc.cdn_stride = int(g->total_pad);
        g->dyn_version += 1;   // the captured loop holds the old descriptor
    }
    GraphKey key;
    key.order = space_order;
    key.time_order = time_order;
    key.brt = g->brt;
    key.keep = g->keep;
    key.obstacle = g->has_obst ? 1 : 0;
    key.dyn_version = g->dyn_version;
    key.sched_version = g->sched_version;
    if (!g->exec || !(key == g->key)) {
        odp_status rc = build_graph(g);
        if (rc != ODP_OK) return rc;
        g->key = key;
    }

    // state of the solve; pageable source, so the copy is staged at once
    SolveState h{};
    h.t = 0.0;
    h.t_end = tau[1];
    h.dt = 0.0;
    h.cfl = cfl;
    h.steps = 0;
    h.max_steps = g->max_steps;
    h.seg = 0;
    h.n_seg = n_tau - 1;
    h.flags = 0;
    h.cur = g->phi_a;
    h.nxt = g->phi_b;
    h.tau = g->tau;
    h.snapshots = g->keep ? g->snapshots : nullptr;
    const size_t bytes = size_t(g->total_pad) * sizeof(float);
    ODP_CUDA(cudaMemcpyAsync(g->tau, tau, sizeof(double) * size_t(n_tau), cudaMemcpyHostToDevice, st));
    ODP_CUDA(cudaMemcpyAsync(g->state, &h, sizeof(h), cudaMemcpyHostToDevice, st));
    // phi(0): the target, or the first set of a target schedule; a schedule's
    // first segment takes the sets at tau[1]
    const float *phi0 = g->l_seq_n ? g->l_seq : g->l;
    ODP_CUDA(cudaMemcpyAsync(g->phi_a, phi0, bytes, cudaMemcpyDeviceToDevice, st));
    if (g->keep) ODP_CUDA(cudaMemcpyAsync(g->snapshots, phi0, bytes, cudaMemcpyDeviceToDevice, st));
    if (g->l_seq_n)
        ODP_CUDA(cudaMemcpyAsync(g->l, g->l_seq + g->total_pad, bytes, cudaMemcpyDeviceToDevice, st));
    if (g->g_seq_n)
        ODP_CUDA(cudaMemcpyAsync(g->obst, g->g_seq + g->total_pad, bytes, cudaMemcpyDeviceToDevice, st));
    ODP_CUDA(launch_alpha_static_any(g, st));
    if (!dynamic_alpha_mask(g)) {   // the first step's dt (later ones: k_advance)
        k_dt<<<1, 1, 0, st>>>(g->state, g->desc);
        ODP_CUDA(cudaGetLastError());
    }
    g->timed = stats != nullptr;
    if (g->timed) ODP_CUDA(cudaEventRecord(g->ev0, st));
    if (g->host_loop) {
        odp_status rc = run_host_loop(g);
        if (rc != ODP_OK) return rc;
    } else {
        ODP_CUDA(cudaGraphLaunch(g->exec, st));
    }
    if (g->timed) ODP_CUDA(cudaEventRecord(g->ev1, st));
    g->solved = true;
    if (stats) return odp_solve_status(g, stats);
    return ODP_OK;
}

static odp_status read_state(odp_grid *g, SolveState *h)
{
    ODP_CUDA(cudaMemcpyAsync(h, g->state, sizeof(*h), cudaMemcpyDeviceToHost, g->stream));
    ODP_CUDA(cudaStreamSynchronize(g->stream));
    return ODP_OK;
}

static odp_status status_of(const SolveState &h)
{
    if (h.flags & FLAG_COPY) return fail(ODP_ECUDA, "a bulk copy into shared memory did not complete");
    if (h.flags & FLAG_NONFINITE) return fail(ODP_ENUMERIC, "a non-finite value appeared in the solve");
    if (h.flags & FLAG_TIMEOUT)
        return fail(ODP_ETIMEOUT, "step limit %lld reached at t = %g", (long long)h.max_steps, h.t);
    return ODP_OK;
}

extern "C" odp_status odp_solve_status(odp_grid *g, odp_solve_stats *stats)
{
    if (!g) return fail(ODP_EINVAL, "grid is NULL");
    if (!g->solved) return fail(ODP_ESTATE, "no solve was issued on this grid");
    ODP_BIND(g);
    SolveState h{};
    odp_status rs = read_state(g, &h);
    if (rs != ODP_OK) return rs;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->steps = h.steps;
        stats->last_dt = h.dt;
        stats->t_final = h.t;
        for (int d = 0; d < g->ndim; ++d) memcpy(&stats->alpha[d], &h.alpha_last[d], sizeof(float));
        if (g->timed) {
            float ms = 0.0f;
            ODP_CUDA(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
            stats->device_ms = ms;
        }
        // algorithmic HBM bytes per node per step: every stage reads phi once
        // and writes its result; stage 2 also reads phi^n; the last stage of a
        // tube reads l (and the obstacle of a reach-avoid solve).
        const double per_stage_rw = 8.0;
        double b = (g->time_order == 1) ? per_stage_rw : (2 * per_stage_rw + 4.0);
        if (g->brt) b += 4.0;
        if (g->has_obst) b += 4.0;
        // the capture model's alpha pass reads phi once per stage; the Rel6D
        // heading-rate pass stops once its ceiling is reached, so its reads
        // are not counted
        if (dynamic_alpha_mask(g) && g->dyn.kind != DYN_REL6D) b += 4.0 * g->time_order;
        // capture model with per-node dissipation: each stage writes and
        // reads three coefficients per node
        if (g->desc.cdn) b += 24.0 * g->time_order;
        stats->bytes = b * double(g->total) * double(h.steps);
        // the once-per-solve alpha reduction (and first k_dt) included
        stats->launches = g->launches_per_step * h.steps + (dynamic_alpha_mask(g) ? 1 : 2);
    }
    return status_of(h);
}

extern "C" odp_status odp_value_readback(odp_grid *g, int tau_index, float *dst, int64_t n_elems,
                                         int on_device)
{
    if (!g || !dst) return fail(ODP_EINVAL, "NULL argument");
    if (!g->solved) return fail(ODP_ESTATE, "no solve was issued on this grid");
    if (n_elems != g->total) return fail(ODP_EINVAL, "destination holds %lld values, grid has %lld",
                                         (long long)n_elems, (long long)g->total);
    if (tau_index < -1 || tau_index >= g->n_tau) return fail(ODP_EINVAL, "tau_index %d out of range", tau_index);
    if (tau_index == g->n_tau - 1) tau_index = -1;
    if (tau_index >= 0 && !g->keep) return fail(ODP_EINVAL, "snapshots were not kept");
    ODP_BIND(g);
    SolveState h{};
    odp_status rs = read_state(g, &h);
    if (rs != ODP_OK) return rs;
    const float *src = (tau_index >= 0) ? g->snapshots + size_t(tau_index) * size_t(g->total_pad) : h.cur;
    ODP_CUDA(cudaMemcpy2DAsync(dst, size_t(g->n_last) * sizeof(float), src, size_t(g->n_pad) * sizeof(float),
                               size_t(g->n_last) * sizeof(float), size_t(g->rows),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream));
    ODP_CUDA(cudaStreamSynchronize(g->stream));
    return status_of(h);
}

extern "C" odp_status odp_time_stage(odp_grid *g, int stage, int reps, double *ms_out)
{
    if (!g || !ms_out) return fail(ODP_EINVAL, "NULL argument");
    if (!g->solved || !g->exec) return fail(ODP_ESTATE, "no solve was issued on this grid");
    if (reps < 1) return fail(ODP_EINVAL, "reps must be >= 1");
    if ((g->time_order == 1) != (stage == 0) || stage < 0 || stage > 2)
        return fail(ODP_EINVAL, "stage %d does not belong to a time order %d solve", stage, g->time_order);
    ODP_BIND(g);
    cudaStream_t s = g->capture_stream;
    ODP_CUDA(cudaStreamSynchronize(g->stream));
    ODP_CUDA(cudaEventRecord(g->ev0, s));
    for (int r = 0; r < reps; ++r) {
        cudaError_t e = launch_stage_any(g, stage, s);
        if (e != cudaSuccess) return fail(ODP_ECUDA, "stage launch: %s", cudaGetErrorString(e));
    }
    ODP_CUDA(cudaEventRecord(g->ev1, s));
    ODP_CUDA(cudaEventSynchronize(g->ev1));
    float ms = 0.0f;
    ODP_CUDA(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
    *ms_out = double(ms) / reps;
    g->timed = false;
    return ODP_OK;
}
