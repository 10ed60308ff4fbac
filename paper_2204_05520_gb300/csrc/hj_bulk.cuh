// hj_bulk.cuh -- bulk-staged stage pass (K2) of a single solve for grids of 3
// or more dimensions whose last axis is a multiple of four nodes.
//
// The same sweep as the plane-streaming pass (hj_plane.cuh): the last two
// axes form the plane (rows of axis nd-2, the last axis fastest), axis nd-3
// is the stream axis, the remaining axes are outer axes; a CTA owns a band of
// plane rows at fixed outer indices for a chunk of the stream axis and walks
// it plane by plane, each compute thread owning one four-node segment.
//
// What differs is who moves the data.  One producer thread per CTA stages,
// with the bulk-copy engine (cp.async.bulk, completion counted in bytes on
// an mbarrier), every value the compute threads read:
//   * centre tiles: plane s of the band with its stencil halo rows above and
//     below (one contiguous run of rows in the C-order storage, so one copy;
//     a periodic row axis adds the wrapped rows), in a ring of RC slots;
//   * neighbour tiles: plane s of the band at each outer-axis neighbour index
//     (one copy each), in a ring of RX slots.
// The compute threads read everything from shared memory: the row-axis and
// last-axis neighbours from the centre tile of plane s, the outer-axis
// neighbours from the neighbour tiles, and the stream-axis neighbours from a
// register window that takes its newest value from the centre tile of plane
// s + r.  Ghost nodes outside a non-periodic axis (Section 3.1.1) are formed
// by the threads that use them.  Each compute warp releases a slot when it
// is done with it; there is no CTA-wide barrier per plane.
//
// Every wait on an mbarrier is bounded in time: a wait that gives up sets
// FLAG_COPY, the compute threads stop, and the producer waits (bounded
// again) for the copies it has in flight before the CTA exits.
#pragma once

#include <type_traits>

#include <type_traits>

#include "hj_kernels.cuh"
#include "hj_plane.cuh"

namespace odp {

// ---------------------------------------------------------------------------
// mbarrier and bulk-copy primitives (PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arrive once and add tx bytes to the barrier's expected transaction count.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t tx)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(tx)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

#ifndef ODP_BULK_WAITMODE
#define ODP_BULK_WAITMODE 0
#endif
// Poll the barrier once: test_wait (no suspension), or try_wait, which may
// suspend the thread for a while (a suspend-time hint in ns caps that).
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
#if ODP_BULK_WAITMODE == 1
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
#elif ODP_BULK_WAITMODE == 2
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity), "r"(200u)
        : "memory");
#else
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
#endif
    return done != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until the barrier's phase with the given parity has completed; false
// if it has not within BULK_WAIT_NS (or an iteration cap as a second bound).
constexpr uint64_t BULK_WAIT_NS = 2000000000ull;   // 2 s
constexpr uint32_t BULK_WAIT_ITERS = 1u << 26;

static __device__ __noinline__ bool mbar_wait_slow(uint64_t *bar, uint32_t parity)
{
    const uint64_t t0 = global_ns();
#ifndef ODP_BULK_BACKOFF
#define ODP_BULK_BACKOFF 0
#endif
    for (uint32_t it = 0; it < BULK_WAIT_ITERS; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (ODP_BULK_BACKOFF && it >= 4) __nanosleep(ODP_BULK_BACKOFF);   // leave issue slots to working warps
        if ((it & 63u) == 63u && global_ns() - t0 > BULK_WAIT_NS) return false;
    }
    return false;
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    return mbar_wait_slow(bar, parity);
}

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global memory into this CTA's shared memory, completion counted on bar.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// the pass
// ---------------------------------------------------------------------------
constexpr int BULK_RC_MAX = 8, BULK_RX_MAX = 6;
// read-once tiles staged beside the neighbour tiles of a plane: l, phi^n,
// the obstacle (each the band's rows of the plane)
constexpr int BULK_AUX = 3;
// barriers (full and empty per centre slot, empty per neighbour slot: at
// most 176 bytes), the ghost-rule count at byte 192 and up to 16 rules of
// 16 bytes from byte 208 (a grid has at most 2 r x 3 = 12), then the rings
constexpr int BULK_GHOST_MAX = 16;
constexpr int BULK_BAR_AREA = 512;
static_assert(8 * (2 * BULK_RC_MAX + BULK_RX_MAX) <= 192, "barriers overlap the ghost table");
static_assert(208 + 16 * BULK_GHOST_MAX <= BULK_BAR_AREA, "the ghost table overlaps the rings");

// One ghost rule of an outer-axis neighbour slot that is not staged: slot
// dst is formed from slots b and i (-1: the centre tile) k cells outside.
struct BulkGhost {
    int dst, b, i;
    float k;
};

// Shared-memory layout of one CTA.
struct BulkSmem {
    uint64_t *full_c, *empty_c, *empty_x;
    int *nghost;
    BulkGhost *ghost;
    float *ring_c, *ring_x;
};

__device__ __forceinline__ BulkSmem bulk_smem(unsigned char *raw, const BulkGeom &bk, int ctile)
{
    BulkSmem s;
    uint64_t *b = reinterpret_cast<uint64_t *>(raw);
    s.full_c = b;
    s.empty_c = b + BULK_RC_MAX;
    s.empty_x = b + 2 * BULK_RC_MAX;
    s.nghost = reinterpret_cast<int *>(raw + 192);
    s.ghost = reinterpret_cast<BulkGhost *>(raw + 208);
    s.ring_c = reinterpret_cast<float *>(raw + BULK_BAR_AREA);
    s.ring_x = s.ring_c + bk.rc * ctile;
    return s;
}

// Where one outer-axis neighbour (offset o along outer axis d) of the CTA's
// pencil comes from: a staged tile (delta: its storage offset from the
// pencil), or a ghost node k cells outside the boundary formed from the
// boundary and inner nodes, each either the centre (-1) or a staged
// neighbour (its slot 0 .. 2r-1 along the same axis).
struct BulkNb {
    int staged, delta;
    int gb, gi;
    float k;
};

template <int O>
__device__ __forceinline__ void bulk_neighbours(const GridDesc &g, int d, int id, BulkNb *nb)
{
    const int n = g.n[d];
    int k = 0;
#pragma unroll
    for (int o = -O; o <= O; ++o) {
        if (o == 0) continue;
        BulkNb q{};
        int jd = id + o;
        if (g.periodic[d]) {
            while (jd < 0) jd += n;
            while (jd >= n) jd -= n;
            q.staged = 1;
            q.delta = (jd - id) * g.stride[d];
        } else if (jd >= 0 && jd < n) {
            q.staged = 1;
            q.delta = (jd - id) * g.stride[d];
        } else {
            const int b = jd < 0 ? 0 : n - 1, in = jd < 0 ? 1 : n - 2;
            q.k = jd < 0 ? float(-jd) : float(jd - (n - 1));
            // slot of offset ob in {-O..-1, 1..O}: ob < 0 -> ob + O, ob > 0 -> ob + O - 1
            const int ob = b - id, oi = in - id;
            q.gb = ob == 0 ? -1 : (ob < 0 ? ob + O : ob + O - 1);
            q.gi = oi == 0 ? -1 : (oi < 0 ? oi + O : oi + O - 1);
        }
        nb[k++] = q;
    }
}

// The producer: one thread issues every copy of the CTA's chunk in the order
// the compute warps consume them.  The centre tiles of the first 2r planes
// (the window fill) complete on their own full barriers; after that, plane s
// has one full barrier, that of the centre tile of plane s + r, on which the
// neighbour tiles of plane s complete too.  Returns false if a wait gave up
// (after waiting, bounded, for the copies already in flight).  The stream
// and row axes are non-periodic (the planner takes no other grid).  (One
// copy per lane of the producer warp measured no faster.)
template <int ND, int O>
__device__ bool bulk_produce(const GridDesc &g, const BulkGeom &bk, const BulkSmem &sm, const float *src, int pencil,
                             const int *idx, int band_lo, int band_rows, int s_begin, int s_end,
                             const float *const *aux, int naux_mask)
{
    constexpr int NOUT = ND - 3, NX = 2 * O * NOUT;
    constexpr int sa = ND - 3;
    const int npad = g.n_pad, nr = g.nr, ns = g.n[sa];
    const int plane = g.stride[sa];
    const int ctile = (bk.rb + 2 * O) * npad, xtile = bk.rb * npad;
    const int nplanes = s_end - s_begin;
    const uint32_t row_bytes = uint32_t(npad) * 4u;
    // centre tile rows t = 0 .. band_rows + 2O - 1 hold grid rows band_lo - O + t;
    // rows outside [0, nr) are ghosts, formed by the compute threads
    const int top = band_lo - O;
    const int r_lo = max(top, 0), r_hi = min(top + band_rows + 2 * O, nr);
    const uint32_t c_bytes = uint32_t(r_hi - r_lo) * row_bytes;
    const int c_off = (r_lo - top) * npad;
    BulkNb nbq[NOUT > 0 ? NOUT : 1][2 * O];
    uint32_t x_bytes = 0;
#pragma unroll
    for (int d = 0; d < NOUT; ++d) {
        bulk_neighbours<O>(g, d, idx[d], nbq[d]);
#pragma unroll
        for (int k = 0; k < 2 * O; ++k)
            if (nbq[d][k].staged) x_bytes += uint32_t(band_rows) * row_bytes;
    }
    // read-once tiles (aux[a] staged when bit a of naux_mask is set)
    int naux = 0;
#pragma unroll
    for (int a = 0; a < BULK_AUX; ++a) naux += (naux_mask >> a) & 1;
    x_bytes += uint32_t(naux) * uint32_t(band_rows) * row_bytes;
    const bool xring = NX > 0 || naux > 0;
    const int xstride = (NX + naux) * xtile;   // floats per neighbour slot
    // slots advance one tile at a time and count their wraps (no division in
    // the loop); the u-th use of a slot (u = wraps so far) first waits for
    // the release of its previous tile, phase u - 1 of the slot's empty
    // barrier.  Source and destination pointers advance one tile at a time.
    int ic = 0, ix = 0;
    int cslot = 0, xslot = 0;
    uint32_t cwrap = 0, xwrap = 0;
    bool ok = true;
    const float *csrc = src + pencil + (s_begin - O) * plane + r_lo * npad;
    const float *xsrc = src + pencil + s_begin * plane + band_lo * npad;
    float *cdst = sm.ring_c + c_off;
    float *xdst = sm.ring_x;
    const uint32_t xrow_bytes = uint32_t(band_rows) * row_bytes;
    for (; ic < nplanes + 2 * O; ++ic) {
        if (cwrap > 0 && !mbar_wait(&sm.empty_c[cslot], (cwrap - 1) & 1u)) {
            ok = false;
            break;
        }
        const bool with_x = xring && ic >= 2 * O;
        if (with_x && xwrap > 0 && !mbar_wait(&sm.empty_x[xslot], (xwrap - 1) & 1u)) {
            ok = false;
            break;
        }
        const int q = s_begin - O + ic;                 // plane of the centre tile
        const bool have = q >= 0 && q < ns;
        mbar_arrive_expect_tx(&sm.full_c[cslot], (have ? c_bytes : 0u) + (with_x ? x_bytes : 0u));
        if (have) bulk_g2s(cdst, csrc, c_bytes, &sm.full_c[cslot]);
        if (with_x) {
#pragma unroll
            for (int d = 0; d < NOUT; ++d)
#pragma unroll
                for (int k = 0; k < 2 * O; ++k)
                    if (nbq[d][k].staged)
                        bulk_g2s(xdst + (d * 2 * O + k) * xtile, xsrc + nbq[d][k].delta, xrow_bytes, &sm.full_c[cslot]);
            // the read-once tiles follow the neighbour tiles in the order
            // l, phi^n, obstacle, each present only when staged
            const int aoff = (s_begin + ix) * plane + pencil + band_lo * npad;
            int apos = NX;
#pragma unroll
            for (int a = 0; a < BULK_AUX; ++a)
                if ((naux_mask >> a) & 1)
                    bulk_g2s(xdst + (apos++) * xtile, aux[a] + aoff, xrow_bytes, &sm.full_c[cslot]);
            ++ix;
            xsrc += plane;
            xdst += xstride;
            if (++xslot == bk.rx) {
                xslot = 0;
                xdst = sm.ring_x;
                ++xwrap;
            }
        }
        csrc += plane;
        cdst += ctile;
        if (++cslot == bk.rc) {
            cslot = 0;
            cdst = sm.ring_c + c_off;
            ++cwrap;
        }
    }
    if (ok) return true;
    // drain: wait (bounded) for the last issued use of every centre slot (the
    // neighbour copies complete on the same barriers)
    for (int slot = 0; slot < bk.rc && slot < ic; ++slot) {
        const int last = slot + ((ic - 1 - slot) / bk.rc) * bk.rc;
        mbar_wait(&sm.full_c[slot], uint32_t(last / bk.rc) & 1u);
    }
    return false;
}

// The value of a centre tile at the thread's segment, or the stream-axis
// ghost formed from the window (plane q outside a non-periodic stream axis).
__device__ __forceinline__ float4 ghost4v(const float4 &pb, const float4 &pi, float k)
{
    return make_float4(keep_sign_ghost(pb.x, pi.x, k), keep_sign_ghost(pb.y, pi.y, k),
                       keep_sign_ghost(pb.z, pi.z, k), keep_sign_ghost(pb.w, pi.w, k));
}

// The bulk-staged stage pass.  ND >= 3, last axis a multiple of 4 nodes,
// alpha static or given per stage (the grid-wide dissipation of Section 2.1).
// STAGE and GOB as in k_stage_plane.
#ifndef ODP_BULK_REGS
#define ODP_BULK_REGS 96
#endif
#ifndef ODP_BULK_REGS6
#define ODP_BULK_REGS6 96
#endif
// Register cap of the bulk-staged pass.  The DubinsCar4D ENO2 pass runs
// bands of 128 compute threads (four compute warps and the producer warp):
// 96 registers (and a 40-byte spill a thread) let four CTAs share an SM,
// measured faster than 104 or 112 (three CTAs) and than bands of 256
// threads at 112.  Rel6D runs three CTAs
// of six warps at 96.  The others keep the plane pass's budget.
template <int ND, int ORDER, int DYN>
constexpr int bulk_max_regs()
{
    return (DYN == DYN_DUBINSCAR4D && ORDER == 2) ? ODP_BULK_REGS
         : (DYN == DYN_REL6D) ? ODP_BULK_REGS6
                              : plane_max_regs<ND, ORDER, DYN>();
}

template <int ND, int ORDER, int DYN, int STAGE, int GOB>
__global__ void __launch_bounds__(512) __maxnreg__((bulk_max_regs<ND, ORDER, DYN>()))
    k_stage_bulk(GridDesc g, DynDesc dy, SolveState *st, const float *__restrict__ l,
                 const float *__restrict__ gob, int stage_rt, int brt)
{
    constexpr int O = ORDER;
    constexpr int NOUT = ND - 3;
    constexpr int NX = 2 * O * NOUT;
    constexpr int sa = ND - 3;
    const int stage = STAGE >= 0 ? STAGE : stage_rt;
    const BulkGeom &bk = g.bk;
    extern __shared__ __align__(128) unsigned char bulk_raw[];
    const int npad = g.n_pad, nr = g.nr, nl = g.n[ND - 1], ns = g.n[sa];
    const int ctile = (bk.rb + 2 * O) * npad, xtile = bk.rb * npad;
    const BulkSmem sm = bulk_smem(bulk_raw, bk, ctile);
    const int cwarps = bk.cwarps;

    const float *__restrict__ src = (stage == 2) ? st->nxt : st->cur;
    float *dst = (stage == 2) ? st->cur : st->nxt;
    const float *prev = st->cur;
    const bool use_l = brt && stage != 1;
    const bool use_g = (GOB >= 0 ? GOB == 1 : gob != nullptr) && stage != 1;
    // read-once tiles the producer stages beside the neighbour tiles: l for
    // the BRT min, phi^n for the Heun average, the obstacle
    const int aux_mask = (use_l ? 1 : 0) | (stage == 2 ? 2 : 0) | (use_g ? 4 : 0);
    const bool xring = NX > 0 || aux_mask != 0;
    // their positions in a neighbour slot, after the NX neighbour tiles
    const int pos_p = NX + (use_l ? 1 : 0), pos_g = pos_p + (stage == 2 ? 1 : 0);
    const int xslot_floats = (pos_g + (use_g ? 1 : 0)) * bk.rb * npad;

    // work item: chunk fastest, then band, then outer pencil.  Outer pencils
    // are numbered block by block (the plane pass's blocks of up to 8
    // indices per outer axis), so CTAs that run together stage each other's
    // pencils as neighbour tiles while they are still in L2.
    const uint32_t item = blockIdx.x;
    const uint32_t q1 = fast_div(item, bk.div_nchunks[O - 1]);
    const int chunk = int(item - q1 * uint32_t(bk.nchunks[O - 1]));
    const uint32_t outer = fast_div(q1, bk.div_nbands);
    const int band = int(q1 - outer * uint32_t(bk.nbands));
    int idx[ND];
    int pencil = 0;
    if (NOUT > 0) {
        const PlaneGeom &pg = g.pg;
        const uint32_t blk0 = fast_div(outer, pg.div_bvol);
        uint32_t wi = outer - blk0 * uint32_t(pg.bvol), blk = blk0;
#pragma unroll
        for (int d = NOUT - 1; d >= 0; --d) {
            const uint32_t wq = fast_div(wi, pg.div_bdim[d]), bq = fast_div(blk, pg.div_nblk[d]);
            idx[d] = int(blk - bq * uint32_t(pg.nblk[d])) * pg.bdim[d] + int(wi - wq * uint32_t(pg.bdim[d]));
            wi = wq;
            blk = bq;
            pencil += idx[d] * g.stride[d];
        }
    }
    const int s_begin = chunk * bk.chunk[O - 1];
    const int s_end = min(ns, s_begin + bk.chunk[O - 1]);
    const int band_lo = band * bk.rb;
    const int band_rows = min(bk.rb, nr - band_lo);

    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int i = 0; i < bk.rc; ++i) {
            mbar_init(&sm.full_c[i], 1);
            mbar_init(&sm.empty_c[i], uint32_t(32 * cwarps));   // every compute thread arrives
        }
        for (int i = 0; i < bk.rx; ++i) {
            mbar_init(&sm.empty_x[i], uint32_t(32 * cwarps));
        }
        mbar_fence_init();
        int ng = 0;
        for (int d = 0; d < NOUT; ++d) {
            BulkNb q[2 * O];
            bulk_neighbours<O>(g, d, idx[d], q);
            for (int k = 0; k < 2 * O; ++k)
                if (!q[k].staged && ng < BULK_GHOST_MAX)
                    sm.ghost[ng++] = BulkGhost{d * 2 * O + k, q[k].gb < 0 ? -1 : d * 2 * O + q[k].gb,
                                               q[k].gi < 0 ? -1 : d * 2 * O + q[k].gi, q[k].k};
        }
        *sm.nghost = ng;
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    if (warp >= cwarps) {
        if (warp == cwarps && lane == 0) {
            const float *aux[BULK_AUX] = {l, prev, gob};
            if (!bulk_produce<ND, O>(g, bk, sm, src, pencil, idx, band_lo, band_rows, s_begin, s_end, aux, aux_mask))
                atomicOr(&st->flags, FLAG_COPY);
        }
        return;
    }

    // this thread's segment: band row j, nodes s0 .. s0 + 3
    const int j = int(fast_div(uint32_t(tid), g.div_segs));
    const int s0 = (tid - j * g.segs) * 4;
    const bool active = j < band_rows;
    const int r = band_lo + (active ? j : 0);
    const int jt = active ? j : 0;
    const int per_l = g.periodic[ND - 1];
    const unsigned *ab = st->alpha_bits[stage == 2 ? 1 : 0];
    float cD[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) cD[d] = 0.5f * bits_to_float(ab[d]) * g.inv_dz[d];
    const float dt = float(st->dt);

    // ghost rows this thread forms (non-periodic row axis)
    const int gtop = r < O ? r + 1 : 0;
    const int gbot = r >= nr - O ? nr - r : 0;
    // only the warps holding one of the grid's first or last r rows form
    // ghost rows (a warp-uniform flag, so the other warps skip the code)
    const bool edge_band = __any_sync(0xffffffffu, active && (gtop != 0 || gbot != 0));
    // last-axis halo columns: wrapped columns of the same tile row, or ghosts
    int lh_off = -2, rh_off = 4;
    bool lghost = false, rghost = false;
    if (per_l) {
        if (s0 == 0) lh_off = nl - 2;
        if (s0 + 4 == nl) rh_off = 4 - nl;
    } else {
        lghost = s0 == 0;
        rghost = s0 + 4 == nl;
    }
    // outer-axis ghost nodes this CTA forms per plane (none inside the grid)
    const int nghost = *sm.nghost;

    // drift coefficients of the segment (the Rel6D x drift is refreshed per plane)
    float cA[ND][4], cS[ND];
    idx[sa] = s_begin;
    idx[ND - 2] = r;
    idx[ND - 1] = s0;
    drift<DYN, ND>(g, dy, idx, cA, cS);
    float4 rx_ve = make_float4(0.f, 0.f, 0.f, 0.f);
    float rx_c = 0.f, rx_wp = 0.f, rx_y = 0.f;
    if (DYN == DYN_REL6D) {
        rx_ve = ldg4(g.coord[ND - 1] + s0);
        rx_c = ldgf(g.cos_tab + idx[2]);
        rx_wp = ldgf(g.coord[4] + idx[4]);
        rx_y = ldgf(g.coord[1] + idx[1]);
    }

    const int so = (O + jt) * npad + s0;   // the segment's offset in a centre tile
    const int xo = jt * npad + s0;         // ... in a neighbour tile
    const int base = pencil + r * npad + s0;
    const int plane = g.stride[sa];
    bool ok = true;

    // ring positions, advanced one tile at a time: the newest centre tile
    // (n), the centre tile whose rows the current plane reads (r), the
    // neighbour tiles (x); slot and phase parity of each
    const int rc = bk.rc, rx = bk.rx;
    int n_slot = 0, r_slot = 0, x_slot = 0;
    uint32_t n_par = 0, r_par = 0;
    auto advance = [&](int &slot, uint32_t &par, int size) {
        if (++slot == size) {
            slot = 0;
            par ^= 1u;
        }
    };
    // a slot is free once every compute thread has arrived (one arrive
    // instruction per warp, no branch); each thread arrives after its own
    // last read of the slot
    auto release = [&](uint64_t *bar) { mbar_arrive(bar); };

    // stream axis: instead of a window of values the thread carries the
    // differences of its segment from plane to plane: ea = w(s) - w(s-1),
    // eb = w(s+1) - w(s) and (ENO2) the second differences da = D2(s-1) =
    // ea - (w(s-1) - w(s-2)), db = D2(s) = eb - ea, the operations of
    // pair_diffs, so the result is that of the window bit for bit.  Each
    // plane reads the values of planes s and s + 1 (and s + 2) from the
    // centre tiles.  The fill reads planes s_begin - O .. s_begin + O - 1.
    auto sub4 = [](const float4 &x, const float4 &y) {
        const float2 lo = f2sub(make_float2(x.x, x.y), make_float2(y.x, y.y));
        const float2 hi = f2sub(make_float2(x.z, x.w), make_float2(y.z, y.w));
        return make_float4(lo.x, lo.y, hi.x, hi.y);
    };
    // ghost k planes outside the boundary plane pb, d = pb - (inner plane)
    auto ghost_d = [](const float4 &pb, const float4 &d, float k) {
        return make_float4(keep_sign_ghost_d(pb.x, d.x, k), keep_sign_ghost_d(pb.y, d.y, k),
                           keep_sign_ghost_d(pb.z, d.z, k), keep_sign_ghost_d(pb.w, d.w, k));
    };
    float4 ea = make_float4(0.f, 0.f, 0.f, 0.f), eb = ea, da = ea, db = ea;
    {
        float4 v[2 * O];
#pragma unroll
        for (int k = 0; k < 2 * O; ++k) {
            if (!mbar_wait(&sm.full_c[n_slot], n_par)) ok = false;
            v[k] = *reinterpret_cast<const float4 *>(sm.ring_c + n_slot * ctile + so);
            advance(n_slot, n_par, rc);
        }
        if (!ok) {
            atomicOr(&st->flags, FLAG_COPY);
            return;
        }
        if (O == 2) {
            if (s_begin == 0) {   // planes -1, -2: ghosts of planes 0 and 1
                v[1] = ghost4v(v[2], v[3 % (2 * O)], 1.0f);
                v[0] = ghost4v(v[2], v[3 % (2 * O)], 2.0f);
            }
            const float4 em2 = sub4(v[1], v[0]);
            ea = sub4(v[2 % (2 * O)], v[1]);
            eb = sub4(v[3 % (2 * O)], v[2 % (2 * O)]);
            da = sub4(ea, em2);
            db = sub4(eb, ea);
        } else {
            ea = sub4(v[1], v[0]);   // plane -1 (s_begin == 0) is set by the first step
        }
    }
    // tiles 0 .. O - 1 are only read here; the rows of plane s_begin are tile O
#pragma unroll
    for (int k = 0; k < O; ++k) {
        release(&sm.empty_c[r_slot]);
        advance(r_slot, r_par, rc);
    }

    float2 fin = make_float2(0.f, 0.f);

    // One plane s.
    // EDGE: the plane may need stream-axis ghost planes ahead (s + O >= ns);
    // planes further in skip those tests
    auto step = [&](int s, auto edge) {
        constexpr bool EDGE = decltype(edge)::value;
        // the centre tile of plane s + O (with the neighbour tiles of plane s)
        if (!mbar_wait(&sm.full_c[n_slot], n_par)) ok = false;
        const float *Tn = sm.ring_c + n_slot * ctile + so;
        advance(n_slot, n_par, rc);
        // the neighbour tiles of plane s completed on the same barrier
        const float *X = sm.ring_x + x_slot * xslot_floats + xo;
        const float *C = sm.ring_c + r_slot * ctile + so;
        const int gi = base + s * plane;
        float4 lx = make_float4(0.f, 0.f, 0.f, 0.f), px = lx, gx = lx;
        // every thread computes (threads past the band's last row compute a
        // copy of its first row), only the valid ones store
        {
#ifndef ODP_BULK_STREAMING
#define ODP_BULK_STREAMING 1
#endif
            // l, phi^n and the obstacle from the tiles the producer staged
            if (use_l) lx = *reinterpret_cast<const float4 *>(X + NX * xtile);
            if (stage == 2) px = *reinterpret_cast<const float4 *>(X + pos_p * xtile);
            if (use_g) gx = *reinterpret_cast<const float4 *>(X + pos_g * xtile);
            const float4 c4 = *reinterpret_cast<const float4 *>(C);
            // stream-axis differences of plane s (ghost planes past a
            // non-periodic end from the carried differences)
            float4 sa_a, sa_b, sa_l = da, sa_m = db, sa_r = db;
            if (O == 2) {
                const int s1 = r_slot + 1 == rc ? 0 : r_slot + 1;
                float4 w1 = *reinterpret_cast<const float4 *>(sm.ring_c + s1 * ctile + so);
                float4 w2 = *reinterpret_cast<const float4 *>(Tn);
                if (EDGE && s + 1 >= ns) {          // planes ns, ns + 1 from planes ns - 1 (c4), ns - 2
                    w1 = ghost_d(c4, ea, 1.0f);
                    w2 = ghost_d(c4, ea, 2.0f);
                } else if (EDGE && s + 2 >= ns) {   // plane ns from planes ns - 1 (w1), ns - 2 (c4)
                    w2 = ghost_d(w1, eb, 1.0f);
                }
                const float4 en = sub4(w2, w1);
                sa_r = sub4(en, eb);
                sa_a = ea;
                sa_b = eb;
                ea = eb;
                eb = en;
                da = db;
                db = sa_r;
            } else {
                float4 w1 = *reinterpret_cast<const float4 *>(Tn);
                if (EDGE && s + 1 >= ns) w1 = ghost_d(c4, ea, 1.0f);
                sa_b = sub4(w1, c4);
                if (s == 0) ea = sub4(c4, ghost_d(c4, sa_b, 1.0f));   // plane -1
                sa_a = ea;
                ea = sa_b;
            }
            if (DYN == DYN_REL6D && s != s_begin) {   // the x drift depends on v_p (the stream axis)
                rel6d_x_drift(ldgf(g.coord[3] + s), rx_ve, rx_c, rx_wp, rx_y, cA[0]);
#pragma unroll
                for (int k = 0; k < 4; ++k) cA[0][k] *= 0.5f * g.inv_dz[0];
            }
            float2 L01 = make_float2(0.0f, 0.0f), L23 = make_float2(0.0f, 0.0f);
            // CTAs at an outer-axis edge: the thread writes the ghost nodes
            // of its segment into the unstaged neighbour slots (its own
            // positions only, so no other thread is involved)
            if (NX > 0) {
#pragma unroll 1
                for (int e = 0; e < nghost; ++e) {
                    const BulkGhost q = sm.ghost[e];
                    float *Xw = const_cast<float *>(X);
                    const float4 pb = *reinterpret_cast<const float4 *>(q.b < 0 ? C : Xw + q.b * xtile);
                    const float4 pi = *reinterpret_cast<const float4 *>(q.i < 0 ? C : Xw + q.i * xtile);
                    *reinterpret_cast<float4 *>(Xw + q.dst * xtile) = ghost4v(pb, pi, q.k);
                }
            }
            // outer axes from the neighbour tiles
#pragma unroll
            for (int d = 0; d < NOUT; ++d) {
                float4 nb[2 * O];
#pragma unroll
                for (int k = 0; k < 2 * O; ++k)
                    nb[k] = *reinterpret_cast<const float4 *>(X + (d * 2 * O + k) * xtile);
                segment_axis<ORDER>(nb[0], nb[O - 1], c4, nb[O], nb[2 * O - 1], cA[d], cS[d], cD[d], L01, L23,
                                    has_drift<DYN, ND>(d), has_bound<DYN, ND>(d));
            }
            // stream axis from the register window
            segment_axis_d<ORDER>(sa_a, sa_b, sa_l, sa_m, sa_r, cA[sa], cS[sa], cD[sa], L01, L23,
                                  has_drift<DYN, ND>(sa), has_bound<DYN, ND>(sa));
            // row axis from the centre tile; ghost rows from this column
            {
                float4 m1 = *reinterpret_cast<const float4 *>(C - npad);
                float4 p1 = *reinterpret_cast<const float4 *>(C + npad);
                float4 m2 = (O == 2) ? *reinterpret_cast<const float4 *>(C - 2 * npad) : m1;
                float4 p2 = (O == 2) ? *reinterpret_cast<const float4 *>(C + 2 * npad) : p1;
                if (edge_band) {
                    if (gtop == 1) {
                        m1 = ghost4(c4, p1, 1.0f);
                        m2 = (O == 2) ? ghost4(c4, p1, 2.0f) : m1;
                    } else if (gtop == 2) {
                        m2 = ghost4(m1, c4, 1.0f);
                    }
                    if (gbot == 1) {
                        p1 = ghost4(c4, m1, 1.0f);
                        p2 = (O == 2) ? ghost4(c4, m1, 2.0f) : p1;
                    } else if (gbot == 2) {
                        p2 = ghost4(p1, c4, 1.0f);
                    }
                }
                segment_axis<ORDER>(m2, m1, c4, p1, p2, cA[ND - 2], cS[ND - 2], cD[ND - 2], L01, L23,
                                    has_drift<DYN, ND>(ND - 2), has_bound<DYN, ND>(ND - 2));
            }
            // last axis: window v[k] = phi(s0 - 2 + k)
            float L[4] = {L01.x, L01.y, L23.x, L23.y};
            {
                float2 lh = *reinterpret_cast<const float2 *>(C + lh_off);
                float2 rh = *reinterpret_cast<const float2 *>(C + rh_off);
                if (!per_l) {   // ghost columns only on a non-periodic last axis (a grid-wide branch)
                    if (lghost) lh = make_float2(keep_sign_ghost(c4.x, c4.y, 2.0f), keep_sign_ghost(c4.x, c4.y, 1.0f));
                    if (rghost) rh = make_float2(keep_sign_ghost(c4.w, c4.z, 1.0f), keep_sign_ghost(c4.w, c4.z, 2.0f));
                }
                const float v[8] = {lh.x, lh.y, c4.x, c4.y, c4.z, c4.w, rh.x, rh.y};
                axis_last<ORDER>(v, cA[ND - 1], cS[ND - 1], cD[ND - 1], L, has_drift<DYN, ND>(ND - 1),
                                 has_bound<DYN, ND>(ND - 1));
            }
            float2 fin_step = fin;
            const float4 out = update_nodes(dt, stage, use_l, c4, L, px, lx, use_g, gx, 4, fin_step);
            if (active && ok) {
                fin = fin_step;
                if (ODP_BULK_STREAMING)
                    __stcs(reinterpret_cast<float4 *>(dst + gi), out);
                else
                    *reinterpret_cast<float4 *>(dst + gi) = out;
            }
        }
        release(&sm.empty_c[r_slot]);
        advance(r_slot, r_par, rc);
        if (xring) {
            release(&sm.empty_x[x_slot]);
            if (++x_slot == rx) x_slot = 0;
        }
    };
#ifndef ODP_BULK_UNROLL2
#define ODP_BULK_UNROLL2 1
#endif
    // two planes per iteration: the carried differences then need no
    // register moves (a small body still, for the instruction cache); the
    // last O planes of the grid take the tests for ghost planes ahead
    using interior = std::false_type;
    using edge = std::true_type;
    const int s_hi = min(s_end, ns - O);
    int s = s_begin;
    if (ODP_BULK_UNROLL2) {
#pragma unroll 1
        for (; s + 1 < s_hi && ok; s += 2) {
            step(s, interior{});
            step(s + 1, interior{});
        }
    }
#pragma unroll 1
    for (; s < s_end && ok; ++s) step(s, edge{});
    if (!ok) atomicOr(&st->flags, FLAG_COPY);
    if (!(fin.x == 0.0f && fin.y == 0.0f)) atomicOr(&st->flags, FLAG_NONFINITE);
}

}  // namespace odp
