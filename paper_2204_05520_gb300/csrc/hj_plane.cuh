// hj_plane.cuh -- plane-streaming stage pass (K2) for grids of 3 or more
// dimensions.
//
// The last two axes form the plane (rows of axis nd-2, the last axis
// fastest), axis nd-3 is the stream axis and axes 0..nd-4 are outer axes.  A
// CTA owns a band of rows of the plane, at fixed outer indices, for a chunk of
// the stream axis, and walks the chunk plane by plane.  Each thread owns one
// four-node segment of the band:
//   * stream axis: the segment's values on planes s-r .. s+r stay in
//     registers (r the stencil radius); plane s+r+1 is loaded one plane ahead;
//   * row axis and last axis: the current plane of the band goes into a
//     double-buffered shared-memory tile with r halo rows above and below and
//     two halo columns at each row end.  The threads owning the band's edge
//     rows and each row's end segments write the halo values (neighbour band,
//     periodic wrap or sign-keeping ghost, Section 3.1.1), loaded one plane
//     ahead, so one barrier per plane suffices;
//   * outer axes: neighbour values are read from global memory.
// The drift coefficients of a segment depend only on the in-plane and outer
// indices for Dubins3D and DubinsCar4D, so they are computed once per thread.
#pragma once

#include <type_traits>

#include "hj_kernels.cuh"

namespace odp {

// Neighbour of an outer axis, read from global memory: the value delta floats
// away, or the ghost k cells outside the boundary from the values db
// (boundary) and di (inner) away (Section 3.1.1).
struct NbPlane {
    int delta, db, di;
    float k;
    int ghost;
};

__device__ __forceinline__ float4 nb_value(const float *__restrict__ src, int gi, const NbPlane &q)
{
    if (!q.ghost) return ldg4(src + gi + q.delta);
    const float4 pb = ldg4(src + gi + q.db), pi = ldg4(src + gi + q.di);
    return make_float4(keep_sign_ghost(pb.x, pi.x, q.k), keep_sign_ghost(pb.y, pi.y, q.k),
                       keep_sign_ghost(pb.z, pi.z, q.k), keep_sign_ghost(pb.w, pi.w, q.k));
}

// The k-th ghost row outside boundary row pb with inner row pi, lane by lane
// (Section 3.1.1).
__device__ __forceinline__ float4 ghost4(const float4 &pb, const float4 &pi, float k)
{
    return make_float4(keep_sign_ghost(pb.x, pi.x, k), keep_sign_ghost(pb.y, pi.y, k),
                       keep_sign_ghost(pb.z, pi.z, k), keep_sign_ghost(pb.w, pi.w, k));
}

// The plane-streaming stage pass.  ND >= 3.  FULL:
// the last axis is a multiple of 4 nodes (no partial segment).
//
// Halo rows of a band: rows of the neighbouring band (or wrapped rows of a
// periodic row axis) are loaded one plane ahead by the band's edge threads;
// ghost rows outside a non-periodic row axis are formed by the threads that
// use them, from their own column of the tile.  Halo columns (FULL): a
// periodic last axis is read at the wrapped columns of the tile row, ghost
// columns are formed from the segment's own values; otherwise the row's
// first and last segments write them into the tile one plane ahead.
// STAGE >= 0 fixes the RK stage at compile time (-1: the stage_rt argument);
// GOB = 0 / 1 fixes whether an obstacle is applied (-1: gob != nullptr).
// Non-finite values are detected by accumulating x - x over the updated nodes
// (0 for finite x, NaN otherwise) and testing the sum once at the end.
// Register budget per model and order, chosen so that whole CTAs fill the
// register file of each SM sub-partition (16384 registers for its warps):
// the DubinsCar4D ENO2 pass (7-warp CTAs) runs 3 CTAs per SM at 80
// registers, the Rel6D upwind pass (5-warp CTAs) 4 CTAs at 96.  The
// DubinsCar4D pass loads its outer-axis neighbours after the plane barrier
// instead of before it, which keeps it within 80 registers.
template <int ND, int ORDER, int DYN>
constexpr int plane_max_regs()
{
    return (DYN == DYN_DUBINSCAR4D && ORDER == 2) ? 80 : (DYN == DYN_REL6D && ORDER == 1) ? 96 : 128;
}

template <int ND, int ORDER, int DYN>
constexpr bool plane_late_outer_loads()
{
    return DYN == DYN_DUBINSCAR4D && ORDER == 2;
}

// Arguments of one plane-streaming stage pass over one grid.
struct PlaneArgs {
    const float *src;             // phi the derivatives are taken of
    const float *prev;            // phi^n for the Heun average (stage 2)
    const float *l;               // target, for the BRT min
    const float *gob;             // reach-avoid obstacle or nullptr
    float *dst;
    const unsigned *alpha_bits;   // alpha of this stage (float bits)
    float dt;
    int stage, brt;
    int *flags;                   // FLAG_NONFINITE is or-ed in here
};

// One work item (band of plane rows x chunk of the stream axis at fixed
// outer indices) of the plane-streaming pass; the CTA calls it with its
// item number.  The launch geometry (bands, chunks, threads, shared bytes)
// is PlaneGeom, computed on the host.
template <int ND, int ORDER, int DYN, bool FULL, int STAGE, int GOB>
__device__ __forceinline__ void plane_pass(const GridDesc &g, const DynDesc &dy, const PlaneArgs &pa, uint32_t item)
{
    const int stage = STAGE >= 0 ? STAGE : pa.stage;
    const int brt = pa.brt;
    const float *__restrict__ l = pa.l;
    const float *__restrict__ gob = pa.gob;
    // per-node dissipation (Algorithm 1's second loop) runs in the generic
    // instantiation only
    const bool local = STAGE < 0 && dy.local_diss != 0;
    const PlaneGeom &pg = g.pg;
    constexpr int O = ORDER;
    constexpr int Q = 2 * O + 1;        // stream-axis window
    constexpr int NOUT = ND - 3;        // outer axes
    constexpr bool LATE = plane_late_outer_loads<ND, ORDER, DYN>();
    extern __shared__ __align__(16) float smem[];
    const int cp = pg.cp;               // tile row pitch: n_pad + 4
    const int tile = 4 + (pg.rb + 2 * O) * cp;

    const int tid = threadIdx.x;
    const float *__restrict__ src = pa.src;
    float *dst = pa.dst;
    const float *prev = pa.prev;
    const unsigned *ab = pa.alpha_bits;
    float cD[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) cD[d] = 0.5f * bits_to_float(ab[d]) * g.inv_dz[d];
    const float dt = pa.dt;
    const bool use_l = brt && stage != 1;
    const bool use_g = (GOB >= 0 ? GOB == 1 : gob != nullptr) && stage != 1;   // reach-avoid obstacle

    // work item: chunk fastest, then band, then outer pencil.  Outer pencils
    // are numbered block by block (blocks of up to 8 indices per outer axis),
    // so CTAs that run together read each other's neighbour planes from L2.
    const uint32_t q1 = fast_div(item, pg.div_nchunks);
    const int chunk = int(item - q1 * uint32_t(pg.nchunks));
    const uint32_t outer = fast_div(q1, pg.div_nbands);
    const int band = int(q1 - outer * uint32_t(pg.nbands));
    int idx[ND];
    int pencil = 0;   // storage offset of the pencil's plane 0
    if (NOUT > 0) {
        const uint32_t blk0 = fast_div(outer, pg.div_bvol);
        uint32_t w = outer - blk0 * uint32_t(pg.bvol), blk = blk0;
#pragma unroll
        for (int d = NOUT - 1; d >= 0; --d) {
            const uint32_t wq = fast_div(w, pg.div_bdim[d]), bq = fast_div(blk, pg.div_nblk[d]);
            idx[d] = int(blk - bq * uint32_t(pg.nblk[d])) * pg.bdim[d] + int(w - wq * uint32_t(pg.bdim[d]));
            w = wq;
            blk = bq;
            pencil += idx[d] * g.stride[d];
        }
    }
    constexpr int sa = ND - 3;
    const int ns = pg.ns, plane = pg.plane;
    const int s_begin = chunk * pg.chunk;
    const int s_end = min(ns, s_begin + pg.chunk);
    const int nr = g.nr, npad = g.n_pad, nl = g.n[ND - 1];
    const int band_lo = band * pg.rb;
    const int band_rows = min(pg.rb, nr - band_lo);
    const int per_r = g.periodic[ND - 2], per_l = g.periodic[ND - 1], per_s = g.periodic[sa];

    // this thread's segment: row band_lo + j, nodes s0 .. s0+3
    const int j = int(fast_div(uint32_t(tid), g.div_segs));
    const int s0 = (tid - j * g.segs) * 4;
    const bool active = j < band_rows;
    const int r = band_lo + (active ? j : 0);
    const int base = pencil + r * npad + s0;   // offset on stream plane 0
    const int so = 4 + (O + j) * cp + s0;                       // offset in a tile
    const int nvalid = FULL ? 4 : min(4, nl - s0);

    // halo-row duty: a band edge row loads the neighbouring band's row (or the
    // wrapped row) into the tile's halo rows; ghost rows have no loader
    bool hrow_duty = false;
    int hdelta = 0, hso = 0;
    if (active && (j < O || j >= band_rows - O)) {
        const int hrow = (j < O) ? band_lo - O + j : band_lo + band_rows + (j - (band_rows - O));
        int q = hrow;
        if (per_r) q = (q < 0) ? q + nr : (q >= nr ? q - nr : q);
        if (q >= 0 && q < nr) {
            hrow_duty = true;
            hdelta = (q - r) * npad;
            hso = 4 + (O + hrow - band_lo) * cp + s0;
        }
    }
    // ghost rows this thread forms: 1 on the boundary row, 2 on the next one
    // (only bands at a non-periodic grid edge have such rows)
    const int gtop = (!per_r && r < O) ? r + 1 : 0;
    const int gbot = (!per_r && r >= nr - O) ? nr - r : 0;
    const bool edge_band = !per_r && (band_lo < O || band_lo + band_rows > nr - O);
    // halo columns
    int lh_off = -2, rh_off = 4;   // relative to the segment's first node in the tile
    bool lghost = false, rghost = false, lcol = false, rcol = false;
    if (FULL) {
        if (per_l) {
            if (s0 == 0) lh_off = nl - 2;
            if (s0 + 4 == nl) rh_off = 4 - nl;
        } else {
            lghost = s0 == 0;
            rghost = s0 + 4 == nl;
        }
    } else {
        lcol = active && s0 == 0;
        rcol = active && s0 + 4 >= nl;
    }

    // neighbours along the outer axes (same offsets for every plane)
    NbPlane nbq[NOUT > 0 ? NOUT : 1][2 * O];
    bool inner = true;
#pragma unroll
    for (int d = 0; d < NOUT; ++d) {
        int k = 0;
#pragma unroll
        for (int o = -O; o <= O; ++o) {
            if (o == 0) continue;
            NbPlane q{};
            int jd = idx[d] + o;
            const int sd = g.stride[d];
            if (g.periodic[d]) {
                while (jd < 0) jd += g.n[d];
                while (jd >= g.n[d]) jd -= g.n[d];
                q.delta = (jd - idx[d]) * sd;
            } else if (jd >= 0 && jd < g.n[d]) {
                q.delta = (jd - idx[d]) * sd;
            } else {
                const int b = jd < 0 ? 0 : g.n[d] - 1, in = jd < 0 ? 1 : g.n[d] - 2;
                q.ghost = 1;
                q.k = jd < 0 ? float(-jd) : float(jd - (g.n[d] - 1));
                q.db = (b - idx[d]) * sd;
                q.di = (in - idx[d]) * sd;
            }
            // the interior path takes every neighbour at o strides, unwrapped
            if (jd != idx[d] + o || q.ghost) inner = false;
            nbq[d][k++] = q;
        }
    }

    // drift coefficients of the segment; for Rel6D also the factors of its x
    // drift that do not depend on v_p, the stream axis
    float cA[ND][4], cS[ND];
    idx[sa] = s_begin;
    idx[ND - 2] = r;
    idx[ND - 1] = s0;
    drift<DYN, ND>(g, dy, idx, cA, cS);
    // the budget-capped passes keep the two drift rows in shared memory
    // (after the two tiles, 32 bytes per thread) and reload them each plane
    // (only active threads touch them: a batched launch may run more threads
    // than this grid's geometry counts, and its shared bytes are sized by it)
    float4 *cA_sm = reinterpret_cast<float4 *>(smem + 2 * tile) + 2 * tid;
    if (LATE && active) {
        cA_sm[0] = make_float4(cA[0][0], cA[0][1], cA[0][2], cA[0][3]);
        cA_sm[1] = make_float4(cA[1][0], cA[1][1], cA[1][2], cA[1][3]);
    }
    float4 rx_ve = make_float4(0.f, 0.f, 0.f, 0.f);
    float rx_c = 0.f, rx_wp = 0.f, rx_y = 0.f;
    if (DYN == DYN_REL6D) {
        rx_ve = ldg4(g.coord[ND - 1] + s0);
        rx_c = ldgf(g.cos_tab + idx[2]);
        rx_wp = ldgf(g.coord[4] + idx[4]);
        rx_y = ldgf(g.coord[1] + idx[1]);
    }

    // halo values of plane p for this thread's duties (loaded one plane ahead)
    float4 hx = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 hl = make_float2(0.f, 0.f), hr = make_float2(0.f, 0.f);
    auto load_halos = [&](int p) {
        const int pb = base + p * plane;
        if (hrow_duty) hx = ldg4(src + pb + hdelta);
        if (!FULL) {
            const float *rowg = src + pb - s0;
            if (lcol) hl = make_float2(last_axis_value(rowg, -2, nl, per_l), last_axis_value(rowg, -1, nl, per_l));
            if (rcol)
                hr = make_float2(last_axis_value(rowg, nl, nl, per_l), last_axis_value(rowg, nl + 1, nl, per_l));
        }
    };

    // stream-axis window: w[(m + i) % Q] holds plane s - O + i at step m = s - s_begin
    float4 w[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) w[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (active) {
#pragma unroll
        for (int k = 0; k < Q; ++k) w[k] = stream_value(src, base, s_begin - O + k, ns, per_s, plane);
        load_halos(s_begin);
    }

    float2 fin = make_float2(0.f, 0.f);   // sum of x - x over the updated nodes
    // One plane: the window slot (u + i) % Q holds plane s - O + i; returns the
    // segment's value on plane s + O + 1.
    auto step = [&](int s, int u, auto inner_tag) -> float4 {
        constexpr bool INNER = decltype(inner_tag)::value;
            float *T = smem + (((s - s_begin) & 1) ? tile : 0);
            const int gi = base + s * plane;
            const float4 c4 = w[(u + O) % Q];
            float4 nb[NOUT > 0 ? NOUT : 1][2 * O];
            float4 lx = make_float4(0.f, 0.f, 0.f, 0.f), px = lx, nx = lx, gx = lx;
            if (active) {
                *reinterpret_cast<float4 *>(T + so) = c4;
                if (hrow_duty) *reinterpret_cast<float4 *>(T + hso) = hx;
                if (!FULL) {
                    if (lcol) {
                        T[so - 2] = hl.x;
                        T[so - 1] = hl.y;
                    }
                    if (rcol) {
                        T[so - s0 + nl] = hr.x;
                        T[so - s0 + nl + 1] = hr.y;
                    }
                }
                // loads for this plane's update and for the next plane
                if (!LATE) {
#pragma unroll
                    for (int d = 0; d < NOUT; ++d)
#pragma unroll
                        for (int k = 0; k < 2 * O; ++k)
                            nb[d][k] = INNER ? ldg4(src + gi + (k < O ? k - O : k - O + 1) * g.stride[d])
                                             : nb_value(src, gi, nbq[d][k]);
                }
                if (use_l) lx = ldg4(l + gi);
                if (use_g) gx = ldg4(gob + gi);
                if (stage == 2) px = *reinterpret_cast<const float4 *>(prev + gi);
                if (s + 1 < s_end) {
                    nx = stream_value(src, base, s + 1 + O, ns, per_s, plane);
                    load_halos(s + 1);
                }
            }
            __syncthreads();

            if (active) {
                if (DYN == DYN_REL6D && s != s_begin) {   // the x drift depends on v_p (the stream axis)
                    rel6d_x_drift(ldgf(g.coord[3] + s), rx_ve, rx_c, rx_wp, rx_y, cA[0]);
#pragma unroll
                    for (int k = 0; k < 4; ++k) cA[0][k] *= 0.5f * g.inv_dz[0];
                }
                if (LATE) {
#pragma unroll
                    for (int d = 0; d < NOUT; ++d)
#pragma unroll
                        for (int k = 0; k < 2 * O; ++k)
                            nb[d][k] = INNER ? ldg4(src + gi + (k < O ? k - O : k - O + 1) * g.stride[d])
                                             : nb_value(src, gi, nbq[d][k]);
                }
                const float *C = T + so;
                float2 L01 = make_float2(0.0f, 0.0f), L23 = make_float2(0.0f, 0.0f);
                // outer axes
                if (LATE) {
                    const float4 a0 = cA_sm[0], a1 = cA_sm[1];
                    cA[0][0] = a0.x;
                    cA[0][1] = a0.y;
                    cA[0][2] = a0.z;
                    cA[0][3] = a0.w;
                    cA[1][0] = a1.x;
                    cA[1][1] = a1.y;
                    cA[1][2] = a1.z;
                    cA[1][3] = a1.w;
                }
#pragma unroll
                for (int d = 0; d < NOUT; ++d) {
                    if (DYN == DYN_REL6D && d == 2 && local)
                        segment_axis_rel6d_theta<ORDER>(nb[d][0], nb[d][O - 1], c4, nb[d][O], nb[d][2 * O - 1],
                                                        cA[d], cS[d], dy, rx_wp, 0.5f * g.inv_dz[2], L01, L23);
                    else
                        segment_axis<ORDER>(nb[d][0], nb[d][O - 1], c4, nb[d][O], nb[d][2 * O - 1], cA[d], cS[d],
                                            cD[d], L01, L23, has_drift<DYN, ND>(d), has_bound<DYN, ND>(d),
                                            local && has_drift<DYN, ND>(d) && !has_bound<DYN, ND>(d));
                }
                // stream axis from the register window
                float2 Pc[2][2];   // capture model: unscaled sums of axes x (stream), y (row)
                // capture model with per-node dissipation: each node's own
                // coefficients, written by the stage's alpha pass
                float4 cdn4[3] = {};
                const bool cap_local = DYN == DYN_CAPTURE && local && g.cdn != nullptr;
                if (cap_local) {
#pragma unroll
                    for (int d = 0; d < 3; ++d) cdn4[d] = ldg4(g.cdn + d * g.cdn_stride + gi);
                }
                if (DYN == DYN_CAPTURE)
                    segment_axis_P<ORDER>(w[u % Q], w[(u + O - 1) % Q], c4, w[(u + O + 1) % Q], w[(u + Q - 1) % Q],
                                          cA[sa], cS[sa], cD[sa], L01, L23, has_drift<DYN, ND>(sa),
                                          has_bound<DYN, ND>(sa), Pc[0][0], Pc[0][1], cap_local ? &cdn4[0] : nullptr);
                else
                    segment_axis<ORDER>(w[u % Q], w[(u + O - 1) % Q], c4, w[(u + O + 1) % Q], w[(u + Q - 1) % Q],
                                        cA[sa], cS[sa], cD[sa], L01, L23, has_drift<DYN, ND>(sa),
                                        has_bound<DYN, ND>(sa),
                                        local && has_drift<DYN, ND>(sa) && !has_bound<DYN, ND>(sa));
                // row axis from the tile; ghost rows from this column
                {
                    float4 m1 = *reinterpret_cast<const float4 *>(C - cp);
                    float4 p1 = *reinterpret_cast<const float4 *>(C + cp);
                    float4 m2 = (O == 2) ? *reinterpret_cast<const float4 *>(C - 2 * cp) : m1;
                    float4 p2 = (O == 2) ? *reinterpret_cast<const float4 *>(C + 2 * cp) : p1;
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
                    if (DYN == DYN_CAPTURE)
                        segment_axis_P<ORDER>(m2, m1, c4, p1, p2, cA[ND - 2], cS[ND - 2], cD[ND - 2], L01, L23,
                                              has_drift<DYN, ND>(ND - 2), has_bound<DYN, ND>(ND - 2), Pc[1][0],
                                              Pc[1][1], cap_local ? &cdn4[1] : nullptr);
                    else
                        segment_axis<ORDER>(m2, m1, c4, p1, p2, cA[ND - 2], cS[ND - 2], cD[ND - 2], L01, L23,
                                            has_drift<DYN, ND>(ND - 2), has_bound<DYN, ND>(ND - 2),
                                            local && has_drift<DYN, ND>(ND - 2) && !has_bound<DYN, ND>(ND - 2));
                }
                // last axis: window v[k] = phi(s0 - 2 + k)
                float L[4] = {L01.x, L01.y, L23.x, L23.y};
                {
                    float2 lh = *reinterpret_cast<const float2 *>(C + lh_off);
                    float2 rh = *reinterpret_cast<const float2 *>(C + rh_off);
                    if (FULL) {
                        if (lghost)
                            lh = make_float2(keep_sign_ghost(c4.x, c4.y, 2.0f), keep_sign_ghost(c4.x, c4.y, 1.0f));
                        if (rghost)
                            rh = make_float2(keep_sign_ghost(c4.w, c4.z, 1.0f), keep_sign_ghost(c4.w, c4.z, 2.0f));
                    }
                    float v[8] = {lh.x, lh.y, c4.x, c4.y, c4.z, c4.w, rh.x, rh.y};
                    if (!FULL && s0 + 4 > nl) {   // partial last segment: the halo columns follow node nl-1
#pragma unroll
                        for (int k = 2; k < 8; ++k)
                            if (s0 + k - 2 >= nl) v[k] = C[k - 2];
                    }
                    float Pth[4];
                    const float cdl[4] = {cdn4[2].x, cdn4[2].y, cdn4[2].z, cdn4[2].w};
                    axis_last<ORDER>(v, cA[ND - 1], cS[ND - 1], cD[ND - 1], L, has_drift<DYN, ND>(ND - 1),
                                     has_bound<DYN, ND>(ND - 1), DYN == DYN_CAPTURE ? Pth : nullptr,
                                     cap_local ? cdl : nullptr);
                    if (DYN == DYN_CAPTURE) {
                        const float Px[4] = {Pc[0][0].x, Pc[0][0].y, Pc[0][1].x, Pc[0][1].y};
                        const float Py[4] = {Pc[1][0].x, Pc[1][0].y, Pc[1][1].x, Pc[1][1].y};
                        capture_term(g, dy, ldgf(g.coord[0] + s), ldgf(g.coord[1] + r), Px, Py, Pth, L);
                    }
                }
                float4 out = update_nodes(dt, stage, use_l, c4, L, px, lx, use_g, gx, nvalid, fin);
                if (FULL || nvalid == 4) {
                    *reinterpret_cast<float4 *>(dst + gi) = out;
                } else {
                    const float o4[4] = {out.x, out.y, out.z, out.w};
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (k < nvalid) dst[gi + k] = o4[k];
                }
            }
        return nx;
    };
    // CTAs whose outer neighbours all lie at plain stride offsets inside the
    // grid (most of them) run the
    // loop unrolled by the window length, so the window is never shifted; the
    // others shift it (smaller code: the two paths share the instruction cache)
    auto run = [&](auto inner_tag) {
        constexpr bool UNROLL = decltype(inner_tag)::value;
        if (UNROLL) {
            for (int s0p = s_begin; s0p < s_end; s0p += Q) {
#pragma unroll
                for (int u = 0; u < Q; ++u) {
                    const int s = s0p + u;
                    if (s >= s_end) break;
                    w[u % Q] = step(s, u, inner_tag);
                }
            }
        } else {
            for (int s = s_begin; s < s_end; ++s) {
                const float4 nx = step(s, 0, inner_tag);
#pragma unroll
                for (int k = 0; k < Q - 1; ++k) w[k] = w[k + 1];
                w[Q - 1] = nx;
            }
        }
    };
    if (inner)
        run(std::true_type{});
    else
        run(std::false_type{});
    if (!(fin.x == 0.0f && fin.y == 0.0f)) atomicOr(pa.flags, FLAG_NONFINITE);
}

// The stage pass of a single solve: buffers, dt and alpha from its state.
template <int ND, int ORDER, int DYN, bool FULL, int STAGE, int GOB>
__global__ void __launch_bounds__(512) __maxnreg__((plane_max_regs<ND, ORDER, DYN>()))
    k_stage_plane(GridDesc g, DynDesc dy, SolveState *st, const float *__restrict__ l, const float *__restrict__ gob,
                  int stage_rt, int brt)
{
    const int stage = STAGE >= 0 ? STAGE : stage_rt;
    PlaneArgs pa;
    pa.src = (stage == 2) ? st->nxt : st->cur;
    pa.dst = (stage == 2) ? st->cur : st->nxt;
    pa.prev = st->cur;
    pa.l = l;
    pa.gob = gob;
    pa.alpha_bits = st->alpha_bits[stage == 2 ? 1 : 0];
    pa.dt = float(st->dt);
    pa.stage = stage;
    pa.brt = brt;
    pa.flags = &st->flags;
    plane_pass<ND, ORDER, DYN, FULL, STAGE, GOB>(g, dy, pa, blockIdx.x);
}

}  // namespace odp
