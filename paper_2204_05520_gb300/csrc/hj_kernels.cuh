// hj_kernels.cuh -- kernels of one solve: the fused stage pass (K2), the
// alpha reductions (K1) and their launch helpers.  Instantiated per model in
// kern_<model>.cu so that the translation units compile in parallel.
//
// Thread layout of the stage pass: one thread owns four consecutive nodes of
// a row (the last axis), loads them and each neighbour row with one 16-byte
// access, and keeps everything in registers.  The Hamiltonian of every model
// here is a sum of per-axis terms, H = sum_d (a_d(z) pbar_d + S_d |pbar_d|)
// (drift coefficient a_d, and S_d = +-bound of the input acting on axis d,
// Algorithm 1 with the bang-bang inputs folded in), and so is the
// Lax-Friedrichs dissipation; the update L = H + 1/2 sum_d alpha_d (p+_d - p-_d)
// is therefore accumulated axis by axis without keeping every derivative.
#pragma once

#include "hj_device.cuh"
#include "odp_launch.h"

namespace odp {

ODP_HD float lane(const float4 &v, int k)
{
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// Neighbour row of a four-node segment along a non-last axis: periodic wrap or
// sign-keeping ghost extrapolation (Section 3.1.1), lane by lane.
ODP_HD float4 row_shift4(const float *__restrict__ src, int base, int id, int stride, int n, int periodic, int off)
{
    int j = id + off;
    if (periodic) {
        while (j < 0) j += n;
        while (j >= n) j -= n;
        return ldg4(src + base + (j - id) * stride);
    }
    if (j >= 0 && j < n) return ldg4(src + base + off * stride);
    const int b = (j < 0) ? 0 : n - 1;
    const int in = (j < 0) ? 1 : n - 2;
    const float k = (j < 0) ? float(-j) : float(j - (n - 1));
    const float4 pb = ldg4(src + base + (b - id) * stride);
    const float4 pi = ldg4(src + base + (in - id) * stride);
    float4 r;
    r.x = keep_sign_ghost(pb.x, pi.x, k);
    r.y = keep_sign_ghost(pb.y, pi.y, k);
    r.z = keep_sign_ghost(pb.z, pi.z, k);
    r.w = keep_sign_ghost(pb.w, pi.w, k);
    return r;
}

// Node j (possibly outside [0, n)) of the last axis of a row.
ODP_HD float last_axis_value(const float *__restrict__ row, int j, int n, int periodic)
{
    if (j >= 0 && j < n) return ldgf(row + j);
    if (periodic) {
        while (j < 0) j += n;
        while (j >= n) j -= n;
        return ldgf(row + j);
    }
    const int b = (j < 0) ? 0 : n - 1;
    const int in = (j < 0) ? 1 : n - 2;
    const float k = (j < 0) ? float(-j) : float(j - (n - 1));
    return keep_sign_ghost(ldgf(row + b), ldgf(row + in), k);
}

// Rel6D x drift of the four nodes of a segment, -v_p + v_e cos th + w_p y
// (unscaled; reading R12 of the model).
ODP_HD void rel6d_x_drift(float vp, const float4 &ve, float c, float wp, float y, float *a)
{
    // explicit roundings: the same value in every kernel that inlines this
#ifdef __CUDA_ARCH__
    const float t = __fmul_rn(wp, y);
    for (int k = 0; k < 4; ++k) a[k] = __fadd_rn(__fadd_rn(-vp, __fmul_rn(lane(ve, k), c)), t);
#else
    for (int k = 0; k < 4; ++k) a[k] = -vp + lane(ve, k) * c + wp * y;
#endif
}

// Half-scaled drift coefficients of the four nodes of a segment,
// cA_d = a_d(z) / (2 h_d), and of the signed input bounds, cS_d = S_d / (2 h_d)
// (Appendix dynamics; Section 4.2 modes).  idx holds the node's axis indices
// (idx[ndim-1] the first node of the segment).
template <int DYN, int ND>
ODP_HD void drift(const GridDesc &g, const DynDesc &dy, const int *idx, float cA[ND][4], float cS[ND])
{
    const float su = mode_sign(dy.umode), sd = mode_sign(dy.dmode);
    for (int d = 0; d < ND; ++d) {
        cS[d] = 0.0f;
        for (int k = 0; k < 4; ++k) cA[d][k] = 0.0f;
    }
    const int s0 = idx[ND - 1];
    if (DYN == DYN_SINGLE_INT) {
        for (int d = 0; d < ND; ++d) cS[d] = su * dy.prm[0];
    } else if (DYN == DYN_ADVECTION) {
        for (int d = 0; d < ND; ++d)
            for (int k = 0; k < 4; ++k) cA[d][k] = dy.prm[d];
    } else if (DYN == DYN_DUBINS3D) {          // (x, y, th), th last
        const float4 c = ldg4(g.cos_tab + s0), s = ldg4(g.sin_tab + s0);
        const float v = dy.prm[0];
        for (int k = 0; k < 4; ++k) {
            cA[0][k] = v * lane(c, k);
            cA[1][k] = v * lane(s, k);
        }
        cS[2] = su * dy.prm[1];
    } else if (DYN == DYN_CAPTURE) {           // (x, y, th), th last (Section 4.2)
        const float4 c = ldg4(g.cos_tab + s0), s = ldg4(g.sin_tab + s0);
        const float v = dy.prm[0];
        for (int k = 0; k < 4; ++k) {
            cA[0][k] = -v + v * lane(c, k);
            cA[1][k] = v * lane(s, k);
        }
        cS[2] = sd * dy.prm[2];                // pursuer turn b: S_b |pbar_th|
    } else if (DYN == DYN_DUBINSCAR4D) {       // (x, y, v, th), th last
        const float4 c = ldg4(g.cos_tab + s0), s = ldg4(g.sin_tab + s0);
        const float v = ldgf(g.coord[2] + idx[2]);
        for (int k = 0; k < 4; ++k) {
            cA[0][k] = v * lane(c, k);
            cA[1][k] = v * lane(s, k);
        }
        cS[2] = su * dy.prm[0];
        cS[3] = su * dy.prm[1];
    } else {                                   // Rel6D (x, y, th, v_p, w_p, v_e), v_e last
        const float x = ldgf(g.coord[0] + idx[0]);
        const float y = ldgf(g.coord[1] + idx[1]);
        const float c = ldgf(g.cos_tab + idx[2]);
        const float s = ldgf(g.sin_tab + idx[2]);
        const float vp = ldgf(g.coord[3] + idx[3]);
        const float wp = ldgf(g.coord[4] + idx[4]);
        const float4 ve = ldg4(g.coord[5] + s0);
        rel6d_x_drift(vp, ve, c, wp, y, cA[0]);
        for (int k = 0; k < 4; ++k) {
            cA[1][k] = lane(ve, k) * s - wp * x;
            cA[2][k] = -wp;
        }
        cS[2] = sd * dy.prm[3];
        cS[3] = su * dy.prm[0];
        cS[4] = su * dy.prm[1];
        cS[5] = sd * dy.prm[2];
    }
    for (int d = 0; d < ND; ++d) {
        const float hh = 0.5f * g.inv_dz[d];
        cS[d] *= hh;
        for (int k = 0; k < 4; ++k) cA[d][k] *= hh;
    }
}

// Contribution of one axis to the Lax-Friedrichs right-hand side at one node
// from its unscaled one-sided differences dm = h p-, dp = h p+:
// a pbar + S |pbar| + 1/2 alpha (p+ - p-) = cA P + cS |P| + cD M with
// P = dp + dm, M = dp - dm, cD = alpha / (2 h) (Algorithm 1).
ODP_HD float axis_term(float dm, float dp, float cA, float cS, float cD)
{
    const float P = dp + dm, M = dp - dm;
    return cA * P + cS * fabsf(P) + cD * M;
}

// Multi-index of a thread's segment (flat thread numbering, used by the
// reductions): idx[0..ND-2] of its row, idx[ND-1] the first node of its
// segment; returns the storage offset of that node.
template <int ND>
ODP_HD int segment_index(const GridDesc &g, uint32_t t, int *idx)
{
    uint32_t row = fast_div(t, g.div_segs);
    const int seg = int(t - row * uint32_t(g.segs));
    const int base = int(row) * g.n_pad + 4 * seg;
    for (int d = ND - 2; d > 0; --d) {
        const uint32_t q = fast_div(row, g.div[d]);
        idx[d] = int(row - q * uint32_t(g.n[d]));
        row = q;
    }
    if (ND >= 2) idx[0] = int(row);
    idx[ND - 1] = 4 * seg;
    return base;
}

// Arguments of one stage pass over one grid.
struct StageArgs {
    const float *src;     // phi the derivatives are taken of
    const float *prev;    // phi^n for the Heun average (stage 2), else unused
    const float *l;       // target, for the BRT min
    const float *gob;     // obstacle g for the reach-avoid max, or nullptr
    float *dst;
    float cD[ODP_MAXD];   // alpha_d / (2 h_d)
    float dt;
    int stage;            // 0 Euler, 1 RK2 stage 1, 2 RK2 stage 2
    int brt;
};

// One non-last axis of a four-node segment that also returns the unscaled
// sums P = dp + dm of its two node pairs (for the capture model's coupled
// term).
template <int ORDER>
ODP_HD void segment_axis_P(const float4 &m2, const float4 &m1, const float4 &c, const float4 &p1, const float4 &p2,
                           const float *cA, float cS, float cD, float2 &L01, float2 &L23, bool has_a, bool has_s,
                           float2 &P01, float2 &P23, const float4 *cDn = nullptr)
{
    // cDn (optional): each node's own dissipation coefficient instead of cD
    float2 dm, dp;
    pair_diffs<ORDER>(make_float2(m2.x, m2.y), make_float2(m1.x, m1.y), make_float2(c.x, c.y),
                      make_float2(p1.x, p1.y), make_float2(p2.x, p2.y), dm, dp);
    pair_terms(dm, dp, make_float2(cA[0], cA[1]), cS, cDn ? make_float2(cDn->x, cDn->y) : f2splat(cD), L01, has_a,
               has_s, &P01);
    pair_diffs<ORDER>(make_float2(m2.z, m2.w), make_float2(m1.z, m1.w), make_float2(c.z, c.w),
                      make_float2(p1.z, p1.w), make_float2(p2.z, p2.w), dm, dp);
    pair_terms(dm, dp, make_float2(cA[2], cA[3]), cS, cDn ? make_float2(cDn->z, cDn->w) : f2splat(cD), L23, has_a,
               has_s, &P23);
}

// The capture model's evader term (Section 4.2): the evader turn a enters
// every axis, x' += a y, y' -= a x, th' -= a, so it contributes
// S_a |s| with s = y pbar_x - x pbar_y - pbar_th, S_a = +-A by its mode;
// pbar_d = P_d / (2 h_d) from the unscaled sums of each axis.
ODP_HD void capture_term(const GridDesc &g, const DynDesc &dy, float x, float y, const float *Px, const float *Py,
                         const float *Pth, float *L)
{
    const float cx = y * (0.5f * g.inv_dz[0]), cy = -x * (0.5f * g.inv_dz[1]), ct = -0.5f * g.inv_dz[2];
    const float Sa = mode_sign(dy.umode) * dy.prm[1];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float s = fmaf(cx, Px[k], fmaf(cy, Py[k], ct * Pth[k]));
        L[k] = fmaf(Sa, fabsf(s), L[k]);
    }
}

// One non-last axis of a four-node segment from its neighbour rows (as two
// pairs of nodes).
template <int ORDER>
ODP_HD void segment_axis(const float4 &m2, const float4 &m1, const float4 &c, const float4 &p1, const float4 &p2,
                         const float *cA, float cS, float cD, float2 &L01, float2 &L23, bool has_a, bool has_s,
                         bool abs_cA = false)
{
    // abs_cA: per-node dissipation of an axis whose rate is the drift alone,
    // alpha_i / (2 h) = |a(z_i)| / (2 h) = |cA| (Algorithm 1's second loop)
    const float2 a01 = make_float2(cA[0], cA[1]), a23 = make_float2(cA[2], cA[3]);
    axis_pair<ORDER>(make_float2(m2.x, m2.y), make_float2(m1.x, m1.y), make_float2(c.x, c.y),
                     make_float2(p1.x, p1.y), make_float2(p2.x, p2.y), a01, cS,
                     abs_cA ? f2abs(a01) : f2splat(cD), L01, has_a, has_s);
    axis_pair<ORDER>(make_float2(m2.z, m2.w), make_float2(m1.z, m1.w), make_float2(c.z, c.w),
                     make_float2(p1.z, p1.w), make_float2(p2.z, p2.w), a23, cS,
                     abs_cA ? f2abs(a23) : f2splat(cD), L23, has_a, has_s);
}

// segment_axis from the axis's differences instead of its five rows: a, b
// the backward and forward differences (f0 - fm1, fp1 - f0) and d2l, d2m,
// d2r the second differences at i-1, i, i+1 (a - (fm1 - fm2), b - a,
// (fp2 - fp1) - b), computed by the caller with the same operations, so the
// result is that of segment_axis bit for bit.
template <int ORDER>
ODP_HD void segment_axis_d(const float4 &a, const float4 &b, const float4 &d2l, const float4 &d2m, const float4 &d2r,
                           const float *cA, float cS, float cD, float2 &L01, float2 &L23, bool has_a, bool has_s)
{
    float2 dm = make_float2(a.x, a.y), dp = make_float2(b.x, b.y);
    if (ORDER == 2) {
        const float2 m = make_float2(d2m.x, d2m.y);
        const float2 cm = f2pick(make_float2(d2l.x, d2l.y), m), cp = f2pick(make_float2(d2r.x, d2r.y), m);
        dm = f2fma(cm, f2splat(0.5f), dm);
        dp = f2fma(cp, f2splat(-0.5f), dp);
    }
    pair_terms(dm, dp, make_float2(cA[0], cA[1]), cS, f2splat(cD), L01, has_a, has_s);
    dm = make_float2(a.z, a.w);
    dp = make_float2(b.z, b.w);
    if (ORDER == 2) {
        const float2 m = make_float2(d2m.z, d2m.w);
        const float2 cm = f2pick(make_float2(d2l.z, d2l.w), m), cp = f2pick(make_float2(d2r.z, d2r.w), m);
        dm = f2fma(cm, f2splat(0.5f), dm);
        dp = f2fma(cp, f2splat(-0.5f), dp);
    }
    pair_terms(dm, dp, make_float2(cA[2], cA[3]), cS, f2splat(cD), L23, has_a, has_s);
}

// The Rel6D heading axis with per-node dissipation: each node's heading-rate
// bound from the interval of its own one-sided differences (the same rule as
// the grid alpha, rel6d_theta_alpha), scaled by 1 / (2 h).
template <int ORDER>
ODP_HD void segment_axis_rel6d_theta(const float4 &m2, const float4 &m1, const float4 &c, const float4 &p1,
                                     const float4 &p2, const float *cA, float cS, const DynDesc &dy, float wp,
                                     float hh, float2 &L01, float2 &L23)
{
    const float2 a01 = make_float2(cA[0], cA[1]), a23 = make_float2(cA[2], cA[3]);
    float2 dm, dp;
    pair_diffs<ORDER>(make_float2(m2.x, m2.y), make_float2(m1.x, m1.y), make_float2(c.x, c.y),
                      make_float2(p1.x, p1.y), make_float2(p2.x, p2.y), dm, dp);
    float2 cD = make_float2(hh * rel6d_theta_alpha(dy, wp, fminf(dm.x, dp.x), fmaxf(dm.x, dp.x)),
                            hh * rel6d_theta_alpha(dy, wp, fminf(dm.y, dp.y), fmaxf(dm.y, dp.y)));
    pair_terms(dm, dp, a01, cS, cD, L01, true, true);
    pair_diffs<ORDER>(make_float2(m2.z, m2.w), make_float2(m1.z, m1.w), make_float2(c.z, c.w),
                      make_float2(p1.z, p1.w), make_float2(p2.z, p2.w), dm, dp);
    cD = make_float2(hh * rel6d_theta_alpha(dy, wp, fminf(dm.x, dp.x), fmaxf(dm.x, dp.x)),
                     hh * rel6d_theta_alpha(dy, wp, fminf(dm.y, dp.y), fmaxf(dm.y, dp.y)));
    pair_terms(dm, dp, a23, cS, cD, L23, true, true);
}

// Update of a four-node segment from its right-hand side L: phi + dt L
// (Euler / RK2 stage), the Heun average with phi^n (b4) on RK2 stage 2, the
// non-finite check of the valid nodes, and the min with l (l4) when use_l
// (the last stage of a step of a tube).  Returns true if a valid node is not
// finite.
ODP_HD bool update_segment(float dt_, int stage, bool use_l, const float4 &c4, const float *L, const float4 &b4,
                           const float4 &l4, bool use_g, const float4 &g4, int nvalid, float4 &out)
{
    const float2 dt = f2splat(dt_);
    float2 v01 = f2fma(dt, make_float2(L[0], L[1]), make_float2(c4.x, c4.y));
    float2 v23 = f2fma(dt, make_float2(L[2], L[3]), make_float2(c4.z, c4.w));
    if (stage == 2) {
        v01 = f2mul(f2splat(0.5f), f2add(make_float2(b4.x, b4.y), v01));
        v23 = f2mul(f2splat(0.5f), f2add(make_float2(b4.z, b4.w), v23));
    }
    const float v[4] = {v01.x, v01.y, v23.x, v23.y};
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (k < nvalid && !isfinite(v[k])) bad = true;
    out = make_float4(v[0], v[1], v[2], v[3]);
    if (use_l) {
        out.x = fminf(out.x, l4.x);
        out.y = fminf(out.y, l4.y);
        out.z = fminf(out.z, l4.z);
        out.w = fminf(out.w, l4.w);
    }
    if (use_g) {
        out.x = fmaxf(out.x, g4.x);
        out.y = fmaxf(out.y, g4.y);
        out.z = fmaxf(out.z, g4.z);
        out.w = fmaxf(out.w, g4.w);
    }
    return bad;
}

// The same update without a per-node finite test: x - x of every valid
// updated node (0 when finite, NaN otherwise) is added to fin instead.
ODP_HD float4 update_nodes(float dt_, int stage, bool use_l, const float4 &c4, const float *L, const float4 &b4,
                           const float4 &l4, bool use_g, const float4 &g4, int nvalid, float2 &fin)
{
    const float2 dt = f2splat(dt_);
    float2 v01 = f2fma(dt, make_float2(L[0], L[1]), make_float2(c4.x, c4.y));
    float2 v23 = f2fma(dt, make_float2(L[2], L[3]), make_float2(c4.z, c4.w));
    if (stage == 2) {
        v01 = f2mul(f2splat(0.5f), f2add(make_float2(b4.x, b4.y), v01));
        v23 = f2mul(f2splat(0.5f), f2add(make_float2(b4.z, b4.w), v23));
    }
    float2 z01 = f2sub(v01, v01), z23 = f2sub(v23, v23);
    if (nvalid < 4) {
        if (nvalid < 4) z23.y = 0.0f;
        if (nvalid < 3) z23.x = 0.0f;
        if (nvalid < 2) z01.y = 0.0f;
    }
    fin = f2add(fin, f2add(z01, z23));
    float4 out = make_float4(v01.x, v01.y, v23.x, v23.y);
    if (use_l) {
        out.x = fminf(out.x, l4.x);
        out.y = fminf(out.y, l4.y);
        out.z = fminf(out.z, l4.z);
        out.w = fminf(out.w, l4.w);
    }
    if (use_g) {
        out.x = fmaxf(out.x, g4.x);
        out.y = fmaxf(out.y, g4.y);
        out.z = fmaxf(out.z, g4.z);
        out.w = fmaxf(out.w, g4.w);
    }
    return out;
}

// update_segment with phi^n, l and the obstacle read at storage offset base.
ODP_HD bool stage_epilogue(const StageArgs &A, int base, const float4 &c4, const float *L, int nvalid, float4 &out)
{
    float4 b4 = make_float4(0.f, 0.f, 0.f, 0.f), l4 = b4, g4 = b4;
    if (A.stage == 2) b4 = *reinterpret_cast<const float4 *>(A.prev + base);
    const bool use_l = A.brt && A.stage != 1;
    if (use_l) l4 = ldg4(A.l + base);
    const bool use_g = A.gob != nullptr && A.stage != 1;
    if (use_g) g4 = ldg4(A.gob + base);
    return update_segment(A.dt, A.stage, use_l, c4, L, b4, l4, use_g, g4, nvalid, out);
}

// Row j (possibly outside [0, n)) of axis `axis` relative to row i0 of the
// segment at storage offset base (periodic wrap or sign-keeping ghost).
ODP_HD float4 axis_row(const float *__restrict__ src, int base, int i0, int j, int stride, int n, int periodic)
{
    if (j >= 0 && j < n) return ldg4(src + base + (j - i0) * stride);
    if (periodic) {
        while (j < 0) j += n;
        while (j >= n) j -= n;
        return ldg4(src + base + (j - i0) * stride);
    }
    const int b = (j < 0) ? 0 : n - 1;
    const int in = (j < 0) ? 1 : n - 2;
    const float k = (j < 0) ? float(-j) : float(j - (n - 1));
    const float4 pb = ldg4(src + base + (b - i0) * stride);
    const float4 pi = ldg4(src + base + (in - i0) * stride);
    float4 r;
    r.x = keep_sign_ghost(pb.x, pi.x, k);
    r.y = keep_sign_ghost(pb.y, pi.y, k);
    r.z = keep_sign_ghost(pb.z, pi.z, k);
    r.w = keep_sign_ghost(pb.w, pi.w, k);
    return r;
}

// One thread of the tiled stage pass (Algorithm 1, one Euler or TVD-RK2
// stage, Section 3.1.3): R rows of axis ndim-2 times one four-node segment of
// the last axis.  Derivatives, pbar, H, Lax-Friedrichs dissipation with the
// grid alpha, update and, on the last stage of a step of a tube, the min with
// l.  Returns true if a non-finite value was produced.
//   stage 0: Euler        phi' = phi + dt L(phi)
//   stage 1: RK2 stage 1  phi1 = phi + dt L(phi)
//   stage 2: RK2 stage 2  phi' = (phi^n + phi1 + dt L(phi1))/2
// t numbers the thread as in GridDesc (segment fastest, then row group,
// then plane).
template <int ND, int ORDER, int DYN, int R>
ODP_HD bool stage_tile(const GridDesc &g, const DynDesc &dy, const StageArgs &A, uint32_t t)
{
    constexpr int O = ORDER;          // stencil radius
    constexpr int NC = R + 2 * O;     // rows of the column along axis ND-2
    const float *__restrict__ src = A.src;
    const uint32_t q = fast_div(t, g.div_segs);
    const int seg = int(t - q * uint32_t(g.segs));
    const uint32_t plane = fast_div(q, g.div_row_groups);
    const int r0 = int(q - plane * uint32_t(g.row_groups)) * R;

    int idx[ND];
    {
        uint32_t pl = plane;
        for (int d = ND - 3; d > 0; --d) {
            const uint32_t q = fast_div(pl, g.div[d]);
            idx[d] = int(pl - q * uint32_t(g.n[d]));
            pl = q;
        }
        if (ND >= 3) idx[0] = int(pl);
    }
    idx[ND - 1] = 4 * seg;
    if (ND >= 2) idx[ND - 2] = r0;
    const int base0 = (int(plane) * g.nr + r0) * g.n_pad + 4 * seg;   // row r0
    const int rstride = g.n_pad;                                       // one row of axis ND-2
    const int nl = g.n[ND - 1];
    const int s0 = idx[ND - 1];
    const int nvalid = nl - s0 < 4 ? nl - s0 : 4;

    // column of rows r0-O .. r0+R-1+O along axis ND-2
    float4 col[NC];
    if (ND >= 2) {
#pragma unroll
        for (int j = 0; j < NC; ++j)
            col[j] = axis_row(src, base0, r0, r0 - O + j, rstride, g.nr, g.periodic[ND - 2]);
    } else {
        col[O] = ldg4(src + base0);
    }

    bool bad = false;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int r = r0 + i;
        if (r >= g.nr) break;
        const int base = base0 + i * rstride;
        if (ND >= 2) idx[ND - 2] = r;
        float cA[ND][4], cS[ND];
        drift<DYN, ND>(g, dy, idx, cA, cS);
        const float4 c4 = col[O + i];
        const float f[4] = {c4.x, c4.y, c4.z, c4.w};
        float2 L01 = make_float2(0.0f, 0.0f), L23 = make_float2(0.0f, 0.0f);

        float2 Pc[2][2];   // capture model: unscaled sums of axes x, y (two node pairs)
        // capture model with per-node dissipation: each node's own
        // coefficients, written by the stage's alpha pass
        float4 cdn4[3] = {};
        const bool cap_local = DYN == DYN_CAPTURE && dy.local_diss && g.cdn != nullptr;
        if (cap_local) {
#pragma unroll
            for (int d = 0; d < 3; ++d) cdn4[d] = ldg4(g.cdn + d * g.cdn_stride + base);
        }
        // outer axes: neighbour rows one by one
#pragma unroll
        for (int d = 0; d < ND - 2; ++d) {
            const int stride = g.stride[d], n = g.n[d], per = g.periodic[d], id = idx[d];
            const float4 m1 = axis_row(src, base, id, id - 1, stride, n, per);
            const float4 p1 = axis_row(src, base, id, id + 1, stride, n, per);
            float4 m2 = m1, p2 = p1;
            if (ORDER == 2) {
                m2 = axis_row(src, base, id, id - 2, stride, n, per);
                p2 = axis_row(src, base, id, id + 2, stride, n, per);
            }
            if (DYN == DYN_CAPTURE)
                segment_axis_P<ORDER>(m2, m1, c4, p1, p2, cA[d], cS[d], A.cD[d], L01, L23, has_drift<DYN, ND>(d),
                                      has_bound<DYN, ND>(d), Pc[0][0], Pc[0][1], cap_local ? &cdn4[d < 3 ? d : 2] : nullptr);
            else if (DYN == DYN_REL6D && d == 2 && dy.local_diss)
                segment_axis_rel6d_theta<ORDER>(m2, m1, c4, p1, p2, cA[d], cS[d], dy, ldgf(g.coord[4] + idx[4]),
                                                0.5f * g.inv_dz[2], L01, L23);
            else
                segment_axis<ORDER>(m2, m1, c4, p1, p2, cA[d], cS[d], A.cD[d], L01, L23, has_drift<DYN, ND>(d),
                                    has_bound<DYN, ND>(d),
                                    dy.local_diss && has_drift<DYN, ND>(d) && !has_bound<DYN, ND>(d));
        }

        // axis ND-2 from the column
        if (ND >= 2) {
            constexpr int d = ND - 2 < 0 ? 0 : ND - 2;
            const float4 m2 = col[i + O - 2 < 0 ? 0 : i + O - 2], m1 = col[i + O - 1];
            const float4 p1 = col[i + O + 1], p2 = col[i + O + 2 < NC ? i + O + 2 : NC - 1];
            if (DYN == DYN_CAPTURE)
                segment_axis_P<ORDER>(m2, m1, c4, p1, p2, cA[d], cS[d], A.cD[d], L01, L23, has_drift<DYN, ND>(d),
                                      has_bound<DYN, ND>(d), Pc[1][0], Pc[1][1], cap_local ? &cdn4[d < 3 ? d : 2] : nullptr);
            else
                segment_axis<ORDER>(m2, m1, c4, p1, p2, cA[d], cS[d], A.cD[d], L01, L23, has_drift<DYN, ND>(d),
                                    has_bound<DYN, ND>(d),
                                    dy.local_diss && has_drift<DYN, ND>(d) && !has_bound<DYN, ND>(d));
        }

        // last axis: an eight-node window w[j] = phi(first node - 2 + j)
        float w[8];
        w[2] = f[0];
        w[3] = f[1];
        w[4] = f[2];
        w[5] = f[3];
        if (s0 >= 2 && s0 + 5 < nl) {
            const float2 lh = ldg2(src + base - 2);
            const float2 rh = ldg2(src + base + 4);
            w[0] = lh.x;
            w[1] = lh.y;
            w[6] = rh.x;
            w[7] = rh.y;
        } else {
            const float *rowp = src + (base - s0);
            const int per = g.periodic[ND - 1];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j < 2 || j >= 6 || s0 + j - 2 >= nl) w[j] = last_axis_value(rowp, s0 + j - 2, nl, per);
        }
        float L[4] = {L01.x, L01.y, L23.x, L23.y};
        float Pth[4];
        constexpr int cl = ND - 1 < 2 ? ND - 1 : 2;
        const float cdl[4] = {cdn4[cl].x, cdn4[cl].y, cdn4[cl].z, cdn4[cl].w};
        axis_last<ORDER>(w, cA[ND - 1], cS[ND - 1], A.cD[ND - 1], L, has_drift<DYN, ND>(ND - 1), has_bound<DYN, ND>(ND - 1),
                         DYN == DYN_CAPTURE ? Pth : nullptr, cap_local ? cdl : nullptr);
        if (DYN == DYN_CAPTURE) {
            const float Px[4] = {Pc[0][0].x, Pc[0][0].y, Pc[0][1].x, Pc[0][1].y};
            const float Py[4] = {Pc[1][0].x, Pc[1][0].y, Pc[1][1].x, Pc[1][1].y};
            capture_term(g, dy, ldgf(g.coord[0] + idx[0]), ldgf(g.coord[1] + idx[1]), Px, Py, Pth, L);
        }

        float4 out;
        const bool bad_here = stage_epilogue(A, base, c4, L, nvalid, out);
        bad = bad || bad_here;
        if (nvalid == 4) {
            *reinterpret_cast<float4 *>(A.dst + base) = out;
        } else {
            const float o[4] = {out.x, out.y, out.z, out.w};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (k < nvalid) A.dst[base + k] = o[k];
        }
    }
    return bad;
}

// Stage pass over a whole grid, reading its buffers, dt and alpha from the
// solve state.
template <int ND, int ORDER, int DYN, int R>
__global__ void __launch_bounds__(256) k_stage(GridDesc g, DynDesc dy, SolveState *st,
                                               const float *__restrict__ l, const float *__restrict__ gob,
                                               int stage, int brt)
{
    StageArgs A;
    A.src = (stage == 2) ? st->nxt : st->cur;
    A.prev = st->cur;
    A.dst = (stage == 2) ? st->cur : st->nxt;
    A.l = l;
    A.gob = gob;
    const unsigned *ab = st->alpha_bits[stage == 2 ? 1 : 0];
#pragma unroll
    for (int d = 0; d < ND; ++d) A.cD[d] = 0.5f * bits_to_float(ab[d]) * g.inv_dz[d];
    A.dt = float(st->dt);
    A.stage = stage;
    A.brt = brt;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= uint32_t(g.nthreads_rb)) return;
    if (stage_tile<ND, ORDER, DYN, R>(g, dy, A, t)) atomicOr(&st->flags, FLAG_NONFINITE);
}

// Grid-wide max of the static alpha components into both stage slots.
template <int ND, int DYN>
__global__ void __launch_bounds__(256) k_alpha_static(GridDesc g, DynDesc dy, SolveState *st)
{
    __shared__ float red[8][ND];
    float a[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) a[d] = 0.0f;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < uint32_t(g.total);
         i += gridDim.x * blockDim.x) {
        int idx[ND];
        unflatten(g, ND, i, idx);
        float la[ND];
        static_alpha<DYN, ND>(g, dy, idx, la);
#pragma unroll
        for (int d = 0; d < ND; ++d) a[d] = fmaxf(a[d], la[d]);
    }
    const int lane_id = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        a[d] = warp_max(a[d]);
        if (lane_id == 0) red[warp][d] = a[d];
    }
    __syncthreads();
    if (threadIdx.x < ND) {
        float m = 0.0f;
        for (int w = 0; w < (blockDim.x >> 5); ++w) m = fmaxf(m, red[w][threadIdx.x]);
        atomicMax(&st->alpha_bits[0][threadIdx.x], __float_as_uint(m));
        atomicMax(&st->alpha_bits[1][threadIdx.x], __float_as_uint(m));
    }
}

// A segment's value on plane p of an axis with n planes stride floats apart
// (periodic wrap or sign-keeping ghost outside [0, n), Section 3.1.1); base
// is the segment's offset on plane 0.
__device__ __forceinline__ float4 stream_value(const float *__restrict__ src, int base, int p, int n, int periodic,
                                               int stride)
{
    if (p >= 0 && p < n) return ldg4(src + base + p * stride);
    if (periodic) {
        while (p < 0) p += n;
        while (p >= n) p -= n;
        return ldg4(src + base + p * stride);
    }
    const int b = p < 0 ? 0 : n - 1, in = p < 0 ? 1 : n - 2;
    const float k = p < 0 ? float(-p) : float(p - (n - 1));
    const float4 pb = ldg4(src + base + b * stride), pi = ldg4(src + base + in * stride);
    return make_float4(keep_sign_ghost(pb.x, pi.x, k), keep_sign_ghost(pb.y, pi.y, k),
                       keep_sign_ghost(pb.z, pi.z, k), keep_sign_ghost(pb.w, pi.w, k));
}

// Rel6D heading-rate alpha of phi (slot 0: cur) or phi1 (slot 1: nxt): the
// largest bound over the nodes of the heading rate given the interval of p_th
// (Section 2.1 global alpha).  A thread owns one four-node segment of an
// (x, y) block and walks the heading axis (axis 2) with the segment's values
// in a register window, so every value is read once.
template <int ORDER>
__global__ void __launch_bounds__(256) k_alpha_rel6d(GridDesc g, DynDesc dy, SolveState *st, int slot)
{
    constexpr int O = ORDER, Q = 2 * O + 1;
    __shared__ float red[8];
    __shared__ int reached;
    // No node's bound exceeds dy.acap (the straddling case at the largest
    // |w_p| of the grid), so once some CTA has reached it the grid maximum
    // is known whatever the other CTAs would find: they skip their reads.
    // (The component is cleared before each step's alpha passes.)
    if (threadIdx.x == 0)
        reached = dy.acap > 0.0f && __ldcg(&st->alpha_bits[slot][2]) >= __float_as_uint(dy.acap);
    __syncthreads();
    if (reached) return;
    const float *__restrict__ src = slot ? st->nxt : st->cur;
    const int nh = g.n[2], inner = g.stride[2];    // heading planes; floats per plane of an (x, y) block
    const uint32_t isegs = uint32_t(inner / 4);
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    float amax = 0.0f;
    if (t < uint32_t(g.n[0] * g.n[1]) * isegs) {
        const uint32_t o = t / isegs;               // (x, y) block
        const int seg = int(t - o * isegs);
        const int base = int(o) * nh * inner + seg * 4;
        const uint32_t row = fast_div(uint32_t(seg), g.div_segs);   // (v_p, w_p) row of the block
        const int s0 = (seg - int(row) * g.segs) * 4;
        const int iwp = int(row - fast_div(row, g.div[4]) * uint32_t(g.n[4]));
        const float wp = ldgf(g.coord[4] + iwp);
        const int nvalid = min(4, g.n[5] - s0);
        const int per = g.periodic[2];
        float4 w[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) w[k] = stream_value(src, base, k - O, nh, per, inner);
        for (int h = 0; h < nh; ++h) {
            const float4 nx = (h + 1 < nh) ? stream_value(src, base, h + 1 + O, nh, per, inner) : w[Q - 1];
            const float4 m2 = w[0], m1 = w[O - 1], c4 = w[O], p1 = w[O + 1], p2 = w[Q - 1];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float dm, dp;
                diffs<ORDER>(lane(m2, k), lane(m1, k), lane(c4, k), lane(p1, k), lane(p2, k), dm, dp);
                if (k < nvalid) amax = fmaxf(amax, rel6d_theta_alpha(dy, wp, fminf(dm, dp), fmaxf(dm, dp)));
            }
#pragma unroll
            for (int k = 0; k < Q - 1; ++k) w[k] = w[k + 1];
            w[Q - 1] = nx;
        }
    }
    amax = warp_max(amax);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = amax;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.0f;
        for (int w = 0; w < (blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
        atomicMax(&st->alpha_bits[slot][2], __float_as_uint(m));
    }
}

// Capture-model alpha of phi (slot 0: cur) or phi1 (slot 1: nxt), every
// component per stage (Section 2.1 global alpha, readings R5 and R20): at
// each node the inputs selectable over its derivative box -- the evader turn
// a from the interval of its switching function y p_x - x p_y - p_th, the
// pursuer turn b from the interval of p_th -- and the largest |f_d| over
// every combination of them.  One thread per four-node segment.
template <int ORDER>
__global__ void __launch_bounds__(256) k_alpha_capture(GridDesc g, DynDesc dy, SolveState *st, int slot)
{
    __shared__ float red[8][3];
    const float *__restrict__ src = slot ? st->nxt : st->cur;
    float amax[3] = {0.0f, 0.0f, 0.0f};
    const float v = dy.prm[0], A = dy.prm[1], B = dy.prm[2];
    const float a_up = dy.umode == MODE_MAX ? A : -A, b_up = dy.dmode == MODE_MAX ? B : -B;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < uint32_t(g.nthreads)) {
        int idx[3];
        const int base = segment_index<3>(g, t, idx);
        const float4 c4 = ldg4(src + base);
        float4 m[2][2], p[2][2];   // axis, offset 1 / 2
        for (int d = 0; d < 2; ++d) {
            m[d][0] = row_shift4(src, base, idx[d], g.stride[d], g.n[d], g.periodic[d], -1);
            p[d][0] = row_shift4(src, base, idx[d], g.stride[d], g.n[d], g.periodic[d], +1);
            m[d][1] = m[d][0];
            p[d][1] = p[d][0];
            if (ORDER == 2) {
                m[d][1] = row_shift4(src, base, idx[d], g.stride[d], g.n[d], g.periodic[d], -2);
                p[d][1] = row_shift4(src, base, idx[d], g.stride[d], g.n[d], g.periodic[d], +2);
            }
        }
        const int s0 = idx[2], nl = g.n[2];
        const float *rowp = src + (base - s0);
        float w[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) w[j] = last_axis_value(rowp, s0 + j - 2, nl, g.periodic[2]);
        const float x = ldgf(g.coord[0] + idx[0]), y = ldgf(g.coord[1] + idx[1]);
        const int nvalid = min(4, nl - s0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (k >= nvalid) break;
            float lo[3], hi[3];
            for (int d = 0; d < 2; ++d) {
                float dm, dp;
                diffs<ORDER>(lane(m[d][1], k), lane(m[d][0], k), lane(c4, k), lane(p[d][0], k), lane(p[d][1], k), dm,
                             dp);
                lo[d] = fminf(dm, dp) * g.inv_dz[d];
                hi[d] = fmaxf(dm, dp) * g.inv_dz[d];
            }
            {
                float dm, dp;
                diffs<ORDER>(w[k], w[k + 1], w[k + 2], w[k + 3], w[k + 4], dm, dp);
                lo[2] = fminf(dm, dp) * g.inv_dz[2];
                hi[2] = fmaxf(dm, dp) * g.inv_dz[2];
            }
            // interval of s_a = y p_x - x p_y - p_th over the box
            const float gc[3] = {y, -x, -1.0f};
            float slo = 0.0f, shi = 0.0f;
            for (int d = 0; d < 3; ++d) {
                slo += gc[d] >= 0.0f ? gc[d] * lo[d] : gc[d] * hi[d];
                shi += gc[d] >= 0.0f ? gc[d] * hi[d] : gc[d] * lo[d];
            }
            float as[2], bs[2];
            int na = 1, nb = 1;
            if (slo > 0.0f) as[0] = a_up;
            else if (shi < 0.0f) as[0] = -a_up;
            else { as[0] = -A; as[1] = A; na = 2; }
            if (lo[2] > 0.0f) bs[0] = b_up;
            else if (hi[2] < 0.0f) bs[0] = -b_up;
            else { bs[0] = -B; bs[1] = B; nb = 2; }
            const float cth = ldgf(g.cos_tab + s0 + k), sth = ldgf(g.sin_tab + s0 + k);
            float aloc[3] = {0.0f, 0.0f, 0.0f};
            for (int ia = 0; ia < na; ++ia) {
                aloc[0] = fmaxf(aloc[0], fabsf(-v + v * cth + as[ia] * y));
                aloc[1] = fmaxf(aloc[1], fabsf(v * sth - as[ia] * x));
                for (int ib = 0; ib < nb; ++ib) aloc[2] = fmaxf(aloc[2], fabsf(bs[ib] - as[ia]));
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                amax[d] = fmaxf(amax[d], aloc[d]);
                // per-node dissipation (Algorithm 1's second loop): this node's own bound
                if (g.cdn) g.cdn[d * g.cdn_stride + base + k] = 0.5f * aloc[d] * g.inv_dz[d];
            }
        }
    }
    const int lane_id = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        amax[d] = warp_max(amax[d]);
        if (lane_id == 0) red[warp][d] = amax[d];
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        float mx = 0.0f;
        for (int w2 = 0; w2 < (blockDim.x >> 5); ++w2) mx = fmaxf(mx, red[w2][threadIdx.x]);
        atomicMax(&st->alpha_bits[slot][threadIdx.x], __float_as_uint(mx));
    }
}

// Threads of the Rel6D heading-rate alpha pass: one per four-node segment
// of a heading plane of every (x, y) block.
inline int64_t alpha_rel6d_threads(const GridDesc &g)
{
    return int64_t(g.n[0]) * g.n[1] * (g.stride[2] / 4);
}

inline int blocks_for(int64_t n, int threads) { return int((n + threads - 1) / threads); }

inline int reduce_blocks(int64_t n)
{
    const int b = blocks_for(n, 256);
    return b < 152 * 8 ? b : 152 * 8;
}

}  // namespace odp

#include "hj_plane.cuh"
#include "hj_bulk.cuh"

namespace odp {

// The bulk-staged pass of a single solve (hj_bulk.cuh): one kernel per RK
// stage and obstacle use.
template <int ND, int ORDER, int DYN>
cudaError_t launch_stage_bulk_t(const GridDesc &g, const DynDesc &dy, SolveState *st, const float *l,
                                const float *gob, int stage, int brt, cudaStream_t s)
{
    const bool ob = gob != nullptr;
    // shared memory for the read-once tiles this stage stages (l for the
    // BRT min, phi^n for the Heun average, the obstacle)
    const int naux = stage == 1 ? 0 : (brt ? 1 : 0) + (stage == 2 ? 1 : 0) + (ob ? 1 : 0);
    const int blocks = g.bk.items[ORDER - 1], th = 32 * (g.bk.cwarps + 1);
    const int sm = int(bulk_smem_bytes(g.bk, g.n_pad, ND, ORDER, naux));
    if (stage == 0) {
        if (ob)
            k_stage_bulk<ND, ORDER, DYN, 0, 1><<<blocks, th, sm, s>>>(g, dy, st, l, gob, stage, brt);
        else
            k_stage_bulk<ND, ORDER, DYN, 0, 0><<<blocks, th, sm, s>>>(g, dy, st, l, gob, stage, brt);
    } else if (stage == 1) {
        k_stage_bulk<ND, ORDER, DYN, 1, 0><<<blocks, th, sm, s>>>(g, dy, st, l, gob, stage, brt);
    } else {
        if (ob)
            k_stage_bulk<ND, ORDER, DYN, 2, 1><<<blocks, th, sm, s>>>(g, dy, st, l, gob, stage, brt);
        else
            k_stage_bulk<ND, ORDER, DYN, 2, 0><<<blocks, th, sm, s>>>(g, dy, st, l, gob, stage, brt);
    }
    return cudaGetLastError();
}

// Resident CTAs per SM of the bulk-staged pass with `threads` threads and
// `smem` shared bytes a CTA (the fewer of its two RK stages).
template <int ND, int ORDER, int DYN>
cudaError_t occupancy_stage_bulk_t(int threads, int smem, int *per_sm)
{
    int a = 0, b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_stage_bulk<ND, ORDER, DYN, 1, 0>, threads, smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_stage_bulk<ND, ORDER, DYN, 2, 0>, threads, smem);
    *per_sm = a < b ? a : b;
    return e;
}

template <int ND, int DYN>
cudaError_t occupancy_stage_bulk_nd(int order, int threads, int smem, int *per_sm)
{
    if constexpr (ND >= 3 && (DYN == DYN_DUBINS3D || DYN == DYN_DUBINSCAR4D || DYN == DYN_REL6D)) {
        if (order == 1) return occupancy_stage_bulk_t<ND, 1, DYN>(threads, smem, per_sm);
        return occupancy_stage_bulk_t<ND, 2, DYN>(threads, smem, per_sm);
    }
    *per_sm = 0;
    return cudaSuccess;
}

template <int ND, int ORDER, int DYN>
cudaError_t configure_stage_bulk_t()
{
    const int bytes = 227 * 1024;
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *f) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    };
    set((const void *)k_stage_bulk<ND, ORDER, DYN, 0, 0>);
    set((const void *)k_stage_bulk<ND, ORDER, DYN, 0, 1>);
    set((const void *)k_stage_bulk<ND, ORDER, DYN, 1, 0>);
    set((const void *)k_stage_bulk<ND, ORDER, DYN, 2, 0>);
    set((const void *)k_stage_bulk<ND, ORDER, DYN, 2, 1>);
    return e;
}

template <int ND, int DYN>
cudaError_t launch_stage_t(const GridDesc &g, const DynDesc &dy, SolveState *st, const float *l,
                           const float *gob, int order, int stage, int brt, cudaStream_t s)
{
    if constexpr (ND >= 3) {
        if constexpr (DYN == DYN_DUBINS3D || DYN == DYN_DUBINSCAR4D || DYN == DYN_REL6D) {
            // bk.use: 1 automatic (the bulk-staged pass where it measured
            // faster: grids of 4 or more dimensions), 2 the bulk-staged pass
            // wherever it applies
            const bool want = g.bk.use == 2 || (g.bk.use == 1 && ND >= 4);
            if (want && g.n[ND - 1] % 4 == 0 && !dy.local_diss && g.bk.smem[order - 1] > 0) {
                if (order == 1) return launch_stage_bulk_t<ND, 1, DYN>(g, dy, st, l, gob, stage, brt, s);
                return launch_stage_bulk_t<ND, 2, DYN>(g, dy, st, l, gob, stage, brt, s);
            }
        }
        if (g.pg.use) {
            // Dubins3D, DubinsCar4D and Rel6D grids whose last axis is a
            // multiple of 4 get one kernel per RK stage and obstacle use; the
            // other models and shapes take both at run time
            const int blocks = g.pg.items, th = g.pg.threads, sm = g.pg.smem[order - 1];
            const bool full = g.n[ND - 1] % 4 == 0;
            constexpr bool SPEC = DYN == DYN_DUBINS3D || DYN == DYN_DUBINSCAR4D || DYN == DYN_REL6D;
            if (SPEC && full && !dy.local_diss) {
                const bool ob = gob != nullptr;
                if (order == 1) {
                    if (stage == 0) {
                        if (ob)
                            k_stage_plane<ND, 1, DYN, true, 0, 1><<<blocks, th, sm, s>>>(g, dy, st, l, gob, stage, brt);
                        else
                            k_stage_plane<ND, 1, DYN, true, 0, 0><<<blocks, th, sm, s>>>(g, dy, st, l, gob, stage, brt);
                    } else if (stage == 1) {
                        k_stage_plane<ND, 1, DYN, true, 1, 0><<<blocks, th, sm, s>>>(g, dy, st, l, gob, stage, brt);
                    } else {
                        if (ob)
                            k_stage_plane<ND, 1, DYN, true, 2, 1><<<blocks, th, sm, s>>>(g, dy, st, l, gob, stage, brt);
                        else
                            k_stage_plane<ND, 1, DYN, true, 2, 0><<<blocks, th, sm, s>>>(g, dy, st, l, gob, stage, brt);
                    }
                } else {
                    if (stage == 0) {
                        if (ob)
                            k_stage_plane<ND, 2, DYN, true, 0, 1><<<blocks, th, sm, s>>>(g, dy, st, l, gob, stage, brt);
                        else
                            k_stage_plane<ND, 2, DYN, true, 0, 0><<<blocks, th, sm, s>>>(g, dy, st, l, gob, stage, brt);
                    } else if (stage == 1) {
                        k_stage_plane<ND, 2, DYN, true, 1, 0><<<blocks, th, sm, s>>>(g, dy, st, l, gob, stage, brt);
                    } else {
                        if (ob)
                            k_stage_plane<ND, 2, DYN, true, 2, 1><<<blocks, th, sm, s>>>(g, dy, st, l, gob, stage, brt);
                        else
                            k_stage_plane<ND, 2, DYN, true, 2, 0><<<blocks, th, sm, s>>>(g, dy, st, l, gob, stage, brt);
                    }
                }
            } else if (order == 1) {
                if (full)
                    k_stage_plane<ND, 1, DYN, true, -1, -1><<<blocks, th, sm, s>>>(g, dy, st, l, gob, stage, brt);
                else
                    k_stage_plane<ND, 1, DYN, false, -1, -1><<<blocks, th, sm, s>>>(g, dy, st, l, gob, stage, brt);
            } else {
                if (full)
                    k_stage_plane<ND, 2, DYN, true, -1, -1><<<blocks, th, sm, s>>>(g, dy, st, l, gob, stage, brt);
                else
                    k_stage_plane<ND, 2, DYN, false, -1, -1><<<blocks, th, sm, s>>>(g, dy, st, l, gob, stage, brt);
            }
            return cudaGetLastError();
        }
    }
    const int grid = blocks_for(g.nthreads_rb, 256), block = 256;
    if (g.R == 4) {
        if (order == 1)
            k_stage<ND, 1, DYN, 4><<<grid, block, 0, s>>>(g, dy, st, l, gob, stage, brt);
        else
            k_stage<ND, 2, DYN, 4><<<grid, block, 0, s>>>(g, dy, st, l, gob, stage, brt);
    } else {
        if (order == 1)
            k_stage<ND, 1, DYN, 1><<<grid, block, 0, s>>>(g, dy, st, l, gob, stage, brt);
        else
            k_stage<ND, 2, DYN, 1><<<grid, block, 0, s>>>(g, dy, st, l, gob, stage, brt);
    }
    return cudaGetLastError();
}

// The plane-streaming tiles stay below the default 48 KB of dynamic shared
// memory; the bulk-staged pass's rings may need more.
template <int ND, int DYN>
cudaError_t configure_stage_t()
{
    if constexpr (ND >= 3 && (DYN == DYN_DUBINS3D || DYN == DYN_DUBINSCAR4D || DYN == DYN_REL6D)) {
        cudaError_t e = configure_stage_bulk_t<ND, 1, DYN>();
        if (e == cudaSuccess) e = configure_stage_bulk_t<ND, 2, DYN>();
        return e;
    }
    return cudaSuccess;
}

template <int ND, int DYN>
cudaError_t launch_alpha_static_t(const GridDesc &g, const DynDesc &dy, SolveState *st, cudaStream_t s)
{
    k_alpha_static<ND, DYN><<<reduce_blocks(g.total), 256, 0, s>>>(g, dy, st);
    return cudaGetLastError();
}

}  // namespace odp
