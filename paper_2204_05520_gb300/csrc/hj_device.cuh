// hj_device.cuh -- per-node arithmetic of Algorithm 1 shared by the kernels.
//
// Paper references (arXiv 2204.05520): Section 3.1.1 (grid, ghost nodes),
// Section 3.1.4 (upwind and ENO2 derivatives), Algorithm 1 (central
// derivative, optimal inputs, Hamiltonian, Lax-Friedrichs dissipation),
// Section 2.1 (global-alpha approximation), Appendix (dynamics).
#pragma once

#include "odp_common.cuh"

namespace odp {

ODP_HD float mode_sign(int mode) { return mode == MODE_MAX ? 1.0f : -1.0f; }

// k-th ghost node outside boundary node pb, from d = pb - pin with pin the
// inner neighbour (Section 3.1.1: extrapolated so that it keeps the sign of
// pb).  Each operation is rounded on its own (no contraction into an FMA),
// so every kernel forms the same ghost value.
ODP_HD float keep_sign_ghost_d(float pb, float d, float k)
{
#ifdef __CUDA_ARCH__
    return __fadd_rn(pb, __fmul_rn(k * (pb >= 0.0f ? 1.0f : -1.0f), fabsf(d)));
#else
    volatile float t = k * (pb >= 0.0f ? 1.0f : -1.0f) * fabsf(d);
    return pb + t;
#endif
}

ODP_HD float keep_sign_ghost(float pb, float pin, float k)
{
#ifdef __CUDA_ARCH__
    return keep_sign_ghost_d(pb, __fsub_rn(pb, pin), k);
#else
    return keep_sign_ghost_d(pb, pb - pin, k);
#endif
}

// Unscaled one-sided differences of one node from its five-node window
// (ENO2) or three-node window (upwind): dm = h p-, dp = h p+.
// ORDER 2: p- = D-phi + (h/2) c, p+ = D+phi - (h/2) c', c (c') the second
// difference of smaller magnitude at i-1 or i (i or i+1), ties keep the
// centred one.
template <int ORDER>
ODP_HD void diffs(float fm2, float fm1, float f0, float fp1, float fp2, float &dm, float &dp)
{
    const float a = f0 - fm1, b = fp1 - f0;
    if (ORDER == 1) {
        dm = a;
        dp = b;
    } else {
        const float d2l = a - (fm1 - fm2);
        const float d2m = b - a;
        const float d2r = (fp2 - fp1) - b;
        const float cm = (fabsf(d2l) < fabsf(d2m)) ? d2l : d2m;
        const float cp = (fabsf(d2r) < fabsf(d2m)) ? d2r : d2m;
        dm = a + 0.5f * cm;
        dp = b - 0.5f * cp;
    }
}

// ---------------------------------------------------------------------------
// Paired float32 arithmetic: two lanes per instruction on sm_100+ (FADD2,
// FFMA2, FMUL2).  Each lane is an ordinary IEEE float32 operation, so the
// results are those of the scalar operations.
// ---------------------------------------------------------------------------
ODP_HD float2 f2add(float2 a, float2 b)
{
#ifdef __CUDA_ARCH__
    return __fadd2_rn(a, b);
#else
    return make_float2(a.x + b.x, a.y + b.y);
#endif
}

ODP_HD float2 f2fma(float2 a, float2 b, float2 c)
{
#ifdef __CUDA_ARCH__
    return __ffma2_rn(a, b, c);
#else
    return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
#endif
}

ODP_HD float2 f2mul(float2 a, float2 b)
{
#ifdef __CUDA_ARCH__
    return __fmul2_rn(a, b);
#else
    return make_float2(a.x * b.x, a.y * b.y);
#endif
}

// a - b lane by lane (a + (-b), rounded once)
ODP_HD float2 f2sub(float2 a, float2 b) { return f2add(a, make_float2(-b.x, -b.y)); }

ODP_HD float2 f2abs(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }

ODP_HD float2 f2splat(float a) { return make_float2(a, a); }

// the smaller-magnitude choice of ENO2, lane by lane: (|x| < |c|) ? x : c
ODP_HD float2 f2pick(float2 x, float2 c)
{
    return make_float2(fabsf(x.x) < fabsf(c.x) ? x.x : c.x, fabsf(x.y) < fabsf(c.y) ? x.y : c.y);
}

// One axis of the Lax-Friedrichs right-hand side for two nodes from their
// five-node (ENO2) or three-node (upwind) stencils along that axis:
// L += cA P + cS |P| + cD M with P = dp + dm, M = dp - dm (unscaled one-sided
// differences, see diffs()); has_a / has_s (compile-time constants at every
// call) drop the terms a model does not have on this axis.  Same operation
// order as diffs() for the ENO2 choice.  pair_diffs / pair_terms are its two
// halves.
template <int ORDER>
ODP_HD void pair_diffs(float2 fm2, float2 fm1, float2 f0, float2 fp1, float2 fp2, float2 &dm, float2 &dp)
{
    const float2 a = f2sub(f0, fm1), b = f2sub(fp1, f0);
    dm = a;
    dp = b;
    if (ORDER == 2) {
        const float2 d2l = f2sub(a, f2sub(fm1, fm2));
        const float2 d2m = f2sub(b, a);
        const float2 d2r = f2sub(f2sub(fp2, fp1), b);
        const float2 cm = f2pick(d2l, d2m), cp = f2pick(d2r, d2m);
        dm = f2fma(cm, f2splat(0.5f), a);
        dp = f2fma(cp, f2splat(-0.5f), b);
    }
}

// The axis's terms from the unscaled one-sided differences of two nodes:
// L += cA P + cS |P| + cD M, cD per lane (the dissipation coefficient
// alpha / (2 h) of each node).
ODP_HD void pair_terms(float2 dm, float2 dp, float2 cA, float cS, float2 cD, float2 &L, bool has_a, bool has_s,
                       float2 *Pout = nullptr)
{
    const float2 P = f2add(dp, dm), M = f2sub(dp, dm);
    if (Pout) *Pout = P;
    if (has_a) L = f2fma(cA, P, L);
    if (has_s) L = f2fma(f2splat(cS), f2abs(P), L);
    L = f2fma(cD, M, L);
}

template <int ORDER>
ODP_HD void axis_pair(float2 fm2, float2 fm1, float2 f0, float2 fp1, float2 fp2, float2 cA, float cS, float2 cD,
                      float2 &L, bool has_a, bool has_s)
{
    float2 dm, dp;
    pair_diffs<ORDER>(fm2, fm1, f0, fp1, fp2, dm, dp);
    pair_terms(dm, dp, cA, cS, cD, L, has_a, has_s);
}

// The last axis of four consecutive nodes from their eight-node window
// w[j] = phi(first - 2 + j), sharing the first and second differences of the
// window between the four nodes (the same float32 operations as diffs()).
// The per-node operations run on node pairs (0, 1) and (2, 3) in paired
// float32 instructions; each lane is the scalar operation, so the results
// are those of the scalar form.
template <int ORDER>
ODP_HD void axis_last(const float *w, const float *cA, float cS, float cD, float *L, bool has_a, bool has_s,
                      float *Pout = nullptr, const float *cDn = nullptr)
{
    // cDn (optional): each node's own dissipation coefficient instead of cD
    float e[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) e[j] = w[j + 1] - w[j];
    float d2[6];
    if (ORDER == 2) {
#pragma unroll
        for (int j = 0; j < 6; ++j) d2[j] = e[j + 1] - e[j];   // the second difference at node j - 1
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k = 2 * h;   // nodes k, k + 1
        const float2 a = make_float2(e[k + 1], e[k + 2]), b = make_float2(e[k + 2], e[k + 3]);
        float2 dm = a, dp = b;
        if (ORDER == 2) {
            // node i: left choice between D2(i - 1), D2(i); right between D2(i + 1), D2(i)
            const float2 cm = f2pick(make_float2(d2[k], d2[k + 1]), make_float2(d2[k + 1], d2[k + 2]));
            const float2 cp = f2pick(make_float2(d2[k + 2], d2[k + 3]), make_float2(d2[k + 1], d2[k + 2]));
            dm = f2fma(cm, f2splat(0.5f), a);
            dp = f2fma(cp, f2splat(-0.5f), b);
        }
        const float2 P = f2add(dp, dm), M = f2sub(dp, dm);
        if (Pout) {
            Pout[k] = P.x;
            Pout[k + 1] = P.y;
        }
        float2 acc = make_float2(L[k], L[k + 1]);
        if (has_a) acc = f2fma(make_float2(cA[k], cA[k + 1]), P, acc);
        if (has_s) acc = f2fma(f2splat(cS), f2abs(P), acc);
        acc = f2fma(cDn ? make_float2(cDn[k], cDn[k + 1]) : f2splat(cD), M, acc);
        L[k] = acc.x;
        L[k + 1] = acc.y;
    }
}

// Which axes carry a drift term (a_d(z) depends on the state) and which a
// bounded input (S_d != 0), per model (Appendix dynamics).  The capture
// model's evader turn enters all three axes; its term S_a |y pbar_x -
// x pbar_y - pbar_th| is added separately (capture_term).
template <int DYN, int ND>
constexpr bool has_drift(int d)
{
    return DYN == DYN_ADVECTION ? true
         : DYN == DYN_SINGLE_INT ? false
         : DYN == DYN_DUBINS3D ? d < 2
         : DYN == DYN_DUBINSCAR4D ? d < 2
         : DYN == DYN_CAPTURE ? d < 2
         : d < 3;   // Rel6D
}

template <int DYN, int ND>
constexpr bool has_bound(int d)
{
    return DYN == DYN_ADVECTION ? false
         : DYN == DYN_SINGLE_INT ? true
         : DYN == DYN_DUBINS3D ? d == 2
         : DYN == DYN_DUBINSCAR4D ? d >= 2
         : DYN == DYN_CAPTURE ? d == 2
         : d >= 2;  // Rel6D
}

// Local dissipation bound a_d(z) (global-alpha reading of Section 2.1): the
// largest |f_d| over the input extremes a node's derivative box can select.
// For every model here except the Rel6D heading rate this does not depend on
// phi ("static" components); the Rel6D component th' = w_e - w_p depends on
// the sign range of p_th and is computed per stage.
template <int DYN, int ND>
ODP_HD void static_alpha(const GridDesc &g, const DynDesc &dy, const int *idx, float *a)
{
    if (DYN == DYN_SINGLE_INT) {
        for (int d = 0; d < ND; ++d) a[d] = dy.prm[0];
    } else if (DYN == DYN_ADVECTION) {
        for (int d = 0; d < ND; ++d) a[d] = fabsf(dy.prm[d]);
    } else if (DYN == DYN_DUBINS3D) {
        a[0] = fabsf(dy.prm[0] * ldgf(g.cos_tab + idx[2]));
        a[1] = fabsf(dy.prm[0] * ldgf(g.sin_tab + idx[2]));
        a[2] = dy.prm[1];
    } else if (DYN == DYN_CAPTURE) {
        for (int d = 0; d < ND; ++d) a[d] = 0.0f;   // every component depends on phi
    } else if (DYN == DYN_DUBINSCAR4D) {
        const float v = ldgf(g.coord[2] + idx[2]);
        a[0] = fabsf(v * ldgf(g.cos_tab + idx[3]));
        a[1] = fabsf(v * ldgf(g.sin_tab + idx[3]));
        a[2] = dy.prm[0];
        a[3] = dy.prm[1];
    } else {
        const float x = ldgf(g.coord[0] + idx[0]);
        const float y = ldgf(g.coord[1] + idx[1]);
        const float c = ldgf(g.cos_tab + idx[2]);
        const float s = ldgf(g.sin_tab + idx[2]);
        const float vp = ldgf(g.coord[3] + idx[3]);
        const float wp = ldgf(g.coord[4] + idx[4]);
        const float ve = ldgf(g.coord[5] + idx[5]);
        a[0] = fabsf(-vp + ve * c + wp * y);
        a[1] = fabsf(ve * s - wp * x);
        a[2] = 0.0f;  // dynamic component
        a[3] = dy.prm[0];
        a[4] = dy.prm[1];
        a[5] = dy.prm[2];
    }
}

// Rel6D heading-rate bound from the interval [lo, hi] of p_th (the switching
// function of w_e): strictly positive or negative selects one extreme,
// otherwise both.
ODP_HD float rel6d_theta_alpha(const DynDesc &dy, float wp, float lo, float hi)
{
    const float b = dy.prm[3];
    const float pos = (dy.dmode == MODE_MAX) ? b : -b;  // w_e chosen when p_th > 0
    if (lo > 0.0f) return fabsf(pos - wp);
    if (hi < 0.0f) return fabsf(-pos - wp);
    return fmaxf(fabsf(b - wp), fabsf(-b - wp));
}

// Multi-index of logical node i (no padding).
ODP_HD void unflatten(const GridDesc &g, int nd, uint32_t i, int *idx)
{
    for (int d = nd - 1; d > 0; --d) {
        const uint32_t q = fast_div(i, g.div[d]);
        idx[d] = int(i - q * uint32_t(g.n[d]));
        i = q;
    }
    idx[0] = int(i);
}

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

}  // namespace odp
