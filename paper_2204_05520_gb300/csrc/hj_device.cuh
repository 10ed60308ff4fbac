// hj_device.cuh -- per-node arithmetic of one Algorithm 1 stage on the GPU.
//
// Paper references (arXiv 2204.05520): Section 3.1.1 (grid, ghost nodes),
// Section 3.1.4 (upwind and ENO2 derivatives), Algorithm 1 (central
// derivative, optimal inputs, Hamiltonian, Lax-Friedrichs dissipation),
// Section 2.1 (global-alpha approximation), Appendix (dynamics).
#pragma once

#include "odp_common.cuh"

namespace odp {

// ---------------------------------------------------------------------------
// neighbours with periodic wrap or sign-keeping ghost extrapolation
// (Section 3.1.1): the k-th ghost outside boundary node b is
// phi_b + k * sign(phi_b) * |phi_b - phi_inner|, sign(0) = +1.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float node_shift(const float *__restrict__ src, int i, int id, int stride,
                                            int n, int periodic, int off)
{
    int j = id + off;
    if (periodic) {
        if (j < 0) j += n;
        if (j < 0) j += n;
        if (j >= n) j -= n;
        if (j >= n) j -= n;
        return __ldg(src + i + (j - id) * stride);
    }
    if (j >= 0 && j < n) return __ldg(src + i + off * stride);
    const int b = (j < 0) ? 0 : n - 1;
    const int in = (j < 0) ? 1 : n - 2;
    const float k = (j < 0) ? float(-j) : float(j - (n - 1));
    const float pb = __ldg(src + i + (b - id) * stride);
    const float pin = __ldg(src + i + (in - id) * stride);
    const float s = (pb >= 0.0f) ? 1.0f : -1.0f;
    return pb + k * s * fabsf(pb - pin);
}

// One-sided derivatives along one axis.  ORDER 1: upwind differences.
// ORDER 2: ENO2, p- = D-phi + (h/2) c, p+ = D+phi - (h/2) c', where c (c')
// is the second difference of smaller magnitude at i-1 or i (i or i+1);
// equal magnitudes keep the centred one.  Second differences are formed
// unscaled and multiplied by 1/h once.
template <int ORDER>
__device__ __forceinline__ void one_sided(const float *__restrict__ src, int i, int id, int stride,
                                          int n, int periodic, float inv_h, float &pm, float &pp)
{
    const float f0 = __ldg(src + i);
    const float fm1 = node_shift(src, i, id, stride, n, periodic, -1);
    const float fp1 = node_shift(src, i, id, stride, n, periodic, +1);
    const float dm = f0 - fm1;
    const float dp = fp1 - f0;
    if (ORDER == 1) {
        pm = dm * inv_h;
        pp = dp * inv_h;
    } else {
        const float fm2 = node_shift(src, i, id, stride, n, periodic, -2);
        const float fp2 = node_shift(src, i, id, stride, n, periodic, +2);
        const float d2l = (f0 - fm1) - (fm1 - fm2);
        const float d2m = (fp1 - f0) - (f0 - fm1);
        const float d2r = (fp2 - fp1) - (fp1 - f0);
        const float cm = (fabsf(d2l) < fabsf(d2m)) ? d2l : d2m;
        const float cp = (fabsf(d2r) < fabsf(d2m)) ? d2r : d2m;
        pm = (dm + 0.5f * cm) * inv_h;
        pp = (dp - 0.5f * cp) * inv_h;
    }
}

__device__ __forceinline__ float mode_sign(int mode) { return mode == MODE_MAX ? 1.0f : -1.0f; }

// ---------------------------------------------------------------------------
// Hamiltonian H = pbar . f(z, u*, d*) with the bang-bang inputs folded in:
// an input with bound b and switching function s contributes
// s * u* = +b|s| in "max" mode and -b|s| in "min" mode (Algorithm 1; the
// Section 4.2 opt_ctrl / opt_dstb rule).
// ---------------------------------------------------------------------------
template <int DYN, int ND>
__device__ __forceinline__ float hamiltonian(const GridDesc &g, const DynDesc &dy, const int *idx,
                                             const float *p)
{
    const float su = mode_sign(dy.umode);
    if (DYN == DYN_SINGLE_INT) {
        float acc = 0.0f;
#pragma unroll
        for (int d = 0; d < ND; ++d) acc += fabsf(p[d]);
        return su * dy.prm[0] * acc;
    } else if (DYN == DYN_ADVECTION) {
        float acc = 0.0f;
#pragma unroll
        for (int d = 0; d < ND; ++d) acc += dy.prm[d] * p[d];
        return acc;
    } else if (DYN == DYN_DUBINS3D) {      // (x, y, th)
        const float c = __ldg(g.cos_tab + idx[2]);
        const float s = __ldg(g.sin_tab + idx[2]);
        return dy.prm[0] * (p[0] * c + p[1] * s) + su * dy.prm[1] * fabsf(p[2]);
    } else if (DYN == DYN_DUBINSCAR4D) {   // (x, y, v, th)
        const float c = __ldg(g.cos_tab + idx[3]);
        const float s = __ldg(g.sin_tab + idx[3]);
        const float v = __ldg(g.coord[2] + idx[2]);
        return v * (p[0] * c + p[1] * s) + su * (dy.prm[0] * fabsf(p[2]) + dy.prm[1] * fabsf(p[3]));
    } else {                               // DYN_REL6D: (x, y, th, v_p, w_p, v_e)
        const float sd = mode_sign(dy.dmode);
        const float x = __ldg(g.coord[0] + idx[0]);
        const float y = __ldg(g.coord[1] + idx[1]);
        const float c = __ldg(g.cos_tab + idx[2]);
        const float s = __ldg(g.sin_tab + idx[2]);
        const float vp = __ldg(g.coord[3] + idx[3]);
        const float wp = __ldg(g.coord[4] + idx[4]);
        const float ve = __ldg(g.coord[5] + idx[5]);
        const float f0 = -vp + ve * c + wp * y;
        const float f1 = ve * s - wp * x;
        return p[0] * f0 + p[1] * f1 - p[2] * wp +
               su * (dy.prm[0] * fabsf(p[3]) + dy.prm[1] * fabsf(p[4])) +
               sd * (dy.prm[3] * fabsf(p[2]) + dy.prm[2] * fabsf(p[5]));
    }
}

// ---------------------------------------------------------------------------
// Local dissipation bound a_d(z) (global-alpha reading of Section 2.1): the
// largest |f_d| over the input extremes a node's derivative box can select.
// For every model here except the Rel6D heading rate this does not depend on
// phi ("static" components); the Rel6D component th' = w_e - w_p depends on
// the sign range of p_th and is computed per stage.
// ---------------------------------------------------------------------------
template <int DYN, int ND>
__device__ __forceinline__ void static_alpha(const GridDesc &g, const DynDesc &dy, const int *idx,
                                             float *a)
{
    if (DYN == DYN_SINGLE_INT) {
#pragma unroll
        for (int d = 0; d < ND; ++d) a[d] = dy.prm[0];
    } else if (DYN == DYN_ADVECTION) {
#pragma unroll
        for (int d = 0; d < ND; ++d) a[d] = fabsf(dy.prm[d]);
    } else if (DYN == DYN_DUBINS3D) {
        a[0] = fabsf(dy.prm[0] * __ldg(g.cos_tab + idx[2]));
        a[1] = fabsf(dy.prm[0] * __ldg(g.sin_tab + idx[2]));
        a[2] = dy.prm[1];
    } else if (DYN == DYN_DUBINSCAR4D) {
        const float v = __ldg(g.coord[2] + idx[2]);
        a[0] = fabsf(v * __ldg(g.cos_tab + idx[3]));
        a[1] = fabsf(v * __ldg(g.sin_tab + idx[3]));
        a[2] = dy.prm[0];
        a[3] = dy.prm[1];
    } else {
        const float x = __ldg(g.coord[0] + idx[0]);
        const float y = __ldg(g.coord[1] + idx[1]);
        const float c = __ldg(g.cos_tab + idx[2]);
        const float s = __ldg(g.sin_tab + idx[2]);
        const float vp = __ldg(g.coord[3] + idx[3]);
        const float wp = __ldg(g.coord[4] + idx[4]);
        const float ve = __ldg(g.coord[5] + idx[5]);
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
__device__ __forceinline__ float rel6d_theta_alpha(const DynDesc &dy, float wp, float lo, float hi)
{
    const float b = dy.prm[3];
    const float pos = (dy.dmode == MODE_MAX) ? b : -b;  // w_e chosen when p_th > 0
    if (lo > 0.0f) return fabsf(pos - wp);
    if (hi < 0.0f) return fabsf(-pos - wp);
    return fmaxf(fabsf(b - wp), fabsf(-b - wp));
}

__device__ __forceinline__ void unflatten(const GridDesc &g, int nd, uint32_t i, int *idx)
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
