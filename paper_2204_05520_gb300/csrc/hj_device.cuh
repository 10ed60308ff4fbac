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

ODP_HD float keep_sign_ghost(float pb, float pin, float k)
{
    // k-th ghost node outside boundary node pb with inner neighbour pin
    // (Section 3.1.1: extrapolated so that it keeps the sign of pb)
    return pb + k * (pb >= 0.0f ? 1.0f : -1.0f) * fabsf(pb - pin);
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
