/*
 * odp_oracle.c -- plain FP64 CPU oracle of the time-dependent HJ level-set
 * method of OptimizedDP (arXiv 2204.05520), Algorithm 1, and of its
 * time-to-reach function by Lax-Friedrichs sweeping, Algorithm 2.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code, header,
 * table or constant with the CUDA library; the two meet only through the
 * seeded inputs both are given.
 *
 * It is written to be checked against the paper by eye, not to be fast: every
 * value is double, every grid point is visited with plain loops over its
 * multi-index, and the two per-point passes of Algorithm 1 (Hamiltonian and
 * derivative range, then dissipation) are kept as two passes.  The only
 * liberty is an OpenMP "parallel for" over grid points, the parallel outer loop
 * of Section 5.1; it changes no result (per-point work is independent and the
 * one reduction is a max).
 *
 * Readings of the paper taken where it is silent or garbled (each is also
 * listed in the design notes of the repository):
 *  R1 time runs as look-back tau = -s from 0 to T:  phi(tau+dt) = phi + dt*L.
 *  R2 Lax-Friedrichs sign: L = H(pbar) + 1/2 sum_d alpha_d (p+_d - p-_d)
 *     (positive viscosity in tau).
 *  R4 mode rule: a "max" input takes +bound when its switching function is
 *     >= 0, a "min" input takes -bound when it is >= 0.
 *  R5 alpha: global per-component bound, alpha_d = max over grid points of the
 *     largest |f_d| over the input extremes that the point's derivative box
 *     can select (a switching interval strictly above or below 0 selects one
 *     extreme, otherwise both).
 *  R7 CFL step dt = cfl / sum_d(alpha_d/dz_d), clipped at the segment end;
 *     a segment ends when its remaining time is <= 1e-12 * its end time.
 *  R8 TVD-RK2 (Heun / Shu-Osher): phi1 = phi + dt L(phi);
 *     phi2 = phi1 + dt L(phi1); phi_new = (phi + phi2)/2; one dt per step from
 *     the stage-1 alpha, stage 2 uses its own alpha.  BRT min once per step.
 *  R9 ghost cells on non-periodic axes: k cells outside the boundary point b,
 *     g_k = phi_b + k*sign(phi_b)*|phi_b - phi_inner|, sign(0) = +1.
 *  R18 per-node alpha (Algorithm 1's second loop, kept as an option): the
 *     dissipation of node i uses alpha_i, the local bound of R5 at that node
 *     (its own derivative box), instead of the grid maximum; the CFL step
 *     still uses the grid maximum.
 *  R20 alpha with coupled inputs: each input's selectable extremes come from
 *     the range of its own switching function over the derivative box, and
 *     alpha_d is the largest |f_d| over every combination of them (a product
 *     set).  For the capture model, whose two inputs share p_th, this bounds
 *     Algorithm 1's max over the box from above.
 *  R17 reach-avoid (Section 4.3, the target and obstacle computation
 *     methods): with an obstacle function g, after each full step
 *     phi <- max(phi, g), taken after the BRT min with l (target first, then
 *     obstacle, in the order the solver options list them); g is
 *     time-invariant here.
 *  R26 time-varying target and obstacle (Section 2.1's time-varying variants,
 *     the target and obstacle computation methods of Section 4.3): with the
 *     sets sampled at every tau, l_k = l(., tau_k) and g_k = g(., tau_k), phi
 *     starts from l_0 and every step of segment (tau_k, tau_k+1] takes its
 *     post-step min with l_k+1 and max with g_k+1, the sets at the end of the
 *     segment in which the step lands.
 *  R27 computation methods (Section 4.3's table; its time indices are
 *     garbled): after each full step, first the target side -- min / max
 *     with the target set of the segment (minVWithVTarget, maxVWithVTarget),
 *     with the value before the step (minVWithVInit, maxVWithVInit: the
 *     "value over time"), or with the initial value phi(0) (minVWithV0,
 *     maxVWithV0) -- then the obstacle side, max / min with g
 *     (maxVWithObstacle, minVWithObstacle).
 *  R10 ENO2: p- = D-phi + (h/2) c, p+ = D+phi - (h/2) c', c (c') the second
 *     difference of smaller magnitude among those at i-1 and i (i and i+1);
 *     on equal magnitude the centred one (at i).  Magnitudes are equal when
 *     they differ by at most 2^-40 times the sum of the magnitudes of the
 *     five window values (the tie margin, OG_ENO_TIE).
 *  R21 time-to-reach Hamiltonian (Section 2.2, Algorithm 2): the control
 *     shortens and the disturbance lengthens the time, so u* = argmin_u and
 *     d* = argmax_d of pbar . f (Algorithm 2's argmin; the equation's printed
 *     min/max of -p.f would pick the opposite control), and the update's H is
 *     the static Hamiltonian Hs = -pbar . f(z, u*, d*) - 1, whose zero is the
 *     TTR equation; Algorithm 2's printed "H_i <- pbar . zdot" drops its sign
 *     and constant (taken literally, a node next to the target never leaves
 *     the initial large value).  sigma_d = |f_d(z, u*, d*)| per axis and
 *     c = 1 / sum_d(sigma_d / dz_d), the multi-axis form of c = dz / sigma;
 *     a node with sum_d(sigma_d / dz_d) = 0 keeps its value.
 *  R22 sweep loop: repeat while max|phi - phi_old| > eps (the printed "<" is
 *     inverted), the change taken over every node after the boundary update;
 *     a sweep cap ends a loop that has not converged.
 *  R23 boundary nodes (first and last node of a non-periodic axis) are not
 *     swept; after the interior pass each non-periodic axis in turn (lower
 *     face, then upper face) sets phi_b <- min(max(2 phi_{b+1} - phi_{b+2},
 *     phi_{b+2}), phi_b) along that axis with the current values, so edges
 *     and corners see the faces of earlier axes.  Periodic axes wrap and have
 *     no boundary.  Every axis needs at least 4 nodes.
 *  R24 Gauss-Seidel order with alternating directions (Section 5.3): sweep k
 *     visits the nodes in nested C-order loops, axis d descending when bit d
 *     of k mod 2^ndim is set, updating phi in place.
 *  R25 Jacobi variant (Section 5.1: parallel updates may need more sweeps):
 *     every interior node of a sweep is computed from the previous sweep's
 *     values; the boundary update is that of R23.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OG_MAXD 8

/* dynamics ids (this library's own numbering) */
enum { OG_SINGLE_INT = 0, OG_DUBINS3D = 1, OG_DUBINSCAR4D = 2, OG_REL6D = 3, OG_ADVECTION = 4,
       OG_CAPTURE = 5 };
enum { OG_MIN = 0, OG_MAX = 1 };
enum { OG_BRS = 0, OG_BRT = 1 };

/* return codes */
enum { OG_OK = 0, OG_EINVAL = -1, OG_ENOMEM = -2, OG_ETIMEOUT = -5, OG_ENUMERIC = -6 };

typedef struct {
    int ndim;
    int64_t n[OG_MAXD];
    double lo[OG_MAXD], hi[OG_MAXD], dz[OG_MAXD];
    int periodic[OG_MAXD];
    int64_t stride[OG_MAXD];
    int64_t total;
} og_grid;

typedef struct {
    int kind;
    int ndim;
    double prm[OG_MAXD];
    int umode, dmode;
} og_dyn;

/* ------------------------------------------------------------------------- */
/* Grid (Section 3.1.1): node counts, bounds, periodic axes.                  */
/* Node i sits at lo + i*dz; dz = (hi-lo)/(n-1), or (hi-lo)/n when periodic.  */
/* ------------------------------------------------------------------------- */
static int og_grid_init(og_grid *g, int ndim, const int64_t *n, const double *lo,
                        const double *hi, const int *periodic)
{
    if (ndim < 1 || ndim > OG_MAXD) return OG_EINVAL;
    g->ndim = ndim;
    for (int d = 0; d < ndim; ++d) {
        if (periodic[d] ? n[d] < 1 : n[d] < 2) return OG_EINVAL;
        if (!(hi[d] > lo[d])) return OG_EINVAL;
        g->n[d] = n[d];
        g->lo[d] = lo[d];
        g->hi[d] = hi[d];
        g->periodic[d] = periodic[d] ? 1 : 0;
        g->dz[d] = periodic[d] ? (hi[d] - lo[d]) / (double)n[d]
                               : (hi[d] - lo[d]) / (double)(n[d] - 1);
    }
    g->total = 1;
    for (int d = ndim - 1; d >= 0; --d) {   /* C order: last axis fastest */
        g->stride[d] = g->total;
        g->total *= n[d];
    }
    return OG_OK;
}

static void og_unflatten(const og_grid *g, int64_t flat, int64_t *idx)
{
    for (int d = 0; d < g->ndim; ++d) {
        idx[d] = flat / g->stride[d];
        flat -= idx[d] * g->stride[d];
    }
}

static void og_state(const og_grid *g, const int64_t *idx, double *z)
{
    for (int d = 0; d < g->ndim; ++d) z[d] = g->lo[d] + (double)idx[d] * g->dz[d];
}

/* phi at the node `off` cells away from idx along axis d, with the periodic
 * wrap or the sign-keeping ghost extrapolation of Section 3.1.1 (reading R9). */
static double og_shifted(const og_grid *g, const double *phi, const int64_t *idx,
                         int64_t flat, int d, int off)
{
    int64_t n = g->n[d];
    int64_t j = idx[d] + off;
    int64_t row = flat - idx[d] * g->stride[d];
    if (g->periodic[d]) {
        j = ((j % n) + n) % n;
        return phi[row + j * g->stride[d]];
    }
    if (j >= 0 && j < n) return phi[row + j * g->stride[d]];
    int64_t b = (j < 0) ? 0 : n - 1;          /* boundary node            */
    int64_t in = (j < 0) ? 1 : n - 2;         /* its inner neighbour      */
    double k = (j < 0) ? (double)(-j) : (double)(j - (n - 1));   /* cells outside */
    double pb = phi[row + b * g->stride[d]];
    double pin = phi[row + in * g->stride[d]];
    double sgn = (pb >= 0.0) ? 1.0 : -1.0;
    return pb + k * sgn * fabs(pb - pin);
}

/* Tie margin of the ENO2 stencil choice (reading R10): the two candidate
 * second differences count as equal in magnitude when their magnitudes differ
 * by at most OG_ENO_TIE times the sum of the magnitudes of the five window
 * values.  On data whose candidates are equal in exact arithmetic (mirror
 * symmetric windows, linear pieces) double rounding leaves differences some
 * 2^-50 of that sum; 2^-40 is far above that noise and far below any
 * difference the method resolves. */
#define OG_ENO_TIE 9.094947017729282e-13   /* 2^-40 */

/* One-sided derivatives p-, p+ along axis d at a node (Section 3.1.4 and
 * Algorithm 1: first-order upwind differences, or second-order ENO, R10).
 *
 * ENO2: with the second differences D2_j = (phi_{j+1} - 2 phi_j + phi_{j-1})
 * / h^2 at j = i-1, i, i+1,
 *   p- = D-phi + (h/2) c,   c  = D2_{i-1} if |D2_{i-1}| < |D2_i|, else D2_i,
 *   p+ = D+phi - (h/2) c',  c' = D2_{i+1} if |D2_{i+1}| < |D2_i|, else D2_i,
 * where "<" means smaller by more than the tie margin above, so that equal
 * magnitudes (a tie) keep the centred D2_i. */
static void og_one_sided(const og_grid *g, const double *phi, const int64_t *idx,
                         int64_t flat, int d, int order, double *pm, double *pp)
{
    double h = g->dz[d];
    double f0 = phi[flat];
    double fm1 = og_shifted(g, phi, idx, flat, d, -1);
    double fp1 = og_shifted(g, phi, idx, flat, d, +1);
    double dm = (f0 - fm1) / h;   /* backward difference D-phi */
    double dp = (fp1 - f0) / h;   /* forward difference  D+phi */
    if (order == 1) {
        *pm = dm;
        *pp = dp;
        return;
    }
    double fm2 = og_shifted(g, phi, idx, flat, d, -2);
    double fp2 = og_shifted(g, phi, idx, flat, d, +2);
    /* second differences in value units (h^2 D2) */
    double s_left = f0 - 2.0 * fm1 + fm2;     /* at i-1 */
    double s_mid = fp1 - 2.0 * f0 + fm1;      /* at i   */
    double s_right = fp2 - 2.0 * fp1 + f0;    /* at i+1 */
    double margin = OG_ENO_TIE * (fabs(fm2) + fabs(fm1) + fabs(f0) + fabs(fp1) + fabs(fp2));
    double c_minus = (fabs(s_left) < fabs(s_mid) - margin) ? s_left : s_mid;
    double c_plus = (fabs(s_right) < fabs(s_mid) - margin) ? s_right : s_mid;
    *pm = dm + 0.5 * c_minus / h;
    *pp = dp - 0.5 * c_plus / h;
}

/* ------------------------------------------------------------------------- */
/* Dynamics plug-ins (Section 4.2: opt_ctrl, opt_dstb, dynamics).             */
/* ------------------------------------------------------------------------- */

static int og_n_ctrl(const og_dyn *dy)
{
    switch (dy->kind) {
    case OG_SINGLE_INT: return dy->ndim;
    case OG_DUBINS3D: return 1;
    case OG_DUBINSCAR4D: return 2;
    case OG_REL6D: return 2;
    case OG_CAPTURE: return 1;
    default: return 0;
    }
}

static int og_n_dstb(const og_dyn *dy)
{
    return dy->kind == OG_REL6D ? 2 : (dy->kind == OG_CAPTURE ? 1 : 0);
}

static double og_ctrl_bound(const og_dyn *dy, int k)
{
    switch (dy->kind) {
    case OG_SINGLE_INT: return dy->prm[0];          /* |u_i| <= u_max            */
    case OG_DUBINS3D: return dy->prm[1];            /* |w| <= w_max              */
    case OG_DUBINSCAR4D: return dy->prm[k];         /* |a| <= a_max, |w| <= w_max */
    case OG_REL6D: return dy->prm[k];               /* |a_p|, |alpha_p|          */
    case OG_CAPTURE: return dy->prm[1];             /* |a| <= A (evader turn)    */
    default: return 0.0;
    }
}

static double og_dstb_bound(const og_dyn *dy, int k)
{
    if (dy->kind == OG_REL6D) return dy->prm[2 + k];   /* |a_e|, |w_e|              */
    if (dy->kind == OG_CAPTURE) return dy->prm[2];     /* |b| <= B (pursuer turn)   */
    return 0.0;
}

/* f(z, u, d) of each model (Appendix; Rel6D is the repository's 6-D
 * relative model built from the 3D pursuit-evasion and 5D Dubins equations). */
static void og_dynamics(const og_dyn *dy, const double *z, const double *u,
                        const double *dd, double *f)
{
    switch (dy->kind) {
    case OG_SINGLE_INT:
        for (int i = 0; i < dy->ndim; ++i) f[i] = u[i];
        break;
    case OG_ADVECTION:
        for (int i = 0; i < dy->ndim; ++i) f[i] = dy->prm[i];
        break;
    case OG_DUBINS3D: {           /* (x, y, th): v cos th, v sin th, w */
        double v = dy->prm[0];
        f[0] = v * cos(z[2]);
        f[1] = v * sin(z[2]);
        f[2] = u[0];
        break;
    }
    case OG_DUBINSCAR4D: {        /* (x, y, v, th): v cos th, v sin th, a, w */
        f[0] = z[2] * cos(z[3]);
        f[1] = z[2] * sin(z[3]);
        f[2] = u[0];
        f[3] = u[1];
        break;
    }
    case OG_REL6D: {              /* (x, y, th, v_p, w_p, v_e) */
        double x = z[0], y = z[1], th = z[2], vp = z[3], wp = z[4], ve = z[5];
        f[0] = -vp + ve * cos(th) + wp * y;
        f[1] = ve * sin(th) - wp * x;
        f[2] = dd[1] - wp;        /* evader turn rate w_e minus pursuer w_p */
        f[3] = u[0];              /* pursuer acceleration a_p               */
        f[4] = u[1];              /* pursuer angular acceleration alpha_p   */
        f[5] = dd[0];             /* evader acceleration a_e                */
        break;
    }
    case OG_CAPTURE: {            /* Section 4.2 pursuit-evasion, (x, y, th) relative */
        double v = dy->prm[0], x = z[0], y = z[1], th = z[2];
        f[0] = -v + v * cos(th) + u[0] * y;
        f[1] = v * sin(th) - u[0] * x;
        f[2] = dd[0] - u[0];      /* pursuer turn b minus evader turn a */
        break;
    }
    default:
        for (int i = 0; i < dy->ndim; ++i) f[i] = 0.0;
    }
}

/* Switching-function coefficients of input k: g = f(z, e_k, 0) - f(z, 0, 0),
 * exact for the input-affine models above. */
static void og_input_column(const og_dyn *dy, const double *z, int is_dstb, int k, double *g)
{
    double u0[OG_MAXD] = {0}, d0[OG_MAXD] = {0}, f0[OG_MAXD], f1[OG_MAXD];
    og_dynamics(dy, z, u0, d0, f0);
    if (is_dstb) d0[k] = 1.0; else u0[k] = 1.0;
    og_dynamics(dy, z, u0, d0, f1);
    for (int i = 0; i < dy->ndim; ++i) g[i] = f1[i] - f0[i];
}

/* Bang-bang choice for one input from its switching function s (R4). */
static double og_bang(double s, double bound, int mode)
{
    if (mode == OG_MAX) return (s >= 0.0) ? bound : -bound;
    return (s >= 0.0) ? -bound : bound;
}

/* Optimal control and disturbance (Algorithm 1, the argmin_d argmax_u step). */
static void og_opt_inputs(const og_dyn *dy, const double *z, const double *p,
                          double *u, double *dd)
{
    double g[OG_MAXD];
    for (int k = 0; k < og_n_ctrl(dy); ++k) {
        og_input_column(dy, z, 0, k, g);
        double s = 0.0;
        for (int i = 0; i < dy->ndim; ++i) s += p[i] * g[i];
        u[k] = og_bang(s, og_ctrl_bound(dy, k), dy->umode);
    }
    for (int k = 0; k < og_n_dstb(dy); ++k) {
        og_input_column(dy, z, 1, k, g);
        double s = 0.0;
        for (int i = 0; i < dy->ndim; ++i) s += p[i] * g[i];
        dd[k] = og_bang(s, og_dstb_bound(dy, k), dy->dmode);
    }
}

/* H_i = pbar . f(z_i, u_opt, d_opt)  (Algorithm 1). */
static double og_hamiltonian(const og_dyn *dy, const double *z, const double *pbar)
{
    double u[OG_MAXD] = {0}, dd[OG_MAXD] = {0}, f[OG_MAXD];
    og_opt_inputs(dy, z, pbar, u, dd);
    og_dynamics(dy, z, u, dd, f);
    double h = 0.0;
    for (int i = 0; i < dy->ndim; ++i) h += pbar[i] * f[i];
    return h;
}

/* Local dissipation bound a_d(z) (reading R5): the largest |f_d| over every
 * combination of input extremes that the derivative box [pmin, pmax] admits. */
static void og_local_alpha(const og_dyn *dy, const double *z, const double *pmin,
                           const double *pmax, double *a)
{
    int nu = og_n_ctrl(dy), nd = og_n_dstb(dy), ni = nu + nd;
    double choice[2 * OG_MAXD][2];
    int count[2 * OG_MAXD];
    double g[OG_MAXD];
    for (int k = 0; k < ni; ++k) {
        int is_d = (k >= nu);
        int kk = is_d ? k - nu : k;
        og_input_column(dy, z, is_d, kk, g);
        /* interval of the switching function s = p . g over the box */
        double slo = 0.0, shi = 0.0;
        for (int i = 0; i < dy->ndim; ++i) {
            if (g[i] >= 0.0) { slo += g[i] * pmin[i]; shi += g[i] * pmax[i]; }
            else             { slo += g[i] * pmax[i]; shi += g[i] * pmin[i]; }
        }
        double bound = is_d ? og_dstb_bound(dy, kk) : og_ctrl_bound(dy, kk);
        int mode = is_d ? dy->dmode : dy->umode;
        if (slo > 0.0) { choice[k][0] = og_bang(1.0, bound, mode); count[k] = 1; }
        else if (shi < 0.0) { choice[k][0] = og_bang(-1.0, bound, mode); count[k] = 1; }
        else { choice[k][0] = -bound; choice[k][1] = bound; count[k] = 2; }
    }
    for (int i = 0; i < dy->ndim; ++i) a[i] = 0.0;
    int combos = 1;
    for (int k = 0; k < ni; ++k) combos *= count[k];
    for (int c = 0; c < combos; ++c) {
        double u[OG_MAXD] = {0}, dd[OG_MAXD] = {0}, f[OG_MAXD];
        int rest = c;
        for (int k = 0; k < ni; ++k) {
            double val = choice[k][rest % count[k]];
            rest /= count[k];
            if (k < nu) u[k] = val; else dd[k - nu] = val;
        }
        og_dynamics(dy, z, u, dd, f);
        for (int i = 0; i < dy->ndim; ++i)
            if (fabs(f[i]) > a[i]) a[i] = fabs(f[i]);
    }
}

/* ------------------------------------------------------------------------- */
/* The two per-point passes of Algorithm 1.                                   */
/* ------------------------------------------------------------------------- */

/* First pass: alpha^max over the grid (global-alpha approximation of
 * Section 2.1, reading R5). */
static void og_alpha(const og_grid *g, const og_dyn *dy, const double *phi, int order,
                     double *alpha)
{
    int nd = g->ndim;
    double amax[OG_MAXD];
    for (int d = 0; d < OG_MAXD; ++d) amax[d] = 0.0;
#pragma omp parallel
    {
        double loc[OG_MAXD];
        for (int d = 0; d < OG_MAXD; ++d) loc[d] = 0.0;
#pragma omp for schedule(static)
        for (int64_t i = 0; i < g->total; ++i) {
            int64_t idx[OG_MAXD];
            double z[OG_MAXD], pm[OG_MAXD], pp[OG_MAXD], lo[OG_MAXD], hi[OG_MAXD], a[OG_MAXD];
            og_unflatten(g, i, idx);
            og_state(g, idx, z);
            for (int d = 0; d < nd; ++d) {
                og_one_sided(g, phi, idx, i, d, order, &pm[d], &pp[d]);
                lo[d] = fmin(pm[d], pp[d]);
                hi[d] = fmax(pm[d], pp[d]);
            }
            og_local_alpha(dy, z, lo, hi, a);
            for (int d = 0; d < nd; ++d)
                if (a[d] > loc[d]) loc[d] = a[d];
        }
#pragma omp critical
        for (int d = 0; d < nd; ++d)
            if (loc[d] > amax[d]) amax[d] = loc[d];
    }
    for (int d = 0; d < nd; ++d) alpha[d] = amax[d];
}

/* Second pass: the Lax-Friedrichs right-hand side at every node,
 * L = H(pbar) + 1/2 sum_d alpha_d (p+_d - p-_d)  (Algorithm 1, reading R2),
 * with the grid alpha, or with the node's own alpha_i when local is set
 * (reading R18). */
static void og_rhs(const og_grid *g, const og_dyn *dy, const double *phi, int order,
                   const double *alpha, int local, double *L)
{
    int nd = g->ndim;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < g->total; ++i) {
        int64_t idx[OG_MAXD];
        double z[OG_MAXD], pm[OG_MAXD], pp[OG_MAXD], pbar[OG_MAXD];
        og_unflatten(g, i, idx);
        og_state(g, idx, z);
        for (int d = 0; d < nd; ++d) {
            og_one_sided(g, phi, idx, i, d, order, &pm[d], &pp[d]);
            pbar[d] = 0.5 * (pp[d] + pm[d]);
        }
        double h = og_hamiltonian(dy, z, pbar);
        double a_loc[OG_MAXD];
        if (local) {
            double lo[OG_MAXD], hi[OG_MAXD];
            for (int d = 0; d < nd; ++d) {
                lo[d] = fmin(pm[d], pp[d]);
                hi[d] = fmax(pm[d], pp[d]);
            }
            og_local_alpha(dy, z, lo, hi, a_loc);
        }
        double diss = 0.0;
        for (int d = 0; d < nd; ++d) diss += 0.5 * (local ? a_loc[d] : alpha[d]) * (pp[d] - pm[d]);
        L[i] = h + diss;
    }
}

/* CFL step of Algorithm 1: (sum_d alpha_d / dz_d)^-1 scaled by cfl. */
static double og_cfl_dt(const og_grid *g, const double *alpha, double cfl)
{
    double s = 0.0;
    for (int d = 0; d < g->ndim; ++d) s += alpha[d] / g->dz[d];
    if (s <= 0.0) return INFINITY;
    return cfl / s;
}

static int og_setup(og_grid *g, og_dyn *dy, int ndim, const int64_t *n, const double *lo,
                    const double *hi, const int *periodic, int kind, const double *prm,
                    int n_prm, int umode, int dmode)
{
    int rc = og_grid_init(g, ndim, n, lo, hi, periodic);
    if (rc) return rc;
    memset(dy, 0, sizeof(*dy));
    dy->kind = kind;
    dy->ndim = ndim;
    dy->umode = umode;
    dy->dmode = dmode;
    int need;
    switch (kind) {
    case OG_SINGLE_INT: need = 1; break;
    case OG_DUBINS3D: need = 2; if (ndim != 3) return OG_EINVAL; break;
    case OG_DUBINSCAR4D: need = 2; if (ndim != 4) return OG_EINVAL; break;
    case OG_REL6D: need = 4; if (ndim != 6) return OG_EINVAL; break;
    case OG_CAPTURE: need = 3; if (ndim != 3) return OG_EINVAL; break;
    case OG_ADVECTION: need = ndim; break;
    default: return OG_EINVAL;
    }
    if (n_prm < need || n_prm > OG_MAXD) return OG_EINVAL;
    for (int k = 0; k < n_prm; ++k) dy->prm[k] = prm[k];
    return OG_OK;
}

/* ------------------------------------------------------------------------- */
/* Exported entry points                                                      */
/* ------------------------------------------------------------------------- */

int og_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void og_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* Node spacing of every axis. */
int og_spacing(int ndim, const int64_t *n, const double *lo, const double *hi,
               const int *periodic, double *dz_out)
{
    og_grid g;
    int rc = og_grid_init(&g, ndim, n, lo, hi, periodic);
    if (rc) return rc;
    for (int d = 0; d < ndim; ++d) dz_out[d] = g.dz[d];
    return OG_OK;
}

/* f(z, u, d) for one state (used by brute-force checks). */
int og_eval_dynamics(int kind, int ndim, const double *prm, int n_prm, const double *z,
                     const double *u, const double *dd, double *f)
{
    og_dyn dy;
    memset(&dy, 0, sizeof(dy));
    dy.kind = kind;
    dy.ndim = ndim;
    for (int k = 0; k < n_prm && k < OG_MAXD; ++k) dy.prm[k] = prm[k];
    og_dynamics(&dy, z, u, dd, f);
    return OG_OK;
}

/* f(z_j, u_j, d_j) for `count` independent triples (inputs padded to 8). */
int og_eval_dynamics_batch(int kind, int ndim, const double *prm, int n_prm, int64_t count,
                           const double *z, const double *u, const double *dd, double *f)
{
    og_dyn dy;
    memset(&dy, 0, sizeof(dy));
    dy.kind = kind;
    dy.ndim = ndim;
    for (int k = 0; k < n_prm && k < OG_MAXD; ++k) dy.prm[k] = prm[k];
    for (int64_t j = 0; j < count; ++j)
        og_dynamics(&dy, z + j * ndim, u + j * OG_MAXD, dd + j * OG_MAXD, f + j * ndim);
    return OG_OK;
}

/* Per-node terms of one Algorithm 1 evaluation on a given phi:
 * p- and p+ (ndim each, node-major), pbar, the optimal inputs, H, the local
 * dissipation bound a_d(z), and the full right-hand side L with the given
 * alpha (or the grid alpha when alpha_in is NULL).  Any output may be NULL. */
int og_terms(int ndim, const int64_t *n, const double *lo, const double *hi,
             const int *periodic, int kind, const double *prm, int n_prm, int umode,
             int dmode, int order, const double *phi, const double *alpha_in,
             double *pm_out, double *pp_out, double *u_out, double *d_out,
             double *h_out, double *a_out, double *alpha_out, double *rhs_out)
{
    og_grid g;
    og_dyn dy;
    int rc = og_setup(&g, &dy, ndim, n, lo, hi, periodic, kind, prm, n_prm, umode, dmode);
    if (rc) return rc;
    if (order != 1 && order != 2) return OG_EINVAL;
    int nu = og_n_ctrl(&dy), ndst = og_n_dstb(&dy);
    double alpha[OG_MAXD];
    og_alpha(&g, &dy, phi, order, alpha);
    if (alpha_out)
        for (int d = 0; d < ndim; ++d) alpha_out[d] = alpha[d];
    if (alpha_in)
        for (int d = 0; d < ndim; ++d) alpha[d] = alpha_in[d];
    for (int64_t i = 0; i < g.total; ++i) {
        int64_t idx[OG_MAXD];
        double z[OG_MAXD], pm[OG_MAXD], pp[OG_MAXD], pbar[OG_MAXD];
        double lo_b[OG_MAXD], hi_b[OG_MAXD], a[OG_MAXD];
        double u[OG_MAXD] = {0}, dd[OG_MAXD] = {0};
        og_unflatten(&g, i, idx);
        og_state(&g, idx, z);
        for (int d = 0; d < ndim; ++d) {
            og_one_sided(&g, phi, idx, i, d, order, &pm[d], &pp[d]);
            pbar[d] = 0.5 * (pp[d] + pm[d]);
            lo_b[d] = fmin(pm[d], pp[d]);
            hi_b[d] = fmax(pm[d], pp[d]);
        }
        og_opt_inputs(&dy, z, pbar, u, dd);
        og_local_alpha(&dy, z, lo_b, hi_b, a);
        double h = og_hamiltonian(&dy, z, pbar);
        for (int d = 0; d < ndim; ++d) {
            if (pm_out) pm_out[i * ndim + d] = pm[d];
            if (pp_out) pp_out[i * ndim + d] = pp[d];
            if (a_out) a_out[i * ndim + d] = a[d];
        }
        for (int k = 0; k < nu; ++k)
            if (u_out) u_out[i * OG_MAXD + k] = u[k];
        for (int k = 0; k < ndst; ++k)
            if (d_out) d_out[i * OG_MAXD + k] = dd[k];
        if (h_out) h_out[i] = h;
        if (rhs_out) {
            double diss = 0.0;
            for (int d = 0; d < ndim; ++d) diss += 0.5 * alpha[d] * (pp[d] - pm[d]);
            rhs_out[i] = h + diss;
        }
    }
    return OG_OK;
}

/* One full time step of size dt from phi (Algorithm 1 update with the
 * Euler or TVD-RK2 integrator of Section 3.1.3, the BRS / BRT post-step and
 * the obstacle max when obst is not NULL), as taken inside og_solve.  out may not alias phi.  alpha_out (ndim) gets the
 * stage-1 alpha (the one the CFL step is computed from). */
int og_step(int ndim, const int64_t *n, const double *lo, const double *hi, const int *periodic,
            int kind, const double *prm, int n_prm, int umode, int dmode, const double *l,
            const double *obst, const double *phi, double dt, int set_kind, int space_order,
            int time_order, int local_alpha, double *out, double *alpha_out)
{
    og_grid g;
    og_dyn dy;
    int rc = og_setup(&g, &dy, ndim, n, lo, hi, periodic, kind, prm, n_prm, umode, dmode);
    if (rc) return rc;
    if (space_order != 1 && space_order != 2) return OG_EINVAL;
    if (time_order != 1 && time_order != 2) return OG_EINVAL;
    int64_t N = g.total;
    double *L = malloc(sizeof(double) * N);
    double *phi1 = (time_order == 2) ? malloc(sizeof(double) * N) : NULL;
    if (!L || (time_order == 2 && !phi1)) { free(L); free(phi1); return OG_ENOMEM; }
    double alpha[OG_MAXD] = {0};
    og_alpha(&g, &dy, phi, space_order, alpha);
    if (alpha_out)
        for (int d = 0; d < ndim; ++d) alpha_out[d] = alpha[d];
    og_rhs(&g, &dy, phi, space_order, alpha, local_alpha, L);
    if (time_order == 1) {
        for (int64_t i = 0; i < N; ++i) out[i] = phi[i] + dt * L[i];
    } else {
        for (int64_t i = 0; i < N; ++i) phi1[i] = phi[i] + dt * L[i];
        og_alpha(&g, &dy, phi1, space_order, alpha);
        og_rhs(&g, &dy, phi1, space_order, alpha, local_alpha, L);
        for (int64_t i = 0; i < N; ++i) out[i] = 0.5 * (phi[i] + (phi1[i] + dt * L[i]));
    }
    if (set_kind == OG_BRT)
        for (int64_t i = 0; i < N; ++i)
            if (l[i] < out[i]) out[i] = l[i];
    if (obst)
        for (int64_t i = 0; i < N; ++i)
            if (obst[i] > out[i]) out[i] = obst[i];
    free(L);
    free(phi1);
    return OG_OK;
}

/* Full solve (Algorithm 1 with the BRS / BRT post-step of Section 4.3).
 *  l           target l(z), total nodes
 *  phi0        NULL: phi(z, 0) = l(z); else the value to start from (resuming a
 *              solve at a kept tau: the schedule then counts from that tau)
 *  tau         n_tau look-back times, tau[0] = 0, strictly increasing
 *  set_kind    OG_BRS (plain PDE) or OG_BRT (phi <- min(phi, l) after each step,
 *              the HJ variational inequality)
 *  obst        NULL, or the obstacle g(z): phi <- max(phi, g) after each step,
 *              after the BRT min (reach-avoid, reading R17)
 *  local_alpha 0: dissipation with the grid alpha (Section 2.1); 1: with each
 *              node's own alpha_i (Algorithm 1's second loop, reading R18)
 *  snapshots   NULL, or n_tau * total doubles: phi at every tau
 *  final_out   total doubles: phi at tau[n_tau-1]
 *  steps_out   NULL or n_tau-1 step counts, one per segment
 *  alpha_out   NULL or ndim doubles: alpha of the last stage
 *  last_dt     NULL or the last step's dt
 */
/* Post-step operations (the computation methods of Section 4.3, reading
 * R27).  Target side, applied first: */
enum { OG_T_NONE = 0,        /* plain PDE (BRS)                                  */
       OG_T_MIN_TARGET = 1,  /* minVWithVTarget: min with the target (BRT)       */
       OG_T_MAX_TARGET = 2,  /* maxVWithVTarget                                  */
       OG_T_MIN_INIT = 3,    /* minVWithVInit: min with the value before the step */
       OG_T_MAX_INIT = 4,    /* maxVWithVInit                                    */
       OG_T_MIN_V0 = 5,      /* minVWithV0: min with the initial value phi(0)    */
       OG_T_MAX_V0 = 6 };    /* maxVWithV0                                       */
/* obstacle side, applied after the target side: */
enum { OG_O_MAX = 1,         /* maxVWithObstacle                                 */
       OG_O_MIN = 2 };       /* minVWithObstacle                                 */

static int og_solve_impl(int ndim, const int64_t *n, const double *lo, const double *hi,
                         const int *periodic, int kind, const double *prm, int n_prm, int umode,
                         int dmode, const double *l, const double *obst, const double *l_seq,
                         const double *g_seq, const double *phi0, const double *tau, int n_tau,
                         int set_kind, int obst_mode, int space_order, int time_order, int local_alpha,
                         double cfl, int64_t max_steps, double *snapshots, double *final_out,
                         int64_t *steps_out, double *alpha_out, double *last_dt)
{
    og_grid g;
    og_dyn dy;
    int rc = og_setup(&g, &dy, ndim, n, lo, hi, periodic, kind, prm, n_prm, umode, dmode);
    if (rc) return rc;
    if (n_tau < 2 || tau[0] != 0.0) return OG_EINVAL;
    for (int k = 1; k < n_tau; ++k)
        if (!(tau[k] > tau[k - 1])) return OG_EINVAL;
    if (space_order != 1 && space_order != 2) return OG_EINVAL;
    if (time_order != 1 && time_order != 2) return OG_EINVAL;
    if (!(cfl > 0.0)) return OG_EINVAL;
    if (set_kind < OG_T_NONE || set_kind > OG_T_MAX_V0) return OG_EINVAL;
    if (obst_mode != OG_O_MAX && obst_mode != OG_O_MIN) return OG_EINVAL;

    int64_t N = g.total;
    double *phi = malloc(sizeof(double) * N);
    double *phi1 = malloc(sizeof(double) * N);
    double *L = malloc(sizeof(double) * N);
    double *v0 = malloc(sizeof(double) * N);
    if (!phi || !phi1 || !L || !v0) { free(phi); free(phi1); free(L); free(v0); return OG_ENOMEM; }
    memcpy(phi, phi0 ? phi0 : (l_seq ? l_seq : l), sizeof(double) * N);
    memcpy(v0, phi, sizeof(double) * N);
    if (snapshots) memcpy(snapshots, phi, sizeof(double) * N);

    double alpha[OG_MAXD] = {0}, alpha2[OG_MAXD] = {0};
    double dt = 0.0;
    int64_t total_steps = 0;
    rc = OG_OK;
    for (int k = 0; k + 1 < n_tau && rc == OG_OK; ++k) {
        double t = tau[k], t_end = tau[k + 1];
        int64_t seg_steps = 0;
        /* sets of this segment: time-varying ones at its end (reading R26) */
        const double *lk = l_seq ? l_seq + (int64_t)(k + 1) * N : l;
        const double *gk = g_seq ? g_seq + (int64_t)(k + 1) * N : obst;
        while (t_end - t > 1e-12 * t_end) {
            if (total_steps >= max_steps) { rc = OG_ETIMEOUT; break; }
            /* stage 1: alpha, dt, phi1 = phi + dt L(phi) */
            og_alpha(&g, &dy, phi, space_order, alpha);
            double dt_cfl = og_cfl_dt(&g, alpha, cfl);
            int last = !(dt_cfl < t_end - t);
            dt = last ? (t_end - t) : dt_cfl;
            og_rhs(&g, &dy, phi, space_order, alpha, local_alpha, L);
            for (int64_t i = 0; i < N; ++i) phi1[i] = phi[i] + dt * L[i];
            if (time_order == 2) {
                /* stage 2 with its own alpha; Heun average */
                og_alpha(&g, &dy, phi1, space_order, alpha2);
                og_rhs(&g, &dy, phi1, space_order, alpha2, local_alpha, L);
                for (int64_t i = 0; i < N; ++i)
                    phi1[i] = 0.5 * (phi[i] + (phi1[i] + dt * L[i]));
            }
            int bad = 0;
            for (int64_t i = 0; i < N; ++i) {
                double v = phi1[i];
                switch (set_kind) {
                case OG_T_MIN_TARGET: if (lk[i] < v) v = lk[i]; break;
                case OG_T_MAX_TARGET: if (lk[i] > v) v = lk[i]; break;
                case OG_T_MIN_INIT: if (phi[i] < v) v = phi[i]; break;   /* phi[i]: before the step */
                case OG_T_MAX_INIT: if (phi[i] > v) v = phi[i]; break;
                case OG_T_MIN_V0: if (v0[i] < v) v = v0[i]; break;
                case OG_T_MAX_V0: if (v0[i] > v) v = v0[i]; break;
                default: break;
                }
                if (gk) {
                    if (obst_mode == OG_O_MAX && gk[i] > v) v = gk[i];
                    if (obst_mode == OG_O_MIN && gk[i] < v) v = gk[i];
                }
                if (!isfinite(v)) bad = 1;
                phi[i] = v;
            }
            if (bad) { rc = OG_ENUMERIC; break; }
            t = last ? t_end : t + dt;
            ++seg_steps;
            ++total_steps;
        }
        if (steps_out) steps_out[k] = seg_steps;
        if (snapshots) memcpy(snapshots + (int64_t)(k + 1) * N, phi, sizeof(double) * N);
    }
    if (final_out) memcpy(final_out, phi, sizeof(double) * N);
    if (alpha_out)
        for (int d = 0; d < ndim; ++d) alpha_out[d] = (time_order == 2) ? alpha2[d] : alpha[d];
    if (last_dt) *last_dt = dt;
    free(phi);
    free(phi1);
    free(L);
    free(v0);
    return rc;
}

int og_solve(int ndim, const int64_t *n, const double *lo, const double *hi,
             const int *periodic, int kind, const double *prm, int n_prm, int umode,
             int dmode, const double *l, const double *obst, const double *phi0,
             const double *tau, int n_tau,
             int set_kind, int space_order, int time_order, int local_alpha, double cfl, int64_t max_steps,
             double *snapshots, double *final_out, int64_t *steps_out,
             double *alpha_out, double *last_dt)
{
    return og_solve_impl(ndim, n, lo, hi, periodic, kind, prm, n_prm, umode, dmode, l, obst, NULL, NULL, phi0,
                         tau, n_tau, set_kind, OG_O_MAX, space_order, time_order, local_alpha, cfl, max_steps,
                         snapshots, final_out, steps_out, alpha_out, last_dt);
}

/* og_solve with time-varying sets (reading R26): l_seq (target) and g_seq
 * (obstacle, or NULL) hold n_tau arrays each, the sets at tau[0..n_tau-1];
 * phi starts from l_seq[0] (or phi0) and the steps of segment k take the
 * post-step min / max with l_seq[k+1] / g_seq[k+1]. */
int og_solve_seq(int ndim, const int64_t *n, const double *lo, const double *hi,
                 const int *periodic, int kind, const double *prm, int n_prm, int umode,
                 int dmode, const double *l_seq, const double *g_seq, const double *phi0,
                 const double *tau, int n_tau,
                 int set_kind, int space_order, int time_order, int local_alpha, double cfl, int64_t max_steps,
                 double *snapshots, double *final_out, int64_t *steps_out,
                 double *alpha_out, double *last_dt)
{
    if (!l_seq) return OG_EINVAL;
    return og_solve_impl(ndim, n, lo, hi, periodic, kind, prm, n_prm, umode, dmode, l_seq, NULL, l_seq, g_seq,
                         phi0, tau, n_tau, set_kind, OG_O_MAX, space_order, time_order, local_alpha, cfl,
                         max_steps, snapshots, final_out, steps_out, alpha_out, last_dt);
}

/* og_solve with any computation method of Section 4.3 (reading R27):
 * target_mode one of OG_T_*, obst_mode OG_O_MAX or OG_O_MIN (used when an
 * obstacle, or obstacle schedule, is given); l_seq / g_seq as og_solve_seq
 * (either may be NULL; then l / obst are the sets of every segment). */
int og_solve_methods(int ndim, const int64_t *n, const double *lo, const double *hi,
                     const int *periodic, int kind, const double *prm, int n_prm, int umode,
                     int dmode, const double *l, const double *obst, const double *l_seq,
                     const double *g_seq, const double *phi0, const double *tau, int n_tau,
                     int target_mode, int obst_mode, int space_order, int time_order, int local_alpha,
                     double cfl, int64_t max_steps, double *snapshots, double *final_out,
                     int64_t *steps_out, double *alpha_out, double *last_dt)
{
    if (!l && !l_seq) return OG_EINVAL;
    return og_solve_impl(ndim, n, lo, hi, periodic, kind, prm, n_prm, umode, dmode, l ? l : l_seq, obst, l_seq,
                         g_seq, phi0, tau, n_tau, target_mode, obst_mode, space_order, time_order, local_alpha,
                         cfl, max_steps, snapshots, final_out, steps_out, alpha_out, last_dt);
}

/* ------------------------------------------------------------------------- */
/* Time-to-reach function by Lax-Friedrichs sweeping (Section 2.2, the TTR    */
/* HJ equation and Algorithm 2; alternating directions of Section 5.3).       */
/* Readings (also in the file header): R21 Hamiltonian and update, R22 the    */
/* sweep loop and its stopping test, R23 boundary nodes, R24 sweep order,     */
/* R25 the Jacobi variant.                                                    */
/* ------------------------------------------------------------------------- */
enum { OG_TTR_GAUSS_SEIDEL = 0, OG_TTR_JACOBI = 1 };

/* Node interior to every non-periodic axis: updated by the sweep itself. */
static int og_ttr_interior(const og_grid *g, const int64_t *idx)
{
    for (int d = 0; d < g->ndim; ++d)
        if (!g->periodic[d] && (idx[d] == 0 || idx[d] == g->n[d] - 1)) return 0;
    return 1;
}

/* phi of the neighbour one cell away along axis d (wrapping on a periodic
 * axis; interior nodes have both neighbours inside on the other axes). */
static double og_ttr_nb(const og_grid *g, const double *phi, const int64_t *idx, int64_t flat,
                        int d, int off)
{
    int64_t j = idx[d] + off;
    if (j < 0) j += g->n[d];
    if (j >= g->n[d]) j -= g->n[d];
    return phi[flat + (j - idx[d]) * g->stride[d]];
}

/* The Lax-Friedrichs value of one interior node (Algorithm 2, reading R21):
 *   pbar_d = (phi(i+e_d) - phi(i-e_d)) / (2 dz_d)      central derivative
 *   u*, d* = argmin_u, argmax_d pbar . f(z, u, d)       optimal inputs
 *   Hs     = -pbar . f(z, u*, d*) - 1                   static Hamiltonian
 *   sigma_d = |dHs/dp_d| = |f_d(z, u*, d*)|
 *   phi_new = (-Hs + sum_d sigma_d (phi(i+e_d) + phi(i-e_d)) / (2 dz_d))
 *             / sum_d (sigma_d / dz_d)
 * A node whose sum_d sigma_d / dz_d is 0 keeps its value. */
static double og_ttr_value(const og_grid *g, const og_dyn *dy, const double *phi,
                           const int64_t *idx, int64_t flat)
{
    int nd = g->ndim;
    double z[OG_MAXD], p[OG_MAXD], up[OG_MAXD], dn[OG_MAXD];
    og_state(g, idx, z);
    for (int d = 0; d < nd; ++d) {
        up[d] = og_ttr_nb(g, phi, idx, flat, d, +1);
        dn[d] = og_ttr_nb(g, phi, idx, flat, d, -1);
        p[d] = (up[d] - dn[d]) / (2.0 * g->dz[d]);
    }
    double u[OG_MAXD] = {0}, dd[OG_MAXD] = {0}, f[OG_MAXD];
    og_opt_inputs(dy, z, p, u, dd);
    og_dynamics(dy, z, u, dd, f);
    double pf = 0.0;
    for (int d = 0; d < nd; ++d) pf += p[d] * f[d];
    double Hs = -pf - 1.0;
    double denom = 0.0, avg = 0.0;
    for (int d = 0; d < nd; ++d) {
        double sigma = fabs(f[d]);
        denom += sigma / g->dz[d];
        avg += sigma * (up[d] + dn[d]) / (2.0 * g->dz[d]);
    }
    if (denom == 0.0) return phi[flat];
    return (-Hs + avg) / denom;
}

/* Boundary nodes after the interior pass (reading R23): for each
 * non-periodic axis in order, the lower face then the upper face,
 *   phi_b <- min(max(2 phi_{b+1} - phi_{b+2}, phi_{b+2}), phi_b)
 * along that axis with the current values. */
static void og_ttr_boundary(const og_grid *g, double *phi)
{
    int64_t idx[OG_MAXD];
    for (int d = 0; d < g->ndim; ++d) {
        if (g->periodic[d]) continue;
        int64_t n = g->n[d], s = g->stride[d];
        for (int side = 0; side < 2; ++side) {
            int64_t b = side ? n - 1 : 0;
            int64_t step = side ? -s : s;      /* toward the interior */
            for (int64_t i = 0; i < g->total; ++i) {
                og_unflatten(g, i, idx);
                if (idx[d] != b) continue;
                double p1 = phi[i + step], p2 = phi[i + 2 * step];
                double e = fmax(2.0 * p1 - p2, p2);
                phi[i] = fmin(e, phi[i]);
            }
        }
    }
}

/* Flat index of the k-th node of sweep `dirs` (reading R24): nested loops in
 * C order over y, axis d visited in descending order when bit d is set. */
static int64_t og_ttr_order(const og_grid *g, int64_t k, unsigned dirs, int64_t *idx)
{
    og_unflatten(g, k, idx);
    int64_t flat = 0;
    for (int d = 0; d < g->ndim; ++d) {
        if ((dirs >> d) & 1u) idx[d] = g->n[d] - 1 - idx[d];
        flat += idx[d] * g->stride[d];
    }
    return flat;
}

/* Algorithm 2.  l: target function (target set T = {l <= 0}), phi starts at
 * 0 on T and `big` elsewhere (Section 2.2).  Sweeps repeat while the largest
 * change of a sweep exceeds eps (reading R22), at most max_sweeps times.
 * scheme: OG_TTR_GAUSS_SEIDEL (in place, alternating directions) or
 * OG_TTR_JACOBI (every interior node from the previous sweep's values,
 * reading R25).  Returns OG_ETIMEOUT if max_sweeps ran out first. */
int og_ttr(int ndim, const int64_t *n, const double *lo, const double *hi, const int *periodic,
           int kind, const double *prm, int n_prm, int umode, int dmode, const double *l,
           double big, double eps, int64_t max_sweeps, int scheme, double *phi_out,
           int64_t *sweeps_out, double *change_out)
{
    og_grid g;
    og_dyn dy;
    int rc = og_setup(&g, &dy, ndim, n, lo, hi, periodic, kind, prm, n_prm, umode, dmode);
    if (rc) return rc;
    if (umode != OG_MIN || dmode != OG_MAX) return OG_EINVAL;
    if (scheme != OG_TTR_GAUSS_SEIDEL && scheme != OG_TTR_JACOBI) return OG_EINVAL;
    if (!(eps >= 0.0) || !(big > 0.0) || max_sweeps < 1) return OG_EINVAL;
    for (int d = 0; d < ndim; ++d)
        if (g.n[d] < 4) return OG_EINVAL;
    int64_t N = g.total;
    double *phi = phi_out;
    double *old = malloc(sizeof(double) * N);
    if (!old) return OG_ENOMEM;
    for (int64_t i = 0; i < N; ++i) phi[i] = (l[i] <= 0.0) ? 0.0 : big;

    int64_t sweeps = 0;
    double change = 0.0;
    rc = OG_ETIMEOUT;
    int64_t idx[OG_MAXD];
    while (sweeps < max_sweeps) {
        memcpy(old, phi, sizeof(double) * N);
        if (scheme == OG_TTR_GAUSS_SEIDEL) {
            unsigned dirs = (unsigned)(sweeps % ((int64_t)1 << ndim));
            for (int64_t k = 0; k < N; ++k) {
                int64_t i = og_ttr_order(&g, k, dirs, idx);
                if (!og_ttr_interior(&g, idx)) continue;
                phi[i] = fmin(og_ttr_value(&g, &dy, phi, idx, i), phi[i]);
            }
        } else {
            for (int64_t i = 0; i < N; ++i) {
                og_unflatten(&g, i, idx);
                if (!og_ttr_interior(&g, idx)) continue;
                phi[i] = fmin(og_ttr_value(&g, &dy, old, idx, i), old[i]);
            }
        }
        og_ttr_boundary(&g, phi);
        change = 0.0;
        for (int64_t i = 0; i < N; ++i) change = fmax(change, fabs(phi[i] - old[i]));
        ++sweeps;
        if (!isfinite(change)) { rc = OG_ENUMERIC; break; }
        if (!(change > eps)) { rc = OG_OK; break; }
    }
    free(old);
    if (sweeps_out) *sweeps_out = sweeps;
    if (change_out) *change_out = change;
    return rc;
}

/* The value Algorithm 2 gives one interior node from phi (reading R21), for
 * tests that enumerate sweep orders themselves. */
int og_ttr_node(int ndim, const int64_t *n, const double *lo, const double *hi, const int *periodic,
                int kind, const double *prm, int n_prm, int umode, int dmode, const double *phi,
                const int64_t *idx, double *value)
{
    og_grid g;
    og_dyn dy;
    int rc = og_setup(&g, &dy, ndim, n, lo, hi, periodic, kind, prm, n_prm, umode, dmode);
    if (rc) return rc;
    int64_t flat = 0;
    for (int d = 0; d < ndim; ++d) {
        if (idx[d] < 0 || idx[d] >= g.n[d]) return OG_EINVAL;
        flat += idx[d] * g.stride[d];
    }
    if (!og_ttr_interior(&g, idx)) return OG_EINVAL;
    *value = og_ttr_value(&g, &dy, phi, idx, flat);
    return OG_OK;
}
