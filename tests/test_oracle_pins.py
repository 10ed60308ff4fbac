"""Pins of the FP64 oracle to facts fixed outside it.

Each test checks the oracle against something it does not compute itself:
hand-derived derivative values, exactness on polynomials, brute-force
maximisation of the Hamiltonian over sampled inputs, exact transports,
closed-form value functions, convergence under refinement, the BRT
invariants and the symmetries of the Dubins car.  A plausible mistake in any
step of Algorithm 1 (a dropped term, a wrong sign, a swapped ENO choice, a
wrong ghost rule, a reversed input mode, a wrong RK2 average) fails one of
them.
"""
import dataclasses
import math
import os

import numpy as np
import pytest

import oracle
from paper_2204_05520_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def box_problem(n, lo, hi, periodic, dynamics="advection", params=None, **kw):
    nd = len(n)
    return inputs.Problem(
        name="t", n=tuple(n), lo=tuple(lo), hi=tuple(hi), periodic=tuple(periodic),
        dynamics=dynamics, params=tuple(params if params is not None else (1.0,) * nd),
        u_mode=kw.pop("u_mode", "max"), d_mode=kw.pop("d_mode", "max"),
        target=kw.pop("target", None), tau=kw.pop("tau", (0.0, 1.0)), **kw)


# ---------------------------------------------------------------------------
# derivatives and ghost cells (Section 3.1.1, Section 3.1.4, Algorithm 1)
# ---------------------------------------------------------------------------

def load_derivative_cases():
    cases = []
    with open(os.path.join(GOLDEN, "derivatives_1d.txt")) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            name, order, per, h, phi, pm, pp = [c.strip() for c in line.split("|")]
            cases.append((name, int(order), per == "1", float(h),
                          np.array(phi.split(), float), np.array(pm.split(), float),
                          np.array(pp.split(), float)))
    return cases


@pytest.mark.parametrize("case", load_derivative_cases(), ids=lambda c: c[0])
def test_hand_derived_derivatives(case):
    name, order, per, h, phi, pm, pp = case
    n = len(phi)
    hi = h * n if per else h * (n - 1)
    p = box_problem((n,), (0.0,), (hi,), (per,))
    t = oracle.terms(p, phi, order=order)
    np.testing.assert_allclose(t["pm"][:, 0], pm, rtol=0, atol=1e-12)
    np.testing.assert_allclose(t["pp"][:, 0], pp, rtol=0, atol=1e-12)


def test_upwind_exact_on_linear_functions():
    # p- = p+ = slope at every interior node of a linear function, on every
    # axis (the ghost rule keeps the boundary sign, so it need not continue the
    # slope at the boundary nodes)
    n = (7, 6, 5)
    p = box_problem(n, (-1.0, 0.0, 2.0), (2.0, 1.0, 3.0), (False,) * 3)
    dz = oracle.spacing(p.n, p.lo, p.hi, p.periodic)
    mesh = np.meshgrid(*inputs.node_coords(p.n, p.lo, p.hi, p.periodic), indexing="ij")
    slopes = (0.7, -1.3, 2.1)
    phi = 5.0 + sum(s * m for s, m in zip(slopes, mesh))
    t = oracle.terms(p, phi, order=1)
    inner = tuple(slice(1, k - 1) for k in n)
    for d, s in enumerate(slopes):
        np.testing.assert_allclose(t["pm"][..., d][inner], s, atol=1e-10)
        np.testing.assert_allclose(t["pp"][..., d][inner], s, atol=1e-10)
    assert np.allclose(dz, [3 / 6, 1 / 5, 1 / 4])


def test_eno2_exact_on_quadratics_in_the_interior():
    # second-order ENO reproduces the derivative of a quadratic exactly
    n = (9, 8, 10)
    p = box_problem(n, (-1.0, -2.0, 0.0), (1.0, 2.0, 3.0), (False,) * 3)
    z = np.meshgrid(*inputs.node_coords(p.n, p.lo, p.hi, p.periodic), indexing="ij")
    phi = 0.5 * z[0] ** 2 - 1.5 * z[1] ** 2 + 0.25 * z[2] ** 2 + z[0] * z[1] - z[2]
    grad = (z[0] + z[1], -3.0 * z[1] + z[0], 0.5 * z[2] - 1.0)
    t = oracle.terms(p, phi, order=2)
    inner = tuple(slice(2, k - 2) for k in n)
    for d in range(3):
        np.testing.assert_allclose(t["pm"][..., d][inner], grad[d][inner], atol=1e-10)
        np.testing.assert_allclose(t["pp"][..., d][inner], grad[d][inner], atol=1e-10)


def test_eno2_tie_margin():
    # Reading R10: ENO2 keeps the centred second difference when the two
    # candidates have equal magnitude in exact arithmetic.  Window at node 2
    # of the periodic array (-0.9, -0.8, -0.6, -0.5, 0.4), h = 1:
    #   second differences at 1, 2, 3: -0.6 + 1.6 - 0.9 = 0.1,
    #   -0.5 + 1.2 - 0.8 = -0.1, 0.4 + 1.0 - 0.6 = 0.8;
    #   D- = 0.2, D+ = 0.1.  |0.1| = |-0.1| is a tie, so c = c' = -0.1 and
    #   p- = 0.2 - 0.05 = 0.15, p+ = 0.1 + 0.05 = 0.15.
    # Double rounding of these decimals gives |0.0999...98| < |-0.1000...09|,
    # so a plain floating-point compare would take c = 0.1 (p- = 0.25).
    p = box_problem((5,), (0.0,), (5.0,), (True,))
    phi = np.array([-0.9, -0.8, -0.6, -0.5, 0.4])
    t = oracle.terms(p, phi, order=2)
    assert t["pm"][2, 0] == pytest.approx(0.15, abs=1e-12)
    assert t["pp"][2, 0] == pytest.approx(0.15, abs=1e-12)
    # a real difference of 1e-9 (far above the 2^-40 margin) is resolved:
    # phi_0 = -0.9 - 1e-9 makes the left difference 0.1 - 1e-9, the smaller,
    # so c = 0.1 - 1e-9 and p- = 0.2 + 0.05 - 5e-10
    phi[0] -= 1e-9
    t = oracle.terms(p, phi, order=2)
    assert t["pm"][2, 0] == pytest.approx(0.25 - 5e-10, abs=1e-12)
    assert t["pp"][2, 0] == pytest.approx(0.15, abs=1e-12)


def test_periodic_wrap_on_every_axis():
    # sin on a periodic axis: p- and p+ are the wrapped one-sided differences
    n = 12
    h = 2 * math.pi / n
    x = h * np.arange(n)
    phi = np.sin(x)
    p = box_problem((n,), (0.0,), (2 * math.pi,), (True,))
    t = oracle.terms(p, phi, order=1)
    np.testing.assert_allclose(t["pm"][:, 0], (phi - np.roll(phi, 1)) / h, atol=1e-12)
    np.testing.assert_allclose(t["pp"][:, 0], (np.roll(phi, -1) - phi) / h, atol=1e-12)


# ---------------------------------------------------------------------------
# optimal inputs and Hamiltonian against brute force (Algorithm 1)
# ---------------------------------------------------------------------------

def input_bounds(problem):
    prm = problem.params
    dyn = problem.dynamics
    if dyn == "single_integrator":
        return [prm[0]] * problem.ndim, []
    if dyn == "dubins3d":
        return [prm[1]], []
    if dyn == "dubinscar4d":
        return [prm[0], prm[1]], []
    if dyn == "rel6d":
        return [prm[0], prm[1]], [prm[2], prm[3]]
    if dyn == "dubins_capture":
        return [prm[1]], [prm[2]]
    return [], []


def brute_force_h(problem, z, pbar, samples=7):
    """ext_d ext_u pbar.f(z,u,d) over a dense sampled input set (endpoints
    included), in both orders of the two extremisations."""
    ub, db = input_bounds(problem)
    grids = [np.linspace(-b, b, samples) for b in ub + db]
    combos = np.array(np.meshgrid(*grids, indexing="ij")).reshape(len(grids), -1).T
    nu = len(ub)
    m = len(z)
    k = len(combos)
    zz = np.repeat(z, k, axis=0)
    uu = np.tile(combos[:, :nu], (m, 1))
    dd = np.tile(combos[:, nu:], (m, 1)) if db else np.zeros((m * k, 1))
    f = oracle.eval_dynamics_batch(problem.dynamics, problem.params, zz, uu, dd)
    val = np.einsum("ij,ij->i", f, np.repeat(pbar, k, axis=0))
    shape = [m] + [samples] * len(grids)
    val = val.reshape(shape)
    ext_u = np.max if problem.u_mode == "max" else np.min
    ext_d = np.max if problem.d_mode == "max" else np.min
    u_axes = tuple(range(1, 1 + nu))
    d_axes = tuple(range(1 + nu, 1 + len(grids)))
    if d_axes:
        h1 = ext_d(ext_u(val, axis=u_axes, keepdims=True), axis=d_axes).reshape(m)
        h2 = ext_u(ext_d(val, axis=d_axes, keepdims=True), axis=u_axes).reshape(m)
    else:
        h1 = h2 = ext_u(val, axis=u_axes).reshape(m)
    return h1, h2


TINY = [
    inputs.dubins3d(n=(9, 9, 8), u_mode="min"),
    inputs.dubins3d(n=(9, 9, 8), u_mode="max"),
    inputs.dubinscar4d(n=(5, 5, 4, 6), u_mode="min"),
    inputs.dubinscar4d(n=(5, 5, 4, 6), u_mode="max"),
    inputs.rel6d(n=(4, 4, 4, 3, 3, 3)),
    inputs.dubins_capture(n=(9, 9, 8)),
    inputs.dubins_capture(n=(9, 9, 8), u_mode="min", d_mode="max"),
    inputs.single_integrator((6, 5), u_mode="min"),
    inputs.single_integrator((6, 5), u_mode="max"),
]


@pytest.mark.parametrize("problem", TINY, ids=lambda p: p.name + "_" + p.u_mode)
@pytest.mark.parametrize("order", [1, 2])
def test_hamiltonian_matches_brute_force(problem, order):
    phi = inputs.random_field(problem.n, seed=7 + order)
    t = oracle.terms(problem, phi, order=order)
    nd = problem.ndim
    pbar = 0.5 * (t["pm"] + t["pp"]).reshape(-1, nd)
    z = np.stack(np.meshgrid(*problem.nodes(), indexing="ij"), axis=-1).reshape(-1, nd)
    rng = np.random.Generator(np.random.PCG64(3))
    pick = rng.choice(len(z), size=min(len(z), 120), replace=False)
    h1, h2 = brute_force_h(problem, z[pick], pbar[pick])
    h = t["H"].reshape(-1)[pick]
    scale = 1.0 + np.abs(h).max()
    np.testing.assert_allclose(h, h1, atol=1e-12 * scale)
    np.testing.assert_allclose(h, h2, atol=1e-12 * scale)


def test_tie_rule_of_the_bang_bang_choice():
    # a zero switching function picks +bound in "max" and -bound in "min" mode
    p = box_problem((5,), (-1.0,), (1.0,), (False,), dynamics="single_integrator",
                    params=(2.0,))
    phi = np.zeros(5)
    for mode, expect in (("max", 2.0), ("min", -2.0)):
        t = oracle.terms(p, phi, order=1, u_mode=mode)
        np.testing.assert_array_equal(t["u"][:, 0], expect)
        np.testing.assert_array_equal(t["H"], 0.0)


# ---------------------------------------------------------------------------
# dissipation coefficients alpha (global-alpha reading, Section 2.1)
# ---------------------------------------------------------------------------

def test_alpha_closed_forms_dubins():
    p = inputs.dubins3d(n=(41, 41, 36), v=1.3, w_max=0.7)
    t = oracle.terms(p, p.target_values())
    th = inputs.node_coords(p.n, p.lo, p.hi, p.periodic)[2]
    expect = [1.3 * np.abs(np.cos(th)).max(), 1.3 * np.abs(np.sin(th)).max(), 0.7]
    np.testing.assert_allclose(t["alpha"], expect, rtol=1e-15)
    np.testing.assert_allclose(t["alpha"], [1.3, 1.3, 0.7], rtol=1e-15)

    p4 = inputs.dubinscar4d(n=(9, 9, 7, 10), a_max=0.6, w_max=1.1)
    t4 = oracle.terms(p4, p4.target_values())
    th4 = inputs.node_coords(p4.n, p4.lo, p4.hi, p4.periodic)[3]
    np.testing.assert_allclose(
        t4["alpha"], [3.0 * np.abs(np.cos(th4)).max(), 3.0 * np.abs(np.sin(th4)).max(), 0.6, 1.1],
        rtol=1e-15)


def test_alpha_rel6d_closed_form_and_theta_rule():
    # 24 nodes per axis: x, y span [-4, 4]; theta hits -pi/2; v in [0.5, 1.5]
    p = inputs.rel6d(n=(24, 6, 24, 3, 3, 3))
    p.lo = (-4.0, -4.0, -math.pi, 0.5, -1.0, 0.5)
    phi = inputs.random_field(p.n, seed=11)
    t = oracle.terms(p, phi, order=1)
    a = t["alpha"]
    assert a[0] == pytest.approx(1.5 + 1.5 + 4.0, abs=1e-12)
    assert a[1] == pytest.approx(1.5 + 4.0, abs=1e-12)
    assert a[3] == a[4] == a[5] == 1.0
    # theta: evader picks w_e = +1 when p_theta >= 0 ("max" mode); a point whose
    # p_theta interval straddles 0 can select both, so a_theta = 1 + |w_p|
    wp = np.meshgrid(*p.nodes(), indexing="ij")[4]
    lo = np.minimum(t["pm"][..., 2], t["pp"][..., 2])
    hi = np.maximum(t["pm"][..., 2], t["pp"][..., 2])
    a_th = np.where(lo > 0, np.abs(1.0 - wp), np.where(hi < 0, np.abs(-1.0 - wp), 1.0 + np.abs(wp)))
    np.testing.assert_allclose(t["a"][..., 2], a_th, atol=1e-15)
    assert a[2] == pytest.approx(a_th.max(), abs=1e-15)


def test_alpha_rel6d_with_unequal_input_bounds():
    # bounds (a_p, alpha_p, a_e, w_e) = (0.7, 0.4, 0.3, 1.2), all different, so
    # each input must drive its own axis (reading R12):
    #   v_p' = a_p -> alpha = 0.7;  w_p' = alpha_p -> 0.4;  v_e' = a_e -> 0.3;
    #   th' = w_e - w_p -> with both signs of p_th somewhere, 1.2 + max|w_p| = 2.2;
    #   x' = -v_p + v_e cos th + w_p y and y' = v_e sin th - w_p x carry no
    #   input: 1.5 + 1.5 + 4 = 7 and 1.5 + 4 = 5.5 as with unit bounds.
    # Swapping the evader's two inputs would give 1.2 on v_e and 1.3 on th.
    p = inputs.rel6d(n=(24, 6, 24, 3, 3, 3), bounds=(0.7, 0.4, 0.3, 1.2))
    p.lo = (-4.0, -4.0, -math.pi, 0.5, -1.0, 0.5)
    t = oracle.terms(p, inputs.random_field(p.n, seed=12), order=1)
    a = t["alpha"]
    assert a[0] == pytest.approx(7.0, abs=1e-12)
    assert a[1] == pytest.approx(5.5, abs=1e-12)
    assert a[2] == pytest.approx(2.2, abs=1e-12)
    assert a[3] == pytest.approx(0.7, abs=1e-15)
    assert a[4] == pytest.approx(0.4, abs=1e-15)
    assert a[5] == pytest.approx(0.3, abs=1e-15)
    # the dynamics themselves: one state, each input alone
    z = np.array([[1.0, -2.0, 0.3, 0.8, 0.5, 1.1]])
    u = np.array([[0.7, 0.0]])
    d = np.array([[0.0, 1.2]])
    f = oracle.eval_dynamics_batch("rel6d", p.params, z, u, d)[0]
    assert f[3] == pytest.approx(0.7) and f[4] == 0.0 and f[5] == 0.0
    assert f[2] == pytest.approx(1.2 - 0.5)
    f = oracle.eval_dynamics_batch("rel6d", p.params, z, np.array([[0.0, 0.4]]), np.array([[0.3, 0.0]]))[0]
    assert f[4] == pytest.approx(0.4) and f[5] == pytest.approx(0.3) and f[3] == 0.0
    assert f[2] == pytest.approx(-0.5)


# ---------------------------------------------------------------------------
# Lax-Friedrichs sign, upwinding, CFL step and TVD-RK2 (Algorithm 1,
# Section 3.1.3): exact transports
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("c", [1.0, -1.0])
def test_advection_cfl1_is_an_exact_shift(c):
    n, k = 16, 5
    h = 2 * math.pi / n
    p = inputs.advection((n,), (c,), horizon=k * h, cfl=1.0)
    l = p.target_values()
    r = oracle.solve(p, l=l)
    assert r["steps"][0] == k
    # phi(z, tau) = l(z + c tau): node i takes the value of node i + k (c > 0)
    expect = np.roll(l.astype(np.float64), -k if c > 0 else k)
    np.testing.assert_allclose(r["final"], expect, atol=1e-12)


def test_advection_2d_one_step_closed_form():
    n = 12
    h = 2 * math.pi / n
    p = inputs.advection((n, n), (1.0, 1.0), horizon=h / 2, cfl=1.0)
    l = p.target_values().astype(np.float64)
    r = oracle.solve(p, l=l)
    assert r["steps"][0] == 1
    expect = 0.5 * (np.roll(l, -1, axis=0) + np.roll(l, -1, axis=1))
    np.testing.assert_allclose(r["final"], expect, atol=1e-12)


def test_rk2_one_step_is_heun_average():
    # c = 1, CFL 1: stage 1 shifts by one node, stage 2 by two, the step
    # averages the start value and the two-node shift
    n = 10
    h = 2 * math.pi / n
    p = inputs.advection((n,), (1.0,), horizon=h, cfl=1.0, time_order=2)
    l = p.target_values().astype(np.float64)
    r = oracle.solve(p, l=l)
    assert r["steps"][0] == 1
    np.testing.assert_allclose(r["final"], 0.5 * (l + np.roll(l, -2)), atol=1e-12)


def transport_error(n, space_order, time_order, cfl=0.5, T=1.0):
    p = inputs.advection((n,), (1.0,), horizon=T, cfl=cfl, space_order=space_order,
                         time_order=time_order)
    r = oracle.solve(p)
    x = inputs.node_coords(p.n, p.lo, p.hi, p.periodic)[0]
    return np.abs(r["final"] - np.sin(x + T)).max()


def test_convergence_orders_on_smooth_transport():
    e1 = [transport_error(n, 1, 1) for n in (64, 128)]
    e2 = [transport_error(n, 2, 2) for n in (64, 128)]
    assert e1[0] / e1[1] > 1.8          # first order
    assert e2[0] / e2[1] > 3.2          # second order
    assert e2[1] < e1[1] / 10


# ---------------------------------------------------------------------------
# whole scheme against closed-form value functions
# ---------------------------------------------------------------------------

def si_errors(n, dims, u_mode, set_kind, T=0.5, r=0.5):
    """Max error against the closed form (a) over the nodes whose domain of
    dependence stays inside the box, (b) over those nodes away from the kinks
    of the exact solution (where a monotone first-order scheme converges at
    rate 1; at kinks the rate drops to 1/2)."""
    p = inputs.single_integrator((n,) * dims, half_width=2.0, radius=r, horizon=T,
                                 u_mode=u_mode, set_kind=set_kind)
    res = oracle.solve(p)
    mesh = np.meshgrid(*p.nodes(), indexing="ij")
    smooth = np.ones(p.n, bool)
    inner = np.ones(p.n, bool)
    for m in mesh:
        inner &= np.abs(m) <= 2.0 - T - 0.1
    if u_mode == "min":          # reach: distance to the box of reachable shifts
        v = np.sqrt(sum(np.maximum(np.abs(m) - T, 0.0) ** 2 for m in mesh)) - r
        for m in mesh:
            smooth &= np.abs(np.abs(m) - T) > 0.3
    elif set_kind == "brs":      # avoid BRS
        v = np.sqrt(sum((np.abs(m) + T) ** 2 for m in mesh)) - r
        for m in mesh:
            smooth &= np.abs(m) > 0.3
    else:                        # avoid BRT is the target itself
        v = p.target_values().astype(np.float64)
    e = np.abs(res["final"] - v)
    return e[inner].max(), e[inner & smooth].max(), res


@pytest.mark.parametrize("dims", [1, 2])
def test_single_integrator_reach_closed_form(dims):
    n0 = 41 if dims == 1 else 21
    e_all0, e_s0, _ = si_errors(n0, dims, "min", "brt")
    e_all1, e_s1, _ = si_errors(2 * n0 - 1, dims, "min", "brt")
    assert e_all1 < 0.16 and e_all1 < e_all0
    assert e_s1 < 0.06
    assert e_s0 / e_s1 > 1.7


def test_single_integrator_reach_1d_far_field_is_exact_shift_of_the_cone():
    # |x| >= t away from the kinks: V = |x| - r - t (upwind on a linear
    # function with |slope| = 1 is exact)
    p = inputs.single_integrator((81,), half_width=2.0, radius=0.5, horizon=0.5)
    res = oracle.solve(p)
    x = p.nodes()[0]
    far = np.abs(x) > 1.0
    np.testing.assert_allclose(res["final"][far], np.abs(x[far]) - 0.5 - 0.5, atol=1e-12)


def test_single_integrator_avoid_brs_closed_form():
    e_all0, e_s0, _ = si_errors(21, 2, "max", "brs")
    e_all1, e_s1, _ = si_errors(41, 2, "max", "brs")
    assert e_all1 < 0.04 and e_all0 / e_all1 > 1.7
    assert e_s0 / e_s1 > 1.6


def test_single_integrator_avoid_brt_equals_target_exactly():
    err, _, res = si_errors(33, 2, "max", "brt")
    assert err == 0.0


def dubins_transport_error(n_xy, n_th, T=0.5, v=1.0):
    """Error of the straight-driving car (w_max = 0) against
    V(z, t) = l(x + v t cos th, y + v t sin th), away from the boundary's
    domain of dependence and from the transported cone apex."""
    p = inputs.dubins3d(n=(n_xy, n_xy, n_th), v=v, w_max=0.0, radius=1.0, horizon=T,
                        set_kind="brs")
    res = oracle.solve(p)
    x, y, th = np.meshgrid(*p.nodes(), indexing="ij")
    rho = np.sqrt((x + v * T * np.cos(th)) ** 2 + (y + v * T * np.sin(th)) ** 2)
    inner = (np.abs(x) < 4 - v * T - 0.5) & (np.abs(y) < 4 - v * T - 0.5) & (rho > 0.5)
    return np.abs(res["final"] - (rho - 1.0))[inner].max()


def test_dubins3d_transport_characteristics():
    e1 = dubins_transport_error(41, 24)
    e2 = dubins_transport_error(81, 24)
    assert e2 < 0.06
    assert e1 / e2 > 1.7


def test_dubinscar4d_transport_characteristics():
    def err(n):
        T = 0.4
        p = inputs.dubinscar4d(n=(n, n, 5, 12), a_max=0.0, w_max=0.0, horizon=T,
                               set_kind="brs", space_order=1, time_order=1)
        res = oracle.solve(p)
        x, y, v, th = np.meshgrid(*p.nodes(), indexing="ij")
        rho = np.sqrt((x + v * T * np.cos(th)) ** 2 + (y + v * T * np.sin(th)) ** 2)
        inner = (np.abs(x) < 3.2) & (np.abs(y) < 3.2) & (rho > 0.5)
        return np.abs(res["final"] - (rho - 1.0))[inner].max()

    e1, e2 = err(41), err(81)   # speeds reach 3 here, so the constant is larger
    assert e2 < 0.2
    assert e1 / e2 > 1.7


def rel6d_exact(mesh, T, r):
    """Closed-form flow of the relative model with all input bounds 0:
    w = x + i y obeys w' = -v_p + v_e exp(i th) - i w_p w, th' = -w_p."""
    x, y, th, vp, wp, ve = mesh
    w0 = x + 1j * y
    rot = np.exp(-1j * wp * T)
    small = np.abs(wp) < 1e-12
    drift = np.where(small, T, (1 - rot) / np.where(small, 1.0, 1j * wp))
    w = rot * w0 - vp * drift + ve * np.exp(1j * th) * T * rot
    return np.abs(w) - r


def test_rel6d_closed_form_flow_matches_ode_integration():
    # the closed form used below is itself checked against RK4 integration
    rng = np.random.Generator(np.random.PCG64(5))
    z0 = np.array([rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(-3, 3), 1.2, -0.7, 0.8])
    T, steps = 0.6, 600
    z = z0.copy()
    f = lambda s: oracle.eval_dynamics("rel6d", (0.0, 0.0, 0.0, 0.0), s)
    hstep = T / steps
    for _ in range(steps):
        k1 = f(z)
        k2 = f(z + 0.5 * hstep * k1)
        k3 = f(z + 0.5 * hstep * k2)
        k4 = f(z + hstep * k3)
        z = z + hstep / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    mesh = [np.array(v) for v in z0]
    assert rel6d_exact(mesh, T, 0.0) == pytest.approx(math.hypot(z[0], z[1]), abs=1e-9)


def test_rel6d_transport_characteristics():
    def err(nxy, nth):
        T = 0.2
        p = inputs.rel6d(n=(nxy, nxy, nth, 2, 3, 2), bounds=(0.0, 0.0, 0.0, 0.0),
                         set_kind="brs", time_order=1, horizon=T)
        res = oracle.solve(p)
        mesh = np.meshgrid(*p.nodes(), indexing="ij")
        exact = rel6d_exact(mesh, T, 0.5)
        inner = (np.abs(mesh[0]) < 2.0) & (np.abs(mesh[1]) < 2.0) & (exact > 0.5)
        return np.abs(res["final"] - exact)[inner].max()

    e1, e2 = err(17, 12), err(33, 24)
    assert e2 < 0.25
    assert e1 / e2 > 1.7


# ---------------------------------------------------------------------------
# BRT invariants and symmetry
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("problem,monotone", [
    (inputs.dubins3d(tau=(0.0, 0.5, 1.0, 1.5, 2.0)), True),
    (inputs.dubinscar4d(n=(17, 17, 9, 16), tau=(0.0, 0.3, 0.6, 0.9), space_order=1), True),
    (inputs.dubinscar4d(n=(17, 17, 9, 16), tau=(0.0, 0.3, 0.6, 0.9)), False),
    (inputs.rel6d(n=(7, 7, 8, 3, 3, 3), tau=(0.0, 0.1, 0.2)), False),
], ids=lambda p: getattr(p, "name", str(p)))
def test_brt_invariants(problem, monotone):
    """V_t <= V_0 = l pointwise (the min with l, exact for every scheme).
    With first-order upwinding and a CFL <= 1 step the Lax-Friedrichs update is
    monotone, so the tube only grows: V(t2) <= V(t1).  ENO2 is not monotone,
    and neither is the sign-keeping ghost rule, which dominates on the
    three-node axes of the small 6-D grid; those cases check V <= l only."""
    res = oracle.solve(problem, snapshots=True)
    s = res["snapshots"]
    l = problem.target_values().astype(np.float64)
    np.testing.assert_array_equal(s[0], l)
    assert (s <= l[None]).all()
    if monotone:
        for k in range(1, len(s)):
            assert (s[k] <= s[k - 1] + 1e-12).all()


def test_dubins3d_rotation_and_mirror_symmetry():
    p = inputs.dubins3d()
    v = oracle.solve(p)["final"]
    nx, ny, nth = p.n
    rng_v = v.max() - v.min()
    # rotation by pi/2: (x, y, th) -> (-y, x, th + pi/2)
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nth), indexing="ij")
    rot = v[nx - 1 - j, i, (k + nth // 4) % nth]
    np.testing.assert_allclose(rot, v, atol=1e-9 * rng_v)
    # mirror: (x, y, th) -> (x, -y, -th)
    mir = v[i, ny - 1 - j, (nth - k) % nth]
    np.testing.assert_allclose(mir, v, atol=1e-9 * rng_v)


def test_step_count_and_last_step_of_the_dubins3d_workload():
    # alpha = (1, 1, 1), dz = (0.2, 0.2, 2 pi / 36): dt = 0.8 / (5 + 5 + 18/pi)
    p = inputs.dubins3d()
    r = oracle.solve(p)
    dt = 0.8 / (5.0 + 5.0 + 18.0 / math.pi)
    assert r["steps"][0] == math.ceil(2.0 / dt) == 40
    assert r["last_dt"] == pytest.approx(2.0 - 39 * dt, rel=1e-9)


def test_invalid_arguments_are_rejected():
    p = inputs.dubins3d(n=(5, 5, 4))
    bad_tau = inputs.dubins3d(n=(5, 5, 4), tau=(0.0, 1.0, 0.5))
    assert oracle.solve(bad_tau, raise_on_error=False)["rc"] == oracle.EINVAL
    short = inputs.dubins3d(n=(1, 5, 4))
    with pytest.raises(oracle.OracleError):
        oracle.solve(short, l=np.zeros(20, np.float32))
    r = oracle.solve(p, max_steps=2, raise_on_error=False)
    assert r["rc"] == oracle.ETIMEOUT


def test_resuming_from_a_kept_value_continues_the_schedule():
    # solving (0, T1, T2) equals solving (0, T1) and resuming from its value
    p = inputs.dubins3d(n=(21, 21, 16), tau=(0.0, 0.6, 1.1), space_order=2, time_order=2)
    full = oracle.solve(p, snapshots=True)
    seg = inputs.dubins3d(n=(21, 21, 16), tau=(0.0, 0.5), space_order=2, time_order=2)
    res = oracle.solve(seg, phi0=full["snapshots"][1])
    np.testing.assert_allclose(res["final"], full["final"], atol=1e-12)
    assert res["steps"][0] == full["steps"][1]


# ---------------------------------------------------------------------------
# reach-avoid: phi <- max(min(phi, l), g) after each step (Section 4.3, the
# target and obstacle computation methods; reading R17)
# ---------------------------------------------------------------------------

def test_reach_avoid_with_an_obstacle_below_the_value_is_the_brt():
    # an obstacle that never exceeds the value changes nothing, bit for bit
    p = inputs.dubins3d(n=(21, 19, 16), horizon=0.7)
    l = p.target_values()
    low = np.full(p.n, float(l.min()) - 1.0, dtype=np.float32)
    ref = oracle.solve(p)
    ra = oracle.solve(p, g=low)
    assert np.array_equal(ref["final"], ra["final"])
    assert np.array_equal(ref["steps"], ra["steps"])


@pytest.mark.parametrize("order", [(1, 1), (2, 2)])
def test_reach_avoid_value_stays_above_the_obstacle(order):
    # after every step phi >= g; where target and obstacle overlap the obstacle
    # wins (min with l first, then max with g)
    p = inputs.reach_avoid(
        inputs.dubins3d(n=(25, 25, 16), space_order=order[0], time_order=order[1],
                        tau=tuple(np.linspace(0.0, 1.0, 6))),
        inputs.cylinder_obstacle(0.8, center=(0.5, 0.0)))
    g = p.obstacle_values().astype(np.float64)
    l = p.target_values().astype(np.float64)
    r = oracle.solve(p, snapshots=True)
    for snap in r["snapshots"][1:]:
        assert np.all(snap >= g)
    both = (g > 0) & (l < 0)
    assert both.any()
    assert np.all(r["final"][both] > 0)
    # the plain tube marks those nodes reachable
    plain = oracle.solve(inputs.dubins3d(n=(25, 25, 16), space_order=order[0], time_order=order[1],
                                         tau=tuple(np.linspace(0.0, 1.0, 6))))
    assert np.all(plain["final"][both] < 0)


def test_reach_avoid_obstacle_acts_only_within_its_domain_of_dependence():
    # the upwind Euler update couples a node to its axis neighbours only and
    # the single integrator's alpha does not depend on phi, so after s steps
    # the obstacle can only have changed nodes within L1 distance s (in cells)
    # of the nodes where it binds
    n = (31, 29)
    base = inputs.single_integrator(n, horizon=2.0)
    obst = inputs.box_obstacle((0.6, -0.4), (1.0, 0.4), dims=(0, 1))
    ra = inputs.reach_avoid(base, obst)
    g = ra.obstacle_values().astype(np.float64)
    l = base.target_values().astype(np.float64)
    steps = 6
    plain = oracle.solve(base, max_steps=steps, raise_on_error=False)
    with_g = oracle.solve(ra, max_steps=steps, raise_on_error=False)
    assert plain["rc"] == with_g["rc"] == -5   # stopped by the step limit
    # nodes where the obstacle can bind at some step: g above the smallest value
    # the plain solve can take there (it only decreases from l)
    bind = g > plain["final"] - 1e-12
    bind |= g > l
    ii, jj = np.nonzero(bind)
    I, J = np.meshgrid(np.arange(n[0]), np.arange(n[1]), indexing="ij")
    dist = np.full(n, 10 ** 6)
    for a, b in zip(ii, jj):
        dist = np.minimum(dist, np.abs(I - a) + np.abs(J - b))
    far = dist > steps
    assert far.sum() > 0.5 * far.size
    assert np.array_equal(plain["final"][far], with_g["final"][far])
    near = dist <= steps
    assert np.abs(plain["final"][near] - with_g["final"][near]).max() > 0


def test_reach_avoid_1d_obstacle_blocks_the_far_side():
    # x' = u, |u| <= 1 on [-4, 4]; target |x| <= 0.5; obstacle [1.5, 2.5].
    # Without the obstacle x = 3 is reached after t = 2.5; with it every node
    # at or beyond the obstacle's far face stays out of the reach-avoid set,
    # while the near side fills in as for the plain tube
    base = inputs.single_integrator((161,), half_width=4.0, horizon=3.0)
    ra = inputs.reach_avoid(base, inputs.box_obstacle((1.5,), (2.5,), dims=(0,)))
    x = base.nodes()[0]
    plain = oracle.solve(base)["final"]
    with_g = oracle.solve(ra)["final"]
    assert plain[np.argmin(np.abs(x - 3.0))] < 0
    assert np.all(with_g[x >= 2.5 - 1e-9] >= 0)
    near = (x > -1.3) & (x < 1.3)
    assert np.all(with_g[near] < 0) and np.all(plain[near] < 0)


# ---------------------------------------------------------------------------
# per-node dissipation: alpha_i of each node instead of the grid maximum
# (Algorithm 1's second loop; reading R18)
# ---------------------------------------------------------------------------

def local(problem):
    return dataclasses.replace(problem, dissipation="local")


@pytest.mark.parametrize("problem", [
    inputs.single_integrator((19, 17), horizon=0.6),
    inputs.single_integrator((9, 8, 7), space_order=2, time_order=2, horizon=0.4),
    inputs.advection((24, 20), (1.0, -0.5), horizon=0.5, cfl=0.8),
], ids=lambda p: p.name)
def test_local_dissipation_equals_global_when_alpha_is_uniform(problem):
    # the single integrator's bound and a constant velocity give every node
    # the grid alpha, so the two dissipations are the same numbers
    a = oracle.solve(problem)
    b = oracle.solve(local(problem))
    assert np.array_equal(a["final"], b["final"])
    assert np.array_equal(a["steps"], b["steps"])


def test_local_dissipation_is_the_upwind_scheme_for_transport():
    # Dubins car with no turning: phi_tau = v cos(th) phi_x + v sin(th) phi_y.
    # With alpha_i = |a_d(z_i)| the Lax-Friedrichs term a pbar + |a|/2 (p+ - p-)
    # is the upwind difference a p+ (a >= 0) or a p- (a < 0), the textbook
    # first-order upwind scheme, written out here independently
    p = local(inputs.dubins3d(n=(23, 21, 16), v=1.3, w_max=0.0, set_kind="brs"))
    rng = np.random.Generator(np.random.PCG64(11))
    phi = rng.uniform(-1.0, 1.0, size=p.n)
    dt = 0.03
    out = oracle.step(p, phi, dt, l=np.zeros(p.n))["out"]
    x, y, th = p.nodes()
    hx, hy = x[1] - x[0], y[1] - y[0]
    ax = (1.3 * np.cos(th))[None, None, :]
    ay = (1.3 * np.sin(th))[None, None, :]
    fx = (phi[2:, 1:-1] - phi[1:-1, 1:-1]) / hx        # D+ along x
    bx = (phi[1:-1, 1:-1] - phi[:-2, 1:-1]) / hx       # D- along x
    fy = (phi[1:-1, 2:] - phi[1:-1, 1:-1]) / hy
    by = (phi[1:-1, 1:-1] - phi[1:-1, :-2]) / hy
    upwind = np.where(ax >= 0, ax * fx, ax * bx) + np.where(ay >= 0, ay * fy, ay * by)
    expect = phi[1:-1, 1:-1] + dt * upwind
    np.testing.assert_allclose(out[1:-1, 1:-1], expect, rtol=0, atol=1e-13)
    # the grid alpha adds dissipation wherever |cos th| or |sin th| < 1
    glob = oracle.step(dataclasses.replace(p, dissipation="global"), phi, dt, l=np.zeros(p.n))["out"]
    assert np.abs(glob[1:-1, 1:-1] - expect).max() > 1e-3


def test_local_dissipation_is_closer_to_the_exact_transport():
    # same transport from a smooth field: the exact solution is the field
    # shifted along (v cos th, v sin th); away from the non-periodic x, y
    # faces the per-node dissipation stays closer to it than the grid one
    v, T = 1.0, 0.6
    target = lambda m: np.sin(1.3 * m[0]) * np.cos(0.9 * m[1])
    base = inputs.dubins3d(n=(61, 61, 16), v=v, w_max=0.0, set_kind="brs", horizon=T)
    base = dataclasses.replace(base, target=target)
    x, y, th = base.nodes()
    X, Y, TH = np.meshgrid(x, y, th, indexing="ij")
    exact = np.sin(1.3 * (X + v * np.cos(TH) * T)) * np.cos(0.9 * (Y + v * np.sin(TH) * T))
    inner = (np.abs(X) < 2.5) & (np.abs(Y) < 2.5)
    err_g = np.abs(oracle.solve(base)["final"] - exact)[inner].max()
    err_l = np.abs(oracle.solve(local(base))["final"] - exact)[inner].max()
    assert err_l < 0.8 * err_g
    assert err_l < 0.05


def test_local_dissipation_keeps_the_brt_monotone():
    p = local(inputs.dubins3d(tau=(0.0, 0.5, 1.0, 1.5, 2.0)))
    s = oracle.solve(p, snapshots=True)["snapshots"]
    l = p.target_values().astype(np.float64)
    assert (s <= l[None]).all()
    for k in range(1, len(s)):
        assert (s[k] <= s[k - 1] + 1e-12).all()


# ---------------------------------------------------------------------------
# the pursuit-evasion capture model of Section 4.2: its evader input enters
# all three components, so its switching function y p_x - x p_y - p_th mixes
# them and the dissipation bound needs interval bounds of it
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("problem", [
    inputs.dubins_capture(n=(9, 9, 8)),
    inputs.dubins_capture(n=(9, 9, 8), u_mode="min", d_mode="max"),
    inputs.rel6d(n=(4, 4, 4, 3, 3, 3)),
], ids=lambda p: p.name + "_" + p.u_mode)
@pytest.mark.parametrize("order", [1, 2])
def test_local_alpha_matches_the_corners_of_the_derivative_box(problem, order):
    # the switching functions are linear in p, so over a node's derivative box
    # their ranges are spanned by its corners: an input's selectable extremes
    # are its bang-bang choices at the corners.  alpha_d is the largest |f_d|
    # over every combination of each input's selectable extremes (reading
    # R20); the choices the inputs make together at one corner never exceed it
    phi = inputs.random_field(problem.n, seed=5 + order)
    t = oracle.terms(problem, phi, order=order)
    nd = problem.ndim
    lo = np.minimum(t["pm"], t["pp"]).reshape(-1, nd)
    hi = np.maximum(t["pm"], t["pp"]).reshape(-1, nd)
    z = np.stack(np.meshgrid(*problem.nodes(), indexing="ij"), axis=-1).reshape(-1, nd)
    ub, db = input_bounds(problem)
    rng = np.random.Generator(np.random.PCG64(4))
    pick = rng.choice(len(z), size=min(len(z), 60), replace=False)
    corners = np.array(np.meshgrid(*[[0, 1]] * nd, indexing="ij")).reshape(nd, -1).T
    a_oracle = t["a"].reshape(-1, nd)[pick]
    dyn, prm = problem.dynamics, problem.params

    def column(zi, k, is_d):
        e = np.zeros(8)
        e[k] = 1.0
        f0 = oracle.eval_dynamics(dyn, prm, zi)
        f1 = oracle.eval_dynamics(dyn, prm, zi, d=e) if is_d else oracle.eval_dynamics(dyn, prm, zi, u=e)
        return f1 - f0

    def choice(s, b, mode):
        up = s >= 0 if mode == "max" else s < 0
        return b if up else -b

    for row, i in enumerate(pick):
        pcs = [np.where(c == 1, hi[i], lo[i]) for c in corners]
        sel, joint = [], [dict() for _ in pcs]
        for k, (b, is_d) in enumerate([(b, False) for b in ub] + [(b, True) for b in db]):
            g = column(z[i], k - (len(ub) if is_d else 0), is_d)
            mode = problem.d_mode if is_d else problem.u_mode
            picks = [choice(float(pc @ g), b, mode) for pc in pcs]
            sel.append(sorted(set(picks)))
            for c, v in enumerate(picks):
                joint[c][k] = v
        best = np.zeros(nd)
        for combo in np.array(np.meshgrid(*sel, indexing="ij")).reshape(len(sel), -1).T:
            u = np.zeros(8)
            d = np.zeros(8)
            u[:len(ub)] = combo[:len(ub)]
            d[:len(db)] = combo[len(ub):]
            best = np.maximum(best, np.abs(oracle.eval_dynamics(dyn, prm, z[i], u=u, d=d)))
        np.testing.assert_allclose(a_oracle[row], best, rtol=0, atol=1e-12)
        for jc in joint:
            u = np.zeros(8)
            d = np.zeros(8)
            u[:len(ub)] = [jc[k] for k in range(len(ub))]
            d[:len(db)] = [jc[len(ub) + k] for k in range(len(db))]
            f = np.abs(oracle.eval_dynamics(dyn, prm, z[i], u=u, d=d))
            assert (f <= a_oracle[row] + 1e-12).all()


def capture_transport_error(n_xy, n_th, T=0.5, v=1.0):
    """Without turning (A = B = 0) the capture dynamics drift with
    (-v + v cos th, v sin th): V(z, t) = l(x + t (v cos th - v), y + t v sin th)."""
    p = inputs.dubins_capture(n=(n_xy, n_xy, n_th), v=v, a_max=0.0, b_max=0.0, radius=1.0,
                              horizon=T, set_kind="brs")
    res = oracle.solve(p)
    x, y, th = np.meshgrid(*p.nodes(), indexing="ij")
    xs, ys = x + T * (v * np.cos(th) - v), y + T * v * np.sin(th)
    rho = np.sqrt(xs ** 2 + ys ** 2)
    inner = (np.abs(x) < 4 - 2 * v * T - 0.5) & (np.abs(y) < 4 - v * T - 0.5) & (rho > 0.5)
    return np.abs(res["final"] - (rho - 1.0))[inner].max()


def test_capture_transport_characteristics():
    e1 = capture_transport_error(41, 24)
    e2 = capture_transport_error(81, 24)
    assert e2 < 0.1
    assert e1 / e2 > 1.6


def test_capture_mirror_symmetry():
    # (x, y, th) -> (x, -y, -th) with a -> -a, b -> -b maps the game onto
    # itself; the symmetric bounds and target make the value symmetric
    p = inputs.dubins_capture(n=(21, 21, 16), horizon=0.6)
    v = oracle.solve(p)["final"]
    mirrored = v[:, ::-1, :][:, :, (-np.arange(16)) % 16]
    np.testing.assert_allclose(v, mirrored, rtol=0, atol=1e-12)
