"""GPU (FP32, CUDA kernels through the C ABI) against the FP64 oracle.

Criterion: max |V_gpu - V_oracle| <= 1e-4 * (max l - min l) on the same
seeded inputs, with equal step counts.

First-order (upwind) runs are compared over the whole solve at that bar.

Second-order ENO runs meet a discontinuity of the method itself: the
stencil choice (Section 3.1.4) switches where the two candidate second
differences have equal magnitude, so float32 rounding of the stored values
can pick the other, equally valid, stencil.  They are checked two ways:

* whole solves against the oracle's own sensitivity: the FP64 oracle moves
  by 0.4e-4 to 6e-4 of the value range when its values are rounded to
  float32 after every step, or its target is perturbed by 1e-7 relative;
  the GPU must stay within twice that (and within 1e-4 wherever the oracle
  itself stays within it);
* step by step: from every kept GPU value the oracle takes one step, and
  every node is held to 1e-4 of the range unless a stencil choice that the
  float32 kernel and the FP64 oracle take differently (a flip, found by
  recomputing both decisions from the same window) reaches it; those nodes
  are held to the bound the flip puts on the step (`eno_flips`).

Small grids span many blocks with a ragged tail; full-size workloads are
checked end to end (DubinsCar4D), step by step at points spread over the
horizon (Rel6D), and by properties that hold at any size.
"""
import dataclasses
import math
import os

import numpy as np
import pytest

import eno_flips
import oracle
import parity
import parity_log
from paper_2204_05520_gb300 import inputs, odp

pytestmark = pytest.mark.gpu
REL_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_05520_gb300 import _build

    _build.build()
    odp.load()
    oracle.build()
    return torch


def gpu_solve(problem, keep=False, l=None, step_limit=None):
    import torch

    l_host = problem.target_values() if l is None else l
    l_dev = torch.from_numpy(l_host).cuda()
    with odp.Grid.for_problem(problem) as g:
        if step_limit:
            odp.set_step_limit(g.handle, step_limit)
        g.set_target(l_dev)
        stats = g.solve_problem(problem, keep_snapshots=keep, stats=True)
        out = torch.empty_like(l_dev)
        g.readback(out)
        snaps = None
        if keep:
            snaps = np.stack([g.readback(torch.empty_like(l_dev), k).cpu().numpy()
                              for k in range(len(problem.tau))])
    return out.cpu().numpy(), stats, snaps


def check_parity(problem, keep=False):
    v, stats, snaps = gpu_solve(problem, keep=keep)
    ref = oracle.solve(problem, snapshots=keep)
    l = problem.target_values().astype(np.float64)
    tol = REL_TOL * (l.max() - l.min())
    assert stats["steps"] == int(ref["steps"].sum())
    err = np.abs(v - ref["final"]).max()
    assert err <= tol, "max err %.3g > tol %.3g" % (err, tol)
    if keep:
        for k in range(len(problem.tau)):
            e = np.abs(snaps[k] - ref["snapshots"][k]).max()
            assert e <= tol, "tau[%d]: max err %.3g > tol %.3g" % (k, e, tol)
    np.testing.assert_allclose(stats["alpha"][: problem.ndim], ref["alpha"], rtol=1e-6)
    return err / (l.max() - l.min())


def alpha_upper_bound(problem):
    """The oracle's alpha on a random field: every derivative box then holds
    both signs somewhere, so no solve of the problem has a larger alpha and
    no CFL step shorter than the one it gives."""
    phi = np.random.default_rng(7).uniform(-1.0, 1.0, problem.n)
    return oracle.terms(problem, phi)["alpha"]


def stage1_problem(problem):
    """The first stage of a TVD-RK2 step as a problem of its own: one Euler
    stage without the post-step set operations."""
    return dataclasses.replace(problem, time_order=1, set_kind="brs", obstacle=None)


def flip_bound(problem, phi, h, alpha, l):
    """(flips of stage 1, flips of stage 2, per-node bound) of one step of
    size h from the GPU's value phi; zero without ENO2."""
    if problem.space_order == 1:
        return 0, 0, np.zeros(phi.shape)
    dz = oracle.spacing(problem.n, problem.lo, problem.hi, problem.periodic)
    s1 = None
    if problem.time_order == 2:
        s1 = oracle.step(stage1_problem(problem), phi, h, l=l)["out"]
    return eno_flips.step_bound(phi, s1, problem.periodic, dz, alpha, h, problem.time_order)


def check_parity_resync(problem, name=None):
    """Step-by-step route: the GPU solves over a schedule of one-step
    segments (spacing just below the shortest CFL step any value of the
    problem can have) keeping every value; from each kept value the oracle
    takes that step.  Nodes no stencil-choice flip reaches are held to the
    1e-4 bar; the others to the bar plus the flip bound."""
    alpha = alpha_upper_bound(problem)
    dz = oracle.spacing(problem.n, problem.lo, problem.hi, problem.periodic)
    spacing = problem.cfl / float(np.sum(alpha / dz)) * (1.0 - 1e-6)
    T = float(problem.tau[-1])
    k = int(math.ceil(T / spacing))
    tau = tuple(min(T, i * spacing) for i in range(k)) + (T,)
    p = dataclasses.replace(problem, tau=tau)
    _, stats, snaps = gpu_solve(p, keep=True)
    l = p.target_values()
    rng_l = float(l.max() - l.min())
    tol = REL_TOL * rng_l
    worst, flips, touched = 0.0, 0, 0
    for i in range(len(tau) - 1):
        h = tau[i + 1] - tau[i]
        seg = dataclasses.replace(problem, tau=(0.0, h))
        ref = oracle.solve(seg, l=l, phi0=snaps[i])
        assert int(ref["steps"].sum()) == 1
        c1, c2, B = flip_bound(problem, snaps[i], h, alpha, l)
        err = np.abs(snaps[i + 1] - ref["final"])
        ratio = float((err / (tol + B)).max())
        assert ratio <= 1.0, "step %d: max err %.3g over the bound (flips %d + %d, %d nodes)" % (
            i, err.max(), c1, c2, int((B > 0).sum()))
        worst = max(worst, float(err[B <= 0.01 * tol].max(initial=0.0)) / rng_l)
        flips += c1 + c2
        touched += int((B > tol).sum())
    assert stats["steps"] == len(tau) - 1
    parity_log.note(name or problem.name, "%d one-step segments, max err/range off flips %.2e, "
                    "ENO2 flips %d, node-steps whose flip bound exceeds the bar %d"
                    % (len(tau) - 1, worst, flips, touched))
    return worst


def check_whole_solve_eno2(problem, spread=None, name=None):
    """Whole ENO2 solve against the FP64 oracle, held to twice the oracle's
    own sensitivity to float32-level changes (float32 storage; target
    perturbed by 1e-7 relative), measured here unless given."""
    v, stats, _ = gpu_solve(problem)
    return parity.check_whole_solve(problem, v, stats["steps"], spread=spread, name=name)


def check(problem):
    if problem.space_order == 2:
        return check_parity_resync(problem)
    return check_parity(problem, keep=len(problem.tau) > 2)


# ---------------------------------------------------------------------------
# every model and scheme on small grids
# ---------------------------------------------------------------------------

CASES = [
    inputs.dubins3d(),                                                   # 41x41x36, Euler, upwind
    inputs.dubins3d(n=(23, 19, 13), space_order=2, time_order=2),
    inputs.dubins3d(n=(17, 21, 12), u_mode="max", set_kind="brs"),
    inputs.dubins3d(n=(31, 31, 24), set_kind="brs", tau=(0.0, 0.3, 0.7, 1.0)),
    inputs.dubinscar4d(n=(21, 19, 11, 16)),                              # ENO2 + RK2
    inputs.dubinscar4d(n=(17, 15, 9, 12), space_order=1, time_order=1),
    inputs.dubinscar4d(n=(13, 13, 7, 10), u_mode="max", set_kind="brs"),
    inputs.rel6d(n=(9, 8, 10, 5, 4, 3), horizon=0.3),                    # upwind + RK2
    inputs.rel6d(n=(7, 7, 8, 3, 4, 3), space_order=2, horizon=0.2),
    inputs.rel6d(n=(8, 9, 8, 3, 3, 4), time_order=1, set_kind="brs", horizon=0.2),
]


@pytest.mark.parametrize("problem", CASES, ids=lambda p: "%s_o%d%d_%s_%s" % (
    p.name, p.space_order, p.time_order, p.set_kind, p.u_mode))
def test_models_match_oracle(problem):
    check(problem)


SI = [((37,), "min", "brt"), ((13, 11), "max", "brs"), ((9, 7, 6), "min", "brs"),
      ((6, 5, 7, 4), "max", "brt"), ((5, 4, 3, 6, 3), "min", "brt"),
      ((3, 4, 3, 3, 2, 4), "min", "brs")]


@pytest.mark.parametrize("n,mode,kind", SI, ids=lambda v: str(v))
@pytest.mark.parametrize("order", [(1, 1), (2, 2)])
def test_single_integrator_every_dimension(n, mode, kind, order):
    p = inputs.single_integrator(n, u_mode=mode, set_kind=kind, space_order=order[0],
                                 time_order=order[1], horizon=0.4)
    check(p)


def test_advection_exact_shift_on_gpu():
    n, k = 64, 7
    h = 2 * math.pi / n
    p = inputs.advection((n,), (1.0,), horizon=k * h, cfl=1.0)
    v, stats, _ = gpu_solve(p)
    assert stats["steps"] == k
    l = p.target_values()
    np.testing.assert_allclose(v, np.roll(l, -k), atol=1e-5)


def test_degenerate_axes():
    # periodic axes of 1 and 2 nodes, non-periodic axes of 2 nodes
    for n, per in (((1, 9), (True, True)), ((2, 7), (True, False)), ((2, 2, 5), (False, False, True))):
        p = inputs.Problem(
            name="deg", n=n, lo=(0.0,) * len(n), hi=(1.0,) * len(n), periodic=per,
            dynamics="advection", params=tuple(0.5 + 0.25 * d for d in range(len(n))),
            u_mode="max", d_mode="max", target=inputs.sine_bump((1,) * len(n)), tau=(0.0, 0.3),
            set_kind="brs", space_order=2, time_order=2)
        check(p)


# ---------------------------------------------------------------------------
# error paths reported by the device
# ---------------------------------------------------------------------------

def test_step_limit_reports_timeout():
    p = inputs.dubins3d(n=(9, 9, 8))
    with pytest.raises(odp.OdpError) as e:
        gpu_solve(p, step_limit=3)
    assert e.value.code == odp.ETIMEOUT


def test_non_finite_target_reports_numeric_error():
    p = inputs.dubins3d(n=(9, 9, 8))
    l = p.target_values()
    l[4, 4, 3] = np.nan
    with pytest.raises(odp.OdpError) as e:
        gpu_solve(p, l=l)
    assert e.value.code == odp.ENUMERIC


def test_missing_target_is_a_state_error():
    p = inputs.dubins3d(n=(9, 9, 8))
    with odp.Grid.for_problem(p) as g:
        with pytest.raises(odp.OdpError) as e:
            g.solve_problem(p)
        assert e.value.code == odp.ESTATE


# ---------------------------------------------------------------------------
# full-size workloads
# ---------------------------------------------------------------------------

def steps_at_full_size(problem, points, name):
    """One GPU solve whose schedule holds a one-step segment (half the CFL
    step) at each of `points`; from the GPU's value at the start of each the
    oracle takes the same step.  Every node is held to the 1e-4 bar plus,
    for ENO2, the bound of any stencil-choice flip that reaches it.  Returns
    (max err / range off flips, last GPU value, l)."""
    import torch

    l = problem.target_values()
    rng_l = float(l.max() - l.min())
    tol = REL_TOL * rng_l
    alpha = alpha_upper_bound(problem)
    dz = oracle.spacing(problem.n, problem.lo, problem.hi, problem.periodic)
    delta = 0.5 * problem.cfl / float(np.sum(alpha / dz))
    tau = [0.0]
    for t in points:
        tau += [t, t + delta]
    if tau[-1] < problem.tau[-1]:
        tau.append(float(problem.tau[-1]))
    worst, flips, touched = 0.0, 0, 0
    with odp.Grid.for_problem(problem) as g:
        g.set_target(torch.from_numpy(l).cuda())
        st = g.solve(tuple(tau), problem.set_kind, problem.space_order, problem.time_order,
                     problem.cfl, keep_snapshots=True, stats=True)
        buf = torch.empty(l.shape, device="cuda")
        for j in range(len(points)):
            phi_a = g.readback(buf, 2 * j + 1).cpu().numpy()
            phi_b = g.readback(buf, 2 * j + 2).cpu().numpy()
            ref = oracle.step(problem, phi_a, delta, l=l)
            c1, c2, B = flip_bound(problem, phi_a, delta, alpha, l)
            err = np.abs(phi_b - ref["out"])
            ratio = float((err / (tol + B)).max())
            assert ratio <= 1.0, "t = %g: max err %.3g over the bound (flips %d + %d)" % (
                points[j], err.max(), c1, c2)
            worst = max(worst, float(err[B <= 0.01 * tol].max(initial=0.0)) / rng_l)
            flips += c1 + c2
            touched += int((B > tol).sum())
            del ref, B, err, phi_a
        last = g.readback(buf, len(tau) - 1).cpu().numpy()
    parity_log.note(name, "one step at t = %s: max err/range off flips %.2e, ENO2 flips %d, "
                    "nodes whose flip bound exceeds the bar %d"
                    % (", ".join("%g" % t for t in points), worst, flips, touched))
    assert np.isfinite(st["t_final"])
    return worst, last, l


def test_dubinscar4d_full_size_step_matches_oracle():
    p = inputs.dubinscar4d()   # 80x80x40x64, ENO2 + RK2
    rel, _, _ = steps_at_full_size(p, (0.5, 2.9), "dubinscar4d full size, steps")
    assert rel <= REL_TOL


def read_sensitivity(workload):
    path = os.path.join(os.path.dirname(__file__), "golden", "eno2_sensitivity.txt")
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            cols = [c.strip() for c in line.split("|")]
            if cols[0] == workload:
                return int(cols[1]), tuple(float(c) for c in cols[2:])
    raise KeyError(workload)


def test_dubinscar4d_full_size_solve_matches_oracle():
    # the whole 265-step ENO2 + TVD-RK2 solve of the 80x80x40x64 grid against
    # the FP64 oracle, held to twice the oracle's own sensitivity of this
    # solve (tests/golden/eno2_sensitivity.txt, written from the oracle alone)
    p = inputs.dubinscar4d()
    steps, spread = read_sensitivity(p.name)
    assert steps == 265
    check_whole_solve_eno2(p, spread=spread, name="dubinscar4d full size")


@pytest.mark.parametrize("problem", [inputs.dubinscar4d(n=(21, 19, 11, 16)),
                                     inputs.dubinscar4d(n=(41, 41, 21, 32))], ids=lambda p: p.name)
def test_eno2_whole_solve_within_the_oracles_own_sensitivity(problem):
    check_whole_solve_eno2(problem)


def test_dubinscar4d_full_size_solve_properties():
    p = inputs.dubinscar4d()
    v, stats, _ = gpu_solve(p)
    l = p.target_values()
    assert stats["steps"] == 265
    assert stats["t_final"] == 3.0
    assert np.isfinite(v).all()
    assert (v <= l).all()
    # the tube grows: strictly more nodes inside than at t = 0
    assert (v <= 0).sum() > (l <= 0).sum()


def test_dubins3d_full_size_matches_oracle_exactly_in_steps():
    r = check_parity(inputs.dubins3d())
    assert r <= REL_TOL


def test_rel6d_full_size_steps_match_oracle():
    # one step from the GPU's state at three points spread over t in [0, 1.5]
    p = inputs.rel6d()         # 24^6, upwind + RK2
    rel, _, _ = steps_at_full_size(p, (0.05, 0.75, 1.45), "rel6d full size, steps")
    assert rel <= REL_TOL


def test_rel6d_full_size_solve_properties():
    p = inputs.rel6d()
    v, stats, _ = gpu_solve(p)
    l = p.target_values()
    assert 185 <= stats["steps"] <= 195
    assert stats["t_final"] == 1.5
    assert np.isfinite(v).all()
    assert (v <= l).all()
    assert stats["alpha"][0] == pytest.approx(7.0) and stats["alpha"][1] == pytest.approx(5.5)


@pytest.mark.parametrize("problem", [
    inputs.dubins3d(n=(21, 23, 16), horizon=0.5),
    dataclasses.replace(inputs.dubinscar4d(n=(11, 13, 7, 12), horizon=0.4), tau=np.array([0.0, 0.1, 0.25, 0.4])),
    inputs.rel6d(n=(6, 6, 8, 4, 4, 4), horizon=0.2),
], ids=["dubins3d_euler", "dubinscar4d_rk2_eno2_snapshots", "rel6d_rk2"])
def test_host_stepped_loop_equals_graph_loop(problem):
    # the same kernels in the same order: bit-identical values, snapshots and steps
    import torch

    l_dev = torch.from_numpy(problem.target_values()).cuda()
    keep = len(problem.tau) > 2
    res = []
    for host in (False, True):
        with odp.Grid.for_problem(problem) as g:
            odp.set_loop_mode(g.handle, host)
            g.set_target(l_dev)
            st = g.solve_problem(problem, keep_snapshots=keep, stats=True)
            vals = [g.readback(torch.empty_like(l_dev), k).cpu().numpy()
                    for k in (range(len(problem.tau)) if keep else [-1])]
            res.append((st["steps"], vals))
    assert res[0][0] == res[1][0] > 0
    for a, b in zip(res[0][1], res[1][1]):
        assert np.array_equal(a, b)


# ---------------------------------------------------------------------------
# reach-avoid: phi <- max(min(phi, l), g) after each step
# ---------------------------------------------------------------------------

RA_CASES = [
    inputs.reach_avoid(inputs.dubins3d(n=(41, 41, 36)), inputs.dubins_obstacle()),
    inputs.reach_avoid(inputs.dubins3d(n=(25, 27, 20), tau=(0.0, 0.4, 1.0, 1.6)),
                       inputs.cylinder_obstacle(0.8, center=(0.5, 0.0))),
    inputs.reach_avoid(inputs.single_integrator((37, 29), horizon=1.5),
                       inputs.box_obstacle((0.6, -0.4), (1.0, 0.4), dims=(0, 1))),
    inputs.reach_avoid(inputs.dubinscar4d(n=(21, 19, 11, 16), horizon=1.0), inputs.dubins_obstacle()),
    inputs.reach_avoid(inputs.rel6d(n=(9, 8, 10, 5, 4, 3), horizon=0.3),
                       inputs.box_obstacle((0.0, -1.5), (2.0, 1.5), dims=(0, 1))),
]


@pytest.mark.parametrize("problem", RA_CASES, ids=lambda p: "%s_o%d%d" % (p.name, p.space_order, p.time_order))
def test_reach_avoid_matches_oracle(problem):
    check(problem)


def test_reach_avoid_full_size_step_matches_oracle():
    p = inputs.workload("dubinscar4d_reach_avoid")   # 80x80x40x64, ENO2 + RK2, obstacle
    rel, last, _ = steps_at_full_size(p, (1.0,), "reach-avoid full size, step")
    assert rel <= REL_TOL
    assert (last >= p.obstacle_values()).all()


def test_removing_the_obstacle_restores_the_plain_tube():
    import torch

    p = inputs.dubins3d(n=(21, 23, 16), horizon=0.8)
    l = torch.from_numpy(p.target_values()).cuda()
    g_vals = inputs.reach_avoid(p, inputs.dubins_obstacle()).obstacle_values()
    out = []
    for obst in (None, g_vals, None):
        with odp.Grid.for_problem(p) as g:
            g.set_target(l)
            g.set_obstacle(g_vals)
            g.set_obstacle(obst)
            g.solve_problem(p)
            out.append(g.readback(torch.empty_like(l)).cpu().numpy())
    assert np.array_equal(out[0], out[2])
    assert not np.array_equal(out[0], out[1])


def test_obstacle_arguments_are_checked():
    p = inputs.dubins3d(n=(9, 9, 8))
    with odp.Grid.for_problem(p) as g:
        with pytest.raises(ValueError):   # the binding checks the size first
            g.set_obstacle(np.zeros((9, 9, 7), np.float32))
        arr = np.zeros(p.n, np.float32)
        assert odp.load().odp_set_obstacle(g.handle, arr.ctypes.data, arr.size - 1, 0) == odp.EINVAL
        g.set_target(p.target_values())
        g.set_obstacle(np.zeros(p.n, np.float32))
        with pytest.raises(odp.OdpError) as e:
            odp.batch_solve([g], [0.5])
        assert e.value.code == odp.EINVAL


# ---------------------------------------------------------------------------
# per-node dissipation (Algorithm 1's second loop) against the oracle
# ---------------------------------------------------------------------------

def per_node(problem):
    return dataclasses.replace(problem, dissipation="local")


LOCAL_CASES = [
    per_node(inputs.dubins3d()),                                          # 41x41x36, Euler, upwind
    per_node(inputs.dubins3d(n=(23, 19, 13), space_order=2, time_order=2)),
    per_node(inputs.dubinscar4d(n=(21, 19, 11, 16))),                    # ENO2 + RK2
    per_node(inputs.dubinscar4d(n=(17, 15, 9, 13), space_order=1, time_order=1)),  # partial segments
    per_node(inputs.rel6d(n=(9, 8, 10, 5, 4, 3), horizon=0.3)),           # upwind + RK2
    per_node(inputs.rel6d(n=(7, 7, 8, 3, 4, 3), space_order=2, horizon=0.2)),
]


@pytest.mark.parametrize("problem", LOCAL_CASES, ids=lambda p: "%s_o%d%d_local" % (
    p.name, p.space_order, p.time_order))
def test_per_node_dissipation_matches_oracle(problem):
    if problem.dynamics == "rel6d":
        # the per-node heading-rate alpha switches with the sign of p_theta, so
        # the whole solve is as sensitive to rounding as ENO2 (1e-7 relative
        # input noise moves the FP64 oracle by 5e-4 of the value range):
        # compared segment by segment at the same bar
        check_parity_resync(problem)
    else:
        check(problem)


def test_per_node_dissipation_changes_dubins_but_not_the_single_integrator():
    import torch

    def run(p):
        l = torch.from_numpy(p.target_values()).cuda()
        with odp.Grid.for_problem(p) as g:
            g.set_target(l)
            g.solve_problem(p)
            return g.readback(torch.empty_like(l)).cpu().numpy()

    si = inputs.single_integrator((29, 27, 13), horizon=0.6)
    assert np.array_equal(run(si), run(per_node(si)))
    d3 = inputs.dubins3d(n=(25, 23, 20), horizon=0.8)
    assert np.abs(run(d3) - run(per_node(d3))).max() > 1e-4


def test_per_node_dissipation_full_size_step_matches_oracle():
    p = per_node(inputs.dubinscar4d())
    rel, _, _ = steps_at_full_size(p, (0.5,), "per-node dissipation full size, step")
    assert rel <= REL_TOL


def test_batch_refuses_per_node_dissipation():
    p = inputs.dubins3d(n=(9, 9, 8))
    with odp.Grid.for_problem(per_node(p)) as g:
        g.set_target(p.target_values())
        with pytest.raises(odp.OdpError) as e:
            odp.batch_solve([g], [0.5])
        assert e.value.code == odp.EINVAL


# ---------------------------------------------------------------------------
# the pursuit-evasion capture model of Section 4.2 (coupled switching
# function; every alpha component reduced per stage)
# ---------------------------------------------------------------------------

CAPTURE_CASES = [
    inputs.dubins_capture(),                                              # 40^3, the paper's grid, T = 1.5
    inputs.dubins_capture(n=(21, 23, 18), space_order=2, time_order=2, horizon=0.5),
    inputs.dubins_capture(n=(25, 25, 20), u_mode="min", d_mode="max", set_kind="brs", horizon=0.5),
    inputs.reach_avoid(inputs.dubins_capture(n=(31, 29, 24), horizon=0.8),
                       inputs.cylinder_obstacle(0.6, center=(1.5, 0.0))),
]


@pytest.mark.parametrize("problem", CAPTURE_CASES, ids=lambda p: "%s_o%d%d_%s_%s" % (
    p.name, p.space_order, p.time_order, p.set_kind, p.u_mode))
def test_capture_model_matches_oracle(problem):
    check(problem)


CAPTURE_LOCAL_CASES = [
    per_node(inputs.dubins_capture()),                                    # 40^3, the paper's grid, T = 1.5
    per_node(inputs.dubins_capture(n=(21, 23, 18), space_order=2, time_order=2, horizon=0.5)),
    per_node(inputs.dubins_capture(n=(25, 25, 20), u_mode="min", d_mode="max", set_kind="brs", horizon=0.5)),
    per_node(inputs.dubins_capture(n=(13, 3, 10), horizon=0.4)),          # 3 rows: the row-blocked pass
]


@pytest.mark.parametrize("problem", CAPTURE_LOCAL_CASES, ids=lambda p: "%s_o%d%d_%s_local" % (
    p.name, p.space_order, p.time_order, p.u_mode))
def test_capture_model_per_node_dissipation_matches_oracle(problem):
    # Algorithm 1's second loop on the coupled-switching model of Section
    # 4.2: each node's alpha_i from interval bounds of y p_x - x p_y - p_th
    # over its derivative box (reading R20).  The per-node bound switches
    # with the signs of those intervals, a discontinuity like ENO2's, so the
    # run is compared step by step (one-step segments) at the 1e-4 bar.
    check_parity_resync(problem)


def test_capture_model_per_node_dissipation_is_refused_by_the_batch():
    p = inputs.dubins_capture(n=(9, 9, 8))
    with odp.Grid.for_problem(per_node(p)) as g:
        g.set_target(p.target_values())
        with pytest.raises(odp.OdpError) as e:
            odp.batch_solve([g], [0.5])
        assert e.value.code == odp.EINVAL


# ---------------------------------------------------------------------------
# the two stage-pass kernels (plane-streaming, bulk-staged) compute the same
# per-node arithmetic: bit-identical values and step counts
# ---------------------------------------------------------------------------

PASS_CASES = [
    inputs.dubinscar4d(n=(21, 19, 11, 16)),                              # ENO2 + RK2, edge CTAs on x
    inputs.dubins3d(),                                                    # upwind + Euler, 41x41x36
    inputs.dubinscar4d(n=(13, 13, 7, 12), u_mode="max", set_kind="brs"),
    inputs.rel6d(n=(7, 7, 8, 4, 4, 4), space_order=2, horizon=0.2),
    inputs.rel6d(n=(6, 5, 8, 5, 4, 8), horizon=0.2),                      # upwind + RK2, periodic outer axis
    inputs.reach_avoid(inputs.dubinscar4d(n=(21, 19, 11, 16), horizon=1.0), inputs.dubins_obstacle()),
    inputs.dubinscar4d(),                                                 # 80x80x40x64
    inputs.rel6d(),                                                       # 24^6
]


@pytest.mark.parametrize("problem", PASS_CASES, ids=lambda p: "%s_o%d%d" % (p.name, p.space_order, p.time_order))
def test_bulk_and_plane_passes_agree_bit_for_bit(problem):
    import torch

    l_dev = torch.from_numpy(problem.target_values()).cuda()
    out = []
    for pass_ in (1, 2):
        with odp.Grid.for_problem(problem) as g:
            odp.set_stage_pass(g.handle, pass_)
            g.set_target(l_dev)
            st = g.solve_problem(problem, stats=True)
            out.append((st["steps"], g.readback(torch.empty_like(l_dev)).cpu().numpy()))
    assert out[0][0] == out[1][0] > 0
    assert np.array_equal(out[0][1], out[1][1])


def test_bulk_pass_is_refused_where_it_does_not_apply():
    p = inputs.dubins3d(n=(23, 19, 13))       # last axis not a multiple of 4 nodes
    with odp.Grid.for_problem(p) as g:
        with pytest.raises(odp.OdpError) as e:
            odp.set_stage_pass(g.handle, 2)
        assert e.value.code == odp.EINVAL
        odp.set_stage_pass(g.handle, 1)
        odp.set_stage_pass(g.handle, 0)
        with pytest.raises(odp.OdpError):
            odp.set_stage_pass(g.handle, 3)
