"""Pins of the oracle's computation methods (Section 4.3's table, reading R27).

Checked against facts outside the methods' own code: with a time-invariant
target the three "min" target methods coincide with the BRT and "None" with
the BRS; every "max" method is the mirror of its "min" twin (phi -> -phi with
the input roles swapped turns one scheme into the other, operation for
operation, so the two solves agree to rounding); and on exact 1-D transport
(upwind, CFL 1: one cell per step) the "value over time" methods give the
running minimum / maximum of the shifted target, a closed form.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2204_05520_gb300 import inputs

FLIP = {"min": "max", "max": "min"}


def _mirror(p):
    return dataclasses.replace(p, u_mode=FLIP[p.u_mode], d_mode=FLIP[p.d_mode])


def _cylinders(p, centers, radius):
    mesh = np.meshgrid(*p.nodes(), indexing="ij")
    return np.stack([(np.sqrt((mesh[0] - cx) ** 2 + (mesh[1] - cy) ** 2) - radius).astype(np.float32)
                     .astype(np.float64) for cx, cy in centers])


def test_min_target_methods_are_the_tube_and_none_is_the_set():
    p = inputs.dubins3d(n=(21, 21, 16), tau=(0.0, 0.4, 0.8))
    l = p.target_values().astype(np.float64)
    brt = oracle.solve(p, l=l)["final"]
    brs = oracle.solve(dataclasses.replace(p, set_kind="brs"), l=l)["final"]
    for m in ("minVWithVTarget", "minVWithV0"):
        assert np.array_equal(oracle.solve_methods(p, m, l=l)["final"], brt)
    assert np.array_equal(oracle.solve_methods(p, "None", l=l)["final"], brs)
    # the value over time of the tube never rises above its start
    v = oracle.solve_methods(p, "minVWithVInit", l=l, snapshots=True)["snapshots"]
    assert np.all(v[1] <= v[0]) and np.all(v[2] <= v[1])


MIRROR_CASES = {
    "dubins3d_upwind_rk2": lambda: inputs.dubins3d(n=(21, 19, 16), tau=(0.0, 0.3, 0.6), time_order=2),
    "capture_upwind_euler": lambda: inputs.dubins_capture(n=(17, 17, 16), tau=(0.0, 0.25, 0.5)),
    "dubinscar4d_eno2_rk2": lambda: inputs.dubinscar4d(n=(11, 10, 7, 12), tau=(0.0, 0.2, 0.4)),
}


@pytest.mark.parametrize("case", sorted(MIRROR_CASES))
@pytest.mark.parametrize("pair", [("maxVWithV0", "minVWithV0"), ("maxVWithVTarget", "minVWithVTarget"),
                                  ("maxVWithVInit", "minVWithVInit")])
def test_max_methods_mirror_min_methods(case, pair):
    p = MIRROR_CASES[case]()
    k = len(p.tau)
    ls = _cylinders(p, [(0.4 * i, -0.2 * i) for i in range(k)], 0.8)
    gs = _cylinders(p, [(2.0 - 0.2 * i, 0.5) for i in range(k)], 0.6)
    mx, mn = pair
    a = oracle.solve_methods(p, mx, "minVWithObstacle", l_seq=ls, g_seq=gs)
    b = oracle.solve_methods(_mirror(p), mn, "maxVWithObstacle", l_seq=-ls, g_seq=-gs)
    span = ls.max() - ls.min()
    assert np.array_equal(a["steps"], b["steps"])
    assert np.abs(a["final"] + b["final"]).max() <= 1e-12 * span


def test_value_over_time_on_exact_transport():
    # x' = c, upwind at CFL 1: every step moves phi one cell (phi_i <- phi_i+1),
    # so after n steps the "value over time" methods hold the running min / max
    # of the target over shifts 0 .. n
    n, steps = 64, 7
    h = 2 * np.pi / n
    p = inputs.advection((n,), velocity=(1.0,), freqs=(2,), horizon=steps * h, cfl=1.0)
    l = p.target_values().astype(np.float64)
    shifts = np.stack([np.roll(l, -j) for j in range(steps + 1)])
    lo = oracle.solve_methods(p, "minVWithVInit", l=l)
    hi = oracle.solve_methods(p, "maxVWithVInit", l=l)
    assert int(lo["steps"].sum()) == steps
    assert np.abs(lo["final"] - shifts.min(axis=0)).max() < 1e-9
    assert np.abs(hi["final"] - shifts.max(axis=0)).max() < 1e-9
    # for pure transport the tube with phi(0) is the same running minimum
    v0 = oracle.solve_methods(p, "minVWithV0", l=l)["final"]
    assert np.abs(v0 - shifts.min(axis=0)).max() < 1e-9


def test_unknown_method_is_refused():
    p = inputs.dubins3d(n=(11, 11, 8))
    with pytest.raises(KeyError):
        oracle.solve_methods(p, "minVWithEverything")
