"""Pins of the oracle's time-varying target and obstacle sets (reading R26:
the steps of segment (tau_k, tau_k+1] take their post-step min / max with the
sets sampled at tau_k+1; phi starts from the set at tau_0).

Checked against facts outside the reading's own code: a constant schedule is
the time-invariant solve, a target that leaves after tau_0 gives the plain
reachable set (BRS), a schedule over three taus is two chained one-segment
solves (which fixes the index convention), and a larger target schedule never
gives a smaller value (the comparison principle of the monotone scheme).
"""
import dataclasses

import numpy as np

import oracle
from paper_2204_05520_gb300 import inputs


def _cylinders(p, centers, radius=0.9):
    mesh = np.meshgrid(*p.nodes(), indexing="ij")
    out = []
    for cx, cy in centers:
        v = np.sqrt((mesh[0] - cx) ** 2 + (mesh[1] - cy) ** 2) - radius
        out.append(v.astype(np.float32).astype(np.float64))
    return np.stack(out)


def _problem(tau):
    return inputs.dubins3d(n=(25, 25, 16), tau=tau)


def test_constant_schedule_is_the_static_solve():
    p = _problem((0.0, 0.4, 0.9))
    l = p.target_values().astype(np.float64)
    g = _cylinders(p, [(2.0, 0.5)], radius=0.6)[0]
    ref = oracle.solve(p, l=l, g=g)
    got = oracle.solve(p, l_seq=np.stack([l] * 3), g_seq=np.stack([g] * 3))
    assert np.array_equal(got["final"], ref["final"])
    assert np.array_equal(got["steps"], ref["steps"])


def test_target_leaving_after_tau0_gives_the_reachable_set():
    p = _problem((0.0, 0.3, 0.7))
    l = p.target_values().astype(np.float64)
    far = np.full_like(l, 1e6)
    got = oracle.solve(p, l_seq=np.stack([l, far, far]))
    brs = oracle.solve(dataclasses.replace(p, set_kind="brs"), l=l)
    assert np.array_equal(got["final"], brs["final"])


def test_three_tau_schedule_is_two_chained_solves():
    tau = (0.0, 0.35, 0.8)
    p = _problem(tau)
    ls = _cylinders(p, [(0.0, 0.0), (0.6, 0.2), (1.2, 0.4)])
    gs = _cylinders(p, [(2.5, 0.0), (2.2, 0.3), (1.9, 0.6)], radius=0.5)
    got = oracle.solve(p, l_seq=ls, g_seq=gs, snapshots=True)
    # segment 0: start from l_0, sets l_1 / g_1
    a = oracle.solve(dataclasses.replace(p, tau=(0.0, tau[1])), l=ls[1], g=gs[1], phi0=ls[0])
    # segment 1: start from segment 0's end, sets l_2 / g_2
    b = oracle.solve(dataclasses.replace(p, tau=(0.0, tau[2] - tau[1])), l=ls[2], g=gs[2], phi0=a["final"])
    span = ls.max() - ls.min()
    assert got["steps"][0] == a["steps"][0] and got["steps"][1] == b["steps"][0]
    assert np.abs(got["snapshots"][1] - a["final"]).max() <= 1e-12 * span
    assert np.abs(got["final"] - b["final"]).max() <= 1e-10 * span
    # the sets do bind: the result differs from holding the first target
    held = oracle.solve(p, l=ls[0], g=gs[0])
    assert np.abs(got["final"] - held["final"]).max() > 0.05


def test_larger_target_schedule_never_gives_a_smaller_value():
    p = _problem((0.0, 0.3, 0.6, 0.9))
    ls = _cylinders(p, [(0.0, 0.0), (0.4, 0.0), (0.8, 0.1), (1.0, 0.3)])
    bump = 0.2 * np.abs(np.sin(np.meshgrid(*p.nodes(), indexing="ij")[0]))
    lo = oracle.solve(p, l_seq=ls)["final"]
    hi = oracle.solve(p, l_seq=ls + bump[None])["final"]
    assert np.all(hi >= lo - 1e-12)
    assert np.any(hi > lo + 1e-6)
