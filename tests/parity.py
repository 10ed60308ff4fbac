"""Whole-solve parity against the FP64 oracle, shared by the GPU tests.

First-order (upwind) solves are held to 1e-4 of the value range.  Second-
order ENO solves are held to twice the oracle's own sensitivity to
float32-level changes of its data (`oracle_sensitivity`): ENO2's stencil
choice (paper Section 3.1.4) is discontinuous, and the FP64 oracle itself
moves by 0.4e-4 to 6e-4 of the range when its values are rounded to float32
after every step or its target is perturbed by 1e-7 relative.
"""
from __future__ import annotations

import numpy as np

import oracle
import parity_log

REL_TOL = 1e-4


def oracle_f32_storage(problem, l):
    """The oracle's whole solve driven one step at a time with its value
    rounded to float32 after every step (the GPU's storage precision).  For
    models whose alpha does not depend on the value (every step the CFL
    step but the last, clipped to the horizon)."""
    dz = oracle.spacing(problem.n, problem.lo, problem.hi, problem.periodic)
    alpha = oracle.terms(problem, l)["alpha"]
    dt = problem.cfl / float(np.sum(alpha / dz))
    T = float(problem.tau[-1])
    phi, t, steps = l.astype(np.float64), 0.0, 0
    while T - t > 1e-12 * T:
        h = min(dt, T - t)
        phi = oracle.step(problem, phi, h, l=l)["out"].astype(np.float32).astype(np.float64)
        t = T if h == T - t else t + h
        steps += 1
    return phi, steps


def oracle_sensitivity(problem, ref):
    """How far float32 storage and a target perturbed by 1e-7 relative move
    the oracle's solve `ref`: (max over the value range for each, then the
    fraction of nodes each moves by more than 1e-4 of the range)."""
    l = problem.target_values()
    rng_l = float(l.max() - l.min())
    a, steps = oracle_f32_storage(problem, l)
    assert steps == int(ref["steps"].sum())
    noise = np.random.default_rng(0).standard_normal(l.shape)
    b = oracle.solve(problem, l=l.astype(np.float64) * (1.0 + 1e-7 * noise))["final"]
    da = np.abs(a.reshape(-1) - ref["final"].reshape(-1))
    db = np.abs(b.reshape(-1) - ref["final"].reshape(-1))
    tol = REL_TOL * rng_l
    return (float(da.max()) / rng_l, float(db.max()) / rng_l,
            float((da > tol).mean()), float((db > tol).mean()))


def check_whole_solve(problem, v, steps, ref=None, spread=None, name=None):
    """GPU result `v` after `steps` steps against the oracle's whole solve:
    the 1e-4 bar for upwind, twice the oracle's own sensitivity (measured
    here unless given) for ENO2, and equal step counts.  Returns the error
    over the value range."""
    if ref is None:
        ref = oracle.solve(problem)
    l = problem.target_values()
    rng_l = float(l.max() - l.min())
    tol = REL_TOL * rng_l
    assert steps == int(ref["steps"].sum()), (steps, ref["steps"])
    d = np.abs(v - ref["final"].reshape(v.shape))
    err = float(d.max()) / rng_l
    if problem.space_order == 1:
        parity_log.note(name or problem.name, "whole solve, %d steps: max err/range %.2e" % (steps, err))
        assert err <= REL_TOL, err
        return err
    if spread is None:
        spread = oracle_sensitivity(problem, ref)
    frac = float((d > tol).mean())
    frac_bar = max(0.01, 2.0 * max(spread[2:])) if len(spread) > 2 else 0.01
    parity_log.note(name or problem.name, "whole solve, %d steps: max err/range %.2e; oracle's own "
                    "sensitivity %.2e (float32 storage) / %.2e (target 1e-7); nodes over 1e-4: %.4f%% "
                    "(bar %.2f%%)" % (steps, err, spread[0], spread[1], 100 * frac, 100 * frac_bar))
    assert err <= max(REL_TOL, 2.0 * max(spread[:2])), (err, spread)
    assert frac <= frac_bar, (frac, frac_bar)
    return err
