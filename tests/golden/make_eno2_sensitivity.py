#!/usr/bin/env python
"""Writes eno2_sensitivity.txt: how far the FP64 oracle's own whole solve
moves under float32-level changes of its data, for the full-size
second-order (ENO2 + TVD-RK2) DubinsCar4D workload.

ENO2's stencil choice (paper Section 3.1.4) is discontinuous, so a whole
ENO2 solve is sensitive to rounding of the stored values.  Two measures,
both from the oracle alone (this script calls only `oracle/` and the seeded
input generators):

* f32store: the oracle's solve with its value rounded to float32 after every
  time step (the storage precision of the GPU path), against the plain FP64
  solve;
* lpert:    the oracle's solve from the target perturbed by 1e-7 relative
  (seeded normal noise, seed 0), against the plain solve.

Each is max |difference| / (max l - min l), with the fraction of nodes whose
difference is above 1e-4 of the range.  The GPU parity test of the
full-size solve holds the GPU to twice the larger of the two maxima, and its
fraction of nodes over 1e-4 to twice the larger fraction (at least 1%).

    python tests/golden/make_eno2_sensitivity.py   # about 40 min on 8 cores
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2204_05520_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "eno2_sensitivity.txt")


def solve_f32_storage(p, l):
    """The oracle's time loop driven one step at a time, rounding the value
    to float32 between steps (alpha is static for this model, so every step
    is the CFL step but the last, which is clipped to the horizon)."""
    dz = oracle.spacing(p.n, p.lo, p.hi, p.periodic)
    alpha = oracle.terms(p, l)["alpha"]
    dt = p.cfl / float(np.sum(alpha / dz))
    T = float(p.tau[-1])
    phi = l.astype(np.float64)
    t, steps = 0.0, 0
    while T - t > 1e-12 * T:
        h = min(dt, T - t)
        phi = oracle.step(p, phi, h, l=l)["out"].astype(np.float32).astype(np.float64)
        t = T if h == T - t else t + h
        steps += 1
    return phi, steps


def main():
    p = inputs.dubinscar4d()
    l = p.target_values()
    rng = float(l.max() - l.min())
    t0 = time.time()
    ref = oracle.solve(p)
    a, steps = solve_f32_storage(p, l)
    assert steps == int(ref["steps"].sum()), (steps, ref["steps"])
    noise = np.random.default_rng(0).standard_normal(l.shape)
    b = oracle.solve(p, l=l.astype(np.float64) * (1.0 + 1e-7 * noise))["final"]
    da = np.abs(a - ref["final"])
    db = np.abs(b - ref["final"])
    f32store = float(da.max()) / rng
    lpert = float(db.max()) / rng
    fa = float((da > 1e-4 * rng).mean())
    fb = float((db > 1e-4 * rng).mean())
    with open(OUT, "w") as fh:
        fh.write("# Sensitivity of the FP64 oracle's whole solve to float32-level changes\n")
        fh.write("# (written by make_eno2_sensitivity.py from the oracle alone; %d threads, %.0f s)\n"
                 % (oracle.num_threads(), time.time() - t0))
        fh.write("# workload | steps | f32store | lpert | f32store nodes > 1e-4 | lpert nodes > 1e-4\n")
        fh.write("#   (max |dV| / value range, then fractions of the nodes)\n")
        fh.write("%s | %d | %.6g | %.6g | %.6g | %.6g\n" % (p.name, steps, f32store, lpert, fa, fb))
    print(open(OUT).read())


if __name__ == "__main__":
    main()
