"""Pins of the oracle's time-to-reach sweeping (Section 2.2, Algorithm 2).

Each test checks the oracle against something it does not compute itself:
the exact discrete solution of the 1-D problem (cells to the target times
h / v) and the sweep counts that Gauss-Seidel and Jacobi orders need for it,
the closed-form Chebyshev distance of the box-input integrator in 2-D and its
convergence under refinement, the reachable tube of the time-dependent
method (Algorithm 1, a different algorithm) at two horizons, the uniqueness
of the limit when no boundary rule takes part (periodic axes), and the
invariants of the time-to-reach function.  A plausible mistake in the update
(a dropped constant, a wrong sign of H, a wrong sigma or c, a wrong average of
the neighbours), in the boundary rule or in the sweep order fails one of them.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2204_05520_gb300 import inputs


def chebyshev_square(n, half_width=2.0, side=0.5, u_max=1.0):
    p = inputs.single_integrator(n, half_width=half_width, u_max=u_max)
    return dataclasses.replace(
        p, target=lambda m: np.max(np.stack([np.abs(c) for c in m]), axis=0) - side)


def test_ttr_1d_exact_discrete_solution():
    # x' = u, |u| <= v: the Lax-Friedrichs fixed point is min(neighbours) + h/v,
    # i.e. (cells to the nearest target node) * h / v, boundary nodes included
    # (the extrapolation is exact on a linear profile).
    v = 1.5
    p = inputs.single_integrator((41,), half_width=2.0, u_max=v, radius=0.5)
    l = p.target_values().astype(np.float64)
    h = 4.0 / 40
    tgt = np.flatnonzero(l <= 0)
    cells = np.array([np.min(np.abs(i - tgt)) for i in range(41)])
    expect = cells * h / v
    gs = oracle.ttr(p)
    assert np.max(np.abs(gs["phi"] - expect)) < 1e-10
    # ascending sweep fixes the right side, descending the left, one more
    # sweep sees no change
    assert gs["sweeps"] == 3
    jac = oracle.ttr(p, scheme="jacobi")
    assert np.max(np.abs(jac["phi"] - expect)) < 1e-10
    # Jacobi moves the front one cell per sweep: the farthest interior node
    # is exact after cells.max()-1 sweeps (the boundary node with it), and
    # one more sweep sees no change
    assert jac["sweeps"] == cells[1:-1].max() + 1


def test_ttr_1d_offcentre_target_and_speed():
    v = 0.5
    p = inputs.single_integrator((33,), half_width=1.0, u_max=v)
    p = dataclasses.replace(p, target=lambda m: np.abs(m[0] - 0.55) - 0.1)
    l = p.target_values().astype(np.float64)
    h = 2.0 / 32
    tgt = np.flatnonzero(l <= 0)
    cells = np.array([np.min(np.abs(i - tgt)) for i in range(33)])
    r = oracle.ttr(p)
    assert np.max(np.abs(r["phi"] - cells * h / v)) < 1e-10


def test_ttr_2d_chebyshev_distance():
    # box input |u_d| <= 1 and a square target [-s, s]^2: the time to reach is
    # the Chebyshev distance max(|x| - s, |y| - s)^+.  Away from the diagonals
    # the Lax-Friedrichs solution converges faster than h; along them (the
    # ridge of the exact solution) the error decays like sqrt(h).
    errs_off, errs_max = [], []
    for n in (41, 81, 161):
        p = chebyshev_square((n, n))
        r = oracle.ttr(p)
        X, Y = np.meshgrid(*p.nodes(), indexing="ij")
        exact = np.maximum(np.maximum(np.abs(X), np.abs(Y)) - 0.5, 0.0)
        err = np.abs(r["phi"] - exact)
        h = 4.0 / (n - 1)
        off = (np.abs(np.abs(X) - np.abs(Y)) > 0.5) & (np.abs(X) < 1.5) & (np.abs(Y) < 1.5)
        errs_off.append(err[off].max())
        errs_max.append(err.max())
        assert err.max() <= 0.75 * np.sqrt(h)
        assert np.all(r["phi"][p.target_values() <= 0] == 0.0)
    assert errs_off[1] < 0.5 * errs_off[0] and errs_off[2] < 0.5 * errs_off[1]
    assert errs_off[2] < 1e-3
    assert errs_max[2] < errs_max[1] < errs_max[0]


def test_ttr_matches_time_dependent_tube():
    # {TTR <= T} is the backward reachable tube of horizon T, which Algorithm 1
    # computes by a different method; the two first-order approximations may
    # disagree only next to the tube's boundary.
    p = inputs.dubins3d(n=(41, 41, 36), tau=(0.0, 1.0, 2.0))
    h = 8.0 / 40
    ttr = oracle.ttr(p)["phi"]
    hj = oracle.solve(p, snapshots=True)["snapshots"]
    for k, T in ((1, 1.0), (2, 2.0)):
        V = hj[k]
        tube, sub = V <= 0, ttr <= T
        dis = tube != sub
        assert dis.sum() <= 0.08 * tube.sum()
        assert np.abs(V[dis]).max() <= 0.75 * h
    # the tube grows with T and TTR is 0 exactly on the target
    assert np.all(ttr[p.target_values() <= 0] == 0.0)
    assert (ttr <= 1.0).sum() < (ttr <= 2.0).sum()


def test_ttr_limit_is_order_independent_without_boundaries():
    # On a torus no boundary extrapolation takes part and the update is
    # monotone in the neighbours, so Gauss-Seidel (any direction pattern) and
    # Jacobi sweeps both decrease to the same largest fixed point.
    p = chebyshev_square((24, 24), half_width=2.0, side=0.6)
    p = dataclasses.replace(p, periodic=(True, True))
    gs = oracle.ttr(p, eps=1e-12)
    jac = oracle.ttr(p, eps=1e-12, scheme="jacobi")
    assert gs["rc"] == 0 and jac["rc"] == 0
    assert np.max(np.abs(gs["phi"] - jac["phi"])) < 1e-9
    assert jac["sweeps"] > gs["sweeps"]
    # the limit is unique, so it has the symmetries of the problem although no
    # sweep order has them: x <-> y and x -> -x (node i <-> (n - i) mod n)
    phi = gs["phi"]
    mirror = phi[(-np.arange(24)) % 24, :]
    assert np.max(np.abs(phi - phi.T)) < 1e-9
    assert np.max(np.abs(phi - mirror)) < 1e-9


def test_ttr_monotone_in_tolerance_and_bounded():
    p = inputs.dubins3d(n=(25, 25, 24))
    loose = oracle.ttr(p, eps=1e-2)["phi"]
    tight = oracle.ttr(p, eps=1e-7)["phi"]
    # sweeps only lower values: a later iterate is below an earlier one
    assert np.all(tight <= loose + 1e-12)
    assert np.all(tight >= 0.0) and tight.max() < 1e4


def test_ttr_big_value_and_sweep_cap():
    p = inputs.dubins3d(n=(25, 25, 24))
    r = oracle.ttr(p, max_sweeps=4, raise_on_error=False)
    assert r["rc"] == oracle.ETIMEOUT and r["sweeps"] == 4 and r["change"] > 1e-5
    # after one sweep a node far from the target still holds the initial value
    one = oracle.ttr(p, max_sweeps=1, big=123.0, raise_on_error=False)
    assert one["phi"].max() == 123.0


@pytest.mark.parametrize("bad", ["umode", "small_axis", "scheme"])
def test_ttr_refusals(bad):
    p = inputs.dubins3d(n=(25, 25, 24))
    if bad == "umode":
        p = dataclasses.replace(p, u_mode="max")
    elif bad == "small_axis":
        p = dataclasses.replace(p, n=(25, 3, 24))
    with pytest.raises((oracle.OracleError, KeyError)) as e:
        oracle.ttr(p, scheme="red_black" if bad == "scheme" else "gauss_seidel")
    if bad != "scheme":
        assert e.value.code == oracle.EINVAL


def _sweep_by_hand(p, phi, k):
    """Sweep k of Algorithm 2 enumerated here from its statement: nested
    loops over the axes in C order, axis d descending when bit d of
    k mod 2^ndim is set (Section 5.3), in-place updates of the interior
    nodes, then the boundary rule axis by axis, lower face then upper face."""
    import itertools

    nd = len(p.n)
    dirs = k % (1 << nd)
    ranges = [range(p.n[d] - 1, -1, -1) if (dirs >> d) & 1 else range(p.n[d]) for d in range(nd)]
    for idx in itertools.product(*ranges):
        if any(not p.periodic[d] and idx[d] in (0, p.n[d] - 1) for d in range(nd)):
            continue
        phi[idx] = min(oracle.ttr_node(p, phi, idx), phi[idx])
    for d in range(nd):
        if p.periodic[d]:
            continue
        for b, s in ((0, 1), (p.n[d] - 1, -1)):
            face = [slice(None)] * nd
            f0 = list(face); f0[d] = b
            f1 = list(face); f1[d] = b + s
            f2 = list(face); f2[d] = b + 2 * s
            e = np.maximum(2.0 * phi[tuple(f1)] - phi[tuple(f2)], phi[tuple(f2)])
            phi[tuple(f0)] = np.minimum(e, phi[tuple(f0)])


@pytest.mark.parametrize("case", ["si2", "dubins3d"])
def test_ttr_sweep_order_matches_enumeration(case):
    # The iterate after k sweeps (the loop cut off by the sweep cap) equals a
    # hand enumeration of the paper's order, bit for bit: this pins the
    # direction pattern, the in-place update and the boundary order.
    if case == "si2":
        p = chebyshev_square((7, 6), half_width=1.5, side=0.4)
    else:
        p = inputs.dubins3d(n=(6, 5, 8), lo=(-2.0, -2.0, -np.pi), hi=(2.0, 2.0, np.pi), radius=0.7)
    l = p.target_values().astype(np.float64)
    phi = np.where(l <= 0, 0.0, 1e4)
    for k in range(6):
        _sweep_by_hand(p, phi, k)
        r = oracle.ttr(p, max_sweeps=k + 1, eps=0.0, raise_on_error=False)
        assert r["sweeps"] == k + 1
        assert np.array_equal(r["phi"], phi), "sweep %d" % k


@pytest.mark.parametrize("case", ["si3", "dubins3d", "dubinscar4d"])
def test_ttr_update_equals_its_upwind_weighted_form(case):
    # With sigma_d = |f_d(z, u*, d*)| each axis's Lax-Friedrichs part equals
    # |f_d| / h_d times the neighbour the flow points to (the smaller one on
    # an input axis), so Algorithm 2's update equals
    # (1 + sum_d w_d phi_nb(d)) / sum_d w_d, w_d = |f_d| / h_d -- the
    # cancellation-free form the CUDA kernel evaluates.  Checked here in
    # float64 against the oracle's printed form at random nodes of random
    # fields.
    rng = np.random.Generator(np.random.PCG64(11))
    if case == "si3":
        p = chebyshev_square((7, 8, 9), u_max=1.3)
    elif case == "dubins3d":
        p = inputs.dubins3d(n=(9, 8, 12), v=1.4, w_max=0.7)
    else:
        p = inputs.dubinscar4d(n=(7, 6, 5, 8), a_max=0.8, w_max=1.2)
    nd = p.ndim
    dz = [(p.hi[d] - p.lo[d]) / (p.n[d] if p.periodic[d] else p.n[d] - 1) for d in range(nd)]
    axes = p.nodes()
    for _ in range(40):
        phi = rng.uniform(0.0, 10.0, size=p.n)
        idx = tuple(int(rng.integers(0 if p.periodic[d] else 1, p.n[d] if p.periodic[d] else p.n[d] - 1))
                    for d in range(nd))
        up, dn = [], []
        for d in range(nd):
            i_up, i_dn = list(idx), list(idx)
            i_up[d] = (idx[d] + 1) % p.n[d]
            i_dn[d] = (idx[d] - 1) % p.n[d]
            up.append(phi[tuple(i_up)])
            dn.append(phi[tuple(i_dn)])
        # flow components and which axes a bounded input drives
        if case == "si3":
            drift, inp = [None] * nd, [p.params[0]] * nd
        elif case == "dubins3d":
            th = axes[2][idx[2]]
            drift = [p.params[0] * np.cos(th), p.params[0] * np.sin(th), None]
            inp = [None, None, p.params[1]]
        else:
            v, th = axes[2][idx[2]], axes[3][idx[3]]
            drift = [v * np.cos(th), v * np.sin(th), None, None]
            inp = [None, None, p.params[0], p.params[1]]
        num, den = 1.0, 0.0
        for d in range(nd):
            if inp[d] is not None:
                w, nb = inp[d] / dz[d], min(up[d], dn[d])
            else:
                w, nb = abs(drift[d]) / dz[d], (up[d] if drift[d] >= 0 else dn[d])
            num += w * nb
            den += w
        got = oracle.ttr_node(p, phi, idx)
        assert abs(got - num / den) <= 1e-12 * max(1.0, abs(got)), (idx, got, num / den)


def _tiled_sweep(p, phi, k, rng):
    """Sweep k in the order the CUDA kernel uses: direction-mapped
    coordinates y (y_d = x_d, or n_d - 1 - x_d on a descending axis), tiles
    of up to 8 nodes per axis (a periodic axis keeps two tiles at least),
    tile hyperplanes in increasing tile-coordinate sum (tiles of one
    hyperplane in random order), inside a tile its own hyperplanes in
    increasing local sum (nodes of one hyperplane in random order); then the
    boundary rule.  Updates use the oracle's per-node value."""
    import itertools

    nd = len(p.n)
    dirs = k % (1 << nd)
    T = [max(1, min(8, p.n[d], p.n[d] // 2 if p.periodic[d] else p.n[d])) for d in range(nd)]
    NT = [(p.n[d] + T[d] - 1) // T[d] for d in range(nd)]
    tiles = list(itertools.product(*[range(m) for m in NT]))
    for S in range(sum(m - 1 for m in NT) + 1):
        plane = [t for t in tiles if sum(t) == S]
        rng.shuffle(plane)
        for t in plane:
            local = list(itertools.product(*[range(T[d]) for d in range(nd)]))
            for s in range(sum(x - 1 for x in T) + 1):
                level = [a for a in local if sum(a) == s]
                rng.shuffle(level)
                for a in level:
                    y = [t[d] * T[d] + a[d] for d in range(nd)]
                    if any(y[d] >= p.n[d] for d in range(nd)):
                        continue
                    x = tuple(p.n[d] - 1 - y[d] if (dirs >> d) & 1 else y[d] for d in range(nd))
                    if any(not p.periodic[d] and x[d] in (0, p.n[d] - 1) for d in range(nd)):
                        continue
                    phi[x] = min(oracle.ttr_node(p, phi, x), phi[x])
    for d in range(nd):
        if p.periodic[d]:
            continue
        for b, s in ((0, 1), (p.n[d] - 1, -1)):
            f0 = [slice(None)] * nd
            f1, f2 = list(f0), list(f0)
            f0[d], f1[d], f2[d] = b, b + s, b + 2 * s
            e = np.maximum(2.0 * phi[tuple(f1)] - phi[tuple(f2)], phi[tuple(f2)])
            phi[tuple(f0)] = np.minimum(e, phi[tuple(f0)])


@pytest.mark.parametrize("case", ["dubins3d", "periodic2d"])
def test_ttr_tiled_hyperplane_order_equals_sequential_sweep(case):
    # Every neighbour a sequential sweep has already updated lies on the
    # previous hyperplane of y, every other one on the next; so the tiled
    # hyperplane walk of the CUDA kernel gives each node the same neighbour
    # values, and the iterates agree bit for bit.
    rng = np.random.Generator(np.random.PCG64(3))
    if case == "dubins3d":
        p = inputs.dubins3d(n=(11, 9, 18), lo=(-2.0, -2.0, -np.pi), hi=(2.0, 2.0, np.pi), radius=0.8)
    else:
        p = chebyshev_square((19, 10), half_width=1.5, side=0.3)
        p = dataclasses.replace(p, periodic=(True, False))
    l = p.target_values().astype(np.float64)
    phi = np.where(l <= 0, 0.0, 1e4)
    for k in range(5):
        _tiled_sweep(p, phi, k, rng)
        r = oracle.ttr(p, max_sweeps=k + 1, eps=0.0, raise_on_error=False)
        assert np.array_equal(r["phi"], phi), "sweep %d" % k
