"""Time-to-reach sweeping on the GPU (FP32, through the C ABI) against the
FP64 oracle (Algorithm 2).

Criterion: max |phi_gpu - phi_oracle| <= 1e-4 * (max phi - min phi) of the
oracle's converged function, with the same number of sweeps within 2% (at
least 2).  The GPU runs the paper's Gauss-Seidel order exactly (hyperplane
wavefronts), so the iterates are the oracle's up to rounding; only the sweep
at which the change first drops to eps can move, because the GPU's change is
a difference of float32 values whose spacing near the largest values (about
1e-6 for values near 8) is a tenth of eps, and a slowly contracting sweep
(ratio near 0.99) turns that into a shift of a few sweeps.  Small
grids span several tiles with ragged last tiles; full-size grids are checked
by the fixed-point property at sampled nodes.
"""
import dataclasses

import numpy as np
import pytest

import oracle
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


def square(n, side=0.5, half_width=2.0, u_max=1.0, periodic=None):
    p = inputs.single_integrator(n, half_width=half_width, u_max=u_max)
    p = dataclasses.replace(p, target=lambda m: np.max(np.stack([np.abs(c) for c in m]), axis=0) - side)
    if periodic is not None:
        p = dataclasses.replace(p, periodic=tuple(periodic))
    return p


def gpu_ttr(problem, eps=1e-5, big=1e4, max_sweeps=100000, host_loop=False, l=None):
    import torch

    l_host = problem.target_values() if l is None else l
    with odp.Grid.for_problem(problem) as g:
        if host_loop:
            odp.set_loop_mode(g.handle, True)
        g.set_target(torch.from_numpy(l_host).cuda())
        stats = g.solve_ttr(eps=eps, big=big, max_sweeps=max_sweeps, stats=True)
        out = torch.empty(problem.n, dtype=torch.float32, device="cuda")
        g.readback(out)
    return out.cpu().numpy(), stats


CASES = {
    "si1_41": lambda: inputs.single_integrator((41,), u_max=1.5),
    "si1_700": lambda: square((700,), side=0.3),
    "si2_45x70": lambda: square((45, 70)),
    "si2_periodic": lambda: square((33, 40), periodic=(True, False), side=0.6),
    "si3_19x23x29": lambda: square((19, 23, 29)),
    "si4_9x10x11x18": lambda: square((9, 10, 11, 18), side=0.8),
    "dubins3d_25x25x24": lambda: inputs.dubins3d(n=(25, 25, 24)),
    "dubins3d_41x41x36": lambda: inputs.dubins3d(n=(41, 41, 36)),
    "dubins3d_fast": lambda: inputs.dubins3d(n=(30, 34, 20), v=1.7, w_max=0.6, radius=0.8),
    "dubinscar4d_14x13x10x16": lambda: inputs.dubinscar4d(n=(14, 13, 10, 16)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_ttr_parity(name):
    p = CASES[name]()
    got, stats = gpu_ttr(p)
    ref = oracle.ttr(p)
    span = ref["phi"].max() - ref["phi"].min()
    err = np.abs(got - ref["phi"]).max()
    assert err <= REL_TOL * span, "max err %.3g > tol %.3g" % (err, REL_TOL * span)
    assert abs(stats["sweeps"] - ref["sweeps"]) <= max(2, 0.02 * ref["sweeps"]), (stats["sweeps"], ref["sweeps"])
    # the target keeps 0 exactly
    assert np.all(got[p.target_values() <= 0] == 0.0)
    assert stats["change"] <= 1e-5


def test_ttr_host_loop_identical():
    p = inputs.dubins3d(n=(25, 25, 24))
    a, sa = gpu_ttr(p)
    b, sb = gpu_ttr(p, host_loop=True)
    assert sa["sweeps"] == sb["sweeps"]
    assert np.array_equal(a, b)
    assert sb["launches"] == sa["launches"]


def test_ttr_sweep_cap_and_partial_iterate():
    # the iterate after a fixed number of sweeps (the cap) matches the
    # oracle's iterate after as many sweeps
    p = inputs.dubins3d(n=(25, 25, 24))
    with pytest.raises(odp.OdpError) as e:
        gpu_ttr(p, max_sweeps=7)
    assert e.value.code == odp.ETIMEOUT
    import torch

    with odp.Grid.for_problem(p) as g:
        g.set_target(torch.from_numpy(p.target_values()).cuda())
        g.solve_ttr(max_sweeps=7)
        out = np.zeros(p.n, dtype=np.float32)
        with pytest.raises(odp.OdpError):
            g.readback(out)          # the readback reports the sweep limit
    ref = oracle.ttr(p, max_sweeps=7, raise_on_error=False)
    assert ref["rc"] == oracle.ETIMEOUT
    span = ref["phi"].max() - ref["phi"].min()
    assert np.abs(out - ref["phi"]).max() <= REL_TOL * span


def test_ttr_degenerate_targets():
    p = inputs.dubins3d(n=(20, 20, 16))
    # every node in the target: one sweep, all zero
    every = np.full(p.n, -1.0, dtype=np.float32)
    got, st = gpu_ttr(p, l=every)
    assert st["sweeps"] == 1 and np.all(got == 0.0)
    ref = oracle.ttr(p, l=every)
    assert ref["sweeps"] == 1
    # no node in the target: nothing decreases, every node keeps `big`
    none = np.ones(p.n, dtype=np.float32)
    got, st = gpu_ttr(p, l=none, big=500.0)
    ref = oracle.ttr(p, l=none, big=500.0)
    assert st["sweeps"] == ref["sweeps"] == 1
    assert np.all(got == 500.0) and np.all(ref["phi"] == 500.0)


def test_ttr_refusals():
    import torch

    p = inputs.dubins3d(n=(20, 20, 16))
    l = torch.from_numpy(p.target_values()).cuda()
    with odp.Grid.for_problem(p) as g:
        with pytest.raises(odp.OdpError) as e:
            g.solve_ttr()
        assert e.value.code == odp.ESTATE      # no target yet
        g.set_target(l)
        for kw in ({"eps": -1.0}, {"big": 0.0}, {"big": float("inf")}, {"max_sweeps": 0}):
            with pytest.raises(odp.OdpError) as e:
                g.solve_ttr(**kw)
            assert e.value.code == odp.EINVAL
    pm = dataclasses.replace(p, u_mode="max")
    with odp.Grid.for_problem(pm) as g:
        g.set_target(l)
        with pytest.raises(odp.OdpError) as e:
            g.solve_ttr()
        assert e.value.code == odp.EINVAL
    small = inputs.dubins3d(n=(20, 3, 16))
    with odp.Grid.for_problem(small) as g:
        g.set_target(torch.from_numpy(small.target_values()).cuda())
        with pytest.raises(odp.OdpError) as e:
            g.solve_ttr()
        assert e.value.code == odp.EINVAL
    r6 = inputs.rel6d(n=(6,) * 6)
    with odp.Grid.for_problem(r6) as g:
        g.set_target(torch.from_numpy(r6.target_values()).cuda())
        with pytest.raises(odp.OdpError) as e:
            g.solve_ttr()
        assert e.value.code == odp.EINVAL


@pytest.mark.parametrize("name", ["dubins3d_100", "dubinscar4d_60"])
def test_ttr_full_size_fixed_point(name):
    # full-size grids: the converged function is a fixed point of Algorithm
    # 2's update, which the oracle evaluates node by node at sampled nodes
    p = inputs.workload("ttr_" + name)
    got, st = gpu_ttr(p)
    assert st["change"] <= 1e-5
    rng = np.random.Generator(np.random.PCG64(7))
    span = float(got.max() - got.min())
    l = p.target_values()
    phi = got.astype(np.float64)
    checked = 0
    while checked < 150:
        idx = tuple(int(rng.integers(1 if not p.periodic[d] else 0,
                                     p.n[d] - 1 if not p.periodic[d] else p.n[d]))
                    for d in range(p.ndim))
        if l[idx] <= 0:
            continue
        v = oracle.ttr_node(p, phi, idx)
        # phi_i = min(F_i(phi), phi_i) at the limit and F_i moves by less
        # than eps plus rounding when its neighbours move by eps
        assert v >= phi[idx] - 1e-4 * span
        assert abs(v - phi[idx]) <= 1e-4 * span, (idx, v, phi[idx])
        checked += 1
    assert np.all(got >= 0.0) and np.all(got[l <= 0] == 0.0)
