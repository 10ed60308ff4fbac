"""Time-varying target and obstacle sets on the GPU against the FP64 oracle
(the steps of segment (tau_k, tau_k+1] take their post-step min / max with
the sets at tau_k+1; phi starts from the target at tau_0).

Criterion as elsewhere: max |V_gpu - V_oracle| <= 1e-4 * (max l - min l) with
equal step counts, on the final value and on the value at every tau.
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


def cylinders(p, centers, radius):
    mesh = np.meshgrid(*p.nodes(), indexing="ij")
    return np.stack([(np.sqrt((mesh[0] - cx) ** 2 + (mesh[1] - cy) ** 2) - radius).astype(np.float32)
                     for cx, cy in centers])


CASES = {
    "dubins3d_upwind_euler": lambda: inputs.dubins3d(n=(25, 25, 16), tau=(0.0, 0.35, 0.8)),
    "dubins3d_upwind_rk2_4taus": lambda: inputs.dubins3d(n=(30, 27, 20), tau=(0.0, 0.2, 0.5, 0.9),
                                                          time_order=2),
    "dubinscar4d_upwind_rk2": lambda: inputs.dubinscar4d(n=(14, 13, 10, 16), tau=(0.0, 0.3, 0.6),
                                                         space_order=1, time_order=2),
}


def schedules(p):
    k = len(p.tau)
    ls = cylinders(p, [(0.5 * i, 0.2 * i) for i in range(k)], 0.9)
    gs = cylinders(p, [(2.5 - 0.3 * i, 0.3 * i) for i in range(k)], 0.5)
    return ls, gs


def gpu_solve(p, ls, gs, host_loop=False):
    import torch

    with odp.Grid.for_problem(p) as g:
        if host_loop:
            odp.set_loop_mode(g.handle, True)
        g.set_target_schedule(torch.from_numpy(ls).cuda())
        if gs is not None:
            g.set_obstacle_schedule(torch.from_numpy(gs).cuda())
        st = g.solve_problem(p, keep_snapshots=True, stats=True)
        snaps = np.stack([g.readback(torch.empty(p.n, device="cuda"), k).cpu().numpy() for k in range(len(p.tau))])
    return snaps, st


@pytest.mark.parametrize("name", sorted(CASES))
def test_time_varying_sets_parity(name):
    p = CASES[name]()
    ls, gs = schedules(p)
    snaps, st = gpu_solve(p, ls, gs)
    ref = oracle.solve(p, l_seq=ls.astype(np.float64), g_seq=gs.astype(np.float64), snapshots=True)
    tol = REL_TOL * float(ls.max() - ls.min())
    assert st["steps"] == int(ref["steps"].sum())
    for k in range(len(p.tau)):
        err = np.abs(snaps[k] - ref["snapshots"][k]).max()
        assert err <= tol, "tau[%d]: %.3g > %.3g" % (k, err, tol)
    # the sets bind: the result is not the solve that holds the first sets
    held = oracle.solve(p, l=ls[0].astype(np.float64), g=gs[0].astype(np.float64))
    assert np.abs(snaps[-1] - held["final"]).max() > 100 * tol


def test_time_varying_host_loop_identical():
    p = CASES["dubins3d_upwind_euler"]()
    ls, gs = schedules(p)
    a, sa = gpu_solve(p, ls, gs)
    b, sb = gpu_solve(p, ls, gs, host_loop=True)
    assert sa["steps"] == sb["steps"]
    assert np.array_equal(a, b)


def test_target_schedule_alone_and_replaced():
    import torch

    p = CASES["dubins3d_upwind_euler"]()
    ls, _ = schedules(p)
    ref = oracle.solve(p, l_seq=ls.astype(np.float64))
    l = p.target_values()
    with odp.Grid.for_problem(p) as g:
        g.set_target_schedule(torch.from_numpy(ls).cuda())
        g.solve_problem(p)
        v = g.readback(torch.empty(p.n, device="cuda")).cpu().numpy()
        assert np.abs(v - ref["final"]).max() <= REL_TOL * float(ls.max() - ls.min())
        # a time-invariant target replaces the schedule
        g.set_target(torch.from_numpy(l).cuda())
        g.solve_problem(p)
        w = g.readback(torch.empty(p.n, device="cuda")).cpu().numpy()
    static = oracle.solve(p)
    assert np.abs(w - static["final"]).max() <= REL_TOL * float(l.max() - l.min())


def test_schedule_refusals():
    import torch

    p = CASES["dubins3d_upwind_euler"]()
    ls, gs = schedules(p)
    with odp.Grid.for_problem(p) as g:
        g.set_target_schedule(torch.from_numpy(ls).cuda())
        # a solve over another tau list
        with pytest.raises(odp.OdpError) as e:
            g.solve(p.tau[:2])
        assert e.value.code == odp.EINVAL
        # the time-to-reach sweep and the batched solve take one target
        with pytest.raises(odp.OdpError) as e:
            g.solve_ttr()
        assert e.value.code == odp.EINVAL
        with pytest.raises(odp.OdpError) as e:
            odp.batch_solve([g], [0.5])
        assert e.value.code == odp.EINVAL
        # a schedule of one set
        with pytest.raises(odp.OdpError) as e:
            g.set_obstacle_schedule(torch.from_numpy(gs[:1]).cuda())
        assert e.value.code == odp.EINVAL
