"""Batched solves (odp_batch_solve): every grid of the batch must end where
the same grid ends when solved alone (same step schedule, same kernel
arithmetic), and where the FP64 oracle ends (1e-4 of the value range)."""
import numpy as np
import pytest

import oracle
import parity
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


def solo(problem):
    import torch

    l = problem.target_values()
    with odp.Grid.for_problem(problem) as g:
        g.set_target(torch.from_numpy(l).cuda())
        st = g.solve_problem(problem, stats=True)
        v = g.readback(torch.empty(l.shape, device="cuda")).cpu().numpy()
    return v, st


def batched(problems, **kw):
    import torch

    grids = []
    try:
        for p in problems:
            g = odp.Grid.for_problem(p)
            g.set_target(torch.from_numpy(p.target_values()).cuda())
            grids.append(g)
        p0 = problems[0]
        st = odp.batch_solve(grids, [p.tau[-1] for p in problems], p0.set_kind, p0.space_order,
                             p0.time_order, p0.cfl)
        outs = [g.readback(torch.empty(p.n, device="cuda")).cpu().numpy()
                for g, p in zip(grids, problems)]
        steps = [odp.solve_status(g.handle)["steps"] for g in grids]
    finally:
        for g in grids:
            g.close()
    return outs, st, steps


def small_dubins_batch(count, seed, sides=(21, 25, 31), horizon=1.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        side = int(rng.choice(sides))
        nth = int(rng.integers(12, 41))
        out.append(inputs.dubins3d(n=(side, side, nth), v=float(rng.uniform(0.5, 2.0)),
                                   w_max=float(rng.uniform(0.5, 1.5)),
                                   radius=float(rng.uniform(0.5, 1.5)), horizon=horizon))
    return out


def test_batch_equals_solo_and_oracle():
    problems = small_dubins_batch(12, seed=3)
    outs, st, steps = batched(problems)
    assert st["rounds"] == max(steps)
    identical = 0
    for p, v, s in zip(problems, outs, steps):
        ref_solo, st_solo = solo(p)
        assert s == st_solo["steps"]
        l = p.target_values()
        rng_l = float(l.max() - l.min())
        assert np.abs(v - ref_solo).max() <= REL_TOL * rng_l
        identical += int(np.array_equal(v, ref_solo))
        ref = oracle.solve(p)
        assert s == int(ref["steps"].sum())
        assert np.abs(v - ref["final"]).max() <= REL_TOL * rng_l
    # the same kernel arithmetic on the same schedule: expected bit-identical
    assert identical == len(problems)


def test_batch_of_mixed_models_rk2_eno2():
    problems = [inputs.dubins3d(n=(21, 23, 16), space_order=2, time_order=2, horizon=0.6),
                inputs.dubinscar4d(n=(11, 13, 7, 12), horizon=0.6),
                inputs.dubins3d(n=(17, 17, 20), space_order=2, time_order=2, horizon=0.3, v=1.7),
                inputs.dubinscar4d(n=(9, 9, 6, 8), horizon=0.4, a_max=0.7)]
    outs, st, steps = batched(problems)
    for p, v, s in zip(problems, outs, steps):
        ref_solo, st_solo = solo(p)
        assert s == st_solo["steps"]
        assert np.array_equal(v, ref_solo)
        # whole ENO2 solves against the oracle, within twice its own
        # sensitivity to float32-level changes
        parity.check_whole_solve(p, v, s, name="batched %s" % p.name)


def test_batch_single_integrator_brs_and_partial_rows():
    # two rows (fewer than four rows per thread) and ragged last axes
    problems = [inputs.single_integrator((2, 37), u_mode="min", set_kind="brs", horizon=0.3),
                inputs.single_integrator((9, 13), u_mode="min", set_kind="brs", horizon=0.5),
                inputs.single_integrator((7, 6, 5), u_mode="min", set_kind="brs", horizon=0.4)]
    outs, _, steps = batched(problems)
    for p, v, s in zip(problems, outs, steps):
        ref = oracle.solve(p)
        l = p.target_values()
        assert s == int(ref["steps"].sum())
        assert np.abs(v - ref["final"]).max() <= REL_TOL * float(l.max() - l.min())


def test_batch_rejects_unsupported_and_bad_arguments():
    import torch

    p = inputs.rel6d(n=(4, 4, 4, 3, 3, 3), horizon=0.1)
    with odp.Grid.for_problem(p) as g:
        g.set_target(torch.from_numpy(p.target_values()).cuda())
        with pytest.raises(odp.OdpError) as e:
            odp.batch_solve([g], [0.1])
        assert e.value.code == odp.EINVAL
    q = inputs.dubins3d(n=(9, 9, 8))
    with odp.Grid.for_problem(q) as g:
        with pytest.raises(odp.OdpError) as e:
            odp.batch_solve([g], [0.1])
        assert e.value.code == odp.ESTATE
        g.set_target(torch.from_numpy(q.target_values()).cuda())
        with pytest.raises(odp.OdpError) as e:
            odp.batch_solve([g], [-1.0])
        assert e.value.code == odp.EINVAL


def test_batch_workload_sample_full_sizes():
    # 32 grids drawn like the 512-grid batched workload (sides 31..101, 36-64
    # theta cells), checked against solo solves
    problems = inputs.batch_problems(count=32, seed=0)
    outs, st, steps = batched(problems)
    assert st["point_updates"] == sum(p.points * s for p, s in zip(problems, steps))
    for p, v, s in zip(problems, outs, steps):
        ref_solo, st_solo = solo(p)
        assert s == st_solo["steps"]
        assert np.array_equal(v, ref_solo)
    # the smallest, the largest and two more grids against the FP64 oracle
    order = sorted(range(len(problems)), key=lambda i: problems[i].points)
    for i in sorted({order[0], order[-1], order[len(order) // 3], order[2 * len(order) // 3]}):
        parity.check_whole_solve(problems[i], outs[i], steps[i], name="batched %s" % problems[i].name)


def test_batch_graph_is_captured_once_and_replayed():
    # the plane-path batch runs as one CUDA graph of its per-round launches:
    # captured by the first call of a batch signature (which also autotunes
    # the stream-chunk cap), replayed by the next; the values are the same
    # both times and equal to the solo solves
    problems = small_dubins_batch(10, seed=11)
    outs1, st1, steps1 = batched(problems)
    outs2, st2, steps2 = batched(problems)
    assert st1["plane_chunk"] in (8, 16, 32, 64) and st2["plane_chunk"] == st1["plane_chunk"]
    assert st1["graph"] == 1 and st2["graph"] == 2
    assert st2["tuned"] == 0
    assert st1["launches"] == st2["launches"] == max(steps1)
    for p, a, b in zip(problems, outs1, outs2):
        assert np.array_equal(a, b)
        assert np.array_equal(a, solo(p)[0])
