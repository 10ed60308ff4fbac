"""Serving loop (odp_server_*): continuous batching under an HBM budget.

Requests that arrive while others are on the GPU join later launches; each
result must equal the same request solved alone (odp_solve_hjb), match the
FP64 oracle (the 1e-4 bar for upwind solves, twice the oracle's own float32
sensitivity for ENO2 solves, equal step counts), and the resident HBM never
exceeds the budget."""
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
        g.solve_problem(problem)
        return g.readback(torch.empty(l.shape, device="cuda")).cpu().numpy()


def mixed_requests(count, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        if rng.uniform() < 0.5:
            side = int(rng.integers(17, 33))
            out.append(inputs.dubins3d(n=(side, side, side), v=float(rng.uniform(0.5, 2.0)),
                                       w_max=float(rng.uniform(0.5, 1.5)),
                                       radius=float(rng.uniform(0.5, 1.5)),
                                       horizon=float(rng.uniform(0.2, 1.0))))
        else:
            side = int(rng.integers(9, 15))
            out.append(inputs.dubinscar4d(n=(side,) * 4, a_max=float(rng.uniform(0.5, 1.5)),
                                          w_max=float(rng.uniform(0.5, 1.5)),
                                          radius=float(rng.uniform(0.5, 1.5)),
                                          horizon=float(rng.uniform(0.2, 0.8))))
    return out


def served_like_requests(count, seed=1):
    """Requests drawn as the served workload draws them (Poisson mix of
    upwind Dubins3D and ENO2 + TVD-RK2 DubinsCar4D, horizons U[0.5, 3]) on
    reduced grids (sides 31-35 and 20-24), so the oracle checks each one."""
    return [p for _, p in inputs.served_requests(100.0, count=count, seed=seed,
                                                 side3=(31, 35), side4=(20, 24))]


def test_results_are_the_same_alone_and_in_the_mix():
    problems = mixed_requests(10, seed=5) + served_like_requests(4)
    assert {p.dynamics for p in problems[10:]} == {"dubins3d", "dubinscar4d"}
    with odp.Server(hbm_budget_bytes=512 << 20) as srv:
        ids = {}
        # arrivals spread over the first steps: later requests join a batch
        # that is already running
        pending = list(enumerate(problems))
        step = 0
        while pending or any(srv.poll(i)["state"] < odp.REQ_DONE for i in ids.values()):
            while pending and len(ids) < 3 * (step + 1):
                k, p = pending.pop(0)
                ids[k] = srv.submit(p)
            srv.step(rounds=4)
            step += 1
            assert step < 10000
        assert srv.info()["launches"] > 1
        for k, p in enumerate(problems):
            st = srv.poll(ids[k])
            assert st["state"] == odp.REQ_DONE and st["steps_done"] == st["steps"]
            v = srv.readback(ids[k], np.empty(p.n, np.float32))
            # the same per-node arithmetic as the single solve
            assert np.array_equal(v, solo(p))
            # and the FP64 oracle's solve of the same request
            parity.check_whole_solve(p, v, st["steps"], name="served %s" % p.name)
            srv.release(ids[k])
        assert srv.info()["used_bytes"] == 0


def test_row_blocked_fallback_in_the_mix():
    # a grid whose last axis is too long for the plane-streaming pass sends
    # the whole step to the persistent row-blocked kernel; every result still
    # equals its solo solve
    problems = [inputs.dubins3d(n=(6, 7, 520), horizon=0.3),
                inputs.dubins3d(n=(21, 21, 20), horizon=0.4),
                inputs.dubinscar4d(n=(10, 11, 9, 12), horizon=0.3)]
    with odp.Server(hbm_budget_bytes=64 << 20) as srv:
        ids = [srv.submit(p) for p in problems]
        steps = 0
        while any(srv.poll(i)["state"] < odp.REQ_DONE for i in ids):
            srv.step(rounds=8)
            steps += 1
            assert steps < 1000
        for i, p in zip(ids, problems):
            v = srv.readback(i, np.empty(p.n, np.float32))
            assert np.array_equal(v, solo(p))
            srv.release(i)


def test_admission_respects_the_budget():
    p = inputs.dubins3d(n=(31, 31, 32), horizon=0.5)
    per = 4 * 3 * 31 * 31 * 32
    with odp.Server(hbm_budget_bytes=int(per * 2.5) + (1 << 16)) as srv:
        ids = [srv.submit(p) for _ in range(5)]
        srv.step(rounds=1)
        info = srv.info()
        assert info["resident"] == 2 and info["queued"] == 3
        assert info["used_bytes"] <= info["budget_bytes"]
        steps = 0
        while ids:
            srv.step(rounds=16)
            steps += 1
            assert steps < 1000
            for i in list(ids):
                if srv.poll(i)["state"] == odp.REQ_DONE:
                    srv.readback(i, np.empty(p.n, np.float32))
                    srv.release(i)
                    ids.remove(i)
            assert srv.info()["used_bytes"] <= srv.info()["budget_bytes"]
        assert srv.info()["used_bytes"] == 0


def test_unsupported_and_oversized_requests_are_refused():
    with odp.Server(hbm_budget_bytes=8 << 20) as srv:
        with pytest.raises(odp.OdpError) as e:
            srv.submit(inputs.rel6d(n=(4, 4, 4, 4, 4, 4)))
        assert e.value.code == odp.EINVAL
        with pytest.raises(odp.OdpError) as e:
            srv.submit(inputs.dubins3d(n=(101, 101, 101)))
        assert e.value.code == odp.ENOMEM


def test_resident_cap_admits_in_arrival_order():
    p = inputs.dubins3d(n=(31, 31, 32), horizon=0.5)
    nodes = 31 * 31 * 32
    ref = solo(p)
    with odp.Server(hbm_budget_bytes=256 << 20) as srv:
        srv.set_max_resident(int(nodes * 2.5))
        ids = [srv.submit(p) for _ in range(5)]
        srv.step(rounds=1)
        info = srv.info()
        assert info["resident"] == 2 and info["queued"] == 3
        steps = 0
        while any(srv.poll(i)["state"] < odp.REQ_DONE for i in ids):
            srv.step(rounds=16)
            steps += 1
            assert srv.info()["resident"] <= 2
            assert steps < 1000
        done = [srv.poll(i)["t_done"] for i in ids]
        assert done == sorted(done)          # first come, first served
        for i in ids:
            assert np.array_equal(srv.readback(i, np.empty(p.n, np.float32)), ref)
            srv.release(i)
        with pytest.raises(odp.OdpError) as e:
            srv.set_max_resident(-1)
        assert e.value.code == odp.EINVAL


def test_cancelled_busy_and_failed_requests():
    p = inputs.dubins3d(n=(31, 31, 32), horizon=0.5)
    per = 4 * 3 * 31 * 31 * 32

    def state(srv, rid):
        try:
            return srv.poll(rid)["state"]
        except odp.OdpError as e:          # a failed request reports ODP_ENUMERIC
            assert e.code == odp.ENUMERIC
            return odp.REQ_FAILED

    with odp.Server(hbm_budget_bytes=int(per * 2.5) + (1 << 16)) as srv:
        ids = [srv.submit(p) for _ in range(4)]
        srv.step(rounds=1)
        assert srv.info()["resident"] == 2 and srv.info()["queued"] == 2
        # a queued request can be cancelled; a running one cannot
        srv.release(ids[3])
        assert srv.info()["queued"] == 1
        with pytest.raises(odp.OdpError) as e:
            srv.poll(ids[3])
        assert e.value.code == odp.EINVAL
        with pytest.raises(odp.OdpError) as e:
            srv.release(ids[0])
        assert e.value.code == odp.EBUSY
        # a target holding a NaN: the device flags the solve, the others finish
        bad = p.target_values().copy()
        bad[15, 15, 5] = np.nan
        rb = srv.submit(p, target=bad)
        ref = solo(p)
        pending, outcome, steps = set(ids[:3] + [rb]), {}, 0
        while pending:
            srv.step(rounds=16)
            steps += 1
            assert steps < 1000
            for i in list(pending):
                st = state(srv, i)
                if st >= odp.REQ_DONE:
                    # finished requests hold their HBM until released
                    if st == odp.REQ_DONE:
                        assert np.array_equal(srv.readback(i, np.empty(p.n, np.float32)), ref)
                    outcome[i] = st
                    srv.release(i)
                    pending.discard(i)
        assert outcome[rb] == odp.REQ_FAILED
        assert all(outcome[i] == odp.REQ_DONE for i in ids[:3])
        assert srv.info()["used_bytes"] == 0
