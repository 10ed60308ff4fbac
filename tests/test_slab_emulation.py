"""The multi-GPU plan for one solve, emulated with CPU ranks (gloo).

One solve shards into slabs along axis 0, one per rank.  Every stage, each
rank exchanges the stencil-deep halo planes with its neighbours, takes the
max-allreduce of its local dissipation bounds for the global alpha (so every
rank computes the same CFL step), and updates its own planes.  Here each rank
evaluates the right-hand side with the FP64 oracle on its slab plus halos
(oracle.terms with the global alpha), replays the time loop (CFL step clipped
at the horizon, Heun average, BRT min), and the slabs gathered on rank 0 must
equal the oracle's single-domain solve.  No GPU takes part.
"""
import dataclasses
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(name):
    from paper_2204_05520_gb300 import inputs

    if name == "dubins3d_eno2_rk2":
        return inputs.dubins3d(n=(23, 17, 12), horizon=0.4, space_order=2, time_order=2)
    if name == "dubinscar4d_eno2_euler":
        return inputs.dubinscar4d(n=(15, 11, 8, 12), horizon=0.3, space_order=2, time_order=1)
    if name == "rel6d_upwind_rk2":
        return inputs.rel6d(n=(10, 8, 7, 5, 5, 5), horizon=0.2, space_order=1, time_order=2)
    raise KeyError(name)


def _slabs(n0, world):
    """Own planes [s0, s1) of axis 0 for each rank (as even as possible)."""
    base, extra = divmod(n0, world)
    out, s = [], 0
    for r in range(world):
        e = s + base + (1 if r < extra else 0)
        out.append((s, e))
        s = e
    return out


def _rank_main(rank, world, port, name, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle

        p = _problem(name)
        O = p.space_order
        n0 = p.n[0]
        h0 = (p.hi[0] - p.lo[0]) / (n0 - 1)          # axis 0 is not periodic here
        s0, s1 = _slabs(n0, world)[rank]
        a0, a1 = max(0, s0 - O), min(n0, s1 + O)     # own planes plus halos
        sub = dataclasses.replace(p, n=(a1 - a0,) + tuple(p.n[1:]),
                                  lo=(p.lo[0] + a0 * h0,) + tuple(p.lo[1:]),
                                  hi=(p.lo[0] + (a1 - 1) * h0,) + tuple(p.hi[1:]))
        own = slice(s0 - a0, s1 - a0)
        l_full = p.target_values().astype(np.float64)
        l_own = l_full[s0:s1]
        phi = l_full[a0:a1].copy()                   # phi(0) = l on the slab and halos

        def exchange(v):
            """Fill the halo planes of v from the neighbours' own planes."""
            reqs, bufs = [], []
            if rank > 0:
                reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(v[own][:O])), rank - 1))
                b = torch.empty((O,) + v.shape[1:], dtype=torch.float64)
                reqs.append(dist.irecv(b, rank - 1))
                bufs.append((slice(0, O), b))
            if rank < world - 1:
                reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(v[own][-O:])), rank + 1))
                b = torch.empty((O,) + v.shape[1:], dtype=torch.float64)
                reqs.append(dist.irecv(b, rank + 1))
                bufs.append((slice(v.shape[0] - O, v.shape[0]), b))
            for q in reqs:
                q.wait()
            for sl, b in bufs:
                v[sl] = b.numpy()

        def rhs_and_alpha(v):
            """L(v) on the own planes with the global alpha (max-allreduce
            of the local bounds of every rank's own nodes)."""
            a_loc = oracle.terms(sub, v)["a"][own].reshape(-1, p.ndim).max(axis=0)
            a = torch.from_numpy(a_loc.copy())
            dist.all_reduce(a, op=dist.ReduceOp.MAX)
            alpha = a.numpy()
            return oracle.terms(sub, v, alpha=alpha)["rhs"][own], alpha

        dz = [h0] + [(p.hi[d] - p.lo[d]) / (p.n[d] if p.periodic[d] else p.n[d] - 1)
                     for d in range(1, p.ndim)]
        t, t_end, steps = 0.0, float(p.tau[-1]), 0
        while t_end - t > 1e-12 * t_end:
            L1, alpha = rhs_and_alpha(phi)
            dt_cfl = p.cfl / sum(alpha[d] / dz[d] for d in range(p.ndim))
            last = not (dt_cfl < t_end - t)
            dt = (t_end - t) if last else dt_cfl
            new = phi[own] + dt * L1
            if p.time_order == 2:
                phi1 = phi.copy()
                phi1[own] = new
                exchange(phi1)
                L2, _ = rhs_and_alpha(phi1)
                new = 0.5 * (phi[own] + (phi1[own] + dt * L2))
            if p.set_kind == "brt":
                new = np.minimum(new, l_own)
            phi[own] = new
            exchange(phi)
            t = t_end if last else t + dt
            steps += 1
        # gather the own planes on rank 0
        mine = torch.from_numpy(np.ascontiguousarray(phi[own]))
        if rank == 0:
            parts = [mine.numpy()]
            for r in range(1, world):
                r0, r1 = _slabs(n0, world)[r]
                b = torch.empty((r1 - r0,) + tuple(p.n[1:]), dtype=torch.float64)
                dist.recv(b, r)
                parts.append(b.numpy())
            out["final"] = np.concatenate(parts, axis=0)
            out["steps"] = steps
        else:
            dist.send(mine, 0)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name,world", [("dubins3d_eno2_rk2", 2), ("dubins3d_eno2_rk2", 3),
                                        ("dubinscar4d_eno2_euler", 3), ("rel6d_upwind_rk2", 2)])
def test_slab_sharded_solve_equals_single_domain(name, world):
    import oracle

    oracle.build()
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:   # no fork of a process holding OpenMP threads
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, name, out), nprocs=world, join=True)
        got = dict(out)
    p = _problem(name)
    ref = oracle.solve(p)
    l = p.target_values().astype(np.float64)
    assert got["steps"] == int(ref["steps"].sum())
    # the same per-node arithmetic; node coordinates of a slab differ from the
    # whole grid's by rounding only
    err = np.abs(got["final"] - ref["final"]).max()
    assert err <= 1e-10 * (l.max() - l.min()), err
