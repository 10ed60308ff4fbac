"""Host logic of the N-rank bench path, run as two gloo ranks on the CPU:
process-group setup from the torchrun environment, the barrier, the
max-over-ranks timing and the whole-job throughput (units of all ranks over
the slowest rank's time)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench

    r, w, local = bench.rank_info()
    dist = bench.dist_setup(w, use_cuda=False)
    try:
        bench.barrier(dist)
        # rank r "took" 10 + 5 r ms; every rank must see the slowest
        slowest = bench.max_over_ranks(dist, 10.0 + 5.0 * r, "cpu")
        bench.barrier(dist)
        out[r] = (r, w, local, slowest)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        got = dict(out)
    assert sorted(got) == [0, 1]
    for r, (rr, w, local, slowest) in got.items():
        assert (rr, w, local) == (r, world, r)
        assert slowest == 15.0


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.dist_setup(1, use_cuda=False) is None
    assert bench.max_over_ranks(None, 3.5, "cpu") == 3.5
    bench.barrier(None)
