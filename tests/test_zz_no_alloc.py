"""The allocation-free entry point (odp_solve_noalloc) against the regular
one (odp_solve_hjb through a grid object).

It is meant for callers that cannot allocate device memory when they need a
solve (code inside a memory pool it does not own, or code that must not let
cudaMalloc/cudaFree synchronise the device): all of its working memory is one
fixed device array inside the library.  Two calls in a row must each match
the regular solve of the same problem, so the second call cannot be
disturbed by what the first one left in the shared array.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

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
    return torch


def regular(problem):
    import torch

    l = problem.target_values()
    with odp.Grid.for_problem(problem) as g:
        g.set_target(torch.from_numpy(l).cuda())
        g.solve_problem(problem)
        return g.readback(torch.empty(l.shape, device="cuda")).cpu().numpy()


def no_alloc(problem):
    import torch

    l = torch.from_numpy(problem.target_values()).cuda()
    out = torch.full(problem.n, float("nan"), device="cuda")
    odp.solve_noalloc(problem, l, out)
    return out.cpu().numpy()


def test_two_calls_in_a_row_match_the_regular_entry_point():
    problems = [inputs.dubins3d(n=(31, 31, 24), horizon=1.0),
                inputs.dubinscar4d(n=(13, 13, 7, 10), horizon=0.5)]
    for p in problems:
        got = no_alloc(p)
        want = regular(p)
        l = p.target_values()
        assert np.isfinite(got).all()
        assert np.abs(got - want).max() <= REL_TOL * float(l.max() - l.min())


def test_a_call_allocates_no_device_memory():
    # after one warm-up call, a second call changes neither the device's free
    # memory nor the memory torch's caching allocator holds
    import torch

    p = inputs.dubins3d(n=(31, 31, 24), horizon=0.5)
    l = torch.from_numpy(p.target_values()).cuda()
    out = torch.empty_like(l)
    odp.solve_noalloc(p, l, out)
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    odp.solve_noalloc(p, l, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0
    assert np.isfinite(out.cpu().numpy()).all()


def test_the_callers_current_device_is_kept():
    import torch

    p = inputs.dubins3d(n=(21, 21, 16), horizon=0.3)
    l = torch.from_numpy(p.target_values()).cuda()
    before = torch.cuda.current_device()
    odp.solve_noalloc(p, l, torch.empty_like(l))
    assert torch.cuda.current_device() == before


def test_a_capturing_stream_is_refused():
    import torch

    p = inputs.dubins3d(n=(21, 21, 16), horizon=0.3)
    l = torch.from_numpy(p.target_values()).cuda()
    out = torch.empty_like(l)
    odp.solve_noalloc(p, l, out)       # first call on this device outside any capture
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    refused = None
    with torch.cuda.graph(g, stream=s):
        out.add_(0.0)                  # the captured graph is not empty
        try:
            odp.solve_noalloc(p, l, out, stream=s)
        except odp.OdpError as e:
            refused = e
    assert refused is not None and refused.code == odp.EINVAL


def test_grids_beyond_the_fixed_array_are_refused():
    import torch

    p = inputs.dubins3d(n=(201, 201, 64), horizon=0.1)   # 2.6M nodes
    l = torch.zeros(p.n, device="cuda")
    with pytest.raises(odp.OdpError) as e:
        odp.solve_noalloc(p, l, torch.empty_like(l))
    assert e.value.code == odp.EINVAL
    assert "scratch" in str(e.value)
