"""The C-ABI library builds for sm_103a, loads on the host and exports every
entry point that include/*.h declares (no compute call: no GPU needed)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_2204_05520_gb300 import _build, odp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(odp_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return odp.load()


def test_header_declares_the_solver_boundary():
    names = declared_entry_points()
    for required in ("odp_grid_create", "odp_set_dynamics", "odp_set_target", "odp_solve_hjb",
                     "odp_value_readback"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_entry_points() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_marshals_every_declared_entry_point(lib):
    # the ctypes binding sets argument and result types for each declared
    # function (an unset one would pass 64-bit arguments as C ints)
    for name in declared_entry_points():
        fn = getattr(lib, name)
        assert fn.restype is not None, name
        assert fn.argtypes is not None, name


def test_library_reports_version_and_no_error(lib):
    assert "sm_103a" in odp.version()
    assert odp.last_error() == ""


def test_argument_errors_need_no_gpu(lib):
    # validation happens before any CUDA call
    with pytest.raises(odp.OdpError) as e:
        odp.grid_create((1, 4), (0.0, 0.0), (1.0, 1.0), (False, False), stream=0)
    assert e.value.code == odp.EINVAL
    with pytest.raises(odp.OdpError) as e:
        odp.grid_create((4,) * 7, (0.0,) * 7, (1.0,) * 7, (False,) * 7, stream=0)
    assert e.value.code == odp.EINVAL
    with pytest.raises(odp.OdpError) as e:
        odp.grid_create((4, 4), (1.0, 0.0), (0.0, 1.0), (False, False), stream=0)
    assert e.value.code == odp.EINVAL


@pytest.mark.parametrize("n", [(41, 41, 36), (80, 80, 40, 64), (24,) * 6, (37,), (13, 11),
                               (101, 101, 64), (31, 31, 37), (2, 2, 5), (3, 4, 3, 3, 2, 4),
                               (4, 13, 200), (6, 101, 64), (5, 3, 40)])
def test_launch_geometry_covers_the_grid(lib, n):
    g = odp.plan_geometry(n)
    nl = n[-1]
    assert g["n_pad"] % 4 == 0 and nl <= g["n_pad"] < nl + 4
    nr = n[-2] if len(n) >= 2 else 1
    assert g["row_groups"] * g["rows_per_thread"] >= nr
    assert g["threads_rb"] == (g["n_pad"] // 4) * g["row_groups"] * g["planes"]
    if len(n) >= 3 and g["plane_pass"]:
        ns = n[-3]
        pencils = int(np.prod(n[:-3])) if len(n) > 3 else 1
        segs = g["n_pad"] // 4
        rb, nb = g["band_rows"], g["bands"]
        assert 1 <= g["chunk"] <= ns
        # bands cover the rows; every band (the last one too) has 4 rows or more
        assert rb * nb >= nr and rb * (nb - 1) < nr and nr - rb * (nb - 1) >= 4
        assert g["ctas"] == pencils * nb * -(-ns // g["chunk"])
        assert g["cta_threads"] == -(-rb * segs // 32) * 32 and g["cta_threads"] <= 512
        assert 0 < g["smem_r1"] < g["smem_r2"] <= 48 * 1024


def test_noalloc_binding_refuses_what_the_entry_point_does_not_solve():
    # reach-avoid, per-node dissipation and intermediate tau points would give
    # a different answer than the grid object's solve: refused before any
    # library call (no GPU needed)
    import dataclasses

    from paper_2204_05520_gb300 import inputs, odp

    p = inputs.dubins3d(n=(9, 9, 8), horizon=0.5)
    bad = [inputs.reach_avoid(p, inputs.dubins_obstacle()),
           dataclasses.replace(p, dissipation="local"),
           dataclasses.replace(p, tau=(0.0, 0.2, 0.5)),
           dataclasses.replace(p, tau=(0.1, 0.5))]
    for q in bad:
        with pytest.raises(ValueError):
            odp.solve_noalloc(q, None, None)
