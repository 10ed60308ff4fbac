"""The stage kernels' shared-window derivative helpers against the one-node
definition, on the CPU (no GPU): tests/host/stencil_check.cu is compiled with
nvcc as a host program that includes the kernels' own device header and
checks, bit for bit, that the last-axis routine (four nodes from one
eight-node window, node pairs in paired arithmetic) and the two-window
paired routine give what diffs() gives node by node (Section 3.1.4's ENO2
choice and the upwind differences), followed by the Lax-Friedrichs terms,
and that the four-node routine fed with precomputed differences (the
bulk-staged pass's stream axis) equals the five-row routine."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2204_05520_gb300 import _build  # noqa: E402


def test_shared_window_helpers_match_the_one_node_definition(tmp_path):
    nvcc = _build.nvcc()
    if not (os.path.isabs(nvcc) and os.path.exists(nvcc)) and shutil.which(nvcc) is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "stencil_check")
    src = os.path.join(ROOT, "tests", "host", "stencil_check.cu")
    csrc = os.path.join(ROOT, "paper_2204_05520_gb300", "csrc")
    cmd = [nvcc, *_build.ARCH, "-std=c++17", "-O2", "-I", csrc, "-I", os.path.join(ROOT, "include"),
           src, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "upwind 0, ENO2 0" in r.stdout


def test_stage_launch_geometry_covers_every_grid_exactly_once(tmp_path):
    """tests/host/geometry_check.cu, linked against the library, runs the
    library's own host geometry functions (plane-streaming and bulk-staged
    passes) on 4,000 seeded 3-6-D shapes and checks that bands, stream
    chunks and pencil blocks cover each grid exactly once and that the
    fast-division tables divide like '/'."""
    nvcc = _build.nvcc()
    if not (os.path.isabs(nvcc) and os.path.exists(nvcc)) and shutil.which(nvcc) is None:
        pytest.skip("nvcc not available")
    lib = _build.build()
    exe = str(tmp_path / "geometry_check")
    src = os.path.join(ROOT, "tests", "host", "geometry_check.cu")
    csrc = os.path.join(ROOT, "paper_2204_05520_gb300", "csrc")
    libdir = os.path.dirname(lib)
    cmd = [nvcc, *_build.ARCH, "-std=c++17", "-O2", "-I", csrc, "-I", os.path.join(ROOT, "include"),
           src, "-o", exe, "-L", libdir, "-lodp", "-Xlinker", "-rpath=" + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "failures: 0" in r.stdout


def test_rel6d_heading_alpha_never_exceeds_its_precomputed_ceiling(tmp_path):
    """tests/host/alpha_ceiling_check.cu, linked against the library: on
    3,000 seeded w_p axes the kernels' per-node heading-rate bound never
    exceeds rel6d_heading_ceiling, and a straddling node reaches it bit for
    bit -- the premise that lets the alpha pass stop reading at the ceiling
    with an unchanged result."""
    nvcc = _build.nvcc()
    if not (os.path.isabs(nvcc) and os.path.exists(nvcc)) and shutil.which(nvcc) is None:
        pytest.skip("nvcc not available")
    lib = _build.build()
    exe = str(tmp_path / "alpha_ceiling_check")
    src = os.path.join(ROOT, "tests", "host", "alpha_ceiling_check.cu")
    csrc = os.path.join(ROOT, "paper_2204_05520_gb300", "csrc")
    libdir = os.path.dirname(lib)
    cmd = [nvcc, *_build.ARCH, "-std=c++17", "-O2", "-I", csrc, "-I", os.path.join(ROOT, "include"),
           src, "-o", exe, "-L", libdir, "-lodp", "-Xlinker", "-rpath=" + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "failures 0" in r.stdout
