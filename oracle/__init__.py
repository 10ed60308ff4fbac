"""FP64 CPU oracle of the time-dependent HJ level-set method (Algorithm 1 of
arXiv 2204.05520) and of its time-to-reach sweeping (Algorithm 2), loaded
through ctypes.

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never imports, links or calls it, and it shares no code with the CUDA library.

``build()`` compiles ``odp_oracle.c`` with gcc (OpenMP over grid points, no
fast-math, no FMA contraction) into ``oracle/_build/liboracle.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "odp_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

DYN_IDS = {"single_integrator": 0, "dubins3d": 1, "dubinscar4d": 2, "rel6d": 3, "advection": 4,
           "dubins_capture": 5}
MODE_IDS = {"min": 0, "max": 1}
SET_IDS = {"brs": 0, "brt": 1}
MAX_INPUTS = 8
TTR_SCHEMES = {"gauss_seidel": 0, "jacobi": 1}
# computation methods of the solver (reading R27)
TARGET_METHODS = {"None": 0, "minVWithVTarget": 1, "maxVWithVTarget": 2, "minVWithVInit": 3,
                  "maxVWithVInit": 4, "minVWithV0": 5, "maxVWithV0": 6}
OBSTACLE_METHODS = {"maxVWithObstacle": 1, "minVWithObstacle": 2}

OK, EINVAL, ENOMEM, ETIMEOUT, ENUMERIC = 0, -1, -2, -5, -6


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__("oracle %s failed with code %d" % (what, code))
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle if the shared object is missing or stale."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
            lib.og_num_threads.restype = i32
            lib.og_set_threads.argtypes = [i32]
            lib.og_spacing.argtypes = [i32, P, P, P, P, P]
            lib.og_eval_dynamics.argtypes = [i32, i32, P, i32, P, P, P, P]
            lib.og_eval_dynamics_batch.argtypes = [i32, i32, P, i32, i64, P, P, P, P]
            lib.og_eval_dynamics_batch.restype = i32
            lib.og_terms.argtypes = [i32, P, P, P, P, i32, P, i32, i32, i32, i32, P, P,
                                     P, P, P, P, P, P, P, P]
            lib.og_solve.argtypes = [i32, P, P, P, P, i32, P, i32, i32, i32, P, P, P, P, i32, i32,
                                     i32, i32, i32, f64, i64, P, P, P, P, P]
            lib.og_solve_seq.argtypes = lib.og_solve.argtypes
            lib.og_solve_methods.argtypes = [i32, P, P, P, P, i32, P, i32, i32, i32, P, P, P, P, P, P, i32,
                                             i32, i32, i32, i32, i32, f64, i64, P, P, P, P, P]
            lib.og_step.argtypes = [i32, P, P, P, P, i32, P, i32, i32, i32, P, P, P, f64, i32, i32,
                                    i32, i32, P, P]
            lib.og_ttr.argtypes = [i32, P, P, P, P, i32, P, i32, i32, i32, P, f64, f64, i64, i32,
                                   P, P, P]
            lib.og_ttr_node.argtypes = [i32, P, P, P, P, i32, P, i32, i32, i32, P, P, P]
            for f in (lib.og_spacing, lib.og_eval_dynamics, lib.og_terms, lib.og_solve,
                      lib.og_solve_seq, lib.og_solve_methods, lib.og_step, lib.og_ttr, lib.og_ttr_node):
                f.restype = i32
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _grid_args(n, lo, hi, periodic):
    n_a = np.ascontiguousarray(n, dtype=np.int64)
    lo_a = np.ascontiguousarray(lo, dtype=np.float64)
    hi_a = np.ascontiguousarray(hi, dtype=np.float64)
    per_a = np.ascontiguousarray([1 if p else 0 for p in periodic], dtype=np.int32)
    return n_a, lo_a, hi_a, per_a


def num_threads() -> int:
    return int(_load().og_num_threads())


def set_threads(t: int) -> None:
    _load().og_set_threads(int(t))


def spacing(n, lo, hi, periodic) -> np.ndarray:
    lib = _load()
    n_a, lo_a, hi_a, per_a = _grid_args(n, lo, hi, periodic)
    out = np.zeros(len(n_a), dtype=np.float64)
    rc = lib.og_spacing(len(n_a), _ptr(n_a), _ptr(lo_a), _ptr(hi_a), _ptr(per_a), _ptr(out))
    if rc:
        raise OracleError(rc, "spacing")
    return out


def eval_dynamics(dynamics: str, params, z, u=(), d=()) -> np.ndarray:
    """f(z, u, d) of one model at one state."""
    lib = _load()
    z_a = np.ascontiguousarray(z, dtype=np.float64)
    prm = np.ascontiguousarray(params, dtype=np.float64)
    u_a = np.zeros(MAX_INPUTS)
    d_a = np.zeros(MAX_INPUTS)
    u_a[: len(u)] = u
    d_a[: len(d)] = d
    f = np.zeros(len(z_a))
    lib.og_eval_dynamics(DYN_IDS[dynamics], len(z_a), _ptr(prm), len(prm), _ptr(z_a),
                         _ptr(u_a), _ptr(d_a), _ptr(f))
    return f


def eval_dynamics_batch(dynamics: str, params, z, u, d) -> np.ndarray:
    """f for arrays of states z (m, ndim) and inputs u, d (m, k <= 8)."""
    lib = _load()
    z_a = np.ascontiguousarray(z, dtype=np.float64)
    m, nd = z_a.shape
    u_a = np.zeros((m, MAX_INPUTS))
    d_a = np.zeros((m, MAX_INPUTS))
    u = np.asarray(u, dtype=np.float64).reshape(m, -1)
    d = np.asarray(d, dtype=np.float64).reshape(m, -1)
    u_a[:, : u.shape[1]] = u
    d_a[:, : d.shape[1]] = d
    prm = np.ascontiguousarray(params, dtype=np.float64)
    f = np.zeros((m, nd))
    lib.og_eval_dynamics_batch(DYN_IDS[dynamics], nd, _ptr(prm), len(prm), m, _ptr(z_a),
                               _ptr(u_a), _ptr(d_a), _ptr(f))
    return f


def terms(problem_or_grid, phi, order=None, alpha=None, dynamics=None, params=None,
          u_mode=None, d_mode=None) -> dict:
    """Per-node terms of one Algorithm 1 evaluation on ``phi``.

    ``problem_or_grid`` is an ``inputs.Problem`` (its grid, dynamics and
    order are used unless overridden).  Returns a dict of numpy arrays:
    pm, pp (shape + (ndim,)), u, d (shape + (8,)), H (shape), a (shape +
    (ndim,)), alpha (ndim,), rhs (shape).
    """
    p = problem_or_grid
    lib = _load()
    n_a, lo_a, hi_a, per_a = _grid_args(p.n, p.lo, p.hi, p.periodic)
    nd = len(n_a)
    dyn = dynamics or p.dynamics
    prm = np.ascontiguousarray(params if params is not None else p.params, dtype=np.float64)
    order = order or p.space_order
    phi64 = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
    N = phi64.size
    out = {
        "pm": np.zeros((N, nd)), "pp": np.zeros((N, nd)),
        "u": np.zeros((N, MAX_INPUTS)), "d": np.zeros((N, MAX_INPUTS)),
        "H": np.zeros(N), "a": np.zeros((N, nd)), "alpha": np.zeros(nd), "rhs": np.zeros(N),
    }
    al = None if alpha is None else np.ascontiguousarray(alpha, dtype=np.float64)
    rc = lib.og_terms(nd, _ptr(n_a), _ptr(lo_a), _ptr(hi_a), _ptr(per_a), DYN_IDS[dyn],
                      _ptr(prm), len(prm), MODE_IDS[u_mode or p.u_mode],
                      MODE_IDS[d_mode or p.d_mode], order, _ptr(phi64), _ptr(al),
                      _ptr(out["pm"]), _ptr(out["pp"]), _ptr(out["u"]), _ptr(out["d"]),
                      _ptr(out["H"]), _ptr(out["a"]), _ptr(out["alpha"]), _ptr(out["rhs"]))
    if rc:
        raise OracleError(rc, "terms")
    shape = tuple(p.n)
    for k in ("pm", "pp", "a"):
        out[k] = out[k].reshape(shape + (nd,))
    for k in ("u", "d"):
        out[k] = out[k].reshape(shape + (MAX_INPUTS,))
    for k in ("H", "rhs"):
        out[k] = out[k].reshape(shape)
    return out


def _obstacle(problem, g):
    """float64 obstacle array: ``g`` if given, else the problem's own
    obstacle (float32 values promoted), else None."""
    if g is None and getattr(problem, "obstacle", None) is not None:
        g = problem.obstacle_values()
    return None if g is None else np.ascontiguousarray(g, dtype=np.float64).reshape(-1)


def _local(problem) -> int:
    """1 when the problem asks for per-node dissipation (reading R18)."""
    return 1 if getattr(problem, "dissipation", "global") == "local" else 0


def step(problem, phi, dt, l=None, g=None) -> dict:
    """One full time step of size ``dt`` from ``phi`` (float64 copy taken),
    as ``solve`` takes it.  Returns dict(out, alpha) with alpha of stage 1."""
    lib = _load()
    p = problem
    n_a, lo_a, hi_a, per_a = _grid_args(p.n, p.lo, p.hi, p.periodic)
    if l is None:
        l = p.target_values()
    l64 = np.ascontiguousarray(l, dtype=np.float64).reshape(-1)
    g64 = _obstacle(p, g)
    phi64 = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
    prm = np.ascontiguousarray(p.params, dtype=np.float64)
    out = np.zeros_like(phi64)
    alpha = np.zeros(len(n_a))
    rc = lib.og_step(len(n_a), _ptr(n_a), _ptr(lo_a), _ptr(hi_a), _ptr(per_a),
                     DYN_IDS[p.dynamics], _ptr(prm), len(prm), MODE_IDS[p.u_mode],
                     MODE_IDS[p.d_mode], _ptr(l64), _ptr(g64), _ptr(phi64), float(dt),
                     SET_IDS[p.set_kind],
                     p.space_order, p.time_order, _local(p), _ptr(out), _ptr(alpha))
    if rc:
        raise OracleError(rc, "step")
    return {"out": out.reshape(tuple(p.n)), "alpha": alpha}


def solve(problem, l=None, snapshots: bool = False, max_steps: int = 10_000_000,
          raise_on_error: bool = True, phi0=None, g=None, l_seq=None, g_seq=None) -> dict:
    """Run the full solve of ``problem`` (an ``inputs.Problem``).

    ``l`` defaults to ``problem.target_values()`` (float32) promoted to float64.
    ``g`` (optional) is an obstacle (reach-avoid); it defaults to the
    problem's own obstacle, if it has one.
    ``phi0`` (optional) is the value to start from instead of ``l``.
    ``l_seq`` / ``g_seq`` (optional, shape (n_tau,) + grid) are time-varying
    target and obstacle sets, one per tau (reading R26); with ``l_seq`` the
    solve starts from ``l_seq[0]``.
    Returns dict(final, snapshots (or None), steps (per segment), alpha,
    last_dt, rc).
    """
    lib = _load()
    p = problem
    n_a, lo_a, hi_a, per_a = _grid_args(p.n, p.lo, p.hi, p.periodic)
    if l is None:
        l = p.target_values()
    l64 = np.ascontiguousarray(l, dtype=np.float64).reshape(-1)
    g64 = _obstacle(p, g)
    p0 = None if phi0 is None else np.ascontiguousarray(phi0, dtype=np.float64).reshape(-1)
    tau = np.ascontiguousarray(p.tau, dtype=np.float64)
    prm = np.ascontiguousarray(p.params, dtype=np.float64)
    N = l64.size
    final = np.zeros(N)
    snaps = np.zeros((len(tau), N)) if snapshots else None
    steps = np.zeros(len(tau) - 1, dtype=np.int64)
    alpha = np.zeros(len(n_a))
    last_dt = ctypes.c_double(0.0)
    if l_seq is not None:
        ls = np.ascontiguousarray(l_seq, dtype=np.float64).reshape(len(tau), -1)
        gs = None if g_seq is None else np.ascontiguousarray(g_seq, dtype=np.float64).reshape(len(tau), -1)
        fn, a_l, a_g = lib.og_solve_seq, ls, gs
    else:
        if g_seq is not None:
            raise ValueError("g_seq needs l_seq")
        fn, a_l, a_g = lib.og_solve, l64, g64
    rc = fn(len(n_a), _ptr(n_a), _ptr(lo_a), _ptr(hi_a), _ptr(per_a),
                      DYN_IDS[p.dynamics], _ptr(prm), len(prm), MODE_IDS[p.u_mode],
                      MODE_IDS[p.d_mode], _ptr(a_l), _ptr(a_g), _ptr(p0), _ptr(tau), len(tau),
                      SET_IDS[p.set_kind],
                      p.space_order, p.time_order, _local(p), float(p.cfl), int(max_steps), _ptr(snaps),
                      _ptr(final), _ptr(steps), _ptr(alpha), ctypes.byref(last_dt))
    if rc and raise_on_error:
        raise OracleError(rc, "solve")
    shape = tuple(p.n)
    return {
        "final": final.reshape(shape),
        "snapshots": None if snaps is None else snaps.reshape((len(tau),) + shape),
        "steps": steps, "alpha": alpha, "last_dt": last_dt.value, "rc": rc,
    }


def ttr(problem, l=None, eps: float = 1e-5, big: float = 1e4, max_sweeps: int = 100_000,
        scheme: str = "gauss_seidel", raise_on_error: bool = True) -> dict:
    """Time-to-reach function of ``problem`` by Lax-Friedrichs sweeping
    (Algorithm 2; readings R21-R25 of ``odp_oracle.c``).

    The target set is {l <= 0}; ``l`` defaults to ``problem.target_values()``
    (float32) promoted to float64, so that target membership is decided on
    the values the CUDA library sees.  ``problem``'s grid, dynamics and
    parameters are used (u_mode "min", d_mode "max").  Returns dict(phi,
    sweeps, change (max |phi - phi_old| of the last sweep), rc).
    """
    lib = _load()
    p = problem
    n_a, lo_a, hi_a, per_a = _grid_args(p.n, p.lo, p.hi, p.periodic)
    if l is None:
        l = p.target_values()
    l64 = np.ascontiguousarray(l, dtype=np.float64).reshape(-1)
    prm = np.ascontiguousarray(p.params, dtype=np.float64)
    phi = np.zeros(l64.size)
    sweeps = ctypes.c_int64(0)
    change = ctypes.c_double(0.0)
    rc = lib.og_ttr(len(n_a), _ptr(n_a), _ptr(lo_a), _ptr(hi_a), _ptr(per_a), DYN_IDS[p.dynamics],
                    _ptr(prm), len(prm), MODE_IDS[p.u_mode], MODE_IDS[p.d_mode], _ptr(l64),
                    float(big), float(eps), int(max_sweeps), TTR_SCHEMES[scheme], _ptr(phi),
                    ctypes.byref(sweeps), ctypes.byref(change))
    if rc and raise_on_error:
        raise OracleError(rc, "ttr")
    return {"phi": phi.reshape(tuple(p.n)), "sweeps": int(sweeps.value), "change": change.value,
            "rc": rc}


def ttr_node(problem, phi, idx) -> float:
    """Algorithm 2's value for one interior node ``idx`` of ``phi``."""
    lib = _load()
    p = problem
    n_a, lo_a, hi_a, per_a = _grid_args(p.n, p.lo, p.hi, p.periodic)
    prm = np.ascontiguousarray(p.params, dtype=np.float64)
    phi64 = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
    i_a = np.ascontiguousarray(idx, dtype=np.int64)
    out = ctypes.c_double(0.0)
    rc = lib.og_ttr_node(len(n_a), _ptr(n_a), _ptr(lo_a), _ptr(hi_a), _ptr(per_a),
                         DYN_IDS[p.dynamics], _ptr(prm), len(prm), MODE_IDS[p.u_mode],
                         MODE_IDS[p.d_mode], _ptr(phi64), _ptr(i_a), ctypes.byref(out))
    if rc:
        raise OracleError(rc, "ttr_node")
    return out.value


def solve_methods(problem, target_method: str, obstacle_method: str = "maxVWithObstacle", l=None, g=None,
                  l_seq=None, g_seq=None, phi0=None, snapshots: bool = False, max_steps: int = 10_000_000,
                  raise_on_error: bool = True) -> dict:
    """``solve`` with any computation method of the solver's table (reading
    R27): ``target_method`` a key of TARGET_METHODS, ``obstacle_method`` a key
    of OBSTACLE_METHODS (used when an obstacle ``g`` or ``g_seq`` is given).
    Returns the dict of ``solve``."""
    lib = _load()
    p = problem
    n_a, lo_a, hi_a, per_a = _grid_args(p.n, p.lo, p.hi, p.periodic)
    if l is None and l_seq is None:
        l = p.target_values()
    tau = np.ascontiguousarray(p.tau, dtype=np.float64)
    l64 = None if l is None else np.ascontiguousarray(l, dtype=np.float64).reshape(-1)
    g64 = None if g is None else np.ascontiguousarray(g, dtype=np.float64).reshape(-1)
    ls = None if l_seq is None else np.ascontiguousarray(l_seq, dtype=np.float64).reshape(len(tau), -1)
    gs = None if g_seq is None else np.ascontiguousarray(g_seq, dtype=np.float64).reshape(len(tau), -1)
    p0 = None if phi0 is None else np.ascontiguousarray(phi0, dtype=np.float64).reshape(-1)
    prm = np.ascontiguousarray(p.params, dtype=np.float64)
    N = p.points
    final = np.zeros(N)
    snaps = np.zeros((len(tau), N)) if snapshots else None
    steps = np.zeros(len(tau) - 1, dtype=np.int64)
    alpha = np.zeros(len(n_a))
    last_dt = ctypes.c_double(0.0)
    rc = lib.og_solve_methods(len(n_a), _ptr(n_a), _ptr(lo_a), _ptr(hi_a), _ptr(per_a), DYN_IDS[p.dynamics],
                              _ptr(prm), len(prm), MODE_IDS[p.u_mode], MODE_IDS[p.d_mode], _ptr(l64), _ptr(g64),
                              _ptr(ls), _ptr(gs), _ptr(p0), _ptr(tau), len(tau), TARGET_METHODS[target_method],
                              OBSTACLE_METHODS[obstacle_method], p.space_order, p.time_order, _local(p),
                              float(p.cfl), int(max_steps), _ptr(snaps), _ptr(final), _ptr(steps), _ptr(alpha),
                              ctypes.byref(last_dt))
    if rc and raise_on_error:
        raise OracleError(rc, "solve_methods")
    shape = tuple(p.n)
    return {"final": final.reshape(shape),
            "snapshots": None if snaps is None else snaps.reshape((len(tau),) + shape),
            "steps": steps, "alpha": alpha, "last_dt": last_dt.value, "rc": rc}
