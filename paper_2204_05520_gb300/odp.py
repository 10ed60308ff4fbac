"""ctypes binding of libodp (include/odp.h).

Each function has the name of the C entry point without the ``odp_`` prefix
and only marshals arguments: shapes and dtypes are checked, torch tensors are
passed by ``data_ptr()`` (device) or as host buffers, numpy arrays as host
buffers, and a negative status raises :class:`OdpError`.  All arithmetic of
the solve runs in the library's CUDA kernels; there is no other code path.
If the library has not been built, :func:`load` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

OK, EINVAL, ENOMEM, ECUDA, ESTATE, ETIMEOUT, ENUMERIC, EBUSY = 0, -1, -2, -3, -4, -5, -6, -7
DYN = {"single_integrator": 0, "dubins3d": 1, "dubinscar4d": 2, "rel6d": 3, "advection": 4,
       "dubins_capture": 5}
MODE = {"min": 0, "max": 1}
SET = {"brs": 0, "brt": 1}

_lock = threading.Lock()
_lib = None


class OdpError(RuntimeError):
    def __init__(self, code: int, where: str, message: str):
        super().__init__("%s failed (%d): %s" % (where, code, message))
        self.code = code


class SolveStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("last_dt", ctypes.c_double),
                ("t_final", ctypes.c_double), ("alpha", ctypes.c_float * 8),
                ("device_ms", ctypes.c_double), ("bytes", ctypes.c_double),
                ("launches", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {"steps": self.steps, "last_dt": self.last_dt, "t_final": self.t_final,
                "alpha": list(self.alpha), "device_ms": self.device_ms, "bytes": self.bytes,
                "launches": self.launches}


class TtrStats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int64), ("change", ctypes.c_double), ("device_ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("launches", ctypes.c_int64), ("tile_planes", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchStats(ctypes.Structure):
    _fields_ = [("device_ms", ctypes.c_double), ("rounds", ctypes.c_int64),
                ("ctas_per_sm", ctypes.c_int32), ("rows_per_thread", ctypes.c_int32),
                ("point_updates", ctypes.c_double), ("bytes", ctypes.c_double),
                ("plane_chunk", ctypes.c_int32), ("graph", ctypes.c_int32), ("launches", ctypes.c_int64),
                ("tuned", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


MAXD = 6
REQ_QUEUED, REQ_RESIDENT, REQ_DONE, REQ_FAILED = 0, 1, 2, 3


class Request(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("n", ctypes.c_int32 * MAXD), ("lo", ctypes.c_double * MAXD),
                ("hi", ctypes.c_double * MAXD), ("periodic", ctypes.c_uint8 * MAXD),
                ("kind", ctypes.c_int), ("n_params", ctypes.c_int32), ("params", ctypes.c_double * 8),
                ("u_mode", ctypes.c_int), ("d_mode", ctypes.c_int), ("target", ctypes.c_void_p),
                ("T", ctypes.c_double), ("set", ctypes.c_int), ("space_order", ctypes.c_int32),
                ("time_order", ctypes.c_int32), ("cfl", ctypes.c_double)]


class RequestStats(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("reserved", ctypes.c_int32), ("steps", ctypes.c_int64),
                ("steps_done", ctypes.c_int64), ("queue_s", ctypes.c_double),
                ("latency_s", ctypes.c_double), ("t_submit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("bytes", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class ServerStats(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_double), ("used_bytes", ctypes.c_double),
                ("queued", ctypes.c_int64), ("resident", ctypes.c_int64), ("launches", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def library_path() -> str:
    return _build.LIB


def load():
    """Load libodp.so (built by ``__graft_entry__.build()`` or ``_build.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError("libodp.so is not built (%s); run __graft_entry__.build()" % path)
        lib = ctypes.CDLL(path)
        P, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        sig = {
            "odp_last_error": ([], ctypes.c_char_p),
            "odp_version": ([], ctypes.c_char_p),
            "odp_grid_create": ([i32, P, P, P, P, P, P], i32),
            "odp_grid_destroy": ([P], i32),
            "odp_grid_points": ([P], i64),
            "odp_set_dynamics": ([P, i32, P, i32, i32, i32], i32),
            "odp_set_target": ([P, P, i64, i32], i32),
            "odp_set_obstacle": ([P, P, i64, i32], i32),
            "odp_set_target_schedule": ([P, P, i32, i64, i32], i32),
            "odp_set_obstacle_schedule": ([P, P, i32, i64, i32], i32),
            "odp_set_dissipation": ([P, i32], i32),
            "odp_set_step_limit": ([P, i64], i32),
            "odp_set_loop_mode": ([P, i32], i32),
            "odp_set_stage_pass": ([P, i32], i32),
            "odp_solve_hjb": ([P, P, i32, i32, i32, i32, f64, i32, P], i32),
            "odp_solve_status": ([P, P], i32),
            "odp_value_readback": ([P, i32, P, i64, i32], i32),
            "odp_time_stage": ([P, i32, i32, P], i32),
            "odp_solve_ttr": ([P, f64, f64, i64, P], i32),
            "odp_plan_geometry": ([i32, P, P, i32], i32),
            "odp_batch_solve": ([P, i32, P, i32, i32, i32, f64, P], i32),
            "odp_batch_set_autotune": ([i32], i32),
            "odp_server_create": ([ctypes.c_size_t, P, P], i32),
            "odp_server_destroy": ([P], i32),
            "odp_server_submit": ([P, P, P], i32),
            "odp_server_step": ([P, i32, P], i32),
            "odp_server_poll": ([P, ctypes.c_uint64, P], i32),
            "odp_server_readback": ([P, ctypes.c_uint64, P, i64, i32], i32),
            "odp_server_release": ([P, ctypes.c_uint64], i32),
            "odp_server_info": ([P, P], i32),
            "odp_server_set_max_resident": ([P, i64], i32),
            "odp_solve_noalloc": ([i32, P, P, P, P, i32, P, i32, i32, i32, P, f64, i32, i32, i32, f64,
                                   P, P], i32),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(rc: int, where: str):
    if rc != OK:
        raise OdpError(rc, where, load().odp_last_error().decode())
    return rc


def last_error() -> str:
    return load().odp_last_error().decode()


def version() -> str:
    return load().odp_version().decode()


def _stream_ptr(stream):
    if stream is None:
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _buffer(x, n_elems: int, writable: bool):
    """(pointer, on_device) of a float32 C-contiguous tensor or array."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float32 or not x.flags["C_CONTIGUOUS"] or x.size != n_elems:
            raise ValueError("need a C-contiguous float32 array of %d values" % n_elems)
        if writable and not x.flags["WRITEABLE"]:
            raise ValueError("array is read-only")
        return ctypes.c_void_p(x.ctypes.data), 0
    import torch

    if not isinstance(x, torch.Tensor):
        raise TypeError("need a numpy array or a torch tensor")
    if x.dtype != torch.float32 or not x.is_contiguous() or x.numel() != n_elems:
        raise ValueError("need a contiguous float32 tensor of %d values" % n_elems)
    return ctypes.c_void_p(x.data_ptr()), 1 if x.is_cuda else 0


def grid_create(n, lo, hi, periodic, stream=None):
    lib = load()
    nd = len(n)
    n_a = (ctypes.c_int32 * nd)(*[int(v) for v in n])
    lo_a = (ctypes.c_double * nd)(*[float(v) for v in lo])
    hi_a = (ctypes.c_double * nd)(*[float(v) for v in hi])
    per_a = (ctypes.c_uint8 * nd)(*[1 if p else 0 for p in periodic])
    out = ctypes.c_void_p()
    _check(lib.odp_grid_create(nd, n_a, lo_a, hi_a, per_a, _stream_ptr(stream), ctypes.byref(out)),
           "odp_grid_create")
    return out


def grid_destroy(g):
    _check(load().odp_grid_destroy(g), "odp_grid_destroy")


def grid_points(g) -> int:
    return int(load().odp_grid_points(g))


def set_dynamics(g, kind, params, u_mode="min", d_mode="max"):
    k = DYN[kind] if isinstance(kind, str) else int(kind)
    prm = (ctypes.c_double * max(1, len(params)))(*[float(v) for v in params])
    _check(load().odp_set_dynamics(g, k, prm, len(params), MODE[u_mode], MODE[d_mode]),
           "odp_set_dynamics")


def set_target(g, l):
    n = grid_points(g)
    ptr, dev = _buffer(l, n, writable=False)
    _check(load().odp_set_target(g, ptr, n, dev), "odp_set_target")


def set_obstacle(g, gv):
    """Reach-avoid obstacle g(z) (float32 array or tensor of the grid's
    shape), or None to remove it."""
    if gv is None:
        _check(load().odp_set_obstacle(g, None, 0, 0), "odp_set_obstacle")
        return
    n = grid_points(g)
    ptr, dev = _buffer(gv, n, writable=False)
    _check(load().odp_set_obstacle(g, ptr, n, dev), "odp_set_obstacle")


def _schedule(g, seq, fn, where):
    n = grid_points(g)
    if seq is None:
        _check(fn(g, None, 0, n, 0), where)
        return
    k = int(seq.shape[0])
    ptr, dev = _buffer(seq, k * n, writable=False)
    _check(fn(g, ptr, k, n, dev), where)


def set_target_schedule(g, l_seq):
    """Time-varying target: one set per tau, shape (n_tau,) + grid (None removes)."""
    _schedule(g, l_seq, load().odp_set_target_schedule, "odp_set_target_schedule")


def set_obstacle_schedule(g, g_seq):
    """Time-varying obstacle: one set per tau, shape (n_tau,) + grid (None removes)."""
    _schedule(g, g_seq, load().odp_set_obstacle_schedule, "odp_set_obstacle_schedule")


def set_dissipation(g, per_node: bool):
    """Lax-Friedrichs dissipation with the grid alpha (False) or each node's
    own alpha (True)."""
    _check(load().odp_set_dissipation(g, 1 if per_node else 0), "odp_set_dissipation")


def set_step_limit(g, max_steps: int):
    _check(load().odp_set_step_limit(g, int(max_steps)), "odp_set_step_limit")


def set_loop_mode(g, host_stepped: bool):
    """Run the time loop as one CUDA graph (False, default) or stepped from the
    host with the same kernels (True; for profilers)."""
    _check(load().odp_set_loop_mode(g, 1 if host_stepped else 0), "odp_set_loop_mode")


def set_stage_pass(g, pass_: int):
    """0: automatic, 1: plane-streaming pass, 2: bulk-staged pass."""
    _check(load().odp_set_stage_pass(g, int(pass_)), "odp_set_stage_pass")


def solve_hjb(g, tau, set_kind="brt", space_order=1, time_order=1, cfl=0.8, keep_snapshots=False,
              stats=False):
    """Enqueue a solve; with ``stats`` wait for it and return its statistics."""
    t = (ctypes.c_double * len(tau))(*[float(v) for v in tau])
    st = SolveStats() if stats else None
    _check(load().odp_solve_hjb(g, t, len(tau), SET[set_kind], int(space_order), int(time_order),
                                float(cfl), 1 if keep_snapshots else 0,
                                ctypes.byref(st) if st is not None else None), "odp_solve_hjb")
    return st.as_dict() if st is not None else None


def solve_ttr(g, eps=1e-5, big=1e4, max_sweeps=100000, stats=False):
    """Enqueue the time-to-reach sweep (Algorithm 2); with ``stats`` wait for
    it and return its statistics."""
    st = TtrStats() if stats else None
    _check(load().odp_solve_ttr(g, float(eps), float(big), int(max_sweeps),
                                ctypes.byref(st) if st is not None else None), "odp_solve_ttr")
    return st.as_dict() if st is not None else None


def solve_status(g) -> dict:
    st = SolveStats()
    _check(load().odp_solve_status(g, ctypes.byref(st)), "odp_solve_status")
    return st.as_dict()


def value_readback(g, out, tau_index: int = -1):
    n = grid_points(g)
    ptr, dev = _buffer(out, n, writable=True)
    _check(load().odp_value_readback(g, int(tau_index), ptr, n, dev), "odp_value_readback")
    return out


def time_stage(g, stage: int, reps: int = 20) -> float:
    """Mean device milliseconds of one launch of the fused stage kernel."""
    ms = ctypes.c_double(0.0)
    _check(load().odp_time_stage(g, int(stage), int(reps), ctypes.byref(ms)), "odp_time_stage")
    return ms.value


def batch_solve(grids, horizons, set_kind="brt", space_order=1, time_order=1, cfl=0.8) -> dict:
    """Solve many grids (``Grid`` objects or handles) in one persistent launch."""
    hs = [g.handle if isinstance(g, Grid) else g for g in grids]
    arr = (ctypes.c_void_p * len(hs))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in hs])
    T = (ctypes.c_double * len(hs))(*[float(t) for t in horizons])
    st = BatchStats()
    _check(load().odp_batch_solve(arr, len(hs), T, SET[set_kind], int(space_order), int(time_order),
                                  float(cfl), ctypes.byref(st)), "odp_batch_solve")
    return st.as_dict()


def solve_noalloc(problem, l, out, stream=None):
    """Solve ``problem`` over [0, T] without allocating device memory: ``l``
    and ``out`` are the caller's device tensors (float32, problem.n), all
    other state lives in the library's fixed device array.  The entry point
    takes a plain solve over tau = {0, T}: a problem with an obstacle,
    per-node dissipation or intermediate tau points is refused (ValueError),
    since its answer would differ from the grid object's solve."""
    if getattr(problem, "obstacle", None) is not None:
        raise ValueError("solve_noalloc: reach-avoid (an obstacle) is not supported")
    if getattr(problem, "dissipation", "global") != "global":
        raise ValueError("solve_noalloc: only grid-wide dissipation is supported")
    if len(problem.tau) != 2 or float(problem.tau[0]) != 0.0:
        raise ValueError("solve_noalloc: the schedule must be tau = (0, T)")
    nd = problem.ndim
    n_pts = problem.points
    lp, ldev = _buffer(l, n_pts, writable=False)
    op, odev = _buffer(out, n_pts, writable=True)
    if not (ldev and odev):
        raise ValueError("l and out must be device tensors")
    n_a = (ctypes.c_int32 * nd)(*[int(v) for v in problem.n])
    lo_a = (ctypes.c_double * nd)(*[float(v) for v in problem.lo])
    hi_a = (ctypes.c_double * nd)(*[float(v) for v in problem.hi])
    per_a = (ctypes.c_uint8 * nd)(*[1 if p else 0 for p in problem.periodic])
    prm = (ctypes.c_double * max(1, len(problem.params)))(*[float(v) for v in problem.params])
    _check(load().odp_solve_noalloc(nd, n_a, lo_a, hi_a, per_a, DYN[problem.dynamics], prm,
                                    len(problem.params), MODE[problem.u_mode], MODE[problem.d_mode],
                                    lp, float(problem.tau[-1]), SET[problem.set_kind],
                                    int(problem.space_order), int(problem.time_order),
                                    float(problem.cfl), op, _stream_ptr(stream)), "odp_solve_noalloc")
    return out


class Server:
    """Continuous-batching solve server (odp_server_*): submit problems, step
    the scheduler, poll, read back, release."""

    def __init__(self, hbm_budget_bytes: int, stream=None):
        self.handle = ctypes.c_void_p()
        _check(load().odp_server_create(int(hbm_budget_bytes), _stream_ptr(stream),
                                        ctypes.byref(self.handle)), "odp_server_create")
        self._targets = {}

    def close(self):
        if self.handle:
            _check(load().odp_server_destroy(self.handle), "odp_server_destroy")
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, problem, target=None) -> int:
        nd = problem.ndim
        l = np.ascontiguousarray(problem.target_values() if target is None else target, dtype=np.float32)
        q = Request()
        q.ndim = nd
        for d in range(nd):
            q.n[d] = int(problem.n[d])
            q.lo[d] = float(problem.lo[d])
            q.hi[d] = float(problem.hi[d])
            q.periodic[d] = 1 if problem.periodic[d] else 0
        q.kind = DYN[problem.dynamics]
        q.n_params = len(problem.params)
        for k, v in enumerate(problem.params):
            q.params[k] = float(v)
        q.u_mode = MODE[problem.u_mode]
        q.d_mode = MODE[problem.d_mode]
        q.target = l.ctypes.data
        q.T = float(problem.tau[-1])
        q.set = SET[problem.set_kind]
        q.space_order = int(problem.space_order)
        q.time_order = int(problem.time_order)
        q.cfl = float(problem.cfl)
        rid = ctypes.c_uint64()
        _check(load().odp_server_submit(self.handle, ctypes.byref(q), ctypes.byref(rid)), "odp_server_submit")
        return rid.value

    def set_max_resident(self, max_nodes: int):
        """Cap the grid nodes of resident (admitted, unfinished) solves; 0: none."""
        _check(load().odp_server_set_max_resident(self.handle, int(max_nodes)), "odp_server_set_max_resident")

    def step(self, rounds: int = 8) -> int:
        done = ctypes.c_int(0)
        _check(load().odp_server_step(self.handle, int(rounds), ctypes.byref(done)), "odp_server_step")
        return done.value

    def poll(self, rid: int) -> dict:
        st = RequestStats()
        _check(load().odp_server_poll(self.handle, ctypes.c_uint64(rid), ctypes.byref(st)), "odp_server_poll")
        return st.as_dict()

    def readback(self, rid: int, out):
        ptr, dev = _buffer(out, out.size if isinstance(out, np.ndarray) else out.numel(), writable=True)
        n = out.size if isinstance(out, np.ndarray) else out.numel()
        _check(load().odp_server_readback(self.handle, ctypes.c_uint64(rid), ptr, n, dev),
               "odp_server_readback")
        return out

    def release(self, rid: int):
        _check(load().odp_server_release(self.handle, ctypes.c_uint64(rid)), "odp_server_release")

    def info(self) -> dict:
        st = ServerStats()
        _check(load().odp_server_info(self.handle, ctypes.byref(st)), "odp_server_info")
        return st.as_dict()


def batch_set_autotune(enabled: bool):
    _check(load().odp_batch_set_autotune(1 if enabled else 0), "odp_batch_set_autotune")


PLAN_FIELDS = ("n_pad", "rows_per_thread", "row_groups", "planes", "threads_rb", "plane_pass",
               "stream_len", "chunk", "ctas", "cta_threads", "smem_r1", "smem_r2", "band_rows", "bands")


def plan_geometry(n) -> dict:
    """Launch geometry for a grid of shape n (host only)."""
    nd = len(n)
    n_a = (ctypes.c_int32 * nd)(*[int(v) for v in n])
    out = (ctypes.c_int64 * len(PLAN_FIELDS))()
    _check(load().odp_plan_geometry(nd, n_a, out, len(PLAN_FIELDS)), "odp_plan_geometry")
    return dict(zip(PLAN_FIELDS, list(out)))


class Grid:
    """Owning wrapper of an odp_grid handle (one problem on one stream)."""

    def __init__(self, n, lo, hi, periodic, stream=None):
        self.shape = tuple(int(v) for v in n)
        self.handle = grid_create(n, lo, hi, periodic, stream)

    @classmethod
    def for_problem(cls, problem, stream=None) -> "Grid":
        g = cls(problem.n, problem.lo, problem.hi, problem.periodic, stream)
        set_dynamics(g.handle, problem.dynamics, problem.params, problem.u_mode, problem.d_mode)
        if getattr(problem, "obstacle", None) is not None:
            set_obstacle(g.handle, problem.obstacle_values())
        if getattr(problem, "dissipation", "global") == "local":
            set_dissipation(g.handle, True)
        return g

    def close(self):
        if self.handle is not None:
            grid_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_target(self, l):
        set_target(self.handle, l)

    def set_obstacle(self, gv):
        set_obstacle(self.handle, gv)

    def set_target_schedule(self, l_seq):
        set_target_schedule(self.handle, l_seq)

    def set_obstacle_schedule(self, g_seq):
        set_obstacle_schedule(self.handle, g_seq)

    def solve(self, tau, set_kind="brt", space_order=1, time_order=1, cfl=0.8,
              keep_snapshots=False, stats=False):
        return solve_hjb(self.handle, tau, set_kind, space_order, time_order, cfl, keep_snapshots,
                         stats)

    def solve_problem(self, problem, keep_snapshots=False, stats=False):
        return self.solve(problem.tau, problem.set_kind, problem.space_order, problem.time_order,
                          problem.cfl, keep_snapshots, stats)

    def readback(self, out, tau_index: int = -1):
        return value_readback(self.handle, out, tau_index)

    def solve_ttr(self, eps=1e-5, big=1e4, max_sweeps=100000, stats=False):
        return solve_ttr(self.handle, eps, big, max_sweeps, stats)
