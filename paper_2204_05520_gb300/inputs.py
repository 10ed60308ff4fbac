"""Seeded synthetic inputs for the HJ level-set workloads.

This module holds none of the level-set method's arithmetic.  It only

* describes problems (grid extents, dynamics name and parameters, scheme,
  tau schedule) as plain data,
* samples analytic target functions l(z) at the grid nodes, and
* draws seeded random numbers (random value fields for tiny tests, the
  parameter draws of the batched and served workloads, Poisson arrivals).

Both sides of every parity check take their inputs from here: the CUDA
library through its binding and the FP64 oracle through the test suite.
Neither side imports the other.

Node placement used to sample a target (Section 3.1.1 of the paper: a
Cartesian grid given by node counts, bounds and periodic dimensions): node i
of an axis sits at lo + i*h with h = (hi - lo)/(n - 1) on a non-periodic
axis and h = (hi - lo)/n on a periodic one (the upper bound is the image of
the lower bound, so it is not a node).

Targets are evaluated in float64 and rounded once to float32; the oracle
promotes the same float32 values back to float64, so both sides start from
identical data.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional, Sequence

import numpy as np

# Dynamics names understood by both sides (each maps them to its own enum).
DYNAMICS = ("single_integrator", "dubins3d", "dubinscar4d", "rel6d", "advection", "dubins_capture")


@dataclasses.dataclass
class Problem:
    """One reachability solve: grid, dynamics, target, scheme and schedule."""

    name: str
    n: tuple
    lo: tuple
    hi: tuple
    periodic: tuple
    dynamics: str
    params: tuple
    u_mode: str  # "min" or "max": role of the control in the Hamiltonian
    d_mode: str  # "min" or "max": role of the disturbance
    target: Callable[[Sequence[np.ndarray]], np.ndarray]
    tau: tuple  # look-back times, tau[0] == 0, strictly increasing
    set_kind: str = "brt"  # "brt" (min with the target after each step) or "brs"
    space_order: int = 1
    time_order: int = 1
    cfl: float = 0.8
    # reach-avoid: obstacle g(z), positive inside the obstacle; after each step
    # phi <- max(phi, g) (after the BRT min with l)
    obstacle: Optional[Callable[[Sequence[np.ndarray]], np.ndarray]] = None
    # Lax-Friedrichs dissipation: "global" (grid alpha, Section 2.1) or
    # "local" (each node's own alpha, Algorithm 1's second loop)
    dissipation: str = "global"

    @property
    def ndim(self) -> int:
        return len(self.n)

    @property
    def points(self) -> int:
        return int(np.prod(self.n, dtype=np.int64))

    def nodes(self) -> list:
        return node_coords(self.n, self.lo, self.hi, self.periodic)

    def target_values(self) -> np.ndarray:
        """l(z) at every node, C order, rounded to float32."""
        mesh = np.meshgrid(*self.nodes(), indexing="ij")
        return np.ascontiguousarray(self.target(mesh), dtype=np.float64).astype(np.float32)

    def obstacle_values(self) -> np.ndarray:
        """g(z) at every node, C order, rounded to float32 (None without an
        obstacle)."""
        if self.obstacle is None:
            return None
        mesh = np.meshgrid(*self.nodes(), indexing="ij")
        return np.ascontiguousarray(self.obstacle(mesh), dtype=np.float64).astype(np.float32)


def node_coords(n, lo, hi, periodic) -> list:
    """Node positions of each axis (float64), see the module docstring."""
    out = []
    for nd, a, b, per in zip(n, lo, hi, periodic):
        h = (b - a) / nd if per else (b - a) / (nd - 1)
        out.append(a + h * np.arange(nd, dtype=np.float64))
    return out


# ----------------------------------------------------------------------------
# analytic targets (implicit surfaces, Section 3.1.2 of the paper)
# ----------------------------------------------------------------------------

def cylinder(radius: float, dims=(0, 1), center=None) -> Callable:
    """Signed distance to a cylinder whose axis spans the ignored dimensions."""

    def f(mesh):
        acc = np.zeros_like(mesh[0])
        for k, d in enumerate(dims):
            c = 0.0 if center is None else center[k]
            acc = acc + (mesh[d] - c) ** 2
        return np.sqrt(acc) - radius

    return f


def ball(radius: float) -> Callable:
    """Signed distance to a ball centred at the origin over all dimensions."""

    def f(mesh):
        acc = np.zeros_like(mesh[0])
        for m in mesh:
            acc = acc + m * m
        return np.sqrt(acc) - radius

    return f


def cylinder_obstacle(radius: float, center, dims=(0, 1)) -> Callable:
    """Obstacle function of a cylinder: radius minus the distance to its axis
    (positive inside)."""
    inside = cylinder(radius, dims=dims, center=center)
    return lambda mesh: -inside(mesh)


def box_obstacle(lo: Sequence[float], hi: Sequence[float], dims: Sequence[int]) -> Callable:
    """Obstacle function of an axis-aligned box over the given dimensions:
    the smallest distance from a face, positive inside, negative outside."""

    def f(mesh):
        acc = None
        for a, b, d in zip(lo, hi, dims):
            v = np.minimum(mesh[d] - a, b - mesh[d])
            acc = v if acc is None else np.minimum(acc, v)
        return acc

    return f


def sine_bump(freqs: Sequence[int]) -> Callable:
    """A smooth periodic field sum_d sin(k_d * z_d) used by transport pins."""

    def f(mesh):
        acc = np.zeros_like(mesh[0])
        for m, k in zip(mesh, freqs):
            acc = acc + np.sin(k * m)
        return acc

    return f


def random_field(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Seeded uniform float32 field for tiny-grid tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=tuple(shape)).astype(np.float32)


# ----------------------------------------------------------------------------
# the three single-solve workloads
# ----------------------------------------------------------------------------

PI = math.pi


def dubins3d(n=(41, 41, 36), v=1.0, w_max=1.0, radius=1.0, horizon=2.0,
             u_mode="min", set_kind="brt", space_order=1, time_order=1,
             lo=(-4.0, -4.0, -PI), hi=(4.0, 4.0, PI), tau=None) -> Problem:
    """Dubins car BRT: x' = v cos(th), y' = v sin(th), th' = w, |w| <= w_max;
    target sqrt(x^2 + y^2) - radius; theta periodic on [-pi, pi)."""
    return Problem(
        name="dubins3d_%dx%dx%d" % tuple(n), n=tuple(n), lo=tuple(lo), hi=tuple(hi),
        periodic=(False, False, True), dynamics="dubins3d", params=(v, w_max),
        u_mode=u_mode, d_mode="max", target=cylinder(radius), tau=tau or (0.0, horizon),
        set_kind=set_kind, space_order=space_order, time_order=time_order)


def dubinscar4d(n=(80, 80, 40, 64), a_max=1.0, w_max=1.0, radius=1.0, horizon=3.0,
                u_mode="min", set_kind="brt", space_order=2, time_order=2,
                lo=(-5.0, -5.0, 0.0, -PI), hi=(5.0, 5.0, 3.0, PI), tau=None) -> Problem:
    """4D Dubins car BRT, state (x, y, v, th): x' = v cos th, y' = v sin th,
    v' = a, th' = w; |a| <= a_max, |w| <= w_max; cylinder target in (x, y)."""
    return Problem(
        name="dubinscar4d_%dx%dx%dx%d" % tuple(n), n=tuple(n), lo=tuple(lo), hi=tuple(hi),
        periodic=(False, False, False, True), dynamics="dubinscar4d", params=(a_max, w_max),
        u_mode=u_mode, d_mode="max", target=cylinder(radius), tau=tau or (0.0, horizon),
        set_kind=set_kind, space_order=space_order, time_order=time_order)


def rel6d(n=(24,) * 6, bounds=(1.0, 1.0, 1.0, 1.0), radius=0.5, horizon=1.5,
          set_kind="brt", space_order=1, time_order=2, tau=None,
          lo=(-4.0, -4.0, -PI, 0.5, -1.0, 0.5), hi=(4.0, 4.0, PI, 1.5, 1.0, 1.5)) -> Problem:
    """6D relative pursuit-evasion, state (x, y, th, v_p, w_p, v_e); pursuer
    controls (a_p, alpha_p) minimise, evader inputs (a_e, w_e) maximise;
    capture target sqrt(x^2 + y^2) - radius."""
    return Problem(
        name="rel6d_%d^6" % n[0] if len(set(n)) == 1 else "rel6d_" + "x".join(map(str, n)),
        n=tuple(n), lo=tuple(lo), hi=tuple(hi),
        periodic=(False, False, True, False, False, False), dynamics="rel6d",
        params=tuple(bounds), u_mode="min", d_mode="max", target=cylinder(radius),
        tau=tau or (0.0, horizon), set_kind=set_kind, space_order=space_order,
        time_order=time_order)


def dubins_capture(n=(40, 40, 40), v=1.0, a_max=1.0, b_max=1.0, radius=0.5, horizon=1.5,
                   u_mode="max", d_mode="min", set_kind="brt", space_order=1, time_order=1,
                   tau=None) -> Problem:
    """Pursuit-evasion of two Dubins cars in relative coordinates (Section 4.2):
    x' = -v + v cos th + a y, y' = v sin th - a x, th' = b - a; evader turn a
    (|a| <= a_max, maximising), pursuer turn b (|b| <= b_max, minimising);
    capture target sqrt(x^2 + y^2) - radius on [-4, 4]^2 x [-pi, pi)."""
    return Problem(
        name="dubins_capture_%dx%dx%d" % tuple(n), n=tuple(n), lo=(-4.0, -4.0, -PI), hi=(4.0, 4.0, PI),
        periodic=(False, False, True), dynamics="dubins_capture", params=(v, a_max, b_max),
        u_mode=u_mode, d_mode=d_mode, target=cylinder(radius), tau=tau or (0.0, horizon),
        set_kind=set_kind, space_order=space_order, time_order=time_order)


def single_integrator(n, half_width=2.0, u_max=1.0, radius=0.5, horizon=0.5,
                      u_mode="min", set_kind="brt", space_order=1, time_order=1,
                      tau=None) -> Problem:
    """x' = u, |u_i| <= u_max on [-w, w]^d with a ball target."""
    d = len(n)
    return Problem(
        name="single_integrator_" + "x".join(map(str, n)), n=tuple(n),
        lo=(-half_width,) * d, hi=(half_width,) * d, periodic=(False,) * d,
        dynamics="single_integrator", params=(u_max,), u_mode=u_mode, d_mode="max",
        target=ball(radius), tau=tau or (0.0, horizon), set_kind=set_kind,
        space_order=space_order, time_order=time_order)


def advection(n, velocity, freqs=None, horizon=1.0, cfl=1.0, space_order=1,
              time_order=1, tau=None) -> Problem:
    """Constant transport z' = c on the periodic box [0, 2 pi)^d."""
    d = len(n)
    return Problem(
        name="advection_" + "x".join(map(str, n)), n=tuple(n), lo=(0.0,) * d,
        hi=(2 * PI,) * d, periodic=(True,) * d, dynamics="advection",
        params=tuple(velocity), u_mode="max", d_mode="max",
        target=sine_bump(freqs or (1,) * d), tau=tau or (0.0, horizon), set_kind="brs",
        space_order=space_order, time_order=time_order, cfl=cfl)


def reach_avoid(problem: Problem, obstacle: Callable) -> Problem:
    """The same solve as a reach-avoid problem with obstacle function g."""
    return dataclasses.replace(problem, name=problem.name + "_reach_avoid", obstacle=obstacle)


def dubins_obstacle() -> Callable:
    """Cylinder obstacle of radius 0.75 centred at (x, y) = (2, 0.5), beside
    the target of the Dubins workloads."""
    return cylinder_obstacle(0.75, center=(2.0, 0.5))


def workload(name: str) -> Problem:
    """The named single-solve workloads at full size."""
    if name == "dubins3d":
        return dubins3d()
    if name == "dubinscar4d":
        return dubinscar4d()
    if name == "rel6d":
        return rel6d()
    if name == "dubinscar4d_reach_avoid":
        return reach_avoid(dubinscar4d(), dubins_obstacle())
    if name.startswith("ttr_"):
        return ttr_workload(name[4:])
    raise KeyError(name)


TTR_SIDES = {"dubins3d": (60, 80, 100), "dubinscar4d": (60, 80, 100)}


def ttr_workload(name: str) -> Problem:
    """Time-to-reach grids of the paper's Section 6 tables (3D Dubins car
    60^3-100^3, 4D Dubins car 60^4-100^4), named "dubins3d_<side>" or
    "dubinscar4d_<side>" (any side >= 4): the Dubins models above on cubic
    grids, cylinder target of radius 1 (the tau schedule is unused)."""
    model, side = name.rsplit("_", 1)
    side = int(side)
    if model == "dubins3d":
        return dataclasses.replace(dubins3d(n=(side,) * 3), name="ttr_dubins3d_%d" % side)
    if model == "dubinscar4d":
        return dataclasses.replace(dubinscar4d(n=(side,) * 4), name="ttr_dubinscar4d_%d" % side)
    raise KeyError(name)


# ----------------------------------------------------------------------------
# batched and served workloads (seeded parameter draws)
# ----------------------------------------------------------------------------

BATCH_SIDES = (31, 41, 51, 61, 81, 101)


def batch_problems(count: int = 512, seed: int = 0, horizon: float = 2.0) -> list:
    """Independent Dubins3D BRT solves with uneven grids: side drawn from
    {31, 41, 51, 61, 81, 101}, 36-64 theta cells, v ~ U[0.5, 2],
    w_max ~ U[0.5, 1.5], target radius ~ U[0.5, 1.5], (x, y) in [-4, 4]^2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        side = int(rng.choice(BATCH_SIDES))
        n_th = int(rng.integers(36, 65))
        v = float(rng.uniform(0.5, 2.0))
        w = float(rng.uniform(0.5, 1.5))
        r = float(rng.uniform(0.5, 1.5))
        out.append(dubins3d(n=(side, side, n_th), v=v, w_max=w, radius=r, horizon=horizon))
    return out


def served_requests(rate: float, count: int = 2000, seed: int = 1,
                    side3=(31, 101), side4=(40, 80)) -> list:
    """Poisson request stream: (arrival_time_s, Problem) pairs.  50/50 mix of
    Dubins3D (cubic grid, side ~ U{31..101}) and DubinsCar4D (side ~ U{40..80}
    in all four dims); horizons ~ U[0.5, 3]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate))
        horizon = float(rng.uniform(0.5, 3.0))
        r = float(rng.uniform(0.5, 1.5))
        w = float(rng.uniform(0.5, 1.5))
        if rng.uniform() < 0.5:
            side = int(rng.integers(side3[0], side3[1] + 1))
            v = float(rng.uniform(0.5, 2.0))
            p = dubins3d(n=(side, side, side), v=v, w_max=w, radius=r, horizon=horizon)
        else:
            side = int(rng.integers(side4[0], side4[1] + 1))
            a = float(rng.uniform(0.5, 1.5))
            p = dubinscar4d(n=(side,) * 4, a_max=a, w_max=w, radius=r, horizon=horizon)
        out.append((t, p))
    return out
