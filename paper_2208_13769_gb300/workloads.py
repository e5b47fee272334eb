"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds none of the method's arithmetic: it only builds problem
statements -- grid sizes, material constants, boundary kinds and values, and
the initial displacement u0 and velocity v0 fields -- from fixed seeds.  Both
the CUDA library and the CPU oracle consume what it produces.

Geometry conventions (node placement of Sec. 7, probe points at half-spacing
offsets): along a bounded axis node k sits at (k + 1/2) dX, with walls at 0 and
n dX; along a periodic axis node k sits at k dX.

Workloads named after the paper's setting:
  * shear_wave      -- periodic square body, transverse standing wave
                       u_x = A sin(2 pi y / L) (64 x 64, lambda 0.5, mu 0.3).
  * clamped_body    -- rectangular body, x- edge clamped (Dirichlet u* = 0),
                       other edges traction-free, initial transverse velocity
                       v_y = v_max x / L (4096 x 2048 and 8192 x 8192 variants).
  * body_batch      -- many independent bodies with seeded sizes, materials,
                       boundary sets and low-mode initial displacements.
  * serving_trace   -- Poisson arrivals of bodies like body_batch's.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Tuple

import numpy as np

PERIODIC, DIRICHLET, NEUMANN = 0, 1, 2
EDGE_NAMES = ("x-", "x+", "y-", "y+")

# omega = dt / tau of the BGK collision (Eq. col).  The paper never fixes the
# relaxation time, so each workload names its own:
#  * OMEGA = 1, the default: the collision replaces f by f^eq (plus the
#    forcing), so the populations' non-equilibrium part, and the rounding
#    noise a reduced-precision storage leaves in it, is gone after each step;
#  * OMEGA_SEC7 = 1.95 for the paper's three runs of Sec. 7 (tension, shear,
#    plate with a hole): they complete at the paper's loads only for omega in
#    about [1.92, 1.99] (at omega = 1 they blow up before t = 2.1);
#  * OMEGA_BODIES = 1.9 for the clamped body and the bodies of the batch and
#    the serving trace: at 4096 x 2048 the clamped body runs 8000 steps for
#    omega in [1.85, 1.93] with either scheme and FP32 or FP16 storage, where
#    at omega = 1 it blows up at its clamped corners after 3250 steps; and
#    FP16 storage keeps its displacement within 1e-4 of the FP64 path (the
#    rounding lands in the non-equilibrium part, which alternates in sign
#    each step and cancels in the displacement), against 1e-2 at omega = 1.
OMEGA = 1.0
OMEGA_SEC7 = 1.95
OMEGA_BODIES = 1.9


@dataclasses.dataclass
class Edge:
    kind: int
    value: tuple = (0.0, 0.0)   # Dirichlet: u* at t=0; Neumann: T0
    rate: tuple = (0.0, 0.0)    # Dirichlet: v*;        Neumann: T1
    times: tuple = (0.0, 0.0, math.inf)  # Neumann: t_on, t_ramp, t_off

    def as_dict(self) -> dict:
        return {"kind": self.kind, "value": self.value, "rate": self.rate, "times": self.times}


@dataclasses.dataclass
class Problem:
    nx: int
    ny: int
    lam: float
    mu: float
    rho0: float = 1.0
    omega: float = OMEGA
    dX: float = 1.0
    body: tuple = (0.0, 0.0)
    edges: List[Edge] = dataclasses.field(default_factory=list)
    u0: Optional[np.ndarray] = None   # [ny][nx][2] float64
    v0: Optional[np.ndarray] = None   # [ny][nx][2] float64
    name: str = ""
    # built on demand instead of u0 / v0 (long request traces): () -> (u0, v0)
    make_initial: Optional[Callable[[], Tuple[np.ndarray, np.ndarray]]] = None
    # a rectangular hole: removed nodes x0 <= x < x1, y0 <= y < y1, and the
    # constant traction on its faces at x0, x1, y0, y1 (None: traction-free)
    hole: Optional[Tuple[int, int, int, int]] = None
    hole_traction: Optional[List[Tuple[float, float]]] = None

    def initial(self) -> Tuple[Optional[np.ndarray], Optional[np.ndarray]]:
        """(u0, v0), built now if the problem holds a recipe instead."""
        if self.make_initial is not None:
            return self.make_initial()
        return self.u0, self.v0

    @property
    def nodes(self) -> int:
        """Nodes of the body (those of a hole removed)."""
        n = self.nx * self.ny
        if self.hole is not None:
            x0, x1, y0, y1 = self.hole
            n -= max(0, x1 - x0) * max(0, y1 - y0)
        return n

    def active(self) -> np.ndarray:
        """[ny][nx] mask of the body's nodes."""
        m = np.ones((self.ny, self.nx), dtype=bool)
        if self.hole is not None:
            x0, x1, y0, y1 = self.hole
            m[y0:y1, x0:x1] = False
        return m

    def edge_dicts(self) -> list:
        return [e.as_dict() for e in self.edges]

    def periodic(self, axis: int) -> bool:
        return self.edges[2 * axis].kind == PERIODIC


def lame_from_nu(mu: float, nu: float) -> float:
    """Plane-strain Lame lambda from shear modulus and Poisson ratio."""
    return 2.0 * mu * nu / (1.0 - 2.0 * nu)


def node_coords(n: int, dX: float, periodic: bool) -> np.ndarray:
    k = np.arange(n, dtype=np.float64)
    return (k if periodic else k + 0.5) * dX


def all_periodic() -> List[Edge]:
    return [Edge(PERIODIC) for _ in range(4)]


def clamped_free_edges() -> List[Edge]:
    """x- clamped (u* = 0, v* = 0); x+, y-, y+ traction-free."""
    return [Edge(DIRICHLET), Edge(NEUMANN), Edge(NEUMANN), Edge(NEUMANN)]


# ----------------------------------------------------------------- workloads

def shear_wave(n: int = 64, amp: float = 0.01, lam: float = 0.5, mu: float = 0.3,
               rho0: float = 1.0, omega: float = OMEGA, dX: float = 1.0) -> Problem:
    """Periodic n x n body, u_x = amp sin(2 pi y / (n dX)), v = 0."""
    y = node_coords(n, dX, True)
    u0 = np.zeros((n, n, 2))
    u0[:, :, 0] = amp * np.sin(2.0 * np.pi * y / (n * dX))[:, None]
    return Problem(nx=n, ny=n, lam=lam, mu=mu, rho0=rho0, omega=omega, dX=dX,
                   edges=all_periodic(), u0=u0, v0=np.zeros_like(u0), name=f"shear_wave_{n}")


def longitudinal_wave(n: int = 64, amp: float = 1e-6, lam: float = 0.5, mu: float = 0.3,
                      rho0: float = 1.0, omega: float = OMEGA, dX: float = 1.0) -> Problem:
    """Periodic n x n body, u_y = amp sin(2 pi y / (n dX)) (a P-wave)."""
    y = node_coords(n, dX, True)
    u0 = np.zeros((n, n, 2))
    u0[:, :, 1] = amp * np.sin(2.0 * np.pi * y / (n * dX))[:, None]
    return Problem(nx=n, ny=n, lam=lam, mu=mu, rho0=rho0, omega=omega, dX=dX,
                   edges=all_periodic(), u0=u0, v0=np.zeros_like(u0), name=f"p_wave_{n}")


def clamped_body(nx: int = 4096, ny: int = 2048, mu: float = 0.3, nu: float = 0.3,
                 vmax: float = 0.05, rho0: float = 1.0, omega: float = OMEGA_BODIES,
                 dX: float = 1.0) -> Problem:
    """Left edge clamped, other edges traction-free, v_y = vmax x / L."""
    x = node_coords(nx, dX, False)
    L = nx * dX
    v0 = np.zeros((ny, nx, 2))
    v0[:, :, 1] = (vmax * x / L)[None, :]
    return Problem(nx=nx, ny=ny, lam=lame_from_nu(mu, nu), mu=mu, rho0=rho0, omega=omega,
                   dX=dX, edges=clamped_free_edges(), u0=np.zeros_like(v0), v0=v0,
                   name=f"clamped_{nx}x{ny}")


def smooth_random(nx: int, ny: int, edges: List[Edge], seed: int, amp: float = 0.02,
                  vamp: float = 0.01, lam: float = 0.45, mu: float = 0.3, rho0: float = 1.0,
                  omega: float = OMEGA, dX: float = 1.0, modes: int = 3) -> Problem:
    """Sum of a few seeded low Fourier modes in u0 and v0 (for parity tests)."""
    rng = np.random.default_rng(seed)
    px = edges[0].kind == PERIODIC
    py = edges[2].kind == PERIODIC
    x = node_coords(nx, dX, px)
    y = node_coords(ny, dX, py)
    Lx, Ly = nx * dX, ny * dX
    X, Y = np.meshgrid(x, y)
    u0 = np.zeros((ny, nx, 2))
    v0 = np.zeros((ny, nx, 2))
    for field, a in ((u0, amp), (v0, vamp)):
        for comp in range(2):
            for _ in range(modes):
                kx = rng.integers(0, 3)
                ky = rng.integers(0, 3)
                ph = rng.uniform(0, 2 * np.pi, size=2)
                c = rng.uniform(-1, 1) * a / modes
                field[:, :, comp] += c * np.sin(2 * np.pi * kx * X / Lx + ph[0]) * np.cos(
                    2 * np.pi * ky * Y / Ly + ph[1])
    return Problem(nx=nx, ny=ny, lam=lam, mu=mu, rho0=rho0, omega=omega, dX=dX,
                   edges=edges, u0=u0, v0=v0, name=f"smooth_{nx}x{ny}_s{seed}")


def affine_patch(nx: int, ny: int, H0, edges_kind: int = NEUMANN, lam: float = 1.0,
                 mu: float = 1.0, rho0: float = 1.0, omega: float = OMEGA, dX: float = 1.0,
                 tractions=None) -> Problem:
    """u0 = H0 X (X node positions from the body centre), v0 = 0.

    tractions: four (T_x, T_y) pairs for Neumann edges (x-, x+, y-, y+)."""
    H0 = np.asarray(H0, dtype=np.float64).reshape(2, 2)
    x = node_coords(nx, dX, False) - 0.5 * nx * dX
    y = node_coords(ny, dX, False) - 0.5 * ny * dX
    X, Y = np.meshgrid(x, y)
    u0 = np.zeros((ny, nx, 2))
    u0[:, :, 0] = H0[0, 0] * X + H0[0, 1] * Y
    u0[:, :, 1] = H0[1, 0] * X + H0[1, 1] * Y
    edges = []
    for k in range(4):
        T = tuple(tractions[k]) if tractions is not None else (0.0, 0.0)
        edges.append(Edge(edges_kind, value=T, rate=T))
    return Problem(nx=nx, ny=ny, lam=lam, mu=mu, rho0=rho0, omega=omega, dX=dX,
                   edges=edges, u0=u0, v0=np.zeros_like(u0), name="affine_patch")


def uniform_motion(nx: int, ny: int, v, lam: float = 0.5, mu: float = 0.3, rho0: float = 1.0,
                   omega: float = OMEGA, dX: float = 1.0) -> Problem:
    """v0 = v everywhere, all four edges Dirichlet moving with v* = v."""
    v = tuple(float(a) for a in v)
    v0 = np.zeros((ny, nx, 2))
    v0[:, :, 0], v0[:, :, 1] = v
    edges = [Edge(DIRICHLET, value=(0.0, 0.0), rate=v) for _ in range(4)]
    return Problem(nx=nx, ny=ny, lam=lam, mu=mu, rho0=rho0, omega=omega, dX=dX,
                   edges=edges, u0=np.zeros_like(v0), v0=v0, name="uniform_motion")


def tension_block(n: int = 40, T1: float = 1.0, lam: float = 1.0, mu: float = 1.0,
                  t_ramp: float = 1.0, omega: float = OMEGA_SEC7) -> Problem:
    """Square block of side l = 1 (dX = 1/n), traction ramped on y+ (Sec. 7).

    The y- edge is clamped; x edges are traction-free."""
    dX = 1.0 / n
    edges = [Edge(NEUMANN), Edge(NEUMANN), Edge(DIRICHLET),
             Edge(NEUMANN, value=(0.0, 0.0), rate=(0.0, T1), times=(0.0, t_ramp, math.inf))]
    z = np.zeros((n, n, 2))
    return Problem(nx=n, ny=n, lam=lam, mu=mu, omega=omega, dX=dX, edges=edges, u0=z, v0=z.copy(),
                   name=f"tension_{n}")


def shear_block(n: int = 40, T1: float = 0.05, lam: float = 1.0, mu: float = 1.0,
                t_ramp: float = 1.0, omega: float = OMEGA_SEC7) -> Problem:
    """Square block of side l = 1 (dX = 1/n) under simple shear (Sec. 7): a
    tangential traction along x1 on y+, ramped from 0 to T1 over t_ramp and
    held (the paper: T1 = 0.05 mu, to t = 8).  The y- edge is clamped, the x
    edges are traction-free (the paper's figure is absent; its probe at the
    centre of the left side moves, so that side is free)."""
    dX = 1.0 / n
    edges = [Edge(NEUMANN), Edge(NEUMANN), Edge(DIRICHLET),
             Edge(NEUMANN, value=(0.0, 0.0), rate=(T1, 0.0), times=(0.0, t_ramp, math.inf))]
    z = np.zeros((n, n, 2))
    return Problem(nx=n, ny=n, lam=lam, mu=mu, omega=omega, dX=dX, edges=edges, u0=z, v0=z.copy(),
                   name=f"shear_{n}")


def plate_with_hole(n: int = 80, hole_frac: float = 0.4, T: float = 0.1, mu: float = 1.0, lam: float = 1.0,
                    t_off: float = 1.0, omega: float = OMEGA_SEC7) -> Problem:
    """Square plate of side l = 1 (dX = 1/n) with a centred square hole of
    side hole_frac l, traction-free except for a sudden traction of T along
    x2 on the top and bottom edges (outward on both) from t = 0 to t_off
    (Sec. 7's plate with a hole: n = 80, hole 0.4 l, T = 0.1 mu, off at
    t = 1)."""
    dX = 1.0 / n
    h = int(round(hole_frac * n))
    a = (n - h) // 2
    pull = dict(value=(0.0, 0.0), times=(0.0, 0.0, t_off))
    edges = [Edge(NEUMANN), Edge(NEUMANN), Edge(NEUMANN, rate=(0.0, -T), **pull),
             Edge(NEUMANN, rate=(0.0, T), **pull)]
    z = np.zeros((n, n, 2))
    return Problem(nx=n, ny=n, lam=lam, mu=mu, omega=omega, dX=dX, edges=edges, u0=z, v0=z.copy(),
                   hole=(a, a + h, a, a + h), name=f"plate_hole_{n}")


# ----------------------------------------------------------------- batches

@dataclasses.dataclass
class BatchSpec:
    problems: List[Problem]
    steps: List[int]


def random_body(rng: np.random.Generator, side_lo: int, side_hi: int, dX: float = 1.0,
                omega: float = OMEGA_BODIES, lazy: bool = False, stable_materials: bool = False) -> Problem:
    """One body: sides U{lo..hi}, mu log-U[0.05, 0.4], nu U[0.2, 0.45],
    periodic or clamped (50/50), low-mode initial displacement of amplitude
    up to 0.1 L, zero velocity.  lazy: keep the recipe of u0 / v0
    (Problem.initial builds them) instead of the arrays.  stable_materials:
    the Poisson ratio drawn from where the method is stable instead (a
    clamped body: 0.25, lambda = mu, the ratio Sec. 7 runs; a periodic one:
    U[0.2, 0.4]); the draws of everything else are the same."""
    nx = int(rng.integers(side_lo, side_hi + 1))
    ny = int(rng.integers(side_lo, side_hi + 1))
    mu = float(math.exp(rng.uniform(math.log(0.05), math.log(0.4))))
    nu = float(rng.uniform(0.2, 0.45))
    periodic = bool(rng.integers(0, 2) == 0)
    if stable_materials:
        nu = 0.2 + (nu - 0.2) * (0.2 / 0.25) if periodic else 0.25
    A_frac = float(rng.uniform(0.0, 0.1))
    theta = float(rng.uniform(0.0, 2 * np.pi))
    phase = float(rng.uniform(0.0, 2 * np.pi))
    axis = int(rng.integers(0, 2))
    edges = all_periodic() if periodic else clamped_free_edges()
    Lx, Ly = nx * dX, ny * dX

    def grid():
        return np.meshgrid(node_coords(nx, dX, periodic), node_coords(ny, dX, periodic))
    L = (Ly if axis == 0 else Lx) if periodic else Lx
    A = A_frac * L

    def build():
        X, Y = grid()
        if periodic:
            mm = np.sin(2 * np.pi * Y / Ly + phase) if axis == 0 else np.sin(2 * np.pi * X / Lx + phase)
        else:
            mm = np.sin(np.pi * X / (2 * Lx))
        u = np.zeros((ny, nx, 2))
        u[:, :, 0] = A * math.cos(theta) * mm
        u[:, :, 1] = A * math.sin(theta) * mm
        return u, np.zeros_like(u)

    name = f"body_{nx}x{ny}_{'per' if periodic else 'clamp'}"
    if lazy:
        return Problem(nx=nx, ny=ny, lam=lame_from_nu(mu, nu), mu=mu, omega=omega, dX=dX, edges=edges,
                       make_initial=build, name=name)
    u0, v0 = build()
    return Problem(nx=nx, ny=ny, lam=lame_from_nu(mu, nu), mu=mu, omega=omega, dX=dX,
                   edges=edges, u0=u0, v0=v0, name=name)


def body_batch(count: int = 256, seed: int = 20220825, side_lo: int = 64, side_hi: int = 1024,
               steps: int = 2000) -> BatchSpec:
    rng = np.random.default_rng(seed)
    probs = [random_body(rng, side_lo, side_hi) for _ in range(count)]
    return BatchSpec(problems=probs, steps=[steps] * count)


@dataclasses.dataclass
class Request:
    arrival: float
    problem: Problem
    steps: int


def serving_trace(rate: float = 200.0, duration: float = 60.0, seed: int = 7,
                  side_lo: int = 128, side_hi: int = 2048, steps_lo: int = 500,
                  steps_hi: int = 20000, max_requests: Optional[int] = None,
                  lazy_fields: bool = True, stable_materials: bool = False) -> List[Request]:
    """Poisson arrivals; each request a body as in body_batch with a
    log-uniform step count (lazy_fields: initial fields built on demand;
    stable_materials: see random_body)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out: List[Request] = []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration:
            break
        prob = random_body(rng, side_lo, side_hi, lazy=lazy_fields, stable_materials=stable_materials)
        steps = int(round(math.exp(rng.uniform(math.log(steps_lo), math.log(steps_hi)))))
        out.append(Request(arrival=t, problem=prob, steps=steps))
        if max_requests is not None and len(out) >= max_requests:
            break
    return out
