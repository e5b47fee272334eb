"""FP64 CPU oracle of the Lagrangian large-deformation LBM (arXiv 2208.13769).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library: ``lbm_oracle.c`` is a plain restatement of
Algorithm 1 (Sec. 5) with the boundary rules of Sec. 6 and the neo-Hooke
material of Sec. 7; this module only compiles it with gcc and marshals
arguments through ctypes.

Parity status per function (pins live in ``tests/test_oracle_pins.py``):
  feq, psi            -- pinned (moment identities of Sec. 5).
  piola, strain_energy -- pinned (finite-difference dW/dF, objectivity, simple
                          shear closed form, linearisation).
  Solver              -- pinned by conservation, exact shear-wave solution and
                          second-order convergence, longitudinal-wave frequency,
                          patch tests (Neumann, rigid rotation, Dirichlet), the
                          printed time steps of Sec. 7; the extrapolated
                          scheme by the order of its one-step miss of the
                          implicit moment.  Large-strain clamped
                          bodies have no closed form: beyond those pins their
                          parity is unpinned.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

PERIODIC, DIRICHLET, NEUMANN = 0, 1, 2
EXPLICIT, PREDICTOR, EXTRAPOLATED = 0, 1, 2


class OracleProblem(C.Structure):
    _fields_ = [
        ("nx", C.c_int32),
        ("ny", C.c_int32),
        ("dX", C.c_double),
        ("lam", C.c_double),
        ("mu", C.c_double),
        ("rho0", C.c_double),
        ("omega", C.c_double),
        ("body", C.c_double * 2),
        ("kind", C.c_int32 * 4),
        ("value", (C.c_double * 2) * 4),
        ("rate", (C.c_double * 2) * 4),
        ("times", (C.c_double * 3) * 4),
        ("scheme", C.c_int32),
        ("hole", C.c_int32 * 4),
        ("hole_T", (C.c_double * 2) * 4),
        ("alt_feq_pbar", C.c_int32),
        ("alt_wall", C.c_int32),
        ("alt_ghost_u", C.c_int32),
        ("alt_ghost_q", C.c_int32),
        ("mu_bar", C.c_double),
    ]


# Alternative readings of the paper's open points (all zero: the readings the
# oracle's header lists).  Keys of the `readings` dict of make_problem:
#   feq_pbar -- 1: f^eq takes Pbar(H) of Eq. (Plin), as Algorithm 1's listing
#   wall     -- 1: anti-bounce-back wall values extrapolated linearly to the wall
#   ghost_u  -- 1: the Neumann ghost of u quadratic instead of linear
#   ghost_q  -- 1: the ghost of Q = P + Pbar quadratic instead of linear; 2: constant
#   mu_bar   -- split stiffness: Pbar and C_s built with mu_bar (0: mu)
READING_KEYS = ("feq_pbar", "wall", "ghost_u", "ghost_q", "mu_bar")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def load(path: str):
    """A compiled oracle library at `path`, with its functions' signatures
    (lib() loads the package's own build; the tests also load copies with
    planted mistakes, to check that the pins catch them)."""
    L = C.CDLL(path)
    dp = C.POINTER(C.c_double)
    L.orc_create.restype = C.c_void_p
    L.orc_create.argtypes = [C.POINTER(OracleProblem), dp, dp]
    L.orc_check.restype = C.c_int
    L.orc_check.argtypes = [C.POINTER(OracleProblem)]
    L.orc_step.restype = C.c_int
    L.orc_step.argtypes = [C.c_void_p, C.c_long]
    L.orc_destroy.argtypes = [C.c_void_p]
    L.orc_read.argtypes = [C.c_void_p] + [dp] * 7
    L.orc_read_populations.argtypes = [C.c_void_p, dp]
    L.orc_read_grad.argtypes = [C.c_void_p, dp]
    L.orc_time.restype = C.c_double
    L.orc_time.argtypes = [C.c_void_p]
    L.orc_dt.restype = C.c_double
    L.orc_dt.argtypes = [C.c_void_p]
    L.orc_step_count.restype = C.c_long
    L.orc_step_count.argtypes = [C.c_void_p]
    L.orc_time_step.argtypes = [C.c_double] * 3 + [dp] * 3
    L.orc_feq.argtypes = [C.c_double, C.c_double, C.c_double, dp, dp, dp]
    L.orc_psi.argtypes = [C.c_double, C.c_double, dp, dp]
    L.orc_lattice.argtypes = [C.c_double, dp, dp, C.POINTER(C.c_int32)]
    L.orc_piola.restype = C.c_double
    L.orc_piola.argtypes = [dp, C.c_double, C.c_double, dp]
    L.orc_strain_energy.restype = C.c_double
    L.orc_strain_energy.argtypes = [dp, C.c_double, C.c_double]
    L.orc_poisson_stress.argtypes = [dp, C.c_double, dp]
    L.orc_threads.restype = C.c_int
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load(build())
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def problem_from(wp, scheme: int = PREDICTOR, readings=None) -> OracleProblem:
    """OracleProblem from a workloads.Problem-like object."""
    return make_problem(wp.nx, wp.ny, wp.dX, wp.lam, wp.mu, wp.rho0, wp.omega, wp.body,
                        wp.edge_dicts(), scheme, hole=getattr(wp, "hole", None),
                        hole_traction=getattr(wp, "hole_traction", None), readings=readings)


def solver_from(wp, scheme: int = PREDICTOR, readings=None) -> "Solver":
    u0, v0 = wp.initial() if hasattr(wp, "initial") else (wp.u0, wp.v0)
    return Solver(problem_from(wp, scheme, readings), u0, v0)


def _f64(x, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


# ---------------------------------------------------------------- unit pieces

def time_step(dX: float, mu: float, rho0: float):
    """(dt, c, Cs^2) under the reading dt = dX / (sqrt(3) C_s) (Sec. 7)."""
    dt, c, cs2 = C.c_double(), C.c_double(), C.c_double()
    lib().orc_time_step(dX, mu, rho0, C.byref(dt), C.byref(c), C.byref(cs2))
    return dt.value, c.value, cs2.value


def lattice(c: float):
    Cv = np.zeros(18)
    w = np.zeros(9)
    opp = np.zeros(9, dtype=np.int32)
    lib().orc_lattice(c, _dp(Cv), _dp(w), opp.ctypes.data_as(C.POINTER(C.c_int32)))
    return Cv.reshape(9, 2), w, opp


def feq(c: float, cs2: float, r: float, j, pbar) -> np.ndarray:
    """Equilibrium of Sec. 5; pbar is a full 2x2 tensor."""
    out = np.zeros(9)
    jj = _f64(j, (2,))
    pb = _f64(pbar, (4,))
    lib().orc_feq(c, cs2, r, _dp(jj), _dp(pb), _dp(out))
    return out


def psi(c: float, cs2: float, S) -> np.ndarray:
    out = np.zeros(9)
    s = _f64(S, (2,))
    lib().orc_psi(c, cs2, _dp(s), _dp(out))
    return out


def piola(H, lam: float, mu: float):
    """(P, J) for the plane-strain neo-Hooke energy of Sec. 7."""
    h = _f64(H, (4,))
    P = np.zeros(4)
    J = lib().orc_piola(_dp(h), lam, mu, _dp(P))
    return P.reshape(2, 2), J


def strain_energy(H, lam: float, mu: float) -> float:
    h = _f64(H, (4,))
    return lib().orc_strain_energy(_dp(h), lam, mu)


def poisson_stress(H, mu: float) -> np.ndarray:
    h = _f64(H, (4,))
    out = np.zeros(4)
    lib().orc_poisson_stress(_dp(h), mu, _dp(out))
    return out.reshape(2, 2)


def threads() -> int:
    return lib().orc_threads()


# ---------------------------------------------------------------- solver

def make_problem(nx, ny, dX, lam, mu, rho0, omega, body, edges,
                 scheme: int = PREDICTOR, hole=None, hole_traction=None, readings=None) -> OracleProblem:
    """edges: four dicts {kind, value, rate, times} in order x-, x+, y-, y+.

    scheme: EXPLICIT (Algorithm 1's time-t source in collision and moment),
    PREDICTOR (the footnote's predictor-corrector for u) or EXTRAPOLATED
    (Sec. 5's linear extrapolation of j to t + dt for the moment's source).
    hole: (x0, x1, y0, y1), the removed nodes of a rectangular hole, or None;
    hole_traction: the constant traction on its faces at x0, x1, y0, y1 (four
    pairs; None: traction-free).  readings: alternative readings (a dict
    with keys from READING_KEYS; None: the oracle's readings)."""
    p = OracleProblem()
    p.scheme = int(scheme)
    p.nx, p.ny = int(nx), int(ny)
    p.dX, p.lam, p.mu, p.rho0, p.omega = float(dX), float(lam), float(mu), float(rho0), float(omega)
    p.body[0], p.body[1] = float(body[0]), float(body[1])
    for k, e in enumerate(edges):
        p.kind[k] = int(e["kind"])
        val = e.get("value", (0.0, 0.0))
        rate = e.get("rate", (0.0, 0.0))
        times = e.get("times", (0.0, 0.0, float("inf")))
        for a in range(2):
            p.value[k][a] = float(val[a])
            p.rate[k][a] = float(rate[a])
        for a in range(3):
            p.times[k][a] = float(times[a])
    if hole is not None:
        for k in range(4):
            p.hole[k] = int(hole[k])
        for k, tr in enumerate(hole_traction or [(0.0, 0.0)] * 4):
            p.hole_T[k][0], p.hole_T[k][1] = float(tr[0]), float(tr[1])
    for key, val in (readings or {}).items():
        if key not in READING_KEYS:
            raise ValueError(f"unknown reading {key!r}")
        if key == "mu_bar":
            p.mu_bar = float(val)
        else:
            setattr(p, "alt_" + key, int(val))
    return p


class Solver:
    """The oracle state for one body; mirrors the library's create/step/read."""

    def __init__(self, problem: OracleProblem, u0=None, v0=None, library=None):
        self.p = problem
        ny, nx = problem.ny, problem.nx
        self._L = L = library if library is not None else lib()
        code = L.orc_check(C.byref(problem))
        if code != 0:
            raise ValueError(f"invalid oracle problem (code {code})")
        u = _f64(u0, (ny, nx, 2)) if u0 is not None else None
        v = _f64(v0, (ny, nx, 2)) if v0 is not None else None
        self._keep = (u, v)
        h = L.orc_create(C.byref(problem), _dp(u) if u is not None else None,
                         _dp(v) if v is not None else None)
        if not h:
            raise ValueError("oracle create failed")
        self._h = C.c_void_p(h)

    def step(self, n: int) -> None:
        self._L.orc_step(self._h, int(n))

    @property
    def t(self) -> float:
        return self._L.orc_time(self._h)

    @property
    def dt(self) -> float:
        return self._L.orc_dt(self._h)

    @property
    def steps(self) -> int:
        return self._L.orc_step_count(self._h)

    def read(self) -> dict:
        ny, nx = self.p.ny, self.p.nx
        out = {
            "u": np.zeros((ny, nx, 2)), "v": np.zeros((ny, nx, 2)),
            "P": np.zeros((ny, nx, 4)), "Pbar": np.zeros((ny, nx, 3)),
            "r": np.zeros((ny, nx)), "J": np.zeros((ny, nx)),
            "sigma": np.zeros((ny, nx, 3)),
        }
        self._L.orc_read(self._h, _dp(out["u"]), _dp(out["v"]), _dp(out["P"]),
                       _dp(out["Pbar"]), _dp(out["r"]), _dp(out["J"]), _dp(out["sigma"]))
        return out

    def grad(self) -> np.ndarray:
        """H = Grad u at the current time, [ny][nx][2][2]."""
        out = np.zeros((self.p.ny, self.p.nx, 2, 2))
        self._L.orc_read_grad(self._h, _dp(out))
        return out

    def populations(self) -> np.ndarray:
        out = np.zeros((9, self.p.ny, self.p.nx))
        self._L.orc_read_populations(self._h, _dp(out))
        return out

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            self._L.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
