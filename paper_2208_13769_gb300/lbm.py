"""ctypes binding of the C ABI in include/lbm.h (liblbm_gb300.so).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  There is no CPU fallback -- if the shared library cannot be
built or loaded, importing the entry points raises.

The module exposes the C functions under their C names (lbm_create, ...),
plus :class:`Body`, a small RAII wrapper that creates a context from a
:class:`paper_2208_13769_gb300.workloads.Problem`.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional, Union

import numpy as np

from . import build as _build

LBM_OK, LBM_E_INVALID, LBM_E_OOM, LBM_E_CUDA, LBM_E_UNSTABLE, LBM_E_TIMEOUT, LBM_E_STATE = range(7)
LBM_F64, LBM_F32, LBM_F16, LBM_BF16 = range(4)
LBM_UCARRY_NATIVE, LBM_UCARRY_COMPENSATED, LBM_UCARRY_COMPENSATED16 = 0, 1, 2


def ucarry_of(compensated) -> int:
    """The lbm_ucarry value of a Body's `compensated` argument: None or True
    (FP32 pair), False (plain), "lo16" (FP32 high word + 16-bit low word)."""
    if compensated is None or compensated is True:
        return LBM_UCARRY_COMPENSATED
    if compensated is False:
        return LBM_UCARRY_NATIVE
    if compensated == "lo16":
        return LBM_UCARRY_COMPENSATED16
    raise ValueError(f"compensated: None, True, False or 'lo16', not {compensated!r}")
LBM_SCHEME_EXPLICIT, LBM_SCHEME_PREDICTOR, LBM_SCHEME_EXTRAPOLATED = 0, 1, 2
LBM_PERIODIC, LBM_DIRICHLET, LBM_NEUMANN = 0, 1, 2
LBM_FIELD_U, LBM_FIELD_V, LBM_FIELD_P, LBM_FIELD_PBAR, LBM_FIELD_R, LBM_FIELD_SIGMA, LBM_FIELD_J = (
    1, 2, 4, 8, 16, 32, 64)
FIELD_COMPS = {LBM_FIELD_U: 2, LBM_FIELD_V: 2, LBM_FIELD_P: 4, LBM_FIELD_PBAR: 3, LBM_FIELD_R: 1,
               LBM_FIELD_SIGMA: 3, LBM_FIELD_J: 1}
FIELD_NAMES = {LBM_FIELD_U: "u", LBM_FIELD_V: "v", LBM_FIELD_P: "P", LBM_FIELD_PBAR: "Pbar",
               LBM_FIELD_R: "r", LBM_FIELD_SIGMA: "sigma", LBM_FIELD_J: "J"}
STORAGE = {"f64": LBM_F64, "f32": LBM_F32, "f16": LBM_F16, "bf16": LBM_BF16}


class lbm_desc(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("dX", C.c_double),
        ("storage", C.c_int32), ("u_carry", C.c_int32), ("scheme", C.c_int32),
        ("f16_scale_log2", C.c_int32),
        ("u0", C.c_void_p), ("v0", C.c_void_p), ("cuda_stream", C.c_void_p),
        ("device", C.c_int32),
    ]


class lbm_tuning(C.Structure):
    _fields_ = [("ring_slots", C.c_int32), ("chunk_rows", C.c_int32), ("aligned", C.c_int32),
                ("plan", C.c_int32)]

    def as_dict(self) -> dict:
        return {"ring_slots": self.ring_slots, "chunk_rows": self.chunk_rows, "aligned": self.aligned,
                "plan": self.plan}


class lbm_field_geometry(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("dX", C.c_double), ("lam", C.c_double),
        ("mu", C.c_double), ("rho0", C.c_double), ("edge_kind", C.c_int32 * 4),
        ("edge_u", (C.c_double * 2) * 4),
    ]


class LbmError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


_lock = threading.Lock()
_lib = None

_SIGNATURES = {
    "lbm_create": (C.c_int, [C.POINTER(lbm_desc), C.POINTER(C.c_void_p)]),
    "lbm_set_material": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double,
                                   C.POINTER(C.c_double)]),
    "lbm_set_boundary": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_double),
                                   C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "lbm_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "lbm_set_hole": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "lbm_profile_steps": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_double)]),
    "lbm_profile_interior": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_double)]),
    "lbm_fields_size": (C.c_int64, [C.c_void_p, C.c_uint32]),
    "lbm_read_fields": (C.c_int, [C.c_void_p, C.c_uint32, C.POINTER(C.c_double), C.c_int64,
                                  C.POINTER(C.c_double)]),
    "lbm_diagnostics": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "lbm_sync": (C.c_int, [C.c_void_p]),
    "lbm_get_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "lbm_memory_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "lbm_state_size": (C.c_int64, [C.c_void_p]),
    "lbm_read_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "lbm_write_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "lbm_destroy": (C.c_int, [C.c_void_p]),
    "lbm_status_string": (C.c_char_p, [C.c_int]),
    "lbm_last_cuda_error": (C.c_char_p, [C.c_void_p]),
    "lbm_diagnostics_noalloc": (C.c_int, [C.POINTER(lbm_field_geometry), C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_void_p, C.POINTER(C.c_void_p)]),
    "lbm_batch_create_tuned": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_void_p, C.POINTER(lbm_tuning),
                                         C.POINTER(C.c_void_p)]),
    "lbm_batch_autotune": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_int64, C.POINTER(lbm_tuning),
                                     C.POINTER(C.c_double)]),
    "lbm_batch_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "lbm_batch_sync": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "lbm_batch_get_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                     C.POINTER(C.c_int32)]),
    "lbm_batch_destroy": (C.c_int, [C.c_void_p]),
    "lbm_selftest_bounded_wait": (C.c_int, [C.c_uint32, C.c_void_p, C.POINTER(C.c_int32)]),
    "lbm_set_tuning": (C.c_int, [C.c_void_p, C.POINTER(lbm_tuning)]),
    "lbm_get_tuning": (C.c_int, [C.c_void_p, C.POINTER(lbm_tuning)]),
    "lbm_autotune": (C.c_int, [C.POINTER(lbm_desc), C.POINTER(C.c_int32), C.c_int64, C.POINTER(lbm_tuning),
                               C.POINTER(C.c_double)]),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """Loads liblbm_gb300.so, building it first when the sources are newer."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library missing: {path}")
            L = C.CDLL(path)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().lbm_status_string(int(status)).decode()


def _check(status: int, what: str, allow=()):
    if status != LBM_OK and status not in allow:
        raise LbmError(status, what)
    return status


def _dbl(a) -> Optional[C.Array]:
    if a is None:
        return None
    return (C.c_double * len(a))(*[float(x) for x in a])


# ------------------------------------------------------------- C names

def lbm_create(desc: lbm_desc) -> C.c_void_p:
    h = C.c_void_p()
    _check(lib().lbm_create(C.byref(desc), C.byref(h)), "lbm_create")
    return h


def lbm_set_material(ctx, lam, mu, rho0, omega, body_force=None):
    return _check(lib().lbm_set_material(ctx, lam, mu, rho0, omega, _dbl(body_force)), "lbm_set_material")


def lbm_set_boundary(ctx, edge, kind, value=None, rate=None, times=None):
    return _check(lib().lbm_set_boundary(ctx, int(edge), int(kind), _dbl(value), _dbl(rate), _dbl(times)),
                  "lbm_set_boundary")


def lbm_step(ctx, nsteps: int):
    st = lib().lbm_step(ctx, int(nsteps))
    if st == LBM_E_CUDA:
        raise LbmError(st, f"lbm_step ({lbm_last_cuda_error(ctx)})")
    return _check(st, "lbm_step")


def lbm_profile_steps(ctx, nsteps: int, allow_unstable: bool = False) -> tuple:
    """Advances nsteps steps launch by launch; returns (status, [interior ms,
    band ms, step ms, interior nodes]), the times averaged over the steps."""
    out = np.zeros(4)
    st = lib().lbm_profile_steps(ctx, int(nsteps), out.ctypes.data_as(C.POINTER(C.c_double)))
    _check(st, "lbm_profile_steps", allow=(LBM_E_UNSTABLE,) if allow_unstable else ())
    return st, out


def lbm_profile_interior(ctx, nlaunches: int, allow_unstable: bool = False) -> tuple:
    """Times nlaunches back-to-back interior launches (the state is saved
    and restored around them); returns (status, [ms per launch, nodes])."""
    out = np.zeros(2)
    st = lib().lbm_profile_interior(ctx, int(nlaunches), out.ctypes.data_as(C.POINTER(C.c_double)))
    _check(st, "lbm_profile_interior", allow=(LBM_E_UNSTABLE,) if allow_unstable else ())
    return st, out


def lbm_fields_size(ctx, mask: int) -> int:
    return int(lib().lbm_fields_size(ctx, int(mask)))


def lbm_read_fields(ctx, mask: int, out: np.ndarray, allow_unstable: bool = False) -> tuple:
    """Fills the float64 host buffer ``out``; returns (status, t)."""
    assert out.dtype == np.float64 and out.flags.c_contiguous
    t = C.c_double()
    st = lib().lbm_read_fields(ctx, int(mask), out.ctypes.data_as(C.POINTER(C.c_double)), out.size,
                               C.byref(t))
    _check(st, "lbm_read_fields", allow=(LBM_E_UNSTABLE,) if allow_unstable else ())
    return st, t.value


def lbm_state_size(ctx) -> int:
    return int(lib().lbm_state_size(ctx))


def lbm_read_state(ctx, allow_unstable: bool = False) -> np.ndarray:
    """The context's state (a uint8 host array in the library's layout)."""
    out = np.empty(lbm_state_size(ctx), dtype=np.uint8)
    st = lib().lbm_read_state(ctx, out.ctypes.data_as(C.c_void_p), out.size)
    _check(st, "lbm_read_state", allow=(LBM_E_UNSTABLE,) if allow_unstable else ())
    return out


def lbm_write_state(ctx, state: np.ndarray) -> None:
    """Replaces the context's state by one lbm_read_state returned."""
    buf = np.ascontiguousarray(state, dtype=np.uint8)
    _check(lib().lbm_write_state(ctx, buf.ctypes.data_as(C.c_void_p), buf.size), "lbm_write_state")


def lbm_diagnostics(ctx, allow_unstable: bool = False) -> tuple:
    out = np.zeros(6)
    st = lib().lbm_diagnostics(ctx, out.ctypes.data_as(C.POINTER(C.c_double)))
    _check(st, "lbm_diagnostics", allow=(LBM_E_UNSTABLE,) if allow_unstable else ())
    return st, out


def lbm_sync(ctx, allow_unstable: bool = False) -> int:
    return _check(lib().lbm_sync(ctx), "lbm_sync", allow=(LBM_E_UNSTABLE,) if allow_unstable else ())


def lbm_get_info(ctx) -> tuple:
    s, d = C.c_int64(), C.c_double()
    _check(lib().lbm_get_info(ctx, C.byref(s), C.byref(d)), "lbm_get_info")
    return s.value, d.value


def lbm_memory_info(ctx) -> tuple:
    a, b = C.c_int64(), C.c_int64()
    _check(lib().lbm_memory_info(ctx, C.byref(a), C.byref(b)), "lbm_memory_info")
    return a.value, b.value


def lbm_destroy(ctx):
    return _check(lib().lbm_destroy(ctx), "lbm_destroy")


def lbm_diagnostics_noalloc(geo: lbm_field_geometry, fields_dev: int, out_dev: int, stream: int = 0) -> int:
    """Diagnostics of caller-owned device fields (device pointers as ints);
    allocates nothing.  Returns the status."""
    return int(lib().lbm_diagnostics_noalloc(C.byref(geo), C.c_void_p(fields_dev), C.c_void_p(out_dev),
                                             C.c_void_p(stream or None)))


def _ctx_array(ctxs):
    return (C.c_void_p * len(ctxs))(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])


def lbm_batch_create(ctxs, stream: int = 0, tuning: Optional["lbm_tuning"] = None) -> C.c_void_p:
    arr = _ctx_array(ctxs)
    h = C.c_void_p()
    if tuning is None:
        st = lib().lbm_batch_create(arr, len(ctxs), C.c_void_p(stream or None), C.byref(h))
    else:
        st = lib().lbm_batch_create_tuned(arr, len(ctxs), C.c_void_p(stream or None), C.byref(tuning), C.byref(h))
    _check(st, "lbm_batch_create")
    return h


def lbm_batch_autotune(ctxs, steps: int = 128) -> tuple:
    """(best lbm_tuning, its ms per step) for a batch of contexts shaped like
    ctxs, timed on scratch copies (ctxs are not touched)."""
    t, ms = lbm_tuning(), C.c_double()
    _check(lib().lbm_batch_autotune(_ctx_array(ctxs), len(ctxs), int(steps), C.byref(t), C.byref(ms)),
           "lbm_batch_autotune")
    return t, ms.value


def lbm_batch_step(batch, nsteps: int):
    return _check(lib().lbm_batch_step(batch, int(nsteps)), "lbm_batch_step")


def lbm_batch_sync(batch, n: int) -> tuple:
    """Returns (first non-OK status or OK, per-member statuses)."""
    st = (C.c_int32 * n)()
    worst = lib().lbm_batch_sync(batch, st)
    if worst == LBM_E_CUDA:
        raise LbmError(worst, "lbm_batch_sync")
    return worst, [int(x) for x in st]


def lbm_batch_get_info(batch) -> tuple:
    s, a, b = C.c_int64(), C.c_int32(), C.c_int32()
    _check(lib().lbm_batch_get_info(batch, C.byref(s), C.byref(a), C.byref(b)), "lbm_batch_get_info")
    return s.value, a.value, b.value


def lbm_batch_destroy(batch):
    return _check(lib().lbm_batch_destroy(batch), "lbm_batch_destroy")


def lbm_selftest_bounded_wait(polls: int, stream: int = 0) -> int:
    """1 if the device-side bounded wait on a never-completing barrier gave
    up after `polls` polls (the expected outcome)."""
    out = C.c_int32(-1)
    _check(lib().lbm_selftest_bounded_wait(int(polls), C.c_void_p(stream or None), C.byref(out)),
           "lbm_selftest_bounded_wait")
    return int(out.value)


def lbm_set_hole(ctx, hole, traction=None):
    """A rectangular hole (x0, x1, y0, y1) of removed nodes; traction: four
    (Tx, Ty) pairs for its faces at x0, x1, y0, y1 (None: traction-free)."""
    h = (C.c_int32 * 4)(*[int(v) for v in hole])
    t = None
    if traction is not None:
        t = (C.c_double * 8)(*[float(v) for pair in traction for v in pair])
    _check(lib().lbm_set_hole(ctx, h, t), "lbm_set_hole")


def lbm_set_tuning(ctx, tuning: "lbm_tuning"):
    return _check(lib().lbm_set_tuning(ctx, C.byref(tuning)), "lbm_set_tuning")


def lbm_get_tuning(ctx) -> "lbm_tuning":
    t = lbm_tuning()
    _check(lib().lbm_get_tuning(ctx, C.byref(t)), "lbm_get_tuning")
    return t


def lbm_autotune(desc: lbm_desc, edge_kinds, steps: int = 129) -> tuple:
    """(best lbm_tuning, its ms per step) for bodies shaped like desc."""
    kinds = (C.c_int32 * 4)(*[int(k) for k in edge_kinds])
    t, ms = lbm_tuning(), C.c_double()
    _check(lib().lbm_autotune(C.byref(desc), kinds, int(steps), C.byref(t), C.byref(ms)), "lbm_autotune")
    return t, ms.value


def tuning_from_dict(d: dict) -> lbm_tuning:
    return lbm_tuning(int(d["ring_slots"]), int(d["chunk_rows"]), int(d["aligned"]), int(d.get("plan", 0)))


def autotune_cached(prob, storage: str = "f32", compensated: Optional[Union[bool, str]] = None,
                    scheme: int = LBM_SCHEME_EXPLICIT, cache_path: Optional[str] = None, steps: int = 129,
                    stream: int = 0, device: int = 0) -> lbm_tuning:
    """The autotuner's choice for bodies of prob's size and edge kinds, from a
    JSON cache (keyed by storage, carry, scheme, size and edge kinds) when it
    holds one, else measured now and stored."""
    import json

    uc = ucarry_of(compensated)
    kinds = [e.kind for e in prob.edges]
    key = f"{storage}:{uc}:{scheme}:{prob.nx}x{prob.ny}:{''.join(str(k) for k in kinds)}:p"
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as fh:
            cache = json.load(fh)
    if key in cache:
        return tuning_from_dict(cache[key])
    d = lbm_desc()
    d.nx, d.ny, d.dX = prob.nx, prob.ny, prob.dX
    d.storage = STORAGE[storage]
    d.u_carry = uc
    d.scheme = scheme
    d.cuda_stream = stream or None
    d.device = device
    t, ms = lbm_autotune(d, kinds, steps)
    if cache_path:
        cache[key] = dict(t.as_dict(), ms_per_step=ms)
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return t


def lbm_last_cuda_error(ctx) -> str:
    return lib().lbm_last_cuda_error(ctx).decode()


def lbm_status_string(status: int) -> str:
    return status_string(status)


# ------------------------------------------------------------- convenience

class Body:
    """One solver context for a workloads.Problem-like object.

    storage: "f64" | "f32" | "f16" | "bf16"; compensated: FP32-pair u-carry
    for "f32" (default True: a plain FP32 u loses Grad u to rounding once
    |u| >> |H| dX; "lo16": the pair with its low word in 16 bits, 12 instead
    of 16 bytes per node, about 35 significant bits); scheme: LBM_SCHEME_EXPLICIT (default: Algorithm 1, the
    time-t source in collision and moment), LBM_SCHEME_PREDICTOR (the
    footnote's predictor-corrector, which Sec. 7's tension run needs) or
    LBM_SCHEME_EXTRAPOLATED (stable only for lambda = mu);
    stream: an integer cudaStream_t handle (e.g. torch's stream.cuda_stream)."""

    def __init__(self, prob, storage: str = "f64", compensated: Optional[Union[bool, str]] = None,
                 scheme: int = LBM_SCHEME_EXPLICIT, stream: int = 0, device: int = 0,
                 f16_scale_log2: int = 0, tuning: Optional["lbm_tuning"] = None):
        self.prob = prob
        d = lbm_desc()
        d.nx, d.ny, d.dX = prob.nx, prob.ny, prob.dX
        d.storage = STORAGE[storage]
        d.u_carry = ucarry_of(compensated)
        d.scheme = scheme
        d.f16_scale_log2 = f16_scale_log2
        u0, v0 = prob.initial() if hasattr(prob, "initial") else (prob.u0, prob.v0)
        self._u0 = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64)
        self._v0 = None if v0 is None else np.ascontiguousarray(v0, dtype=np.float64)
        d.u0 = None if self._u0 is None else self._u0.ctypes.data
        d.v0 = None if self._v0 is None else self._v0.ctypes.data
        d.cuda_stream = stream or None
        d.device = device
        self.ctx = lbm_create(d)
        self._u0 = self._v0 = None  # copied to the device by lbm_create
        if tuning is not None:
            lbm_set_tuning(self.ctx, tuning)
        lbm_set_material(self.ctx, prob.lam, prob.mu, prob.rho0, prob.omega, prob.body)
        for k, e in enumerate(prob.edges):
            lbm_set_boundary(self.ctx, k, e.kind, e.value, e.rate, e.times)
        if getattr(prob, "hole", None) is not None:
            lbm_set_hole(self.ctx, prob.hole, prob.hole_traction)

    def step(self, n: int) -> None:
        lbm_step(self.ctx, n)

    def read(self, mask: int = 127, allow_unstable: bool = False) -> dict:
        n = lbm_fields_size(self.ctx, mask)
        buf = np.empty(n, dtype=np.float64)
        st, t = lbm_read_fields(self.ctx, mask, buf, allow_unstable=allow_unstable)
        out, off = {"t": t, "status": st}, 0
        ny, nx = self.prob.ny, self.prob.nx
        for bit in (1, 2, 4, 8, 16, 32, 64):
            if mask & bit:
                k = FIELD_COMPS[bit]
                blk = buf[off:off + k * nx * ny].reshape(ny, nx, k)
                out[FIELD_NAMES[bit]] = blk[:, :, 0] if k == 1 else blk
                off += k * nx * ny
        return out

    def diagnostics(self, allow_unstable: bool = False):
        return lbm_diagnostics(self.ctx, allow_unstable)[1]

    def save_state(self, allow_unstable: bool = False) -> np.ndarray:
        """Checkpoint: the body's state after its last step (host bytes)."""
        return lbm_read_state(self.ctx, allow_unstable)

    def load_state(self, state: np.ndarray) -> None:
        """Resume from a checkpoint of a body of the same size, format,
        scheme and material."""
        lbm_write_state(self.ctx, state)

    def info(self):
        return lbm_get_info(self.ctx)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            lbm_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several Body objects (one storage format) advanced by shared launches;
    each member's results are bit-identical to stepping it alone with the
    interior kernel (plan 2; to rounding for a small member whose own default
    plan is edge tiles only)."""

    def __init__(self, bodies, stream: int = 0, tuning: Optional["lbm_tuning"] = None):
        self.bodies = list(bodies)
        self.handle = lbm_batch_create([b.ctx for b in self.bodies], stream, tuning)

    def step(self, n: int) -> None:
        lbm_batch_step(self.handle, n)

    def sync(self) -> list:
        return lbm_batch_sync(self.handle, len(self.bodies))[1]

    def info(self) -> dict:
        s, a, b = lbm_batch_get_info(self.handle)
        return {"steps": s, "interior_ctas": a, "edge_ctas": b}

    def close(self):
        if getattr(self, "handle", None) is not None:
            lbm_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
