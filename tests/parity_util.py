"""Shared helpers of the parity tests (GPU library vs the FP64 oracle)."""
import numpy as np

import oracle
from paper_2208_13769_gb300 import lbm


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def run_both(prob, steps, storage="f64", compensated=None, scheme=oracle.PREDICTOR, chunks=None):
    """Advance the oracle and the GPU library by `steps` from the same inputs;
    returns (oracle fields, gpu fields)."""
    s = oracle.solver_from(prob, scheme)
    s.step(steps)
    ref = s.read()
    with lbm.Body(prob, storage=storage, compensated=compensated, scheme=scheme) as b:
        for n in (chunks or [steps]):
            b.step(n)
        got = b.read(allow_unstable=True)
    return ref, got


def moment_scale(ref, prob):
    """Natural scale of the zeroth moment r = sum_i f_i: the populations are
    of order |r| + rho0 |v| / c + |Pbar| / c^2 (c = dX / dt = sqrt(3 mu / rho0)),
    and the rounding of r is relative to them, not to |r| alone."""
    c = np.sqrt(3.0 * prob.mu / prob.rho0)
    return (np.linalg.norm(ref["r"]) + prob.rho0 * np.linalg.norm(ref["v"]) / c
            + np.linalg.norm(ref["Pbar"]) / c ** 2)


def compare(ref, got, tol, keys=("u", "v", "P"), prob=None):
    errs = {}
    for k in keys:
        if k == "r" and prob is not None:
            errs[k] = np.linalg.norm(np.asarray(got[k]) - ref[k]) / moment_scale(ref, prob)
        else:
            errs[k] = rel_l2(got[k], ref[k])
    bad = {k: e for k, e in errs.items() if not (e <= tol)}
    assert not bad, (bad, errs)
    return errs
