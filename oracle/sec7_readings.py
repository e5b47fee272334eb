"""The runs of Sec. 7 under each reading of the paper's open points.

TEST INFRASTRUCTURE ONLY (it runs the FP64 oracle of this package and
nothing else).  The paper prints three runs that complete at its loads: the
tension block (T* ramped to mu by t = 1, to t = 3), the shear block (T*
ramped to 0.05 mu, to t = 8) and the plate with a square hole (a sudden
0.1 mu until t = 1, to t = 3, lengthened by about 18 %).  This script runs
each of them under every combination of

  omega = dt / tau                          (R3: the paper never fixes tau)
  the time level of 1S in the moment        (R14: Algorithm 1 / predictor / R17)
  the ghost extrapolation at traction edges (R6: linear or quadratic, for u and Q)
  the wall values of anti-bounce-back       (R7: edge node or linear to the wall)
  the Pbar of f^eq                          (R4: kinetic or Pbar(H) literally)

and prints, per combination, the time each run blows up ("ok": it reached
its end) and the plate's peak centre-line elongation (the paper's probe Q2).

    python -m oracle.sec7_readings [--procs N] [--quick]
"""
from __future__ import annotations

import argparse
import itertools
import multiprocessing as mp
import os

import numpy as np

RUNS = ("tension", "shear", "plate")


def _problem(name):
    from paper_2208_13769_gb300 import workloads as W

    if name == "tension":
        return W.tension_block(), 3.0
    if name == "shear":
        return W.shear_block(), 8.0
    return W.plate_with_hole(), 3.0


def run_one(args):
    """(name, omega, scheme, readings) -> (blow-up time or None, peak
    elongation of the centre line along x2)."""
    name, omega, scheme, readings = args
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import oracle

    prob, t_end = _problem(name)
    prob.omega = omega
    s = oracle.solver_from(prob, scheme, readings)
    n = int(round(t_end / s.dt))
    act = prob.active()
    c = prob.nx // 2
    peak, k = 0.0, 0
    while k < n:
        m = min(4, n - k)
        s.step(m)
        k += m
        o = s.read()
        u = o["u"]
        if not np.all(np.isfinite(u)) or np.abs(u).max() > 5.0 or np.where(act, o["J"], 1.0).min() <= 0.0:
            return s.t, peak
        peak = max(peak, float(u[-1, c, 1] - u[0, c, 1]))
    return None, peak


def combinations(quick: bool):
    omegas = (1.0, 1.5, 1.8, 1.95) if quick else (1.0, 1.5, 1.8, 1.9, 1.92, 1.95, 1.99)
    for omega, scheme in itertools.product(omegas, (0, 1, 2)):
        for gu, gq, wall in itertools.product((0, 1), (0, 1), (0, 1)):
            yield omega, scheme, dict(ghost_u=gu, ghost_q=gq, wall=wall)
    for omega, scheme in itertools.product((1.0, 1.95), (0, 1)):
        yield omega, scheme, dict(feq_pbar=1)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--quick", action="store_true", help="fewer values of omega")
    a = ap.parse_args(argv)
    combos = list(combinations(a.quick))
    jobs = [(name, om, sch, rd) for om, sch, rd in combos for name in RUNS]
    with mp.get_context("spawn").Pool(a.procs) as pool:
        res = pool.map(run_one, jobs, chunksize=2)
    by = {(n, om, sch, tuple(sorted(rd.items()))): r for (n, om, sch, rd), r in zip(jobs, res)}
    scheme_name = {0: "explicit", 1: "predictor", 2: "extrapolated"}

    def rd_name(rd):
        if rd.get("feq_pbar"):
            return "Pbar(H) in f^eq"
        g = "u " + ("quad" if rd["ghost_u"] else "lin") + ", Q " + ("quad" if rd["ghost_q"] else "lin")
        return g + (", wall linear" if rd["wall"] else "")

    print("| omega | scheme | readings | tension | shear | plate | plate peak elongation |")
    print("|---|---|---|---|---|---|---|")
    for om, sch, rd in combos:
        cells = []
        for name in RUNS:
            blow, _ = by[(name, om, sch, tuple(sorted(rd.items())))]
            cells.append("ok" if blow is None else f"{blow:.2f}")
        peak = by[("plate", om, sch, tuple(sorted(rd.items())))][1]
        print(f"| {om} | {scheme_name[sch]} | {rd_name(rd)} | " + " | ".join(cells) + f" | {peak:.3f} |")


if __name__ == "__main__":
    main()
