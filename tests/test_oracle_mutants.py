"""The oracle's pins must catch plausible mistakes: each case below plants
one mistake in a copy of the oracle's C source (on the CPU), compiles it,
and checks that the independent link-by-link restatement of
tests/brute_force.py then disagrees with it on at least one tiny body.  The
unmodified source agrees (test_oracle_pins)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from test_oracle_pins import _tiny_cases

SRC = os.path.join(os.path.dirname(oracle.__file__), "lbm_oracle.c")

# (what the mistake is, text of the source, replacement, occurrence to change)
MUTANTS = [
    ("bounce-back sign", "return fc - 2.0 / s->Cs2 * s->w[i] * cj;", "return fc + 2.0 / s->Cs2 * s->w[i] * cj;", 0),
    ("Dirichlet ghost value", "return 2.0 * ub[a] - v0;", "return ub[a];", 0),
    ("Neumann ghost of u", "return ghost_extrap(s->p.alt_ghost_u, v0, v1, v2);",
     "return 3.0 * v0 - 3.0 * v1 + v2;", 0),
    ("ghost of Q", "return ghost_extrap(s->p.alt_ghost_q, v0, v1, v2);", "return v0;", 0),
    ("forcing prefactor", "dt * (1.0 - 0.5 * omega) * ps[i]", "dt * ps[i]", 0),
    ("tangential wall entry from Pbar(H)", "Ptt += tv[a] * Pfw[2 * a + b] * tv[b];",
     "Ptt += tv[a] * Pbw[2 * a + b] * tv[b];", 0),
    ("corner traction not divided", "T[0] /= nlen;", "T[0] /= 1.0;", 0),
    ("half source dropped in the moment", "double jn = s->m[a][id] + 0.5 * dt * s->S[a][id];",
     "double jn = s->m[a][id];", 0),
    ("trapezoid without dt", "s->u[a][id] = s->u[a][id] + dt / (2.0 * p->rho0) * (jn + s->j[a][id]);",
     "s->u[a][id] = s->u[a][id] + 1.0 / (2.0 * p->rho0) * (jn + s->j[a][id]);", 0),
    ("F^-1 instead of F^-T", "double FiT[4] = {F[3] / J, -F[2] / J, -F[1] / J, F[0] / J};",
     "double FiT[4] = {F[3] / J, -F[1] / J, -F[2] / J, F[0] / J};", 0),
    ("diagonal weight", "1.0 / 9.0 : 1.0 / 36.0", "1.0 / 9.0 : 1.0 / 32.0", 0),
    ("initial r sign", "s->r[id] = -p->rho0 * (H[0] + H[3]);", "s->r[id] = p->rho0 * (H[0] + H[3]);", 0),
    # the hole of reading R16
    ("hole ghost", "return ghost_extrap(s->p.alt_ghost_u, U[a][IDX(s, x, y)]", "return ghost_extrap(1, U[a][IDX(s, x, y)]",
     0),
    ("hole corner normal", "if (!cx && !cy) cx = cy = 1;", "if (!cx && !cy) cx = 1;", 0),
    ("hole face traction", "s->p.hole_T[ex > 0 ? 0 : 1]", "s->p.hole_T[ex > 0 ? 1 : 0]", 0),
    # the extrapolated scheme of reading R17
    ("extrapolation held constant", "double je = 2.0 * s->j[a][id] - s->jp[a][id];",
     "double je = s->j[a][id];", 0),
    ("extrapolation slope reversed", "double je = 2.0 * s->j[a][id] - s->jp[a][id];",
     "double je = 2.0 * s->jp[a][id] - s->j[a][id];", 0),
    ("no history before the first step", "s->jp[a][id] = s->j[a][id]; /* R17", "s->jp[a][id] = 0.0; /* R17", 0),
    ("history not advanced", "s->jp[a][id] = s->j[a][id];\n", "s->jp[a][id] = s->jp[a][id];\n", 0),
]


def _build_mutant(tmp_path, old, new, occurrence):
    text = open(SRC).read()
    at = -1
    for _ in range(occurrence + 1):
        at = text.index(old, at + 1)
    text = text[:at] + new + text[at + len(old):]
    src = tmp_path / "mutant.c"
    src.write_text(text)
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                    "-o", str(so), str(src), "-lm"], check=True)
    return oracle.load(str(so))


def _disagrees(L, scheme):
    from brute_force import BruteForce

    for name, prob in sorted(_tiny_cases().items()):
        bf = BruteForce(prob, scheme)
        u0, v0 = prob.initial()
        s = oracle.Solver(oracle.problem_from(prob, scheme), u0, v0, library=L)
        try:
            for _ in range(3):
                bf.step()
                s.step(1)
                got, ref = bf.fields(), s.read()
                for k in ("u", "v", "r"):
                    scale = max(np.abs(got[k]).max(), 1e-30)
                    if not np.abs(got[k] - ref[k]).max() <= 1e-12 * scale:
                        return name
        finally:
            s.close()
    return None


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc needed to build the mutants")
@pytest.mark.parametrize("what,old,new,occ", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, what, old, new, occ):
    L = _build_mutant(tmp_path, old, new, occ)
    caught = (_disagrees(L, oracle.PREDICTOR) or _disagrees(L, oracle.EXPLICIT)
              or _disagrees(L, oracle.EXTRAPOLATED))
    assert caught is not None, f"planted mistake not caught: {what}"
