"""The FP32 form whose compensated displacement carry keeps its low word in
16 bits (LBM_UCARRY_COMPENSATED16, Body(compensated="lo16")): u = hi + lo
with hi an FP32 plane and lo stored as FP16 of lo 2^k (k fixed per body),
12 bytes per node for both components instead of the pair's 16.

The displacement then keeps about 35 significant bits, far more than the
rounding of the FP32 populations leaves in it, so the form is held to the
FP32 bounds of the pair (u, v and P within 1e-5 of the FP64 oracle at the
stated horizons), through every path that stores the carry: the interior
kernel, the edge tiles, the seam images of periodic bodies, batches and
checkpoints."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2208_13769_gb300 import lbm
from paper_2208_13769_gb300 import workloads as W
from parity_util import compare, run_both
from test_gpu_parity import CASES, FP32_STEPS, TOL, Pp, N0, D0

pytestmark = pytest.mark.gpu

LO16 = "lo16"


@pytest.mark.parametrize("name", sorted(FP32_STEPS))
def test_lo16_carry_parity(name):
    prob, _ = CASES[name]
    ref, got = run_both(prob, FP32_STEPS[name], "f32", compensated=LO16)
    compare(ref, got, TOL["f32"])


def test_lo16_carry_clamped_body_full_horizon():
    """The clamped body (192 x 96, omega 1.9) for its full 5000 steps."""
    prob = W.clamped_body(nx=192, ny=96, nu=0.25, vmax=0.01)
    ref, got = run_both(prob, 5000, "f32", compensated=LO16)
    compare(ref, got, TOL["f32"])


def test_lo16_carry_shear_wave_at_its_1000_steps():
    prob, _ = CASES["shear_wave_64"]
    ref, got = run_both(prob, 1000, "f32", compensated=LO16)
    compare(ref, got, TOL["f32"])


def test_lo16_carry_agrees_with_the_pair_to_its_precision():
    """On a body large enough for the interior kernel, after 300 steps u
    differs from the pair's by the FP32 populations' own rounding noise
    (once the two carries differ in a last bit, the populations round apart),
    well below the FP32 bound; the memory per node update is 8 bytes
    smaller."""
    prob = W.smooth_random(600, 400, W.clamped_free_edges(), seed=41, amp=0.01, vamp=0.004, lam=0.3, mu=0.3)
    out, moved = {}, {}
    for comp in (True, LO16):
        with lbm.Body(prob, storage="f32", compensated=comp, scheme=lbm.LBM_SCHEME_EXPLICIT) as b:
            assert lbm.lbm_get_tuning(b.ctx).plan == 2  # the interior kernel runs
            _, moved[comp] = lbm.lbm_memory_info(b.ctx)
            b.step(300)
            out[comp] = b.read(lbm.LBM_FIELD_U | lbm.LBM_FIELD_V)
    du = np.linalg.norm(out[LO16]["u"] - out[True]["u"]) / np.linalg.norm(out[True]["u"])
    assert du <= 2e-6, du
    assert moved[True] - moved[LO16] == 8, moved


@pytest.mark.parametrize("layout", ["x_periodic", "both_periodic"])
def test_lo16_carry_across_periodic_seams_matches_the_oracle(layout):
    """Plan 2 (the interior kernel across the seams, the seam images copied
    after each step, in the carry's own layout) and the default plan, against
    the oracle; plan 2 bit-identical to the same body in a batch."""
    edges = {"x_periodic": [Pp, Pp, D0, N0], "both_periodic": W.all_periodic()}
    prob = W.smooth_random(660, 620, edges[layout], seed=31, amp=0.01, vamp=0.004, lam=0.3, mu=0.3)
    s = oracle.solver_from(prob, oracle.EXPLICIT)
    s.step(60)
    ref = s.read()
    for plan in (0, 2):
        with lbm.Body(prob, storage="f32", compensated=LO16, scheme=lbm.LBM_SCHEME_EXPLICIT,
                      tuning=lbm.lbm_tuning(0, 0, -1, plan)) as b:
            b.step(60)
            got = b.read()
        compare(ref, got, TOL["f32"])
    with lbm.Body(prob, storage="f32", compensated=LO16, tuning=lbm.lbm_tuning(0, 0, -1, 2)) as alone:
        alone.step(60)
        a = alone.read(lbm.LBM_FIELD_U | lbm.LBM_FIELD_V)
    with lbm.Body(prob, storage="f32", compensated=LO16) as member:
        with lbm.Batch([member]) as batch:
            batch.step(60)
        m = member.read(lbm.LBM_FIELD_U | lbm.LBM_FIELD_V)
    assert np.array_equal(a["u"], m["u"]) and np.array_equal(a["v"], m["v"])


def test_lo16_carry_batch_members_are_bit_identical_to_single_bodies():
    probs = [W.smooth_random(nx, ny, W.clamped_free_edges(), seed=50 + i, amp=0.01, vamp=0.004, lam=0.3, mu=0.3)
             for i, (nx, ny) in enumerate(((700, 300), (96, 50), (400, 512)))]
    alone = []
    for p in probs:
        with lbm.Body(p, storage="f32", compensated=LO16, tuning=lbm.lbm_tuning(0, 0, -1, 2)) as b:
            b.step(90)
            alone.append(b.read(lbm.LBM_FIELD_U | lbm.LBM_FIELD_V))
    members = [lbm.Body(p, storage="f32", compensated=LO16) for p in probs]
    try:
        with lbm.Batch(members) as batch:
            batch.step(90)
        for m, a in zip(members, alone):
            got = m.read(lbm.LBM_FIELD_U | lbm.LBM_FIELD_V)
            assert np.array_equal(got["u"], a["u"]) and np.array_equal(got["v"], a["v"])
    finally:
        for m in members:
            m.close()


def test_lo16_carry_checkpoint_continues_bit_identically():
    """A saved state restores into a body of the same form and continues
    bit-identically; the pair's body refuses it (another carry layout)."""
    prob = W.smooth_random(600, 400, W.clamped_free_edges(), seed=43, amp=0.01, vamp=0.004, lam=0.3, mu=0.3)
    with lbm.Body(prob, storage="f32", compensated=LO16) as a:
        a.step(40)
        state = a.save_state()
        a.step(40)
        ref = a.read(lbm.LBM_FIELD_U | lbm.LBM_FIELD_V)
    with lbm.Body(prob, storage="f32", compensated=LO16) as b:
        b.load_state(state)
        b.step(40)
        got = b.read(lbm.LBM_FIELD_U | lbm.LBM_FIELD_V)
    assert np.array_equal(got["u"], ref["u"]) and np.array_equal(got["v"], ref["v"])
    with lbm.Body(prob, storage="f32", compensated=True) as c:
        with pytest.raises(lbm.LbmError):
            c.load_state(state)


def test_lo16_carry_saturates_without_overflow_beyond_its_range():
    """A displacement 4 times beyond the range of the low word (a rigid
    shift of 32 max(nx, ny) dX plus a small smooth field): the low word
    saturates instead of overflowing, the state stays finite and u keeps
    about FP32 precision against the FP64 path."""
    base = W.smooth_random(96, 50, W.all_periodic(), seed=44, amp=0.01, vamp=0.004, lam=0.3, mu=0.3)
    u0, v0 = base.initial()
    shift = 32 * max(base.nx, base.ny) * base.dX
    prob = dataclasses.replace(base, u0=u0 + shift, v0=v0)
    out = {}
    for st, comp in (("f64", None), ("f32", LO16)):
        with lbm.Body(prob, storage=st, compensated=comp) as b:
            b.step(50)
            out[st] = b.read(lbm.LBM_FIELD_U | lbm.LBM_FIELD_V)
            assert out[st]["status"] == lbm.LBM_OK
    assert np.all(np.isfinite(out["f32"]["u"]))
    du = out["f32"]["u"] - out["f64"]["u"]
    assert np.abs(du).max() <= 64 * np.finfo(np.float32).eps * shift, np.abs(du).max()
