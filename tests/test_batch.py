"""Batched stepping: several bodies advanced by shared launches give exactly
the results of stepping each body alone (the same kernels and arithmetic per
node), and exactly the oracle's within the FP64 tolerance."""
import numpy as np
import pytest

import oracle
from paper_2208_13769_gb300 import lbm
from paper_2208_13769_gb300 import workloads as W
from parity_util import compare

pytestmark = pytest.mark.gpu

Pp = W.Edge(W.PERIODIC)
N0 = W.Edge(W.NEUMANN)
D0 = W.Edge(W.DIRICHLET)


def _members():
    """Uneven sizes, every boundary kind, bodies with and without interior,
    periodic axes shorter than a tile, a ramped traction, differing
    materials and schemes."""
    return [
        (W.shear_wave(64), lbm.LBM_SCHEME_PREDICTOR),
        (W.smooth_random(96, 50, W.clamped_free_edges(), seed=12, amp=0.01, vamp=0.005, lam=0.3, mu=0.3),
         lbm.LBM_SCHEME_PREDICTOR),
        (W.smooth_random(4, 5, [D0, N0, N0, D0], seed=17, amp=0.02, lam=0.3, mu=0.3), lbm.LBM_SCHEME_PREDICTOR),
        (W.smooth_random(20, 8, W.all_periodic(), seed=13, amp=0.02, lam=0.45), lbm.LBM_SCHEME_PREDICTOR),
        (W.smooth_random(70, 37, [Pp, Pp, D0, N0], seed=14, amp=0.01, lam=0.2, mu=0.2), lbm.LBM_SCHEME_EXPLICIT),
        (W.smooth_random(300, 260, W.clamped_free_edges(), seed=21, amp=0.01, vamp=0.004, lam=0.3, mu=0.3),
         lbm.LBM_SCHEME_PREDICTOR),
        (W.tension_block(40, T1=0.1), lbm.LBM_SCHEME_PREDICTOR),
    ]


def _fields(body):
    return body.read(lbm.LBM_FIELD_U | lbm.LBM_FIELD_V | lbm.LBM_FIELD_R | lbm.LBM_FIELD_P)


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
def test_batch_is_bitwise_the_single_body_step(storage):
    steps = 150  # a warm-up step, two graph chunks of 64, plain steps
    members = _members()
    alone = []
    for prob, scheme in members:
        with lbm.Body(prob, storage=storage, scheme=scheme) as b:
            b.step(steps)
            alone.append(_fields(b))
    bodies = [lbm.Body(prob, storage=storage, scheme=scheme) for prob, scheme in members]
    try:
        with lbm.Batch(bodies) as batch:
            batch.step(steps - 20)
            batch.step(20)
            assert all(s == lbm.LBM_OK for s in batch.sync())
            info = batch.info()
            assert info["steps"] == steps and info["interior_ctas"] > 0 and info["edge_ctas"] > 0
        for k, b in enumerate(bodies):
            got = _fields(b)
            assert got["t"] == alone[k]["t"]
            for key in ("u", "v", "r", "P"):
                assert np.array_equal(got[key], alone[k][key]), (k, key)
    finally:
        for b in bodies:
            b.close()


def test_batch_members_at_different_step_counts():
    """A member already advanced an odd number of steps on its own joins with
    its own phase; the batch advances everyone by the same count."""
    members = _members()[:4]
    pre = [0, 3, 1, 0]
    steps = 70
    alone = []
    for (prob, scheme), k0 in zip(members, pre):
        with lbm.Body(prob, storage="f32", scheme=scheme) as b:
            b.step(k0 + steps)
            alone.append(_fields(b))
    bodies = [lbm.Body(prob, storage="f32", scheme=scheme) for prob, scheme in members]
    try:
        for b, k0 in zip(bodies, pre):
            if k0:
                b.step(k0)
        with lbm.Batch(bodies) as batch:
            batch.step(steps)
        for k, b in enumerate(bodies):
            got = _fields(b)
            for key in ("u", "v", "r"):
                assert np.array_equal(got[key], alone[k][key]), (k, key)
    finally:
        for b in bodies:
            b.close()


def test_batch_member_matches_the_oracle():
    prob = W.smooth_random(96, 50, W.clamped_free_edges(), seed=12, amp=0.01, vamp=0.005, lam=0.3, mu=0.3)
    other = W.shear_wave(64)
    s = oracle.solver_from(prob, oracle.PREDICTOR)
    s.step(200)
    ref = s.read()
    s.close()
    pr = lbm.LBM_SCHEME_PREDICTOR
    with lbm.Body(prob, storage="f64", scheme=pr) as b, lbm.Body(other, storage="f64", scheme=pr) as b2:
        with lbm.Batch([b2, b]) as batch:
            batch.step(200)
        compare(ref, b.read(), 1e-12, keys=("u", "v", "P", "Pbar", "J", "sigma"))


def test_batch_reports_an_unstable_member_only():
    bad = W.smooth_random(40, 30, W.all_periodic(), seed=3, amp=0.0)
    x = np.arange(40)
    bad.u0[:, :, 0] = -2.0 * np.sin(2 * np.pi * x / 40)[None, :] * 40 / (2 * np.pi) * 1.5
    good = W.shear_wave(64)
    with lbm.Body(good, storage="f32") as g, lbm.Body(bad, storage="f32") as b:
        with lbm.Batch([g, b]) as batch:
            batch.step(5)
            st = batch.sync()
        assert st == [lbm.LBM_OK, lbm.LBM_E_UNSTABLE]


def test_batch_argument_and_phase_errors():
    p1 = W.shear_wave(64)
    with lbm.Body(p1, storage="f32") as a, lbm.Body(p1, storage="f64") as b, lbm.Body(p1, storage="f32") as c:
        L = lbm.lib()
        with pytest.raises(lbm.LbmError) as ei:
            lbm.Batch([a, b])  # mixed formats
        assert ei.value.status == lbm.LBM_E_INVALID
        with pytest.raises(lbm.LbmError):
            lbm.Batch([a, a])  # repeated member
        with pytest.raises(lbm.LbmError):
            lbm.Batch([])
        with lbm.Body(p1, storage="f32", scheme=lbm.LBM_SCHEME_EXTRAPOLATED) as x:
            with pytest.raises(lbm.LbmError) as ei:
                lbm.Batch([a, x])  # the extrapolated scheme runs as a single body only
            assert ei.value.status == lbm.LBM_E_INVALID
        with lbm.Batch([a, c]) as batch:
            batch.step(2)
            c.step(1)  # a member stepped on its own: out of phase
            assert L.lbm_batch_step(batch.handle, 1) == lbm.LBM_E_STATE


def test_batch_tuning_changes_the_split_not_the_result():
    """Every decomposition of a batch's interior tiles (ring depth, rows per
    tile, strip grid) gives bit-identical members; the batch autotuner
    returns one of its candidates and leaves the members untouched; bad
    tunings are refused."""
    members = _members()[:6]
    ref = []
    for prob, scheme in members:
        with lbm.Body(prob, storage="f32", scheme=scheme) as b:
            b.step(90)
            ref.append(_fields(b))
    for ring, chunk, aligned in ((4, 0, -1), (6, 8, 1), (8, 40, 0), (5, 256, 2), (4, 48, 0), (4, 64, 2)):
        bodies = [lbm.Body(prob, storage="f32", scheme=scheme) for prob, scheme in members]
        try:
            with lbm.Batch(bodies, tuning=lbm.lbm_tuning(ring, chunk, aligned)) as batch:
                batch.step(90)
                batch.sync()
            for k, b in enumerate(bodies):
                got = _fields(b)
                for key in ("u", "v", "r", "P"):
                    assert np.array_equal(got[key], ref[k][key]), (ring, chunk, aligned, k, key)
        finally:
            for b in bodies:
                b.close()
    bodies = [lbm.Body(prob, storage="f32", scheme=scheme) for prob, scheme in members]
    try:
        for b in bodies:
            b.step(3)
        before = [b.read(lbm.LBM_FIELD_U)["u"] for b in bodies]
        best, ms = lbm.lbm_batch_autotune([b.ctx for b in bodies], 16)
        assert best.ring_slots in (4, 5, 6) and best.chunk_rows in (0, 32, 64, 128, 256) and 0 < ms < 10
        assert best.aligned in (0, 1, 2)
        for b, u in zip(bodies, before):
            assert lbm.lbm_get_info(b.ctx)[0] == 3
            assert np.array_equal(b.read(lbm.LBM_FIELD_U)["u"], u)
        for bad in (lbm.lbm_tuning(3, 0, 1), lbm.lbm_tuning(9, 0, 1), lbm.lbm_tuning(5, 7, 1), lbm.lbm_tuning(4, 0, 3)):
            with pytest.raises(lbm.LbmError) as ei:
                lbm.Batch(bodies, tuning=bad)
            assert ei.value.status == lbm.LBM_E_INVALID
    finally:
        for b in bodies:
            b.close()


@pytest.mark.auto_plan
def test_batch_of_small_bodies_agrees_with_their_default_plan():
    """With the library's default plan a small body stepped alone runs edge
    tiles only, while the batch advances it with the interior kernel: the
    two agree to rounding (FP64: 1e-12), and the batch matches the oracle."""
    members = [m for m in _members() if m[0].nx * m[0].ny < (1 << 17)]
    steps = 70
    alone = []
    for prob, scheme in members:
        with lbm.Body(prob, storage="f64", scheme=scheme) as b:
            b.step(steps)
            alone.append(_fields(b))
            assert lbm.lbm_get_tuning(b.ctx).plan == 1
    bodies = [lbm.Body(prob, storage="f64", scheme=scheme) for prob, scheme in members]
    try:
        with lbm.Batch(bodies) as batch:
            batch.step(steps)
        for (prob, scheme), b, ref in zip(members, bodies, alone):
            got = _fields(b)
            for k in ("u", "v", "P"):
                scale = max(np.linalg.norm(ref[k]), 1e-30)
                assert np.linalg.norm(got[k] - ref[k]) <= 1e-12 * scale, (prob.name, k)
            s = oracle.solver_from(prob, scheme)
            s.step(steps)
            compare(s.read(), got, 1e-12)
    finally:
        for b in bodies:
            b.close()
