"""Checkpoint and resume: a body saved after N steps and restored into a
fresh context (or into itself) continues exactly as the uninterrupted run,
bit for bit, in every storage format and with time-dependent boundary data
(a traction ramp, moving walls); states of another body are refused."""
import numpy as np
import pytest

from paper_2208_13769_gb300 import lbm
from paper_2208_13769_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MASK = lbm.LBM_FIELD_U | lbm.LBM_FIELD_V | lbm.LBM_FIELD_R | lbm.LBM_FIELD_P


def _problems():
    moving = [W.Edge(W.DIRICHLET, value=(0.0, 0.0), rate=(0.003, -0.002))] * 4
    return [
        W.tension_block(40, T1=0.1),  # ramped traction: the step count sets the boundary data
        W.smooth_random(33, 40, moving, seed=15, amp=0.01, lam=0.45),
        W.smooth_random(150, 90, W.clamped_free_edges(), seed=31, amp=0.01, vamp=0.004, lam=0.3, mu=0.3),
        W.smooth_random(100, 70, W.all_periodic(), seed=11, amp=0.02, lam=0.45),
    ]


def _same(a, b, what):
    assert a["t"] == b["t"], what
    for k in ("u", "v", "r", "P"):
        assert np.array_equal(a[k], b[k]), (what, k)


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
def test_resume_in_a_fresh_context_is_bitwise_the_uninterrupted_run(storage):
    n = 75  # a 64-step graph and plain steps on each side of the checkpoint
    for prob in _problems():
        with lbm.Body(prob, storage=storage) as whole:
            whole.step(2 * n)
            ref = whole.read(MASK)
        with lbm.Body(prob, storage=storage) as first:
            first.step(n)
            state = first.save_state()
            assert state.size == lbm.lbm_state_size(first.ctx) > 0
            at_save = first.read(MASK)
        with lbm.Body(prob, storage=storage) as second:
            second.load_state(state)
            assert lbm.lbm_get_info(second.ctx)[0] == n
            _same(second.read(MASK), at_save, (prob.name, storage, "restored"))
            assert np.array_equal(second.save_state(), state)  # the round trip keeps every byte
            second.step(n)
            _same(second.read(MASK), ref, (prob.name, storage, "resumed"))


def test_extrapolated_scheme_resumes_bitwise():
    """The extrapolated scheme's state holds two more carry planes (j of two
    time levels); a resumed run continues bit for bit."""
    n = 75
    prob = W.smooth_random(150, 90, W.clamped_free_edges(), seed=31, amp=0.01, vamp=0.004, lam=0.3, mu=0.3)
    xs = lbm.LBM_SCHEME_EXTRAPOLATED
    with lbm.Body(prob, storage="f32", scheme=xs) as whole:
        whole.step(2 * n)
        ref = whole.read(MASK)
    with lbm.Body(prob, storage="f32", scheme=xs) as first:
        first.step(n)
        state = first.save_state()
    with lbm.Body(prob, storage="f32") as other:  # another scheme: refused
        with pytest.raises(lbm.LbmError):
            other.load_state(state)
    with lbm.Body(prob, storage="f32", scheme=xs) as second:
        second.load_state(state)
        second.step(n)
        _same(second.read(MASK), ref, "extrapolated resumed")


def test_rollback_within_one_context():
    prob = W.tension_block(40, T1=0.1)
    with lbm.Body(prob, storage="f32") as b:
        b.step(30)
        state = b.save_state()
        b.step(100)
        ref = b.read(MASK)
        b.load_state(state)
        b.step(100)
        _same(b.read(MASK), ref, "rollback")
        d1 = b.diagnostics()
        b.load_state(state)
        b.step(100)
        assert np.array_equal(b.diagnostics(), d1)


def test_states_of_another_body_are_refused():
    a = W.smooth_random(40, 30, W.clamped_free_edges(), seed=3, amp=0.01, lam=0.3, mu=0.3)
    b = W.smooth_random(41, 30, W.clamped_free_edges(), seed=3, amp=0.01, lam=0.3, mu=0.3)
    with lbm.Body(a, storage="f32") as ba:
        ba.step(5)
        state = ba.save_state()
        with lbm.Body(b, storage="f32") as bb:  # another size
            with pytest.raises(lbm.LbmError) as e:
                bb.load_state(state)
            assert e.value.status == lbm.LBM_E_INVALID
        with lbm.Body(a, storage="f16") as bc:  # another storage format
            with pytest.raises(lbm.LbmError):
                bc.load_state(state)
        soft = W.smooth_random(40, 30, W.clamped_free_edges(), seed=3, amp=0.01, lam=0.2, mu=0.2)
        with lbm.Body(soft, storage="f32") as bd:  # another material: another time step
            with pytest.raises(lbm.LbmError):
                bd.load_state(state)
        with lbm.Body(a, storage="f32") as be:
            with pytest.raises(lbm.LbmError):
                be.load_state(state[:-1])  # truncated
            bad = state.copy()
            bad[0] ^= 0xFF  # not a state
            with pytest.raises(lbm.LbmError):
                be.load_state(bad)
            be.load_state(state)  # the good one still loads
            be.step(5)


def test_interior_profiling_leaves_the_state_as_it_was():
    """lbm_profile_interior runs interior launches that compute no solution,
    between a device-side save and restore of the state: the body then
    continues bit for bit as if the call had not been made."""
    prob = W.smooth_random(150, 90, W.clamped_free_edges(), seed=31, amp=0.01, vamp=0.004, lam=0.3, mu=0.3)
    for storage in ("f32", "f16"):
        with lbm.Body(prob, storage=storage) as whole:
            whole.step(140)
            ref = whole.read(MASK)
        with lbm.Body(prob, storage=storage) as b:
            b.step(70)
            st, out = lbm.lbm_profile_interior(b.ctx, 33)
            assert st == lbm.LBM_OK and out[0] > 0 and out[1] == (150 - 4) * (90 - 4)
            b.step(70)
            _same(b.read(MASK), ref, (storage, "after profiling"))
