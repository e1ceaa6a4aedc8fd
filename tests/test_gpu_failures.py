"""Failure detection with host-side fault injection (rt_debug_inject): nothing
is made to fault or hang on the GPU.  A bounded device wait given a zero
budget gives up at once, drains its copies in flight, sets the error word and
the step reports RT_ETIMEOUT; a checkpoint restores the context, after which
the run matches an uninterrupted one bit for bit."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1404_5776_gb300 as m
    m.build()
    return m


def _radii(r=6.0):
    return dict(r_Sinv=r, r_T=r, r_U=r, r_K=r, r_M=r)


@pytest.fixture(scope="module")
def system():
    s = synth.diamond_system(2, "spd13", 6.0, 6.0)
    K0, _, _ = synth.ground_state_dense(s, 2 * s.n_atoms)
    return s, K0


def test_hotelling_maxiter_injection(rt, system):
    s, _ = system
    ctx = rt.RT(s, **_radii())
    ctx.debug_inject(rt.RT_FAULT_HOTELLING_MAXITER1)
    with pytest.raises(rt.RTError) as e:
        ctx.inverse()
    assert e.value.status == rt.RT_ENOTCONV
    it, res = ctx.inverse()  # one-shot: the next inverse converges
    assert res < 1e-10
    ctx.close()


def test_nan_in_h_is_reported(rt, system):
    s, K0 = system
    for precision in ("fp64", "fp32"):
        ctx = rt.RT(s, precision=precision, **_radii())
        ctx.inverse()
        ctx.set_density_dense(0, 0, K0)
        ctx.debug_inject(rt.RT_FAULT_NAN_IN_H)
        ctx.step(2)
        with pytest.raises(rt.RTError) as e:
            ctx.observables(0, 0)
        assert e.value.status == rt.RT_ENUMERIC, precision
        ctx.close()


@pytest.mark.parametrize("incremental", [0, 1])
def test_wait_timeout_then_resume_from_checkpoint(rt, system, incremental):
    """A bounded wait that gives up poisons the context; a restore that is
    rejected (a truncated checkpoint) leaves it poisoned; a valid restore
    resumes it.  The literal path resumes bit for bit; the reference split
    forms dK = K - K_ref again from the restored K (one FP64 rounding)."""
    s, K0 = system
    kw = dict(precision="fp32", **_radii())
    if incremental:
        kw.update(incremental=1, field_poly=1)
    ref = rt.RT(s, **kw)
    ref.inverse()
    ref.set_density_dense(0, 0, K0)
    ref.kick(0, 0, 0, 1e-3)
    ref.step(3)
    ref_obs = ref.observables(0, 0)
    K_ref = ref.matrix(0, rt.RT_MAT_K)
    ref.close()

    ctx = rt.RT(s, **kw)
    ctx.inverse()
    ctx.set_density_dense(0, 0, K0)
    ctx.kick(0, 0, 0, 1e-3)
    ctx.step(1)
    state = ctx.get_state()
    ctx.debug_inject(rt.RT_FAULT_WAIT_TIMEOUT_0)
    with pytest.raises(rt.RTError) as e:
        ctx.step(1)
    assert e.value.status == rt.RT_ETIMEOUT
    with pytest.raises(rt.RTError) as e:  # poisoned until a checkpoint is restored
        ctx.step(1)
    assert e.value.status == rt.RT_ESTATE
    with pytest.raises(rt.RTError) as e:  # a rejected restore clears nothing
        ctx.set_state(state[:-8])
    assert e.value.status == rt.RT_EINVAL
    with pytest.raises(rt.RTError) as e:
        ctx.step(1)
    assert e.value.status == rt.RT_ESTATE
    ctx.set_state(state)
    ctx.step(2)
    obs = ctx.observables(0, 0)
    K = ctx.matrix(0, rt.RT_MAT_K)
    ctx.close()
    if incremental:
        assert np.abs(K - K_ref).max() <= 1e-12 * np.abs(K_ref).max()
        assert np.abs(obs[-2:, 3] - ref_obs[-2:, 3]).max() <= 1e-12 * np.abs(ref_obs[-2:, 3]).max()
    else:
        assert np.array_equal(K, K_ref)
        assert np.array_equal(obs[-2:], ref_obs[-2:])


def test_unknown_fault_flag_rejected(rt, system):
    s, _ = system
    ctx = rt.RT(s, **_radii())
    with pytest.raises(rt.RTError) as e:
        ctx.debug_inject(1 << 10)
    assert e.value.status == rt.RT_EINVAL
    ctx.close()
