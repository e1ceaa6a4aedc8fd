"""Stored trajectories of the 64-atom correctness workload (tests/golden/).

The files are written by tests/golden/make_golden.py from the oracle.  On the
CPU: the oracle still reproduces their first steps, and they carry the
properties the method fixes (Tr(K0 S) = n/2 at half filling, charge kept
to the truncation level, a linear response along the kick only at first
order).  On the GPU: 200 steps through the C ABI match them.
"""
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


def _load(prop):
    return np.loadtxt(make_golden.path(prop))


@pytest.mark.parametrize("prop", ["em", "cn"])
def test_oracle_reproduces_stored_steps(prop):
    ref = _load(prop)
    rows = make_golden.trajectory(prop, steps=8)
    assert np.array_equal(rows[:, 0], ref[:8, 0])
    for c in range(1, 5):
        assert np.abs(rows[:, c] - ref[:8, c]).max() <= 1e-12 * np.abs(ref[:8, c]).max(), c


@pytest.mark.parametrize("prop", ["em", "cn"])
def test_stored_trajectory_properties(prop):
    ref = _load(prop)
    assert ref.shape == (make_golden.STEPS, 5)
    assert np.allclose(ref[:, 0], 0.05 * np.arange(1, make_golden.STEPS + 1), rtol=0, atol=1e-12)
    # half filling of 256 functions: Tr(K S) = 128, kept to the truncation level
    assert np.abs(ref[:, 1] - 128.0).max() < 1e-4
    # the x response oscillates about its start (no secular drift larger than the swing)
    dx = ref[:, 2] - ref[0, 2]
    assert np.abs(dx).max() > 1e-2
    assert abs(dx.mean()) < np.abs(dx).max()


@pytest.mark.gpu
@pytest.mark.parametrize("prop", ["em", "cn"])
def test_gpu_matches_stored_trajectory(prop):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1404_5776_gb300 as rt
    rt.build()
    ref = _load(prop)
    s, K0, _ = make_golden.workload()
    ctx = rt.RT(s, dt=0.05, prop=prop, **make_golden.RADII)
    ctx.inverse()
    ctx.set_density_dense(0, 0, K0)
    ctx.kick(0, 0, 0, make_golden.KAPPA)
    ctx.step(make_golden.STEPS)
    obs = ctx.observables(0, 0)
    ctx.close()
    assert obs.shape[0] == make_golden.STEPS
    assert np.abs(obs[:, 0] - ref[:, 0]).max() < 1e-12
    for c in range(4):
        g, r = obs[:, 1 + 2 * c], ref[:, 1 + c]
        assert np.abs(g - r).max() <= 1e-10 * np.abs(r).max(), c
    ind_g = obs[:, 3] - obs[0, 3]
    ind_r = ref[:, 2] - ref[0, 2]
    assert np.abs(ind_g - ind_r).max() <= 1e-7 * np.abs(ind_r).max()
