"""Stored trajectories of the 64-atom correctness workloads (tests/golden/).

The files are written by tests/golden/make_golden.py from the oracle.  On the
CPU: the oracle still reproduces their first steps, and they carry the
properties the method fixes (Tr(K0 S) = number of occupied states, charge kept
to the truncation level, an induced dipole along the drive).  On the GPU: 200
steps through the C ABI match them (4-function cell here, FP64; the
13-function trajectories are the mixed-precision references of
test_gpu_reference_split.py).
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


@pytest.mark.parametrize("case", make_golden.CASES13)
def test_oracle_reproduces_stored_steps_13(case):
    prop, drive, rebuild = case
    ref = np.loadtxt(make_golden.path13(prop, drive, rebuild))
    rows = make_golden.trajectory13(prop, drive, rebuild, steps=2)
    assert np.array_equal(rows[:, 0], ref[:2, 0])
    for c in range(1, 5):
        assert np.abs(rows[:, c] - ref[:2, c]).max() <= 1e-12 * np.abs(ref[:2, c]).max(), c


@pytest.mark.parametrize("case", make_golden.CASES13)
def test_stored_trajectory_properties_13(case):
    ref = np.loadtxt(make_golden.path13(*case))
    assert ref.shape == (make_golden.STEPS, 5)
    assert np.allclose(ref[:, 0], 0.05 * np.arange(1, make_golden.STEPS + 1), rtol=0, atol=1e-12)
    # two doubly occupied states per atom: Tr(K S) = 128 after the first step; the
    # truncation at 6 A (42 of 64 blocks per atom) is not exactly unitary, and the
    # charge drifts by ~1e-3 relative over 200 steps (CN with two Hotelling
    # iterations from a cold start: by ~1.5e-2)
    assert abs(ref[0, 1] - 128.0) < 1e-3
    drift = np.abs(ref[:, 1] - ref[0, 1]).max() / 128.0
    assert drift < (3e-2 if case[0] == "cn" else 2e-3)
    # the x dipole responds to the x drive and oscillates without a secular drift larger than its swing
    dx = ref[:, 2] - ref[0, 2]
    assert np.abs(dx).max() > 1e-3 * np.abs(ref[:, 2]).max()
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
