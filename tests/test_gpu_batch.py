"""Batched contexts: several systems of uneven size and block size, each with
x, y and z kicks, advanced together by one rt_step, against the oracle run
system by system and kick by kick.

Bars: FP64 mode 1e-10 relative on K and on every trace.  Mixed precision in
the reference split (the mode that carries the precision claim): the dipole
along each kick within 1e-6 of its induced swing, max_t |P - P_FP64| /
max_t |P_FP64(t) - P_FP64(t_1)|.  The literal FP32 path (FP32 products on the
whole K) is checked at its own, looser level: 1e-6 of |P|, and 3e-4 of the
induced swing after 10 steps (the cluster's swing is ~20 times smaller than the
cells'); it does not meet the 1e-6 induced bar.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

R = 6.0
KAPPA = 1e-3


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1404_5776_gb300 as m
    m.build()
    return m


@pytest.fixture(scope="module")
def systems():
    pos, species = synth.si_h_cluster(target=60)
    cluster = synth.build_system(pos, None, species, 5.0, 5.0)         # 1 + 4 functions, open
    return [synth.diamond_system(2, "spd13", 6.0, 6.0),                # 64 atoms x 13
            cluster,
            synth.diamond_system(3, "sp4", 6.0, 6.0, seed=3)]          # 216 atoms x 4


def _radii():
    return dict(r_Sinv=R, r_T=R, r_U=R, r_K=R, r_M=R)


def _oracle_runs(systems, steps, prop):
    out = []
    for s in systems:
        n_occ = int(np.sum(s.bsize)) // 2
        K0, _, _ = synth.ground_state_dense(s, n_occ)
        per_kick = []
        for d in range(3):
            ref = oracle.Propagator(s, oracle.Params(prop=prop, **_radii()))
            ref.set_density_dense(K0)
            ref.kick(d, KAPPA)
            rows = [ref.step()["obs"] for _ in range(steps)]
            per_kick.append((ref.K.val.copy(), np.array(rows)))
        out.append((K0, per_kick))
    return out


def _gpu_run(rt, systems, refs, steps, prop, precision):
    ctx = rt.RT(systems, prop=prop, precision=precision, n_kick=3, **_radii())
    ctx.inverse()
    for si, (K0, _) in enumerate(refs):
        for d in range(3):
            ctx.set_density_dense(si, d, K0)
            ctx.kick(si, d, d, KAPPA)
    ctx.step(steps)
    return ctx


@pytest.mark.parametrize("prop", ["em", "cn"])
def test_batched_systems_and_kicks_fp64(rt, systems, prop):
    steps = 6
    refs = _oracle_runs(systems, steps, prop)
    ctx = _gpu_run(rt, systems, refs, steps, prop, "fp64")
    for si, (_, per_kick) in enumerate(refs):
        for d, (Kref, rows) in enumerate(per_kick):
            Kg = ctx.matrix(si, rt.RT_MAT_K, kick=d)
            assert np.abs(Kg - Kref).max() <= 1e-10 * np.abs(Kref).max(), (si, d)
            obs = ctx.observables(si, d)
            assert obs.shape[0] == steps
            for c in range(4):  # Tr(KS), Tr(K Dx), Tr(K Dy), Tr(K Dz)
                g = obs[:, 1 + 2 * c]
                r = rows[:, c].real
                assert np.abs(g - r).max() <= 1e-10 * np.abs(r).max(), (si, d, c)
            # the kicked direction responds: its induced dipole matches too
            ind_g = obs[:, 3 + 2 * d] - obs[0, 3 + 2 * d]
            ind_r = rows[:, 1 + d].real - rows[0, 1 + d].real
            assert np.abs(ind_g - ind_r).max() <= 1e-7 * max(np.abs(ind_r).max(), 1e-300), (si, d)
    ctx.close()


def test_batched_systems_and_kicks_mixed_literal(rt, systems):
    """The literal FP32 path, at its own accuracy level (see the module docstring)."""
    steps = 10
    refs = _oracle_runs(systems, steps, "em")
    ctx = _gpu_run(rt, systems, refs, steps, "em", "fp32")
    for si, (_, per_kick) in enumerate(refs):
        for d, (_, rows) in enumerate(per_kick):
            obs = ctx.observables(si, d)
            p64 = rows[:, 1 + d].real
            err = np.abs(obs[:, 3 + 2 * d] - p64).max()
            assert err <= 1e-6 * np.abs(p64).max(), (si, d)
            assert err <= 3e-4 * np.abs(p64 - p64[0]).max(), (si, d)
            q64 = rows[:, 0].real
            assert np.abs(obs[:, 1] - q64).max() <= 1e-6 * np.abs(q64).max(), (si, d)
    ctx.close()


@pytest.mark.parametrize("full_step", [0, 1])
def test_batched_reference_split(rt, systems, full_step):
    """Mixed precision in the reference split for every (system, kick) of the
    batch (block sizes 13 and 4, the cluster padded from 1 to 4), with U built
    once (full_step = 0) or from the field polynomial at every step."""
    steps = 10
    refs = _oracle_runs(systems, steps, "em")
    kw = dict(prop="em", precision="fp32", n_kick=3, incremental=1, full_step=full_step)
    if full_step:
        kw["field_poly"] = 1
    ctx = rt.RT(systems, **kw, **_radii())
    ctx.inverse()
    for si, (K0, _) in enumerate(refs):
        for d in range(3):
            ctx.set_density_dense(si, d, K0)
            ctx.kick(si, d, d, KAPPA)
    if not full_step:
        ctx.propagator(0.0)
    ctx.step(steps)
    for si, (_, per_kick) in enumerate(refs):
        for d, (_, rows) in enumerate(per_kick):
            obs = ctx.observables(si, d)
            p64 = rows[:, 1 + d].real
            err = np.abs(obs[:, 3 + 2 * d] - p64).max()
            assert err <= 1e-6 * np.abs(p64 - p64[0]).max(), (si, d, full_step)
            q64 = rows[:, 0].real
            assert np.abs(obs[:, 1] - q64).max() <= 1e-10 * np.abs(q64).max(), (si, d)
    ctx.close()
