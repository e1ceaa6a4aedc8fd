"""Mixed precision in the reference split against FP64, over 200-step runs.

The accuracy bar of the mixed-precision mode is the dipole error relative to
the induced swing,

    max_t |P_mixed(t) - P_FP64(t)| / max_t |P_FP64(t) - P_FP64(t_1)|  <= 1e-6,

with P = Re Tr(K D_x) along the field or kick and t_1 the first step (the
spectrum of Sec. II.B is built from the induced part P(t) - P(0) only).  The
error relative to |P| is checked as well (a much looser reading: P carries a
static dipole ~500 times the induced swing), and Tr(K S) to 1e-8 relative.

The reference split keeps the part of the step that acts on the O(1) density
K_ref in FP64 and runs the FP32 block products on dK = K - K_ref only, with
U - I stochastically rounded to FP32 at every step:
  * full step, EM with the field polynomial: U(E) and
    R(E) = sym(cut(cut(U(E) K_ref) U(E)^dagger)) - K_ref are polynomials in the
    field value (exact for H = H0 - E D), formed in FP64;
  * propagation step (U built once in FP64): R formed once; any propagator.

Against the oracle: 64 atoms x 13 functions, radii 6 A, 200 steps, stored in
tests/golden/ by make_golden.py (the oracle takes about a second per step).
Against the library's FP64 path (itself pinned to the oracle at 1e-10): 512
atoms x 13 functions, 200 steps, every propagator."""
import os
import sys

import numpy as np
import pytest

import synth

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402

pytestmark = pytest.mark.gpu

BAR_INDUCED = 1e-6
STEPS = make_golden.STEPS


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1404_5776_gb300 as m
    m.build()
    return m


@pytest.fixture(scope="module")
def w13():
    return make_golden.workload13()


def _errors(p_mixed, p_ref):
    """(error / induced swing, error / |P|) of a dipole trace."""
    err = np.abs(p_mixed - p_ref).max()
    return err / np.abs(p_ref - p_ref[0]).max(), err / np.abs(p_ref).max()


def _run13(rt, w13, prop, drive, full_step, steps=STEPS, **extra):
    s, K0, _ = w13
    kw = dict(prop=prop, precision="fp32", incremental=1, full_step=1 if full_step else 0, obs_capacity=steps + 8)
    if full_step:
        kw["field_poly"] = 1
    kw.update(extra)
    ctx = rt.RT(s, dt=0.05, **kw, **make_golden.RADII13)
    if drive == "pulse":
        f = make_golden.PULSE13
        ctx.set_field(kind=rt.RT_FIELD_GAUSSIAN, dir=0, E0=f["E0"], t0=f["t0"], sigma=f["sigma"], omega=f["omega"])
    ctx.inverse()
    ctx.set_density_dense(0, 0, K0)
    if drive == "kick":
        ctx.kick(0, 0, 0, make_golden.KAPPA)
    if not full_step:
        ctx.propagator(0.0)
    ctx.step(steps)
    obs = ctx.observables(0, 0)
    return ctx, obs


def _check_against(obs, ref, what):
    assert obs.shape[0] == ref.shape[0]
    assert np.abs(obs[:, 0] - ref[:, 0]).max() < 1e-12
    ind, rel_p = _errors(obs[:, 3], ref[:, 2])
    assert ind <= BAR_INDUCED, (what, ind)
    assert rel_p <= 1e-8, (what, rel_p)  # implied by the induced reading (|P| ~ 500 x the swing)
    swing = np.abs(ref[:, 2] - ref[0, 2]).max()
    for c, col in ((5, 3), (7, 4)):  # the other two dipole components, on the same scale
        assert np.abs(obs[:, c] - ref[:, col]).max() <= BAR_INDUCED * swing, (what, c)
    q = ref[:, 1]
    assert np.abs(obs[:, 1] - q).max() <= 1e-8 * np.abs(q).max(), what  # Tr(K S)
    assert np.all(obs[:, 9] < 1e-6)  # K hermitian to FP32 level before symmetrising


@pytest.mark.parametrize("drive", ["kick", "pulse"])
def test_full_step_em_matches_stored_oracle(rt, w13, drive):
    """EM full step (U(t + dt/2) rebuilt at every step) in the reference split,
    after a delta kick and under a Gaussian pulse (where U and R change at
    every step), against 200 stored oracle steps."""
    ref = np.loadtxt(make_golden.path13("em", drive, True))
    ctx, obs = _run13(rt, w13, "em", drive, True)
    ctx.close()
    _check_against(obs, ref, ("em", drive))


@pytest.mark.parametrize("prop", ["em", "cn", "etrs", "m4"])
def test_propagation_step_matches_stored_oracle(rt, w13, prop):
    """U built once in FP64 after the kick and reused (the field is zero after
    it, so for EM this is the full step's trajectory), 200 steps."""
    ref = np.loadtxt(make_golden.path13(prop, "kick", prop == "em"))
    ctx, obs = _run13(rt, w13, prop, "kick", False)
    ctx.close()
    _check_against(obs, ref, (prop, "propagation step"))


@pytest.fixture(scope="module")
def w512():
    s = synth.diamond_system(4, "spd13", 6.0, 6.0)
    # chemical potential (mid-gap at two doubly occupied states per atom) and
    # spectral bounds from the 64-atom cell of the same model
    _, w, _ = synth.ground_state_dense(synth.diamond_system(2, "spd13", 6.0, 6.0), 128)
    return s, 0.5 * (w[127] + w[128]), float(w.min()) - 0.5, float(w.max()) + 0.5


def _pair512(rt, w512, prop, full_step, steps):
    s, mu, e_lo, e_hi = w512
    radii = dict(r_Sinv=6.0, r_T=6.0, r_U=6.0, r_K=6.0, r_M=6.0)
    out = {}
    for mode in ("fp64", "split"):
        kw = dict(prop=prop, full_step=1 if full_step else 0, obs_capacity=steps + 8)
        if mode == "split":
            kw.update(precision="fp32", incremental=1)
            if full_step:
                kw["field_poly"] = 1
        ctx = rt.RT(s, dt=0.05, **kw, **radii)
        ctx.inverse()
        # ground state by the library's Chebyshev expansion: the same K0 for both runs
        ctx.ground_state(0, 200, mu, 0.01, e_lo, e_hi)
        ctx.kick(0, 0, 0, 1e-3)
        if not full_step:
            ctx.propagator(0.0)
        ctx.step(steps)
        out[mode] = ctx.observables(0, 0)
        ctx.close()
    return out["fp64"], out["split"]


@pytest.mark.parametrize("prop,full_step", [("em", True), ("em", False), ("cn", False), ("etrs", False),
                                            ("m4", False)])
def test_512_atoms_against_fp64(rt, w512, prop, full_step):
    """512 atoms x 13 functions (n = 6656), radii 6 A, 200 steps: the reference
    split against the library's FP64 path from the same K(0+)."""
    o64, o32 = _pair512(rt, w512, prop, full_step, STEPS)
    assert o64.shape[0] == o32.shape[0] == STEPS
    ind, rel_p = _errors(o32[:, 3], o64[:, 3])
    assert ind <= BAR_INDUCED, (prop, full_step, ind)
    assert rel_p <= 1e-8, (prop, full_step, rel_p)
    assert np.abs(o32[:, 1] - o64[:, 1]).max() <= 1e-8 * np.abs(o64[:, 1]).max()


def test_unitarity_of_the_split_propagator(rt, w13):
    """The reference split applies the FP64 propagator (rounded per step without
    bias): its S-unitarity error equals the FP64 propagator's."""
    s = w13[0]
    out = {}
    for mode in ("fp64", "split"):
        kw = dict(prop="em", field_poly=1)
        if mode == "split":
            kw.update(precision="fp32", incremental=1)
        ctx = rt.RT(s, dt=0.05, **kw, **make_golden.RADII13)
        ctx.inverse()
        ctx.propagator(0.0)
        out[mode] = ctx.unitarity(0, True)
        ctx.close()
    assert abs(out["split"][0] - out["fp64"][0]) <= 1e-12
    assert abs(out["split"][1] - out["fp64"][1]) <= 1e-12


def test_checkpoint_resume_within_the_bar(rt, w13):
    """A checkpoint of a reference-split run holds K = K_ref + dK itself; a run
    restored from it forms a new reference and continues on the same
    trajectory (to the mixed bar; the split point differs, so not bit for bit)."""
    s, K0, _ = w13
    ref = np.loadtxt(make_golden.path13("em", "kick", True))
    ctx = rt.RT(s, dt=0.05, prop="em", precision="fp32", incremental=1, field_poly=1, obs_capacity=STEPS + 8,
                **make_golden.RADII13)
    ctx.inverse()
    ctx.set_density_dense(0, 0, K0)
    ctx.kick(0, 0, 0, make_golden.KAPPA)
    ctx.step(60)
    state = ctx.get_state()
    ctx.step(40)
    ctx.set_state(state)
    ctx.step(STEPS - 60)
    obs = ctx.observables(0, 0)  # steps 1..60, then 61..200 of the resumed run
    ctx.close()
    _check_against(obs, ref, "resumed")
