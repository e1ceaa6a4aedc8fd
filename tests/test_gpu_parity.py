"""CUDA path (through the C ABI) against the CPU oracle, element by element.

Tolerance: FP64 mode 1e-10 relative (the stated FP64 parity bar) on K, on the
dipole Tr(K D_x) and on S^-1; patterns bit-exact.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

REL = 1e-10


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1404_5776_gb300 as m
    m.build()
    return m


def _radii(r, **over):
    d = dict(r_Sinv=r, r_T=r, r_U=r, r_K=r, r_M=r)
    d.update(over)
    return d


def relerr(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


# --------------------------------------------------------------------------
# patterns (bit-exact)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("ncell,radii", [(2, (3.0, 6.0, 8.0, 20.0)), (4, (6.0, 7.0, 10.0))])
def test_patterns_bit_exact(rt, ncell, radii):
    s = synth.diamond_system(ncell, "sp4", 6.0, 6.0)
    names = ["r_Sinv", "r_T", "r_U", "r_K", "r_M"]
    for r in radii:
        ctx = rt.RT(s, **{n: r for n in names})
        for which in (rt.RT_PAT_SINV, rt.RT_PAT_U, rt.RT_PAT_K):
            rp, col = ctx.pattern(0, which)
            ref = oracle.pattern(s.pos, s.cell, r)
            assert np.array_equal(rp, ref.rowptr) and np.array_equal(col, ref.col), (r, which)
        # P_A = P_{max(r_S, r_H)} and the given S pattern round-trips
        rp, col = ctx.pattern(0, rt.RT_PAT_A)
        ref = oracle.pattern(s.pos, s.cell, 6.0)
        assert np.array_equal(rp, ref.rowptr) and np.array_equal(col, ref.col)
        ctx.close()


def test_patterns_open_system_and_full_size(rt):
    rng = np.random.default_rng(11)
    pos = rng.uniform(0, 20.0, size=(300, 3))
    s = synth.build_system(pos, None, ["sp4"] * 300, 4.0, 4.0)
    ctx = rt.RT(s, **_radii(7.5))
    rp, col = ctx.pattern(0, rt.RT_PAT_U)
    ref = oracle.pattern(s.pos, None, 7.5)
    assert np.array_equal(rp, ref.rowptr) and np.array_equal(col, ref.col)
    ctx.close()


# --------------------------------------------------------------------------
# Hotelling S^-1 (Sec. V.A)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("basis,r", [("sp4", 6.0), ("spd13", 6.0), ("sp4", 20.0)])
def test_hotelling_matches_oracle(rt, basis, r):
    s = synth.diamond_system(2, basis, 6.0, 6.0)
    ctx = rt.RT(s, **_radii(r))
    it, res = ctx.inverse()
    X = ctx.matrix(0, rt.RT_MAT_SINV)
    ref = oracle.hotelling(oracle.BlockMatrix(s.bsize, oracle.Pattern(s.s_rowptr, s.s_col), s.s_val),
                           oracle.pattern(s.pos, s.cell, r), tol=1e-10, maxit=100)
    assert it == ref.iters
    assert abs(res - ref.residual) <= 1e-8 * max(ref.residual, 1e-14) + 1e-15
    assert relerr(X, ref.X.val) < REL
    ctx.close()


# --------------------------------------------------------------------------
# the step (EM and CN), FP64
# --------------------------------------------------------------------------

def _run_pair(rt, s, prop, radii, steps, n_occ, kappa=1e-3, field=None, hot_iters=2, full_step=1,
              use_graph=1, field_first=False, **gpu_params):
    K0, _, _ = synth.ground_state_dense(s, n_occ)
    ctx = rt.RT(s, dt=0.05, prop=prop, hot_step_iters=hot_iters, full_step=full_step, use_graph=use_graph,
                **radii, **gpu_params)
    if field and field_first:
        ctx.set_field(**field)
    ctx.inverse()
    if field and not field_first:
        ctx.set_field(**field)
    ctx.set_density_dense(0, 0, K0)
    ctx.kick(0, 0, 0, kappa)
    if not full_step:
        ctx.propagator(0.0)
    ctx.step(steps)
    obs = ctx.observables(0, 0)
    Kg = ctx.matrix(0, rt.RT_MAT_K)
    Ug = ctx.matrix(0, rt.RT_MAT_U)
    ctx.close()
    of = None
    if field:
        of = {"kind": {1: "gaussian", 2: "constant"}[field["kind"]], "E0": field["E0"], "t0": field.get("t0", 0.0),
              "sigma": field.get("sigma", 1.0), "omega": field.get("omega", 0.0)}
    ref = oracle.Propagator(s, oracle.Params(dt=0.05, prop=prop, hot_step_iters=hot_iters, field=of,
                                             field_dir=field["dir"] if field else 0, **radii))
    ref.set_density_dense(K0)
    ref.kick(0, kappa)
    rows = []
    for _ in range(steps):
        out = ref.step(rebuild=bool(full_step))
        rows.append([out["t"]] + [v for z in out["obs"] for v in (z.real, z.imag)])
    return obs, Kg, Ug, np.array(rows), ref


@pytest.mark.parametrize("prop", ["em", "cn"])
@pytest.mark.parametrize("basis,r,n_per_atom", [("sp4", 6.0, 2), ("spd13", 6.0, 2), ("sp4", 20.0, 2)])
def test_step_parity(rt, prop, basis, r, n_per_atom):
    s = synth.diamond_system(2, basis, 6.0, 6.0)
    obs, Kg, Ug, rows, ref = _run_pair(rt, s, prop, _radii(r), 10, n_per_atom * s.n_atoms)
    assert relerr(Kg, ref.K.val) < REL
    assert relerr(Ug, ref.U.val) < REL
    assert np.allclose(obs[:, 0], rows[:, 0], rtol=0, atol=1e-12)
    # charge and dipole: Tr(KS), Tr(K Dx) (relative to their magnitude)
    for col in (1, 3, 5, 7):
        assert relerr(obs[:, col], rows[:, col]) < REL, col
    # the induced part of the dipole also matches (relative to its own amplitude)
    ind_g = obs[:, 3] - obs[0, 3]
    ind_r = rows[:, 3] - rows[0, 3]
    assert np.abs(ind_g - ind_r).max() <= 1e-7 * np.abs(ind_r).max()


def test_step_parity_gaussian_pulse_and_no_graph(rt):
    s = synth.diamond_system(2, "sp4", 6.0, 6.0)
    field = dict(kind=rt.RT_FIELD_GAUSSIAN, dir=1, E0=2e-3, t0=0.2, sigma=0.15, omega=1.1)
    obs, Kg, _, rows, ref = _run_pair(rt, s, "em", _radii(6.0), 12, s.n // 2, kappa=0.0, field=field, use_graph=0)
    assert relerr(Kg, ref.K.val) < REL
    for col in (1, 3, 5, 7):
        assert relerr(obs[:, col], rows[:, col]) < REL


@pytest.mark.parametrize("prop", ["etrs", "m4"])
@pytest.mark.parametrize("basis,radii", [("sp4", dict(r_Sinv=6.0, r_T=6.0, r_U=7.0, r_K=6.0, r_M=7.0)),
                                         ("spd13", dict(r_Sinv=6.0, r_T=7.0, r_U=6.0, r_K=6.0, r_M=6.0))])
def test_etrs_m4_parity_under_pulse(rt, prop, basis, radii):
    """ETRS and fourth-order Magnus (Sec. II.A) under a Gaussian pulse, so that
    T(t), T(t+dt) and the Gauss-Legendre samples T(t1), T(t2) all differ; with
    r_T > r_U the exponent is cut to P_U, with r_T < r_U it is zero-extended."""
    s = synth.diamond_system(2, basis, 6.0, 6.0)
    field = dict(kind=rt.RT_FIELD_GAUSSIAN, dir=2, E0=5e-3, t0=0.15, sigma=0.1, omega=1.3)
    obs, Kg, Ug, rows, ref = _run_pair(rt, s, prop, radii, 8, 2 * s.n_atoms, field=field)
    assert relerr(Kg, ref.K.val) < REL
    assert relerr(Ug, ref.U.val) < REL
    for col in (1, 3, 5, 7):
        assert relerr(obs[:, col], rows[:, col]) < REL, col
    ind_g = obs[:, 7] - obs[0, 7]
    ind_r = rows[:, 7] - rows[0, 7]
    assert np.abs(ind_g - ind_r).max() <= 1e-7 * np.abs(ind_r).max()


@pytest.mark.parametrize("prop", ["etrs", "m4"])
def test_etrs_m4_propagation_step(rt, prop):
    """Propagation step (U built once at t = 0, reused) for both propagators."""
    s = synth.diamond_system(2, "sp4", 6.0, 6.0)
    field = dict(kind=rt.RT_FIELD_CONSTANT, dir=0, E0=1e-3)
    obs, Kg, _, rows, ref = _run_pair(rt, s, prop, _radii(6.0), 6, s.n // 2, field=field, full_step=0)
    assert relerr(Kg, ref.K.val) < REL
    assert relerr(obs[:, 3], rows[:, 3]) < REL


@pytest.mark.parametrize("basis,radii", [("sp4", dict(r_Sinv=6.0, r_T=6.0, r_U=7.0, r_K=6.0, r_M=7.0)),
                                         ("spd13", dict(r_Sinv=6.0, r_T=7.0, r_U=6.0, r_K=6.0, r_M=6.0))])
@pytest.mark.parametrize("field_first", [False, True])
def test_field_polynomial_em_matches_oracle(rt, basis, radii, field_first):
    """EM with U formed as the polynomial sum_m E^m V_m in the field value:
    the literal truncated series of the oracle, step by step, under a pulse
    along z (the field axis set after rt_inverse forces the coefficients to
    be formed again)."""
    s = synth.diamond_system(2, basis, 6.0, 6.0)
    field = dict(kind=rt.RT_FIELD_GAUSSIAN, dir=2, E0=5e-3, t0=0.15, sigma=0.1, omega=1.3)
    obs, Kg, Ug, rows, ref = _run_pair(rt, s, "em", radii, 8, 2 * s.n_atoms, field=field, field_first=field_first,
                                       field_poly=1)
    assert relerr(Kg, ref.K.val) < REL
    assert relerr(Ug, ref.U.val) < REL
    for col in (1, 3, 5, 7):
        assert relerr(obs[:, col], rows[:, col]) < REL, col
    ind_g = obs[:, 7] - obs[0, 7]
    ind_r = rows[:, 7] - rows[0, 7]
    assert np.abs(ind_g - ind_r).max() <= 1e-7 * np.abs(ind_r).max()


def test_field_polynomial_mixed_blocks_and_terms(rt):
    """Block sizes 1 and 4 in an open cluster, 7 Taylor terms, kick."""
    pos, species = synth.si_h_cluster(target=60)
    s = synth.build_system(pos, None, species, 5.0, 5.0)
    n_occ = int(np.sum(s.bsize)) // 2
    K0, _, _ = synth.ground_state_dense(s, n_occ)
    ctx = rt.RT(s, dt=0.05, field_poly=1, taylor_terms=7, **_radii(7.0))
    ctx.inverse()
    ctx.set_density_dense(0, 0, K0)
    ctx.kick(0, 0, 0, 1e-3)
    ctx.step(5)
    obs = ctx.observables(0, 0)
    Kg = ctx.matrix(0, rt.RT_MAT_K)
    ctx.close()
    ref = oracle.Propagator(s, oracle.Params(dt=0.05, taylor_terms=7, **_radii(7.0)))
    ref.set_density_dense(K0)
    ref.kick(0, 1e-3)
    rows = [ref.step()["obs"] for _ in range(5)]
    assert relerr(Kg, ref.K.val) < REL
    assert relerr(obs[:, 3], np.array([r[1].real for r in rows])) < REL


def test_propagation_step_reuses_u(rt):
    s = synth.diamond_system(2, "sp4", 6.0, 6.0)
    obs, Kg, _, rows, ref = _run_pair(rt, s, "em", _radii(6.0), 8, s.n // 2, full_step=0)
    assert relerr(Kg, ref.K.val) < REL


def test_mixed_block_sizes_cluster(rt):
    """1- and 4-function atoms (padded to 4 on the device) in an open cluster."""
    pos, species = synth.si_h_cluster(target=60)
    s = synth.build_system(pos, None, species, 5.0, 5.0)
    n_occ = int(np.sum(s.bsize)) // 2
    obs, Kg, _, rows, ref = _run_pair(rt, s, "em", _radii(7.0), 6, n_occ)
    assert relerr(Kg, ref.K.val) < REL
    for col in (1, 3):
        assert relerr(obs[:, col], rows[:, col]) < REL


def test_several_tiles_and_ragged_tail(rt):
    """512 atoms x 13 functions: many CTAs with a partial last one."""
    s = synth.diamond_system(4, "spd13", 6.0, 6.0)
    obs, Kg, _, rows, ref = _run_pair(rt, s, "em", _radii(6.0, r_Sinv=6.0), 2, 2 * s.n_atoms)
    assert relerr(Kg, ref.K.val) < REL
    assert relerr(obs[:, 3], rows[:, 3]) < REL


# --------------------------------------------------------------------------
# ground state, unitarity, checkpoint, graph replay
# --------------------------------------------------------------------------

def test_ground_state_foe(rt):
    s = synth.diamond_system(2, "sp4", 6.0, 6.0)
    ctx = rt.RT(s, **_radii(8.0))
    ctx.inverse()
    ctx.ground_state(0, 60, -0.3, 0.05, -1.0, 1.0)
    Kg = ctx.matrix(0, rt.RT_MAT_K)
    ctx.close()
    ref = oracle.Propagator(s, oracle.Params(**_radii(8.0)))
    ref.ground_state(60, -0.3, 0.05, -1.0, 1.0)
    assert relerr(Kg, ref.K.val) < REL


@pytest.mark.parametrize("metric", [True, False])
def test_unitarity_matches_oracle(rt, metric):
    s = synth.diamond_system(2, "sp4", 6.0, 6.0)
    ctx = rt.RT(s, **_radii(6.0))
    ctx.inverse()
    ctx.propagator(0.0)
    mx, mean = ctx.unitarity(0, metric)
    ctx.close()
    ref = oracle.Propagator(s, oracle.Params(**_radii(6.0)))
    U, _ = ref.propagator(0.0)
    pw = oracle.pattern(s.pos, s.cell, 6.0 + 6.0)
    rmx, rmean = oracle.unitarity(U, ref.S if metric else None, pw)
    assert abs(mx - rmx) <= 1e-9 * rmx + 1e-15
    assert abs(mean - rmean) <= 1e-9 * rmean + 1e-15


def test_checkpoint_resume_bit_exact(rt):
    s = synth.diamond_system(2, "sp4", 6.0, 6.0)
    K0, _, _ = synth.ground_state_dense(s, s.n // 2)
    ctx = rt.RT(s, prop="cn", **_radii(6.0))
    ctx.inverse()
    ctx.set_density_dense(0, 0, K0)
    ctx.kick(0, 0, 0, 1e-3)
    ctx.step(3)
    state = ctx.get_state()
    ctx.step(4)
    K_a = ctx.matrix(0, rt.RT_MAT_K)
    obs_a = ctx.observables(0, 0)
    ctx.set_state(state)
    ctx.step(4)
    K_b = ctx.matrix(0, rt.RT_MAT_K)
    obs_b = ctx.observables(0, 0)
    ctx.close()
    assert np.array_equal(K_a, K_b)
    assert np.array_equal(obs_a[-4:], obs_b[-4:])


@pytest.mark.parametrize("prop", ["em", "etrs", "m4"])
def test_checkpoint_resume_mixed_propagation_step(rt, prop):
    """Mixed mode with U built once and reused (full_step = 0): only U - I is
    current (FP32), so the checkpoint carries U = I + (U - I) and the resumed
    run applies the same propagator (the kick left its own operator in U)."""
    s = synth.diamond_system(2, "sp4", 6.0, 6.0)
    K0, _, _ = synth.ground_state_dense(s, s.n // 2)
    ctx = rt.RT(s, prop=prop, precision="fp32", full_step=0, **_radii(6.0))
    ctx.inverse()
    ctx.set_density_dense(0, 0, K0)
    ctx.kick(0, 0, 0, 1e-3)
    ctx.propagator(0.0)
    ctx.step(2)
    state = ctx.get_state()
    ctx.step(3)
    K_a = ctx.matrix(0, rt.RT_MAT_K)
    obs_a = ctx.observables(0, 0)
    ctx.set_state(state)
    ctx.step(3)
    K_b = ctx.matrix(0, rt.RT_MAT_K)
    obs_b = ctx.observables(0, 0)
    ctx.close()
    assert np.abs(K_b - K_a).max() <= 1e-12 * np.abs(K_a).max()
    scale = np.abs(obs_a[-3:, 1]).max()  # Tr(KS)
    for col in (1, 3, 5, 7):  # Tr(KS), Tr(K Dx,y,z)
        assert np.abs(obs_b[-3:, col] - obs_a[-3:, col]).max() <= 1e-12 * scale, col


def test_graph_and_direct_launch_identical(rt):
    s = synth.diamond_system(2, "sp4", 6.0, 6.0)
    K0, _, _ = synth.ground_state_dense(s, s.n // 2)
    outs = []
    for g in (1, 0):
        ctx = rt.RT(s, use_graph=g, **_radii(6.0))
        ctx.inverse()
        ctx.set_density_dense(0, 0, K0)
        ctx.kick(0, 0, 0, 1e-3)
        ctx.step(6)
        outs.append((ctx.matrix(0, rt.RT_MAT_K), ctx.observables(0, 0)))
        ctx.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


def test_errors_are_reported(rt):
    s = synth.diamond_system(2, "sp4", 6.0, 6.0)
    ctx = rt.RT(s, **_radii(6.0))
    with pytest.raises(rt.RTError) as e:
        ctx.kick(0, 0, 0, 1e-3)  # before rt_inverse
    assert e.value.status == rt.RT_ESTATE
    with pytest.raises(rt.RTError) as e:
        ctx.kick(5, 0, 0, 1e-3)
    assert e.value.status == rt.RT_EINVAL
    ctx.close()
