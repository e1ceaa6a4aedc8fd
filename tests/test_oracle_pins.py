"""Pins of the CPU oracle to what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks it against a
closed form, a library routine for a special case, an invariant, or a
brute-force restatement on tiny inputs.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sl

import oracle
import synth
from oracle import dense as od

BIG = 30.0  # larger than the tiny cell's diagonal: nothing is truncated


def _prop(sys, prop="em", r=BIG, dt=0.05, terms=6, **kw):
    p = oracle.Params(r_Sinv=r, r_T=r, r_U=r, r_K=r, r_M=r, dt=dt, prop=prop, taylor_terms=terms, **kw)
    return oracle.Propagator(sys, p)


# --------------------------------------------------------------------------
# patterns
# --------------------------------------------------------------------------

def _pattern_by_images(pos, cell, r):
    """Independent restatement: minimum over the 27 explicit images."""
    n = len(pos)
    d = pos[None, :, :] - pos[:, None, :]
    best = np.full((n, n), np.inf)
    for nx in (-1, 0, 1):
        for ny in (-1, 0, 1):
            for nz in (-1, 0, 1):
                dd = d + np.array([nx, ny, nz]) * cell
                best = np.minimum(best, (dd ** 2).sum(-1))
    return best


@pytest.mark.parametrize("r", [3.0, 6.0, 8.0])
def test_pattern_matches_explicit_images(tiny_sp4, r):
    s = tiny_sp4
    P = oracle.pattern(s.pos, s.cell, r)
    d2 = _pattern_by_images(s.pos, s.cell, r)
    # no near-ties for these radii (jittered lattice)
    assert np.min(np.abs(d2 - r * r)) > 1e-6
    ref = d2 < r * r
    got = np.zeros_like(ref)
    got[P.rows(), P.col] = True
    assert np.array_equal(got, ref)
    assert np.array_equal(got, got.T)
    assert all(np.all(np.diff(P.col[P.rowptr[i]:P.rowptr[i + 1]]) > 0) for i in range(s.n_atoms))


def test_pattern_dense_at_large_radius_and_counts(tiny_sp4):
    s = tiny_sp4
    P = oracle.pattern(s.pos, s.cell, BIG)
    assert P.nnzb == s.n_atoms ** 2
    # 64-atom cell at 6 A: 42.25 blocks per atom (includes the diagonal)
    assert oracle.pattern(s.pos, s.cell, 6.0).nnzb / 64 == pytest.approx(42.25)
    # open system: plain Euclidean distance
    pos = np.array([[0.0, 0, 0], [1.0, 0, 0], [2.5, 0, 0]])
    Q = oracle.pattern(pos, None, 1.6)
    assert list(Q.rowptr) == [0, 2, 5, 7] and list(Q.col) == [0, 1, 0, 1, 2, 1, 2]


# --------------------------------------------------------------------------
# truncated product against dense masked products (brute force)
# --------------------------------------------------------------------------

def _random_block(bsize, pat, rng, cplx=True):
    M = oracle.zeros(bsize, pat)
    M.val = rng.standard_normal(len(M.val)) + (1j * rng.standard_normal(len(M.val)) if cplx else 0)
    return M


@pytest.mark.parametrize("a_dag,b_dag", [(False, False), (False, True), (True, False), (True, True)])
def test_spgemm_matches_masked_dense(a_dag, b_dag):
    rng = np.random.default_rng(5)
    pos = rng.uniform(0, 9.0, size=(14, 3))
    cell = np.array([9.0, 9.0, 9.0])
    bsize = np.array([1, 4, 13, 4, 1, 13, 4, 4, 1, 13, 4, 1, 4, 13], dtype=np.int32)
    PA, PB, PC = (oracle.pattern(pos, cell, r) for r in (4.0, 5.0, 4.5))
    A = _random_block(bsize, PA, rng)
    B = _random_block(bsize, PB, rng)
    C = oracle.spgemm(A, B, PC, a_dag=a_dag, b_dag=b_dag)
    Ad, Bd = A.to_dense(), B.to_dense()
    Ad = Ad.conj().T if a_dag else Ad
    Bd = Bd.conj().T if b_dag else Bd
    ref = od.cut(Ad @ Bd, od.atom_mask(bsize, PC))
    np.testing.assert_allclose(C.to_dense(), ref, atol=1e-12, rtol=0)


def test_spgemm_upper_only_and_row_range():
    rng = np.random.default_rng(6)
    pos = rng.uniform(0, 8.0, size=(10, 3))
    bsize = np.full(10, 4, dtype=np.int32)
    P = oracle.pattern(pos, None, 5.0)
    A, B = _random_block(bsize, P, rng), _random_block(bsize, P, rng)
    full = oracle.spgemm(A, B, P)
    up = oracle.spgemm(A, B, P, upper_only=True)
    rows = P.rows()
    for q in range(P.nnzb):
        blk = slice(up.voff[q], up.voff[q + 1])
        if P.col[q] >= rows[q]:
            np.testing.assert_array_equal(up.val[blk], full.val[blk])
        else:
            assert np.all(up.val[blk] == 0)
    part = oracle.spgemm(A, B, P, rows=(3, 7))
    for q in range(P.nnzb):
        blk = slice(part.voff[q], part.voff[q + 1])
        if 3 <= rows[q] < 7:
            np.testing.assert_array_equal(part.val[blk], full.val[blk])
        else:
            assert np.all(part.val[blk] == 0)


# --------------------------------------------------------------------------
# Hotelling (Sec. V.A)
# --------------------------------------------------------------------------

def test_hotelling_matches_lu_inverse(tiny_spd13):
    s = tiny_spd13
    S = oracle.BlockMatrix(s.bsize, oracle.Pattern(s.s_rowptr, s.s_col), s.s_val)
    res = oracle.hotelling(S, oracle.pattern(s.pos, s.cell, BIG), tol=1e-13)
    assert res.status == "converged"
    Sinv = np.linalg.inv(s.to_dense("S"))
    np.testing.assert_allclose(res.X.to_dense(), Sinv, atol=1e-11 * np.abs(Sinv).max())
    # untruncated: R_{k+1} = R_k^2 for R = I - S X, so ||R_{k+1}||_F <= ||R_k||_F^2,
    # i.e. h_{k+1} <= sqrt(n) h_k^2 for the normalised residuals h
    h = res.history
    n = s.n
    assert h[-1] < 1e-13
    for a, b in zip(h[:-1], h[1:]):
        assert b <= math.sqrt(n) * a * a * (1 + 1e-9) + 1e-14


def test_hotelling_scalar_block():
    """b = 1, one atom: X -> 1/s."""
    P = oracle.Pattern(np.array([0, 1], np.int32), np.array([0], np.int32))
    S = oracle.BlockMatrix(np.array([1], np.int32), P, np.array([2.5]))
    res = oracle.hotelling(S, P, tol=1e-15, maxit=60)
    assert res.X.val[0] == pytest.approx(0.4, rel=1e-15)
    # from X0 = 1/||S|| = 0.4 the answer is exact at once
    S2 = oracle.BlockMatrix(np.array([1, 1], np.int32),
                            oracle.Pattern(np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32)),
                            np.array([2.0, 0.5, 0.5, 1.0]))
    r2 = oracle.hotelling(S2, S2.pat, tol=1e-15, maxit=80)
    np.testing.assert_allclose(r2.X.to_dense(), np.linalg.inv([[2.0, 0.5], [0.5, 1.0]]), atol=1e-15)


# --------------------------------------------------------------------------
# closed forms for time-independent H (untruncated)
# --------------------------------------------------------------------------

def _closed_form_run(sys, K0, g, m):
    """K(m) from the generalised eigenpairs: K~ = V^T S K S V evolves as
    K~_ab(m) = g_a^m conj(g_b)^m K~_ab(0)."""
    S, H = sys.to_dense("S"), sys.to_dense("H")
    w, V = sl.eigh(H, S)
    Kt = V.T @ S @ K0 @ S @ V
    G = g(w) ** m
    Kt_m = (G[:, None] * np.conj(G)[None, :]) * Kt
    Vinv = V.T @ S  # V^T S V = I
    Vi = np.linalg.inv(Vinv)
    return Vi @ Kt_m @ Vi.T


def _kicked_density(sys, kappa=1e-3):
    K0, _, _ = synth.ground_state_dense(sys, sys.n // 2)
    S, Dx = sys.to_dense("S"), sys.to_dense("Dx")
    V = sl.expm(1j * kappa * np.linalg.solve(S, Dx))
    return V @ K0 @ V.conj().T


@pytest.mark.parametrize("prop", ["em", "cn"])
def test_step_matches_eigenpair_closed_form(tiny_sp4, prop):
    s, dt, m = tiny_sp4, 0.05, 12
    K1 = _kicked_density(s)
    if prop == "em":
        g = lambda e: sum((-1j * dt * e) ** n / math.factorial(n) for n in range(6))
    else:
        g = lambda e: (1 - 0.5j * dt * e) / (1 + 0.5j * dt * e)
    ref = _closed_form_run(s, K1, g, m)
    pr = _prop(s, prop, dt=dt, hot_step_iters=3)
    pr.K = oracle.from_dense(s.bsize, pr.pats["K"], K1)
    for _ in range(m):
        pr.step()
    np.testing.assert_allclose(pr.K.to_dense(), ref, atol=1e-11, rtol=0)
    # and the dense mode of the oracle agrees with the same closed form
    S, H = s.to_dense("S"), s.to_dense("H")
    U = od.em_propagator(np.linalg.inv(S), H, dt) if prop == "em" else od.cn_propagator_exact(S, H, dt)
    Kd = K1
    for _ in range(m):
        Kd = U @ Kd @ U.conj().T
    np.testing.assert_allclose(Kd, ref, atol=1e-11, rtol=0)


def test_orthogonal_basis_reduces_to_expm():
    """S = I: many Taylor terms give exp(-i H dt) (scipy.linalg.expm)."""
    rng = np.random.default_rng(3)
    n_at = 6
    bsize = np.full(n_at, 4, np.int32)
    P = oracle.pattern(rng.uniform(0, 5, (n_at, 3)), None, 100.0)
    Hd = rng.standard_normal((24, 24))
    Hd = 0.5 * (Hd + Hd.T)
    H = oracle.from_dense(bsize, P, Hd)
    I = oracle.identity(bsize, P)
    U, _ = oracle.taylor_em(oracle.spgemm(I, H, P), 0.05, 30, P)
    np.testing.assert_allclose(U.to_dense(), sl.expm(-0.05j * Hd), atol=1e-14)
    # six terms: the truncated exponential series exactly
    U6, _ = oracle.taylor_em(H, 0.05, 6, P)
    ref6 = sum(np.linalg.matrix_power(-0.05j * Hd, k) / math.factorial(k) for k in range(6))
    np.testing.assert_allclose(U6.to_dense(), ref6, atol=1e-15)


def test_unitarity_closed_forms(tiny_sp4):
    """CN: U^dagger S U = S to rounding.  EM-6: U^dagger S U - S = V^-T (|g|^2 - 1) V^-1."""
    s, dt = tiny_sp4, 0.05
    S, H = s.to_dense("S"), s.to_dense("H")
    w, V = sl.eigh(H, S)
    prc = _prop(s, "cn", dt=dt, hot_step_iters=4)
    Uc, _ = prc.propagator(0.0)
    pw = prc.pats["U"]
    mx, _ = oracle.unitarity(Uc, prc.S, pw)
    assert mx < 1e-13
    pre = _prop(s, "em", dt=dt)
    Ue, _ = pre.propagator(0.0)
    mx_e, _ = oracle.unitarity(Ue, pre.S, pw)
    g = sum((-1j * dt * w) ** n / math.factorial(n) for n in range(6))
    Vinv = V.T @ S
    E = Vinv.T @ np.diag(np.abs(g) ** 2 - 1) @ Vinv
    assert mx_e == pytest.approx(np.abs(E).max(), rel=1e-6)
    # per eigenpair |g|^2 - 1 ~ y^6/360 (y = dt e) for small y
    y = dt * w
    np.testing.assert_allclose(np.abs(g) ** 2 - 1, y ** 6 / 360, rtol=0.05, atol=1e-15)


def test_invariants_cn_truncated(tiny_spd13):
    """Truncated CN: K stays hermitian, Tr(KS) starts at N_occ and drifts little."""
    s = tiny_spd13
    n_occ = 2 * s.n_atoms
    K0, _, _ = synth.ground_state_dense(s, n_occ)
    pr = _prop(s, "cn", r=7.0, dt=0.05, hot_step_iters=2)
    pr.set_density_dense(K0)
    q0 = oracle.observables(pr.K, pr.S, pr.D)[0]
    pr.kick(0, 1e-3)
    for _ in range(3):
        out = pr.step()
    Kd = pr.K.to_dense()
    assert np.abs(Kd - Kd.conj().T).max() == 0.0
    assert abs(out["obs"][0].imag) < 1e-12
    assert abs(out["obs"][0].real - q0.real) < 1e-2 * n_occ


def test_charge_dipole_and_kick(tiny_sp4):
    s = tiny_sp4
    K0, _, _ = synth.ground_state_dense(s, s.n // 2)
    pr = _prop(s, "em")
    pr.set_density_dense(K0)
    q, px = oracle.observables(pr.K, pr.S, pr.D)[:2]
    assert q.real == pytest.approx(s.n // 2, abs=1e-10) and abs(q.imag) < 1e-14
    # kick with kappa -> 0 is the identity
    pr.kick(0, 0.0)
    np.testing.assert_array_equal(pr.K.to_dense(), oracle.from_dense(s.bsize, pr.pats["K"], K0).to_dense())
    # the induced dipole is linear in kappa: ratio 2 for kappa and 2 kappa
    resp = []
    for kap in (1e-4, 2e-4):
        pk = _prop(s, "em")
        pk.set_density_dense(K0)
        pk.kick(0, kap)
        for _ in range(10):
            o = pk.step()
        resp.append(o["obs"][1].real - px.real)
    assert resp[1] / resp[0] == pytest.approx(2.0, rel=1e-3)


def test_kick_matches_expm(tiny_sp4):
    s = tiny_sp4
    K0, _, _ = synth.ground_state_dense(s, s.n // 2)
    pr = _prop(s, "em")
    pr.set_density_dense(K0)
    pr.kick(1, 5e-3)
    S, Dy = s.to_dense("S"), s.to_dense("Dy")
    V = sl.expm(5e-3j * np.linalg.solve(S, Dy))
    np.testing.assert_allclose(pr.K.to_dense(), V @ K0 @ V.conj().T, atol=1e-13)


def test_foe_matches_fermi_dirac(tiny_sp4):
    """Chebyshev FOE against the exact Fermi-Dirac density from eigh."""
    s = tiny_sp4
    S, H = s.to_dense("S"), s.to_dense("H")
    w = sl.eigh(H, S, eigvals_only=True)
    mu = 0.5 * (w[s.n // 2 - 1] + w[s.n // 2])
    pr = _prop(s, "em")
    lo, hi = w.min() - 0.05, w.max() + 0.05
    pr.ground_state(200, mu, 0.05, lo, hi)
    ref = od.fermi_dense(H, S, mu, 0.05)
    np.testing.assert_allclose(pr.K.to_dense().real, ref, atol=1e-9)
    # idempotency K S K = K at small kT (gapped): max deviation small
    pr.ground_state(400, mu, 0.004, lo, hi)
    K = pr.K.to_dense().real
    assert np.abs(K @ S @ K - K).max() < 5e-3
    assert np.trace(K @ S) == pytest.approx(s.n // 2, abs=0.05)


# --------------------------------------------------------------------------
# the truncated step against a dense masked restatement
# --------------------------------------------------------------------------

@pytest.mark.parametrize("prop", ["em", "cn"])
def test_truncated_step_matches_masked_dense(tiny_spd13, prop):
    s = tiny_spd13
    r = 6.0
    dt = 0.05
    pr = _prop(s, prop, r=r, dt=dt, hot_step_iters=2, hot_tol=0.0, hot_maxit=12)
    K0, _, _ = synth.ground_state_dense(s, 2 * s.n_atoms)
    pr.set_density_dense(K0)
    mK = od.atom_mask(s.bsize, pr.pats["K"])
    S, H = s.to_dense("S"), s.to_dense("H")
    # dense restatement with masks (Hotelling: same fixed iteration count)
    mS = od.atom_mask(s.bsize, pr.pats["Sinv"])
    Xd, k, _ = od.hotelling(S, iters=pr.hot.iters, mask=mS)
    np.testing.assert_allclose(pr.Sinv.to_dense(), Xd, atol=1e-13)
    Kd = od.cut(K0.astype(complex), mK)
    up = od.upper_block_mask(s.bsize) & mK
    Xcn = Xd.astype(complex)
    for _ in range(2):
        pr.step()
        if prop == "em":
            U = od.em_propagator(Xd, H, dt, 6, mK, mK)
        else:
            U, Xcn, _ = od.cn_propagator_hotelling(S, H, dt, Xcn, 2, mK)
        Kd = od.sandwich(U, Kd, mK, mK, up)
    np.testing.assert_allclose(pr.K.to_dense(), Kd, atol=1e-12)
