"""Pins (CPU, FP64) for the algebraic reformulations the CUDA path uses on top
of the paper's step, each restated here with the oracle's truncated products
and compared with the literal computation:

* T(E) = cut(S^-1 (H0 - E D)) = cut(S^-1 H0) - E cut(S^-1 D)    (the FP32 EM path)
* delta-form sandwich: with dU = U - I, M = cut_M(dU K), W = K + M,
  K' = K + M + cut_K(W dU^dagger)  equals  cut_K(cut_M(U K) U^dagger)   (r_M >= r_K)
* incremental form: sandwich(K_ref + dK) = K_ref + R + dK + M + N with
  R = sandwich(K_ref) - K_ref, M = cut(dU dK), N = cut((dK + M) dU^dagger)
* field polynomial: U(E) = sum_m E^m V_m with V_m = sum_n c_n Q_{n,m},
  Q_{1,0} = T0, Q_{1,1} = -T_D, Q_{n,m} = cut(T0 Q_{n-1,m}) + cut(Q_{1,1} Q_{n-1,m-1}),
  equals the literal truncated series of T(E) at every E.
* reference split with the field polynomial: with U(E) = sum_m E^m V_m,
  sym(cut_K(cut_M(U(E) K_ref) U(E)^dagger)) = sum_p E^p B_p,
  B_p = sum_{m+m'=p} sym(cut_K(cut_M(V_m K_ref) V_m'^dagger)), at every E.
* ETRS in the delta form (the mixed path): with dU_a = exp(-i dt/2 T(t)) - I,
  dU_b = exp(-i dt/2 T(t+dt)) - I and T(t) = T0 - E(t) T_D,
  I + dU_a + dU_b + cut(dU_b dU_a)  equals  cut(U_b U_a)  from cut(S^-1 H(t)).
* M4 in the delta form (the mixed path): Om from T1, T2 = T0 - E(t_{1,2}) T_D,
  I + sum_{n>=1} Om^n / n!  equals the literal M4 propagator from cut(S^-1 H(t_{1,2})).
The hermitian mirroring of K' (upper blocks computed, lower mirrored) is the
same on both sides and is applied to both."""
import math

import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def setup():
    s = synth.diamond_system(2, "sp4", 6.0, 6.0)
    pats = {r: oracle.pattern(s.pos, s.cell, r) for r in (4.0, 5.0, 6.0, 7.0)}
    S = oracle.BlockMatrix(s.bsize, oracle.Pattern(s.s_rowptr, s.s_col), s.s_val)
    hp = oracle.Pattern(s.h_rowptr, s.h_col)
    H0 = oracle.BlockMatrix(s.bsize, hp, s.h_val)
    D = oracle.BlockMatrix(s.bsize, hp, s.d_val[0])
    Sinv = oracle.hotelling(S, pats[6.0], 1e-12, 100).X
    K0, _, _ = synth.ground_state_dense(s, s.n // 2)
    return s, pats, S, H0, D, Sinv, K0


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_T_is_linear_in_the_field(setup):
    s, pats, S, H0, D, Sinv, _ = setup
    pT = pats[5.0]
    T0 = oracle.spgemm(Sinv, H0, pT)
    TD = oracle.spgemm(Sinv, D, pT)
    for E in (1e-3, -0.05):
        TE = oracle.spgemm(Sinv, oracle.hamiltonian(H0, D, E), pT)
        assert rel(TE.val, T0.val - E * TD.val) < 1e-13


def _sandwich_direct(U, K, pM, pK):
    Kn, _ = oracle.sandwich(U, K, pM)
    assert Kn.pat is pK or np.array_equal(Kn.pat.col, pK.col)
    return Kn


def _delta_sandwich(dU, K, pM, pK):
    M = oracle.spgemm(dU, K, pM)
    W = oracle.axpy(1.0, K, M)                      # K + M on P_M
    Kn = oracle.axpy(1.0, M, K.copy())              # K + M on P_K
    oracle.spgemm(W, dU, pK, b_dag=True, upper_only=True, out=(X := oracle.zeros(K.bsize, pK)))
    up = oracle.BlockMatrix(K.bsize, pK, Kn.val + X.val, Kn.voff)
    oracle.mirror_upper(up)
    return up


def _propagator(setup, r_T, r_U, dt=0.05, terms=6):
    s, pats, S, H0, D, Sinv, _ = setup
    T = oracle.spgemm(Sinv, H0, pats[r_T])
    U, _ = oracle.taylor_em(T, dt, terms, pats[r_U])
    return U


@pytest.mark.parametrize("r_K,r_M", [(5.0, 5.0), (5.0, 7.0), (6.0, 6.0)])
def test_delta_form_equals_direct_sandwich(setup, r_K, r_M):
    s, pats, *_ , K0 = setup
    U = _propagator(setup, 5.0, 6.0)
    pK, pM = pats[r_K], pats[r_M]
    K = oracle.from_dense(s.bsize, pK, K0.astype(complex))
    dU = oracle.axpy(-1.0, oracle.identity(s.bsize, U.pat), U)
    direct = _sandwich_direct(U, K, pM, pK)
    delta = _delta_sandwich(dU, K, pM, pK)
    assert rel(delta.val, direct.val) < 1e-13


def test_incremental_form_equals_direct_sandwich(setup):
    s, pats, *_, K0 = setup
    U = _propagator(setup, 5.0, 6.0)
    pK = pM = pats[6.0]
    dU = oracle.axpy(-1.0, oracle.identity(s.bsize, U.pat), U)
    K_ref = oracle.from_dense(s.bsize, pK, K0.astype(complex))
    rng = np.random.default_rng(3)
    dK = oracle.BlockMatrix(s.bsize, pK, 1e-3 * (rng.standard_normal(K_ref.val.shape)
                                                 + 1j * rng.standard_normal(K_ref.val.shape)))
    oracle.mirror_upper(dK)  # hermitian perturbation
    K = oracle.axpy(1.0, dK, K_ref.copy())
    direct = _sandwich_direct(U, K, pM, pK)
    R = oracle.axpy(-1.0, K_ref, _sandwich_direct(U, K_ref, pM, pK))
    d_new = _delta_sandwich(dU, dK, pM, pK)          # dK + M + N
    incr = oracle.axpy(1.0, R, oracle.axpy(1.0, K_ref, d_new))
    assert rel(incr.val, direct.val) < 1e-13


def _field_poly_V(setup, terms, pT, pU, dt=0.05):
    """V_m of U(E) = sum_m E^m V_m, formed from the oracle's truncated products."""
    s, pats, S, H0, D, Sinv, _ = setup
    T0 = oracle.spgemm(Sinv, H0, pT)
    Q1 = [T0, oracle.BlockMatrix(s.bsize, pT, -oracle.spgemm(Sinv, D, pT).val)]
    deg = terms - 1
    V = [oracle.identity(s.bsize, pU)] + [oracle.zeros(s.bsize, pU) for _ in range(deg)]

    def coef(n):
        return (-1j * dt) ** n / math.factorial(n)

    for m in range(min(deg, 1) + 1):
        if deg >= 1:
            V[m] = oracle.axpy(coef(1), oracle.restrict(Q1[m], pU), V[m])
    prev = Q1
    for n in range(2, deg + 1):
        cur = []
        for m in range(n + 1):
            acc = oracle.zeros(s.bsize, pU)
            if m <= n - 1:
                acc = oracle.axpy(1.0, oracle.spgemm(Q1[0], prev[m], pU), acc)
            if m >= 1:
                acc = oracle.axpy(1.0, oracle.spgemm(Q1[1], prev[m - 1], pU), acc)
            cur.append(acc)
            V[m] = oracle.axpy(coef(n), acc, V[m])
        prev = cur
    return V


def _horner(coeffs, E):
    v = coeffs[-1].val.copy()
    for c in coeffs[-2::-1]:
        v = v * E + c.val
    return v


@pytest.mark.parametrize("terms", [2, 6, 7])
def test_field_polynomial_equals_literal_series(setup, terms):
    s, pats, S, H0, D, Sinv, _ = setup
    pT, pU = pats[4.0], pats[6.0]
    dt = 0.05
    V = _field_poly_V(setup, terms, pT, pU, dt)
    for E in (0.0, 2e-3, -0.03):
        poly = _horner(V, E)
        TE = oracle.spgemm(Sinv, oracle.hamiltonian(H0, D, E), pT)
        U_lit, _ = oracle.taylor_em(TE, dt, terms, pU)
        assert rel(poly, U_lit.val) < 1e-12, (terms, E)


@pytest.mark.parametrize("r_K,r_M", [(5.0, 5.0), (5.0, 7.0)])
def test_reference_part_is_a_polynomial_in_the_field(setup, r_K, r_M):
    """The FP64 part of the reference split for a field-dependent propagator:
    the literal sandwich of K_ref with U(E) from the truncated series of
    T(E) = cut(S^-1 (H0 - E D)) equals sum_p E^p B_p with the B_p formed once
    from the V_m (every cut is linear)."""
    s, pats, S, H0, D, Sinv, K0 = setup
    pT, pU, pK, pM = pats[5.0], pats[6.0], pats[r_K], pats[r_M]
    dt, terms = 0.05, 6
    deg = terms - 1
    V = _field_poly_V(setup, terms, pT, pU, dt)
    K_ref = oracle.from_dense(s.bsize, pK, K0.astype(complex))
    A = [oracle.spgemm(Vm, K_ref, pM) for Vm in V]
    Bp = [oracle.zeros(s.bsize, pK) for _ in range(2 * deg + 1)]
    cross_only = oracle.zeros(s.bsize, pK)
    for m in range(deg + 1):
        for m2 in range(deg + 1):
            X = oracle.zeros(s.bsize, pK)
            oracle.spgemm(A[m], V[m2], pK, b_dag=True, upper_only=True, out=X)
            oracle.mirror_upper(X)
            Bp[m + m2] = oracle.axpy(1.0, X, Bp[m + m2])
            if m != m2 and m + m2 == 1:
                cross_only = oracle.axpy(1.0, X, cross_only)
    for E in (0.0, 4e-3, -0.05):
        TE = oracle.spgemm(Sinv, oracle.hamiltonian(H0, D, E), pT)
        U_lit, _ = oracle.taylor_em(TE, dt, terms, pU)
        direct = _sandwich_direct(U_lit, K_ref, pM, pK)
        assert rel(_horner(Bp, E), direct.val) < 1e-12, E
        if E != 0.0:  # the first-order cross terms carry the field's effect: dropping them is visible
            assert rel(_horner(Bp, E) - E * cross_only.val, direct.val) > 1e-6


PULSE = {"kind": "gaussian", "E0": 0.02, "t0": 0.1, "sigma": 0.2, "omega": 1.1}


def _field_split(ref):
    T0 = oracle.spgemm(ref.Sinv, ref.H0, ref.pats["T"])
    TD = oracle.spgemm(ref.Sinv, ref.D[ref.p.field_dir], ref.pats["T"])
    return T0, TD


def _T_of(T0, TD, E):
    return oracle.BlockMatrix(T0.bsize, T0.pat, T0.val - E * TD.val, T0.voff)


@pytest.mark.parametrize("r_T,r_U", [(5.0, 7.0), (7.0, 5.0)])
def test_etrs_delta_form_equals_literal(setup, r_T, r_U):
    s = setup[0]
    p = oracle.Params(prop="etrs", r_Sinv=6.0, r_T=r_T, r_U=r_U, r_K=6.0, r_M=6.0, field=PULSE, field_dir=1)
    ref = oracle.Propagator(s, p)
    T0, TD = _field_split(ref)
    pU = ref.pats["U"]
    I = oracle.identity(s.bsize, pU)
    for t in (0.0, 0.15):
        Ua, _ = oracle.taylor_em(_T_of(T0, TD, oracle.field_value(PULSE, t)), 0.5 * p.dt, p.taylor_terms, pU)
        Ub, _ = oracle.taylor_em(_T_of(T0, TD, oracle.field_value(PULSE, t + p.dt)), 0.5 * p.dt, p.taylor_terms, pU)
        dUa = oracle.axpy(-1.0, I, Ua)
        dUb = oracle.axpy(-1.0, I, Ub)
        delta = oracle.axpy(1.0, oracle.spgemm(dUb, dUa, pU), oracle.axpy(1.0, dUb, oracle.axpy(1.0, dUa, I)))
        U_lit, _ = ref.propagator(t)
        assert rel(delta.val, U_lit.val) < 1e-13, t
        # the correction term is second order in dt: dropping it is visible
        assert rel(oracle.axpy(1.0, dUb, oracle.axpy(1.0, dUa, I)).val, U_lit.val) > 1e-6


@pytest.mark.parametrize("r_T,r_U", [(5.0, 7.0), (7.0, 5.0)])
def test_m4_delta_form_equals_literal(setup, r_T, r_U):
    s = setup[0]
    p = oracle.Params(prop="m4", r_Sinv=6.0, r_T=r_T, r_U=r_U, r_K=6.0, r_M=6.0, field=PULSE, field_dir=2)
    ref = oracle.Propagator(s, p)
    T0, TD = _field_split(ref)
    pU = ref.pats["U"]
    r3 = math.sqrt(3.0)
    for t in (0.0, 0.15):
        T1 = _T_of(T0, TD, oracle.field_value(PULSE, t + (0.5 - r3 / 6.0) * p.dt))
        T2 = _T_of(T0, TD, oracle.field_value(PULSE, t + (0.5 + r3 / 6.0) * p.dt))
        C21 = oracle.spgemm(T2, T1, pU)
        C12 = oracle.spgemm(T1, T2, pU)
        tsum = oracle.axpy(1.0, oracle.restrict(T2, pU), oracle.restrict(T1, pU))
        Om = oracle.BlockMatrix(s.bsize, pU, -0.5j * p.dt * tsum.val
                                - (r3 * p.dt * p.dt / 12.0) * (C21.val - C12.val), tsum.voff)
        dU = Om.copy()
        P = Om
        for n in range(2, p.taylor_terms):
            P = oracle.spgemm(Om, P, pU)
            dU = oracle.axpy(1.0 / math.factorial(n), P, dU)
        U_lit, _ = ref.propagator(t)
        I = oracle.identity(s.bsize, pU)
        assert rel(oracle.axpy(1.0, I, dU).val, U_lit.val) < 1e-13, t
