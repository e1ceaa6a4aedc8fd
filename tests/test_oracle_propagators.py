"""Pins of the ETRS and fourth-order Magnus propagators of the oracle (Sec. II.A).

* Time-independent H: ETRS is two half-step Taylor exponentials, per
  generalised eigenpair g(e) = [sum_{n<6} (-i dt/2 e)^n / n!]^2; M4 reduces to
  exactly the EM propagator (the commutator vanishes, M = -i dt T).
* Time-dependent H: the global error at a fixed final time falls as dt^2 for
  EM and ETRS and as dt^4 for M4 (Taylor series long enough to be exact).
"""
import math

import numpy as np
import pytest
import scipy.linalg as sl

import oracle
import synth


def _prop(sys, prop, dt=0.05, terms=6, field=None, r=30.0):
    p = oracle.Params(r_Sinv=r, r_T=r, r_U=r, r_K=r, r_M=r, dt=dt, prop=prop, taylor_terms=terms, field=field)
    return oracle.Propagator(sys, p)


def test_etrs_closed_form(tiny_sp4):
    s, dt = tiny_sp4, 0.05
    S, H = s.to_dense("S"), s.to_dense("H")
    w, V = sl.eigh(H, S)
    g = sum((-0.5j * dt * w) ** n / math.factorial(n) for n in range(6)) ** 2
    U_ref = V @ np.diag(g) @ V.T @ S  # U = V G V^-1, V^-1 = V^T S
    pr = _prop(s, "etrs", dt)
    U, _ = pr.propagator(0.0)
    np.testing.assert_allclose(U.to_dense(), U_ref, atol=1e-12)


def test_m4_equals_em_for_static_h(tiny_sp4):
    em = _prop(tiny_sp4, "em")
    m4 = _prop(tiny_sp4, "m4")
    Ue, _ = em.propagator(0.0)
    Um, _ = m4.propagator(0.0)
    np.testing.assert_allclose(Um.to_dense(), Ue.to_dense(), atol=1e-14)


def _open_cluster():
    pos, _ = synth.diamond_positions(1)
    return synth.build_system(pos, None, ["sp4"] * 8, 20.0, 20.0)


def _final_density(sys, prop, dt, T, field):
    pr = _prop(sys, prop, dt=dt, terms=16, field=field)
    K0, _, _ = synth.ground_state_dense(sys, sys.n // 2)
    pr.set_density_dense(K0)
    for _ in range(int(round(T / dt))):
        pr.step()
    return pr.K.to_dense()


def test_convergence_orders():
    s = _open_cluster()
    field = {"kind": "gaussian", "E0": 0.05, "t0": 0.6, "sigma": 0.25, "omega": 2.0}
    T = 1.2
    ref = _final_density(s, "m4", 0.0125, T, field)
    orders = {}
    for prop in ("em", "etrs", "m4"):
        e1 = np.abs(_final_density(s, prop, 0.1, T, field) - ref).max()
        e2 = np.abs(_final_density(s, prop, 0.05, T, field) - ref).max()
        orders[prop] = math.log2(e1 / e2)
    assert 1.6 < orders["em"] < 2.5
    assert 1.6 < orders["etrs"] < 2.5
    assert orders["m4"] > 3.4
