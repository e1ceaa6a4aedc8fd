"""Spectra post-processing (paper Sec. II.B) against the closed-form linear
response of a delta kick.

With H v = e S v (v^T S v = 1), K0 = sum_occ v v^T and the kick
V = exp(+i kappa S^-1 D), to first order in kappa
    Tr(K(t) D) - Tr(K0 D) = 2 kappa sum_{a occ, b virt} |d_ab|^2 sin((e_b - e_a) t),
d_ab = v_a^T D v_b.  Hence Im alpha(w) is a sum of lines at e_b - e_a and the
f-sum int S(w) dw = (1/3) 2 sum_{a occ, b virt} (e_b - e_a) |d_ab|^2 for a kick
along one axis.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sl

import synth
from oracle import dense as od
from paper_1404_5776_gb300 import spectra


@pytest.fixture(scope="module")
def model():
    pos, _ = synth.diamond_positions(1)
    s = synth.build_system(pos, None, ["sp4"] * 8, 20.0, 20.0)  # open 8-atom cluster
    S, H, Dx = s.to_dense("S"), s.to_dense("H"), s.to_dense("Dx")
    w, V = sl.eigh(H, S)
    n_occ = s.n // 2
    d = V.T @ Dx @ V
    a, b = np.meshgrid(np.arange(n_occ), np.arange(n_occ, s.n), indexing="ij")
    wab = (w[b] - w[a]).ravel()
    dab2 = (d[a, b] ** 2).ravel()
    return s, S, H, Dx, w, V, n_occ, wab, dab2


def test_closed_form_matches_propagation(model):
    s, S, H, Dx, w, V, n_occ, wab, dab2 = model
    kappa, dt, n = 1e-5, 0.02, 300
    K0 = V[:, :n_occ] @ V[:, :n_occ].T
    Vk = sl.expm(1j * kappa * np.linalg.solve(S, Dx))
    K = Vk @ K0 @ Vk.conj().T
    U = sl.expm(-1j * dt * np.linalg.solve(S, H))
    p0 = od.trace(K0, Dx).real
    t = dt * np.arange(1, n + 1)
    sim = []
    for _ in range(n):
        K = U @ K @ U.conj().T
        sim.append(od.trace(K, Dx).real - p0)
    closed = 2 * kappa * (dab2[None, :] * np.sin(np.outer(t, wab))).sum(1)
    assert np.abs(np.array(sim) - closed).max() <= 1e-3 * np.abs(closed).max()


def test_f_sum_and_lines(model):
    s, S, H, Dx, w, V, n_occ, wab, dab2 = model
    kappa, dt, T, gamma = 1e-3, 0.02, 400.0, 0.02
    t = dt * np.arange(1, int(T / dt) + 1)
    dP = 2 * kappa * (dab2[None, :] * np.sin(np.outer(t, wab))).sum(1)
    om = np.linspace(0.0, 10.0 * wab.max(), 20000)
    ax = spectra.polarizability(t, dP, kappa, om, damping=gamma)
    Sw = spectra.strength_function(om, [ax, 0 * ax, 0 * ax])
    ref = (1.0 / 3.0) * 2.0 * np.sum(wab * dab2)
    # the Lorentzian tails beyond the grid hold ~3e-3 of the weight
    assert spectra.f_sum(om, Sw) == pytest.approx(ref, rel=1e-2)
    # the main peaks sit at excitation energies e_b - e_a of strong lines
    strong = wab[wab * dab2 > 0.05 * (wab * dab2).max()]
    for pk in spectra.peaks(om, Sw, 4):
        assert np.min(np.abs(strong - pk)) < 2 * gamma


def test_field_denominator_equals_kick_limit():
    """With E given on the grid, alpha = FT[P]/FT[E]; a narrow pulse of area
    kappa gives the same alpha as the kick formula at low frequency."""
    dt = 0.01
    t = dt * np.arange(1, 4001)
    w0 = 0.7
    sig = 0.02
    kappa = 1e-3
    E = kappa / (sig * math.sqrt(2 * math.pi)) * np.exp(-((t - 0.2) ** 2) / (2 * sig ** 2))
    # response of a single line to that pulse (convolution of the kick response)
    resp = np.array([np.sum(E[:k + 1] * np.sin(w0 * (t[k] - t[:k + 1]))) * dt for k in range(len(t))])
    om = np.array([0.3, 0.5])
    a_field = spectra.polarizability(t, resp, None, om, damping=0.01, E=E)
    # the same line kicked at the pulse centre; its transform carries e^{i w 0.2}
    kick = np.sin(w0 * (t - 0.2)) * (t > 0.2) * kappa
    a_kick = spectra.polarizability(t, kick, kappa, om, damping=0.01) * np.exp(-1j * om * 0.2)
    np.testing.assert_allclose(a_field, a_kick, rtol=2e-2)
