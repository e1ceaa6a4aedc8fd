"""Pins for the seeded input generator (Gaussian integrals, geometry, folding)."""
import math

import numpy as np
import pytest

import synth


def _two_atoms(species, sep_ang, direction=(0.3, -0.5, 0.8)):
    d = np.asarray(direction, float)
    d = d / np.linalg.norm(d)
    pos = np.array([[1.0, 2.0, 3.0], [1.0, 2.0, 3.0] + sep_ang * d])
    return synth.build_system(pos, None, species, 20.0, 20.0)


def test_s_s_overlap_closed_form():
    # normalised s Gaussians: S = (2 sqrt(ab)/(a+b))^(3/2) exp(-ab R^2/(a+b))
    sysm = _two_atoms(["sp4", "h1"], 2.0)
    S = sysm.to_dense("S")
    a = synth.SPECIES["sp4"]["shells"][0][1]
    b = synth.SPECIES["h1"]["shells"][0][1]
    R = 2.0 * synth.BOHR_PER_ANG
    ref = (2 * math.sqrt(a * b) / (a + b)) ** 1.5 * math.exp(-a * b * R * R / (a + b))
    assert S[0, 4] == pytest.approx(ref, rel=1e-13)
    assert S[4, 0] == pytest.approx(ref, rel=1e-13)
    np.testing.assert_allclose(np.diag(S), 1.0, rtol=0, atol=1e-14)


def _grid_functions(basis, centre, X, Y, Z):
    """Basis functions evaluated on a grid, each normalised numerically."""
    out = []
    for (l, a) in basis.shells:
        dx, dy, dz = X - centre[0], Y - centre[1], Z - centre[2]
        g = np.exp(-a * (dx * dx + dy * dy + dz * dz))
        if l == 0:
            fs = [g]
        elif l == 1:
            fs = [dx * g, dy * g, dz * g]
        else:
            fs = [dx * dy * g, dx * dz * g, dy * dz * g, (dx * dx - dy * dy) * g,
                  (2 * dz * dz - dx * dx - dy * dy) * g]
        out += fs
    return out


def test_overlap_and_dipole_by_quadrature():
    """p and d overlaps and first moments against a 3D trapezoid quadrature."""
    sep = 2.35
    sysm = _two_atoms(["spd13", "sp4"], sep)
    S = sysm.to_dense("S")
    Dx = sysm.to_dense("Dx")
    Dz = sysm.to_dense("Dz")
    A = sysm.pos[0] * synth.BOHR_PER_ANG
    B = sysm.pos[1] * synth.BOHR_PER_ANG
    h = 0.25
    lo = np.minimum(A, B) - 8.0
    hi = np.maximum(A, B) + 8.0
    ax = [np.arange(lo[d], hi[d] + h, h) for d in range(3)]
    X, Y, Z = np.meshgrid(*ax, indexing="ij")
    fa = _grid_functions(synth.make_basis("spd13"), A, X, Y, Z)
    fb = _grid_functions(synth.make_basis("sp4"), B, X, Y, Z)
    fa = [f / math.sqrt(np.sum(f * f) * h ** 3) for f in fa]
    fb = [f / math.sqrt(np.sum(f * f) * h ** 3) for f in fb]
    F = fa + fb
    n = len(F)
    assert n == S.shape[0] == 17
    Sq = np.array([[np.sum(F[i] * F[j]) * h ** 3 for j in range(n)] for i in range(n)])
    # the quadrature fixes each function's sign; compare magnitudes of the
    # normalised cross overlaps and the exact signs of the same-function pairs
    np.testing.assert_allclose(np.abs(S), np.abs(Sq), atol=2e-7)
    Dxq = np.array([[np.sum(F[i] * X * F[j]) * h ** 3 for j in range(n)] for i in range(n)])
    Dzq = np.array([[np.sum(F[i] * Z * F[j]) * h ** 3 for j in range(n)] for i in range(n)])
    np.testing.assert_allclose(np.abs(Dx), np.abs(Dxq), atol=2e-6)
    np.testing.assert_allclose(np.abs(Dz), np.abs(Dzq), atol=2e-6)
    # signs agree where the values are not tiny (same function ordering and phase)
    big = np.abs(Sq) > 1e-3
    assert np.all(np.sign(S[big]) == np.sign(Sq[big]))


def test_matrices_symmetric_and_gamma_folding(tiny_sp4):
    s = tiny_sp4
    S, H, Dx = s.to_dense("S"), s.to_dense("H"), s.to_dense("Dx")
    assert np.array_equal(S, S.T) and np.array_equal(H, H.T) and np.array_equal(Dx, Dx.T)
    # Gamma-point folding: block (i,j) sums all images of j within r_S
    L = s.cell
    i, j = 0, 5
    tot = np.zeros((4, 4))
    for nx in (-1, 0, 1):
        for ny in (-1, 0, 1):
            for nz in (-1, 0, 1):
                dvec = s.pos[j] + np.array([nx, ny, nz]) * L - s.pos[i]
                d2 = (dvec[0] * dvec[0] + dvec[1] * dvec[1]) + dvec[2] * dvec[2]
                if d2 < 6.0 * 6.0:
                    two = synth.build_system(np.array([s.pos[i], s.pos[i] + dvec]), None,
                                             ["sp4", "sp4"], 20.0, 20.0)
                    tot += two.to_dense("S")[0:4, 4:8]
    np.testing.assert_allclose(S[0:4, 20:24], tot, atol=1e-15)


def test_model_checks(tiny_sp4):
    """S is SPD and well conditioned; gap at half filling; dt * spectral radius small."""
    S = tiny_sp4.to_dense("S")
    w = np.linalg.eigvalsh(S)
    assert w.min() > 0 and w.max() / w.min() < 1e4
    K0, e, gap = synth.ground_state_dense(tiny_sp4, tiny_sp4.n // 2)
    assert gap > 0.05
    assert 0.05 * np.abs(e).max() <= 0.3
    assert np.trace(K0 @ S) == pytest.approx(tiny_sp4.n // 2, abs=1e-10)


def test_positions_seeded_and_wrapped():
    p1, c = synth.diamond_positions(2, seed=0)
    p2, _ = synth.diamond_positions(2, seed=0)
    assert np.array_equal(p1, p2)
    assert np.all(p1 >= 0) and np.all(p1 < c)
    assert len(p1) == 64
