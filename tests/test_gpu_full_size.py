"""Parity at the benchmark's size (4096 atoms x 13 functions), on sampled
outputs the oracle computes row by row.

Sandwich (r = 8 A): the library builds U and steps a seeded hermitian K once;
the oracle recomputes sampled rows of M = cut(U K) and of the upper blocks of
K' = cut(M U^dagger) from the library's own U and K (its truncated product
restricted to those rows), and the two are compared block by block.  FP64 at
1e-10 relative; the mixed path (FP32 block products in the delta form) at
1e-6 of the largest block entry of the sampled rows.

Taylor powers (r = 8 and 10 A, the radius the benchmark headlines): from the
library's own T = cut(S^-1 H), the oracle forms the full truncated powers
T^2, T^3, T^4 and sampled rows of T^5 and of U = sum_n (-i dt)^n T^n / n!
(eq. matrix_exp, six terms); the library's U on those rows is compared with
them, U - I at 1e-10 of its largest entry in FP64, and at 1e-6 in the literal
mixed path, whose powers are the FP32 real block products (k_gemm13_r32)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

R = 8.0
SAMPLE = (0, 777, 2048, 4095)


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1404_5776_gb300 as m
    m.build()
    return m


@pytest.fixture(scope="module")
def workload():
    s = synth.diamond_system(8, "spd13", 7.0, 7.0)
    pat = oracle.pattern(s.pos, s.cell, R)
    # a seeded hermitian K on P_K: upper blocks random, lower blocks their adjoints
    rng = np.random.default_rng(7)
    n = s.n_atoms
    rows = pat.rows().astype(np.int64)
    cols = pat.col.astype(np.int64)
    keys = rows * n + cols                      # ascending (block-CSR order)
    tq = np.searchsorted(keys, cols * n + rows)  # index of the transposed block
    vals = (rng.standard_normal((pat.nnzb, 13, 13)) + 1j * rng.standard_normal((pat.nnzb, 13, 13))) * 1e-2
    diag = rows == cols
    vals[diag] = 0.5 * (vals[diag] + np.conj(np.transpose(vals[diag], (0, 2, 1))))
    lower = rows > cols
    vals[lower] = np.conj(np.transpose(vals[tq[lower]], (0, 2, 1)))
    Kb = oracle.BlockMatrix(s.bsize, pat, vals.reshape(-1))
    return s, pat, Kb


@pytest.fixture(scope="module")
def cell4096():
    return synth.diamond_system(8, "spd13", 7.0, 7.0)


@pytest.mark.parametrize("radius", [8.0, 10.0])
def test_taylor_powers_rows_at_full_size(rt, cell4096, radius):
    s = cell4096
    radii = dict(r_Sinv=radius, r_T=radius, r_U=radius, r_K=radius, r_M=radius)
    got = {}
    T = None
    for precision in ("fp64", "fp32"):
        ctx = rt.RT(s, precision=precision, full_step=0, dt=0.05, **radii)
        ctx.inverse()
        ctx.propagator(0.0)
        if T is None:
            T = ctx.matrix(0, rt.RT_MAT_T)
            rpT, colT = ctx.pattern(0, rt.RT_PAT_T)
            rpU, colU = ctx.pattern(0, rt.RT_PAT_U)
        got[precision] = ctx.matrix(0, rt.RT_MAT_U)
        ctx.close()
    pT, pU = oracle.Pattern(rpT, colT), oracle.Pattern(rpU, colU)
    assert pT == oracle.pattern(s.pos, s.cell, radius)  # the patterns themselves are pinned bit for bit
    Tb = oracle.BlockMatrix(s.bsize, pT, T)
    dt = 0.05
    coef = [(-1j * dt) ** n / np.prod(np.arange(1, n + 1)) for n in range(6)]
    P = oracle.restrict(Tb, pU)
    Uo = oracle.axpy(coef[1], P, oracle.identity(s.bsize, pU))
    for n in range(2, 5):  # full powers: row i of T^5 needs rows of T^4 over the 4-hop neighbourhood
        P = oracle.spgemm(Tb, P, pU)
        Uo = oracle.axpy(coef[n], P, Uo)
    P5 = oracle.zeros(s.bsize, pU)
    for i in SAMPLE:
        oracle.spgemm(Tb, P, pU, rows=(i, i + 1), out=P5)
    Uo = oracle.axpy(coef[5], P5, Uo)
    ident = oracle.identity(s.bsize, pU).val
    for precision, bar in (("fp64", 1e-10), ("fp32", 1e-6)):
        worst, scale = 0.0, 0.0
        for i in SAMPLE:
            sl = slice(Uo.voff[pU.rowptr[i]], Uo.voff[pU.rowptr[i + 1]])
            ref = Uo.val[sl] - ident[sl]
            worst = max(worst, float(np.abs(got[precision][sl] - ident[sl] - ref).max()))
            scale = max(scale, float(np.abs(ref).max()))
        assert worst <= bar * scale, (precision, radius, worst, scale)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sandwich_rows_at_full_size(rt, workload, precision):
    s, pat, Kb = workload
    ctx = rt.RT(s, precision=precision, full_step=0, r_Sinv=R, r_T=R, r_U=R, r_K=R, r_M=R)
    ctx.inverse()
    rp, col = ctx.pattern(0, rt.RT_PAT_K)
    assert np.array_equal(rp, pat.rowptr) and np.array_equal(col, pat.col)
    ctx.set_density(0, 0, Kb.val)
    ctx.propagator(0.0)
    U = ctx.matrix(0, rt.RT_MAT_U)
    ctx.step(1)
    K1 = ctx.matrix(0, rt.RT_MAT_K)
    ctx.close()
    Ub = oracle.BlockMatrix(s.bsize, pat, U)
    M = oracle.zeros(s.bsize, pat)
    Kn = oracle.zeros(s.bsize, pat)
    for i in SAMPLE:
        oracle.spgemm(Ub, Kb, pat, rows=(i, i + 1), out=M)
        oracle.spgemm(M, Ub, pat, b_dag=True, rows=(i, i + 1), upper_only=True, out=Kn)
    worst, scale = 0.0, 0.0
    for i in SAMPLE:
        for q in range(pat.rowptr[i], pat.rowptr[i + 1]):
            j = pat.col[q]
            if j < i:
                continue
            ref = Kn.val[Kn.voff[q]:Kn.voff[q + 1]].reshape(13, 13)
            if j == i:
                ref = 0.5 * (ref + ref.conj().T)
            got = K1[Kn.voff[q]:Kn.voff[q + 1]].reshape(13, 13)
            worst = max(worst, float(np.abs(got - ref).max()))
            scale = max(scale, float(np.abs(ref).max()))
    bar = 1e-10 if precision == "fp64" else 1e-6
    assert worst <= bar * scale, (worst, scale)
