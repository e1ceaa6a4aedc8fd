"""Truncation studies through the C ABI (paper Sec. IV-V) on a 64-atom cell:
the trends the paper reports, and the limits that hold exactly."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1404_5776_gb300 as m
    m.build()
    return m


def test_range_sweep_converges(rt):
    from paper_1404_5776_gb300 import studies
    s = synth.diamond_system(2, "sp4", 6.0, 6.0)
    recs = studies.truncation_sweep(rt, s, [4.0, 6.0, 8.0, 12.0])
    e_sinv = [r["err_Sinv"]["mean"] for r in recs]
    e_drop = [r["err_SinvH_drop"]["mean"] for r in recs]
    e_tot = [r["err_SinvH_total"]["mean"] for r in recs]
    assert all(a >= b for a, b in zip(e_sinv, e_sinv[1:])), e_sinv
    assert all(a >= b for a, b in zip(e_drop, e_drop[1:])), e_drop
    assert all(a >= b for a, b in zip(e_tot, e_tot[1:])), e_tot
    # r = 12 A keeps every pair of the 64-atom cell: nothing is dropped, and
    # S^-1 is the converged Hotelling inverse
    dense = recs[-1]
    assert dense["blocks_per_atom_Sinv"] == 64
    assert dense["err_SinvH_drop"]["max"] == 0.0
    assert dense["err_Sinv"]["max"] < 1e-8
    assert dense["err_SinvH_total"]["max"] < 1e-8
    # the propagator's unitarity improves with the range and is at the
    # Taylor-truncation level when nothing is cut
    u = [r["unitarity_UdSU_minus_S"]["mean"] for r in recs]
    assert u[-1] <= u[0]
    assert u[-1] < 1e-9


def test_unitarity_vs_dt_and_terms(rt):
    from paper_1404_5776_gb300 import studies
    s = synth.diamond_system(2, "sp4", 6.0, 6.0)
    recs = studies.unitarity_vs_dt_terms(rt, s, [0.02, 0.05, 0.1, 0.2], [3, 4, 6], r=12.0)
    by = {(r["terms"], r["dt"]): r["UdSU_minus_S"]["max"] for r in recs}
    for nt in (3, 4, 6):
        seq = [by[(nt, dt)] for dt in (0.02, 0.05, 0.1, 0.2)]
        assert all(a <= b for a, b in zip(seq, seq[1:])), (nt, seq)
    for dt in (0.1, 0.2):
        seq = [by[(nt, dt)] for nt in (3, 4, 6)]
        assert seq[0] > seq[-1], (dt, seq)
    # the error of an n-term series scales as dt^n for small dt (leading term of
    # the defect |g|^2 - 1, g the truncated exponential of a real eigenvalue):
    # even n gives dt^n, odd n dt^(n+1)
    ratio = by[(4, 0.1)] / by[(4, 0.05)]
    assert 8.0 < ratio < 32.0, ratio
