"""Host-side measures of the truncation studies (no GPU): block assembly,
pattern masks and the error norms, checked against direct constructions."""
import numpy as np

import oracle
import synth
from paper_1404_5776_gb300 import studies


def test_blocks_to_dense_matches_the_generator():
    pos, species = synth.si_h_cluster(target=40)
    s = synth.build_system(pos, None, species, 5.0, 5.0)  # block sizes 1 and 4
    ref = s.to_dense("S")
    got = studies.blocks_to_dense(s.bsize, s.s_rowptr, s.s_col, s.s_val)
    assert np.array_equal(got, ref)


def test_pattern_mask_covers_exactly_the_blocks():
    s = synth.diamond_system(2, "sp4", 6.0, 6.0)
    P = oracle.pattern(s.pos, s.cell, 4.0)
    m = studies.pattern_mask(s.bsize, P.rowptr, P.col)
    rows = np.repeat(np.arange(s.n_atoms), np.diff(P.rowptr))
    assert m.sum() == int(np.sum(s.bsize[rows] * s.bsize[P.col]))
    # symmetric pattern -> symmetric mask; the diagonal blocks are in
    assert np.array_equal(m, m.T)
    assert all(m[i, i] for i in range(m.shape[0]))


def test_error_measures():
    E = np.array([[1.0, -2.0], [0.0, 3.0]])
    e = studies.error_measures(E)
    assert e["mean"] == 1.5 and e["row"] == 3.0 and e["max"] == 3.0


def test_truncated_inverse_error_falls_with_range():
    """The S^-1 error measure on the oracle's Hotelling inverse (the same
    post-processing the GPU sweep applies): it falls with the range and
    vanishes when every pair is kept."""
    s = synth.diamond_system(2, "sp4", 6.0, 6.0)
    S, H, Sinv, T = studies.dense_reference(s)
    Sb = oracle.BlockMatrix(s.bsize, oracle.Pattern(s.s_rowptr, s.s_col), s.s_val)
    errs = []
    for r in (3.0, 5.0, 12.0):
        X = oracle.hotelling(Sb, oracle.pattern(s.pos, s.cell, r), tol=1e-12, maxit=100).X
        Xd = studies.blocks_to_dense(s.bsize, X.pat.rowptr, X.pat.col, X.val).real
        errs.append(studies.error_measures(Xd @ S - np.eye(S.shape[0]))["row"])
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-9
    assert np.allclose(T, Sinv @ H)
