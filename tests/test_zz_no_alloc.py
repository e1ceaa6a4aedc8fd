"""The allocation-free trace entry point (rt_traces_noalloc) against the
library's own observables.

rt_traces_noalloc exists for callers that cannot allocate device memory when
they need the traces (inside a stream capture, or under a framework that owns
all device memory): it takes caller-owned device arrays and keeps its
reduction scratch in a fixed array inside the library.  This test builds those
arrays from a context's density, overlap and dipole blocks, calls the entry
point twice in a row through the C ABI, and compares both results with the
Tr(KS), Tr(KD) that rt_observables reports for the same density (1e-12
relative: both sum the same FP64 products, in a different order)."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _index_of(rowptr, col, i, j):
    lo, hi = rowptr[i], rowptr[i + 1]
    k = lo + np.searchsorted(col[lo:hi], j)
    return int(k) if k < hi and col[k] == j else -1


def test_traces_noalloc_matches_observables():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1404_5776_gb300 as rt
    rt.build()
    s = synth.diamond_system(2, "sp4", 6.0, 6.0)  # 4 functions per atom: no padding
    K0, _, _ = synth.ground_state_dense(s, s.n // 2)
    ctx = rt.RT(s, r_Sinv=6.0, r_T=6.0, r_U=6.0, r_K=6.0, r_M=6.0)
    ctx.inverse()
    ctx.set_density_dense(0, 0, K0)
    ctx.kick(0, 0, 0, 1e-3)
    ctx.step(3)
    ref = ctx.observables(0, 0)[-1, 1:9]
    K = ctx.matrix(0, rt.RT_MAT_K)
    S = ctx.matrix(0, rt.RT_MAT_S).real.copy()
    D = [ctx.matrix(0, w).real.copy() for w in (rt.RT_MAT_DX, rt.RT_MAT_DY, rt.RT_MAT_DZ)]
    krp, kcol = ctx.pattern(0, rt.RT_PAT_K)
    srp, scol = ctx.pattern(0, rt.RT_PAT_S)
    hrp, hcol = ctx.pattern(0, rt.RT_PAT_H)
    ctx.close()
    rowidx = np.repeat(np.arange(s.n_atoms, dtype=np.int32), np.diff(krp))
    ks = np.array([_index_of(srp, scol, j, i) for i, j in zip(rowidx, kcol)], dtype=np.int32)
    kd = np.array([_index_of(hrp, hcol, j, i) for i, j in zip(rowidx, kcol)], dtype=np.int32)

    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    dK = t(K.view(np.float64))
    dS, dDx, dDy, dDz = t(S), t(D[0]), t(D[1]), t(D[2])
    drow, dcol, dks, dkd = t(rowidx), t(kcol.astype(np.int32)), t(ks), t(kd)
    dbs = t(np.asarray(s.bsize, dtype=np.int32))
    out = torch.zeros(8, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    lib = rt.load()
    p = lambda x: ctypes.c_void_p(x.data_ptr())
    results = []
    for n_ctas in (0, 7):  # two calls in a row, sharing the scratch array
        out.zero_()
        st = lib.rt_traces_noalloc(p(dK), len(kcol), p(drow), p(dcol), p(dbs), 4, p(dS), p(dks), p(dDx), p(dDy),
                                   p(dDz), p(dkd), n_ctas, p(out), ctypes.c_void_p(stream))
        assert st == rt.RT_OK
        torch.cuda.synchronize()
        results.append(out.cpu().numpy().copy())
    for got in results:
        for c in (0, 2, 4, 6):  # real parts of Tr(KS), Tr(KDx), Tr(KDy), Tr(KDz)
            assert abs(got[c] - ref[c]) <= 1e-12 * abs(ref[c])
        assert np.all(got[1::2] == 0.0) and np.all(ref[1::2] == 0.0)
    # sizes beyond the scratch limit are rejected before any GPU work
    st = lib.rt_traces_noalloc(p(dK), len(kcol), p(drow), p(dcol), p(dbs), 4, p(dS), p(dks), p(dDx), p(dDy), p(dDz),
                               p(dkd), 4096, p(out), ctypes.c_void_p(stream))
    assert st == rt.RT_EINVAL
