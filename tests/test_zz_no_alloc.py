"""The allocation-free trace entry point (rt_traces_noalloc) against the oracle.

rt_traces_noalloc exists for callers that cannot allocate device memory when
they need the traces (inside a stream capture, or under a framework that owns
all device memory): it takes caller-owned device arrays and keeps its
reduction scratch in a fixed array inside the library.

The density here is the oracle's own K(0+) after a delta kick (the library
computes nothing but the traces), laid out the way the library stores blocks:
every atom padded to the largest block size B = 13, so the 4-function atoms of
the mixed cell carry padding that the entry point has to mask out.  The test
calls the entry point through the C ABI several times in a row (the calls share
the scratch array), with the automatic CTA count, a few CTAs that each sum many
blocks, and the maximum number of CTAs (more CTAs than blocks: most partials
are zero), and compares every result with the oracle's trace_product at 1e-12
relative (both sum the same FP64 products, in a different order)."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _padded(bm, B):
    """Block values of an oracle BlockMatrix as B x B padded blocks (zeros outside the true sizes)."""
    rows = bm.pat.rows()
    out = np.zeros((bm.pat.nnzb, B, B), dtype=bm.val.dtype)
    for q in range(bm.pat.nnzb):
        bi, bj = bm.bsize[rows[q]], bm.bsize[bm.pat.col[q]]
        out[q, :bi, :bj] = bm.val[bm.voff[q]:bm.voff[q + 1]].reshape(bi, bj)
    return out


def _transpose_map(src, dst):
    """For each block (i,j) of src, the index of block (j,i) in dst, or -1."""
    rows = src.rows()
    return np.array([oracle.find(dst, j, i) for i, j in zip(rows, src.col)], dtype=np.int32)


def test_traces_noalloc_matches_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1404_5776_gb300 as rt
    rt.build()
    pos, cell = synth.diamond_positions(2)
    species = ["spd13" if a % 2 == 0 else "sp4" for a in range(len(pos))]
    s = synth.build_system(pos, cell, species, 6.0, 6.0)
    B = int(max(s.bsize))
    assert B == 13 and int(min(s.bsize)) == 4  # padded atoms present
    K0, _, _ = synth.ground_state_dense(s, s.n // 2)
    r = 6.0
    ref = oracle.Propagator(s, oracle.Params(r_Sinv=r, r_T=r, r_U=r, r_K=r, r_M=r))
    ref.set_density_dense(K0)
    ref.kick(0, 1e-3)
    K = ref.K
    want = np.array(oracle.observables(K, ref.S, ref.D))

    pk, ps, ph = K.pat, ref.S.pat, ref.D[0].pat
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    dK = t(_padded(K, B).reshape(-1).view(np.float64))
    dS = t(_padded(ref.S, B).real.reshape(-1))
    dD = [t(_padded(d, B).real.reshape(-1)) for d in ref.D]
    drow, dcol = t(pk.rows().astype(np.int32)), t(pk.col.astype(np.int32))
    dks, dkd = t(_transpose_map(pk, ps)), t(_transpose_map(pk, ph))
    dbs = t(np.asarray(s.bsize, dtype=np.int32))
    out = torch.zeros(8, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    lib = rt.load()
    p = lambda x: ctypes.c_void_p(x.data_ptr())

    def call(n_ctas):
        return lib.rt_traces_noalloc(p(dK), pk.nnzb, p(drow), p(dcol), p(dbs), B, p(dS), p(dks), p(dD[0]), p(dD[1]),
                                     p(dD[2]), p(dkd), n_ctas, p(out), ctypes.c_void_p(stream))

    assert pk.nnzb < rt.RT_NOALLOC_MAX_CTAS * 8  # the last case has more warps than blocks
    for n_ctas in (0, 3, 0, rt.RT_NOALLOC_MAX_CTAS):  # calls in a row, sharing the scratch array
        out.fill_(np.nan)
        assert call(n_ctas) == rt.RT_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for c in range(4):  # Tr(KS), Tr(KDx), Tr(KDy), Tr(KDz)
            assert abs(got[2 * c] - want[c].real) <= 1e-12 * abs(want[c].real)
            assert got[2 * c + 1] == 0.0 and abs(want[c].imag) <= 1e-12 * abs(want[c].real)
    # sizes beyond the scratch limit are rejected before any GPU work
    assert call(rt.RT_NOALLOC_MAX_CTAS + 1) == rt.RT_EINVAL
