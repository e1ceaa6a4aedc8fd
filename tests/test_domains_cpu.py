"""Domain decomposition of one system over ranks (host side, CPU).

The plan (Morton-ordered domains, halo rows per product, point-to-point
exchange, all-reduce of the traces) is checked with two gloo ranks: each rank
owns a contiguous range of block rows in the Morton numbering, every row it
neither owns nor receives is set to NaN, and after the halo exchange its rows
of M = cut(U K) and of K' = cut(M U^dagger) (the sandwich of Sec. II.A, full
rows) are computed with the oracle's row-range product.  They must equal the
single-rank products bit for bit (same products, same k order), and the
all-reduced partial traces Tr(K' S), Tr(K' D_xyz) must match the single-rank
traces to rounding."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import synth
from paper_1404_5776_gb300 import domains

R = 6.0


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _morton_system():
    pos, cell = synth.diamond_positions(3)
    order = domains.morton_order(pos, cell)
    s = synth.build_system(pos[order], cell, ["sp4"] * len(pos), 6.0, 6.0)
    return s, pos, cell, order


def test_morton_order_is_a_local_permutation():
    pos, cell = synth.diamond_positions(3)
    order = domains.morton_order(pos, cell)
    assert sorted(order.tolist()) == list(range(len(pos)))
    d = synth.min_image_d2(pos[order[:-1]], pos[order[1:]], cell)
    rng = np.random.default_rng(0)
    perm = rng.permutation(len(pos))
    d_rand = synth.min_image_d2(pos[perm[:-1]], pos[perm[1:]], cell)
    assert np.sqrt(d).mean() < 0.6 * np.sqrt(d_rand).mean()


def test_permuted_pattern_matches_the_pattern_of_permuted_positions():
    pos, cell = synth.diamond_positions(2)
    order = domains.morton_order(pos, cell)
    p_old = oracle.pattern(pos, cell, R)
    rp, col, src = domains.permute_pattern(p_old.rowptr, p_old.col, order)
    p_new = oracle.pattern(pos[order], cell, R)
    assert np.array_equal(rp, p_new.rowptr) and np.array_equal(col, p_new.col)
    rows_old = p_old.rows()
    inv = np.empty(len(order), dtype=np.int64)
    inv[order] = np.arange(len(order))
    assert np.array_equal(inv[rows_old[src]], p_new.rows()) and np.array_equal(inv[p_old.col[src]], col)


def test_balanced_ranges():
    w = np.arange(1, 101, dtype=float)
    rr = domains.balanced_ranges(w, 4)
    assert rr[0][0] == 0 and rr[-1][1] == 100 and all(a < b for a, b in rr)
    assert all(rr[p][1] == rr[p + 1][0] for p in range(3))
    tot = [w[a:b].sum() for a, b in rr]
    assert max(tot) - min(tot) <= w.max()
    with pytest.raises(ValueError):
        domains.balanced_ranges(np.ones(2), 3)


def test_halo_plan_is_exact():
    s, *_ = _morton_system()
    pat = oracle.pattern(s.pos, s.cell, R)
    ranges = domains.balanced_ranges(np.diff(pat.rowptr), 3)
    plan = domains.plan_halo(pat.rowptr, pat.col, ranges)
    own = domains.owner_of_rows(ranges, s.n_atoms)
    for p, (r0, r1) in enumerate(ranges):
        want = set(pat.col[pat.rowptr[r0]:pat.rowptr[r1]].tolist()) - set(range(r0, r1))
        got = set(plan.halo(p).tolist())
        assert got == want
        for q in range(3):
            for k in plan.need.get((p, q), []):
                assert own[k] == q
    # a compact (Morton) domain needs far fewer halo rows than a scattered one
    rng = np.random.default_rng(1)
    perm = rng.permutation(s.n_atoms)
    p_rand = oracle.pattern(s.pos[perm], s.cell, R)
    plan_r = domains.plan_halo(p_rand.rowptr, p_rand.col, ranges)
    assert len(plan.halo(0)) < len(plan_r.halo(0))


def _single_rank(s):
    """U (EM, 6 terms), K(0+) after an x kick, M = cut(U K), K' = cut(M U^dagger) full rows."""
    p = oracle.Params(r_Sinv=R, r_T=R, r_U=R, r_K=R, r_M=R)
    ref = oracle.Propagator(s, p)
    K0, _, _ = synth.ground_state_dense(s, s.n // 2)
    ref.set_density_dense(K0)
    ref.kick(0, 1e-3)
    U, _ = ref.propagator(0.0)
    pat = ref.pats["K"]
    M = oracle.spgemm(U, ref.K, ref.pats["M"])
    Kn = oracle.spgemm(M, U, pat, b_dag=True)
    return ref, U, M, Kn


def _partial_traces(Kn, X, r0, r1):
    tot = 0.0 + 0.0j
    rows = Kn.pat.rows()
    for q in range(Kn.pat.rowptr[r0], Kn.pat.rowptr[r1]):
        i, j = rows[q], Kn.pat.col[q]
        qx = oracle.find(X.pat, j, i)
        if qx < 0:
            continue
        kb = Kn.val[Kn.voff[q]:Kn.voff[q + 1]].reshape(Kn.bsize[i], Kn.bsize[j])
        xb = X.val[X.voff[qx]:X.voff[qx + 1]].reshape(X.bsize[j], X.bsize[i])
        tot += np.sum(kb * xb.T)
    return tot


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s, *_ = _morton_system()
    ref, U, M_full, Kn_full = _single_rank(s)
    pU, pK, pM = ref.pats["U"], ref.pats["K"], ref.pats["M"]
    ranges = domains.balanced_ranges(np.diff(pK.rowptr), world)
    r0, r1 = ranges[rank]

    def local(A, keep):
        """This rank's copy: the rows in `keep` kept, every other row NaN."""
        B = A.copy()
        mask = np.ones(s.n_atoms, bool)
        mask[keep] = False
        for k in np.nonzero(mask)[0]:
            B.val[B.voff[A.pat.rowptr[k]]:B.voff[A.pat.rowptr[k + 1]]] = np.nan
        return B

    own = np.arange(r0, r1)
    # M = cut(U K): own rows of U, own + halo rows of K (halo over P_U)
    plan_m = domains.plan_halo(pU.rowptr, pU.col, ranges)
    Kl = local(ref.K, own)
    domains.exchange_rows(dist, plan_m, rank, pK.rowptr, Kl.voff, Kl.val)
    Ul = local(U, own)
    M = oracle.zeros(s.bsize, pM)
    oracle.spgemm(Ul, Kl, pM, rows=(r0, r1), out=M)
    # K' = cut(M U^dagger): block (j, k) of U for (i, j) in P_K: halo of U over P_K
    plan_k = domains.plan_halo(pK.rowptr, pK.col, ranges)
    domains.exchange_rows(dist, plan_k, rank, pU.rowptr, Ul.voff, Ul.val)
    Kn = oracle.zeros(s.bsize, pK)
    oracle.spgemm(M, Ul, pK, b_dag=True, rows=(r0, r1), out=Kn)
    sl_m = slice(M.voff[pM.rowptr[r0]], M.voff[pM.rowptr[r1]])
    sl_k = slice(Kn.voff[pK.rowptr[r0]], Kn.voff[pK.rowptr[r1]])
    exact_m = bool(np.array_equal(M.val[sl_m], M_full.val[sl_m]))
    exact_k = bool(np.array_equal(Kn.val[sl_k], Kn_full.val[sl_k]))
    part = np.zeros(8)
    for c, X in enumerate([ref.S] + ref.D):
        z = _partial_traces(Kn, X, r0, r1)
        part[2 * c], part[2 * c + 1] = z.real, z.imag
    tot = domains.allreduce_traces(dist, part)
    want = np.array(oracle.observables(Kn_full, ref.S, ref.D))
    ok_tr = bool(np.allclose(tot[0::2], want.real, rtol=1e-12, atol=0)
                 and np.allclose(tot[1::2], want.imag, rtol=0, atol=1e-9 * np.abs(want.real).max()))
    out[rank] = (exact_m, exact_k, ok_tr, len(plan_m.halo(rank)), r1 - r0)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_sandwich_with_halo_exchange_is_bit_exact():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(600)
        assert p.exitcode == 0
    for rank in range(2):
        exact_m, exact_k, ok_tr, n_halo, n_own = out[rank]
        assert exact_m and exact_k and ok_tr, out[rank]
        # two halves of a 16 A periodic cell: the 6 A halo is the other half
        assert 0 < n_halo <= 216 - n_own
