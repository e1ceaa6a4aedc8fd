"""Truncation studies (paper Sec. IV: time-step and Taylor-term dependence of
the propagator unitarity; Sec. V: truncation of S^-1 and S^-1 H, their effect
on unitarity, size dependence, and density-matrix truncation).

Every matrix comes from the library through the C ABI (Hotelling S^-1, T, U,
rt_unitarity, steps); the host only measures them.  The untruncated reference
is the dense inverse of S (LU) and the dense product S^-1 H, so these sweeps
suit systems whose n x n dense matrices fit in host memory.

Error measures (the paper names them without a normalisation):
  mean  = average absolute value over all n x n elements;
  row   = average over rows of the row sum of absolute values (an intensive
          measure that does not fall as 1/N when the system grows).
For S^-1 the error matrix is X S - I (X the truncated Hotelling inverse).
For S^-1 H two errors are given: "drop", the elements that the cut to r_T
removes from the untruncated S^-1 H (the paper's definition: untruncated
S^-1 in the product), and "total", the library's T = cut(X H) against the
untruncated S^-1 H.
"""
from __future__ import annotations

import time
from typing import Iterable, Sequence

import numpy as np


def blocks_to_dense(bsize, rowptr, col, vals) -> np.ndarray:
    """Dense matrix from blocks in rowptr order (row-major, true sizes)."""
    bsize = np.asarray(bsize, dtype=np.int64)
    foff = np.concatenate([[0], np.cumsum(bsize)])
    n = int(foff[-1])
    out = np.zeros((n, n), dtype=vals.dtype)
    o = 0
    for i in range(len(bsize)):
        bi = int(bsize[i])
        for q in range(int(rowptr[i]), int(rowptr[i + 1])):
            j = int(col[q])
            bj = int(bsize[j])
            out[foff[i]:foff[i] + bi, foff[j]:foff[j] + bj] = vals[o:o + bi * bj].reshape(bi, bj)
            o += bi * bj
    return out


def pattern_mask(bsize, rowptr, col) -> np.ndarray:
    """Boolean n x n mask of the elements inside the blocks of a pattern."""
    bsize = np.asarray(bsize, dtype=np.int64)
    foff = np.concatenate([[0], np.cumsum(bsize)])
    n = int(foff[-1])
    m = np.zeros((n, n), dtype=bool)
    for i in range(len(bsize)):
        for q in range(int(rowptr[i]), int(rowptr[i + 1])):
            j = int(col[q])
            m[foff[i]:foff[i + 1], foff[j]:foff[j + 1]] = True
    return m


def error_measures(E: np.ndarray) -> dict:
    a = np.abs(E)
    return {"mean": float(a.mean()), "row": float(a.sum(axis=1).mean()), "max": float(a.max())}


def dense_reference(system):
    """Untruncated S^-1 (dense LU inverse) and S^-1 H0 of a system."""
    S = system.to_dense("S")
    H = system.to_dense("H")
    Sinv = np.linalg.inv(S)
    return S, H, Sinv, Sinv @ H


def _dense_of(rt, ctx, system, pat, mat, kick=0):
    rp, col = ctx.pattern(0, pat)
    v = ctx.matrix(0, mat, kick)
    return blocks_to_dense(system.bsize, rp, col, v), (rp, col)


def truncation_sweep(rt, system, radii: Sequence[float], dt: float = 0.05, taylor_terms: int = 6,
                     prop: str = "em", r_K: float | None = None, steps: int = 0, kappa: float = 1e-3,
                     K0_dense: np.ndarray | None = None, reference=None) -> list:
    """One record per radius r (r_Sinv = r_T = r_U = r): Hotelling iterations
    and residual, S^-1 and S^-1 H errors, U unitarity in both forms, and, when
    steps > 0 and K0 is given, the drift of Tr(K S) over a kicked run."""
    S, H, Sinv_ref, T_ref = reference if reference is not None else dense_reference(system)
    n = S.shape[0]
    I = np.eye(n)
    out = []
    for r in radii:
        rk = r if r_K is None else r_K
        t0 = time.perf_counter()
        ctx = rt.RT(system, dt=dt, prop=prop, taylor_terms=taylor_terms, r_Sinv=r, r_T=r, r_U=r, r_K=rk, r_M=rk)
        try:
            iters, resid = ctx.inverse()
            ctx.propagator(0.0)
            X, _ = _dense_of(rt, ctx, system, rt.RT_PAT_SINV, rt.RT_MAT_SINV)
            rec = {"r": float(r), "hotelling_iters": int(iters), "hotelling_residual": float(resid)}
            for name, pat in (("Sinv", rt.RT_PAT_SINV), ("T", rt.RT_PAT_T), ("U", rt.RT_PAT_U), ("K", rt.RT_PAT_K)):
                rec[f"blocks_per_atom_{name}"] = ctx.pattern(0, pat)[1].size / system.n_atoms
            rec["err_Sinv"] = error_measures(X.real @ S - I)
            if prop == "em":
                T, (rp, col) = _dense_of(rt, ctx, system, rt.RT_PAT_T, rt.RT_MAT_T)
                mask = pattern_mask(system.bsize, rp, col)
                rec["err_SinvH_drop"] = error_measures(np.where(mask, 0.0, T_ref))
                rec["err_SinvH_total"] = error_measures(T.real - T_ref)
            mx, mn = ctx.unitarity(0, True)
            rec["unitarity_UdSU_minus_S"] = {"max": mx, "mean": mn}
            mx, mn = ctx.unitarity(0, False)
            rec["unitarity_UdU_minus_I"] = {"max": mx, "mean": mn}
            if steps > 0 and K0_dense is not None:
                ctx.set_density_dense(0, 0, K0_dense)
                ctx.kick(0, 0, 0, kappa)
                ctx.step(steps)
                obs = ctx.observables(0, 0)
                q = obs[:, 1]
                rec["charge_drift"] = float(np.abs(q - q[0]).max() / abs(q[0]))
                rec["dipole_x"] = obs[:, 3].tolist()
            rec["seconds"] = round(time.perf_counter() - t0, 3)
        finally:
            ctx.close()
        out.append(rec)
    return out


def size_sweep(rt, systems: Iterable, r_Sinv: float, r_T: float) -> list:
    """S^-1 H error at fixed ranges against system size (Sec. V)."""
    out = []
    for system in systems:
        S, H, Sinv_ref, T_ref = dense_reference(system)
        ctx = rt.RT(system, r_Sinv=r_Sinv, r_T=r_T, r_U=r_T, r_K=r_T, r_M=r_T)
        try:
            iters, resid = ctx.inverse()
            ctx.propagator(0.0)
            T, (rp, col) = _dense_of(rt, ctx, system, rt.RT_PAT_T, rt.RT_MAT_T)
            mask = pattern_mask(system.bsize, rp, col)
            X, _ = _dense_of(rt, ctx, system, rt.RT_PAT_SINV, rt.RT_MAT_SINV)
            out.append({"n_atoms": int(system.n_atoms), "n": int(S.shape[0]), "hotelling_iters": int(iters),
                        "err_Sinv": error_measures(X.real @ S - np.eye(S.shape[0])),
                        "err_SinvH_drop": error_measures(np.where(mask, 0.0, T_ref)),
                        "err_SinvH_total": error_measures(T.real - T_ref),
                        "unitarity_UdSU_minus_S": dict(zip(("max", "mean"), ctx.unitarity(0, True)))})
        finally:
            ctx.close()
    return out


def unitarity_vs_dt_terms(rt, system, dts: Sequence[float], terms: Sequence[int], r: float,
                          prop: str = "em") -> list:
    """Unitarity of U(t=0) against the time step and the number of Taylor terms
    (Sec. IV), both forms."""
    out = []
    for nt in terms:
        for dt in dts:
            ctx = rt.RT(system, dt=dt, prop=prop, taylor_terms=nt, r_Sinv=r, r_T=r, r_U=r, r_K=r, r_M=r)
            try:
                ctx.inverse()
                ctx.propagator(0.0)
                s_mx, s_mn = ctx.unitarity(0, True)
                i_mx, i_mn = ctx.unitarity(0, False)
            finally:
                ctx.close()
            out.append({"terms": int(nt), "dt": float(dt), "UdSU_minus_S": {"max": s_mx, "mean": s_mn},
                        "UdU_minus_I": {"max": i_mx, "mean": i_mn}})
    return out
