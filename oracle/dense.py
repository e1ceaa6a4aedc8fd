"""Dense mode of the oracle (numpy, FP64 complex).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Full n x n matrices.  Without masks nothing is truncated, which is the
setting where the method has closed forms (generalised eigenpairs of H v =
e S v).  With boolean masks each product is cut exactly as in the
block-sparse mode, which gives an independent dense restatement of the
truncated step for small cells.

S^-1 can be taken from a dense LU inverse (the paper's ScaLAPACK
alternative, Sec. V.A) or from Hotelling's iteration.
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np


def atom_mask(bsize, pat) -> np.ndarray:
    """Element mask of a block pattern (rowptr/col) for given block sizes."""
    bsize = np.asarray(bsize)
    foff = np.concatenate([[0], np.cumsum(bsize)])
    n = int(foff[-1])
    m = np.zeros((n, n), dtype=bool)
    rp, col = pat.rowptr, pat.col
    for i in range(len(bsize)):
        for q in range(rp[i], rp[i + 1]):
            j = col[q]
            m[foff[i]:foff[i + 1], foff[j]:foff[j + 1]] = True
    return m


def cut(X, mask):
    return X if mask is None else np.where(mask, X, 0.0)


def inverse_lu(S):
    """Dense inverse by LU factorisation (Sec. V.A alternative to Hotelling)."""
    return np.linalg.inv(S)


def hotelling(S, iters=None, tol=1e-12, maxit=200, mask=None, X0=None):
    """X <- X(2I - S X) from X0 = I/||S||_inf, products cut to `mask`."""
    n = S.shape[0]
    I = np.eye(n)
    X = X0 if X0 is not None else I / np.abs(S).sum(1).max()
    X = cut(X, mask)
    k = 0
    while True:
        Y = cut(S @ X, mask)
        res = np.linalg.norm(I - Y) / math.sqrt(n)
        if iters is None and (res < tol or k >= maxit):
            break
        if iters is not None and k >= iters:
            break
        X = cut(X @ (2 * I - Y), mask)
        k += 1
    return X, k, res


def taylor_em(T, dt, terms, mask_u=None):
    """sum_{n<terms} (-i dt)^n T^n / n!, powers cut to mask_u."""
    n = T.shape[0]
    U = np.eye(n, dtype=np.complex128)
    P = np.eye(n)
    coef = 1.0 + 0.0j
    for k in range(1, terms):
        P = T if k == 1 else cut(T @ P, mask_u)
        coef = coef * (-1j * dt) / k
        U = U + coef * P
    return cut(U, mask_u)


def em_propagator(Sinv, H, dt, terms=6, mask_t=None, mask_u=None):
    T = cut(Sinv @ H, mask_t)
    return taylor_em(T, dt, terms, mask_u)


def cn_propagator_exact(S, H, dt):
    """(S + i dt/2 H)^-1 (S - i dt/2 H) by a dense solve."""
    return np.linalg.solve(S + 0.5j * dt * H, S - 0.5j * dt * H)


def cn_propagator_hotelling(S, H, dt, X, iters, mask_u=None):
    A = S + 0.5j * dt * H
    B = S - 0.5j * dt * H
    n = S.shape[0]
    I = np.eye(n)
    res = 0.0
    for _ in range(iters):
        Y = cut(A @ X, mask_u)
        res = np.linalg.norm(I - Y) / math.sqrt(n)
        X = cut(X @ (2 * I - Y), mask_u)
    return cut(X @ B, mask_u), X, res


def sandwich(U, K, mask_m=None, mask_k=None, mask_upper=None):
    """K' = U K U^dagger, M cut to mask_m, K' to mask_k, hermitian by construction
    (upper blocks mirrored, diagonal blocks symmetrised) when mask_upper given."""
    M = cut(U @ K, mask_m)
    Kn = cut(M @ U.conj().T, mask_k)
    if mask_upper is None:
        return Kn
    up = np.where(mask_upper, Kn, 0.0)
    # mask_upper covers blocks with i < j plus diagonal blocks
    strict = np.where(mask_upper & ~mask_upper.T, up, 0.0)
    diag = np.where(mask_upper & mask_upper.T, Kn, 0.0)
    return strict + strict.conj().T + 0.5 * (diag + diag.conj().T)


def upper_block_mask(bsize):
    bsize = np.asarray(bsize)
    a = np.repeat(np.arange(len(bsize)), bsize)
    return a[:, None] <= a[None, :]


def trace(K, X):
    return complex(np.sum(K * X.T))


def generalized_eig(H, S):
    import scipy.linalg as sl
    w, V = sl.eigh(H, S)
    return w, V


def fermi_dense(H, S, mu, kT):
    """K = sum_a f(e_a) v_a v_a^T (V^T S V = I) — exact Fermi-Dirac density."""
    w, V = generalized_eig(H, S)
    f = 0.5 * (1.0 - np.tanh(0.5 * (w - mu) / kT))
    return (V * f) @ V.T
