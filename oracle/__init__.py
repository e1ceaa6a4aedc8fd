"""CPU FP64 oracle for the truncated density-matrix RT-TDDFT time step.

TEST INFRASTRUCTURE ONLY.  This package is the checker, never the product:
only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import it.  It shares no code with the CUDA path (it only takes its
inputs from the ``synth`` generator).

The oracle follows O'Rourke & Bowler (arXiv:1404.5776) step by step:

* Sec. II.A, eq. (Liouville) and the formal solution K(t) = U K(t0) U^dagger:
  one step is the sandwich K <- U K U^dagger.
* eq. (EM): exponential-midpoint propagator U = exp(-i S^-1 H(t+dt/2) dt),
  with the exponential taken as the truncated Taylor series of eq.
  (matrix_exp), six terms in total (Sec. IV.B).
* Sec. V.A: S^-1 by Hotelling's iteration X <- X(2I - S X), once at t=0,
  and only the truncated product T = S^-1 H enters the propagator.
* Sec. II.A spatial cut-off: every product is cut to its output radius.
* Sec. II.B: the field enters as delta v = -E_j(t) r, so H(t) = H0 - E(t) D_j;
  the dipole observable is Tr(K D_j) and the charge is Tr(K S) (Sec. IV).
* Crank-Nicolson form U = (S + i dt/2 H)^-1 (S - i dt/2 H), with the inverse
  by the same Hotelling iteration warm-started from the previous step (an
  added propagator mode; the paper uses EM throughout).
* Sec. II.A also defines the enforced-time-reversal-symmetry propagator
  U_ETRS = exp(-i dt/2 S^-1 H(t+dt)) exp(-i dt/2 S^-1 H(t)) and the fourth-order
  Magnus propagator U_M4 = exp(M), M = -i dt/2 [T(t1) + T(t2)]
  - (sqrt(3) dt^2 / 12) [T(t2), T(t1)], t_{2,1} = t + (1/2 +- sqrt(3)/6) dt,
  T = S^-1 H; every exponential by the same truncated Taylor series.

Two modes share these definitions: the truncated block-sparse mode here (C
kernels in ``oracle.c`` for patterns and products) and the dense mode in
``oracle.dense`` (numpy, no truncation unless masks are given).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (plain C11, OpenMP, no FP contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        L.or_pattern_count.restype = ctypes.c_int64
        L.or_pattern_count.argtypes = [ctypes.c_int, P, P, ctypes.c_double, P]
        L.or_pattern_fill.restype = None
        L.or_pattern_fill.argtypes = [ctypes.c_int, P, P, ctypes.c_double, P, P]
        L.or_min_image_d2.restype = None
        L.or_min_image_d2.argtypes = [ctypes.c_int, P, P, P, P]
        L.or_spgemm.restype = None
        L.or_spgemm.argtypes = [ctypes.c_int, P,
                                P, P, P, P, ctypes.c_int,
                                P, P, P, P, ctypes.c_int,
                                P, P, P, P,
                                ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.or_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------------------
# patterns (Sec. II.A spatial cut-off)
# ----------------------------------------------------------------------------

@dataclass
class Pattern:
    rowptr: np.ndarray  # int32 [n+1]
    col: np.ndarray     # int32 [nnzb]

    @property
    def nnzb(self):
        return int(self.rowptr[-1])

    def rows(self):
        return np.repeat(np.arange(len(self.rowptr) - 1, dtype=np.int32), np.diff(self.rowptr))

    def __eq__(self, other):
        return np.array_equal(self.rowptr, other.rowptr) and np.array_equal(self.col, other.col)


def pattern(pos, cell, r: float) -> Pattern:
    """P_r = {(i,j): minimum-image |R_i - R_j| < r}, brute force in C."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n = len(pos)
    cellp = None if cell is None else np.ascontiguousarray(cell, dtype=np.float64)
    rowptr = np.zeros(n + 1, dtype=np.int32)
    L = lib()
    nnz = L.or_pattern_count(n, _p(pos), None if cellp is None else _p(cellp), float(r), _p(rowptr))
    col = np.zeros(max(nnz, 1), dtype=np.int32)
    L.or_pattern_fill(n, _p(pos), None if cellp is None else _p(cellp), float(r), _p(rowptr), _p(col))
    return Pattern(rowptr, col[:nnz])


# ----------------------------------------------------------------------------
# block-sparse matrices
# ----------------------------------------------------------------------------

@dataclass
class BlockMatrix:
    """Atom-blocked matrix on a pattern; values complex128, row-major blocks."""
    bsize: np.ndarray
    pat: Pattern
    val: np.ndarray
    voff: np.ndarray = None

    def __post_init__(self):
        if self.voff is None:
            self.voff = block_offsets(self.bsize, self.pat)
        self.val = np.ascontiguousarray(self.val, dtype=np.complex128)
        assert len(self.val) == self.voff[-1]

    def copy(self):
        return BlockMatrix(self.bsize, self.pat, self.val.copy(), self.voff)

    def block(self, i, j):
        q = find(self.pat, i, j)
        if q < 0:
            return None
        bi, bj = self.bsize[i], self.bsize[j]
        return self.val[self.voff[q]:self.voff[q + 1]].reshape(bi, bj)

    def to_dense(self):
        foff = np.concatenate([[0], np.cumsum(self.bsize)])
        n = int(foff[-1])
        out = np.zeros((n, n), dtype=np.complex128)
        rows = self.pat.rows()
        for q in range(self.pat.nnzb):
            i, j = rows[q], self.pat.col[q]
            out[foff[i]:foff[i + 1], foff[j]:foff[j + 1]] = \
                self.val[self.voff[q]:self.voff[q + 1]].reshape(self.bsize[i], self.bsize[j])
        return out


def block_offsets(bsize, pat: Pattern):
    rows = pat.rows()
    sz = bsize[rows].astype(np.int64) * bsize[pat.col].astype(np.int64)
    return np.concatenate([[0], np.cumsum(sz)]).astype(np.int64)


def find(pat: Pattern, i, j):
    lo, hi = pat.rowptr[i], pat.rowptr[i + 1]
    k = lo + np.searchsorted(pat.col[lo:hi], j)
    if k < hi and pat.col[k] == j:
        return int(k)
    return -1


def from_dense(bsize, pat: Pattern, dense) -> BlockMatrix:
    foff = np.concatenate([[0], np.cumsum(bsize)])
    rows = pat.rows()
    parts = [dense[foff[i]:foff[i + 1], foff[j]:foff[j + 1]].reshape(-1)
             for i, j in zip(rows, pat.col)]
    val = np.concatenate(parts) if parts else np.zeros(0)
    return BlockMatrix(bsize, pat, val.astype(np.complex128))


def zeros(bsize, pat: Pattern) -> BlockMatrix:
    voff = block_offsets(bsize, pat)
    return BlockMatrix(bsize, pat, np.zeros(voff[-1], dtype=np.complex128), voff)


def identity(bsize, pat: Pattern, scale=1.0) -> BlockMatrix:
    M = zeros(bsize, pat)
    for i in range(len(bsize)):
        q = find(pat, i, i)
        assert q >= 0, "pattern lacks a diagonal block"
        b = bsize[i]
        M.val[M.voff[q]:M.voff[q + 1]] = (scale * np.eye(b)).reshape(-1)
    return M


def restrict(A: BlockMatrix, pat: Pattern) -> BlockMatrix:
    """A on another pattern: blocks outside `pat` dropped, missing ones zero (cut)."""
    out = zeros(A.bsize, pat)
    rows = pat.rows()
    for q in range(pat.nnzb):
        qa = find(A.pat, rows[q], pat.col[q])
        if qa >= 0:
            out.val[out.voff[q]:out.voff[q + 1]] = A.val[A.voff[qa]:A.voff[qa + 1]]
    return out


def axpy(alpha, X: BlockMatrix, Y: BlockMatrix) -> BlockMatrix:
    """alpha*X + Y on Y's pattern (X restricted to it)."""
    if X.pat is Y.pat or X.pat == Y.pat:
        return BlockMatrix(Y.bsize, Y.pat, alpha * X.val + Y.val, Y.voff)
    return BlockMatrix(Y.bsize, Y.pat, alpha * restrict(X, Y.pat).val + Y.val, Y.voff)


def spgemm(A: BlockMatrix, B: BlockMatrix, pat_c: Pattern, a_dag=False, b_dag=False,
           rows=None, upper_only=False, out: BlockMatrix = None) -> BlockMatrix:
    """C = cut_{P_C}(op(A) op(B)) (truncated block product, C kernel)."""
    C = out if out is not None else zeros(A.bsize, pat_c)
    n = len(A.bsize)
    r0, r1 = (0, n) if rows is None else rows
    bs = np.ascontiguousarray(A.bsize, dtype=np.int32)
    lib().or_spgemm(n, _p(bs),
                    _p(A.pat.rowptr), _p(A.pat.col), _p(A.voff), _p(A.val), int(a_dag),
                    _p(B.pat.rowptr), _p(B.pat.col), _p(B.voff), _p(B.val), int(b_dag),
                    _p(C.pat.rowptr), _p(C.pat.col), _p(C.voff), _p(C.val),
                    int(r0), int(r1), int(upper_only))
    return C


def mirror_upper(C: BlockMatrix) -> float:
    """Fill lower blocks from upper ones (C_ji = C_ij^dagger); symmetrise the
    diagonal blocks to (C_ii + C_ii^dagger)/2.  Returns the largest
    |C_ii - C_ii^dagger| element seen before symmetrising."""
    rows = C.pat.rows()
    herm = 0.0
    for q in range(C.pat.nnzb):
        i, j = rows[q], C.pat.col[q]
        bi, bj = C.bsize[i], C.bsize[j]
        blk = C.val[C.voff[q]:C.voff[q + 1]].reshape(bi, bj)
        if i == j:
            herm = max(herm, float(np.abs(blk - blk.conj().T).max()))
            C.val[C.voff[q]:C.voff[q + 1]] = (0.5 * (blk + blk.conj().T)).reshape(-1)
        elif i < j:
            qm = find(C.pat, j, i)
            C.val[C.voff[qm]:C.voff[qm + 1]] = blk.conj().T.reshape(-1)
    return herm


# ----------------------------------------------------------------------------
# method steps
# ----------------------------------------------------------------------------

def inf_norm(A: BlockMatrix) -> float:
    """max_i sum_j |A_ij| over all matrix elements (Gershgorin bound)."""
    foff = np.concatenate([[0], np.cumsum(A.bsize)])
    rs = np.zeros(int(foff[-1]))
    rows = A.pat.rows()
    for q in range(A.pat.nnzb):
        i, j = rows[q], A.pat.col[q]
        blk = np.abs(A.val[A.voff[q]:A.voff[q + 1]]).reshape(A.bsize[i], A.bsize[j])
        rs[foff[i]:foff[i + 1]] += blk.sum(1)
    return float(rs.max())


def residual_I_minus(Y: BlockMatrix) -> float:
    """||I - Y||_F / sqrt(n) over the entries of Y's pattern."""
    I = identity(Y.bsize, Y.pat)
    d = I.val - Y.val
    n = int(np.sum(Y.bsize))
    return float(np.sqrt(np.sum(np.abs(d) ** 2)) / math.sqrt(n))


@dataclass
class HotellingResult:
    X: BlockMatrix
    iters: int
    residual: float
    status: str             # "converged" | "stagnated" | "maxit" | "diverged"
    history: List[float] = field(default_factory=list)


def hotelling(A: BlockMatrix, pat_x: Pattern, tol=1e-10, maxit=100, X0: BlockMatrix = None,
              stagnation=0.9, fixed_iters: Optional[int] = None) -> HotellingResult:
    """Hotelling's iteration X <- X(2I - A X) with products cut to P_X (Sec. V.A).

    X0 defaults to I/||A||_inf.  Each iteration first forms Y = cut(A X) and its
    residual ||I - Y||_F/sqrt(n); it stops when the residual is below tol
    (converged), stops growing smaller by more than the factor `stagnation`
    (stagnated at the truncation floor), exceeds 1 (diverged) or after maxit.
    With fixed_iters the update runs exactly that many times (no tests).
    """
    X = restrict(X0, pat_x) if X0 is not None else identity(A.bsize, pat_x, 1.0 / inf_norm(A))
    hist = []
    it = 0
    nmax = fixed_iters if fixed_iters is not None else maxit
    status = "maxit"
    while True:
        Y = spgemm(A, X, pat_x)
        res = residual_I_minus(Y)
        hist.append(res)
        if fixed_iters is None:
            if not np.isfinite(res) or res > 1.0:
                status = "diverged"
                break
            if res < tol:
                status = "converged"
                break
            if len(hist) > 1 and res > stagnation * hist[-2]:
                status = "stagnated"
                break
        if it >= nmax:
            status = "fixed" if fixed_iters is not None else "maxit"
            break
        Z = axpy(-1.0, Y, identity(A.bsize, pat_x, 2.0))
        X = spgemm(X, Z, pat_x)
        it += 1
    return HotellingResult(X, it, hist[-1], status, hist)


def field_value(field, t):
    """E(t) of the supported external fields (Sec. II.B / Sec. IV.A Gaussian pulse)."""
    if field is None:
        return 0.0
    kind = field.get("kind", "none")
    if kind == "none":
        return 0.0
    if kind == "gaussian":
        E0, t0, sig, w = field["E0"], field["t0"], field["sigma"], field.get("omega", 0.0)
        x = t - t0
        return E0 * math.exp(-(x * x) / (2.0 * sig * sig)) * math.cos(w * x)
    if kind == "constant":
        return field["E0"]
    raise ValueError(kind)


def hamiltonian(H0: BlockMatrix, D: BlockMatrix, E: float) -> BlockMatrix:
    """H(t) = H0 - E(t) D_j  (delta v_ext = -E_j(t) r, Sec. II.B)."""
    return axpy(-E, D, H0)


def taylor_em(T: BlockMatrix, dt: float, terms: int, pat_u: Pattern):
    """U = sum_{n=0}^{terms-1} (-i dt)^n T^n / n!  with T^n = cut_{r_U}(T T^{n-1})
    (eq. matrix_exp, eq. EM).  Returns (U, [T^1..T^{terms-1}])."""
    U = identity(T.bsize, pat_u)
    powers = []
    P = T
    coef = 1.0 + 0.0j
    for n in range(1, terms):
        if n > 1:
            P = spgemm(T, P, pat_u)
        coef = coef * (-1j * dt) / n
        powers.append(P)
        U = axpy(coef, P, U)
    return U, powers


def sandwich(U: BlockMatrix, K: BlockMatrix, pat_m: Pattern):
    """K' = U K U^dagger (formal solution, Sec. II.A):
    M = cut_{r_M}(U K); K'_ij = sum_k M_ik U_jk^dagger on the upper blocks of
    P_K, then K'_ji = K'_ij^dagger and diagonal blocks made hermitian."""
    M = spgemm(U, K, pat_m)
    Kn = zeros(K.bsize, K.pat)
    spgemm(M, U, K.pat, b_dag=True, upper_only=True, out=Kn)
    herm = mirror_upper(Kn)
    return Kn, herm


def trace_product(K: BlockMatrix, X: BlockMatrix) -> complex:
    """Tr(K X) = sum_{ij} sum_{ab} K_ij[a,b] X_ji[b,a] over blocks present in both."""
    tot = 0.0 + 0.0j
    rows = K.pat.rows()
    for q in range(K.pat.nnzb):
        i, j = rows[q], K.pat.col[q]
        qx = find(X.pat, j, i)
        if qx < 0:
            continue
        kb = K.val[K.voff[q]:K.voff[q + 1]].reshape(K.bsize[i], K.bsize[j])
        xb = X.val[X.voff[qx]:X.voff[qx + 1]].reshape(X.bsize[j], X.bsize[i])
        tot += np.sum(kb * xb.T)
    return complex(tot)


def observables(K: BlockMatrix, S: BlockMatrix, D: List[BlockMatrix]):
    """[Tr(KS), Tr(KDx), Tr(KDy), Tr(KDz)] (Sec. IV charge; Sec. II.B dipole)."""
    return [trace_product(K, S)] + [trace_product(K, d) for d in D]


def unitarity(U: BlockMatrix, S: Optional[BlockMatrix], pat_w: Pattern):
    """E = cut_{P_U}(U^dagger cut_{P_W}(S U)) - S on P_U  (with S=None: U^dagger U - I).

    The paper prints U^dagger U - I (eq. s_unit); in the non-orthogonal basis
    the conserved form is U^dagger S U = S.  Returns (max|E|, mean|E|)."""
    W = spgemm(S, U, pat_w) if S is not None else U
    E = spgemm(U, W, U.pat, a_dag=True)
    ref = restrict(S, U.pat) if S is not None else identity(U.bsize, U.pat)
    d = np.abs(E.val - ref.val)
    return float(d.max()), float(d.mean())


def chebyshev_fermi_coeffs(order, mu, kT, e_lo, e_hi, jackson=False):
    """Chebyshev coefficients of f(e) = 1/(1+exp((e-mu)/kT)) on [e_lo, e_hi]
    by Chebyshev-Gauss quadrature with M = 4*(order+1) nodes."""
    a = 0.5 * (e_hi + e_lo)
    w = 0.5 * (e_hi - e_lo)
    M = 4 * (order + 1)
    th = math.pi * (np.arange(M) + 0.5) / M
    e = a + w * np.cos(th)
    f = 0.5 * (1.0 - np.tanh(0.5 * (e - mu) / kT))
    c = np.array([(2.0 if n else 1.0) / M * np.sum(f * np.cos(n * th)) for n in range(order + 1)])
    if jackson:
        N = order + 1
        n = np.arange(N)
        g = ((N - n + 1) * np.cos(math.pi * n / (N + 1)) +
             np.sin(math.pi * n / (N + 1)) / math.tan(math.pi / (N + 1))) / (N + 1)
        c = c * g
    return c, a, w


def fermi_operator_expansion(T: BlockMatrix, Sinv: BlockMatrix, pat_k: Pattern, order, mu, kT,
                             e_lo, e_hi, jackson=False) -> BlockMatrix:
    """K0 = f(S^-1 H) S^-1 by a Chebyshev expansion (setup step, not timed):
    X = (T - a I)/w, Y_0 = S^-1, Y_1 = cut(X Y_0), Y_{n+1} = 2 cut(X Y_n) - Y_{n-1},
    K0 = sum c_n Y_n, then K0 <- (K0 + K0^T)/2 (all on P_K)."""
    c, a, w = chebyshev_fermi_coeffs(order, mu, kT, e_lo, e_hi, jackson)
    Y0 = restrict(Sinv, pat_k)

    def apply_X(Y):
        TY = spgemm(T, Y, pat_k)
        return BlockMatrix(Y.bsize, pat_k, (TY.val - a * Y.val) / w, Y.voff)

    K = BlockMatrix(Y0.bsize, pat_k, c[0] * Y0.val, Y0.voff)
    if order >= 1:
        Y1 = apply_X(Y0)
        K.val = K.val + c[1] * Y1.val
        Ym, Yc = Y0, Y1
        for nn in range(2, order + 1):
            XY = apply_X(Yc)
            Yn = BlockMatrix(Yc.bsize, pat_k, 2.0 * XY.val - Ym.val, Yc.voff)
            K.val = K.val + c[nn] * Yn.val
            Ym, Yc = Yc, Yn
    # symmetrise K0 <- (K0 + K0^T)/2
    Kt = K.copy()
    rows = pat_k.rows()
    for q in range(pat_k.nnzb):
        i, j = rows[q], pat_k.col[q]
        qm = find(pat_k, j, i)
        blk = K.val[K.voff[qm]:K.voff[qm + 1]].reshape(K.bsize[j], K.bsize[i])
        Kt.val[Kt.voff[q]:Kt.voff[q + 1]] = 0.5 * (K.val[K.voff[q]:K.voff[q + 1]] + blk.T.reshape(-1))
    return Kt


# ----------------------------------------------------------------------------
# a propagation driver
# ----------------------------------------------------------------------------

@dataclass
class Params:
    r_Sinv: float = 8.0
    r_T: float = 8.0
    r_U: float = 8.0
    r_K: float = 8.0
    r_M: float = 8.0
    dt: float = 0.05
    prop: str = "em"          # "em" | "cn"
    taylor_terms: int = 6
    hot_tol: float = 1e-10
    hot_maxit: int = 100
    hot_step_iters: int = 2   # CN: Hotelling iterations per step
    kick_terms: int = 12
    field: Optional[dict] = None
    field_dir: int = 0


class Propagator:
    """Truncated-mode oracle run: setup (patterns, S^-1), kick, steps."""

    def __init__(self, sys, p: Params, hotelling_fixed: Optional[int] = None):
        self.sys = sys
        self.p = p
        bs = np.asarray(sys.bsize)
        self.bsize = bs
        pos, cell = sys.pos, sys.cell
        self.pats = {}
        for name, r in [("Sinv", p.r_Sinv), ("T", p.r_T), ("U", p.r_U), ("K", p.r_K), ("M", p.r_M),
                        ("A", max(sys.r_S, sys.r_H))]:
            self.pats[name] = self._pat(r)
        self.S = BlockMatrix(bs, Pattern(sys.s_rowptr, sys.s_col), sys.s_val.astype(np.complex128))
        hp = Pattern(sys.h_rowptr, sys.h_col)
        self.H0 = BlockMatrix(bs, hp, sys.h_val.astype(np.complex128))
        self.D = [BlockMatrix(bs, hp, d.astype(np.complex128)) for d in sys.d_val]
        self.hot = hotelling(self.S, self.pats["Sinv"], p.hot_tol, p.hot_maxit, fixed_iters=hotelling_fixed)
        self.Sinv = self.hot.X
        self.t = 0.0
        self.K = None
        self.X = None   # CN warm start
        self.U = None

    def _pat(self, r):
        key = float(r)
        if not hasattr(self, "_pcache"):
            self._pcache = {}
        if key not in self._pcache:
            self._pcache[key] = pattern(self.sys.pos, self.sys.cell, r)
        return self._pcache[key]

    def set_density_dense(self, K0_dense):
        self.K = from_dense(self.bsize, self.pats["K"], np.asarray(K0_dense, dtype=np.complex128))

    def set_density(self, K: BlockMatrix):
        self.K = restrict(K, self.pats["K"])

    def kick(self, direction: int, kappa: float):
        """K(0+) = V K0 V^dagger, V = exp(+i kappa S^-1 D_j) (delta-kick of
        strength kappa: H = H0 - kappa delta(t) D_j), Taylor series with
        kick_terms terms, powers cut to r_U."""
        TD = spgemm(self.Sinv, self.D[direction], self.pats["T"])
        V, _ = taylor_em(TD, -kappa, self.p.kick_terms, self.pats["U"])
        self.K, _ = sandwich(V, self.K, self.pats["M"])

    def ground_state(self, order, mu, kT, e_lo, e_hi, jackson=False):
        T0 = spgemm(self.Sinv, self.H0, self.pats["T"])
        self.K = fermi_operator_expansion(T0, self.Sinv, self.pats["K"], order, mu, kT, e_lo, e_hi, jackson)

    def _T(self, t):
        """T(t) = cut_{r_T}(S^-1 H(t))."""
        H = hamiltonian(self.H0, self.D[self.p.field_dir], field_value(self.p.field, t))
        return spgemm(self.Sinv, H, self.pats["T"])

    def propagator(self, t):
        """U for [t, t+dt]: eq. EM (H at the midpoint t + dt/2), the CN form,
        ETRS or the fourth-order Magnus form (Sec. II.A)."""
        p = self.p
        E = field_value(p.field, t + 0.5 * p.dt)
        Hm = hamiltonian(self.H0, self.D[p.field_dir], E)
        info = {"iters": 0, "resid": 0.0}
        if p.prop == "etrs":
            Ua, _ = taylor_em(self._T(t), 0.5 * p.dt, p.taylor_terms, self.pats["U"])
            Ub, _ = taylor_em(self._T(t + p.dt), 0.5 * p.dt, p.taylor_terms, self.pats["U"])
            self.U = spgemm(Ub, Ua, self.pats["U"])
            return self.U, info
        if p.prop == "m4":
            r3 = math.sqrt(3.0)
            T1 = self._T(t + (0.5 - r3 / 6.0) * p.dt)
            T2 = self._T(t + (0.5 + r3 / 6.0) * p.dt)
            pu = self.pats["U"]
            comm = axpy(-1.0, spgemm(T1, T2, pu), spgemm(T2, T1, pu))  # [T2, T1]
            Msum = axpy(1.0, restrict(T1, pu), restrict(T2, pu))
            Om = BlockMatrix(T1.bsize, pu, -0.5j * p.dt * Msum.val - (r3 * p.dt * p.dt / 12.0) * comm.val, Msum.voff)
            U = identity(T1.bsize, pu)
            P = Om
            for n in range(1, p.taylor_terms):
                if n > 1:
                    P = spgemm(Om, P, pu)
                U = axpy(1.0 / math.factorial(n), P, U)
            self.U = U
            return U, info
        if p.prop == "em":
            T = spgemm(self.Sinv, Hm, self.pats["T"])
            U, _ = taylor_em(T, p.dt, p.taylor_terms, self.pats["U"])
        else:
            pa = self.pats["A"]
            Sa = restrict(self.S, pa)
            Ha = restrict(Hm, pa)
            A = axpy(0.5j * p.dt, Ha, Sa)
            B = axpy(-0.5j * p.dt, Ha, Sa)
            X = self.X if self.X is not None else restrict(self.Sinv, self.pats["U"])
            res = 0.0
            for _ in range(p.hot_step_iters):
                Y = spgemm(A, X, self.pats["U"])
                res = residual_I_minus(Y)
                Z = axpy(-1.0, Y, identity(self.bsize, self.pats["U"], 2.0))
                X = spgemm(X, Z, self.pats["U"])
            self.X = X
            U = spgemm(X, B, self.pats["U"])
            info = {"iters": p.hot_step_iters, "resid": res}
        self.U = U
        return U, info

    def step(self, rebuild=True):
        info = {"iters": 0, "resid": 0.0}
        if rebuild or self.U is None:
            _, info = self.propagator(self.t)
        self.K, herm = sandwich(self.U, self.K, self.pats["M"])
        self.t += self.p.dt
        obs = observables(self.K, self.S, self.D)
        return {"t": self.t, "obs": obs, "herm": herm, **info}
