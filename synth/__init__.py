"""Seeded synthetic inputs for the density-matrix RT-TDDFT step.

This module makes the *inputs* of the method and nothing else: atom
positions, the non-orthogonal overlap S, a tight-binding Hamiltonian H0 and
the position-operator matrices D_x, D_y, D_z, all in atom-blocked
block-CSR form, plus (for small cells) a reference ground-state density
from a dense generalised diagonalisation.  It holds none of the
propagation arithmetic (no truncated products, no propagators, no
observables), so both the CPU oracle and the CUDA path can take their
inputs from here without sharing method code.

Units: positions, cell lengths and cut-off radii in Angstrom; integrals,
energies and time in atomic units (bohr, hartree).

Model (synthetic stand-in for the paper's PAO bases, Sec. III / Sec. V):
  * diamond lattice, a = 5.43 A, 8 atoms per conventional cell, Gaussian
    jitter per coordinate, positions wrapped into the periodic cell;
  * 4-function atoms: one s and one p shell (a minimal sp basis);
    13-function atoms: two s, two p and one d shell (5 real harmonics);
    1-function atoms (cluster hydrogen): one s shell;
  * S: overlaps of normalised Cartesian Gaussians (Obara-Saika recursion),
    d shells transformed to the 5 real solid harmonics;
  * H0: off-site Wolfsberg-Helmholz  H_ij = K/2 (e_a + e_b) S_ij exp(-R/lam);
    on-site diag(e_a) plus seeded symmetric noise;
  * D_x,y,z: first-moment integrals;  in a periodic cell each pair's moment
    is taken about the wrapped midpoint of the pair (hermitian sawtooth);
  * periodic cells use Gamma-point folding: a block sums every image of
    atom j within the radius; a block exists iff the minimum-image distance
    is below the radius (strict inequality).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

BOHR_PER_ANG = 1.0 / 0.529177210903
A_DIAMOND = 5.43

# Shell tables: list of (l, exponent in bohr^-2); energies per shell (Ha).
# sp valence shells; the 13-function basis adds a compact second s/p pair and a
# d shell.  The parameters are synthetic, chosen for (i) a gapped spectrum at
# valence filling (2 doubly occupied states per atom, which is half filling
# for the 4-function basis), (ii) a well-conditioned S whose inverse is short
# ranged at the 6-12 A radii used, (iii) dt * spectral radius << 1.
SPECIES = {
    "sp4": dict(shells=[(0, 0.30), (1, 0.30)], eps=[-0.45, -0.35]),
    "spd13": dict(shells=[(0, 0.30), (1, 0.30), (0, 1.20), (1, 1.20), (2, 0.80)],
                  eps=[-0.60, -0.35, 0.00, 0.20, 0.30]),
    "h1": dict(shells=[(0, 0.35)], eps=[-0.40]),
}
# Wolfsberg-Helmholz constant: larger than the textbook 1.75 so that the compact
# (well-conditioned, short-ranged S^-1) Gaussians still give a gapped sp3 spectrum.
K_WH = 3.5
LAMBDA_WH = None  # optional extra exp(-R/lambda) damping of H (bohr); None = off
ONSITE_NOISE = 0.1  # Ha, uniform +- on the diagonal of each on-site block


def _cart_list(l):
    if l == 0:
        return [(0, 0, 0)]
    if l == 1:
        return [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    if l == 2:
        return [(2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0), (1, 0, 1), (0, 1, 1)]
    raise ValueError(l)


# Cartesian d (xx, yy, zz, xy, xz, yz) -> 5 real harmonics (xy, xz, yz,
# x^2-y^2, 2z^2-x^2-y^2); overall scale is fixed later by normalisation.
_D_SPH = np.array([
    [0, 0, 0, 1, 0, 0],
    [0, 0, 0, 0, 1, 0],
    [0, 0, 0, 0, 0, 1],
    [1, -1, 0, 0, 0, 0],
    [-1, -1, 2, 0, 0, 0],
], dtype=np.float64)


def _overlap_1d(alpha, beta, xa, xb, la, lb):
    """1D Obara-Saika overlap table E[i][j] for i <= la, j <= lb (vectorised).

    alpha, beta scalars; xa, xb arrays (bohr).  Returns list of lists of arrays.
    """
    p = alpha + beta
    mu = alpha * beta / p
    xab = xa - xb
    xp = (alpha * xa + beta * xb) / p
    xpa = xp - xa
    xpb = xp - xb
    s00 = math.sqrt(math.pi / p) * np.exp(-mu * xab * xab)
    E = [[None] * (lb + 1) for _ in range(la + 1)]
    E[0][0] = s00
    inv2p = 0.5 / p
    for i in range(la + 1):
        for j in range(lb + 1):
            if i == 0 and j == 0:
                continue
            if i > 0:
                v = xpa * E[i - 1][j]
                if i > 1:
                    v = v + (i - 1) * inv2p * E[i - 2][j]
                if j > 0:
                    v = v + j * inv2p * E[i - 1][j - 1]
            else:
                v = xpb * E[i][j - 1]
                if j > 1:
                    v = v + (j - 1) * inv2p * E[i][j - 2]
            E[i][j] = v
    return E


@dataclasses.dataclass
class Basis:
    name: str
    shells: list            # [(l, alpha)]
    eps_func: np.ndarray    # on-site energy per final function
    ncart: int
    nfunc: int
    cart_index: list        # per shell: (offset in cart list, l)
    transform: np.ndarray   # nfunc x ncart (spherical transform * normalisation)


def make_basis(name: str) -> Basis:
    spec = SPECIES[name]
    shells = spec["shells"]
    cart_index = []
    ncart = 0
    rows = []
    eps = []
    nf = 0
    for (l, a), e in zip(shells, spec["eps"]):
        cart_index.append((ncart, l))
        nc = len(_cart_list(l))
        if l < 2:
            for c in range(nc):
                r = np.zeros(0)
                rows.append((ncart + c, None))
            nf += nc
            eps += [e] * nc
        else:
            for k in range(5):
                rows.append((ncart, _D_SPH[k]))
            nf += 5
            eps += [e] * 5
        ncart += nc
    T = np.zeros((nf, ncart))
    for f, (off, vec) in enumerate(rows):
        if vec is None:
            T[f, off] = 1.0
        else:
            T[f, off:off + 6] = vec
    b = Basis(name, shells, np.array(eps), ncart, nf, cart_index, T)
    # normalise: on-site self overlap of each final function is 1
    Sc = _cart_block(b, b, np.zeros((1, 3)), np.zeros((1, 3)))[0][0]
    d = np.einsum("fa,ab,fb->f", T, Sc, T)
    b.transform = T / np.sqrt(d)[:, None]
    return b


def _cart_block(ba: Basis, bb: Basis, A, B, moment_about=None):
    """Cartesian overlap blocks [npair, ncart_a, ncart_b] between atoms at A, B (bohr).

    With moment_about=C (array [npair,3]) also returns the three first-moment
    blocks <a|(x_d - C_d)|b>.
    """
    npair = A.shape[0]
    S = np.zeros((npair, ba.ncart, bb.ncart))
    M = np.zeros((3, npair, ba.ncart, bb.ncart)) if moment_about is not None else None
    for (oa, la), (_, alpha) in zip(ba.cart_index, ba.shells):
        for (ob, lb), (_, beta) in zip(bb.cart_index, bb.shells):
            extra = 1 if moment_about is not None else 0
            E = [_overlap_1d(alpha, beta, A[:, d], B[:, d], la, lb + extra) for d in range(3)]
            ca = _cart_list(la)
            cb = _cart_list(lb)
            for ia, pa in enumerate(ca):
                for ib, pb in enumerate(cb):
                    ex = E[0][pa[0]][pb[0]]
                    ey = E[1][pa[1]][pb[1]]
                    ez = E[2][pa[2]][pb[2]]
                    S[:, oa + ia, ob + ib] = ex * ey * ez
                    if M is not None:
                        comps = (ex, ey, ez)
                        for d in range(3):
                            # x - C = (x - B) + (B - C):  E[i][j+1] + (B-C) E[i][j]
                            mom = E[d][pa[d]][pb[d] + 1] + (B[:, d] - moment_about[:, d]) * comps[d]
                            prod = mom
                            for e in range(3):
                                if e != d:
                                    prod = prod * comps[e]
                            M[d, :, oa + ia, ob + ib] = prod
    return S, M


def min_image_d2(xi, xj, cell):
    """Minimum-image squared distance (Angstrom^2), evaluated term by term.

    dx = xj - xi; dx -= L * rint(dx / L); d2 = (dx*dx + dy*dy) + dz*dz.
    Each operation is a separately rounded IEEE double operation.
    """
    d2 = None
    for d in range(3):
        dx = xj[..., d] - xi[..., d]
        if cell is not None:
            L = cell[d]
            dx = dx - L * np.rint(dx / L)
        t = dx * dx
        d2 = t if d2 is None else d2 + t
    return d2


@dataclasses.dataclass
class System:
    """One synthetic system in atom-blocked block-CSR form (host arrays)."""
    n_atoms: int
    pos: np.ndarray            # [n,3] Angstrom, wrapped into the cell
    cell: Optional[np.ndarray]  # [3] Angstrom or None (open)
    bsize: np.ndarray          # [n] int32 functions per atom
    r_S: float
    r_H: float
    s_rowptr: np.ndarray
    s_col: np.ndarray
    s_val: np.ndarray          # concatenated row-major blocks
    h_rowptr: np.ndarray
    h_col: np.ndarray
    h_val: np.ndarray
    d_val: list                # three arrays on the H pattern
    eps_func: np.ndarray       # on-site energies per function (diagnostic)
    species: list

    @property
    def n(self):
        return int(self.bsize.sum())

    @property
    def foff(self):
        return np.concatenate([[0], np.cumsum(self.bsize)]).astype(np.int64)

    def block_offsets(self, rowptr, col):
        """Value offset of each block of a pattern with this system's block sizes."""
        rows = np.repeat(np.arange(self.n_atoms), np.diff(rowptr))
        sz = self.bsize[rows].astype(np.int64) * self.bsize[col].astype(np.int64)
        return np.concatenate([[0], np.cumsum(sz)])

    def to_dense(self, which: str):
        """Dense n x n matrix of S, H or Dx/Dy/Dz (for small tests)."""
        if which == "S":
            rp, cl, v = self.s_rowptr, self.s_col, self.s_val
        else:
            rp, cl = self.h_rowptr, self.h_col
            v = {"H": self.h_val, "Dx": self.d_val[0], "Dy": self.d_val[1], "Dz": self.d_val[2]}[which]
        return blocks_to_dense(self.bsize, rp, cl, v)


def blocks_to_dense(bsize, rowptr, col, val, dtype=np.float64):
    bsize = np.asarray(bsize)
    foff = np.concatenate([[0], np.cumsum(bsize)])
    n = int(foff[-1])
    out = np.zeros((n, n), dtype=dtype)
    o = 0
    for i in range(len(bsize)):
        for q in range(rowptr[i], rowptr[i + 1]):
            j = col[q]
            bi, bj = bsize[i], bsize[j]
            out[foff[i]:foff[i] + bi, foff[j]:foff[j] + bj] = val[o:o + bi * bj].reshape(bi, bj)
            o += bi * bj
    return out


def dense_to_blocks(bsize, rowptr, col, dense):
    bsize = np.asarray(bsize)
    foff = np.concatenate([[0], np.cumsum(bsize)])
    parts = []
    for i in range(len(bsize)):
        for q in range(rowptr[i], rowptr[i + 1]):
            j = col[q]
            parts.append(dense[foff[i]:foff[i] + bsize[i], foff[j]:foff[j] + bsize[j]].reshape(-1))
    if not parts:
        return np.zeros(0, dtype=dense.dtype)
    return np.concatenate(parts)


# ----------------------------------------------------------------------------
# geometry
# ----------------------------------------------------------------------------

def _morton_sort(pos: np.ndarray, L: float, bits: int = 10) -> np.ndarray:
    """Atoms reordered along a Morton (Z-order) curve over the periodic cube of
    side L: coordinates quantised to 2^bits steps, bits interleaved x, y, z."""
    q = np.clip((pos / L * (1 << bits)).astype(np.int64), 0, (1 << bits) - 1)
    code = np.zeros(len(pos), dtype=np.int64)
    for b in range(bits):
        for d in range(3):
            code |= ((q[:, d] >> b) & 1) << (3 * b + d)
    return pos[np.argsort(code, kind="stable")]


def diamond_positions(ncell: int, a: float = A_DIAMOND, jitter: float = 0.05, seed: int = 0,
                      order: str = "lattice"):
    """ncell^3 conventional diamond cells (8 atoms each), seeded jitter, wrapped.

    order "lattice": cell by cell (z fastest), the 8 basis atoms of a cell in
    turn; "morton": the same atoms sorted along a Morton curve (spatially
    compact runs of atoms, as a linear-scaling code orders its partitions)."""
    basis = np.array([
        [0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0],
        [.25, .25, .25], [.25, .75, .75], [.75, .25, .75], [.75, .75, .25],
    ])
    g = np.arange(ncell)
    cx, cy, cz = np.meshgrid(g, g, g, indexing="ij")
    cells = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)
    pos = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    rng = np.random.default_rng(seed)
    pos = pos + rng.normal(0.0, jitter, size=pos.shape)
    L = ncell * a
    pos = np.mod(pos, L)
    pos[pos >= L] -= L
    if order == "morton":
        pos = _morton_sort(pos, L)
    elif order != "lattice":
        raise ValueError(f"unknown atom order {order!r}")
    return pos, np.array([L, L, L], dtype=np.float64)


def si_h_cluster(target: int = 1200, a: float = A_DIAMOND, seed: int = 2, bond_h: float = 1.48):
    """Sphere cut from diamond Si, dangling bonds H-terminated (open system).

    Returns positions (Angstrom, shifted to be non-negative), species list.
    """
    nn = a * math.sqrt(3) / 4
    basis = np.array([
        [0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0],
        [.25, .25, .25], [.25, .75, .75], [.75, .25, .75], [.75, .75, .25],
    ])
    m = 8
    g = np.arange(-m, m)
    cx, cy, cz = np.meshgrid(g, g, g, indexing="ij")
    cells = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)
    lat = ((cells[:, None, :] + basis[None]) * a).reshape(-1, 3)
    centre = np.array([0.1, 0.2, 0.3]) * a
    dist = np.linalg.norm(lat - centre, axis=1)
    order = np.argsort(dist)
    best = None
    for rad in np.linspace(6.0, 20.0, 281):
        si = lat[dist < rad]
        # bonds to missing neighbours
        dmat = np.linalg.norm(si[:, None, :] - si[None, :, :], axis=2) if len(si) < 1500 else None
        if dmat is None:
            break
        nb = ((dmat > 0.1) & (dmat < nn * 1.1)).sum(1)
        keep = nb >= 2  # drop nearly isolated atoms
        si = si[keep]
        dmat = dmat[np.ix_(keep, keep)]
        nb = ((dmat > 0.1) & (dmat < nn * 1.1)).sum(1)
        tot = len(si) + int((4 - nb).sum())
        if best is None or abs(tot - target) < abs(best[0] - target):
            best = (tot, rad)
    rad = best[1]
    si = lat[dist < rad]
    dmat = np.linalg.norm(si[:, None, :] - si[None, :, :], axis=2)
    nb = ((dmat > 0.1) & (dmat < nn * 1.1)).sum(1)
    keep = nb >= 2
    si = si[keep]
    siset = {tuple(np.round(p, 6)) for p in si}
    # tetrahedral bond directions per sublattice
    dirs_a = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]]) / math.sqrt(3)
    hs = []
    for p in si:
        frac = np.mod(p / a, 1.0)
        # sublattice B sits at +(1/4,1/4,1/4) from an fcc site
        onB = np.any(np.all(np.abs(np.mod(frac - 0.25, 0.5)) < 1e-6, axis=-1)) if False else None
        for sgn in (1.0, -1.0):
            pass
        # find missing neighbours explicitly
        cands = []
        for sgn in (1.0, -1.0):
            for d in dirs_a:
                q = p + sgn * d * nn
                cands.append((sgn, d, q))
        for sgn, d, q in cands:
            # a true lattice neighbour exists at q if q is a lattice point
            fq = q / a
            isl = np.any(np.linalg.norm(lat - q, axis=1) < 1e-6)
            if not isl:
                continue
            if tuple(np.round(q, 6)) in siset:
                continue
            hs.append(p + sgn * d * bond_h)
    hs = np.array(hs)
    rng = np.random.default_rng(seed)
    pos = np.concatenate([si, hs])
    pos = pos + rng.normal(0.0, 0.02, size=pos.shape)
    pos = pos - pos.min(0) + 1.0
    species = ["sp4"] * len(si) + ["h1"] * len(hs)
    return pos, species


# ----------------------------------------------------------------------------
# pair lists and integrals
# ----------------------------------------------------------------------------

def _neighbour_pairs(pos, cell, r):
    """All (i, j) with minimum-image distance < r, i <= j, as arrays (cell lists)."""
    n = len(pos)
    r2 = r * r
    if cell is None:
        lo = pos.min(0)
        span = pos.max(0) - lo + 1e-9
        nb = np.maximum(1, np.floor(span / r).astype(int))
        binsz = span / nb
    else:
        nb = np.maximum(1, np.floor(cell / r).astype(int))
        lo = np.zeros(3)
        binsz = cell / nb
    idx = np.minimum(np.floor((pos - lo) / binsz).astype(int), nb - 1)
    lin = (idx[:, 0] * nb[1] + idx[:, 1]) * nb[2] + idx[:, 2]
    order = np.argsort(lin, kind="stable")
    start = np.searchsorted(lin[order], np.arange(nb.prod() + 1))
    I, J = [], []
    offs = []
    rngs = [range(-1, 2) if nb[d] >= 3 else range(0, nb[d]) for d in range(3)]
    seen_bins = set()
    for ox in (range(-1, 2) if nb[0] >= 3 else [None]):
        for oy in (range(-1, 2) if nb[1] >= 3 else [None]):
            for oz in (range(-1, 2) if nb[2] >= 3 else [None]):
                offs.append((ox, oy, oz))
    for b in range(nb.prod()):
        bx, by, bz = b // (nb[1] * nb[2]), (b // nb[2]) % nb[1], b % nb[2]
        ai = order[start[b]:start[b + 1]]
        if len(ai) == 0:
            continue
        nbrs = set()
        for ox, oy, oz in offs:
            xs = [bx + ox] if ox is not None else list(range(nb[0]))
            ys = [by + oy] if oy is not None else list(range(nb[1]))
            zs = [bz + oz] if oz is not None else list(range(nb[2]))
            for x in xs:
                for y in ys:
                    for z in zs:
                        if cell is None:
                            if not (0 <= x < nb[0] and 0 <= y < nb[1] and 0 <= z < nb[2]):
                                continue
                        x2, y2, z2 = x % nb[0], y % nb[1], z % nb[2]
                        nbrs.add((x2 * nb[1] + y2) * nb[2] + z2)
        aj = np.concatenate([order[start[c]:start[c + 1]] for c in sorted(nbrs)])
        d2 = min_image_d2(pos[ai][:, None, :], pos[aj][None, :, :], cell)
        m = (d2 < r2) & (ai[:, None] <= aj[None, :])
        ii, jj = np.nonzero(m)
        I.append(ai[ii])
        J.append(aj[jj])
    I = np.concatenate(I) if I else np.zeros(0, int)
    J = np.concatenate(J) if J else np.zeros(0, int)
    o = np.lexsort((J, I))
    return I[o], J[o]


def _image_shifts(pos, cell, I, J, r):
    """For each pair (i,j) the list of image displacement vectors within r (Angstrom).

    Returns (pair_index, disp[3]) arrays over all contributing images.
    """
    dx0 = pos[J] - pos[I]
    if cell is None:
        return np.arange(len(I)), dx0
    pidx, disp = [], []
    r2 = r * r
    for nx in (-1, 0, 1):
        for ny in (-1, 0, 1):
            for nz in (-1, 0, 1):
                d = dx0 + np.array([nx, ny, nz]) * cell
                d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
                m = d2 < r2
                pidx.append(np.nonzero(m)[0])
                disp.append(d[m])
    pidx = np.concatenate(pidx)
    disp = np.concatenate(disp)
    return pidx, disp


def _pair_blocks(basis_i: Basis, basis_j: Basis, pos_i_bohr, disp_bohr, mids_wrapped_bohr, want_d):
    """Final (spherical, normalised) S and D blocks for pairs i->j with displacement."""
    A = pos_i_bohr
    B = pos_i_bohr + disp_bohr
    C = A + 0.5 * disp_bohr
    Sc, Mc = _cart_block(basis_i, basis_j, A, B, moment_about=C if want_d else None)
    Ti, Tj = basis_i.transform, basis_j.transform
    S = np.einsum("fa,pab,gb->pfg", Ti, Sc, Tj, optimize=True)
    D = None
    if want_d:
        D = []
        for d in range(3):
            Md = np.einsum("fa,pab,gb->pfg", Ti, Mc[d], Tj, optimize=True)
            if mids_wrapped_bohr is not None:
                Md = Md + mids_wrapped_bohr[:, d][:, None, None] * S
            D.append(Md)
    return S, D


def build_system(pos, cell, species: Sequence[str], r_S: float, r_H: float,
                 noise_seed: int = 1, chunk: int = 20000) -> System:
    """Build S, H0, D on block-CSR patterns P_{r_S} (S) and P_{r_H} (H, D)."""
    pos = np.asarray(pos, dtype=np.float64)
    n = len(pos)
    species = list(species)
    bases = {s: make_basis(s) for s in set(species)}
    bsize = np.array([bases[s].nfunc for s in species], dtype=np.int32)
    r_max = max(r_S, r_H)
    if cell is not None and r_max >= float(np.min(cell)):
        raise ValueError("radius must be below the cell length for +-1 image folding")
    I, J = _neighbour_pairs(pos, cell, r_max)
    d2 = min_image_d2(pos[I], pos[J], cell)
    pidx, disp = _image_shifts(pos, cell, I, J, r_max)
    # per-image S and D
    eps_all = {s: bases[s].eps_func for s in bases}
    # group pairs by species combination
    spec_arr = np.array(species)
    S_pairs = {}
    D_pairs = {}
    Hoff_pairs = {}
    rng = np.random.default_rng(noise_seed)
    noise = {}
    # on-site noise blocks (symmetric), drawn in atom order
    for i in range(n):
        b = bsize[i]
        noise[i] = np.diag(rng.uniform(-ONSITE_NOISE, ONSITE_NOISE, size=b))
    dist_img = np.sqrt((disp * disp).sum(1)) * BOHR_PER_ANG
    mids = None
    if cell is not None:
        m = pos[I[pidx]] + 0.5 * disp
        m = np.mod(m, cell)
        mids = m * BOHR_PER_ANG
    img_r2 = (disp[:, 0] * disp[:, 0] + disp[:, 1] * disp[:, 1]) + disp[:, 2] * disp[:, 2]
    npair = len(I)
    Sblk = [None] * npair
    Hblk = [None] * npair
    Dblk = [[None] * npair for _ in range(3)]
    for si in bases:
        for sj in bases:
            sel = np.nonzero((spec_arr[I[pidx]] == si) & (spec_arr[J[pidx]] == sj))[0]
            if len(sel) == 0:
                continue
            bi, bj = bases[si], bases[sj]
            for c0 in range(0, len(sel), chunk):
                s = sel[c0:c0 + chunk]
                A = pos[I[pidx[s]]] * BOHR_PER_ANG
                Dv = disp[s] * BOHR_PER_ANG
                mw = mids[s] if mids is not None else None
                Sb, Db = _pair_blocks(bi, bj, A, Dv, mw, True)
                if cell is None:
                    # open system: moment about the origin
                    Sc, Mc = _cart_block(bi, bj, A, A + Dv, moment_about=np.zeros_like(A))
                    Db = [np.einsum("fa,pab,gb->pfg", bi.transform, Mc[d], bj.transform, optimize=True)
                          for d in range(3)]
                ea = bi.eps_func[None, :, None]
                eb = bj.eps_func[None, None, :]
                decay = 1.0 if LAMBDA_WH is None else np.exp(-dist_img[s] / LAMBDA_WH)[:, None, None]
                Hb = 0.5 * K_WH * (ea + eb) * Sb * decay
                inS = img_r2[s] < r_S * r_S
                inH = img_r2[s] < r_H * r_H
                for t, p in enumerate(pidx[s]):
                    if inS[t]:
                        Sblk[p] = Sb[t] if Sblk[p] is None else Sblk[p] + Sb[t]
                    if inH[t]:
                        is_self = (I[p] == J[p]) and np.all(np.abs(disp[s[t]]) < 1e-12)
                        h = Hb[t]
                        if is_self:
                            # on-site: 1/2 (e_a + e_b) S_ab (diagonal e_a) plus noise
                            h = 0.5 * (bi.eps_func[:, None] + bi.eps_func[None, :]) * Sb[t] + noise[I[p]]
                        Hblk[p] = h if Hblk[p] is None else Hblk[p] + h
                        for d in range(3):
                            Dblk[d][p] = Db[d][t] if Dblk[d][p] is None else Dblk[d][p] + Db[d][t]
    # assemble symmetric block-CSR on both patterns (mirror i<j blocks)
    def assemble(radius, blocks_list):
        keep = d2 < radius * radius
        ii, jj = I[keep], J[keep]
        idx = np.nonzero(keep)[0]
        rows = np.concatenate([ii, jj[ii != jj]])
        cols = np.concatenate([jj, ii[ii != jj]])
        src = np.concatenate([idx, idx[ii != jj]])
        tr = np.concatenate([np.zeros(len(ii), bool), np.ones(int((ii != jj).sum()), bool)])
        o = np.lexsort((cols, rows))
        rows, cols, src, tr = rows[o], cols[o], src[o], tr[o]
        rowptr = np.zeros(n + 1, dtype=np.int32)
        np.add.at(rowptr, rows + 1, 1)
        rowptr = np.cumsum(rowptr).astype(np.int32)
        outs = []
        for blocks in blocks_list:
            parts = []
            for p, t in zip(src, tr):
                b = blocks[p]
                if b is None:
                    b = np.zeros((bsize[I[p]], bsize[J[p]]))
                elif I[p] == J[p]:
                    b = 0.5 * (b + b.T)  # exact symmetry of on-site blocks
                parts.append((b.T if t else b).reshape(-1))
            outs.append(np.concatenate(parts) if parts else np.zeros(0))
        return rowptr, cols.astype(np.int32), outs

    s_rowptr, s_col, (s_val,) = assemble(r_S, [Sblk])
    h_rowptr, h_col, (h_val, dx, dy, dz) = assemble(r_H, [Hblk] + Dblk)
    eps_func = np.concatenate([bases[s].eps_func for s in species])
    return System(n, pos, None if cell is None else np.asarray(cell, float), bsize, r_S, r_H,
                  s_rowptr, s_col, s_val, h_rowptr, h_col, h_val, [dx, dy, dz], eps_func, species)


def diamond_system(ncell: int, basis: str = "sp4", r_S: float = 6.0, r_H: float = 6.0,
                   jitter: float = 0.05, seed: int = 0, noise_seed: int = 1, order: str = "lattice") -> System:
    pos, cell = diamond_positions(ncell, jitter=jitter, seed=seed, order=order)
    return build_system(pos, cell, [basis] * len(pos), r_S, r_H, noise_seed=noise_seed)


def ground_state_dense(sys: System, n_occ: int):
    """Reference ground state by dense generalised diagonalisation (small cells only).

    Returns (K0 dense n x n, eigenvalues, gap): K0 = C_occ C_occ^T with C^T S C = I,
    so Tr(K0 S) = n_occ.
    """
    import scipy.linalg as sl
    S = sys.to_dense("S")
    H = sys.to_dense("H")
    w, C = sl.eigh(H, S)
    Co = C[:, :n_occ]
    K0 = Co @ Co.T
    gap = float(w[n_occ] - w[n_occ - 1]) if n_occ < len(w) else float("nan")
    return K0, w, gap
