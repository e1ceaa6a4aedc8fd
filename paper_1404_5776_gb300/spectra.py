"""Optical spectra from the recorded dipole (paper Sec. II.B, linear response).

Post-processing of the observables that rt_step records (host side, numpy):

  alpha_ij(w) = int dt e^{iwt} P_i(t) / int dt e^{iwt} E_j(t)
  S(w)        = (2 w / pi) Im( (1/3) Tr alpha(w) )
  f-sum       = int_0^inf S(w) dw

For a delta kick E_j(t) = kappa delta(t) the denominator is kappa.  The
response signal is the change of Tr(K D_i) after the kick (the library returns
Tr(K D) without the electron charge and spin factor, which scale alpha and the
f-sum by the same constant).  A damping exp(-gamma t) turns the finite record
into Lorentzian lines of half width gamma.
"""
from __future__ import annotations

import numpy as np


def polarizability(t, dP, kappa, omegas, damping=0.0, E=None):
    """alpha(w) for each w in `omegas` from samples dP(t) = P(t) - P(0).

    t: sample times (uniform spacing, starting one step after the kick);
    dP: response samples; kappa: kick strength (used when E is None);
    E: field samples at t (then alpha = FT[P] / FT[E] on the same grid).
    The integral is the trapezoid rule on [0, t_max] with dP(0) = 0.
    """
    t = np.asarray(t, dtype=float)
    dP = np.asarray(dP, dtype=float)
    omegas = np.asarray(omegas, dtype=float)
    tt = np.concatenate([[0.0], t])
    pp = np.concatenate([[0.0], dP]) * np.exp(-damping * tt)
    phase = np.exp(1j * np.outer(omegas, tt))
    num = np.trapezoid(phase * pp[None, :], tt, axis=1)
    if E is None:
        return num / kappa
    ee = np.concatenate([[0.0], np.asarray(E, dtype=float)]) * np.exp(-damping * tt)
    den = np.trapezoid(phase * ee[None, :], tt, axis=1)
    return num / den


def strength_function(omegas, alphas):
    """S(w) = (2w/pi) Im((1/3) sum_j alpha_jj(w)); `alphas` = [alpha_xx, alpha_yy, alpha_zz]
    (missing directions may be passed as zeros, keeping the 1/3)."""
    omegas = np.asarray(omegas, dtype=float)
    tr = sum(np.asarray(a) for a in alphas) / 3.0
    return 2.0 * omegas / np.pi * tr.imag


def f_sum(omegas, S):
    """int S(w) dw over the sampled frequencies (trapezoid rule)."""
    return float(np.trapezoid(np.asarray(S, dtype=float), np.asarray(omegas, dtype=float)))


def peaks(omegas, S, n=5):
    """Frequencies of the n largest local maxima of S."""
    S = np.asarray(S)
    idx = [i for i in range(1, len(S) - 1) if S[i] > S[i - 1] and S[i] >= S[i + 1]]
    idx.sort(key=lambda i: -S[i])
    return np.asarray(omegas)[idx[:n]]
