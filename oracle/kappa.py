"""FP64 absorption-coefficient table, Eq. (tau) of Section 3 (test infrastructure).

kappa(nu_j, T) = u(T) * sum over lines l with |nu_j - nu0_l| <= cutoff of
                 S_l(T) * f_l(nu_j - nu0_l; T)                          [cm^-1]

with a single absorbing gas, u the ideal-gas number density at the table's
(p_ref, x_ref), S_l(T) from Eq. (S) and f the Lorentz or Voigt shape.  The
spectral grid is nu_j = nu_min + j * dnu evaluated in float64, and the cutoff
test |nu_j - nu0| <= cutoff is applied in float64 exactly as written (edge
inclusive, no renormalisation of the truncated profile, no pedestal).

Parity: pinned (single-line area against closed forms, superposition over
lines, direct evaluation at each temperature node).
"""
from __future__ import annotations

import numpy as np

from . import physics as ph


def grid_nu(spec, js):
    """nu_j = nu_min + j * dnu in float64 (the grid the cutoff test uses)."""
    return spec.nu_min + np.asarray(js, dtype=np.int64).astype(np.float64) * spec.dnu


def line_terms(lines, T, p_atm, x, profile):
    """Per-line factors at one temperature: (u * S(T), gamma_L, alpha_D)."""
    S = ph.line_intensity(lines.S_ref, lines.nu0, lines.E_lower, T, lines.T_ref, lines.q_exp)
    A = ph.number_density(x, p_atm, T) * S
    g = ph.lorentz_hwhm(lines.gamma_ref, p_atm, T, lines.T_ref, lines.n_T)
    a = ph.doppler_hwhm(lines.nu0, T, lines.mass_amu) if profile == "voigt" else None
    return A, g, a


def _fixed_window(lines, spec):
    """Fixed points per line: j = jf - n/2 + 1 .. jf + n/2, jf = floor((nu0 - nu_min)/dnu)."""
    n = int(spec.points_per_line)
    jf = np.floor((lines.nu0 - spec.nu_min) / spec.dnu).astype(np.int64)
    lo = np.maximum(jf - n // 2 + 1, 0)
    hi = np.minimum(jf + n // 2, spec.n_nu - 1)
    return lo, hi


def _pairs(lines, spec, js):
    """All (column, line) pairs with |nu_j - nu0| <= cutoff, exact float64 test
    (or, with points_per_line > 0, the fixed window of each line)."""
    if getattr(spec, "points_per_line", 0) > 0:
        lo, hi = _fixed_window(lines, spec)
        js = np.asarray(js, dtype=np.int64)
        col_l, lid_l = [], []
        for i, j in enumerate(js):
            ls = np.nonzero((lo <= j) & (hi >= j))[0]
            col_l.append(np.full(ls.size, i, dtype=np.int64))
            lid_l.append(ls)
        col = np.concatenate(col_l) if col_l else np.zeros(0, np.int64)
        lid = np.concatenate(lid_l) if lid_l else np.zeros(0, np.int64)
        return col, lid, grid_nu(spec, js)[col] - lines.nu0[lid]
    nu_j = grid_nu(spec, js)
    slack = 1e-9 * max(1.0, abs(spec.nu_min) + spec.n_nu * spec.dnu)
    lo = np.searchsorted(lines.nu0, nu_j - spec.cutoff - slack, side="left")
    hi = np.searchsorted(lines.nu0, nu_j + spec.cutoff + slack, side="right")
    cnt = hi - lo
    col = np.repeat(np.arange(len(js)), cnt)
    start = np.repeat(lo - np.concatenate(([0], np.cumsum(cnt)[:-1])), cnt)
    lid = start + np.arange(int(cnt.sum()))
    dnu = nu_j[col] - lines.nu0[lid]
    keep = np.abs(dnu) <= spec.cutoff
    return col[keep], lid[keep], dnu[keep]


def kappa_columns(lines, spec, js, T_nodes=None, p_atm=None, x=None, chunk=512):
    """kappa[k, i] at columns js[i] and temperatures T_nodes[k] (default: the
    spec's T grid at its p_ref, x_ref).  Returns (nT, len(js)) float64."""
    js = np.asarray(js, dtype=np.int64)
    T_nodes = spec.T_nodes() if T_nodes is None else np.atleast_1d(np.asarray(T_nodes, np.float64))
    p_atm = spec.p_ref_atm if p_atm is None else p_atm
    x = spec.x_ref if x is None else x
    out = np.zeros((len(T_nodes), len(js)), dtype=np.float64)
    terms = [line_terms(lines, float(T), p_atm, x, spec.profile) for T in T_nodes]
    for c0 in range(0, len(js), chunk):
        sl = slice(c0, min(len(js), c0 + chunk))
        col, lid, dnu = _pairs(lines, spec, js[sl])
        if col.size == 0:
            continue
        n = sl.stop - sl.start
        for k, (A, g, a) in enumerate(terms):
            if spec.profile == "lorentz":
                f = ph.lorentz_profile(dnu, g[lid])
            else:
                f = ph.voigt_profile(dnu, g[lid], a[lid])
            out[k, sl] = np.bincount(col, weights=A[lid] * f, minlength=n)
    return out


def kappa_table(lines, spec, chunk=512):
    """Full table kappa[k][j], shape (nT, n_nu), float64."""
    return kappa_columns(lines, spec, np.arange(spec.n_nu), chunk=chunk)


def line_ranges(lines, spec):
    """Inclusive grid-index range [j_lo, j_hi] of each line's cutoff window,
    decided by the float64 test |nu_j - nu0| <= cutoff (empty when j_lo > j_hi)."""
    if getattr(spec, "points_per_line", 0) > 0:
        return _fixed_window(lines, spec)
    nu0 = lines.nu0
    n = spec.n_nu
    lo = np.floor((nu0 - spec.cutoff - spec.nu_min) / spec.dnu).astype(np.int64) - 1
    hi = np.ceil((nu0 + spec.cutoff - spec.nu_min) / spec.dnu).astype(np.int64) + 1
    lo = np.clip(lo, 0, n)
    hi = np.clip(hi, -1, n - 1)

    def inc(j):
        ok = (j >= 0) & (j < n)
        return ok & (np.abs(grid_nu(spec, np.clip(j, 0, n - 1)) - nu0) <= spec.cutoff)

    for _ in range(6):
        lo = np.where((lo <= hi) & ~inc(lo), lo + 1, lo)
    for _ in range(6):
        hi = np.where((hi >= lo) & ~inc(hi), hi - 1, hi)
    return lo, hi


def profile_evals(lines, spec):
    """Exact number of (T node, line, nu_j) profile evaluations of the table."""
    lo, hi = line_ranges(lines, spec)
    return int(np.maximum(hi - lo + 1, 0).sum()) * int(spec.nT)
