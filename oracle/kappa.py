"""FP64 absorption-coefficient table, Eq. (tau) of Section 3 (test infrastructure).

kappa(nu_j, T) = u(T) * sum over lines l with |nu_j - nu0_l| <= cutoff of
                 S_l(T) * f_l(nu_j - nu0_l; T)                          [cm^-1]

with a single absorbing gas, u the ideal-gas number density at the table's
(p_ref, x_ref), S_l(T) from Eq. (S) and f the Lorentz or Voigt shape.  The
spectral grid is nu_j = nu_min + j * dnu evaluated in float64, and the cutoff
test |nu_j - nu0| <= cutoff is applied in float64 exactly as written (edge
inclusive, no renormalisation of the truncated profile, no pedestal).

With spec.kappa_min > 0 the points per line adapt to the temperature and the
line's intensity (the next version Section 4 announces: "dynamically adapt the
number of points depending on the local temperature and the intensity of the
line"; the paper gives no rule).  Reading: at T node T_k, line l is evaluated
only where its Lorentz wing reaches kappa_min,
    |nu_j - nu0_l| <= w_lk = min(cutoff, sqrt(A_lk gamma_lk / (pi kappa_min))),
A_lk = u(T_k) S_l(T_k) and gamma_lk the Lorentz half-width at T_k (the distance at
which A gamma / (pi dnu^2), the far wing of both profiles, equals kappa_min);
w_lk and the test are float64.

Parity: pinned (single-line area against closed forms, superposition over
lines, direct evaluation at each temperature node; adaptive windows: the cutoff
table as kappa_min -> 0, every dropped Lorentz term below kappa_min and every
kept one's wing at or above it, monotone in kappa_min).
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


def adaptive_halfwidth(A, gamma, spec):
    """w = min(cutoff, sqrt(A gamma / (pi kappa_min))) per line [cm^-1] (adaptive points)."""
    w = np.sqrt(A * gamma / (np.pi * spec.kappa_min))
    return np.where(w <= spec.cutoff, w, spec.cutoff)


def kappa_columns(lines, spec, js, T_nodes=None, p_atm=None, x=None, chunk=512):
    """kappa[k, i] at columns js[i] and temperatures T_nodes[k] (default: the
    spec's T grid at its p_ref, x_ref).  Returns (nT, len(js)) float64."""
    js = np.asarray(js, dtype=np.int64)
    T_nodes = spec.T_nodes() if T_nodes is None else np.atleast_1d(np.asarray(T_nodes, np.float64))
    p_atm = spec.p_ref_atm if p_atm is None else p_atm
    x = spec.x_ref if x is None else x
    out = np.zeros((len(T_nodes), len(js)), dtype=np.float64)
    terms = [line_terms(lines, float(T), p_atm, x, spec.profile) for T in T_nodes]
    adaptive = getattr(spec, "kappa_min", 0.0) > 0
    wins = [adaptive_halfwidth(A, g, spec) for A, g, _ in terms] if adaptive else None
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
            wt = A[lid] * f
            if adaptive:   # the line's own window at this node
                wt = np.where(np.abs(dnu) <= wins[k][lid], wt, 0.0)
            out[k, sl] = np.bincount(col, weights=wt, minlength=n)
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


def window_range(lines, spec, w):
    """Inclusive grid-index range [j_lo, j_hi] of |nu_j - nu0_l| <= w_l (float64 test)."""
    nu0 = lines.nu0
    n = spec.n_nu
    lo = np.floor((nu0 - w - spec.nu_min) / spec.dnu).astype(np.int64) - 1
    hi = np.ceil((nu0 + w - spec.nu_min) / spec.dnu).astype(np.int64) + 1
    lo = np.clip(lo, 0, n)
    hi = np.clip(hi, -1, n - 1)

    def inc(j):
        ok = (j >= 0) & (j < n)
        return ok & (np.abs(grid_nu(spec, np.clip(j, 0, n - 1)) - nu0) <= w)

    for _ in range(6):
        lo = np.where((lo <= hi) & ~inc(lo), lo + 1, lo)
    for _ in range(6):
        hi = np.where((hi >= lo) & ~inc(hi), hi - 1, hi)
    return lo, hi


def adaptive_ranges(lines, spec):
    """Per T node k, the grid-index range of each line's adaptive window: (lo, hi),
    each of shape (nT, n_lines)."""
    los, his = [], []
    for T in spec.T_nodes():
        A, g, _ = line_terms(lines, float(T), spec.p_ref_atm, spec.x_ref, "lorentz")
        lo, hi = window_range(lines, spec, adaptive_halfwidth(A, g, spec))
        los.append(lo)
        his.append(hi)
    return np.stack(los), np.stack(his)


def profile_evals(lines, spec):
    """Exact number of (T node, line, nu_j) profile evaluations of the table."""
    if getattr(spec, "kappa_min", 0.0) > 0:
        lo, hi = adaptive_ranges(lines, spec)
        return int(np.maximum(hi - lo + 1, 0).sum())
    lo, hi = line_ranges(lines, spec)
    return int(np.maximum(hi - lo + 1, 0).sum()) * int(spec.nT)
