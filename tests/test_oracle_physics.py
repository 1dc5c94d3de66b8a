"""Pins of the FP64 oracle's physics (Section 3, Eqs. S, tau, planck) against
published constants, closed forms and independent library routines."""
import math

import numpy as np
import pytest
from scipy import integrate

import synth
from oracle import kappa as K
from oracle import physics as ph

# Published constants used as pins (CODATA 2018).
C2_PUBLISHED_CM_K = 1.438776877        # second radiation constant, cm K
LOSCHMIDT_273 = 2.686780111e25          # m^-3 at 273.15 K and 101.325 kPa
SIGMA_SB = 5.670374419e-8               # Stefan-Boltzmann, W m^-2 K^-4


def test_second_radiation_constant():
    assert ph.C2_CM == pytest.approx(C2_PUBLISHED_CM_K, rel=1e-9)


def test_eq_s_identity_at_reference():
    rng = np.random.default_rng(5)
    S, nu0, E = rng.uniform(1e-22, 1e-19, 50), rng.uniform(2000, 3000, 50), rng.uniform(0, 5000, 50)
    assert np.allclose(ph.line_intensity(S, nu0, E, 296.0), S, rtol=1e-15, atol=0)


def test_eq_s_population_ratio_from_si_energies():
    # Boltzmann population of the lower state computed from the level energy in joules.
    T, Tref = 1500.0, 296.0
    E = np.array([0.0, 1000.0, 3000.0, 5000.0])   # cm^-1
    nu0 = 1e7 * np.ones_like(E)                    # stimulated emission negligible
    E_J = E * 100.0 * ph.H_PLANCK * ph.C_LIGHT
    pop = np.exp(-E_J / (ph.K_BOLTZ * T)) / np.exp(-E_J / (ph.K_BOLTZ * Tref))
    ratio = ph.line_intensity(np.ones_like(E), nu0, E, T) / (Tref / T)
    assert np.allclose(ratio, pop, rtol=1e-12)
    # hot gas populates high levels: S grows with T for large E, falls like 1/T for E = 0
    S_lo = ph.line_intensity(1.0, 2300.0, 5000.0, 800.0)
    S_hi = ph.line_intensity(1.0, 2300.0, 5000.0, 1600.0)
    assert S_hi > S_lo
    assert ph.line_intensity(1.0, 1e7, 0.0, 592.0) == pytest.approx(0.5, rel=1e-14)


def test_eq_s_stimulated_emission_factor():
    # E = 0 and Q ratio removed: the remaining factor is (1 - exp(-h c nu/kT)) / same at T_ref.
    T = 2000.0
    nu0 = np.array([500.0, 2000.0, 3000.0])
    x = 100.0 * nu0 * ph.H_PLANCK * ph.C_LIGHT / ph.K_BOLTZ
    expect = (1.0 - np.exp(-x / T)) / (1.0 - np.exp(-x / 296.0))
    got = ph.line_intensity(np.ones(3), nu0, np.zeros(3), T) / (296.0 / T)
    assert np.allclose(got, expect, rtol=1e-12)


def test_number_density_loschmidt():
    assert ph.number_density(1.0, 1.0, 273.15) == pytest.approx(LOSCHMIDT_273 * 1e-6, rel=1e-8)
    # linear in x and p, inverse in T
    assert ph.number_density(0.1, 3.0, 546.3) == pytest.approx(0.15 * LOSCHMIDT_273 * 1e-6, rel=1e-8)


def test_widths_reference_and_scaling():
    assert ph.lorentz_hwhm(0.07, 1.0, 296.0) == pytest.approx(0.07, rel=1e-15)
    assert ph.lorentz_hwhm(0.07, 2.0, 296.0 * 16.0) == pytest.approx(0.07 * 2.0 / 8.0, rel=1e-14)
    # Doppler HWHM = sqrt(2 ln2) * thermal speed sqrt(kT/m) * nu0 / c
    v_th = math.sqrt(ph.K_BOLTZ * 1000.0 / (44.0 * ph.AMU))
    assert ph.doppler_hwhm(2500.0, 1000.0) == pytest.approx(
        2500.0 * math.sqrt(2 * math.log(2)) * v_th / ph.C_LIGHT, rel=1e-14)


def _gauss(d, a):
    return math.sqrt(math.log(2) / math.pi) / a * math.exp(-math.log(2) * d * d / (a * a))


def _lor(d, g):
    return (g / math.pi) / (d * d + g * g)


@pytest.mark.parametrize("dnu,gamma,alpha", [(0.0, 0.02, 0.005), (0.01, 0.02, 0.005),
                                              (0.3, 0.03, 0.006), (0.0, 0.003, 0.006),
                                              (0.02, 0.003, 0.006), (2.0, 0.05, 0.004)])
def test_voigt_equals_convolution_integral(dnu, gamma, alpha):
    # V = integral of Gaussian(t) * Lorentzian(dnu - t), by adaptive quadrature.
    f = lambda t: _gauss(t, alpha) * _lor(dnu - t, gamma)
    span = 12 * alpha
    pts = sorted({-span, dnu - 5 * gamma, dnu, dnu + 5 * gamma, span})
    val = 0.0
    edges = [-math.inf] + [p for p in pts] + [math.inf]
    for a, b in zip(edges[:-1], edges[1:]):
        if b > a:
            val += integrate.quad(f, a, b, epsabs=0, epsrel=1e-13, limit=500)[0]
    assert float(ph.voigt_profile(dnu, gamma, alpha)) == pytest.approx(val, rel=1e-9)


@pytest.mark.parametrize("y", [0.1, 0.5, 1.0, 2.0, 5.0])
def test_voigt_centre_erfc(y):
    alpha = 0.004
    gamma = y * alpha / math.sqrt(math.log(2))
    expect = math.exp(y * y) * math.erfc(y) * math.sqrt(math.log(2)) / (alpha * math.sqrt(math.pi))
    assert float(ph.voigt_profile(0.0, gamma, alpha)) == pytest.approx(expect, rel=1e-12)


def test_voigt_limits():
    g = 0.05
    for d in (0.0, 0.05, 0.5, 10.0):
        assert float(ph.voigt_profile(d, g, 1e-7 * g)) == pytest.approx(_lor(d, g), rel=1e-10)
    a = 0.006
    for d in (0.0, 0.003, 0.006, 0.01):
        assert float(ph.voigt_profile(d, 1e-10 * a, a)) == pytest.approx(_gauss(d, a), rel=1e-6)


def test_voigt_unit_area():
    g, a = 0.02, 0.006
    f = lambda t: float(ph.voigt_profile(t, g, a))
    area = 2 * (integrate.quad(f, 0, 1, epsrel=1e-13, limit=400)[0]
                + integrate.quad(f, 1, math.inf, epsrel=1e-12, limit=400)[0])
    assert area == pytest.approx(1.0, rel=1e-9)


def _single_line_case(profile, gamma=0.05, dnu=0.005):
    lines = synth.Lines(nu0=np.array([2300.0 + 0.5 * dnu]), S_ref=np.array([3e-20]),
                        gamma_ref=np.array([gamma]), E_lower=np.array([1200.0]))
    spec = synth.Spectral(nu_min=2250.0, dnu=dnu, n_nu=int(round(100 / dnu)), cutoff=25.0,
                          profile=profile, nT=1, T_min=296.0, T_max=296.0, p_ref_atm=1.0,
                          x_ref=1.0)
    return lines, spec


def test_kappa_single_lorentz_line_area():
    # Sum_j kappa_j dnu over the cutoff window = u S (2/pi) atan(cutoff/gamma): a midpoint
    # rule over [-25, 25] whose error is exponentially small for gamma/dnu = 10.
    lines, spec = _single_line_case("lorentz")
    tab = K.kappa_table(lines, spec)[0]
    u = ph.number_density(1.0, 1.0, 296.0)
    area = tab.sum() * spec.dnu / (u * 3e-20)
    assert area == pytest.approx(2 / math.pi * math.atan(25.0 / 0.05), rel=1e-10)
    assert np.count_nonzero(tab) == 10000


def test_kappa_single_voigt_line_area():
    lines, spec = _single_line_case("voigt")
    tab = K.kappa_table(lines, spec)[0]
    u = ph.number_density(1.0, 1.0, 296.0)
    area = tab.sum() * spec.dnu / (u * 3e-20)
    alpha = float(ph.doppler_hwhm(lines.nu0[0], 296.0))
    f = lambda t: float(ph.voigt_profile(t, 0.05, alpha))
    expect = 2 * integrate.quad(f, 0, 25.0, epsrel=1e-13, limit=400)[0]
    assert area == pytest.approx(expect, rel=1e-9)


def test_kappa_superposition_and_nodes():
    case = synth.config(0)
    spec = synth.Spectral(nu_min=2100.0, dnu=0.02, n_nu=2000, cutoff=25.0, profile="voigt",
                          nT=3, T_min=500.0, T_max=1500.0, p_ref_atm=2.0, x_ref=0.2)
    lines = case.lines
    js = np.arange(0, spec.n_nu, 7)
    full = K.kappa_columns(lines, spec, js)
    a = K.kappa_columns(lines.subset(slice(0, 250)), spec, js)
    b = K.kappa_columns(lines.subset(slice(250, 500)), spec, js)
    assert np.allclose(full, a + b, rtol=1e-13, atol=0)
    # each row equals the table evaluated at that temperature alone
    for k, T in enumerate(spec.T_nodes()):
        row = K.kappa_columns(lines, spec, js, T_nodes=[T])[0]
        assert np.array_equal(row, full[k])
    # density scaling: kappa is proportional to x * p at fixed widths only through u
    # (the widths depend on p), so check x alone
    half = K.kappa_columns(lines, spec, js, x=0.1)
    assert np.allclose(half, 0.5 * full, rtol=1e-14)


def test_kappa_cutoff_edge_inclusive():
    # A grid in binary fractions: points at exactly +-cutoff are included.
    lines = synth.Lines(nu0=np.array([2.0]), S_ref=np.array([1e-20]), gamma_ref=np.array([0.1]),
                        E_lower=np.array([0.0]))
    spec = synth.Spectral(nu_min=0.0, dnu=0.25, n_nu=17, cutoff=1.0, profile="lorentz")
    tab = K.kappa_table(lines, spec)[0]
    assert np.array_equal(np.nonzero(tab)[0], np.arange(4, 13))
    lo, hi = K.line_ranges(lines, spec)
    assert (lo[0], hi[0]) == (4, 12)
    assert K.profile_evals(lines, spec) == 9


def test_line_ranges_match_pairs():
    case = synth.config(0)
    lo, hi = K.line_ranges(case.lines, case.spec)
    js = np.arange(case.spec.n_nu)
    col, lid, _ = K._pairs(case.lines, case.spec, js)
    cnt = np.bincount(lid, minlength=case.lines.n)
    assert np.array_equal(cnt, np.maximum(hi - lo + 1, 0))
    assert K.profile_evals(case.lines, case.spec) == col.size


def test_planck_stefan_boltzmann():
    T = 1000.0
    dnu = 0.5
    nu = (np.arange(80000) + 0.5) * dnu      # cm^-1, midpoints up to 40000 cm^-1
    total = ph.planck_wavenumber(nu, T).sum() * dnu * 100.0
    assert total == pytest.approx(SIGMA_SB * T ** 4 / math.pi, rel=1e-8)


def test_fixed_points_per_line_window():
    # Section 3: 16 contributions per line; the window is the 8 grid points at or
    # below the centre and the 8 above it
    from dataclasses import replace
    case = synth.config(0)
    spec = replace(case.spec, points_per_line=16)
    lo, hi = K.line_ranges(case.lines, spec)
    inner = (lo > 0) & (hi < spec.n_nu - 1)
    assert np.all(hi[inner] - lo[inner] + 1 == 16)
    nu_lo = K.grid_nu(spec, lo[inner] + 7)
    nu_hi = K.grid_nu(spec, lo[inner] + 8)
    assert np.all(nu_lo <= case.lines.nu0[inner]) and np.all(nu_hi > case.lines.nu0[inner])
    tab = K.kappa_table(case.lines, spec)[0]
    assert K.profile_evals(case.lines, spec) == int(np.sum(hi - lo + 1))
    assert np.count_nonzero(tab) <= 500 * 16


def _adaptive_case(profile="lorentz", kappa_min=1e-3):
    from dataclasses import replace
    rng = synth.rng_for(9, 60)
    lines = synth.make_lines(400, 2000.0, 2040.0, rng)
    spec = synth.Spectral(nu_min=2005.0, dnu=0.01, n_nu=3001, cutoff=25.0, profile=profile, nT=4,
                          T_min=700.0, T_max=1900.0, p_ref_atm=1.5, x_ref=0.08)
    return lines, spec, replace(spec, kappa_min=kappa_min)


def test_adaptive_points_reduce_to_the_cutoff_table():
    # kappa_min -> 0 makes every window the cutoff window: the same table, bit for bit
    lines, spec, _ = _adaptive_case()
    from dataclasses import replace
    tiny = replace(spec, kappa_min=1e-300)
    assert np.array_equal(K.kappa_table(lines, tiny), K.kappa_table(lines, spec))
    assert K.profile_evals(lines, tiny) == K.profile_evals(lines, spec)


def test_adaptive_points_drop_only_terms_below_kappa_min():
    # Every (node, line, point) of the cutoff set: kept iff its Lorentz wing A gamma / (pi dnu^2)
    # reaches kappa_min (within the cutoff); the exact Lorentz value of a dropped term is then
    # below kappa_min, so 0 <= full - adaptive <= (dropped terms) * kappa_min at every entry.
    lines, spec, ad = _adaptive_case()
    full, adap = K.kappa_table(lines, spec), K.kappa_table(lines, ad)
    lo, hi = K.adaptive_ranges(lines, ad)
    clo, chi = K.line_ranges(lines, spec)
    js = np.arange(spec.n_nu)
    nu = K.grid_nu(spec, js)
    for k, T in enumerate(spec.T_nodes()):
        A, g, _ = K.line_terms(lines, float(T), spec.p_ref_atm, spec.x_ref, "lorentz")
        dropped = np.zeros(spec.n_nu)
        kept_n = 0
        for l in range(lines.n):
            if chi[l] < clo[l]:
                continue
            jj = js[clo[l]:chi[l] + 1]
            d = nu[jj] - lines.nu0[l]
            keep = (jj >= lo[k, l]) & (jj <= hi[k, l])
            wing = A[l] * g[l] / (math.pi * d * d)
            assert np.all(wing[keep & (d != 0)] >= ad.kappa_min)
            val = A[l] * g[l] / (math.pi * (d * d + g[l] * g[l]))
            assert np.all(val[~keep] < ad.kappa_min)
            dropped[jj[~keep]] += 1
            kept_n += int(keep.sum())
        diff = full[k] - adap[k]
        assert np.all(diff >= -1e-12 * full[k]) and np.all(diff <= dropped * ad.kappa_min * (1 + 1e-12))
        assert kept_n == int(np.maximum(hi[k] - lo[k] + 1, 0).sum())
    assert K.profile_evals(lines, ad) < K.profile_evals(lines, spec)


def test_adaptive_points_monotone_in_kappa_min():
    from dataclasses import replace
    lines, spec, _ = _adaptive_case("voigt")
    prev_t, prev_n = None, None
    for km in (1e-4, 1e-3, 1e-2, 1e-1):
        s = replace(spec, kappa_min=km)
        t, n = K.kappa_table(lines, s), K.profile_evals(lines, s)
        if prev_t is not None:
            assert n <= prev_n and np.all(t <= prev_t * (1 + 1e-12))
        prev_t, prev_n = t, n
