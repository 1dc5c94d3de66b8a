"""FP64 physics of the line-by-line method (Section 3, Eqs. S, tau, I, planck).

Test infrastructure only (see the package docstring).

Units: wavenumbers in cm^-1, line intensities in cm/molecule, number density
in molecule/cm^3, absorption coefficients in cm^-1, temperatures in K,
pressures in atm.  The Planck function uses SI (wavenumber in m^-1).

Readings of the paper (where it is silent):
* Eq. (S) takes the partition-function ratio Q(T_ref)/Q(T) = (T_ref/T)^q_exp.
* The density u_g of Eq. (tau) is the ideal-gas number density x p / (k_B T).
* Lorentz half-width gamma = gamma_ref (p / 1 atm) (T_ref / T)^n_T;
  Doppler half-width alpha = (nu0 / c) sqrt(2 ln2 k_B T / m).
* Eq. (planck) is taken in its wavenumber form 2 h c^2 nu^3 / (exp(c2 nu / T) - 1).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import wofz

# CODATA 2018 exact SI constants and derived values.
H_PLANCK = 6.62607015e-34        # J s
C_LIGHT = 299792458.0            # m / s
K_BOLTZ = 1.380649e-23           # J / K
AMU = 1.66053906660e-27          # kg
ATM = 101325.0                   # Pa
C2_M = H_PLANCK * C_LIGHT / K_BOLTZ   # second radiation constant, m K
C2_CM = 100.0 * C2_M                  # cm K
LN2 = math.log(2.0)


def line_intensity(S_ref, nu0, E_lower, T, T_ref=296.0, q_exp=1.0):
    """Eq. (S): S(T) = S(T_ref) * Q(T_ref)/Q(T) * Boltzmann ratio * stimulated-emission ratio.

    Parity: pinned (T = T_ref identity; SI-route Boltzmann and stimulated-emission factors).
    """
    S_ref = np.asarray(S_ref, dtype=np.float64)
    nu0 = np.asarray(nu0, dtype=np.float64)
    E_lower = np.asarray(E_lower, dtype=np.float64)
    q_ratio = (T_ref / T) ** q_exp
    boltz = np.exp(-C2_CM * E_lower / T) / np.exp(-C2_CM * E_lower / T_ref)
    stim = (-np.expm1(-C2_CM * nu0 / T)) / (-np.expm1(-C2_CM * nu0 / T_ref))
    return S_ref * q_ratio * boltz * stim


def number_density(x, p_atm, T):
    """Absorber number density u_g of Eq. (tau) from the ideal-gas law [molecule / cm^3].

    Parity: pinned (Loschmidt constant).
    """
    return x * p_atm * ATM / (K_BOLTZ * T) * 1e-6


def lorentz_hwhm(gamma_ref, p_atm, T, T_ref=296.0, n_T=0.75):
    """Pressure-broadened half-width at (T, p) [cm^-1].  Parity: pinned (T_ref, 1 atm identity)."""
    return np.asarray(gamma_ref, dtype=np.float64) * p_atm * (T_ref / T) ** n_T


def doppler_hwhm(nu0, T, mass_amu=44.0):
    """Doppler half-width at half maximum [cm^-1].  Parity: pinned (Gaussian limit test)."""
    return np.asarray(nu0, dtype=np.float64) / C_LIGHT * math.sqrt(
        2.0 * LN2 * K_BOLTZ * T / (mass_amu * AMU))


def lorentz_profile(dnu, gamma):
    """Lorentz line shape f (unit area), f = (gamma/pi) / (dnu^2 + gamma^2) [cm].

    Parity: pinned (truncated-area closed form (2/pi) atan(cutoff/gamma)).
    """
    dnu = np.asarray(dnu, dtype=np.float64)
    return (gamma / math.pi) / (dnu * dnu + gamma * gamma)


def voigt_profile(dnu, gamma, alpha):
    """Voigt line shape (unit area): Re w(z) sqrt(ln2) / (alpha sqrt(pi)),
    z = sqrt(ln2) (dnu + i gamma) / alpha, with w the Faddeeva function taken
    from scipy.special.wofz (a library primitive).

    Parity: pinned (convolution integral by quadrature, V(0) via libm erfc,
    Lorentz and Gaussian limits, unit area).
    """
    dnu = np.asarray(dnu, dtype=np.float64)
    s = math.sqrt(LN2) / np.asarray(alpha, dtype=np.float64)
    z = (dnu + 1j * np.asarray(gamma, dtype=np.float64)) * s
    return wofz(z).real * s / math.sqrt(math.pi)


def planck_wavenumber(nu_cm, T):
    """Eq. (planck), wavenumber form: 2 h c^2 nu^3 / (exp(c2 nu / T) - 1)
    with nu in m^-1; returns W m^-2 sr^-1 (m^-1)^-1.

    Parity: pinned (Stefan-Boltzmann integral sigma T^4 / pi).
    """
    nu_m = 100.0 * np.asarray(nu_cm, dtype=np.float64)
    return 2.0 * H_PLANCK * C_LIGHT ** 2 * nu_m ** 3 / np.expm1(C2_M * nu_m / T)
