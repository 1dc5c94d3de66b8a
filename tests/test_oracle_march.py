"""Pins of the oracle's spectrally resolved marching of Eq. (I): the isothermal
closed form I_in e^-tau + I_b (1 - e^-tau), transparency, the optically thick
limit, and the power reduction."""
import math

import numpy as np
import pytest

import synth
from oracle import physics as ph
from oracle import trace as OT


def _slab(T=1200.0, n=10):
    return synth.uniform_grid(n, 1, 1, 0.1, math.inf, math.inf, T)


def test_isothermal_column_closed_form():
    g = _slab()
    spec = synth.Spectral(nu_min=2000.0, dnu=0.5, n_nu=200, nT=1, T_min=1200.0, T_max=1200.0)
    kap = np.linspace(1e-3, 0.2, 200)[None, :]               # cm^-1 per wavenumber
    Iin = np.linspace(0.0, 3.0, 200)
    I, pw = OT.march(g, spec, kap, [[0.0, 0.0, 0.0]], [[1.0, 0.0, 0.0]], I_in=Iin)
    tau = kap[0] * 100.0 * 1.0                                # 10 cells x 0.1 m
    Ib = ph.planck_wavenumber(spec.nu_min + np.arange(200) * spec.dnu, 1200.0)
    expect = Iin * np.exp(-tau) + Ib * (-np.expm1(-tau))
    assert np.allclose(I[0], expect, rtol=1e-13)
    assert pw[0] == pytest.approx(np.sum(Iin - expect) * 100.0 * spec.dnu, rel=1e-12)


def test_transparent_and_thick_limits():
    g = synth.Grid(6, 1, 1, 0.05, math.inf, math.inf,
                   np.array([800, 900, 1000, 1100, 1200, 1500], dtype=np.float32))
    spec = synth.Spectral(nu_min=2100.0, dnu=1.0, n_nu=5, nT=2, T_min=800.0, T_max=1500.0)
    Iin = np.array([0.1, 0.2, 0.3, 0.4, 0.5])
    I0, _ = OT.march(g, spec, np.zeros((2, 5)), [[0.0, 0.0, 0.0]], [[1.0, 0.0, 0.0]], I_in=Iin)
    assert np.array_equal(I0[0], Iin)
    Ith, _ = OT.march(g, spec, np.full((2, 5), 1e6), [[0.0, 0.0, 0.0]], [[1.0, 0.0, 0.0]], I_in=Iin)
    Ib_last = ph.planck_wavenumber(spec.nu_min + np.arange(5) * spec.dnu, 1500.0)
    assert np.allclose(Ith[0], Ib_last, rtol=1e-12)


def test_oblique_ray_path_length():
    # an oblique ray through a uniform 3-D box: tau = kappa * 100 * chord
    g = synth.uniform_grid(5, 5, 5, 0.2, 0.2, 0.2, 1000.0)
    spec = synth.Spectral(nu_min=2000.0, dnu=1.0, n_nu=3, nT=1, T_min=1000.0, T_max=1000.0)
    d = np.array([0.48, 0.6, 0.64], dtype=np.float32)
    d = (d / np.linalg.norm(d.astype(np.float64))).astype(np.float32)
    p = np.array([0.01, 0.02, 0.03], dtype=np.float32)
    kap = np.array([[0.01, 0.02, 0.05]])
    I, _ = OT.march(g, spec, kap, [p], [d])
    chord = min((1.0 - float(p[a])) / float(d[a]) for a in range(3))
    Ib = ph.planck_wavenumber(spec.nu_min + np.arange(3) * spec.dnu, 1000.0)
    expect = Ib * (-np.expm1(-kap[0] * 100.0 * chord))
    assert np.allclose(I[0], expect, rtol=1e-6)
