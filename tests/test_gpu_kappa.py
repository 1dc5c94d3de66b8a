"""GPU parity of rt_build_kappa (Eqs. S and tau) against the FP64 oracle.

Tolerance: 1e-5 relative per table entry (binary32 line sum with Kahan
compensation; the error budget is about 1e-6 for Eq. S with a double-float
Boltzmann exponent, <= 1.5e-6 for the binary32 Voigt function at y >= 0.5,
and a few ulps for the compensated sum).  The number of profile evaluations
is an integer decision taken in binary64 on both sides and must match exactly.
"""
import ctypes as ct

import numpy as np
import pytest

import synth
from oracle import kappa as okappa

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def rt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_cs_0703028_gb300 as rt
    rt.lib()
    return rt


def _gpu_table(rt, lines, spec, memory="host"):
    import torch
    evals = torch.zeros(1, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    kap = rt.build_kappa(lines, spec, memory=memory, evals=evals, status=status)
    torch.cuda.synchronize()
    return kap.cpu().numpy().astype(np.float64), int(evals.item()), int(status.item())


def _rel(got, ref):
    return np.abs(got - ref) / np.abs(ref)


def test_c0_lorentz_full_table(rt):
    case = synth.config(0)
    got, ev, st = _gpu_table(rt, case.lines, case.spec)
    ref = okappa.kappa_table(case.lines, case.spec)
    assert st == 0
    assert ev == okappa.profile_evals(case.lines, case.spec)
    assert np.all(ref > 0)
    assert _rel(got, ref).max() <= TOL


@pytest.mark.parametrize("n_nu,nT,p_ref,T_lo,T_hi", [(5003, 5, 1.0, 600.0, 2200.0),
                                                     (3001, 3, 0.5, 1500.0, 2500.0),
                                                     (4096, 2, 5.0, 500.0, 900.0)])
def test_voigt_tiles_and_ragged_tail(rt, n_nu, nT, p_ref, T_lo, T_hi):
    rng = synth.rng_for(9, n_nu)
    lines = synth.make_lines(400, 1960.0, 2090.0, rng)   # some centres outside the window
    spec = synth.Spectral(nu_min=2000.0, dnu=0.01, n_nu=n_nu, cutoff=25.0, profile="voigt",
                          nT=nT, T_min=T_lo, T_max=T_hi, p_ref_atm=p_ref, x_ref=0.2)
    got, ev, st = _gpu_table(rt, lines, spec)
    ref = okappa.kappa_table(lines, spec)
    assert st == 0
    assert ev == okappa.profile_evals(lines, spec)
    nz = ref > 0
    assert np.array_equal(got > 0, nz)
    assert _rel(got[nz], ref[nz]).max() <= TOL


def test_dense_lines_many_chunks(rt):
    # about 3000 lines per 1024-point tile: several staged chunks per block
    rng = synth.rng_for(9, 77)
    lines = synth.make_lines(5000, 1990.0, 2110.0, rng)
    spec = synth.Spectral(nu_min=2000.0, dnu=0.02, n_nu=4000, cutoff=25.0, profile="voigt",
                          nT=2, T_min=800.0, T_max=2000.0)
    got, ev, st = _gpu_table(rt, lines, spec)
    ref = okappa.kappa_table(lines, spec)
    assert ev == okappa.profile_evals(lines, spec)
    assert _rel(got, ref).max() <= TOL


def test_device_resident_lines_match_host(rt):
    case = synth.config(0)
    a, ev_a, st_a = _gpu_table(rt, case.lines, case.spec, memory="host")
    b, ev_b, st_b = _gpu_table(rt, case.lines, case.spec, memory="device")
    assert st_a == 0 and st_b == 0 and ev_a == ev_b
    assert np.array_equal(a, b)


def test_device_resident_unsorted_lines_flagged(rt):
    import torch
    case = synth.config(0)
    ul = case.lines.subset(np.arange(case.lines.n)[::-1])
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rt.build_kappa(ul, case.spec, memory="device", status=status)
    st = rt.lib().rt_status_read(ct.c_void_p(status.data_ptr()), None)
    assert st == rt.RT_E_UNSORTED


def test_empty_line_list_and_single_point(rt):
    case = synth.config(0)
    empty = case.lines.subset(np.arange(0))
    got, ev, st = _gpu_table(rt, empty, case.spec)
    assert ev == 0 and np.all(got == 0)
    spec1 = synth.Spectral(nu_min=2250.0, dnu=0.02, n_nu=1, cutoff=25.0, profile="lorentz",
                           nT=1, T_min=1000.0, T_max=1000.0)
    got, ev, st = _gpu_table(rt, case.lines, spec1)
    ref = okappa.kappa_table(case.lines, spec1)
    assert ev == okappa.profile_evals(case.lines, spec1)
    assert _rel(got, ref).max() <= TOL


@pytest.fixture(scope="module")
def c1_columns():
    case = synth.config(1)
    rng = np.random.default_rng(123)
    cols = np.unique(np.concatenate([rng.integers(0, case.spec.n_nu, 600),
                                     np.arange(0, 8), np.arange(case.spec.n_nu - 8, case.spec.n_nu)]))
    return case, cols, okappa.kappa_columns(case.lines, case.spec, cols)


def test_c1_full_size_table_sampled_columns(rt, c1_columns):
    # Full 64 x 100k Voigt table in the benchmark's launch configuration;
    # 600 random columns (all 64 temperatures) plus both edges against the oracle.
    case, cols, ref = c1_columns
    got, ev, st = _gpu_table(rt, case.lines, case.spec)
    assert st == 0
    assert ev == okappa.profile_evals(case.lines, case.spec)
    assert got.shape == (64, 100000)
    assert np.all(np.isfinite(got)) and np.all(got > 0)
    assert _rel(got[:, cols], ref).max() <= TOL


@pytest.mark.parametrize("profile", ["lorentz", "voigt"])
def test_fixed_points_per_line(rt, profile):
    from dataclasses import replace
    rng = synth.rng_for(9, 80)
    lines = synth.make_lines(2000, 1990.0, 2110.0, rng)
    spec = synth.Spectral(nu_min=2000.0, dnu=0.01, n_nu=10000, cutoff=25.0, profile=profile, nT=3,
                          T_min=800.0, T_max=1600.0, points_per_line=16)
    got, ev, st = _gpu_table(rt, lines, spec)
    ref = okappa.kappa_table(lines, spec)
    assert ev == okappa.profile_evals(lines, spec)
    nz = ref > 0
    assert np.array_equal(got > 0, nz)
    assert _rel(got[nz], ref[nz]).max() <= TOL


def test_two_gas_mixture_accumulates(rt):
    import torch
    from dataclasses import replace
    rng = synth.rng_for(9, 81)
    co2 = synth.make_lines(600, 2000.0, 2200.0, rng)
    h2o = replace(synth.make_lines(400, 2050.0, 2250.0, rng, S_lo=1e-23, S_hi=1e-20), mass_amu=18.0,
                  n_T=0.6, q_exp=1.5)
    s1 = synth.Spectral(nu_min=2020.0, dnu=0.02, n_nu=8000, cutoff=25.0, profile="voigt", nT=4,
                        T_min=700.0, T_max=1900.0, x_ref=0.1)
    s2 = replace(s1, x_ref=0.05, accumulate=1)
    out = torch.empty((s1.nT, s1.n_nu), dtype=torch.float32, device="cuda")
    rt.build_kappa(co2, s1, out=out)
    rt.build_kappa(h2o, s2, out=out)
    torch.cuda.synchronize()
    ref = okappa.kappa_table(co2, s1) + okappa.kappa_table(h2o, replace(s2, accumulate=0))
    got = out.cpu().numpy().astype(np.float64)
    assert _rel(got, ref).max() <= TOL


def test_offsets_of_millions_of_grid_points(rt):
    # A 50 cm^-1 cutoff on a 1e-5 cm^-1 grid: offsets of a point from a line centre
    # reach 4.5e6 grid points (binary32 offsets with an ulp of 0.5 grid point).
    rng = synth.rng_for(9, 82)
    lines = synth.make_lines(60, 1955.0, 2045.0, rng)
    spec = synth.Spectral(nu_min=2000.0, dnu=1e-5, n_nu=3000, cutoff=50.0, profile="voigt", nT=2,
                          T_min=800.0, T_max=1600.0)
    got, ev, st = _gpu_table(rt, lines, spec)
    ref = okappa.kappa_table(lines, spec)
    assert st == 0
    assert ev == okappa.profile_evals(lines, spec)
    assert np.all(ref > 0)
    assert _rel(got, ref).max() <= TOL


@pytest.mark.parametrize("profile,memory", [("voigt", "host"), ("voigt", "device"), ("lorentz", "host")])
def test_odd_line_count(rt, profile, memory):
    # the line sum takes lines in pairs; an odd count adds a padding line that must add nothing
    rng = synth.rng_for(9, 83)
    lines = synth.make_lines(401, 1985.0, 2075.0, rng)
    spec = synth.Spectral(nu_min=2000.0, dnu=0.01, n_nu=5000, cutoff=25.0, profile=profile, nT=3,
                          T_min=700.0, T_max=1900.0)
    got, ev, st = _gpu_table(rt, lines, spec, memory=memory)
    ref = okappa.kappa_table(lines, spec)
    assert st == 0
    assert ev == okappa.profile_evals(lines, spec)
    nz = ref > 0
    assert np.array_equal(got > 0, nz)
    assert _rel(got[nz], ref[nz]).max() <= TOL


def test_fixed_points_per_line_accumulates(rt):
    # two gases with 16 points per line, the second accumulated into the first's table
    import torch
    from dataclasses import replace
    rng = synth.rng_for(9, 84)
    co2 = synth.make_lines(800, 1995.0, 2105.0, rng)
    h2o = replace(synth.make_lines(500, 1995.0, 2105.0, rng, S_lo=1e-23, S_hi=1e-20), mass_amu=18.0,
                  n_T=0.6, q_exp=1.5)
    s1 = synth.Spectral(nu_min=2000.0, dnu=0.01, n_nu=10000, cutoff=25.0, profile="voigt", nT=3,
                        T_min=800.0, T_max=1600.0, points_per_line=16)
    s2 = replace(s1, x_ref=0.05, accumulate=1)
    out = torch.empty((s1.nT, s1.n_nu), dtype=torch.float32, device="cuda")
    rt.build_kappa(co2, s1, out=out)
    rt.build_kappa(h2o, s2, out=out)
    torch.cuda.synchronize()
    ref = okappa.kappa_table(co2, s1) + okappa.kappa_table(h2o, replace(s2, accumulate=0))
    got = out.cpu().numpy().astype(np.float64)
    nz = ref > 0
    assert np.array_equal(got > 0, nz)
    assert _rel(got[nz], ref[nz]).max() <= TOL


@pytest.mark.parametrize("profile,kappa_min", [("lorentz", 1e-3), ("voigt", 1e-3), ("voigt", 0.3)])
def test_adaptive_points_per_line(rt, profile, kappa_min):
    # each line at each T node only where its Lorentz wing reaches kappa_min (windows decided
    # in binary64 on both sides: the evaluation counts must match exactly); points no window
    # reaches stay exactly zero
    from dataclasses import replace
    rng = synth.rng_for(9, 82)
    lines = synth.make_lines(2000, 1990.0, 2110.0, rng)
    spec = synth.Spectral(nu_min=2000.0, dnu=0.01, n_nu=10001, cutoff=25.0, profile=profile, nT=3,
                          T_min=800.0, T_max=1600.0, p_ref_atm=1.3, x_ref=0.07, kappa_min=kappa_min)
    got, ev, st = _gpu_table(rt, lines, spec)
    ref = okappa.kappa_table(lines, spec)
    assert st == 0
    assert ev == okappa.profile_evals(lines, spec)
    assert ev < okappa.profile_evals(lines, replace(spec, kappa_min=0.0))
    nz = ref > 0
    assert np.array_equal(got > 0, nz)
    assert _rel(got[nz], ref[nz]).max() <= TOL


def test_adaptive_points_accumulate_and_device_lines(rt):
    import torch
    from dataclasses import replace
    rng = synth.rng_for(9, 83)
    co2 = synth.make_lines(700, 2000.0, 2200.0, rng)
    h2o = replace(synth.make_lines(500, 2050.0, 2250.0, rng, S_lo=1e-23, S_hi=1e-20), mass_amu=18.0,
                  n_T=0.6, q_exp=1.5)
    s1 = synth.Spectral(nu_min=2020.0, dnu=0.02, n_nu=8000, cutoff=25.0, profile="voigt", nT=4,
                        T_min=700.0, T_max=1900.0, x_ref=0.1, kappa_min=1e-2)
    s2 = replace(s1, x_ref=0.05, accumulate=1)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    tab = rt.build_kappa(co2, s1, memory="device", status=status)
    rt.build_kappa(h2o, s2, out=tab, memory="device", status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = okappa.kappa_table(co2, s1) + okappa.kappa_table(h2o, s2)
    got = tab.cpu().numpy().astype(np.float64)
    nz = ref > 0
    assert np.array_equal(got > 0, nz)
    assert _rel(got[nz], ref[nz]).max() <= TOL


def test_adaptive_points_exclude_fixed_points(rt):
    import torch
    from dataclasses import replace
    c0 = synth.config(0)
    bad = replace(c0.spec, kappa_min=1e-3, points_per_line=16)
    with pytest.raises(rt.RtError):
        rt.build_kappa(c0.lines, bad)
    with pytest.raises(rt.RtError):
        rt.build_kappa(c0.lines, replace(c0.spec, kappa_min=-1.0))


def test_c1_full_size_adaptive_points_sampled_columns(rt, c1_columns):
    # Adaptive points per line on the full 64 x 100k Voigt table of the 20k-line list (the
    # configuration `bench.py --workload next` times): 600 random columns and both edges
    # against the oracle's adaptive table; the evaluation count over the whole table exact.
    from dataclasses import replace
    case, cols, _ = c1_columns
    spec = replace(case.spec, kappa_min=1e-3)
    ref = okappa.kappa_columns(case.lines, spec, cols)
    got, ev, st = _gpu_table(rt, case.lines, spec)
    assert st == 0
    assert ev == okappa.profile_evals(case.lines, spec)
    nz = ref > 0
    assert np.array_equal(got[:, cols] > 0, nz)
    assert _rel(got[:, cols][nz], ref[nz]).max() <= TOL
