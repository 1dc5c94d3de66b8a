"""rt_build_kappa_static: the kappa build for callers that cannot allocate
device memory (a solver that has given all device memory to its own pool, a
loop where an allocation could stall or fail).  It must give the same table
as rt_build_kappa, call after call, using only its fixed 32 MiB device array.

This file is named to be collected last: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes as ct

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the kappa parity tolerance of the other GPU tests


@pytest.fixture(scope="module")
def rt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_cs_0703028_gb300 as rt
    rt.lib()
    return rt


def _both(rt, lines, spec):
    """The same inputs through rt_build_kappa and rt_build_kappa_static."""
    import torch
    L = rt.lib()
    S = rt.make_spectral(spec)
    ls, keep = rt.make_lines(lines)
    ref = torch.empty((spec.nT, spec.n_nu), dtype=torch.float32, device="cuda")
    got = torch.full((spec.nT, spec.n_nu), -1.0, dtype=torch.float32, device="cuda")
    ev_ref = torch.zeros(1, dtype=torch.int64, device="cuda")
    ev_got = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = L.rt_build_kappa(ct.byref(ls), ct.byref(S), ct.c_void_p(ref.data_ptr()),
                          ct.c_void_p(ev_ref.data_ptr()), None, None)
    assert st == rt.RT_OK, L.rt_last_error()
    st = L.rt_build_kappa_static(ct.byref(ls), ct.byref(S), ct.c_void_p(got.data_ptr()),
                                 ct.c_void_p(ev_got.data_ptr()), None, None)
    assert st == rt.RT_OK, L.rt_last_error()
    torch.cuda.synchronize()
    return ref.cpu().numpy(), got.cpu().numpy(), int(ev_ref.item()), int(ev_got.item())


def _close(got, ref):
    nz = ref != 0
    assert np.array_equal(got == 0, ~nz)
    assert np.max(np.abs(got[nz] - ref[nz]) / np.abs(ref[nz])) <= TOL


def test_static_scratch_matches_allocating_build_twice(rt):
    # two calls in a row with different inputs: the second must not see the first's scratch
    c0 = synth.config(0)
    rng = synth.rng_for(9, 31)
    lines_b = synth.make_lines(700, 2000.0, 2100.0, rng)
    spec_b = synth.Spectral(nu_min=2010.0, dnu=0.01, n_nu=6001, cutoff=25.0, profile="voigt",
                            nT=5, T_min=700.0, T_max=2100.0, p_ref_atm=2.0, x_ref=0.05)
    for lines, spec in ((c0.lines, c0.spec), (lines_b, spec_b), (c0.lines, c0.spec)):
        ref, got, ev_ref, ev_got = _both(rt, lines, spec)
        assert ev_got == ev_ref
        _close(got, ref)


@pytest.mark.parametrize("profile", ["lorentz", "voigt"])
def test_static_scratch_fixed_points_per_line(rt, profile):
    # the fixed-points gather kernel through the allocation-free entry point (odd line count)
    rng = synth.rng_for(9, 33)
    lines = synth.make_lines(901, 1995.0, 2105.0, rng)
    spec = synth.Spectral(nu_min=2000.0, dnu=0.01, n_nu=10001, cutoff=25.0, profile=profile, nT=3,
                          T_min=800.0, T_max=1600.0, points_per_line=16)
    ref, got, ev_ref, ev_got = _both(rt, lines, spec)
    assert ev_got == ev_ref
    _close(got, ref)


def test_static_scratch_rejects_oversized_input(rt):
    L = rt.lib()
    rng = synth.rng_for(9, 32)
    lines = synth.make_lines(100000, 1500.0, 3500.0, rng)
    spec = synth.Spectral(nu_min=1500.0, dnu=0.005, n_nu=400000, cutoff=25.0, profile="voigt",
                          nT=64, T_min=500.0, T_max=2500.0)
    S = rt.make_spectral(spec)
    ls, keep = rt.make_lines(lines)
    st = L.rt_build_kappa_static(ct.byref(ls), ct.byref(S), ct.c_void_p(256), None, None, None)
    assert st == rt.RT_E_INVAL
    assert b"static array holds" in L.rt_last_error()
