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


def _both(rt, lines, spec, memory="host", tables=None):
    """The same inputs through rt_build_kappa and rt_build_kappa_static (into the given
    (ref, got) tables when spec.accumulate is set)."""
    import torch
    L = rt.lib()
    S = rt.make_spectral(spec)
    ls, keep = rt.make_lines(lines, memory=memory)
    if tables is None:
        ref = torch.empty((spec.nT, spec.n_nu), dtype=torch.float32, device="cuda")
        got = torch.full((spec.nT, spec.n_nu), -1.0, dtype=torch.float32, device="cuda")
    else:
        ref, got = tables
    ev_ref = torch.zeros(1, dtype=torch.int64, device="cuda")
    ev_got = torch.zeros(1, dtype=torch.int64, device="cuda")
    status = torch.zeros(2, dtype=torch.int32, device="cuda")   # required for device-resident lines
    st = L.rt_build_kappa(ct.byref(ls), ct.byref(S), ct.c_void_p(ref.data_ptr()),
                          ct.c_void_p(ev_ref.data_ptr()), ct.c_void_p(status.data_ptr()), None)
    assert st == rt.RT_OK, L.rt_last_error()
    st = L.rt_build_kappa_static(ct.byref(ls), ct.byref(S), ct.c_void_p(got.data_ptr()),
                                 ct.c_void_p(ev_got.data_ptr()), ct.c_void_p(status.data_ptr() + 4), None)
    assert st == rt.RT_OK, L.rt_last_error()
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [0, 0]
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


def test_static_scratch_adaptive_points_per_line(rt):
    # adaptive points per line: the per-(node, line) windows live in the static array too
    rng = synth.rng_for(9, 35)
    lines = synth.make_lines(1500, 1995.0, 2105.0, rng)
    spec = synth.Spectral(nu_min=2000.0, dnu=0.01, n_nu=10001, cutoff=25.0, profile="voigt", nT=4,
                          T_min=800.0, T_max=1600.0, kappa_min=1e-3)
    for _ in range(2):
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


def test_static_scratch_device_resident_lines_and_accumulation(rt):
    # lines already in device memory (the call reads them there and reports through the
    # status word), then a second gas added into the same tables (accumulate = 1)
    import torch
    from dataclasses import replace
    rng = synth.rng_for(9, 34)
    co2 = synth.make_lines(1200, 2000.0, 2080.0, rng)
    h2o = replace(synth.make_lines(500, 1990.0, 2090.0, rng, S_lo=1e-23, S_hi=1e-20), mass_amu=18.0,
                  n_T=0.6, q_exp=1.5)
    spec = synth.Spectral(nu_min=2005.0, dnu=0.01, n_nu=7001, cutoff=25.0, profile="voigt", nT=6,
                          T_min=600.0, T_max=2100.0, p_ref_atm=1.5, x_ref=0.08)
    ref, got, ev_ref, ev_got = _both(rt, co2, spec, memory="device")
    assert ev_got == ev_ref
    _close(got, ref)
    tabs = (torch.from_numpy(ref).cuda(), torch.from_numpy(got).cuda())
    ref2, got2, ev_ref2, ev_got2 = _both(rt, h2o, replace(spec, accumulate=1, x_ref=0.05), memory="device",
                                         tables=tabs)
    assert ev_got2 == ev_ref2
    assert np.all(ref2 >= ref) and np.any(ref2 > ref)   # the second gas was added
    _close(got2, ref2)


def _driver():
    """The CUDA driver API (libcuda), for reading the device's default memory pool."""
    import ctypes.util
    for name in ("libcuda.so.1", ctypes.util.find_library("cuda")):
        if name:
            try:
                return ct.CDLL(name)
            except OSError:
                pass
    pytest.skip("libcuda not found")


def test_static_scratch_allocates_nothing(rt):
    # The allocating build takes its scratch from the device's default memory pool
    # (stream-ordered allocation), which raises the pool's high-water mark of used
    # memory; the allocation-free build must leave that mark at zero.
    import torch
    cu = _driver()
    USED_MEM_HIGH = 8   # CU_MEMPOOL_ATTR_USED_MEM_HIGH
    dev = ct.c_int()
    assert cu.cuDeviceGet(ct.byref(dev), torch.cuda.current_device()) == 0
    pool = ct.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ct.byref(pool), dev) == 0

    def high():
        v = ct.c_uint64()
        assert cu.cuMemPoolGetAttribute(pool, USED_MEM_HIGH, ct.byref(v)) == 0
        return v.value

    def reset():
        zero = ct.c_uint64(0)
        assert cu.cuMemPoolSetAttribute(pool, USED_MEM_HIGH, ct.byref(zero)) == 0

    L = rt.lib()
    c0 = synth.config(0)
    S = rt.make_spectral(c0.spec)
    ls, keep = rt.make_lines(c0.lines)
    out = torch.empty((c0.spec.nT, c0.spec.n_nu), dtype=torch.float32, device="cuda")
    for fn in (L.rt_build_kappa, L.rt_build_kappa_static):   # warm: module loading, symbol look-up
        assert fn(ct.byref(ls), ct.byref(S), ct.c_void_p(out.data_ptr()), None, None, None) == rt.RT_OK
    torch.cuda.synchronize()
    reset()
    assert L.rt_build_kappa(ct.byref(ls), ct.byref(S), ct.c_void_p(out.data_ptr()), None, None, None) == 0
    torch.cuda.synchronize()
    assert high() > 0          # the check sees the allocating build's scratch
    reset()
    assert high() == 0
    for _ in range(2):
        st = L.rt_build_kappa_static(ct.byref(ls), ct.byref(S), ct.c_void_p(out.data_ptr()), None, None, None)
        assert st == rt.RT_OK, L.rt_last_error()
    torch.cuda.synchronize()
    assert high() == 0
