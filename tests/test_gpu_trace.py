"""GPU parity of rt_trace / rt_tally (Section 3 Monte-Carlo ray tracing)
against the FP64 oracle on the same Philox rays.

Tolerances: cell-visit sequences and segment lengths are specified in binary32
and must be bit-exact; per-cell absorbed power within 1e-4 relative for cells
whose oracle tally is >= 1e-6 of the largest, else within 1e-10 of the emitted
power; the GPU's binary64 energy balance within 1e-5 (deposits are binary32).
"""
import ctypes as ct
import math

import numpy as np
import pytest

import synth
from oracle import kappa as okappa
from oracle import trace as otrace

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_cs_0703028_gb300 as rt
    rt.lib()
    return rt


def _tables_equal_input(rt, K64):
    import torch
    return torch.from_numpy(K64.astype(np.float32)).cuda()


def _check_tally(ab_gpu, ab_ref, emitted):
    big = ab_ref >= 1e-6 * ab_ref.max()
    rel = np.abs(ab_gpu[big] - ab_ref[big]) / ab_ref[big]
    assert rel.max() <= 1e-4, rel.max()
    small = ~big
    assert np.all(np.abs(ab_gpu[small] - ab_ref[small]) <= 1e-10 * emitted)


def _run(rt, grid, spec, kap_dev, n, seed=0, ray_begin=0, n_total=None, flags=0, rec_n=0):
    gs, keep = rt.make_grid(grid)
    tally = rt.Tally(grid.ncells)
    tally.zero()
    rec = rt.Record(rec_n, grid.nx + grid.ny + grid.nz + 4) if rec_n else None
    rt.trace(gs, kap_dev, spec, tally, n_rays=n, ray_begin=ray_begin, n_rays_total=n_total or n,
             seed=seed, flags=flags, record=rec)
    ab, sc, st = tally.read()
    return ab, sc, int(tally.steps.item()), rec


def test_c0_slab_walk_with_oracle_table(rt):
    # the walk alone: both sides use the oracle's table (GPU: rounded to binary32)
    case = synth.config(0)
    K = okappa.kappa_table(case.lines, case.spec)
    ab, sc, steps, _ = _run(rt, case.grid, case.spec, _tables_equal_input(rt, K), case.n_rays)
    K32 = K.astype(np.float32).astype(np.float64)
    o = otrace.trace(case.grid, case.spec, K32, n_rays=case.n_rays)
    _check_tally(ab, o.absorbed, o.emitted)
    assert steps == o.steps
    assert sc[0] == pytest.approx(o.emitted, rel=1e-5)
    assert sc[2] == pytest.approx(o.escaped, rel=1e-4)
    assert sc[3] < 1e-5


def test_c0_slab_end_to_end(rt):
    case = synth.config(0)
    kap = rt.build_kappa(case.lines, case.spec)
    ab, sc, steps, _ = _run(rt, case.grid, case.spec, kap, case.n_rays)
    o = otrace.trace_case(case)
    _check_tally(ab, o.absorbed, o.emitted)
    assert sc[0] == pytest.approx(o.emitted, rel=1e-5)


def test_c0_isothermal_column_beam(rt):
    # escaped / injected = exp(-kappa_j L) for every nu_j; compared as optical
    # depth -ln(escaped) against the oracle's kappa_j * 100 * L within 1e-5
    # relative while the transmitted fraction is a normal binary32 (> 1e-30).
    # With x = 0.1 this column is opaque at every wavenumber (tau >= 270), so the
    # absorber is diluted to x = 1e-4 (table and field alike): tau from 0.27 up.
    from dataclasses import replace
    case = synth.config(0)
    spec = replace(case.spec, x_ref=1e-4)
    grid = synth.uniform_grid(64, 1, 1, 1.0 / 64, math.inf, math.inf, 1000.0, 1.0, 1e-4)
    kap = rt.build_kappa(case.lines, spec)
    n = spec.n_nu
    ab, sc, steps, rec = _run(rt, grid, spec, kap, n, flags=rt.RT_SRC_BEAM, rec_n=n)
    esc = rec.escaped.cpu().numpy().astype(np.float64)
    tau_ref = okappa.kappa_table(case.lines, spec)[0] * 100.0 * 1.0
    ok = esc > 1e-30
    assert ok.sum() > 5000
    assert np.allclose(-np.log(esc[ok]), tau_ref[ok], rtol=1e-5, atol=0)
    assert np.all(esc[tau_ref > 80] < 1e-30)
    assert np.all(rec.n_visits.cpu().numpy() == 64)
    assert steps == 64 * n


def test_visit_sequences_bit_exact_c1_geometry(rt):
    case = synth.config(1)
    K = np.full((case.spec.nT, case.spec.n_nu), 1e-3)
    n = 10000
    import torch
    kd = torch.full((case.spec.nT, case.spec.n_nu), 1e-3, dtype=torch.float32, device="cuda")
    ab, sc, steps, rec = _run(rt, case.grid, case.spec, kd, n, n_total=case.n_rays, rec_n=n)
    o = otrace.trace(case.grid, case.spec, K, n_rays=n, n_total=case.n_rays, n_record=n)
    nv = rec.n_visits.cpu().numpy()
    assert np.array_equal(nv, o.rec["n"])
    cells = rec.cells.cpu().numpy()
    ds = rec.ds.cpu().numpy()
    mask = np.arange(cells.shape[1])[None, :] < nv[:, None]
    assert np.array_equal(cells[mask], o.rec["cells"][mask])
    assert np.array_equal(ds[mask].view(np.uint32), o.rec["ds"][mask].view(np.uint32))
    assert steps == o.steps


@pytest.mark.parametrize("tau_cut", [False, True])
def test_uneven_grid_with_pressure_field(rt, tau_cut):
    # anisotropic cells, p and x fields (density scale), T clamped at both ends
    rng = synth.rng_for(9, 5)
    g = synth.gaussian_hotspot_grid(9, 0.9, 700.0, 2100.0, 0.2, dims=(9, 6, 4))
    g.hy, g.hz = 0.13, 0.21
    g.p_atm = rng.uniform(0.5, 3.0, g.ncells).astype(np.float32)
    g.x = rng.uniform(0.05, 0.2, g.ncells).astype(np.float32)
    lines = synth.make_lines(300, 2000.0, 2100.0, rng)
    spec = synth.Spectral(nu_min=2020.0, dnu=0.02, n_nu=3000, cutoff=25.0, profile="voigt",
                          nT=6, T_min=800.0, T_max=2000.0, p_ref_atm=1.0, x_ref=0.1)
    K = okappa.kappa_table(lines, spec)
    n = 50000
    flags = rt.RT_TAU_CUT if tau_cut else 0
    ab, sc, steps, _ = _run(rt, g, spec, _tables_equal_input(rt, K), n, seed=5, flags=flags)
    o = otrace.trace(g, spec, K.astype(np.float32).astype(np.float64), seed=5, n_rays=n,
                     tau_cut=tau_cut)
    _check_tally(ab, o.absorbed, o.emitted)
    assert steps == o.steps
    assert sc[3] < 1e-5


def test_ray_ranges_accumulate(rt):
    import torch
    case = synth.config(0)
    kap = rt.build_kappa(case.lines, case.spec)
    gs, keep = rt.make_grid(case.grid)
    t1, t2 = rt.Tally(64), rt.Tally(64)
    t1.zero(); t2.zero()
    n = 40000
    rt.trace(gs, kap, case.spec, t1, n_rays=n, n_rays_total=n)
    rt.trace(gs, kap, case.spec, t2, n_rays=n // 2, ray_begin=0, n_rays_total=n)
    rt.trace(gs, kap, case.spec, t2, n_rays=n // 2, ray_begin=n // 2, n_rays_total=n)
    a1, s1, _ = t1.read()
    a2, s2, _ = t2.read()
    assert np.allclose(a1, a2, rtol=1e-12, atol=0)
    assert s1[0] == pytest.approx(s2[0], rel=1e-12)


def test_nonfinite_temperature_reported(rt):
    case = synth.config(0)
    g = synth.uniform_grid(64, 1, 1, 1 / 64, math.inf, math.inf, 1000.0)
    g.T[10] = np.nan
    kap = rt.build_kappa(case.lines, case.spec)
    gs, keep = rt.make_grid(g)
    tally = rt.Tally(64)
    tally.zero()
    rt.trace(gs, kap, case.spec, tally, n_rays=1000)
    ab, sc, st = tally.read(check=False)
    assert st == rt.RT_E_NONFINITE


@pytest.fixture(scope="module")
def c1_full_gpu(rt):
    """Full-size workload in the benchmark's launch configuration: the 64 x 100k
    table and all 1e7 rays, recording the first 2000 rays."""
    case = synth.config(1)
    kap = rt.build_kappa(case.lines, case.spec)
    ab, sc, steps, rec = _run(rt, case.grid, case.spec, kap, case.n_rays, rec_n=2000)
    return case, ab, sc, steps, rec


def test_c1_full_run_sampled_rays_and_balance(rt, c1_full_gpu):
    case, ab, sc, steps, rec = c1_full_gpu
    n = 2000
    o = otrace.trace_case(case, n_rays=n, n_record=n)
    # the sampled rays' weights, walls and visits against the oracle
    w = rec.weight.cpu().numpy().astype(np.float64)
    esc = rec.escaped.cpu().numpy().astype(np.float64)
    assert np.allclose(w, o.rec["w"], rtol=1e-4, atol=0)
    # walls: compared as the ray's optical depth -ln(escaped / w), whose error is
    # the table's relative error (<= 1e-5) times tau, while escaped / w is a normal
    # binary32 value
    frac_g = esc / w
    frac_o = o.rec["escaped"] / o.rec["w"]
    ok = frac_g > 1e-30
    tau_g, tau_o = -np.log(frac_g[ok]), -np.log(frac_o[ok])
    assert np.all(np.abs(tau_g - tau_o) <= 2e-5 * tau_o + 1e-5)
    assert np.all(frac_o[~ok] < 1e-25)
    assert np.array_equal(rec.n_visits.cpu().numpy(), o.rec["n"])
    # whole run: energy balance and plausibility
    assert sc[3] < 1e-5
    assert np.all(ab >= 0) and np.all(np.isfinite(ab))
    assert steps > case.n_rays


def test_c1_ray_subset_tallies(rt):
    case = synth.config(1)
    kap = rt.build_kappa(case.lines, case.spec)
    n = 1500
    ab, sc, steps, _ = _run(rt, case.grid, case.spec, kap, n, n_total=case.n_rays)
    o = otrace.trace_case(case, n_rays=n)
    _check_tally(ab, o.absorbed, o.emitted)
    assert steps == o.steps
    assert sc[0] == pytest.approx(o.emitted, rel=1e-5)


def _with_group(rt, mode, fn):
    before = rt.get_tuning()
    try:
        rt.set_tuning(walk_group=mode)
        return fn()
    finally:
        rt.set_tuning(**before)


def test_wavenumber_grouped_walk_matches_oracle(rt):
    # The walk over rays grouped by wavenumber (walk_group = 2: counting pass over the
    # rays' Philox draws, warps walk runs of equal-wavenumber rays) traces the same
    # rays: per-cell tallies against the oracle at 1e-4, against the ungrouped walk up
    # to the binary64 summation order, the same step count.
    case = synth.config(1)
    kap = rt.build_kappa(case.lines, case.spec)
    n = 1500
    ab_g, sc_g, st_g, _ = _with_group(rt, 2, lambda: _run(rt, case.grid, case.spec, kap, n, n_total=case.n_rays))
    ab_u, sc_u, st_u, _ = _with_group(rt, 1, lambda: _run(rt, case.grid, case.spec, kap, n, n_total=case.n_rays))
    o = otrace.trace_case(case, n_rays=n)
    _check_tally(ab_g, o.absorbed, o.emitted)
    assert st_g == o.steps == st_u
    assert np.allclose(ab_g, ab_u, rtol=1e-12, atol=1e-13 * ab_u.max())
    assert sc_g[0] == pytest.approx(sc_u[0], rel=1e-12)


def test_wavenumber_grouped_walk_records_bit_exact_visits(rt):
    # record rows follow the ray's index, whatever order the grouped walk takes the rays in;
    # many rays per wavenumber (n_nu = 64): the grouping runs through its shared histogram
    import torch
    spec = synth.Spectral(nu_min=2000.0, dnu=0.5, n_nu=64, cutoff=25.0, profile="voigt", nT=13,
                          T_min=800.0, T_max=2000.0)
    g = synth.gaussian_hotspot_grid(12, 1.0, 800.0, 2000.0, 0.2, dims=(12, 9, 7))
    K = np.full((spec.nT, spec.n_nu), 2e-3)
    kd = torch.full((spec.nT, spec.n_nu), 2e-3, dtype=torch.float32, device="cuda")
    n = 8000
    ab, sc, steps, rec = _with_group(rt, 2, lambda: _run(rt, g, spec, kd, n, seed=3, rec_n=n))
    o = otrace.trace(g, spec, K, seed=3, n_rays=n, n_record=n)
    nv = rec.n_visits.cpu().numpy()
    assert np.array_equal(nv, o.rec["n"])
    cells = rec.cells.cpu().numpy()
    mask = np.arange(cells.shape[1])[None, :] < nv[:, None]
    assert np.array_equal(cells[mask], o.rec["cells"][mask])
    assert np.array_equal(rec.ds.cpu().numpy()[mask].view(np.uint32), o.rec["ds"][mask].view(np.uint32))
    _check_tally(ab, o.absorbed, o.emitted)
