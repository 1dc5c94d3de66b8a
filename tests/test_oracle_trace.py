"""Pins of the FP64 ray-tracing oracle (Section 3, Fig. ray, Eq. I first term,
Eq. planck) against an independent Philox implementation, closed forms of
plane-parallel radiative exchange, brute-force quadrature of the estimator and
geometric invariants of the cell walk."""
import ctypes
import ctypes.util
import math
import os

import numpy as np
import pytest
from scipy.special import expn

import synth
from oracle import kappa as K
from oracle import physics as ph
from oracle import trace as OT

SIGMA_SB = 5.670374419e-8


# ---------------------------------------------------------------- Philox
def _curand():
    cands = [os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64", "libcurand.so"),
             "/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")]
    for c in cands:
        if c and os.path.exists(c):
            return ctypes.CDLL(c)
    pytest.skip("libcurand not found")


def _curand_host_philox(seed, nblocks):
    lib = _curand()
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0   # PHILOX4_32_10
    assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
    out = np.zeros(4 * nblocks, dtype=np.uint32)
    assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
    lib.curandDestroyGenerator(gen)
    return out.reshape(-1, 4)


@pytest.mark.parametrize("seed", [0, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_cuda_host_generator(seed):
    # The CUDA toolkit's host Philox4x32-10 generator lays out output block b at
    # counter (b >> 16, 0, b & 0xffff, 0) under key (seed_lo, seed_hi).
    blocks = [0, 1, 2, 3, 4095, 65535, 65536, 65537, 70001]
    ref = _curand_host_philox(seed, max(blocks) + 1)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for b in blocks:
        got = OT.philox4x32_10([b >> 16, 0, b & 0xFFFF, 0], key)
        assert np.array_equal(got, ref[b]), b


# ---------------------------------------------------------------- helpers
def _slab4(kappa_nodes=(0.002, 0.02), T_cells=(600.0, 900.0, 1200.0, 1400.0), h=0.25):
    """4-cell plane-parallel slab, one spectral sample, kappa linear in T between 2 nodes."""
    spec = synth.Spectral(nu_min=2300.0, dnu=1.0, n_nu=1, cutoff=25.0, profile="lorentz",
                          nT=2, T_min=500.0, T_max=1500.0)
    grid = synth.Grid(4, 1, 1, h, math.inf, math.inf, np.array(T_cells, dtype=np.float32))
    tab = np.array([[kappa_nodes[0]], [kappa_nodes[1]]], dtype=np.float64)
    return spec, grid, tab


def _slab_cell_kappa(spec, grid, tab):
    k, fr, sc = OT.cell_prep(grid, spec)
    return np.array([(1 - float(f)) * tab[kk, 0] + float(f) * tab[kk + 1, 0] for kk, f in zip(k, fr)])


def _e3_exchange(kap_m, Ib, h, dnu_m):
    """Closed-form plane-parallel exchange matrix P[i, j] (W/m^2) and wall losses."""
    n = len(kap_m)
    tau = kap_m * h
    P = np.zeros((n, n))
    walls = np.zeros(n)
    E3 = lambda x: expn(3, x)
    for i in range(n):
        emit = 4 * math.pi * kap_m[i] * h * Ib[i] * dnu_m
        for j in range(n):
            if j == i:
                continue
            lo, hi = min(i, j), max(i, j)
            tg = tau[lo + 1:hi].sum()
            P[i, j] = 2 * math.pi * Ib[i] * dnu_m * (E3(tg) - E3(tg + tau[i]) - E3(tg + tau[j])
                                                     + E3(tg + tau[i] + tau[j]))
        tl, tr = tau[:i].sum(), tau[i + 1:].sum()
        walls[i] = 2 * math.pi * Ib[i] * dnu_m * (E3(tl) - E3(tl + tau[i]) + E3(tr) - E3(tr + tau[i]))
        P[i, i] = emit - 2 * math.pi * Ib[i] * dnu_m * (1 - 2 * E3(tau[i]))
    return P, walls


def test_slab_exchange_closed_form_is_conservative():
    spec, grid, tab = _slab4()
    kap = 100 * _slab_cell_kappa(spec, grid, tab)
    Ib = ph.planck_wavenumber(2300.0, grid.T.astype(np.float64))
    P, walls = _e3_exchange(kap, Ib, 0.25, 100.0)
    emit = 4 * math.pi * kap * 0.25 * Ib * 100.0
    assert np.allclose(P.sum(1) + walls, emit, rtol=1e-13)


def test_slab_bruteforce_estimator_matches_e3():
    # Deterministic expectation of the estimator: midpoint quadrature over the
    # emission position x in each cell and the direction cosine mu.
    spec, grid, tab = _slab4()
    kap = 100 * _slab_cell_kappa(spec, grid, tab)
    Ib = ph.planck_wavenumber(2300.0, grid.T.astype(np.float64))
    P, walls = _e3_exchange(kap, Ib, 0.25, 100.0)
    nx_, nmu = 512, 2048
    got = np.zeros((4, 4))
    got_w = np.zeros(4)
    for i in range(4):
        emit = 4 * math.pi * kap[i] * 0.25 * Ib[i] * 100.0
        fx = ((np.arange(nx_) + 0.5) / nx_).astype(np.float32)
        mu = (-1 + (np.arange(nmu) + 0.5) * (2.0 / nmu))
        X, M = np.meshgrid(fx, mu, indexing="ij")
        n = X.size
        pos = np.zeros((n, 3), np.float32)
        pos[:, 0] = (np.float32(i) + X.ravel().astype(np.float32)) * np.float32(0.25)
        d = np.zeros((n, 3), np.float32)
        d[:, 0] = M.ravel()
        d[:, 1] = np.sqrt(1 - M.ravel() ** 2)
        ix3 = np.zeros((n, 3), np.int32)
        ix3[:, 0] = i
        ab, esc = OT.walk_rays(grid, spec, tab, ix3, pos, d, np.zeros(n, np.int64),
                               np.full(n, emit / n))
        got[i] = ab
        got_w[i] = esc.sum()
    assert np.allclose(got, P, rtol=2e-6, atol=1e-9 * P.max())
    assert np.allclose(got_w, walls, rtol=2e-6)


def test_slab_monte_carlo_within_4_sigma_of_e3():
    spec, grid, tab = _slab4()
    kap = 100 * _slab_cell_kappa(spec, grid, tab)
    Ib = ph.planck_wavenumber(2300.0, grid.T.astype(np.float64))
    P, walls = _e3_exchange(kap, Ib, 0.25, 100.0)
    expect = P.sum(0)
    nb, per = 16, 200_000
    runs = []
    for b in range(nb):
        r = OT.trace(grid, spec, tab, seed=7, ray_begin=b * per, n_rays=per, n_total=per)
        runs.append(np.concatenate([r.absorbed, [r.escaped, r.emitted]]))
        assert r.energy_residual < 1e-12
    runs = np.array(runs)
    mean = runs.mean(0)
    sem = runs.std(0, ddof=1) / math.sqrt(nb)
    full = np.concatenate([expect, [walls.sum(), (4 * math.pi * kap * 0.25 * Ib * 100).sum()]])
    assert np.all(np.abs(mean - full) <= 4 * sem + 1e-12 * full.max()), (mean, full, sem)


def test_isothermal_column_beam_transmissivity():
    # Every wavenumber of the 1-D isothermal column: escaped / injected = exp(-kappa L).
    case = synth.config(0)
    tab = K.kappa_table(case.lines, case.spec)
    n = case.spec.n_nu
    r = OT.trace(case.grid, case.spec, tab, n_rays=n, mode=OT.MODE_BEAM, n_record=n)
    esc = r.rec["escaped"]
    tau = tab[0] * 100.0 * 1.0
    ok = tau < 700
    assert ok.sum() > 1000
    assert np.allclose(-np.log(esc[ok]), tau[ok], rtol=1e-13, atol=0)
    thin = tau < 30
    assert np.allclose(esc[thin], np.exp(-tau[thin]), rtol=1e-12)
    assert r.energy_residual < 1e-12
    # straight run through all 64 cells with ds = h
    assert np.all(r.rec["n"] == 64)
    assert np.array_equal(r.rec["cells"][0, :64], np.arange(64))
    assert np.all(r.rec["ds"][:, :64] == np.float32(1.0 / 64))


@pytest.mark.parametrize("cfg", [0, 1])
def test_energy_conservation(cfg):
    case = synth.config(cfg)
    n = 20000 if cfg == 0 else 3000
    r = OT.trace_case(case, n_rays=n)
    assert r.energy_residual < 1e-12
    assert r.absorbed_total > 0 and r.escaped > 0


def _chord(pos, d, n, h, bound=False):
    """float64 ray-box exit parameter of a ray stored in binary32; with bound=True
    also the rounding bound of the binary32 walk's exit: the wall plane (|wall|),
    the position (|x|) and the product with 1/d each carry half an ulp, amplified
    by 1/|d_a|, plus a few ulps of the result itself."""
    t, err = math.inf, 0.0
    u = 2.0 ** -24
    for a in range(3):
        if not math.isfinite(h[a]) or d[a] == 0:
            continue
        hf = float(np.float32(h[a]))
        wall = n[a] * hf if d[a] > 0 else 0.0
        ta = (wall - float(pos[a])) / float(d[a])
        if ta < t:
            t = ta
            err = u * (abs(wall) + abs(float(pos[a]))) / abs(float(d[a])) + 8 * u * ta
    return (t, err) if bound else t


def test_walk_geometry_invariants():
    grid = synth.gaussian_hotspot_grid(11, 1.0, 800.0, 2000.0, 0.2, dims=(11, 7, 5))
    spec = synth.Spectral(nu_min=2000.0, dnu=0.1, n_nu=10, nT=2, T_min=800.0, T_max=2000.0)
    tab = np.full((2, 10), 1e-3)
    n = 4000
    r = OT.trace(grid, spec, tab, seed=3, n_rays=n, n_record=n)
    cell, j, pos, dirs, w = OT.sample_rays(grid, spec, tab, seed=3, n=n)
    h = (grid.hx, grid.hy, grid.hz)
    dims = (grid.nx, grid.ny, grid.nz)
    for k in range(n):
        nv = r.rec["n"][k]
        cells = r.rec["cells"][k, :nv]
        ds = r.rec["ds"][k, :nv].astype(np.float64)
        assert cells[0] == cell[k]
        # sum of segment lengths = ray-box chord (parameter units of the stored direction)
        chord, err = _chord(pos[k], dirs[k], dims, h, bound=True)
        assert abs(ds.sum() - chord) <= err, (k, ds.sum(), chord, err)
        # consecutive visits are face neighbours
        ix = np.stack([cells % 11, (cells // 11) % 7, cells // 77], 1)
        assert np.all(np.abs(np.diff(ix, axis=0)).sum(1) == 1)
        assert nv <= 11 + 7 + 5
        assert np.all(ds >= 0)


def test_walk_matches_dense_sampling_of_the_segment():
    # Brute force: sample the float64 ray densely; the distinct cells it passes
    # equal the walk's visits with positive length.
    grid = synth.uniform_grid(6, 5, 4, 0.2, 0.25, 0.3, 1000.0)
    spec = synth.Spectral(nu_min=2000.0, dnu=0.1, n_nu=4, nT=1, T_min=1000.0, T_max=1000.0)
    tab = np.full((1, 4), 1e-3)
    n = 500
    r = OT.trace(grid, spec, tab, seed=11, n_rays=n, n_record=n)
    cell, j, pos, dirs, w = OT.sample_rays(grid, spec, tab, seed=11, n=n)
    h = np.array([0.2, 0.25, 0.3], dtype=np.float32).astype(np.float64)   # the walk's binary32 sizes
    checked = 0
    for k in range(n):
        nv = r.rec["n"][k]
        ds = r.rec["ds"][k, :nv]
        if np.any((ds > 0) & (ds < 1e-4)):
            continue  # near a cell edge: dense sampling cannot resolve it
        chord = _chord(pos[k], dirs[k], (6, 5, 4), h)
        ts = (np.arange(200000) + 0.5) / 200000 * chord
        p = pos[k].astype(np.float64)[None, :] + ts[:, None] * dirs[k].astype(np.float64)[None, :]
        ii = np.floor(p / h).astype(np.int64)
        ii = np.minimum(ii, np.array([5, 4, 3]))   # samples within rounding of the far wall
        flat = ii[:, 0] + 6 * (ii[:, 1] + 5 * ii[:, 2])
        seq = flat[np.concatenate(([True], flat[1:] != flat[:-1]))]
        vis = r.rec["cells"][k, :nv][ds > 0]
        assert np.array_equal(seq, vis), k
        checked += 1
    assert checked > 400


def test_emission_weights_gray_medium_stefan_boltzmann():
    # Gray absorber (kappa independent of nu) in one isothermal cell: the sum of the
    # per-(cell, nu) emitted powers over a wide spectral grid is 4 kappa sigma T^4 V.
    T = 1200.0
    spec = synth.Spectral(nu_min=1.0, dnu=2.0, n_nu=12000, nT=1, T_min=T, T_max=T)   # midpoints
    grid = synth.uniform_grid(1, 1, 1, 0.1, 0.2, 0.3, T)
    kap_cm = 0.01
    tab = np.full((1, spec.n_nu), kap_cm)
    n = 400000
    cell, j, pos, dirs, w = OT.sample_rays(grid, spec, tab, seed=1, n=n, n_total=n)
    P = w * n / (1 * spec.n_nu)               # power of each sampled (cell, j)
    uj, first = np.unique(j, return_index=True)
    assert uj.size == spec.n_nu
    total = P[first].sum()
    V = 0.1 * 0.2 * 0.3
    assert total == pytest.approx(4 * (100 * kap_cm) * SIGMA_SB * T ** 4 * V, rel=1e-6)


def test_directions_are_unit_and_isotropic():
    grid = synth.uniform_grid(8, 8, 8, 0.125, 0.125, 0.125, 1000.0)
    spec = synth.Spectral(nu_min=2000.0, dnu=0.1, n_nu=4, nT=1, T_min=1000.0, T_max=1000.0)
    tab = np.full((1, 4), 1e-3)
    n = 200000
    cell, j, pos, dirs, w = OT.sample_rays(grid, spec, tab, seed=5, n=n)
    d = dirs.astype(np.float64)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=4e-7)
    assert np.all(np.abs(d.mean(0)) < 4 * math.sqrt(1 / 3 / n))
    assert np.allclose((d ** 2).mean(0), 1 / 3, atol=4 * math.sqrt(4 / 45 / n))
    # positions inside their cells, cells and j uniform
    ix = np.stack([cell % 8, (cell // 8) % 8, cell // 64], 1)
    assert np.all((pos >= ix * 0.125) & (pos <= (ix + 1) * 0.125))
    cnt = np.bincount(cell, minlength=512)
    assert cnt.min() > 0.7 * n / 512


def test_cell_prep_brackets():
    spec = synth.Spectral(nu_min=2000.0, dnu=0.1, n_nu=4, nT=5, T_min=800.0, T_max=1600.0)
    T = np.array([800.0, 1000.0, 1100.0, 1600.0, 700.0, 1700.0, 1599.0], dtype=np.float32)
    grid = synth.Grid(7, 1, 1, 0.1, 0.1, 0.1, T, np.full(7, 2.0, np.float32),
                      np.full(7, 0.05, np.float32))
    k, fr, sc = OT.cell_prep(grid, spec)
    assert list(k) == [0, 1, 1, 3, 0, 3, 3]
    assert np.allclose(fr, [0, 0, 0.5, 1, 0, 1, 199 / 200], atol=1e-6)
    # density scale (p x) / (p_ref x_ref) with the table at 1 atm, x = 0.1: here p x = p_ref x_ref
    assert np.allclose(sc, 1.0, atol=1e-7)


def test_cell_density_scale_is_the_number_density_ratio():
    # u_g of Eq. tau is x p / (k_B T); the table holds it at (p_ref, x_ref) and the cell's own
    # T through the node bracket, so a cell's kappa is scaled by (p x) / (p_ref x_ref).  Cells
    # with p x != p_ref x_ref: an inverted ratio, a dropped factor or a p- or x-only scale fails.
    T = np.full(7, 1000.0, dtype=np.float32)
    p = np.array([2.0, 1.0, 3.0, 0.5, 1.5, 2.5, 1.2], dtype=np.float32)
    x = np.array([0.1, 0.05, 0.2, 0.3, 0.05, 0.01, 0.15], dtype=np.float32)
    for p_ref, x_ref in ((1.0, 0.1), (1.5, 0.05)):
        spec = synth.Spectral(nu_min=2000.0, dnu=0.1, n_nu=4, nT=5, T_min=800.0, T_max=1600.0,
                              p_ref_atm=p_ref, x_ref=x_ref)
        grid = synth.Grid(7, 1, 1, 0.1, 0.1, 0.1, T, p, x)
        _, _, sc = OT.cell_prep(grid, spec)
        expect = p.astype(np.float64) * x.astype(np.float64) / (p_ref * x_ref)
        assert np.allclose(sc, expect, rtol=3e-7, atol=0), (p_ref, x_ref, sc, expect)
        if p_ref == 1.0:
            assert sc[0] == pytest.approx(2.0, rel=1e-7) and sc[1] == pytest.approx(0.5, rel=1e-7)
        # a missing field stands for the table's reference value
        _, _, sp = OT.cell_prep(synth.Grid(7, 1, 1, 0.1, 0.1, 0.1, T, p, None), spec)
        _, _, sx = OT.cell_prep(synth.Grid(7, 1, 1, 0.1, 0.1, 0.1, T, None, x), spec)
        assert np.allclose(sp, p.astype(np.float64) / p_ref, rtol=3e-7, atol=0)
        assert np.allclose(sx, x.astype(np.float64) / x_ref, rtol=3e-7, atol=0)


def test_per_cell_kappa_beam_through_a_layered_slab():
    # Per-cell kappa (each cell's own value, no T interpolation): a collimated beam
    # through a slab of 16 layers with kappa varying by layer and wavenumber is
    # attenuated by exp(-100 h sum_c kappa_c) (Beer-Lambert, Eq. I first term), and
    # layer c absorbs exp(-tau_<c) - exp(-tau_<=c) of it.
    nc, n_nu, h = 16, 64, 1.0 / 16
    spec = synth.Spectral(nu_min=2000.0, dnu=0.5, n_nu=n_nu, nT=2, T_min=800.0, T_max=1600.0)
    grid = synth.Grid(nc, 1, 1, h, math.inf, math.inf, np.linspace(800, 1600, nc).astype(np.float32))
    c = np.arange(nc)[:, None]
    j = np.arange(n_nu)[None, :]
    Kc = 0.02 * (1.0 + c) * (0.25 + np.sin(0.3 * j + 0.7 * c) ** 2)
    r = OT.trace(grid, spec, Kc, n_rays=n_nu, mode=OT.MODE_BEAM, n_record=n_nu, per_cell=True)
    tau_cum = np.concatenate([np.zeros((1, n_nu)), np.cumsum(100.0 * h * Kc, axis=0)])
    assert np.allclose(r.rec["escaped"], np.exp(-tau_cum[-1]), rtol=1e-12, atol=0)
    layer = (np.exp(-tau_cum[:-1]) - np.exp(-tau_cum[1:])).sum(axis=1)
    assert np.allclose(r.absorbed, layer, rtol=1e-12, atol=0)
    assert r.energy_residual < 1e-12


def test_per_cell_kappa_emission_is_each_cells_own_gray_emission():
    # Gray cells at their own temperature and kappa: the per-(cell, nu) emitted powers
    # summed over a wide grid give 4 kappa_c sigma T_c^4 V per cell, with kappa_c the
    # cell's own value (the table's T bracket and density scale are not applied).
    Ts = np.array([900.0, 1200.0, 1500.0], dtype=np.float32)
    spec = synth.Spectral(nu_min=1.0, dnu=2.0, n_nu=12000, nT=2, T_min=500.0, T_max=2500.0,
                          p_ref_atm=1.0, x_ref=0.1)
    grid = synth.Grid(3, 1, 1, 0.1, 0.2, 0.3, Ts, np.full(3, 2.0, np.float32), np.full(3, 0.2, np.float32))
    kc = np.array([0.01, 0.003, 0.02])
    Kc = np.repeat(kc[:, None], spec.n_nu, axis=1)
    n = 2_000_000
    cell, j, pos, dirs, w = OT.sample_rays(grid, spec, Kc, seed=2, n=n, n_total=n, per_cell=True)
    P = w * n / (3 * spec.n_nu)
    key = cell * spec.n_nu + j
    uk, first = np.unique(key, return_index=True)
    assert uk.size == 3 * spec.n_nu
    per_cell = np.bincount(cell[first], weights=P[first], minlength=3)
    V = 0.1 * 0.2 * 0.3
    expect = 4 * (100 * kc) * SIGMA_SB * Ts.astype(np.float64) ** 4 * V
    assert np.allclose(per_cell, expect, rtol=1e-6, atol=0)
