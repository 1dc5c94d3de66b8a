"""GPU parity of the two alternative walks.

* rt_trace_lbl sums the lines at each visited cell's own state.  On cells whose
  temperatures are table nodes, at the table's pressure and mole fraction, that
  equals the oracle's table walk: per-cell tallies within 1e-4 relative (cells
  >= 1e-6 of the largest), as for rt_trace.
* rt_trace_mlp with a network whose output is the constant log kappa0 must give
  the table walk's tallies for the constant table kappa0 (no BF16 rounding is
  involved: zero weights give exact zero activations), within 1e-5.
"""
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


def _node_grid(seed=0, n=8):
    rng = np.random.default_rng(seed)
    T = (800.0 + 100.0 * rng.integers(0, 13, n ** 3)).astype(np.float32)
    return synth.Grid(n, n, n, 1.0 / n, 1.0 / n, 1.0 / n, T, np.full(n ** 3, 1.0, np.float32),
                      np.full(n ** 3, 0.1, np.float32))


def _tally(rt, run, ncells):
    t = rt.Tally(ncells)
    t.zero()
    run(t)
    ab, sc, st = t.read()
    return ab, sc, int(t.steps.item())


def _close(ab, ref, emitted, rtol):
    big = ref >= 1e-6 * ref.max()
    assert np.max(np.abs(ab[big] - ref[big]) / ref[big]) <= rtol
    assert np.all(np.abs(ab[~big] - ref[~big]) <= 1e-10 * emitted)


@pytest.mark.parametrize("profile", ["voigt", "lorentz"])
def test_lbl_walk_matches_oracle_on_node_temperatures(rt, profile):
    rng = synth.rng_for(9, 40)
    lines = synth.make_lines(300, 2000.0, 2060.0, rng)
    spec = synth.Spectral(nu_min=2010.0, dnu=0.02, n_nu=2000, cutoff=25.0, profile=profile,
                          nT=13, T_min=800.0, T_max=2000.0, p_ref_atm=1.0, x_ref=0.1)
    g = _node_grid()
    gs, keep = rt.make_grid(g)
    n = 20000
    ab, sc, steps = _tally(rt, lambda t: rt.trace_lbl(gs, lines, spec, t, n_rays=n, seed=4), g.ncells)
    K = okappa.kappa_table(lines, spec)
    o = otrace.trace(g, spec, K, seed=4, n_rays=n)
    _close(ab, o.absorbed, o.emitted, 1e-4)
    assert steps == o.steps
    assert sc[0] == pytest.approx(o.emitted, rel=2e-5)
    assert sc[3] < 1e-5


def test_mlp_walk_with_constant_network_matches_table_walk(rt):
    import torch
    case = synth.config(1)
    g = synth.gaussian_hotspot_grid(12, 1.0, 800.0, 2000.0, 0.2)
    spec = case.spec
    kappa0 = 0.37
    off = synth.mlp_offsets()
    params = np.zeros(synth.MLP_NPARAM, np.float32)
    mean, scale = -1.0, 2.0
    params[off["b5"][0]] = (math.log(kappa0) - mean) / scale
    norm = rt.make_norm([math.log(2000.0), 600.0, 0.5, 0.01], [math.log(3000.0), 2200.0, 5.0, 0.3],
                        mean, scale)
    gs, keep = rt.make_grid(g)
    n = 30000
    P = torch.from_numpy(params).cuda()
    ab_m, sc_m, st_m = _tally(rt, lambda t: rt.trace_mlp(gs, P, norm, spec, t, n_rays=n, seed=2), g.ncells)
    tab = torch.full((spec.nT, spec.n_nu), kappa0, dtype=torch.float32, device="cuda")
    ab_t, sc_t, st_t = _tally(rt, lambda t: rt.trace(gs, tab, spec, t, n_rays=n, seed=2), g.ncells)
    assert st_m == st_t
    _close(ab_m, ab_t, sc_t[0], 1e-5)
    assert sc_m[0] == pytest.approx(sc_t[0], rel=1e-5)
    assert sc_m[3] < 1e-5


def test_mlp_walk_matches_table_of_the_same_network(rt):
    # A random network tabulated with rt_mlp_forward (binary32 first layer and SiLU) at
    # the T nodes: on cells whose temperatures are nodes (p, x at the reference), the
    # surrogate walk (first layer as a split-BF16 tensor-core product, packed-BF16 SiLU)
    # must reproduce the table walk's tallies to within the BF16 activation rounding.
    import torch
    spec = synth.Spectral(nu_min=2000.0, dnu=0.02, n_nu=2000, cutoff=25.0, profile="voigt", nT=13,
                          T_min=800.0, T_max=2000.0, p_ref_atm=1.0, x_ref=0.1)
    g = _node_grid(4)
    params = synth.mlp_init(3)
    lo = [math.log(2000.0), 600.0, 0.5, 0.01]
    hi = [math.log(3000.0), 2200.0, 5.0, 0.3]
    norm = rt.make_norm(lo, hi, -3.0, 1.0)
    P = torch.from_numpy(params).cuda()
    j = np.arange(spec.n_nu, dtype=np.float32)
    nu = (j * np.float32(spec.dnu) + np.float32(spec.nu_min)).astype(np.float32)
    T_nodes = np.asarray(spec.T_nodes(), dtype=np.float32)
    raw = np.zeros((spec.nT, spec.n_nu, 4), np.float32)
    raw[..., 0] = np.log(nu)[None, :]
    raw[..., 1] = T_nodes[:, None]
    raw[..., 2] = 1.0
    raw[..., 3] = 0.1
    logk = rt.mlp_forward(P, norm, torch.from_numpy(raw.reshape(-1, 4)).cuda())
    tab = torch.exp(logk).reshape(spec.nT, spec.n_nu).contiguous()
    gs, keep = rt.make_grid(g)
    n = 40000
    ab_m, sc_m, st_m = _tally(rt, lambda t: rt.trace_mlp(gs, P, norm, spec, t, n_rays=n, seed=5), g.ncells)
    ab_t, sc_t, st_t = _tally(rt, lambda t: rt.trace(gs, tab, spec, t, n_rays=n, seed=5), g.ncells)
    assert st_m == st_t  # the same rays and visits
    big = ab_t >= 1e-3 * ab_t.max()
    rel = np.abs(ab_m[big] - ab_t[big]) / ab_t[big]
    assert np.median(rel) < 1e-2 and rel.max() < 5e-2, (np.median(rel), rel.max())
    assert sc_m[0] == pytest.approx(sc_t[0], rel=1e-2)


def _oracle_logk(params, lo, hi, mean, scale, raw):
    """FP64 oracle network (oracle/mlp.py) at raw inputs (n, 4): mean + scale * y."""
    from oracle import mlp as omlp
    lo32 = np.asarray(lo, np.float32).astype(np.float64)   # the binding passes binary32 ranges
    hi32 = np.asarray(hi, np.float32).astype(np.float64)
    y, _ = omlp.forward(np.asarray(params, np.float64), omlp.normalise(raw, lo32, hi32))
    return float(np.float32(mean)) + float(np.float32(scale)) * y


def _mlp_case(rt, seed=3):
    """A random network whose output moves with every input: the initial first layer
    x3 and head x20 give log kappa an rms spread of about 0.18, of which 0.07-0.15 per
    input (an exchanged or dropped input changes the tallies by several per cent)."""
    import torch
    lo = [math.log(2000.0), 600.0, 0.5, 0.01]
    hi = [math.log(3000.0), 2200.0, 5.0, 0.3]
    params = synth.mlp_init(seed)
    off = synth.mlp_offsets()
    for name, f in (("W1", 3.0), ("w5", 20.0)):
        o, shape = off[name]
        params[o:o + int(np.prod(shape))] *= np.float32(f)
    norm = rt.make_norm(lo, hi, -3.0, 1.0)
    return params, torch.from_numpy(params).cuda(), norm, lo, hi


def test_mlp_walk_matches_oracle_on_node_temperatures(rt):
    # The surrogate walk against the FP64 oracle: oracle/mlp.py tabulates the same
    # network at (log nu_j, T_k, p_ref, x_ref) in binary64 and oracle/trace.c walks
    # the same rays through that table.  Cells sit on T nodes at the table's p and x,
    # so the table walk's kappa is the network's value at each cell exactly; the
    # difference is the BF16 rounding of the tensor-core products.
    spec = synth.Spectral(nu_min=2000.0, dnu=0.02, n_nu=2000, cutoff=25.0, profile="voigt", nT=13,
                          T_min=800.0, T_max=2000.0, p_ref_atm=1.0, x_ref=0.1)
    g = _node_grid(4)
    params, P, norm, lo, hi = _mlp_case(rt)
    nu = spec.nu_min + np.arange(spec.n_nu) * spec.dnu
    raw = np.zeros((spec.nT, spec.n_nu, 4))
    raw[..., 0] = np.log(nu)[None, :]
    raw[..., 1] = np.asarray(spec.T_nodes(), np.float32)[:, None]
    raw[..., 2] = np.float32(1.0)
    raw[..., 3] = np.float32(0.1)
    K = np.exp(_oracle_logk(params, lo, hi, -3.0, 1.0, raw.reshape(-1, 4))).reshape(spec.nT, spec.n_nu)
    gs, keep = rt.make_grid(g)
    n = 40000
    ab, sc, steps = _tally(rt, lambda t: rt.trace_mlp(gs, P, norm, spec, t, n_rays=n, seed=5), g.ncells)
    o = otrace.trace(g, spec, K, seed=5, n_rays=n)
    assert steps == o.steps  # the same rays and visits
    big = o.absorbed >= 1e-3 * o.absorbed.max()
    rel = np.abs(ab[big] - o.absorbed[big]) / o.absorbed[big]
    assert np.median(rel) < 1e-2 and rel.max() < 5e-2, (np.median(rel), rel.max())
    assert sc[0] == pytest.approx(o.emitted, rel=1e-2)
    assert sc[3] < 1e-5


def test_mlp_walk_matches_oracle_with_pressure_and_mole_fraction_fields(rt):
    # Cells at arbitrary T, p and x: the network takes each cell's own state, so the
    # oracle evaluates it per cell (binary64, oracle/mlp.py) and walks the rays with
    # those per-cell values (oracle/trace.c, per-cell mode).
    rng = np.random.default_rng(21)
    n3 = 6
    nc = n3 ** 3
    g = synth.Grid(n3, n3, n3, 1.0 / n3, 1.0 / n3, 1.0 / n3,
                   rng.uniform(800.0, 2000.0, nc).astype(np.float32),
                   rng.uniform(0.5, 5.0, nc).astype(np.float32),
                   rng.uniform(0.01, 0.3, nc).astype(np.float32))
    spec = synth.Spectral(nu_min=2400.0, dnu=0.05, n_nu=1500, cutoff=25.0, profile="voigt", nT=13,
                          T_min=800.0, T_max=2000.0, p_ref_atm=1.0, x_ref=0.1)
    params, P, norm, lo, hi = _mlp_case(rt, seed=7)
    n = 30000
    _, j = otrace.emission_indices(nc, spec.n_nu, 6, 0, n)
    cols = np.unique(j)
    nu = spec.nu_min + cols * spec.dnu
    raw = np.zeros((nc, cols.size, 4))
    raw[..., 0] = np.log(nu)[None, :]
    raw[..., 1] = g.T[:, None]
    raw[..., 2] = g.p_atm[:, None]
    raw[..., 3] = g.x[:, None]
    logk = _oracle_logk(params, lo, hi, -3.0, 1.0, raw.reshape(-1, 4)).reshape(nc, cols.size)
    assert logk.std(axis=0).mean() > 0.1  # the cells' states matter to the network
    gs, keep = rt.make_grid(g)
    ab, sc, steps = _tally(rt, lambda t: rt.trace_mlp(gs, P, norm, spec, t, n_rays=n, seed=6), nc)
    o = otrace.trace(g, spec, np.exp(logk), seed=6, n_rays=n, columns=cols, per_cell=True)
    assert steps == o.steps
    big = o.absorbed >= 1e-3 * o.absorbed.max()
    rel = np.abs(ab[big] - o.absorbed[big]) / o.absorbed[big]
    assert np.median(rel) < 1e-2 and rel.max() < 5e-2, (np.median(rel), rel.max())
    assert sc[0] == pytest.approx(o.emitted, rel=1e-2)
    assert sc[3] < 1e-5
