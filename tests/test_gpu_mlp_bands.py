"""GPU parity of the spectral-band ensemble of surrogate networks (one network per
band of wavenumbers).

* Training several networks in one library call (rt_mlp_train_steps_nets) gives
  each network, bit for bit, the parameters of its own rt_mlp_train_steps run on
  its own samples: the ensemble only adds a network index to the same kernels.
* The ensemble's forward pass matches the FP64 oracle network (oracle/mlp.py) per
  network, within the BF16 tolerance of the single-network tests.
* The banded walk (rt_trace_mlp_bands) matches the FP64 oracle: each band's
  network tabulated in binary64 at node temperatures (or evaluated per cell for
  p/x fields), walked by oracle/trace.c on the same rays; with one band it equals
  rt_trace_mlp.
* The band samples lie in their band and their targets are the table's values.
"""
import math

import numpy as np
import pytest

import synth
from oracle import mlp as omlp
from oracle import trace as otrace

pytestmark = pytest.mark.gpu

LO = [math.log(2000.0), 600.0, 0.5, 0.01]
HI = [math.log(3000.0), 2200.0, 5.0, 0.3]


@pytest.fixture(scope="module")
def rt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_cs_0703028_gb300 as rt
    rt.lib()
    return rt


def _spread_net(seed, w1=3.0, w5=20.0):
    """A random network whose output moves with every input (first layer and head scaled)."""
    p = synth.mlp_init(seed)
    off = synth.mlp_offsets()
    for name, f in (("W1", w1), ("w5", w5)):
        o, shape = off[name]
        p[o:o + int(np.prod(shape))] *= np.float32(f)
    return p


def _band_norms(rt, spec, band_pts, mean=-3.0, scale=1.0):
    nb = -(-spec.n_nu // band_pts)
    j0 = np.arange(nb) * band_pts
    j1 = np.minimum(j0 + band_pts, spec.n_nu) - 1
    lo = np.tile(np.array(LO), (nb, 1))
    hi = np.tile(np.array(HI), (nb, 1))
    lo[:, 0] = np.log(spec.nu_min + j0 * spec.dnu)
    hi[:, 0] = np.maximum(np.log(spec.nu_min + j1 * spec.dnu), lo[:, 0] + 1e-6)
    return rt.norms_tensor(lo, hi, np.full(nb, mean), np.full(nb, scale)), lo, hi


def _oracle_logk_band(params, lo, hi, raw, mean=-3.0, scale=1.0):
    lo32 = np.asarray(lo, np.float32).astype(np.float64)
    hi32 = np.asarray(hi, np.float32).astype(np.float64)
    y, _ = omlp.forward(np.asarray(params, np.float64), omlp.normalise(raw, lo32, hi32))
    return float(np.float32(mean)) + float(np.float32(scale)) * y


def _tally(rt, run, ncells):
    t = rt.Tally(ncells)
    t.zero()
    run(t)
    ab, sc, st = t.read()
    return ab, sc, int(t.steps.item())


def test_ensemble_training_equals_separate_training(rt):
    import torch
    n_nets, n, batch, steps = 3, 1536, 512, 4
    rng = np.random.default_rng(5)
    params = [synth.mlp_init(10 + b) * np.float32(1.5) for b in range(n_nets)]
    raw = [(np.array(LO) + (np.array(HI) - np.array(LO)) * rng.uniform(0, 1, (n, 4))).astype(np.float32)
           for _ in range(n_nets)]
    tgt = [rng.normal(-3.0 + b, 2.0, n).astype(np.float32) for b in range(n_nets)]
    norms_h = [(LO, HI, -3.0 + b, 2.0 + 0.5 * b) for b in range(n_nets)]
    sep = []
    for b in range(n_nets):
        tr = rt.MlpTrainer(torch.from_numpy(params[b].copy()).cuda(), rt.make_norm(*norms_h[b]))
        tr.steps(torch.from_numpy(raw[b]).cuda(), torch.from_numpy(tgt[b]).cuda(), batch, 1e-3, 1e-4, 1, steps,
                 steps)
        sep.append(tr.params.cpu().numpy())
    P = torch.from_numpy(np.concatenate(params)).cuda()
    norms = rt.norms_tensor([h[0] for h in norms_h], [h[1] for h in norms_h], [h[2] for h in norms_h],
                            [h[3] for h in norms_h])
    tr = rt.MlpEnsembleTrainer(P, norms)
    losses = torch.zeros(steps, dtype=torch.float32, device="cuda")
    tr.steps(torch.from_numpy(np.stack(raw)).cuda(), torch.from_numpy(np.stack(tgt)).cuda(), batch, 1e-3, 1e-4,
             1, steps, steps, losses=losses)
    got = tr.params.cpu().numpy().reshape(n_nets, -1)
    for b in range(n_nets):
        assert np.array_equal(got[b], sep[b]), b
    assert np.all(np.isfinite(losses.cpu().numpy())) and float(losses[0]) > 0


def test_ensemble_forward_matches_oracle(rt):
    import torch
    n_nets, n = 4, 700   # ragged last tile
    rng = np.random.default_rng(8)
    params = [_spread_net(20 + b) for b in range(n_nets)]
    lo = np.tile(np.array(LO), (n_nets, 1))
    hi = np.tile(np.array(HI), (n_nets, 1))
    lo[:, 0] = np.log(2000.0 + 200.0 * np.arange(n_nets))
    hi[:, 0] = np.log(2150.0 + 200.0 * np.arange(n_nets))
    raw = lo[:, None, :] + (hi - lo)[:, None, :] * rng.uniform(0, 1, (n_nets, n, 4))
    raw = raw.astype(np.float32)
    norms = rt.norms_tensor(lo, hi, -1.0 - np.arange(n_nets), 1.0 + np.arange(n_nets))
    out = rt.mlp_forward_nets(torch.from_numpy(np.concatenate(params)).cuda(), norms,
                              torch.from_numpy(raw).cuda()).cpu().numpy().astype(np.float64)
    for b in range(n_nets):
        ref = _oracle_logk_band(params[b], lo[b], hi[b], raw[b].astype(np.float64), -1.0 - b, 1.0 + b)
        assert np.max(np.abs(out[b] - ref)) <= 2e-2 * np.std(ref) * 4 + 1e-3, b


def _node_grid(seed=4, n=8):
    rng = np.random.default_rng(seed)
    T = (800.0 + 100.0 * rng.integers(0, 13, n ** 3)).astype(np.float32)
    return synth.Grid(n, n, n, 1.0 / n, 1.0 / n, 1.0 / n, T, np.full(n ** 3, 1.0, np.float32),
                      np.full(n ** 3, 0.1, np.float32))


@pytest.mark.parametrize("band_pts", [300, 2000])
def test_banded_walk_matches_oracle_on_node_temperatures(rt, band_pts):
    import torch
    spec = synth.Spectral(nu_min=2000.0, dnu=0.02, n_nu=2000, cutoff=25.0, profile="voigt", nT=13,
                          T_min=800.0, T_max=2000.0, p_ref_atm=1.0, x_ref=0.1)
    nb = -(-spec.n_nu // band_pts)        # 300: 7 bands, the last one 200 points
    params = [_spread_net(30 + b) for b in range(nb)]
    norms, lo, hi = _band_norms(rt, spec, band_pts)
    nu = spec.nu_min + np.arange(spec.n_nu) * spec.dnu
    K = np.zeros((spec.nT, spec.n_nu))
    Tn = np.asarray(spec.T_nodes(), np.float32).astype(np.float64)
    for b in range(nb):
        js = np.arange(b * band_pts, min((b + 1) * band_pts, spec.n_nu))
        raw = np.zeros((spec.nT, js.size, 4))
        raw[..., 0] = np.log(nu[js])[None, :]
        raw[..., 1] = Tn[:, None]
        raw[..., 2] = np.float32(1.0)
        raw[..., 3] = np.float32(0.1)
        K[:, js] = np.exp(_oracle_logk_band(params[b], lo[b], hi[b], raw.reshape(-1, 4))).reshape(spec.nT, -1)
    g = _node_grid()
    gs, keep = rt.make_grid(g)
    n = 40000
    P = torch.from_numpy(np.concatenate(params)).cuda()
    ab, sc, steps = _tally(rt, lambda t: rt.trace_mlp_bands(gs, band_pts, P, norms, spec, t, n_rays=n, seed=5),
                           g.ncells)
    o = otrace.trace(g, spec, K, seed=5, n_rays=n)
    assert steps == o.steps
    big = o.absorbed >= 1e-3 * o.absorbed.max()
    rel = np.abs(ab[big] - o.absorbed[big]) / o.absorbed[big]
    assert np.median(rel) < 1e-2 and rel.max() < 5e-2, (np.median(rel), rel.max())
    assert sc[0] == pytest.approx(o.emitted, rel=1e-2)
    assert sc[3] < 1e-5


def test_banded_walk_with_pressure_and_mole_fraction_fields(rt):
    import torch
    rng = np.random.default_rng(23)
    n3 = 6
    nc = n3 ** 3
    g = synth.Grid(n3, n3, n3, 1.0 / n3, 1.0 / n3, 1.0 / n3,
                   rng.uniform(800.0, 2000.0, nc).astype(np.float32),
                   rng.uniform(0.5, 5.0, nc).astype(np.float32),
                   rng.uniform(0.01, 0.3, nc).astype(np.float32))
    spec = synth.Spectral(nu_min=2400.0, dnu=0.05, n_nu=1500, cutoff=25.0, profile="voigt", nT=13,
                          T_min=800.0, T_max=2000.0, p_ref_atm=1.0, x_ref=0.1)
    band_pts = 400   # 4 bands, the last one 300 points
    nb = -(-spec.n_nu // band_pts)
    params = [_spread_net(40 + b) for b in range(nb)]
    norms, lo, hi = _band_norms(rt, spec, band_pts)
    n = 30000
    _, j = otrace.emission_indices(nc, spec.n_nu, 6, 0, n)
    cols = np.unique(j)
    nu = spec.nu_min + cols * spec.dnu
    logk = np.zeros((nc, cols.size))
    for b in range(nb):
        sel = (cols // band_pts) == b
        raw = np.zeros((nc, int(sel.sum()), 4))
        raw[..., 0] = np.log(nu[sel])[None, :]
        raw[..., 1] = g.T[:, None]
        raw[..., 2] = g.p_atm[:, None]
        raw[..., 3] = g.x[:, None]
        logk[:, sel] = _oracle_logk_band(params[b], lo[b], hi[b], raw.reshape(-1, 4)).reshape(nc, -1)
    gs, keep = rt.make_grid(g)
    P = torch.from_numpy(np.concatenate(params)).cuda()
    ab, sc, steps = _tally(rt, lambda t: rt.trace_mlp_bands(gs, band_pts, P, norms, spec, t, n_rays=n, seed=6), nc)
    o = otrace.trace(g, spec, np.exp(logk), seed=6, n_rays=n, columns=cols, per_cell=True)
    assert steps == o.steps
    big = o.absorbed >= 1e-3 * o.absorbed.max()
    rel = np.abs(ab[big] - o.absorbed[big]) / o.absorbed[big]
    assert np.median(rel) < 1e-2 and rel.max() < 5e-2, (np.median(rel), rel.max())
    assert sc[0] == pytest.approx(o.emitted, rel=1e-2)


def test_one_band_equals_single_network_walk(rt):
    import torch
    spec = synth.Spectral(nu_min=2000.0, dnu=0.02, n_nu=2000, cutoff=25.0, profile="voigt", nT=13,
                          T_min=800.0, T_max=2000.0, p_ref_atm=1.0, x_ref=0.1)
    p = _spread_net(50)
    P = torch.from_numpy(p).cuda()
    g = synth.gaussian_hotspot_grid(10, 1.0, 800.0, 2000.0, 0.2)
    gs, keep = rt.make_grid(g)
    norm = rt.make_norm(LO, HI, -3.0, 1.0)
    norms = rt.norms_tensor([LO], [HI], [-3.0], [1.0])
    n = 20000
    a1, s1, n1 = _tally(rt, lambda t: rt.trace_mlp(gs, P, norm, spec, t, n_rays=n, seed=9), g.ncells)
    a2, s2, n2 = _tally(rt, lambda t: rt.trace_mlp_bands(gs, 5000, P, norms, spec, t, n_rays=n, seed=9), g.ncells)
    assert n1 == n2
    assert np.allclose(a1, a2, rtol=1e-12, atol=1e-12 * a1.max())
    assert s1[0] == pytest.approx(s2[0], rel=1e-12)


def test_band_samples_lie_in_their_band(rt):
    import torch
    spec = synth.Spectral(nu_min=2000.0, dnu=0.05, n_nu=1000, cutoff=25.0, profile="voigt", nT=5,
                          T_min=800.0, T_max=1600.0, p_ref_atm=1.0, x_ref=0.1)
    rng = np.random.default_rng(2)
    tab = rng.uniform(0.5, 2.0, (2, spec.nT, spec.n_nu)).astype(np.float32)
    p_nodes = torch.tensor([1.0, 2.0], dtype=torch.float32, device="cuda")
    band_pts, n = 128, 3000   # 8 bands, the last one 104 points
    inp, tg = rt.mlp_make_samples_bands(torch.from_numpy(tab).cuda(), p_nodes, spec, band_pts, 0.05, 0.2, 3, n)
    inp, tg = inp.cpu().numpy().astype(np.float64), tg.cpu().numpy().astype(np.float64)
    for b in range(-(-spec.n_nu // band_pts)):
        nu = np.exp(inp[b, :, 0])
        j = np.rint((nu - spec.nu_min) / spec.dnu).astype(int)
        assert j.min() >= b * band_pts and j.max() < min((b + 1) * band_pts, spec.n_nu)
        kT = np.rint((inp[b, :, 1] - spec.T_min) / 200.0).astype(int)
        kp = np.rint(inp[b, :, 2]).astype(int) - 1
        x = inp[b, :, 3]
        assert np.all((x >= 0.05) & (x <= 0.2))
        ref = np.log(tab[kp, kT, j].astype(np.float64) * x / 0.1)
        assert np.allclose(tg[b], ref, rtol=0, atol=2e-6 * np.abs(ref).max() + 1e-6)


@pytest.mark.parametrize("mix", [1.0, 0.5])
def test_band_samples_follow_the_emission_weights(rt, mix):
    # With emission_mix m, a sample's wavenumber follows (1 - m) uniform + m kappa I_b(nu, T)
    # over its band (at its own T and p node): the empirical frequencies match within 5 sigma.
    import torch
    spec = synth.Spectral(nu_min=2000.0, dnu=0.5, n_nu=16, cutoff=25.0, profile="voigt", nT=3,
                          T_min=800.0, T_max=1600.0, p_ref_atm=1.0, x_ref=0.1)
    rng = np.random.default_rng(4)
    tab = rng.uniform(0.2, 5.0, (1, spec.nT, spec.n_nu)).astype(np.float32)
    p_nodes = torch.tensor([1.0], dtype=torch.float32, device="cuda")
    n = 60000
    inp, _ = rt.mlp_make_samples_bands(torch.from_numpy(tab).cuda(), p_nodes, spec, 8, 0.05, 0.2, 11, n,
                                       emission_mix=mix)
    inp = inp.cpu().numpy().astype(np.float64)
    c2 = 1.438776877
    for b in range(2):
        j = np.rint((np.exp(inp[b, :, 0]) - spec.nu_min) / spec.dnu).astype(int) - 8 * b
        kT = np.rint((inp[b, :, 1] - spec.T_min) / 400.0).astype(int)
        for k in range(spec.nT):
            sel = kT == k
            js = np.arange(8 * b, 8 * b + 8)
            nu = spec.nu_min + js * spec.dnu
            w = tab[0, k, js].astype(np.float64) * nu ** 3 / np.expm1(c2 * nu / spec.T_nodes()[k])
            p = (1 - mix) / 8 + mix * w / w.sum()
            cnt = np.bincount(j[sel], minlength=8)
            m = sel.sum()
            assert np.all(np.abs(cnt - m * p) <= 5 * np.sqrt(m * p * (1 - p)) + 1), (b, k, cnt, m * p)


def test_banded_walk_at_the_learned_part_size(rt):
    # The 64^3 learned-part workload in the benchmark's configuration: 6250 networks of 16
    # wavenumbers over 100k wavenumbers, 5e7 rays grouped by band.  The visits do not depend
    # on kappa, so the step count must equal the table walk's on the same rays exactly; the
    # tally must close its energy balance; and a sample of rays' emission weights must follow
    # each ray's own band network (recorded weights against the FP64 oracle network).
    import torch
    case = synth.config(2)
    spec, g = case.spec, case.grid
    band_pts = 16
    nb = -(-spec.n_nu // band_pts)
    base = _spread_net(60)
    P = torch.from_numpy(np.tile(base, nb)).cuda()
    norms, lo, hi = _band_norms(rt, spec, band_pts)
    gs, keep = rt.make_grid(g)
    n = case.n_rays
    t = rt.Tally(g.ncells)
    t.zero()
    rec = rt.Record(2000, g.nx + g.ny + g.nz + 4)
    rt.trace_mlp_bands(gs, band_pts, P, norms, spec, t, n_rays=n, record=rec)
    ab, sc, st = t.read()
    steps_b = int(t.steps.item())
    kap = torch.full((spec.nT, spec.n_nu), 1e-3, dtype=torch.float32, device="cuda")
    t2 = rt.Tally(g.ncells)
    t2.zero()
    rt.trace(gs, kap, spec, t2, n_rays=n)
    t2.read()
    assert steps_b == int(t2.steps.item())
    assert sc[3] < 1e-5
    # the recorded rays' weights: 4 pi V kappa I_b dnu ncells n_nu / N with kappa from the ray's band network
    cell, j = otrace.emission_indices(g.ncells, spec.n_nu, 0, 0, 2000)
    w_gpu = rec.weight.cpu().numpy().astype(np.float64)
    T = g.T[cell].astype(np.float64)
    nu = spec.nu_min + j * spec.dnu
    raw = np.stack([np.log(nu), T, np.full_like(T, np.float32(spec.p_ref_atm)),
                    np.full_like(T, np.float32(spec.x_ref))], 1)
    logk = np.array([_oracle_logk_band(base, lo[jj // band_pts], hi[jj // band_pts], raw[i:i + 1])[0]
                     for i, jj in enumerate(j)])
    from oracle import physics as ph
    V = g.hx * g.hy * g.hz
    w_ref = (4 * math.pi * V * 100.0 * np.exp(logk) * ph.planck_wavenumber(nu, T) * 100.0 * spec.dnu
             * g.ncells * spec.n_nu / n)
    rel = np.abs(w_gpu - w_ref) / w_ref
    assert np.median(rel) < 1e-2 and rel.max() < 5e-2, (np.median(rel), rel.max())


def test_evaluation_count_and_dark_rays(rt):
    # RT_COUNT_EVALS adds the network evaluations in steps[1] and leaves the walk as it
    # was; with the optical-depth cut every counted step is a lit step (no dark ray runs
    # ahead), so the evaluations cover at least the steps of the tile's longest ray; without
    # the cut a dark ray takes its remaining steps without evaluations
    import torch
    spec = synth.Spectral(nu_min=2000.0, dnu=0.02, n_nu=2000, cutoff=25.0, profile="voigt", nT=13,
                          T_min=800.0, T_max=2000.0, p_ref_atm=1.0, x_ref=0.1)
    p = _spread_net(51)
    P = torch.from_numpy(p).cuda()
    g = synth.gaussian_hotspot_grid(12, 1.0, 800.0, 2000.0, 0.2)
    gs, keep = rt.make_grid(g)
    norms = rt.norms_tensor([LO], [HI], [2.0], [1.0])   # large kappa: most rays go dark
    n = 30000

    def run(flags):
        t = rt.Tally(g.ncells, counters=2)
        t.zero()
        rt.trace_mlp_bands(gs, 5000, P, norms, spec, t, n_rays=n, seed=3, flags=flags)
        ab, sc, st = t.read()
        assert st == 0
        return ab, sc, int(t.steps[0].item()), int(t.steps[1].item())

    a0, s0, n0, e0 = run(0)
    a1, s1, n1, e1 = run(rt.RT_COUNT_EVALS)
    assert e0 == 0 and e1 > 0
    assert n0 == n1
    assert np.allclose(a0, a1, rtol=1e-12, atol=1e-12 * a0.max())
    # the evaluations serve fewer ray-steps than were taken: dark rays ran ahead
    assert e1 * 128 < n1
    _, _, nc, ec = run(rt.RT_COUNT_EVALS | rt.RT_TAU_CUT)
    assert ec * 128 >= nc   # with the cut every step is evaluated
