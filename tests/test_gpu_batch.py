"""Batched tracing of enclosures of uneven size (one persistent launch) against
per-enclosure rt_trace calls and the oracle, and replay as a CUDA graph.

Enclosure e draws its rays with Philox counter word 3 = e, so its batched tally
equals rt_trace(..., enclosure=e) up to the order of binary64 atomic additions
(1e-9 relative), and the oracle's tally within the walk tolerance (1e-4)."""
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


@pytest.fixture(scope="module")
def setup(rt):
    import torch
    rng = synth.rng_for(9, 60)
    encl = synth.batched_enclosures(12, rng, side_lo=3, side_hi=14, rays_per_cell=8)
    lines = synth.make_lines(300, 2000.0, 2060.0, rng)
    spec = synth.Spectral(nu_min=2010.0, dnu=0.02, n_nu=2000, cutoff=25.0, profile="voigt",
                          nT=8, T_min=600.0, T_max=2000.0)
    K = okappa.kappa_table(lines, spec)
    kap = torch.from_numpy(K.astype(np.float32)).cuda()
    return encl, spec, K, kap


def _single(rt, g, spec, kap, n, e):
    gs, keep = rt.make_grid(g)
    t = rt.Tally(g.ncells)
    t.zero()
    rt.trace(gs, kap, spec, t, n_rays=n, n_rays_total=n, seed=7, enclosure=e)
    ab, sc, _ = t.read()
    return ab, sc, int(t.steps.item())


@pytest.mark.parametrize("rays_per_item,threads", [(0, 0), (64, 128), (1000, 256)])
def test_batch_matches_per_enclosure_traces(rt, setup, rays_per_item, threads):
    encl, spec, K, kap = setup
    B = rt.Batch([g for g, _ in encl], [n for _, n in encl], spec, seed=7,
                 rays_per_item=rays_per_item, threads=threads)
    B.trace(kap)
    for e, ((g, n), t) in enumerate(zip(encl, B.tallies)):
        ab, sc, st = t.read()
        ab1, sc1, st1 = _single(rt, g, spec, kap, n, e)
        assert int(t.steps.item()) == st1
        assert np.allclose(ab, ab1, rtol=1e-9, atol=1e-12 * sc1[0])
        assert sc[0] == pytest.approx(sc1[0], rel=1e-12)
        assert sc[3] < 1e-5
    B.close()


def test_batch_enclosure_matches_oracle(rt, setup):
    encl, spec, K, kap = setup
    B = rt.Batch([g for g, _ in encl], [n for _, n in encl], spec, seed=7)
    B.trace(kap)
    for e in (0, 5, 11):
        g, n = encl[e]
        ab, sc, _ = B.tallies[e].read()
        o = otrace.trace(g, spec, K.astype(np.float32).astype(np.float64), seed=7, n_rays=n,
                         enclosure=e)
        big = o.absorbed >= 1e-6 * o.absorbed.max()
        assert np.max(np.abs(ab[big] - o.absorbed[big]) / o.absorbed[big]) <= 1e-4
        assert sc[0] == pytest.approx(o.emitted, rel=1e-5)
    B.close()


def test_batch_replays_as_cuda_graph(rt, setup):
    import torch
    encl, spec, K, kap = setup
    B = rt.Batch([g for g, _ in encl], [n for _, n in encl], spec, seed=7)
    B.trace(kap)
    eager = [t.read()[0].copy() for t in B.tallies]
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        B.zero(stream=s)
        B.trace(kap, stream=s)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        for t, ref in zip(B.tallies, eager):
            assert np.allclose(t.read()[0], ref, rtol=1e-9, atol=0)
    B.close()
