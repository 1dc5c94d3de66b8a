"""GPU parity of rt_march (spectrally resolved Eq. I along rays) against the
oracle's binary64 marching on the same binary32 walk.  Tolerance: 1e-5 of the
largest |I_out| of the path per sample and 1e-5 relative on the power sum, from
binary32 exponentials over about a hundred cells."""
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


def _paths(g, n, seed):
    rng = np.random.default_rng(seed)
    ext = np.array([g.nx * g.hx if math.isfinite(g.hx) else 1.0,
                    g.ny * g.hy if math.isfinite(g.hy) else 1.0,
                    g.nz * g.hz if math.isfinite(g.hz) else 1.0])
    pos = (rng.uniform(0.02, 0.98, (n, 3)) * ext).astype(np.float32)
    d = rng.normal(size=(n, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    return pos, d


@pytest.mark.parametrize("kind", ["box", "slab"])
def test_march_matches_oracle(rt, kind):
    import torch
    rng = synth.rng_for(9, 70)
    lines = synth.make_lines(300, 2000.0, 2070.0, rng)
    spec = synth.Spectral(nu_min=2010.0, dnu=0.02, n_nu=3000, cutoff=25.0, profile="voigt", nT=6,
                          T_min=800.0, T_max=2000.0, x_ref=1e-3)
    if kind == "box":
        g = synth.gaussian_hotspot_grid(10, 1.0, 800.0, 2000.0, 0.2, dims=(10, 8, 6))
    else:
        g = synth.Grid(40, 1, 1, 0.025, math.inf, math.inf,
                       np.linspace(800, 2000, 40).astype(np.float32))
    K = okappa.kappa_table(lines, spec)
    Iin = (1e-3 * (1.0 + np.sin(np.arange(spec.n_nu) * 0.01))).astype(np.float32)
    pos, d = _paths(g, 64, 3)
    gs, keep = rt.make_grid(g)
    I, pw = rt.march(gs, torch.from_numpy(K.astype(np.float32)).cuda(), spec, torch.from_numpy(pos).cuda(),
                     torch.from_numpy(d).cuda(), I_in=torch.from_numpy(Iin).cuda())
    I = I.cpu().numpy().astype(np.float64)
    pw = pw.cpu().numpy()
    Io, pwo = otrace.march(g, spec, K.astype(np.float32).astype(np.float64), pos, d, I_in=Iin.astype(np.float64))
    scale = np.abs(Io).max(axis=1, keepdims=True)
    assert np.all(np.abs(I - Io) <= 1e-5 * scale)
    assert np.allclose(pw, pwo, rtol=1e-5, atol=1e-7 * np.abs(pwo).max())
