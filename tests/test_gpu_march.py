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


def _cells_crossed(g, pos, d):
    """Cells a straight path from pos (inside) along d crosses before its first wall, in
    binary64: one plus the interior planes i h (0 < i < n) strictly between start and exit."""
    n = np.array([g.nx, g.ny, g.nz])
    h = np.array([g.hx, g.hy, g.hz])
    p = pos.astype(np.float64)
    v = d.astype(np.float64)
    out = np.ones(len(p), dtype=np.int64)
    for r in range(len(p)):
        t_exit = np.inf
        for a in range(3):
            if math.isfinite(h[a]) and v[r, a] != 0.0:
                wall = n[a] * h[a] if v[r, a] > 0 else 0.0
                t_exit = min(t_exit, (wall - p[r, a]) / v[r, a])
        for a in range(3):
            if math.isfinite(h[a]) and v[r, a] != 0.0 and math.isfinite(t_exit):
                i0 = math.floor(p[r, a] / h[a])
                i1 = math.floor((p[r, a] + t_exit * v[r, a]) / h[a])
                i1 = min(max(i1, 0), n[a] - 1)
                out[r] += abs(i1 - i0)
    return out


@pytest.mark.parametrize("kind,n_nu", [("box", 3000), ("slab", 3000), ("box", 3002), ("box", 2999)])
def test_march_matches_oracle(rt, kind, n_nu):
    # the kernel loads 4, 2 or 1 table entries at a time as n_nu is a multiple of 4,
    # even or odd; 3002 and 2999 also leave a ragged last group of wavenumbers
    import torch
    rng = synth.rng_for(9, 70)
    lines = synth.make_lines(300, 2000.0, 2070.0, rng)
    spec = synth.Spectral(nu_min=2010.0, dnu=0.02, n_nu=n_nu, cutoff=25.0, profile="voigt", nT=6,
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
    nvis = torch.zeros(pos.shape[0], dtype=torch.int32, device="cuda")
    I, pw = rt.march(gs, torch.from_numpy(K.astype(np.float32)).cuda(), spec, torch.from_numpy(pos).cuda(),
                     torch.from_numpy(d).cuda(), I_in=torch.from_numpy(Iin).cuda(), nvis=nvis)
    # cells crossed = 1 + the interior grid planes the segment to the first wall crosses
    assert np.array_equal(nvis.cpu().numpy(), _cells_crossed(g, pos, d))
    I = I.cpu().numpy().astype(np.float64)
    pw = pw.cpu().numpy()
    Io, pwo = otrace.march(g, spec, K.astype(np.float32).astype(np.float64), pos, d, I_in=Iin.astype(np.float64))
    scale = np.abs(Io).max(axis=1, keepdims=True)
    assert np.all(np.abs(I - Io) <= 1e-5 * scale)
    assert np.allclose(pw, pwo, rtol=1e-5, atol=1e-7 * np.abs(pwo).max())
