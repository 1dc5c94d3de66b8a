"""Degenerate inputs through the C ABI: zero rays, zero paths, zero samples, and a
grid of one cell (Section 3's finite volumes reduced to a single isothermal cube)."""
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


def test_zero_rays_leave_the_tally_untouched(rt):
    import torch
    case = synth.config(0)
    kap = rt.build_kappa(case.lines, case.spec)
    gs, keep = rt.make_grid(case.grid)
    tally = rt.Tally(case.grid.ncells)
    tally.zero()
    rt.trace(gs, kap, case.spec, tally, n_rays=0, n_rays_total=10)
    rt.trace_lbl(gs, case.lines, case.spec, tally, n_rays=0, n_rays_total=10)
    torch.cuda.synchronize()
    ab, sc, _ = tally.read()
    assert not ab.any() and not np.asarray(sc).any()
    assert int(tally.steps.item()) == 0


def test_zero_paths_and_zero_samples(rt):
    import torch
    case = synth.config(0)
    kap = rt.build_kappa(case.lines, case.spec)
    gs, keep = rt.make_grid(case.grid)
    z3 = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    I, pw = rt.march(gs, kap, case.spec, z3, z3)
    assert pw.numel() == 0 and (I is None or I.numel() == 0)
    params = torch.from_numpy(synth.mlp_init(0)).cuda()
    norm = rt.make_norm([7.6, 800.0, 0.5, 0.01], [8.0, 2000.0, 2.0, 0.3], 0.0, 1.0)
    out = rt.mlp_forward(params, norm, torch.zeros((0, 4), dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    assert out.numel() == 0


def test_single_cell_grid_matches_oracle(rt):
    # one 1 cm cube: every ray starts and ends in the same cell, so the tally is the
    # emitted power less what escapes through the six faces
    import torch
    case = synth.config(0)
    K = okappa.kappa_table(case.lines, case.spec)
    grid = synth.uniform_grid(1, 1, 1, 0.01, 0.01, 0.01, 1000.0, 1.0, 0.1)
    gs, keep = rt.make_grid(grid)
    tally = rt.Tally(1)
    tally.zero()
    n = 20000
    rt.trace(gs, torch.from_numpy(K.astype(np.float32)).cuda(), case.spec, tally, n_rays=n, n_rays_total=n)
    torch.cuda.synchronize()
    ab, sc, _ = tally.read()
    o = otrace.trace(grid, case.spec, K.astype(np.float32).astype(np.float64), n_rays=n)
    assert int(tally.steps.item()) == o.steps == n
    assert ab[0] == pytest.approx(o.absorbed[0], rel=1e-4)
    assert sc[0] == pytest.approx(o.emitted, rel=1e-5)
    assert sc[2] == pytest.approx(o.escaped, rel=1e-4)
    assert sc[3] < 1e-5
