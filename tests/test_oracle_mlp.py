"""Pins of the FP64 surrogate-network oracle: finite differences, degenerate
closed forms, Adam's first-step property."""
import numpy as np
import pytest

import synth
from oracle import mlp as M


def _data(n=64, seed=0):
    rng = np.random.default_rng(seed)
    U = rng.uniform(-1, 1, (n, 4))
    t = rng.normal(0, 1, n)
    return U, t


def test_layout_size():
    assert synth.MLP_NPARAM == 50305
    off = synth.mlp_offsets()
    assert off["b5"][0] == 50304


@pytest.mark.parametrize("name", ["W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4", "w5", "b5"])
def test_gradient_matches_central_differences(name):
    flat = synth.mlp_init(0).astype(np.float64) * 3.0   # larger weights: non-trivial curvature
    U, t = _data()
    loss, g = M.loss_and_grad(flat, U, t)
    off, shape = synth.mlp_offsets()[name]
    n = int(np.prod(shape))
    rng = np.random.default_rng(1)
    idx = off + rng.choice(n, size=min(n, 12), replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(flat)
        e[i] = h
        lp, _ = M.loss_and_grad(flat + e, U, t)
        lm, _ = M.loss_and_grad(flat - e, U, t)
        fd = (lp - lm) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-10), (name, i)


def test_degenerate_network_closed_form():
    # all weights zero except biases: every hidden unit is silu(b), output = b5 + sum(w5) silu(b4)
    d = {k: np.zeros(s) for k, (o, s) in synth.mlp_offsets().items()}
    d["b4"][:] = 0.7
    d["w5"][:] = 0.01
    d["b5"][0] = -0.3
    flat = M.flatten(d)
    U, _ = _data(5)
    y, _ = M.forward(flat, U)
    s = 0.7 / (1 + np.exp(-0.7))
    assert np.allclose(y, -0.3 + 128 * 0.01 * s, rtol=1e-15)
    # the first layer is a plain affine map of the inputs
    d["W1"][0, :] = [1.0, 2.0, 3.0, 4.0]
    d["b4"][:] = 0.0
    d["W2"][0, 0] = 1.0
    d["W3"][0, 0] = 1.0
    d["W4"][0, 0] = 1.0
    d["w5"][:] = 0.0
    d["w5"][0] = 1.0
    d["b5"][0] = 0.0
    y, _ = M.forward(M.flatten(d), U)
    z = U @ np.array([1.0, 2.0, 3.0, 4.0])
    expect = M.silu(M.silu(M.silu(M.silu(z))))
    assert np.allclose(y, expect, rtol=1e-14)


def test_silu_grad_closed_form():
    z = np.linspace(-8, 8, 101)
    h = 1e-6
    assert np.allclose(M.silu_grad(z), (M.silu(z + h) - M.silu(z - h)) / (2 * h), rtol=1e-7, atol=1e-10)


def test_adam_first_step_is_signed_lr():
    flat = synth.mlp_init(0).astype(np.float64)
    U, t = _data()
    _, g = M.loss_and_grad(flat, U, t)
    m = np.zeros_like(flat)
    v = np.zeros_like(flat)
    new, m, v = M.adam_step(flat, g, m, v, 1, lr=1e-3, eps=0.0)
    nz = g != 0
    assert np.allclose((new - flat)[nz], -1e-3 * np.sign(g[nz]), rtol=1e-12)


def test_normalise_maps_to_unit_box():
    raw = np.array([[np.log(2000.0), 600.0, 0.5, 0.01], [np.log(3000.0), 2200.0, 5.0, 0.3]])
    lo = raw[0]
    hi = raw[1]
    u = M.normalise(raw, lo, hi)
    assert np.allclose(u, [[-1, -1, -1, -1], [1, 1, 1, 1]])
