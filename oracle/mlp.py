"""FP64 oracle of the kappa surrogate network (test infrastructure).

The network replaces the table lookup of the ray walk (Section 3, Eq. tau
evaluated at a cell's state): inputs (log nu, T, p, x) mapped affinely to
[-1, 1], four hidden layers of width 128 with SiLU, a linear scalar output
that predicts the standardised log kappa.  Parameters are one flat vector with
the layout of ``synth.MLP_LAYOUT`` (W[out][in] row-major).  Training uses the
mean-squared error and Adam (Kingma and Ba, 2015).

Parity: pinned (central finite differences of the loss for every parameter
tensor; closed-form outputs for degenerate weights; Adam's first step moves
each parameter by lr in the direction of -sign(g)).
"""
from __future__ import annotations

import numpy as np

import synth


def unflatten(flat):
    flat = np.asarray(flat, dtype=np.float64)
    return {k: flat[o:o + int(np.prod(s))].reshape(s) for k, (o, s) in synth.mlp_offsets().items()}


def flatten(d):
    out = np.zeros(synth.MLP_NPARAM, dtype=np.float64)
    for k, (o, s) in synth.mlp_offsets().items():
        out[o:o + int(np.prod(s))] = np.asarray(d[k], dtype=np.float64).ravel()
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def normalise(raw, lo, hi):
    """Affine map of raw inputs (n, 4) from [lo, hi] per feature to [-1, 1]."""
    raw = np.asarray(raw, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return 2.0 * (raw - lo) / (hi - lo) - 1.0


def forward(flat, U):
    """Network output (n,) for normalised inputs U (n, 4); returns (y, cache)."""
    P = unflatten(flat)
    h = np.asarray(U, dtype=np.float64)
    zs, hs = [], [h]
    for i in (1, 2, 3, 4):
        z = h @ P[f"W{i}"].T + P[f"b{i}"]
        h = silu(z)
        zs.append(z)
        hs.append(h)
    y = h @ P["w5"] + P["b5"][0]
    return y, (zs, hs)


def loss_and_grad(flat, U, target):
    """Mean-squared error 0.5 * mean((y - target)^2) and its gradient (flat)."""
    P = unflatten(flat)
    y, (zs, hs) = forward(flat, U)
    n = y.shape[0]
    r = y - np.asarray(target, dtype=np.float64)
    loss = 0.5 * float(np.mean(r * r))
    dy = r / n
    g = {"w5": hs[4].T @ dy, "b5": np.array([dy.sum()])}
    dh = np.outer(dy, P["w5"])
    for i in (4, 3, 2, 1):
        dz = dh * silu_grad(zs[i - 1])
        g[f"W{i}"] = dz.T @ hs[i - 1]
        g[f"b{i}"] = dz.sum(0)
        dh = dz @ P[f"W{i}"]
    return loss, flatten(g)


def adam_step(flat, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1); returns new (flat, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v
