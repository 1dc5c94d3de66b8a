"""Surrogate-network pipeline: line-by-line training tables, samples, training.

Every numeric step runs in the library's kernels (rt_build_kappa for the
tables, rt_mlp_make_samples for the samples, rt_mlp_train_steps for the
forward and backward passes and Adam over all steps with a cosine learning
rate); this module only orders the calls and forms the input/output
normalisation (ranges and the targets' mean and spread).

Two forms: one network for the whole spectral window (train_surrogate), and a
spectral-band ensemble (train_bands) with one network per band of band_pts
wavenumbers, all trained together by rt_mlp_train_steps_nets.
"""
from __future__ import annotations

import math
from dataclasses import replace

import numpy as np

from . import (MlpEnsembleTrainer, MlpTrainer, RT_MLP_NPARAM, build_kappa, make_norm, mlp_make_samples,
               mlp_make_samples_bands, norms_tensor)


def training_tables(lines, spec, p_nodes):
    """kappa[kp][kT][j] (CUDA float32) from rt_build_kappa at each pressure node."""
    import torch
    out = torch.empty((len(p_nodes), spec.nT, spec.n_nu), dtype=torch.float32, device="cuda")
    for i, p in enumerate(p_nodes):
        build_kappa(lines, replace(spec, p_ref_atm=float(p)), out=out[i])
    return out


def input_ranges(spec, p_nodes, x_lo, x_hi):
    lo = [math.log(spec.nu_min), spec.T_min, float(min(p_nodes)), x_lo]
    hi = [math.log(spec.nu_min + (spec.n_nu - 1) * spec.dnu), spec.T_max, float(max(p_nodes)), x_hi]
    return lo, hi


def train_surrogate(lines, spec, p_nodes, x_lo=0.01, x_hi=0.3, n_samples=2_000_000, batch=8192,
                    epochs=1, lr0=1e-3, lr1=1e-5, seed=0, params=None, log_every=0, objective="mse"):
    """Train the network on samples drawn from line-by-line tables; returns
    (params, norm, history) with history = [(step, loss)].  objective "mse": the
    mean-squared error of the standardised log kappa over uniformly drawn samples."""
    import torch
    import synth
    if objective != "mse":
        raise ValueError(f"unknown training objective {objective!r}")
    p_nodes = np.asarray(p_nodes, dtype=np.float32)
    tables = training_tables(lines, spec, p_nodes)
    pn = torch.from_numpy(p_nodes).cuda()
    inputs, targets = mlp_make_samples(tables, pn, spec, x_lo, x_hi, seed, n_samples)
    del tables
    head = targets[:65536].cpu().numpy().astype(np.float64)
    lo, hi = input_ranges(spec, p_nodes, x_lo, x_hi)
    norm = make_norm(lo, hi, float(head.mean()), float(head.std()))
    if params is None:
        params = torch.from_numpy(synth.mlp_init(seed, spread_biases=True)).cuda()
    tr = MlpTrainer(params, norm)
    nb = n_samples // batch
    total = nb * epochs
    # all steps in one library call (batch b = s mod nb, cosine learning rate), the
    # per-step losses kept on the device and read once
    losses = torch.zeros(max(total, 1), dtype=torch.float32, device="cuda")
    tr.steps(inputs[:nb * batch], targets[:nb * batch], batch, lr0, lr1, 1, total, total, losses=losses)
    hist = []
    if log_every and total:
        lh = losses.cpu().numpy()
        hist = [(s, float(lh[s])) for s in range(total) if s % log_every == 0 or s == total - 1]
    return params, norm, hist


def save(path, params, norm):
    """Store parameters and normalisation (numpy .npz)."""
    np.savez(path, params=params.detach().cpu().numpy(), in_lo=np.array(norm.in_lo[:]),
             in_hi=np.array(norm.in_hi[:]), out=np.array([norm.out_mean, norm.out_scale]))


def load(path):
    """Parameters (CUDA tensor) and normalisation stored by save()."""
    import torch
    d = np.load(path)
    return (torch.from_numpy(d["params"].astype(np.float32)).cuda(),
            make_norm(d["in_lo"], d["in_hi"], float(d["out"][0]), float(d["out"][1])))


def band_count(spec, band_pts):
    return -(-int(spec.n_nu) // int(band_pts))


def band_norms(spec, band_pts, p_nodes, x_lo, x_hi, targets):
    """Device norms [n_bands, 10] of a spectral-band ensemble: each band's own log nu
    range (its first and last wavenumber), the T, p, x ranges of the training set,
    and the band's target mean and spread (targets [n_bands, n])."""
    import torch
    nb = band_count(spec, band_pts)
    j0 = np.arange(nb, dtype=np.float64) * band_pts
    j1 = np.minimum(j0 + band_pts, spec.n_nu) - 1
    lo_nu = np.log(spec.nu_min + j0 * spec.dnu)
    hi_nu = np.log(spec.nu_min + j1 * spec.dnu)
    hi_nu = np.where(hi_nu > lo_nu, hi_nu, lo_nu + 1e-6)   # a one-point band still gets a range
    lo = np.stack([lo_nu, np.full(nb, spec.T_min), np.full(nb, float(min(p_nodes))), np.full(nb, x_lo)], 1)
    hi = np.stack([hi_nu, np.full(nb, spec.T_max), np.full(nb, float(max(p_nodes))), np.full(nb, x_hi)], 1)
    t64 = targets.double()
    mean = t64.mean(1)
    scale = t64.std(1).clamp_min(1e-3)
    return norms_tensor(lo, hi, mean, scale, device=targets.device)


def train_bands(lines, spec, p_nodes, x_lo=0.01, x_hi=0.3, band_pts=64, n_per_band=12800, batch=256,
                steps=24000, lr0=3e-3, lr1=1e-5, seed=0, group=2048, log_every=0, emission_mix=0.5):
    """Train a spectral-band ensemble on samples drawn from line-by-line tables: one
    network per band_pts wavenumbers, groups of up to `group` networks per library
    call; a fraction emission_mix of the samples drawn in proportion to kappa I_b.  Returns (params [n_bands * RT_MLP_NPARAM], norms [n_bands, 10], history)
    with history = [(step, mean loss over the networks)] of the first group."""
    import torch
    import synth
    p_nodes = np.asarray(p_nodes, dtype=np.float32)
    tables = training_tables(lines, spec, p_nodes)
    pn = torch.from_numpy(p_nodes).cuda()
    inputs, targets = mlp_make_samples_bands(tables, pn, spec, band_pts, x_lo, x_hi, seed, n_per_band,
                                             emission_mix=emission_mix)
    del tables
    nb = band_count(spec, band_pts)
    norms = band_norms(spec, band_pts, p_nodes, x_lo, x_hi, targets)
    params = torch.from_numpy(synth.mlp_init(seed, spread_biases=True)).cuda().repeat(nb).contiguous()
    hist = []
    for g0 in range(0, nb, group):
        g1 = min(nb, g0 + group)
        pv = params[g0 * RT_MLP_NPARAM:g1 * RT_MLP_NPARAM]
        tr = MlpEnsembleTrainer(pv, norms[g0:g1])
        losses = torch.zeros(max(steps, 1), dtype=torch.float32, device="cuda")
        tr.steps(inputs[g0:g1], targets[g0:g1], batch, lr0, lr1, 1, steps, steps, losses=losses)
        if g0 == 0 and log_every:
            lh = losses.cpu().numpy()
            hist = [(s_, float(lh[s_])) for s_ in range(steps) if s_ % log_every == 0 or s_ == steps - 1]
        del tr
    return params, norms, hist
