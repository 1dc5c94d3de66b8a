"""Autotuner for launch shapes (no effect on results, only on speed).

Each tuner times its candidates on the caller's actual workload with CUDA
events (after one warm-up launch each), keeps the fastest, and caches the
choice in a JSON file keyed by a signature of the workload's sizes
(``$RT_GB300_TUNE_CACHE`` or ``~/.cache/paper_cs_0703028_gb300/tune.json``).

* ``tune_kappa``: temperature nodes per rt_build_kappa block (1, 2, 4, 8).
* ``tune_batch``: rays per work item and threads per block of the batched walk.
* ``tune_walk``: resident blocks per SM (4 or 5) and refill threshold (12 or 16) of the rt_trace walk,
  then whether grouping its rays by wavenumber pays.
"""
from __future__ import annotations

import json
import os

from . import Batch, Tally, build_kappa, set_tuning, trace


def _cache_path():
    p = os.environ.get("RT_GB300_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_cs_0703028_gb300", "tune.json")


def _load():
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key, value):
    data = _load()
    data[key] = value
    path = _cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def _time(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def tune_kappa(lines, spec, candidates=(1, 2, 4, 8), reps=3, use_cache=True):
    """Pick the temperature nodes per block of rt_build_kappa; returns (best, {tpb: ms})."""
    import torch
    key = f"kappa:{spec.profile}:{lines.n}:{spec.n_nu}:{spec.nT}:{spec.dnu}:{spec.cutoff}"
    if use_cache and key in _load():
        best = int(_load()[key]["best"])
        set_tuning(kappa_t_per_block=best)
        return best, _load()[key]["ms"]
    out = torch.empty((spec.nT, spec.n_nu), dtype=torch.float32, device="cuda")
    times = {}
    for c in candidates:
        set_tuning(kappa_t_per_block=c)
        times[int(c)] = _time(lambda: build_kappa(lines, spec, out=out), reps)
    best = min(times, key=times.get)
    set_tuning(kappa_t_per_block=best)
    _store(key, {"best": best, "ms": times})
    return best, times


def tune_batch(grids, n_rays, spec, kappa, candidates=None, reps=2, use_cache=True, seed=0):
    """Pick (rays_per_item, threads) of the batched walk; returns (best, {str: ms})."""
    if candidates is None:
        candidates = [(r, t) for r in (1024, 4096, 16384) for t in (128, 256)]
    sig = sum(g.nx * g.ny * g.nz for g in grids)
    key = f"batch:{len(grids)}:{sig}:{int(sum(n_rays))}:{spec.n_nu}:{spec.nT}"
    if use_cache and key in _load():
        b = _load()[key]["best"]
        return (int(b[0]), int(b[1])), _load()[key]["ms"]
    times = {}
    for rpi, th in candidates:
        B = Batch(grids, n_rays, spec, seed=seed, rays_per_item=rpi, threads=th)
        times[f"{rpi},{th}"] = _time(lambda: B.trace(kappa), reps)
        B.close()
    best = min(times, key=times.get)
    rpi, th = (int(v) for v in best.split(","))
    _store(key, {"best": [rpi, th], "ms": times})
    return (rpi, th), times


def tune_walk(grid_struct, ncells, spec, kappa, n_rays, candidates=None, reps=2, use_cache=True,
              n_rays_group=None):
    """Pick the walk's (resident blocks per SM, refill threshold) on the caller's trace
    (n_rays rays, no wavenumber grouping), then, with that shape, whether grouping the
    rays by wavenumber pays on n_rays_group rays (default n_rays): grouping costs a
    counting pass over the rays and gains only when many rays share each wavenumber.
    Returns ((blocks, refill, group), {"blocks,refill[,group]": ms}) with group 1 (off)
    or 2 (on) as rt_tuning.walk_group."""
    if candidates is None:
        candidates = [(b, r) for b in (4, 5) for r in (12, 16)]
    ng = int(n_rays if n_rays_group is None else n_rays_group)
    key = f"walk:{ncells}:{spec.n_nu}:{spec.nT}:{int(n_rays)}:{ng}"
    cached = _load().get(key) if use_cache else None
    if cached and tuple(int(v) for v in cached["best"][:2]) in [tuple(c) for c in candidates]:
        b, r, g = (int(v) for v in cached["best"])   # a cached shape that is still a candidate
        set_tuning(walk_blocks_per_sm=b, walk_refill_idle=r, walk_group=g)
        return (b, r, g), cached["ms"]
    tally = Tally(ncells)
    times = {}
    set_tuning(walk_group=1)
    for b, r in candidates:
        set_tuning(walk_blocks_per_sm=b, walk_refill_idle=r)
        times[f"{b},{r}"] = _time(lambda: (tally.zero(), trace(grid_struct, kappa, spec, tally, n_rays)), reps)
    best = min(times, key=times.get)
    b, r = (int(v) for v in best.split(","))
    set_tuning(walk_blocks_per_sm=b, walk_refill_idle=r)
    tg = {}
    for g in (1, 2):
        set_tuning(walk_group=g)
        tg[g] = _time(lambda: (tally.zero(), trace(grid_struct, kappa, spec, tally, ng)), 1)
        times[f"{b},{r},{g}"] = tg[g]
    g = min(tg, key=tg.get)
    set_tuning(walk_group=g)
    _store(key, {"best": [b, r, g], "ms": times})
    return (b, r, g), times
