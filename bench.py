"""Benchmark of the Monte-Carlo line-by-line hot path on GB300.

One step = one pass of the whole path over the 32^3-box workload (20k Voigt
lines, 64 temperature nodes x 100k wavenumbers, 1e7 rays): rt_build_kappa
(line geometry, Eq. S prefactors, Eq. tau table) -> rt_tally_zero -> rt_trace
(cell prep, walk) -> rt_tally (binary64 reduction, energy balance).

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on a
bounded ray/column sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

FP32_LANES_PER_SM = 128
MUFU_LANES_PER_SM = 16
# algorithmic work of one profile evaluation, per pipe, in lane operations (FMA = 1):
# a far-wing Voigt evaluation is 1 MUFU reciprocal + 6 binary32 operations (grid
# coordinate, |z|^2, series, accumulation and its share of the Kahan update);
# Lorentz is 1 reciprocal + 4.  The roofline is set by the pipe with the larger
# (count / measured rate): max(FP32 ops / FP32 rate, MUFU ops / MUFU rate).
OPS_PER_EVAL = {"voigt": {"mufu": 1, "fp32": 6}, "lorentz": {"mufu": 1, "fp32": 4},
                # one (cell, nu) update of Eq. I: two exponentials and a reciprocal
                # (attenuation and Planck), interpolation, scale, the update itself
                "march": {"mufu": 3, "fp32": 10},
                # a near-centre Voigt value (fixed points per line): Weideman's N = 24
                # rational series (23 complex multiply-adds, one division), the square
                # root and reciprocal of the width, the compensated add
                "voigt_near": {"mufu": 3, "fp32": 110}}


def alu_roofline(evals_per_s, profile, probe, n_sm, clock_mhz):
    """Roofline of the line sum from the measured FP32 and MUFU ceilings (rt_alu_probe)."""
    ops = OPS_PER_EVAL[profile]
    rate = {"fp32": probe["fma_lane_ops_per_s"], "mufu": probe["rcp_lane_ops_per_s"]}
    pipe = max(ops, key=lambda k: ops[k] / rate[k])
    other = "fp32" if pipe == "mufu" else "mufu"
    achieved = evals_per_s * ops[pipe] / 1e12
    peak = rate[pipe] / 1e12
    mufu_name = "MUFU (ex2, rcp)" if profile == "march" else "MUFU reciprocal"
    return {"bound": "alu", "pipe": {"mufu": mufu_name, "fp32": "FP32"}[pipe],
            "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
            "other_pipe_frac": evals_per_s * ops[other] / rate[other],
            "ops_per_eval": ops,
            "peak_source": "measured by rt_alu_probe (independent chains on every SM)",
            "derived_peaks_tops": {"fp32": n_sm * FP32_LANES_PER_SM * clock_mhz * 1e6 / 1e12,
                                   "mufu": n_sm * MUFU_LANES_PER_SM * clock_mhz * 1e6 / 1e12}}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def ray_range(rank: int, world: int, rays_per_rank: int):
    """Weak scaling: rank r traces rays [r * R, (r + 1) * R) of an N*R-ray estimate."""
    return rank * rays_per_rank, rays_per_rank, world * rays_per_rank


def _clock_sampler(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                 "-lms", "200"], stdout=open(path, "w"), stderr=subprocess.DEVNULL)
    except (OSError, FileNotFoundError):
        return None


def _clock_summary(path, dev_index):
    rows = []
    try:
        for line in open(path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or f[0] != str(dev_index):
                continue
            rows.append(f)
    except OSError:
        return None
    if not rows:
        return None
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    reasons = set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for r in rows:
        for n, v in zip(names, r[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": sorted(reasons), "samples": len(rows)}


def _profiled_traffic(summary, sources):
    """DRAM bytes per launch from a committed ncu summary, or None once the
    kernel's sources have changed since the counters were taken."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", summary)
    try:
        text = open(path).read()
    except OSError:
        return None
    m_sha = re.search(r"source_sha: ([0-9a-f]{12})", text)
    m_tr = re.search(r"traffic_bytes_per_launch \| (\d+)", text)
    if not m_sha or not m_tr:
        return None
    h = hashlib.sha1()
    for s in sources:
        h.update(hashlib.sha1(open(os.path.join(ROOT, "paper_cs_0703028_gb300", "csrc", s), "rb")
                              .read()).hexdigest().encode() + b"  " +
                 os.path.join("paper_cs_0703028_gb300", "csrc", s).encode() + b"\n")
    return int(m_tr.group(1)) if h.hexdigest()[:12] == m_sha.group(1) else None


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def run_gpu(args):
    import torch
    import torch.distributed as dist
    import paper_cs_0703028_gb300 as rt

    world, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    case = synth.config(1)
    spec, lines, grid = case.spec, case.lines, case.grid
    ray_begin, n_rays, n_total = ray_range(rank, world, case.n_rays)

    stream = torch.cuda.current_stream()
    # inputs resident in HBM
    lines_dev, keep_lines = rt.make_lines(lines, memory="device")
    gs, keep_grid = rt.make_grid(grid)
    S = rt.make_spectral(spec)
    kappa = torch.empty((spec.nT, spec.n_nu), dtype=torch.float32, device="cuda")
    evals = torch.zeros(1, dtype=torch.int64, device="cuda")
    bstatus = torch.zeros(1, dtype=torch.int32, device="cuda")
    tally = rt.Tally(grid.ncells)
    L = rt.lib()
    import ctypes as ct
    sp = ct.c_void_p(stream.cuda_stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2
    host_sc = np.zeros(4, dtype=np.float64)

    kb0 = torch.cuda.Event(enable_timing=True)
    kb1 = torch.cuda.Event(enable_timing=True)
    kt0 = torch.cuda.Event(enable_timing=True)
    kt1 = torch.cuda.Event(enable_timing=True)

    def step(timers=None):
        if timers:
            timers[0].record(stream)
        st = L.rt_build_kappa(ct.byref(lines_dev), ct.byref(S), ct.c_void_p(kappa.data_ptr()),
                              ct.c_void_p(evals.data_ptr()), ct.c_void_p(bstatus.data_ptr()), sp)
        if st:
            raise rt.RtError(st, "rt_build_kappa", L.rt_last_error().decode())
        if timers:
            timers[1].record(stream)
        st = L.rt_tally_zero(ct.byref(tally.buf), grid.ncells, sp)
        if timers:
            timers[2].record(stream)
        st |= L.rt_trace(ct.byref(gs), ct.c_void_p(kappa.data_ptr()), ct.byref(S), ray_begin, n_rays,
                         n_total, case.seed, 0, 0, ct.byref(tally.buf), None, sp)
        if timers:
            timers[3].record(stream)
        if st:
            raise rt.RtError(st, "rt_trace", L.rt_last_error().decode())
        st = L.rt_tally(ct.byref(tally.buf), grid.ncells, None, host_sc.ctypes.data, sp)
        if st:
            raise rt.RtError(st, "rt_tally", L.rt_last_error().decode())

    # launch shape of the walk, picked on this workload (untimed; results do not depend on it)
    from paper_cs_0703028_gb300 import autotune
    step()
    torch.cuda.synchronize()
    walk_blocks, walk_tune_ms = autotune.tune_walk(gs, grid.ncells, spec, kappa, n_rays, use_cache=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evals.zero_()
    evals_per_step = None
    steps_per_step = int(tally.steps.item())

    clk_path = os.path.join(tempfile.gettempdir(), f"rt_clocks_{os.getpid()}.csv")
    sampler = _clock_sampler(clk_path) if rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    s0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    s1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(float(i))          # evict the previous step's data from L2 (untimed)
        s0[i].record(stream)
        step(ev[i])
        s1[i].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    if sampler:
        sampler.terminate()
        sampler.wait()
    ms_total = sum(a.elapsed_time(b) for a, b in zip(s0, s1))
    ms_build = sum(e[0].elapsed_time(e[1]) for e in ev) / args.steps
    ms_trace = sum(e[2].elapsed_time(e[3]) for e in ev) / args.steps
    evals_per_step = int(evals.item()) // args.steps
    if world > 1:
        t = torch.tensor([ms_total], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    value = steps_per_step * world / (ms_step * 1e-3)

    # ---- end to end through the public API with host buffers (pinned)
    lines_host = [torch.from_numpy(np.ascontiguousarray(getattr(lines, k))).pin_memory()
                  for k in ("nu0", "S_ref", "gamma_ref", "E_lower")]
    Lh = rt.rt_lines(lines.n, *[t.data_ptr() for t in lines_host], lines.T_ref, lines.n_T,
                     lines.q_exp, lines.mass_amu, rt.RT_MEM_HOST, 0)
    T_host = torch.from_numpy(grid.T).pin_memory()
    p_host = torch.from_numpy(grid.p_atm).pin_memory()
    x_host = torch.from_numpy(grid.x).pin_memory()
    T_dev, p_dev, x_dev = keep_grid
    ab_host = torch.zeros(grid.ncells, dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in lines_host + [T_host, p_host, x_host])
    d2h = ab_host.numel() * 8 + 4 * 8

    def e2e_step():
        T_dev.copy_(T_host, non_blocking=True)
        p_dev.copy_(p_host, non_blocking=True)
        x_dev.copy_(x_host, non_blocking=True)
        st = L.rt_build_kappa(ct.byref(Lh), ct.byref(S), ct.c_void_p(kappa.data_ptr()), None, None, sp)
        st |= L.rt_tally_zero(ct.byref(tally.buf), grid.ncells, sp)
        st |= L.rt_trace(ct.byref(gs), ct.c_void_p(kappa.data_ptr()), ct.byref(S), ray_begin, n_rays,
                         n_total, case.seed, 0, 0, ct.byref(tally.buf), None, sp)
        st |= L.rt_tally(ct.byref(tally.buf), grid.ncells, ab_host.data_ptr(), host_sc.ctypes.data, sp)
        if st:
            raise RuntimeError("e2e step failed: " + L.rt_last_error().decode())

    for _ in range(max(1, args.warmup // 2)):
        e2e_step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e_ms = 0.0
    for i in range(args.steps):
        flush.fill_(float(i))
        e0.record(stream)
        e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        e_ms += e0.elapsed_time(e1)
    e2e_value = steps_per_step * world / (e_ms / args.steps * 1e-3)

    # for context (not the metric): the same trace with the optical-depth cut, which
    # stops rays once tau > 100 (lost fraction < 4e-44) and so counts fewer visits
    cut = rt.Tally(grid.ncells)
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    for rep in range(2):
        cut.zero()
        c0.record(stream)
        st = L.rt_trace(ct.byref(gs), ct.c_void_p(kappa.data_ptr()), ct.byref(S), ray_begin, n_rays,
                        n_total, case.seed, 0, rt.RT_TAU_CUT, ct.byref(cut.buf), None, sp)
        c1.record(stream)
        if st:
            raise rt.RtError(st, "rt_trace (tau cut)", L.rt_last_error().decode())
    torch.cuda.synchronize()
    _, cut_sc, _ = cut.read()
    cut_info = {"trace_ms": c0.elapsed_time(c1), "ray_cell_steps": int(cut.steps.item()),
                "absorbed_total_rel_diff": abs(float(cut_sc[1]) - float(host_sc[1])) / float(host_sc[1])}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    peaks = _peaks()
    clocks = _clock_summary(clk_path, local) if sampler else None
    sm_clock_mhz = peaks.get("sm_max_mhz", 2070.0)
    props = torch.cuda.get_device_properties(local)
    probe = rt.alu_probe()  # measured FP32 and MUFU ceilings
    roof = alu_roofline(evals_per_step / (ms_build * 1e-3), spec.profile, probe,
                        props.multi_processor_count, sm_clock_mhz)
    traffic = _profiled_traffic("k_kappa_box32_voigt20k.md", ["rt_kappa.cu", "rt_common.cuh"])
    # the walk, second kernel of the step: algorithmic 12 B per ray-cell step (the cell's
    # 4-byte T bracket and two 4-byte kappa gathers) against HBM
    hbm_peak = _peaks().get("hbm_gbs", 6771.5)
    walk_gbs = steps_per_step * 12 / (ms_trace * 1e-3) / 1e9
    walk_traffic = _profiled_traffic("k_walk_box32_voigt20k.md", ["rt_trace.cu", "rt_walk.cuh", "rt_common.cuh"])
    out = {
        "metric": "ray-cell steps/s + line-profile evals/s; surrogate vs plain at <=1% tally err",
        "value": value,
        "unit": "ray-cell steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded line list, Gaussian hot-spot field; no HITRAN data)",
        "config": {"workload": "box32_voigt20k: 32^3 cells 1 m^3, 20k Voigt lines 2000-3000 cm^-1, "
                               "64 T x 100k nu table, 1e7 rays per GPU",
                   "ncells": grid.ncells, "n_lines": lines.n, "n_nu": spec.n_nu, "nT": spec.nT,
                   "rays_per_gpu": n_rays, "l2": "flushed between steps (256 MB write, untimed)"},
        "line_profile_evals_per_s": evals_per_step * world / (ms_step * 1e-3),
        "ray_cell_steps_per_step": steps_per_step,
        "profile_evals_per_step": evals_per_step,
        "kernels_ms": {"rt_build_kappa": ms_build, "rt_trace": ms_trace},
        "energy_residual": float(host_sc[3]),
        # per step: k_line_geometry, k_prefactor, k_tile_lines, k_kappa; k_cell_prep, walk
        # table copy, k_walk; k_reduce, k_final
        "gpu_launches": 9 * args.steps,
        "tuning": {"walk_blocks_per_sm": walk_blocks[0], "walk_refill_idle": walk_blocks[1],
                   "walk_candidates_ms": walk_tune_ms},
        "roofline": {"kernel": "k_kappa (rt_build_kappa)", **roof, "traffic": traffic,
                     "timed": "rt_build_kappa (k_kappa and its three small set-up kernels)"},
        "e2e": {"value": e2e_value, "unit": "ray-cell steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "walk_roofline": {"kernel": "k_walk (rt_trace)", "bound": "hbm", "achieved": walk_gbs,
                          "peak": hbm_peak, "unit": "GB/s", "frac": walk_gbs / hbm_peak,
                          "traffic": walk_traffic, "bytes_per_step": 12,
                          "note": "tables L2-resident; latency- and issue-bound (profiles/)"},
        "trace_with_tau_cut": cut_info,
        "clocks": clocks,
    }
    if world == 1 and not args.no_surrogate:
        out["surrogate"] = surrogate_summary(args)
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(case, evals_per_step, steps_per_step, budget_s=args.cpu_seconds)
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def cpu_baseline(case, evals_full, steps_full, budget_s=15.0):
    """The FP64 oracle, as it stands, on a bounded ray sample of the same step:
    the kappa columns those rays use (all 64 T) and the walk of those rays;
    throughput extrapolated to the full step."""
    from oracle import kappa as okappa
    from oracle import trace as otrace
    threads = otrace.default_threads()
    n = 64
    t_k = t_w = 0.0
    ev = st = rays = 0
    rb = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        _, j = otrace.emission_indices(case.grid.ncells, case.spec.n_nu, case.seed, rb, n)
        cols = np.unique(j)
        a = time.perf_counter()
        K = okappa.kappa_columns(case.lines, case.spec, cols)
        b = time.perf_counter()
        lo, hi = okappa.line_ranges(case.lines, case.spec)
        nu = okappa.grid_nu(case.spec, cols)
        col_evals = np.searchsorted(case.lines.nu0, nu + case.spec.cutoff, "right") - \
            np.searchsorted(case.lines.nu0, nu - case.spec.cutoff, "left")
        r = otrace.trace(case.grid, case.spec, K, seed=case.seed, ray_begin=rb, n_rays=n,
                         n_total=case.n_rays, columns=cols, threads=threads)
        c = time.perf_counter()
        t_k += b - a
        t_w += c - b
        ev += int(col_evals.sum()) * case.spec.nT
        st += r.steps
        rays += n
        rb += n
    evals_per_s = ev / t_k
    steps_per_s = st / t_w
    t_full = evals_full / evals_per_s + steps_full / steps_per_s
    return {"value": steps_full / t_full, "unit": "ray-cell steps/s", "cores": threads,
            "kind": "oracle",
            "sample": f"rays [0, {rays}) of the 1e7-ray step and the {ev // case.spec.nT} (line, nu) "
                      f"pairs of their columns at all 64 T; kappa oracle numpy/scipy on 1 core, walk "
                      f"oracle C on {threads} threads; full-step time extrapolated from "
                      f"{evals_per_s:.3g} evals/s and {steps_per_s:.3g} steps/s",
            "line_profile_evals_per_s": evals_per_s, "ray_cell_steps_per_s": steps_per_s}


def run_reference(args):
    world, rank = _dist()
    if rank != 0:
        return
    case = synth.config(1)
    from oracle import kappa as okappa
    # full-step work (exact profile-evaluation count, ray-cell steps from a ray sample)
    evals_full = okappa.profile_evals(case.lines, case.spec)
    from oracle import trace as otrace
    K1 = np.full((case.spec.nT, case.spec.n_nu), 1e-3)
    probe = otrace.trace(case.grid, case.spec, K1, seed=case.seed, n_rays=20000, n_total=case.n_rays)
    steps_full = int(probe.steps * (case.n_rays / 20000))
    per = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_baseline(case, evals_full, steps_full, budget_s=per)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(case, evals_full, steps_full, budget_s=per))
    el = time.perf_counter() - t0
    v = statistics.median([x["value"] for x in vals])
    ms_step = steps_full / v * 1e3
    cb = dict(vals[-1])
    cb["value"] = v
    out = {"impl": "reference", "metric": "ray-cell steps/s + line-profile evals/s; surrogate vs plain at "
                                          "<=1% tally err",
           "value": v, "unit": "ray-cell steps/s", "n_gpus": 0, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "box32_voigt20k: 32^3 cells 1 m^3, 20k Voigt lines 2000-3000 cm^-1, "
                                  "64 T x 100k nu table, 1e7 rays per GPU"},
           "cpu_baseline": cb, "wall_s": el,
           "e2e": {"value": v, "unit": "ray-cell steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def _ev_time(fn, reps=1):
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def surrogate_summary(args):
    """Compact form of run_surrogate for the default benchmark line."""
    import io
    import contextlib
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        run_surrogate(args)
    r = json.loads(buf.getvalue().strip().splitlines()[-1])
    w = r["walks"]
    return {"workload": r["config"]["workload"],
            "steps_per_s": {k: w[k]["ray_cell_steps_per_s"] for k in w},
            "speedup_vs_lbl": r["speedup_vs_lbl"],
            "tally_error_vs_table_median": r["tally_error_vs_table"]["median"],
            "meets_1pct_target": r["tally_error_vs_table"]["max"] <= 0.01,
            "tensor_roofline": r["tensor_roofline"],
            "training": r["training"]}


def run_surrogate(args):
    """Table walk vs surrogate-network walk vs on-the-fly line-by-line walk on the
    64^3 learned-part workload (same rays), after training the network."""
    import torch
    import paper_cs_0703028_gb300 as rt
    from paper_cs_0703028_gb300 import surrogate
    case = synth.config(2)
    spec = case.spec
    ex = case.extra
    p_nodes = np.exp(np.linspace(np.log(ex["train_p"][0]), np.log(ex["train_p"][1]), ex["train_p"][2]))
    t0 = time.time()
    params, norm, hist = surrogate.train_surrogate(case.lines, spec, p_nodes, ex["train_x"][0],
                                                   ex["train_x"][1], n_samples=args.samples,
                                                   batch=8192, epochs=args.epochs, log_every=500)
    torch.cuda.synchronize()
    train_s = time.time() - t0
    # device time of the training steps alone (one rt_mlp_train_steps call over K
    # 8192-sample batches of synthetic inputs within the training ranges; no table
    # build, no sampling)
    K, B = 100, 8192
    lo, hi = surrogate.input_ranges(spec, p_nodes, ex["train_x"][0], ex["train_x"][1])
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1)
    lo_t = torch.tensor(lo, dtype=torch.float32, device="cuda")
    hi_t = torch.tensor(hi, dtype=torch.float32, device="cuda")
    xs = lo_t + (hi_t - lo_t) * torch.rand((K * B, 4), device="cuda", generator=gen)
    ys = torch.randn(K * B, device="cuda", generator=gen)
    tr = rt.MlpTrainer(params.clone(), norm)
    tl = torch.zeros(K, dtype=torch.float32, device="cuda")
    run_k = (lambda: tr.steps(xs, ys, B, 1e-4, 1e-5, 1, K, K, losses=tl))
    run_k()
    step_ms = _ev_time(run_k) / K
    del xs, ys, tr, tl
    g = case.grid
    gs, keep = rt.make_grid(g)
    kap = rt.build_kappa(case.lines, spec)
    n = args.rays
    out = {}
    runs = {"table": (lambda t: rt.trace(gs, kap, spec, t, n_rays=n, n_rays_total=n)),
            "mlp": (lambda t: rt.trace_mlp(gs, params, norm, spec, t, n_rays=n, n_rays_total=n)),
            "lbl": (lambda t: rt.trace_lbl(gs, case.lines, spec, t, n_rays=n // 50, n_rays_total=n))}
    tallies = {}
    for name, fn in runs.items():
        t = rt.Tally(g.ncells)
        t.zero()
        fn(t)
        t.zero()
        ms = _ev_time(lambda: fn(t))
        ab, sc, _ = t.read()
        steps = int(t.steps.item())
        tallies[name] = ab
        out[name] = {"ray_cell_steps_per_s": steps / (ms * 1e-3), "ms": ms, "steps": steps,
                     "energy_residual": float(sc[3])}
    ref = tallies["table"]
    big = ref >= 1e-3 * ref.max()
    err = np.abs(tallies["mlp"][big] - ref[big]) / ref[big]
    res = {"metric": "ray-cell steps/s, surrogate walk vs on-the-fly line-by-line walk",
           "value": out["mlp"]["ray_cell_steps_per_s"], "unit": "ray-cell steps/s",
           "higher_is_better": True, "config": {"workload": "box64 learned part, 20k Voigt lines, "
                                                           f"{n} rays (line-by-line walk: {n // 50})"},
           "walks": out, "speedup_vs_lbl": out["mlp"]["ray_cell_steps_per_s"] / out["lbl"]["ray_cell_steps_per_s"],
           "tally_error_vs_table": {"median": float(np.median(err)), "p90": float(np.percentile(err, 90)),
                                    "max": float(err.max()), "cells": int(big.sum()),
                                    "total": float(tallies["mlp"].sum() / ref.sum() - 1.0)},
           "training": {"seconds": train_s, "samples": args.samples, "epochs": args.epochs,
                        "loss_first": hist[0][1], "loss_last": hist[-1][1],
                        "device_ms_per_step": step_ms, "samples_per_s": B / (step_ms * 1e-3),
                        "step_note": f"{K} steps of {B} samples in one rt_mlp_train_steps call, CUDA events"}}
    # tensor-core work: three 128x128 layers, 2 * 128 * 128 flops each per network evaluation
    # (one per ray-cell step in the walk; forward + two backward products per training sample)
    peak = _peaks().get("bf16_tflops", 1978.3)
    eval_flops = 3 * 2 * 128 * 128
    walk_tf = out["mlp"]["ray_cell_steps_per_s"] * eval_flops / 1e12
    train_tf = args.samples * args.epochs * 3 * eval_flops / train_s / 1e12
    res["tensor_roofline"] = {"bound": "tensor", "unit": "TFLOP/s", "peak": peak,
                              "peak_source": "measured bf16 burst (MEASURED_PEAKS.json)",
                              "walk_achieved": walk_tf, "walk_frac": walk_tf / peak,
                              "training_achieved": train_tf, "training_frac": train_tf / peak,
                              "training_note": "wall clock incl. tables, sampling and Adam; 8192-sample batches",
                              "training_step_achieved": B * 3 * eval_flops / (step_ms * 1e-3) / 1e12,
                              "training_step_frac": B * 3 * eval_flops / (step_ms * 1e-3) / 1e12 / peak}
    print(json.dumps(res), flush=True)


def run_batched(args):
    """256 enclosures in one persistent (graph-replayed) launch vs 256 rt_trace calls."""
    import torch
    import paper_cs_0703028_gb300 as rt
    from paper_cs_0703028_gb300 import autotune
    case = synth.config(3)
    encl = case.extra["enclosures"]
    scale = args.rays_scale
    grids = [g for g, _ in encl]
    rays = [max(1, int(r * scale)) for _, r in encl]
    kap = rt.build_kappa(case.lines, case.spec)
    (rpi, th), tune_ms = autotune.tune_batch(grids, rays, case.spec, kap, reps=1)
    B = rt.Batch(grids, rays, case.spec, rays_per_item=rpi, threads=th)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    gph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gph, stream=s):
        B.zero(stream=s)
        B.trace(kap, stream=s)
    gph.replay()
    ms_graph = _ev_time(gph.replay, reps=args.steps)
    steps = sum(int(t.steps.item()) for t in B.tallies)
    singles = [(rt.make_grid(g), rt.Tally(g.ncells)) for g in grids]

    def separate():
        for e, ((gs, _), t) in enumerate(singles):
            t.zero()
            rt.trace(gs, kap, case.spec, t, n_rays=rays[e], n_rays_total=rays[e], enclosure=e)
    separate()
    ms_sep = _ev_time(separate, reps=args.steps)
    res = {"metric": "ray-cell steps/s, 256 enclosures", "value": steps / (ms_graph * 1e-3),
           "unit": "ray-cell steps/s", "higher_is_better": True,
           "config": {"workload": f"batched256: sides 8..48, {sum(rays)} rays ({scale:g} x 1e3 per cell)",
                      "cells": int(sum(g.ncells for g in grids))},
           "graph_ms": ms_graph, "separate_launches_ms": ms_sep, "speedup": ms_sep / ms_graph,
           "steps": steps, "autotuned": {"rays_per_item": rpi, "threads": th, "candidates_ms": tune_ms}}
    B.close()
    print(json.dumps(res), flush=True)


def pressure_reading_error(rt, case, kap, n_rays=1_000_000):
    """Per-cell tally error of the table walk (T-node table at p_ref, kappa scaled by the
    cell's density p x / (p_ref x_ref); the widths' pressure dependence is not tabulated)
    against the on-the-fly line-by-line walk at each cell's own (T, p, x), same rays, on the
    16^3 version of the 128^3 fields; and with p = p_ref everywhere, which leaves only the
    linear-in-T interpolation, so that the pressure reading's share shows."""
    import torch
    from dataclasses import replace
    g16 = synth.multi_gaussian_grid(16, 1.0, synth.rng_for(4, 1))
    out = {"grid": "16^3, same recipe and seed as the 128^3 fields", "rays": n_rays}
    for name, grid in (("p_field_1_3_atm", g16),
                       ("p_ref_everywhere", replace(g16, p_atm=np.full_like(g16.p_atm, case.spec.p_ref_atm)))):
        gs, keep = rt.make_grid(grid)
        tallies = {}
        for walk in ("table", "lbl"):
            t = rt.Tally(grid.ncells)
            t.zero()
            if walk == "table":
                rt.trace(gs, kap, case.spec, t, n_rays=n_rays, n_rays_total=n_rays)
            else:
                rt.trace_lbl(gs, case.lines, case.spec, t, n_rays=n_rays, n_rays_total=n_rays)
            tallies[walk] = t.read()[0]
        ref, got = tallies["lbl"], tallies["table"]
        big = ref >= 1e-3 * ref.max()
        err = np.abs(got[big] - ref[big]) / ref[big]
        out[name] = {"median": float(np.median(err)), "p90": float(np.percentile(err, 90)),
                     "max": float(err.max()), "cells": int(big.sum()),
                     "total": float(got.sum() / ref.sum() - 1.0)}
    torch.cuda.synchronize()
    return out


def _resident_build(rt, lines):
    """A kappa build of device-resident lines (inputs already in HBM, as in the timed
    step of the 32^3 workload): returns build(spec, out, evals=None)."""
    import ctypes as ct
    import torch
    Ld, keep = rt.make_lines(lines, memory="device")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    L = rt.lib()

    def build(spec, out, evals=None):
        S = rt.make_spectral(spec)
        st = L.rt_build_kappa(ct.byref(Ld), ct.byref(S), ct.c_void_p(out.data_ptr()),
                              None if evals is None else ct.c_void_p(evals.data_ptr()),
                              ct.c_void_p(status.data_ptr()),
                              ct.c_void_p(torch.cuda.current_stream().cuda_stream))
        if st:
            raise rt.RtError(st, "rt_build_kappa", L.rt_last_error().decode())
    build.keep = (Ld, keep, status)
    return build


def run_next(args):
    """The rows after the hot path, on the 32^3 workload's line list and table: the
    paper's spectrally resolved marching (Eq. I per wavenumber along 4096 straight
    paths), the fixed 16 points per line, and a second gas accumulated into the table."""
    import torch
    from dataclasses import replace
    import paper_cs_0703028_gb300 as rt
    case = synth.config(1)
    spec = case.spec
    probe = rt.alu_probe()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    clock = _peaks().get("sm_max_mhz", 2070.0)
    kap = rt.build_kappa(case.lines, spec)
    gs, keep = rt.make_grid(case.grid)
    rng = np.random.default_rng(7)
    n = 4096
    pos = torch.from_numpy((rng.uniform(0.02, 0.98, (n, 3)) * 1.0).astype(np.float32)).cuda()
    d = rng.normal(size=(n, 3))
    d = torch.from_numpy((d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)).cuda()
    nvis = torch.zeros(n, dtype=torch.int32, device="cuda")
    march = lambda: rt.march(gs, kap, spec, pos, d, want_I=False, nvis=nvis)
    for _ in range(args.warmup):
        march()
    ms_march = _ev_time(march, reps=args.steps)
    updates = int(nvis.sum().item()) * spec.n_nu
    out = {"march": {"paths": n, "cells_crossed": int(nvis.sum().item()), "updates": updates,
                     "ms": ms_march, "updates_per_s": updates / (ms_march * 1e-3),
                     "roofline": alu_roofline(updates / (ms_march * 1e-3), "march", probe, n_sm, clock),
                     "note": "per call: cell preparation, the paths' walk and the marching kernel"}}
    # fixed 16 points per line (lines resident in HBM)
    co2 = _resident_build(rt, case.lines)
    s16 = replace(spec, points_per_line=16)
    ev = torch.zeros(1, dtype=torch.int64, device="cuda")
    k16 = torch.empty((spec.nT, spec.n_nu), dtype=torch.float32, device="cuda")
    co2(s16, k16, ev)
    torch.cuda.synchronize()
    ev16 = int(ev.item())
    for _ in range(args.warmup):
        co2(s16, k16)
    ms16 = _ev_time(lambda: co2(s16, k16), reps=args.steps)
    out["points_per_line_16"] = {"evals": ev16, "ms": ms16, "evals_per_s": ev16 / (ms16 * 1e-3),
                                 "roofline": alu_roofline(ev16 / (ms16 * 1e-3), "voigt_near", probe, n_sm,
                                                          clock),
                                 "note": "per call: line geometry, prefactors and the gather kernel"}
    # a second gas (an H2O-like list: 10k lines, mass 18 u) accumulated into the CO2 table
    h2o = replace(synth.make_lines(10000, 2000.0, 3000.0, synth.rng_for(1, 9), S_lo=1e-23, S_hi=1e-20),
                  mass_amu=18.0, n_T=0.6, q_exp=1.5)
    s2 = replace(spec, x_ref=0.05, accumulate=1)
    h2o_build = _resident_build(rt, h2o)
    tab = torch.empty((spec.nT, spec.n_nu), dtype=torch.float32, device="cuda")
    e1 = torch.zeros(1, dtype=torch.int64, device="cuda")
    e2 = torch.zeros(1, dtype=torch.int64, device="cuda")
    co2(spec, tab, e1)
    h2o_build(s2, tab, e2)
    torch.cuda.synchronize()
    ev2 = int(e1.item()) + int(e2.item())

    def two_gas():
        co2(spec, tab)
        h2o_build(s2, tab)
    for _ in range(args.warmup):
        two_gas()
    ms2 = _ev_time(two_gas, reps=args.steps)
    out["two_gases"] = {"evals": ev2, "ms": ms2, "evals_per_s": ev2 / (ms2 * 1e-3),
                        "roofline": alu_roofline(ev2 / (ms2 * 1e-3), "voigt", probe, n_sm, clock)}
    res = {"metric": "Eq. I updates/s (marching), line-profile evals/s (variants)",
           "value": out["march"]["updates_per_s"], "unit": "(cell, nu) updates/s", "higher_is_better": True,
           "config": {"workload": "next32: 32^3 box, 20k Voigt lines, 64 T x 100k nu; 4096 paths"},
           **out}
    print(json.dumps(res), flush=True)


def run_box128(args):
    """The 128^3 workload: 100k lines, 64 T x 400k nu table, and the walk."""
    import torch
    import paper_cs_0703028_gb300 as rt
    case = synth.config(4)
    spec = case.spec
    n = int(case.n_rays * args.rays_scale)
    gs, keep = rt.make_grid(case.grid)
    kap = torch.empty((spec.nT, spec.n_nu), dtype=torch.float32, device="cuda")
    evals = torch.zeros(1, dtype=torch.int64, device="cuda")
    build = _resident_build(rt, case.lines)  # lines resident in HBM
    build(spec, kap, evals)
    torch.cuda.synchronize()
    ev = int(evals.item())
    for _ in range(args.warmup):
        build(spec, kap)
    ms_build = _ev_time(lambda: build(spec, kap), reps=args.steps)
    from paper_cs_0703028_gb300 import autotune
    walk_shape, walk_ms = autotune.tune_walk(gs, case.grid.ncells, spec, kap, min(n, 10_000_000),
                                             use_cache=False)
    t = rt.Tally(case.grid.ncells)
    t.zero()
    rt.trace(gs, kap, spec, t, n_rays=min(n, 10_000_000), n_rays_total=n)
    t.zero()
    ms_trace = _ev_time(lambda: rt.trace(gs, kap, spec, t, n_rays=n, n_rays_total=n))
    ab, sc, _ = t.read()
    steps = int(t.steps.item())
    hbm = _peaks().get("hbm_gbs", 6771.5)
    res = {"metric": "ray-cell steps/s + line-profile evals/s", "value": steps / (ms_trace * 1e-3),
           "unit": "ray-cell steps/s", "higher_is_better": True,
           "config": {"workload": f"box128_voigt100k: 128^3 cells, 100k Voigt lines, 64 T x 400k nu, {n} rays"},
           "build_ms": ms_build, "evals": ev, "line_profile_evals_per_s": ev / (ms_build * 1e-3),
           "trace_ms": ms_trace, "steps": steps, "energy_residual": float(sc[3]),
           "walk_hbm_frac_at_16B_per_step": steps * 16 / (ms_trace * 1e-3) / (hbm * 1e9),
           "build_roofline": alu_roofline(ev / (ms_build * 1e-3), spec.profile, rt.alu_probe(),
                                          torch.cuda.get_device_properties(0).multi_processor_count,
                                          _peaks().get("sm_max_mhz", 2070.0)),
           "tuning": {"walk_blocks_per_sm": walk_shape[0], "walk_refill_idle": walk_shape[1],
                      "walk_candidates_ms_1e7_rays": walk_ms},
           "pressure_reading_error_vs_lbl": pressure_reading_error(rt, case, kap)}
    print(json.dumps(res), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--workload", default="box32", choices=["box32", "surrogate", "batched", "box128", "next"])
    ap.add_argument("--samples", type=int, default=20_000_000)
    ap.add_argument("--epochs", type=int, default=1)
    ap.add_argument("--rays", type=int, default=2_000_000)
    ap.add_argument("--rays-scale", type=float, default=1.0)
    args = ap.parse_args()
    if args.workload == "surrogate":
        return run_surrogate(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "box128":
        return run_box128(args)
    if args.workload == "next":
        return run_next(args)
    if args.warmup < 3 and args.impl == "gb300":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
