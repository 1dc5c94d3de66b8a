"""The C-ABI library loads, exports every entry point include/rt.h declares,
and rejects bad arguments on the host before any launch (no GPU needed)."""
import ctypes as ct
import math
import os
import re

import numpy as np
import pytest

import paper_cs_0703028_gb300 as rt
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rt_[a-z_]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = _declared()
    for n in ("rt_build_kappa", "rt_trace", "rt_tally", "rt_tally_zero", "rt_status_read",
              "rt_last_error", "rt_version", "rt_kappa_table_elems"):
        assert n in names


def test_library_exports_every_declared_symbol():
    L = rt.lib()
    for n in _declared():
        assert hasattr(L, n), n
        assert n in rt._SIGNATURES, f"binding misses {n}"


def test_version_and_table_size():
    assert b"sm_103a" in rt.lib().rt_version()
    s = rt.make_spectral(synth.config(1).spec)
    assert rt.lib().rt_kappa_table_elems(ct.byref(s)) == 64 * 100000
    assert rt.lib().rt_kappa_table_elems(None) == 0


def _status(call):
    st = call()
    return st, rt.lib().rt_last_error().decode()


def test_build_kappa_rejects_bad_input_on_host():
    L = rt.lib()
    case = synth.config(0)
    spec = rt.make_spectral(case.spec)
    lines, keep = rt.make_lines(case.lines)
    dummy = ct.c_void_p(16)   # never dereferenced: validation fails first
    st, msg = _status(lambda: L.rt_build_kappa(None, ct.byref(spec), dummy, None, None, None))
    assert st == rt.RT_E_INVAL
    bad = rt.make_spectral(case.spec)
    bad.dnu = 0.0
    assert L.rt_build_kappa(ct.byref(lines), ct.byref(bad), dummy, None, None, None) == rt.RT_E_INVAL
    bad = rt.make_spectral(case.spec)
    bad.profile = 7
    assert L.rt_build_kappa(ct.byref(lines), ct.byref(bad), dummy, None, None, None) == rt.RT_E_INVAL
    bad = rt.make_spectral(case.spec)
    bad.nT, bad.T_max = 4, bad.T_min
    assert L.rt_build_kappa(ct.byref(lines), ct.byref(bad), dummy, None, None, None) == rt.RT_E_INVAL
    # unsorted and non-finite line lists
    ul = case.lines.subset(np.arange(case.lines.n)[::-1])
    ls, keep2 = rt.make_lines(ul)
    st, msg = _status(lambda: L.rt_build_kappa(ct.byref(ls), ct.byref(spec), dummy, None, None, None))
    assert st == rt.RT_E_UNSORTED and "ascending" in msg
    nl = case.lines.subset(np.arange(case.lines.n))
    nl.S_ref[3] = math.nan
    ls, keep3 = rt.make_lines(nl)
    assert L.rt_build_kappa(ct.byref(ls), ct.byref(spec), dummy, None, None, None) == rt.RT_E_NONFINITE
    nl = case.lines.subset(np.arange(case.lines.n))
    nl.gamma_ref[0] = -1.0
    ls, keep4 = rt.make_lines(nl)
    assert L.rt_build_kappa(ct.byref(ls), ct.byref(spec), dummy, None, None, None) == rt.RT_E_NONFINITE
    # device-resident lines need a status word
    dl = rt.rt_lines(case.lines.n, 16, 16, 16, 16, 296.0, 0.75, 1.0, 44.0, rt.RT_MEM_DEVICE, 0)
    assert L.rt_build_kappa(ct.byref(dl), ct.byref(spec), dummy, None, None, None) == rt.RT_E_INVAL


def test_trace_rejects_bad_input_on_host():
    L = rt.lib()
    case = synth.config(0)
    spec = rt.make_spectral(case.spec)
    g = rt.rt_grid(64, 1, 1, 0, 1 / 64, math.inf, math.inf, 16, None, None)
    t = rt.rt_tally_buf(16, 16, 16, 16)
    k = ct.c_void_p(16)
    assert L.rt_trace(None, k, ct.byref(spec), 0, 10, 10, 0, 0, 0, ct.byref(t), None, None) == rt.RT_E_INVAL
    bad = rt.rt_grid(0, 1, 1, 0, 1.0, 1.0, 1.0, 16, None, None)
    assert L.rt_trace(ct.byref(bad), k, ct.byref(spec), 0, 10, 10, 0, 0, 0, ct.byref(t), None, None) == rt.RT_E_INVAL
    bad = rt.rt_grid(4, 4, 4, 0, math.inf, math.inf, math.inf, 16, None, None)
    assert L.rt_trace(ct.byref(bad), k, ct.byref(spec), 0, 10, 10, 0, 0, 0, ct.byref(t), None, None) == rt.RT_E_INVAL
    bad = rt.rt_grid(4, 4, 4, 0, -1.0, 1.0, 1.0, 16, None, None)
    assert L.rt_trace(ct.byref(bad), k, ct.byref(spec), 0, 10, 10, 0, 0, 0, ct.byref(t), None, None) == rt.RT_E_INVAL
    # n_rays_total smaller than n_rays, unknown flags, NULL tally member, NULL kappa
    assert L.rt_trace(ct.byref(g), k, ct.byref(spec), 0, 10, 5, 0, 0, 0, ct.byref(t), None, None) == rt.RT_E_INVAL
    assert L.rt_trace(ct.byref(g), k, ct.byref(spec), 0, 10, 10, 0, 0, 1 << 9, ct.byref(t), None, None) == rt.RT_E_INVAL
    tb = rt.rt_tally_buf(16, None, 16, 16)
    assert L.rt_trace(ct.byref(g), k, ct.byref(spec), 0, 10, 10, 0, 0, 0, ct.byref(tb), None, None) == rt.RT_E_INVAL
    assert L.rt_trace(ct.byref(g), None, ct.byref(spec), 0, 10, 10, 0, 0, 0, ct.byref(t), None, None) == rt.RT_E_INVAL
    assert L.rt_tally(ct.byref(t), 0, None, None, None) == rt.RT_E_INVAL
    assert L.rt_status_read(None, None) == rt.RT_E_INVAL


def test_tuning_round_trip_and_validation():
    # launch shapes only; the calls touch no device
    before = rt.get_tuning()
    try:
        rt.set_tuning(kappa_t_per_block=4, walk_blocks_per_sm=4, walk_refill_idle=12, walk_group=2)
        assert rt.get_tuning() == {"kappa_t_per_block": 4, "walk_blocks_per_sm": 4, "walk_refill_idle": 12,
                                   "walk_group": 2}
        rt.set_tuning(walk_refill_idle=16)  # other fields keep their value
        assert rt.get_tuning()["walk_blocks_per_sm"] == 4 and rt.get_tuning()["walk_group"] == 2
        for bad in ({"kappa_t_per_block": 9}, {"walk_blocks_per_sm": 3}, {"walk_refill_idle": 8},
                    {"walk_group": 3}):
            with pytest.raises(rt.RtError):
                rt.set_tuning(**bad)
        with pytest.raises(TypeError):
            rt.set_tuning(rays_per_block=1)
        rt.set_tuning(kappa_t_per_block=0, walk_blocks_per_sm=0, walk_refill_idle=0, walk_group=0)  # defaults
        assert rt.get_tuning() == {"kappa_t_per_block": 8, "walk_blocks_per_sm": 5, "walk_refill_idle": 16,
                                   "walk_group": 0}
    finally:
        rt.set_tuning(**before)


def test_adaptive_points_spec_rejected_on_host():
    L = rt.lib()
    case = synth.config(0)
    lines, keep = rt.make_lines(case.lines)
    dummy = ct.c_void_p(16)
    for km in (-1e-3, math.nan, math.inf):
        bad = rt.make_spectral(case.spec)
        bad.kappa_min = km
        st, msg = _status(lambda: L.rt_build_kappa(ct.byref(lines), ct.byref(bad), dummy, None, None, None))
        assert st == rt.RT_E_INVAL and "kappa_min" in msg
    # adaptive windows and fixed points per line exclude each other
    bad = rt.make_spectral(case.spec)
    bad.kappa_min, bad.points_per_line = 1e-3, 128
    st, msg = _status(lambda: L.rt_build_kappa(ct.byref(lines), ct.byref(bad), dummy, None, None, None))
    assert st == rt.RT_E_INVAL and "exclude" in msg


def test_ensemble_entry_points_reject_bad_input_on_host():
    # every case fails validation before any allocation or launch
    L = rt.lib()
    case = synth.config(0)
    spec = rt.make_spectral(case.spec)
    d = ct.c_void_p(16)
    samp = lambda bp=32, lo=0.01, hi=0.3, mix=0.5, n=100, tables=d: L.rt_mlp_make_samples_bands(
        tables, 2, d, ct.byref(spec), bp, lo, hi, mix, 1, n, d, d, None)
    assert samp(mix=1.5) == rt.RT_E_INVAL
    assert samp(mix=math.nan) == rt.RT_E_INVAL
    assert samp(bp=0) == rt.RT_E_INVAL
    assert samp(lo=0.0) == rt.RT_E_INVAL
    assert samp(n=-1) == rt.RT_E_INVAL
    assert samp(tables=None) == rt.RT_E_INVAL
    big = rt.make_spectral(case.spec)
    big.n_nu = 70000
    st, msg = _status(lambda: L.rt_mlp_make_samples_bands(d, 2, d, ct.byref(big), 1, 0.01, 0.3, 0.5, 1, 100,
                                                           d, d, None))
    assert st == rt.RT_E_INVAL and "65535" in msg

    train = lambda nn=2, n=1024, b=256, lr0=1e-3, s0=1, ns=4, tot=4: L.rt_mlp_train_steps_nets(
        nn, d, d, d, d, d, d, n, b, d, lr0, 1e-5, s0, ns, tot, None, None, None)
    assert train(nn=0) == rt.RT_E_INVAL
    assert train(b=2048) == rt.RT_E_INVAL
    assert train(b=0) == rt.RT_E_INVAL
    assert train(lr0=math.nan) == rt.RT_E_INVAL
    assert train(s0=0) == rt.RT_E_INVAL
    assert train(s0=3, ns=4, tot=4) == rt.RT_E_INVAL
    assert train(ns=0) == rt.RT_OK            # no step: nothing allocated or launched

    fwd = lambda nn=2, n=100, p=d: L.rt_mlp_forward_nets(nn, p, d, d, n, d, None, None)
    assert fwd(nn=0) == rt.RT_E_INVAL
    assert fwd(nn=65536) == rt.RT_E_INVAL
    assert fwd(n=-1) == rt.RT_E_INVAL
    assert fwd(p=None) == rt.RT_E_INVAL
    assert fwd(n=0, p=None) == rt.RT_OK       # no sample: buffers are not read

    g = rt.rt_grid(64, 1, 1, 0, 1 / 64, math.inf, math.inf, 16, None, None)
    t = rt.rt_tally_buf(16, 16, 16, 16)
    walk = lambda bp=32, p=d, nm=d, flags=0, n=10, s=spec: L.rt_trace_mlp_bands(
        ct.byref(g), bp, p, nm, ct.byref(s), 0, n, max(n, 10), 0, 0, flags, ct.byref(t), None, None)
    assert walk(p=None) == rt.RT_E_INVAL
    assert walk(nm=None) == rt.RT_E_INVAL
    assert walk(bp=0) == rt.RT_E_INVAL
    assert walk(flags=rt.RT_SRC_BEAM) == rt.RT_E_INVAL
    st, msg = _status(lambda: walk(bp=1, s=big))
    assert st == rt.RT_E_INVAL and "65535" in msg
    st, msg = _status(lambda: walk(n=1 << 32))
    assert st == rt.RT_E_INVAL and "2^32" in msg


def test_wait_probe_rejects_bad_input_on_host():
    L = rt.lib()
    assert L.rt_wait_probe(1000, 1, None, None) == rt.RT_E_INVAL
    assert L.rt_wait_probe(0, 1, ct.c_void_p(16), None) == rt.RT_E_INVAL
    assert L.rt_wait_probe((1 << 24) + 1, 1, ct.c_void_p(16), None) == rt.RT_E_INVAL


def test_table_walk_rejects_the_evaluation_counter_flag():
    L = rt.lib()
    case = synth.config(0)
    spec = rt.make_spectral(case.spec)
    g = rt.rt_grid(64, 1, 1, 0, 1 / 64, math.inf, math.inf, 16, None, None)
    t = rt.rt_tally_buf(16, 16, 16, 16)
    st, msg = _status(lambda: L.rt_trace(ct.byref(g), ct.c_void_p(16), ct.byref(spec), 0, 10, 10, 0, 0,
                                         rt.RT_COUNT_EVALS, ct.byref(t), None, None))
    assert st == rt.RT_E_INVAL and "unknown bits" in msg


def test_evaluation_counter_needs_two_counters():
    # the binding refuses RT_COUNT_EVALS with a one-counter tally before any call
    t = rt.Tally(8, device="cpu")
    with pytest.raises(rt.RtError):
        rt.trace_mlp_bands(None, 16, None, None, None, t, n_rays=1, flags=rt.RT_COUNT_EVALS)
    with pytest.raises(rt.RtError):
        rt.trace_mlp(None, None, None, None, t, n_rays=1, flags=rt.RT_COUNT_EVALS)
