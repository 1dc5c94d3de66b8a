"""Python front of the FP64 ray-tracing oracle in ``trace.c`` (test infrastructure).

Section 3 (Fig. "Monte-Carlo ray-tracing", Eq. I first term, Eq. planck): the
estimator of absorbed power per finite volume.  See ``trace.c`` for the
readings of the paper it implements.  Parity: pinned (plane-parallel E3
exchange closed form, brute-force quadrature of the estimator, isothermal
column exp(-kappa L), energy balance, DDA chord and adjacency, Philox against
the CUDA toolkit's host Philox generator).
"""
from __future__ import annotations

import ctypes as ct
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle_trace.so")
_lock = threading.Lock()
_lib = None

MODE_EMIT, MODE_BEAM = 0, 1


def build(force: bool = False) -> str:
    """Compile trace.c (binary32 geometry needs -ffp-contract=off)."""
    src = os.path.join(_HERE, "trace.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-fno-strict-aliasing", "-pthread", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class OgGrid(ct.Structure):
    _fields_ = [("nx", ct.c_int32), ("ny", ct.c_int32), ("nz", ct.c_int32), ("pad", ct.c_int32),
                ("hx", ct.c_double), ("hy", ct.c_double), ("hz", ct.c_double),
                ("T", ct.c_void_p), ("p", ct.c_void_p), ("x", ct.c_void_p)]


class OgSpec(ct.Structure):
    _fields_ = [("nu_min", ct.c_double), ("dnu", ct.c_double), ("n_nu", ct.c_int64),
                ("nT", ct.c_int32), ("pad", ct.c_int32), ("T_min", ct.c_double),
                ("T_max", ct.c_double), ("p_ref", ct.c_double), ("x_ref", ct.c_double)]


class OgTable(ct.Structure):
    _fields_ = [("kappa", ct.c_void_p), ("ncol", ct.c_int64), ("col_of_j", ct.c_void_p),
                ("per_cell", ct.c_int32), ("pad", ct.c_int32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ct.CDLL(build())
            P = ct.c_void_p
            L.oracle_philox.argtypes = [P, P, P]
            L.oracle_trace.argtypes = [P, P, P, ct.c_uint64, ct.c_uint32, ct.c_uint64, ct.c_uint64,
                                       ct.c_uint64, ct.c_int, ct.c_int, ct.c_int, P, P, P,
                                       ct.c_int64, ct.c_int32, P, P, P, P, P]
            L.oracle_sample_rays.argtypes = [P, P, P, ct.c_uint64, ct.c_uint32, ct.c_uint64,
                                             ct.c_uint64, ct.c_uint64, ct.c_int, P, P, P, P, P]
            L.oracle_emission_indices.argtypes = [ct.c_int64, ct.c_int64, ct.c_uint64,
                                                  ct.c_uint32, ct.c_uint64, ct.c_uint64, P, P]
            L.oracle_emission_indices.restype = None
            L.oracle_walk_rays.argtypes = [P, P, P, ct.c_int64, P, P, P, P, P, P, P]
            L.oracle_cell_prep.argtypes = [P, P, P, P, P]
            L.oracle_march.argtypes = [P, P, P, ct.c_int64, P, P, P, P, P]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


class _Inputs:
    """Keeps the numpy buffers behind the ctypes structs alive."""

    def __init__(self, grid, spec, kappa=None, columns=None, per_cell=False):
        self.T = np.ascontiguousarray(grid.T, dtype=np.float32)
        self.p = None if grid.p_atm is None else np.ascontiguousarray(grid.p_atm, dtype=np.float32)
        self.x = None if grid.x is None else np.ascontiguousarray(grid.x, dtype=np.float32)
        self.g = OgGrid(grid.nx, grid.ny, grid.nz, 0, float(grid.hx), float(grid.hy),
                        float(grid.hz), _p(self.T), _p(self.p), _p(self.x))
        self.s = OgSpec(float(spec.nu_min), float(spec.dnu), int(spec.n_nu), int(spec.nT), 0,
                        float(spec.T_min), float(spec.T_max), float(spec.p_ref_atm),
                        float(spec.x_ref))
        if kappa is not None:
            self.K = np.ascontiguousarray(kappa, dtype=np.float64)
            ncol = self.K.shape[1]
            rows = grid.nx * grid.ny * grid.nz if per_cell else max(1, int(spec.nT))
            if self.K.ndim != 2 or self.K.shape[0] != rows:
                raise ValueError(f"kappa must be ({rows}, ncol), got {self.K.shape}")
            if columns is None:
                self.map = None
            else:
                self.map = np.full(spec.n_nu, -1, dtype=np.int64)
                self.map[np.asarray(columns, dtype=np.int64)] = np.arange(ncol)
            self.t = OgTable(_p(self.K), ncol, _p(self.map), int(bool(per_cell)), 0)
        else:
            self.t = OgTable(None, 0, None, 0, 0)


def philox4x32_10(counter, key):
    """Philox4x32-10 of one 128-bit counter (4 words) under a 64-bit key (2 words)."""
    c = np.asarray(counter, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox(_p(c), _p(k), _p(out))
    return out


def emission_indices(ncells, n_nu, seed, ray_begin, n, enclosure=0):
    cell = np.zeros(n, dtype=np.int64)
    j = np.zeros(n, dtype=np.int64)
    lib().oracle_emission_indices(int(ncells), int(n_nu), int(seed), int(enclosure),
                                  int(ray_begin), int(n), _p(cell), _p(j))
    return cell, j


def default_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


class TraceResult:
    def __init__(self, absorbed, scalars, steps, rec=None):
        self.absorbed = absorbed
        self.emitted, self.absorbed_total, self.escaped = (float(v) for v in scalars)
        self.steps = int(steps)
        self.rec = rec

    @property
    def energy_residual(self) -> float:
        return abs(self.emitted - self.absorbed_total - self.escaped) / self.emitted


def trace(grid, spec, kappa, seed=0, ray_begin=0, n_rays=1000, n_total=None, mode=MODE_EMIT,
          columns=None, tau_cut=False, enclosure=0, n_record=0, max_visits=None, threads=None,
          per_cell=False):
    """Run the estimator on rays [ray_begin, ray_begin + n_rays) of an N = n_total run.

    kappa: (nT, ncol) float64 table, or with per_cell=True (ncells, ncol): each
    cell's own absorption coefficient at its state (no T interpolation, no
    density scale); columns: the j of each table column (None = all n_nu
    columns).  Returns a TraceResult; with n_record > 0 the first n_record
    rays' visit sequences are returned in ``rec``.
    """
    n_total = n_rays if n_total is None else n_total
    I = _Inputs(grid, spec, kappa, columns, per_cell)
    ncells = grid.nx * grid.ny * grid.nz
    absorbed = np.zeros(ncells, dtype=np.float64)
    scalars = np.zeros(3, dtype=np.float64)
    steps = np.zeros(1, dtype=np.uint64)
    rec = None
    args_rec = [0, 0, None, None, None, None, None]
    if n_record > 0:
        mv = int(max_visits or (grid.nx + grid.ny + grid.nz + 4))
        rec = {"cells": np.full((n_record, mv), -1, dtype=np.int32),
               "ds": np.zeros((n_record, mv), dtype=np.float32),
               "n": np.zeros(n_record, dtype=np.int32),
               "escaped": np.zeros(n_record, dtype=np.float64),
               "w": np.zeros(n_record, dtype=np.float64)}
        args_rec = [n_record, mv, _p(rec["cells"]), _p(rec["ds"]), _p(rec["n"]),
                    _p(rec["escaped"]), _p(rec["w"])]
    e = lib().oracle_trace(ct.byref(I.g), ct.byref(I.s), ct.byref(I.t), int(seed), int(enclosure),
                           int(ray_begin), int(n_rays), int(n_total), int(mode), int(bool(tau_cut)),
                           int(threads or default_threads()), _p(absorbed), _p(scalars),
                           _p(steps), *args_rec)
    if e != 0:
        raise RuntimeError(f"oracle_trace failed with code {e}")
    return TraceResult(absorbed, scalars, steps[0], rec)


def sample_rays(grid, spec, kappa, seed=0, ray_begin=0, n=16, n_total=None, mode=MODE_EMIT,
                columns=None, enclosure=0, per_cell=False):
    n_total = n if n_total is None else n_total
    I = _Inputs(grid, spec, kappa, columns, per_cell)
    cell = np.zeros(n, dtype=np.int64)
    j = np.zeros(n, dtype=np.int64)
    pos = np.zeros((n, 3), dtype=np.float32)
    dirs = np.zeros((n, 3), dtype=np.float32)
    w = np.zeros(n, dtype=np.float64)
    e = lib().oracle_sample_rays(ct.byref(I.g), ct.byref(I.s), ct.byref(I.t), int(seed),
                                 int(enclosure), int(ray_begin), int(n), int(n_total), int(mode),
                                 _p(cell), _p(j), _p(pos), _p(dirs), _p(w))
    if e != 0:
        raise RuntimeError(f"oracle_sample_rays failed with code {e}")
    return cell, j, pos, dirs, w


def walk_rays(grid, spec, kappa, ix3, pos, dirs, j, w, columns=None, per_cell=False):
    """Walk explicitly given rays; returns (absorbed per cell, escaped per ray)."""
    I = _Inputs(grid, spec, kappa, columns, per_cell)
    n = int(len(j))
    ix3 = np.ascontiguousarray(ix3, dtype=np.int32)
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    dirs = np.ascontiguousarray(dirs, dtype=np.float32)
    j = np.ascontiguousarray(j, dtype=np.int64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    absorbed = np.zeros(grid.nx * grid.ny * grid.nz, dtype=np.float64)
    esc = np.zeros(n, dtype=np.float64)
    e = lib().oracle_walk_rays(ct.byref(I.g), ct.byref(I.s), ct.byref(I.t), n, _p(ix3), _p(pos),
                               _p(dirs), _p(j), _p(w), _p(absorbed), _p(esc))
    if e != 0:
        raise RuntimeError(f"oracle_walk_rays failed with code {e}")
    return absorbed, esc


def cell_prep(grid, spec):
    I = _Inputs(grid, spec)
    n = grid.nx * grid.ny * grid.nz
    k = np.zeros(n, dtype=np.int32)
    fr = np.zeros(n, dtype=np.float32)
    sc = np.zeros(n, dtype=np.float32)
    e = lib().oracle_cell_prep(ct.byref(I.g), ct.byref(I.s), _p(k), _p(fr), _p(sc))
    if e != 0:
        raise RuntimeError("oracle_cell_prep failed")
    return k, fr, sc


def trace_case(case, ray_begin=0, n_rays=None, n_record=0, tau_cut=False, threads=None,
               kappa_fn=None):
    """Trace a ray subset of a workload with the oracle's own kappa columns.

    Only the columns the traced rays use are built (kappa_fn(lines, spec, js)
    -> (nT, len(js)) float64; default the oracle's Eq. tau sum).
    """
    from . import kappa as okappa
    n_rays = case.n_rays if n_rays is None else n_rays
    g = case.grid
    _, j = emission_indices(g.ncells, case.spec.n_nu, case.seed, ray_begin, n_rays)
    cols = np.unique(j)
    kfn = kappa_fn or okappa.kappa_columns
    K = kfn(case.lines, case.spec, cols)
    res = trace(g, case.spec, K, seed=case.seed, ray_begin=ray_begin, n_rays=n_rays,
                n_total=case.n_rays, columns=cols, tau_cut=tau_cut, n_record=n_record,
                threads=threads)
    res.columns = cols
    res.kappa = K
    return res


def march(grid, spec, kappa, pos, dirs, I_in=None, columns=None):
    """Eq. (I) marched per spectral sample along given rays (start position inside
    the grid, direction).  Returns (I_out (n, n_nu), power (n,) = sum_j (I_in - I_out) dnu)."""
    I = _Inputs(grid, spec, kappa, columns)
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    dirs = np.ascontiguousarray(dirs, dtype=np.float32)
    n = int(pos.shape[0])
    Iin = None if I_in is None else np.ascontiguousarray(I_in, dtype=np.float64)
    out = np.zeros((n, spec.n_nu), dtype=np.float64)
    pw = np.zeros(n, dtype=np.float64)
    e = lib().oracle_march(ct.byref(I.g), ct.byref(I.s), ct.byref(I.t), n, _p(pos), _p(dirs), _p(Iin),
                           _p(out), _p(pw))
    if e != 0:
        raise RuntimeError(f"oracle_march failed with code {e}")
    return out, pw
