"""GB300 (sm_103a) Monte-Carlo line-by-line radiative transfer.

Thin Python binding of the C ABI declared in ``include/rt.h`` (ctypes, the
same names: the kappa build, the walks, tallies, the surrogate network, the
batched walk, the spectral marching, launch shapes); the helpers below only
marshal arguments: every step of the computation runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.

The method follows Section 3 of Collange, Daumas and Defour, "Graphic
processors to speed-up simulations for the design of high performance solar
receptors": the absorption coefficient of a gas from its line list (Eqs. S,
tau) and Monte-Carlo rays traced through finite volumes with Beer-Lambert
attenuation (Eq. I) and Planck emission (Eq. planck).

There is no CPU fallback: if the CUDA library cannot be loaded, importing
this package raises.
"""
from __future__ import annotations

import ctypes as ct
import math
import os

from . import _build

__all__ = ["RtError", "lib", "rt_lines", "rt_spectral", "rt_grid", "rt_tally_buf", "rt_record",
           "make_lines", "make_spectral", "make_grid", "Tally", "Record", "build_kappa", "trace",
           "PROFILE", "RT_SRC_EMIT", "RT_SRC_BEAM", "RT_TAU_CUT", "RT_MEM_HOST", "RT_MEM_DEVICE"]

RT_OK, RT_E_INVAL, RT_E_NOMEM, RT_E_CUDA, RT_E_STEPCAP, RT_E_TIMEOUT, RT_E_UNSORTED, RT_E_NONFINITE = range(8)
STATUS_NAMES = {0: "RT_OK", 1: "RT_E_INVAL", 2: "RT_E_NOMEM", 3: "RT_E_CUDA", 4: "RT_E_STEPCAP",
                5: "RT_E_TIMEOUT", 6: "RT_E_UNSORTED", 7: "RT_E_NONFINITE"}
PROFILE = {"lorentz": 0, "voigt": 1}
RT_MEM_HOST, RT_MEM_DEVICE = 0, 1
RT_SRC_EMIT, RT_SRC_BEAM, RT_TAU_CUT, RT_COUNT_EVALS = 0, 1, 1 << 4, 1 << 5


class RtError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


class rt_lines(ct.Structure):
    _fields_ = [("n", ct.c_int64), ("nu0", ct.c_void_p), ("S_ref", ct.c_void_p),
                ("gamma_ref", ct.c_void_p), ("E_lower", ct.c_void_p), ("T_ref", ct.c_double),
                ("n_T", ct.c_double), ("q_exp", ct.c_double), ("mass_amu", ct.c_double),
                ("memory", ct.c_int32), ("pad", ct.c_int32)]


class rt_spectral(ct.Structure):
    _fields_ = [("nu_min", ct.c_double), ("dnu", ct.c_double), ("n_nu", ct.c_int64),
                ("cutoff", ct.c_double), ("profile", ct.c_int32), ("nT", ct.c_int32),
                ("T_min", ct.c_double), ("T_max", ct.c_double), ("p_ref_atm", ct.c_double),
                ("x_ref", ct.c_double), ("points_per_line", ct.c_int32), ("accumulate", ct.c_int32),
                ("kappa_min", ct.c_double)]


class rt_grid(ct.Structure):
    _fields_ = [("nx", ct.c_int32), ("ny", ct.c_int32), ("nz", ct.c_int32), ("pad", ct.c_int32),
                ("hx", ct.c_double), ("hy", ct.c_double), ("hz", ct.c_double),
                ("T", ct.c_void_p), ("p_atm", ct.c_void_p), ("x", ct.c_void_p)]


class rt_tally_buf(ct.Structure):
    _fields_ = [("absorbed", ct.c_void_p), ("scalars", ct.c_void_p), ("steps", ct.c_void_p),
                ("status", ct.c_void_p)]


class rt_record(ct.Structure):
    _fields_ = [("n_rays", ct.c_int64), ("max_visits", ct.c_int32), ("pad", ct.c_int32),
                ("cells", ct.c_void_p), ("ds", ct.c_void_p), ("n_visits", ct.c_void_p),
                ("weight", ct.c_void_p), ("escaped", ct.c_void_p)]


_P = ct.c_void_p
_SIGNATURES = {
    "rt_version": ([], ct.c_char_p),
    "rt_last_error": ([], ct.c_char_p),
    "rt_kappa_table_elems": ([_P], ct.c_size_t),
    "rt_build_kappa": ([_P, _P, _P, _P, _P, _P], ct.c_int),
    "rt_build_kappa_static": ([_P, _P, _P, _P, _P, _P], ct.c_int),
    "rt_trace": ([_P, _P, _P, ct.c_uint64, ct.c_uint64, ct.c_uint64, ct.c_uint64, ct.c_uint32,
                  ct.c_int32, _P, _P, _P], ct.c_int),
    "rt_tally_zero": ([_P, ct.c_int64, _P], ct.c_int),
    "rt_tally": ([_P, ct.c_int64, _P, _P, _P], ct.c_int),
    "rt_status_read": ([_P, _P], ct.c_int),
    "rt_mlp_forward": ([_P, _P, _P, ct.c_int64, _P, _P, _P], ct.c_int),
    "rt_mlp_train_step": ([_P, _P, _P, _P, _P, _P, ct.c_int64, _P, ct.c_float, ct.c_int32, ct.c_int32,
                           _P, _P, _P], ct.c_int),
    "rt_mlp_train_steps": ([_P, _P, _P, _P, _P, _P, ct.c_int64, ct.c_int64, _P, ct.c_double, ct.c_double,
                            ct.c_int32, ct.c_int32, ct.c_int32, _P, _P, _P], ct.c_int),
    "rt_tc_selftest": ([_P, _P, _P, _P, _P], ct.c_int),
    "rt_tc_selftest_mn": ([_P, _P, _P, _P, _P], ct.c_int),
    "rt_alu_probe": ([_P, _P], ct.c_int),
    "rt_wait_probe": ([ct.c_uint32, ct.c_int32, _P, _P], ct.c_int),
    "rt_trace_mlp": ([_P, _P, _P, _P, ct.c_uint64, ct.c_uint64, ct.c_uint64, ct.c_uint64, ct.c_uint32,
                      ct.c_int32, _P, _P, _P], ct.c_int),
    "rt_mlp_make_samples": ([_P, ct.c_int32, _P, _P, ct.c_float, ct.c_float, ct.c_uint64, ct.c_int64,
                             _P, _P, _P], ct.c_int),
    "rt_mlp_make_samples_bands": ([_P, ct.c_int32, _P, _P, ct.c_int32, ct.c_float, ct.c_float, ct.c_float,
                                   ct.c_uint64, ct.c_int64, _P, _P, _P], ct.c_int),
    "rt_mlp_train_steps_nets": ([ct.c_int32, _P, _P, _P, _P, _P, _P, ct.c_int64, ct.c_int64, _P, ct.c_double,
                                 ct.c_double, ct.c_int32, ct.c_int32, ct.c_int32, _P, _P, _P], ct.c_int),
    "rt_mlp_forward_nets": ([ct.c_int32, _P, _P, _P, ct.c_int64, _P, _P, _P], ct.c_int),
    "rt_trace_mlp_bands": ([_P, ct.c_int32, _P, _P, _P, ct.c_uint64, ct.c_uint64, ct.c_uint64, ct.c_uint64,
                            ct.c_uint32, ct.c_int32, _P, _P, _P], ct.c_int),
    "rt_trace_lbl": ([_P, _P, _P, ct.c_uint64, ct.c_uint64, ct.c_uint64, ct.c_uint64, ct.c_uint32,
                      ct.c_int32, _P, _P, _P], ct.c_int),
    "rt_batch_create": ([ct.c_int32, _P, _P, ct.c_uint64, ct.c_int32, _P, _P], ct.c_int),
    "rt_batch_trace": ([_P, _P, _P], ct.c_int),
    "rt_batch_destroy": ([_P], ct.c_int),
    "rt_trace_batch": ([ct.c_int32, _P, _P, _P, ct.c_uint64, ct.c_int32, _P, _P], ct.c_int),
    "rt_march": ([_P, _P, _P, ct.c_int64, _P, _P, _P, _P, _P, _P, _P, _P], ct.c_int),
    "rt_set_tuning": ([_P], ct.c_int),
    "rt_get_tuning": ([_P], ct.c_int),
}


class rt_mlp_norm(ct.Structure):
    _fields_ = [("in_lo", ct.c_float * 4), ("in_hi", ct.c_float * 4), ("out_mean", ct.c_float),
                ("out_scale", ct.c_float)]


RT_MLP_NPARAM = 50305
RT_MLP_GRAD_ONLY = 1

_lib = None


def lib():
    """Load (building first if needed) the CUDA library; raises if it cannot."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path) or os.environ.get("RT_GB300_AUTOBUILD", "1") == "1":
            path = _build.build()
        L = ct.CDLL(path)
        for name, (args, res) in _SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(st: int, where: str):
    if st != RT_OK:
        raise RtError(st, where, lib().rt_last_error().decode())


def __getattr__(name):  # rt_* entry points by their C names
    if name in _SIGNATURES:
        return getattr(lib(), name)
    raise AttributeError(name)


def _ptr(t):
    return None if t is None else ct.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ct.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------- marshalling
def make_lines(lines, memory: str = "host"):
    """rt_lines from an object with nu0, S_ref, gamma_ref, E_lower (float64 arrays)
    and T_ref, n_T, q_exp, mass_amu.  memory='host' keeps numpy arrays;
    'device' copies them to CUDA tensors.  Returns (struct, keepalive)."""
    import numpy as np
    arrs = [np.ascontiguousarray(getattr(lines, k), dtype=np.float64)
            for k in ("nu0", "S_ref", "gamma_ref", "E_lower")]
    n = int(arrs[0].shape[0])
    if memory == "device":
        import torch
        keep = [torch.from_numpy(a).cuda() for a in arrs]
        ptrs = [k.data_ptr() if n else None for k in keep]
        mem = RT_MEM_DEVICE
    else:
        keep = arrs
        ptrs = [a.ctypes.data if n else None for a in arrs]
        mem = RT_MEM_HOST
    s = rt_lines(n, *ptrs, float(lines.T_ref), float(lines.n_T), float(lines.q_exp),
                 float(lines.mass_amu), mem, 0)
    return s, keep


def make_spectral(spec) -> rt_spectral:
    return rt_spectral(float(spec.nu_min), float(spec.dnu), int(spec.n_nu), float(spec.cutoff),
                       PROFILE[spec.profile] if isinstance(spec.profile, str) else int(spec.profile),
                       int(spec.nT), float(spec.T_min), float(spec.T_max), float(spec.p_ref_atm),
                       float(spec.x_ref), int(getattr(spec, "points_per_line", 0)),
                       int(getattr(spec, "accumulate", 0)), float(getattr(spec, "kappa_min", 0.0)))


def make_grid(grid, device="cuda"):
    """rt_grid with the fields copied to CUDA float32 tensors. Returns (struct, keepalive)."""
    import torch

    def dev(a):
        if a is None:
            return None
        t = a if isinstance(a, torch.Tensor) else torch.from_numpy(a)
        return t.to(device=device, dtype=torch.float32).contiguous()

    T, p, x = dev(grid.T), dev(grid.p_atm), dev(grid.x)
    s = rt_grid(int(grid.nx), int(grid.ny), int(grid.nz), 0, float(grid.hx), float(grid.hy),
                float(grid.hz), T.data_ptr(), None if p is None else p.data_ptr(),
                None if x is None else x.data_ptr())
    return s, (T, p, x)


class Tally:
    """Device tally buffers (caller-owned torch tensors) of a grid of ncells cells.

    ``absorbed`` and ``scalars`` are views of one binary64 buffer ``flat`` =
    [absorbed[ncells] | emitted, absorbed total, escaped, residual], so that ranks
    that traced disjoint ray ranges combine their tallies with one all-reduce
    (``shard.combine_tally``)."""

    def __init__(self, ncells: int, device="cuda", counters: int = 1):
        import torch
        self.ncells = int(ncells)
        self.flat = torch.zeros(self.ncells + 4, dtype=torch.float64, device=device)
        self.absorbed = self.flat[:self.ncells]
        self.scalars = self.flat[self.ncells:]
        # [ray-cell steps] or, counters = 2 for a surrogate walk with RT_COUNT_EVALS,
        # [ray-cell steps, network evaluations]
        self.steps = torch.zeros(int(counters), dtype=torch.int64, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.buf = rt_tally_buf(self.absorbed.data_ptr(), self.scalars.data_ptr(),
                                self.steps.data_ptr(), self.status.data_ptr())

    def zero(self, stream=None):
        _check(lib().rt_tally_zero(ct.byref(self.buf), self.ncells, _stream_ptr(stream)), "rt_tally_zero")
        if self.steps.numel() > 1:  # the evaluation counter (rt_tally_zero clears steps[0])
            self.steps[1:].zero_()

    def read(self, stream=None, absorbed=True, check=True):
        """rt_tally: returns (absorbed float64 numpy or None, scalars[4], status)."""
        import numpy as np
        sc = np.zeros(4, dtype=np.float64)
        ab = np.zeros(self.ncells, dtype=np.float64) if absorbed else None
        st = lib().rt_tally(ct.byref(self.buf), self.ncells,
                            None if ab is None else ab.ctypes.data, sc.ctypes.data, _stream_ptr(stream))
        if check:
            _check(st, "rt_tally")
        return ab, sc, st


class Record:
    """Optional per-ray record buffers for the first n rays of a trace call."""

    def __init__(self, n: int, max_visits: int, device="cuda"):
        import torch
        self.n, self.max_visits = int(n), int(max_visits)
        self.cells = torch.full((self.n, self.max_visits), -1, dtype=torch.int32, device=device)
        self.ds = torch.zeros((self.n, self.max_visits), dtype=torch.float32, device=device)
        self.n_visits = torch.zeros(self.n, dtype=torch.int32, device=device)
        self.weight = torch.zeros(self.n, dtype=torch.float32, device=device)
        self.escaped = torch.zeros(self.n, dtype=torch.float32, device=device)
        self.buf = rt_record(self.n, self.max_visits, 0, self.cells.data_ptr(), self.ds.data_ptr(),
                             self.n_visits.data_ptr(), self.weight.data_ptr(), self.escaped.data_ptr())


def build_kappa(lines, spec, out=None, stream=None, memory="host", evals=None, status=None):
    """Run rt_build_kappa; returns the (nT, n_nu) float32 CUDA tensor."""
    import torch
    S = make_spectral(spec)
    L, keep = make_lines(lines, memory)
    if out is None:
        out = torch.empty((int(spec.nT), int(spec.n_nu)), dtype=torch.float32, device="cuda")
    st = lib().rt_build_kappa(ct.byref(L), ct.byref(S), _ptr(out), _ptr(evals), _ptr(status),
                              _stream_ptr(stream))
    _check(st, "rt_build_kappa")
    if memory == "host":
        # host arrays are read by the call's copies before it returns
        pass
    out._rt_keep = keep
    return out


def trace(grid_struct, kappa, spec, tally: Tally, n_rays: int, ray_begin: int = 0,
          n_rays_total: int | None = None, seed: int = 0, enclosure: int = 0, flags: int = 0,
          record: Record | None = None, stream=None):
    """Run rt_trace (asynchronous); accumulates into ``tally``."""
    S = make_spectral(spec)
    st = lib().rt_trace(ct.byref(grid_struct), _ptr(kappa), ct.byref(S), int(ray_begin), int(n_rays),
                        int(n_rays_total if n_rays_total is not None else n_rays), int(seed),
                        int(enclosure), int(flags), ct.byref(tally.buf),
                        None if record is None else ct.byref(record.buf), _stream_ptr(stream))
    _check(st, "rt_trace")


# ---------------------------------------------------------------- surrogate network
def make_norm(in_lo, in_hi, out_mean, out_scale) -> "rt_mlp_norm":
    n = rt_mlp_norm()
    for i in range(4):
        n.in_lo[i] = float(in_lo[i])
        n.in_hi[i] = float(in_hi[i])
    n.out_mean = float(out_mean)
    n.out_scale = float(out_scale)
    return n


def mlp_forward(params, norm, inputs, out=None, stream=None):
    """rt_mlp_forward on CUDA tensors: params [RT_MLP_NPARAM], inputs [n, 4] -> log kappa [n]."""
    import torch
    n = int(inputs.shape[0])
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=inputs.device)
    st = lib().rt_mlp_forward(_ptr(params), ct.byref(norm), _ptr(inputs), n, _ptr(out), None,
                              _stream_ptr(stream))
    _check(st, "rt_mlp_forward")
    return out


class MlpTrainer:
    """Parameters, Adam moments, gradient and loss buffers (CUDA tensors)."""

    def __init__(self, params, norm):
        import torch
        self.params = params
        self.norm = norm
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.grad = torch.zeros_like(params)
        self.loss = torch.zeros(1, dtype=torch.float32, device=params.device)
        self.status = torch.zeros(1, dtype=torch.int32, device=params.device)
        self.step_no = 0

    def step(self, inputs, targets, lr, grad_only=False, stream=None):
        if not grad_only:
            self.step_no += 1
        st = lib().rt_mlp_train_step(_ptr(self.params), _ptr(self.m), _ptr(self.v), _ptr(self.grad),
                                     _ptr(inputs), _ptr(targets), int(inputs.shape[0]),
                                     ct.byref(self.norm), float(lr), max(1, self.step_no),
                                     RT_MLP_GRAD_ONLY if grad_only else 0, _ptr(self.loss),
                                     _ptr(self.status), _stream_ptr(stream))
        _check(st, "rt_mlp_train_step")
        return self.loss

    def steps(self, inputs, targets, batch, lr0, lr1, step_first, n_steps, total_steps, losses=None,
              stream=None):
        """rt_mlp_train_steps: n_steps Adam steps over consecutive batches with the cosine
        learning rate from lr0 to lr1 over total_steps; losses (optional float32 CUDA
        tensor [n_steps]) receives each step's loss."""
        st = lib().rt_mlp_train_steps(_ptr(self.params), _ptr(self.m), _ptr(self.v), _ptr(self.grad),
                                      _ptr(inputs), _ptr(targets), int(inputs.shape[0]), int(batch),
                                      ct.byref(self.norm), float(lr0), float(lr1), int(step_first),
                                      int(n_steps), int(total_steps), _ptr(losses), _ptr(self.status),
                                      _stream_ptr(stream))
        _check(st, "rt_mlp_train_steps")
        self.step_no = int(step_first) - 1 + int(n_steps)


def _check_eval_counter(tally, flags):
    # RT_COUNT_EVALS makes the library write a second steps counter
    if (int(flags) & RT_COUNT_EVALS) and tally.steps.numel() < 2:
        raise RtError(RT_E_INVAL, "trace_mlp", "RT_COUNT_EVALS needs a Tally with counters=2")


def trace_mlp(grid_struct, params, norm, spec, tally: Tally, n_rays: int, ray_begin: int = 0,
              n_rays_total: int | None = None, seed: int = 0, enclosure: int = 0, flags: int = 0,
              record: Record | None = None, stream=None):
    """Run rt_trace_mlp (asynchronous); accumulates into ``tally``."""
    _check_eval_counter(tally, flags)
    S = make_spectral(spec)
    st = lib().rt_trace_mlp(ct.byref(grid_struct), _ptr(params), ct.byref(norm), ct.byref(S),
                            int(ray_begin), int(n_rays),
                            int(n_rays_total if n_rays_total is not None else n_rays), int(seed),
                            int(enclosure), int(flags), ct.byref(tally.buf),
                            None if record is None else ct.byref(record.buf), _stream_ptr(stream))
    _check(st, "rt_trace_mlp")


def norms_tensor(in_lo, in_hi, out_mean, out_scale, device="cuda"):
    """Device array of rt_mlp_norm for an ensemble: in_lo, in_hi (n, 4), out_mean,
    out_scale (n,), any array-likes (torch or numpy); returns float32 [n, 10]."""
    import torch

    def t(a):
        return torch.as_tensor(a, dtype=torch.float32).to(device)
    lo, hi = t(in_lo).reshape(-1, 4), t(in_hi).reshape(-1, 4)
    return torch.cat([lo, hi, t(out_mean).reshape(-1, 1), t(out_scale).reshape(-1, 1)], 1).contiguous()


def mlp_forward_nets(params, norms, inputs, out=None, stream=None):
    """rt_mlp_forward_nets: params [n_nets * RT_MLP_NPARAM], norms [n_nets, 10] (device),
    inputs [n_nets, n, 4] -> log kappa [n_nets, n]."""
    import torch
    nn_, n = int(inputs.shape[0]), int(inputs.shape[1])
    if out is None:
        out = torch.empty((nn_, n), dtype=torch.float32, device=inputs.device)
    _check(lib().rt_mlp_forward_nets(nn_, _ptr(params), _ptr(norms), _ptr(inputs), n, _ptr(out), None,
                                     _stream_ptr(stream)), "rt_mlp_forward_nets")
    return out


class MlpEnsembleTrainer:
    """Parameters, Adam moments and gradients of n_nets networks (CUDA tensors
    [n_nets * RT_MLP_NPARAM]) with their device norms [n_nets, 10]."""

    def __init__(self, params, norms):
        import torch
        self.params = params
        self.norms = norms
        self.n_nets = int(norms.shape[0])
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.grad = torch.zeros_like(params)
        self.status = torch.zeros(1, dtype=torch.int32, device=params.device)

    def steps(self, inputs, targets, batch, lr0, lr1, step_first, n_steps, total_steps, losses=None,
              stream=None):
        """rt_mlp_train_steps_nets over inputs [n_nets, n, 4], targets [n_nets, n]."""
        n = int(targets.shape[1])
        st = lib().rt_mlp_train_steps_nets(self.n_nets, _ptr(self.params), _ptr(self.m), _ptr(self.v),
                                           _ptr(self.grad), _ptr(inputs), _ptr(targets), n, int(batch),
                                           _ptr(self.norms), float(lr0), float(lr1), int(step_first),
                                           int(n_steps), int(total_steps), _ptr(losses), _ptr(self.status),
                                           _stream_ptr(stream))
        _check(st, "rt_mlp_train_steps_nets")


def mlp_make_samples_bands(tables, p_nodes, spec, band_pts, x_lo, x_hi, seed, n_per_band, stream=None,
                           emission_mix=0.0):
    """rt_mlp_make_samples_bands: (inputs [n_bands, n, 4], targets [n_bands, n]) CUDA tensors."""
    import torch
    nb = -(-int(spec.n_nu) // int(band_pts))
    inputs = torch.empty((nb, n_per_band, 4), dtype=torch.float32, device=tables.device)
    targets = torch.empty((nb, n_per_band), dtype=torch.float32, device=tables.device)
    S = make_spectral(spec)
    st = lib().rt_mlp_make_samples_bands(_ptr(tables), int(p_nodes.shape[0]), _ptr(p_nodes), ct.byref(S),
                                         int(band_pts), float(x_lo), float(x_hi), float(emission_mix), int(seed),
                                         int(n_per_band),
                                         _ptr(inputs), _ptr(targets), _stream_ptr(stream))
    _check(st, "rt_mlp_make_samples_bands")
    return inputs, targets


def trace_mlp_bands(grid_struct, band_pts, params, norms, spec, tally: Tally, n_rays: int, ray_begin: int = 0,
                    n_rays_total: int | None = None, seed: int = 0, enclosure: int = 0, flags: int = 0,
                    record: Record | None = None, stream=None):
    """Run rt_trace_mlp_bands (asynchronous); accumulates into ``tally``."""
    _check_eval_counter(tally, flags)
    S = make_spectral(spec)
    st = lib().rt_trace_mlp_bands(ct.byref(grid_struct), int(band_pts), _ptr(params), _ptr(norms), ct.byref(S),
                                  int(ray_begin), int(n_rays),
                                  int(n_rays_total if n_rays_total is not None else n_rays), int(seed),
                                  int(enclosure), int(flags), ct.byref(tally.buf),
                                  None if record is None else ct.byref(record.buf), _stream_ptr(stream))
    _check(st, "rt_trace_mlp_bands")


def trace_lbl(grid_struct, lines, spec, tally: Tally, n_rays: int, ray_begin: int = 0,
              n_rays_total: int | None = None, seed: int = 0, enclosure: int = 0, flags: int = 0,
              record: Record | None = None, stream=None, memory="host"):
    """Run rt_trace_lbl (asynchronous); accumulates into ``tally``."""
    S = make_spectral(spec)
    L, keep = make_lines(lines, memory)
    st = lib().rt_trace_lbl(ct.byref(grid_struct), ct.byref(L), ct.byref(S), int(ray_begin), int(n_rays),
                            int(n_rays_total if n_rays_total is not None else n_rays), int(seed),
                            int(enclosure), int(flags), ct.byref(tally.buf),
                            None if record is None else ct.byref(record.buf), _stream_ptr(stream))
    _check(st, "rt_trace_lbl")
    return keep


def mlp_make_samples(tables, p_nodes, spec, x_lo, x_hi, seed, n, stream=None):
    """rt_mlp_make_samples: (inputs [n, 4], targets [n]) CUDA tensors."""
    import torch
    inputs = torch.empty((n, 4), dtype=torch.float32, device=tables.device)
    targets = torch.empty(n, dtype=torch.float32, device=tables.device)
    S = make_spectral(spec)
    st = lib().rt_mlp_make_samples(_ptr(tables), int(p_nodes.shape[0]), _ptr(p_nodes), ct.byref(S),
                                   float(x_lo), float(x_hi), int(seed), int(n), _ptr(inputs),
                                   _ptr(targets), _stream_ptr(stream))
    _check(st, "rt_mlp_make_samples")
    return inputs, targets


class rt_enclosure(ct.Structure):
    _fields_ = [("grid", rt_grid), ("n_rays", ct.c_uint64), ("tally", rt_tally_buf)]


class rt_batch_opts(ct.Structure):
    _fields_ = [("rays_per_item", ct.c_int32), ("threads", ct.c_int32)]


class rt_tuning(ct.Structure):
    _fields_ = [("kappa_t_per_block", ct.c_int32), ("walk_blocks_per_sm", ct.c_int32),
                ("walk_refill_idle", ct.c_int32), ("walk_group", ct.c_int32), ("reserved", ct.c_int32 * 4)]


_TUNING_FIELDS = ("kappa_t_per_block", "walk_blocks_per_sm", "walk_refill_idle", "walk_group")


def set_tuning(**shapes):
    """Set process-wide launch shapes by field name (rt_tuning); others keep their value."""
    t = rt_tuning()
    _check(lib().rt_get_tuning(ct.byref(t)), "rt_get_tuning")
    for k, v in shapes.items():
        if k not in _TUNING_FIELDS:
            raise TypeError(f"unknown tuning field {k!r}")
        if v is not None:
            setattr(t, k, int(v))
    _check(lib().rt_set_tuning(ct.byref(t)), "rt_set_tuning")


def get_tuning() -> dict:
    t = rt_tuning()
    _check(lib().rt_get_tuning(ct.byref(t)), "rt_get_tuning")
    return {k: getattr(t, k) for k in _TUNING_FIELDS}


class Batch:
    """A plan over many enclosures: grids (synth.Grid-like), ray counts, one Tally each."""

    def __init__(self, grids, n_rays, spec, seed=0, flags=0, rays_per_item=0, threads=0):
        self.grids = [make_grid(g) for g in grids]
        self.tallies = [Tally(g.ncells) for g in grids]
        for t in self.tallies:
            t.zero()
        arr = (rt_enclosure * len(grids))()
        for i, ((gs, _), t, n) in enumerate(zip(self.grids, self.tallies, n_rays)):
            arr[i].grid = gs
            arr[i].n_rays = int(n)
            arr[i].tally = t.buf
        self.encl = arr
        self.spec = make_spectral(spec)
        self.opts = rt_batch_opts(int(rays_per_item), int(threads))
        self.plan = ct.c_void_p()
        _check(lib().rt_batch_create(len(grids), arr, ct.byref(self.spec), int(seed), int(flags),
                                     ct.byref(self.opts), ct.byref(self.plan)), "rt_batch_create")

    def trace(self, kappa, stream=None):
        _check(lib().rt_batch_trace(self.plan, _ptr(kappa), _stream_ptr(stream)), "rt_batch_trace")

    def zero(self, stream=None):
        for t in self.tallies:
            t.zero(stream)

    def close(self):
        if self.plan:
            lib().rt_batch_destroy(self.plan)
            self.plan = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def march(grid_struct, kappa, spec, pos, dirs, I_in=None, want_I=True, nvis=None, stream=None):
    """rt_march on CUDA tensors pos, dirs [n, 3]; returns (I_out [n, n_nu] or None, power [n]).
    ``nvis`` (optional int32 CUDA tensor [n]) receives the number of cells each path crosses."""
    import torch
    n = int(pos.shape[0])
    S = make_spectral(spec)
    I_out = torch.empty((n, int(spec.n_nu)), dtype=torch.float32, device="cuda") if want_I else None
    power = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = lib().rt_march(ct.byref(grid_struct), _ptr(kappa), ct.byref(S), n, _ptr(pos), _ptr(dirs),
                        _ptr(I_in), _ptr(I_out), _ptr(power), _ptr(nvis), None, _stream_ptr(stream))
    _check(st, "rt_march")
    return I_out, power


def alu_probe(stream=None) -> dict:
    """rt_alu_probe: measured binary32 FMA and MUFU reciprocal lane operations per second."""
    import numpy as np
    out = np.zeros(2, dtype=np.float64)
    _check(lib().rt_alu_probe(out.ctypes.data, _stream_ptr(stream)), "rt_alu_probe")
    return {"fma_lane_ops_per_s": float(out[0]), "rcp_lane_ops_per_s": float(out[1])}
