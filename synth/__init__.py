"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws and lays out inputs: line lists, spectral windows,
finite-volume grids with T / p / x fields, and the five workload recipes.
It holds none of the method's arithmetic (no line strengths at temperature,
no profiles, no optical depths), so both the CPU oracle and the CUDA path
can take their inputs from it without sharing any computation.

The paper's own inputs (HITRAN-class CO2/H2O line lists and the solar
receptor geometry of Section 3) are not available; these generators stand in
for them with the shapes of the paper's workload: a few hundred to 1e5 lines
in the 4.3 um band, 1e4..4e5 spectral samples, grids of finite volumes with
smooth temperature fields, and up to 1e9 Monte-Carlo rays.

Layout conventions (shared with the C-ABI):
  * line arrays are float64, sorted by ascending centre nu0 [cm^-1];
  * spectral grid nu_j = nu_min + j * dnu for j = 0 .. n_nu-1 (nu_max excluded);
  * temperature grid T_k = T_min + k * (T_max - T_min) / (nT - 1), k = 0 .. nT-1
    (nT = 1 means a single isothermal row at T_min);
  * fields are float32 arrays of ncells = nx*ny*nz values, x fastest
    (flat index = ix + nx * (iy + ny * iz));
  * an infinite cell size (hy = hz = inf) makes a plane-parallel slab.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

__all__ = [
    "Lines", "Spectral", "Grid", "Case", "make_lines", "uniform_grid",
    "gaussian_hotspot_grid", "multi_gaussian_grid", "config", "CONFIG_NAMES",
    "batched_enclosures", "rng_for",
]


@dataclass
class Lines:
    """Spectral line list (float64, sorted by nu0)."""
    nu0: np.ndarray          # line centre [cm^-1]
    S_ref: np.ndarray        # intensity at T_ref [cm / molecule]
    gamma_ref: np.ndarray    # Lorentz half-width at T_ref and 1 atm [cm^-1]
    E_lower: np.ndarray      # lower-state energy [cm^-1]
    T_ref: float = 296.0     # reference temperature [K]
    n_T: float = 0.75        # temperature exponent of the Lorentz width
    q_exp: float = 1.0       # partition-function exponent, Q ~ T^q_exp
    mass_amu: float = 44.0   # absorber molecular mass [u] (CO2)

    @property
    def n(self) -> int:
        return int(self.nu0.shape[0])

    def subset(self, idx) -> "Lines":
        return replace(self, nu0=self.nu0[idx].copy(), S_ref=self.S_ref[idx].copy(),
                       gamma_ref=self.gamma_ref[idx].copy(), E_lower=self.E_lower[idx].copy())


@dataclass
class Spectral:
    """Spectral window, profile choice and temperature grid of the kappa table."""
    nu_min: float
    dnu: float
    n_nu: int
    cutoff: float = 25.0
    profile: str = "voigt"   # "lorentz" | "voigt"
    nT: int = 1
    T_min: float = 296.0
    T_max: float = 296.0
    p_ref_atm: float = 1.0   # table pressure [atm]
    x_ref: float = 0.1       # table absorber mole fraction
    points_per_line: int = 0  # > 0: fixed number of grid points per line instead of the cutoff
    accumulate: int = 0       # add into an existing table (one build per absorbing gas)
    kappa_min: float = 0.0    # > 0: adaptive points per line, each line evaluated where its wing >= kappa_min

    @property
    def nu_max(self) -> float:
        return self.nu_min + self.n_nu * self.dnu

    def T_nodes(self) -> np.ndarray:
        if self.nT == 1:
            return np.array([self.T_min], dtype=np.float64)
        k = np.arange(self.nT, dtype=np.float64)
        return self.T_min + k * ((self.T_max - self.T_min) / (self.nT - 1))


@dataclass
class Grid:
    """Finite-volume grid with cell-constant fields (float32, x fastest)."""
    nx: int
    ny: int
    nz: int
    hx: float
    hy: float
    hz: float
    T: np.ndarray
    p_atm: Optional[np.ndarray] = None
    x: Optional[np.ndarray] = None

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz


@dataclass
class Case:
    """One workload: a line list, a spectral spec, a grid and a ray budget."""
    name: str
    lines: Lines
    spec: Spectral
    grid: Grid
    n_rays: int
    seed: int = 0
    extra: dict = field(default_factory=dict)


def rng_for(config_index: int, stream: int = 0) -> np.random.Generator:
    """Data seed 0 with the config index (and a stream number) as sub-seed."""
    return np.random.default_rng([0, int(config_index), int(stream)])


def make_lines(n: int, nu_lo: float, nu_hi: float, rng: np.random.Generator,
               S_lo: float = 1e-22, S_hi: float = 1e-19,
               g_lo: float = 0.05, g_hi: float = 0.1,
               E_hi: float = 5000.0) -> Lines:
    """n synthetic lines: centres U[nu_lo, nu_hi), S log-uniform, widths and
    lower-state energies uniform; returned sorted by centre."""
    nu0 = rng.uniform(nu_lo, nu_hi, n)
    S = np.exp(rng.uniform(math.log(S_lo), math.log(S_hi), n))
    g = rng.uniform(g_lo, g_hi, n)
    E = rng.uniform(0.0, E_hi, n)
    order = np.argsort(nu0, kind="stable")
    return Lines(nu0=nu0[order].copy(), S_ref=S[order].copy(),
                 gamma_ref=g[order].copy(), E_lower=E[order].copy())


def _centres(n: int, h: float) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) * h


def uniform_grid(nx, ny, nz, hx, hy, hz, T, p_atm=None, x=None) -> Grid:
    n = nx * ny * nz
    Tf = np.full(n, T, dtype=np.float32)
    pf = None if p_atm is None else np.full(n, p_atm, dtype=np.float32)
    xf = None if x is None else np.full(n, x, dtype=np.float32)
    return Grid(nx, ny, nz, hx, hy, hz, Tf, pf, xf)


def _mesh(nx, ny, nz, h):
    zc, yc, xc = np.meshgrid(_centres(nz, h), _centres(ny, h), _centres(nx, h), indexing="ij")
    return xc, yc, zc


def gaussian_hotspot_grid(n: int, side: float, T_lo: float, T_hi: float, sigma: float,
                          centre=None, p_atm: float = 1.0, x: float = 0.1,
                          dims=None) -> Grid:
    """Cubic (or dims-shaped) box with T = T_lo + (T_hi - T_lo) exp(-|r - r_c|^2 / 2 sigma^2)."""
    nx, ny, nz = dims if dims is not None else (n, n, n)
    h = side / n
    xc, yc, zc = _mesh(nx, ny, nz, h)
    if centre is None:
        centre = (0.5 * nx * h, 0.5 * ny * h, 0.5 * nz * h)
    r2 = (xc - centre[0]) ** 2 + (yc - centre[1]) ** 2 + (zc - centre[2]) ** 2
    T = T_lo + (T_hi - T_lo) * np.exp(-r2 / (2.0 * sigma * sigma))
    ncell = nx * ny * nz
    return Grid(nx, ny, nz, h, h, h, T.astype(np.float32).reshape(ncell),
                np.full(ncell, p_atm, dtype=np.float32), np.full(ncell, x, dtype=np.float32))


def _norm(v: np.ndarray) -> np.ndarray:
    lo, hi = float(v.min()), float(v.max())
    return (v - lo) / (hi - lo) if hi > lo else np.zeros_like(v)


def _gauss_sum(xc, yc, zc, rng, k, side, s_lo, s_hi):
    acc = np.zeros_like(xc)
    for _ in range(k):
        c = rng.uniform(0.0, side, 3)
        s = rng.uniform(s_lo, s_hi)
        acc += np.exp(-((xc - c[0]) ** 2 + (yc - c[1]) ** 2 + (zc - c[2]) ** 2) / (2 * s * s))
    return acc


def multi_gaussian_grid(n: int, side: float, rng: np.random.Generator,
                        T_lo=500.0, T_hi=2500.0, p_lo=1.0, p_hi=3.0, x=0.1) -> Grid:
    """Random smooth fields: T from a normalised sum of 8 Gaussians, p from 4."""
    h = side / n
    xc, yc, zc = _mesh(n, n, n, h)
    T = T_lo + (T_hi - T_lo) * _norm(_gauss_sum(xc, yc, zc, rng, 8, side, 0.05, 0.3))
    p = p_lo + (p_hi - p_lo) * _norm(_gauss_sum(xc, yc, zc, rng, 4, side, 0.05, 0.3))
    nc = n ** 3
    return Grid(n, n, n, h, h, h, T.astype(np.float32).reshape(nc),
                p.astype(np.float32).reshape(nc), np.full(nc, x, dtype=np.float32))


def batched_enclosures(n_encl: int, rng: np.random.Generator, side_lo=8, side_hi=48,
                       h=1.0 / 32, T_lo=600.0, T_hi=2000.0, rays_per_cell=1000):
    """Independent enclosures with uneven sizes and random Gaussian hot spots."""
    out = []
    for _ in range(n_encl):
        nx, ny, nz = (int(v) for v in rng.integers(side_lo, side_hi + 1, 3))
        dims_len = np.array([nx, ny, nz], dtype=np.float64) * h
        c = rng.uniform(0.0, 1.0, 3) * dims_len
        sig = rng.uniform(0.1, 0.3) * float(dims_len.mean())
        xc, yc, zc = _mesh(nx, ny, nz, h)
        r2 = (xc - c[0]) ** 2 + (yc - c[1]) ** 2 + (zc - c[2]) ** 2
        T = T_lo + (T_hi - T_lo) * np.exp(-r2 / (2 * sig * sig))
        nc = nx * ny * nz
        g = Grid(nx, ny, nz, h, h, h, T.astype(np.float32).reshape(nc),
                 np.full(nc, 1.0, dtype=np.float32), np.full(nc, 0.1, dtype=np.float32))
        out.append((g, rays_per_cell * nc))
    return out


CONFIG_NAMES = ("c0_slab64_lorentz500", "c1_box32_voigt20k", "c2_mlp_box64",
                "c3_batched256", "c4_box128_voigt100k")


def config(index: int, n_rays: Optional[int] = None) -> Case:
    """The five workload recipes (index 0..4).

    0: 1-D isothermal slab of 64 cells over 1 m, T=1000 K, 500 Lorentz lines,
       25k spectral points at 0.02 cm^-1, 1e5 rays.
    1: 32^3 box of 1 m^3 with a Gaussian hot spot (800-2000 K, sigma 0.15 m),
       20k Voigt lines over 2000-3000 cm^-1, 100k points at 0.01, 64 T nodes, 1e7 rays.
    2: learned-part workload: the index-1 line list, 64^3 box with the index-1
       field, 5e7 rays (training tables span 600-2200 K, 0.5-5 atm).
    3: 256 enclosures of 8..48 cells per side sharing the index-1 line list,
       T nodes over 600-2000 K, 1e3 rays per cell.
    4: 128^3 box with random smooth T (500-2500 K) and p (1-3 atm) fields,
       100k Voigt lines over 1500-3500 cm^-1, 400k points at 0.005, 1e9 rays.
    """
    if index == 0:
        rng = rng_for(0)
        lines = make_lines(500, 2000.0, 2500.0, rng)
        spec = Spectral(nu_min=2000.0, dnu=0.02, n_nu=25000, cutoff=25.0, profile="lorentz",
                        nT=1, T_min=1000.0, T_max=1000.0, p_ref_atm=1.0, x_ref=0.1)
        grid = uniform_grid(64, 1, 1, 1.0 / 64, math.inf, math.inf, 1000.0, 1.0, 0.1)
        return Case(CONFIG_NAMES[0], lines, spec, grid, n_rays or 100_000)
    if index in (1, 2, 3):
        rng = rng_for(1)
        lines = make_lines(20000, 2000.0, 3000.0, rng)
        if index == 1:
            spec = Spectral(nu_min=2000.0, dnu=0.01, n_nu=100000, cutoff=25.0, profile="voigt",
                            nT=64, T_min=800.0, T_max=2000.0, p_ref_atm=1.0, x_ref=0.1)
            grid = gaussian_hotspot_grid(32, 1.0, 800.0, 2000.0, 0.15)
            return Case(CONFIG_NAMES[1], lines, spec, grid, n_rays or 10_000_000)
        if index == 2:
            spec = Spectral(nu_min=2000.0, dnu=0.01, n_nu=100000, cutoff=25.0, profile="voigt",
                            nT=64, T_min=600.0, T_max=2200.0, p_ref_atm=1.0, x_ref=0.1)
            grid = gaussian_hotspot_grid(64, 1.0, 800.0, 2000.0, 0.15)
            return Case(CONFIG_NAMES[2], lines, spec, grid, n_rays or 50_000_000,
                        extra={"train_T": (600.0, 2200.0, 64), "train_p": (0.5, 5.0, 16),
                               "train_x": (0.01, 0.3), "n_samples": 20_000_000})
        spec = Spectral(nu_min=2000.0, dnu=0.01, n_nu=100000, cutoff=25.0, profile="voigt",
                        nT=64, T_min=600.0, T_max=2000.0, p_ref_atm=1.0, x_ref=0.1)
        encl = batched_enclosures(256, rng_for(3))
        return Case(CONFIG_NAMES[3], lines, spec, encl[0][0], sum(r for _, r in encl),
                    extra={"enclosures": encl})
    if index == 4:
        rng = rng_for(4)
        lines = make_lines(100000, 1500.0, 3500.0, rng)
        spec = Spectral(nu_min=1500.0, dnu=0.005, n_nu=400000, cutoff=25.0, profile="voigt",
                        nT=64, T_min=500.0, T_max=2500.0, p_ref_atm=1.0, x_ref=0.1)
        grid = multi_gaussian_grid(128, 1.0, rng_for(4, 1))
        return Case(CONFIG_NAMES[4], lines, spec, grid, n_rays or 1_000_000_000)
    raise ValueError(f"unknown config index {index}")


# ---------------------------------------------------------------- surrogate network
MLP_WIDTH = 128
MLP_LAYOUT = (("W1", (128, 4)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)),
              ("W3", (128, 128)), ("b3", (128,)), ("W4", (128, 128)), ("b4", (128,)),
              ("w5", (128,)), ("b5", (1,)))
MLP_NPARAM = sum(int(np.prod(s)) for _, s in MLP_LAYOUT)   # 50,305


def mlp_offsets():
    """Offsets of each tensor in the flat float32 parameter vector (row-major W[out][in])."""
    off, out = 0, {}
    for name, shape in MLP_LAYOUT:
        out[name] = (off, shape)
        off += int(np.prod(shape))
    return out


def mlp_init(seed: int = 0, spread_biases: bool = False) -> np.ndarray:
    """Flat float32 initial parameters: W ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)); biases 0,
    or with spread_biases also U(-1/sqrt(fan_in), 1/sqrt(fan_in)) (the first layer's
    kinks then lie at different points of the input range instead of all at its
    centre, which speeds up fitting a spectrum's lines)."""
    rng = np.random.default_rng([0, 2, 100 + int(seed)])
    flat = np.zeros(MLP_NPARAM, dtype=np.float32)
    fan = {"b1": 4, "b2": 128, "b3": 128, "b4": 128, "b5": 128}
    for name, (off, shape) in mlp_offsets().items():
        n = int(np.prod(shape))
        if name.startswith("W") or name == "w5":
            fan_in = shape[-1] if len(shape) == 2 else shape[0]
            flat[off:off + n] = rng.uniform(-1, 1, n).astype(np.float32) / np.float32(np.sqrt(fan_in))
    if spread_biases:
        rb = np.random.default_rng([0, 2, 200 + int(seed)])
        for name, (off, shape) in mlp_offsets().items():
            if name in fan:
                n = int(np.prod(shape))
                flat[off:off + n] = rb.uniform(-1, 1, n).astype(np.float32) / np.float32(np.sqrt(fan[name]))
    return flat
