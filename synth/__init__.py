"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module draws random numbers and lays out workload descriptions. It holds
none of the solver's arithmetic: no discretisation, no time-stepping matrices,
no Krylov step. Both sides import it so that they see byte-identical inputs.

Random numbers
--------------
* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014): state_i = seed + (i+1)*0x9E3779B97F4A7C15, output
  = mix(state_i). Being counter-based, element i depends only on (seed, i).
* uniform on [-1, 1): 2 * (x >> 11) * 2^-53 - 1.
* standard normal: Box-Muller on pairs of uniforms in (0, 1].
* Gaussian-correlated field: white normal noise convolved separably with a
  Gaussian kernel of standard deviation ell/sqrt(2) cells (so the covariance is
  exp(-r^2 / (2 ell^2))), truncated at 4 standard deviations, zero padding at
  the domain edge, then shifted and scaled to zero sample mean and unit sample
  variance.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Return outputs offset..offset+n-1 of the SplitMix64 stream for `seed`."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles uniform on [-1, 1)."""
    x = splitmix64(seed, n, offset) >> np.uint64(11)
    return 2.0 * x.astype(np.float64) * (2.0 ** -53) - 1.0


def _unit_open(seed: int, n: int, offset: int) -> np.ndarray:
    """n doubles uniform on (0, 1]."""
    x = splitmix64(seed, n, offset) >> np.uint64(11)
    return (x.astype(np.float64) + 1.0) * (2.0 ** -53)


def normal(seed: int, n: int) -> np.ndarray:
    """n standard normal doubles by Box-Muller."""
    m = (n + 1) // 2
    u1 = _unit_open(seed, m, 0)
    u2 = _unit_open(seed, m, m)
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:n]


def correlated_field(seed: int, shape: tuple, ell: float) -> np.ndarray:
    """Zero-mean, unit-variance Gaussian field with correlation length ell cells.

    `shape` is (nz, ny, nx) (x fastest). Returns a C-contiguous float64 array.
    """
    from scipy.ndimage import convolve1d

    g = normal(seed, int(np.prod(shape))).reshape(shape)
    sd = ell / math.sqrt(2.0)
    rad = int(math.ceil(4.0 * sd))
    x = np.arange(-rad, rad + 1, dtype=np.float64)
    ker = np.exp(-0.5 * (x / sd) ** 2)
    ker /= np.sqrt(np.sum(ker ** 2))
    for ax in range(len(shape)):
        if shape[ax] > 1:
            g = convolve1d(g, ker, axis=ax, mode="constant", cval=0.0)
    g = g - g.mean()
    g = g / g.std()
    return np.ascontiguousarray(g)


# ---------------------------------------------------------------------------
# Workload descriptions (sizes, coefficients, seeds). Only data, no arithmetic
# of the solver.
# ---------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    dims: tuple            # (nx, ny, nz); nz == 1 for 2-D
    kind: str              # "convdiff", "diffreact", "richards"
    s: int                 # block width (coupled steps or stages)
    tau: float
    tol: float = 1e-10
    precond: str = "jacobi"
    velocity: tuple = (0.0, 0.0, 0.0)
    diffusion: str = "const"      # "const" or "lognormal_iid"
    seed_coef: int = 0
    seed_rhs: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        nx, ny, nz = self.dims
        return nx * ny * nz


def convdiff_2d_64(s: int = 4) -> Workload:
    """2-D convection-diffusion, 64x64 cells, D=1, v=(1,0.5), implicit Euler,
    tau=1e-3, block GMRES(30) + Jacobi, tol 1e-10, RHS U[-1,1] seed 1."""
    return Workload("convdiff2d_64x64", (64, 64, 1), "convdiff", s, 1e-3, 1e-10,
                    "jacobi", (1.0, 0.5, 0.0), "const", 0, 1)


def convdiff_3d(n: int = 128, s: int = 8) -> Workload:
    """3-D convection-diffusion, n^3 cells, D=exp(g) with g iid N(0,1) (seed 2),
    v=(1,0.5,0), implicit Euler tau=1e-3, block GMRES(30) + ILU(0), tol 1e-10,
    RHS U[-1,1] (seed 2)."""
    return Workload(f"convdiff3d_{n}^3", (n, n, n), "convdiff", s, 1e-3, 1e-10,
                    "ilu0", (1.0, 0.5, 0.0), "lognormal_iid", 2, 2)


def diffreact_2d(n: int = 512) -> Workload:
    """2-D nonlinear diffusion-reaction u_t = div((1+u^2) grad u) + u(1-u) + src,
    n x n cells, Neumann, u0 = 0.5, moving-circle source, SDIRK2 window of s=2
    stages pipelined through 4 steps, tau=1e-2."""
    return Workload(f"diffreact2d_{n}x{n}", (n, n, 1), "diffreact", 2, 1e-2, 1e-8,
                    "ilu0", extra={"steps": 4, "u0": 0.5})


def richards_3d(n: int = 96, s: int = 8) -> Workload:
    """3-D Richards, n^3 cells, van Genuchten alpha=1, n=2, theta_r=0.05,
    theta_s=0.4, K_S = exp(2 g) with g correlated (ell = 8 cells, seed 4),
    implicit Euler tau=1/96 in windows of s steps."""
    return Workload(f"richards3d_{n}^3", (n, n, n), "richards", s, 1.0 / 96.0, 1e-8,
                    "ilu0", seed_coef=4,
                    extra={"steps": 18, "alpha": 1.0, "n_vg": 2.0, "theta_r": 0.05,
                           "theta_s": 0.4, "sigma": 2.0, "ell": 8.0, "dt_D": 1.0 / 16.0})


def diffusion_field(w: Workload) -> np.ndarray:
    """Per-cell diffusion coefficient, shape (nz, ny, nx)."""
    nx, ny, nz = w.dims
    if w.diffusion == "const":
        return np.ones((nz, ny, nx))
    if w.diffusion == "lognormal_iid":
        return np.exp(normal(w.seed_coef, w.n)).reshape(nz, ny, nx)
    raise ValueError(w.diffusion)


def permeability_field(w: Workload) -> np.ndarray:
    """Saturated conductivity K_S = exp(sigma * g), g correlated, (nz, ny, nx)."""
    nx, ny, nz = w.dims
    g = correlated_field(w.seed_coef, (nz, ny, nx), w.extra["ell"])
    return np.exp(w.extra["sigma"] * g)


def rhs_block(w: Workload, s: int | None = None) -> np.ndarray:
    """Right-hand sides b(t_k), one column per coupled step, N x s row-major,
    iid U[-1,1]; column k of row r is element r*s + k of the stream."""
    s = w.s if s is None else s
    return uniform(w.seed_rhs, w.n * s).reshape(w.n, s)


def request_stream(seed: int, count: int, rate: float, grids=(32, 48, 64, 96, 128),
                   widths=(2, 4, 8, 16), precisions=("fp32", "fp64")) -> list:
    """Seeded Poisson stream of slab-solve requests: exponential inter-arrival
    times of mean 1/rate seconds, grid (cells per direction), block width s
    and inner precision drawn uniformly. Returns a list of dicts
    {rid, arrival, n, s, precision} in arrival order."""
    u = 0.5 * (uniform(seed, 4 * count) + 1.0)          # [0, 1)
    t, out = 0.0, []
    for i in range(count):
        t += -np.log1p(-u[4 * i]) / rate
        out.append({"rid": i, "arrival": t,
                    "n": int(grids[min(int(u[4 * i + 1] * len(grids)), len(grids) - 1)]),
                    "s": int(widths[min(int(u[4 * i + 2] * len(widths)), len(widths) - 1)]),
                    "precision": precisions[min(int(u[4 * i + 3] * len(precisions)),
                                                len(precisions) - 1)]})
    return out


def batch_jobs(seed: int, count: int, grids2d=(32, 48, 64), grids3d=(16, 24, 32),
               widths=(2, 4, 8, 16)) -> list:
    """Seeded mix of small slab solves for one batched launch: half 2-D
    (n x n cells), half 3-D (n^3), grid and block width s drawn uniformly.
    Returns dicts {jid, dims, s, seed_coef, seed_rhs}; each job's diffusion
    field is log-normal iid from seed_coef, its right-hand side U[-1,1] from
    seed_rhs."""
    u = 0.5 * (uniform(seed, 3 * count) + 1.0)          # [0, 1)
    out = []
    for i in range(count):
        three = u[3 * i] >= 0.5
        g = grids3d if three else grids2d
        n = int(g[min(int(u[3 * i + 1] * len(g)), len(g) - 1)])
        s = int(widths[min(int(u[3 * i + 2] * len(widths)), len(widths) - 1)])
        out.append({"jid": i, "dims": (n, n, n) if three else (n, n, 1), "s": s,
                    "seed_coef": 1000 + 2 * i, "seed_rhs": 1001 + 2 * i})
    return out
