"""Seeded synthetic inputs for the PHIF solver and its oracle.

This module only draws random numbers and lays them out on the grid. It holds
none of the method's arithmetic (no discretisation, no factorisation), so both
the FP64 CPU oracle and the CUDA path may import it.

Layout conventions (shared input format, not solver code):

* A d-dimensional grid has ``ns[i]`` interior nodes along axis ``i``
  (x first).  The unit cube is split into ``ns[i] + 1`` intervals, so
  ``h_i = 1 / (ns[i] + 1)``.
* A *pixel* (voxel in 3D) is one grid interval square/cube.  Per-pixel
  coefficient arrays have shape ``(ns_y+1, ns_x+1)`` in 2D and
  ``(ns_z+1, ns_y+1, ns_x+1)`` in 3D (C order, x fastest).
* DOF index of interior node with 0-based indices ``(i, j, k)`` is
  ``i + ns_x*(j + ns_y*k)``; node vectors have length ``prod(ns)``.

The workloads follow the numerical section of the paper (Sec. 4): synthetic
random coefficient fields on the unit square/cube with zero Dirichlet data.
The paper's own field (uniform samples, Gaussian blur of width 4h, median
quantisation to {1e-2, 1e2}) is provided as :func:`paper_quantized_field`;
the benchmark workloads use i.i.d. log-uniform per-pixel fields instead.
"""
from __future__ import annotations

import dataclasses
import numpy as np

SEED_BASE = 1808 * 100


def rng(seed: int) -> np.random.Generator:
    """numpy PCG64 generator; every workload is derived from one integer seed."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def pixel_shape(ns):
    """Shape of a per-pixel array for a grid with interior sizes ``ns`` (x first)."""
    return tuple(int(n) + 1 for n in reversed(ns))


def log_uniform_pixels(ns, lo: float, hi: float, seed: int) -> np.ndarray:
    """i.i.d. per-pixel field with log10(a) ~ U[log10 lo, log10 hi]."""
    g = rng(seed)
    e = g.uniform(np.log10(lo), np.log10(hi), size=pixel_shape(ns))
    return np.power(10.0, e)


def normal_rhs(ns, seed: int, nrhs: int = 1) -> np.ndarray:
    """f ~ N(0, 1) at every interior node; shape (N,) or (nrhs, N)."""
    n = int(np.prod(ns))
    g = rng(seed)
    if nrhs == 1:
        return g.standard_normal(n)
    return g.standard_normal((nrhs, n))


def gaussian_bump_log_field(ns, seed: int, count: int = 20, amp: float = 3.0) -> np.ndarray:
    """log a*(x) = sum of ``count`` isotropic Gaussian bumps, sampled at pixel centres.

    Centres ~ U(0,1)^d, widths ~ U[0.05, 0.15], signs +-1 equiprobable,
    peak height ``amp``.
    """
    g = rng(seed)
    d = len(ns)
    centres = g.uniform(0.0, 1.0, size=(count, d))
    widths = g.uniform(0.05, 0.15, size=count)
    signs = np.where(g.uniform(size=count) < 0.5, -1.0, 1.0)
    axes = [(np.arange(n + 1) + 0.5) / (n + 1) for n in ns]  # pixel centres, x first
    grids = np.meshgrid(*reversed(axes), indexing="ij")      # C order: (z,) y, x
    grids = list(reversed(grids))                            # x first
    out = np.zeros(pixel_shape(ns))
    for c, w, s in zip(centres, widths, signs):
        r2 = sum((grids[i] - c[i]) ** 2 for i in range(d))
        out += s * amp * np.exp(-0.5 * r2 / (w * w))
    return out


def paper_quantized_field(ns, seed: int, lo: float = 1e-2, hi: float = 1e2) -> np.ndarray:
    """The paper's high-contrast field (Sec. 4), on pixels instead of nodes.

    Uniform samples, smoothed by an isotropic Gaussian of width 4h (periodic
    wrap, truncated at 3 widths), then set to ``lo`` at or below the median and
    ``hi`` above it.
    """
    g = rng(seed)
    shp = pixel_shape(ns)
    u = g.uniform(size=shp)
    sigma = 4.0  # in units of h
    rad = int(np.ceil(3 * sigma))
    t = np.arange(-rad, rad + 1)
    kern = np.exp(-0.5 * (t / sigma) ** 2)
    kern /= kern.sum()
    for ax in range(u.ndim):
        acc = np.zeros_like(u)
        for off, wgt in zip(t, kern):
            acc += wgt * np.roll(u, off, axis=ax)
        u = acc
    mu = np.median(u)
    return np.where(u <= mu, lo, hi)


@dataclasses.dataclass
class Problem:
    """One synthetic instance: grid, per-pixel a, node b, right-hand sides."""
    ns: tuple
    a: np.ndarray            # per-pixel coefficient
    b: float | np.ndarray    # scalar or per-node
    f: np.ndarray            # (N,) or (nrhs, N)
    leaf: int
    tol: float
    name: str = ""

    @property
    def n(self) -> int:
        return int(np.prod(self.ns))


def make_problem(ns, lo, hi, b, leaf, tol, seed, nrhs=1, name=""):
    a = log_uniform_pixels(ns, lo, hi, seed)
    f = normal_rhs(ns, seed + 1, nrhs)
    return Problem(tuple(int(x) for x in ns), a, b, f, leaf, tol, name)


def config_problem(index: int, **over) -> Problem:
    """The five benchmark workloads (index 0..2 here; 3 and 4 have helpers).

    0: 2D 127^2, log10 a ~ U[-2,2], b=0, leaf 8, tol 1e-3.
    1: 2D 1023^2, log10 a ~ U[-4,4], b=0, leaf 16, tol 1e-3 (1e-6 variant).
    2: 3D 63^3, log10 a ~ U[-3,3], b=1e-2, leaf 8, tol 1e-3.
    """
    seed = SEED_BASE + index
    if index == 0:
        p = make_problem((127, 127), 1e-2, 1e2, 0.0, 8, 1e-3, seed, name="2d-127sq-leaf8")
    elif index == 1:
        p = make_problem((1023, 1023), 1e-4, 1e4, 0.0, 16, 1e-3, seed, name="2d-1023sq-leaf16")
    elif index == 2:
        p = make_problem((63, 63, 63), 1e-3, 1e3, 1e-2, 8, 1e-3, seed, name="3d-63cube-leaf8")
    else:
        raise ValueError("config index must be 0, 1 or 2; use batched_problems / inverse_problem")
    for k, v in over.items():
        setattr(p, k, v)
    return p


def batched_sides(count: int = 64, lo: int = 127, hi: int = 511, seed: int = SEED_BASE + 3) -> list:
    """Grid sides drawn uniformly from the integers lo..hi inclusive."""
    return [int(s) for s in rng(seed).integers(lo, hi + 1, size=count)]


def batched_problems(count: int = 64, nrhs: int = 32, seed: int = SEED_BASE + 3,
                     sides=None) -> list:
    """Many independent 2D problems with log10 a ~ U[-3,3], nrhs N(0,1) RHS each."""
    sides = batched_sides(count, seed=seed) if sides is None else list(sides)
    out = []
    for i, s in enumerate(sides):
        out.append(make_problem((s, s), 1e-3, 1e3, 0.0, 8, 1e-3, seed * 1000 + i,
                                nrhs=nrhs, name=f"batch{i}-{s}sq"))
    return out


def inverse_problem(ns=(511, 511), seed: int = SEED_BASE + 4):
    """Coefficient-recovery workload: log a* from 20 bumps, f = 1, initial log a = 0."""
    log_a_star = gaussian_bump_log_field(ns, seed)
    f = np.ones(int(np.prod(ns)))
    return log_a_star, f
