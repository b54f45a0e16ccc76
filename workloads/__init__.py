"""Seeded synthetic workloads shaped like the paper's KISS-GP experiments.

This module is the only code shared by the FP64 oracle and the CUDA path's
tests and benchmark.  It holds configuration values and seeded random draws
only: no interpolation, kernel, Lanczos or variance arithmetic lives here.

Five workloads (C1..C5), each shaped like one of the paper's settings:

  C1  1-D, n = 1,000, grid of 100 points on [-0.05, 1.05], k = 50, FP64
  C2  1-D, n = 1,000,000, grid of 10,000 points, k = 100, FP32 (headline)
  C3  3-D, n = 500,000, 64^3 grid, k = 100, FP32 (+ BF16 cache)
  C4  2-D, n = 200,000, 256^2 grid, k = 64, FP32 + backward
  C5  256 independent 1-D GPs of uneven size, k = 64, FP32 + BF16 cache

Where a configuration does not state the grid bounds, the grid is placed so
that every x in [0, 1] has its four cubic-interpolation neighbours inside the
grid: spacing h = 1 / (g - 5) and first node at -2 h (KISS-GP regular grid,
Sec. 2.3).  Outputscale is 1 wherever a configuration is silent, and the noise
variance of C3/C4 is the generating noise variance.

Every array is drawn from numpy's PCG64 with seed 180306058 + config index and
a fixed sub-stream per array, then rounded to the run's dtype.  Arrays are
returned as float64 copies of the rounded values so both sides see the same
numbers.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

BASE_SEED = 180306058

# sub-stream ids
_S_XTRAIN, _S_YNOISE, _S_XTEST, _S_Z, _S_HYPER, _S_XSAMPLE = range(6)


@dataclasses.dataclass
class Workload:
    name: str
    index: int
    dim: int
    n: int
    grid_size: List[int]
    grid_lo: List[float]
    grid_hi: List[float]
    lengthscale: List[float]
    outputscale: float
    noise: float
    k: int
    t: int                      # test points for mean/variance
    dtype: str                  # "f64" or "f32": arithmetic type of the path
    cache_dtypes: Sequence[str] = ("f32",)
    s: int = 0                  # posterior samples
    t_sample: int = 0           # test points for samples
    target: str = "sin2pi"      # which synthetic target function

    @property
    def m(self) -> int:
        return int(np.prod(self.grid_size))

    @property
    def seed(self) -> int:
        return BASE_SEED + self.index

    def rng(self, stream: int) -> np.random.Generator:
        return np.random.default_rng([self.seed, stream])

    # -- rounding to the run dtype ---------------------------------------
    def _round(self, a: np.ndarray) -> np.ndarray:
        if self.dtype == "f32":
            return a.astype(np.float32).astype(np.float64)
        return a.astype(np.float64)

    def x_train(self) -> np.ndarray:
        x = self.rng(_S_XTRAIN).random((self.n, self.dim))
        return self._round(x)

    def y_train(self, x: Optional[np.ndarray] = None) -> np.ndarray:
        if x is None:
            x = self.x_train()
        rng = self.rng(_S_YNOISE)
        if self.target == "sin2pi":
            f = np.sin(2 * np.pi * x[:, 0])
            sd = 0.1
        elif self.target == "sin8pi":
            f = np.sin(8 * np.pi * x[:, 0]) + 0.5 * np.sin(2 * np.pi * x[:, 0])
            sd = 0.05
        elif self.target == "sum_sin":
            f = np.sin(2 * np.pi * x).sum(axis=1)
            sd = 0.1
        elif self.target == "sincos":
            f = np.sin(4 * np.pi * x[:, 0]) * np.cos(4 * np.pi * x[:, 1])
            sd = 0.05
        elif self.target == "sin2pi_noise":
            f = np.sin(2 * np.pi * x[:, 0])
            sd = math.sqrt(self.noise)
        else:
            raise ValueError(self.target)
        y = f + sd * rng.standard_normal(self.n)
        return self._round(y)

    def x_test(self, t: Optional[int] = None) -> np.ndarray:
        t = self.t if t is None else t
        x = self.rng(_S_XTEST).random((t, self.dim))
        return self._round(x)

    def x_sample(self, t: Optional[int] = None) -> np.ndarray:
        t = self.t_sample if t is None else t
        x = self.rng(_S_XSAMPLE).random((t, self.dim))
        return self._round(x)

    def z(self, k: int, s: int) -> np.ndarray:
        """Standard normal draws (k x s) for user-supplied sampling noise."""
        z = self.rng(_S_Z).standard_normal((k, s))
        return z.astype(np.float32).astype(np.float64)

    def scaled(self, n: Optional[int] = None, t: Optional[int] = None,
               grid_size: Optional[List[int]] = None, k: Optional[int] = None,
               name: Optional[str] = None) -> "Workload":
        """A smaller copy with the same structure (for oracle-sized tests)."""
        w = dataclasses.replace(self)
        if n is not None:
            w.n = n
        if t is not None:
            w.t = t
        if k is not None:
            w.k = k
        if grid_size is not None:
            w.grid_size = list(grid_size)
            lo, hi = zip(*[_interior_grid(g) for g in grid_size])
            w.grid_lo, w.grid_hi = list(lo), list(hi)
        w.name = name or (self.name + "-scaled")
        return w


def _interior_grid(g: int):
    """Bounds of a g-point regular grid whose 4-point stencils cover [0, 1]."""
    h = 1.0 / (g - 5)
    lo = -2.0 * h
    hi = lo + (g - 1) * h
    return lo, hi


def _wl(name, index, dim, n, g, ls, noise, k, t, dtype, target, outputscale=1.0,
        lo=None, hi=None, cache_dtypes=("f32",), s=0, t_sample=0):
    gs = [g] * dim
    if lo is None:
        b = [_interior_grid(g)] * dim
        lo = [x[0] for x in b]
        hi = [x[1] for x in b]
    return Workload(name=name, index=index, dim=dim, n=n, grid_size=gs,
                    grid_lo=list(lo), grid_hi=list(hi), lengthscale=[ls] * dim,
                    outputscale=outputscale, noise=noise, k=k, t=t, dtype=dtype,
                    cache_dtypes=cache_dtypes, s=s, t_sample=t_sample,
                    target=target)


C1 = _wl("C1-1d-n1e3-fp64", 0, 1, 1000, 100, 0.1, 0.01, 50, 1000, "f64",
         "sin2pi", lo=[-0.05], hi=[1.05], cache_dtypes=("f64",))
C2 = _wl("C2-1d-n1e6-m1e4-k100-fp32", 1, 1, 1_000_000, 10_000, 0.02, 0.0025,
         100, 1_000_000, "f32", "sin8pi", s=1000, t_sample=10_000)
C3 = _wl("C3-3d-n5e5-m64^3-k100", 2, 3, 500_000, 64, 0.15, 0.01, 100,
         2_000_000, "f32", "sum_sin", cache_dtypes=("f32", "bf16"))
C4 = _wl("C4-2d-n2e5-m256^2-k64-grad", 3, 2, 200_000, 256, 0.08, 0.0025, 64,
         65_536, "f32", "sincos")

CONFIGS = [C1, C2, C3, C4]


@dataclasses.dataclass
class BatchedWorkload:
    """C5: many independent 1-D KISS-GPs of uneven size."""
    name: str = "C5-batched-256x1d-k64"
    index: int = 4
    count: int = 256
    n_lo: int = 1_000
    n_hi: int = 200_000
    k: int = 64
    t: int = 16_384
    s: int = 256

    def members(self, count: Optional[int] = None, n_hi: Optional[int] = None,
                t: Optional[int] = None) -> List[Workload]:
        count = self.count if count is None else count
        n_hi = self.n_hi if n_hi is None else n_hi
        t = self.t if t is None else t
        rng = np.random.default_rng([BASE_SEED + self.index, _S_HYPER])
        logn = rng.uniform(math.log(self.n_lo), math.log(n_hi), size=count)
        ls = rng.uniform(0.02, 0.2, size=count)
        nz = rng.uniform(1e-3, 1e-1, size=count)
        out = []
        for i in range(count):
            n = int(round(math.exp(logn[i])))
            g = int(min(max(n // 20, 256), 8192))
            w = _wl(f"C5[{i}]", 1000 + i, 1, n, g, float(ls[i]), float(nz[i]),
                    self.k, t, "f32", "sin2pi_noise",
                    cache_dtypes=("bf16", "f32"), s=self.s, t_sample=t)
            out.append(w)
        return out


C5 = BatchedWorkload()


def by_name(name: str) -> Workload:
    for c in CONFIGS:
        if c.name == name or c.name.startswith(name):
            return c
    raise KeyError(name)
