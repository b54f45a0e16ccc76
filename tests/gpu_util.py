"""Helpers shared by the GPU parity tests (oracle side + binding side)."""
from __future__ import annotations

import numpy as np

import workloads
from oracle import grid as og
from oracle import love as ol
from oracle import ski as os_


def small_workload(dim=1, g=40, n=2000, ls=0.15, noise=0.01, k=20, t=3000, dtype="f32", seed_index=50):
    """A scaled-down workload with the structure of the measured ones."""
    lo, hi = workloads._interior_grid(g)
    return workloads.Workload(
        name=f"small-{dim}d-g{g}-n{n}", index=seed_index, dim=dim, n=n, grid_size=[g] * dim,
        grid_lo=[lo] * dim, grid_hi=[hi] * dim, lengthscale=[ls] * dim, outputscale=1.0,
        noise=noise, k=k, t=t, dtype=dtype,
        target={1: "sin2pi", 2: "sincos", 3: "sum_sin"}[dim])


def oracle_ski(wl, x=None, y=None):
    x = wl.x_train() if x is None else x
    y = wl.y_train(x) if y is None else y
    return os_.SKI(og.grid_from_workload(wl), x, wl.noise, y)


def oracle_cache(wl, k=None, want_grad=False, **kw):
    ski = oracle_ski(wl)
    return ski, ol.precompute(ski, k=wl.k if k is None else k, want_grad=want_grad, **kw)


def gpu_ski(love, torch, wl, x=None, y=None, with_y=True):
    dt = torch.float64 if wl.dtype == "f64" else torch.float32
    x = wl.x_train() if x is None else x
    y = wl.y_train(x) if y is None else y
    xt = torch.tensor(x, dtype=dt, device="cuda")
    yt = torch.tensor(y, dtype=dt, device="cuda") if with_y else None
    return love.ski_build(xt, yt, wl.grid_size, wl.grid_lo, wl.grid_hi, wl.lengthscale,
                          wl.outputscale, wl.noise)


def round_to(a, dtype):
    """Round an FP64 array as the library stores it (RNE)."""
    import torch
    if dtype == "f64":
        return np.asarray(a, dtype=np.float64)
    if dtype == "f32":
        return np.asarray(a, dtype=np.float32).astype(np.float64)
    t = torch.tensor(np.asarray(a, dtype=np.float64)).to(torch.bfloat16)
    return t.to(torch.float64).numpy()


def rounded_cache(cache, dtype):
    """Copy of an oracle cache with Rt and a rounded to the cache dtype."""
    import dataclasses
    c = dataclasses.replace(cache)
    c.Rt = round_to(cache.Rt, dtype)
    if cache.a is not None:
        c.a = round_to(cache.a, dtype)
    return c
