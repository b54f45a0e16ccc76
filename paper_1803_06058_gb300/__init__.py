"""GB300 (sm_103a) LOVE for KISS-GP: thin Python binding of liblove.so.

The binding marshals arguments only: torch supplies device memory (through
the library's allocator callback, backed by torch's caching allocator) and
streams; every step of the method runs in the library's CUDA kernels.  The
names mirror the C ABI (include/love.h):

    ski_build(x_train, y_train, grid_size, grid_lo, grid_hi, lengthscale,
              outputscale, noise)                         -> Ski
    love_precompute(ski, k, cache_dtype, want_mean, want_sampler, want_grad,
                    prior_exact, ...)                     -> Cache
    love_predict_mean_var(cache, x_test)                 -> (mean, var)
    love_sample(cache, x_test, s, z=None, seed=0)        -> samples (s x t)
    love_var_backward(cache, x_test, grad_var)           -> (grad_x, grad_l, grad_noise)
    love_var(cache, x_test, lengthscale=None, noise=None) autograd op

There is no CPU fallback: importing works without a GPU, but every call needs
liblove.so and a CUDA device, and raises otherwise.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import (BF16, F32, F64, PRIOR_EXACT, WANT_GRAD, WANT_MEAN, WANT_SAMPLER,  # noqa: F401
                   LoveError, check)

_DT = {"f32": F32, "f64": F64, "bf16": BF16, torch.float32: F32, torch.float64: F64,
       torch.bfloat16: BF16}
_TORCH = {F32: torch.float32, F64: torch.float64}


def lib():
    return _lib.load()


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None) -> C.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


# -- device memory through torch's caching allocator -------------------------
@_lib.ALLOC_FN
def _torch_alloc(ctx, nbytes, stream):
    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))
    except Exception:  # OOM -> NULL -> LOVE_ERR_OOM
        return None


@_lib.FREE_FN
def _torch_free(ctx, ptr, nbytes, stream):
    if ptr:
        torch.cuda.caching_allocator_delete(int(ptr))


TORCH_ALLOCATOR = _lib.love_allocator(_torch_alloc, _torch_free, None)


def _desc(dim, n, grid_size, grid_lo, grid_hi, lengthscale, outputscale, noise, dtype,
          use_torch_allocator=True, additive=False):
    d = _lib.love_ski_desc()
    d.dim = dim
    d.n = n
    for e in range(3):
        d.grid_size[e] = int(grid_size[e]) if e < dim else 1
        d.grid_lo[e] = float(grid_lo[e]) if e < dim else 0.0
        d.grid_hi[e] = float(grid_hi[e]) if e < dim else 1.0
        d.lengthscale[e] = float(lengthscale[e]) if e < dim else 1.0
    d.outputscale = float(outputscale)
    d.noise = float(noise)
    d.dtype = dtype
    d.allocator = C.pointer(TORCH_ALLOCATOR) if use_torch_allocator else None
    d.additive = 1 if additive else 0
    return d


class Ski:
    """KISS-GP structure of a training set (handle of ski_build)."""

    def __init__(self, handle, desc, dtype, n, dim, m):
        self.handle = handle
        self.desc = desc
        self.dtype = dtype
        self.n = n
        self.dim = dim
        self.m = m

    def __del__(self):
        if getattr(self, "handle", None) and _lib._lib is not None:
            _lib._lib.ski_destroy(self.handle)
            self.handle = None


class Cache:
    """LOVE cache (handle of love_precompute / love_cache_import / love_cache_load)."""

    def __init__(self, handle, dtype, dim):
        self.handle = handle
        self.dtype = dtype
        self.dim = dim

    def info(self) -> dict:
        inf = _lib.love_cache_info_t()
        check("love_cache_info", lib().love_cache_info(self.handle, C.byref(inf)))
        return {f: (list(getattr(inf, f)) if f in ("grid_size", "phase_ms") else getattr(inf, f))
                for f, _ in inf._fields_}

    def device_status(self, reset=False, stream=None) -> dict:
        st = _lib.love_device_status_t()
        check("love_get_device_status",
              lib().love_get_device_status(self.handle, int(reset), C.byref(st), _stream(stream)))
        return {"bits": st.bits, "domain_errors": st.domain_errors, "clamped": st.clamped}

    def __del__(self):
        if getattr(self, "handle", None) and _lib._lib is not None:
            _lib._lib.love_cache_destroy(self.handle)
            self.handle = None


def _as_points(x: torch.Tensor, dim: int, dtype: torch.dtype) -> torch.Tensor:
    if x.dim() == 1:
        x = x.reshape(-1, 1)
    if x.shape[-1] != dim:
        raise ValueError(f"points must be (t, {dim})")
    if not x.is_cuda or x.dtype != dtype or not x.is_contiguous():
        raise ValueError(f"points must be a contiguous CUDA {dtype} tensor")
    return x


def ski_build(x_train: torch.Tensor, y_train: Optional[torch.Tensor], grid_size: Sequence[int],
              grid_lo: Sequence[float], grid_hi: Sequence[float], lengthscale: Sequence[float],
              outputscale: float, noise: float, stream=None, use_torch_allocator=True,
              additive: bool = False) -> Ski:
    """KISS-GP structure of a training set.  additive=True: the additive
    composition of 1-D kernels (block-diagonal K_UU, m = sum of grid_size)."""
    if x_train.dim() == 1:
        x_train = x_train.reshape(-1, 1)
    n, dim = x_train.shape
    dt = _DT[x_train.dtype]
    x_train = _as_points(x_train, dim, x_train.dtype)
    if y_train is not None and (not y_train.is_contiguous() or y_train.dtype != x_train.dtype
                                or y_train.numel() != n or not y_train.is_cuda):
        raise ValueError("y_train must be a contiguous CUDA tensor of n values, same dtype as x")
    d = _desc(dim, n, grid_size, grid_lo, grid_hi, lengthscale, outputscale, noise, dt,
              use_torch_allocator, additive)
    h = C.c_void_p()
    check("ski_build", lib().ski_build(C.byref(d), _ptr(x_train), _ptr(y_train), _stream(stream),
                                       C.byref(h)))
    sizes = [int(grid_size[e]) for e in range(dim)]
    m = sum(sizes) if additive else int(np.prod(sizes))
    return Ski(h, d, dt, n, dim, m)


def ski_mvm(ski: Ski, v: torch.Tensor, stream=None) -> torch.Tensor:
    out = torch.empty_like(v)
    check("ski_mvm", lib().ski_mvm(ski.handle, _ptr(v), _ptr(out), _stream(stream)))
    return out


def ski_mvm_kuu(ski: Ski, v: torch.Tensor, stream=None) -> torch.Tensor:
    out = torch.empty_like(v)
    check("ski_mvm_kuu", lib().ski_mvm_kuu(ski.handle, _ptr(v), _ptr(out), _stream(stream)))
    return out


def ski_mvm_kuu_noalloc(ski: Ski, v: torch.Tensor, out: Optional[torch.Tensor] = None,
                        stream=None) -> torch.Tensor:
    """K_UU v through the entry point that allocates nothing (its FFT scratch is
    a fixed device array inside the library); pass `out` to keep this call
    allocation-free on the Python side as well."""
    if out is None:
        out = torch.empty_like(v)
    check("ski_mvm_kuu_noalloc", lib().ski_mvm_kuu_noalloc(ski.handle, _ptr(v), _ptr(out), _stream(stream)))
    return out


def love_precompute(ski: Ski, k: int, cache_dtype: str = None, want_mean: bool = True,
                    want_sampler: bool = False, want_grad: bool = False, prior_exact: bool = False,
                    breakdown_tol: float = 0.0, cg_tol: float = 0.0, cg_max_iter: int = 0,
                    sampler_k: int = 0, sampler_seed: int = 0, reorth: str = "always", reorth_eta: float = 0.0,
                    cg_plain: bool = False, time_reorth: bool = False, stream=None) -> Cache:
    """reorth: "always" (two Gram-Schmidt passes every step), "detect" (the
    second pass only where |Q_j^T y'| > reorth_eta |y'|) or "lowsync" (the second
    pass folded into the first through Q^T Q, checked like "detect").  cg_plain: mean CG
    without the spectral preconditioner (1-D grids use it by default).
    time_reorth: record the sweeps' device time (info()["reorth_ms"])."""
    o = _opts(ski.dtype, k, cache_dtype, want_mean, want_sampler, want_grad, prior_exact, breakdown_tol, cg_tol,
              cg_max_iter, sampler_k, sampler_seed, reorth, reorth_eta, cg_plain)
    if time_reorth:
        o.flags |= _lib.TIME_REORTH
    h = C.c_void_p()
    keff = C.c_int(0)
    check("love_precompute", lib().love_precompute(ski.handle, C.byref(o), _stream(stream),
                                                   C.byref(h), C.byref(keff)))
    return Cache(h, ski.dtype, ski.dim)


_REORTH = {"always": 0, "detect": 1, "lowsync": 2}


def _opts(dtype, k, cache_dtype, want_mean, want_sampler, want_grad, prior_exact, breakdown_tol, cg_tol,
          cg_max_iter, sampler_k, sampler_seed, reorth="always", reorth_eta=0.0, cg_plain=False):
    o = _lib.love_precompute_opts()
    o.k = k
    o.cache_dtype = dtype if cache_dtype is None else _DT[cache_dtype]
    o.flags = ((WANT_MEAN if want_mean else 0) | (WANT_SAMPLER if want_sampler else 0)
               | (WANT_GRAD if want_grad else 0) | (PRIOR_EXACT if prior_exact else 0))
    o.breakdown_tol = breakdown_tol
    o.cg_tol = cg_tol
    o.cg_max_iter = cg_max_iter
    o.sampler_k = sampler_k
    o.sampler_seed = sampler_seed
    o.reorth = _REORTH[reorth]
    o.reorth_eta = reorth_eta
    o.cg_plain = 1 if cg_plain else 0
    return o


def love_precompute_batched(skis: Sequence[Ski], k: int, cache_dtype: str = None, want_mean: bool = True,
                            want_sampler: bool = False, want_grad: bool = False, prior_exact: bool = False,
                            breakdown_tol: float = 0.0, cg_tol: float = 0.0, cg_max_iter: int = 0,
                            sampler_k: int = 0, sampler_seed: int = 0, workers: int = 0, reorth: str = "always",
                            reorth_eta: float = 0.0, cg_plain: bool = False, streams: bool = False, stream=None):
    """love_precompute for every ski (shared options), run concurrently; returns (caches, k_eff).
    1-D FP32 batches run their Lanczos steps as one batched run (one launch per phase
    per step for all GPs, captured into a CUDA graph; caches[b].info()["batched_rows"]
    is the sweep chunk size it picked); streams=True runs each GP's own
    love_precompute on a pool stream instead."""
    B = len(skis)
    if B == 0:
        return [], []
    o = _opts(skis[0].dtype, k, cache_dtype, want_mean, want_sampler, want_grad, prior_exact, breakdown_tol,
              cg_tol, cg_max_iter, sampler_k, sampler_seed, reorth, reorth_eta, cg_plain)
    if streams:
        o.flags |= _lib.BATCH_STREAMS
    hs = (C.c_void_p * B)(*[s.handle for s in skis])
    out = (C.c_void_p * B)()
    keff = (C.c_int * B)()
    check("love_precompute_batched", lib().love_precompute_batched(B, hs, C.byref(o), workers, _stream(stream),
                                                                   out, keff))
    return [Cache(C.c_void_p(out[b]), skis[b].dtype, skis[b].dim) for b in range(B)], list(keff)


class Batch:
    """Caches served together (handle of love_batch_create); keeps the caches alive."""

    def __init__(self, handle, caches, t_sizes):
        self.handle = handle
        self.caches = list(caches)
        self.t_sizes = list(t_sizes)
        self.dtype = caches[0].dtype
        self.dim = caches[0].dim

    def info(self) -> dict:
        inf = _lib.love_batch_info_t()
        check("love_batch_info", lib().love_batch_info(self.handle, C.byref(inf)))
        return {"lanes_per_point": inf.lanes_per_point, "ctas_per_sm": inf.ctas_per_sm,
                "candidate_ms": list(inf.candidate_ms)[:inf.n_candidates], "chunks": inf.chunks,
                "graph_captures": inf.graph_captures, "graph_captures_dropped": inf.graph_captures_dropped}

    def __del__(self):
        if getattr(self, "handle", None) and _lib._lib is not None:
            _lib._lib.love_batch_destroy(self.handle)
            self.handle = None


def love_batch_create(caches: Sequence[Cache], t_sizes: Sequence[int], stream=None) -> Batch:
    B = len(caches)
    off = [0]
    for t in t_sizes:
        off.append(off[-1] + int(t))
    hs = (C.c_void_p * B)(*[c.handle for c in caches])
    to = (C.c_int64 * (B + 1))(*off)
    h = C.c_void_p()
    check("love_batch_create", lib().love_batch_create(B, hs, to, _stream(stream), C.byref(h)))
    return Batch(h, caches, t_sizes)


def love_predict_batched(batch: Batch, x_test: torch.Tensor, want_mean: bool = True, stream=None,
                         out_mean=None, out_var=None):
    """x_test: the concatenated test points of all GPs (sum t_b, dim)."""
    dt = _TORCH[batch.dtype]
    x_test = _as_points(x_test, batch.dim, dt)
    T = x_test.shape[0]
    if T != sum(batch.t_sizes):
        raise ValueError("x_test rows must equal the batch's total test points")
    var = out_var if out_var is not None else torch.empty(T, dtype=dt, device=x_test.device)
    mean = None
    if want_mean:
        mean = out_mean if out_mean is not None else torch.empty(T, dtype=dt, device=x_test.device)
    check("love_predict_batched", lib().love_predict_batched(batch.handle, _ptr(x_test), _ptr(mean), _ptr(var),
                                                             _stream(stream)))
    return mean, var


def love_sample_batched(batch: Batch, x_test: torch.Tensor, s: int, seed: int = 0, stream=None, out=None):
    """s samples per GP; returns a flat tensor: GP b's s x t_b block starts at s * t_off[b]."""
    dt = _TORCH[batch.dtype]
    x_test = _as_points(x_test, batch.dim, dt)
    T = x_test.shape[0]
    if T != sum(batch.t_sizes):
        raise ValueError("x_test rows must equal the batch's total test points")
    out = out if out is not None else torch.empty(s * T, dtype=dt, device=x_test.device)
    check("love_sample_batched", lib().love_sample_batched(batch.handle, _ptr(x_test), s, seed, _ptr(out),
                                                           _stream(stream)))
    return out


def love_batch_serve(batch: Batch, x_test: torch.Tensor, mean: Optional[torch.Tensor], var: torch.Tensor,
                     s: int = 0, seed: int = 0, samples: Optional[torch.Tensor] = None, use_graph: bool = True,
                     stream=None):
    """Predict (and sample) the whole batch into caller buffers; with use_graph the launches
    are captured into one CUDA graph on first use and replayed afterwards."""
    dt = _TORCH[batch.dtype]
    x_test = _as_points(x_test, batch.dim, dt)
    check("love_batch_serve", lib().love_batch_serve(batch.handle, _ptr(x_test), _ptr(mean), _ptr(var), s, seed,
                                                     _ptr(samples), int(use_graph), _stream(stream)))


def batch_split(batch: Batch, flat: torch.Tensor, s: int = 0):
    """Views of a batched output per GP: (t_b,) for predict outputs, (s, t_b) for samples."""
    res, off = [], 0
    for t in batch.t_sizes:
        if s:
            res.append(flat[off * s:(off + t) * s].view(s, t))
        else:
            res.append(flat[off:off + t])
        off += t
    return res


def love_predict_mean_var(cache: Cache, x_test: torch.Tensor, want_mean: bool = True,
                          stream=None, out_mean=None, out_var=None):
    dt = _TORCH[cache.dtype]
    x_test = _as_points(x_test, cache.dim, dt)
    t = x_test.shape[0]
    var = out_var if out_var is not None else torch.empty(t, dtype=dt, device=x_test.device)
    mean = None
    if want_mean:
        mean = out_mean if out_mean is not None else torch.empty(t, dtype=dt, device=x_test.device)
    check("love_predict_mean_var",
          lib().love_predict_mean_var(cache.handle, t, _ptr(x_test), _ptr(mean), _ptr(var),
                                      _stream(stream)))
    return mean, var


def love_predict_mean_var_host(cache: Cache, x_test: torch.Tensor, want_mean: bool = True,
                               stream=None, out_mean=None, out_var=None):
    """love_predict_mean_var on host (CPU) tensors; pinned tensors are read and
    written by the kernel directly.  Outputs are pinned CPU tensors unless given.
    Returns when the results are in the host tensors."""
    dt = _TORCH[cache.dtype]
    if x_test.is_cuda:
        raise ValueError("love_predict_mean_var_host takes host tensors")
    x_test = x_test.to(dt).reshape(-1, cache.dim).contiguous()
    t = x_test.shape[0]
    pin = x_test.is_pinned()
    var = out_var if out_var is not None else torch.empty(t, dtype=dt, pin_memory=pin)
    mean = None
    if want_mean:
        mean = out_mean if out_mean is not None else torch.empty(t, dtype=dt, pin_memory=pin)
    check("love_predict_mean_var_host",
          lib().love_predict_mean_var_host(cache.handle, t, _ptr(x_test), _ptr(mean), _ptr(var), _stream(stream)))
    return mean, var


def love_predict_covariance(cache: Cache, x1: torch.Tensor, x2: Optional[torch.Tensor] = None,
                            stream=None) -> torch.Tensor:
    """t1 x t2 posterior cross-covariances (x2 defaults to x1)."""
    dt = _TORCH[cache.dtype]
    x1 = _as_points(x1, cache.dim, dt)
    x2 = x1 if x2 is None else _as_points(x2, cache.dim, dt)
    out = torch.empty((x1.shape[0], x2.shape[0]), dtype=dt, device=x1.device)
    check("love_predict_covariance", lib().love_predict_covariance(cache.handle, x1.shape[0], _ptr(x1), x2.shape[0],
                                                                   _ptr(x2), _ptr(out), _stream(stream)))
    return out


def love_predict_var_root(cache: Cache, x_test: torch.Tensor, stream=None, out_var=None) -> torch.Tensor:
    """Variance from the posterior root: |S^T w*|^2 (needs want_sampler)."""
    dt = _TORCH[cache.dtype]
    x_test = _as_points(x_test, cache.dim, dt)
    t = x_test.shape[0]
    var = out_var if out_var is not None else torch.empty(t, dtype=dt, device=x_test.device)
    check("love_predict_var_root", lib().love_predict_var_root(cache.handle, t, _ptr(x_test), _ptr(var),
                                                               _stream(stream)))
    return var


def love_sample(cache: Cache, x_test: torch.Tensor, s: int, z: Optional[torch.Tensor] = None,
                seed: int = 0, stream=None) -> torch.Tensor:
    dt = _TORCH[cache.dtype]
    x_test = _as_points(x_test, cache.dim, dt)
    t = x_test.shape[0]
    out = torch.empty((s, t), dtype=dt, device=x_test.device)
    if z is not None and (z.dtype != dt or not z.is_contiguous() or not z.is_cuda):
        raise ValueError("z must be a contiguous CUDA tensor (k_s x s) of the cache dtype")
    check("love_sample", lib().love_sample(cache.handle, t, _ptr(x_test), s, _ptr(z), seed,
                                           _ptr(out), _stream(stream)))
    return out


def love_sampler_precompute(cache: Cache, k: int = 0, seed: int = 0, stream=None) -> Cache:
    """Sampler root S (Sec. 3.3) for an existing cache (pre-computed, imported or
    loaded): k Lanczos steps on K_UU - Rt Rt^T (0 -> the cache's k_eff).
    Replaces any root the cache held; returns the same cache."""
    check("love_sampler_precompute", lib().love_sampler_precompute(cache.handle, int(k), int(seed),
                                                                   _stream(stream)))
    return cache


def love_var_backward(cache: Cache, x_test: torch.Tensor, grad_var: torch.Tensor,
                      want_x: bool = True, want_hyper: bool = True, stream=None):
    dt = _TORCH[cache.dtype]
    x_test = _as_points(x_test, cache.dim, dt)
    t = x_test.shape[0]
    gx = torch.empty_like(x_test) if want_x else None
    gl = (C.c_double * cache.dim)() if want_hyper else None
    gn = C.c_double(0.0) if want_hyper else None
    check("love_var_backward",
          lib().love_var_backward(cache.handle, t, _ptr(x_test), _ptr(grad_var.contiguous()), _ptr(gx),
                                  C.cast(gl, _lib.DP) if want_hyper else None,
                                  C.byref(gn) if want_hyper else None, _stream(stream)))
    return gx, (list(gl) if want_hyper else None), (gn.value if want_hyper else None)


class _LoveVar(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, ls, noise, cache):
        ctx.cache = cache
        ctx.save_for_backward(x)
        ctx.hyper = (ls is not None, noise is not None)
        _, var = love_predict_mean_var(cache, x.detach().contiguous(), want_mean=False)
        return var

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        want_h = ctx.hyper[0] or ctx.hyper[1]
        gx, gl, gn = love_var_backward(ctx.cache, x.detach().contiguous(), g.contiguous().to(x.dtype),
                                       want_x=ctx.needs_input_grad[0], want_hyper=want_h)
        gls = torch.tensor(gl, dtype=x.dtype, device=x.device) if ctx.hyper[0] else None
        gno = torch.tensor(gn, dtype=x.dtype, device=x.device) if ctx.hyper[1] else None
        return gx, gls, gno, None


def love_var(cache: Cache, x: torch.Tensor, lengthscale: Optional[torch.Tensor] = None,
             noise: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Differentiable LOVE variance: gradients flow to x (through the cubic
    interpolation weights) and, if passed, to the lengthscale and noise tensors
    (whose values must be the ones the cache was built with)."""
    return _LoveVar.apply(x, lengthscale, noise, cache)


def love_cache_import(grid_size, grid_lo, grid_hi, lengthscale, outputscale, noise, Rt, a=None,
                      S=None, alpha=None, beta=None, P=None, dtype="f32", cache_dtype=None,
                      prior_exact=False, stream=None, additive=False) -> Cache:
    """Build a cache from host (numpy) arrays computed elsewhere."""
    import numpy as np
    dim = len(grid_size)
    dt = _DT[dtype]
    cdt = dt if cache_dtype is None else _DT[cache_dtype]
    d = _desc(dim, 1, grid_size, grid_lo, grid_hi, lengthscale, outputscale, noise, dt, additive=additive)
    Rt = np.ascontiguousarray(Rt, dtype=np.float64)
    m, k = Rt.shape
    flags = ((WANT_MEAN if a is not None else 0) | (WANT_SAMPLER if S is not None else 0)
             | (WANT_GRAD if P is not None else 0) | (PRIOR_EXACT if prior_exact else 0))

    def dp(arr):
        if arr is None:
            return None
        arr = np.ascontiguousarray(arr, dtype=np.float64)
        keep.append(arr)
        return arr.ctypes.data_as(_lib.DP)

    keep = []
    ks = 0 if S is None else np.asarray(S).shape[1]
    h = C.c_void_p()
    check("love_cache_import",
          lib().love_cache_import(C.byref(d), k, cdt, flags, dp(Rt), dp(a), ks, dp(S), dp(alpha),
                                  dp(beta), dp(P), _stream(stream), C.byref(h)))
    return Cache(h, dt, dim)


def love_cache_export(cache: Cache, stream=None) -> dict:
    import numpy as np
    inf = cache.info()
    m, k, ks = inf["m"], inf["k_eff"], inf["sampler_k"]
    Rt = np.zeros((m, k))
    a = np.zeros(m)
    S = np.zeros((m, ks)) if ks else None
    has_p = bool(inf["flags"] & WANT_GRAD)
    P = np.zeros((m, k)) if has_p else None
    al = np.zeros(k)
    be = np.zeros(max(k - 1, 1))

    def dp(arr):
        return None if arr is None else arr.ctypes.data_as(_lib.DP)

    check("love_cache_export", lib().love_cache_export(cache.handle, dp(Rt), dp(a), dp(S), dp(P),
                                                       dp(al), dp(be), _stream(stream)))
    return {"Rt": Rt, "a": a if inf["flags"] & WANT_MEAN else None, "S": S, "P": P,
            "alpha": al, "beta": be[: max(k - 1, 0)], "info": inf}


def love_cache_save(cache: Cache, path: str, stream=None):
    check("love_cache_save", lib().love_cache_save(cache.handle, path.encode(), _stream(stream)))


def love_cache_load(path: str, stream=None) -> Cache:
    h = C.c_void_p()
    check("love_cache_load", lib().love_cache_load(path.encode(), C.pointer(TORCH_ALLOCATOR),
                                                   _stream(stream), C.byref(h)))
    c = Cache(h, F32, 1)
    inf = c.info()
    c.dtype = inf["dtype"]
    c.dim = inf["dim"]
    return c


def version() -> str:
    return lib().love_version().decode()
