"""LOVE pre-compute, predictive mean/variance, sampler and gradients (oracle).

TEST INFRASTRUCTURE ONLY.  FP64 throughout.

Pre-compute (Sec. 3.2, Algorithm 1):
  b = (1/m) W^T K_UU 1                    probe, the average column of W^T K_UU
  Q_k, T_k = lanczos(K^, b)               k steps, full reorthogonalisation
  T_k = L L^T                             tridiagonal Cholesky (O(k))
  R^T = K_UU W Q_k,  R' = T_k^{-1} R       so that  R^T R' ~ C  (eq. pred_covar_ski_cache)
The cache stores one symmetric factor  Rt = K_UU W Q_k L^{-T}  (m x k):
  Rt Rt^T = K_UU W Q_k T_k^{-1} Q_k^T W^T K_UU = R^T R',
so the variance of eq. pred_covar_ski_fast (i = j) is  p(x*) - |Rt^T w*|^2.

Prior term p(x*): Algorithm 1 uses k(x*, x*) while the sampling derivation
(eq. pred_covar_ski_interp_form12) uses the SKI prior w*^T K_UU w*.  The
default here is the SKI prior; prior="exact" selects k(x*, x*) = s_f.

Mean (eq. pred_mean_ski, zero prior mean): a = K_UU W K^^{-1} y with the solve by
CG (Sec. 2.1); mu(x*) = w*^T a.

Sampler (Sec. 3.3): Lanczos on K_UU - R^T R' = K_UU - Rt Rt^T (eq. lancapprox)
gives Q', T'; with T' = L' L'^T, S = Q' L' (m x k') and samples are
mu + W*^T S v, v ~ N(0, I) (eqs. sample, pred_covar_ski_interp_form).  If T' is
not positive definite (the difference of two nearly equal PSD matrices in
finite precision), the eigendecomposition T' = V diag(lam) V^T with lam
clamped at 0 gives S = Q' V diag(sqrt(lam)) instead (flagged).

Gradients (not in the paper; derived from eq. pred_covar_ski_cache by matrix
calculus with every K^^{-1} replaced by M M^T, M = Q L^{-T}, Q held fixed):
  d var_i / d x*_e  = 2 (dw_i/dx_e)^T K w_i - 2 (Rt^T dw_i/dx_e) . (Rt^T w_i)
  d var_i / d l_e   = (w_i - P v_i)^T (dK/dl_e) (w_i - P v_i),   P = W M, v_i = Rt^T w_i
  d var_i / d s^2   = |L^{-T} v_i|^2
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import scipy.linalg

from . import lanczos as lz
from .grid import Grid
from .rng import rademacher_probe
from .ski import SKI


@dataclasses.dataclass
class LoveCache:
    grid: Grid
    noise: float
    k_eff: int
    alpha: np.ndarray
    beta: np.ndarray
    chol_d: np.ndarray
    chol_e: np.ndarray
    Rt: np.ndarray                      # m x k_eff
    a: Optional[np.ndarray] = None      # m (mean cache)
    P: Optional[np.ndarray] = None      # m x k_eff  (W Q L^{-T}, for gradients)
    S: Optional[np.ndarray] = None      # m x k'     (sampler root)
    sampler_fallback: bool = False
    beta_last: float = 0.0
    cg_iters: int = 0

    @property
    def L(self) -> np.ndarray:
        return lz.bidiag_dense(self.chol_d, self.chol_e)


def rt_from_q(ski: SKI, Q: np.ndarray, d: np.ndarray, e: np.ndarray):
    """Rt = K_UU W Q L^{-T}; also returns P = W Q L^{-T}."""
    L = lz.bidiag_dense(d, e)
    WQ = ski.W @ Q.T                          # m x k   (W_X Q_k)
    R0 = ski.grid.kuu_matmul(WQ)              # m x k   (K_UU W_X Q_k = R^T)
    # X L^T = R0  <=>  L X^T = R0^T
    Rt = scipy.linalg.solve_triangular(L, R0.T, lower=True).T
    P = scipy.linalg.solve_triangular(L, WQ.T, lower=True).T
    return Rt, P


def mean_cache(ski: SKI, tol: float = 1e-12, max_iter: int = 10000):
    """a = K_UU W (W^T K_UU W + s^2 I)^{-1} y by CG (eq. pred_mean_ski)."""
    z, it, _ = lz.cg(ski.mvm, ski.y, tol=tol, max_iter=max_iter)
    return ski.mvm_kux(z), it


def precompute(ski: SKI, k: int, tau: float = 1e-12, want_mean: bool = True,
               cg_tol: float = 1e-12, cg_max_iter: int = 10000,
               want_grad: bool = False) -> LoveCache:
    b = ski.probe()
    Q, alpha, beta, beta_last = lz.lanczos(ski.mvm, b, k, tau)
    d, e = lz.tridiag_cholesky(alpha, beta)
    Rt, P = rt_from_q(ski, Q, d, e)
    a, it = (None, 0)
    if want_mean and ski.y is not None:
        a, it = mean_cache(ski, cg_tol, cg_max_iter)
    return LoveCache(grid=ski.grid, noise=ski.noise, k_eff=alpha.shape[0],
                     alpha=alpha, beta=beta, chol_d=d, chol_e=e, Rt=Rt, a=a,
                     P=P if want_grad else None, beta_last=beta_last, cg_iters=it)


def prior(grid: Grid, x: np.ndarray, mode: str = "ski") -> np.ndarray:
    if mode == "exact":
        return np.full(np.atleast_2d(x).reshape(-1, grid.dim).shape[0], grid.outputscale)
    return grid.local_kernel_quadform(x)


def predict(cache: LoveCache, x: np.ndarray, prior_mode: str = "ski"):
    """(mean, var) at test points: mu = w^T a, var = p - |Rt^T w|^2 (Alg. 1)."""
    Ws = cache.grid.W(x)                      # m x t
    V = Ws.T @ cache.Rt                       # t x k   (Rt^T w_i as rows)
    var = prior(cache.grid, x, prior_mode) - np.sum(V * V, axis=1)
    mean = None if cache.a is None else Ws.T @ cache.a
    return mean, var


def predict_cov(cache: LoveCache, x1: np.ndarray, x2: np.ndarray, prior_mode: str = "ski") -> np.ndarray:
    """Posterior cross-covariances (eq. pred_covar_ski_fast with i != j, Alg. 1 on
    two point sets): cov[i, j] = p(x1_i, x2_j) - (Rt^T w1_i) . (Rt^T w2_j), with p
    the SKI prior w1^T K_UU w2 or, in "exact" mode, outputscale * k(x1_i, x2_j)."""
    grid = cache.grid
    W1, W2 = grid.W(x1), grid.W(x2)                                   # m x t1, m x t2
    if prior_mode == "exact":
        a = np.atleast_2d(x1).reshape(-1, grid.dim)
        b = np.atleast_2d(x2).reshape(-1, grid.dim)
        d2 = np.zeros((a.shape[0], b.shape[0]))
        for e in range(grid.dim):
            d2 += (a[:, e][:, None] - b[:, e][None, :]) ** 2 / (2.0 * grid.lengthscale[e] ** 2)
        P = grid.outputscale * np.exp(-d2)
    else:
        P = W1.T @ grid.kuu_matmul(W2.toarray())
    return P - (W1.T @ cache.Rt) @ (W2.T @ cache.Rt).T


# -- sampler ------------------------------------------------------------------
def sampler_precompute(cache: LoveCache, k: int, seed: int, tau: float = 1e-12):
    """S with S S^T ~ K_UU - Rt Rt^T via Lanczos (Sec. 3.3)."""
    grid, Rt = cache.grid, cache.Rt

    def mvm(v):
        return grid.kuu_matmul(v) - Rt @ (Rt.T @ v)

    r = rademacher_probe(seed, grid.m)
    Q, alpha, beta, _ = lz.lanczos(mvm, r, k, tau)
    try:
        d, e = lz.tridiag_cholesky(alpha, beta)
        S = Q.T @ lz.bidiag_dense(d, e)
        fallback = False
    except lz.NotPositiveDefinite:
        lam, V = np.linalg.eigh(lz.tridiag_dense(alpha, beta))
        S = Q.T @ (V * np.sqrt(np.maximum(lam, 0.0))[None, :])
        fallback = True
    cache.S = S
    cache.sampler_fallback = fallback
    return S, fallback


def predict_root(cache: LoveCache, x: np.ndarray) -> np.ndarray:
    """Predictive variance from the posterior root of Sec. 3.3 (S S^T ~ K_UU - C):
    var(x*) = |S^T w*|^2, a sum of squares (no cancellation), exact at Krylov
    exhaustion, a rank-k' truncation of the posterior covariance otherwise."""
    G = cache.grid.W(x).T @ cache.S              # t x k'
    return np.einsum("tk,tk->t", G, G)


def sample(cache: LoveCache, x: np.ndarray, Z: np.ndarray) -> np.ndarray:
    """Samples F (s x t): F[j, i] = mu_i + (W*^T S Z)[i, j]  (eq. sample)."""
    Ws = cache.grid.W(x)
    G = Ws.T @ cache.S                        # t x k'
    mu = np.zeros(G.shape[0]) if cache.a is None else Ws.T @ cache.a
    return (mu[:, None] + G @ Z).T


# -- gradients ----------------------------------------------------------------
def var_grad(cache: LoveCache, ski: SKI, x: np.ndarray, g: np.ndarray,
             prior_mode: str = "ski", chunk: int = 256):
    """Vector-Jacobian product of sum_i g_i var_i.

    Returns grad_x (t x d), grad_lengthscale (d), grad_noise.  Needs P
    (pre-compute with want_grad) -- or recomputes it from the SKI.
    """
    grid = cache.grid
    x = np.atleast_2d(np.asarray(x, dtype=np.float64)).reshape(-1, grid.dim)
    g = np.asarray(g, dtype=np.float64)
    t, dim = x.shape
    Ws = grid.W(x)
    V = Ws.T @ cache.Rt                                   # t x k
    grad_x = np.zeros((t, dim))
    for e in range(dim):
        dWs = grid.W(x, deriv_dim=e)
        dV = dWs.T @ cache.Rt
        dp = 2.0 * grid.local_kernel_quadform(x, deriv_x=e) if prior_mode == "ski" else 0.0
        grad_x[:, e] = g * (dp - 2.0 * np.sum(dV * V, axis=1))
    P = cache.P
    if P is None:
        raise ValueError("pre-compute with want_grad=True to keep P = W Q L^-T")
    grad_l = np.zeros(dim)
    Wd = Ws.toarray()                                     # m x t (small t only)
    for s0 in range(0, t, chunk):
        sl = slice(s0, min(t, s0 + chunk))
        U = Wd[:, sl] - P @ V[sl].T                       # m x c: w_i - P v_i
        for e in range(dim):
            KU = grid.kuu_matmul(U, deriv_dim=e)
            q = np.sum(U * KU, axis=0)
            if prior_mode == "exact":
                q = q - grid.local_kernel_quadform(x[sl], deriv_l=e)
            grad_l[e] += float(g[sl] @ q)
    Y = scipy.linalg.solve_triangular(cache.L.T, V.T, lower=False)   # L^{-T} v_i
    grad_noise = float(g @ np.sum(Y * Y, axis=0))
    return grad_x, grad_l, grad_noise


def cache_with_grid(cache: LoveCache, grid: Grid) -> LoveCache:
    c = dataclasses.replace(cache)
    c.grid = grid
    return c
