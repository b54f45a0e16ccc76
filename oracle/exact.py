"""The exact SKI posterior that LOVE approximates (oracle; test infrastructure only).

eq. pred_covar_approx / pred_covar_ski_cache: with the KISS-GP kernel,
    var(x*)  = p(x*) - w*^T C w*,   C = K_UU W (W^T K_UU W + s^2 I)^{-1} W^T K_UU
    mu(x*)   = w*^T K_UU W (W^T K_UU W + s^2 I)^{-1} y          (eq. pred_mean_ski)
Three independent evaluations:
  dense     n x n Cholesky of K^ (tiny n)
  push      the m x m push-through form  C = K G (K G + s^2 I)^{-1} K,  G = W W^T
            (from (W^T K W + s^2 I)^{-1} W^T = W^T (K W W^T + s^2 I)^{-1})
  cg        one FP64 CG solve per test point (Sec. 3.1, "Limitations": the
            KISS-GP variance computed from scratch)
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import lanczos as lz
from .love import prior
from .ski import SKI


def exact_dense(ski: SKI, x: np.ndarray, prior_mode: str = "ski"):
    grid = ski.grid
    Khat = ski.dense()
    Ws = grid.W(x).toarray()                                  # m x t
    Kd = grid.dense_kuu()
    kstar = ski.W.toarray().T @ (Kd @ Ws)                     # n x t
    cf = scipy.linalg.cho_factor(Khat, lower=True)
    sol = scipy.linalg.cho_solve(cf, kstar)
    var = prior(grid, x, prior_mode) - np.sum(kstar * sol, axis=0)
    mean = None
    if ski.y is not None:
        mean = kstar.T @ scipy.linalg.cho_solve(cf, ski.y)
    return mean, var


def pushthrough_C(ski: SKI) -> np.ndarray:
    grid = ski.grid
    Kd = grid.dense_kuu()
    G = (ski.W @ ski.W.T).toarray()
    A = Kd @ G + ski.noise * np.eye(grid.m)
    X = np.linalg.solve(A, Kd)                                # (K G + s^2 I)^{-1} K
    return Kd @ (G @ X)


def exact_pushthrough(ski: SKI, x: np.ndarray, prior_mode: str = "ski", C=None):
    grid = ski.grid
    if C is None:
        C = pushthrough_C(ski)
    Ws = grid.W(x)
    WC = Ws.T @ C                                             # t x m
    var = prior(grid, x, prior_mode) - np.einsum("tm,tm->t", WC, Ws.T.toarray())
    mean = None
    if ski.y is not None:
        mean = Ws.T @ mean_weights_pushthrough(ski)
    return mean, var


def mean_weights_pushthrough(ski: SKI) -> np.ndarray:
    """a = K_UU W (W^T K_UU W + s^2 I)^{-1} y = K_UU (G K_UU + s^2 I)^{-1} W y,
    G = W W^T (push-through identity), by one dense m x m solve; the predictive
    mean is w*^T a (eq. pred_mean_ski)."""
    grid = ski.grid
    Kd = grid.dense_kuu()
    G = (ski.W @ ski.W.T).tocsr()
    return Kd @ np.linalg.solve(np.asarray(G @ Kd) + ski.noise * np.eye(grid.m), ski.W @ ski.y)


def exact_cg(ski: SKI, x: np.ndarray, prior_mode: str = "ski", tol: float = 1e-12,
             max_iter: int = 20000):
    grid = ski.grid
    Ws = grid.W(x)
    t = Ws.shape[1]
    var = prior(grid, x, prior_mode).copy()
    for i in range(t):
        kstar = ski.WT @ grid.kuu_matmul(Ws[:, i].toarray().ravel())
        z, _, _ = lz.cg(ski.mvm, kstar, tol=tol, max_iter=max_iter)
        var[i] -= kstar @ z
    return var
