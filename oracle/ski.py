"""The SKI operator (oracle; test infrastructure only).

eq. ski:  K~_XX = W_X^T K_UU W_X, and the operator Lanczos and CG see is
K^_XX = K~_XX + sigma^2 I (Sec. 2, Algorithm 1 input mvm_K_XX).  mvm_K_UX of
Algorithm 1 is  V -> K_UU W_X V.
"""
from __future__ import annotations

import numpy as np

from .grid import Grid


class SKI:
    def __init__(self, grid: Grid, x_train: np.ndarray, noise: float,
                 y_train: np.ndarray | None = None):
        self.grid = grid
        self.x = np.atleast_2d(np.asarray(x_train, dtype=np.float64)).reshape(-1, grid.dim)
        self.n = self.x.shape[0]
        self.noise = float(noise)
        self.y = None if y_train is None else np.asarray(y_train, dtype=np.float64)
        self.W = grid.W(self.x)            # m x n
        self.WT = self.W.T.tocsr()         # n x m

    def mvm(self, v: np.ndarray) -> np.ndarray:
        """(W^T K_UU W + sigma^2 I) v  for v of length n (or n x r)."""
        return self.WT @ self.grid.kuu_matmul(self.W @ v) + self.noise * v

    def mvm_kux(self, V: np.ndarray) -> np.ndarray:
        """K_UU W V  (m x r) -- Algorithm 1's mvm_K_UX."""
        return self.grid.kuu_matmul(self.W @ V)

    def probe(self) -> np.ndarray:
        """b = (1/m) W^T K_UU 1, the average column of W^T K_UU (Sec. 3.2)."""
        ones = np.ones(self.grid.m)
        return (self.WT @ self.grid.kuu_matmul(ones)) / self.grid.m

    def dense(self) -> np.ndarray:
        """Dense K^_XX for tiny n (brute-force checks)."""
        Wd = self.W.toarray()
        return Wd.T @ self.grid.dense_kuu() @ Wd + self.noise * np.eye(self.n)
