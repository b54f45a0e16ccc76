"""KISS-GP grid, RBF kernel and interpolation matrix (oracle; test infrastructure only).

Sec. 2.3: the m inducing points lie on a regular grid, so for a stationary
kernel K_UU is Toeplitz (1-D) or a Kronecker product of Toeplitz factors (a
product kernel over dimensions).  The kernel used throughout is the
RBF kernel k(x, x') = s_f * exp(-|x - x'|^2 / (2 l^2)); for d > 1 it is the
product over dimensions with one lengthscale per dimension, so

    K_UU = s_f * T_1 (x) T_2 (x) ... (x) T_d,   T_e[a, b] = exp(-((a-b) h_e)^2 / (2 l_e^2)).

Grid linear index: row-major over dimensions, the last dimension fastest.
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence

import numpy as np
import scipy.linalg
import scipy.sparse as sp

from . import keys


@dataclasses.dataclass
class Grid:
    size: List[int]
    lo: List[float]
    hi: List[float]
    lengthscale: List[float]
    outputscale: float = 1.0

    @property
    def dim(self) -> int:
        return len(self.size)

    @property
    def m(self) -> int:
        return int(np.prod(self.size))

    @property
    def h(self) -> List[float]:
        return [(self.hi[e] - self.lo[e]) / (self.size[e] - 1) for e in range(self.dim)]

    @property
    def strides(self) -> List[int]:
        st = [1] * self.dim
        for e in range(self.dim - 2, -1, -1):
            st[e] = st[e + 1] * self.size[e + 1]
        return st

    # -- Toeplitz factors ---------------------------------------------------
    def toeplitz_col(self, e: int) -> np.ndarray:
        """First column of T_e: exp(-(j h_e)^2 / (2 l_e^2)), j = 0..g_e-1."""
        j = np.arange(self.size[e], dtype=np.float64)
        r = j * self.h[e]
        return np.exp(-(r ** 2) / (2.0 * self.lengthscale[e] ** 2))

    def toeplitz_col_dl(self, e: int) -> np.ndarray:
        """First column of dT_e/dl_e: T_e entry * r^2 / l_e^3."""
        j = np.arange(self.size[e], dtype=np.float64)
        r = j * self.h[e]
        ls = self.lengthscale[e]
        return np.exp(-(r ** 2) / (2.0 * ls ** 2)) * (r ** 2) / ls ** 3

    def dense_kuu(self, deriv_dim: int = -1) -> np.ndarray:
        """Dense K_UU (or dK_UU/dl_e for e = deriv_dim) for tiny grids."""
        out = np.array([[self.outputscale]])
        for e in range(self.dim):
            c = self.toeplitz_col_dl(e) if e == deriv_dim else self.toeplitz_col(e)
            out = np.kron(out, scipy.linalg.toeplitz(c))
        return out

    def kuu_matmul(self, V: np.ndarray, deriv_dim: int = -1) -> np.ndarray:
        """K_UU @ V (or dK_UU/dl_e @ V) through one Toeplitz product per mode.

        V is m or m x r.  Each mode product multiplies the fibres of that mode
        by T_e; Toeplitz products use scipy.linalg.matmul_toeplitz (an FFT
        library routine) for long modes and a dense Toeplitz matrix for short
        ones.
        """
        V = np.asarray(V, dtype=np.float64)
        vec = V.ndim == 1
        if vec:
            V = V[:, None]
        r = V.shape[1]
        X = V.reshape(list(self.size) + [r])
        for e in range(self.dim):
            c = self.toeplitz_col_dl(e) if e == deriv_dim else self.toeplitz_col(e)
            Xe = np.moveaxis(X, e, 0)
            sh = Xe.shape
            flat = Xe.reshape(sh[0], -1)
            if sh[0] <= 2048:
                flat = scipy.linalg.toeplitz(c) @ flat
            else:
                flat = scipy.linalg.matmul_toeplitz((c, c), flat)
            X = np.moveaxis(flat.reshape(sh), 0, e)
        out = self.outputscale * X.reshape(self.m, r)
        return out[:, 0] if vec else out

    # -- interpolation -------------------------------------------------------
    def interp(self, x: np.ndarray, check: bool = True):
        """Per-dimension base indices, weights and weight derivatives."""
        x = np.atleast_2d(np.asarray(x, dtype=np.float64))
        if x.shape[1] != self.dim:
            x = x.reshape(-1, self.dim)
        out = []
        for e in range(self.dim):
            out.append(keys.interp_1d(x[:, e], self.lo[e], self.h[e], self.size[e], check))
        return out

    def stencil(self, x: np.ndarray, check: bool = True, deriv_dim: int = -1):
        """Rows (grid indices) and values of the 4^d nonzeros of each w_x.

        Returns (rows[n, 4^d], vals[n, 4^d]).  With deriv_dim = e the values
        are those of d w_x / d x_e (the e-th factor replaced by its derivative).
        """
        per = self.interp(x, check)
        n = per[0][0].shape[0]
        rows = np.zeros((n, 1), dtype=np.int64)
        vals = np.ones((n, 1), dtype=np.float64)
        st = self.strides
        for e, (i, w, dw) in enumerate(per):
            idx = (i[:, None] + np.arange(-1, 3)[None, :]) * st[e]
            we = dw if e == deriv_dim else w
            rows = (rows[:, :, None] + idx[:, None, :]).reshape(n, -1)
            vals = (vals[:, :, None] * we[:, None, :]).reshape(n, -1)
        return rows, vals

    def W(self, x: np.ndarray, check: bool = True, deriv_dim: int = -1) -> sp.csr_matrix:
        """Sparse interpolation matrix W_X (m x n), columns w_x (eq. ski)."""
        rows, vals = self.stencil(x, check, deriv_dim)
        n = rows.shape[0]
        cols = np.repeat(np.arange(n), rows.shape[1])
        return sp.csr_matrix((vals.ravel(), (rows.ravel(), cols)), shape=(self.m, n))

    def local_kernel_quadform(self, x: np.ndarray, deriv_x: int = -1,
                              deriv_l: int = -1, check: bool = True) -> np.ndarray:
        """w_x^T K_UU w_x evaluated on the 4^d nonzeros of w_x.

        For the product kernel the 4^d x 4^d block of K_UU factorises, so
        w^T K w = s_f * prod_e (w_e^T T_e^loc w_e) with T_e^loc[r, s] = T_e[|r-s|].
        deriv_x = e gives (d w / d x_e)^T K w (one factor uses dw_e on the left);
        deriv_l = e gives w^T (dK/dl_e) w.
        """
        per = self.interp(x, check)
        out = np.full(per[0][0].shape[0], self.outputscale)
        for e, (_, w, dw) in enumerate(per):
            c = self.toeplitz_col_dl(e) if e == deriv_l else self.toeplitz_col(e)
            Tloc = scipy.linalg.toeplitz(c[:4])
            left = dw if e == deriv_x else w
            out = out * np.einsum("nr,rs,ns->n", left, Tloc, w)
        return out


def grid_from_workload(wl) -> Grid:
    return Grid(size=list(wl.grid_size), lo=list(wl.grid_lo), hi=list(wl.grid_hi),
                lengthscale=list(wl.lengthscale), outputscale=float(wl.outputscale))


@dataclasses.dataclass
class AdditiveGrid:
    """Additive composition of one-dimensional KISS-GP kernels (Sec. 3, "Extension
    to additive kernel compositions"): k~(x, x') = sum_e w_e(x_e)^T K_e w_e(x'_e),
    written as one SKI kernel with the stacked interpolation vector
    w(x) = [w_1(x_1); ...; w_d(x_d)] (4 nonzeros per component) and the
    block-diagonal K_UU = diag(K_1, ..., K_d), K_e = s_f T_e on grid e.

    Same interface as Grid (W, kuu_matmul, dense_kuu, local_kernel_quadform, m,
    dim), so the LOVE oracle runs on it unchanged.  Grid index of node j of
    component e: offset(e) + j, offset(e) = size[0] + ... + size[e-1].
    """
    size: List[int]
    lo: List[float]
    hi: List[float]
    lengthscale: List[float]
    outputscale: float = 1.0

    @property
    def dim(self) -> int:
        return len(self.size)

    @property
    def m(self) -> int:
        return int(np.sum(self.size))

    @property
    def h(self) -> List[float]:
        return [(self.hi[e] - self.lo[e]) / (self.size[e] - 1) for e in range(self.dim)]

    @property
    def offsets(self) -> List[int]:
        return [int(np.sum(self.size[:e])) for e in range(self.dim)]

    def component(self, e: int) -> Grid:
        return Grid([self.size[e]], [self.lo[e]], [self.hi[e]], [self.lengthscale[e]], self.outputscale)

    def toeplitz_col(self, e: int) -> np.ndarray:
        return self.component(e).toeplitz_col(0)

    def dense_kuu(self, deriv_dim: int = -1) -> np.ndarray:
        return scipy.linalg.block_diag(*[self.component(e).dense_kuu(0 if e == deriv_dim else -1)
                                         for e in range(self.dim)])

    def kuu_matmul(self, V: np.ndarray, deriv_dim: int = -1) -> np.ndarray:
        out = np.zeros_like(np.asarray(V, dtype=np.float64))
        for e, off in enumerate(self.offsets):
            sl = slice(off, off + self.size[e])
            out[sl] = self.component(e).kuu_matmul(np.asarray(V, dtype=np.float64)[sl],
                                                   deriv_dim=0 if e == deriv_dim else -1)
        return out

    def interp(self, x: np.ndarray, check: bool = True):
        x = np.atleast_2d(np.asarray(x, dtype=np.float64))
        if x.shape[1] != self.dim:
            x = x.reshape(-1, self.dim)
        return [keys.interp_1d(x[:, e], self.lo[e], self.h[e], self.size[e], check) for e in range(self.dim)]

    def stencil(self, x: np.ndarray, check: bool = True, deriv_dim: int = -1):
        """Rows and values of the 4 d nonzeros of the stacked w_x (component by
        component; deriv_dim = e: d w_x / d x_e, nonzero in component e only)."""
        per = self.interp(x, check)
        rows, vals = [], []
        for e, ((i, w, dw), off) in enumerate(zip(per, self.offsets)):
            rows.append(off + i[:, None] + np.arange(-1, 3)[None, :])
            if deriv_dim < 0:
                vals.append(w)
            else:
                vals.append(dw if e == deriv_dim else np.zeros_like(w))
        return np.concatenate(rows, axis=1), np.concatenate(vals, axis=1)

    def W(self, x: np.ndarray, check: bool = True, deriv_dim: int = -1) -> sp.csr_matrix:
        rows, vals = self.stencil(x, check, deriv_dim)
        n = rows.shape[0]
        cols = np.repeat(np.arange(n), rows.shape[1])
        return sp.csr_matrix((vals.ravel(), (rows.ravel(), cols)), shape=(self.m, n))

    def local_kernel_quadform(self, x: np.ndarray, deriv_x: int = -1,
                              deriv_l: int = -1, check: bool = True) -> np.ndarray:
        """w_x^T K_UU w_x = s_f sum_e w_e^T T_e^loc w_e (a sum over components)."""
        per = self.interp(x, check)
        out = np.zeros(per[0][0].shape[0])
        for e, (_, w, dw) in enumerate(per):
            c = self.component(e)
            cc = c.toeplitz_col_dl(0) if e == deriv_l else c.toeplitz_col(0)
            if deriv_l >= 0 and e != deriv_l:
                continue
            if deriv_x >= 0 and e != deriv_x:
                continue
            Tloc = scipy.linalg.toeplitz(cc[:4])
            left = dw if e == deriv_x else w
            out = out + self.outputscale * np.einsum("nr,rs,ns->n", left, Tloc, w)
        return out


def additive_grid_from_workload(wl) -> AdditiveGrid:
    return AdditiveGrid(size=list(wl.grid_size), lo=list(wl.grid_lo), hi=list(wl.grid_hi),
                        lengthscale=list(wl.lengthscale), outputscale=float(wl.outputscale))
