"""Pins for the oracle's interpolation, grid and kernel (Sec. 2.3, eq. ski).

Each check is against something other than the oracle's own formula: exact
rational values of Keys' kernel, polynomial reproduction, brute-force loops,
dense Kronecker products, and scipy's FFT Toeplitz product.
"""
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg

from oracle import grid as G
from oracle import keys as K

GOLD = os.path.join(os.path.dirname(__file__), "golden", "keys_weights.txt")


def _golden():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        rows.append([float(Fraction(t)) for t in line.split()])
    return np.array(rows)


def test_keys_golden_values():
    gold = _golden()
    h, lo, g = 0.5, -1.0, 40
    for f, *w in gold:
        x = lo + (10 + f) * h                  # base node 10, fraction f
        i, wt, _ = K.interp_1d(np.array([x]), lo, h, g)
        assert i[0] == 10
        np.testing.assert_allclose(wt[0], w, rtol=0, atol=1e-15)


def test_keys_partition_of_unity_and_quadratic_reproduction():
    rng = np.random.default_rng(0)
    lo, h, g = 0.0, 0.1, 50
    x = rng.uniform(0.2, 4.6, 1000)
    i, w, _ = K.interp_1d(x, lo, h, g)
    nodes = lo + (i[:, None] + np.arange(-1, 3)[None, :]) * h
    np.testing.assert_allclose(w.sum(1), 1.0, atol=1e-14)
    np.testing.assert_allclose((w * nodes).sum(1), x, atol=1e-13)
    np.testing.assert_allclose((w * nodes ** 2).sum(1), x ** 2, atol=1e-12)
    # a = -1/2 does not reproduce cubics: the error is visible
    assert np.max(np.abs((w * nodes ** 3).sum(1) - x ** 3)) > 1e-6


def test_keys_node_hit_and_domain():
    i, w, _ = K.interp_1d(np.array([0.375]), 0.0, 0.125, 20)
    assert i[0] == 3
    np.testing.assert_array_equal(w[0], [0, 1, 0, 0])
    K.interp_1d(np.array([2.24]), 0.0, 0.125, 20)          # base 17: nodes 16..19
    with pytest.raises(K.DomainError):
        K.interp_1d(np.array([0.05]), 0.0, 0.125, 20)      # needs node -1
    with pytest.raises(K.DomainError):
        K.interp_1d(np.array([2.3]), 0.0, 0.125, 20)       # needs node 20
    with pytest.raises(K.DomainError):
        K.interp_1d(np.array([np.nan]), 0.0, 0.125, 20)


def test_keys_derivative_matches_finite_differences_and_is_continuous():
    s = np.linspace(-1.95, 1.95, 391)
    s = s[np.min(np.abs(s[:, None] - np.array([-1, 0, 1])[None, :]), axis=1) > 1e-3]
    hfd = 1e-6
    fd = (K.u(s + hfd) - K.u(s - hfd)) / (2 * hfd)
    np.testing.assert_allclose(K.du(s), fd, atol=1e-8)
    # C1 across the knots at |s| = 1 and 0
    for knot in (-1.0, 0.0, 1.0):
        assert abs(K.du(knot - 1e-12) - K.du(knot + 1e-12)) < 1e-9
    # weight derivatives are d w / d x
    lo, h, g = 0.0, 0.1, 50
    x = np.array([1.234, 2.011, 3.5501])
    _, w, dw = K.interp_1d(x, lo, h, g)
    _, wp, _ = K.interp_1d(x + 1e-7, lo, h, g)
    _, wm, _ = K.interp_1d(x - 1e-7, lo, h, g)
    np.testing.assert_allclose(dw, (wp - wm) / 2e-7, atol=1e-6)


def _brute_W(grid, x):
    """Interpolation matrix by explicit loops over points and stencil nodes."""
    m = grid.m
    n = x.shape[0]
    Wd = np.zeros((m, n))
    for p in range(n):
        per = []
        for e in range(grid.dim):
            s = (x[p, e] - grid.lo[e]) / grid.h[e]
            i = int(np.floor(s))
            per.append([(i + r - 1, float(K.u(s - (i + r - 1)))) for r in range(4)])
        import itertools
        for combo in itertools.product(*per):
            idx = 0
            wv = 1.0
            for e, (node, we) in enumerate(combo):
                idx = idx * grid.size[e] + node
                wv *= we
            Wd[idx, p] += wv
    return Wd


@pytest.mark.parametrize("dim,g", [(1, 12), (2, 9), (3, 7)])
def test_W_matches_brute_force(dim, g):
    lo, hi = -2.0 / (g - 5), -2.0 / (g - 5) + (g - 1) / (g - 5)
    grid = G.Grid([g] * dim, [lo] * dim, [hi] * dim, [0.3] * dim)
    x = np.random.default_rng(dim).random((25, dim))
    np.testing.assert_allclose(grid.W(x).toarray(), _brute_W(grid, x), atol=1e-14)


@pytest.mark.parametrize("dim,g", [(1, 30), (2, 8), (3, 6)])
def test_kuu_matmul_matches_dense_kron(dim, g):
    grid = G.Grid([g] * dim, [0.0] * dim, [1.0] * dim, [0.2, 0.35, 0.5][:dim], 1.7)
    V = np.random.default_rng(1).standard_normal((grid.m, 3))
    Kd = np.zeros((grid.m, grid.m))
    # brute force: kernel between every pair of grid points
    pts = np.stack(np.meshgrid(*[np.linspace(0, 1, g)] * dim, indexing="ij"), -1).reshape(-1, dim)
    d2 = (pts[:, None, :] - pts[None, :, :]) ** 2 / (2 * np.array(grid.lengthscale) ** 2)
    Kd = 1.7 * np.exp(-d2.sum(-1))
    np.testing.assert_allclose(grid.dense_kuu(), Kd, atol=1e-13)
    np.testing.assert_allclose(grid.kuu_matmul(V), Kd @ V, atol=1e-12)
    # derivative w.r.t. lengthscale e, against central differences of K
    for e in range(dim):
        hh = 1e-6
        gp = G.Grid(grid.size, grid.lo, grid.hi, list(grid.lengthscale), 1.7)
        gm = G.Grid(grid.size, grid.lo, grid.hi, list(grid.lengthscale), 1.7)
        gp.lengthscale[e] += hh
        gm.lengthscale[e] -= hh
        fd = (gp.dense_kuu() - gm.dense_kuu()) / (2 * hh)
        np.testing.assert_allclose(grid.dense_kuu(deriv_dim=e), fd, atol=1e-7)
        np.testing.assert_allclose(grid.kuu_matmul(V, deriv_dim=e), fd @ V, atol=1e-6)


def test_long_mode_uses_fft_toeplitz_consistently():
    g = 2500                                         # > 2048 -> matmul_toeplitz path
    grid = G.Grid([g], [0.0], [1.0], [0.01])
    v = np.random.default_rng(2).standard_normal(g)
    dense = scipy.linalg.toeplitz(grid.toeplitz_col(0)) @ v
    np.testing.assert_allclose(grid.kuu_matmul(v), dense, atol=1e-11)


@pytest.mark.parametrize("dim,g", [(1, 20), (2, 9), (3, 7)])
def test_local_prior_equals_dense_quadratic_form(dim, g):
    lo, hi = -2.0 / (g - 5), -2.0 / (g - 5) + (g - 1) / (g - 5)
    grid = G.Grid([g] * dim, [lo] * dim, [hi] * dim, [0.25] * dim, 1.3)
    x = np.random.default_rng(3).random((17, dim))
    Wd = grid.W(x).toarray()
    Kd = grid.dense_kuu()
    np.testing.assert_allclose(grid.local_kernel_quadform(x),
                               np.einsum("mt,mn,nt->t", Wd, Kd, Wd), atol=1e-13)
    for e in range(dim):
        dWd = grid.W(x, deriv_dim=e).toarray()
        np.testing.assert_allclose(grid.local_kernel_quadform(x, deriv_x=e),
                                   np.einsum("mt,mn,nt->t", dWd, Kd, Wd), atol=1e-10)
        Kl = grid.dense_kuu(deriv_dim=e)
        np.testing.assert_allclose(grid.local_kernel_quadform(x, deriv_l=e),
                                   np.einsum("mt,mn,nt->t", Wd, Kl, Wd), atol=1e-11)


def test_interior_grid_rule_covers_unit_interval():
    import workloads
    for wl in workloads.CONFIGS:
        grid = G.grid_from_workload(wl)
        edge = np.array([[0.0] * wl.dim, [1.0] * wl.dim, [1 - 1e-7] * wl.dim])
        grid.interp(edge)                             # raises on a domain error
