"""Pins for the oracle's Lanczos, LOVE pre-compute, predict and exact posterior.

What the paper and the mathematics fix (Sec. 2.1, 2.2, 3.2, Algorithm 1):
Q orthonormal and T tridiagonal, q_1 = b/|b|, T positive definite, k = n
Lanczos reproducing the exact (SKI) variance, 0 <= var <= prior, and three
independent evaluations of the exact SKI posterior agreeing with one another
and with a closed form at n = 1.
"""
import numpy as np
import pytest
import scipy.linalg

import workloads
from oracle import exact as E
from oracle import grid as G
from oracle import lanczos as LZ
from oracle import love as L
from oracle import ski as S


def _small(dim=1, g=24, n=300, ls=0.15, noise=0.05, seed=0, outputscale=1.0):
    lo, hi = -2.0 / (g - 5), -2.0 / (g - 5) + (g - 1) / (g - 5)
    grid = G.Grid([g] * dim, [lo] * dim, [hi] * dim, [ls] * dim, outputscale)
    rng = np.random.default_rng(seed)
    x = rng.random((n, dim))
    y = np.sin(2 * np.pi * x[:, 0]) + 0.1 * rng.standard_normal(n)
    return S.SKI(grid, x, noise, y), rng.random((40, dim))


def test_ski_mvm_matches_dense_and_probe_is_average_column():
    ski, _ = _small(dim=2, g=9, n=120)
    A = ski.dense()
    v = np.random.default_rng(5).standard_normal(ski.n)
    np.testing.assert_allclose(ski.mvm(v), A @ v, atol=1e-12)
    WtK = ski.W.toarray().T @ ski.grid.dense_kuu()
    np.testing.assert_allclose(ski.probe(), WtK.mean(axis=1), atol=1e-14)


def test_lanczos_structure():
    ski, _ = _small(n=400, g=30)
    b = ski.probe()
    Q, a, bt, _ = LZ.lanczos(ski.mvm, b, 12)
    k = Q.shape[0]
    np.testing.assert_allclose(Q[0], b / np.linalg.norm(b), atol=1e-15)
    assert np.max(np.abs(Q @ Q.T - np.eye(k))) < 1e-12
    T = LZ.tridiag_dense(a, bt)
    QAQ = Q @ np.stack([ski.mvm(q) for q in Q]).T
    scale = np.max(np.abs(QAQ))
    assert np.max(np.abs(QAQ - T)) < 1e-10 * scale            # tridiagonal, = T
    assert np.all(np.linalg.eigvalsh(T) > 0)                   # T is PD (Sec. 3.2)
    d, e = LZ.tridiag_cholesky(a, bt)
    Lm = LZ.bidiag_dense(d, e)
    np.testing.assert_allclose(Lm @ Lm.T, T, atol=1e-10 * scale)


def test_lanczos_ritz_values_on_known_spectrum():
    lam = np.linspace(1.0, 50.0, 40)
    D = np.diag(lam)
    b = np.ones(40)
    Q, a, bt, blast = LZ.lanczos(lambda v: D @ v, b, 40)
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(LZ.tridiag_dense(a, bt))), lam, atol=1e-9)
    assert blast < 1e-8


def test_tridiag_cholesky_rejects_indefinite():
    with pytest.raises(LZ.NotPositiveDefinite):
        LZ.tridiag_cholesky(np.array([1.0, 1.0]), np.array([2.0]))


def test_cg_matches_dense_solve():
    ski, _ = _small(n=200)
    x, it, res = LZ.cg(ski.mvm, ski.y, tol=1e-13)
    np.testing.assert_allclose(x, np.linalg.solve(ski.dense(), ski.y), rtol=1e-9, atol=1e-9)
    assert res <= 1e-13


def test_lanczos_single_solve_at_exhaustion():
    """eq. lanczos_single_solve: A^{-1} b = |b| Q T^{-1} e_1 after exhaustion."""
    ski, _ = _small(n=150, g=20)
    b = ski.probe()
    Q, a, bt, _ = LZ.lanczos(ski.mvm, b, 150)
    T = LZ.tridiag_dense(a, bt)
    e1 = np.zeros(T.shape[0]); e1[0] = 1
    approx = np.linalg.norm(b) * Q.T @ np.linalg.solve(T, e1)
    np.testing.assert_allclose(approx, np.linalg.solve(ski.dense(), b), rtol=1e-8)


@pytest.mark.parametrize("dim,g,n", [(1, 24, 300), (2, 8, 250), (3, 6, 200)])
def test_exact_posterior_three_ways_agree(dim, g, n):
    ski, xs = _small(dim=dim, g=g, n=n)
    md, vd = E.exact_dense(ski, xs)
    mp, vp = E.exact_pushthrough(ski, xs)
    vc = E.exact_cg(ski, xs[:8])
    np.testing.assert_allclose(vp, vd, rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(vc, vd[:8], rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(mp, md, atol=1e-10)


def test_exact_posterior_closed_form_one_training_point():
    """n = 1: var = p - (w*^T K w_1)^2 / (w_1^T K w_1 + s^2)."""
    ski, xs = _small(n=1, g=16)
    Kd = ski.grid.dense_kuu()
    w1 = ski.W.toarray()[:, 0]
    Ws = ski.grid.W(xs).toarray()
    p = np.einsum("mt,mn,nt->t", Ws, Kd, Ws)
    closed = p - (Ws.T @ Kd @ w1) ** 2 / (w1 @ Kd @ w1 + ski.noise)
    _, vd = E.exact_dense(ski, xs)
    _, vp = E.exact_pushthrough(ski, xs)
    np.testing.assert_allclose(vd, closed, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(vp, closed, rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("dim,g,n", [(1, 24, 300), (2, 8, 250)])
def test_love_reproduces_exact_at_krylov_exhaustion(dim, g, n):
    ski, xs = _small(dim=dim, g=g, n=n)
    c = L.precompute(ski, k=n)                  # runs to breakdown (<= m)
    assert c.k_eff <= ski.grid.m
    m_, v = L.predict(c, xs)
    md, vd = E.exact_dense(ski, xs)
    np.testing.assert_allclose(v, vd, rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(m_, md, atol=1e-9)


def test_love_cache_is_the_papers_R_Rprime():
    """Rt Rt^T = R^T R' with R^T = K W Q and R' = T^{-1} R (Sec. 3.2)."""
    ski, _ = _small(n=200, g=20)
    c = L.precompute(ski, k=8)
    Q, a, bt, _ = LZ.lanczos(ski.mvm, ski.probe(), 8)
    RT = ski.grid.dense_kuu() @ (ski.W.toarray() @ Q.T)         # m x k
    Rp = np.linalg.solve(LZ.tridiag_dense(a, bt), RT.T)           # k x m
    np.testing.assert_allclose(c.Rt @ c.Rt.T, RT @ Rp, atol=1e-10 * np.abs(RT @ Rp).max())


def test_love_bounds_and_monotone_in_k():
    """var_SKI <= var_LOVE(k) <= p, non-increasing in k (nested Krylov spaces)."""
    ski, xs = _small(n=500, g=40, ls=0.08, noise=0.01)
    _, vex = E.exact_pushthrough(ski, xs)
    p = L.prior(ski.grid, xs)
    prev = p.copy()
    for k in (1, 2, 4, 8, 16, 32):
        c = L.precompute(ski, k=k, want_mean=False)
        _, v = L.predict(c, xs)
        assert np.all(v >= vex - 1e-12 * p)
        assert np.all(v <= p + 1e-14)
        assert np.all(v <= prev + 1e-12 * p)
        prev = v


def test_love_error_falls_with_k_on_c1():
    """Fig. 2's shape: the error against the exact variance drops fast in k."""
    wl = workloads.C1
    grid = G.grid_from_workload(wl)
    x = wl.x_train()
    ski = S.SKI(grid, x, wl.noise, wl.y_train(x))
    xs = wl.x_test(200)
    _, vex = E.exact_pushthrough(ski, xs)
    errs = []
    for k in (2, 5, 10, 20, 50):
        c = L.precompute(ski, k=k, want_mean=False)
        _, v = L.predict(c, xs)
        errs.append(np.median(np.abs(v - vex) / vex))
    assert errs[-1] < 1e-8
    assert all(errs[i + 1] <= errs[i] * 1.0001 for i in range(len(errs) - 1))
    assert errs[0] > 1e3 * errs[-1]


def test_exact_prior_mode_uses_outputscale():
    ski, xs = _small(n=100, g=20, outputscale=2.5)
    c = L.precompute(ski, k=10, want_mean=False)
    _, v_ski = L.predict(c, xs)
    _, v_ex = L.predict(c, xs, prior_mode="exact")
    p = ski.grid.local_kernel_quadform(xs)
    np.testing.assert_allclose(v_ex - v_ski, 2.5 - p, atol=1e-13)


def test_cross_covariance_is_the_exact_posterior_covariance_at_exhaustion():
    """predict_cov at Krylov exhaustion equals W1^T (K_UU - C) W2 with C from the
    independent push-through solve; with x1 = x2 it is symmetric PSD and its
    diagonal is the LOVE variance."""
    from oracle import exact as E
    from oracle import love as L
    from oracle import grid as og
    from oracle import ski as os_
    rng = np.random.default_rng(21)
    g = 18
    lo, hi = -2.0 / (g - 5), 1.0 + 2.0 / (g - 5)
    grid = og.Grid([g], [lo], [hi], [0.2], 1.3)
    x = rng.uniform(0, 1, (300, 1))
    ski = os_.SKI(grid, x, 0.05, np.sin(6 * x[:, 0]))
    c = L.precompute(ski, k=300)
    x1 = rng.uniform(0, 1, (40, 1))
    x2 = rng.uniform(0, 1, (25, 1))
    C = E.pushthrough_C(ski)
    target = grid.W(x1).T @ (grid.dense_kuu() - C) @ grid.W(x2)
    got = L.predict_cov(c, x1, x2)
    assert np.max(np.abs(got - target)) < 1e-9 * np.max(np.abs(target))
    S = L.predict_cov(c, x1, x1)
    np.testing.assert_allclose(S, S.T, atol=1e-12)
    assert np.min(np.linalg.eigvalsh(S)) > -1e-10
    np.testing.assert_allclose(np.diag(S), L.predict(c, x1)[1], rtol=1e-9, atol=1e-14)
    # the exact-prior form: outputscale * k on the diagonal
    Se = L.predict_cov(c, x1, x1, prior_mode="exact")
    np.testing.assert_allclose(np.diag(Se), L.predict(c, x1, prior_mode="exact")[1], rtol=1e-9, atol=1e-14)
