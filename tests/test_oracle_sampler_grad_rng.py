"""Pins for the oracle's sampler (Sec. 3.3), gradients and generators.

Sampler: at Krylov exhaustion W*^T S S^T W* equals the exact Cholesky-sampling
covariance W*^T (K - C) W* (eq. pred_covar_ski_interp_form12); the sample
covariance converges to it.  Gradients: central finite differences of the
oracle variance (test points) and of the exact SKI variance at Krylov
exhaustion (hyperparameters).  Generators: published known-answer values.
"""
import numpy as np
import pytest

from oracle import exact as E
from oracle import grid as G
from oracle import love as L
from oracle import rng as R
from oracle import ski as S


def _small(dim=1, g=20, n=300, ls=0.2, noise=0.05, seed=0):
    lo, hi = -2.0 / (g - 5), -2.0 / (g - 5) + (g - 1) / (g - 5)
    grid = G.Grid([g] * dim, [lo] * dim, [hi] * dim, [ls] * dim, 1.0)
    rng = np.random.default_rng(seed)
    x = rng.random((n, dim))
    y = np.sin(2 * np.pi * x[:, 0]) + 0.1 * rng.standard_normal(n)
    return S.SKI(grid, x, noise, y), rng.random((30, dim))


def test_sampler_root_matches_exact_posterior_covariance_at_exhaustion():
    ski, xs = _small(g=20, n=300)
    c = L.precompute(ski, k=300)
    S_, fb = L.sampler_precompute(c, k=ski.grid.m, seed=7, tau=1e-13)
    C = E.pushthrough_C(ski)
    Ws = ski.grid.W(xs).toarray()
    target = Ws.T @ (ski.grid.dense_kuu() - C) @ Ws
    got = Ws.T @ S_ @ S_.T @ Ws
    assert np.max(np.abs(got - target)) < 1e-9 * np.max(np.abs(np.diag(target)))
    # diag equals the LOVE variance there
    _, v = L.predict(c, xs)
    np.testing.assert_allclose(np.diag(got), v, rtol=1e-6, atol=1e-12)


def test_root_variance_is_the_exact_variance_at_exhaustion():
    """|S^T w*|^2 with the posterior root: a sum of squares, and at Krylov
    exhaustion (S S^T = K_UU - C) the exact SKI variance, here computed by the
    independent push-through solve."""
    ski, xs = _small(g=20, n=300)
    c = L.precompute(ski, k=300)
    L.sampler_precompute(c, k=ski.grid.m, seed=7, tau=1e-13)
    _, v_exact = E.exact_pushthrough(ski, xs)
    vr = L.predict_root(c, xs)
    assert np.all(vr >= 0)
    np.testing.assert_allclose(vr, v_exact, rtol=1e-6, atol=1e-9 * np.max(v_exact))


def _positive_part(M, iters=100):
    """M_+ = (M + M sign(M)) / 2, with sign(M) from the Newton iteration
    X <- (X + X^{-1}) / 2 started at M (Higham, Functions of Matrices, Ch. 5):
    no eigensolver, so it shares no step with the sampler's eigen fallback."""
    X = M.copy()
    for _ in range(iters):
        Xn = 0.5 * (X + np.linalg.inv(X))
        done = np.max(np.abs(Xn - X)) <= 1e-15 * np.max(np.abs(Xn))
        X = Xn
        if done:
            break
    return 0.5 * (M + M @ X)


def test_sampler_eigen_fallback_gives_the_positive_part():
    """Sec. 3.3 with T' indefinite: the oracle's fallback root S = Q' V diag(sqrt(max(lam, 0)))
    satisfies S S^T = M_+ (the positive part of M = K_UU - Rt Rt^T) at Krylov exhaustion.
    M is made clearly indefinite by one extra cache column along the eigenvector of
    K_UU - Rt Rt^T's smallest eigenvalue; the grid's lengthscale is short (K_UU
    well conditioned) so M_+ from the Newton sign iteration is accurate to rounding.
    A clamp taken after the square root, |lam| in place of max(lam, 0), or V^T in
    place of V each break the equality."""
    import dataclasses
    g = 24
    ski, _ = _small(g=g, n=400, ls=0.6 / (g - 5), noise=0.05)
    c = L.precompute(ski, k=400)
    K = ski.grid.dense_kuu()
    lam, V = np.linalg.eigh(K - c.Rt @ c.Rt.T)
    shift = 3 * lam[:5].mean() + 0.3 * lam[-1]             # pushes one eigenvalue well below 0
    c2 = dataclasses.replace(c)
    c2.Rt = np.hstack([c.Rt, np.sqrt(shift) * V[:, :1]])
    M = K - c2.Rt @ c2.Rt.T
    assert np.linalg.eigvalsh(M)[0] < -0.1 * lam[-1]
    S_, fb = L.sampler_precompute(c2, k=g, seed=5, tau=1e-14)
    assert fb and S_.shape == (g, g)
    Mp = _positive_part(M)
    # exhaustion: S S^T = Q' T'_+ Q'^T with Q' orthonormal and complete; rounding of
    # the Lanczos run and the eigensolve, ~g eps |M|
    assert np.max(np.abs(S_ @ S_.T - Mp)) <= 1e-12 * np.max(np.abs(Mp))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sampler_eigen_fallback_at_rounding_level_matches_exact_posterior(seed):
    """Sec. 3.3 where T' is indefinite only by rounding (K_UU - Rt Rt^T has eigenvalues
    near -1e-15 |K_UU|, as the root of a real workload does): at Krylov exhaustion
    the fallback root's covariance W*^T S S^T W* equals the exact SKI posterior
    covariance W*^T (K_UU - C) W* of the push-through solve (eq.
    pred_covar_ski_interp_form12), to the same 1e-9 as the positive definite case."""
    ski, xs = _small(g=30, n=3000, ls=0.3, noise=0.01, seed=seed)
    c = L.precompute(ski, k=ski.grid.m, tau=1e-13)
    S_, fb = L.sampler_precompute(c, k=ski.grid.m, seed=7, tau=1e-14)
    assert fb, "this case is meant to take the eigen fallback"
    C = E.pushthrough_C(ski)
    Ws = ski.grid.W(xs).toarray()
    target = Ws.T @ (ski.grid.dense_kuu() - C) @ Ws
    got = Ws.T @ S_ @ S_.T @ Ws
    assert np.all(np.isfinite(S_))
    assert np.max(np.abs(got - target)) < 1e-9 * np.max(np.abs(np.diag(target)))


def test_sample_covariance_converges_and_sample_is_deterministic():
    ski, xs = _small(g=16, n=200, noise=0.1)
    c = L.precompute(ski, k=200)
    S_, _ = L.sampler_precompute(c, k=ski.grid.m, seed=3)
    mu, v = L.predict(c, xs)
    z = np.random.default_rng(11).standard_normal((S_.shape[1], 40000))
    F = L.sample(c, xs, z)
    np.testing.assert_array_equal(F, L.sample(c, xs, z))
    np.testing.assert_allclose(F.mean(0), mu, atol=6 * np.sqrt(v.max() / 40000))
    Ws = ski.grid.W(xs).toarray()
    cov = Ws.T @ S_ @ S_.T @ Ws
    emp = np.cov(F.T)
    assert np.mean(np.abs(emp - cov)) < 0.03 * np.mean(np.abs(np.diag(cov)))


def _fd_points(grid, xs, hfd):
    """Keep points whose FD stencil stays inside one interpolation cell."""
    keep = np.ones(xs.shape[0], bool)
    for e in range(grid.dim):
        s = (xs[:, e] - grid.lo[e]) / grid.h[e]
        f = s - np.floor(s)
        keep &= (f > 2 * hfd / grid.h[e]) & (f < 1 - 2 * hfd / grid.h[e])
    return xs[keep]


@pytest.mark.parametrize("dim,g", [(1, 20), (2, 8)])
def test_grad_x_matches_central_differences(dim, g):
    ski, xs = _small(dim=dim, g=g, n=250)
    c = L.precompute(ski, k=12, want_grad=True)
    hfd = 1e-6
    xs = _fd_points(ski.grid, xs, hfd)
    gvec = np.random.default_rng(4).standard_normal(xs.shape[0])
    gx, _, _ = L.var_grad(c, ski, xs, gvec)
    for e in range(dim):
        xp, xm = xs.copy(), xs.copy()
        xp[:, e] += hfd
        xm[:, e] -= hfd
        fd = (L.predict(c, xp)[1] - L.predict(c, xm)[1]) / (2 * hfd)
        np.testing.assert_allclose(gx[:, e], gvec * fd, rtol=1e-5, atol=1e-8 * np.abs(gvec * fd).max())


def test_grad_x_at_h_1e4_within_truncation_bound():
    """At the stated FD step h = 1e-4 the central-difference truncation error is
    h^2/6 |var'''| <= h^2/6 * C/h_grid^3 * |var|; with h_grid = 1/15 the relative
    error stays under ~1e-3."""
    ski, xs = _small(dim=1, g=20, n=250)
    c = L.precompute(ski, k=12, want_grad=True)
    hfd = 1e-4
    xs = _fd_points(ski.grid, xs, hfd)
    gx, _, _ = L.var_grad(c, ski, xs, np.ones(xs.shape[0]))
    fd = (L.predict(c, xs + hfd)[1] - L.predict(c, xs - hfd)[1]) / (2 * hfd)
    rel = np.abs(gx[:, 0] - fd) / np.maximum(np.abs(fd), 1e-3 * np.abs(fd).max())
    assert np.max(rel) < 1e-3


def _exact_var(grid_kwargs, x, y, noise, xs):
    grid = G.Grid(**grid_kwargs)
    ski = S.SKI(grid, x, noise, y)
    return E.exact_pushthrough(ski, xs)[1]


@pytest.mark.parametrize("prior_mode", ["ski", "exact"])
def test_grad_hyper_matches_fd_of_exact_at_exhaustion(prior_mode):
    """2-D, 12^2 grid, n = 400: LOVE's fixed-Q gradient equals d/dtheta of the
    exact SKI variance when the Krylov space is exhausted."""
    g, dim, n = 12, 2, 400
    lo, hi = -2.0 / (g - 5), -2.0 / (g - 5) + (g - 1) / (g - 5)
    kw = dict(size=[g, g], lo=[lo, lo], hi=[hi, hi], lengthscale=[0.3, 0.22], outputscale=1.0)
    rng = np.random.default_rng(9)
    x = rng.random((n, dim))
    y = rng.standard_normal(n)
    xs = rng.random((25, dim))
    noise = 0.05
    grid = G.Grid(**kw)
    ski = S.SKI(grid, x, noise, y)
    c = L.precompute(ski, k=n, want_grad=True, tau=1e-14)
    gvec = rng.standard_normal(xs.shape[0])
    _, gl, gn = L.var_grad(c, ski, xs, gvec, prior_mode=prior_mode)

    def total(kw_, noise_):
        grid_ = G.Grid(**kw_)
        ski_ = S.SKI(grid_, x, noise_, y)
        return float(gvec @ E.exact_pushthrough(ski_, xs, prior_mode=prior_mode)[1])

    h = 1e-5
    for e in range(dim):
        kp = {**kw, "lengthscale": list(kw["lengthscale"])}
        km = {**kw, "lengthscale": list(kw["lengthscale"])}
        kp["lengthscale"][e] += h
        km["lengthscale"][e] -= h
        fd = (total(kp, noise) - total(km, noise)) / (2 * h)
        assert abs(gl[e] - fd) <= 1e-6 * max(abs(fd), 1e-3)
    fdn = (total(kw, noise + h) - total(kw, noise - h)) / (2 * h)
    assert abs(gn - fdn) <= 1e-6 * max(abs(fdn), 1e-3)


def test_splitmix64_known_answers():
    # SplitMix64 seeded with 0 (Steele et al. 2014): first outputs
    assert R.splitmix64_output(0, 0) == 0xE220A8397B1DCDAF
    assert R.splitmix64_output(0, 1) == 0x6E789E6AA1B965F4
    assert R.splitmix64_output(0, 2) == 0x06C45D188009454F
    v = R.splitmix64_outputs(0, 3)
    assert [int(a) for a in v] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    r = R.rademacher_probe(12345, 100000)
    assert set(np.unique(r)) == {-1.0, 1.0}
    assert abs(r.mean()) < 0.02


def test_philox_known_answers_and_normals():
    # Philox4x32-10 known-answer vectors (Salmon et al. 2011)
    ctr = np.array([[0, 0, 0, 0],
                    [0xFFFFFFFF] * 4,
                    [0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]], dtype=np.uint64)
    key = np.array([[0, 0], [0xFFFFFFFF] * 2, [0xA4093822, 0x299F31D0]], dtype=np.uint64)
    out = R.philox4x32_10(ctr, key)
    exp = np.array([[0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8],
                    [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD],
                    [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]], dtype=np.uint32)
    np.testing.assert_array_equal(out, exp)
    z = R.philox_normals(99, 200001)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
