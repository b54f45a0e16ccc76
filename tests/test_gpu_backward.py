"""GPU parity of love_var_backward (d var / d x*, d/d lengthscale, d/d noise).

The reference is the oracle's var_grad on the same cache (formula derived from
eq. pred_covar_ski_cache with K^^{-1} ~ Q T^{-1} Q^T, Q fixed), itself pinned by
finite differences (test_oracle_sampler_grad_rng.py).

Tolerances: FP64 path 1e-9 relative.  FP32 path: every term is a dot product
of FP32 gathers (4^d products per entry) accumulated in double-float, so the
error is a few 4^d * 2^-24 of the size of the terms that cancel (see _scales);
asserted as |error| <= tol * size with tol = 1e-6 (d = 1), 4e-6 (d = 2), 1.6e-5 (d = 3),
i.e. 16 * 4^(d-1) * 2^-24.
"""
import numpy as np
import pytest

from gpu_util import gpu_ski, oracle_cache, rounded_cache, small_workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def love():
    import __graft_entry__ as g
    g.build()
    import paper_1803_06058_gb300 as pkg
    return pkg


def _import(love, wl, c, dtype, prior_exact=False):
    return love.love_cache_import(wl.grid_size, wl.grid_lo, wl.grid_hi, wl.lengthscale, wl.outputscale,
                                  wl.noise, c.Rt, a=c.a, alpha=c.alpha, beta=c.beta, P=c.P, dtype=dtype,
                                  prior_exact=prior_exact)


def _scales(c, ski_o, xs, g):
    """Size of the terms each gradient is the (nearly cancelling) sum of, for
    FP32 tolerances: the kernel's rounding error is a few 2^-24 of these.
      x:      2 |g_i| |dw_i|^T K |w_i|            (|dw|_1 |w|_1 s_f bound)
      l_e:    sum_i |g_i| (|w_i| + |P| |v_i|)^T K'_e (|w_i| + |P| |v_i|)   (K'_e >= 0)
      noise:  sum_i |g_i| v_i^T L^-1 L^-T v_i       (positive terms)"""
    from oracle import love as ol
    grid = c.grid
    per = grid.interp(xs)
    sx = 0.0
    for e in range(grid.dim):
        b = np.ones(xs.shape[0]) * grid.outputscale
        for f, (_, w, dw) in enumerate(per):
            b = b * np.abs(dw if f == e else w).sum(1)
        sx = max(sx, np.max(2 * np.abs(g) * b))
    Wa = abs(grid.W(xs)).toarray()                                  # m x t
    V = np.abs(grid.W(xs).T @ c.Rt)                                 # t x k
    U = Wa + np.abs(c.P) @ V.T
    sl = max(float(np.abs(g) @ np.sum(U * grid.kuu_matmul(U, deriv_dim=e), axis=0)) for e in range(grid.dim))
    _, _, gn = ol.var_grad(c, ski_o, xs, np.abs(g))
    return sx, sl, abs(gn) + 1e-30


@pytest.mark.parametrize("dim,g", [(1, 40), (2, 14), (3, 8)])
@pytest.mark.parametrize("prior_exact", [False, True])
def test_backward_fp64_imported(love, dim, g, prior_exact):
    from oracle import love as ol
    wl = small_workload(dim=dim, g=g, n=1500, k=16, t=200, dtype="f64", ls=0.2)
    ski_o, c = oracle_cache(wl, want_grad=True)
    dev = _import(love, wl, c, "f64", prior_exact)
    xs = wl.x_test()
    gv = np.random.default_rng(4).standard_normal(xs.shape[0])
    gx, gl, gn = love.love_var_backward(dev, torch.tensor(xs, device="cuda"), torch.tensor(gv, device="cuda"))
    gx_o, gl_o, gn_o = ol.var_grad(c, ski_o, xs, gv, prior_mode="exact" if prior_exact else "ski")
    np.testing.assert_allclose(gx.cpu().numpy(), gx_o, rtol=1e-9, atol=1e-9 * np.abs(gx_o).max())
    np.testing.assert_allclose(gl, gl_o, rtol=1e-8, atol=1e-10 * np.abs(gl_o).max())
    np.testing.assert_allclose(gn, gn_o, rtol=1e-9)


@pytest.mark.parametrize("dim,g", [(1, 60), (2, 20), (3, 10)])
def test_backward_fp32_imported(love, dim, g):
    from oracle import love as ol
    wl = small_workload(dim=dim, g=g, n=2000, k=24, t=500, ls=0.2)
    ski_o, c = oracle_cache(wl, want_grad=True)
    rc = rounded_cache(c, "f32")
    rc.P = np.asarray(np.asarray(c.P, np.float32), np.float64)
    dev = _import(love, wl, rc, "f32")
    xs = np.asarray(wl.x_test(), np.float32).astype(np.float64)
    gv = np.asarray(np.random.default_rng(5).standard_normal(xs.shape[0]), np.float32).astype(np.float64)
    gx, gl, gn = love.love_var_backward(dev, torch.tensor(xs, dtype=torch.float32, device="cuda"),
                                        torch.tensor(gv, dtype=torch.float32, device="cuda"))
    gx_o, gl_o, gn_o = ol.var_grad(rc, ski_o, xs, gv)
    sx, sl, sn = _scales(rc, ski_o, xs, gv)
    tol = {1: 1e-6, 2: 4e-6, 3: 1.6e-5}[dim]
    assert np.max(np.abs(gx.double().cpu().numpy() - gx_o)) <= tol * sx
    assert np.max(np.abs(np.array(gl) - gl_o)) <= tol * sl
    assert abs(gn - gn_o) <= tol * sn


def test_backward_matches_finite_differences_of_gpu_variance(love):
    """FP64: d var/dx* from the kernel vs central differences of the GPU's own
    love_predict_mean_var (points away from interpolation knots)."""
    wl = small_workload(dim=2, g=16, n=2000, k=20, t=300, dtype="f64", ls=0.25)
    ski = gpu_ski(love, torch, wl)
    cache = love.love_precompute(ski, k=20, want_mean=False, want_grad=True)
    xs = wl.x_test()
    h = (wl.grid_hi[0] - wl.grid_lo[0]) / (wl.grid_size[0] - 1)
    fr = ((xs - wl.grid_lo[0]) / h) % 1.0
    xs = xs[np.all((fr > 0.05) & (fr < 0.95), axis=1)]
    gx, _, _ = love.love_var_backward(cache, torch.tensor(xs, device="cuda"),
                                      torch.ones(xs.shape[0], dtype=torch.float64, device="cuda"),
                                      want_hyper=False)
    gx = gx.cpu().numpy()
    hfd = 1e-6
    for e in range(2):
        xp, xm = xs.copy(), xs.copy()
        xp[:, e] += hfd
        xm[:, e] -= hfd
        _, vp = love.love_predict_mean_var(cache, torch.tensor(xp, device="cuda"), want_mean=False)
        _, vm = love.love_predict_mean_var(cache, torch.tensor(xm, device="cuda"), want_mean=False)
        fd = (vp - vm).cpu().numpy() / (2 * hfd)
        np.testing.assert_allclose(gx[:, e], fd, rtol=1e-4, atol=1e-5 * np.abs(fd).max())


def test_backward_pipeline_fp32_scaled_c4(love):
    """The 2-D gradient workload at reduced size: GPU pre-compute with
    want_grad vs the oracle pre-compute and gradient at the same k."""
    from oracle import love as ol
    import workloads
    wl = workloads.C4.scaled(n=20000, t=2000, grid_size=[48, 48], k=32)
    ski_o, c = oracle_cache(wl, want_grad=True)
    ski = gpu_ski(love, torch, wl)
    cache = love.love_precompute(ski, k=32, want_mean=False, want_grad=True)
    xs = np.asarray(wl.x_test(), np.float32).astype(np.float64)
    gv = np.ones(xs.shape[0])
    gx, gl, gn = love.love_var_backward(cache, torch.tensor(xs, dtype=torch.float32, device="cuda"),
                                        torch.ones(xs.shape[0], dtype=torch.float32, device="cuda"))
    gx_o, gl_o, gn_o = ol.var_grad(c, ski_o, xs, gv)
    sx, sl, sn = _scales(c, ski_o, xs, gv)
    # FP32 Lanczos vs FP64 Lanczos: the caches differ at ~1e-7 relative, amplified
    # by the same cancellation as the variance
    assert np.max(np.abs(gx.double().cpu().numpy() - gx_o)) <= 1e-3 * sx
    assert np.max(np.abs(np.array(gl) - gl_o)) <= 1e-3 * sl
    assert abs(gn - gn_o) <= 1e-3 * sn


def test_autograd_function(love):
    wl = small_workload(dim=1, g=40, n=1500, k=16, t=100, dtype="f64", ls=0.2)
    ski = gpu_ski(love, torch, wl)
    cache = love.love_precompute(ski, k=16, want_mean=False, want_grad=True)
    x = torch.tensor(wl.x_test(), device="cuda", requires_grad=True)
    ls = torch.tensor(wl.lengthscale, dtype=torch.float64, device="cuda", requires_grad=True)
    nz = torch.tensor(wl.noise, dtype=torch.float64, device="cuda", requires_grad=True)
    var = love.love_var(cache, x, ls, nz)
    w = torch.linspace(0.5, 1.5, x.shape[0], dtype=torch.float64, device="cuda")
    (var * w).sum().backward()
    gx, gl, gn = love.love_var_backward(cache, x.detach(), w)
    assert torch.allclose(x.grad, gx)
    np.testing.assert_allclose(ls.grad.cpu().numpy(), gl)
    assert abs(nz.grad.item() - gn) <= 1e-12 * abs(gn)
    _, v2 = love.love_predict_mean_var(cache, x.detach(), want_mean=False)
    assert torch.equal(var.detach(), v2)
