"""GPU parity of love_predict_covariance (posterior cross-covariances, eq.
pred_covar_ski_fast with i != j) against the oracle's predict_cov on the same
(rounded) imported cache.

Tolerance: each entry is p - v1 . v2 with v = Rt^T w gathered in FP32 over 4^d
cache rows and the dot product on the split-TF32 tensor path (~FP32), so the
error is a few 4^d 2^-24 of sqrt(p_i p_j) (the size of the cancelling terms):
FP32 1e-6 (d = 1), 4e-6 (d = 2), 1.6e-5 (d = 3); FP64 1e-10.
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
    data = "f32" if dtype == "bf16" else dtype
    return love.love_cache_import(wl.grid_size, wl.grid_lo, wl.grid_hi, wl.lengthscale, wl.outputscale,
                                  wl.noise, c.Rt, a=c.a, dtype=data, cache_dtype=dtype, prior_exact=prior_exact)


@pytest.mark.parametrize("dim,g", [(1, 60), (2, 18), (3, 9)])
@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16"])
def test_covariance_on_imported_cache(love, dim, g, dtype):
    from oracle import love as ol
    wl = small_workload(dim=dim, g=g, n=1500, k=20, t=300, dtype="f64" if dtype == "f64" else "f32", ls=0.2)
    _, c = oracle_cache(wl)
    rc = rounded_cache(c, dtype)
    dev = _import(love, wl, rc, dtype)
    tdt = np.float64 if dtype == "f64" else np.float32
    x = np.asarray(wl.x_test(), tdt)
    x1, x2 = x[:130], x[130:300]
    cov = love.love_predict_covariance(dev, torch.tensor(x1, device="cuda"), torch.tensor(x2, device="cuda"))
    assert cov.shape == (130, 170)
    ref = ol.predict_cov(rc, x1.astype(np.float64), x2.astype(np.float64))
    p1 = ol.prior(rc.grid, x1.astype(np.float64))
    p2 = ol.prior(rc.grid, x2.astype(np.float64))
    scale = np.sqrt(np.outer(p1, p2))
    tol = 1e-10 if dtype == "f64" else {1: 1e-6, 2: 4e-6, 3: 1.6e-5}[dim]
    assert np.max(np.abs(cov.double().cpu().numpy() - ref) / scale) <= tol


def test_covariance_diagonal_is_the_variance_and_symmetric(love):
    """With x1 = x2: symmetric up to rounding, and the diagonal equals the
    variance of love_predict_mean_var (FP32 pipeline)."""
    from oracle import love as ol
    from oracle import grid as og
    wl = small_workload(dim=2, g=32, n=20000, k=40, t=600, ls=0.2, noise=0.0025)
    ski = gpu_ski(love, torch, wl)
    cache = love.love_precompute(ski, k=40, want_mean=False)
    x = torch.tensor(np.asarray(wl.x_test(), np.float32), device="cuda")
    cov = love.love_predict_covariance(cache, x).double().cpu().numpy()
    _, var = love.love_predict_mean_var(cache, x, want_mean=False)
    p = ol.prior(og.grid_from_workload(wl), x.double().cpu().numpy())
    assert np.max(np.abs(np.diag(cov) - var.double().cpu().numpy()) / p) <= 4e-6
    assert np.max(np.abs(cov - cov.T) / np.sqrt(np.outer(p, p))) <= 4e-6


def test_covariance_exact_prior_and_domain_errors(love):
    from oracle import love as ol
    wl = small_workload(dim=1, g=40, n=1000, k=16, t=50, dtype="f64", ls=0.2)
    _, c = oracle_cache(wl)
    dev = _import(love, wl, c, "f64", prior_exact=True)
    x = np.asarray(wl.x_test(), np.float64)
    cov = love.love_predict_covariance(dev, torch.tensor(x, device="cuda")).cpu().numpy()
    ref = ol.predict_cov(c, x, x, prior_mode="exact")
    np.testing.assert_allclose(cov, ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())
    bad = x.copy()
    bad[3, 0] = 5.0                               # far outside the grid
    cov = love.love_predict_covariance(dev, torch.tensor(bad, device="cuda")).cpu().numpy()
    assert np.all(np.isnan(cov[3, :])) and np.all(np.isnan(cov[:, 3]))
    assert np.all(np.isfinite(np.delete(np.delete(cov, 3, 0), 3, 1)))
    assert dev.device_status()["domain_errors"] > 0
    e = love.love_predict_covariance(dev, torch.tensor(x[:0], device="cuda"), torch.tensor(x, device="cuda"))
    assert e.shape == (0, x.shape[0])
