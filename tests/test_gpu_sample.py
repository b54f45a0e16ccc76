"""GPU parity of the sampler (Sec. 3.3) against the FP64 oracle.

* Pre-compute, FP64 (1-D, m = 100): the GPU and the oracle run the same
  Lanczos on K_UU - Rt Rt^T from the same SplitMix64 Rademacher probe, so the
  roots S agree element by element (Cholesky of T' is unique) and so do the
  samples for the same Z.
* Test phase on an imported root: love_sample(Z) = mu + W*^T S Z computed by
  the oracle on the same (rounded) S, mu and Z.
* On-device normals: Philox4x32-10 + Box-Muller against the oracle's
  generator (FP64 Box-Muller, rounded to the dtype).
* FP32 pipeline: the sample covariance of many samples converges to
  W*^T S S^T W* and its diagonal to the LOVE variance.
"""
import numpy as np
import pytest

import workloads
from gpu_util import gpu_ski, oracle_cache, rounded_cache, small_workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def love():
    import __graft_entry__ as g
    g.build()
    import paper_1803_06058_gb300 as pkg
    return pkg


def test_sampler_fp64_matches_oracle(love):
    from oracle import love as ol
    wl = small_workload(dim=1, g=40, n=800, k=30, t=300, dtype="f64", ls=0.15, noise=0.01)
    _, c_o = oracle_cache(wl)
    S_o, fb_o = ol.sampler_precompute(c_o, k=20, seed=77)
    ski = gpu_ski(love, torch, wl)
    cache = love.love_precompute(ski, k=30, want_mean=True, want_sampler=True, sampler_k=20, sampler_seed=77)
    inf = cache.info()
    ex = love.love_cache_export(cache)
    assert inf["sampler_fallback"] == int(fb_o)
    xs = wl.x_test()
    Ws = c_o.grid.W(xs).toarray()
    cov_o = Ws.T @ S_o @ S_o.T @ Ws
    cov_g = Ws.T @ ex["S"] @ ex["S"].T @ Ws
    assert np.max(np.abs(cov_g - cov_o)) <= 1e-8 * np.max(np.abs(np.diag(cov_o)))
    if not fb_o:
        kk = min(S_o.shape[1], ex["S"].shape[1])
        np.testing.assert_allclose(ex["S"][:, :kk], S_o[:, :kk], atol=1e-8 * np.abs(S_o).max())
        Z = np.random.default_rng(3).standard_normal((inf["sampler_k"], 64))
        F = love.love_sample(cache, torch.tensor(xs, device="cuda"), 64,
                             z=torch.tensor(Z, device="cuda")).cpu().numpy()
        c_o.S = S_o[:, : inf["sampler_k"]]
        F_o = ol.sample(c_o, xs, Z)
        np.testing.assert_allclose(F, F_o, atol=1e-8 * np.abs(F_o).max())


@pytest.mark.parametrize("dim,g", [(1, 50), (2, 16), (3, 8)])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_sample_on_imported_root(love, dim, g, dtype):
    from oracle import love as ol
    wl = small_workload(dim=dim, g=g, n=1500, k=20, t=333, dtype=dtype, ls=0.25)
    _, c_o = oracle_cache(wl)
    S_o, _ = ol.sampler_precompute(c_o, k=24, seed=5)
    rc = rounded_cache(c_o, dtype)
    rc.S = np.asarray(np.asarray(S_o, np.float32 if dtype == "f32" else np.float64), np.float64)
    dev = love.love_cache_import(wl.grid_size, wl.grid_lo, wl.grid_hi, wl.lengthscale, wl.outputscale,
                                 wl.noise, rc.Rt, a=rc.a, S=rc.S, dtype=dtype)
    ks = rc.S.shape[1]
    s = 129
    tdt = torch.float32 if dtype == "f32" else torch.float64
    Z = np.asarray(np.random.default_rng(9).standard_normal((ks, s)), np.float32 if dtype == "f32" else np.float64)
    xs = np.asarray(wl.x_test(), np.float32 if dtype == "f32" else np.float64)
    F = love.love_sample(dev, torch.tensor(xs, device="cuda"), s, z=torch.tensor(Z, device="cuda"))
    F_o = ol.sample(rc, xs.astype(np.float64), Z.astype(np.float64))
    scale = np.abs(F_o).max()
    tol = 2e-6 if dtype == "f32" else 1e-12
    assert F.shape == (s, xs.shape[0])
    assert np.max(np.abs(F.double().cpu().numpy() - F_o)) <= tol * scale * (4 ** dim)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_device_normals_match_philox_oracle(love, dtype):
    from oracle import love as ol
    from oracle import rng
    wl = small_workload(dim=1, g=30, n=500, k=10, t=50, dtype=dtype)
    _, c_o = oracle_cache(wl)
    S_o, _ = ol.sampler_precompute(c_o, k=12, seed=1)
    rc = rounded_cache(c_o, dtype)
    rc.S = np.asarray(np.asarray(S_o, np.float32 if dtype == "f32" else np.float64), np.float64)
    dev = love.love_cache_import(wl.grid_size, wl.grid_lo, wl.grid_hi, wl.lengthscale, wl.outputscale,
                                 wl.noise, rc.Rt, a=rc.a, S=rc.S, dtype=dtype)
    ks, s, seed = rc.S.shape[1], 37, 0xABCDEF12345
    xs = np.asarray(wl.x_test(), np.float32 if dtype == "f32" else np.float64)
    F = love.love_sample(dev, torch.tensor(xs, device="cuda"), s, seed=seed).double().cpu().numpy()
    Z = rng.philox_normals(seed, ks * s).reshape(ks, s)
    Z = np.asarray(Z, np.float32 if dtype == "f32" else np.float64).astype(np.float64)
    F_o = ol.sample(rc, xs.astype(np.float64), Z)
    tol = 2e-6 if dtype == "f32" else 1e-12
    assert np.max(np.abs(F - F_o)) <= tol * np.abs(F_o).max()


def test_fp32_pipeline_sample_covariance(love):
    """FP32 pipeline: samples' empirical covariance converges to W*^T S S^T W*, and the
    root's diagonal matches the LOVE variance (Sec. 3.3, eq. pred_covar_ski_interp_form12) within the FP32 tolerance."""
    wl = small_workload(dim=1, g=60, n=3000, k=30, t=40, ls=0.1, noise=0.01)
    ski = gpu_ski(love, torch, wl)
    cache = love.love_precompute(ski, k=30, want_mean=True, want_sampler=True, sampler_k=40, sampler_seed=3)
    ex = love.love_cache_export(cache)
    xs = np.asarray(wl.x_test(), np.float32)
    xt = torch.tensor(xs, device="cuda")
    mean, var = love.love_predict_mean_var(cache, xt)
    s = 20000
    F = love.love_sample(cache, xt, s, seed=11).double().cpu().numpy()
    from oracle import grid as og
    Ws = og.grid_from_workload(wl).W(xs.astype(np.float64)).toarray()
    cov = Ws.T @ ex["S"] @ ex["S"].T @ Ws
    v = var.double().cpu().numpy()
    p = __import__("oracle").love.prior(og.grid_from_workload(wl), xs.astype(np.float64))
    assert np.max(np.abs(np.diag(cov) - v) / p) <= 5e-6
    np.testing.assert_allclose(F.mean(0), mean.double().cpu().numpy(), atol=8 * np.sqrt(v.max() / s))
    emp = np.cov(F.T)
    assert np.mean(np.abs(emp - cov)) <= 0.05 * np.mean(np.diag(cov))


def test_sample_edge_cases(love):
    wl = small_workload(dim=1, g=30, n=500, k=10, t=50)
    ski = gpu_ski(love, torch, wl)
    cache = love.love_precompute(ski, k=10, want_mean=True, want_sampler=False)
    with pytest.raises(love.LoveError, match="STATE"):
        love.love_sample(cache, torch.zeros((4, 1), device="cuda"), 3)
    cache = love.love_precompute(ski, k=10, want_mean=True, want_sampler=True)
    out = love.love_sample(cache, torch.zeros((0, 1), device="cuda"), 5)
    assert out.shape == (5, 0)
    bad = torch.tensor([[0.5], [2.0], [0.25]], device="cuda")
    F = love.love_sample(cache, bad, 4, seed=1).cpu().numpy()
    assert np.all(np.isnan(F[:, 1])) and np.all(np.isfinite(F[:, [0, 2]]))


@pytest.mark.parametrize("dim,g", [(1, 50), (2, 16), (3, 8)])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_variance_from_root_on_imported_root(love, dim, g, dtype):
    """love_predict_var_root = |S^T w*|^2 against the oracle on the same
    (rounded) root.  A sum of squares: relative error of a 4^d-row FP32 gather
    and a k'-term FP32 sum, (4^d + k') 2^-24 < 1e-5; FP64 1e-12."""
    from oracle import love as ol
    wl = small_workload(dim=dim, g=g, n=1500, k=20, t=333, dtype=dtype, ls=0.25)
    _, c_o = oracle_cache(wl)
    S_o, _ = ol.sampler_precompute(c_o, k=24, seed=5)
    rc = rounded_cache(c_o, dtype)
    rc.S = np.asarray(np.asarray(S_o, np.float32 if dtype == "f32" else np.float64), np.float64)
    dev = love.love_cache_import(wl.grid_size, wl.grid_lo, wl.grid_hi, wl.lengthscale, wl.outputscale,
                                 wl.noise, rc.Rt, a=rc.a, S=rc.S, dtype=dtype)
    xs = np.asarray(wl.x_test(), np.float32 if dtype == "f32" else np.float64)
    v = love.love_predict_var_root(dev, torch.tensor(xs, device="cuda")).double().cpu().numpy()
    v_o = ol.predict_root(rc, xs.astype(np.float64))
    tol = 1e-5 if dtype == "f32" else 1e-12
    np.testing.assert_allclose(v, v_o, rtol=tol, atol=tol * v_o.max() * 1e-3)


def test_variance_from_root_pipeline_properties(love):
    """FP32 pipeline with the sampler: 0 <= |S^T w*|^2 <= p, and without a
    sampler the call is refused (LOVE_ERR_STATE)."""
    from oracle import love as ol
    from oracle import grid as og
    wl = small_workload(dim=1, g=200, n=20000, k=40, t=2000, ls=0.1, noise=0.0025)
    ski = gpu_ski(love, torch, wl)
    cache = love.love_precompute(ski, k=40, want_mean=False, want_sampler=True)
    xs = np.asarray(wl.x_test(), np.float32)
    v = love.love_predict_var_root(cache, torch.tensor(xs, device="cuda")).double().cpu().numpy()
    p = ol.prior(og.grid_from_workload(wl), xs.astype(np.float64))
    assert np.all(v >= 0) and np.all(v <= p * (1 + 1e-5))
    c2 = love.love_precompute(ski, k=10, want_mean=False)
    with pytest.raises(love.LoveError):
        love.love_predict_var_root(c2, torch.tensor(xs, device="cuda"))
