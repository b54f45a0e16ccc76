"""GPU parity of the additive composition of one-dimensional kernels (the
paper's Sec. 3 extension, eq. multi_dimensional_kernel_block): stacked
interpolation vectors, block-diagonal K_UU.  Reference: the oracle's
AdditiveGrid, itself pinned against sums of separate 1-D SKI kernels and the
exact posterior (test_oracle_additive.py).  Tolerances as for the product
grids: FP64 1e-9 relative; FP32 |d var| / p <= 2e-6 (a 4d-row gather, d <= 3)."""
import numpy as np
import pytest

from gpu_util import small_workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def love():
    import __graft_entry__ as g
    g.build()
    import paper_1803_06058_gb300 as pkg
    return pkg


def _setup(love, wl, dtype):
    from oracle import grid as og
    from oracle import ski as os_
    x = wl.x_train()
    y = wl.y_train(x)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    ski = love.ski_build(torch.tensor(x, dtype=tdt, device="cuda"), torch.tensor(y, dtype=tdt, device="cuda"),
                         wl.grid_size, wl.grid_lo, wl.grid_hi, wl.lengthscale, wl.outputscale, wl.noise,
                         additive=True)
    npdt = np.float64 if dtype == "f64" else np.float32
    xr = np.asarray(x, npdt).astype(np.float64)
    yr = np.asarray(y, npdt).astype(np.float64)
    grid = og.additive_grid_from_workload(wl)
    return ski, os_.SKI(grid, xr, wl.noise, yr), grid


@pytest.mark.parametrize("dim,g", [(2, 30), (3, 24)])
def test_additive_fp64_pipeline(love, dim, g):
    from oracle import love as ol
    wl = small_workload(dim=dim, g=g, n=3000, k=30, t=500, dtype="f64", ls=0.2)
    ski, ski_o, grid = _setup(love, wl, "f64")
    # the SKI product against the oracle's block form
    v = np.random.default_rng(1).standard_normal(wl.n)
    out = love.ski_mvm(ski, torch.tensor(v, device="cuda")).cpu().numpy()
    np.testing.assert_allclose(out, ski_o.mvm(v), rtol=1e-10, atol=1e-10 * np.abs(out).max())
    c_o = ol.precompute(ski_o, k=30, cg_tol=1e-12)
    cache = love.love_precompute(ski, k=30, want_mean=True)
    assert abs(cache.info()["k_eff"] - c_o.k_eff) <= 1
    xs = wl.x_test()
    m, var = love.love_predict_mean_var(cache, torch.tensor(xs, device="cuda"))
    m_ref, v_ref = ol.predict(c_o, xs)
    np.testing.assert_allclose(var.cpu().numpy(), v_ref, rtol=1e-9)
    np.testing.assert_allclose(m.cpu().numpy(), m_ref, atol=1e-9 * np.std(ski_o.y))
    p = ol.prior(grid, xs)
    assert np.all(var.cpu().numpy() <= p * (1 + 1e-12))


def test_additive_fp32_pipeline_and_sampler(love):
    from oracle import love as ol
    wl = small_workload(dim=2, g=60, n=20000, k=40, t=1000, ls=0.15, noise=0.0025)
    ski, ski_o, grid = _setup(love, wl, "f32")
    c_o = ol.precompute(ski_o, k=40, want_mean=False)
    cache = love.love_precompute(ski, k=40, want_mean=False, want_sampler=True)
    xs = np.asarray(wl.x_test(), np.float32).astype(np.float64)
    _, var = love.love_predict_mean_var(cache, torch.tensor(xs, dtype=torch.float32, device="cuda"),
                                        want_mean=False)
    _, v_ref = ol.predict(c_o, xs)
    p = ol.prior(grid, xs)
    err = np.abs(var.double().cpu().numpy() - v_ref) / p
    print(f"additive 2-D FP32: |dvar|/p max {err.max():.3e} median {np.median(err):.3e}")
    assert err.max() <= 2e-6
    # samples through the root: their covariance diagonal is |S^T w|^2 >= 0
    vr = love.love_predict_var_root(cache, torch.tensor(xs, dtype=torch.float32, device="cuda"))
    assert torch.all(vr >= 0)
    F = love.love_sample(cache, torch.tensor(xs[:200], dtype=torch.float32, device="cuda"), 64, seed=3)
    assert F.shape == (64, 200) and torch.all(torch.isfinite(F))


def test_additive_sampler_fp64_matches_oracle(love):
    from oracle import love as ol
    wl = small_workload(dim=2, g=20, n=1500, k=20, t=200, dtype="f64", ls=0.25)
    ski, ski_o, grid = _setup(love, wl, "f64")
    c_o = ol.precompute(ski_o, k=20, want_mean=False)
    cache = love.love_precompute(ski, k=20, want_mean=False, want_sampler=True, sampler_k=24, sampler_seed=5)
    S_o, _ = ol.sampler_precompute(c_o, k=24, seed=5)
    xs = wl.x_test()
    Ws = grid.W(xs)
    cov_o = (Ws.T @ S_o) @ (Ws.T @ S_o).T
    ks = cache.info()["sampler_k"]
    Z = np.random.default_rng(7).standard_normal((ks, 4000))
    F = love.love_sample(cache, torch.tensor(xs, device="cuda"), 4000, z=torch.tensor(Z, device="cuda"))
    ex = love.love_cache_export(cache)
    G = Ws.T @ ex["S"][:, :ks]
    np.testing.assert_allclose(F.cpu().numpy(), (G @ Z).T, atol=1e-9 * np.abs(G @ Z).max())
    cov_g = G @ G.T
    assert np.max(np.abs(cov_g - cov_o)) <= 1e-7 * np.max(np.abs(np.diag(cov_o)))


def test_additive_unsupported_calls_and_save_load(love, tmp_path):
    wl = small_workload(dim=2, g=20, n=1000, k=10, t=50, dtype="f64", ls=0.25)
    ski, _, _ = _setup(love, wl, "f64")
    cache = love.love_precompute(ski, k=10, want_mean=False)
    xs = torch.tensor(wl.x_test(), device="cuda")
    with pytest.raises(love.LoveError):
        love.love_predict_covariance(cache, xs)
    with pytest.raises(love.LoveError):
        love.love_precompute(ski, k=10, want_mean=False, want_grad=True)
    path = str(tmp_path / "add.love")
    love.love_cache_save(cache, path)
    c2 = love.love_cache_load(path)
    _, v1 = love.love_predict_mean_var(cache, xs, want_mean=False)
    _, v2 = love.love_predict_mean_var(c2, xs, want_mean=False)
    assert torch.equal(v1, v2)
