"""GPU parity of the SKI operator, the K_UU FFT product and the LOVE test phase.

Every call goes through the C ABI (liblove.so) via the binding; every expected
value comes from the FP64 oracle on the same seeded inputs.

Tolerances (derived from the arithmetic):
  FP64 path: relative 1e-11 (FFT of length N adds ~log2(N) * 1e-16 per stage).
  FP32 K_UU / SKI products: |err| <= 2e-6 * (|K| |v|) -- FP32 FFT of length N
    has error ~ log2(N) * 2^-24 relative to the largest term.
  FP32 predict on an imported cache: the oracle evaluates the same FP32-rounded
    cache in FP64, so only the kernel's arithmetic differs.  Each v_c is a sum of
    4^d FP32 products, so |d v_c| <= gamma_{4^d} (|w|^T |R_c|) with
    gamma_n ~ n 2^-24, and |d |v|^2| <= 2 gamma_{4^d} |w|_1^2 p (|w|_1 <= 1.25^d).
    Asserted: |d var| / p <= 6e-7 (d = 1), 3e-6 (d = 2), 1.5e-5 (d = 3); the
    observed errors are ~5-10x below these worst-case bounds.
"""
import numpy as np
import pytest

from gpu_util import gpu_ski, oracle_cache, oracle_ski, rounded_cache, small_workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def love():
    import __graft_entry__ as g
    g.build()
    import paper_1803_06058_gb300 as pkg
    return pkg


@pytest.mark.parametrize("dim,g", [(1, 100), (1, 3000), (1, 10000), (2, 64), (3, 20)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_kuu_fft_product_matches_oracle(love, dim, g, dtype):
    wl = small_workload(dim=dim, g=g, n=500, dtype=dtype)
    ski = gpu_ski(love, torch, wl)
    grid = oracle_ski(wl).grid
    v = np.random.default_rng(1).standard_normal(grid.m)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    vt = torch.tensor(v, dtype=tdt, device="cuda")
    if dtype == "f32":
        v = vt.double().cpu().numpy()
    out = love.ski_mvm_kuu(ski, vt).double().cpu().numpy()
    ref = grid.kuu_matmul(v)
    scale = np.abs(grid.kuu_matmul(np.abs(v))).max()
    tol = 1e-11 if dtype == "f64" else 2e-6
    assert np.max(np.abs(out - ref)) <= tol * scale


@pytest.mark.parametrize("dim,g,n", [(1, 100, 1000), (1, 10000, 20000), (2, 40, 5000), (3, 16, 4000)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_ski_mvm_matches_oracle(love, dim, g, n, dtype):
    wl = small_workload(dim=dim, g=g, n=n, dtype=dtype)
    ski = gpu_ski(love, torch, wl)
    oski = oracle_ski(wl)
    v = np.random.default_rng(2).standard_normal(n)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    vt = torch.tensor(v, dtype=tdt, device="cuda")
    v = vt.double().cpu().numpy()
    out = love.ski_mvm(ski, vt).double().cpu().numpy()
    ref = oski.mvm(v)
    scale = np.abs(oski.mvm(np.abs(v))).max()
    tol = 1e-11 if dtype == "f64" else 3e-6
    assert np.max(np.abs(out - ref)) <= tol * scale


def test_ski_build_rejects_points_outside_the_grid(love):
    wl = small_workload(dim=1, g=40, n=100)
    x = wl.x_train()
    x[7] = 1.5
    with pytest.raises(love.LoveError, match="DOMAIN"):
        gpu_ski(love, torch, wl, x=x)


def _import(love, wl, cache, cdt, prior_exact=False):
    return love.love_cache_import(wl.grid_size, wl.grid_lo, wl.grid_hi, wl.lengthscale,
                                  wl.outputscale, wl.noise, cache.Rt, a=cache.a, dtype=wl.dtype,
                                  cache_dtype=cdt, prior_exact=prior_exact)


@pytest.mark.parametrize("dim,g,n,k", [(1, 60, 3000, 25), (2, 24, 3000, 30), (3, 12, 3000, 30)])
@pytest.mark.parametrize("cdt", ["f32", "bf16"])
def test_predict_on_imported_cache_fp32(love, dim, g, n, k, cdt):
    wl = small_workload(dim=dim, g=g, n=n, k=k, t=4097)
    _, c = oracle_cache(wl)
    rc = rounded_cache(c, cdt)
    dev = _import(love, wl, rc, cdt)
    xs = wl.x_test()
    mean, var = love.love_predict_mean_var(dev, torch.tensor(xs, dtype=torch.float32, device="cuda"))
    from oracle import love as ol
    xs32 = np.asarray(xs, np.float32).astype(np.float64)
    m_ref, v_ref = ol.predict(rc, xs32)
    p = ol.prior(rc.grid, xs32)
    v_ref_c = np.maximum(v_ref, 0.0)
    tol = {1: 6e-7, 2: 3e-6, 3: 1.5e-5}[dim]
    got = var.double().cpu().numpy()
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - v_ref_c) / p) <= tol
    mtol = 4e-6 * (np.abs(rc.a).max())
    assert np.max(np.abs(mean.double().cpu().numpy() - m_ref)) <= mtol


@pytest.mark.parametrize("dim,g,n,k", [(1, 60, 2000, 25), (2, 20, 2000, 30), (3, 10, 2000, 20)])
def test_predict_on_imported_cache_fp64(love, dim, g, n, k):
    wl = small_workload(dim=dim, g=g, n=n, k=k, t=1000, dtype="f64")
    _, c = oracle_cache(wl)
    dev = _import(love, wl, c, "f64")
    xs = wl.x_test()
    mean, var = love.love_predict_mean_var(dev, torch.tensor(xs, device="cuda"))
    from oracle import love as ol
    m_ref, v_ref = ol.predict(c, xs)
    np.testing.assert_allclose(var.cpu().numpy(), v_ref, rtol=1e-10, atol=1e-15)
    np.testing.assert_allclose(mean.cpu().numpy(), m_ref, rtol=1e-11, atol=1e-13)


def test_predict_edge_cases(love):
    wl = small_workload(dim=1, g=50, n=1500, k=15, t=33)
    _, c = oracle_cache(wl)
    rc = rounded_cache(c, "f32")
    dev = _import(love, wl, rc, "f32")
    # t = 0 is a no-op
    e = torch.empty((0, 1), device="cuda")
    m0, v0 = love.love_predict_mean_var(dev, e)
    assert v0.numel() == 0
    # nodes exactly, the ends of [0, 1], and points outside
    h = (wl.grid_hi[0] - wl.grid_lo[0]) / (wl.grid_size[0] - 1)
    pts = np.array([0.0, 1.0, wl.grid_lo[0] + 10 * h, 0.5, -0.5, 2.0, np.nan, 0.25])
    pts32 = np.asarray(pts, np.float32).astype(np.float64)
    mean, var = love.love_predict_mean_var(dev, torch.tensor(pts32, dtype=torch.float32, device="cuda").reshape(-1, 1))
    got = var.double().cpu().numpy()
    bad = [4, 5, 6]
    assert np.all(np.isnan(got[bad])) and np.all(np.isnan(mean.double().cpu().numpy()[bad]))
    st = dev.device_status(reset=True)
    assert st["domain_errors"] == 3 and st["bits"] & (1 << 2)
    from oracle import love as ol
    good = [0, 1, 2, 3, 7]
    _, v_ref = ol.predict(rc, pts32[good])
    p = ol.prior(rc.grid, pts32[good])
    assert np.max(np.abs(got[good] - np.maximum(v_ref, 0)) / p) <= 6e-7
    assert dev.device_status()["domain_errors"] == 0


def test_predict_exact_prior(love):
    wl = small_workload(dim=2, g=16, n=1500, k=20, t=500)
    wl.outputscale = 1.7
    _, c = oracle_cache(wl)
    rc = rounded_cache(c, "f32")
    dev = _import(love, wl, rc, "f32", prior_exact=True)
    xs = np.asarray(wl.x_test(), np.float32).astype(np.float64)
    _, var = love.love_predict_mean_var(dev, torch.tensor(xs, dtype=torch.float32, device="cuda"))
    from oracle import love as ol
    _, v_ref = ol.predict(rc, xs, prior_mode="exact")
    assert np.max(np.abs(var.double().cpu().numpy() - np.maximum(v_ref, 0)) / 1.7) <= 3e-6
