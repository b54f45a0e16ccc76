"""GPU parity of the LOVE pre-compute (Lanczos with full reorthogonalisation,
tridiagonal Cholesky, cache build, mean CG) against the FP64 oracle.

FP64 path: the GPU runs the same algorithm in the same precision; variances
agree to 1e-9 relative (Lanczos rounding grows ~ k eps cond(T)).
FP32 path: Lanczos vectors and MVMs in FP32 with double-float dot products;
variances are compared as |d var| / p <= 1e-6 (the scaled error of the
paper's SMAE, Sec. 4), because var / p ~ 1e-4..1e-7 makes FP32 cancellation
error dominate any relative measure; the relative error is asserted only on
a sparse-data case where var >= 1e-2 p.
"""
import numpy as np
import pytest

import workloads
from gpu_util import gpu_ski, oracle_cache, small_workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def love():
    import __graft_entry__ as g
    g.build()
    import paper_1803_06058_gb300 as pkg
    return pkg


def _predict(love, cache, xs, dtype):
    tdt = torch.float64 if dtype == "f64" else torch.float32
    has_mean = bool(cache.info()["flags"] & love.WANT_MEAN)
    m, v = love.love_predict_mean_var(cache, torch.tensor(xs, dtype=tdt, device="cuda"), want_mean=has_mean)
    return (m.double().cpu().numpy() if has_mean else None), v.double().cpu().numpy()


def test_c1_fp64_pipeline_matches_oracle(love):
    from oracle import love as ol
    wl = workloads.C1
    ski_o, c_o = oracle_cache(wl, cg_tol=1e-12)
    ski = gpu_ski(love, torch, wl)
    cache = love.love_precompute(ski, k=wl.k, want_mean=True)
    inf = cache.info()
    assert abs(inf["k_eff"] - c_o.k_eff) <= 1
    xs = wl.x_test()
    m, v = _predict(love, cache, xs, "f64")
    m_ref, v_ref = ol.predict(c_o, xs)
    np.testing.assert_allclose(v, v_ref, rtol=1e-9)
    np.testing.assert_allclose(m, m_ref, atol=1e-9)
    ex = love.love_cache_export(cache)
    kk = min(inf["k_eff"], c_o.k_eff)
    np.testing.assert_allclose(ex["alpha"][:kk], c_o.alpha[:kk], rtol=1e-9)
    C_gpu = ex["Rt"] @ ex["Rt"].T
    C_ref = c_o.Rt @ c_o.Rt.T
    assert np.max(np.abs(C_gpu - C_ref)) <= 1e-9 * np.max(np.abs(C_ref))


@pytest.mark.parametrize("dim,g,n,k", [(1, 200, 20000, 40), (2, 32, 20000, 40), (3, 14, 20000, 40)])
def test_fp32_pipeline_matches_oracle(love, dim, g, n, k):
    from oracle import love as ol
    wl = small_workload(dim=dim, g=g, n=n, k=k, t=2000, ls=0.1 if dim == 1 else 0.2, noise=0.0025)
    ski_o, c_o = oracle_cache(wl)
    ski = gpu_ski(love, torch, wl)
    cache = love.love_precompute(ski, k=k, want_mean=True)
    xs = np.asarray(wl.x_test(), np.float32).astype(np.float64)
    m, v = _predict(love, cache, xs, "f32")
    m_ref, v_ref = ol.predict(c_o, xs)
    p = ol.prior(c_o.grid, xs)
    assert np.all(v >= 0) and np.all(v <= p * (1 + 1e-6))
    assert np.max(np.abs(v - v_ref) / p) <= 1e-6
    ystd = np.std(ski_o.y)
    assert np.max(np.abs(m - m_ref)) <= 1e-4 * ystd


def test_fp32_relative_error_on_sparse_data(love):
    """n = 200, s^2 = 0.3: var >= 1e-2 p, so relative error is meaningful (<= 1e-4)."""
    from oracle import love as ol
    wl = small_workload(dim=1, g=64, n=200, k=40, t=1000, ls=0.05, noise=0.3)
    _, c_o = oracle_cache(wl)
    ski = gpu_ski(love, torch, wl)
    cache = love.love_precompute(ski, k=wl.k, want_mean=False)
    xs = np.asarray(wl.x_test(), np.float32).astype(np.float64)
    _, v = _predict(love, cache, xs, "f32")
    _, v_ref = ol.predict(c_o, xs)
    p = ol.prior(c_o.grid, xs)
    assert np.min(v_ref / p) >= 1e-2
    assert np.max(np.abs(v - v_ref) / v_ref) <= 1e-4


def test_fp32_variance_non_increasing_in_k_and_bounded(love):
    wl = small_workload(dim=1, g=120, n=8000, k=40, t=3000, ls=0.08, noise=0.01)
    ski = gpu_ski(love, torch, wl)
    xs = np.asarray(wl.x_test(), np.float32).astype(np.float64)
    from oracle import grid as og
    from oracle import love as ol
    p = ol.prior(og.grid_from_workload(wl), xs)
    prev = None
    for k in (4, 8, 16, 32):
        cache = love.love_precompute(ski, k=k, want_mean=False)
        _, v = _predict(love, cache, xs, "f32")
        assert np.all(v >= 0) and np.all(v <= p * (1 + 1e-6))
        if prev is not None:
            assert np.all(v <= prev + 1e-6 * p)
        prev = v


def test_breakdown_is_reported_through_k_eff(love):
    """A Krylov space of dimension < k (m = 30 grid points) ends the Lanczos run
    early; the returned cache has k_eff < k columns and still matches."""
    from oracle import love as ol
    wl = small_workload(dim=1, g=30, n=3000, k=60, t=500, dtype="f64", ls=0.2)
    _, c_o = oracle_cache(wl)
    ski = gpu_ski(love, torch, wl)
    cache = love.love_precompute(ski, k=60, want_mean=False)
    assert cache.info()["k_eff"] < 60
    xs = wl.x_test()
    _, v = _predict(love, cache, xs, "f64")
    _, v_ref = ol.predict(c_o, xs)
    np.testing.assert_allclose(v, v_ref, rtol=1e-8)


def test_cache_save_load_roundtrip(love, tmp_path):
    wl = small_workload(dim=2, g=16, n=3000, k=12, t=300)
    ski = gpu_ski(love, torch, wl)
    cache = love.love_precompute(ski, k=12, want_mean=True)
    path = str(tmp_path / "c.love")
    love.love_cache_save(cache, path)
    c2 = love.love_cache_load(path)
    a, b = love.love_cache_export(cache), love.love_cache_export(c2)
    np.testing.assert_array_equal(a["Rt"], b["Rt"])
    np.testing.assert_array_equal(a["a"], b["a"])
    np.testing.assert_array_equal(a["alpha"], b["alpha"])
    xs = torch.tensor(wl.x_test(), dtype=torch.float32, device="cuda")
    m1, v1 = love.love_predict_mean_var(cache, xs)
    m2, v2 = love.love_predict_mean_var(c2, xs)
    assert torch.equal(v1, v2) and torch.equal(m1, m2)


def test_cache_load_refuses_a_corrupted_header(love, tmp_path):
    """A saved cache whose leading dimension field is changed (offset 144 of the
    224-byte header) no longer matches its buffer sizes: the load is refused
    before anything reaches the device, and the intact file (mean, sampler root
    and gradient tables) still loads."""
    import struct
    wl = small_workload(dim=1, g=40, n=2000, k=10, t=100)
    ski = gpu_ski(love, torch, wl)
    cache = love.love_precompute(ski, k=10, want_mean=True, want_sampler=True, want_grad=True)
    path = tmp_path / "c.love"
    love.love_cache_save(cache, str(path))
    raw = bytearray(path.read_bytes())
    assert raw[:8] == b"LOVECACH"
    ld = struct.unpack_from("<i", raw, 144)[0]
    assert ld == -(-(cache.info()["k_eff"] + 1) // 4) * 4
    bad = tmp_path / "bad.love"
    struct.pack_into("<i", raw, 144, ld + 4)
    bad.write_bytes(bytes(raw))
    with pytest.raises(love.LoveError):
        love.love_cache_load(str(bad))
    c2 = love.love_cache_load(str(path))
    a, b = love.love_cache_export(cache), love.love_cache_export(c2)
    for key in ("Rt", "a", "S", "P", "alpha"):
        np.testing.assert_array_equal(a[key], b[key])
