"""Full-size parity on the 1-D, n = 1e6, m = 1e4, k = 100, FP32 workload, in the
launch configuration bench.py times: the GPU cache and all 1e6 predictive
variances are checked by properties that hold at any size (finite, 0 <= var <= p,
k_eff = k), and every one of the 1e6 variances against the FP64 oracle LOVE run
on the same data at the same k (|d var| / p <= 1e-6, the FP32 tolerance; the
oracle's O(k) predict runs on the host in chunks of 1e5 points)."""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def love():
    import __graft_entry__ as g
    g.build()
    import paper_1803_06058_gb300 as pkg
    return pkg


def test_c2_fullsize_variances(love):
    from oracle import grid as og
    from oracle import love as ol
    from oracle import ski as os_
    wl = workloads.C2
    x = wl.x_train()
    y = wl.y_train(x)
    xs = wl.x_test()
    ski = love.ski_build(torch.tensor(x, dtype=torch.float32, device="cuda"),
                         torch.tensor(y, dtype=torch.float32, device="cuda"), wl.grid_size,
                         wl.grid_lo, wl.grid_hi, wl.lengthscale, wl.outputscale, wl.noise)
    cache = love.love_precompute(ski, k=wl.k, want_mean=True)
    assert cache.info()["k_eff"] == wl.k
    mean, var = love.love_predict_mean_var(cache, torch.tensor(xs, dtype=torch.float32, device="cuda"))
    v = var.double().cpu().numpy()
    grid = og.grid_from_workload(wl)
    p = ol.prior(grid, xs)
    assert np.all(np.isfinite(v)) and np.all(np.isfinite(mean.cpu().numpy()))
    assert np.all(v >= 0) and np.all(v <= p * (1 + 1e-6))
    assert cache.device_status()["domain_errors"] == 0
    # oracle on the same data, same k, FP64
    oc = ol.precompute(os_.SKI(grid, x, wl.noise, y), k=wl.k, want_mean=False)
    v_ref = np.empty_like(v)
    for a in range(0, xs.shape[0], 100_000):
        _, v_ref[a:a + 100_000] = ol.predict(oc, xs[a:a + 100_000])
    err = np.abs(v - v_ref) / p
    rel = np.abs(v - v_ref) / v_ref
    print(f"C2 all {xs.shape[0]} points: |dvar|/p max {err.max():.3e} median {np.median(err):.3e}; "
          f"relative median {np.median(rel):.3e}; var/p median {np.median(v_ref / p):.3e}")
    assert err.max() <= 1e-6


def test_c2_fullsize_mean(love):
    """Predictive mean of the full-size workload (Sec. 3, eq. pred_mean_ski)
    against the oracle's exact SKI mean by the push-through identity (one dense
    m x m solve, m = 1e4) at 2,000 sampled test points: |d mu| <= 1e-4 std(y),
    the FP32 mean tolerance; the CG stopping rule bounds the error of the
    fitted values at the training points by 1e-6 |y|."""
    from oracle import exact as oe
    from oracle import grid as og
    from oracle import ski as os_
    wl = workloads.C2
    x = wl.x_train()
    y = wl.y_train(x)
    ski = love.ski_build(torch.tensor(x, dtype=torch.float32, device="cuda"),
                         torch.tensor(y, dtype=torch.float32, device="cuda"), wl.grid_size,
                         wl.grid_lo, wl.grid_hi, wl.lengthscale, wl.outputscale, wl.noise)
    cache = love.love_precompute(ski, k=8, want_mean=True)
    inf = cache.info()
    assert 0 < inf["cg_iters"] < 4000
    xs = wl.x_test()
    idx = np.random.default_rng(1).choice(xs.shape[0], 2000, replace=False)
    xs = np.asarray(xs[idx], np.float32).astype(np.float64)
    mu, _ = love.love_predict_mean_var(cache, torch.tensor(xs, dtype=torch.float32, device="cuda"))
    grid = og.grid_from_workload(wl)
    xr = np.asarray(x, np.float32).astype(np.float64)
    yr = np.asarray(y, np.float32).astype(np.float64)
    a = oe.mean_weights_pushthrough(os_.SKI(grid, xr, wl.noise, yr))
    mu_ref = grid.W(xs).T @ a
    err = np.abs(mu.double().cpu().numpy() - mu_ref) / np.std(yr)
    print(f"C2 mean: cg_iters {inf['cg_iters']}, |d mu|/std(y) max {err.max():.3e} median {np.median(err):.3e}")
    assert err.max() <= 1e-4
