"""GPU parity of the sampler pre-compute (Sec. 3.3) at the precision and path
the 1-D n = 1e6 workload runs: an FP32 cache, whose K_UU - Rt Rt^T is
indefinite well above the rounding level, so T' is not positive definite and
both sides take the root of T''s positive part (the oracle's eigen fallback).

Same cache: love_sampler_precompute runs the GPU sampler on a cache imported
from the oracle (Rt rounded to FP32), and the oracle's sampler runs on the same
rounded Rt, so both see the same operator M = K_UU - Rt Rt^T and the same
SplitMix64 probe.  The GPU's Lanczos run and the eigenpairs of T' are FP64
(their rounding moves the root covariance by ~1e-12 of its scale), so the root
covariances W*^T S S^T W* agree to the FP32 arithmetic of the root itself:
  * S = Q' B (B = V diag(sqrt(lam_+)), B B^T = T'_+) is formed in FP32: entry-wise
    |dS| <= gamma |Q'| |B| with gamma = k' 2^-24, so
    |dS^T w| <= gamma |B|_F |Q'|_F |w| <= gamma sqrt(tr T'_+) sqrt(k') |w|,
    and with tr T'_+ <= sqrt(k') |T'_+|_F and |S^T w| <= sqrt(|T'_+|_F) |w| a
    covariance entry moves by at most 2 gamma k'^(3/4) |T'_+|_F |w_i| |w_j|,
    below 2 k'^2 2^-24 |T'_+|_F |w_i| |w_j|;
  * S stored in FP32: a relative 2^-24 per element, 2^-23 |S^T w_i| |S^T w_j| on a product.
Pipeline: the GPU's own FP32 cache against the oracle's FP64 one.  The two
operators differ by the FP32 error of C = Rt Rt^T, which the variance parity
bounds by 1e-6 p per quadratic form; on the oracle alone, rounding Rt to FP32
(|dC| ~ 1e-7 p) moves the root covariance by up to 10x that, so the pipeline
bound is 10 x 1e-6 sqrt(p_i p_j).
Samples: the empirical covariance of s samples from the root differs from
W*^T S S^T W* by sampling noise only; its element-wise mean absolute error
(the measure of the paper's Sec. 4 sampling table) is compared with the
expected value of that noise.
"""
import numpy as np
import pytest

import workloads
from gpu_util import rounded_cache

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEED = 1234


@pytest.fixture(scope="module")
def love():
    import __graft_entry__ as g
    g.build()
    import paper_1803_06058_gb300 as pkg
    return pkg


def _oracle(wl):
    from oracle import grid as og
    from oracle import love as ol
    from oracle import ski as os_
    x = wl.x_train()
    y = wl.y_train(x)
    grid = og.grid_from_workload(wl)
    return x, y, grid, ol.precompute(os_.SKI(grid, x, wl.noise, y), k=wl.k, want_mean=False)


def _root_cov(Ws, S):
    G = Ws.T @ S
    return G @ G.T, G


def _same_cache_check(love, wl, xs, ks):
    """GPU sampler on the oracle's FP32-rounded cache vs the oracle sampler on it."""
    from oracle import love as ol
    _, _, grid, c_o = _oracle(wl)
    rc = rounded_cache(c_o, "f32")
    S_o, fb_o = ol.sampler_precompute(rc, k=ks, seed=SEED)
    dev = love.love_cache_import(wl.grid_size, wl.grid_lo, wl.grid_hi, wl.lengthscale, wl.outputscale,
                                 wl.noise, rc.Rt, dtype="f32")
    love.love_sampler_precompute(dev, k=ks, seed=SEED)
    inf = dev.info()
    S_g = love.love_cache_export(dev)["S"]
    # an FP32 cache makes K_UU - Rt Rt^T indefinite: both take the positive-part root
    assert fb_o and inf["sampler_fallback"] == 1
    assert inf["sampler_k"] == S_o.shape[1] == ks
    Ws = grid.W(xs)
    cov_o, G_o = _root_cov(Ws, S_o)
    cov_g, _ = _root_cov(Ws, S_g)
    wn = np.sqrt(np.asarray(Ws.multiply(Ws).sum(axis=0)).ravel())       # |w_i|_2
    gn = np.linalg.norm(G_o, axis=1)                                      # |S^T w_i|
    tplus_f = np.linalg.norm(S_o.T @ S_o)                                 # |T'_+|_F
    tol = 2 * ks ** 2 * 2.0 ** -24 * tplus_f * np.outer(wn, wn) + 2.0 ** -23 * np.outer(gn, gn)
    err = np.abs(cov_g - cov_o)
    scale = np.max(np.diag(cov_o))
    print(f"{wl.name}: same-cache root covariance max|d|/max diag {err.max() / scale:.3e}, "
          f"max |d|/tol {np.max(err / tol):.3e}")
    assert np.all(np.isfinite(S_g))
    assert np.all(err <= tol)


def test_sampler_same_fp32_cache_scaled_1d(love):
    """n = 1e5, m = 2,000, k = k' = 100: the 1-D n = 1e6 workload's structure at a
    size whose T' the oracle and the GPU both find indefinite."""
    wl = workloads.C2.scaled(n=100_000, grid_size=[2000], t=300, name="C2-scaled-n1e5-m2e3")
    _same_cache_check(love, wl, wl.x_test(), 100)


def test_sampler_same_fp32_cache_fullsize_1d(love):
    """The full 1-D n = 1e6, m = 1e4, k = k' = 100 workload, at 1,000 of the
    sample points."""
    wl = workloads.C2
    _same_cache_check(love, wl, wl.x_sample(1000), 100)


def _pipeline_check(love, wl, xs, ks):
    from oracle import love as ol
    x, y, grid, c_o = _oracle(wl)
    S_o, _ = ol.sampler_precompute(c_o, k=ks, seed=SEED)
    ski = love.ski_build(torch.tensor(x, dtype=torch.float32, device="cuda"),
                         torch.tensor(y, dtype=torch.float32, device="cuda"), wl.grid_size, wl.grid_lo,
                         wl.grid_hi, wl.lengthscale, wl.outputscale, wl.noise)
    cache = love.love_precompute(ski, k=wl.k, want_mean=True, want_sampler=True, sampler_k=ks,
                                 sampler_seed=SEED, reorth="lowsync")
    inf = cache.info()
    S_g = love.love_cache_export(cache)["S"]
    Ws = grid.W(xs)
    cov_o, _ = _root_cov(Ws, S_o)
    cov_g, _ = _root_cov(Ws, S_g)
    p = ol.prior(grid, xs)
    rel = np.abs(cov_g - cov_o) / np.sqrt(np.outer(p, p))
    print(f"{wl.name}: pipeline root covariance max |d|/sqrt(p p') {rel.max():.3e} "
          f"(covariance scale {np.max(np.diag(cov_o)) / p.max():.3e} p), GPU fallback {inf['sampler_fallback']}")
    assert inf["sampler_fallback"] == 1
    assert np.all(np.diag(cov_g) >= 0) and np.all(np.diag(cov_g) <= p)
    assert rel.max() <= 10 * 1e-6
    return cache, cov_g


def test_sampler_pipeline_scaled_1d(love):
    wl = workloads.C2.scaled(n=100_000, grid_size=[2000], t=300, name="C2-scaled-n1e5-m2e3")
    _pipeline_check(love, wl, wl.x_test(), 100)


def test_sampler_pipeline_fullsize_1d_and_sample_covariance(love):
    """Full size, in the bench's launch configuration (k = k' = 100, s = 1,000
    samples at 10,000 points); root covariance on 1,000 of the points, and the
    samples' empirical covariance against the root's on the same points."""
    wl = workloads.C2
    xs_all = wl.x_sample()
    idx = np.random.default_rng(5).choice(xs_all.shape[0], 1000, replace=False)
    cache, cov_g = _pipeline_check(love, wl, xs_all[idx], 100)
    s = wl.s
    F = love.love_sample(cache, torch.tensor(xs_all, dtype=torch.float32, device="cuda"), s,
                         seed=77).double().cpu().numpy()
    assert F.shape == (s, xs_all.shape[0]) and np.all(np.isfinite(F))
    emp = np.cov(F[:, idx].T)
    mae = np.mean(np.abs(emp - cov_g))
    d = np.diag(cov_g)
    # E|emp_ij - cov_ij| for Gaussian samples: sqrt(2/pi) sqrt((c_ii c_jj + c_ij^2) / (s - 1))
    expect = np.mean(np.sqrt(2 / np.pi) * np.sqrt((np.outer(d, d) + cov_g ** 2) / (s - 1)))
    print(f"sample covariance MAE {mae:.3e} vs sampling noise {expect:.3e} (mean variance {d.mean():.3e})")
    assert mae <= 1.2 * expect
