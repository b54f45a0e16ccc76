"""GPU parity of the batched Lanczos run behind love_precompute_batched for 1-D
FP32 batches (one launch per phase per step over a ragged chunk list of all
GPs, the steps captured into one CUDA graph):

  * each GP's variances and means against its own love_precompute cache: both
    are FP32 runs of the same algorithm (Sec. 2.2 Lanczos with full
    reorthogonalisation, Sec. 3 cache) whose rounding differs (the K_UU product
    is a real-input split FFT in double-float here, and the summation orders
    differ), so they agree to twice the 1-D FP32 variance tolerance,
    |d var| / p <= 2e-6, and take the same number of steps;
  * two GPs against the FP64 oracle's LOVE at the same k: |d var| / p <= 1e-6,
    the single-GP bound;
  * ragged k: a GP with m < k stops by m steps beside GPs that run up to k, and
    every GP takes the single-GP run's number of steps (breakdown included);
  * both reorthogonalisation forms (two passes always / detection);
  * the sweep chunk size is one of the tuner's candidates;
  * a batch holding a 2-D GP runs per GP (bitwise the love_precompute cache).
"""
import numpy as np
import pytest

import workloads
from gpu_util import gpu_ski, oracle_cache, small_workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K = 32


@pytest.fixture(scope="module")
def love():
    import __graft_entry__ as g
    g.build()
    import paper_1803_06058_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def members():
    ms = workloads.C5.members(count=9, n_hi=20_000, t=1200)
    # a GP whose grid is smaller than k: k_eff = m = 24
    ms.append(small_workload(dim=1, g=24, n=3000, ls=0.2, noise=0.02, k=K, t=1200, seed_index=77))
    return ms


def _var(love, cache, x, want_mean=True):
    xt = torch.tensor(np.asarray(x, np.float32), device="cuda")
    m, v = love.love_predict_mean_var(cache, xt, want_mean=want_mean)
    return (m.double().cpu().numpy() if want_mean else None), v.double().cpu().numpy()


@pytest.mark.parametrize("reorth", ["always", "detect"])
def test_batched_lanczos_matches_single(love, members, reorth):
    from oracle import love as ol
    skis = [gpu_ski(love, torch, wl) for wl in members]
    caches, keff = love.love_precompute_batched(skis, k=K, want_mean=True, reorth=reorth, workers=4)
    for b, wl in enumerate(members):
        inf = caches[b].info()
        assert inf["batched_rows"] in (256, 512, 1024, 2048)
        c1 = love.love_precompute(skis[b], k=K, want_mean=True, reorth=reorth)
        # the same step count, breakdown included (smooth kernels exhaust the Krylov space early)
        assert c1.info()["k_eff"] == keff[b] <= min(K, wl.grid_size[0])
        xs = wl.x_test()[:1200]
        mb, vb = _var(love, caches[b], xs)
        m1, v1 = _var(love, c1, xs)
        from oracle import grid as og
        p = ol.prior(og.grid_from_workload(wl), xs)
        d = np.max(np.abs(vb - v1) / p)
        print(f"{wl.name}: m = {wl.grid_size[0]}, n = {wl.n}, batched vs single max |dvar|/p {d:.2e}")
        assert d <= 2e-6
        assert np.max(np.abs(mb - m1)) <= 2e-5 * max(1.0, np.max(np.abs(m1)))


def test_batched_lanczos_matches_oracle(love, members):
    from oracle import grid as og
    from oracle import love as ol
    picks = [0, len(members) - 1]
    skis = [gpu_ski(love, torch, members[b]) for b in picks]
    caches, keff = love.love_precompute_batched(skis, k=K, want_mean=False, reorth="always")
    for i, b in enumerate(picks):
        wl = members[b]
        _, c_o = oracle_cache(wl, k=keff[i], want_mean=False)
        xs = wl.x_test()[:1200]
        _, v_o = ol.predict(c_o, xs)
        _, vb = _var(love, caches[i], xs, want_mean=False)
        p = ol.prior(og.grid_from_workload(wl), xs)
        d = np.max(np.abs(vb - v_o) / p)
        print(f"{wl.name}: batched vs oracle max |dvar|/p {d:.2e}")
        assert d <= 1e-6


def test_batch_with_a_2d_gp_runs_per_gp(love, members):
    wl2 = small_workload(dim=2, g=20, n=4000, k=K, t=500)
    skis = [gpu_ski(love, torch, members[0]), gpu_ski(love, torch, wl2)]
    caches, keff = love.love_precompute_batched(skis, k=K, want_mean=True)
    for b in range(2):
        assert caches[b].info()["batched_rows"] == 0
        c1 = love.love_precompute(skis[b], k=K, want_mean=True)
        e1, e2 = love.love_cache_export(c1), love.love_cache_export(caches[b])
        np.testing.assert_array_equal(e1["Rt"], e2["Rt"])
        np.testing.assert_array_equal(e1["a"], e2["a"])
