"""GPU parity of the batched entry points (many independent 1-D GPs of uneven
size, the 256-GP workload's members at reduced n and t):

  * love_precompute_batched with streams=True (each GP's own love_precompute
    on a pool stream) gives, per GP, the cache love_precompute gives (same
    kernels on another stream: bitwise equal); the batched Lanczos kernels of
    the default form are checked in test_gpu_batched_lanczos.py;
  * love_predict_batched (one launch, autotuned shape) matches per-GP
    love_predict_mean_var to the FP32 variance tolerance |d var| / p <= 1e-6
    (only the lanes-per-point summation order can differ) and two GPs match
    the FP64 oracle LOVE at the same k to the same tolerance;
  * love_sample_batched equals per-GP love_sample with seed + b (bitwise);
  * love_batch_serve replays a captured CUDA graph with identical results;
  * ragged edges: a GP with no test points, a batch of one GP.
"""
import numpy as np
import pytest

import workloads
from gpu_util import oracle_cache

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def love():
    import __graft_entry__ as g
    g.build()
    import paper_1803_06058_gb300 as pkg
    return pkg


def _ski(love, wl):
    x = wl.x_train()
    y = wl.y_train(x)
    return love.ski_build(torch.tensor(x, dtype=torch.float32, device="cuda"),
                          torch.tensor(y, dtype=torch.float32, device="cuda"), wl.grid_size,
                          wl.grid_lo, wl.grid_hi, wl.lengthscale, wl.outputscale, wl.noise)


@pytest.fixture(scope="module")
def batch_setup(love):
    members = workloads.C5.members(count=10, n_hi=20_000, t=1500)
    t_sizes = [wl.t for wl in members]
    t_sizes[3] = 0          # a GP with no test points
    t_sizes[5] = 777        # a ragged chunk tail
    skis = [_ski(love, wl) for wl in members]
    caches, keff = love.love_precompute_batched(skis, k=32, want_mean=True, want_sampler=True, workers=4,
                                                streams=True)
    xs = [np.asarray(wl.x_test()[:t], np.float32).astype(np.float64) for wl, t in zip(members, t_sizes)]
    x_all = torch.tensor(np.concatenate(xs), dtype=torch.float32, device="cuda")
    return members, t_sizes, skis, caches, keff, xs, x_all


def test_precompute_batched_equals_single(love, batch_setup):
    members, t_sizes, skis, caches, keff, xs, x_all = batch_setup
    for b in (0, 4, 9):
        c1 = love.love_precompute(skis[b], k=32, want_mean=True, want_sampler=True)
        assert c1.info()["k_eff"] == keff[b]
        e1, e2 = love.love_cache_export(c1), love.love_cache_export(caches[b])
        np.testing.assert_array_equal(e1["Rt"], e2["Rt"])
        np.testing.assert_array_equal(e1["a"], e2["a"])
        np.testing.assert_array_equal(e1["S"], e2["S"])


def test_predict_batched_matches_single_and_oracle(love, batch_setup):
    from oracle import grid as og
    from oracle import love as ol
    members, t_sizes, skis, caches, keff, xs, x_all = batch_setup
    batch = love.love_batch_create(caches, t_sizes)
    inf = batch.info()
    assert inf["lanes_per_point"] in (4, 8, 16) and inf["ctas_per_sm"] in (4, 8, 16)
    assert len(inf["candidate_ms"]) == 9
    mean, var = love.love_predict_batched(batch, x_all)
    ms, vs = love.batch_split(batch, mean), love.batch_split(batch, var)
    for b, wl in enumerate(members):
        if t_sizes[b] == 0:
            assert vs[b].numel() == 0
            continue
        m1, v1 = love.love_predict_mean_var(caches[b], torch.tensor(xs[b], dtype=torch.float32, device="cuda"))
        p = ol.prior(og.grid_from_workload(wl), xs[b])
        vb = vs[b].double().cpu().numpy()
        assert np.max(np.abs(vb - v1.double().cpu().numpy()) / p) <= 1e-6
        assert torch.allclose(ms[b], m1, rtol=0, atol=1e-6 * float(m1.abs().max()) + 1e-12)
        if b in (0, 7):
            _, c_o = oracle_cache(wl, k=32)
            _, v_ref = ol.predict(c_o, xs[b])
            assert np.max(np.abs(vb - v_ref) / p) <= 1e-6
    for c in caches:
        assert c.device_status()["domain_errors"] == 0


def test_sample_batched_equals_single(love, batch_setup):
    members, t_sizes, skis, caches, keff, xs, x_all = batch_setup
    batch = love.love_batch_create(caches, t_sizes)
    s = 48
    out = love.love_sample_batched(batch, x_all, s, seed=11)
    parts = love.batch_split(batch, out, s=s)
    for b in range(len(members)):
        if t_sizes[b] == 0:
            continue
        ref = love.love_sample(caches[b], torch.tensor(xs[b], dtype=torch.float32, device="cuda"), s, seed=11 + b)
        assert torch.equal(parts[b], ref)


def test_batch_serve_graph_replay(love, batch_setup):
    members, t_sizes, skis, caches, keff, xs, x_all = batch_setup
    batch = love.love_batch_create(caches, t_sizes)
    T = x_all.shape[0]
    s = 16
    mean = torch.empty(T, device="cuda")
    var = torch.empty(T, device="cuda")
    smp = torch.empty(s * T, device="cuda")
    m_ref, v_ref = love.love_predict_batched(batch, x_all)
    s_ref = love.love_sample_batched(batch, x_all, s, seed=3)
    for _ in range(3):          # eager + capture, then two replays
        mean.fill_(0)
        var.fill_(0)
        smp.fill_(0)
        love.love_batch_serve(batch, x_all, mean, var, s=s, seed=3, samples=smp, use_graph=True)
        torch.cuda.synchronize()
        assert torch.equal(mean, m_ref) and torch.equal(var, v_ref) and torch.equal(smp, s_ref)


def test_batch_serve_recaptures_after_work_space_grows(love, batch_setup):
    """A graph captured by love_batch_serve holds the work space's address; a
    love_sample_batched call with more samples grows (moves) that work space, so
    the graph must be dropped and the next serve call capture again: its
    results stay bitwise those of the eager calls."""
    members, t_sizes, skis, caches, keff, xs, x_all = batch_setup
    batch = love.love_batch_create(caches, t_sizes)
    T = x_all.shape[0]
    s = 8
    mean = torch.empty(T, device="cuda")
    var = torch.empty(T, device="cuda")
    smp = torch.empty(s * T, device="cuda")
    m_ref, v_ref = love.love_predict_batched(batch, x_all)
    s_ref = love.love_sample_batched(batch, x_all, s, seed=5)

    def serve_and_check():
        mean.fill_(0)
        var.fill_(0)
        smp.fill_(0)
        love.love_batch_serve(batch, x_all, mean, var, s=s, seed=5, samples=smp, use_graph=True)
        torch.cuda.synchronize()
        assert torch.equal(mean, m_ref) and torch.equal(var, v_ref) and torch.equal(smp, s_ref)

    serve_and_check()                       # eager call + capture
    serve_and_check()                       # replay
    inf = batch.info()
    assert inf["graph_captures"] == 1 and inf["graph_captures_dropped"] == 0
    big = love.love_sample_batched(batch, x_all, 64, seed=9)   # grows the work space
    torch.cuda.synchronize()
    assert batch.info()["graph_captures_dropped"] == 1
    serve_and_check()                       # captures again with the new work space
    serve_and_check()                       # and replays it
    assert batch.info()["graph_captures"] == 2
    ref_big = love.love_sample(caches[0], torch.tensor(xs[0], dtype=torch.float32, device="cuda"), 64, seed=9)
    assert torch.equal(love.batch_split(batch, big, 64)[0], ref_big)


def test_batch_of_one_and_errors(love, batch_setup):
    members, t_sizes, skis, caches, keff, xs, x_all = batch_setup
    b1 = love.love_batch_create([caches[0]], [t_sizes[0]])
    m, v = love.love_predict_batched(b1, x_all[:t_sizes[0]])
    m1, v1 = love.love_predict_mean_var(caches[0], x_all[:t_sizes[0]])
    from oracle import grid as og
    from oracle import love as ol
    p = ol.prior(og.grid_from_workload(members[0]), xs[0])
    assert np.max(np.abs(v.double().cpu().numpy() - v1.double().cpu().numpy()) / p) <= 1e-6
    with pytest.raises(ValueError):
        love.love_predict_batched(b1, x_all)          # wrong number of rows
    c_nomean = love.love_precompute(skis[1], k=8, want_mean=False)
    b2 = love.love_batch_create([c_nomean], [10])
    with pytest.raises(love.LoveError):
        love.love_predict_batched(b2, x_all[:10], want_mean=True)   # LOVE_ERR_STATE
    with pytest.raises(love.LoveError):
        love.love_sample_batched(b2, x_all[:10], 4)                 # no sampler
