"""love_predict_mean_var_host (the predict call on host buffers) against the
device-buffer call on the same cache: page-locked buffers are read and written
by the kernel over the CPU-GPU link, pageable ones go through device staging
in chunks; either way the kernel is the same, so the results are identical."""
import numpy as np
import pytest

from gpu_util import gpu_ski, small_workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def love():
    import __graft_entry__ as g
    g.build()
    import paper_1803_06058_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def cache(love):
    wl = small_workload(dim=2, g=24, n=4000, k=20, t=5000, ls=0.2)
    ski = gpu_ski(love, torch, wl)
    return wl, love.love_precompute(ski, k=20, want_mean=True)


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("want_mean", [True, False])
def test_host_buffers_match_device_buffers(love, cache, pinned, want_mean):
    wl, c = cache
    x = torch.tensor(np.asarray(wl.x_test(), np.float32))
    if pinned:
        x = x.pin_memory()
    m_d, v_d = love.love_predict_mean_var(c, x.cuda(), want_mean=want_mean)
    m_h, v_h = love.love_predict_mean_var_host(c, x, want_mean=want_mean)
    assert v_h.device.type == "cpu" and v_h.is_pinned() == pinned
    assert torch.equal(v_h, v_d.cpu())
    if want_mean:
        assert torch.equal(m_h, m_d.cpu())
    else:
        assert m_h is None


def test_host_buffers_in_chunks_and_empty(love, cache):
    """More points than one staging chunk (2^20) on pageable memory, and t = 0."""
    wl, c = cache
    rng = np.random.default_rng(5)
    x = torch.tensor(rng.uniform(0, 1, (1_200_000, 2)).astype(np.float32))
    _, v_h = love.love_predict_mean_var_host(c, x, want_mean=False)
    _, v_d = love.love_predict_mean_var(c, x.cuda(), want_mean=False)
    assert torch.equal(v_h, v_d.cpu())
    _, v0 = love.love_predict_mean_var_host(c, x[:0], want_mean=False)
    assert v0.shape == (0,)
