"""ski_mvm_kuu_noalloc: the K_UU product for callers that cannot allocate.

Real-time loops that forbid allocator calls (an allocation can block or
synchronise the device), frameworks that have reserved all device memory, and
code inside the caching allocator's own callbacks use this entry point; its FFT
scratch is a fixed file-scope device array (4 MiB) instead of memory from the
handle's allocator.  This file is collected
last, so a failure here leaves every other test already run.  The test passes
alone in a fresh process and after the other tests: the first call on a device
looks up the array's address, every later call reuses it.
"""
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


@pytest.mark.parametrize("dim,g", [(1, 10000), (1, 100), (2, 64)])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_noalloc_matches_allocating_entry_point_twice(love, dim, g, dtype):
    wl = small_workload(dim=dim, g=g, n=500, dtype=dtype)
    ski = gpu_ski(love, torch, wl)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    tol = 1e-11 if dtype == "f64" else 2e-6
    rng = np.random.default_rng(7)
    for _ in range(2):                                  # two calls in a row share the scratch
        v = torch.tensor(rng.standard_normal(ski.m), dtype=tdt, device="cuda")
        ref = love.ski_mvm_kuu(ski, v)
        got = love.ski_mvm_kuu_noalloc(ski, v)
        scale = ref.abs().max().item()
        assert (got - ref).abs().max().item() <= tol * scale


def test_noalloc_rejects_grids_beyond_the_scratch(love):
    wl = small_workload(dim=1, g=300000, n=200)         # N = 2^20 complex doubles > 4 MiB
    ski = gpu_ski(love, torch, wl)
    v = torch.zeros(ski.m, dtype=torch.float32, device="cuda")
    with pytest.raises(love.LoveError, match="UNSUPPORTED"):
        love.ski_mvm_kuu_noalloc(ski, v)
