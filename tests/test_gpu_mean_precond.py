"""GPU checks of the preconditioned grid-space mean solve (1-D grids): the mean
cache a = K_UU W K^^{-1} y of eq. pred_mean_ski, solved by right-preconditioned
GMRES with the spectral approximation of (B K_UU + s^2 I)^{-1}, reaches the
same solution as the plain CG of Sec. 2.1 (both accept an iterate only when
r^T K r <= tol^2 s^2 |y|^2, checked exactly), in far fewer iterations.
Tolerances: FP32 |d mu| <= 1e-4 std(y) (the FP32 mean tolerance); FP64 1e-8
std(y): the stopping rule at the FP64 default tol = 1e-12 leaves mean errors of
~1e-9 std(y) on these problems (both solvers stop on the same rule, at
different points below it)."""
import numpy as np
import pytest

import workloads
from gpu_util import gpu_ski, small_workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def love():
    import __graft_entry__ as g
    g.build()
    import paper_1803_06058_gb300 as pkg
    return pkg


def _mean_ref(wl, x, y, xs):
    from oracle import exact as oe
    from oracle import grid as og
    from oracle import ski as os_
    grid = og.grid_from_workload(wl)
    a = oe.mean_weights_pushthrough(os_.SKI(grid, x, wl.noise, y))
    return grid.W(xs).T @ a


def _mean(love, cache, xs, dtype):
    tdt = torch.float64 if dtype == "f64" else torch.float32
    mu, _ = love.love_predict_mean_var(cache, torch.tensor(xs, dtype=tdt, device="cuda"))
    return mu.double().cpu().numpy()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("layout", ["uniform", "clustered"])
def test_pcg_mean_matches_the_exact_mean(love, dtype, layout):
    """Uniform x (the stencil average fits G well) and clustered x (three
    narrow clusters, so G is far from its average and the preconditioner is
    poor): both reach the exact SKI mean, the plain CG too.  In the clustered
    case GMRES stalls and, after its 4 cycles of 40 steps, the plain CG takes
    over from zero, so the count is at most 160 + the plain CG's."""
    wl = small_workload(dim=1, g=400, n=20000, k=8, t=500, dtype=dtype, ls=0.03, noise=0.0025)
    x = wl.x_train()
    if layout == "clustered":
        rng = np.random.default_rng(7)
        c = rng.choice([0.15, 0.5, 0.8], size=x.shape[0])
        x = np.clip(c[:, None] + 0.03 * rng.standard_normal(x.shape), 0.0, 1.0)
    y = wl.y_train(x)
    rd = np.float64 if dtype == "f64" else np.float32
    xr, yr = np.asarray(x, rd).astype(np.float64), np.asarray(y, rd).astype(np.float64)
    xs = np.asarray(wl.x_test(), rd).astype(np.float64)
    ref = _mean_ref(wl, xr, yr, xs)
    ski = gpu_ski(love, torch, wl, x=x, y=y)
    # clustered: empty grid regions make the system harder (condition ~
    # lambda_max / s^2 without the data's help), and the same stopping rule
    # leaves up to ~1e-6 std(y) in FP64
    tol = (1e-8 if layout == "uniform" else 1e-6) if dtype == "f64" else 1e-4
    its, errs = {}, {}
    for plain in (False, True):
        cache = love.love_precompute(ski, k=8, want_mean=True, cg_plain=plain)
        its[plain] = cache.info()["cg_iters"]
        errs[plain] = np.max(np.abs(_mean(love, cache, xs, dtype) - ref)) / np.std(yr)
        print(f"{layout} {dtype} plain={plain}: iters {its[plain]}, |d mu|/std(y) {errs[plain]:.3e}")
    assert errs[False] <= tol and errs[True] <= tol
    if layout == "uniform":
        assert 0 < its[False] and its[False] * 5 <= its[True]
    else:
        assert 0 < its[False] <= 160 + its[True]


def test_pcg_zero_targets(love):
    wl = small_workload(dim=1, g=100, n=3000, k=8, t=100)
    x = wl.x_train()
    ski = gpu_ski(love, torch, wl, x=x, y=np.zeros(x.shape[0]))
    cache = love.love_precompute(ski, k=8, want_mean=True)
    assert cache.info()["cg_iters"] == 0
    mu = _mean(love, cache, np.asarray(wl.x_test(), np.float64), "f32")
    assert np.all(mu == 0.0)


def test_pcg_c2_fullsize_mean_and_iterations(love):
    """The 1-D n = 1e6, m = 1e4 workload: the preconditioned solve matches the
    exact mean (push-through, 2,000 sampled test points) with at least 20x
    fewer iterations than the plain CG."""
    wl = workloads.C2
    x = wl.x_train()
    y = wl.y_train(x)
    ski = gpu_ski(love, torch, wl, x=x, y=y)
    xs = wl.x_test()
    idx = np.random.default_rng(1).choice(xs.shape[0], 2000, replace=False)
    xs = np.asarray(xs[idx], np.float32).astype(np.float64)
    xr, yr = np.asarray(x, np.float32).astype(np.float64), np.asarray(y, np.float32).astype(np.float64)
    ref = _mean_ref(wl, xr, yr, xs)
    its, ms = {}, {}
    for plain in (False, True):
        cache = love.love_precompute(ski, k=8, want_mean=True, cg_plain=plain)
        inf = cache.info()
        its[plain], ms[plain] = inf["cg_iters"], inf["phase_ms"][1]
        err = np.max(np.abs(_mean(love, cache, xs, "f32") - ref)) / np.std(yr)
        print(f"C2 plain={plain}: iters {its[plain]}, CG {ms[plain]:.2f} ms, |d mu|/std(y) {err:.3e}")
        assert err <= 1e-4
    assert its[False] * 20 <= its[True]
