"""Oracle pins for the additive composition of one-dimensional KISS-GP kernels
(Sec. 3, "Extension to additive kernel compositions", eq.
multi_dimensional_kernel_block): the stacked interpolation vector and the
block-diagonal K_UU against the sum of separate one-dimensional SKI kernels,
and LOVE on it against the exact posterior."""
import numpy as np

from oracle import exact as E
from oracle import grid as G
from oracle import love as L
from oracle import ski as S


def _grid(gs, ls, sf=1.2):
    lo = [-2.0 / (g - 5) for g in gs]
    hi = [1.0 + 2.0 / (g - 5) for g in gs]
    return G.AdditiveGrid(list(gs), lo, hi, list(ls), sf)


def test_block_form_equals_the_sum_of_one_dimensional_kernels():
    """w(x)^T diag(K_e) w(x') = sum_e w_e(x_e)^T K_e w_e(x'_e): the SKI matrix of
    the block form against the sum of plain 1-D Grid SKI matrices."""
    rng = np.random.default_rng(1)
    ag = _grid([20, 16, 24], [0.2, 0.3, 0.15])
    x = rng.uniform(0, 1, (150, 3))
    ski = S.SKI(ag, x, 0.05, None)
    ref = 0.05 * np.eye(150)
    for e in range(3):
        c = ag.component(e)
        We = c.W(x[:, e:e + 1]).toarray()
        ref = ref + We.T @ c.dense_kuu() @ We
    np.testing.assert_allclose(ski.dense(), ref, rtol=0, atol=1e-13)
    # the prior is the diagonal of W*^T K W*, a sum over components
    xs = rng.uniform(0, 1, (40, 3))
    Ws = ag.W(xs).toarray()
    np.testing.assert_allclose(ag.local_kernel_quadform(xs), np.einsum("mt,mn,nt->t", Ws, ag.dense_kuu(), Ws),
                               rtol=1e-13)
    # 4 nonzeros per component in the stacked vector
    assert ag.W(xs).nnz == 40 * 4 * 3
    # block-diagonal K_UU product against the dense block matrix
    v = rng.standard_normal((ag.m, 3))
    np.testing.assert_allclose(ag.kuu_matmul(v), ag.dense_kuu() @ v, atol=1e-12)


def test_love_on_the_additive_kernel_reaches_the_exact_posterior():
    rng = np.random.default_rng(2)
    ag = _grid([18, 14], [0.25, 0.2])
    x = rng.uniform(0, 1, (220, 2))
    ski = S.SKI(ag, x, 0.03, np.sin(3 * x).sum(1))
    c = L.precompute(ski, k=220)
    xs = rng.uniform(0, 1, (30, 2))
    m, v = L.predict(c, xs)
    me, ve = E.exact_dense(ski, xs)
    assert np.max(np.abs(v - ve)) <= 1e-9 * np.max(np.abs(ve))
    assert np.max(np.abs(m - me)) <= 1e-8 * np.max(np.abs(me))
    assert np.all(v > 0) and np.all(v <= L.prior(ag, xs) * (1 + 1e-12))


def test_one_component_is_the_plain_one_dimensional_grid():
    rng = np.random.default_rng(3)
    ag = _grid([30], [0.15])
    g1 = G.Grid([30], list(ag.lo), list(ag.hi), [0.15], ag.outputscale)
    x = rng.uniform(0, 1, (100, 1))
    c_a = L.precompute(S.SKI(ag, x, 0.02, None), k=10)
    c_1 = L.precompute(S.SKI(g1, x, 0.02, None), k=10)
    xs = rng.uniform(0, 1, (25, 1))
    np.testing.assert_allclose(L.predict(c_a, xs)[1], L.predict(c_1, xs)[1], rtol=1e-12)
