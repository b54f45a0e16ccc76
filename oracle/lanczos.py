"""Lanczos with full reorthogonalisation, tridiagonal Cholesky, CG (oracle).

TEST INFRASTRUCTURE ONLY.

Lanczos (Sec. 2.2): from a probe b, q_1 = b/|b|; each step multiplies the
newest basis vector by A and orthogonalises the result against the basis; the
coefficients form the symmetric tridiagonal T_k, with A ~ Q_k T_k Q_k^T.

Full reorthogonalisation (Sec. 5, "Numerical stability of Lanczos"): the oracle
always reorthogonalises (the paper's detection criterion is not stated) and
uses classical Gram-Schmidt applied twice (CGS2) to the raw product A q_j:

    v   = A q_j
    c   = Q_j^T v ;  v -= Q_j c      (pass 1; c_j = alpha_j = q_j^T A q_j,
                                      and in exact arithmetic c_{j-1} = beta_{j-1},
                                      c_i = 0 otherwise: the three-term recurrence)
    c'  = Q_j^T v ;  v -= Q_j c'     (pass 2; c' is discarded, not folded into T)
    beta_j = |v| ;  q_{j+1} = v / beta_j

Breakdown (not in the paper): stop after step j when beta_j <= tau * max_i |alpha_i|;
k_eff = j.  T_k's diagonal is alpha_1..alpha_keff, its off-diagonal beta_1..beta_{keff-1}.
"""
from __future__ import annotations

import numpy as np


class NotPositiveDefinite(ArithmeticError):
    """A non-positive pivot in the tridiagonal Cholesky (LOVE_ERR_NOT_PD)."""


def lanczos(matvec, b: np.ndarray, k: int, tau: float = 1e-12):
    """k Lanczos steps with CGS2 full reorthogonalisation.

    Returns (Q[k_eff, n], alpha[k_eff], beta[k_eff - 1], beta_last) -- the basis
    vectors as rows.  beta_last is the norm left after the final step (the
    residual coupling, zero at exact Krylov exhaustion).
    """
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    k = min(k, n)
    Q = np.zeros((k, n))
    alpha = np.zeros(k)
    beta = np.zeros(k)
    Q[0] = b / np.linalg.norm(b)
    k_eff = k
    for j in range(k):
        Qj = Q[: j + 1]
        v = matvec(Q[j])
        c = Qj @ v
        alpha[j] = c[j]
        v = v - Qj.T @ c
        c2 = Qj @ v
        v = v - Qj.T @ c2
        beta[j] = np.linalg.norm(v)
        if j == k - 1:
            break
        if beta[j] <= tau * np.max(np.abs(alpha[: j + 1])):
            k_eff = j + 1
            break
        Q[j + 1] = v / beta[j]
    return Q[:k_eff].copy(), alpha[:k_eff].copy(), beta[: k_eff - 1].copy(), float(beta[k_eff - 1])


def tridiag_dense(alpha: np.ndarray, beta: np.ndarray) -> np.ndarray:
    k = alpha.shape[0]
    T = np.diag(alpha)
    if k > 1:
        T += np.diag(beta, 1) + np.diag(beta, -1)
    return T


def tridiag_cholesky(alpha: np.ndarray, beta: np.ndarray):
    """T = L L^T for symmetric tridiagonal T; L lower bidiagonal.

    l_11 = sqrt(alpha_1); e_j = beta_j / l_jj; l_{j+1,j+1} = sqrt(alpha_{j+1} - e_j^2).
    Returns (diag[k], sub[k-1]).  Raises NotPositiveDefinite on a pivot <= 0.
    """
    k = alpha.shape[0]
    d = np.zeros(k)
    e = np.zeros(max(k - 1, 0))
    piv = alpha[0]
    for j in range(k):
        if j > 0:
            e[j - 1] = beta[j - 1] / d[j - 1]
            piv = alpha[j] - e[j - 1] ** 2
        if not piv > 0.0:
            raise NotPositiveDefinite(f"pivot {j}: {piv}")
        d[j] = np.sqrt(piv)
    return d, e


def bidiag_dense(d: np.ndarray, e: np.ndarray) -> np.ndarray:
    L = np.diag(d)
    if d.shape[0] > 1:
        L += np.diag(e, -1)
    return L


def cg(matvec, b: np.ndarray, tol: float = 1e-12, max_iter: int = 10000, x0=None):
    """Linear conjugate gradients (Sec. 2.1) on a positive definite operator.

    Stops when |r| <= tol * |b|.  Returns (x, iterations, relative residual).
    """
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - matvec(x) if x0 is not None else b.copy()
    p = r.copy()
    rr = float(r @ r)
    bn = float(np.linalg.norm(b))
    if bn == 0.0:
        return x, 0, 0.0
    it = 0
    while it < max_iter and np.sqrt(rr) > tol * bn:
        Ap = matvec(p)
        a = rr / float(p @ Ap)
        x = x + a * p
        r = r - a * Ap
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it, float(np.sqrt(rr) / bn)
