"""Cubic-convolution interpolation weights (oracle; test infrastructure only).

Sec. 2.3 of the paper expresses a point x through its 4 closest inducing points
with cubic interpolation (Keys 1981); the paper does not state Keys' free
parameter; a = -0.5 is taken here (the value for which the
interpolation reproduces quadratics).

Keys' kernel, with s = |distance| in grid units:
    u(s) = (a+2) s^3 - (a+3) s^2 + 1          for 0 <= s <= 1
    u(s) = a s^3 - 5a s^2 + 8a s - 4a         for 1 <  s <  2
    u(s) = 0                                  otherwise
"""
from __future__ import annotations

import numpy as np

KEYS_A = -0.5


def u(s):
    """Keys cubic-convolution kernel u(s) (even in s)."""
    a = KEYS_A
    s = np.abs(np.asarray(s, dtype=np.float64))
    out = np.zeros_like(s)
    m1 = s <= 1.0
    m2 = (s > 1.0) & (s < 2.0)
    s1 = s[m1]
    s2 = s[m2]
    out[m1] = (a + 2) * s1 ** 3 - (a + 3) * s1 ** 2 + 1.0
    out[m2] = a * s2 ** 3 - 5 * a * s2 ** 2 + 8 * a * s2 - 4 * a
    return out


def du(s):
    """Derivative u'(s) of the Keys kernel (odd in s)."""
    a = KEYS_A
    s = np.asarray(s, dtype=np.float64)
    sg = np.sign(s)
    r = np.abs(s)
    out = np.zeros_like(r)
    m1 = r <= 1.0
    m2 = (r > 1.0) & (r < 2.0)
    r1 = r[m1]
    r2 = r[m2]
    out[m1] = 3 * (a + 2) * r1 ** 2 - 2 * (a + 3) * r1
    out[m2] = 3 * a * r2 ** 2 - 10 * a * r2 + 8 * a
    return out * sg


class DomainError(ValueError):
    """A point whose 4-point stencil leaves the grid (LOVE_ERR_DOMAIN)."""


def interp_1d(x, lo, h, g, check=True):
    """Base index and the 4 weights (and d/dx weights) of points x.

    s = (x - lo)/h, i = floor(s), f = s - i.  The stencil nodes are
    i-1, i, i+1, i+2 with weights u(s - node) = u(1+f), u(f), u(1-f), u(2-f).
    Returns (i, w[n,4], dw[n,4]) where dw = d w / d x = u'(s - node) / h.
    """
    x = np.asarray(x, dtype=np.float64)
    s = (x - lo) / h
    finite = np.isfinite(s)
    i = np.floor(np.where(finite, s, 0.0)).astype(np.int64)
    if check:
        bad = ~finite | (i - 1 < 0) | (i + 2 > g - 1)
        if np.any(bad):
            raise DomainError(f"{int(bad.sum())} points outside the interpolable grid")
    offs = np.arange(-1, 3)
    d = s[:, None] - (i[:, None] + offs[None, :])
    w = u(d)
    dw = du(d) / h
    return i, w, dw
