"""Plain FP64 CPU oracle for LOVE (LanczOs Variance Estimates) on KISS-GP.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path (the seeded input generators live in the separate
``workloads`` module, which holds no method arithmetic).

Everything here is written for a reader who checks it against the paper
(Pleiss, Gardner, Weinberger, Wilson, "Constant-Time Predictive Distributions
for Gaussian Processes", ICML 2018):

  keys      cubic-convolution interpolation weights (Sec. 2.3, Keys 1981)
  grid      KISS-GP regular grid, RBF Toeplitz / Kronecker K_UU (Sec. 2.3)
  ski       the SKI operator  W^T K_UU W + sigma^2 I  (eq. ski)
  lanczos   Lanczos with full reorthogonalisation, CG (Sec. 2.1, 2.2, Sec. 5)
  love      LOVE pre-compute, predictive mean/variance, sampler, gradients
            (Sec. 3.2, 3.3, Algorithm 1)
  exact     the exact SKI posterior the method approximates (eqs.
            pred_covar_approx, pred_covar_ski_cache)
  rng       SplitMix64 and Philox4x32-10 counter-based generators

Pins (what each function is checked against, other than itself) are in
``tests/test_oracle_*.py``.  Parity unpinned: none of the functions above is
unpinned; the Philox Box-Muller normals are pinned through the Philox
known-answer vectors plus distribution moments only.
"""
from . import keys, grid, ski, lanczos, love, exact, rng  # noqa: F401
