"""CPU FP64 oracle of the rank-revealing leverage-score estimator.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The CUDA library in
``paper_2105_11004_gb300`` shares no code with it and never calls it.

Contents:
* ``oracle.rng``       -- splitmix64 hash/sign, Box-Muller streams, entries of G and Omega;
* ``oracle.linalg``    -- column-pivoted Householder QR, back-substitution;
* ``oracle.exact``     -- exact leverage scores (QR route, Gram route Alg. 5), Alg. 7;
* ``oracle.estimator`` -- Alg. 10 step by step (Alg. 3 -> Alg. 4 -> Alg. 8), SRHT variant;
* ``oracle.backward``  -- gradient of sum_i w_i theta~_i and the exact
                          closed-form gradient 2 (I - H) W (A^+)^T;
* ``oracle.rank``      -- singular values, the SVD rank rule, strong-RRQR measures and swaps;
* ``oracle.precond``   -- Alg. 11 (N = V_k Sigma_k^{-1}) and LSQR on A N.

Pins (tests/test_oracle_*.py): splitmix64 reference outputs, brute-force
pseudo-inverse leverage, sum(theta) = rank, 0 <= theta <= 1, theta = 1 on rows
alone in their direction, invariance under A -> A T, explicit S A and G B
products, a hand-solved back-substitution, identity-sketch reduction to the
exact scores, JL statistics, the ranks the paper states for its fixed-spectrum
matrices, the Gu-Eisenstat determinant identity, the spectrum of A N, central
finite differences and the closed-form gradient. Every function has at least
one such pin. The paper prints no numeric example of theta~ itself, so no
stored value comes from the paper except the ranks.
"""
from . import rng, linalg, exact, estimator, backward, rank, precond  # noqa: F401
