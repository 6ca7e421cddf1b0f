"""CPU FP64 oracle of the rank-revealing leverage-score estimator.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The CUDA library in
``paper_2105_11004_gb300`` shares no code with it and never calls it.

Contents:
* ``oracle.rng``       -- splitmix64 hash/sign and Box-Muller streams;
* ``oracle.linalg``    -- column-pivoted Householder QR, back-substitution;
* ``oracle.exact``     -- exact leverage scores (QR route, Gram route Alg. 5);
* ``oracle.estimator`` -- Alg. 10 step by step (Alg. 3 -> Alg. 4 -> Alg. 8);
* ``oracle.backward``  -- gradient of sum_i w_i theta~_i and the exact
                          closed-form gradient 2 (I - H) W (A^+)^T.

Pins (tests/test_oracle_*.py): splitmix64 reference outputs, brute-force
pseudo-inverse leverage, sum(theta) = rank, 0 <= theta <= 1, theta = 1 on rows
alone in their direction, invariance under A -> A T, identity-sketch
reduction to the exact scores, JL statistics, central finite differences and
the closed-form gradient. Parity unpinned: actual theta~ values at the
workload sizes (the paper prints no numeric example).
"""
from . import rng, linalg, exact, estimator, backward  # noqa: F401
