"""The update rule behind the incremental BUILD, checked on the CPU.

The CUDA BUILD keeps the gain g(c) = sum_o min(d(o,c) - d_n(o), 0) of every
candidate and, after adding medoid m, changes it only through the points
U = {o : d(o,m) < d_n(o)}: by d_n - d_n' where d(o,c) < d_n', by
d_n - d(o,c) where d_n' <= d(o,c) < d_n, else 0 (d_n' the new distance).
This file restates that rule in numpy (row o of D serves candidate c by
symmetry) and checks that the greedy choices it produces are those of
Alg. 1 evaluated from scratch -- the brute-force greedy BUILD of
tests/bruteforce.py and the oracle's BUILD -- on integer matrices rich in
ties and duplicates, where every sum is exact.  It tests the arithmetic
argument, not the kernel (the GPU tests compare the kernel with the
oracle)."""
import numpy as np
import pytest

import bruteforce as bf
import oracle


def incremental_build(D, k):
    """Medoids and per-step gains by the incremental rule (int64 sums)."""
    A = np.asarray(bf.sq(D), dtype=np.int64)
    n = A.shape[0]
    gains = A.sum(axis=0)               # step 0: distance sums
    is_med = np.zeros(n, bool)
    dn = None
    med, steps, rows = [], [], 0
    for t in range(k):
        key = np.where(is_med, np.iinfo(np.int64).max, gains)
        c = int(np.argmin(key))         # lowest index on ties
        med.append(c)
        steps.append(int(gains[c]))
        is_med[c] = True
        row = A[c]                      # d(c, o) = d(o, c)
        if dn is None:                  # gains after step 0: every row
            dn = row.copy()
            gains = np.zeros(n, np.int64)
            for o in range(n):
                gains += np.minimum(A[o] - dn[o], 0)
            rows += 2 * n
            continue
        U = np.nonzero(row < dn)[0]
        for o in U:
            vn, vo, d = row[o], dn[o], A[o]
            gains += np.where(d < vn, vo - vn, np.where(d < vo, vo - d, 0))
        rows += len(U)
        dn = np.minimum(dn, row)
    return med, steps, rows


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_incremental_rule_equals_greedy_build_tiny(seed):
    for D in bf.tiny_instances(300 + seed, 40, n_lo=3, n_hi=11):
        n = D.shape[0]
        for k in sorted({1, 2, max(1, n // 2), n}):
            med, steps, _ = incremental_build(D, k)
            bmed, bsteps = bf.greedy_build(D, k)
            assert med == bmed
            assert steps == [int(v) for v in bsteps]


def test_incremental_rule_equals_oracle_build_with_duplicates():
    """Clustered integer points with many exact duplicates (gains of 0 and
    empty updates late in the BUILD) and a ragged n: medoids and every
    step's gain equal the oracle's BUILD; the rows the rule streams stay far
    below the plain pass's sum of (n - t)."""
    g = np.random.default_rng(17)
    centres = g.integers(0, 200, size=(12, 2))
    X = centres[g.integers(0, 12, size=301)] + g.integers(-3, 4, size=(301, 2))
    D = np.abs(X[:, None, :] - X[None, :, :]).sum(-1).astype(np.int32)
    k = 40
    med, steps, rows = incremental_build(D, k)
    omed, _, ogains = oracle.pam_build(D, k)
    assert med == omed.tolist()
    assert steps == [int(v) for v in ogains]
    assert rows < sum(301 - t for t in range(k)) / 4
