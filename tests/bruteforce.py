"""Brute-force definitions used to pin the oracle (numpy, tiny inputs).

Each function is the plain definition from the paper, evaluated by
exhaustive recomputation -- nothing here shares code with ``oracle/`` or the
CUDA path:

* ``td``            Eq. (2): sum over points of the distance to the nearest
                    medoid.
* ``swap_deltas``   Delta(i, c) = TD(M - m_i + c) - TD(M) for every slot i
                    and non-medoid c (the quantity SWAP minimises, Sec. 2).
* ``best_swap``     lexicographic minimum of (Delta, i, c).
* ``steepest``      repeated best swap while Delta < 0 (PAM SWAP, Alg. 2).
* ``fastpam2``      the FastPAM2 reading of Sec. 3.2 (best swap per slot,
                    the global best first, then the other improving slots),
                    every Delta by full TD recomputation.
* ``greedy_build``  each step adds argmin_c TD(M + c) (BUILD, Alg. 1; the
                    first step is the 1-medoid of Eq. (3)).
* ``optimum``       the global optimum by enumerating all C(n, k) sets.
"""
import itertools

import numpy as np


def sq(D, n=None):
    n = D.shape[0] if n is None else n
    return np.asarray(D[:n, :n], dtype=np.float64)


def td(D, med):
    A = sq(D)
    return float(A[:, list(med)].min(axis=1).sum())


def swap_deltas(D, med):
    """Array [k, n] of Delta(i, c); +inf where c is a medoid."""
    A = sq(D)
    n = A.shape[0]
    med = list(med)
    base = td(A, med)
    out = np.full((len(med), n), np.inf)
    for i in range(len(med)):
        for c in range(n):
            if c in med:
                continue
            trial = med.copy()
            trial[i] = c
            out[i, c] = td(A, trial) - base
    return out


def best_swap(D, med):
    dl = swap_deltas(D, med)
    best = (np.inf, -1, -1)
    for i in range(dl.shape[0]):
        for c in range(dl.shape[1]):
            if dl[i, c] < best[0]:
                best = (dl[i, c], i, c)
    return best


def steepest(D, med, max_iter=1000):
    med = list(med)
    trace = []
    for _ in range(max_iter):
        d, i, c = best_swap(D, med)
        if not d < 0:
            break
        trace.append((d, i, c))
        med[i] = c
    return med, trace


def fastpam2(D, med, fp2_tol=0.0, max_iter=1000):
    """FastPAM2 as read from Sec. 3.2: per slot the best (Delta_i*, c_i*)
    over all non-medoids (lowest c on ties); apply the global best (lowest
    slot on ties); then visit the other slots with Delta_i* < 0 in
    ascending (Delta_i*, i), skip one whose c_i* is a medoid by now, and
    apply it iff its Delta against the current medoids, recomputed from
    scratch, is < -fp2_tol * |Delta*|.  Returns (medoids, trace)."""
    med = list(med)
    trace = []
    for _ in range(max_iter):
        dl = swap_deltas(D, med)
        bc = [int(np.argmin(dl[i])) for i in range(len(med))]
        bd = [float(dl[i, bc[i]]) for i in range(len(med))]
        bi = int(np.argmin(bd))
        if not bd[bi] < 0:
            break
        dstar = bd[bi]
        trace.append((dstar, bi, bc[bi]))
        med[bi] = bc[bi]
        rest = sorted((bd[i], i) for i in range(len(med))
                      if i != bi and bd[i] < 0)
        for _, i in rest:
            if bc[i] in med:
                continue
            trial = med.copy()
            trial[i] = bc[i]
            d = td(D, trial) - td(D, med)
            if d < -fp2_tol * abs(dstar):
                trace.append((d, i, bc[i]))
                med[i] = bc[i]
    return med, trace


def greedy_build(D, k):
    A = sq(D)
    n = A.shape[0]
    col = A.sum(axis=0)
    med = [int(np.argmin(col))]
    steps = [float(col[med[0]])]
    for _ in range(1, k):
        base = td(A, med)
        best, bc = np.inf, -1
        for c in range(n):
            if c in med:
                continue
            v = td(A, med + [c]) - base
            if v < best:
                best, bc = v, c
        med.append(bc)
        steps.append(best)
    return med, steps


def optimum(D, k):
    A = sq(D)
    n = A.shape[0]
    best = np.inf
    for comb in itertools.combinations(range(n), k):
        best = min(best, A[:, list(comb)].min(axis=1).sum())
    return float(best)


def cache(D, med):
    """(near, dn, ds) as the two smallest (distance, slot) pairs."""
    A = sq(D)
    n = A.shape[0]
    near = np.empty(n, np.int64)
    dn = np.empty(n)
    ds = np.empty(n)
    for o in range(n):
        pairs = sorted((A[o, m], j) for j, m in enumerate(med))
        near[o] = pairs[0][1]
        dn[o] = pairs[0][0]
        ds[o] = pairs[1][0] if len(pairs) > 1 else np.inf
    return near, dn, ds


# ------------------------------------------------------------ instances --

def tiny_instances(seed, count, n_lo=3, n_hi=10, kinds=("grid1", "grid2",
                                                        "sym")):
    """Tiny integer matrices rich in ties and duplicate points."""
    g = np.random.default_rng(seed)
    out = []
    for t in range(count):
        n = int(g.integers(n_lo, n_hi + 1))
        kind = kinds[t % len(kinds)]
        if kind == "grid1":
            x = g.integers(0, 6, size=(n, 1))
            D = np.abs(x[:, None, :] - x[None, :, :]).sum(-1)
        elif kind == "grid2":
            x = g.integers(0, 4, size=(n, 2))
            D = np.abs(x[:, None, :] - x[None, :, :]).sum(-1)
        else:  # symmetric non-metric dissimilarity, zero diagonal
            U = g.integers(0, 9, size=(n, n))
            D = np.triu(U, 1)
            D = D + D.T
        ld = (n + 3) // 4 * 4
        M = np.zeros((n, ld), np.int32)
        M[:, :n] = D
        out.append(M)
    return out


def tiny_float_instances(seed, count, n_lo=4, n_hi=10):
    g = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(g.integers(n_lo, n_hi + 1))
        x = g.normal(size=(n, 3))
        D = np.sqrt(((x[:, None, :] - x[None, :, :]) ** 2).sum(-1))
        D = D.astype(np.float32)
        up = np.triu(D, 1)
        D = up + up.T
        ld = (n + 3) // 4 * 4
        M = np.zeros((n, ld), np.float32)
        M[:, :n] = D
        out.append(M)
    return out
