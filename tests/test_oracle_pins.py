"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests retypes an oracle formula: the expected values come from
the paper's worked example (Fig. 1), from brute-force recomputation of the TD
objective (Eq. (2)) in numpy, from enumeration of all medoid sets, or from
invariants the paper states (Sec. 2 and 3).
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import bruteforce as bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def fig1():
    with open(os.path.join(GOLDEN, "fig1_alternating.json")) as f:
        g = json.load(f)
    names = list(g["points"].keys())
    x = np.array([g["points"][a] for a in names], np.int64)
    n = len(x)
    D = np.zeros((n, 8), np.int32)
    D[:, :n] = np.abs(x[:, None] - x[None, :])
    return g, names, D


# ------------------------------------------------------------------ P1 --

@pytest.mark.parametrize("variant", ["pam_bruteforce", "pam", "fastpam1",
                                     "fasterpam", "fastpam2"])
def test_fig1_worked_example(variant):
    """Fig. 1: from medoids {B, E} SWAP makes B->A (loss 7), then E->D
    (loss 6), then stops."""
    g, names, D = fig1()
    idx = {a: i for i, a in enumerate(names)}
    start = [idx[a] for a in g["start_medoids"]]
    out = oracle.swap(D, start, variant=variant, n=6)
    assert out["swaps"] == len(g["swaps"])
    med = list(start)
    for (delta, slot, cand), sw in zip(out["trace"], g["swaps"]):
        assert med[slot] == idx[sw["remove"]]
        assert cand == idx[sw["add"]]
        med[slot] = cand
        assert oracle.td(D, med, n=6) == sw["loss_after"]
    assert out["td"] == g["swaps"][-1]["loss_after"]
    assert out["td_bookkept"] == out["td"]
    assert out["converged"]
    if variant in ("pam_bruteforce", "pam", "fastpam1"):
        assert out["iterations"] == out["swaps"] + 1


def test_fig1_build_then_swap():
    """BUILD on the Fig. 1 points: first medoid is the 1-medoid (C and D tie
    at distance sum 14, lowest index wins), then the greedy step adds A;
    SWAP then moves C -> D and reaches the loss 6 of Fig. 1."""
    g, names, D = fig1()
    med, tdb, steps = oracle.pam_build(D, 2, n=6)
    bmed, bsteps = bf.greedy_build(D[:, :6], 2)
    assert list(med) == bmed == [names.index("C"), names.index("A")]
    assert tdb == 7 == bf.td(D[:, :6], med)
    out = oracle.swap(D, med, variant="fastpam1", n=6)
    assert out["td"] == g["swaps"][-1]["loss_after"]
    assert out["swaps"] == 1 and out["iterations"] == 2


# ------------------------------------------------------------------ P2 --

def test_eval_matches_bruteforce_integer():
    """Per candidate, min_i Delta(i, c) and its lowest slot from the
    FastPAM1 decomposition (Eq. (7)), from PAM's change function (Eq. (5))
    and from full TD recomputation all equal brute force exactly."""
    for D in bf.tiny_instances(11, 150):
        n = D.shape[0]
        g = np.random.default_rng(n * 7 + int(D.sum()))
        for k in range(1 if n > 2 else 2, n):
            if k < 2:
                continue
            med = list(g.choice(n, size=k, replace=False))
            dl = bf.swap_deltas(D, med)
            want = dl.min(axis=0)
            wslot = dl.argmin(axis=0)
            wbest = bf.best_swap(D, med)
            for method in ("fastpam1", "pam", "bruteforce"):
                cd, cs, best = oracle.eval_swaps(D, med, method=method)
                for c in range(n):
                    if c in med:
                        assert cs[c] == -1
                        continue
                    assert cd[c] == want[c], (method, n, k, c)
                    assert cs[c] == wslot[c], (method, n, k, c)
                assert best == (wbest[0], wbest[1], wbest[2]), method


def test_eval_matches_bruteforce_float():
    for D in bf.tiny_float_instances(12, 60):
        n = D.shape[0]
        g = np.random.default_rng(n)
        for k in range(2, n):
            med = list(g.choice(n, size=k, replace=False))
            dl = bf.swap_deltas(D, med)
            want = dl.min(axis=0)
            scale = bf.td(D, med) + 1.0
            cd, cs, best = oracle.eval_swaps(D, med, method="fastpam1")
            for c in range(n):
                if c in med:
                    continue
                assert abs(cd[c] - want[c]) <= 1e-12 * scale
                # slot: exact argmin unless an exact-arithmetic tie
                assert dl[cs[c], c] <= want[c] + 1e-12 * scale


def test_swap_delta_single_pair():
    for D in bf.tiny_instances(13, 60):
        n = D.shape[0]
        g = np.random.default_rng(n + 3)
        k = int(g.integers(2, n))
        med = list(g.choice(n, size=k, replace=False))
        dl = bf.swap_deltas(D, med)
        for i in range(k):
            for c in range(n):
                if c not in med:
                    assert oracle.swap_delta(D, med, i, c) == dl[i, c]


def test_cache_and_removal_loss():
    """nearest / d_n / d_s are the two smallest (distance, slot) pairs; the
    removal loss of slot i equals TD(M - m_i) - TD(M) (the loss of removing
    the medoid and reassigning its points to their second nearest)."""
    for D in bf.tiny_instances(14, 80):
        n = D.shape[0]
        g = np.random.default_rng(n + 5)
        k = int(g.integers(2, n + 1))
        med = list(g.choice(n, size=k, replace=False))
        near, sec, dn, ds = oracle.cache(D, med)
        bn, bdn, bds = bf.cache(D, med)
        assert (near == bn).all() and (dn == bdn).all() and (ds == bds).all()
        rl = oracle.removal_loss(near, dn, ds, k)
        base = bf.td(D, med)
        for i in range(k):
            rest = med[:i] + med[i + 1:]
            assert rl[i] == bf.td(D, rest) - base


# --------------------------------------------------------------- P3-P5 --

def test_fastpam1_equals_pam_trajectory():
    """FastPAM1 makes exactly the swaps of PAM (Sec. 3.1) -- checked against
    an independent brute-force steepest descent on integer data."""
    for D in bf.tiny_instances(21, 120, n_lo=5, n_hi=11):
        n = D.shape[0]
        g = np.random.default_rng(n * 13)
        k = int(g.integers(2, min(n, 5)))
        start = list(g.choice(n, size=k, replace=False))
        bmed, btrace = bf.steepest(D, start)
        for variant in ("pam_bruteforce", "pam", "fastpam1"):
            out = oracle.swap(D, start, variant=variant)
            assert [tuple(t) for t in out["trace"]] == \
                [(float(d), i, c) for d, i, c in btrace], variant
            assert list(out["medoids"]) == bmed
            assert out["iterations"] == out["swaps"] + 1


@pytest.mark.parametrize("variant", ["fastpam1", "fastpam2", "fasterpam"])
def test_monotone_and_locally_optimal(variant):
    """TD strictly decreases at every accepted swap and the final medoids
    admit no swap with Delta < 0 (Sec. 2).  Iteration counts: steepest
    descent makes one swap per pass and a final pass without one
    (iterations = swaps + 1, Sec. 5); FastPAM2 applies at least the best
    swap in every pass but the last, and every FasterPAM scan but the last
    holds a swap (a whole scan without one ends the run, Alg. 4)."""
    insts = bf.tiny_instances(31, 60, n_lo=5, n_hi=11)
    insts += [np.ascontiguousarray(M) for M in
              bf.tiny_float_instances(32, 30, n_lo=5, n_hi=11)]
    for D in insts:
        n = D.shape[0]
        g = np.random.default_rng(n * 17)
        k = int(g.integers(2, min(n, 5)))
        start = list(g.choice(n, size=k, replace=False))
        out = oracle.swap(D, start, variant=variant)
        med = list(start)
        prev = bf.td(D, med)
        for d, i, c in out["trace"]:
            assert d < 0
            med[i] = c
            cur = bf.td(D, med)
            assert abs((cur - prev) - d) <= 1e-9 * (1 + prev)
            assert cur < prev
            prev = cur
        assert list(out["medoids"]) == med
        assert abs(out["td"] - prev) <= 1e-9 * (1 + prev)
        assert abs(out["td_bookkept"] - out["td"]) <= 1e-9 * (1 + prev)
        assert bf.swap_deltas(D, med).min() >= -1e-9 * (1 + prev)
        assert out["converged"]
        if variant == "fastpam1":
            assert out["iterations"] == out["swaps"] + 1
        else:
            assert out["swaps"] >= out["iterations"] - 1 >= 0


def test_fasterpam_scan_rule():
    """Alg. 4 read as a cyclic scan: after the final swap at index p the
    scan visits the other n - 1 indices without a swap, so the positions
    visited are (absolute index of the last swap) + n."""
    for D in bf.tiny_instances(33, 40, n_lo=6, n_hi=11):
        n = D.shape[0]
        g = np.random.default_rng(n)
        k = int(g.integers(2, 5))
        start = list(g.choice(n, size=k, replace=False))
        out = oracle.swap(D, start, variant="fasterpam")
        if out["swaps"] == 0:
            assert out["visited"] == n and out["iterations"] == 1
        else:
            assert out["visited"] % n == (out["trace"][-1][2] + n) % n
            # replay the scan with brute force to confirm eagerness
            med = list(start)
            pos = 0
            for d, i, c in out["trace"]:
                while pos % n != c:  # candidates before c did not improve
                    p = pos % n
                    if p not in med:
                        assert bf.swap_deltas(D, med)[:, p].min() >= 0
                    pos += 1
                dl = bf.swap_deltas(D, med)[:, c]
                assert dl.min() == d and int(dl.argmin()) == i
                med[i] = c
                pos += 1


def test_fastpam2_first_swap_is_fastpam1_swap():
    for D in bf.tiny_instances(41, 60, n_lo=6, n_hi=11):
        n = D.shape[0]
        g = np.random.default_rng(n * 3)
        k = int(g.integers(2, 5))
        start = list(g.choice(n, size=k, replace=False))
        f1 = oracle.swap(D, start, variant="fastpam1", max_iter=1)
        f2 = oracle.swap(D, start, variant="fastpam2", max_iter=1)
        if f1["swaps"]:
            assert f2["trace"][0] == f1["trace"][0]
        else:
            assert f2["swaps"] == 0


@pytest.mark.parametrize("fp2_tol", [0.0, 0.25, 1.0])
def test_fastpam2_matches_bruteforce_replay(fp2_tol):
    """Every swap FastPAM2 applies (the best one and the additional ones,
    their order, the skip of a candidate that became a medoid, the
    threshold) equals a replay of the Sec. 3.2 reading in which each Delta
    is a full TD recomputation.  Integer data: the deltas are exact."""
    cases = 0
    for D in bf.tiny_instances(43, 240, n_lo=6, n_hi=12):
        n = D.shape[0]
        g = np.random.default_rng(n * 7 + cases)
        k = int(g.integers(2, min(6, n - 1) + 1))
        start = [int(x) for x in g.choice(n, size=k, replace=False)]
        got = oracle.swap(D, start, variant="fastpam2", fastpam2_tol=fp2_tol)
        med, trace = bf.fastpam2(D, start, fp2_tol=fp2_tol)
        assert got["converged"]
        assert [tuple(t) for t in got["trace"]] == \
            [(float(d), i, c) for d, i, c in trace]
        assert list(got["medoids"]) == med
        assert got["td"] == bf.td(D, med)
        cases += len(trace) > got["iterations"] - 1
    if fp2_tol < 1.0:  # an extra swap rarely beats -|Delta*| itself
        assert cases > 0  # some iteration applied an additional swap


# ------------------------------------------------------------------ P6 --

def test_build_is_greedy_td():
    """BUILD: the first medoid is the 1-medoid of Eq. (3); each further
    medoid is argmin_c TD(M + c) (lowest index on ties); the bookkept TD
    equals Eq. (2) after every step."""
    insts = bf.tiny_instances(51, 90, n_lo=3, n_hi=12)
    for D in insts:
        n = D.shape[0]
        for k in range(1, n + 1):
            med, tdb, steps = oracle.pam_build(D, k)
            bmed, bsteps = bf.greedy_build(D, k)
            assert list(med) == bmed
            assert np.allclose(steps, bsteps, rtol=0, atol=0)
            assert tdb == bf.td(D, med)


def test_build_float_bookkeeping():
    for D in bf.tiny_float_instances(52, 40):
        n = D.shape[0]
        k = max(1, n // 3)
        med, tdb, steps = oracle.pam_build(D, k)
        assert abs(tdb - bf.td(D, med)) <= 1e-9 * (1 + tdb)
        bmed, _ = bf.greedy_build(D, k)
        assert list(med) == bmed


# ------------------------------------------------------------------ P7 --

def test_degenerate_k():
    for D in bf.tiny_instances(61, 40, n_lo=3, n_hi=9):
        n = D.shape[0]
        # k = n: every point is a medoid
        med, tdb, _ = oracle.pam_build(D, n)
        assert tdb == 0 and sorted(med) == list(range(n))
        out = oracle.swap(D, med, variant="fastpam1")
        assert out["swaps"] == 0 and out["td"] == 0
        # k = 1: BUILD gives the global optimum; SWAP from any medoid
        # reaches it (the 1-medoid, lowest index on ties)
        med1, td1, _ = oracle.pam_build(D, 1)
        assert td1 == bf.optimum(D, 1)
        for v in ("fastpam1", "fasterpam", "fastpam2", "pam"):
            out = oracle.swap(D, [n - 1], variant=v)
            assert out["td"] == td1


def test_local_optimum_vs_enumeration():
    """For k = 1..3 and n <= 12: the local optimum is never below the
    global optimum; on metric data it is within the locality gap of 5
    (Sec. 3.2, Arya et al.)."""
    for D in bf.tiny_instances(71, 45, n_lo=5, n_hi=12,
                               kinds=("grid1", "grid2")):
        n = D.shape[0]
        for k in (1, 2, 3):
            if k >= n:
                continue
            opt = bf.optimum(D, k)
            out = oracle.run(D, k, variant="fastpam1")
            assert out["td"] >= opt
            assert out["td"] <= 5 * opt + 1e-9


def test_iteration_cap_reports_not_converged():
    D = bf.tiny_instances(81, 1, n_lo=10, n_hi=10, kinds=("grid2",))[0]
    start = [0, 1, 2]
    full = oracle.swap(D, start, variant="fastpam1")
    if full["swaps"] >= 1:
        out = oracle.swap(D, start, variant="fastpam1", max_iter=1)
        assert not out["converged"] and out["swaps"] == 1


def test_thread_count_does_not_change_results():
    from paper_2008_05171_gb300 import workloads as wl
    X = wl.gmm_points(300, 4, 6, seed="t-threads")
    D = wl.euclidean_f32(X)
    med, _, _ = oracle.pam_build(D, 6)
    a = oracle.eval_swaps(D, med)
    oracle.set_threads(1)
    try:
        b = oracle.eval_swaps(D, med)
    finally:
        oracle.set_threads(os.cpu_count() or 1)
    assert (a[0] == b[0]).all() and (a[1] == b[1]).all() and a[2] == b[2]


def test_build_gains_step_matches_build():
    for D in bf.tiny_instances(91, 30, n_lo=4, n_hi=12):
        n = D.shape[0]
        k = max(1, n // 2)
        med, _, steps = oracle.pam_build(D, k)
        for t in range(k):
            g = oracle.build_gains(D, med[:t])
            assert int(np.argmin(g)) == med[t] and g[med[t]] == steps[t]
            base = bf.td(D, list(med[:t])) if t else 0.0
            for c in range(n):
                if c in med[:t]:
                    assert g[c] == np.inf
                elif t:
                    assert g[c] == bf.td(D, list(med[:t]) + [c]) - base


# ------------------------------------------------------------------ CLARA

def test_clara_single_full_sample_is_pam():
    """CLARA with one 'sample' holding every point is PAM on the full data
    (Sec. 2.1): same medoids and TD as BUILD + FastPAM1."""
    from paper_2008_05171_gb300 import workloads as wl
    X = wl.gmm_points(150, 3, 4, seed="clara-pin").astype(np.float32)
    D = oracle.euclid_f32(X)
    S = np.arange(150, dtype=np.int32)[None, :]
    med, lab, tds, best = oracle.clara(X, 4, S)
    ref = oracle.run(D, 4, variant="fastpam1")
    assert best == 0
    assert med.tolist() == ref["medoids"].tolist()
    assert abs(tds[0] - ref["td"]) <= 1e-5 * ref["td"]


def test_clara_best_sample_has_least_full_td():
    from paper_2008_05171_gb300 import workloads as wl
    X = wl.gmm_points(400, 2, 5, seed="clara-pin2").astype(np.float32)
    D = oracle.euclid_f32(X)
    S = wl.clara_samples(400, 5, 30, seed="clara-pin2")
    med, lab, tds, best = oracle.clara(X, 5, S)
    assert best == int(np.argmin(tds))
    full = bf.td(D, med)
    assert abs(full - tds[best]) <= 1e-5 * full
    # each sample's TD is the TD of PAM on that sample, assigned to all data
    for q in range(5):
        Dq = oracle.euclid_f32(X, idx=S[q])
        r = oracle.run(Dq, 5, variant="fastpam1")
        gm = S[q][r["medoids"]]
        assert abs(bf.td(D, gm) - tds[q]) <= 1e-5 * tds[q]
    assert (lab == np.argmin(D[:, :400][:, med], axis=1)).all()


def test_euclid_f32_is_the_fp64_distance_rounded_once():
    """The batch and CLARA matrices are Euclidean distances of float32
    points computed in FP64 and rounded once to float32: every entry lies
    within half a float32 ulp of scipy's FP64 distance (an independent
    routine with its own summation order), the diagonal is zero, the matrix
    is bitwise symmetric and the row padding is zero.  A float32 sum, a
    dropped coordinate or a missing square root fails it."""
    from scipy.spatial.distance import cdist
    g = np.random.default_rng(416)
    for d in (1, 2, 3, 8, 17, 32):
        m = int(g.integers(5, 70))
        X = (g.normal(size=(m, d)) * g.uniform(0.01, 100.0)).astype(np.float32)
        X[-1] = X[0]                                   # a duplicate: distance 0
        ld = (m + 3) // 4 * 4 + 4
        D = oracle.euclid_f32(X, ld=ld)
        ref = cdist(X.astype(np.float64), X.astype(np.float64))
        got = D[:, :m].astype(np.float64)
        half_ulp = 0.5 * np.spacing(D[:, :m]).astype(np.float64)
        assert (np.abs(got - ref) <= half_ulp * (1 + 1e-6) + 1e-300).all(), d
        assert (np.diag(D[:, :m]) == 0).all()
        assert (D[:, :m] == D[:, :m].T).all()
        assert (D[:, m:] == 0).all()
        assert D[0, m - 1] == 0 and D[m - 1, 0] == 0
    # sample indices select rows and columns of the full matrix
    X = g.normal(size=(40, 5)).astype(np.float32)
    idx = np.array([3, 17, 0, 39, 8], np.int64)
    assert (oracle.euclid_f32(X, idx=idx)[:, :5] == oracle.euclid_f32(X)[np.ix_(idx, idx)]).all()


# --------------------------------------------------------- FastCLARANS --

def _clarans_bruteforce(D, med, cand, maxneighbor):
    """CLARANS over the given draws with every (slot, draw) Delta recomputed
    from the TD objective (Eq. (2)): for a non-medoid draw c, the best slot
    is the lowest one with the least TD after putting c there."""
    med = list(int(m) for m in med)
    fails, pos, trace = 0, 0, []
    while pos < len(cand):
        c = int(cand[pos])
        pos += 1
        if c in med:
            continue
        base = bf.td(D, med)
        best, bi = None, -1
        for i in range(len(med)):
            trial = med.copy()
            trial[i] = c
            d = bf.td(D, trial) - base
            if best is None or d < best:
                best, bi = d, i
        if best < 0:
            med[bi] = c
            trace.append((best, bi, c))
            fails = 0
        else:
            fails += 1
            if fails >= maxneighbor:
                return med, pos, trace, True
    return med, pos, trace, False


def test_clarans_matches_bruteforce_replay():
    """FastCLARANS (Sec. 3.4) evaluates a draw against all k medoids with
    Eq. (7); each decision must equal the brute-force TD recomputation over
    all slots, on tiny integer matrices rich in ties, random starts, draw
    streams with repeats and medoids, and every stopping count."""
    g = np.random.default_rng(31)
    for D in bf.tiny_instances(131, 90, n_lo=4, n_hi=10):
        n = D.shape[0]
        k = int(g.integers(2, n))
        med = g.choice(n, size=k, replace=False).astype(np.int32)
        cand = g.integers(0, n, size=3 * n).astype(np.int32)
        mn = int(g.integers(1, n + 1))
        ref_med, ref_pos, ref_tr, ref_stop = _clarans_bruteforce(D, med, cand, mn)
        out = oracle.clarans(D, med, cand, mn)
        assert out["medoids"].tolist() == ref_med
        assert out["consumed"] == ref_pos and out["stopped"] == ref_stop
        assert [(round(d), i, c) for d, i, c in out["trace"]] == \
            [(round(d), i, c) for d, i, c in ref_tr]
        assert out["td"] == bf.td(D, ref_med)


def test_clarans_on_cyclic_draws_is_fasterpam():
    """With the draws 0, 1, ..., n-1 repeated and maxneighbor = n - k (every
    non-medoid failed once since the last swap), the randomized search
    makes exactly FasterPAM's scan (Alg. 4): same swaps in the same order."""
    g = np.random.default_rng(5)
    for t, D in enumerate(bf.tiny_instances(77, 20, n_lo=8, n_hi=10) +
                          [bf.tiny_float_instances(78, 1, 10, 10)[0]]):
        n = D.shape[0]
        k = 3 if n > 4 else 2
        start = g.choice(n, size=k, replace=False).astype(np.int32)
        ref = oracle.swap(D, start, variant="fasterpam", trace_cap=1000)
        cyc = np.tile(np.arange(n, dtype=np.int32), 50)
        out = oracle.clarans(D, start, cyc, n - k, trace_cap=1000)
        assert out["stopped"]
        assert out["medoids"].tolist() == ref["medoids"].tolist()
        assert [(i, c) for _, i, c in out["trace"]] == [(i, c) for _, i, c in ref["trace"]]
    # the worked example of Fig. 1: from {B, E} the swaps B->A, E->D
    gj, names, D = fig1()
    start = np.array([names.index("B"), names.index("E")], np.int32)
    out = oracle.clarans(D, start, np.tile(np.arange(6, dtype=np.int32), 10), 4)
    assert sorted(names[m] for m in out["medoids"]) == ["A", "D"]
    assert [names[c] for _, _, c in out["trace"]] == ["A", "D"]


# ------------------------------------------- distance-weighted initialisation --

def test_init_weighted_picks_by_the_weight_intervals():
    """Draw t picks the point whose interval of the running weight sum holds
    u_t W, weights = distances to the nearest medoid drawn so far (the
    k-means++ seeding with linear distances, Sec. 2.3 / 3.3): with u_1 at
    the middle of point o's interval the second medoid is o, for every o
    with positive weight, on integer matrices (weights = distances)."""
    for D in bf.tiny_instances(401, 12, n_lo=6, n_hi=10, kinds=("grid2", "sym")):
        n = D.shape[0]
        A = bf.sq(D)
        first = 2
        w = A[:, first].copy()                 # distances to the first medoid
        W = w.sum()
        if W == 0:
            continue
        prefix = np.cumsum(w) - w
        for o in range(n):
            if w[o] == 0:
                continue
            u1 = (prefix[o] + 0.5 * w[o]) / W
            med = oracle.init_weighted(D, 2, [(first + 0.5) / n, u1])
            assert med.tolist() == [first, o]


def test_init_weighted_frequencies_follow_distances():
    """Over many uniform u_1 the second medoid is o with frequency close to
    d(o, m_1) / sum_p d(p, m_1) (chi-square, fixed seed)."""
    D = bf.tiny_instances(402, 1, n_lo=9, n_hi=9, kinds=("grid2",))[0]
    A = bf.sq(D)
    first = 0
    g = np.random.default_rng(3)
    counts = np.zeros(A.shape[0])
    for u1 in g.random(4000):
        counts[oracle.init_weighted(D, 2, [0.0, u1])[1]] += 1
    p = A[:, first] / A[:, first].sum()
    m = p > 0
    chi2 = (((counts[m] - 4000 * p[m]) ** 2) / (4000 * p[m])).sum()
    assert counts[~m].sum() == 0 and chi2 < 30.0   # ~ 8 degrees of freedom


def test_init_weighted_distinct_and_degenerate():
    g = np.random.default_rng(9)
    for D in bf.tiny_instances(403, 20, n_lo=4, n_hi=10):
        n = D.shape[0]
        u = g.random(n)
        med = oracle.init_weighted(D, n, u)
        assert sorted(med.tolist()) == list(range(n))          # k = n: every point once
        assert med[0] == int(np.floor(u[0] * n))              # draw 0 is uniform
    Z = np.zeros((6, 8), np.int32)                            # all points coincide
    assert oracle.init_weighted(Z, 4, [0.5, 0.9, 0.1, 0.3]).tolist() == [3, 0, 1, 2]
    F = bf.tiny_float_instances(404, 1, 8, 8)[0]
    med = oracle.init_weighted(F, 3, [0.99999, 0.5, 0.5])
    assert med[0] == 7 and len(set(med.tolist())) == 3


def _float_matrix(seed, n, d=3):
    """A float32 Euclidean matrix (distances with full 24-bit mantissas)."""
    g = np.random.default_rng(seed)
    X = (g.normal(size=(n, d)) * 3.7).astype(np.float32)
    return oracle.euclid_f32(X)


def test_init_weighted_float_weights_follow_the_distances():
    """On float matrices the weights of a draw are the distances to the
    nearest medoid (Sec. 3.3): u_1 at the middle of point o's interval of
    the exact running sum picks o, and the interval boundaries sit where
    the exact FP64 distances put them to 2^-40 of the total weight: u_1 just
    above the sum of the weights before o picks o, just below it picks the
    previous point of positive weight.  The expected intervals come from
    numpy's FP64 distances, not from the oracle's summation."""
    import math
    for seed, n in ((421, 9), (422, 31), (423, 64)):
        D = _float_matrix(seed, n)
        A = bf.sq(D)
        first = n // 3
        w = A[:, first].copy()
        W = math.fsum(w)
        pre = [math.fsum(w[:o]) for o in range(n)]
        pos = [o for o in range(n) if w[o] > 0]
        delta = 2.0 ** -40 * W
        u0 = (first + 0.5) / n
        for j, o in enumerate(pos):
            mid = (pre[o] + 0.5 * w[o]) / W
            assert oracle.init_weighted(D, 2, [u0, mid]).tolist() == [first, o]
            if j > 0 and w[o] > 4 * delta:
                above = (pre[o] + delta) / W
                below = (pre[o] - delta) / W
                assert oracle.init_weighted(D, 2, [u0, above])[1] == o
                assert oracle.init_weighted(D, 2, [u0, below])[1] == pos[j - 1]


def test_init_weighted_float_frequencies_follow_distances():
    """Float matrix: over many uniform u_1 the second medoid is o with
    frequency close to d(o, m_1) / sum_p d(p, m_1) (chi-square, fixed seed,
    ~10 degrees of freedom)."""
    D = _float_matrix(424, 11)
    A = bf.sq(D)
    g = np.random.default_rng(4)
    counts = np.zeros(11)
    for u1 in g.random(5000):
        counts[oracle.init_weighted(D, 2, [0.0, u1])[1]] += 1
    p = A[:, 0] / A[:, 0].sum()
    m = p > 0
    chi2 = (((counts[m] - 5000 * p[m]) ** 2) / (5000 * p[m])).sum()
    assert counts[~m].sum() == 0 and chi2 < 35.0


def _lab_bruteforce(D, k, ranks):
    """LAB (Sec. 3.3) from its definition: at step t the subsample is the
    set of non-medoids at the given ranks (index order), and the next medoid
    is the subsample point c minimising the subsample's TD with c added
    (TD of the subsample alone at t = 0), lowest index on ties."""
    A = bf.sq(D)
    n = A.shape[0]
    med = []
    for t in range(k):
        free = [o for o in range(n) if o not in med]
        S = [free[r] for r in ranks[t]]
        best, pick = None, None
        for c in sorted(S):
            cols = med + [c]
            v = A[np.ix_(S, cols)].min(axis=1).sum()
            if best is None or v < best:
                best, pick = v, c
        med.append(pick)
    return med


def test_init_lab_matches_subsample_td_bruteforce():
    """Each LAB step is the argmin of the subsample's TD with the candidate
    added (integer matrices rich in ties: exact)."""
    g = np.random.default_rng(411)
    for D in bf.tiny_instances(411, 60, n_lo=6, n_hi=12):
        n = D.shape[0]
        k = int(g.integers(1, n + 1))
        s = int(g.integers(1, n - k + 2))
        ranks = np.array([g.choice(n - t, s, replace=False) for t in range(k)])
        assert oracle.init_lab(D, k, ranks).tolist() == _lab_bruteforce(D, k, ranks)


def test_init_lab_float_matches_subsample_td_bruteforce():
    """Float matrices: each LAB step is the argmin of the subsample's TD
    with the candidate added, computed in numpy FP64, wherever the best
    choice beats the runner-up by more than 1e-9 of the subsample's TD; the
    reported gain equals the FP64 TD change to 1e-12 of it."""
    g = np.random.default_rng(425)
    checked = 0
    for t0 in range(40):
        n = int(g.integers(6, 30))
        D = _float_matrix(4250 + t0, n, d=int(g.integers(1, 6)))
        A = bf.sq(D)
        k = int(g.integers(1, min(n, 6) + 1))
        s = int(g.integers(2, n - k + 2))
        ranks = np.array([g.choice(n - t, s, replace=False) for t in range(k)])
        med_o, gains_o = oracle.init_lab(D, k, ranks, gains=True)
        med = []
        for t in range(k):
            free = [o for o in range(n) if o not in med]
            S = [free[r] for r in ranks[t]]
            base = A[np.ix_(S, med)].min(axis=1).sum() if med else 0.0
            vals = sorted((A[np.ix_(S, med + [c])].min(axis=1).sum(), c) for c in S)
            scale = max(1.0, abs(vals[0][0]))
            assert abs(gains_o[t] - (vals[0][0] - base)) <= 1e-12 * max(1.0, abs(base), scale)
            if len(vals) > 1 and vals[1][0] - vals[0][0] <= 1e-9 * scale:
                break                          # a near-tie: the rest is not comparable
            assert med_o[t] == vals[0][1], (t0, t)
            med.append(vals[0][1])
            checked += 1
    assert checked > 60


def test_init_lab_full_sample_is_build():
    """With the whole non-medoid set as every subsample (ranks 0..n-t-1,
    the rest of the row -1 = unused), LAB is BUILD (Alg. 1): medoids and
    gains equal the oracle's BUILD, which is pinned to greedy brute force
    above; integer and float data."""
    insts = bf.tiny_instances(412, 30, n_lo=5, n_hi=12) + \
        bf.tiny_float_instances(413, 10, 5, 12)
    for D in insts:
        n = D.shape[0]
        for k in sorted({1, 2, max(1, n // 2), n}):
            ranks = np.full((k, n), -1, np.int32)
            for t in range(k):
                ranks[t, :n - t] = np.arange(n - t)
            med_l, gains_l = oracle.init_lab(D, k, ranks, gains=True)
            med_b, _, gains_b = oracle.pam_build(D, k)
            assert med_l.tolist() == list(med_b)
            assert np.allclose(gains_l, gains_b, rtol=0, atol=1e-9 * max(1.0, abs(gains_b[0])))


def test_init_lab_rank_mapping_and_errors():
    """Ranks name non-medoids in index order: with a one-point subsample
    the step-t choice is exactly that point; out-of-range or repeated ranks
    are rejected; LAB's subsample size is 10 + ceil(sqrt(n))."""
    D = bf.tiny_instances(414, 1, n_lo=8, n_hi=8)[0]
    ranks = np.array([[5], [5], [0], [4]], np.int32)
    # step 0 picks 5; non-medoids {0..4,6,7}: rank 5 -> 6; then {0..4,7}:
    # rank 0 -> 0; then {1..4,7}: rank 4 -> 7
    assert oracle.init_lab(D, 4, ranks).tolist() == [5, 6, 0, 7]
    with pytest.raises(ValueError):
        oracle.init_lab(D, 2, np.array([[0, 0], [1, 2]], np.int32))
    with pytest.raises(ValueError):
        oracle.init_lab(D, 2, np.array([[0, 1], [7, 2]], np.int32))
    assert [oracle.lab_sample_size(n) for n in (1, 2, 4, 5, 20000, 50000)] == \
        [11, 12, 12, 13, 152, 234]


def test_td_points_is_eq2_on_the_fp64_matrix():
    """TD of feature vectors (no matrix) = Eq. (2) by brute force with numpy
    FP64 distances; labels = lowest nearest slot; duplicated points give
    ties that go to the lower slot."""
    g = np.random.default_rng(415)
    for _ in range(20):
        n, d = int(g.integers(5, 60)), int(g.integers(1, 9))
        X = g.normal(size=(n, d)).astype(np.float32)
        X[-1] = X[0]                       # a duplicate: equal distances
        k = int(g.integers(1, n))
        med = g.choice(n, k, replace=False)
        A = np.sqrt(((X[:, None, :].astype(np.float64) - X[None, :, :]) ** 2).sum(-1))
        ref = A[:, med].min(axis=1).sum()
        v, lab = oracle.td_points(X, med, return_labels=True)
        assert abs(v - ref) <= 1e-12 * max(1.0, ref)
        assert (lab == np.argmin(A[:, med], axis=1)).all()
