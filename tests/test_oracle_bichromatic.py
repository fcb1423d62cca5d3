"""Pins of the bichromatic oracle (the paper's Outlook: medoids among m
locations, TD over n consumers, d(x_c, x_l) = D[l, c]) against what the
definitions and the square case fix:

* with m = n and a symmetric zero-diagonal matrix it is the square case:
  BUILD and FastPAM1 equal the pinned square oracle bit for bit;
* TD is Eq. (2) over the consumers (numpy min over the medoid rows);
* BUILD's first location is the bichromatic medoid argmin_l sum_c d(c, l),
  and every BUILD gain is the brute-force TD drop of the best addition;
* every FastPAM1 Delta (Eq. (7)) equals the TD recomputed after the swap;
* the run ends in a local optimum (no single swap lowers TD) and its
  bookkept TD is the recomputed TD.
A wrong index (rows and columns exchanged), a dropped term of Eq. (7) or a
wrong sign fails one of these on rectangular instances."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2008_05171_gb300 import workloads as wl


def rect_int(m, n, seed):
    L, C = wl.bichromatic_points(m, n, seed=seed, integer=True)
    return wl.cross_manhattan_int32(L, C)


def rect_float(m, n, seed):
    L, C = wl.bichromatic_points(m, n, seed=seed)
    return wl.cross_euclidean_f32(L, C)


def np_td(D, med, n):
    return float(D[np.asarray(med), :n].astype(np.float64).min(axis=0).sum())


@pytest.mark.parametrize("kind", ["int", "float"])
def test_square_symmetric_case_is_the_square_oracle(kind):
    if kind == "int":
        Dh = wl.manhattan_int32(wl.int_coords(140, 2, 1000, seed="bi-sq"))
    else:
        Dh = wl.euclidean_f32(wl.gmm_points(140, 4, 6, seed="bi-sq-f"))
    n = 140
    for k in (1, 2, 7):
        mb, tb, gb = oracle.bi_build(Dh, k, n=n)
        ms, ts, gs = oracle.pam_build(Dh, k, n=n)
        assert mb.tolist() == ms.tolist() and tb == ts and gb.tolist() == gs.tolist()
        rb = oracle.bi_run(Dh, k, n=n, trace_cap=500)
        rs = oracle.run(Dh, k, variant="fastpam1", n=n, trace_cap=500)
        assert rb["medoids"].tolist() == rs["medoids"].tolist()
        assert rb["trace"] == [(d, i, int(c)) for d, i, c in rs["trace"]]
        assert rb["td"] == rs["td"] and rb["iterations"] == rs["iterations"]


def test_td_is_eq2_over_the_consumers():
    D = rect_float(23, 57, 1)
    med = [3, 17, 9]
    td, lab = oracle.bi_td(D, med, n=57, return_labels=True)
    assert td == pytest.approx(np_td(D, med, 57), rel=1e-12)
    cols = D[np.asarray(med), :57]
    assert lab.tolist() == np.argmin(cols, axis=0).tolist()  # lowest slot on ties


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_build_first_location_is_the_bichromatic_medoid_and_gains_are_bruteforce(seed):
    m, n, k = 19, 33, 4
    D = rect_int(m, n, seed)
    med, td, steps = oracle.bi_build(D, k, n=n)
    sums = D[:, :n].astype(np.int64).sum(axis=1)
    assert med[0] == int(np.argmin(sums)) and steps[0] == sums.min()
    for t in range(1, k):
        base = np_td(D, med[:t], n)
        gains = [np_td(D, list(med[:t]) + [l], n) - base if l not in med[:t] else np.inf
                 for l in range(m)]
        assert med[t] == int(np.argmin(gains)) and steps[t] == min(gains)
    assert td == np_td(D, med, n)


@pytest.mark.parametrize("m,n,k", [(11, 17, 3), (25, 9, 4), (8, 40, 2)])
def test_eq7_deltas_equal_bruteforce_recomputation(m, n, k):
    for kind in ("int", "float"):
        D = rect_int(m, n, (m, n)) if kind == "int" else rect_float(m, n, (m, n))
        rng = np.random.default_rng(m * 100 + n)
        med = rng.choice(m, size=k, replace=False).astype(np.int32)
        cd7, cs7, b7 = oracle.bi_eval_swaps(D, med, method="fastpam1", n=n)
        cdb, csb, bb = oracle.bi_eval_swaps(D, med, method="bruteforce", n=n)
        tol = 0.0 if kind == "int" else 1e-9 * np_td(D, med, n)
        fin = np.isfinite(cdb)
        assert (np.isfinite(cd7) == fin).all()
        assert np.abs(cd7[fin] - cdb[fin]).max() <= tol
        if kind == "int":
            assert cs7.tolist() == csb.tolist() and b7 == bb
        # one swap by hand: TD(M - m_i + l) - TD(M)
        l = int(np.flatnonzero(fin)[0])
        i = int(cs7[l])
        trial = med.copy()
        trial[i] = l
        assert cd7[l] == pytest.approx(np_td(D, trial, n) - np_td(D, med, n), abs=tol + 1e-12)


@pytest.mark.parametrize("kind", ["int", "float"])
def test_run_ends_in_a_local_optimum_with_exact_bookkeeping(kind):
    m, n, k = 30, 70, 5
    D = rect_int(m, n, 7) if kind == "int" else rect_float(m, n, 7)
    r = oracle.bi_run(D, k, n=n, trace_cap=200)
    assert r["converged"] and r["swaps"] == len(r["trace"])
    med = r["medoids"]
    assert len(set(med.tolist())) == k and all(0 <= x < m for x in med)
    td = np_td(D, med, n)
    assert r["td"] == pytest.approx(td, rel=1e-12)
    assert r["td_bookkept"] == pytest.approx(td, rel=1e-9)
    for i in range(k):
        for l in range(m):
            if l in med:
                continue
            trial = med.copy()
            trial[i] = l
            assert np_td(D, trial, n) >= td - 1e-9 * td
    # every applied swap lowered TD by its Delta
    cur = r["build_medoids"].copy()
    for dlt, i, l in r["trace"]:
        before = np_td(D, cur, n)
        cur[i] = l
        assert dlt < 0 and dlt == pytest.approx(np_td(D, cur, n) - before, abs=1e-9 * before)
    assert cur.tolist() == med.tolist()


def test_k1_and_k_equal_m():
    D = rect_int(9, 25, 5)
    r = oracle.bi_run(D, 1, n=25)
    sums = D[:, :25].astype(np.int64).sum(axis=1)
    assert r["medoids"].tolist() == [int(np.argmin(sums))] and r["swaps"] == 0
    s = oracle.bi_swap(D, [8], n=25)  # from the worst single location
    assert s["medoids"].tolist() == [int(np.argmin(sums))]
    full = oracle.bi_run(D, 9, n=25)
    assert sorted(full["medoids"].tolist()) == list(range(9)) and full["swaps"] == 0


def test_tiny_exhaustive_optimum_bounds_the_run():
    m, n, k = 9, 14, 3
    D = rect_int(m, n, 13)
    best = min(np_td(D, list(c), n) for c in itertools.combinations(range(m), k))
    r = oracle.bi_run(D, k, n=n)
    assert r["td"] >= best
