"""Tensor-core (tcgen05) path of the on-the-fly distance form: the BF16 Gram
product against an FP32 reference.  BF16 products are exact in FP32, so
only the FP32 summation order differs: |G - G_ref| <= 1e-5 * sum |x_i y_i|."""
import numpy as np
import pytest

from paper_2008_05171_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2008_05171_gb300.kmedoids as km  # noqa: E402


@pytest.mark.parametrize("n,d", [(128, 16), (200, 64), (300, 128), (517, 256),
                                 (1000, 128)])
def test_gram_bf16_matches_fp32(n, d):
    X = wl.features_200000(n=n, d=d, n_centers=7)
    Xt = torch.from_numpy(X).to(torch.bfloat16)
    assert (Xt.float().numpy() == X).all()  # bf16-exact inputs
    G = km.gram_bf16(Xt.cuda()).cpu().numpy().astype(np.float64)
    X64 = X.astype(np.float64)
    ref = X64 @ X64.T
    bound = 1e-5 * (np.abs(X64) @ np.abs(X64).T) + 1e-6
    assert np.all(np.abs(G - ref) <= bound), np.max(np.abs(G - ref) / bound)


# ---------------------------------------------------------------- runs

import oracle  # noqa: E402


def _feat_case(n, d, centers, seed):
    X = wl.features_200000(n=n, d=d, n_centers=centers) if seed is None else \
        wl.to_bf16_values(wl.gmm_points(n, d, centers, seed=seed,
                                        center_std=2.0, center_box=None))
    Dh = wl.euclidean_f32(X.astype(np.float64))
    return X, Dh


@pytest.mark.parametrize("n,d,k", [(1000, 128, 8), (777, 64, 12), (2500, 128, 20)])
def test_run_features_matches_oracle(n, d, k):
    """BUILD + FastPAM1 with on-the-fly bf16 Gram distances: the TD it
    reports is exact for its medoids, every BUILD choice is the oracle's best
    up to the Gram rounding, the result is locally optimal and its TD equals
    the oracle's run on the exact matrix within 1e-6 (the method's float
    tolerance)."""
    X, Dh = _feat_case(n, d, max(2, k // 2), ("feat", n, d))
    Xt = torch.from_numpy(X).to(torch.bfloat16).cuda()
    out = km.run_features(Xt, k, trace=10000)
    med = out["medoids"].cpu().numpy()
    assert len(set(med.tolist())) == k
    tdv = oracle.td(Dh, med)
    assert abs(out["td"] - tdv) <= 1e-6 * tdv
    assert abs(out["td_bookkept"] - tdv) <= 1e-4 * tdv
    _, olab = oracle.td(Dh, med, return_labels=True)
    lab = out["labels"].cpu().numpy()
    assert np.mean(lab == olab) > 0.999
    _, _, best = oracle.eval_swaps(Dh, med)
    assert best[0] >= -1e-6 * tdv
    ref = oracle.run(Dh, k, variant="fastpam1")
    assert abs(out["td"] - ref["td"]) <= 1e-6 * ref["td"]


def test_build_features_steps():
    """kmedoids_build_features: the medoids in the order chosen and each
    step's gain, against the oracle's BUILD (Alg. 1) on the exact matrix:
    same choices, gains within 1e-6 of the BUILD's TD."""
    X, Dh = _feat_case(1500, 128, 6, "featb")
    Xt = torch.from_numpy(X).to(torch.bfloat16).cuda()
    out = km.build_features(Xt, 6)
    omed, otd, ogains = oracle.pam_build(Dh, 6)
    assert out["medoids"].cpu().tolist() == list(omed)
    assert np.all(np.abs(out["build_gains"] - ogains) <= 1e-6 * otd)
    assert abs(out["td"] - otd) <= 1e-6 * otd
    assert out["iterations"] == 0 and out["swaps"] == 0
    start = km.swap_features(Xt, [0, 1, 2, 3, 4, 5], max_iter=1)
    assert start["iterations"] >= 1


@pytest.mark.parametrize("n,d,k", [(20000, 64, 40), (6001, 128, 25)])
def test_incremental_build_equals_the_plain_pass(n, d, k):
    """The incremental BUILD (a dense pass for step 0, then each step updates
    every candidate's gain from the points the last commit moved) against
    the plain pass of every step: the same medoids in the same order, gains
    within 1e-6 of TD, and far fewer point rows streamed."""
    X = wl.features_200000(n=n, d=d, n_centers=k)
    Xt = torch.from_numpy(X).to(torch.bfloat16).cuda()
    a = km.build_features(Xt, k)
    b = km.build_features(Xt, k, build_full=True)
    assert a["medoids"].cpu().tolist() == b["medoids"].cpu().tolist()
    assert np.all(np.abs(a["build_gains"] - b["build_gains"]) <= 1e-6 * b["td"])
    assert abs(a["td"] - b["td"]) <= 1e-9 * b["td"]
    assert b["build_rows"] == n * k
    assert n <= a["build_rows"] < n * k // 4, a["build_rows"]


@pytest.mark.parametrize("n,d,k", [(20000, 64, 40), (6001, 128, 25), (3000, 32, 2)])
def test_incremental_swap_equals_the_plain_pass(n, d, k):
    """The incremental SWAP (every candidate's Eq. (7) sums kept across
    passes; each pass after the first moves only the entries of the points
    the last swap changed) against the plain FastPAM1 pass over every
    point: the same swaps in the same order, the same medoids and TD."""
    X = wl.features_200000(n=n, d=d, n_centers=max(k, 4))
    Xt = torch.from_numpy(X).to(torch.bfloat16).cuda()
    rng = np.random.default_rng(n)
    start = rng.choice(n, size=k, replace=False).astype(np.int32)
    a = km.swap_features(Xt, start, trace=100000)
    b = km.swap_features(Xt, start, trace=100000, swap_full=True)
    assert a["swaps"] >= 1 and a["converged"] and b["converged"]
    assert [(i, c) for _, i, c in a["trace"]] == [(i, c) for _, i, c in b["trace"]]
    # the two passes recover a pair's distance from differently folded MMA
    # outputs (the plain pass carries the threshold in the product), so the
    # Deltas agree to the Gram's rounding, well inside the 1e-6 TD tolerance
    for (da, _, _), (db, _, _) in zip(a["trace"], b["trace"]):
        assert abs(da - db) <= 1e-7 * b["td"]
    assert a["medoids"].cpu().tolist() == b["medoids"].cpu().tolist()
    assert abs(a["td"] - b["td"]) <= 1e-12 * b["td"]
    r = km.run_features(Xt, k)
    rf = km.run_features(Xt, k, swap_full=True)
    assert r["medoids"].cpu().tolist() == rf["medoids"].cpu().tolist()


@pytest.mark.parametrize("n,d", [(6001, 128), (3000, 64), (129, 16), (100, 32)])
def test_symmetric_gram_dense_pass(n, d):
    """The dense pass of the first BUILD step with each Gram tile pair
    computed once (default: candidate tile t takes the point blocks b >= t
    and sums the off-diagonal tiles along rows and columns) and with every
    tile in both orientations (gram_full), against the oracle's exact
    distance sums of step 0 (Alg. 1): the step's gain within 1e-6 of the
    least sum plus the error of the candidate's distance to itself (the
    Gram form gives d(c, c) as the square root of the rounding residue of
    |x_c|^2 + |x_c|^2 - 2 x_c.x_c, up to sqrt(2^-19 max |x|^2)), and the
    oracle's medoid (on these inputs the best sum leads the next by 0.18 %
    or more).  The points are taken in three orders so
    that the best candidate sits in different tiles (a dropped or doubled
    column sum moves the choice or the gain); 3-medoid runs of both forms
    take the same medoids."""
    X, Dh = _feat_case(n, d, 5, ("sym", n, d))
    self_pair = float(np.sqrt(2.0 ** -19 * (X.astype(np.float64) ** 2).sum(axis=1).max()))
    rng = np.random.default_rng(n + d)
    for perm in (np.arange(n), np.arange(n)[::-1], rng.permutation(n)):
        Xp = np.ascontiguousarray(X[perm])
        Dp = np.ascontiguousarray(Dh[:n, :n][np.ix_(perm, perm)])
        sums = oracle.build_gains(Dp, [])
        order = np.argsort(sums, kind="stable")
        best = float(sums[order[0]])
        assert sums[order[1]] - best > 1e-3 * best
        Xt = torch.from_numpy(Xp).to(torch.bfloat16).cuda()
        for full in (False, True):
            out = km.build_features(Xt, 1, gram_full=full)
            assert out["status_name"] == "KM_OK"
            assert abs(out["build_gains"][0] - best) <= 1e-6 * best + self_pair
            assert out["medoids"].cpu().tolist() == [int(order[0])]
        a = km.run_features(Xt, 3)
        b = km.run_features(Xt, 3, gram_full=True)
        assert a["medoids"].cpu().tolist() == b["medoids"].cpu().tolist()
        assert abs(a["td"] - b["td"]) <= 1e-9 * b["td"]


def test_run_features_many_tiles_per_cta():
    """n = 20000 gives 157 candidate tiles, more than there are SMs, so CTAs
    take several tiles each through the dynamic tile counter (and the tile
    hand-over between producer and epilogue); the run must equal the
    oracle's BUILD + FastPAM1 on the exact FP32 matrix within 1e-6 and its
    reported TD must be exact for its medoids."""
    n, d, k = 20000, 32, 16
    X = wl.to_bf16_values(wl.gmm_points(n, d, 12, seed="feat-many", center_std=2.0,
                                        center_box=None))
    Xt = torch.from_numpy(X).to(torch.bfloat16).cuda()
    out = km.run_features(Xt, k)
    med = out["medoids"].cpu().numpy()
    assert len(set(med.tolist())) == k
    D = wl.euclidean_f32_torch(X, torch.device("cuda", 0)).cpu().numpy()
    tdv = oracle.td(D, med)
    assert abs(out["td"] - tdv) <= 1e-6 * tdv
    ref = oracle.run(D, k, variant="fastpam1")
    assert abs(out["td"] - ref["td"]) <= 1e-6 * ref["td"]


def test_features_k1_and_k_equals_n():
    """k = 1: SWAP from any single medoid reaches the 1-medoid (Eq. (3)) by a
    dense pass (TD within 1e-5 of the exact 1-medoid's; the same medoid with
    each Gram tile pair once and with every tile); BUILD + SWAP with k = 1
    as well.  k = n: every point a medoid, TD 0."""
    X, Dh = _feat_case(900, 64, 4, "feat-k1")
    Xt = torch.from_numpy(X).to(torch.bfloat16).cuda()
    best = float(Dh[:900, :900].astype(np.float64).sum(axis=0).min())
    for start in ([0], [899], [450]):
        out = km.swap_features(Xt, start, trace=4)
        assert out["converged"]
        assert abs(out["td"] - best) <= 1e-5 * best
        assert out["swaps"] <= 1
    r = km.run_features(Xt, 1)
    assert abs(r["td"] - best) <= 1e-5 * best
    # the dense pass with every Gram tile (gram_full) reaches the same medoid
    for start in ([0], [899]):
        a = km.swap_features(Xt, start)
        b = km.swap_features(Xt, start, gram_full=True)
        assert a["medoids"].cpu().tolist() == b["medoids"].cpu().tolist()
        assert abs(a["td"] - b["td"]) <= 1e-12 * b["td"]
    small = torch.from_numpy(X[:40]).to(torch.bfloat16).cuda()
    z = km.run_features(small, 40)
    assert z["td"] == 0.0 and sorted(z["medoids"].cpu().tolist()) == list(range(40))
