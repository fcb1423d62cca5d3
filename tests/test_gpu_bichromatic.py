"""Bichromatic form (the paper's Outlook): medoids among m locations, TD
over n consumers, an m x n matrix of d(consumer, location) with rows =
locations.  The CUDA path against the FP64 bichromatic oracle:

* integer matrices (int32 and 16-bit): BUILD gains, medoids, the whole
  FastPAM1 swap trajectory, TD and labels bit-exact, for m < n, m > n,
  ragged tiles and padded rows;
* float matrices: the same medoids and trajectory (the sums are exact fixed
  point, the decisions the oracle's wherever they are not near ties) and TD
  to 1e-9;
* m = n with a symmetric matrix reproduces the square entry point;
* k = 1 gives the bichromatic medoid; SWAP from given locations; FasterPAM,
  FastPAM2 and FastCLARANS end in a local optimum of the oracle with its
  exact TD; invalid arguments are rejected."""
import numpy as np
import pytest

import oracle
from paper_2008_05171_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2008_05171_gb300.kmedoids as km  # noqa: E402


def rect(m, n, seed, integer=True, ld=None):
    L, C = wl.bichromatic_points(m, n, seed=seed, integer=integer)
    if integer:
        return wl.cross_manhattan_int32(L, C, ld=ld)
    return wl.cross_euclidean_f32(L, C, ld=ld)


def as_u16(Dh, n):
    ld = (Dh.shape[1] + 7) // 8 * 8
    U = np.zeros((Dh.shape[0], ld), np.uint16)
    U[:, :n] = Dh[:, :n]
    return torch.from_numpy(U.view(np.int16)).cuda()


@pytest.mark.parametrize("m,n,k", [(300, 2500, 12), (3000, 900, 20), (1031, 2049, 7),
                                   (64, 5000, 5)])
def test_int_run_is_bit_exact(m, n, k):
    Dh = rect(m, n, (m, n))
    ref = oracle.bi_run(Dh, k, n=n, trace_cap=10000)
    _, _, gains = oracle.bi_build(Dh, k, n=n)
    for D in (torch.from_numpy(Dh).cuda(), as_u16(Dh, n)):
        out = km.run_bichromatic(D, k, n, trace=10000)
        assert out["status_name"] == "KM_OK"
        assert list(out["build_gains"]) == gains.tolist()
        assert out["medoids"].cpu().tolist() == ref["medoids"].tolist()
        assert [(int(d), i, c) for d, i, c in out["trace"]] == \
            [(int(d), i, int(c)) for d, i, c in ref["trace"]]
        assert out["td_i64"] == int(ref["td"])
        _, lab = oracle.bi_td(Dh, ref["medoids"], n=n, return_labels=True)
        assert out["labels"].cpu().tolist() == lab.tolist()
        assert out["iterations"] == ref["iterations"]


@pytest.mark.parametrize("m,n,k", [(700, 3000, 15), (2100, 1300, 25)])
def test_float_run_matches_oracle(m, n, k):
    Dh = rect(m, n, ("f", m, n), integer=False)
    ref = oracle.bi_run(Dh, k, n=n, trace_cap=10000)
    out = km.run_bichromatic(torch.from_numpy(Dh).cuda(), k, n, trace=10000)
    assert out["medoids"].cpu().tolist() == ref["medoids"].tolist()
    assert [(i, c) for _, i, c in out["trace"]] == [(i, int(c)) for _, i, c in ref["trace"]]
    assert abs(out["td"] - ref["td"]) <= 1e-9 * ref["td"]
    for (dg, _, _), (do, _, _) in zip(out["trace"], ref["trace"]):
        assert abs(dg - do) <= 1e-9 * ref["td"]


def test_square_symmetric_matrix_reproduces_the_square_entry_point():
    Dh = wl.manhattan_int32(wl.int_coords(1500, 2, 1000, seed="bi-square"))
    D = torch.from_numpy(Dh).cuda()
    a = km.run_bichromatic(D, 11, 1500, trace=1000)
    b = km.run(D, 11, trace=1000)
    assert a["medoids"].cpu().tolist() == b["medoids"].cpu().tolist()
    assert a["trace"] == b["trace"] and a["td_i64"] == b["td_i64"]


def test_k1_is_the_bichromatic_medoid_and_swap_from_given_locations():
    m, n = 500, 1800
    Dh = rect(m, n, "k1")
    D = torch.from_numpy(Dh).cuda()
    sums = Dh[:, :n].astype(np.int64).sum(axis=1)
    out = km.run_bichromatic(D, 1, n)
    assert out["medoids"].cpu().tolist() == [int(np.argmin(sums))]
    worst = int(np.argmax(sums))
    s1 = km.swap_bichromatic(D, [worst], n)
    assert s1["medoids"].cpu().tolist() == [int(np.argmin(sums))]
    start = np.random.default_rng(3).choice(m, size=9, replace=False).astype(np.int32)
    s = km.swap_bichromatic(D, start, n, trace=1000)
    ref = oracle.bi_swap(Dh, start, n=n, trace_cap=1000)
    assert s["medoids"].cpu().tolist() == ref["medoids"].tolist()
    assert [(int(d), i, c) for d, i, c in s["trace"]] == \
        [(int(d), i, int(c)) for d, i, c in ref["trace"]]


@pytest.mark.parametrize("variant", ["fasterpam", "fastpam2", "fastclarans"])
def test_other_variants_end_in_a_local_optimum(variant):
    m, n, k = 900, 2200, 10
    Dh = rect(m, n, ("v", variant))
    D = torch.from_numpy(Dh).cuda()
    kw = {}
    if variant == "fastclarans":
        draws = np.random.default_rng(5).integers(0, m, size=200000).astype(np.int32)
        kw = dict(draws=torch.from_numpy(draws).cuda(), maxneighbor=m - k)
    out = km.run_bichromatic(D, k, n, variant=variant, **kw)
    assert out["status_name"] == "KM_OK", out["status_name"]
    med = out["medoids"].cpu().numpy()
    assert len(set(med.tolist())) == k and med.max() < m
    assert out["td_i64"] == int(oracle.bi_td(Dh, med, n=n))
    if variant != "fastclarans":  # FastCLARANS stops on failed draws, not at an optimum
        _, _, best = oracle.bi_eval_swaps(Dh, med, n=n)
        assert best[0] >= 0, best


def test_invalid_arguments():
    Dh = rect(100, 300, "inv")
    D = torch.from_numpy(Dh).cuda()
    with pytest.raises(km.KmError):
        km.swap_bichromatic(D, [1, 100], 300)      # location out of range
    with pytest.raises(km.KmError):
        km.swap_bichromatic(D, [4, 4], 300)        # repeated
    with pytest.raises(km.KmError):
        km.run_bichromatic(D, 101, 300)            # k > m
    with pytest.raises(km.KmError):
        km.run_bichromatic(D, 5, 300, check_input=True)
