"""FastCLARANS (Sec. 3.4) on the CUDA path against the FP64 oracle.

The caller's candidate draws are evaluated in windows on the GPU; the first
improving draw in draw order is applied, and the failure count follows the
sequential algorithm, so the swaps, the draws consumed and evaluated and
the stopping point must equal the oracle's exactly on integer data (and the
medoids and TD on float data)."""
import numpy as np
import pytest

import oracle
from paper_2008_05171_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2008_05171_gb300.kmedoids as km  # noqa: E402


def _case(n, k, seed, float_data=False):
    if float_data:
        Dh = wl.euclidean_f32(wl.gmm_points(n, 8, max(2, k), seed=seed))
    else:
        Dh = wl.manhattan_int32(wl.int_coords(n, 2, 1000, seed=seed))
    g = wl.rng_for(("draws", seed))
    start = g.choice(n, size=k, replace=False).astype(np.int32)
    return Dh, start, g


@pytest.mark.parametrize("n,k,length,mn", [(300, 4, 2000, 7), (1500, 10, 9000, 37),
                                           (2100, 25, 20000, 2075), (900, 12, 500, 400)])
def test_clarans_int_exact(n, k, length, mn):
    Dh, start, g = _case(n, k, ("clarans", n, k))
    draws = g.integers(0, n, size=length).astype(np.int32)
    ref = oracle.clarans(Dh, start, draws, mn, trace_cap=100000)
    out = km.swap(torch.from_numpy(Dh).cuda(), start, variant="fastclarans",
                  draws=torch.from_numpy(draws).cuda(), maxneighbor=mn, trace=100000)
    assert out["medoids"].cpu().tolist() == ref["medoids"].tolist()
    assert out["swaps"] == ref["swaps"]
    assert [(int(d), i, c) for d, i, c in out["trace"]] == \
        [(int(d), i, c) for d, i, c in ref["trace"]]
    assert out["visited"] == ref["consumed"] and out["iterations"] == ref["evaluated"]
    assert out["converged"] == ref["stopped"]
    assert out["td_i64"] == ref["td"]


def test_clarans_cyclic_draws_equal_fasterpam():
    """Draws 0..n-1 repeated, maxneighbor = n - k: the GPU search makes the
    GPU FasterPAM's swaps (and the oracle's)."""
    n, k = 1200, 9
    Dh, start, _ = _case(n, k, "clarans-cyc")
    D = torch.from_numpy(Dh).cuda()
    draws = torch.from_numpy(np.tile(np.arange(n, dtype=np.int32), 40)).cuda()
    out = km.swap(D, start, variant="fastclarans", draws=draws, maxneighbor=n - k, trace=10000)
    fp = km.swap(D, start, variant="fasterpam", trace=10000)
    assert out["converged"]
    assert out["medoids"].cpu().tolist() == fp["medoids"].cpu().tolist()
    assert [(i, c) for _, i, c in out["trace"]] == [(i, c) for _, i, c in fp["trace"]]


def test_clarans_float_matches_oracle():
    n, k = 2500, 20
    Dh, start, g = _case(n, k, "clarans-f", float_data=True)
    draws = g.integers(0, n, size=12000).astype(np.int32)
    mn = int(0.025 * (n - k))
    ref = oracle.clarans(Dh, start, draws, mn, trace_cap=100000)
    out = km.swap(torch.from_numpy(Dh).cuda(), start, variant="fastclarans",
                  draws=torch.from_numpy(draws).cuda(), maxneighbor=mn, trace=100000)
    assert out["medoids"].cpu().tolist() == ref["medoids"].tolist()
    assert out["visited"] == ref["consumed"] and out["swaps"] == ref["swaps"]
    assert abs(out["td"] - ref["td"]) <= 1e-9 * ref["td"]
    for (d1, i1, c1), (d2, i2, c2) in zip(out["trace"], ref["trace"]):
        assert (i1, c1) == (i2, c2) and abs(d1 - d2) <= 1e-9 * ref["td"]


def test_clarans_draws_exhausted_and_invalid():
    n, k = 400, 5
    Dh, start, g = _case(n, k, "clarans-x")
    D = torch.from_numpy(Dh).cuda()
    draws = torch.from_numpy(g.integers(0, n, size=30).astype(np.int32)).cuda()
    out = km.swap(D, start, variant="fastclarans", draws=draws, maxneighbor=1000)
    ref = oracle.clarans(Dh, start, draws.cpu().numpy(), 1000)
    assert not out["converged"] and not ref["stopped"]
    assert out["medoids"].cpu().tolist() == ref["medoids"].tolist()
    assert out["visited"] == 30
    with pytest.raises(km.KmError):
        km.swap(D, start[:1], variant="fastclarans", draws=draws, maxneighbor=5)  # k = 1
    with pytest.raises(km.KmError):
        km.swap(D, start, variant="fastclarans", maxneighbor=5)  # no draws
