"""Parity at the full benchmark sizes, in the launch configuration bench.py
times (automatic kernel geometry, BUILD + FastPAM1 via kmedoids_run).

The oracle cannot replay a whole n = 50000 run, so these tests check what
it can compute one by one: the final TD recomputed by Eq. (2), local
optimality of the result (one oracle FastPAM1 pass: no swap has Delta < 0),
sampled BUILD steps against the oracle's gains for the same prefix, and
sampled accepted swaps replayed from their pre-swap state (Delta within
1e-9 * TD and within 1e-6 * TD of the oracle's best).  At n = 20000 the
oracle also runs the whole method and the TDs must agree within 1e-6.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2008_05171_gb300.kmedoids as km  # noqa: E402
from paper_2008_05171_gb300 import workloads as wl  # noqa: E402


def _run_and_check(points, k, full_oracle):
    D = wl.euclidean_f32_torch(points, torch.device("cuda", 0))
    n = D.shape[0]
    b = km.build(D, k)
    out = km.run(D, k, trace=100000)
    torch.cuda.synchronize()
    Dh = D.cpu().numpy()
    bmed = b["medoids"].cpu().numpy()
    med = out["medoids"].cpu().numpy()
    assert len(set(med.tolist())) == k
    # exact TD of the result
    tdv = oracle.td(Dh, med)
    assert abs(out["td"] - tdv) <= 1e-9 * tdv
    assert abs(out["td_bookkept"] - tdv) <= 1e-9 * tdv
    # local optimality (Sec. 2): no single swap improves
    _, _, best = oracle.eval_swaps(Dh, med)
    assert best[0] >= -1e-9 * tdv, best
    # BUILD: sampled steps against the oracle's gains for the same prefix
    gains = out["build_gains"]
    for t in sorted({0, 1, k // 2, k - 1}):
        g = oracle.build_gains(Dh, bmed[:t])
        scale = abs(g[bmed[t]]) if t == 0 else tdv
        assert g[bmed[t]] <= g.min() + 1e-6 * scale, t
        assert abs(gains[t] - g[bmed[t]]) <= 1e-6 * scale, t
    # sampled accepted swaps replayed from their pre-swap state (P9)
    trace = out["trace"]
    assert out["iterations"] == out["swaps"] + 1
    assert len(trace) == out["swaps"]
    sample = sorted({0, len(trace) // 2, len(trace) - 1}) if trace else []
    cur = bmed.copy()
    for j, (d, i, c) in enumerate(trace):
        if j in sample:
            tcur = oracle.td(Dh, cur)
            dor = oracle.swap_delta(Dh, cur, i, c)
            assert abs(d - dor) <= 1e-9 * tcur, (j, d, dor)
            _, _, bst = oracle.eval_swaps(Dh, cur)
            assert dor <= bst[0] + 1e-6 * tcur
        cur[i] = c
    assert cur.tolist() == med.tolist()
    if full_oracle:
        ref = oracle.run(Dh, k, variant="fastpam1")
        assert abs(out["td"] - ref["td"]) <= 1e-6 * ref["td"]
    del D
    torch.cuda.empty_cache()
    return out


def test_fullsize_gmm_20000_k100():
    """n=20000, d=16, 100-cluster mixture, k=100 (the benchmark input)."""
    out = _run_and_check(wl.gmm_20000_points(), 100, full_oracle=True)
    assert out["swaps"] >= 1


def test_fullsize_gmm_50000_k200():
    """n=50000, d=32, 200 clusters, Dirichlet weights, k=200 (10 GB)."""
    _run_and_check(wl.gmm_50000_points(), 200, full_oracle=False)


def test_fullsize_fasterpam_20000():
    """FasterPAM at full size: every applied swap improves TD and the result
    is locally optimal."""
    D = wl.euclidean_f32_torch(wl.gmm_20000_points(), torch.device("cuda", 0))
    out = km.run(D, 100, variant="fasterpam", trace=100000)
    Dh = D.cpu().numpy()
    med = out["medoids"].cpu().numpy()
    tdv = oracle.td(Dh, med)
    assert abs(out["td"] - tdv) <= 1e-9 * tdv
    assert all(d < 0 for d, _, _ in out["trace"])
    _, _, best = oracle.eval_swaps(Dh, med)
    assert best[0] >= -1e-9 * tdv
