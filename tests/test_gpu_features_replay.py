"""On-the-fly form (bf16 tensor-core Gram distances) replayed step by step by
the FP64 oracle on the exact Euclidean matrix of the same features.

Every BUILD step (Alg. 1) and every accepted FastPAM1 swap (Alg. 3) of the
GPU run is re-evaluated by the oracle from the GPU's own pre-step state:

* the GPU's choice is the oracle's best wherever the best leads the
  runner-up by more than 1e-6 TD (the method's float tolerance); in a closer
  race it is within 1e-6 TD of the best.  When no race of a run is that
  close the oracle's own BUILD + FastPAM1 therefore makes exactly the GPU's
  choices and ends at the same medoids;
* the GPU's reported gain or Delta equals the oracle's value of the same
  choice within 1e-6 TD (P9);
* the final medoids admit no swap better than -1e-6 TD, and the reported TD
  is the exact TD of the medoids (1e-6 relative).

The tolerance covers what the Gram form changes: the FP32 accumulation of
x_o.x_c (relative error ~1e-6 on d^2 here) and the fixed-point rounding of
each distance (half a unit of 2^-q, q from the data's diameter), both
random in sign, summed over the few thousand pairs a candidate's Delta
collects."""
import numpy as np
import pytest

import oracle
from paper_2008_05171_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2008_05171_gb300.kmedoids as km  # noqa: E402


def _second_best_swap(Dh, med, cd, best):
    """Least Delta over every (slot, candidate) pair except the best one."""
    _, bs, bc = best
    rest = cd.copy()
    rest[bc] = np.inf
    for m in med:
        rest[m] = np.inf
    other = min((oracle.swap_delta(Dh, med, i, bc) for i in range(len(med)) if i != bs),
                default=np.inf)
    return min(float(rest.min()), other)


@pytest.mark.parametrize("n,d,k,centers", [(20000, 64, 40, 40), (6000, 128, 25, 20)])
def test_features_build_and_swaps_replayed_by_oracle(n, d, k, centers):
    X = wl.features_200000(n=n, d=d, n_centers=centers)
    Xt = torch.from_numpy(X).to(torch.bfloat16).cuda()
    Dh = wl.euclidean_f32_torch(X.astype(np.float64), "cuda").cpu().numpy()

    # ---------------------------------------------------------------- BUILD
    b = km.build_features(Xt, k)
    med_b = b["medoids"].cpu().numpy().astype(np.int32)
    assert len(set(med_b.tolist())) == k
    tol = 1e-6 * oracle.td(Dh, med_b)
    races = 0
    for t in range(k):
        g = oracle.build_gains(Dh, med_b[:t])
        c = int(med_b[t])
        order = np.argsort(g, kind="stable")
        best = int(order[0])
        if g[order[1]] - g[best] > tol:
            assert c == best, (t, c, best, g[c] - g[best])
        else:
            races += 1
            assert g[c] <= g[best] + tol, (t, g[c] - g[best])
        assert abs(b["build_gains"][t] - g[c]) <= tol, (t, b["build_gains"][t], g[c])
    assert abs(b["td"] - oracle.td(Dh, med_b)) <= 1e-6 * b["td"]

    # ------------------------------------------------- SWAP from the BUILD
    s = km.swap_features(Xt, med_b, trace=100000)
    assert s["converged"]
    med = med_b.copy()
    for j, (dg, slot, cand) in enumerate(s["trace"]):
        cd, _, best = oracle.eval_swaps(Dh, med)
        do = oracle.swap_delta(Dh, med, slot, cand)
        assert do < 0 and abs(dg - do) <= tol, (j, dg, do)
        if _second_best_swap(Dh, med, cd, best) - best[0] > tol:
            assert (slot, cand) == (best[1], best[2]), (j, slot, cand, best)
        else:
            races += 1
            assert do <= best[0] + tol, (j, do, best)
        med[slot] = cand
    assert s["medoids"].cpu().numpy().tolist() == med.tolist()
    _, _, best = oracle.eval_swaps(Dh, med)
    assert best[0] >= -tol, best                      # locally optimal (P5)
    tdo = oracle.td(Dh, med)
    assert abs(s["td"] - tdo) <= 1e-6 * tdo
    assert s["swaps"] == len(s["trace"])
    print("features replay n=%d d=%d k=%d: %d BUILD steps, %d swaps, %d close races"
          % (n, d, k, k, s["swaps"], races))
