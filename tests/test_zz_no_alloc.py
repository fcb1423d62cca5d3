"""kmedoids_eval_swaps_static: the FastPAM1 evaluation pass for callers that
cannot allocate device memory (frozen memory pools, plugins that must not use
the host application's allocator, real-time loops).  Its scratch is a fixed
array inside the library image instead of a caller workspace.

The test calls it through the C ABI twice in a row, on two different inputs,
and checks each result against kmedoids_eval_swaps with an ordinary
workspace: bit-exact on integer distances, within 1e-9 * TD on float ones
(the tolerance the other parity tests use for per-candidate Delta values).
This file is collected last so a run that stops at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from paper_2008_05171_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2008_05171_gb300.kmedoids as km  # noqa: E402


def _compare(Dh, med, exact):
    D = torch.from_numpy(Dh).cuda()
    cd_s, cs_s, best_s = km.eval_swaps_static(D, med)
    cd_w, cs_w, best_w = km.eval_swaps(D, med)
    torch.cuda.synchronize()
    cd_s, cd_w = cd_s.cpu().numpy(), cd_w.cpu().numpy()
    cs_s, cs_w = cs_s.cpu().numpy(), cs_w.cpu().numpy()
    if exact:
        assert (cd_s == cd_w).all() and (cs_s == cs_w).all()
        assert best_s == best_w
    else:
        tdv = float(np.sort(Dh[:, :Dh.shape[0]][:, med], axis=1)[:, 0].sum())
        fin = np.isfinite(cd_w)
        assert (np.isfinite(cd_s) == fin).all()
        assert np.max(np.abs(cd_s[fin] - cd_w[fin])) <= 1e-9 * tdv
        assert abs(best_s[0] - best_w[0]) <= 1e-9 * tdv


def test_static_scratch_matches_workspace_twice():
    Di = wl.manhattan_int32(wl.int_coords(3000, 2, 1000, seed="zz-int"))
    med_i = np.random.default_rng(1).choice(3000, 25, replace=False)
    Df = wl.euclidean_f32(wl.gmm_points(2300, 8, 20, seed="zz-f32"))
    med_f = np.random.default_rng(2).choice(2300, 40, replace=False)
    # two calls in a row share the scratch array: the second must not see
    # anything left over by the first
    _compare(Di, med_i, exact=True)
    _compare(Df, med_f, exact=False)
    _compare(Di, med_i, exact=True)


def test_static_scratch_rejects_oversize():
    D = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(km.KmError) as e:
        km.eval_swaps_static(D, [0, 1], n=40000)
    assert e.value.status == 7
