"""The cheap initialisations of Sec. 3.3 on the CUDA path against the oracle.

Distance-weighted seeding and LAB draw their random numbers from the caller
(uniform numbers, subsample ranks); both sides weigh and score in the exact
fixed point of the SWAP sums, so the chosen medoids must be identical on
integer and on float data.  Sizes span one to several 32-point chunks per
thread of the seeding kernel (n > 32768), ragged tails, k = 1 and k = n,
coincident points (zero total weight) and the LAB limits."""
import numpy as np
import pytest

import oracle
from paper_2008_05171_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2008_05171_gb300.kmedoids as km  # noqa: E402


def _int_matrix(n, seed):
    return wl.manhattan_int32(wl.int_coords(n, 2, 1000, seed=seed))


def _float_matrix(n, seed, d=8, centers=20):
    return wl.euclidean_f32(wl.gmm_points(n, d, centers, seed=seed))


def _ranks(n, k, s, seed):
    g = wl.rng_for(("lab", seed))
    r = np.full((k, s), -1, np.int32)
    for t in range(k):
        m = min(s, n - t)
        r[t, :m] = g.choice(n - t, m, replace=False)
    return r


@pytest.mark.parametrize("n,k,float_data", [(1000, 10, False), (2999, 60, False),
                                            (2500, 40, True), (1031, 1, True),
                                            (64, 64, False)])
def test_init_weighted_matches_oracle(n, k, float_data):
    Dh = _float_matrix(n, ("w", n)) if float_data else _int_matrix(n, ("w", n))
    D = torch.from_numpy(Dh).cuda()
    for rep in range(3):
        u = wl.rng_for(("u", n, k, rep)).random(k)
        med = km.init_weighted(D, k, u).cpu().numpy()
        ref = oracle.init_weighted(Dh, k, u)
        assert med.tolist() == ref.tolist()
        assert len(set(med.tolist())) == k


def test_init_weighted_many_chunks_per_thread():
    """n = 36000 int32 (4 chunks of 32 points per thread in the search for
    the threshold's chunk); built on the device, checked against the
    oracle on the host copy."""
    n, k = 36000, 50
    P = torch.from_numpy(wl.int_coords(n, 2, 1000, seed="w-big").astype(np.int32)).cuda()
    D = torch.empty((n, n), dtype=torch.int32, device="cuda")
    for r0 in range(0, n, 4096):
        r1 = min(n, r0 + 4096)
        D[r0:r1] = (P[r0:r1, None, :] - P[None, :, :]).abs().sum(-1).to(torch.int32)
    u = wl.rng_for("u-big").random(k)
    med = km.init_weighted(D, k, u).cpu().numpy()
    Dh = D.cpu().numpy()
    del D
    assert med.tolist() == oracle.init_weighted(Dh, k, u).tolist()


def test_init_weighted_zero_weights_and_errors():
    Z = torch.zeros((100, 100), dtype=torch.float32, device="cuda")
    u = [0.37, 0.9, 0.1, 0.5]
    assert km.init_weighted(Z, 4, u).cpu().tolist() == \
        oracle.init_weighted(np.zeros((100, 100), np.float32), 4, u).tolist() == [37, 0, 1, 2]
    D = torch.from_numpy(_int_matrix(50, "w-err")).cuda()
    with pytest.raises(km.KmError) as e:
        km.init_weighted(D, 3, [0.1, 1.0, 0.2])
    assert e.value.status == 1


@pytest.mark.parametrize("n,k,float_data", [(1000, 10, False), (3000, 40, False),
                                            (2500, 30, True), (700, 1, True)])
def test_init_lab_matches_oracle(n, k, float_data):
    Dh = _float_matrix(n, ("l", n)) if float_data else _int_matrix(n, ("l", n))
    D = torch.from_numpy(Dh).cuda()
    s = oracle.lab_sample_size(n)
    ranks = _ranks(n, k, s, (n, k))
    med, gains = km.init_lab(D, k, ranks)
    ref, rg = oracle.init_lab(Dh, k, ranks, gains=True)
    assert med.cpu().tolist() == ref.tolist()
    assert np.array_equal(gains, rg)


def test_init_lab_full_subsamples_equal_build():
    """Whole non-medoid set as every subsample (s = n, padded rows): LAB is
    BUILD, on the GPU too (integer data: identical medoids and gains)."""
    n, k = 900, 12
    Dh = _int_matrix(n, "l-full")
    D = torch.from_numpy(Dh).cuda()
    ranks = np.full((k, n), -1, np.int32)
    for t in range(k):
        ranks[t, :n - t] = np.arange(n - t)
    med, gains = km.init_lab(D, k, ranks)
    b = km.build(D, k)
    assert med.cpu().tolist() == b["medoids"].cpu().tolist()
    assert gains.tolist() == list(b["build_gains"])


def test_init_lab_limits_and_errors():
    n = 300
    D = torch.from_numpy(_int_matrix(n, "l-err")).cuda()
    bad = _ranks(n, 3, 20, "e")
    bad[1, 0] = n - 1                   # outside [0, n - 1) at step 1
    with pytest.raises(km.KmError) as e:
        km.init_lab(D, 3, bad)
    assert e.value.status == 1
    rep = _ranks(n, 3, 20, "e")
    rep[2, 1] = rep[2, 0]
    with pytest.raises(km.KmError):
        km.init_lab(D, 3, rep)
    empty = _ranks(n, 3, 20, "e")
    empty[0, :] = -1
    with pytest.raises(km.KmError):
        km.init_lab(D, 3, empty)
    with pytest.raises(km.KmError) as e:
        km.init_lab(D, 2, np.zeros((2, 4097), np.int32))
    assert e.value.status == 7
    # the largest subsample: s = 4096 entries at n = 5000 (unused padding)
    n2 = 5000
    Dh = _float_matrix(n2, "l-max", d=4, centers=8)
    ranks = _ranks(n2, 5, 4096, "max")
    med, _ = km.init_lab(torch.from_numpy(Dh).cuda(), 5, ranks)
    assert med.cpu().tolist() == oracle.init_lab(Dh, 5, ranks).tolist()


def test_weighted_start_then_fasterpam_matches_oracle():
    """The paper's recommended pipeline (Sec. 6): distance-weighted start,
    then FasterPAM to convergence; integer data, identical swaps."""
    n, k = 2000, 20
    Dh = _int_matrix(n, "w-fp")
    D = torch.from_numpy(Dh).cuda()
    u = wl.rng_for("u-fp").random(k)
    start = km.init_weighted(D, k, u)
    out = km.swap(D, start, variant="fasterpam", trace=10000)
    ref = oracle.swap(Dh, oracle.init_weighted(Dh, k, u), variant="fasterpam")
    assert out["medoids"].cpu().tolist() == ref["medoids"].tolist()
    assert out["td_i64"] == int(ref["td"])
    assert out["swaps"] == ref["swaps"]
