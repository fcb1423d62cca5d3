"""The compressed integer form (KM_U16): 16-bit unsigned distances, half
the bytes per matrix pass.  Every entry point of the matrix form must give
exactly what it gives on the same matrix stored as int32, and the oracle's
results: BUILD gains, FastPAM1 / FastPAM2 / FasterPAM / FastCLARANS
trajectories, the evaluation pass, the cache, the initialisations.  Sizes
span several 1024-column stages with ragged tails, values up to 65535."""
import numpy as np
import pytest

import oracle
from paper_2008_05171_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2008_05171_gb300.kmedoids as km  # noqa: E402


def _pair(n, seed, scale=1, ld=None):
    """(int32 host matrix, uint16 device matrix with row stride ld)."""
    Di = wl.manhattan_int32(wl.int_coords(n, 2, 1000, seed=seed)) * scale
    assert Di.max() <= 65535
    ld = ld or (n + 7) // 8 * 8
    U = np.zeros((n, ld), np.uint16)
    U[:, :n] = Di[:, :n]
    return np.ascontiguousarray(Di[:, :n]).astype(np.int32), torch.from_numpy(U.view(np.int16)).cuda()


@pytest.mark.parametrize("n,k,scale", [(1000, 10, 1), (2053, 25, 16), (3100, 40, 32)])
def test_u16_run_equals_int32_and_oracle(n, k, scale):
    Di, U = _pair(n, ("u16", n), scale)
    out = km.run(U, k, n=n, trace=100000)
    ref = oracle.run(Di, k, variant="fastpam1", trace_cap=100000)
    assert out["medoids"].cpu().tolist() == ref["medoids"].tolist()
    assert out["td_i64"] == int(ref["td"])
    assert [(int(d), i, c) for d, i, c in out["trace"]] == \
        [(int(d), i, c) for d, i, c in ref["trace"]]
    bmed, _, bg = oracle.pam_build(Di, k)
    assert list(out["build_gains"]) == list(bg)
    lab = out["labels"].cpu().numpy()
    _, olab = oracle.td(Di, ref["medoids"], return_labels=True)
    assert (lab == olab).all()


@pytest.mark.parametrize("variant", ["fasterpam", "fastpam2"])
def test_u16_variants_equal_oracle(variant):
    n, k = 2500, 30
    Di, U = _pair(n, ("u16v", variant), 8)
    start = np.sort(np.random.default_rng(3).choice(n, k, replace=False)).astype(np.int32)
    out = km.swap(U, start, n=n, variant=variant, trace=100000)
    ref = oracle.swap(Di, start, variant=variant, trace_cap=100000)
    assert out["medoids"].cpu().tolist() == ref["medoids"].tolist()
    assert out["td_i64"] == int(ref["td"]) and out["swaps"] == ref["swaps"]


def test_u16_clarans_eval_cache_and_inits():
    n, k = 1800, 15
    Di, U = _pair(n, "u16-misc", 30)
    Dd = torch.from_numpy(Di).cuda()
    g = np.random.default_rng(4)
    start = np.sort(g.choice(n, k, replace=False)).astype(np.int32)
    draws = g.integers(0, n, size=6000).astype(np.int32)
    a = km.swap(U, start, n=n, variant="fastclarans", draws=torch.from_numpy(draws).cuda(),
                maxneighbor=60, trace=10000)
    r = oracle.clarans(Di, start, draws, 60, trace_cap=10000)
    assert a["medoids"].cpu().tolist() == r["medoids"].tolist() and a["td_i64"] == r["td"]
    cd_u, cs_u, best_u = km.eval_swaps(U, start, n=n)
    cd_i, cs_i, best_i = km.eval_swaps(Dd, start)
    assert torch.equal(cd_u, cd_i) and torch.equal(cs_u, cs_i) and best_u == best_i
    near_u, sec_u, dn_u, ds_u, rl_u = km.cache(U, start, n=n)
    near_i, sec_i, dn_i, ds_i, rl_i = km.cache(Dd, start)
    assert torch.equal(near_u, near_i) and torch.equal(sec_u, sec_i)
    assert torch.equal(dn_u, dn_i) and torch.equal(ds_u, ds_i) and torch.equal(rl_u, rl_i)
    u = g.random(k)
    assert km.init_weighted(U, k, u, n=n).cpu().tolist() == oracle.init_weighted(Di, k, u).tolist()
    s = oracle.lab_sample_size(n)
    ranks = np.stack([g.choice(n - t, s, replace=False) for t in range(k)]).astype(np.int32)
    med_l, gains_l = km.init_lab(U, k, ranks, n=n)
    ref_l, ref_g = oracle.init_lab(Di, k, ranks, gains=True)
    assert med_l.cpu().tolist() == ref_l.tolist() and np.array_equal(gains_l, ref_g)


def test_u16_full_range_and_stride_rules():
    """Values up to 65535 (a scaled matrix) and a padded stride; a stride
    that is not a multiple of 8 is rejected."""
    n, k = 1500, 12
    Di = wl.manhattan_int32(wl.int_coords(n, 2, 1000, seed="u16-range"))
    Di = (Di.astype(np.int64) * 65535 // Di.max()).astype(np.int32)
    U = np.zeros((n, 1512), np.uint16)
    U[:, :n] = Di
    Ud = torch.from_numpy(U.view(np.int16)).cuda()
    out = km.run(Ud, k, n=n)
    ref = oracle.run(Di, k, variant="fastpam1")
    assert out["medoids"].cpu().tolist() == ref["medoids"].tolist()
    assert out["td_i64"] == int(ref["td"])
    bad = torch.zeros((100, 100), dtype=torch.int16, device="cuda")   # ld 100 % 8 != 0
    with pytest.raises(km.KmError) as e:
        km.run(bad, 3)
    assert e.value.status == 1
