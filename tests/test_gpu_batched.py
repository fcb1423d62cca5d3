"""Batched form (many PAM instances in one persistent launch) and CLARA
against the FP64 oracle.

The instance and sample matrices are built on the device with the same
FP64 recipe as the oracle, so the matrices are bitwise equal (checked);
then every instance's BUILD + FastPAM1 result must match the oracle's run:
same medoids, swaps and passes, TD within 1e-9 relative.  CLARA must pick
the same sample with the same medoids and per-sample TDs within 1e-6."""
import numpy as np
import pytest

import oracle
from paper_2008_05171_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2008_05171_gb300.kmedoids as km  # noqa: E402


def _instances(count, n_lo, n_hi, k_hi, seed):
    g = np.random.default_rng(seed)
    specs = []
    for i in range(count):
        n = int(g.integers(n_lo, n_hi + 1))
        k = int(g.integers(1, min(k_hi, n) + 1))
        specs.append((n, k))
    specs += [(7, 7), (5, 1), (9, 2)]  # k = n, k = 1, tiny
    return specs


@pytest.mark.parametrize("tune", [0, 1])
def test_batched_matches_oracle(tune):
    specs = _instances(36, 20, 700, 30, 123)
    P, offs = wl.batched_points(specs, d=8, seed="batched-test")
    inst, arena_len, nmed = km.batch_layout(specs)
    inst_dev = torch.from_numpy(inst.view(np.uint8).copy()).cuda()
    arena = torch.zeros(arena_len, dtype=torch.float32, device="cuda")
    km.batched_distances(torch.from_numpy(P).cuda(), offs, inst_dev, arena)
    med, res = km.run_batched(arena, inst_dev, nmed, tune=tune)
    med = med.cpu().numpy()
    res = np.frombuffer(res.cpu().numpy().tobytes(), dtype=km.BATCH_RESULT_DTYPE)
    A = arena.cpu().numpy()
    for i, (n, k) in enumerate(specs):
        o, ld, mo = int(inst[i]["offset"]), int(inst[i]["ld"]), int(inst[i]["medoid_offset"])
        Dg = A[o:o + n * ld].reshape(n, ld)
        Do = oracle.euclid_f32(P[offs[i]:offs[i] + n])
        assert (Dg[:, :n] == Do[:, :n]).all(), i  # bitwise equal matrices
        ref = oracle.run(Do, k, variant="fastpam1")
        got = med[mo:mo + k]
        assert got.tolist() == ref["medoids"].tolist(), (i, n, k)
        assert res[i]["status"] == 0
        assert abs(res[i]["td"] - ref["td"]) <= 1e-9 * max(1.0, ref["td"])
        if k < n:
            assert res[i]["swaps"] == ref["swaps"], i
            assert res[i]["iterations"] == ref["iterations"], i


def test_clara_matches_oracle():
    X = wl.gmm_points(6000, 8, 10, seed="clara-test").astype(np.float32)
    k, samples = 5, 4
    S = wl.clara_samples(6000, samples, 80 + 4 * k, seed="clara-test")
    out = km.clara(torch.from_numpy(X).cuda(), k, torch.from_numpy(S).cuda())
    omed, olab, otds, obest = oracle.clara(X, k, S)
    assert out["best_sample"] == obest
    assert np.allclose(out["sample_td"], otds, rtol=1e-6, atol=0)
    assert out["medoids"].cpu().numpy().tolist() == omed.tolist()
    lab = out["labels"].cpu().numpy()
    assert np.mean(lab == olab) > 0.999
    assert abs(out["td"] - otds[obest]) <= 1e-6 * otds[obest]
