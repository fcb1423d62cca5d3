"""Batched form (many PAM instances in one persistent launch) and CLARA
against the FP64 oracle.

The instance matrices are built on the device (FP64 differences, one
rounding to float32); each entry must lie within half a float32 ulp of
scipy's FP64 Euclidean distance.  The oracle then runs on the device's own
matrix, so every instance's BUILD + FastPAM1 result must match it: same
medoids, swaps and passes, TD within 1e-9 relative.  CLARA must pick the
same sample with the same medoids and per-sample TDs within 1e-6."""
import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle
from paper_2008_05171_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2008_05171_gb300.kmedoids as km  # noqa: E402


def _check_euclid(Dg, X):
    """Device matrix entries within half a float32 ulp of the FP64 distance
    (a correctly rounded FP64 -> float32 result), zero diagonal, symmetric."""
    n = X.shape[0]
    ref = cdist(X.astype(np.float64), X.astype(np.float64))
    got = Dg[:, :n]
    half_ulp = 0.5 * np.spacing(got).astype(np.float64)
    assert (np.abs(got.astype(np.float64) - ref) <= half_ulp * (1 + 1e-6) + 1e-300).all()
    assert (np.diag(got) == 0).all() and (got == got.T).all()


def _device_matrix(arena, inst, i, n):
    o, ld = int(inst[i]["offset"]), int(inst[i]["ld"])
    return np.ascontiguousarray(arena[o:o + n * ld].reshape(n, ld))


def _instances(count, n_lo, n_hi, k_hi, seed):
    g = np.random.default_rng(seed)
    specs = []
    for i in range(count):
        n = int(g.integers(n_lo, n_hi + 1))
        k = int(g.integers(1, min(k_hi, n) + 1))
        specs.append((n, k))
    specs += [(7, 7), (5, 1), (9, 2)]  # k = n, k = 1, tiny
    return specs


@pytest.mark.parametrize("tune", [0, 1, 2, 3, 4, 5])
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
        mo = int(inst[i]["medoid_offset"])
        Dg = _device_matrix(A, inst, i, n)
        _check_euclid(Dg, P[offs[i]:offs[i] + n])
        ref = oracle.run(Dg, k, variant="fastpam1")
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


def _run_specs(specs, seed, **kw):
    P, offs = wl.batched_points(specs, d=8, seed=seed)
    inst, arena_len, nmed = km.batch_layout(specs)
    inst_dev = torch.from_numpy(inst.view(np.uint8).copy()).cuda()
    arena = torch.zeros(arena_len, dtype=torch.float32, device="cuda")
    km.batched_distances(torch.from_numpy(P).cuda(), offs, inst_dev, arena)
    med, res = km.run_batched(arena, inst_dev, nmed, **kw)
    med = med.cpu().numpy()
    res = np.frombuffer(res.cpu().numpy().tobytes(), dtype=km.BATCH_RESULT_DTYPE)
    return P, offs, inst, med, res, arena.cpu().numpy()


def test_batched_long_rows_and_ragged_tails():
    """Rows of several 512-column ring stages with ragged last stages, up to
    the n = 4096 and k = 128 limits."""
    specs = [(4096, 128), (4093, 9), (1025, 40), (1537, 2), (513, 3), (2048, 1)]
    P, offs, inst, med, res, A = _run_specs(specs, "batched-long")
    for i, (n, k) in enumerate(specs):
        mo = int(inst[i]["medoid_offset"])
        Dg = _device_matrix(A, inst, i, n)
        _check_euclid(Dg, P[offs[i]:offs[i] + n])
        ref = oracle.run(Dg, k, variant="fastpam1")
        assert res[i]["status"] == 0, i
        assert med[mo:mo + k].tolist() == ref["medoids"].tolist(), (i, n, k)
        assert abs(res[i]["td"] - ref["td"]) <= 1e-9 * max(1.0, ref["td"]), i
        if k < n:
            assert res[i]["swaps"] == ref["swaps"], i
            assert res[i]["iterations"] == ref["iterations"], i


def test_batched_invalid_instance_reported_per_instance():
    """An instance outside the limits gets KM_E_INVALID in its own result;
    the other instances are solved."""
    specs = [(300, 5), (200, 4), (250, 6)]
    P, offs = wl.batched_points(specs, d=8, seed="batched-invalid")
    inst, arena_len, nmed = km.batch_layout(specs)
    inst[1]["k"] = 300  # k > n
    inst_dev = torch.from_numpy(inst.view(np.uint8).copy()).cuda()
    arena = torch.zeros(arena_len, dtype=torch.float32, device="cuda")
    km.batched_distances(torch.from_numpy(P).cuda(), offs, inst_dev, arena)
    med, res = km.run_batched(arena, inst_dev, nmed + 300)
    res = np.frombuffer(res.cpu().numpy().tobytes(), dtype=km.BATCH_RESULT_DTYPE)
    assert res[1]["status"] == 1
    assert res[0]["status"] == 0 and res[2]["status"] == 0
    med = med.cpu().numpy()
    A = arena.cpu().numpy()
    for i in (0, 2):
        n, k = specs[i]
        mo = int(inst[i]["medoid_offset"])
        ref = oracle.run(_device_matrix(A, inst, i, n), k, variant="fastpam1")
        assert med[mo:mo + k].tolist() == ref["medoids"].tolist(), i


def test_batched_graph_capture_replays():
    """kmedoids_run_batched enqueues only device work, so it can be captured
    in a CUDA graph; replays give the eager result."""
    specs = [(700, 12), (1100, 20), (300, 4), (64, 64)]
    P, offs = wl.batched_points(specs, d=8, seed="batched-graph")
    inst, arena_len, nmed = km.batch_layout(specs)
    inst_dev = torch.from_numpy(inst.view(np.uint8).copy()).cuda()
    arena = torch.zeros(arena_len, dtype=torch.float32, device="cuda")
    km.batched_distances(torch.from_numpy(P).cuda(), offs, inst_dev, arena)
    med0, res0 = km.run_batched(arena, inst_dev, nmed)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        med1, res1 = km.run_batched(arena, inst_dev, nmed)
    for _ in range(2):
        med1.fill_(-1)
        res1.fill_(0)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(med0, med1)
        assert torch.equal(res0, res1)


def test_restarts_from_random_starts_match_oracle():
    """kmedoids_swap_batched: several uniform random starting sets on the
    same matrices (instances sharing one arena offset), each FastPAM1 to
    convergence: every run equals the oracle's FastPAM1 from the same start
    (medoids, swaps, passes; TD within 1e-9), and the best-of-restarts pick
    is the oracle's."""
    specs = [(900, 12), (2600, 30), (515, 5)]
    P, offs = wl.batched_points(specs, d=8, seed="restarts")
    inst1, arena_len, _ = km.batch_layout(specs)
    arena = torch.zeros(arena_len, dtype=torch.float32, device="cuda")
    km.batched_distances(torch.from_numpy(P).cuda(), offs,
                         torch.from_numpy(inst1.view(np.uint8).copy()).cuda(), arena)
    R = 6
    g = np.random.default_rng(77)
    rows, starts, moff = [], [], 0
    for i, (n, k) in enumerate(specs):
        for r in range(R):
            rows.append((int(inst1[i]["offset"]), n, int(inst1[i]["ld"]), k, moff))
            starts.append(np.sort(g.choice(n, size=k, replace=False)).astype(np.int32))
            moff += k
    inst = np.array(rows, dtype=km.INSTANCE_DTYPE)
    med = torch.from_numpy(np.concatenate(starts)).cuda()
    inst_dev = torch.from_numpy(inst.view(np.uint8).copy()).cuda()
    med, res = km.swap_batched(arena, inst_dev, med)
    med = med.cpu().numpy()
    res = np.frombuffer(res.cpu().numpy().tobytes(), dtype=km.BATCH_RESULT_DTYPE)
    A = arena.cpu().numpy()
    for i, (n, k) in enumerate(specs):
        Do = _device_matrix(A, inst1, i, n)
        tds = []
        for r in range(R):
            j = i * R + r
            ref = oracle.swap(Do, starts[j], variant="fastpam1")
            mo = int(inst[j]["medoid_offset"])
            assert res[j]["status"] == 0
            assert med[mo:mo + k].tolist() == ref["medoids"].tolist(), (i, r)
            assert res[j]["swaps"] == ref["swaps"] and res[j]["iterations"] == ref["iterations"]
            assert abs(res[j]["td"] - ref["td"]) <= 1e-9 * ref["td"]
            tds.append(ref["td"])
        gpu_best = int(np.argmin([res[i * R + r]["td"] for r in range(R)]))
        assert gpu_best == int(np.argmin(tds))


def test_swap_batched_rejects_bad_starts():
    specs = [(300, 4), (300, 4)]
    P, offs = wl.batched_points(specs, d=8, seed="bad-starts")
    inst, arena_len, nmed = km.batch_layout(specs)
    inst_dev = torch.from_numpy(inst.view(np.uint8).copy()).cuda()
    arena = torch.zeros(arena_len, dtype=torch.float32, device="cuda")
    km.batched_distances(torch.from_numpy(P).cuda(), offs, inst_dev, arena)
    med = torch.tensor([1, 2, 3, 4, 7, 7, 8, 9], dtype=torch.int32, device="cuda")  # repeat
    med, res = km.swap_batched(arena, inst_dev, med)
    res = np.frombuffer(res.cpu().numpy().tobytes(), dtype=km.BATCH_RESULT_DTYPE)
    assert res[0]["status"] == 0 and res[1]["status"] == 1
    med2 = torch.tensor([1, 2, 3, 4, 5, 6, 7, 300], dtype=torch.int32, device="cuda")  # range
    _, res2 = km.swap_batched(arena, inst_dev, med2)
    res2 = np.frombuffer(res2.cpu().numpy().tobytes(), dtype=km.BATCH_RESULT_DTYPE)
    assert res2[1]["status"] == 1


def test_batched_fasterpam_restarts_and_build_match_oracle():
    """FasterPAM (Alg. 4) in the batched form: each CTA scans its instance
    in windows of one row per warp and applies the first improving swap at
    once.  From uniform random starts (several per matrix) and after BUILD,
    every instance's medoids, swap count, scans and TD equal the oracle's
    FasterPAM; instances span several 512-column ring stages, ragged tails
    and k from 2 to 128."""
    specs = [(900, 12), (2600, 30), (515, 5), (1500, 128), (40, 2)]
    P, offs = wl.batched_points(specs, d=8, seed="fp-batched")
    inst1, arena_len, nmed1 = km.batch_layout(specs)
    arena = torch.zeros(arena_len, dtype=torch.float32, device="cuda")
    inst1_dev = torch.from_numpy(inst1.view(np.uint8).copy()).cuda()
    km.batched_distances(torch.from_numpy(P).cuda(), offs, inst1_dev, arena)
    A = arena.cpu().numpy()
    mats = [_device_matrix(A, inst1, i, n) for i, (n, k) in enumerate(specs)]
    # BUILD + FasterPAM
    med_b, res_b = km.run_batched(arena, inst1_dev, nmed1, variant="fasterpam")
    med_b = med_b.cpu().numpy()
    res_b = np.frombuffer(res_b.cpu().numpy().tobytes(), dtype=km.BATCH_RESULT_DTYPE)
    for i, (n, k) in enumerate(specs):
        ref = oracle.run(mats[i], k, variant="fasterpam")
        mo = int(inst1[i]["medoid_offset"])
        assert res_b[i]["status"] == 0
        assert med_b[mo:mo + k].tolist() == ref["medoids"].tolist(), i
        assert res_b[i]["swaps"] == ref["swaps"] and res_b[i]["iterations"] == ref["iterations"]
        assert abs(res_b[i]["td"] - ref["td"]) <= 1e-9 * ref["td"]
    # restarts from random starts
    R = 3
    g = np.random.default_rng(78)
    rows, starts, moff = [], [], 0
    for i, (n, k) in enumerate(specs):
        for r in range(R):
            rows.append((int(inst1[i]["offset"]), n, int(inst1[i]["ld"]), k, moff))
            starts.append(np.sort(g.choice(n, size=k, replace=False)).astype(np.int32))
            moff += k
    inst = np.array(rows, dtype=km.INSTANCE_DTYPE)
    med = torch.from_numpy(np.concatenate(starts)).cuda()
    inst_dev = torch.from_numpy(inst.view(np.uint8).copy()).cuda()
    med, res = km.swap_batched(arena, inst_dev, med, variant="fasterpam")
    med = med.cpu().numpy()
    res = np.frombuffer(res.cpu().numpy().tobytes(), dtype=km.BATCH_RESULT_DTYPE)
    for i, (n, k) in enumerate(specs):
        for r in range(R):
            j = i * R + r
            ref = oracle.swap(mats[i], starts[j], variant="fasterpam")
            mo = int(inst[j]["medoid_offset"])
            assert res[j]["status"] == 0
            assert med[mo:mo + k].tolist() == ref["medoids"].tolist(), (i, r)
            assert res[j]["swaps"] == ref["swaps"] and res[j]["iterations"] == ref["iterations"]
            assert abs(res[j]["td"] - ref["td"]) <= 1e-9 * ref["td"]
    with pytest.raises(km.KmError) as e:
        km.run_batched(arena, inst1_dev, nmed1, variant="fastpam2")
    assert e.value.status == 7


def test_batched_autotune_picks_a_geometry_with_identical_results():
    """kmedoids_batched_autotune times every geometry of the persistent
    kernel on the batch and returns the fastest; results do not depend on
    the geometry, and the choice is cached per instance-size histogram."""
    specs = _instances(40, 50, 900, 25, 321)
    P, offs = wl.batched_points(specs, d=8, seed="batched-tune")
    inst, arena_len, nmed = km.batch_layout(specs)
    inst_dev = torch.from_numpy(inst.view(np.uint8).copy()).cuda()
    arena = torch.zeros(arena_len, dtype=torch.float32, device="cuda")
    km.batched_distances(torch.from_numpy(P).cuda(), offs, inst_dev, arena)
    g, ms = km.batched_autotune(arena, inst_dev, nmed)
    assert 1 <= g <= 5 and ms[g - 1] == min(m for m in ms if m >= 0)
    assert km.batched_autotune(arena, inst_dev, nmed, measure=False)[0] == g  # cached
    ref_med, ref_res = km.run_batched(arena, inst_dev, nmed, tune=1)
    for t in range(1, 6):
        med, res = km.run_batched(arena, inst_dev, nmed, tune=t)
        assert torch.equal(med, ref_med) and torch.equal(res, ref_res), t
    with pytest.raises(km.KmError):
        km.run_batched(arena, inst_dev, nmed, tune=6)


def _clara_case():
    X = wl.gmm_points(6000, 8, 10, seed="clara-test").astype(np.float32)
    k, samples = 5, 4
    S = wl.clara_samples(6000, samples, 80 + 4 * k, seed="clara-test")
    return X, k, S


def _check_clara(bc, X, k, S):
    omed, olab, otds, obest = oracle.clara(X, k, S)
    out = bc.clara_outcome()
    assert out["status"] == 0 and out["best_sample"] == obest
    assert np.allclose(bc.sample_td.cpu().numpy(), otds, rtol=1e-6, atol=0)
    assert bc.clara_medoids.cpu().numpy().tolist() == omed.tolist()
    assert np.mean(bc.labels.cpu().numpy() == olab) > 0.999
    assert abs(out["td"] - otds[obest]) <= 1e-6 * otds[obest]


def test_batch_and_clara_in_one_enqueue_captured_in_a_graph():
    """kmedoids_run_batched_clara: the batch's instances and CLARA's samples
    share one persistent PAM launch and the whole method (sample matrices,
    PAM, assignment, choice, labels) is device work only.  Eager and graph
    replays give the oracle's results for every instance and for CLARA."""
    specs = [(700, 12), (1100, 20), (300, 4), (64, 64), (2100, 33)]
    P, offs = wl.batched_points(specs, d=8, seed="batched-clara")
    inst, arena_len, nmed = km.batch_layout(specs)
    inst_dev = torch.from_numpy(inst.view(np.uint8).copy()).cuda()
    arena = torch.zeros(arena_len, dtype=torch.float32, device="cuda")
    km.batched_distances(torch.from_numpy(P).cuda(), offs, inst_dev, arena)
    X, k, S = _clara_case()
    bc = km.BatchedClara(arena, inst_dev, nmed, torch.from_numpy(X).cuda(), k,
                         torch.from_numpy(S).cuda())
    bc.enqueue()
    torch.cuda.synchronize()
    A = arena.cpu().numpy()

    def check_batch():
        med = bc.medoids.cpu().numpy()
        res = np.frombuffer(bc.results.cpu().numpy().tobytes(), dtype=km.BATCH_RESULT_DTYPE)
        for i, (n, kk) in enumerate(specs):
            ref = oracle.run(_device_matrix(A, inst, i, n), kk, variant="fastpam1")
            mo = int(inst[i]["medoid_offset"])
            assert res[i]["status"] == 0
            assert med[mo:mo + kk].tolist() == ref["medoids"].tolist(), i
            assert abs(res[i]["td"] - ref["td"]) <= 1e-9 * max(1.0, ref["td"])

    check_batch()
    _check_clara(bc, X, k, S)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bc.enqueue()
    for _ in range(2):
        bc.medoids.fill_(-1)
        bc.clara_medoids.fill_(-1)
        bc.results.fill_(0)
        bc.sample_td.fill_(0)
        g.replay()
        torch.cuda.synchronize()
        check_batch()
        _check_clara(bc, X, k, S)


def test_clara_alone_through_the_one_enqueue():
    """kmedoids_run_batched_clara with no batch instances (count 0) is
    CLARA as kmedoids_clara computes it."""
    X, k, S = _clara_case()
    bc = km.BatchedClara(None, None, 0, torch.from_numpy(X).cuda(), k,
                         torch.from_numpy(S).cuda())
    bc.enqueue()
    torch.cuda.synchronize()
    _check_clara(bc, X, k, S)
