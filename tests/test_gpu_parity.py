"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

Integer dissimilarities: bit-exact medoids, labels, TD, BUILD gains, swap
trajectories and per-candidate Delta values.  Float dissimilarities: the
tolerance the method allows -- TD within 1e-6 relative, per-candidate Delta
within 1e-9 * TD (the GPU sums each distance as an exact 64-bit fixed-point
value, the oracle sums FP64 values), and every accepted swap replayed by the
oracle from the same pre-swap state.
Sizes span several 1024-column chunks and candidate tiles with ragged
tails, padded row strides, and the degenerate k = 1, 2, n cases.
"""
import numpy as np
import pytest

import oracle
from paper_2008_05171_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2008_05171_gb300.kmedoids as km  # noqa: E402


def dev(Dh):
    return torch.from_numpy(np.ascontiguousarray(Dh)).cuda()


def int_instance(n, seed, hi=1000, dim=2, ld=None):
    X = wl.int_coords(n, dim, hi, seed=seed)
    return wl.manhattan_int32(X, ld=ld)


def float_instance(n, d, centers, seed, ld=None):
    X = wl.gmm_points(n, d, centers, seed=seed)
    return wl.euclidean_f32(X, ld=ld)


def rand_medoids(n, k, seed):
    return np.random.default_rng(seed).choice(n, size=k, replace=False)


INT_CASES = [(5, 2, None), (37, 3, 40), (300, 7, None), (1000, 10, None),
             (2100, 20, 2112), (2500, 40, None)]


# ------------------------------------------------------------------ cache

@pytest.mark.parametrize("n,k,ld", INT_CASES)
def test_cache_int(n, k, ld):
    Dh = int_instance(n, ("cache", n), ld=ld)
    med = rand_medoids(n, k, n)
    near, sec, dn, ds, rl = km.cache(dev(Dh), med)
    onear, osec, odn, ods = oracle.cache(Dh, med)
    assert (near.cpu().numpy() == onear).all()
    assert (sec.cpu().numpy() == osec).all()
    assert (dn.cpu().numpy() == odn).all()
    assert (ds.cpu().numpy() == ods).all()
    orl = oracle.removal_loss(onear, odn, ods, k)
    assert (rl.cpu().numpy() == orl).all()


def test_cache_float_and_k1():
    Dh = float_instance(1500, 8, 12, "cache-f")
    med = rand_medoids(1500, 12, 5)
    near, sec, dn, ds, rl = km.cache(dev(Dh), med)
    onear, osec, odn, ods = oracle.cache(Dh, med)
    assert (near.cpu().numpy() == onear).all()
    assert (dn.cpu().numpy().astype(np.float64) == odn).all()
    assert (ds.cpu().numpy().astype(np.float64) == ods).all()
    orl = oracle.removal_loss(onear, odn, ods, 12)
    assert np.allclose(rl.cpu().numpy(), orl, rtol=1e-12, atol=1e-9)
    near, sec, dn, ds, rl = km.cache(dev(Dh), [7])
    assert (near.cpu().numpy() == 0).all() and (sec.cpu().numpy() == -1).all()
    assert (dn.cpu().numpy() == Dh[:, 7]).all()


# ------------------------------------------------------------- evaluation

@pytest.mark.parametrize("n,k,ld", INT_CASES)
def test_eval_int_exact(n, k, ld):
    Dh = int_instance(n, ("eval", n), ld=ld)
    med = rand_medoids(n, k, n + 1)
    cd, cs, best = km.eval_swaps(dev(Dh), med)
    ocd, ocs, obest = oracle.eval_swaps(Dh, med, method="fastpam1")
    cd = cd.cpu().numpy()
    cs = cs.cpu().numpy()
    assert (cs == ocs).all()
    assert (cd == ocd).all()
    assert best == obest


@pytest.mark.parametrize("n,d,c,k", [(700, 4, 8, 8), (3000, 16, 30, 30),
                                     (2049, 8, 20, 64)])
def test_eval_float(n, d, c, k):
    Dh = float_instance(n, d, c, ("evalf", n))
    med = rand_medoids(n, k, n)
    cd, cs, best = km.eval_swaps(dev(Dh), med)
    ocd, ocs, obest = oracle.eval_swaps(Dh, med, method="fastpam1")
    cd = cd.cpu().numpy()
    cs = cs.cpu().numpy()
    tdv = oracle.td(Dh, med)
    tol = 1e-9 * tdv
    nm = ocs >= 0
    assert (cs[~nm] == -1).all()
    assert np.max(np.abs(cd[nm] - ocd[nm])) <= tol
    # the slot chosen is optimal up to the tolerance (exact ties may differ)
    for c_ in np.nonzero(nm & (cs != ocs))[0]:
        dl = oracle.swap_delta(Dh, med, cs[c_], c_)
        assert dl <= ocd[c_] + tol
    assert abs(best[0] - obest[0]) <= tol


# ----------------------------------------------------------------- BUILD

@pytest.mark.parametrize("n,k,ld", INT_CASES + [(1000, 1000, None)])
def test_build_int_exact(n, k, ld):
    Dh = int_instance(n, ("build", n), ld=ld)
    out = km.build(dev(Dh), k)
    omed, otd, ogains = oracle.pam_build(Dh, k)
    assert out["medoids"].cpu().numpy().tolist() == omed.tolist()
    assert out["td_i64"] == int(otd)
    assert out["build_gains"].tolist() == ogains.tolist()
    assert out["build_steps"] == k


def test_build_float():
    Dh = float_instance(2600, 16, 25, "build-f")
    k = 25
    out = km.build(dev(Dh), k)
    med = out["medoids"].cpu().numpy()
    tdv = oracle.td(Dh, med)
    assert abs(out["td"] - tdv) <= 1e-9 * tdv
    # replay each step: the GPU's choice is the oracle's best up to 1e-6*TD
    gains = out["build_gains"]
    for t in range(k):
        g = oracle.build_gains(Dh, med[:t])
        best = g.min()
        scale = abs(g[med[t]]) if t == 0 else tdv
        assert g[med[t]] <= best + 1e-6 * scale
        assert abs(gains[t] - g[med[t]]) <= 1e-6 * scale
        if g[med[t]] != best:
            second = np.partition(g, 1)[1]
            assert second - best <= 1e-6 * scale  # only near-ties may differ


@pytest.mark.parametrize("n,k,ld", [(37, 3, 40), (2100, 20, 2112), (2500, 40, None)])
def test_build_incremental_equals_full_pass_int(n, k, ld):
    """The default BUILD keeps every candidate's gain and updates it from
    the rows of the points whose d_n dropped; the plain pass (build_full)
    streams every candidate row each step.  Integer data: identical medoids,
    gains and TD, and the rows each streamed."""
    Dh = int_instance(n, ("inc", n), ld=ld)
    D = dev(Dh)
    a = km.build(D, k)
    b = km.build(D, k, build_full=True)
    assert a["medoids"].cpu().tolist() == b["medoids"].cpu().tolist()
    assert a["build_gains"].tolist() == b["build_gains"].tolist()
    assert a["td_i64"] == b["td_i64"]
    assert b["build_rows"] == sum(n - t for t in range(k))
    # step 0 and the first gains read every row once each; then |U| rows
    assert 2 * n <= a["build_rows"] <= 2 * n + (k - 2) * n
    assert a["build_launches"] == b["build_launches"] == k


def test_build_incremental_ties_and_empty_updates():
    """Many duplicate points (25 distinct positions, k = 40): later steps
    add duplicates with gain 0, no point's d_n drops (an empty update), and
    the lowest index must win every tie -- bit-exact against the oracle,
    for int32 and the 16-bit form."""
    n, k = 1500, 40
    X = wl.int_coords(n, 2, 5, seed="dups")
    Dh = wl.manhattan_int32(X)
    omed, otd, ogains = oracle.pam_build(Dh, k)
    out = km.build(dev(Dh), k)
    assert out["medoids"].cpu().tolist() == omed.tolist()
    assert out["build_gains"].tolist() == ogains.tolist()
    assert out["td_i64"] == int(otd) == 0
    ld = (n + 7) // 8 * 8
    U = np.zeros((n, ld), np.uint16)
    U[:, :n] = Dh[:, :n]
    u = km.build(torch.from_numpy(U.view(np.int16)).cuda(), k, n=n)
    assert u["medoids"].cpu().tolist() == omed.tolist()


def test_build_incremental_float_matches_full_pass():
    """Float data: the incremental gains are exact fixed-point sums
    (floor(d 2^f) per term), the plain pass sums FP32 with compensation;
    on a clustered matrix both pick the same medoids and their gains agree
    with the oracle's FP64 gains to 1e-9 of TD."""
    Dh = float_instance(3100, 16, 30, "inc-f", ld=3104)
    k = 30
    D = dev(Dh)
    a = km.build(D, k, n=3100)
    b = km.build(D, k, n=3100, build_full=True)
    assert a["medoids"].cpu().tolist() == b["medoids"].cpu().tolist()
    med = a["medoids"].cpu().numpy()
    tdv = oracle.td(Dh, med)
    assert abs(a["td"] - tdv) <= 1e-9 * tdv
    for t in (0, 1, 2, k // 2, k - 1):
        g = oracle.build_gains(Dh, med[:t])
        assert abs(a["build_gains"][t] - g[med[t]]) <= 1e-9 * (abs(g[med[t]]) if t == 0 else tdv)
    assert a["build_rows"] < b["build_rows"] / 3


# ------------------------------------------------------------ full runs

def assert_same_run(out, ref):
    assert out["medoids"].cpu().numpy().tolist() == ref["medoids"].tolist()
    assert out["td_i64"] == int(ref["td"])
    assert out["swaps"] == ref["swaps"]
    assert out["iterations"] == ref["iterations"]
    assert [(int(d), i, c) for d, i, c in out["trace"]] == \
        [(int(d), i, c) for d, i, c in ref["trace"]]


@pytest.mark.parametrize("variant", ["fastpam1", "fasterpam", "fastpam2"])
@pytest.mark.parametrize("n,k,ld", INT_CASES)
def test_swap_int_exact(variant, n, k, ld):
    Dh = int_instance(n, ("swap", n), ld=ld)
    start = rand_medoids(n, k, n + 7)
    out = km.swap(dev(Dh), start, variant=variant, trace=100000)
    ref = oracle.swap(Dh, start, variant=variant, trace_cap=100000)
    assert_same_run(out, ref)
    if variant == "fasterpam":
        assert out["visited"] == ref["visited"]
    lab = out["labels"].cpu().numpy()
    _, olab = oracle.td(Dh, ref["medoids"], return_labels=True)
    assert (lab == olab).all()


def test_run_manhattan_1000_exact():
    """Integer workload: n=1000 Manhattan int32, k=10, BUILD + FastPAM1."""
    Dh, k = wl.manhattan_1000()
    out = km.run(dev(Dh), k, trace=1000)
    ref = oracle.run(Dh, k, variant="fastpam1")
    assert_same_run(out, ref)
    assert out["build_gains"].tolist() == oracle.pam_build(Dh, k)[2].tolist()
    for v in ("fasterpam", "fastpam2"):
        o2 = km.run(dev(Dh), k, variant=v, trace=1000)
        r2 = oracle.run(Dh, k, variant=v)
        assert_same_run(o2, r2)


def replay_float(Dh, start, out, sample=None, kind="fastpam1"):
    """Every accepted swap: |Delta_gpu - Delta_oracle| <= 1e-9 * TD and
    Delta_oracle < 0; for FastPAM1 it is within 1e-6 * TD of the oracle's
    best swap of that state, for FasterPAM within 1e-6 * TD of the best slot
    for that candidate (Alg. 4 swaps each candidate with its best slot)."""
    med = np.array(start, np.int32)
    trace = out["trace"]
    idx = range(len(trace)) if sample is None else sample
    for j, (d, i, c) in enumerate(trace):
        if j in idx:
            tdv = oracle.td(Dh, med)
            dor = oracle.swap_delta(Dh, med, i, c)
            assert abs(d - dor) <= 1e-9 * tdv, (j, d, dor)
            assert dor < 1e-9 * tdv
            if kind in ("fastpam1", "fasterpam"):
                cd, _, best = oracle.eval_swaps(Dh, med)
                ref = best[0] if kind == "fastpam1" else cd[c]
                assert dor <= ref + 1e-6 * tdv
        med[i] = c
    assert med.tolist() == out["medoids"].cpu().numpy().tolist()
    return med


@pytest.mark.parametrize("variant", ["fastpam1", "fasterpam", "fastpam2"])
def test_swap_float(variant):
    Dh = float_instance(2500, 16, 20, ("swapf", variant))
    start = rand_medoids(2500, 20, 3)
    out = km.swap(dev(Dh), start, variant=variant, trace=100000)
    kind = "fastpam1" if variant == "fastpam1" else (
        "fasterpam" if variant == "fasterpam" else "fastpam2")
    med = replay_float(Dh, start, out, kind=kind)
    tdv = oracle.td(Dh, med)
    assert abs(out["td"] - tdv) <= 1e-9 * tdv
    assert abs(out["td_bookkept"] - tdv) <= 1e-9 * tdv
    _, _, best = oracle.eval_swaps(Dh, med)
    assert best[0] >= -1e-9 * tdv  # locally optimal
    ref = oracle.swap(Dh, start, variant=variant)
    if variant == "fastpam1":
        assert abs(out["td"] - ref["td"]) <= 1e-6 * ref["td"]


def test_run_float_gmm():
    Dh = float_instance(4000, 16, 40, "runf")
    k = 40
    out = km.run(dev(Dh), k, trace=10000)
    ref = oracle.run(Dh, k, variant="fastpam1")
    assert abs(out["td"] - ref["td"]) <= 1e-6 * ref["td"]
    if out["medoids"].cpu().numpy().tolist() != ref["medoids"].tolist():
        # divergence is allowed only through near-ties
        replay_float(Dh, ref["build_medoids"], out)


# --------------------------------------------------------- degenerate k

@pytest.mark.parametrize("dtype", ["int", "float"])
def test_k_equals_one(dtype):
    Dh = int_instance(900, "k1") if dtype == "int" else \
        float_instance(900, 4, 3, "k1f")
    for v in ("fastpam1", "fasterpam", "fastpam2"):
        out = km.swap(dev(Dh), [899], variant=v, trace=10)
        ref = oracle.swap(Dh, [899], variant=v)
        assert out["medoids"].cpu().numpy().tolist() == ref["medoids"].tolist()
        assert out["iterations"] == ref["iterations"]
        assert out["swaps"] == ref["swaps"]
        assert abs(out["td"] - ref["td"]) <= 1e-6 * ref["td"]
    out = km.run(dev(Dh), 1)
    omed, otd, _ = oracle.pam_build(Dh, 1)
    assert out["medoids"].cpu().numpy().tolist() == omed.tolist()
    assert out["swaps"] == 0


def test_k_equals_n_and_tiny():
    Dh = int_instance(6, "kn")
    out = km.run(dev(Dh), 6)
    assert out["td_i64"] == 0 and out["swaps"] == 0
    assert sorted(out["medoids"].cpu().numpy().tolist()) == list(range(6))
    for n in (2, 3, 4):
        Dh = int_instance(n, ("tiny", n))
        for k in range(1, n + 1):
            out = km.run(dev(Dh), k, trace=64)
            ref = oracle.run(Dh, k, variant="fastpam1")
            assert out["medoids"].cpu().numpy().tolist() == ref["medoids"].tolist()
            assert out["td_i64"] == int(ref["td"])


def test_all_distances_equal():
    Dh = np.zeros((64, 64), np.int32)
    out = km.run(dev(Dh), 5, trace=64)
    ref = oracle.run(Dh, 5, variant="fastpam1")
    assert out["medoids"].cpu().numpy().tolist() == ref["medoids"].tolist()
    assert out["td_i64"] == 0 and out["swaps"] == 0


def test_duplicates_and_ties():
    X = np.repeat(wl.int_coords(150, 2, 8, seed="dup"), 3, axis=0)
    Dh = wl.manhattan_int32(X)
    for v in ("fastpam1", "fasterpam", "fastpam2"):
        out = km.run(dev(Dh), 12, variant=v, trace=10000)
        ref = oracle.run(Dh, 12, variant=v)
        assert_same_run(out, ref)


def test_max_iter_not_converged():
    Dh = int_instance(800, "cap")
    start = rand_medoids(800, 10, 1)
    full = oracle.swap(Dh, start, variant="fastpam1")
    assert full["swaps"] >= 2
    out = km.swap(dev(Dh), start, max_iter=1, trace=10)
    assert out["status_name"] == "KM_E_NOT_CONVERGED"
    assert out["swaps"] == 1 and out["iterations"] == 1
    assert out["trace"][0][1:] == full["trace"][0][1:]


@pytest.mark.parametrize("kind", ["i32", "f32", "u16"])
def test_swap_loop_graph_equals_host_driven_loop(kind):
    """FastPAM1 without per-pass timing runs its SWAP loop as one CUDA graph
    (a conditional WHILE node: pass, swap, device-side loop condition); with
    profile = 1 the host drives the passes.  Both take the same swaps in the
    same order; the launch counts show which loop ran.  A max_iter cap ends both after that many
    passes, not converged."""
    if kind == "f32":
        Dh = float_instance(2500, 8, 12, "graph-f")
    else:
        Dh = int_instance(2500, ("graph", kind))
    D = dev(Dh)
    if kind == "u16":  # 16-bit entries, rows padded to 8 elements
        U = np.zeros((2500, 2504), np.uint16)
        U[:, :2500] = Dh
        D = torch.from_numpy(U.view(np.int16)).cuda()
    g = km.run(D, 14, n=2500, trace=1000)
    h = km.run(D, 14, n=2500, trace=1000, profile=True)
    assert g["medoids"].cpu().tolist() == h["medoids"].cpu().tolist()
    assert g["trace"] == h["trace"] and g["td"] == h["td"]
    assert g["iterations"] == h["iterations"] and g["swaps"] >= 1
    # graph: pass, swap and condition per body, one body per pass; host
    # loop: pass and swap per launch, launched in batches of 1, 2, 4, .. 64
    # between reads of the state (the passes after convergence exit at once)
    launched, batch = 0, 1
    while launched < h["iterations"]:
        launched, batch = launched + batch, min(2 * batch, 64)
    assert g["kernel_launches"] - 3 * g["iterations"] == h["kernel_launches"] - 2 * launched
    start = rand_medoids(2500, 14, 5)
    for cap in (1, 2, 3):
        a = km.swap(D, start, n=2500, max_iter=cap, trace=10)
        b = km.swap(D, start, n=2500, max_iter=cap, trace=10, profile=True)
        assert a["status_name"] == b["status_name"] == "KM_E_NOT_CONVERGED"
        assert a["iterations"] == b["iterations"] == cap
        assert a["trace"] == b["trace"] and a["swaps"] == cap
    # a second call with the same arguments replays the cached graph
    g2 = km.run(D, 14, n=2500, trace=1000)
    assert g2["medoids"].cpu().tolist() == g["medoids"].cpu().tolist()
    assert g2["kernel_launches"] == g["kernel_launches"]


def test_swap_loop_graph_cache_evicts_and_rebuilds():
    """More distinct argument sets than the graph cache keeps (8): every run
    still equals the oracle, including a repeat of the first after it was
    evicted."""
    Dh = int_instance(900, "graph-cache")
    D = dev(Dh)
    ks = list(range(3, 14))
    for k in ks + [ks[0]]:
        out = km.run(D, k, trace=500)
        ref = oracle.run(Dh, k, variant="fastpam1")
        assert out["medoids"].cpu().tolist() == ref["medoids"].tolist(), k
        assert out["td_i64"] == int(ref["td"]), k


@pytest.mark.parametrize("fill", [0x00, 0xA5, 0xFF])
def test_workspace_contents_do_not_matter(fill):
    """Every call initialises what it reads of the caller's workspace: the
    same BUILD, BUILD + SWAP and SWAP results (state records, counters,
    TD, trace) from a workspace filled with any byte pattern."""
    Dh = int_instance(1500, "dirty")
    D = dev(Dh)
    ref_b = oracle.pam_build(Dh, 11)
    ref = oracle.run(Dh, 11, variant="fastpam1")
    opts = km.options(trace=1000)
    ws = km.workspace(1500, 11, km.KM_I32, opts)
    for call in ("build", "run", "swap"):
        ws.fill_(fill)
        if call == "build":
            out = km.build(D, 11, ws=ws, trace=1000)
            assert out["medoids"].cpu().tolist() == ref_b[0].tolist()
            assert out["build_steps"] == 11 and out["td_i64"] == int(ref_b[1])
        elif call == "run":
            out = km.run(D, 11, ws=ws, trace=1000)
            assert_same_run(out, ref)
            assert out["build_steps"] == 11
        else:
            out = km.swap(D, ref_b[0], ws=ws, trace=1000)
            assert_same_run(out, ref)


def test_invalid_medoids_and_workspace():
    Dh = int_instance(100, "inv")
    D = dev(Dh)
    with pytest.raises(km.KmError):
        km.swap(D, [1, 1, 2])
    with pytest.raises(km.KmError):
        km.swap(D, [1, 200])
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(km.KmError) as e:
        km.run(D, 5, ws=ws)
    assert e.value.status == 2


def test_stream_and_workspace_reuse():
    Dh = int_instance(1200, "reuse")
    D = dev(Dh)
    code = km.KM_I32
    ws = km.workspace(1200, 9, code, km.options(trace=100))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = km.run(D, 9, ws=ws, trace=100)
        b = km.run(D, 9, ws=ws, trace=100)
    s.synchronize()
    assert a["medoids"].cpu().tolist() == b["medoids"].cpu().tolist()
    assert a["td_i64"] == b["td_i64"]


@pytest.mark.parametrize("variant", ["fastpam1", "fasterpam", "fastpam2"])
def test_measured_geometry_same_result(variant):
    """tune = -1 times every geometry that fits on the first call for a shape
    and keeps the fastest; the result equals the automatic choice's (exact
    sums, total orders), the chosen entries are reported, and a second call
    reuses them."""
    Dh = int_instance(3000, ("tune", variant))
    D = dev(Dh)
    a = km.run(D, 12, variant=variant)
    b = km.run(D, 12, variant=variant, tune=-1)
    c = km.run(D, 12, variant=variant, tune=-1)
    for r in (b, c):
        assert r["medoids"].cpu().tolist() == a["medoids"].cpu().tolist()
        assert r["td_i64"] == a["td_i64"] and r["swaps"] == a["swaps"]
        assert r["build_geometry"] == 0  # incremental BUILD: no table entry
        # the eager variants run in their own persistent kernel (geometry 0)
        assert (r["swap_geometry"] == 0) if variant == "fasterpam" else \
            (1 <= r["swap_geometry"] <= 16)
    assert (b["swap_geometry"], b["build_geometry"]) == (c["swap_geometry"], c["build_geometry"])
    # no timing passes the second time (the eager SWAP kernel has none, and
    # BUILD was tuned for this shape by the first parameter of this test)
    if variant == "fasterpam":
        assert c["kernel_launches"] <= b["kernel_launches"]
    else:
        assert c["kernel_launches"] < b["kernel_launches"]


@pytest.mark.parametrize("rows", [1, 4, 16])
def test_fasterpam_window_lengths_same_trajectory(rows):
    """FasterPAM and FastCLARANS evaluate adaptive windows of scan positions
    (one per CTA after a swap, doubling after a window without one); the
    trajectory is that of the sequential scan (Alg. 4) whatever the tile
    rows, i.e. whatever the largest window: integer data from a random
    start with frequent swaps (k = 40), against the oracle."""
    n, k = 2600, 40
    Dh = int_instance(n, ("win", rows))
    start = rand_medoids(n, k, 99)
    out = km.swap(dev(Dh), start, variant="fasterpam", rows_per_tile=rows, trace=100000)
    ref = oracle.swap(Dh, start, variant="fasterpam", trace_cap=100000)
    assert_same_run(out, ref)
    assert out["visited"] == ref["visited"]
    # candidates evaluated by the sequential scan: the non-medoid positions
    # visited, replaying the swaps where the scan meets their candidates
    med, ev, sw, p = list(start), 0, 0, 0
    trace = ref["trace"]
    while p < ref["visited"]:
        r = p % n
        if r not in med:
            ev += 1
            if sw < len(trace) and trace[sw][2] == r:
                med[trace[sw][1]] = r
                sw += 1
        p += 1
    assert sw == len(trace) and out["evaluated"] == ev


def test_apply_rescans_large_k():
    """The swap's cache update rescans a point with a whole warp (lanes over
    the slots, butterfly merge of top-2 lists): k = 150 (several slots per
    lane), ties from duplicated points; every FastPAM1 decision and the
    final labels equal the oracle's."""
    n, k = 3000, 150
    P = np.repeat(wl.int_coords(n // 2, 2, 60, seed="rescan"), 2, axis=0)
    Dh = wl.manhattan_int32(P)
    start = rand_medoids(n, k, 5)
    out = km.swap(dev(Dh), start, variant="fastpam1", trace=100000)
    ref = oracle.swap(Dh, start, variant="fastpam1", trace_cap=100000)
    assert_same_run(out, ref)
    # labels come from the incrementally updated cache
    _, olab = oracle.td(Dh, ref["medoids"], return_labels=True)
    assert (out["labels"].cpu().numpy() == olab).all()


def test_check_input_reports_broken_matrices():
    """check_input: one extra pass over D verifies the method's assumptions
    (zero diagonal, symmetry; finite entries >= 0 for float data) before any
    other work; valid matrices run unchanged (int32, float32, 16-bit)."""
    n, k = 1100, 9
    Dh = int_instance(n, "check")
    ref = km.run(dev(Dh), k, trace=1000)
    ok = km.run(dev(Dh), k, trace=1000, check_input=True)
    assert ok["medoids"].cpu().tolist() == ref["medoids"].cpu().tolist()
    assert ok["td_i64"] == ref["td_i64"]
    A = Dh.copy()
    A[700, 3] += 1                                   # d(700, 3) != d(3, 700)
    with pytest.raises(km.KmError) as e:
        km.run(dev(A), k, check_input=True)
    assert e.value.status == 1 and "symmetric" in str(e.value)
    B = Dh.copy()
    B[1099, 1099] = 5                                # last diagonal entry, ragged tile
    with pytest.raises(km.KmError) as e:
        km.swap(dev(B), rand_medoids(n, k, 1), check_input=True)
    assert e.value.status == 1 and "diagonal" in str(e.value)
    F = wl.euclidean_f32(wl.gmm_points(700, 4, 5, seed="check-f"))
    assert km.run(dev(F), 5, check_input=True)["converged"]
    G = F.copy()
    G[10, 20] = G[20, 10] = np.float32(np.nan)
    with pytest.raises(km.KmError) as e:
        km.run(dev(G), 5, check_input=True)
    assert e.value.status == 6
    U = np.zeros((n, 1104), np.uint16)
    U[:, :n] = Dh[:, :n]
    Ud = torch.from_numpy(U.view(np.int16)).cuda()
    assert km.run(Ud, k, n=n, check_input=True)["td_i64"] == ref["td_i64"]
    U[5, 6] += 1
    with pytest.raises(km.KmError) as e:
        km.run(torch.from_numpy(U.view(np.int16)).cuda(), k, n=n, check_input=True)
    assert e.value.status == 1


@pytest.mark.parametrize("variant", ["fasterpam", "fastpam2"])
def test_tiny_and_nearly_full_k_all_variants(variant):
    """Every k from 1 to n on tiny matrices (fewer points than the eager
    kernel has CTAs), k = n - 1 on a larger one, int32 and 16-bit: the
    variant's result equals the oracle's."""
    for n in (2, 3, 5, 9):
        Dh = int_instance(n, ("tiny-v", n))
        for k in range(1, n + 1):
            start = rand_medoids(n, k, n * 10 + k)
            out = km.swap(dev(Dh), start, variant=variant, trace=64)
            ref = oracle.swap(Dh, start, variant=variant)
            assert out["medoids"].cpu().tolist() == ref["medoids"].tolist(), (n, k)
            assert out["td_i64"] == int(ref["td"])
    n = 700
    Dh = int_instance(n, "nearly-full")
    start = rand_medoids(n, n - 1, 3)
    out = km.swap(dev(Dh), start, variant=variant)
    ref = oracle.swap(Dh, start, variant=variant)
    assert out["medoids"].cpu().tolist() == ref["medoids"].tolist()
    U = np.zeros((n, 704), np.uint16)
    U[:, :n] = Dh[:, :n]
    start = rand_medoids(n, 9, 4)
    out = km.swap(torch.from_numpy(U.view(np.int16)).cuda(), start, n=n, variant=variant)
    ref = oracle.swap(np.ascontiguousarray(Dh[:, :n]), start, variant=variant)
    assert out["medoids"].cpu().tolist() == ref["medoids"].tolist()
    assert out["td_i64"] == int(ref["td"])


@pytest.mark.parametrize("variant", ["fasterpam", "fastclarans"])
def test_windowed_streaming_path_for_the_eager_variants(variant):
    """A fixed geometry runs FasterPAM / FastCLARANS on the windowed
    streaming kernel (one launch per window, adaptive window length) instead
    of the persistent eager kernel: same decisions, swaps and counts as the
    oracle and as the eager kernel."""
    n, k = 1900, 24
    Dh = int_instance(n, ("windowed", variant))
    start = rand_medoids(n, k, 21)
    kw = {}
    if variant == "fastclarans":
        draws = np.random.default_rng(5).integers(0, n, size=20000).astype(np.int32)
        kw = dict(draws=torch.from_numpy(draws).cuda(), maxneighbor=90)
    a = km.swap(dev(Dh), start, variant=variant, tune=3, trace=100000, **kw)
    b = km.swap(dev(Dh), start, variant=variant, trace=100000, **kw)
    assert a["swap_geometry"] == 3 and b["swap_geometry"] == 0
    for key in ("swaps", "td_i64", "visited", "iterations", "evaluated"):
        assert a[key] == b[key], key
    assert a["medoids"].cpu().tolist() == b["medoids"].cpu().tolist()
    if variant == "fasterpam":
        ref = oracle.swap(Dh, start, variant=variant, trace_cap=100000)
        assert_same_run(a, ref)
    else:
        ref = oracle.clarans(Dh, start, draws, 90, trace_cap=100000)
        assert a["medoids"].cpu().tolist() == ref["medoids"].tolist()
        assert a["iterations"] == ref["evaluated"] and a["visited"] == ref["consumed"]
