#!/usr/bin/env python3
"""Benchmark of the k-medoids hot path on GB300.

One step = one whole run of the method on one synthetic input resident in
HBM: PAM BUILD (k greedy steps) + the per-point cache + FastPAM1 SWAP to
convergence (best swap per pass, cache update after each swap), i.e.
kmedoids_run() through the C ABI.  Default workload: n=50000 points, d=32
float32 Gaussian mixture (200 clusters, centres U[-10,10]^32, sigma
U[0.5,2], Dirichlet(1) weights), Euclidean float32 50000x50000 matrix
(10 GB, larger than L2), k=200; the same figures for the n=20000, k=100
mixture (1.6 GB) ride along in a ``k100`` block.

metric: SWAP dTD point-evals per second -- (n-k)*n (candidate, point) pairs
per FastPAM1 evaluation pass divided by the median pass time (CUDA events
around every evaluation launch of the timed runs) -- plus the full run time
(ms_per_step: BUILD + cache + every SWAP pass and swap) and the pass's
fraction of the measured HBM bandwidth.  Multi-GPU: replicas only (the
method's passes are one sequential chain; each rank runs its own instance).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# the headline metric, worded as the method's benchmark states it
METRIC = "SWAP \u0394TD point-evals/sec + full PAM run time at k=100/200; % HBM roofline vs FP32 path"

WORKLOADS = {
    "gmm_20000": dict(n=20000, d=16, centers=100, k=100, recipe="gmm_20000_points",
                      desc="n=20000 d=16 f32 GMM (100 clusters, centres U[-10,10]^16, "
                           "sigma=1, equal weights), Euclidean f32 20000x20000 matrix, "
                           "k=100, BUILD + FastPAM1 SWAP to convergence"),
    "features_200000": dict(n=200000, d=128, centers=200, k=200, recipe="features_200000",
                            desc="n=200000 d=128 bf16 features of a 200-cluster mixture "
                                 "(centres N(0,4I), sigma=1), Euclidean distances on the fly "
                                 "from a tcgen05 BF16 Gram with FP32 accumulation (no n x n "
                                 "matrix), exact FP32 cache, k=200, BUILD + FastPAM1 SWAP"),
    "batched_512": dict(n=0, d=8, centers=0, k=0, recipe="batched",
                        desc="512 independent PAM instances (n ~ U[200,4000], d=8 float32 "
                             "uniform in [0,1)^8, k ~ U[5,50], Euclidean matrices in one "
                             "11.5 GB arena) in one persistent launch, plus CLARA on "
                             "n=1e6 d=32 float32 (100-cluster mixture), k=100, 10 samples "
                             "of 80+4k=480 points"),
    "clarans_20000": dict(n=20000, d=16, centers=100, k=100, recipe="gmm_20000_points",
                          desc="FastCLARANS (Sec. 3.4) on the gmm_20000 matrix (n=20000 d=16 "
                               "f32 GMM, 100 clusters): k=100, a uniform random start, "
                               "uniform random candidate draws with replacement, stop after "
                               "maxneighbor = 2.5% of n-k = 497 consecutive failed draws"),
    "fasterpam_20000": dict(n=20000, d=16, centers=100, k=100, recipe="gmm_20000_points",
                            desc="the paper's recommended pipeline (Sec. 4.3, Sec. 6) on the "
                                 "gmm_20000 matrix (n=20000 d=16 f32 GMM, 100 clusters): "
                                 "distance-weighted initialisation (Sec. 3.3) from fixed "
                                 "uniform numbers, then eager FasterPAM (Alg. 4) to "
                                 "convergence, k=100"),
    "u16_20000": dict(n=20000, d=2, centers=0, k=100, recipe="manhattan_u16",
                      desc="the compressed integer form: n=20000 2-D integer points uniform in "
                           "[0,1000)^2, exact Manhattan distances (<= 2000) stored as uint16 "
                           "(20000x20000, 0.8 GB), k=100, BUILD + FastPAM1 SWAP to convergence; "
                           "the same matrix as int32 timed beside it"),
    "bichromatic_100000": dict(n=100000, m=20000, d=2, centers=200, k=100,
                               recipe="bichromatic_100000",
                               desc="facility placement (the paper's Outlook): n=100000 "
                                    "consumers around 200 towns (2-D Gaussian mixture), "
                                    "m=20000 candidate locations uniform over the square, "
                                    "Euclidean f32 20000x100000 location-by-consumer matrix "
                                    "(8 GB), k=100 locations, BUILD (plain pass) + FastPAM1 "
                                    "SWAP over the consumers to convergence"),
    "gmm_50000": dict(n=50000, d=32, centers=200, k=200, recipe="gmm_50000_points",
                      desc="n=50000 d=32 f32 GMM (200 clusters, centres U[-10,10]^32, "
                           "sigma U[0.5,2], Dirichlet(1) weights), Euclidean f32 "
                           "50000x50000 matrix (10 GB), k=200, BUILD + FastPAM1 SWAP "
                           "to convergence"),
}


def load_json(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return None


def peaks():
    p = load_json(os.path.join(ROOT, "MEASURED_PEAKS.json"))
    if p and p.get("hbm_gbs"):
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def tensor_peak():
    """Sustained dense bf16 peak (the pass runs inside a seconds-long step)."""
    p = load_json(os.path.join(ROOT, "MEASURED_PEAKS.json"))
    if p and p.get("bf16_tflops_sustained"):
        return float(p["bf16_tflops_sustained"]), "measured sustained"
    return 1700.0, "fallback sustained"


def source_hash(files=("km_stream.cu", "km_device.cuh")):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2008_05171_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def max_over_ranks(ms, world, device):
    """Slowest rank's time: the timed region ends when every rank is done."""
    if world <= 1:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch
        torch.distributed.barrier()


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def make_input(wl_name, device):
    """Synthetic matrix on the device (FP64 direct differences -> FP32; the
    16-bit workload: exact integer Manhattan distances)."""
    from paper_2008_05171_gb300 import workloads as wl
    import torch
    spec = WORKLOADS[wl_name]
    if spec["recipe"] == "manhattan_u16":
        n = spec["n"]
        P = torch.from_numpy(wl.int_coords(n, 2, 1000, seed=("u16", n)).astype(np.int32)).to(device)
        D = torch.empty((n, n), dtype=torch.int16, device=device)
        for r0 in range(0, n, 2048):
            r1 = min(n, r0 + 2048)
            D[r0:r1] = (P[r0:r1, None, :] - P[None, :, :]).abs().sum(-1).to(torch.int16)
        return D, spec
    X = getattr(wl, spec["recipe"])()
    D = wl.euclidean_f32_torch(X, device)
    return D, spec


def evals_of(n, k, res):
    """Element evaluations of BUILD and SWAP in one run: BUILD streams
    build_rows rows of n elements (the incremental BUILD: every row once for
    the distance sums and once for the first gains, then the rows of the
    points whose d_n dropped; the plain pass: n - t candidate rows at step
    t), a SWAP pass n - k candidate rows."""
    rows = int(res.get("build_rows") or 0)
    build = rows * n if rows > 0 else sum((n - t) * n for t in range(k))
    swap = res["iterations"] * (n - k) * n
    return build, swap


def run_features(args, rank, world, local_rank):
    """The on-the-fly distance form: kmedoids_run_features on bf16 features."""
    import torch
    import paper_2008_05171_gb300.kmedoids as km
    from paper_2008_05171_gb300 import workloads as wl
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    spec = WORKLOADS[args.workload]
    n, d, k = spec["n"], spec["d"], spec["k"]
    Xh = wl.features_200000(n=n, d=d, n_centers=spec["centers"])
    X = torch.from_numpy(Xh).to(torch.bfloat16).to(dev)
    torch.cuda.synchronize()

    def step():
        return km.run_features(X, k, profile=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    clocks = Clocks(local_rank)
    clocks.start()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    results = []
    torch.cuda.synchronize()
    for i in range(args.steps):
        ev[i][0].record(stream)
        results.append(step())
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world, dev)
    sw = swap_pass_figures(n, k, None, results)
    # the SWAP is incremental: its first pass sums every point (the full
    # FastPAM1 evaluation of every pair), each later one only the entries of
    # the points the last swap changed; value is the full pass's throughput
    first_ms = float(np.median([r["eval_ms_first"] for r in results]))
    sw["first_pass_ms"] = first_ms
    sw["later_passes_median_ms"] = sw.pop("median_ms")
    sw["kind"] = ("incremental: pass 1 over every point, later passes over the points the "
                  "last swap changed (one entry per point: its old terms out, its new terms in)")
    pass_ms = max_over_ranks(first_ms, world, dev)
    value = world * (n - k) * n / (pass_ms / 1e3)
    r0 = results[-1]
    peak, pk = tensor_peak()
    flops = 2.0 * n * n * d  # Gram of all candidates x all points, one pass
    # BUILD: every candidate against the point rows its passes streamed (all
    # points in step 0, then the points each commit moved: incremental)
    b_rows = int(r0.get("build_rows") or n * k)
    b_flops = 2.0 * n * d * b_rows / max(1, r0["build_launches"])
    b_ms = r0["build_eval_ms"] / max(1, r0["build_launches"])
    s_ms = first_ms

    def roof(ms, name, share, fl):
        ach = fl / (ms / 1e3) / 1e12
        return {"bound": "tensor", "achieved": round(ach, 1), "peak": peak, "unit": "TFLOP/s",
                "frac": round(ach / peak, 4), "peak_source": pk + " bf16 (MEASURED_PEAKS.json)",
                "kernel": name, "algorithmic_flops_per_launch": fl,
                "avg_launch_ms": round(ms, 4), "share_ms": share, "traffic": None}

    # the plain FastPAM1 pass over every point (swap_full) beside it, untimed
    rp = km.run_features(X, k, profile=True, swap_full=True)
    torch.cuda.synchronize()
    plain = {"ms_per_step": rp["build_ms"] + rp["swap_ms"], "swap_pass_median_ms": rp["eval_ms_median"],
             "swap_passes": rp["eval_launches"],
             "same_medoids": rp["medoids"].cpu().tolist() == r0["medoids"].cpu().tolist(),
             "frac_of_sustained_bf16": round(flops / (rp["eval_ms_median"] / 1e3) / 1e12 / peak, 4)}
    # the dense pass of BUILD step 0 (every candidate's distance sum) with
    # each Gram tile pair computed once, against every tile (gram_full)
    def step0(full):
        t, med = [], None
        for _ in range(3):
            r1 = km.build_features(X, 1, labels=False, profile=True, gram_full=full)
            t.append(r1["build_eval_ms"])
            med = r1["medoids"].cpu().tolist()
        return float(np.median(t)), med
    s0_ms, s0_med = step0(False)
    f0_ms, f0_med = step0(True)
    sym = {"step0_ms": s0_ms, "step0_gram_full_ms": f0_ms, "speedup": round(f0_ms / s0_ms, 3),
           "same_medoid": s0_med == f0_med,
           "pairs_per_s": n * n / (s0_ms / 1e3),
           "kind": "each 128x128 Gram tile pair once (tiles b >= t), distances summed along "
                   "rows and columns; gram_full = every tile in both orientations"}
    rb = roof(b_ms, "k_feat_pass<BUILD> (step 0 dense, then incremental updates)",
              r0["build_eval_ms"], b_flops)
    rb["build_rows_streamed"] = b_rows
    rs = roof(s_ms, "k_feat_pass<SWAP> (the first pass: every point)", r0["eval_ms"], flops)
    dom, other = (rb, rs) if r0["build_eval_ms"] >= r0["eval_ms"] else (rs, rb)
    e2e = None
    if not args.no_e2e:
        Xp = torch.empty(X.shape, dtype=X.dtype, pin_memory=True)
        Xp.copy_(X)
        Xd = torch.empty_like(X)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        Xd.copy_(Xp, non_blocking=True)
        r = km.run_features(Xd, k)
        med_h = r["medoids"].cpu()
        lab_h = r["labels"].cpu()
        b.record(stream)
        torch.cuda.synchronize()
        e_ms = a.elapsed_time(b)
        e2e = {"value": world * r["iterations"] * (n - k) * n / (e_ms / 1e3),
               "unit": "point-evals/s", "steps": 1,
               "h2d_bytes_per_step": int(X.numel() * 2),
               "d2h_bytes_per_step": int(4 * k + 4 * n)}
        del med_h, lab_h
    line = {
        "metric": METRIC,
        "value": value, "unit": "point-evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16 Gram / f32 (FP64 TD)",
        "data": "synthetic",
        "config": features_config(args.workload, spec, world),
        "value_definition": "(n-k)*n point-evals of the first FastPAM1 SWAP pass (every point) "
                            "/ its median time over the steps; ms_per_step = the whole BUILD + "
                            "SWAP run (later passes incremental)",
        "swap_pass": sw,
        "plain_swap_run": plain,
        "symmetric_gram": sym,
        "full_run_ms": total_ms / args.steps, "swap_iterations": r0["iterations"],
        "swaps": r0["swaps"], "swap_iter_ms": s_ms, "build_step_ms": b_ms, "td": r0["td"],
        "kernel_ms_per_step": {"build_eval": r0["build_eval_ms"], "swap_eval": r0["eval_ms"],
                               "build_total": r0["build_ms"], "swap_total": r0["swap_ms"]},
        "roofline": dom, "roofline_other": other,
        "gpu_launches": int(sum(r["kernel_launches"] for r in results)),
        "clocks": ck, "e2e": e2e,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # TD error of the result: the GPU's TD (bf16 Gram decisions, exact
        # FP32 cache, FP64 sums) against the FP64 oracle's TD of the same
        # medoids on the exact Euclidean distances of the same features
        import oracle
        td_ref = oracle.td_points(np.asarray(Xh, np.float32), r0["medoids"].cpu().numpy())
        line["td_fp64_oracle"] = td_ref
        line["td_rel_error"] = abs(r0["td"] - td_ref) / td_ref
    if world == 1 and not args.no_matrix_compare:
        line["fp32_matrix_path"] = matrix_path_beside(Xh, k, r0, dev, stream)
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        ns = 8000
        Ds = torch.from_numpy(wl.euclidean_f32(Xh[:ns].astype(np.float64)))
        cb = cpu_baseline(Ds, dict(spec, n=ns), args.cpu_seconds)
        cb["sample"] = "first %d points of the same features as an FP32 matrix; " % ns + cb["sample"]
        line["cpu_baseline"] = cb
    return line


def run_batched(args, rank, world, local_rank):
    """Batched instances + CLARA in one enqueue (kmedoids_run_batched_clara):
    the 512 instances and CLARA's 10 samples share one persistent PAM
    launch, with the sample matrices, the full-data assignment and the
    choice of the best sample around it, all device work; the step is one
    replay of that sequence captured in a CUDA graph.  The kernel geometry
    comes from kmedoids_batched_autotune on this batch."""
    import torch
    import paper_2008_05171_gb300.kmedoids as km
    from paper_2008_05171_gb300 import workloads as wl
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    specs = wl.batched_specs(512)
    if args.instances:
        specs = specs[:args.instances]
    P, offs = wl.batched_points(specs, d=8)
    inst, arena_len, nmed = km.batch_layout(specs)
    inst_dev = torch.from_numpy(inst.view(np.uint8).copy()).to(dev)
    arena = torch.empty(arena_len, dtype=torch.float32, device=dev)
    km.batched_distances(torch.from_numpy(P).to(dev), offs, inst_dev, arena)
    kc, samples = 100, 10
    Xc = torch.from_numpy(wl.clara_points()).to(dev)
    Sc = torch.from_numpy(wl.clara_samples(Xc.shape[0], samples, 80 + 4 * kc)).to(dev)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    # the geometry of the persistent kernel, measured on this batch
    geometry, tune_ms = km.batched_autotune(arena, inst_dev, nmed)
    bc = km.BatchedClara(arena, inst_dev, nmed, Xc, kc, Sc, tune=geometry)
    bc.enqueue()                      # eager once (warms the launch paths)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        bc.enqueue()
    torch.cuda.synchronize()
    # the batch alone and CLARA alone, timed once beside the graph (not part
    # of value): the persistent kernel's roofline and CLARA's share
    a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a_.record(stream)
    km.run_batched(arena, inst_dev, nmed, tune=geometry)
    b_.record(stream)
    torch.cuda.synchronize()
    b_ms = a_.elapsed_time(b_)
    bc_only = km.BatchedClara(None, None, 0, Xc, kc, Sc, tune=geometry)
    bc_only.enqueue()
    torch.cuda.synchronize()
    a_.record(stream)
    bc_only.enqueue()
    b_.record(stream)
    torch.cuda.synchronize()
    clara_ms = a_.elapsed_time(b_)
    del bc_only

    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    barrier(world)
    clocks = Clocks(local_rank)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    torch.cuda.synchronize()
    for i in range(args.steps):
        ev[i][0].record(stream)
        graph.replay()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    r = np.frombuffer(bc.results.cpu().numpy().tobytes(), dtype=km.BATCH_RESULT_DTYPE)
    assert (r["status"] == 0).all()
    cl = bc.clara_outcome()
    ev_b = 0
    bytes_b = 0
    for (n, k), it in zip(specs, r["iterations"]):
        ev_b += sum((n - t) * n for t in range(k)) + int(it) * (n - k) * n
        bytes_b += 4 * (sum((n - t) * n for t in range(k)) + int(it) * (n - k) * n)
    ev_c = Xc.shape[0] * kc * samples
    value = world * args.steps * (ev_b + ev_c) / (total_ms / 1e3)
    # kernels per replay: CLARA's descriptors, distances, order, the
    # persistent PAM kernel, medoid map, assignment(s), selection, labels
    launches = args.steps * 9
    e2e = None
    if not args.no_e2e:
        # the public calls from host data: points, offsets and descriptors
        # in, distances, then the one enqueue of batch + CLARA, results out
        Ph = torch.from_numpy(P).pin_memory()
        Oh = torch.from_numpy(np.asarray(offs, dtype=np.int64)).pin_memory()
        Ih = torch.from_numpy(inst.view(np.uint8).copy()).pin_memory()
        Xh = Xc.cpu().pin_memory()
        Sh = Sc.cpu().pin_memory()
        med_h = torch.empty(nmed, dtype=torch.int32).pin_memory()
        res_h = torch.empty(len(specs) * 24, dtype=torch.uint8).pin_memory()
        cmed_h = torch.empty(kc, dtype=torch.int32).pin_memory()
        lab_h = torch.empty(Xc.shape[0], dtype=torch.int32).pin_memory()
        P_d = torch.empty(P.shape, dtype=torch.float32, device=dev)
        O_d = torch.empty(len(offs), dtype=torch.int64, device=dev)
        I_d = torch.empty_like(inst_dev)
        X_d = torch.empty_like(Xc)
        S_d = torch.empty_like(Sc)
        be = km.BatchedClara(arena, I_d, nmed, X_d, kc, S_d, tune=geometry)

        def e2e_step():
            P_d.copy_(Ph, non_blocking=True)
            O_d.copy_(Oh, non_blocking=True)
            I_d.copy_(Ih, non_blocking=True)
            X_d.copy_(Xh, non_blocking=True)
            S_d.copy_(Sh, non_blocking=True)
            km.batched_distances(P_d, O_d, I_d, arena)
            be.enqueue()
            med_h.copy_(be.medoids[:nmed], non_blocking=True)
            res_h.copy_(be.results, non_blocking=True)
            cmed_h.copy_(be.clara_medoids, non_blocking=True)
            lab_h.copy_(be.labels, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        for _ in range(args.steps):
            e2e_step()
        eb.record(stream)
        torch.cuda.synchronize()
        e_ms = ea.elapsed_time(eb)
        h2d = (Ph.numel() * 4 + Oh.numel() * 8 + Ih.numel() + Xh.numel() * 4 + Sh.numel() * 4)
        d2h = med_h.numel() * 4 + res_h.numel() + cmed_h.numel() * 4 + lab_h.numel() * 4
        e2e = {"value": world * args.steps * (ev_b + ev_c) / (e_ms / 1e3), "unit": "point-evals/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": e_ms / args.steps,
               "includes": "host->device copies of points and features, the batched "
                           "distance matrices, batch + CLARA in one enqueue, results back"}
        del be
    peak, pk = peaks()
    ach = bytes_b / (b_ms / 1e3) / 1e9
    # DRAM traffic per launch: the ratio of DRAM bytes to algorithmic bytes
    # from one ncu capture of a smaller batch (traffic is proportional to the
    # rows streamed), applied to this launch; null once the kernel changed
    traffic = None
    ent = (load_json(os.path.join(ROOT, "profiles", "traffic.json")) or {}).get("batch_pam")
    if ent and ent.get("source_hash") == source_hash(("km_batched.cu", "km_device.cuh")):
        traffic = round(ent["dram_bytes_per_algorithmic_byte"] * bytes_b)
    warps, stages = km.batched_geometry_info(geometry)
    line = {
        "metric": BATCHED_METRIC,
        "value": value, "unit": "point-evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (fixed-point dTD, FP64 TD)",
        "data": "synthetic",
        "config": batched_config(args, specs, arena_len, world),
        "value_definition": "(element evaluations of every instance's BUILD steps and SWAP "
                            "passes + CLARA's point-medoid assignments) / replay time",
        "step": "one CUDA-graph replay of kmedoids_run_batched_clara: 512 instances and "
                "10 CLARA samples in one persistent PAM launch, CLARA's matrices, "
                "assignment, choice and labels around it",
        "autotune": {"geometry": geometry, "warps_per_cta": warps, "ring_stages": stages,
                     "ms_per_geometry": tune_ms},
        "batched_alone_ms": b_ms, "clara_alone_ms": clara_ms,
        "instances_per_s": len(specs) / (total_ms / args.steps / 1e3),
        "batched_swaps": int(r["swaps"].sum()), "batched_passes": int(r["iterations"].sum()),
        "clara_td": cl["td"], "clara_best_sample": cl["best_sample"],
        "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(ach / peak, 4),
                     "kernel": "k_batch_pam<%d,%d> (the batch alone)" % (warps, stages),
                     "algorithmic_bytes_per_launch": bytes_b, "avg_launch_ms": round(b_ms, 3),
                     "peak_source": pk, "traffic": traffic},
        "clocks": ck, "e2e": e2e, "gpu_launches": launches,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = oracle_batched(specs, args.cpu_seconds)
        cb.pop("seconds")
        line["cpu_baseline"] = cb
    return line


def eager_roofline(r, n, kernel, workload=None):
    """The eager kernel (one persistent launch per call): the rows the
    sequential scan evaluates, 4 B per (candidate, point) pair, over the
    launch's CUDA-event time.  Its decisions are sequential (Alg. 4), so it
    is bound by the latency of one window + barrier + swap per accepted
    swap, far below HBM bandwidth; the fraction says so."""
    peak, pk = peaks()
    nbytes = int(r["evaluated"]) * n * 4
    ms = float(r["eval_ms"])
    ach = nbytes / (ms / 1e3) / 1e9
    traffic = None
    ent = (load_json(os.path.join(ROOT, "profiles", "traffic.json")) or {}).get("eager")
    if ent and workload and ent.get("workload") == workload and \
            ent.get("source_hash") == source_hash(("km_eager.cu", "km_device.cuh")):
        traffic = ent.get("dram_bytes_per_launch")
    return {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
            "frac": round(ach / peak, 4), "kernel": kernel,
            "algorithmic_bytes_per_launch": nbytes, "avg_launch_ms": round(ms, 5),
            "peak_source": pk, "traffic": traffic,
            "note": "sequential eager decisions: one window evaluation, grid barrier and "
                    "swap per accepted swap (latency-bound)"}


def fasterpam_inputs(n, k):
    from paper_2008_05171_gb300 import workloads as wl
    return wl.rng_for(("fasterpam", n, k)).random(k)


def replay_evaluated(start, trace, visited, n):
    """Candidates the sequential FasterPAM scan evaluates: non-medoid
    positions up to `visited`, applying each swap where the scan meets its
    candidate."""
    med = list(int(x) for x in start)
    inset = set(med)
    ev, sw = 0, 0
    for p in range(visited):
        r = p % n
        if r in inset:
            continue
        ev += 1
        if sw < len(trace) and trace[sw][2] == r:
            inset.discard(med[trace[sw][1]])
            med[trace[sw][1]] = r
            inset.add(r)
            sw += 1
    return ev


def oracle_fasterpam_run(Dh, n, k):
    """The oracle's distance-weighted start + FasterPAM (one core), timed."""
    import oracle
    u = fasterpam_inputs(n, k)
    t0 = time.perf_counter()
    start = oracle.init_weighted(Dh, k, u)
    r = oracle.swap(Dh, start, variant="fasterpam", trace_cap=100000)
    dt = time.perf_counter() - t0
    ev = replay_evaluated(start, r["trace"], r["visited"], n)
    return {"value": (ev * n + k * n) / dt, "unit": "point-evals/s", "cores": 1,
            "kind": "oracle", "seconds": dt,
            "sample": "the whole workload: distance-weighted start + FasterPAM of the FP64 C "
                      "oracle (one core) on the same matrix and uniform numbers: %d candidates "
                      "evaluated, %d swaps, %.1f s" % (ev, r["swaps"], dt)}


def run_fasterpam(args, rank, world, local_rank):
    """Distance-weighted start + FasterPAM to convergence per step."""
    import torch
    import paper_2008_05171_gb300.kmedoids as km
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    D, spec = make_input(args.workload, dev)
    n, k = spec["n"], spec["k"]
    u = torch.from_numpy(fasterpam_inputs(n, k)).to(dev)
    ws = km.workspace(n, k, km.KM_F32, km.options(profile=True, trace=100000), device=dev)
    torch.cuda.synchronize()

    def step(Dm, trace=0):
        start = km.init_weighted(Dm, k, u, ws=ws)
        return km.swap(Dm, start, ws=ws, variant="fasterpam", profile=True, trace=trace)

    for _ in range(args.warmup):
        step(D)
    torch.cuda.synchronize()
    barrier(world)
    clocks = Clocks(local_rank)
    clocks.start()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    results = []
    for i in range(args.steps):
        ev[i][0].record(stream)
        results.append(step(D))
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world, dev)
    r0 = results[-1]
    evals = sum(int(r["evaluated"]) * n + k * n for r in results)
    value = world * evals / (total_ms / 1e3)
    # latency per accepted swap: device timestamps of consecutive swaps
    # (one untimed traced run)
    rt = step(D, trace=100000)
    ts = np.asarray(rt["trace_time_ns"], dtype=np.int64)
    gaps = np.diff(ts) / 1e3 if len(ts) > 1 else np.zeros(1)
    per_swap = {"median_us": float(np.median(gaps)), "mean_us": float(np.mean(gaps)),
                "p90_us": float(np.percentile(gaps, 90)), "swaps": int(rt["swaps"]),
                "note": "intervals between the device timestamps of consecutive applied "
                        "swaps (windows without a swap in between included)"}
    e2e = None
    if not args.no_e2e:
        Dh = torch.empty(D.shape, dtype=D.dtype, pin_memory=True)
        Dh.copy_(D)
        Dd = torch.empty_like(D)
        med_h = torch.empty(k, dtype=torch.int32, pin_memory=True)
        lab_h = torch.empty(n, dtype=torch.int32, pin_memory=True)
        torch.cuda.synchronize()
        e_ms, e_ev = 0.0, 0
        for _ in range(max(1, min(args.steps, 3))):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            km.upload(Dh, D=Dd)
            r = step(Dd)
            med_h.copy_(r["medoids"], non_blocking=True)
            lab_h.copy_(r["labels"], non_blocking=True)
            b.record(stream)
            torch.cuda.synchronize()
            e_ms += a.elapsed_time(b)
            e_ev += int(r["evaluated"]) * n + k * n
        e2e = {"value": world * e_ev / (e_ms / 1e3), "unit": "point-evals/s",
               "h2d_bytes_per_step": int(D.numel() * 4), "d2h_bytes_per_step": 4 * k + 4 * n}
        del Dh, Dd
    line = {
        "metric": METRIC,
        "value": value, "unit": "point-evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (exact 64-bit fixed-point dTD sums, FP64 TD)", "data": "synthetic",
        "config": {"workload": args.workload + ": " + spec["desc"], "n": n, "k": k,
                   "l2": "matrix larger than L2 (no flush needed)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "full_run_ms": total_ms / args.steps, "swaps": int(r0["swaps"]),
        "per_swap": per_swap,
        "evaluated": int(r0["evaluated"]), "visited": int(r0["visited"]),
        "scans": int(r0["iterations"]), "fasterpam_ms": float(r0["swap_ms"]), "td": r0["td"],
        "roofline": eager_roofline(r0, n, "k_eager<float> (FasterPAM)", args.workload),
        "gpu_launches": int(sum(r["kernel_launches"] for r in results)) + 2 * args.steps,
        "clocks": ck, "e2e": e2e,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = oracle_fasterpam_run(D.cpu().numpy(), n, k)
        cb.pop("seconds")
        line["cpu_baseline"] = cb
    return line


def run_clarans(args, rank, world, local_rank):
    """FastCLARANS from a fixed random start over fixed random draws."""
    import torch
    import paper_2008_05171_gb300.kmedoids as km
    from paper_2008_05171_gb300 import workloads as wl
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    D, spec = make_input(args.workload, dev)
    n, k = spec["n"], spec["k"]
    mn = int(0.025 * (n - k))
    g = wl.rng_for(("clarans", n, k))
    start = np.sort(g.choice(n, size=k, replace=False)).astype(np.int32)
    draws = torch.from_numpy(g.integers(0, n, size=400_000).astype(np.int32)).to(dev)
    ws = km.workspace(n, k, km.KM_F32, km.options(profile=True), device=dev)
    torch.cuda.synchronize()

    def step():
        return km.swap(D, start, ws=ws, variant="fastclarans", draws=draws, maxneighbor=mn,
                       profile=True, tune=args.tune)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    clocks = Clocks(local_rank)
    clocks.start()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    results = []
    for i in range(args.steps):
        ev[i][0].record(stream)
        results.append(step())
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world, dev)
    r0 = results[-1]
    evals = sum(int(r["iterations"]) * n for r in results)  # draws evaluated x points
    value = world * evals / (total_ms / 1e3)
    line = {
        "metric": METRIC,
        "value": value, "unit": "point-evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (exact 64-bit fixed-point dTD sums, FP64 TD)", "data": "synthetic",
        "config": {"workload": args.workload + ": " + spec["desc"], "n": n, "k": k,
                   "maxneighbor": mn, "draws_available": int(draws.numel()),
                   "l2": "matrix larger than L2 (no flush needed)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "draws_consumed": int(r0["visited"]), "draws_evaluated": int(r0["iterations"]),
        "swaps": int(r0["swaps"]),
        "stopped_by_maxneighbor": bool(r0["converged"]), "td": r0["td"],
        "roofline": eager_roofline(r0, n, "k_eager<float> (FastCLARANS)"),
        "gpu_launches": int(sum(r["kernel_launches"] for r in results)),
        "clocks": ck, "e2e": None,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = oracle_clarans_sample(D.cpu().numpy(), n, k, args.cpu_seconds)
        cb.pop("seconds")
        line["cpu_baseline"] = cb
    return line


def run_bichromatic(args, rank, world, local_rank):
    """Bichromatic BUILD + FastPAM1 per step on the m x n location-by-consumer
    matrix; value = (m - k) n point-evals per SWAP pass / median pass."""
    import torch
    import paper_2008_05171_gb300.kmedoids as km
    from paper_2008_05171_gb300 import workloads as wl
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    spec = WORKLOADS[args.workload]
    m, n, k = spec["m"], spec["n"], spec["k"]
    L, C = getattr(wl, spec["recipe"])()
    D = wl.cross_euclidean_f32_torch(L, C, dev)
    stream = torch.cuda.current_stream()
    opts = km.options(profile=True)
    ws = torch.empty(int(km.load().kmedoids_bichromatic_workspace_size(m, n, k, km.KM_F32,
                                                                        ctypes.byref(opts))),
                     dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()

    def step():
        return km.run_bichromatic(D, k, n, ws=ws, profile=True, tune=args.tune)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    clocks = Clocks(local_rank)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    results = []
    for i in range(args.steps):
        ev[i][0].record(stream)
        results.append(step())
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world, dev)
    med_ms = max_over_ranks(float(np.median([r["eval_ms_median"] for r in results])), world, dev)
    mean_ms = sum(r["eval_ms"] for r in results) / max(1, sum(r["eval_launches"] for r in results))
    evals = (m - k) * n
    value = world * evals / (med_ms / 1e3)
    peak, peak_kind = peaks()
    r0 = results[-1]
    ach = evals * 4 / (mean_ms / 1e3) / 1e9
    ent = (load_json(os.path.join(ROOT, "profiles", "traffic.json")) or {}).get(
        "swap_eval@" + args.workload)
    traffic = ent.get("dram_bytes_per_launch") if ent and \
        ent.get("source_hash") == source_hash(("km_stream.cu", "km_device.cuh")) else None
    roofline = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "traffic": traffic,
                "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"
                if peak_kind == "measured" else "fallback 6.8 TB/s",
                "kernel": "k_stream<float,SWAP> over the location rows",
                "algorithmic_bytes_per_launch": evals * 4, "avg_launch_ms": round(mean_ms, 5)}
    e2e = None
    if not args.no_e2e:
        Dh = torch.empty(D.shape, dtype=D.dtype, pin_memory=True)
        Dh.copy_(D)
        Dd = torch.empty_like(D)
        med_h = torch.empty(k, dtype=torch.int32, pin_memory=True)
        lab_h = torch.empty(n, dtype=torch.int32, pin_memory=True)
        torch.cuda.synchronize()
        e_ms, e_evals = 0.0, 0
        for i in range(-1, args.steps):  # one untimed warm-up step
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            km.upload(Dh, n=n, D=Dd)
            r = km.run_bichromatic(Dd, k, n, ws=ws, tune=args.tune)
            med_h.copy_(r["medoids"], non_blocking=True)
            lab_h.copy_(r["labels"], non_blocking=True)
            b.record(stream)
            torch.cuda.synchronize()
            if i >= 0:
                e_ms += a.elapsed_time(b)
                e_evals += r["iterations"] * evals
        e_ms = max_over_ranks(e_ms, world, dev)
        e2e = {"value": world * e_evals / (e_ms / 1e3), "unit": "point-evals/s",
               "steps": args.steps, "ms_per_step": e_ms / args.steps,
               "h2d_bytes_per_step": int(D.numel() * 4), "d2h_bytes_per_step": int(4 * k + 4 * n),
               "note": "SWAP point-evals / (matrix upload from pinned host memory + BUILD + "
                       "SWAP + medoids and labels read back)"}
        del Dh, Dd
    line = {
        "metric": METRIC, "value": value, "unit": "point-evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (exact 64-bit fixed-point dTD sums, FP64 TD)", "data": "synthetic",
        "config": {"workload": args.workload + ": " + spec["desc"], "m": m, "n": n, "k": k,
                   "matrix_bytes": int(D.numel() * 4),
                   "l2": "matrix larger than L2 (129 MB): no flush needed",
                   "parallelism": "single GPU" if world == 1 else "replicas"},
        "value_definition": "(m-k)*n point-evals per FastPAM1 SWAP evaluation pass / median "
                            "pass time; ms_per_step = the whole BUILD + SWAP run",
        "swap_pass": {"median_ms": med_ms, "mean_ms": mean_ms,
                      "passes_per_run": int(r0["iterations"]), "point_evals_per_pass": evals},
        "full_run_ms": total_ms / args.steps, "swap_iterations": r0["iterations"],
        "swaps": r0["swaps"], "td": r0["td"],
        "kernel_ms_per_step": {"build_eval": r0["build_eval_ms"], "swap_eval": r0["eval_ms"],
                               "build_total": r0["build_ms"], "swap_total": r0["swap_ms"]},
        "roofline": roofline,
        "gpu_launches": int(sum(r["kernel_launches"] for r in results)),
        "clocks": ck, "e2e": e2e,
    }
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline_bichromatic(D, spec, args.cpu_seconds)
    return line


def cpu_baseline_bichromatic(D, spec, budget_s, m_sample=1000):
    """The FP64 bichromatic oracle on the host cores: FastPAM1 evaluation
    passes (Eq. (7) over every consumer) of the first m_sample locations,
    from a fixed medoid set among them, as many as fit in about budget_s."""
    import oracle
    n, k = spec["n"], spec["k"]
    Dh = D[:m_sample].cpu().numpy() if hasattr(D, "cpu") else np.asarray(D)[:m_sample]
    med = np.arange(0, m_sample, m_sample // k, dtype=np.int32)[:k]
    t0 = time.perf_counter()
    passes = 0
    while time.perf_counter() - t0 < budget_s or passes == 0:
        oracle.bi_eval_swaps(Dh, med, n=n)
        passes += 1
    dt = time.perf_counter() - t0
    return {"value": passes * (m_sample - k) * n / dt, "unit": "point-evals/s",
            "cores": oracle.num_threads(), "kind": "oracle", "seconds": dt,
            "sample": "%d FastPAM1 evaluation passes of the first %d locations against all "
                      "n=%d consumers (k=%d evenly spaced medoids among them; FP64 C oracle, "
                      "OpenMP over locations), %.1f s" % (passes, m_sample, n, k, dt)}


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2008_05171_gb300.kmedoids as km
    if args.workload.startswith("clarans"):
        return run_clarans(args, rank, world, local_rank)
    if args.workload.startswith("fasterpam"):
        return run_fasterpam(args, rank, world, local_rank)
    if args.workload.startswith("features"):
        return run_features(args, rank, world, local_rank)
    if args.workload.startswith("batched"):
        return run_batched(args, rank, world, local_rank)
    if args.workload.startswith("bichromatic"):
        return run_bichromatic(args, rank, world, local_rank)
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    D, spec = make_input(args.workload, dev)
    n, k = spec["n"], spec["k"]
    esize = D.element_size()
    stream = torch.cuda.current_stream()
    ws = km.workspace(n, k, km._dtype_code(D), km.options(profile=True), device=dev)
    torch.cuda.synchronize()

    # tune=-1: the first (warm-up) call times every kernel geometry that fits
    # on this matrix and the library keeps the fastest for the timed steps
    def step():
        return km.run(D, k, ws=ws, labels=True, profile=True, tune=args.tune,
                      build_full=args.build_full)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    clocks = Clocks(local_rank)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    results = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        ev[i][0].record(stream)
        results.append(step())
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ck = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    sw = swap_pass_figures(n, k, esize, results)
    pass_ms = max_over_ranks(sw["median_ms"], world, dev)
    value = world * (n - k) * n / (pass_ms / 1e3)
    r0 = results[-1]

    # roofline of the kernel with the larger share of the step
    build_launch_ms = sum(r["build_eval_ms"] for r in results) / \
        max(1, sum(r["build_launches"] for r in results))
    # BUILD: rows streamed by the BUILD evaluation launches (incremental
    # update passes, or the plain pass's candidate rows), averaged per launch
    build_bytes = evals_of(n, k, r0)[0] * esize / max(1, r0["build_launches"])
    incremental = int(r0["build_geometry"]) == 0
    peak, peak_kind = peaks()
    kern = {
        "swap_eval": {"launch_ms": sw["mean_ms"], "bytes": (n - k) * n * esize,
                      "share_ms": r0["eval_ms"]},
        "build_eval": {"launch_ms": build_launch_ms, "bytes": build_bytes,
                       "share_ms": r0["build_eval_ms"]},
    }
    dom = max(kern, key=lambda x: kern[x]["share_ms"])
    prof = load_json(os.path.join(ROOT, "profiles", "traffic.json")) or {}

    def traffic_of(name):
        key, files = name, ("km_stream.cu", "km_device.cuh")
        if name == "build_eval" and incremental:
            key, files = "build_update", ("km_build.cu", "km_device.cuh")
        key += "_u16" if esize == 2 else ""
        ent = prof.get(key + "@" + args.workload) or prof.get(key)
        if ent and ent.get("source_hash") == source_hash(files) and \
                ent.get("workload") == args.workload:
            return ent.get("dram_bytes_per_launch")
        return None

    def kernel_name(name):
        t = {4: "float", 2: "uint16"}.get(esize, "?")
        if name == "build_eval" and incremental:
            return "k_build_update<%s> (incremental BUILD)" % t
        return "k_stream<%s,%s>" % (t, "SWAP" if name == "swap_eval" else "BUILD")

    def roof(name):
        kk = kern[name]
        ach = kk["bytes"] / (kk["launch_ms"] / 1e3) / 1e9
        return {"bound": "hbm", "achieved": round(ach, 1), "peak": peak,
                "unit": "GB/s", "frac": round(ach / peak, 4),
                "traffic": traffic_of(name),
                "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"
                if peak_kind == "measured" else "fallback 6.8 TB/s",
                "kernel": kernel_name(name),
                "algorithmic_bytes_per_launch": kk["bytes"],
                "avg_launch_ms": round(kk["launch_ms"], 5)}

    roofline = roof(dom)
    other = roof("swap_eval" if dom == "build_eval" else "build_eval")

    # end to end through the public call: the matrix copied from pinned host
    # memory, the run, medoids and labels read back -- every timed step
    e2e = None
    if not args.no_e2e:
        Dh = torch.empty(D.shape, dtype=D.dtype, pin_memory=True)
        Dh.copy_(D)
        Dd = torch.empty_like(D)
        med_h = torch.empty(k, dtype=torch.int32, pin_memory=True)
        lab_h = torch.empty(n, dtype=torch.int32, pin_memory=True)
        torch.cuda.synchronize()
        e_ms, e_evals = 0.0, 0
        for i in range(-1, args.steps):  # one untimed warm-up step
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            km.upload(Dh, D=Dd)  # SM loads from pinned host memory over the link
            r = km.run(Dd, k, ws=ws, labels=True, tune=args.tune, build_full=args.build_full)
            med_h.copy_(r["medoids"], non_blocking=True)
            lab_h.copy_(r["labels"], non_blocking=True)
            b.record(stream)
            torch.cuda.synchronize()
            if i >= 0:
                e_ms += a.elapsed_time(b)
                e_evals += r["iterations"] * (n - k) * n
        e_ms = max_over_ranks(e_ms, world, dev)
        e2e = {"value": world * e_evals / (e_ms / 1e3), "unit": "point-evals/s",
               "steps": args.steps, "ms_per_step": e_ms / args.steps,
               "h2d_bytes_per_step": int(D.numel() * esize),
               "d2h_bytes_per_step": int(4 * k + 4 * n),
               "note": "SWAP point-evals of the run / (matrix H2D by kmedoids_upload_matrix "
                       "from pinned host memory + BUILD + SWAP + medoids and labels D2H)"}
        del Dh, Dd

    line = {
        "metric": METRIC, "value": value, "unit": "point-evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (exact 64-bit fixed-point dTD sums, FP64 TD)" if esize == 4 else
                 "u16 distances (int32 compares, int64 sums)",
        "data": "synthetic",
        "config": matrix_config(args.workload, spec, world),
        "value_definition": "(n-k)*n point-evals per FastPAM1 SWAP evaluation pass / median "
                            "pass time (CUDA events around every evaluation launch of the "
                            "timed runs); ms_per_step = the whole BUILD + SWAP run",
        "swap_pass": sw,
        "geometry": {"swap": int(r0["swap_geometry"]), "build": int(r0["build_geometry"]),
                     "picked_by": {-1: "measured on the first call (tune=-1)",
                                   0: "preference order (tune=0)"}.get(
                                       args.tune, "fixed (tune=%d)" % args.tune)},
        "full_run_ms": total_ms / args.steps,
        "swap_iterations": r0["iterations"], "swaps": r0["swaps"],
        "td": r0["td"],
        "kernel_ms_per_step": {"build_eval": r0["build_eval_ms"],
                               "swap_eval": r0["eval_ms"],
                               "build_total": r0["build_ms"],
                               "swap_total": r0["swap_ms"]},
        "build": {"mode": "incremental" if incremental else "plain pass",
                  "rows_streamed": int(r0["build_rows"]),
                  "plain_pass_rows": sum(n - t for t in range(k))},
        "roofline": roofline, "roofline_other": other,
        "gpu_launches": int(sum(r["kernel_launches"] for r in results)),
        "clocks": ck, "e2e": e2e, "wall_s": wall,
    }
    # the same run without per-pass events (as a caller makes it): the
    # FastPAM1 loop runs as one graph and the call reads its results once
    for _ in range(2):
        km.run(D, k, ws=ws, labels=True, tune=args.tune, build_full=args.build_full)
    torch.cuda.synchronize()
    g_ms = []
    for _ in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rg = km.run(D, k, ws=ws, labels=True, tune=args.tune, build_full=args.build_full)
        b.record(stream)
        torch.cuda.synchronize()
        g_ms.append(a.elapsed_time(b))
    line["run_without_pass_events"] = {
        "ms_per_step": max_over_ranks(sum(g_ms), world, dev) / args.steps,
        "swap_loop": "one graph (conditional WHILE node)",
        "same_medoids": rg["medoids"].cpu().tolist() == r0["medoids"].cpu().tolist(),
        "kernel_launches": int(rg["kernel_launches"])}
    if incremental and not args.no_e2e:
        # the plain BUILD (every step streams all candidate rows) on the same
        # matrix, timed the same way (not part of value)
        for _ in range(2):
            km.run(D, k, ws=ws, profile=True, tune=args.tune, build_full=True)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rf = km.run(D, k, ws=ws, profile=True, tune=args.tune, build_full=True)
        b.record(stream)
        torch.cuda.synchronize()
        line["build"]["plain_pass_run"] = {
            "ms_per_step": a.elapsed_time(b), "build_ms": rf["build_ms"],
            "same_medoids": rf["medoids"].cpu().tolist() == r0["medoids"].cpu().tolist(),
            "td": rf["td"]}
    if esize == 2:
        # the same matrix as int32, timed the same way (not part of value)
        Di = D.to(torch.int32)
        wsi = km.workspace(n, k, km.KM_I32, km.options(profile=True), device=dev)
        for _ in range(2):
            km.run(Di, k, ws=wsi, profile=True, tune=args.tune, build_full=args.build_full)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ri = km.run(Di, k, ws=wsi, profile=True, tune=args.tune, build_full=args.build_full)
        b.record(stream)
        torch.cuda.synchronize()
        line["int32_same_matrix"] = {
            "ms_per_step": a.elapsed_time(b),
            "swap_iter_ms": ri["eval_ms"] / max(1, ri["eval_launches"]),
            "build_step_ms": ri["build_eval_ms"] / max(1, ri["build_launches"]),
            "same_medoids": ri["medoids"].cpu().tolist() == r0["medoids"].cpu().tolist()}
        del Di, wsi
    cb_D = D.to(torch.int32) if esize == 2 else D
    if args.workload == "gmm_50000" and not args.no_k100:
        del ws
        line["k100"] = k100_block(args, km, dev, stream, peak)
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(cb_D, spec, args.cpu_seconds)
    return line


def matrix_path_beside(Xh, k, rf, dev, stream):
    """The plain FP32 matrix path on the same points: the n x n matrix of
    FP64 direct-difference distances rounded once to FP32 (torch cdist
    without the Gram shortcut, in row blocks; 160 GB at n = 200000), then
    kmedoids_run (BUILD + FastPAM1) on it.  Reports whether the feature
    form ended at the same medoids and the TD of both medoid sets on the
    same matrix."""
    import torch
    import paper_2008_05171_gb300.kmedoids as km
    n = Xh.shape[0]
    ld = (n + 3) // 4 * 4
    t0 = time.perf_counter()
    X64 = torch.from_numpy(np.asarray(Xh, np.float64)).to(dev)
    D = torch.zeros((n, ld), dtype=torch.float32, device=dev)
    B = 2048
    for i0 in range(0, n, B):
        i1 = min(n, i0 + B)
        D[i0:i1, :n] = torch.cdist(X64[i0:i1], X64, p=2.0,
                                   compute_mode="donot_use_mm_for_euclid_dist").float()
    # bitwise symmetric with a zero diagonal, as the matrix form assumes
    T = 8192
    for i0 in range(0, n, T):
        i1 = min(n, i0 + T)
        for j0 in range(i0, n, T):
            j1 = min(n, j0 + T)
            blk = D[i0:i1, j0:j1]
            if j0 == i0:
                up = torch.triu(blk, 1)
                blk.copy_(up + up.T)
            else:
                D[j0:j1, i0:i1] = blk.T
    del X64
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    ws = km.workspace(n, k, km.KM_F32, km.options(profile=True), device=dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    rm = km.run(D, k, n=n, ws=ws, labels=True, profile=True, tune=0)
    b.record(stream)
    torch.cuda.synchronize()
    mf = rf["medoids"].cpu().numpy()
    mm = rm["medoids"].cpu().numpy()
    # TD of the feature form's medoids on the same FP32 matrix
    mf_t = torch.from_numpy(mf.astype(np.int64)).to(dev)
    td_f = 0.0
    for i0 in range(0, n, 8192):
        td_f += float(D[i0:i0 + 8192, :n].index_select(1, mf_t).min(dim=1).values
                      .double().sum().item())
    out = {"matrix_bytes": int(n) * ld * 4, "matrix_build_s": round(gen_s, 2),
           "run_ms": a.elapsed_time(b), "swap_pass_ms": rm["eval_ms_median"],
           "build_ms": rm["build_ms"], "swap_iterations": rm["iterations"],
           "swaps": rm["swaps"], "td_matrix_path": rm["td"],
           "td_feature_medoids_on_matrix": td_f,
           "same_medoids": sorted(mf.tolist()) == sorted(mm.tolist()),
           "same_slot_order": mf.tolist() == mm.tolist(),
           "td_rel_diff": abs(td_f - rm["td"]) / rm["td"],
           "medoids_differing": int(len(set(mf.tolist()) ^ set(mm.tolist())) // 2)}
    del D, ws
    torch.cuda.empty_cache()
    return out


def features_config(wl_name, spec, world):
    """The workload description of the on-the-fly form (both arms)."""
    return {"workload": wl_name + ": " + spec["desc"], "n": spec["n"], "d": spec["d"],
            "k": spec["k"], "l2": "features (51 MB) L2-resident by design; no matrix",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def matrix_config(wl_name, spec, world):
    """The workload description of a matrix workload; both arms print the
    same dict."""
    n = spec["n"]
    esize = 2 if spec["recipe"] == "manhattan_u16" else 4
    return {"workload": wl_name + ": " + spec["desc"], "n": n, "k": spec["k"],
            "matrix_bytes": n * n * esize,
            "l2": "matrix larger than L2 (129 MB): no flush needed",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def swap_pass_figures(n, k, esize, results):
    """FastPAM1 evaluation passes of the timed runs: median (over runs of
    each run's median pass) and mean pass time, and (matrix form: esize
    bytes per element) the HBM roofline of the median pass."""
    med = float(np.median([r["eval_ms_median"] for r in results]))
    mean = sum(r["eval_ms"] for r in results) / max(1, sum(r["eval_launches"] for r in results))
    out = {"median_ms": med, "mean_ms": mean,
           "passes_per_run": int(results[-1]["iterations"]),
           "point_evals_per_pass": (n - k) * n}
    if esize:
        peak, _ = peaks()
        gbs = (n - k) * n * esize / (med / 1e3) / 1e9
        out.update(median_pass_gbs=round(gbs, 1), median_pass_frac_of_hbm=round(gbs / peak, 4))
    return out


def k100_block(args, km, dev, stream, peak):
    """The k = 100 case of the metric: BUILD + FastPAM1 on the n = 20000
    mixture (1.6 GB matrix), warm-up and timed runs as for the headline."""
    import torch
    spec = WORKLOADS["gmm_20000"]
    D, _ = make_input("gmm_20000", dev)
    n, k = spec["n"], spec["k"]
    ws = km.workspace(n, k, km.KM_F32, km.options(profile=True), device=dev)
    for _ in range(args.warmup):
        km.run(D, k, ws=ws, profile=True, tune=args.tune, build_full=args.build_full)
    torch.cuda.synchronize()
    res, ms = [], []
    for _ in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        res.append(km.run(D, k, ws=ws, profile=True, tune=args.tune,
                          build_full=args.build_full))
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    sw = swap_pass_figures(n, k, 4, res)
    out = {"workload": "gmm_20000: " + spec["desc"], "n": n, "k": k,
           "swap_point_evals_per_s": (n - k) * n / (sw["median_ms"] / 1e3),
           "swap_pass": sw, "full_run_ms": float(np.mean(ms)),
           "build_ms": res[-1]["build_ms"], "swap_iterations": res[-1]["iterations"],
           "td": res[-1]["td"], "swap_geometry": int(res[-1]["swap_geometry"])}
    del D, ws
    torch.cuda.empty_cache()
    return out


def oracle_medoids(n, k):
    """The medoid set the oracle's timed passes start from: k distinct points
    drawn uniformly (fixed seed).  A pass's cost does not depend on which
    medoids are current beyond the share of points near them."""
    from paper_2008_05171_gb300 import workloads as wl
    g = wl.rng_for(("bench-oracle-medoids", n, k))
    return np.sort(g.choice(n, size=k, replace=False)).astype(np.int32)


def cpu_baseline(D, spec, budget_s, pam=True):
    """The FP64 oracle on the host cores on a bounded sample of the same
    workload: FastPAM1 evaluation passes (Eq. (7), every non-medoid candidate
    against all n points) over the same matrix, as many as fit in about
    budget_s seconds (at least one); the value is the metric's point-evals
    per second of those passes."""
    import oracle
    n, k = spec["n"], spec["k"]
    Dh = D.cpu().numpy() if hasattr(D, "cpu") else D
    threads = oracle.num_threads()
    med = oracle_medoids(n, k)
    t0 = time.perf_counter()
    passes = 0
    while time.perf_counter() - t0 < budget_s or passes == 0:
        oracle.eval_swaps(Dh, med, method="fastpam1")
        passes += 1
    dt = time.perf_counter() - t0
    out = {"value": passes * (n - k) * n / dt, "unit": "point-evals/s", "cores": threads,
           "kind": "oracle", "seconds": dt,
           "sample": "%d FastPAM1 evaluation passes ((n-k)*n point-evals each) of the same "
                     "n=%d k=%d matrix from a fixed uniform random medoid set (FP64 C "
                     "oracle, OpenMP over candidates), %.1f s" % (passes, n, k, dt)}
    if pam:
        out["pam_vs_fastpam1"] = pam_vs_fastpam1(Dh, med, threads)
    return out


def pam_vs_fastpam1(Dh, med, threads, n_sub=4000):
    """One SWAP evaluation pass of original PAM (Eq. (5): every (medoid,
    candidate) pair summed over all points) and of FastPAM1 (Eq. (7)) with
    the oracle on the first n_sub points and the first medoids among them:
    the same-host speedup the paper quotes for the O(k) improvement.  Also
    FastPAM1 on one thread."""
    import oracle
    Ds = np.ascontiguousarray(Dh[:n_sub, :n_sub])
    k = len(med)
    sub = [int(m) for m in med if m < n_sub][:k]
    sub += [i for i in range(n_sub) if i not in set(sub)][:k - len(sub)]
    sub = np.array(sub, np.int32)
    out = {"n": n_sub, "k": k, "threads": threads}
    for name, method in (("pam_pass_s", "pam"), ("fastpam1_pass_s", "fastpam1")):
        t0 = time.perf_counter()
        oracle.eval_swaps(Ds, sub, method=method)
        out[name] = time.perf_counter() - t0
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.eval_swaps(Ds, sub, method="fastpam1")
        out["fastpam1_pass_1thread_s"] = time.perf_counter() - t0
    finally:
        oracle.set_threads(threads)
    out["speedup_pam_over_fastpam1"] = out["pam_pass_s"] / out["fastpam1_pass_s"]
    return out


BATCHED_METRIC = METRIC


def batched_config(args, specs, arena_len, world):
    if arena_len is None:
        arena_len = sum(n * ((n + 3) // 4 * 4) for n, _ in specs)
    return {"workload": args.workload + ": " + WORKLOADS[args.workload]["desc"],
            "instances": len(specs), "arena_bytes": int(arena_len * 4),
            "l2": "arena %.1f GB > L2 (129 MB): no flush needed" % (arena_len * 4 / 1e9),
            "parallelism": "replicas" if world > 1 else "single GPU"}


def oracle_batched(specs, budget_s):
    """The FP64 oracle's BUILD + FastPAM1 on the batch's instances in order
    until about budget_s seconds of solver time (matrix construction not
    timed, as on the GPU side where the arena is built before the step)."""
    import oracle
    from paper_2008_05171_gb300 import workloads as wl
    head = specs[:64]
    P, offs = wl.batched_points(head, d=8)
    ev, el, done = 0, 0.0, 0
    for (n, k), o in zip(head, offs):
        D = oracle.euclid_f32(P[o:o + n])
        t0 = time.perf_counter()
        r = oracle.run(D, k, variant="fastpam1")
        el += time.perf_counter() - t0
        ev += sum((n - t) * n for t in range(k)) + r["iterations"] * (n - k) * n
        done += 1
        if el >= budget_s:
            break
    return {"value": ev / el, "unit": "point-evals/s", "cores": oracle.num_threads(),
            "kind": "oracle", "seconds": el,
            "sample": "BUILD + FastPAM1 on the first %d of the %d instances (FP64 C oracle, "
                      "OpenMP over candidates), %.1f s of solver time" % (done, len(specs), el)}


def oracle_clarans_sample(Dh, n, k, budget_s):
    """The oracle's FastCLARANS from the workload's start over a prefix of
    its draws, the prefix doubled until one run takes about budget_s / 3
    (the oracle evaluates draws one after another on one core)."""
    import oracle
    from paper_2008_05171_gb300 import workloads as wl
    mn = int(0.025 * (n - k))
    g = wl.rng_for(("clarans", n, k))
    start = np.sort(g.choice(n, size=k, replace=False)).astype(np.int32)
    draws = g.integers(0, n, size=400_000).astype(np.int32)
    length = 64
    while True:
        t0 = time.perf_counter()
        r = oracle.clarans(Dh, start, draws[:length], mn)
        dt = time.perf_counter() - t0
        if dt >= budget_s / 3 or r["stopped"] or length >= len(draws):
            break
        length *= 2
    return {"value": r["evaluated"] * n / dt, "unit": "point-evals/s", "cores": 1,
            "kind": "oracle", "seconds": dt,
            "sample": "FastCLARANS of the FP64 C oracle (one core) from the same start over "
                      "the first %d of the same draws: %d evaluated, %d swaps, %.1f s"
                      % (length, r["evaluated"], r["swaps"], dt)}


def run_reference(args, rank, world):
    """The oracle as the reference arm: timed on the host cores on a bounded
    sample of the workload per step (rank 0 only)."""
    if rank != 0:
        return None
    import torch
    spec = WORKLOADS[args.workload]
    from paper_2008_05171_gb300 import workloads as wl
    if args.workload.startswith("bichromatic"):
        m, n, k = spec["m"], spec["n"], spec["k"]
        L, C = getattr(wl, spec["recipe"])()
        Ds = wl.cross_euclidean_f32(L[:1000], C)  # the sample's location rows
        vals, secs, cb = [], [], None
        for _ in range(args.warmup + args.steps):
            cb = cpu_baseline_bichromatic(Ds, spec, min(8.0, args.cpu_seconds))
            vals.append(cb["value"])
            secs.append(cb.pop("seconds"))
        v = float(np.mean(vals[args.warmup:]))
        cb["value"] = v
        ld = (n + 3) // 4 * 4
        return {"impl": "reference", "metric": METRIC, "value": v, "unit": "point-evals/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * float(np.mean(secs[args.warmup:])),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload + ": " + spec["desc"], "m": m, "n": n,
                           "k": k, "matrix_bytes": int(m * ld * 4),
                           "l2": "matrix larger than L2 (129 MB): no flush needed",
                           "parallelism": "single GPU" if world == 1 else "replicas"},
                "cpu_baseline": cb,
                "e2e": {"value": v, "unit": "point-evals/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
    if args.workload.startswith("batched"):
        # the oracle on the first instances of the batch (bounded sample)
        vals, secs, cb = [], [], None
        for _ in range(args.warmup + args.steps):
            cb = oracle_batched(wl.batched_specs(512), min(8.0, args.cpu_seconds))
            vals.append(cb["value"])
            secs.append(cb["seconds"])
        v = float(np.mean(vals[args.warmup:]))
        cb = dict(cb, value=v)
        cb.pop("seconds")
        return {"impl": "reference", "metric": BATCHED_METRIC, "value": v, "unit": "point-evals/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * float(np.mean(secs[args.warmup:])),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": batched_config(args, wl.batched_specs(512), None, world),
                "cpu_baseline": cb,
                "e2e": {"value": v, "unit": "point-evals/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
    if spec["recipe"] == "manhattan_u16":
        # the same integer matrix (the oracle reads it as int32)
        D, _ = make_input(args.workload, torch.device("cuda", 0)) if torch.cuda.is_available() \
            else (None, None)
        if D is None:
            P = wl.int_coords(spec["n"], 2, 1000, seed=("u16", spec["n"]))
            D = torch.from_numpy(wl.manhattan_int32(P)[:, :spec["n"]].copy())
        D = D.to(torch.int32)
        X = None
    else:
        X = getattr(wl, spec["recipe"])()
    if args.workload.startswith("fasterpam"):
        dev = torch.device("cuda", 0) if torch.cuda.is_available() else torch.device("cpu")
        Dh = (wl.euclidean_f32_torch(X, dev) if dev.type == "cuda"
              else torch.from_numpy(wl.euclidean_f32(X))).cpu().numpy()
        vals, secs, cb = [], [], None
        for _ in range(args.warmup + args.steps):
            cb = oracle_fasterpam_run(Dh, spec["n"], spec["k"])
            vals.append(cb["value"])
            secs.append(cb.pop("seconds"))
        v = float(np.mean(vals[args.warmup:]))
        cb["value"] = v
        return {"impl": "reference", "metric": METRIC, "value": v, "unit": "point-evals/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * float(np.mean(secs[args.warmup:])),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload + ": " + spec["desc"], "n": spec["n"],
                           "k": spec["k"]},
                "cpu_baseline": cb,
                "e2e": {"value": v, "unit": "point-evals/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
    if args.workload.startswith("clarans"):
        dev = torch.device("cuda", 0) if torch.cuda.is_available() else torch.device("cpu")
        Dh = (wl.euclidean_f32_torch(X, dev) if dev.type == "cuda"
              else torch.from_numpy(wl.euclidean_f32(X))).cpu().numpy()
        vals, secs, cb = [], [], None
        for _ in range(args.warmup + args.steps):
            cb = oracle_clarans_sample(Dh, spec["n"], spec["k"], min(8.0, args.cpu_seconds))
            vals.append(cb["value"])
            secs.append(cb.pop("seconds"))
        v = float(np.mean(vals[args.warmup:]))
        cb["value"] = v
        return {"impl": "reference", "metric": METRIC, "value": v, "unit": "point-evals/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * float(np.mean(secs[args.warmup:])),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload + ": " + spec["desc"], "n": spec["n"],
                           "k": spec["k"]},
                "cpu_baseline": cb,
                "e2e": {"value": v, "unit": "point-evals/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
    feat = args.workload.startswith("features")
    spec_s = spec
    if feat:
        # no n x n matrix exists in this form: time the oracle on a subsample
        spec_s = dict(spec, n=8000)
        X = X[:8000].astype(np.float64)
    dev = torch.device("cuda", 0) if torch.cuda.is_available() else torch.device("cpu")
    if X is None:
        pass  # the integer matrix built above
    elif dev.type == "cuda":
        D = wl.euclidean_f32_torch(X, dev)
    else:
        D = torch.from_numpy(wl.euclidean_f32(X))
    Dh = D.cpu().numpy()
    del D
    # each step: as many FastPAM1 evaluation passes as fit in the budget
    budget = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_baseline(Dh, spec_s, budget / 4, pam=False)
    vals, secs, evals = [], [], 0
    for i in range(args.steps):
        cb = cpu_baseline(Dh, spec_s, budget, pam=(i == args.steps - 1))
        secs.append(cb.pop("seconds"))
        vals.append(cb["value"])
    v = float(np.mean(vals))
    cb["value"] = v
    if feat:
        cb["sample"] = "first 8000 points of the same features as an FP32 matrix; " + \
            cb["sample"]
        config = features_config(args.workload, spec, world)
    else:
        config = matrix_config(args.workload, spec, world)
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "point-evals/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(secs)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config,
            "value_definition": "(n-k)*n point-evals per FastPAM1 evaluation pass of the FP64 "
                                "C oracle / pass time, on the host cores",
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "point-evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="gmm_50000", choices=sorted(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-k100", action="store_true",
                    help="gmm_50000: skip the k=100 (gmm_20000) block")
    ap.add_argument("--no-matrix-compare", action="store_true",
                    help="features_*: skip the FP32 matrix path run beside the feature form")
    ap.add_argument("--build-full", action="store_true",
                    help="matrix workloads: time the plain BUILD pass (every candidate "
                         "row each step) instead of the incremental BUILD")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    # smaller cases of the same recipes, for profiler captures only
    ap.add_argument("--n", type=int, default=None, help="features_*: number of points")
    ap.add_argument("--k", type=int, default=None, help="features_*: number of medoids")
    ap.add_argument("--instances", type=int, default=None,
                    help="batched_*: first INSTANCES instances of the batch")
    ap.add_argument("--tune", type=int, default=-1,
                    help="matrix workloads: kernel geometry (-1 measured on the first "
                         "call, 0 the library's preference order, 1..16 fixed)")
    args = ap.parse_args()
    spec = WORKLOADS[args.workload]
    if args.workload.startswith("features") and (args.n or args.k):
        n, k = args.n or spec["n"], args.k or spec["k"]
        WORKLOADS[args.workload] = dict(spec, n=n, k=k, desc=spec["desc"] +
                                        " [reduced to n=%d k=%d for profiling]" % (n, k))
    if args.workload.startswith("batched") and args.instances:
        WORKLOADS[args.workload] = dict(spec, desc=spec["desc"] +
                                        " [first %d instances, for profiling]" % args.instances)
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "ours":
            torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        line = run_ours(args, rank, world, local_rank)
    if rank == 0 and line is not None:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
