"""The multi-process paths of bench.py on CPU with the gloo backend, world
size 2: the slowest-rank timing reduction, and the reference arm launched
the way the multi-GPU bench is (torchrun, one process per rank), where rank
0 alone runs the oracle and prints one JSON line and the other rank exits 0
without output."""
import json
import os
import socket
import subprocess
import sys
import tempfile

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        bench.barrier(world)
        got = bench.max_over_ranks(10.0 * (rank + 1) + 0.25, world, "cpu")
        with open(os.path.join(out_dir, "r%d" % rank), "w") as f:
            f.write(repr(got))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    import torch.multiprocessing as mp
    port = _free_port()
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_worker, args=(2, port, d), nprocs=2, join=True, start_method="spawn")
        vals = [float(open(os.path.join(d, "r%d" % r)).read()) for r in range(2)]
    assert vals == [20.25, 20.25]


def test_reference_arm_under_torchrun_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--workload", "batched_512", "--gpus", "2", "--steps", "1",
           "--warmup", "3", "--cpu-seconds", "0.2"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [json.loads(x) for x in p.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
