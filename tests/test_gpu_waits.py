"""Bounded device waits: a wait that cannot be satisfied gives up after the
caller's limit with KM_E_TIMEOUT, and the context stays usable.

kmedoids_wait_selftest runs the library's own wait routines (the mbarrier
phase wait of the pipelined kernels, the consumer barrier, the eager
kernel's grid barrier) on a condition nothing ever fulfils; no copy, MMA or
tensor memory is in flight when they give up.  A normal run on the same
stream must then succeed and equal the oracle, and the production kernels
must honour a caller-given limit that their waits stay within."""
import time

import numpy as np
import pytest

import oracle
from paper_2008_05171_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2008_05171_gb300.kmedoids as km  # noqa: E402


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_unsatisfiable_wait_times_out_and_context_survives(kind):
    limit = 2_000_000  # 2 ms
    t0 = time.perf_counter()
    st, msg = km.wait_selftest(kind, limit)
    dt = time.perf_counter() - t0
    assert st == 5, (st, msg)                      # KM_E_TIMEOUT
    assert "gave up" in msg and str(limit) in msg
    assert dt >= limit * 1e-9                       # it waited its limit ...
    assert dt < 5.0                                 # ... and not the 4 s default
    # the same stream still runs the method: bit-exact integer run
    Dh = wl.manhattan_int32(wl.int_coords(500, 2, 1000, seed=("waits", kind)))
    out = km.run(torch.from_numpy(Dh).cuda(), 7)
    ref = oracle.run(Dh, 7, variant="fastpam1")
    assert out["medoids"].cpu().tolist() == ref["medoids"].tolist()
    assert out["td_i64"] == int(ref["td"])


def test_caller_wait_limit_reaches_every_kernel():
    """A limit of half a second (far above any wait of these small runs) is
    accepted by the matrix, eager and on-the-fly forms, which then run as
    usual."""
    Dh = wl.manhattan_int32(wl.int_coords(1200, 2, 1000, seed="waits-limit"))
    D = torch.from_numpy(Dh).cuda()
    for variant in ("fastpam1", "fasterpam"):
        out = km.run(D, 9, variant=variant, wait_limit_ns=500_000_000)
        ref = oracle.run(Dh, 9, variant=variant)
        assert out["medoids"].cpu().tolist() == ref["medoids"].tolist(), variant
    X = wl.features_200000(n=2000, d=32, n_centers=10)
    Xt = torch.from_numpy(X).to(torch.bfloat16).cuda()
    a = km.run_features(Xt, 5, wait_limit_ns=500_000_000)
    b = km.run_features(Xt, 5)
    assert a["medoids"].cpu().tolist() == b["medoids"].cpu().tolist()
    assert a["td"] == b["td"]
