"""The bounds-checking build (-DKM_BOUNDS_CHECK, libkmedoids_bounds.so): its
index check records an index out of range as KM_E_BOUNDS with the index,
the bound and the place of the check (self-test kind 3, which accesses no
memory with the index), and on valid inputs it changes nothing: the matrix,
eager, FastPAM2, on-the-fly and initialisation paths give the oracle's
results with every check compiled in.  Runs in a child process that loads
the bounds-checking library (KMEDOIDS_BOUNDS_CHECK=1)."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2008_05171_gb300.kmedoids as km  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
sys.path.insert(0, ROOT)
import numpy as np
import torch
import oracle
import paper_2008_05171_gb300.kmedoids as km
from paper_2008_05171_gb300 import workloads as wl
lib = km.load()
assert km.LIB_PATH.endswith("libkmedoids_bounds.so")
assert lib.kmedoids_bounds_checked() == 1
st, msg = km.wait_selftest(3, 0)
assert st == 8 and "index 5 out of range [0, 3) at km_selftest.cu:" in msg, (st, msg)
Dh = wl.manhattan_int32(wl.int_coords(1800, 2, 1000, seed="bounds"))
D = torch.from_numpy(Dh).cuda()
for v in ("fastpam1", "fasterpam", "fastpam2"):
    out = km.run(D, 13, variant=v, trace=1000)
    ref = oracle.run(Dh, 13, variant=v)
    assert out["medoids"].cpu().tolist() == ref["medoids"].tolist(), v
    assert out["td_i64"] == int(ref["td"]), v
    assert out["status_name"] == "KM_OK", (v, out["status_name"])
X = wl.gmm_points(1500, 8, 12, seed="bounds-f")
Dfh = wl.euclidean_f32(X)
outf = km.run(torch.from_numpy(Dfh).cuda(), 12, build_full=True)
reff = oracle.run(Dfh, 12, variant="fastpam1")
assert outf["medoids"].cpu().tolist() == reff["medoids"].tolist()
Xf = wl.features_200000(n=3000, d=32, n_centers=12)
a = km.run_features(torch.from_numpy(Xf).to(torch.bfloat16).cuda(), 8)
assert a["status_name"] == "KM_OK" and len(set(a["medoids"].cpu().tolist())) == 8
u = np.random.default_rng(3).random(13)
med = km.init_weighted(D, 13, u)
assert med.cpu().tolist() == oracle.init_weighted(Dh, 13, u).tolist()
print("ok")
'''


def test_regular_build_compiles_the_checks_out():
    if os.environ.get("KMEDOIDS_BOUNDS_CHECK") == "1":
        pytest.skip("this process runs the bounds-checking build")
    assert km.load().kmedoids_bounds_checked() == 0
    st, msg = km.wait_selftest(3, 0)
    assert st == 0, (st, msg)


def test_bounds_checking_build_records_and_changes_nothing():
    from paper_2008_05171_gb300 import build as b
    b.build(bounds_check=True)
    env = dict(os.environ, KMEDOIDS_BOUNDS_CHECK="1")
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout[-2000:] + r.stderr[-4000:]
