"""kmedoids_upload_matrix: the matrix from host memory into a device buffer
with another row pitch, pad columns cleared -- byte-exact against the host
data on every access width (16-, 4- and 2-byte loads from page-locked
memory, the copy engines for pageable memory), and a run on the uploaded
matrix equals the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2008_05171_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2008_05171_gb300.kmedoids as km  # noqa: E402


def _host(n, host_ld, dtype, pinned, seed):
    rng = np.random.default_rng(seed)
    if dtype == torch.float32:
        a = rng.random((n, host_ld), np.float32) * 100
    elif dtype == torch.int32:
        a = rng.integers(-2**31, 2**31 - 1, (n, host_ld), dtype=np.int64).astype(np.int32)
    else:
        a = rng.integers(0, 2**16, (n, host_ld), dtype=np.int64).astype(np.uint16).view(np.int16)
    H = torch.from_numpy(a)
    if pinned:
        H = H.pin_memory()
    return H[:, :n] if host_ld > n else H


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("n,host_ld,ld,dtype", [
    (4096, 4096, 4096, torch.float32),   # flat 16-byte copy
    (3001, 3001, 3004, torch.float32),   # rows, 4-byte loads
    (2000, 2004, 2008, torch.int32),     # rows, 16-byte loads, wider host rows
    (1001, 1001, 1008, torch.int16),     # 16-bit rows, 2-byte loads
    (1000, 1000, 1000, torch.int16),     # 16-bit flat
    (7, 9, 16, torch.int16),             # tiny, fewer rows than CTAs
])
def test_upload_is_byte_exact_and_clears_padding(n, host_ld, ld, dtype, pinned):
    H = _host(n, host_ld, dtype, pinned, (n, host_ld, ld))
    D = torch.full((n, ld), -1, dtype=dtype, device="cuda")
    km.upload(H, D=D)
    Dc = D.cpu()
    assert torch.equal(Dc[:, :n], H[:, :n])
    assert bool((Dc[:, n:] == 0).all())


@pytest.mark.parametrize("pinned", [True, False])
def test_upload_of_a_rectangular_matrix(pinned):
    """kmedoids_upload_rows: m location rows of n consumer columns (the
    bichromatic form), into a padded device buffer."""
    H = torch.from_numpy(np.random.default_rng(9).random((300, 1001), np.float32))
    if pinned:
        H = H.pin_memory()
    D = torch.full((300, 1004), -1.0, dtype=torch.float32, device="cuda")
    km.upload(H, n=1001, D=D)
    Dc = D.cpu()
    assert torch.equal(Dc[:, :1001], H[:, :1001]) and bool((Dc[:, 1001:] == 0).all())


def test_upload_rejects_a_device_source():
    lib = km.load()
    import ctypes
    X = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    Y = torch.empty_like(X)
    st = lib.kmedoids_upload_matrix(ctypes.c_void_p(X.data_ptr()), 64, km.KM_F32, 64,
                                    ctypes.c_void_p(Y.data_ptr()), 64, None)
    assert st == 1 and b"device address" in lib.kmedoids_last_error()


def test_run_on_an_uploaded_matrix():
    Dh = wl.manhattan_int32(wl.int_coords(1500, 2, 1000, seed="upload-run"))
    H = torch.from_numpy(Dh).pin_memory()
    D = km.upload(H)
    assert D.shape == (1500, 1500)
    out = km.run(D, 9)
    ref = oracle.run(Dh, 9, variant="fastpam1")
    assert out["medoids"].cpu().tolist() == ref["medoids"].tolist()
    assert out["td_i64"] == int(ref["td"])
