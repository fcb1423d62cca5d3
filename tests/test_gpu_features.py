"""Tensor-core (tcgen05) path of the on-the-fly distance form: the BF16 Gram
product against an FP32 reference.  BF16 products are exact in FP32, so
only the FP32 summation order differs: |G - G_ref| <= 1e-5 * sum |x_i y_i|."""
import numpy as np
import pytest

from paper_2008_05171_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2008_05171_gb300.kmedoids as km  # noqa: E402


@pytest.mark.parametrize("n,d", [(128, 16), (200, 64), (300, 128), (517, 256),
                                 (1000, 128)])
def test_gram_bf16_matches_fp32(n, d):
    X = wl.features_200000(n=n, d=d, n_centers=7)
    Xt = torch.from_numpy(X).to(torch.bfloat16)
    assert (Xt.float().numpy() == X).all()  # bf16-exact inputs
    G = km.gram_bf16(Xt.cuda()).cpu().numpy().astype(np.float64)
    X64 = X.astype(np.float64)
    ref = X64 @ X64.T
    bound = 1e-5 * (np.abs(X64) @ np.abs(X64).T) + 1e-6
    assert np.all(np.abs(G - ref) <= bound), np.max(np.abs(G - ref) / bound)
