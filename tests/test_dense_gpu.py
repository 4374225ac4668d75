"""The hand-written dense pixel-grid stencil (the dense comparison of bench.py) against
scipy.ndimage.correlate in FP64, through the C ABI."""
import numpy as np
import pytest
import scipy.ndimage as ndi
import torch

import paper_2112_03592_gb300 as G

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(20, 37, 70), (1, 9, 130), (40, 8, 64), (3, 2, 5)])
@pytest.mark.parametrize("k", [3, 5])
@pytest.mark.parametrize("bc", [G.APR_BC_REFLECT, G.APR_BC_ZERO])
def test_dense_convolve_matches_scipy(shape, k, bc):
    rng = np.random.default_rng(sum(shape) + k)
    img = rng.uniform(50, 500, size=shape).astype(np.float32)
    w = rng.normal(size=(k, k, k)).astype(np.float32)
    got = G.apr_dense_convolve(torch.as_tensor(img, device="cuda"), torch.as_tensor(w.reshape(-1), device="cuda"), k, bc)
    torch.cuda.synchronize()
    mode = "reflect" if bc == G.APR_BC_REFLECT else "constant"
    ref = ndi.correlate(img.astype(np.float64), w.astype(np.float64), mode=mode, cval=0.0)
    err = np.max(np.abs(got.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert err <= 1e-5, err
