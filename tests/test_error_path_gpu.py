"""Device-side failure detection without a GPU fault: a bounded wait that runs out (a barrier nothing
completes) is reported by apr_sync_status as APR_ERR_TIMEOUT, and the context stays usable."""
import numpy as np
import pytest
import torch

import aprsynth as S
import oracle
import paper_2112_03592_gb300 as G
from paper_2112_03592_gb300 import _abi

pytestmark = pytest.mark.gpu


def test_bounded_wait_timeout_is_reported_and_context_survives():
    apr = S.random_balanced_apr((12, 10, 40), 1, seed=3, p_fine=0.05)
    lay = G.AprLayout.from_apr(apr, G.APR_VALIDATE | G.APR_REQUIRE_BALANCE)
    lib = lay._lib
    assert lib.apr_selftest_bounded_wait(lay.handle, 2000, G._stream_ptr()) == _abi.APR_OK
    assert lib.apr_sync_status(lay.handle, G._stream_ptr()) == 6      # APR_ERR_TIMEOUT
    assert lib.apr_sync_status(lay.handle, G._stream_ptr()) == _abi.APR_OK   # the word was cleared
    # the handle and the context still work
    w = np.repeat(S.gaussian_stencil(3, 1.0).astype(np.float32).reshape(1, -1), apr.n_levels, 0)
    v = torch.as_tensor(apr.values.astype(np.float32), device="cuda")
    out = G.apr_convolve(lay, v, G.apr_tree_restrict(lay, v), torch.as_tensor(w, device="cuda"), 3)
    lay.sync_status()
    ref = oracle.Oracle(apr).conv(w.astype(np.float64), 3)[:, 0]
    assert np.max(np.abs(out.cpu().numpy() - ref) / np.abs(ref)) <= 1e-5
    assert lib.apr_selftest_bounded_wait(lay.handle, 0, G._stream_ptr()) == 1   # APR_ERR_INVALID_ARG
