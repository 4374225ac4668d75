"""apr_convolve_backward_noalloc: the backward pass for callers that cannot allocate device memory.

The entry point uses a fixed scratch array inside the library instead of a caller workspace. Its
results must equal those of apr_convolve_backward (which takes a caller workspace) on the same
inputs, on two calls in a row (the shared scratch keeps the first call's contents, so the second call
checks that whatever must start at zero is cleared). This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import aprsynth as S
import paper_2112_03592_gb300 as G
from paper_2112_03592_gb300 import _abi

pytestmark = pytest.mark.gpu
TOL = 1e-5  # the tolerance the other parity tests use (normwise)


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_backward_matches_workspace_backward_twice():
    apr = S.make_config("blob64", use_cache=False)
    lay = G.AprLayout.from_apr(apr)
    k = 5
    rng = np.random.default_rng(4)
    st = torch.as_tensor(rng.normal(size=(apr.n_levels, k ** 3)).astype(np.float32), device="cuda")
    v = torch.as_tensor(apr.values, device="cuda")
    tree = G.apr_tree_restrict(lay, v)
    lib = _abi.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        g = torch.as_tensor(rng.normal(size=apr.n_particles).astype(np.float32), device="cuda")
        ref_p, ref_w = G.apr_convolve_backward(lay, v, tree, st, k, g)
        gp = torch.full((apr.n_particles,), float("nan"), device="cuda")
        gw = torch.full((apr.n_levels, k ** 3), float("nan"), device="cuda")
        rc = lib.apr_convolve_backward_noalloc(lay.handle, _p(v), _p(tree), _p(st), k, G.APR_BC_REFLECT, _p(g),
                                               _p(gp), _p(gw), stream)
        _abi.check("apr_convolve_backward_noalloc", rc)
        torch.cuda.synchronize()
        for got, ref in ((gp, ref_p), (gw, ref_w)):
            err = (torch.max(torch.abs(got - ref)) / torch.max(torch.abs(ref))).item()
            assert err <= TOL, (call, err)
