"""apr_convolve_backward_noalloc: the backward pass for callers that cannot allocate device memory.

The entry point uses a fixed scratch array inside the library instead of a caller workspace. Its
results must equal those of apr_convolve_backward (which takes a caller workspace) on the same
inputs, on two calls in a row (the shared scratch keeps the first call's contents, so the second call
checks that whatever must start at zero is cleared). Both paths are deterministic, so they must
agree bit for bit. An APR whose backward scratch exceeds the fixed array is refused with
APR_ERR_UNSUPPORTED. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import aprsynth as S
import paper_2112_03592_gb300 as G
from paper_2112_03592_gb300 import _abi

pytestmark = pytest.mark.gpu
SCRATCH = 16 << 20   # bytes of the library's fixed scratch array


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("k", [3, 5])
def test_noalloc_backward_matches_workspace_backward_twice(k):
    apr = S.make_config("blob64", use_cache=False)
    lay = G.AprLayout.from_apr(apr)
    rng = np.random.default_rng(4 + k)
    st = torch.as_tensor(rng.normal(size=(apr.n_levels, k ** 3)).astype(np.float32), device="cuda")
    v = torch.as_tensor(apr.values, device="cuda")
    tree = G.apr_tree_restrict(lay, v)
    lib = _abi.load()
    assert lib.apr_backward_workspace_bytes(lay.handle, k) <= SCRATCH
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
        assert torch.equal(gp, ref_p), (call, "particle gradients differ")
        assert torch.equal(gw, ref_w), (call, "stencil gradients differ")


def _all_finest_layout(dims):
    """Host-only index of an APR whose every pixel is a particle of the finest level (33.5 M
    particles for 256 x 256 x 512): its backward scratch exceeds the fixed array."""
    l_max = int(np.ceil(np.log2(max(dims))))
    coarse_rows = sum(-(-dims[0] // (1 << (l_max - l))) * -(-dims[1] // (1 << (l_max - l))) for l in range(l_max))
    rows = dims[0] * dims[1]
    rp = np.concatenate([np.zeros(coarse_rows, np.int64), np.arange(rows + 1, dtype=np.int64) * dims[2]])
    y = np.tile(np.arange(dims[2], dtype=np.int32), rows)
    return G.AprLayout(dims, 0, l_max, rp, y, G.APR_HOST_ONLY)   # only the size check runs on it


def test_noalloc_backward_refuses_an_apr_larger_than_its_scratch():
    lay = _all_finest_layout((256, 256, 512))
    lib = _abi.load()
    assert lib.apr_backward_workspace_bytes(lay.handle, 5) > SCRATCH
    null = ctypes.c_void_p(0)
    rc = lib.apr_convolve_backward_noalloc(lay.handle, null, null, null, 5, G.APR_BC_REFLECT, null, null, null, null)
    assert rc == _abi.APR_ERR_UNSUPPORTED
