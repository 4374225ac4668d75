"""Gradient magnitude (Sec. 4.3): three convolutions on one staged patch, CUDA vs oracle."""
import numpy as np
import pytest
import torch

import aprsynth as S
import oracle
import paper_2112_03592_gb300 as G

pytestmark = pytest.mark.gpu
FLAGS = G.APR_VALIDATE | G.APR_REQUIRE_BALANCE

CASES = {
    "blob64": lambda: S.make_config("blob64", use_cache=False),
    "rand_ragged": lambda: S.random_balanced_apr((21, 13, 150), 1, seed=7, p_fine=0.01),
    "all_max": lambda: S.uniform_level_apr((9, 17, 70), 7, l_min=2),
    "tiny": lambda: S.random_balanced_apr((2, 3, 5), 0, seed=9, p_fine=0.3),
}


def stacks(apr, k, kind):
    if kind == "sobel":
        sob = G.sobel_stencils(3)
        return np.stack([G.apr_rescale_stencil(sob[a], apr.l_max, apr.l_min) for a in range(3)]).astype(np.float32)
    return np.random.default_rng(1).normal(size=(3, apr.n_levels, k ** 3)).astype(np.float32)


@pytest.mark.parametrize("bc", [G.APR_BC_REFLECT, G.APR_BC_ZERO])
@pytest.mark.parametrize("k,kind", [(3, "sobel"), (5, "random")])
@pytest.mark.parametrize("case", list(CASES))
def test_gradient_magnitude_matches_oracle(case, k, kind, bc):
    apr = CASES[case]()
    W = stacks(apr, k, kind)
    lay = G.AprLayout.from_apr(apr, FLAGS)
    v = torch.as_tensor(apr.values.astype(np.float32), device="cuda")
    tree = G.apr_tree_restrict(lay, v)
    got = G.apr_gradient_magnitude(lay, v, tree, torch.as_tensor(W, device="cuda"), k, bc).cpu().numpy()
    lay.sync_status()
    ref = oracle.gradient_magnitude(apr, apr.values.astype(np.float32), W.astype(np.float64), k, bc)
    assert np.all(np.isfinite(got))
    err = np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-30)
    assert err <= 1e-5, f"normwise error {err:.3e}"
