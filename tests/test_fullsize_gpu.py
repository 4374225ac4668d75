"""Full-size workload (1024x1024x512 pixels, ~8M particles, 5^3 stencils): sampled parity against the
oracle in the launch configuration the benchmark times, plus properties that hold at any size."""
import numpy as np
import pytest
import torch

import aprsynth as S
import oracle
import paper_2112_03592_gb300 as G

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def big():
    apr = S.make_config("blob1024")
    lay = G.AprLayout.from_apr(apr, G.APR_VALIDATE | G.APR_REQUIRE_BALANCE)
    o = oracle.Oracle(apr)
    return apr, lay, o


@pytest.mark.parametrize("mode", ["plain", "restricted"])
def test_fullsize_sampled_parity(big, mode):
    apr, lay, o = big
    k = 5
    w = S.gaussian_stencil(k, 1.5).astype(np.float32)
    st = np.repeat(w.reshape(1, -1), apr.n_levels, 0) if mode == "plain" else G.apr_restrict_stencil(w, apr.l_max, apr.l_min)
    v = torch.as_tensor(apr.values, device="cuda")
    tree = G.apr_tree_restrict(lay, v)
    out = G.apr_convolve(lay, v, tree, torch.as_tensor(st, device="cuda"), k)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    sample = np.sort(rng.choice(apr.n_particles, 20000, replace=False))
    lev = apr.particle_coords()[0]
    # make sure every level is sampled, including its first and last particle
    for l in range(apr.l_min, apr.l_max + 1):
        idx = np.nonzero(lev == l)[0]
        if idx.size:
            sample = np.union1d(sample, [idx[0], idx[-1]])
    ref = o.conv(st.astype(np.float64), k, sample=sample)[:, 0]
    got = out.cpu().numpy()[sample]
    err = np.max(np.abs(got - ref) / np.abs(ref))
    assert err <= 1e-5, err
    tref = o.tree()[:, 0]
    tgot = tree.cpu().numpy()
    assert np.max(np.abs(tgot - tref) / np.abs(tref)) <= 1e-5


def test_fullsize_linearity_and_constant(big):
    apr, lay, _ = big
    k = 5
    st = torch.as_tensor(G.apr_restrict_stencil(S.gaussian_stencil(5, 1.5).astype(np.float32), apr.l_max, apr.l_min), device="cuda")
    c = torch.full((apr.n_particles,), 3.0, device="cuda")
    tree = G.apr_tree_restrict(lay, c)
    out = G.apr_convolve(lay, c, tree, st, k)
    torch.cuda.synchronize()
    assert torch.max(torch.abs(out - 3.0)).item() <= 3.0 * 1e-5
