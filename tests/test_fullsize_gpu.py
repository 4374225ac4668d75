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


def test_fullsize_backward_identities(big):
    """At full size: the stencil gradient and the particle gradient satisfy the identities of a
    linear map, sum_l w_l . dL/dw_l = <g, out> = <x, dL/dx>, and are finite."""
    apr, lay, _ = big
    k = 5
    st = torch.as_tensor(G.apr_restrict_stencil(S.gaussian_stencil(5, 1.5).astype(np.float32), apr.l_max, apr.l_min), device="cuda")
    x = torch.as_tensor(apr.values, device="cuda")
    g = torch.as_tensor(np.random.default_rng(3).normal(size=apr.n_particles).astype(np.float32), device="cuda")
    tree = G.apr_tree_restrict(lay, x)
    out = G.apr_convolve(lay, x, tree, st, k)
    gp, gw = G.apr_convolve_backward(lay, x, tree, st, k, g)
    torch.cuda.synchronize()
    lay.sync_status()
    gw64, gp64 = gw.double().cpu().numpy(), gp.double().cpu().numpy()
    assert np.all(np.isfinite(gw64)) and np.all(np.isfinite(gp64))
    o64, g64, x64 = out.double().cpu().numpy(), g.double().cpu().numpy(), x.double().cpu().numpy()
    ref = float(np.dot(g64, o64))
    scale = float(np.dot(np.abs(g64), np.abs(o64)))
    assert abs(float(np.sum(st.double().cpu().numpy() * gw64)) - ref) <= 1e-5 * scale
    assert abs(float(np.dot(x64, gp64)) - ref) <= 1e-5 * scale


def test_fullsize_sampled_backward_parity(big):
    """Gradients of a sampled set of outputs (dL/dout zero elsewhere) vs the oracle at full size."""
    apr, lay, o = big
    k = 5
    st_h = G.apr_restrict_stencil(S.gaussian_stencil(5, 1.5).astype(np.float32), apr.l_max, apr.l_min)
    st = torch.as_tensor(st_h, device="cuda")
    x = torch.as_tensor(apr.values, device="cuda")
    rng = np.random.default_rng(4)
    sample = np.sort(rng.choice(apr.n_particles, 20000, replace=False))
    g_full = np.zeros(apr.n_particles, np.float32)
    g_full[sample] = rng.normal(size=sample.size).astype(np.float32)
    tree = G.apr_tree_restrict(lay, x)
    gp, gw = G.apr_convolve_backward(lay, x, tree, st, k, torch.as_tensor(g_full, device="cuda"))
    torch.cuda.synchronize()
    ref_gp, ref_gw = o.conv_backward(st_h.astype(np.float64), k, g_full.astype(np.float64), sample=sample)
    got_gw = gw.double().cpu().numpy()
    assert np.max(np.abs(got_gw - ref_gw.reshape(got_gw.shape))) <= 1e-5 * np.max(np.abs(ref_gw))
    got_gp = gp.double().cpu().numpy()
    assert np.max(np.abs(got_gp - ref_gp[:, 0])) <= 1e-5 * np.max(np.abs(ref_gp))
