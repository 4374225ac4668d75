"""Full-size multi-channel (256^3 blob APR, ~1M particles, 16 channels) and Richardson-Lucy (512^3 blob
APR, 2.9M particles) workloads, in the launch configuration bench.py times: sampled parity against
the oracle, bit-exact BF16 tree, and properties that hold at any size."""
import numpy as np
import pytest
import torch

import aprsynth as S
import oracle
import paper_2112_03592_gb300 as G

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
FLAGS = G.APR_VALIDATE | G.APR_REQUIRE_BALANCE


@pytest.fixture(scope="module")
def mc():
    import bench
    apr = S.make_config(bench.MC_WORKLOAD)
    lay = G.AprLayout.from_apr(apr, FLAGS)
    x, w, g = bench.mc_inputs(apr)
    return apr, lay, x, w, g


def bf(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda").to(torch.bfloat16).contiguous()


def test_fullsize_mc_tree_bit_exact_and_sampled_forward(mc):
    apr, lay, x, w, g = mc
    xd, wd = bf(x), bf(w)
    tree = G.apr_tree_restrict_bf16(lay, xd)
    out = G.apr_convolve_mc(lay, xd, tree, wd)
    torch.cuda.synchronize()
    lay.sync_status()
    o = oracle.Oracle(apr, x)
    np.testing.assert_array_equal(tree.float().cpu().numpy().astype(np.float64), o.tree_bf16())
    sample = np.sort(np.random.default_rng(0).choice(apr.n_particles, 4000, replace=False))
    ref = o.conv(w, 3, sample=sample, C_out=16)
    got = out.cpu().numpy()[sample]
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))


def test_fullsize_mc_backward_identities_and_sampled_parity(mc):
    apr, lay, x, w, g = mc
    xd, wd = bf(x), bf(w)
    tree = G.apr_tree_restrict_bf16(lay, xd)
    out = G.apr_convolve_mc(lay, xd, tree, wd)
    gp, gw = G.apr_convolve_mc_backward(lay, xd, tree, wd, bf(g))
    torch.cuda.synchronize()
    lay.sync_status()
    o64, g64 = out.double().cpu().numpy(), np.asarray(g, np.float64)
    ref = float(np.sum(g64 * o64))
    scale = float(np.sum(np.abs(g64) * np.abs(o64)))
    w64 = wd.double().cpu().numpy()
    assert np.all(np.isfinite(gw.cpu().numpy())) and np.all(np.isfinite(gp.cpu().numpy()))
    # <w, dL/dw> = <g, out> = <x, dL/dx> for the linear layer (the tree rounding taken as identity in
    # the adjoint makes <x, dL/dx> use the unrounded average: compare with the same tolerance scale)
    assert abs(float(np.sum(w64 * gw.double().cpu().numpy())) - ref) <= 1e-5 * scale
    # gradients of a sampled subset of outputs vs the oracle
    sample = np.sort(np.random.default_rng(1).choice(apr.n_particles, 3000, replace=False))
    gs = np.zeros_like(g)
    gs[sample] = g[sample]
    gp2, gw2 = G.apr_convolve_mc_backward(lay, xd, tree, wd, bf(gs))
    torch.cuda.synchronize()
    rgp, rgw = oracle.Oracle(apr, x).conv_backward(w, 3, gs, C_out=16, sample=sample)
    # each weight-gradient entry sums ~3000 targets x 16 channels of products; the tensor cores
    # accumulate them in FP32 over ~200 MMA steps per CTA plus the cross-CTA reduction, so the bound
    # is relative to the sum of the terms' magnitudes (an upper bound from |x|, |g|), not to the
    # signed result
    _, abs_gw = oracle.Oracle(apr, np.abs(x)).conv_backward(w, 3, np.abs(gs), C_out=16, sample=sample)
    e_w = np.max(np.abs(gw2.cpu().numpy() - rgw)) / np.max(abs_gw)
    e_p = np.max(np.abs(gp2.cpu().numpy() - rgp)) / np.max(np.abs(rgp))
    print(f"full-size multi-channel sampled backward: weight grad {e_w:.3e} (of sum |terms|), data grad {e_p:.3e}")
    assert e_w <= 1e-5, e_w
    assert e_p <= 1e-5, e_p


def test_fullsize_rl_identity_psf_and_constant_image():
    import bench
    apr = S.make_config(bench.RL_WORKLOAD)
    lay = G.AprLayout.from_apr(apr, FLAGS)
    u = torch.as_tensor(apr.values, device="cuda")
    delta = np.zeros((apr.n_levels, 125), np.float32)
    delta[:, 62] = 1.0
    est = G.apr_richardson_lucy(lay, u, torch.as_tensor(delta, device="cuda"), 5, 3)
    torch.cuda.synchronize()
    # identity PSF: i_1 = i_0 * (u / i_0) = u, exactly (u > 0), and then stays u
    assert torch.equal(est, u)
    c = torch.full_like(u, 7.25)
    st = torch.as_tensor(G.apr_restrict_stencil(S.gaussian_stencil(5, 1.5).astype(np.float32), apr.l_max, apr.l_min),
                         device="cuda")
    est = G.apr_richardson_lucy(lay, c, st, 5, bench.RL_ITERS)
    torch.cuda.synchronize()
    lay.sync_status()
    assert float(torch.max(torch.abs(est - 7.25))) <= 7.25 * 1e-5
