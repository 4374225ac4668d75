"""APR CNN (16 bf16 channels, 3^3 per-level weights, ReLU, residual read-out): element-wise kernels
bit for bit, every layer of the network against the oracle fed the GPU's own bf16 inputs (1e-5), and
the whole network's forward and weight gradients vs the FP64 oracle network as a sanity bound."""
import numpy as np
import pytest
import torch

import aprsynth as S
import oracle
import paper_2112_03592_gb300 as G
from paper_2112_03592_gb300.surrogate import AprCnn

pytestmark = pytest.mark.gpu
FLAGS = G.APR_VALIDATE | G.APR_REQUIRE_BALANCE


def f32(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")


def test_elementwise_kernels_bit_exact():
    rng = np.random.default_rng(0)
    n = 1000
    x = (rng.normal(size=n) * 100).astype(np.float32)
    c = (rng.normal(size=(n, 16)) * 3).astype(np.float32)
    g = rng.normal(size=(n, 16)).astype(np.float32)
    scale = np.float32(0.0123)
    e = G.apr_mc_embed_bf16(f32(x), float(scale)).float().cpu().numpy()
    ref = np.zeros((n, 16))
    ref[:, 0] = oracle.round_bf16_array(scale * x)
    np.testing.assert_array_equal(e, ref)
    np.testing.assert_array_equal(G.apr_mc_relu_bf16(f32(c)).float().cpu().numpy(),
                                  oracle.round_bf16_array(np.maximum(c, 0)))
    np.testing.assert_array_equal(G.apr_mc_relu_backward_bf16(f32(c), f32(g)).float().cpu().numpy(),
                                  oracle.round_bf16_array(np.where(c > 0, g, 0)))
    inv = np.float32(1.0) / scale
    np.testing.assert_array_equal(G.apr_mc_readout(f32(c), f32(x), float(inv)).cpu().numpy(),
                                  (x + np.float32(inv) * c[:, 0]).astype(np.float32))
    rb = G.apr_mc_readout_backward_bf16(f32(x), float(inv)).float().cpu().numpy()
    ref = np.zeros((n, 16))
    ref[:, 0] = oracle.round_bf16_array(np.float32(inv) * x)
    np.testing.assert_array_equal(rb, ref)


CASES = {
    "blob64": lambda: S.make_config("blob64", use_cache=False),
    "rand_ragged": lambda: S.random_balanced_apr((21, 13, 150), 1, seed=7, p_fine=0.01),
}


@pytest.mark.parametrize("case", list(CASES))
def test_cnn_forward_and_gradients_match_oracle(case):
    apr = CASES[case]()
    lay = G.AprLayout.from_apr(apr, FLAGS)
    x = apr.values.astype(np.float32)
    scale = float(np.float32(1.0 / x.mean()))
    model = AprCnn(4, seed=1)
    Wb = model.stack_weights(lay)
    Wh = [w.float().cpu().numpy().astype(np.float64) for w in Wb]
    y = model.forward(lay, f32(x), scale, keep=True, weights=Wb)
    gy = np.random.default_rng(2).normal(size=apr.n_particles).astype(np.float32)
    grads = model.backward(f32(gy))
    torch.cuda.synchronize()
    lay.sync_status()
    ref_y = oracle.cnn_forward(apr, x, Wh, scale)
    # end to end only as a sanity bound (the layer-by-layer test holds each step to 1e-5): bf16
    # rounding decisions taken on FP32 (GPU) and FP64 (oracle) values can differ by one bf16 unit at
    # a few activations, and those differences propagate
    d_got = y.double().cpu().numpy() - x
    d_ref = ref_y - x
    err = np.max(np.abs(d_got - d_ref)) / np.max(np.abs(d_ref))
    assert err <= 1e-2, f"forward residual normwise error {err:.3e}"
    ref_g = oracle.cnn_backward(apr, x, Wh, scale, gy)
    for i, (gg, rg) in enumerate(zip(grads, ref_g)):
        gg = gg.double().cpu().numpy()
        e = np.max(np.abs(gg - rg)) / np.max(np.abs(rg))
        assert np.all(np.isfinite(gg)) and e <= 2e-2, f"layer {i} weight gradient normwise error {e:.3e}"


def _nerr(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    assert np.all(np.isfinite(got))
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-30))


@pytest.mark.parametrize("case", list(CASES))
def test_cnn_layer_by_layer_matches_oracle(case):
    """Every step of the network on the GPU against the oracle fed the GPU's own bf16 inputs of that
    step: embedding and activations bit for bit, bf16 trees bit for bit, each convolution and each
    convolution transpose (data and weight gradients) normwise 1e-5, read-out and its transpose bit
    for bit. Layer order, level indexing and the read-out scale are fixed by this chain."""
    apr = CASES[case]()
    lay = G.AprLayout.from_apr(apr, FLAGS)
    x = apr.values.astype(np.float32)
    scale = float(np.float32(1.0 / x.mean()))
    model = AprCnn(4, seed=1)
    Wb = model.stack_weights(lay)
    Wh = [w.float().cpu().numpy().astype(np.float64) for w in Wb]
    y = model.forward(lay, f32(x), scale, keep=True, weights=Wb)
    torch.cuda.synchronize()
    lay.sync_status()
    _, _, _, saved = model._saved
    host = lambda t: t.float().cpu().numpy().astype(np.float64)
    ref_h0 = np.zeros((apr.n_particles, 16))
    ref_h0[:, 0] = oracle.round_bf16_array(np.float32(scale) * x)
    np.testing.assert_array_equal(host(saved[0][0]), ref_h0)
    for i, (h, tree, c) in enumerate(saved):
        hh = host(h)
        o = oracle.Oracle(apr, hh)
        np.testing.assert_array_equal(host(tree), o.tree_bf16())
        e = _nerr(host(c), o.conv(Wh[i], 3, C_out=16))
        assert e <= 1e-5, f"layer {i} convolution normwise error {e:.3e}"
        if i + 1 < len(saved):
            np.testing.assert_array_equal(host(saved[i + 1][0]), oracle.round_bf16_array(np.maximum(host(c), 0.0)))
    c_last = saved[-1][2].float().cpu().numpy()
    inv = np.float32(1.0 / scale)  # the FP32 factor the read-out receives
    np.testing.assert_array_equal(y.cpu().numpy(), (x + inv * c_last[:, 0]).astype(np.float32))
    # backward, step by step
    gy = np.random.default_rng(2).normal(size=apr.n_particles).astype(np.float32)
    g = G.apr_mc_readout_backward_bf16(f32(gy), float(inv))
    ref_g = np.zeros((apr.n_particles, 16))
    ref_g[:, 0] = oracle.round_bf16_array(inv * gy)
    np.testing.assert_array_equal(host(g), ref_g)
    for i in reversed(range(len(saved))):
        h, tree, _ = saved[i]
        gp, gw = G.apr_convolve_mc_backward(lay, h, tree, Wb[i], g, need_particles=i > 0)
        torch.cuda.synchronize()
        o = oracle.Oracle(apr, host(h))
        o.tree_bf16()
        rp, rw = o.conv_backward(Wh[i], 3, host(g), C_out=16)
        e = _nerr(gw.double().cpu().numpy(), rw)
        assert e <= 1e-5, f"layer {i} weight gradient normwise error {e:.3e}"
        if i > 0:
            e = _nerr(gp.double().cpu().numpy(), rp)
            assert e <= 1e-5, f"layer {i} data gradient normwise error {e:.3e}"
            g = G.apr_mc_relu_backward_bf16(saved[i - 1][2], gp)
            c_prev = saved[i - 1][2].float().cpu().numpy()
            np.testing.assert_array_equal(host(g), oracle.round_bf16_array(np.where(c_prev > 0, gp.cpu().numpy(), 0)))


def test_cnn_training_reduces_loss():
    from paper_2112_03592_gb300.surrogate import train
    apr = CASES["blob64"]()
    lay = G.AprLayout.from_apr(apr, FLAGS)
    x = f32(apr.values)
    w = S.gaussian_stencil(3, 1.0).astype(np.float32)
    st = torch.as_tensor(G.apr_restrict_stencil(w, apr.l_max, apr.l_min), device="cuda")
    target = G.apr_richardson_lucy(lay, x, st, 3, 5)
    model = AprCnn(4, seed=0)
    hist = train(model, [(lay, x, target, float(1.0 / x.mean()))], steps=60, lr=3e-3)
    assert np.isfinite(hist).all() and np.mean(hist[-10:]) < 0.5 * np.mean(hist[:5])


def test_fused_relu_layer_equals_convolution_then_relu():
    apr = CASES["rand_ragged"]()
    lay = G.AprLayout.from_apr(apr, FLAGS)
    rng = np.random.default_rng(5)
    x = torch.as_tensor((rng.integers(-64, 65, size=(apr.n_particles, 16)) / 8.0).astype(np.float32), device="cuda").to(torch.bfloat16)
    w = torch.as_tensor(rng.normal(scale=0.1, size=(apr.n_levels, 16, 16, 27)).astype(np.float32), device="cuda").to(torch.bfloat16)
    tree = G.apr_tree_restrict_bf16(lay, x)
    fused = G.apr_convolve_mc_relu_bf16(lay, x, tree, w)
    plain = G.apr_mc_relu_bf16(G.apr_convolve_mc(lay, x, tree, w))
    torch.cuda.synchronize()
    assert torch.equal(fused, plain)
