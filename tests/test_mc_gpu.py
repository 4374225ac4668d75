"""Multi-channel (bfloat16, 16 -> 16 channels, 3^3) CUDA path vs the oracle, through the C ABI.

Features and weights are bfloat16 numbers (multiples of 1/8 and 1/16), so the oracle sees exactly
the GPU's inputs; the BF16 tree is compared bit for bit, outputs and gradients (FP32 accumulation on
the tensor cores vs FP64) normwise against 1e-5.
"""
import numpy as np
import pytest
import torch

import aprsynth as S
import oracle
import paper_2112_03592_gb300 as G

pytestmark = pytest.mark.gpu
FLAGS = G.APR_VALIDATE | G.APR_REQUIRE_BALANCE
C = 16
NORM = 1e-5   # max |gpu - oracle| / max |oracle|

CASES = {
    "blob64": lambda: S.make_config("blob64", use_cache=False),
    "rand_ragged": lambda: S.random_balanced_apr((21, 13, 150), 1, seed=7, p_fine=0.01),
    "rand_thin": lambda: S.random_balanced_apr((3, 40, 9), 0, seed=8, p_fine=0.05),
    "all_max": lambda: S.uniform_level_apr((9, 17, 70), 7, l_min=2),
    "uniform_coarse": lambda: S.uniform_level_apr((32, 32, 32), 3, l_min=3),
    "tiny": lambda: S.random_balanced_apr((2, 3, 5), 0, seed=9, p_fine=0.3),
    "single": lambda: S.uniform_level_apr((1, 1, 1), 0, l_min=0),
    # level grids 2 cells wide along z and x: with reflection a coarse particle has up to 4 x 4 x 3
    # pre-images (two of them here reach more than 32), and the 5^3 mirror lists take the d < 2R path
    "thin_2x2": lambda: S.random_balanced_apr((2, 2, 40), 0, seed=22, p_fine=0.3),
}


def bf16_inputs(apr, seed):
    """Features k/8 in [-8, 8], weights k/16 in [-1, 1]: all exact in bfloat16."""
    rng = np.random.default_rng(seed)
    x = rng.integers(-64, 65, size=(apr.n_particles, C)) / 8.0
    w = rng.integers(-16, 17, size=(apr.n_levels, C, C, 27)) / 16.0
    g = rng.integers(-64, 65, size=(apr.n_particles, C)) / 8.0
    return x, w, g


def to_bf16(a):
    t = torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda").to(torch.bfloat16)
    assert np.array_equal(t.float().cpu().numpy().astype(np.float64), np.asarray(a, np.float64))
    return t.contiguous()


def assert_norm(got, ref, tol=NORM):
    ref = np.asarray(ref, np.float64)
    got = np.asarray(got, np.float64)
    assert got.shape == ref.shape
    assert np.all(np.isfinite(got)), "non-finite GPU outputs"
    if ref.size == 0:
        return
    err = np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-30)
    assert err <= tol, f"normwise error {err:.3e} > {tol}"


def run_gpu(apr, x, w, g, bc):
    lay = G.AprLayout.from_apr(apr, FLAGS)
    xd = to_bf16(x)
    tree = G.apr_tree_restrict_bf16(lay, xd)
    wd = to_bf16(w)
    out = G.apr_convolve_mc(lay, xd, tree, wd, bc)
    gp, gw = G.apr_convolve_mc_backward(lay, xd, tree, wd, to_bf16(g), bc)
    torch.cuda.synchronize()
    lay.sync_status()
    return (tree.float().cpu().numpy().astype(np.float64), out.cpu().numpy(), gp.cpu().numpy(),
            gw.cpu().numpy())


@pytest.mark.parametrize("bc", [G.APR_BC_REFLECT, G.APR_BC_ZERO])
@pytest.mark.parametrize("case", list(CASES))
def test_mc_forward_backward_match_oracle(case, bc):
    apr = CASES[case]()
    x, w, g = bf16_inputs(apr, seed=len(case) + 3 * bc)
    tree, out, gp, gw = run_gpu(apr, x, w, g, bc)
    o = oracle.Oracle(apr, x)
    ref_tree = o.tree_bf16()
    np.testing.assert_array_equal(tree, ref_tree)           # bit-exact BF16 tree
    assert_norm(out, o.conv(w, 3, bc, C_out=C))
    ref_gp, ref_gw = o.conv_backward(w, 3, g, bc, C_out=C)
    assert_norm(gp, ref_gp)
    assert_norm(gw, ref_gw)


def test_mc_backward_is_deterministic():
    apr = CASES["blob64"]()
    x, w, g = bf16_inputs(apr, seed=11)
    a = run_gpu(apr, x, w, g, G.APR_BC_REFLECT)
    b = run_gpu(apr, x, w, g, G.APR_BC_REFLECT)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_mc_rejects_unsupported_shapes():
    apr = CASES["tiny"]()
    lay = G.AprLayout.from_apr(apr, FLAGS)
    lib = lay._lib
    x = torch.zeros((apr.n_particles, C), dtype=torch.bfloat16, device="cuda")
    t = torch.zeros((max(lay.n_tree, 1), C), dtype=torch.bfloat16, device="cuda")
    w = torch.zeros((apr.n_levels, C, C, 27), dtype=torch.bfloat16, device="cuda")
    out = torch.zeros((apr.n_particles, C), dtype=torch.float32, device="cuda")
    p = lambda a: a.data_ptr()
    s = G._stream_ptr()
    assert lib.apr_convolve_mc(lay.handle, p(x), p(t), p(w), 8, 16, 3, 0, p(out), s) == 3   # UNSUPPORTED
    assert lib.apr_convolve_mc(lay.handle, p(x), p(t), p(w), 16, 16, 5, 0, p(out), s) == 3
    assert lib.apr_convolve_mc(lay.handle, p(x), p(t), p(w), 16, 16, 3, 7, p(out), s) == 1   # bad bc
    assert lib.apr_convolve_mc(lay.handle, p(x) + 2, p(t), p(w), 16, 16, 3, 0, p(out), s) == 1  # misaligned
    assert lib.apr_tree_restrict_bf16(lay.handle, p(x), p(t), 8, s) == 3


def test_bf16_tree_golden_two_levels_up():
    """The hand-derived bf16 tree of tests/golden/tree_bf16.txt (FP32 accumulation in child order
    loses a term that the exact average keeps) in channel 0, bit for bit on the GPU."""
    from test_oracle_cnn_pins import _golden_bf16_tree
    child, root = _golden_bf16_tree()
    ps = []
    for z in range(4):
        for x in range(4):
            for y in range(4):
                ps.append((2, z, x, y, child[(z // 2, x // 2, y // 2)]))
    apr = S.apr_from_particles((4, 4, 4), 0, ps)
    lay = G.AprLayout.from_apr(apr, FLAGS)
    xm = np.zeros((apr.n_particles, C))
    xm[:, 0] = apr.values
    tree = G.apr_tree_restrict_bf16(lay, to_bf16(xm)).float().cpu().numpy()
    torch.cuda.synchronize()
    ref = oracle.Oracle(apr, xm).tree_bf16()
    np.testing.assert_array_equal(tree.astype(np.float64), ref)
    tc = oracle.Oracle(apr, xm).tree_coords()
    i0 = [i for i, c in enumerate(tc) if tuple(int(v) for v in c) == (0, 0, 0, 0)][0]
    assert tree[i0, 0] == root[(0, 0, 0, 0)]
