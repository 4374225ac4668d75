"""Pins of the oracle's APR CNN (Sec. 6 outlook) and of the parts of the oracle that only the CNN
and the stencil-size limit use, against things other than the oracle itself (CPU only).

- cnn_forward on an all-finest-level APR == a dense composition written from library routines:
  scipy.ndimage.correlate (reflect) per channel pair, np.maximum, torch's float -> bfloat16 cast and
  the residual read-out x + c / scale (scale != 1, so a misplaced scale fails).
- cnn_backward == torch autograd of the same dense network (rounding off), including a channel whose
  pre-activation is exactly zero (torch's ReLU has derivative 0 there; a mask c >= 0 fails).
- cnn_backward == FP64 central differences of cnn_forward (rounding off) on a multi-level APR, where
  the tree and the coarse fill take part.
- ora_check_coarse_fill counts uncovered taps: a closed-form count on a hand-built unbalanced APR,
  and a positive count at radius 3 on the 64^3 blob workload (Sec. 5.1 footnote: a 5^3 patch
  reaches one coarser level only under 2:1 balance).
- bf16 tree: a hand-derived golden where the FP32 accumulation in child order and the exact average
  round to different bfloat16 values two levels above the particles.
"""
import numpy as np
import pytest
import scipy.ndimage as ndi
import torch

import aprsynth as S
import oracle

GOLD = __import__("pathlib").Path(__file__).parent / "golden"


def _bf16(a):
    """torch's float32 -> bfloat16 cast (round to nearest even), as float64."""
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _finest(dims, rng):
    apr = S.uniform_level_apr(dims, S.l_max_for(dims))
    x = rng.integers(-64, 65, size=apr.n_particles) / 8.0
    return apr, x


def _weights(rng, L, n_layers, zero_co=None):
    Ws = []
    for i in range(n_layers):
        W = rng.integers(-16, 17, size=(L, 16, 16, 27)) / 16.0
        if zero_co is not None and i == 0:
            W[:, zero_co] = 0.0
        Ws.append(W)
    return Ws


def _dense_net(img, Ws, scale, level_idx):
    """The network on a dense image (every pixel a particle of the finest level)."""
    h = np.zeros((16,) + img.shape)
    h[0] = _bf16(np.float32(scale) * img.astype(np.float32))
    c = None
    for i, W in enumerate(Ws):
        w = W[level_idx].reshape(16, 16, 3, 3, 3)
        c = np.zeros_like(h)
        for co in range(16):
            for ci in range(16):
                if np.any(h[ci]):
                    c[co] += ndi.correlate(h[ci], w[co, ci], mode="reflect")
        if i + 1 < len(Ws):
            h = _bf16(np.maximum(c, 0.0))
    return img + c[0] / float(np.float32(scale))


@pytest.mark.parametrize("dims", [(6, 7, 9), (8, 8, 8)])
def test_cnn_forward_all_finest_equals_dense_composition(dims):
    rng = np.random.default_rng(3)
    apr, x = _finest(dims, rng)
    Ws = _weights(rng, apr.n_levels, 3)
    scale = 0.25  # exact in FP32 and bf16; every product and sum below is exact in FP64
    y = oracle.cnn_forward(apr, x, Ws, scale)
    img = x.reshape(dims)  # all-finest particles in l -> z -> x -> y order are the raster order
    ref = _dense_net(img, Ws, scale, apr.n_levels - 1).reshape(-1)
    np.testing.assert_array_equal(y, ref)


def _torch_net(img, Ws, scale, level_idx):
    """Same network in torch FP64 without roundings (autograd gives the weight gradients)."""
    t = [torch.tensor(W[level_idx].reshape(16, 16, 3, 3, 3), dtype=torch.float64, requires_grad=True) for W in Ws]
    x = torch.tensor(img, dtype=torch.float64)
    h = torch.zeros((1, 16) + img.shape, dtype=torch.float64)
    h[0, 0] = float(np.float32(scale)) * x
    c = None
    for i, w in enumerate(t):
        # half-sample symmetric reflection of radius 1 repeats the edge cell
        hp = torch.nn.functional.pad(h, (1, 1, 1, 1, 1, 1), mode="replicate")
        c = torch.nn.functional.conv3d(hp, w)  # conv3d is a correlation
        if i + 1 < len(t):
            h = torch.relu(c)
    y = x + c[0, 0] / float(np.float32(scale))
    return y, t


def test_cnn_backward_all_finest_equals_torch_autograd():
    dims = (5, 6, 7)
    rng = np.random.default_rng(4)
    apr, x = _finest(dims, rng)
    x = x + rng.uniform(-0.01, 0.01, size=x.size)  # no bf16-exactness needed with rounding off
    Ws = [rng.normal(scale=0.2, size=(apr.n_levels, 16, 16, 27)) for _ in range(3)]
    Ws[0][:, 5] = 0.0  # channel 5 of the first hidden layer is exactly 0: ReLU derivative 0 there
    scale = 0.5
    gy = rng.normal(size=x.size)
    got = oracle.cnn_backward(apr, x, Ws, scale, gy, rounding=False)
    y, t = _torch_net(x.reshape(dims), Ws, scale, apr.n_levels - 1)
    (y.reshape(-1) * torch.tensor(gy)).sum().backward()
    yo = oracle.cnn_forward(apr, x, Ws, scale, rounding=False)
    np.testing.assert_allclose(yo, y.detach().numpy().reshape(-1), rtol=0, atol=1e-12 * np.abs(yo).max())
    for i in range(3):
        ref = t[i].grad.numpy().reshape(16, 16, 27)
        g = got[i][apr.n_levels - 1]
        np.testing.assert_allclose(g, ref, rtol=0, atol=1e-10 * np.abs(ref).max())
        assert np.all(got[i][: apr.n_levels - 1] == 0.0)  # no particles on coarser levels
    assert np.all(got[1][:, :, 5] == 0.0)  # nothing flows into layer 1 from the all-zero channel
    assert np.all(got[0][:, 5] == 0.0)     # ... nor back through its ReLU at exactly 0


def test_cnn_backward_matches_central_differences_multilevel():
    apr = S.random_balanced_apr((8, 8, 12), 1, seed=5, p_fine=0.05)
    assert apr.n_levels >= 3
    rng = np.random.default_rng(6)
    x = rng.uniform(50.0, 150.0, size=apr.n_particles)
    Ws = [rng.normal(scale=0.15, size=(apr.n_levels, 16, 16, 27)) for _ in range(4)]
    scale = float(np.float32(1.0 / x.mean()))
    gy = rng.normal(size=apr.n_particles)
    grads = oracle.cnn_backward(apr, x, Ws, scale, gy, rounding=False)

    def loss(Wl):
        return float(gy @ oracle.cnn_forward(apr, x, Wl, scale, rounding=False))

    h = 1e-6
    for i in range(4):
        gmax = np.abs(grads[i]).max()
        assert gmax > 0
        flat = np.argsort(-np.abs(grads[i]).ravel())[:4]  # the largest entries ...
        flat = np.concatenate([flat, rng.choice(grads[i].size, 4, replace=False)])  # ... and random ones
        for f in flat:
            idx = np.unravel_index(f, grads[i].shape)
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[i][idx] += h
            Wm[i][idx] -= h
            fd = (loss(Wp) - loss(Wm)) / (2 * h)
            assert abs(fd - grads[i][idx]) <= 1e-6 * gmax, (i, idx, fd, grads[i][idx])


# ------------------------------------------------------------------------------------------
# the coarse-fill checker
# ------------------------------------------------------------------------------------------
def _unbalanced_apr():
    """8^3 image, l_max = 3, l_min = 1: octant [0,4)^3 split into 64 level-3 particles, the other
    seven octants level-1 particles (edge 4): finest particles touch particles two levels coarser."""
    ps = []
    for z in range(4):
        for x in range(4):
            for y in range(4):
                ps.append((3, z, x, y, 1.0))
    for z in range(2):
        for x in range(2):
            for y in range(2):
                if (z, x, y) != (0, 0, 0):
                    ps.append((1, z, x, y, 2.0))
    return S.apr_from_particles((8, 8, 8), 1, ps)


def test_coarse_fill_checker_counts_uncovered_taps_closed_form():
    o = oracle.Oracle(_unbalanced_apr())
    # A tap of a level-3 particle p = (a, b, c) in [0,4)^3 is uncovered iff p + e lies in the grid
    # but outside the octant (there only a level-1 particle covers it); the level-1 particles' taps
    # are covered by level-1 particles and the level-1 tree node. Per axis, the offsets in [-1, 1]
    # that stay in [0, 8) sum to 2 + 3 + 3 + 3 = 11 over a = 0..3 and those that stay in [0, 4) to
    # 2 + 3 + 3 + 2 = 10, so the count is 11^3 - 10^3.
    assert o.check_coarse_fill(1) == 11 ** 3 - 10 ** 3
    # radius 0 touches no other cell
    assert o.check_coarse_fill(0) == 0


def test_coarse_fill_checker_finds_radius3_gaps_on_blob64():
    apr = S.make_config("blob64")
    o = oracle.Oracle(apr)
    assert o.check_coarse_fill(2) == 0  # 2:1 balance covers every 5^3 tap
    assert o.check_coarse_fill(3) > 0   # a 7^3 patch reaches two coarser levels


# ------------------------------------------------------------------------------------------
# bf16 tree: FP32 accumulation in child order, two levels above the particles
# ------------------------------------------------------------------------------------------
def _golden_bf16_tree():
    rows = [l.split("|") for l in (GOLD / "tree_bf16.txt").read_text().splitlines()
            if l.strip() and not l.startswith("#")]
    child = {tuple(int(v) for v in r[1].split()): float(r[2]) for r in rows if r[0].strip() == "child"}
    root = {tuple(int(v) for v in r[1].split()): float(r[2]) for r in rows if r[0].strip() == "node"}
    return child, root


def test_bf16_tree_two_levels_up_golden():
    child, root = _golden_bf16_tree()
    # 4^3 image, every pixel a level-2 particle; each level-1 node's 8 particles carry its value
    ps = []
    for z in range(4):
        for x in range(4):
            for y in range(4):
                ps.append((2, z, x, y, child[(z // 2, x // 2, y // 2)]))
    apr = S.apr_from_particles((4, 4, 4), 0, ps)
    o = oracle.Oracle(apr, apr.values.astype(np.float64))
    t = o.tree_bf16()[:, 0]
    tc = o.tree_coords()
    got = {(int(c[0]), int(c[1]), int(c[2]), int(c[3])): v for c, v in zip(tc, t)}
    for (z, x, y), v in child.items():
        assert got[(1, z, x, y)] == v
    for key, v in root.items():
        assert got[key] == v
    # the exact average of the same children rounds elsewhere: the golden pins the FP32 reading
    exact = sum(child.values()) / 8.0
    assert _bf16(exact) != root[(0, 0, 0, 0)]
