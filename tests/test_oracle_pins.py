"""Pins of the FP64 oracle against things other than itself (CPU only).

P1  all-max-level APR: APR convolution == dense correlation of the image (scipy.ndimage), Sec. 4.1.
P2  uniform level-l APR + restricted stencil == block mean of the dense correlation of the
    upsampled image (R_l K_w P_l with R_l P_l = I), Eq. (restrict_stenc).
P3  constant image + normalised stencils stays constant.
P4  tree value == mean of the full-resolution reconstruction over the node's pixels (Sec. 3.4).
P5  brute force: level-l patch values == block means of the full-resolution reconstruction
    (Sec. 3.5 footnote), densely correlated and sampled at the level-l particles.
P6  backward == transpose of the forward map, built column by column (tiny inputs).
P7  restriction commutes with the stencil flip.
P9  restricted stencils: golden hand derivations, identity at s = 1, sum preserved.
Golden tree values of hand-built APRs (including an image edge with missing children).
"""
import numpy as np
import pytest
import scipy.ndimage as ndi

import aprsynth as S
import oracle
from oracle import Oracle, restrict_stencil

GOLD = __import__("pathlib").Path(__file__).parent / "golden"


def _stack(ws, L):
    ws = np.asarray(ws, np.float64)
    if ws.ndim == 3:
        ws = np.repeat(ws[None], L, 0)
    return ws.reshape(L, -1)


def _block_mean(F, s):
    z, x, y = F.shape
    return F.reshape(z // s, s, x // s, s, y // s, s).mean(axis=(1, 3, 5))


# ------------------------------------------------------------------------------------------ P1
@pytest.mark.parametrize("dims", [(9, 7, 12), (8, 8, 8), (5, 11, 6)])
@pytest.mark.parametrize("k", [3, 5])
@pytest.mark.parametrize("bc", [oracle.BC_REFLECT, oracle.BC_ZERO])
def test_p1_all_max_level_equals_dense_correlation(dims, k, bc):
    rng = np.random.default_rng(sum(dims) * 10 + k + bc)
    l_max = S.l_max_for(dims)
    img = rng.uniform(-3.0, 7.0, size=dims)
    apr = S.uniform_level_apr(dims, l_max, values_fn=lambda d: img)
    w = rng.normal(size=(k, k, k))                    # not symmetric: catches flips / axis swaps
    o = Oracle(apr, img[tuple(apr.particle_coords()[1:])])
    out = o.conv(_stack(w, apr.n_levels), k, bc=bc)[:, 0]
    mode = "reflect" if bc == oracle.BC_REFLECT else "constant"
    ref = ndi.correlate(img, w, mode=mode, cval=0.0)
    _, z, x, y = apr.particle_coords()
    np.testing.assert_allclose(out, ref[z, x, y], rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------------------------------ P2
@pytest.mark.parametrize("k,sigma", [(3, 1.0), (5, 1.5)])
@pytest.mark.parametrize("level_drop", [1, 2])
def test_p2_uniform_level_restricted_equals_block_mean(k, sigma, level_drop):
    dims = (16, 32, 24)
    l_max = S.l_max_for(dims)
    l = l_max - level_drop
    s = 1 << level_drop
    rng = np.random.default_rng(k * 7 + level_drop)
    d = S.level_dims(dims, l_max, l)
    u = rng.uniform(0.0, 100.0, size=d)
    apr = S.uniform_level_apr(dims, l, values_fn=lambda dd: u)
    w = S.gaussian_stencil(k, sigma) * rng.uniform(0.5, 1.5, size=(k, k, k))  # not separable
    wl = restrict_stencil(w, l_max, l)
    o = Oracle(apr, u[tuple(apr.particle_coords()[1:])])
    out = o.conv(wl.reshape(wl.shape[0], -1), k)[:, 0]
    fine = np.kron(u, np.ones((s, s, s)))
    ref = _block_mean(ndi.correlate(fine, w, mode="reflect"), s)
    _, z, x, y = apr.particle_coords()
    np.testing.assert_allclose(out, ref[z, x, y], rtol=1e-12, atol=1e-10)


# ------------------------------------------------------------------------------------------ P3
@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("k", [3, 5])
def test_p3_constant_image_stays_constant(seed, k):
    apr = S.random_balanced_apr((16, 16, 16), 1, seed=seed, values="const")
    o = Oracle(apr)
    np.testing.assert_allclose(o.tree()[:, 0], 7.25, rtol=1e-14)
    w = S.gaussian_stencil(k, 1.0)
    for ws in (_stack(w, apr.n_levels), restrict_stencil(w, apr.l_max, apr.l_min).reshape(apr.n_levels, -1)):
        out = o.conv(ws, k)[:, 0]
        np.testing.assert_allclose(out, 7.25, rtol=1e-13)


# ------------------------------------------------------------------------------------------ P4
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_p4_tree_is_volume_mean_of_reconstruction(seed):
    apr = S.random_balanced_apr((16, 16, 16), 1, seed=seed)
    o = Oracle(apr)
    F = S.paint_full(apr)
    tc = o.tree_coords()
    tv = o.tree()[:, 0]
    assert len(tv) > 0
    for (l, z, x, y), v in zip(tc, tv):
        s = 1 << (apr.l_max - l)
        ref = F[z * s:(z + 1) * s, x * s:(x + 1) * s, y * s:(y + 1) * s].mean()
        assert abs(v - ref) <= 1e-12 * max(1.0, abs(ref))


# ------------------------------------------------------------------------------------------ P5
@pytest.mark.parametrize("seed", [3, 4])
@pytest.mark.parametrize("k", [3, 5])
@pytest.mark.parametrize("bc", [oracle.BC_REFLECT, oracle.BC_ZERO])
def test_p5_brute_force_block_mean_patches(seed, k, bc):
    dims = (16, 32, 16)
    apr = S.random_balanced_apr(dims, 1, seed=seed, p_fine=0.02)
    rng = np.random.default_rng(seed + 100)
    L = apr.n_levels
    ws = rng.normal(size=(L, k, k, k))
    o = Oracle(apr)
    out = o.conv(ws.reshape(L, -1), k, bc=bc)[:, 0]
    F = S.paint_full(apr)
    lev, z, x, y = apr.particle_coords()
    ref = np.zeros(apr.n_particles)
    mode = "reflect" if bc == oracle.BC_REFLECT else "constant"
    for l in range(apr.l_min, apr.l_max + 1):
        m = lev == l
        if not m.any():
            continue
        U = _block_mean(F, 1 << (apr.l_max - l))
        C = ndi.correlate(U, ws[l - apr.l_min], mode=mode, cval=0.0)
        ref[m] = C[z[m], x[m], y[m]]
    np.testing.assert_allclose(out, ref, rtol=1e-11, atol=1e-10)


def test_p5_generated_workload_has_coarse_fill_property():
    apr = S.make_config("blob64", use_cache=False)
    S.validate_apr(apr)
    o = Oracle(apr)
    assert o.check_coarse_fill(2) == 0


# ------------------------------------------------------------------------------------------ P6
@pytest.mark.parametrize("k,bc,C,Cout", [(3, 0, 1, 1), (5, 0, 1, 1), (3, 1, 1, 1), (3, 0, 2, 3)])
def test_p6_backward_is_transpose(k, bc, C, Cout):
    apr = S.random_balanced_apr((8, 8, 8), 1, seed=11, p_fine=0.02)
    N, L = apr.n_particles, apr.n_levels
    assert 20 < N < 400
    rng = np.random.default_rng(5)
    W = rng.normal(size=(L, Cout, C, k ** 3))
    o = Oracle(apr, np.zeros((N, C)))
    # dense matrix of the forward map, one unit input at a time
    A = np.zeros((N * Cout, N * C))
    for j in range(N * C):
        x = np.zeros(N * C)
        x[j] = 1.0
        o.set_values(x.reshape(N, C))
        A[:, j] = o.conv(W, k, bc=bc, C_out=Cout).reshape(-1)
    G = rng.normal(size=(N, Cout))
    xv = rng.normal(size=(N, C))
    o.set_values(xv)
    gp, gw = o.conv_backward(W, k, G, bc=bc, C_out=Cout)
    np.testing.assert_allclose(gp.reshape(-1), A.T @ G.reshape(-1), rtol=1e-12, atol=1e-12)
    # weight gradient: the map is linear in W; differentiate one unit stencil entry at a time
    gw_ref = np.zeros_like(W)
    for idx in np.ndindex(*W.shape):
        E = np.zeros_like(W)
        E[idx] = 1.0
        gw_ref[idx] = np.sum(o.conv(E, k, bc=bc, C_out=Cout) * G)
    np.testing.assert_allclose(gw, gw_ref, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------------------------------ P7, P9
def _golden_restrict():
    rows = []
    for line in (GOLD / "restrict_1d.txt").read_text().splitlines():
        if not line.strip() or line.startswith("#"):
            continue
        head, fine, coarse = line.split("|")
        k, s = map(int, head.split())
        rows.append((k, s, np.array(fine.split(), float), np.array(coarse.split(), float)))
    return rows


@pytest.mark.parametrize("case", range(4))
def test_p9_restriction_golden(case):
    k, s, fine, coarse = _golden_restrict()[case]
    w = fine[:, None, None] * fine[None, :, None] * fine[None, None, :]
    lmax = int(np.log2(s))
    wl = restrict_stencil(w, lmax, 0)[0]
    ref = coarse[:, None, None] * coarse[None, :, None] * coarse[None, None, :]
    np.testing.assert_allclose(wl, ref, rtol=0, atol=1e-15)


def test_p9_restriction_identity_and_sum():
    rng = np.random.default_rng(9)
    for k in (3, 5):
        w = rng.normal(size=(k, k, k))
        st = restrict_stencil(w, 6, 0)
        np.testing.assert_allclose(st[-1], w, atol=1e-15)
        np.testing.assert_allclose(st.reshape(7, -1).sum(1), w.sum(), rtol=1e-12)
        r = k // 2
        for l in range(6):  # support of w_l within +-1 for s >= 2 (Eq. restrict_stenc, r <= 2)
            m = np.zeros((k, k, k), bool)
            m[r - 1:r + 2, r - 1:r + 2, r - 1:r + 2] = True
            assert np.all(st[l][~m] == 0.0)


def test_p7_flip_commutes_with_restriction():
    rng = np.random.default_rng(2)
    w = rng.normal(size=(5, 5, 5))
    a = restrict_stencil(w[::-1, ::-1, ::-1], 5, 0)
    b = restrict_stencil(w, 5, 0)[:, ::-1, ::-1, ::-1]
    np.testing.assert_allclose(a, b, atol=1e-14)


# ------------------------------------------------------------------------------------------ golden tree
def _tiny_case(case):
    if case == "A":
        ps = [(2, a, b, c, 1 + 4 * a + 2 * b + c) for a in range(2) for b in range(2) for c in range(2)]
        cells = [(z, x, y) for z in range(2) for x in range(2) for y in range(2) if (z, x, y) != (0, 0, 0)]
        ps += [(1, z, x, y, 10.0 * (1 + i)) for i, (z, x, y) in enumerate(cells)]
        return S.apr_from_particles((4, 4, 4), 1, ps)
    ps = [(2, 2, b, c, 2.0 * (1 + 2 * b + c)) for b in range(2) for c in range(2)]
    cells = [(z, x, y) for z in range(2) for x in range(2) for y in range(2) if (z, x, y) != (1, 0, 0)]
    ps += [(1, z, x, y, 10.0 * (1 + i)) for i, (z, x, y) in enumerate(cells)]
    return S.apr_from_particles((3, 4, 4), 1, ps)


@pytest.mark.parametrize("case", ["A", "B"])
def test_golden_tree_tiny(case):
    gold = {}
    for line in (GOLD / "tree_tiny.txt").read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            c, rest = line.split("|")
            l, z, x, y, v = rest.split()
            gold[c.strip()] = ((int(l), int(z), int(x), int(y)), float(v))
    apr = _tiny_case(case)
    S.validate_apr(apr)
    o = Oracle(apr)
    (coords, v) = gold[case]
    tc = o.tree_coords()
    assert tc.shape[0] == 1 and tuple(tc[0]) == coords
    assert o.tree()[0, 0] == v


def test_invalid_layouts_are_detected():
    apr = _tiny_case("A")
    # drop one fine particle: a hole in the partition
    ps = [(2, a, b, c, 1.0) for a in range(2) for b in range(2) for c in range(2)][:-1]
    ps += [(1, z, x, y, 1.0) for z in range(2) for x in range(2) for y in range(2) if (z, x, y) != (0, 0, 0)]
    hole = S.apr_from_particles((4, 4, 4), 1, ps)
    with pytest.raises(ValueError):
        Oracle(hole).tree()
    # a particle that is also an ancestor of other particles (overlap)
    ps2 = [(2, a, b, c, 1.0) for a in range(2) for b in range(2) for c in range(2)]
    ps2 += [(1, z, x, y, 1.0) for z in range(2) for x in range(2) for y in range(2)]
    assert Oracle(S.apr_from_particles((4, 4, 4), 1, ps2)).error != 0
    assert Oracle(apr).error == 0


# ------------------------------------------------------------------------------------------ bf16
def test_bf16_rounding_matches_torch():
    import torch
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-6, 6, size=2000),
                        [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, -(1.0 + 2 ** -9), 0.0, 255.5, 256.5]])
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([oracle.round_bf16(x) for x in v])
    np.testing.assert_array_equal(got, ref)


def test_bf16_tree_is_rounded_average_level_by_level():
    apr = S.random_balanced_apr((16, 16, 16), 1, seed=6)
    rng = np.random.default_rng(1)
    vals = rng.integers(-64, 65, size=(apr.n_particles, 3)) / 8.0
    o = Oracle(apr, vals)
    t = o.tree_bf16()
    # every value is a bfloat16, and the finest-level nodes are the rounded exact averages
    assert all(oracle.round_bf16(x) == x for x in t.ravel())
    tc = o.tree_coords()
    exact = Oracle(apr, vals).tree()
    fin = tc[:, 0] == apr.l_max - 1
    np.testing.assert_array_equal(t[fin], np.vectorize(oracle.round_bf16)(exact[fin]))


# ---- Richardson-Lucy (Sec. 6.2)
def test_rl_identity_psf_gives_observed_after_one_iteration():
    apr = S.random_balanced_apr((12, 10, 20), 1, seed=31, p_fine=0.05)
    rng = np.random.default_rng(2)
    u = rng.uniform(1.0, 5.0, apr.n_particles)
    i0 = rng.uniform(0.5, 2.0, apr.n_particles)
    delta = np.zeros((apr.n_levels, 27))
    delta[:, 13] = 1.0
    got = oracle.richardson_lucy(apr, u, delta, 3, 1, estimate=i0)
    np.testing.assert_allclose(got, u, rtol=1e-14)


@pytest.mark.parametrize("bc", [0, 1])
def test_rl_on_pixels_equals_dense_rl(bc):
    from scipy import ndimage
    dims = (7, 9, 11)
    apr = S.uniform_level_apr(dims, S.l_max_for(dims), l_min=2)
    rng = np.random.default_rng(3)
    u = rng.uniform(1.0, 10.0, apr.n_particles)
    w = rng.uniform(0.0, 1.0, (3, 3, 3))          # non-symmetric: a missing flip fails
    w /= w.sum()
    W = np.zeros((apr.n_levels, 27))
    W[:] = w.reshape(-1)
    got = oracle.richardson_lucy(apr, u, W, 3, 3, bc=bc)
    mode = "reflect" if bc == 0 else "constant"
    U = u.reshape(dims)                             # all-finest APR: particle order = z, x, y raster
    I = U.copy()
    for _ in range(3):
        c = ndimage.correlate(I, w, mode=mode, cval=0.0)
        ratio = np.where(c > 0, U / np.where(c > 0, c, 1.0), 0.0)
        I = I * ndimage.correlate(ratio, w[::-1, ::-1, ::-1], mode=mode, cval=0.0)
    np.testing.assert_allclose(got, I.reshape(-1), rtol=1e-12)


def test_rl_constant_image_is_a_fixed_point():
    apr = S.random_balanced_apr((16, 16, 24), 1, seed=32, p_fine=0.03)
    u = np.full(apr.n_particles, 4.5)
    w = S.gaussian_stencil(5, 1.5)
    W = oracle.restrict_stencil(w, apr.l_max, apr.l_min).reshape(apr.n_levels, -1)
    got = oracle.richardson_lucy(apr, u, W, 5, 4)
    np.testing.assert_allclose(got, u, rtol=1e-12)


# ---- gradient magnitude with level-rescaled Sobel stencils (Sec. 4.3, Eq. adapt_grad)
def _sobel():
    d, sm = np.array([-0.5, 0.0, 0.5]), np.array([0.25, 0.5, 0.25])
    return np.stack([np.einsum("i,j,k->ijk", d, sm, sm), np.einsum("i,j,k->ijk", sm, d, sm),
                     np.einsum("i,j,k->ijk", sm, sm, d)])


@pytest.mark.parametrize("level", [None, 3])
def test_gradient_magnitude_of_a_linear_ramp(level):
    """A linear ramp has the same gradient everywhere: at pixels (all-finest APR) the Sobel estimate
    is exact, and on a uniform coarse level the cell means are the ramp at the cell centres, so the
    level-rescaled stencil (w / 2^(l_max - l)) recovers the pixel-unit gradient."""
    dims = (16, 16, 32)
    lmax = S.l_max_for(dims)
    lev = lmax if level is None else level
    apr = S.uniform_level_apr(dims, lev, l_min=min(lev, 2))
    l, z, x, y = apr.particle_coords()
    s = 1 << (lmax - lev)
    alpha, beta, gamma = 0.7, -1.3, 0.4
    # cell means of f = alpha*Z + beta*X + gamma*Y over the pixels of each cell (centres)
    cz, cx, cy = (z + 0.5) * s - 0.5, (x + 0.5) * s - 0.5, (y + 0.5) * s - 0.5
    vals = 5.0 + alpha * cz + beta * cx + gamma * cy
    sob = _sobel().reshape(3, -1)
    W = np.stack([np.stack([sob[a] * 2.0 ** -(lmax - lv) for lv in range(apr.l_min, apr.l_max + 1)]) for a in range(3)])
    got = oracle.gradient_magnitude(apr, vals, W, 3)
    dz, dx, dy = apr.level_dims(lev)
    inner = (z >= 1) & (z < dz - 1) & (x >= 1) & (x < dx - 1) & (y >= 1) & (y < dy - 1)
    np.testing.assert_allclose(got[inner], np.sqrt(alpha ** 2 + beta ** 2 + gamma ** 2), rtol=1e-12)
    if level is not None:   # without the rescaling the coarse estimate is s times too large
        W1 = np.stack([np.repeat(sob[a][None], apr.n_levels, 0) for a in range(3)])
        g1 = oracle.gradient_magnitude(apr, vals, W1, 3)
        np.testing.assert_allclose(g1[inner], s * np.sqrt(alpha ** 2 + beta ** 2 + gamma ** 2), rtol=1e-12)


def test_multichannel_conv_on_pixels_equals_channel_sum_of_dense_correlations():
    """With 16 channels on an all-finest APR, out[co] = sum_ci correlate(x[ci], W[co][ci]) (reflect)."""
    dims = (6, 7, 9)
    apr = S.uniform_level_apr(dims, S.l_max_for(dims), l_min=2)
    rng = np.random.default_rng(11)
    C = 16
    x = rng.normal(size=(apr.n_particles, C))
    W = rng.normal(size=(apr.n_levels, C, C, 27))
    got = Oracle(apr, x).conv(W, 3, C_out=C)
    lev = apr.l_max - apr.l_min
    X = x.reshape(dims + (C,))
    for co in range(0, C, 5):
        ref = sum(ndi.correlate(X[..., ci], W[lev, co, ci].reshape(3, 3, 3), mode="reflect") for ci in range(C))
        np.testing.assert_allclose(got[:, co], ref.reshape(-1), rtol=1e-10, atol=1e-10)
