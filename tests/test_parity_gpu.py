"""CUDA path vs the FP64 oracle, element by element, through the C ABI (needs a GB300)."""
import numpy as np
import pytest
import torch

import aprsynth as S
import oracle
import paper_2112_03592_gb300 as G
from paper_2112_03592_gb300 import _abi

pytestmark = pytest.mark.gpu
FLAGS = G.APR_VALIDATE | G.APR_REQUIRE_BALANCE
REL = 1e-5    # FP32 vs FP64: max relative error (positive data)
NORM = 1e-5   # sign-mixed data: max |diff| / max |reference|


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def stencil_stack(apr, k, mode, seed=0):
    L = apr.n_levels
    if mode == "gauss":
        w = S.gaussian_stencil(k, 1.0 if k == 3 else 1.5).astype(np.float32)
        return np.repeat(w.reshape(1, -1), L, 0)
    if mode == "restricted":
        w = S.gaussian_stencil(k, 1.0 if k == 3 else 1.5).astype(np.float32)
        return G.apr_restrict_stencil(w, apr.l_max, apr.l_min)
    rng = np.random.default_rng(seed)
    st = rng.normal(size=(L, k ** 3)).astype(np.float32)
    if mode == "mixed_shell" and k == 5:
        # even level indices: zero outside the central 3^3 (computed with radius 1); level 1: zero
        # outside the core except one corner tap (radius 2); the rest: all taps
        w = st.reshape(L, 5, 5, 5)
        for i in range(L):
            if i % 2 == 0 or i == 1:
                core = w[i, 1:4, 1:4, 1:4].copy()
                w[i] = 0.0
                w[i, 1:4, 1:4, 1:4] = core
        if L > 1:
            w[1, 0, 0, 0] = 0.5
    return st


def gpu_forward(apr, st, k, bc):
    lay = G.AprLayout.from_apr(apr, FLAGS)
    v = dev(apr.values.astype(np.float32))
    tree = G.apr_tree_restrict(lay, v)
    out = G.apr_convolve(lay, v, tree, dev(st), k, bc)
    torch.cuda.synchronize()
    lay.sync_status()
    return lay, v, tree, out


def assert_rel(got, ref, tol=REL):
    ref = np.asarray(ref, np.float64)
    got = np.asarray(got, np.float64)
    assert np.all(np.isfinite(got)), "non-finite GPU outputs"
    err = np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-30))
    assert err <= tol, f"max relative error {err:.3e} > {tol}"


def assert_norm(got, ref, tol=NORM):
    ref = np.asarray(ref, np.float64)
    got = np.asarray(got, np.float64)
    assert np.all(np.isfinite(got)), "non-finite GPU outputs"
    err = np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-30)
    assert err <= tol, f"normwise error {err:.3e} > {tol}"


CASES = {
    "blob64": lambda: S.make_config("blob64", use_cache=False),
    "rand_ragged": lambda: S.random_balanced_apr((21, 13, 150), 1, seed=7, p_fine=0.01),
    "rand_thin": lambda: S.random_balanced_apr((3, 40, 9), 0, seed=8, p_fine=0.05),
    "all_max": lambda: S.uniform_level_apr((9, 17, 70), 7, l_min=2),
    "uniform_coarse": lambda: S.uniform_level_apr((32, 32, 32), 3, l_min=3),
    "tiny": lambda: S.random_balanced_apr((2, 3, 5), 0, seed=9, p_fine=0.3),
    "single": lambda: S.uniform_level_apr((1, 1, 1), 0, l_min=0),
    "row": lambda: S.random_balanced_apr((1, 1, 200), 0, seed=13, p_fine=0.05),
    "plane": lambda: S.random_balanced_apr((1, 37, 90), 1, seed=14, p_fine=0.03),
    # level grids 2 cells wide along z and x: with reflection a coarse particle has up to 4 x 4 x 3
    # pre-images (two of them here reach more than 32), and the 5^3 mirror lists take the d < 2R path
    "thin_2x2": lambda: S.random_balanced_apr((2, 2, 40), 0, seed=22, p_fine=0.3),
}


@pytest.mark.parametrize("case", list(CASES))
def test_tree_restrict_matches_oracle(case):
    apr = CASES[case]()
    lay = G.AprLayout.from_apr(apr, FLAGS)
    v = dev(apr.values.astype(np.float32))
    tree = G.apr_tree_restrict(lay, v).cpu().numpy()
    ref = oracle.Oracle(apr).tree()[:, 0]
    assert tree.shape == ref.shape
    if ref.size:
        assert_rel(tree, ref)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("k", [3, 5])
@pytest.mark.parametrize("bc", [G.APR_BC_REFLECT, G.APR_BC_ZERO])
@pytest.mark.parametrize("mode", ["gauss", "restricted", "random", "mixed_shell"])
def test_convolve_matches_oracle(case, k, bc, mode):
    apr = CASES[case]()
    st = stencil_stack(apr, k, mode, seed=k + 10 * bc)
    _, _, _, out = gpu_forward(apr, st, k, bc)
    ref = oracle.Oracle(apr).conv(st.astype(np.float64), k, bc=bc)[:, 0]
    got = out.cpu().numpy()
    if mode in ("random", "mixed_shell") or bc == G.APR_BC_ZERO:
        assert_norm(got, ref)
    else:
        assert_rel(got, ref)


@pytest.mark.parametrize("k", [3, 5])
def test_single_particle_closed_form(k):
    # a 1-cell grid reflects every neighbour onto the cell itself: out = v * sum(w); zero boundary
    # keeps only the centre tap
    apr = CASES["single"]()
    w = np.random.default_rng(k).normal(size=(1, k ** 3)).astype(np.float32)
    v = float(apr.values[0])
    for bc, ref in ((G.APR_BC_REFLECT, v * float(w.astype(np.float64).sum())),
                    (G.APR_BC_ZERO, v * float(w[0, k ** 3 // 2]))):
        _, _, _, out = gpu_forward(apr, w, k, bc)
        assert abs(float(out.cpu()[0]) - ref) <= 1e-5 * max(abs(ref), 1e-30) + 1e-6 * abs(v) * float(np.abs(w).sum())


def test_constant_image_stays_constant():
    apr = S.random_balanced_apr((24, 20, 130), 1, seed=4, values="const")
    for k in (3, 5):
        st = stencil_stack(apr, k, "restricted")
        _, _, tree, out = gpu_forward(apr, st, k, G.APR_BC_REFLECT)
        assert_rel(tree.cpu().numpy(), np.full(tree.numel(), 7.25))
        assert_rel(out.cpu().numpy(), np.full(out.numel(), 7.25))


@pytest.mark.parametrize("case", ["blob64", "rand_ragged", "rand_thin", "tiny", "single", "row", "plane"])
@pytest.mark.parametrize("k", [3, 5])
@pytest.mark.parametrize("bc", [G.APR_BC_REFLECT, G.APR_BC_ZERO])
@pytest.mark.parametrize("mode", ["random", "restricted", "mixed_shell"])
def test_backward_matches_oracle(case, k, bc, mode):
    apr = CASES[case]()
    st = stencil_stack(apr, k, mode, seed=3)
    lay, v, tree, _ = gpu_forward(apr, st, k, bc)
    g = np.random.default_rng(1).normal(size=apr.n_particles).astype(np.float32)
    gp, gw = G.apr_convolve_backward(lay, v, tree, dev(st), k, dev(g), bc)
    torch.cuda.synchronize()
    rp, rw = oracle.Oracle(apr).conv_backward(st.astype(np.float64), k, g.astype(np.float64), bc=bc)
    assert_norm(gp.cpu().numpy(), rp[:, 0])
    assert_norm(gw.cpu().numpy(), rw.reshape(gw.shape))


def test_backward_is_deterministic():
    apr = CASES["blob64"]()
    st = stencil_stack(apr, 5, "random")
    lay, v, tree, _ = gpu_forward(apr, st, 5, 0)
    g = dev(np.random.default_rng(2).normal(size=apr.n_particles).astype(np.float32))
    a = [t.clone() for t in G.apr_convolve_backward(lay, v, tree, dev(st), 5, g, 0)]
    b = G.apr_convolve_backward(lay, v, tree, dev(st), 5, g, 0)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_autograd_function_and_finite_differences():
    apr = S.random_balanced_apr((10, 12, 20), 1, seed=12, p_fine=0.02)
    lay = G.AprLayout.from_apr(apr, FLAGS)
    k = 3
    st = torch.tensor(stencil_stack(apr, k, "random", seed=5), device="cuda", requires_grad=True)
    v = torch.tensor(apr.values, device="cuda", requires_grad=True)
    out = G.AprConv.apply(v, st, lay, k)
    gsel = torch.randn(out.shape, device="cuda")
    (out * gsel).sum().backward()
    # the map is bilinear in (values, stencils): central differences in float64 via the oracle are exact
    o = oracle.Oracle(apr)
    W = st.detach().cpu().double().numpy()
    x0 = apr.values.astype(np.float64)
    G_ = gsel.cpu().double().numpy()
    rng = np.random.default_rng(0)
    for j in rng.choice(apr.n_particles, 5, replace=False):
        e = np.zeros_like(x0)
        e[j] = 1.0
        o.set_values(x0 + e)
        fp = np.sum(o.conv(W, k)[:, 0] * G_)
        o.set_values(x0 - e)
        fm = np.sum(o.conv(W, k)[:, 0] * G_)
        fd = (fp - fm) / 2.0
        assert abs(v.grad[j].item() - fd) <= 1e-4 * max(1.0, abs(fd))
    o.set_values(x0)
    _, rw = o.conv_backward(W, k, G_)
    assert_norm(st.grad.cpu().numpy(), rw.reshape(st.shape))


def test_structure_on_device_is_bit_exact():
    apr = CASES["blob64"]()
    lay = G.AprLayout.from_apr(apr, FLAGS)
    o = oracle.Oracle(apr)
    rp, ty = o.tree_layout()
    assert np.array_equal(lay.export(_abi.APR_STRUCT_ROW_PTR), apr.row_ptr.astype(np.uint32))
    assert np.array_equal(lay.export(_abi.APR_STRUCT_Y_IDX), apr.y_idx.astype(np.uint16))
    assert np.array_equal(lay.export(_abi.APR_STRUCT_TREE_ROW_PTR), rp.astype(np.uint32))
    assert np.array_equal(lay.export(_abi.APR_STRUCT_TREE_Y_IDX), ty.astype(np.uint16))
    # the tree kernels' child maps on the device equal the host-built ones (pinned on the CPU)
    host = G.AprLayout.from_apr(apr, FLAGS | G.APR_HOST_ONLY)
    assert np.array_equal(lay.export(_abi.APR_STRUCT_TREE_NODE_MAP), host.export(_abi.APR_STRUCT_TREE_NODE_MAP))


def test_misaligned_caller_allocation_is_refused():
    """A caller allocator whose blocks are off the 16-byte grid the kernels' vector loads need: the
    build fails with APR_ERR_CUDA, hands every block back, and the library keeps working."""
    import ctypes
    apr = S.make_config("blob64", use_cache=False)
    lib = _abi.load()
    held = {}

    def alloc(nbytes, stream, ctx):
        p = int(torch.cuda.caching_allocator_alloc(int(nbytes) + 16, torch.cuda.current_device(),
                                                   stream if stream else 0))
        held[p + 4] = p
        return p + 4

    def free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(held.pop(int(ptr)))

    fa, ff = _abi.ALLOC_FN(alloc), _abi.FREE_FN(free)
    al = _abi.AprAllocator(fa, ff, None)
    rp = np.ascontiguousarray(apr.row_ptr.astype(np.int64))
    yi = np.ascontiguousarray(apr.y_idx.astype(np.int32))
    L = _abi.AprHostLayout()
    L.l_min, L.l_max = apr.l_min, apr.l_max
    for a in range(3):
        L.dims[a] = int(apr.dims[a])
    L.row_ptr = rp.ctypes.data_as(ctypes.c_void_p)
    L.y_idx = yi.ctypes.data_as(ctypes.c_void_p)
    L.n_particles = int(yi.size)
    h = ctypes.c_void_p()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.apr_build_device_ex(ctypes.byref(L), FLAGS, stream, ctypes.byref(al), ctypes.byref(h))
    torch.cuda.synchronize()
    assert rc == _abi.APR_ERR_CUDA and not h.value and not held
    lay = G.AprLayout.from_apr(apr, FLAGS, allocator="torch")
    assert lay.layout_bytes() > 0


def test_backward_parts_compose_to_backward():
    apr = CASES["rand_ragged"]()
    st = stencil_stack(apr, 5, "random", seed=8)
    lay, v, tree, _ = gpu_forward(apr, st, 5, G.APR_BC_REFLECT)
    g = dev(np.random.default_rng(3).normal(size=apr.n_particles).astype(np.float32))
    ref_p, ref_w = G.apr_convolve_backward(lay, v, tree, dev(st), 5, g)
    gp, gt = G.apr_convolve_adjoint(lay, dev(st), 5, g)
    G.apr_tree_restrict_adjoint(lay, gt, gp)
    gw = G.apr_convolve_stencil_grad(lay, v, tree, 5, g)
    torch.cuda.synchronize()
    assert torch.equal(gp, ref_p) and torch.equal(gw, ref_w)


def test_convolve_adjoint_dot_product():
    # <A x, y> == <x, A^T y> for the convolution alone (tree values as an independent input)
    apr = CASES["blob64"]()
    lay = G.AprLayout.from_apr(apr, FLAGS)
    rng = np.random.default_rng(7)
    st = dev(rng.normal(size=(apr.n_levels, 27)).astype(np.float32))
    x = rng.normal(size=apr.n_particles)
    t = rng.normal(size=lay.n_tree)
    y = rng.normal(size=apr.n_particles)
    out = G.apr_convolve(lay, dev(x.astype(np.float32)), dev(t.astype(np.float32)), st, 3)
    gp, gt = G.apr_convolve_adjoint(lay, st, 3, dev(y.astype(np.float32)))
    torch.cuda.synchronize()
    lhs = float(np.dot(out.cpu().double().numpy(), y))
    rhs = float(np.dot(x, gp.cpu().double().numpy()) + np.dot(t, gt.cpu().double().numpy()))
    assert abs(lhs - rhs) <= 1e-5 * max(1.0, abs(lhs)), (lhs, rhs)


@pytest.mark.parametrize("C", [2, 5])
def test_tree_restrict_multichannel_fp32(C):
    apr = CASES["rand_ragged"]()
    lay = G.AprLayout.from_apr(apr, FLAGS)
    vals = np.random.default_rng(C).uniform(1.0, 9.0, size=(apr.n_particles, C))
    tree = G.apr_tree_restrict(lay, dev(vals.astype(np.float32))).cpu().numpy()
    ref = oracle.Oracle(apr, vals.astype(np.float32)).tree()
    assert tree.shape == ref.shape
    assert_rel(tree, ref)


@pytest.mark.parametrize("bc", [G.APR_BC_REFLECT, G.APR_BC_ZERO])
def test_convolve_auto_equals_restrict_then_convolve(bc):
    apr = CASES["rand_ragged"]()
    st = dev(stencil_stack(apr, 5, "restricted"))
    lay, v, tree, out = gpu_forward(apr, st.cpu().numpy(), 5, bc)
    auto = G.apr_convolve_auto(lay, v, st, 5, bc)
    torch.cuda.synchronize()
    assert torch.equal(auto, out)
    small = torch.empty(max(lay.n_tree * 4 - 4, 0), dtype=torch.uint8, device="cuda")
    if lay.n_tree > 0:
        with pytest.raises(RuntimeError):
            G.apr_convolve_auto(lay, v, st, 5, bc, workspace=small)


def test_index_in_torch_caching_allocator_gives_identical_results():
    """apr_build_device_ex with callbacks into torch's caching allocator: the handle's index lives in
    torch memory (torch counts it), results are bit-identical to the library's stream-ordered
    allocation, and apr_destroy gives the memory back."""
    apr = S.make_config("blob64", use_cache=False)
    st = dev(stencil_stack(apr, 5, "restricted"))
    v = dev(apr.values.astype(np.float32))
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    lay_t = G.AprLayout.from_apr(apr, FLAGS, allocator="torch")
    torch.cuda.synchronize()
    grown = torch.cuda.memory_allocated() - before
    assert grown >= lay_t.layout_bytes() > 0
    lay_c = G.AprLayout.from_apr(apr, FLAGS)
    outs = []
    for lay in (lay_t, lay_c):
        tree = G.apr_tree_restrict(lay, v)
        out = G.apr_convolve(lay, v, tree, st, 5)
        gp, gw = G.apr_convolve_backward(lay, v, tree, st, 5, out)
        torch.cuda.synchronize()
        lay.sync_status()
        outs.append((tree, out, gp, gw))
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    nbytes = lay_t.layout_bytes()
    held = torch.cuda.memory_allocated()
    lay_t.close()
    torch.cuda.synchronize()
    assert held - torch.cuda.memory_allocated() >= nbytes
