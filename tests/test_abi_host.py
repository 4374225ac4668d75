"""C-ABI library on the host (no GPU): symbols, index structure, stencil helpers, invalid layouts."""
import ctypes
import pathlib
import re

import numpy as np
import pytest

import aprsynth as S
import oracle
import paper_2112_03592_gb300 as G
from paper_2112_03592_gb300 import _abi

HEADER = pathlib.Path(__file__).resolve().parents[1] / "include" / "apr.h"
HOST = G.APR_VALIDATE | G.APR_REQUIRE_BALANCE | G.APR_HOST_ONLY


def declared_functions():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(apr_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = _abi.load()
    names = declared_functions()
    assert len(names) >= 15, names
    for n in names:
        assert hasattr(lib, n), f"{n} missing from {_abi.lib_path()}"
        assert n in _abi.SIGNATURES, f"{n} not bound in the Python binding"


def test_status_strings():
    lib = _abi.load()
    for code in range(8):
        assert lib.apr_status_string(code)


def _check_structure(apr):
    lay = G.AprLayout.from_apr(apr, flags=HOST)
    o = oracle.Oracle(apr)
    assert o.error == 0
    assert lay.n_tree == o.n_tree
    rp, ty = o.tree_layout()
    assert np.array_equal(lay.export(_abi.APR_STRUCT_ROW_PTR), apr.row_ptr.astype(np.uint32))
    assert np.array_equal(lay.export(_abi.APR_STRUCT_Y_IDX), apr.y_idx.astype(np.uint16))
    assert np.array_equal(lay.export(_abi.APR_STRUCT_TREE_ROW_PTR), rp.astype(np.uint32))
    assert np.array_equal(lay.export(_abi.APR_STRUCT_TREE_Y_IDX), ty.astype(np.uint16))
    # work list: exactly the (level, tile, y-block) bricks holding particles
    lev, z, x, y = apr.particle_coords()
    T, B = _abi.APR_TILE_ZX, _abi.APR_BLOCK_Y
    ref = sorted(set(zip(lev.tolist(), (z // T).tolist(), (x // T).tolist(), (y // B).tolist())))
    got = [tuple(r) for r in lay.export(_abi.APR_STRUCT_FWD_ITEMS).tolist()]
    assert got == ref
    tc = o.tree_coords()
    tref = sorted(set(zip(tc[:, 0].tolist(), tc[:, 1].tolist(), tc[:, 2].tolist(), (tc[:, 3] // B).tolist())))
    assert [tuple(r) for r in lay.export(_abi.APR_STRUCT_TREE_ITEMS).tolist()] == tref
    # data-adjoint work list: the tiles with a cell within Chebyshev distance 2 of a particle of their
    # level (the cells a 5^3 window around a target reaches), by dense dilation of each level's grid
    from scipy import ndimage
    bref = []
    for l in range(apr.l_min, apr.l_max + 1):
        sel = lev == l
        if not sel.any():
            continue
        dz, dx, dy = apr.level_dims(l)
        grid = np.zeros((dz, dx, dy), bool)
        grid[z[sel], x[sel], y[sel]] = True
        near = ndimage.binary_dilation(grid, structure=np.ones((5, 5, 5), bool))
        nz, nx, ny = np.nonzero(near)
        bref += sorted(set(zip([l] * nz.size, (nz // T).tolist(), (nx // T).tolist(), (ny // B).tolist())))
    assert [tuple(r) for r in lay.export(_abi.APR_STRUCT_BWD_ITEMS).tolist()] == bref


@pytest.mark.parametrize("maker", [
    lambda: S.make_config("blob64", use_cache=False),
    lambda: S.random_balanced_apr((12, 16, 10), 1, seed=1),
    lambda: S.random_balanced_apr((9, 5, 70), 1, seed=2, p_fine=0.01),
    lambda: S.random_balanced_apr((3, 1, 130), 0, seed=3),
    lambda: S.uniform_level_apr((16, 8, 8), 4),
    lambda: S.uniform_level_apr((16, 8, 8), 2, l_min=1),
])
def test_structure_bit_exact_vs_oracle(maker):
    _check_structure(maker())


def test_restrict_and_rescale_stencils_vs_oracle():
    rng = np.random.default_rng(0)
    for k in (3, 5):
        w = rng.uniform(-1, 1, size=(k, k, k)).astype(np.float32)
        a = G.apr_restrict_stencil(w, 9, 2)
        b = oracle.restrict_stencil(w.astype(np.float64), 9, 2).reshape(a.shape)
        np.testing.assert_allclose(a, b, rtol=0, atol=2e-7 * np.abs(b).max())
        c = G.apr_rescale_stencil(w, 9, 2)
        np.testing.assert_array_equal(c, (w.reshape(1, -1) * (2.0 ** -(9 - np.arange(2, 10)))[:, None]).astype(np.float32))
    with pytest.raises(G.AprError):
        G.apr_restrict_stencil(np.ones((7, 7, 7), np.float32), 5, 1)


def test_restricted_5cubed_stencils_have_3cubed_support_below_l_max():
    """Eq. restrict_stenc with cell edge s >= 2 maps a 5^3 stencil to support 2 ceil(2/s) + 1 = 3 per
    axis: the library's restricted stack is exactly zero outside the central 3^3 on every level below
    l_max (the condition under which the convolution kernels apply radius-1 tiles), and so is the
    oracle's independent construction; at l_max the stencil is unchanged and its outer taps are not
    zero."""
    rng = np.random.default_rng(3)
    w = rng.uniform(0.1, 1.0, size=(5, 5, 5)).astype(np.float32)
    l_max, l_min = 10, 3
    a = G.apr_restrict_stencil(w, l_max, l_min).reshape(-1, 5, 5, 5)
    b = oracle.restrict_stencil(w.astype(np.float64), l_max, l_min).reshape(-1, 5, 5, 5)
    shell = np.ones((5, 5, 5), bool)
    shell[1:4, 1:4, 1:4] = False
    for i, l in enumerate(range(l_min, l_max + 1)):
        if l < l_max:
            assert np.all(a[i][shell] == 0.0) and np.all(b[i][shell] == 0.0), l
            assert np.all(a[i][~shell] != 0.0)
        else:
            np.testing.assert_array_equal(a[i], w)
            assert np.all(a[i][shell] != 0.0)


# ---------------------------------------------------------------------------- invalid layouts
def _layout(apr, **kw):
    d = dict(dims=apr.dims, l_min=apr.l_min, l_max=apr.l_max, row_ptr=apr.row_ptr.copy(), y_idx=apr.y_idx.copy())
    d.update(kw)
    return d


def _build(d, flags=HOST):
    return G.AprLayout(d["dims"], d["l_min"], d["l_max"], d["row_ptr"], d["y_idx"], flags)


def _expect(code, d, flags=HOST):
    with pytest.raises(G.AprError) as e:
        _build(d, flags)
    assert e.value.code == code


def test_invalid_layouts_rejected():
    apr = S.random_balanced_apr((8, 8, 8), 1, seed=5)
    _build(_layout(apr))  # the valid one builds
    rp = apr.row_ptr.copy()
    rp[3] = rp[4] + 1  # not monotone
    _expect(2, _layout(apr, row_ptr=rp))
    rp = apr.row_ptr.copy()
    rp[-1] -= 1  # does not end at n_particles
    _expect(2, _layout(apr, row_ptr=rp))
    y = apr.y_idx.copy()
    big = int(np.argmax(np.diff(apr.row_ptr)))
    b = int(apr.row_ptr[big])
    y[b], y[b + 1] = y[b + 1], y[b]  # unsorted y
    _expect(2, _layout(apr, y_idx=y))
    y = apr.y_idx.copy()
    y[-1] = 1000  # outside the grid
    _expect(2, _layout(apr, y_idx=y))
    _expect(2, _layout(apr, l_max=apr.l_max + 1))
    _expect(1, _layout(apr, dims=(0, 8, 8)))


def _tiny(ps, dims=(4, 4, 4), l_min=1):
    return S.apr_from_particles(dims, l_min, ps)


def test_partition_and_balance_violations_rejected():
    full8 = [(2, a, b, c, 1.0) for a in range(2) for b in range(2) for c in range(2)]
    others = [(1, z, x, y, 1.0) for z in range(2) for x in range(2) for y in range(2) if (z, x, y) != (0, 0, 0)]
    ok = _tiny(full8 + others)
    _build(_layout(ok))
    hole = _tiny(full8[:-1] + others)                       # a missing cell
    _expect(2, _layout(hole))
    _build(_layout(hole), flags=G.APR_HOST_ONLY)            # without APR_VALIDATE it is not checked
    overlap = _tiny(full8 + others + [(1, 0, 0, 0, 1.0)])   # a particle over finer particles
    _expect(2, _layout(overlap))
    # unbalanced: level-3 particles touching a level-1 particle (8x8x8 image)
    ps = [(1, z, x, y, 1.0) for z in range(2) for x in range(2) for y in range(2) if (z, x, y) != (0, 0, 0)]
    ps += [(2, z, x, y, 1.0) for z in range(2) for x in range(2) for y in range(2) if (z, x, y) != (1, 1, 1)]
    ps += [(3, z, x, y, 1.0) for z in range(2, 4) for x in range(2, 4) for y in range(2, 4)]
    unb = S.apr_from_particles((8, 8, 8), 1, ps)
    S.validate_apr(unb, check_balance=False)
    _build(_layout(unb), flags=G.APR_VALIDATE | G.APR_HOST_ONLY)     # a valid partition ...
    _expect(2, _layout(unb), flags=HOST)                             # ... but not 2:1 balanced


def test_compute_calls_reject_bad_arguments_without_a_device():
    """Argument checks run before any launch: host-only handles, null buffers, unsupported sizes and
    flags return their status codes on a machine without a GPU."""
    import ctypes
    apr = S.random_balanced_apr((8, 8, 16), 0, seed=1, p_fine=0.05)
    lay = G.AprLayout.from_apr(apr, G.APR_VALIDATE | G.APR_REQUIRE_BALANCE | G.APR_HOST_ONLY)
    lib, h = lay._lib, lay.handle
    P = ctypes.c_void_p
    dummy = P(16)
    inv = 1  # APR_ERR_INVALID_ARG
    assert lib.apr_convolve(h, dummy, dummy, dummy, 3, 0, dummy, P(0)) == inv          # host-only handle
    assert lib.apr_gradient_magnitude(h, dummy, dummy, dummy, 3, 0, dummy, P(0)) == inv
    assert lib.apr_convolve_auto(h, dummy, dummy, 3, 0, dummy, dummy, 1 << 20, P(0)) == inv
    assert lib.apr_convolve_auto_workspace_bytes(h) == 4 * max(lay.n_tree, 1)
    assert lib.apr_convolve_mc_relu_bf16(h, dummy, dummy, dummy, 16, 16, 3, 0, dummy, P(0)) == inv
    assert lib.apr_richardson_lucy(h, dummy, dummy, 3, 0, 2, dummy, dummy, 1 << 20, P(0)) == inv
    assert lib.apr_convolve_mc(h, dummy, dummy, dummy, 16, 16, 3, 0, dummy, P(0)) == inv
    assert lib.apr_tree_restrict_bf16(h, dummy, dummy, 16, P(0)) == inv
    assert lib.apr_selftest_bounded_wait(h, 1000, P(0)) == inv
    assert lib.apr_mc_relu_bf16(P(0), 10, dummy, P(0)) == inv                           # null input
    assert lib.apr_mc_embed_bf16(dummy, -1, ctypes.c_float(1.0), dummy, P(0)) == inv   # negative size
    assert lib.apr_mc_readout(P(0), dummy, 4, ctypes.c_float(1.0), dummy, P(0)) == inv
    assert lib.apr_mc_backward_workspace_bytes(h, 8, 16, 3) == 0                        # unsupported shape
    assert lib.apr_restrict_stencil(dummy, 7, 9, 2, dummy) == 3                          # k = 7 unsupported
    bad = _abi.AprHostLayout()
    out = P()
    assert lib.apr_build_device(ctypes.byref(bad), 1 << 7, P(0), ctypes.byref(out)) == inv  # unknown flag


def test_sobel_stencils_helper():
    """apr_sobel_stencils: derivative (-1/2, 0, 1/2) along one axis, smoothing (1/4, 1/2, 1/4) across
    (Sec. 4.3); a linear ramp of slope 1 along the axis correlates to 1, the other axes to 0."""
    import numpy as np
    sob = G.sobel_stencils(3)
    d, sm = np.array([-0.5, 0.0, 0.5]), np.array([0.25, 0.5, 0.25])
    ref = np.stack([np.einsum("i,j,k->ijk", d, sm, sm), np.einsum("i,j,k->ijk", sm, d, sm),
                    np.einsum("i,j,k->ijk", sm, sm, d)]).astype(np.float32)
    np.testing.assert_array_equal(sob, ref)
    g = np.meshgrid(np.arange(3.0), np.arange(3.0), np.arange(3.0), indexing="ij")
    for a in range(3):
        for b in range(3):
            assert abs(float(np.sum(sob[a] * g[b])) - (1.0 if a == b else 0.0)) < 1e-6
    lib = _abi.load()
    assert lib.apr_sobel_stencils(3, None) == 1   # APR_ERR_INVALID_ARG
    out = np.zeros(3 * 125, np.float32)
    assert lib.apr_sobel_stencils(5, out.ctypes.data_as(ctypes.c_void_p)) == 3   # APR_ERR_UNSUPPORTED


def test_build_device_ex_rejects_incomplete_allocator():
    apr = S.random_balanced_apr((8, 8, 8), 1, seed=1)
    lib = _abi.load()
    L = _abi.AprHostLayout()
    rp = np.ascontiguousarray(apr.row_ptr.astype(np.int64))
    yi = np.ascontiguousarray(apr.y_idx.astype(np.int32))
    L.l_min, L.l_max = apr.l_min, apr.l_max
    for a in range(3):
        L.dims[a] = apr.dims[a]
    L.row_ptr, L.y_idx, L.n_particles = rp.ctypes.data_as(ctypes.c_void_p), yi.ctypes.data_as(ctypes.c_void_p), apr.n_particles
    al = _abi.AprAllocator()  # both callbacks NULL
    h = ctypes.c_void_p()
    assert lib.apr_build_device_ex(ctypes.byref(L), 0, None, ctypes.byref(al), ctypes.byref(h)) == 1  # INVALID_ARG
    assert not h.value
