"""apr_convolve_backward runs the stencil gradient on the library's second stream while the data and
tree adjoints run on the caller's: captured into a CUDA graph (fork / join through events) and
replayed, and called eagerly on a side stream, it gives bit for bit the results of the three parts
called one after the other on one stream."""
import numpy as np
import pytest
import torch

import aprsynth as S
import paper_2112_03592_gb300 as G

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k", [3, 5])
def test_concurrent_backward_equals_sequential_parts(k):
    apr = S.random_balanced_apr((40, 24, 130), 3, seed=31, p_fine=0.03)
    lay = G.AprLayout.from_apr(apr, G.APR_VALIDATE | G.APR_REQUIRE_BALANCE)
    rng = np.random.default_rng(k)
    dev = torch.device("cuda")
    vals = torch.as_tensor(rng.normal(size=apr.n_particles).astype(np.float32) + 2, device=dev)
    gout = torch.as_tensor(rng.normal(size=apr.n_particles).astype(np.float32), device=dev)
    st = torch.as_tensor(rng.normal(size=(apr.n_levels, k ** 3)).astype(np.float32), device=dev)
    tree = G.apr_tree_restrict(lay, vals)
    # the parts, one after the other
    gp_ref = torch.empty_like(vals)
    gt = torch.empty(lay.n_tree, device=dev)
    G.apr_convolve_adjoint(lay, st, k, gout, G.APR_BC_REFLECT, grad_particles=gp_ref, grad_tree=gt)
    G.apr_tree_restrict_adjoint(lay, gt, gp_ref)
    gw_ref = G.apr_convolve_stencil_grad(lay, vals, tree, k, gout, G.APR_BC_REFLECT)
    torch.cuda.synchronize()
    # eager, on a side stream
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        gp, gw = G.apr_convolve_backward(lay, vals, tree, st, k, gout, G.APR_BC_REFLECT, stream=side)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    assert torch.equal(gp, gp_ref) and torch.equal(gw, gw_ref)
    # captured and replayed
    gp2 = torch.full_like(vals, float("nan"))
    gw2 = torch.full_like(gw_ref, float("nan"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        G.apr_convolve_backward(lay, vals, tree, st, k, gout, G.APR_BC_REFLECT, grad_particles=gp2, grad_stencils=gw2)
    for _ in range(2):
        gp2.fill_(float("nan"))
        gw2.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(gp2, gp_ref) and torch.equal(gw2, gw_ref)
    lay.sync_status()


def test_tree_adjoint_level_by_level():
    """apr_tree_restrict_adjoint_levels called level by level, coarsest first, equals the whole tree
    adjoint bit for bit; after tree level t the particles of level t + 1 already hold their final
    gradient (what a caller copies out early)."""
    apr = S.random_balanced_apr((40, 24, 130), 2, seed=33, p_fine=0.03)
    lay = G.AprLayout.from_apr(apr, G.APR_VALIDATE | G.APR_REQUIRE_BALANCE)
    assert apr.l_max - apr.l_min >= 3
    rng = np.random.default_rng(9)
    dev = torch.device("cuda")
    gout = torch.as_tensor(rng.normal(size=apr.n_particles).astype(np.float32), device=dev)
    st = torch.as_tensor(rng.normal(size=(apr.n_levels, 125)).astype(np.float32), device=dev)
    gp0, gt0 = G.apr_convolve_adjoint(lay, st, 5, gout)
    gp_ref, gt_ref = gp0.clone(), gt0.clone()
    G.apr_tree_restrict_adjoint(lay, gt_ref, gp_ref)
    gp, gt = gp0.clone(), gt0.clone()
    first = [apr.level_row_offset(l) for l in range(apr.l_min, apr.l_max + 2)]
    rp = apr.row_ptr
    for t in range(apr.l_min, apr.l_max):
        G.apr_tree_restrict_adjoint_levels(lay, gt, gp, t, t)
        torch.cuda.synchronize()
        lo, hi = int(rp[first[t + 1 - apr.l_min]]), int(rp[first[t + 2 - apr.l_min]])
        assert torch.equal(gp[lo:hi], gp_ref[lo:hi]), t
    assert torch.equal(gp, gp_ref) and torch.equal(gt, gt_ref)
    with pytest.raises(RuntimeError):
        G.apr_tree_restrict_adjoint_levels(lay, gt, gp, apr.l_max - 1, apr.l_min)
    lay.sync_status()
