"""A 5^3 convolution or data adjoint over the whole work list runs the levels below l_max split by
radius (radius-1 tiles in their own launch on the library's second stream, beside the l_max tiles;
the tiles of lower levels with outer taps in a persistent radius-2 launch), or as one launch when the
last call's stack had outer taps below l_max; apr_convolve_auto starts the l_max launch beside the
tree restriction (those tiles read no tree node). Whichever launches a call takes, every tile is
computed by the same code: the results equal, bit for bit, the single launch over all work items
(apr_convolve_tiles / apr_convolve_adjoint_tiles), also when consecutive calls switch between
restricted, plain and mixed stacks without waiting (so the choice rests on an older call), and
inside a captured CUDA graph."""
import numpy as np
import pytest
import torch

import aprsynth as S
import paper_2112_03592_gb300 as G

pytestmark = pytest.mark.gpu

FLAGS = G.APR_VALIDATE | G.APR_REQUIRE_BALANCE


def stacks(apr):
    w = S.gaussian_stencil(5, 1.5).astype(np.float32)
    L = apr.n_levels
    restricted = G.apr_restrict_stencil(w, apr.l_max, apr.l_min)
    plain = np.repeat(w.reshape(1, -1), L, 0)
    mixed = restricted.copy().reshape(L, 5, 5, 5)
    mixed[L // 2, 0, 4, 2] = 0.25        # one level below l_max with a single outer tap
    return {"restricted": restricted, "plain": plain, "mixed": mixed.reshape(L, -1)}


def reference(lay, vals, tree, st, gout, bc, n_fwd, n_bwd):
    """The single launch over all work items (the radius-2 kernel, radius-1 tiles inside)."""
    out = torch.zeros_like(vals)
    G.apr_convolve_tiles(lay, vals, tree, st, 5, 0, n_fwd, bc, out=out)
    gp = torch.zeros_like(vals)
    gt = torch.zeros(lay.n_tree, device=vals.device)
    G.apr_convolve_adjoint_tiles(lay, st, 5, gout, gp, gt, 0, n_bwd, bc)
    return out, gp, gt


@pytest.mark.parametrize("bc", [G.APR_BC_REFLECT, G.APR_BC_ZERO])
def test_split_equals_single_launch_across_stack_switches(bc):
    apr = S.random_balanced_apr((48, 40, 150), 2, seed=41, p_fine=0.03)
    assert apr.l_max - apr.l_min >= 3
    lay = G.AprLayout.from_apr(apr, FLAGS)
    n_fwd = len(lay.export(G._abi.APR_STRUCT_FWD_ITEMS))
    n_bwd = len(lay.export(G._abi.APR_STRUCT_BWD_ITEMS))
    rng = np.random.default_rng(7)
    dev = torch.device("cuda")
    vals = torch.as_tensor(rng.normal(size=apr.n_particles).astype(np.float32) + 2, device=dev)
    gout = torch.as_tensor(rng.normal(size=apr.n_particles).astype(np.float32), device=dev)
    tree = G.apr_tree_restrict(lay, vals)
    sts = {name: torch.as_tensor(s, device=dev) for name, s in stacks(apr).items()}
    refs = {name: reference(lay, vals, tree, st, gout, bc, n_fwd, n_bwd) for name, st in sts.items()}
    torch.cuda.synchronize()
    order = ["restricted", "plain", "plain", "restricted", "mixed", "restricted", "mixed", "plain"]
    got = []
    for name in order:      # no synchronisation in between: each choice rests on an earlier call
        out = G.apr_convolve(lay, vals, tree, sts[name], 5, bc)
        gp = torch.empty_like(vals)
        gt = torch.empty(lay.n_tree, device=dev)
        G.apr_convolve_adjoint(lay, sts[name], 5, gout, bc, grad_particles=gp, grad_tree=gt)
        tree2 = torch.full_like(tree, float("nan"))
        auto = G.apr_convolve_auto(lay, vals, sts[name], 5, bc, workspace=tree2)
        got.append((name, out, gp, gt, auto, tree2))
    torch.cuda.synchronize()
    lay.sync_status()
    for name, out, gp, gt, auto, tree2 in got:
        r_out, r_gp, r_gt = refs[name]
        assert torch.equal(out, r_out), name
        assert torch.equal(gp, r_gp), name
        assert torch.equal(gt, r_gt), name
        assert torch.equal(auto, r_out), name
        assert torch.equal(tree2, tree), name
    # captured after each kind of stack, replayed with each stack's values copied in
    st_buf = torch.empty_like(sts["restricted"])
    for first in ["restricted", "plain"]:
        st_buf.copy_(sts[first])
        G.apr_convolve(lay, vals, tree, st_buf, 5, bc)
        torch.cuda.synchronize()
        out = torch.empty_like(vals)
        gp = torch.empty_like(vals)
        gt = torch.empty(lay.n_tree, device=dev)
        g = torch.cuda.CUDAGraph()
        out2 = torch.empty_like(vals)
        tree2 = torch.empty_like(tree)
        with torch.cuda.graph(g):
            G.apr_convolve(lay, vals, tree, st_buf, 5, bc, out=out)
            G.apr_convolve_adjoint(lay, st_buf, 5, gout, bc, grad_particles=gp, grad_tree=gt)
            G.apr_convolve_auto(lay, vals, st_buf, 5, bc, out=out2, workspace=tree2)
        for name in ["restricted", "mixed", "plain"]:
            st_buf.copy_(sts[name])
            out.fill_(float("nan"))
            out2.fill_(float("nan"))
            tree2.fill_(float("nan"))
            g.replay()
            torch.cuda.synchronize()
            r_out, r_gp, r_gt = refs[name]
            assert torch.equal(out, r_out) and torch.equal(gp, r_gp) and torch.equal(gt, r_gt), (first, name)
            assert torch.equal(out2, r_out) and torch.equal(tree2, tree), (first, name)
    lay.sync_status()


def test_richardson_lucy_split_equals_across_stack_switches():
    """apr_richardson_lucy with a restricted PSF takes the split launches; with a plain one the single
    launch: both equal the same iteration run through apr_convolve_tiles."""
    apr = S.random_balanced_apr((40, 32, 96), 2, seed=43, p_fine=0.03)
    lay = G.AprLayout.from_apr(apr, FLAGS)
    dev = torch.device("cuda")
    u = torch.as_tensor(apr.values.astype(np.float32), device=dev)
    for name in ["restricted", "plain", "restricted"]:
        st = torch.as_tensor(stacks(apr)[name], device=dev)
        est = G.apr_richardson_lucy(lay, u, st, 5, 2)
        torch.cuda.synchronize()
        # the same two iterations through the tile-range entry point (single launch)
        n_fwd = len(lay.export(G._abi.APR_STRUCT_FWD_ITEMS))
        stf = torch.flip(st.reshape(-1, 5, 5, 5), dims=(1, 2, 3)).reshape(st.shape).contiguous()
        ref = u.clone()
        for _ in range(2):
            tree = G.apr_tree_restrict(lay, ref)
            conv = torch.zeros_like(u)
            G.apr_convolve_tiles(lay, ref, tree, st, 5, 0, n_fwd, out=conv)
            ratio = torch.where(conv > 0, u / conv, torch.zeros_like(u))
            tree = G.apr_tree_restrict(lay, ratio)
            back = torch.zeros_like(u)
            G.apr_convolve_tiles(lay, ratio, tree, stf, 5, 0, n_fwd, out=back)
            ref = ref * back
        torch.cuda.synchronize()
        np.testing.assert_allclose(est.cpu().numpy(), ref.cpu().numpy(), rtol=2e-6, atol=0)
    lay.sync_status()
