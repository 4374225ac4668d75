"""The local work of z-slab shards on the GPU (CudaLocal: tile-range convolution and adjoint on the
whole-APR layout), the exchange and all-reduces emulated on one GPU: the stitched outputs and
gradients of all ranks equal the whole-volume oracle (the collectives themselves run as gloo ranks
in test_slab_gloo.py)."""
import numpy as np
import pytest
import torch

import aprsynth as S
import oracle
from paper_2112_03592_gb300.slab import CudaLocal, SlabPlan

pytestmark = pytest.mark.gpu

CASES = {
    "rand": lambda: S.random_balanced_apr((40, 24, 30), 3, seed=21, p_fine=0.02),
    "c2_shaped": lambda: S.random_balanced_apr((512, 8, 1024), 3, seed=23, p_fine=0.0005),
}


@pytest.mark.parametrize("case,world", [("rand", 3), ("c2_shaped", 8)])
@pytest.mark.parametrize("k,bc", [(3, 0), (5, 0), (5, 1)])
def test_slab_local_gpu_matches_whole_volume(case, world, k, bc):
    apr = CASES[case]()
    rng = np.random.default_rng(5)
    vals = rng.normal(size=apr.n_particles) + 3.0
    gout = rng.normal(size=apr.n_particles)
    W = rng.normal(size=(apr.n_levels, k ** 3))
    o = oracle.Oracle(apr, vals)
    ref = o.conv(W, k, bc)[:, 0]
    ref_gp, ref_gw = o.conv_backward(W, k, gout, bc)
    plan = SlabPlan(apr, world, k // 2)
    st = torch.as_tensor(W.astype(np.float32), device="cuda")
    v_all = torch.as_tensor(vals.astype(np.float32), device="cuda")
    g_all = torch.as_tensor(gout.astype(np.float32), device="cuda")
    locs = [CudaLocal(apr, plan, r, st, k, bc) for r in range(world)]
    # the tree: the sum over ranks of each rank's restriction of its own particles (the all-reduce)
    tree = None
    for r, loc in enumerate(locs):
        mine = torch.zeros_like(v_all)
        ix = torch.as_tensor(plan.owned[r], device="cuda")
        mine[ix] = v_all[ix]
        t = loc.restrict(mine)
        tree = t if tree is None else tree + t
    out = np.full(apr.n_particles, np.nan)
    gp = np.zeros(apr.n_particles)
    gt_sum = torch.zeros(tree.numel(), device="cuda")
    gw_sum = np.zeros((apr.n_levels, k ** 3))
    for r, loc in enumerate(locs):
        need = torch.as_tensor(plan.needed[r], device="cuda")
        v = torch.zeros_like(v_all)
        v[need] = v_all[need]                          # the rank's values after the exchange
        own = plan.owned[r]
        out[own] = loc.convolve(v, tree, own).cpu().numpy()[own]
        g = torch.zeros_like(g_all)
        ixo = torch.as_tensor(own, device="cuda")
        g[ixo] = g_all[ixo]
        p, t, w = loc.adjoint(v, tree, g, own)
        gp += p.double().cpu().numpy()                 # direct shares, added back to their owners
        gt_sum += t
        gw_sum += w.double().cpu().numpy().reshape(apr.n_levels, -1)
    torch.cuda.synchronize()
    for r, loc in enumerate(locs):
        own = plan.owned[r]
        gp[own] += loc.tree_transpose(gt_sum).double().cpu().numpy()[own]
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-5 * np.abs(ref).max())
    np.testing.assert_allclose(gp, ref_gp[:, 0], rtol=0, atol=1e-5 * np.abs(ref_gp).max())
    np.testing.assert_allclose(gw_sum, ref_gw.reshape(apr.n_levels, -1), rtol=0, atol=1e-5 * np.abs(ref_gw).max())
