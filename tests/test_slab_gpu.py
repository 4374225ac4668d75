"""The local work of a z-slab shard on the GPU: each rank's sub-APR (built with APR_SUBDOMAIN) fed
with the whole image's values of its region gives the whole-volume oracle's outputs and gradients
for the particles it owns."""
import numpy as np
import pytest
import torch

import aprsynth as S
import oracle
from paper_2112_03592_gb300.slab import SlabConv

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k,bc", [(3, 0), (5, 0), (5, 1)])
def test_slab_local_gpu_matches_whole_volume(k, bc):
    apr = S.random_balanced_apr((40, 24, 30), 3, seed=21, p_fine=0.02)
    rng = np.random.default_rng(5)
    vals = rng.normal(size=apr.n_particles) + 3.0
    gout = rng.normal(size=apr.n_particles)
    W = rng.normal(size=(apr.n_levels, k ** 3))
    o = oracle.Oracle(apr, vals)
    ref = o.conv(W, k, bc)[:, 0]
    ref_gp, ref_gw = o.conv_backward(W, k, gout, bc)
    world = 3
    gw_sum = np.zeros((apr.n_levels, k ** 3))
    gp = np.zeros(apr.n_particles)
    for rank in range(world):
        sc = SlabConv(apr, rank, world, k, stencils=torch.as_tensor(W.astype(np.float32), device="cuda"), bc=bc)
        loc = np.concatenate([np.arange(a, b) for a, b in sc.plan.local[rank]])
        own = sc.plan.owned_positions_global(rank)
        lv = torch.as_tensor(vals[loc].astype(np.float32), device="cuda")
        out = sc._local_forward(lv).cpu().numpy()[sc.own_loc]
        np.testing.assert_allclose(out, ref[own], rtol=1e-5, atol=1e-5 * np.abs(ref).max())
        # backward of the owned outputs only; halo shares added back by global position
        g = np.zeros(sc.sub.n_particles, np.float32)
        g[sc.own_loc] = gout[own]
        gl, gw = sc._local_backward(lv, torch.as_tensor(g, device="cuda"))
        np.add.at(gp, loc, gl.cpu().numpy().astype(np.float64))
        gw_sum += gw.cpu().numpy().reshape(apr.n_levels, -1)
    scale = np.abs(ref_gp).max()
    np.testing.assert_allclose(gp, ref_gp[:, 0], rtol=0, atol=1e-5 * scale)
    np.testing.assert_allclose(gw_sum, ref_gw.reshape(apr.n_levels, -1), rtol=0, atol=1e-5 * np.abs(ref_gw).max())
