"""z-slab sharding with halo exchange, run as gloo ranks on host processes (no GPU).

Each rank convolves its sub-APR with the oracle standing in for the CUDA kernels; the stitched
owned outputs, the transposed (backward) results and the all-reduced stencil gradient must equal
the whole-volume oracle. The exchange, the plan and the stitching are the product code under test.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import aprsynth as S
import oracle
from paper_2112_03592_gb300.slab import SlabConv, SlabPlan

CASES = {
    "rand": lambda: S.random_balanced_apr((40, 24, 30), 3, seed=21, p_fine=0.02),
    "rand_odd": lambda: S.random_balanced_apr((37, 9, 70), 4, seed=22, p_fine=0.03),
}


def _stencils(apr, k, seed=0):
    return np.random.default_rng(seed).normal(size=(apr.n_levels, k ** 3))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, case, k, bc, outdir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        apr = CASES[case]()
        W = _stencils(apr, k)
        rng = np.random.default_rng(5)
        vals = rng.normal(size=apr.n_particles) + 3.0
        gout = rng.normal(size=apr.n_particles)

        def fwd(sub, v):
            return torch.as_tensor(oracle.Oracle(sub, v.numpy()).conv(W, k, bc)[:, 0])

        def bwd(sub, v, g):
            gp, gw = oracle.Oracle(sub, v.numpy()).conv_backward(W, k, g.numpy(), bc)
            return torch.as_tensor(gp[:, 0]), torch.as_tensor(gw.reshape(apr.n_levels, -1))

        sc = SlabConv(apr, rank, world, k, bc=bc, compute=fwd, compute_backward=bwd)
        own = sc.plan.owned_positions_global(rank)
        v_own = torch.as_tensor(vals[own])
        out = sc.forward(v_own)
        gp, gw = sc.backward(v_own, torch.as_tensor(gout[own]))
        np.savez(os.path.join(outdir, f"r{rank}.npz"), own=own, out=out.numpy(), gp=gp.numpy(), gw=gw.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("k,bc", [(3, 0), (5, 0), (5, 1)])
@pytest.mark.parametrize("case", list(CASES))
def test_slab_sharded_conv_matches_whole_volume(case, k, bc, world, tmp_path):
    mp.spawn(_worker, args=(world, _free_port(), case, k, bc, str(tmp_path)), nprocs=world, join=True)
    apr = CASES[case]()
    W = _stencils(apr, k)
    rng = np.random.default_rng(5)
    vals = rng.normal(size=apr.n_particles) + 3.0
    gout = rng.normal(size=apr.n_particles)
    o = oracle.Oracle(apr, vals)
    ref = o.conv(W, k, bc)[:, 0]
    ref_gp, ref_gw = o.conv_backward(W, k, gout, bc)
    out = np.full(apr.n_particles, np.nan)
    gp = np.full(apr.n_particles, np.nan)
    seen = np.zeros(apr.n_particles, int)
    for r in range(world):
        z = np.load(tmp_path / f"r{r}.npz")
        out[z["own"]] = z["out"]
        gp[z["own"]] = z["gp"]
        seen[z["own"]] += 1
        np.testing.assert_allclose(z["gw"], ref_gw.reshape(apr.n_levels, -1), rtol=1e-11, atol=1e-11)
    assert np.all(seen == 1), "every particle is owned by exactly one rank"
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(gp, ref_gp[:, 0], rtol=1e-11, atol=1e-11)


def test_slab_plan_partitions_and_aligns():
    apr = CASES["rand_odd"]()
    for world in (1, 2, 3, 4):
        p = SlabPlan(apr, world, 2)
        A = 1 << (apr.l_max - apr.l_min)
        assert p.bounds[0][0] == 0 and p.bounds[-1][1] == apr.dims[0]
        for (a, b), (c, d) in zip(p.bounds, p.bounds[1:]):
            assert b == c and b % A == 0
        owned = np.concatenate([p.owned_positions_global(i) for i in range(world)])
        assert np.array_equal(np.sort(owned), np.arange(apr.n_particles))
        for i in range(world):
            # the owned particles sit inside the rank's sub-APR at the listed local positions
            loc = p.own_local_positions(i)
            assert loc.size == p.n_owned(i) and len(set(loc.tolist())) == loc.size
            assert np.array_equal(p.sub[i].y_idx[loc], np.asarray(apr.y_idx)[p.owned_positions_global(i)])
    with pytest.raises(ValueError):
        SlabPlan(apr, 100, 1)
