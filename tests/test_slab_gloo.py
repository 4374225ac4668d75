"""z-slab sharding with per-level halos, run as gloo ranks on host processes (no GPU).

Each rank's local work is the oracle standing in for the CUDA kernels (the whole-APR index, the
particle values the plan gives the rank, the all-reduced tree); the stitched owned outputs, the
transposed (backward) results and the all-reduced stencil gradient must equal the whole-volume
oracle. The plan, the exchange, the all-reduces and the stitching are the product code under test.
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
    # the shape of the 1024x1024x512 workload's level structure: l_max 10, l_min 3, 512 z rows
    "c2_shaped": lambda: S.random_balanced_apr((512, 8, 1024), 3, seed=23, p_fine=0.0005),
}


def _stencils(apr, k, seed=0):
    return np.random.default_rng(seed).normal(size=(apr.n_levels, k ** 3))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleLocal:
    """A rank's local work done by the FP64 oracle on the whole-APR index."""

    def __init__(self, apr, W, k, bc):
        self.apr, self.W, self.k, self.bc = apr, W, k, bc

    def _o(self, v, tree=None):
        o = oracle.Oracle(self.apr, v.numpy())
        if tree is not None:
            o.set_tree(tree.numpy())
        return o

    def restrict(self, v):
        return torch.as_tensor(self._o(v).tree()[:, 0].copy())

    def convolve(self, v, tree, owned):
        out = np.zeros(self.apr.n_particles)
        out[owned] = self._o(v, tree).conv(self.W, self.k, self.bc, sample=owned)[:, 0]
        return torch.as_tensor(out)

    def adjoint(self, v, tree, g, owned):
        gp, gt, gw = self._o(v, tree).conv_backward_parts(self.W, self.k, g.numpy(), self.bc, sample=owned)
        return (torch.as_tensor(gp[:, 0].copy()), torch.as_tensor(gt[:, 0].copy()),
                torch.as_tensor(gw.reshape(self.apr.n_levels, -1)))

    def tree_transpose(self, gt):
        return torch.as_tensor(oracle.Oracle(self.apr).tree_transpose(gt.numpy())[:, 0].copy())


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
        sc = SlabConv(apr, rank, world, k, bc=bc, local=OracleLocal(apr, W, k, bc))
        own = sc.own
        v_own = torch.as_tensor(vals[own])
        out = sc.forward(v_own)
        gp, gw = sc.backward(v_own, torch.as_tensor(gout[own]))
        np.savez(os.path.join(outdir, f"r{rank}.npz"), own=own, out=out.numpy(), gp=gp.numpy(), gw=gw.numpy(),
                 held=sc.plan.held_fraction(rank))
    finally:
        dist.destroy_process_group()


def _check(case, k, bc, world, tmp_path):
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
    held = []
    for r in range(world):
        z = np.load(tmp_path / f"r{r}.npz")
        out[z["own"]] = z["out"]
        gp[z["own"]] = z["gp"]
        seen[z["own"]] += 1
        held.append(float(z["held"]))
        np.testing.assert_allclose(z["gw"], ref_gw.reshape(apr.n_levels, -1), rtol=1e-11, atol=1e-11 * np.abs(ref_gw).max())
    assert np.all(seen == 1), "every particle is owned by exactly one rank"
    np.testing.assert_allclose(out, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())
    np.testing.assert_allclose(gp, ref_gp[:, 0], rtol=1e-11, atol=1e-11 * np.abs(ref_gp).max())
    return held


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("k,bc", [(3, 0), (5, 0), (5, 1)])
@pytest.mark.parametrize("case", ["rand", "rand_odd"])
def test_slab_sharded_conv_matches_whole_volume(case, k, bc, world, tmp_path):
    mp.spawn(_worker, args=(world, _free_port(), case, k, bc, str(tmp_path)), nprocs=world, join=True)
    _check(case, k, bc, world, tmp_path)


@pytest.mark.parametrize("world", [2, 4, 8])
def test_slab_c2_shaped_scales_to_8_ranks(world, tmp_path):
    """l_min 3, l_max 10, 512 z rows: 2, 4 and 8 ranks each hold little more than 1/world of the
    particles, and the stitched results equal the whole-volume oracle."""
    mp.spawn(_worker, args=(world, _free_port(), "c2_shaped", 5, 0, str(tmp_path)), nprocs=world, join=True)
    held = _check("c2_shaped", 5, 0, world, tmp_path)
    assert max(held) <= 1.0 / world + 0.15, held


def test_slab_plan_partitions_and_aligns():
    for case in ("rand_odd", "c2_shaped"):
        apr = CASES[case]()
        for world in (1, 2, 3, 4, 8):
            p = SlabPlan(apr, world, 2)
            assert p.bounds[0][0] == 0 and p.bounds[-1][1] == apr.dims[0]
            for (a, b), (c, d) in zip(p.bounds, p.bounds[1:]):
                assert b == c and b % p.B == 0
            owned = np.concatenate([p.owned[i] for i in range(world)])
            assert np.array_equal(np.sort(owned), np.arange(apr.n_particles))
            for i in range(world):
                assert np.all(np.isin(p.owned[i], p.needed[i]))
                for lv in p.levels:  # a sharded level's cells lie inside one slab
                    if lv["sharded"]:
                        assert p.B % lv["s"] == 0
    apr = CASES["c2_shaped"]()
    p = SlabPlan(apr, 8, [1] * (apr.n_levels - 1) + [2])
    assert p.B == 64 and not p.levels[0]["sharded"] and all(lv["sharded"] for lv in p.levels[1:])
    with pytest.raises(ValueError):
        SlabPlan(apr, 1000, 1)
