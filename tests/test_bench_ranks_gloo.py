"""The multi-rank reporting of bench.py (replicas: barrier, slowest rank's time, whole-job value)
as gloo ranks on host processes."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        dist.barrier()
        t = bench.max_over_ranks(1.0 + 0.5 * rank)   # rank-dependent step time
        np.save(os.path.join(outdir, f"r{rank}.npy"), np.array([t]))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = [float(np.load(tmp_path / f"r{r}.npy")[0]) for r in range(world)]
    assert got == [1.5, 1.5]


def test_max_over_ranks_single_process():
    import bench
    assert bench.max_over_ranks(2.5) == 2.5
