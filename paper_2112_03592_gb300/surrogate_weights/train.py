"""Trains the APR CNN surrogate of 20 Richardson-Lucy iterations and writes its weights here.

Training set: seeded 256^3 blob images (400 blobs, sigma 2-12 px, Poisson noise) turned into APRs,
seeds 1000 .. 1000 + n - 1, each mapped to its 20-iteration Richardson-Lucy output (restricted 5^3
Gaussian PSF sigma 1.5 and its flip, Sec. 6.2) computed on the GPU with apr_richardson_lucy. The
model and the loss are those of paper_2112_03592_gb300.surrogate (Adam on FP32 master weights).

    python -m paper_2112_03592_gb300.surrogate_weights.train [--n 200] [--steps 3000] [--out FILE]

Needs a CUDA device. The APRs are generated in parallel processes (spawned before any GPU use).
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
DEFAULT_OUT = os.path.join(HERE, "rl20_blob256.npz")
SEED0 = 1000


def _make(seed):
    sys.path.insert(0, ROOT)
    import aprsynth as S
    return S.make_config("blob256", seed=seed)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=200, help="training APRs")
    ap.add_argument("--steps", type=int, default=3000, help="Adam steps")
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--workers", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--out", default=DEFAULT_OUT)
    a = ap.parse_args(argv)

    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(a.workers) as pool:
        aprs = pool.map(_make, [SEED0 + i for i in range(a.n)])
    t_gen = time.perf_counter() - t0

    import numpy as np
    import torch
    sys.path.insert(0, ROOT)
    import aprsynth as S
    import paper_2112_03592_gb300 as G
    from paper_2112_03592_gb300.surrogate import AprCnn, train

    dev = torch.device("cuda")
    w = S.gaussian_stencil(5, 1.5).astype(np.float32)
    flags = G.APR_VALIDATE | G.APR_REQUIRE_BALANCE
    t0 = time.perf_counter()
    samples = []
    for apr in aprs:
        lay = G.AprLayout.from_apr(apr, flags)
        x = torch.as_tensor(apr.values, device=dev)
        st = torch.as_tensor(G.apr_restrict_stencil(w, apr.l_max, apr.l_min), device=dev)
        t = G.apr_richardson_lucy(lay, x, st, 5, 20)
        samples.append((lay, x, t, float(1.0 / float(x.mean()))))
    torch.cuda.synchronize()
    t_rl = time.perf_counter() - t0
    model = AprCnn(4, n_dist=8, seed=0)
    t0 = time.perf_counter()
    hist = train(model, samples, a.steps, lr=a.lr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    np.savez(a.out, **{f"layer{i}": wl.float().cpu().numpy() for i, wl in enumerate(model.W)},
             n_train=a.n, seed0=SEED0, steps=a.steps, lr=a.lr,
             loss_first=float(np.mean(hist[:20])), loss_last=float(np.mean(hist[-20:])))
    print(f"trained on {a.n} APRs ({sum(x.n_particles for x in aprs)} particles): generation {t_gen:.1f} s, "
          f"RL20 targets {t_rl:.1f} s, {a.steps} steps {t_train:.1f} s; loss {np.mean(hist[:20]):.5f} -> "
          f"{np.mean(hist[-20:]):.5f}; wrote {a.out}")


if __name__ == "__main__":
    main()
