#!/usr/bin/env python
"""Benchmark: APR-native convolution hot path on the 1024x1024x512-pixel blob APR (~8M particles).

One step = APR tree restriction (Sec. 3.4) + APR convolution with the per-level restricted 5^3
Gaussian stencils (Sec. 4.1-4.2) + its backward (gradients w.r.t. particle values, through the tree,
and w.r.t. the stencils). The index and the work lists are built once (apr_build_device) and reused,
as the paper allows for repeated convolutions (Sec. 6.1.2). Inputs are synthetic (seeded blob
image, Poisson noise). The data set (~0.1 GB) is smaller than L2, so L2 is flushed (a 512 MB write)
before every timed step, outside the step's own timing events.

Prints one JSON line. --impl reference times the FP64 CPU oracle on a bounded sample instead.
Multi-GPU: the path has no exchange step here, so N ranks run N independent replicas (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "blob1024"
K = 5
SIGMA = 1.5
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except OSError:
        return PEAKS_FALLBACK, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0=None, t1=None):
        """Median SM clock and active throttle reasons over the samples taken in [t0, t1] (all
        samples if none fall inside, e.g. a timed region shorter than the sampling period)."""
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines
        if t0 is not None:
            inside = [x for x in lines if t0 <= x[0] <= t1]
            lines = inside if inside else lines
        for _, ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm),
                "window": "timed region" if t0 is not None and any(t0 <= x[0] <= t1 for x in self.lines)
                else "warm-up and timed region (timed region shorter than the 50 ms sampling period)"}


TRAFFIC_SOURCES = ["paper_2112_03592_gb300/csrc/apr_kernels.cu", "paper_2112_03592_gb300/csrc/apr_device.cuh",
                   "paper_2112_03592_gb300/csrc/apr_tile.cuh", "paper_2112_03592_gb300/csrc/apr_plan.cu"]


MC_TRAFFIC_SOURCES = ["paper_2112_03592_gb300/csrc/apr_mc.cu", "paper_2112_03592_gb300/csrc/apr_device.cuh",
                      "paper_2112_03592_gb300/csrc/apr_plan.cu"]


def kernel_source_hash(sources=None):
    """sha1 prefix of the sources the single-channel (or the given) kernels are built from."""
    import hashlib
    h = hashlib.sha1()
    for rel in sources or TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def recorded_traffic(call, section=None):
    """DRAM bytes of one call of `call` (the sum over its launches) from the committed ncu summary,
    if the kernel sources are unchanged since that capture (sha1 prefix match); else None.
    section "mc": the multi-channel record (its own sources and hash)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)
        if section:
            rec = rec[section]
        sha = kernel_source_hash(MC_TRAFFIC_SOURCES if section == "mc" else None)
    except (OSError, KeyError, ValueError):
        return None
    if sha != rec.get("sha1_prefix"):
        return None
    return rec.get("dram_bytes_per_call", {}).get(call)


def conv_launches(apr, st_h, k):
    """Kernels of one apr_convolve (or apr_convolve_adjoint) call on the whole work list: for k = 5
    with levels below l_max, three when no such level has taps outside the central 3^3 (radius-1
    launch, persistent radius-2 launch, l_max launch), else two (one launch over all tiles and the
    hint kernel beside it); otherwise one."""
    import numpy as np
    if k != 5 or apr.l_max == apr.l_min:
        return 1
    w = np.asarray(st_h, np.float32).reshape(apr.n_levels, 5, 5, 5)[:-1]
    outer = w.copy()
    outer[:, 1:4, 1:4, 1:4] = 0
    return 2 if np.any(outer != 0) else 3


def make_replayers(fns, use_graph):
    """The step's parts as CUDA graphs (one graph per part, replayed on the current stream), so the
    timed region has no host launch gaps; the plain callables when use_graph is false. Each part
    has run eagerly before (allocations, kernel attributes)."""
    if not use_graph:
        return list(fns)
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for f in fns:
            f()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    out = []
    for f in fns:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            f()
        out.append(g.replay)
    torch.cuda.synchronize()
    return out


def max_over_ranks(x: float, device=None) -> float:
    """Max of a per-rank float over the process group (the step time every rank reports is the
    slowest rank's); identity without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def algorithmic_bytes(apr, lay, k):
    """Bytes the method must move (no index overhead, no re-reads):
    conv forward  = N_p (4 in + 2 y + 4 out) + N_t (4 + 2) + (R_p + R_t) 4 + stencils
    tree restrict = N_p (4 + 2) + N_t (4 write + 2) + (R_p + R_t) 4   (tree read-back of finer levels ~ N_t 4)
    """
    Np, Nt = apr.n_particles, lay.n_tree
    Rp = int(apr.row_ptr.size - 1)
    Rt = sum(apr.level_dims(l)[0] * apr.level_dims(l)[1] for l in range(apr.l_min, apr.l_max))
    st = apr.n_levels * k ** 3 * 4
    conv = Np * 10 + Nt * 6 + (Rp + Rt) * 4 + st
    restrict = Np * 6 + Nt * 10 + (Rp + Rt) * 4
    return conv, restrict


def dense_pixel_conv(dims, w, steps, flush, stream):
    """Time a dense FP32 k^3 correlation of a pixel image of `dims` (cuDNN through torch conv3d,
    TF32 disabled, zero padding); returns ms and pixel-equivalent GB/s, or None if it does not fit."""
    import torch
    import torch.nn.functional as F
    prev = torch.backends.cudnn.allow_tf32
    torch.backends.cudnn.allow_tf32 = False
    try:
        img = torch.rand((1, 1) + tuple(int(d) for d in dims), device=stream.device)
        ker = torch.as_tensor(w, device=stream.device).reshape((1, 1) + w.shape)
        pad = w.shape[0] // 2
        out = F.conv3d(img, ker, padding=pad)
        ts = []
        for _ in range(max(3, steps)):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            out = F.conv3d(img, ker, padding=pad)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        ms = statistics.median(ts[1:])
        nbytes = float(img.numel()) * 4
        del out
        # the hand-written dense stencil (2.5-D blocked, apr_dense_convolve), same image, reflect
        import paper_2112_03592_gb300 as G
        img3 = img.reshape(img.shape[2:])
        ker1 = ker.reshape(-1).contiguous()
        out3 = G.apr_dense_convolve(img3, ker1, w.shape[0])
        th = []
        for _ in range(max(3, steps)):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            G.apr_dense_convolve(img3, ker1, w.shape[0], out=out3)
            b.record(stream)
            b.synchronize()
            th.append(a.elapsed_time(b))
        ms_h = statistics.median(th[1:])
        del img, img3, out3
        torch.cuda.empty_cache()
        return {"ms": round(ms, 4), "pixel_GBps": round(nbytes / (ms * 1e-3) / 1e9, 2),
                "library": "cuDNN via torch.nn.functional.conv3d, FP32 (TF32 off), zero padding",
                "hand_written": {"ms": round(ms_h, 4), "pixel_GBps": round(nbytes / (ms_h * 1e-3) / 1e9, 2),
                                 "kernel": "dense_conv_kernel (apr_dense_convolve), FP32, 2.5-D blocked, reflect",
                                 "hbm_frac_read_write": round(2 * nbytes / (ms_h * 1e-3) / 1e9 / float(_peaks()[0]["hbm_gbs"]), 4)},
                "note": "context for the pixel-equivalent metric; not part of the APR path"}
    except RuntimeError as e:
        return {"unavailable": str(e).splitlines()[0][:200]}
    finally:
        torch.backends.cudnn.allow_tf32 = prev


def layer_step(args, lay, st, b, dev, stream, flush, world, clocks=False):
    """Times the layer step with stencil stack st on the buffers b: tree restriction and convolution
    (apr_convolve_auto, the paper's forward pipeline: the l_max tiles, which read no tree node, run
    beside the restriction) and the backward (apr_convolve_backward: data adjoint and tree adjoint on
    this stream, the stencil gradient concurrently on the library's second stream), device-resident
    (CUDA events around the step, L2 flushed before every step) and end to end from pinned host
    buffers; and, in a separate pass, each of the five parts alone (tree restriction | convolution |
    convolution adjoint | tree adjoint | stencil gradient, one after the other, CUDA events per part)
    and the forward pipeline alone. Returns the per-part times (the pipeline last), the step and e2e
    means (max over ranks), the copy sizes and the clock record."""
    import torch

    import paper_2112_03592_gb300 as G
    vals, gout, tree, out, gp, gw, gtree = (b[k] for k in ("vals", "gout", "tree", "out", "gp", "gw", "gtree"))
    parts_fns = [lambda: G.apr_tree_restrict(lay, vals, tree),
                 lambda: G.apr_convolve(lay, vals, tree, st, K, G.APR_BC_REFLECT, out),
                 lambda: G.apr_convolve_adjoint(lay, st, K, gout, G.APR_BC_REFLECT, grad_particles=gp, grad_tree=gtree),
                 lambda: G.apr_tree_restrict_adjoint(lay, gtree, gp),
                 lambda: G.apr_convolve_stencil_grad(lay, vals, tree, K, gout, G.APR_BC_REFLECT, grad_stencils=gw),
                 lambda: G.apr_convolve_auto(lay, vals, st, K, G.APR_BC_REFLECT, out, workspace=tree)]
    step_fns = [parts_fns[5],
                lambda: G.apr_convolve_backward(lay, vals, tree, st, K, gout, G.APR_BC_REFLECT, grad_particles=gp,
                                                grad_stencils=gw)]
    for f in parts_fns + step_fns[1:]:
        f()
    run_part = make_replayers(parts_fns, not args.no_graph)
    # the step as one graph (forward pipeline, then the backward)
    run_step = make_replayers([lambda: [f() for f in step_fns]], not args.no_graph)

    def parts_pass(e=None):
        if e is not None:
            e[0].record(stream)
        for j, f in enumerate(run_part):
            f()
            if e is not None:
                e[j + 1].record(stream)

    # each part alone, one after the other
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(args.steps)]
    for _ in range(args.warmup):
        flush.zero_()
        parts_pass()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()
        parts_pass(ev[i])
    torch.cuda.synchronize()
    parts = [[ev[i][j].elapsed_time(ev[i][j + 1]) for i in range(args.steps)] for j in range(6)]

    # the step
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    clk = ClockSampler(dev.index).__enter__() if clocks else None
    for _ in range(args.warmup):
        flush.zero_()
        for f in run_step:
            f()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        evs[i][0].record(stream)
        for f in run_step:
            f()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    clock_rec = None
    if clk is not None:
        time.sleep(0.12)
        clk.__exit__()
        clock_rec = clk.summary(t0, t1)
    if world > 1:
        torch.distributed.barrier()
    lay.sync_status()
    step_ms = max_over_ranks(sum(e[0].elapsed_time(e[1]) for e in evs) / args.steps, dev)

    # end to end through the public API with host buffers: H2D of the step's inputs (values,
    # upstream gradient), the step, D2H of its results (outputs, both gradients). Copies that the
    # kernels do not wait for run on a second stream: dL/dout goes in (after the values, so that they
    # have the host link to themselves) while the tree restriction and the convolution run, the
    # outputs come back while the backward runs, and the particle
    # gradient while the stencil gradient runs (so here the backward's three parts are called one
    # after the other: overlapping that copy saves more than running the stencil gradient beside
    # the adjoints)
    h_vals = vals.cpu().pin_memory()
    h_gout = gout.cpu().pin_memory()
    h_out = torch.empty(out.numel()).pin_memory()
    h_gp = torch.empty(gp.numel()).pin_memory()
    h_gw = torch.empty_like(gw, device="cpu").pin_memory()
    cs = torch.cuda.Stream(device=dev)
    ev_v, ev_g, ev_out, ev_gp, ev_stage = (torch.cuda.Event() for _ in range(5))
    # a streaming input pipeline: the values of step i+1 come in (host to device, into a staging
    # buffer) while step i runs, and each step starts with a device copy of its values from there;
    # every step's timed region still holds one full host-to-device copy of values and dL/dout
    staging = torch.empty_like(vals)
    staging.copy_(h_vals)
    ev_stage.record(stream)
    torch.cuda.synchronize()

    def e2e_step():
        cs.wait_stream(stream)                  # the previous step has finished with gout
        stream.wait_event(ev_stage)             # this step's values have landed in the staging buffer
        vals.copy_(staging, non_blocking=True)
        ev_v.record(stream)
        with torch.cuda.stream(cs):
            cs.wait_event(ev_v)
            gout.copy_(h_gout, non_blocking=True)
            ev_g.record(cs)
            staging.copy_(h_vals, non_blocking=True)  # the next step's values
            ev_stage.record(cs)
        run_part[5]()                           # tree restriction + convolution
        ev_out.record(stream)
        with torch.cuda.stream(cs):
            cs.wait_event(ev_out)
            h_out.copy_(out, non_blocking=True)
        stream.wait_event(ev_g)
        run_part[2]()
        run_part[3]()
        ev_gp.record(stream)
        with torch.cuda.stream(cs):
            cs.wait_event(ev_gp)
            h_gp.copy_(gp, non_blocking=True)
        run_part[4]()
        h_gw.copy_(gw, non_blocking=True)
        stream.wait_stream(cs)                  # the step ends when every copy has landed

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        a, bb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_step()
        bb.record(stream)
        bb.synchronize()
        e2e_ms.append(a.elapsed_time(bb))
    e2e = max_over_ranks(sum(e2e_ms) / len(e2e_ms), dev)
    return {"parts": parts, "step_ms": step_ms, "e2e_ms": e2e, "wall": t1 - t0, "clocks": clock_rec,
            "h2d": int(h_vals.numel() * 4 + h_gout.numel() * 4),
            "d2h": int(h_out.numel() * 4 + h_gp.numel() * 4 + h_gw.numel() * 4)}


def run_ours(args, rank, world):
    import numpy as np
    import torch

    import aprsynth as S
    import paper_2112_03592_gb300 as G

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    apr = S.make_config(WORKLOAD)
    t_build = time.perf_counter()
    lay = G.AprLayout.from_apr(apr, G.APR_VALIDATE | G.APR_REQUIRE_BALANCE)
    t_build = time.perf_counter() - t_build
    w = S.gaussian_stencil(K, SIGMA).astype(np.float32)
    st_h = G.apr_restrict_stencil(w, apr.l_max, apr.l_min)
    Np = apr.n_particles
    st = torch.as_tensor(st_h, device=dev)
    vals = torch.as_tensor(apr.values, device=dev)
    gout = torch.as_tensor(np.random.default_rng(0).normal(size=Np).astype(np.float32), device=dev)
    tree = torch.empty(lay.n_tree, device=dev)
    out = torch.empty(Np, device=dev)
    gp = torch.empty(Np, device=dev)
    gw = torch.empty((apr.n_levels, K ** 3), device=dev)
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=dev)  # 512 MB > L2 (129 MB)
    stream = torch.cuda.current_stream()

    gtree = torch.empty(lay.n_tree, device=dev)
    bufs = dict(vals=vals, gout=gout, tree=tree, out=out, gp=gp, gw=gw, gtree=gtree)
    T = layer_step(args, lay, st, bufs, dev, stream, flush, world, clocks=True)
    parts, step_ms, e2e, wall, clocks = T["parts"], T["step_ms"], T["e2e_ms"], T["wall"], T["clocks"]
    t_restrict, t_conv, t_adj, t_tadj, t_sgrad, t_pipe = parts

    # gradient magnitude with level-rescaled Sobel filters (Sec. 4.3): three 3^3 convolutions on one
    # staged patch, timed alone (L2 flushed before each launch)
    sob = G.sobel_stencils(3)
    sob_st = torch.as_tensor(np.stack([G.apr_rescale_stencil(sob[a], apr.l_max, apr.l_min) for a in range(3)]),
                             device=dev)
    gm_out = torch.empty(Np, device=dev)
    G.apr_gradient_magnitude(lay, vals, tree, sob_st, 3, G.APR_BC_REFLECT, gm_out)
    gm_ms = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        G.apr_gradient_magnitude(lay, vals, tree, sob_st, 3, G.APR_BC_REFLECT, gm_out)
        b.record(stream)
        b.synchronize()
        gm_ms.append(a.elapsed_time(b))
    gm_ms = statistics.mean(gm_ms)

    # context: a dense FP32 5^3 convolution of the same-size pixel image with cuDNN (torch conv3d,
    # TF32 off), the stand-in for the paper's dense pixel baseline (same pixel-equivalent metric)
    dense = None
    if not args.no_dense and world == 1:
        dense = dense_pixel_conv(apr.dims, w, args.steps, flush, stream)

    # forward-only pipeline (tree restriction + convolution), the paper's timed pipeline
    mean = lambda v: sum(v) / len(v)
    fwd_ms = mean(t_pipe)
    conv_ms, adj_ms = mean(t_conv), mean(t_adj)
    conv_bytes, restrict_bytes = algorithmic_bytes(apr, lay, K)
    peaks, src = _peaks()
    hbm = float(peaks["hbm_gbs"])
    pix_bytes = float(np.prod(apr.dims)) * 4.0
    # our kernels per step: restriction (one per level holding tree nodes), convolution, convolution
    # adjoint, push-down (one per level holding tree nodes), stencil-gradient partials, reduction
    n_tree_levels = len(set(lay.export(G._abi.APR_STRUCT_TREE_ITEMS)[:, 0].tolist()))
    nc = conv_launches(apr, st_h, K)
    launches_per_step = n_tree_levels + nc + nc + n_tree_levels + 2
    # the dominant call of the step: the convolution adjoint (its radius-1 tiles in one launch on the
    # library's second stream beside the launch over the l_max tiles; the call also clears the two
    # gradient outputs). Its algorithmic bytes equal the forward's: dL/dout in, dL/dparticles and
    # dL/dtree out, y indices and row pointers.
    dom_ms, dom_call = (adj_ms, "apr_convolve_adjoint") if adj_ms >= conv_ms else (conv_ms, "apr_convolve")
    dom_name = dom_call + (": conv_bwd_data_r1_kernel (levels below l_max, radius 1) beside conv_bwd_data_kernel<2> "
                           "(l_max), conv_bwd_data_r2_pool_kernel after the radius-1 launch"
                           if dom_call == "apr_convolve_adjoint" else
                           ": conv_fwd_r1_kernel (levels below l_max, radius 1) beside conv_fwd_kernel<2> (l_max), "
                           "conv_fwd_r2_pool_kernel after the radius-1 launch")
    traffic = recorded_traffic(dom_call)
    rec = {
        "metric": "APR conv Gparticles/s & pixel-equiv GB/s",
        "value": round(world * Np / (step_ms * 1e-3) / 1e9, 4),
        "unit": "Gparticles/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(step_ms, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded 2000-blob image with Poisson noise -> APR)",
        "config": {"workload": "blob APR 1024x1024x512 pixels (z=512), 5^3 Gaussian sigma=1.5, restricted per-level stencils",
                   "n_particles": Np, "n_tree": lay.n_tree, "levels": [apr.l_min, apr.l_max],
                   "computational_ratio": round(float(np.prod(apr.dims)) / Np, 2),
                   "step": "tree restrict + convolve (apr_convolve_auto) + convolve_backward (data + stencil grads)",
                   "backward": "apr_convolve_backward: data adjoint and tree adjoint on the step's stream, stencil "
                               "gradient concurrently on the library's second stream (fork / join events)",
                   "l2": "flushed before every step (512 MB write, outside the step events)",
                   "launch": "the step as one CUDA graph (the parts and the end-to-end step: one graph per part)"
                             if not args.no_graph else "eager",
                   "parallelism": f"replicas x{world}"},
        "pixel_equiv_GBps": round(world * pix_bytes / (step_ms * 1e-3) / 1e9, 2),
        "forward_pipeline": {"ms": round(fwd_ms, 5),
                             "Gparticles_per_s": round(Np / (fwd_ms * 1e-3) / 1e9, 3),
                             "pixel_equiv_GBps": round(pix_bytes / (fwd_ms * 1e-3) / 1e9, 2),
                             "paper_context": "up to 1 TB/s pixel-equivalent on one RTX 2080 Max-Q (paper abstract)"},
        "dense_pixel_conv": dense,
        "gradient_magnitude": {"ms": round(gm_ms, 5), "Gparticles_per_s": round(Np / (gm_ms * 1e-3) / 1e9, 3),
                               "filters": "3^3 Sobel along z, x, y, rescaled per level (Eq. adapt_grad)",
                               "hbm_frac_conv_bytes": round(algorithmic_bytes(apr, lay, 3)[0] / (gm_ms * 1e-3) / 1e9 / hbm, 4)},
        "step_ms_parts": {"tree_restrict": round(mean(t_restrict), 5), "convolve": round(conv_ms, 5),
                          "convolve_adjoint": round(adj_ms, 5), "tree_restrict_adjoint": round(mean(t_tadj), 5),
                          "stencil_grad": round(mean(t_sgrad), 5),
                          "timing": "each part alone, one after the other (a separate pass; the step overlaps "
                                    "the stencil gradient with the data and tree adjoints)"},
        "roofline": {"kernel": dom_name, "bound": "hbm",
                     "achieved": round(conv_bytes / (dom_ms * 1e-3) / 1e9, 2), "peak": hbm,
                     "unit": "GB/s", "frac": round(conv_bytes / (dom_ms * 1e-3) / 1e9 / hbm, 4),
                     "traffic": traffic, "traffic_source": "profiles/traffic.json (ncu dram bytes of the call's "
                     "launches, same source)" if traffic else None, "peak_source": src + " (hbm_gbs, copy bandwidth)",
                     "algorithmic_bytes_per_launch": conv_bytes,
                     "per_launch": "per call: algorithmic bytes of the whole call / the call's event time (its "
                                   "launches on two streams, joined)",
                     "convolve_frac": round(conv_bytes / (conv_ms * 1e-3) / 1e9 / hbm, 4)},
        "e2e": {"value": round(world * Np / (e2e * 1e-3) / 1e9, 4), "unit": "Gparticles/s",
                "h2d_bytes_per_step": T["h2d"], "d2h_bytes_per_step": T["d2h"],
                "ms_per_step": round(e2e, 4),
                "copies": "pinned host buffers; dL/dout in and outputs out on a second stream, overlapped with "
                          "the step's kernels (the backward's parts called one after the other, so the particle "
                          "gradient goes out while the stencil gradient runs); the values of the next step "
                          "come in during the step (a staging buffer, copied to the values at step start)"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "wall_s_timed_region": round(wall, 4),
        "layout_bytes": lay.layout_bytes(),
        "layout_build_s": round(t_build, 3),   # once per APR: validation, index, work lists, tile plans, upload
    }
    # the plain method on the same APR (Sec. 4.1): the 5^3 Gaussian itself at every level (radius 2
    # everywhere), the same step, buffers and timing
    if not args.no_plain:
        st_plain = torch.as_tensor(np.repeat(w.reshape(1, -1), apr.n_levels, 0), device=dev).contiguous()
        P = layer_step(args, lay, st_plain, bufs, dev, stream, flush, world)
        pall = [mean(v) for v in P["parts"]]
        pp = pall[:5]
        p_dom_ms, p_dom = ((pp[2], "conv_bwd_data_kernel<2> (apr_convolve_adjoint: one launch over all tiles)")
                           if pp[2] >= pp[1] else (pp[1], "conv_fwd_kernel<2> (apr_convolve: one launch over all tiles)"))
        npc = conv_launches(apr, st_plain.cpu().numpy(), K)
        rec["plain5"] = {
            "value": round(world * Np / (P["step_ms"] * 1e-3) / 1e9, 4), "unit": "Gparticles/s",
            "ms_per_step": round(P["step_ms"], 5),
            "config": "same APR and step, 5^3 Gaussian sigma=1.5 at every level (no per-level restriction)",
            "step_ms_parts": dict(zip(("tree_restrict", "convolve", "convolve_adjoint", "tree_restrict_adjoint",
                                       "stencil_grad"), (round(v, 5) for v in pp))),
            "forward_pipeline": {"ms": round(pall[5], 5),
                                 "pixel_equiv_GBps": round(pix_bytes / (pall[5] * 1e-3) / 1e9, 2)},
            "roofline": {"kernel": p_dom, "bound": "hbm", "achieved": round(conv_bytes / (p_dom_ms * 1e-3) / 1e9, 2),
                         "peak": hbm, "unit": "GB/s", "frac": round(conv_bytes / (p_dom_ms * 1e-3) / 1e9 / hbm, 4),
                         "convolve_frac": round(conv_bytes / (pp[1] * 1e-3) / 1e9 / hbm, 4),
                         "algorithmic_bytes_per_launch": conv_bytes, "peak_source": src + " (hbm_gbs)"},
            "e2e": {"value": round(world * Np / (P["e2e_ms"] * 1e-3) / 1e9, 4), "unit": "Gparticles/s",
                    "h2d_bytes_per_step": P["h2d"], "d2h_bytes_per_step": P["d2h"], "ms_per_step": round(P["e2e_ms"], 4)},
            "gpu_launches": (2 * n_tree_levels + 2 * npc + 2) * args.steps,
        }
    if rank == 0 and not args.no_cpu_baseline:
        rec["cpu_baseline"] = cpu_baseline(apr, st_h, gout.cpu().numpy(), budget_s=args.cpu_budget)
        rec["cpu_multicore"] = cpu_multicore(apr, st_h, gout.cpu().numpy())
    return rec


def cpu_multicore(apr, st, gout, reps=2):
    """The multi-core FP32 CPU implementation (cpubase/: rows of a level in parallel, dynamic
    scheduling) timed on the whole step (tree restriction, convolution, backward) on all host
    threads; one untimed run first."""
    import numpy as np

    import cpubase
    c = cpubase.CpuApr(apr)
    stf = np.ascontiguousarray(st, np.float32).reshape(apr.n_levels, -1)

    def step():
        t = c.tree_restrict(apr.values)
        t1 = time.perf_counter()
        c.convolve(apr.values, t, stf, K)
        t2 = time.perf_counter()
        c.backward(apr.values, t, stf, K, gout)
        return t1, t2

    step()
    ts, parts = [], []
    for _ in range(reps):
        t0 = time.perf_counter()
        t1, t2 = step()
        t3 = time.perf_counter()
        ts.append(t3 - t0)
        parts.append((t1 - t0, t2 - t1, t3 - t2))
    sec = statistics.mean(ts)
    pm = [statistics.mean(p[i] for p in parts) for i in range(3)]
    return {"value": round(apr.n_particles / sec / 1e9, 6), "unit": "Gparticles/s", "cores": c.threads,
            "kind": "FP32 multi-threaded CPU implementation (cpubase/; rows of a level in parallel, dynamic scheduling)",
            "ms_per_step": round(1e3 * sec, 2),
            "step_ms_parts": {"tree_restrict": round(1e3 * pm[0], 2), "convolve": round(1e3 * pm[1], 2),
                              "backward": round(1e3 * pm[2], 2)},
            "sample": f"the whole step on all {apr.n_particles} particles, mean of {reps} runs after one untimed run"}


MC_WORKLOAD = "blob256"
MC_C = 16


def mc_inputs(apr, seed=0):
    """bfloat16-exact features (k/8 in [-8, 8]), weights ~ N(0, 1/432) rounded to bf16, upstream
    gradients (k/8); returned as float64 arrays holding bf16 values."""
    import numpy as np
    import torch
    rng = np.random.default_rng(seed)
    x = rng.integers(-64, 65, size=(apr.n_particles, MC_C)) / 8.0
    w = torch.as_tensor(rng.normal(scale=432 ** -0.5, size=(apr.n_levels, MC_C, MC_C, 27)).astype(np.float32))
    w = w.to(torch.bfloat16).to(torch.float64).numpy()
    g = rng.integers(-64, 65, size=(apr.n_particles, MC_C)) / 8.0
    return x, w, g


def mc_algorithmic(apr, lay):
    """Per launch of the multi-channel forward: bytes (features 32 B in, y 2 B, outputs 64 B out per
    particle; tree 32 + 2 B per node; row pointers; weights) and tensor FLOPs (2 * 27 * 16 * 16 per
    particle)."""
    Np, Nt = apr.n_particles, lay.n_tree
    Rp = int(apr.row_ptr.size - 1)
    Rt = sum(apr.level_dims(l)[0] * apr.level_dims(l)[1] for l in range(apr.l_min, apr.l_max))
    byts = Np * (32 + 2 + 64) + Nt * (32 + 2) + (Rp + Rt) * 4 + apr.n_levels * MC_C * MC_C * 27 * 2
    flops = 2 * 27 * MC_C * MC_C * Np
    return byts, flops


def run_mc(args, rank, world, full=True):
    """Multi-channel step on the 256^3 blob APR: BF16 tree + 16->16 convolution + its backward."""
    import numpy as np
    import torch

    import aprsynth as S
    import paper_2112_03592_gb300 as G

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    apr = S.make_config(MC_WORKLOAD)
    lay = G.AprLayout.from_apr(apr, G.APR_VALIDATE | G.APR_REQUIRE_BALANCE)
    Np = apr.n_particles
    xh, wh, gh = mc_inputs(apr)
    bf = lambda a: torch.as_tensor(a.astype(np.float32), device=dev).to(torch.bfloat16).contiguous()
    x, w, g = bf(xh), bf(wh), bf(gh)
    tree = torch.empty((lay.n_tree, MC_C), dtype=torch.bfloat16, device=dev)
    out = torch.empty((Np, MC_C), device=dev)
    gp = torch.empty((Np, MC_C), device=dev)
    gw = torch.empty((apr.n_levels, MC_C, MC_C, 27), device=dev)
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    # BF16 tree | forward | data adjoint (+ tree push-down) | weight gradient
    parts_fns = [lambda: G.apr_tree_restrict_bf16(lay, x, tree),
                 lambda: G.apr_convolve_mc(lay, x, tree, w, G.APR_BC_REFLECT, out),
                 lambda: G.apr_convolve_mc_backward(lay, x, tree, w, g, G.APR_BC_REFLECT, need_weights=False, grad_particles=gp),
                 lambda: G.apr_convolve_mc_backward(lay, x, tree, w, g, G.APR_BC_REFLECT, need_particles=False, grad_weights=gw)]
    for f in parts_fns:
        f()
    run_part = make_replayers(parts_fns, not args.no_graph)

    def step(e=None):
        if e is not None:
            e[0].record(stream)
        for j, f in enumerate(run_part):
            f()
            if e is not None:
                e[j + 1].record(stream)

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    clk = ClockSampler(dev.index).__enter__() if full else None
    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        step(ev[i])
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    if clk is not None:
        time.sleep(0.12)
        clk.__exit__()
    lay.sync_status()
    parts = [statistics.mean(ev[i][j].elapsed_time(ev[i][j + 1]) for i in range(args.steps)) for j in range(4)]
    step_ms = sum(parts)
    step_ms = max_over_ranks(step_ms, dev)
    byts, flops = mc_algorithmic(apr, lay)
    peaks, src = _peaks()
    hbm, tc = float(peaks["hbm_gbs"]), float(peaks.get("bf16_tflops", 1900.0))
    names = ["tree_restrict_bf16", "convolve_mc", "data_adjoint", "weight_grad"]
    dom = max(range(1, 4), key=lambda j: parts[j])
    mc_traffic = recorded_traffic(names[dom], "mc")
    n_tree_levels = len(set(lay.export(G._abi.APR_STRUCT_TREE_ITEMS)[:, 0].tolist()))
    # per step: BF16 tree (one launch per level), weight layout + forward, weight layout + data
    # adjoint, push-down (one per level), weight gradient + its reduction
    launches_per_step = n_tree_levels + 2 + 2 + n_tree_levels + 2
    rec = {
        "metric": "APR conv Gparticles/s & pixel-equiv GB/s",
        "value": round(world * Np / (step_ms * 1e-3) / 1e9, 4), "unit": "Gparticles/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(step_ms, 5), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16",
        "data": "synthetic (seeded 400-blob 256^3 image with Poisson noise -> APR; random bf16 features and weights)",
        "config": {"workload": "blob APR 256^3 pixels, 16 -> 16 channels bf16 (FP32 accumulation), 3^3 per-level weights",
                   "n_particles": Np, "n_tree": lay.n_tree, "levels": [apr.l_min, apr.l_max],
                   "step": "bf16 tree + convolve_mc + backward (data adjoint with tree push-down, weight gradient)",
                   "l2": "flushed before every step (512 MB write, outside the step events)",
                   "launch": "CUDA graphs (one per part)" if not args.no_graph else "eager",
                   "parallelism": f"replicas x{world}"},
        "step_ms_parts": {n: round(t, 5) for n, t in zip(names, parts)},
        "roofline": {"kernel": {1: "mc_fwd_kernel (apr_convolve_mc)", 2: "mc_bwd_data_kernel (+ push-down)",
                                3: "mc_wgrad_kernel (+ reduce)"}[dom],
                     "bound": "hbm", "achieved": round(byts / (parts[dom] * 1e-3) / 1e9, 2), "peak": hbm, "unit": "GB/s",
                     "frac": round(byts / (parts[dom] * 1e-3) / 1e9 / hbm, 4), "traffic": mc_traffic,
                     "traffic_source": "profiles/traffic.json (mc: ncu dram bytes of the call's launches, same "
                     "source)" if mc_traffic else None,
                     "peak_source": src + " (hbm_gbs)", "algorithmic_bytes_per_launch": byts,
                     "tensor_tflops": round(flops / (parts[dom] * 1e-3) / 1e12, 2),
                     "tensor_frac": round(flops / (parts[dom] * 1e-3) / 1e12 / tc, 4),
                     "forward_frac": round(byts / (parts[1] * 1e-3) / 1e9 / hbm, 4),
                     "forward_tensor_frac": round(flops / (parts[1] * 1e-3) / 1e12 / tc, 4)},
        "gpu_launches": launches_per_step * args.steps,
    }
    if not full:
        return rec
    # end to end with host buffers: H2D of features and upstream gradient, D2H of outputs and grads
    h_x, h_g = x.cpu().pin_memory(), g.cpu().pin_memory()
    h_out, h_gp = torch.empty_like(out, device="cpu").pin_memory(), torch.empty_like(gp, device="cpu").pin_memory()
    h_gw = torch.empty_like(gw, device="cpu").pin_memory()

    # copies the kernels do not wait for run on a second stream: dL/dout goes in (after the features)
    # while the tree and the forward run, the outputs come back while the data adjoint runs and the
    # particle gradient while the weight gradient runs
    cs = torch.cuda.Stream(device=dev)
    ev_x, ev_g, ev_out, ev_gp, ev_stage = (torch.cuda.Event() for _ in range(5))
    # streaming input: the next step's features come in (into a staging buffer) during this step
    staging = torch.empty_like(x)
    staging.copy_(h_x)
    ev_stage.record(stream)
    torch.cuda.synchronize()

    def e2e_step():
        cs.wait_stream(stream)                  # the previous step has finished with g
        stream.wait_event(ev_stage)
        x.copy_(staging, non_blocking=True)
        ev_x.record(stream)
        with torch.cuda.stream(cs):
            cs.wait_event(ev_x)
            g.copy_(h_g, non_blocking=True)
            ev_g.record(cs)
            staging.copy_(h_x, non_blocking=True)   # the next step's features
            ev_stage.record(cs)
        run_part[0]()
        run_part[1]()
        ev_out.record(stream)
        with torch.cuda.stream(cs):
            cs.wait_event(ev_out)
            h_out.copy_(out, non_blocking=True)
        stream.wait_event(ev_g)
        run_part[2]()
        ev_gp.record(stream)
        with torch.cuda.stream(cs):
            cs.wait_event(ev_gp)
            h_gp.copy_(gp, non_blocking=True)
        run_part[3]()
        h_gw.copy_(gw, non_blocking=True)
        stream.wait_stream(cs)                  # the step ends when every copy has landed

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_step()
        b.record(stream)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e = max_over_ranks(statistics.mean(e2e_ms), dev)
    rec["e2e"] = {"value": round(world * Np / (e2e * 1e-3) / 1e9, 4), "unit": "Gparticles/s",
                  "h2d_bytes_per_step": int(h_x.numel() * 2 + h_g.numel() * 2),
                  "d2h_bytes_per_step": int(h_out.numel() * 4 + h_gp.numel() * 4 + h_gw.numel() * 4),
                  "ms_per_step": round(e2e, 4),
                  "copies": "pinned host buffers; dL/dout in, outputs and particle gradients out on a second "
                            "stream, overlapped with the step's kernels; the next step's features come in during "
                            "the step (a staging buffer, copied to the features at step start)"}
    rec["clocks"] = clk.summary(t0, t1)
    if rank == 0 and not args.no_cpu_baseline:
        rec["cpu_baseline"] = mc_cpu_baseline(apr, xh, wh, gh, budget_s=args.cpu_budget)
    return rec


def mc_cpu_baseline(apr, x, w, g, budget_s=20.0):
    """The FP64 oracle with 16 channels on a bounded sample: full BF16 tree fill, then forward and
    backward of a random sample of output particles (rate per particle of the whole step)."""
    import numpy as np

    import oracle
    o = oracle.Oracle(apr, x)
    t0 = time.perf_counter()
    o.tree_bf16()
    t_fill = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    n = 200

    def run(smp):
        o.conv(w, 3, sample=smp, C_out=MC_C)
        o.conv_backward(w, 3, g, sample=smp, C_out=MC_C)

    t0 = time.perf_counter()
    run(np.sort(rng.choice(apr.n_particles, n, replace=False)))
    t_probe = time.perf_counter() - t0
    n2 = int(min(apr.n_particles, max(n, n * (budget_s - t_fill) / max(t_probe, 1e-6) * 0.6)))
    step_s, t_fixed, t_s = oracle_sampled_step(apr.n_particles, t_fill, run, n2, rng)
    return {"value": round(apr.n_particles / step_s / 1e9, 9), "unit": "Gparticles/s", "cores": 1, "kind": "oracle",
            "sample": f"full bf16 tree fill ({t_fill:.2f} s) + 16-channel forward and backward of {n2} random output "
                      f"particles ({t_s:.2f} s, of which {t_fixed:.2f} s does not depend on the sample), scaled to all "
                      f"{apr.n_particles} outputs; FP64, 1 thread"}


RL_WORKLOAD = "blob512"
RL_ITERS = 20


def run_rl(args, rank, world, full=True):
    """Richardson-Lucy on the 512^3 blob APR: 20 iterations with the restricted 5^3 Gaussian PSF
    (sigma 1.5) and its flip; one step = the whole 20-iteration deconvolution from i_0 = u."""
    import numpy as np
    import torch

    import aprsynth as S
    import paper_2112_03592_gb300 as G

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    apr = S.make_config(RL_WORKLOAD)
    lay = G.AprLayout.from_apr(apr, G.APR_VALIDATE | G.APR_REQUIRE_BALANCE)
    Np = apr.n_particles
    w = S.gaussian_stencil(K, SIGMA).astype(np.float32)
    st_h = G.apr_restrict_stencil(w, apr.l_max, apr.l_min)
    st = torch.as_tensor(st_h, device=dev)
    u = torch.as_tensor(apr.values, device=dev)
    est = torch.empty_like(u)
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def rl():
        est.copy_(u)
        G.apr_richardson_lucy(lay, u, st, K, RL_ITERS, G.APR_BC_REFLECT, estimate=est)

    rl()
    step = make_replayers([rl], not args.no_graph)[0]
    clk = ClockSampler(dev.index).__enter__() if full else None
    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    t1 = time.perf_counter()
    if clk is not None:
        time.sleep(0.12)
        clk.__exit__()
    lay.sync_status()
    step_ms = max_over_ranks(statistics.mean(ms), dev)
    # one convolution alone, for the roofline of the dominant kernel (the fused-epilogue convolution)
    tree = G.apr_tree_restrict(lay, u)
    out = torch.empty_like(u)
    ev = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        G.apr_convolve(lay, u, tree, st, K, G.APR_BC_REFLECT, out)
        b.record(stream)
        b.synchronize()
        ev.append(a.elapsed_time(b))
    conv_ms = statistics.mean(ev)
    conv_bytes, _ = algorithmic_bytes(apr, lay, K)
    conv_bytes += Np * 4   # the fused epilogue reads one more value per particle
    peaks, src = _peaks()
    hbm = float(peaks["hbm_gbs"])
    n_tree_levels = len(set(lay.export(G._abi.APR_STRUCT_TREE_ITEMS)[:, 0].tolist()))
    pix = float(np.prod(apr.dims))
    rec = {
        "metric": "APR conv Gparticles/s & pixel-equiv GB/s",
        "value": round(world * Np * RL_ITERS / (step_ms * 1e-3) / 1e9, 4),
        "unit": "Gparticles/s (particle-iterations of Richardson-Lucy; 2 convolutions each)",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded 200-blob 512^3 image with Poisson noise -> APR)",
        "config": {"workload": "blob APR 512^3 pixels: 20 Richardson-Lucy iterations, restricted 5^3 Gaussian PSF sigma=1.5 and its flip",
                   "n_particles": Np, "n_tree": lay.n_tree, "levels": [apr.l_min, apr.l_max],
                   "step": "20 iterations from i_0 = u (per iteration: 2 tree restrictions, 2 convolutions with fused divide / multiply)",
                   "launch": "one CUDA graph for the 20 iterations" if not args.no_graph else "eager",
                   "l2": "flushed before every step (512 MB write, outside the step events)",
                   "parallelism": f"replicas x{world}"},
        "pixel_equiv_GBps_per_conv": round(pix * 4 * 2 * RL_ITERS / (step_ms * 1e-3) / 1e9, 2),
        "roofline": {"kernel": "apr_convolve (one call timed alone: conv_fwd_r1_kernel beside conv_fwd_kernel<2>, "
                               "conv_fwd_r2_pool_kernel)", "bound": "hbm",
                     "achieved": round(conv_bytes / (conv_ms * 1e-3) / 1e9, 2), "peak": hbm, "unit": "GB/s",
                     "frac": round(conv_bytes / (conv_ms * 1e-3) / 1e9 / hbm, 4), "traffic": None,
                     "peak_source": src + " (hbm_gbs)", "algorithmic_bytes_per_launch": conv_bytes,
                     "conv_ms": round(conv_ms, 5)},
        "gpu_launches": RL_ITERS * 2 * (n_tree_levels + conv_launches(apr, st_h, K)) * args.steps,
    }
    if not full:
        return rec
    h_u, h_est = torch.as_tensor(apr.values).pin_memory(), torch.empty(Np).pin_memory()
    e2e = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        u.copy_(h_u, non_blocking=True)
        step()
        h_est.copy_(est, non_blocking=True)
        b.record(stream)
        b.synchronize()
        if i >= args.warmup:
            e2e.append(a.elapsed_time(b))
    e2e_ms = max_over_ranks(statistics.mean(e2e), dev)
    rec["e2e"] = {"value": round(world * Np * RL_ITERS / (e2e_ms * 1e-3) / 1e9, 4), "unit": rec["unit"],
                  "h2d_bytes_per_step": int(h_u.numel() * 4), "d2h_bytes_per_step": int(h_est.numel() * 4),
                  "ms_per_step": round(e2e_ms, 4)}
    rec["clocks"] = clk.summary(t0, t1)
    if rank == 0 and not args.no_cpu_baseline:
        rec["cpu_baseline"] = rl_cpu_baseline(apr, st_h, budget_s=args.cpu_budget)
    return rec


def rl_cpu_baseline(apr, st, budget_s=20.0):
    """The FP64 oracle's Richardson-Lucy iteration on a bounded sample: the full tree fill (twice per
    iteration) and the two convolutions of one iteration evaluated for a random sample of output
    particles; rate = particle-iterations per second."""
    import numpy as np

    import oracle
    W = st.reshape(apr.n_levels, -1).astype(np.float64)
    o = oracle.Oracle(apr)
    t0 = time.perf_counter()
    o.tree()
    t_fill = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    n = 1000
    s = np.sort(rng.choice(apr.n_particles, n, replace=False))
    t0 = time.perf_counter()
    o.conv(W, K, sample=s)
    t_probe = time.perf_counter() - t0
    n2 = int(min(apr.n_particles, max(n, n * (budget_s - t_fill) / max(2 * t_probe, 1e-6) * 0.8)))
    s = np.sort(rng.choice(apr.n_particles, n2, replace=False))
    t0 = time.perf_counter()
    o.conv(W, K, sample=s)
    o.conv(W[:, ::-1].copy(), K, sample=s)
    t_s = time.perf_counter() - t0
    per = 2 * t_fill / apr.n_particles + t_s / n2
    return {"value": round(1.0 / per / 1e9, 9), "unit": "Gparticles/s (particle-iterations)", "cores": 1,
            "kind": "oracle",
            "sample": f"full tree fill ({t_fill:.2f} s, counted twice per iteration, scaled by sample/N) + the two "
                      f"convolutions of one iteration for {n2} random output particles ({t_s:.2f} s), FP64, 1 thread"}


def pixels_per_particle(apr):
    """Pixels each particle covers (cell edge 2^(l_max - l) per axis, clipped at the image edge)."""
    import numpy as np
    l, z, x, y = apr.particle_coords()
    s = (1 << (apr.l_max - l)).astype(np.int64)
    ext = [np.minimum(s, d - c * s) for c, d in zip((z, x, y), apr.dims)]
    return (ext[0] * ext[1] * ext[2]).astype(np.float64)


SURROGATE_WEIGHTS = os.path.join(ROOT, "paper_2112_03592_gb300", "surrogate_weights", "rl20_blob256.npz")


def run_surrogate(args, rank, world, pretrained=None):
    """APR CNN surrogate of 20 Richardson-Lucy iterations: trained on seeded 256^3 blob APRs (here,
    or the committed weights written by surrogate_weights/train.py when `pretrained` names them),
    evaluated on the 1024x1024x512 blob APR against the plain 20-iteration filter (time and PSNR)."""
    import numpy as np
    import torch

    import aprsynth as S
    import paper_2112_03592_gb300 as G
    from paper_2112_03592_gb300.surrogate import AprCnn, psnr, train

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    w = S.gaussian_stencil(K, SIGMA).astype(np.float32)
    flags = G.APR_VALIDATE | G.APR_REQUIRE_BALANCE
    model = AprCnn(4, n_dist=8, seed=0)
    if pretrained:
        z = np.load(pretrained)
        model.W = [torch.as_tensor(z[f"layer{i}"], device=dev).contiguous() for i in range(4)]
        hist = [float(z["loss_first"])] * 10 + [float(z["loss_last"])] * 10
        t_data = t_train = 0.0
        train_desc = (f"{int(z['n_train'])} seeded 256^3 blob APRs (seeds {int(z['seed0'])}..), {int(z['steps'])} Adam "
                      f"steps, lr {float(z['lr'])}; committed weights (surrogate_weights/train.py)")
    else:
        t0 = time.perf_counter()
        samples = []
        for i in range(args.sur_train):
            a = S.make_config("blob256", seed=100 + i)
            lay = G.AprLayout.from_apr(a, flags)
            x = torch.as_tensor(a.values, device=dev)
            st = torch.as_tensor(G.apr_restrict_stencil(w, a.l_max, a.l_min), device=dev)
            t = G.apr_richardson_lucy(lay, x, st, K, RL_ITERS)
            samples.append((lay, x, t, float(1.0 / float(x.mean()))))
        t_data = time.perf_counter() - t0
        t0 = time.perf_counter()
        hist = train(model, samples, args.sur_steps, lr=args.sur_lr)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        train_desc = f"{args.sur_train} seeded 256^3 blob APRs, {args.sur_steps} Adam steps, lr {args.sur_lr}"

    apr = S.make_config(WORKLOAD)
    clean = S.make_config(WORKLOAD, clean=True)
    lay = G.AprLayout.from_apr(apr, flags)
    Np = apr.n_particles
    x = torch.as_tensor(apr.values, device=dev)
    st = torch.as_tensor(G.apr_restrict_stencil(w, apr.l_max, apr.l_min), device=dev)
    scale = float(1.0 / float(x.mean()))
    Wb = model.stack_weights(lay)
    est = torch.empty_like(x)
    holder = [None]

    def rl():
        est.copy_(x)
        G.apr_richardson_lucy(lay, x, st, K, RL_ITERS, estimate=est)

    def cnn():
        holder[0] = model.forward(lay, x, scale, weights=Wb)

    rl()
    cnn()
    run_rl_, run_cnn = make_replayers([rl, cnn], not args.no_graph)
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def timed(f):
        ts = []
        for i in range(args.warmup + args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            f()
            b.record(stream)
            b.synchronize()
            if i >= args.warmup:
                ts.append(a.elapsed_time(b))
        return statistics.mean(ts)

    rl_ms = timed(run_rl_)
    cnn_ms = timed(run_cnn)
    n_tree_levels = len(set(lay.export(G._abi.APR_STRUCT_TREE_ITEMS)[:, 0].tolist()))
    y = holder[0]
    wts = torch.as_tensor(pixels_per_particle(apr), device=dev)
    ref_clean = torch.as_tensor(clean.values, device=dev)
    rec = {
        "metric": "surrogate vs iterative at PSNR",
        "value": round(rl_ms / cnn_ms, 3), "unit": "x (time of 20 RL iterations / time of CNN inference)",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(cnn_ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (FP32 accumulation)",
        "data": "synthetic (seeded blob images with Poisson noise -> APR); noise-free particle means as ground truth",
        "config": {"workload": "4-layer APR CNN (16 ch bf16, 3^3 per-level weights, ReLU, residual) vs 20 Richardson-Lucy "
                               "iterations (restricted 5^3 Gaussian PSF sigma=1.5), on the 1024x1024x512 blob APR",
                   "n_particles": Np, "train": train_desc, "launch": "CUDA graphs" if not args.no_graph else "eager"},
        "rl20_ms": round(rl_ms, 4), "cnn_ms": round(cnn_ms, 4),
        "cnn_Gparticles_per_s": round(Np / (cnn_ms * 1e-3) / 1e9, 4),
        "psnr_db": {"cnn_vs_rl20": round(psnr(y, est, wts), 3), "input_vs_rl20": round(psnr(x, est, wts), 3),
                    "rl20_vs_clean": round(psnr(est, ref_clean, wts), 3), "cnn_vs_clean": round(psnr(y, ref_clean, wts), 3),
                    "input_vs_clean": round(psnr(x, ref_clean, wts), 3),
                    "weighting": "pixels covered by each particle (pixel-equivalent)"},
        "training": {"loss_first": round(float(np.mean(hist[:10])), 6), "loss_last": round(float(np.mean(hist[-10:])), 6),
                     "data_s": round(t_data, 1), "train_s": round(t_train, 1)},
        # per CNN inference: embedding, 4 x (tree restriction per level, weight layout, convolution;
        # hidden ReLUs fused into the convolution), read-out; per RL run: 2 x (tree + convolution) per iteration
        "gpu_launches": (2 + 4 * (n_tree_levels + 2) +
                         RL_ITERS * 2 * (n_tree_levels + conv_launches(apr, st.cpu().numpy(), 5))) * args.steps,
    }
    return rec


def oracle_sampled_step(N, t_fill, run, n, rng):
    """Estimate the oracle's whole-step time from sampled runs. run(sample) evaluates the step's
    outputs (and gradients) at the sampled output particles; its cost is a part that does not depend
    on the sample (the tree transpose runs over every node) plus a part per sampled particle. A
    16-particle run measures the first, an n-particle run the second; the step is estimated as
    fill + fixed + per-particle x N. Returns (estimated step seconds, fixed s, sampled-run s)."""
    import numpy as np
    s0 = np.sort(rng.choice(N, min(16, N), replace=False))
    t0 = time.perf_counter()
    run(s0)
    t_fixed = time.perf_counter() - t0
    s = np.sort(rng.choice(N, min(n, N), replace=False))
    t0 = time.perf_counter()
    run(s)
    t_s = time.perf_counter() - t0
    per = max(t_s - t_fixed, 1e-12) / max(s.size - s0.size, 1)
    return t_fill + t_fixed + per * N, t_fixed, t_s


def cpu_baseline(apr, st, gout, budget_s=20.0, sample_n=None):
    """The FP64 oracle (single thread, as it stands) on a bounded sample of the same step: the full
    tree fill, then forward and backward for a random sample of output particles. The tree fill
    time is scaled by sample/N (it is linear in N) so the rate is per particle of the whole step."""
    import numpy as np

    import oracle
    o = oracle.Oracle(apr)
    t0 = time.perf_counter()
    o.tree()
    t_fill = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    n = sample_n or 2000
    W = st.astype(np.float64)
    g64 = gout.astype(np.float64)

    def run(smp):
        o.conv(W, K, sample=smp)
        o.conv_backward(W, K, g64, sample=smp)

    t0 = time.perf_counter()
    run(np.sort(rng.choice(apr.n_particles, n, replace=False)))
    t_probe = time.perf_counter() - t0
    # size the real sample to the time budget
    n2 = int(min(apr.n_particles, max(n, n * (budget_s - t_fill) / max(t_probe, 1e-6) * 0.6)))
    step_s, t_fixed, t_s = oracle_sampled_step(apr.n_particles, t_fill, run, n2, rng)
    return {"value": round(apr.n_particles / step_s / 1e9, 9), "unit": "Gparticles/s", "cores": 1, "kind": "oracle",
            "sample": f"full tree fill ({t_fill:.2f} s) + forward and backward of {n2} random output particles "
                      f"({t_s:.2f} s, of which {t_fixed:.2f} s does not depend on the sample), scaled to all "
                      f"{apr.n_particles} outputs; FP64, 1 thread"}


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step is a bounded sample of the workload."""
    import numpy as np

    import aprsynth as S
    import oracle
    apr = S.make_config(WORKLOAD)
    w = S.gaussian_stencil(K, SIGMA)
    st = oracle.restrict_stencil(w.astype(np.float32).astype(np.float64), apr.l_max, apr.l_min).reshape(apr.n_levels, -1)
    gout = np.random.default_rng(0).normal(size=apr.n_particles)
    o = oracle.Oracle(apr)
    rng = np.random.default_rng(1)
    n = args.ref_sample

    def run(smp):
        o.conv(st, K, sample=smp)
        o.conv_backward(st, K, gout, sample=smp)

    est, wall = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        o.set_values(apr.values)
        o.tree()
        t_fill = time.perf_counter() - t0
        step_s, t_fixed, t_s = oracle_sampled_step(apr.n_particles, t_fill, run, n, rng)
        if i >= args.warmup:
            est.append(step_s)
            wall.append(t_fill + t_fixed + t_s)
    val = apr.n_particles / statistics.mean(est) / 1e9
    return {"metric": "APR conv Gparticles/s & pixel-equiv GB/s", "value": round(val, 9), "unit": "Gparticles/s",
            "impl": "reference", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * statistics.mean(wall), 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded 2000-blob image with Poisson noise -> APR)",
            "config": {"workload": "blob APR 1024x1024x512 pixels (z=512), 5^3 Gaussian sigma=1.5, restricted per-level stencils",
                       "step": f"oracle: full tree fill + forward and backward of {n} random output particles (and of 16, "
                               "for the part that does not depend on the sample); the whole step's time is estimated "
                               "as fill + fixed part + per-output time x N_p; ms_per_step is the sampled step's wall time"},
            "cpu_baseline": {"value": round(val, 9), "unit": "Gparticles/s", "cores": 1, "kind": "oracle",
                             "sample": f"{n} random output particles per step (plus the full tree fill)"},
            "e2e": {"value": round(val, 9), "unit": "Gparticles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_reference_mc(args, rank, world):
    """The oracle as the reference arm of the multi-channel workload (bounded sample per step)."""
    import numpy as np

    import aprsynth as S
    import oracle
    apr = S.make_config(MC_WORKLOAD)
    x, w, g = mc_inputs(apr)
    o = oracle.Oracle(apr, x)
    rng = np.random.default_rng(1)
    n = max(1, args.ref_sample // 10)

    def run(smp):
        o.conv(w, 3, sample=smp, C_out=MC_C)
        o.conv_backward(w, 3, g, sample=smp, C_out=MC_C)

    t_fill, t_samp, est = [], [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        o.set_values(x)
        o.tree_bf16()
        tf = time.perf_counter() - t0
        step_s, t_fixed, t_s = oracle_sampled_step(apr.n_particles, tf, run, n, rng)
        if i >= args.warmup:
            t_fill.append(tf)
            t_samp.append(t_fixed + t_s)
            est.append(step_s)
    val = apr.n_particles / statistics.mean(est) / 1e9
    return {"metric": "APR conv Gparticles/s & pixel-equiv GB/s", "value": round(val, 9), "unit": "Gparticles/s",
            "impl": "reference", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * (statistics.mean(t_fill) + statistics.mean(t_samp)), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded 400-blob 256^3 image with Poisson noise -> APR; random bf16 features and weights)",
            "config": {"workload": "blob APR 256^3 pixels, 16 -> 16 channels bf16 (FP32 accumulation), 3^3 per-level weights",
                       "step": f"oracle: full bf16 tree fill + 16-channel forward and backward of {n} random output "
                               "particles (and of 16, for the part that does not depend on the sample); the whole step's time "
                               "is estimated as fill + fixed part + per-output time x N_p"},
            "cpu_baseline": {"value": round(val, 9), "unit": "Gparticles/s", "cores": 1, "kind": "oracle",
                             "sample": f"{n} random output particles per step (plus the full bf16 tree fill)"},
            "e2e": {"value": round(val, 9), "unit": "Gparticles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_reference_rl(args, rank, world):
    """The oracle as the reference arm of the Richardson-Lucy workload (bounded sample per step)."""
    import numpy as np

    import aprsynth as S
    import oracle
    apr = S.make_config(RL_WORKLOAD)
    w = S.gaussian_stencil(K, SIGMA)
    W = oracle.restrict_stencil(w.astype(np.float32).astype(np.float64), apr.l_max, apr.l_min).reshape(apr.n_levels, -1)
    W_flip = W[:, ::-1].copy()
    o = oracle.Oracle(apr)
    rng = np.random.default_rng(1)
    n = max(1, args.ref_sample // 3)
    t_fill, t_samp = [], []
    for i in range(args.warmup + args.steps):
        s = np.sort(rng.choice(apr.n_particles, n, replace=False))
        t0 = time.perf_counter()
        o.set_values(apr.values)
        o.tree()
        t1 = time.perf_counter()
        o.conv(W, K, sample=s)
        o.conv(W_flip, K, sample=s)
        t2 = time.perf_counter()
        if i >= args.warmup:
            t_fill.append(t1 - t0)
            t_samp.append(t2 - t1)
    per = 2 * statistics.mean(t_fill) / apr.n_particles + statistics.mean(t_samp) / n
    val = 1.0 / per / 1e9
    unit = "Gparticles/s (particle-iterations of Richardson-Lucy; 2 convolutions each)"
    return {"metric": "APR conv Gparticles/s & pixel-equiv GB/s", "value": round(val, 9), "unit": unit,
            "impl": "reference", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * (statistics.mean(t_fill) + statistics.mean(t_samp)), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded 200-blob 512^3 image with Poisson noise -> APR)",
            "config": {"workload": "blob APR 512^3 pixels: 20 Richardson-Lucy iterations, restricted 5^3 Gaussian PSF sigma=1.5 and its flip",
                       "step": f"oracle: one iteration's tree fill (counted twice) + its two convolutions for {n} random "
                               "output particles; rate = particle-iterations per second"},
            "cpu_baseline": {"value": round(val, 9), "unit": unit, "cores": 1, "kind": "oracle",
                             "sample": f"{n} random output particles per step (plus the full tree fill)"},
            "e2e": {"value": round(val, 9), "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def ncu_launches(part, reps=3):
    """Runs one part of the default step `reps` times on the 1024x1024x512 APR (parts mc_*: of the
    multi-channel step on the 256^3 APR), for an ncu capture of that kernel (no timing); prints a
    one-line JSON note."""
    import numpy as np
    import torch

    import aprsynth as S
    import paper_2112_03592_gb300 as G
    if part.startswith("mc_"):
        apr = S.make_config(MC_WORKLOAD)
        lay = G.AprLayout.from_apr(apr, G.APR_VALIDATE | G.APR_REQUIRE_BALANCE)
        xh, wh, gh = mc_inputs(apr)
        bf = lambda a: torch.as_tensor(a.astype(np.float32), device="cuda").to(torch.bfloat16).contiguous()
        x, w, g = bf(xh), bf(wh), bf(gh)
        tree = G.apr_tree_restrict_bf16(lay, x)
        out = torch.empty((apr.n_particles, MC_C), device="cuda")
        gp = torch.empty((apr.n_particles, MC_C), device="cuda")
        gw = torch.empty((apr.n_levels, MC_C, MC_C, 27), device="cuda")
        run = {"mc_convolve": lambda: G.apr_convolve_mc(lay, x, tree, w, G.APR_BC_REFLECT, out),
               "mc_adjoint": lambda: G.apr_convolve_mc_backward(lay, x, tree, w, g, G.APR_BC_REFLECT,
                                                                need_weights=False, grad_particles=gp),
               "mc_wgrad": lambda: G.apr_convolve_mc_backward(lay, x, tree, w, g, G.APR_BC_REFLECT,
                                                              need_particles=False, grad_weights=gw)}[part]
        for _ in range(reps):
            run()
        torch.cuda.synchronize()
        lay.sync_status()
        print(json.dumps({"ncu_launches": part, "reps": reps, "workload": MC_WORKLOAD}))
        return
    apr = S.make_config(WORKLOAD)
    lay = G.AprLayout.from_apr(apr, G.APR_VALIDATE | G.APR_REQUIRE_BALANCE)
    w = S.gaussian_stencil(K, SIGMA).astype(np.float32)
    st = torch.as_tensor(G.apr_restrict_stencil(w, apr.l_max, apr.l_min), device="cuda")
    v = torch.as_tensor(apr.values, device="cuda")
    g = torch.as_tensor(np.random.default_rng(0).normal(size=apr.n_particles).astype(np.float32), device="cuda")
    tree = G.apr_tree_restrict(lay, v)
    gp, gt = torch.empty_like(v), torch.empty(lay.n_tree, device="cuda")
    run = {"restrict": lambda: G.apr_tree_restrict(lay, v, tree),
           "convolve": lambda: G.apr_convolve(lay, v, tree, st, K),
           "adjoint": lambda: G.apr_convolve_adjoint(lay, st, K, g, grad_particles=gp, grad_tree=gt),
           "stencil_grad": lambda: G.apr_convolve_stencil_grad(lay, v, tree, K, g)}[part]
    for _ in range(reps):
        run()
    torch.cuda.synchronize()
    lay.sync_status()
    print(json.dumps({"ncu_launches": part, "reps": reps, "workload": WORKLOAD}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--ref-sample", type=int, default=3000)
    ap.add_argument("--sur-train", type=int, default=8, help="surrogate: training APRs")
    ap.add_argument("--sur-steps", type=int, default=1500, help="surrogate: Adam steps")
    ap.add_argument("--sur-lr", type=float, default=2e-3, help="surrogate: learning rate")
    ap.add_argument("--sur-pretrained", action="store_true",
                    help="surrogate workload: evaluate the committed weights instead of training")
    ap.add_argument("--workload", default="blob1024", choices=["blob1024", "blob256_mc", "blob512_rl", "surrogate"],
                    help="blob1024: single-channel FP32 step (default); blob256_mc: 16-channel bf16 step; "
                         "blob512_rl: 20 Richardson-Lucy iterations")
    ap.add_argument("--no-mc", action="store_true", help="skip the multi-channel summary of the default line")
    ap.add_argument("--no-graph", action="store_true", help="launch eagerly instead of replaying CUDA graphs")
    ap.add_argument("--no-dense", action="store_true", help="skip the dense pixel convolution context timing")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain 5^3 (unrestricted) arm of the default line")
    ap.add_argument("--no-rl", action="store_true", help="skip the Richardson-Lucy summary of the default line")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate summary of the default line")
    ap.add_argument("--ncu-launches", choices=["restrict", "convolve", "adjoint", "stencil_grad", "mc_convolve", "mc_adjoint",
                                                    "mc_wgrad"],
                    help="run one part of the step 3 times for an ncu capture, no timing")
    args = ap.parse_args()
    if args.ncu_launches:
        ncu_launches(args.ncu_launches)
        return
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        fn = {"blob256_mc": run_reference_mc, "blob512_rl": run_reference_rl}.get(args.workload, run_reference)
        print(json.dumps(fn(args, rank, world)))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    if args.workload == "blob256_mc":
        rec = run_mc(args, rank, world, full=True)
    elif args.workload == "blob512_rl":
        rec = run_rl(args, rank, world, full=True)
    elif args.workload == "surrogate":
        rec = run_surrogate(args, rank, world, pretrained=SURROGATE_WEIGHTS if args.sur_pretrained else None)
    else:
        rec = run_ours(args, rank, world)
        if not args.no_mc:
            mc = run_mc(args, rank, world, full=False)
            rec["multichannel"] = {k: mc[k] for k in ("value", "unit", "ms_per_step", "dtype", "config", "step_ms_parts",
                                                      "roofline", "gpu_launches")}
        if not args.no_rl:
            rl = run_rl(args, rank, world, full=False)
            rec["rl"] = {k: rl[k] for k in ("value", "unit", "ms_per_step", "config", "roofline", "gpu_launches")}
        if not args.no_surrogate:
            if os.path.exists(SURROGATE_WEIGHTS):
                sr = run_surrogate(args, rank, world, pretrained=SURROGATE_WEIGHTS)
                rec["surrogate"] = {k: sr[k] for k in ("value", "unit", "config", "rl20_ms", "cnn_ms", "psnr_db",
                                                       "training", "gpu_launches")}
            else:
                rec["surrogate"] = {"unavailable": "no trained weights (run surrogate_weights/train.py)"}
    if rank == 0:
        print(json.dumps(rec))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
