"""APR-native CNN surrogate of an iterated APR filter (the learned per-level filters Sec. 6 proposes).

Architecture: the particle intensities x (float32) are embedded into 16 bfloat16 channels (channel 0
= bf16(scale * x)); n_layers APR convolutions 16 -> 16 with per-level 3^3 weights (apr_convolve_mc,
tensor cores, FP32 accumulation), each but the last followed by ReLU rounded to bf16; the output is
the residual y = x + c_last[:, 0] / scale. A level's weights are chosen by its distance to the finest
level, l_max - l (its cell edge 2^(l_max - l) pixels), so one model applies to APRs of any size.
Every step of inference runs in the library's kernels (trees, convolutions, activations, read-out and
their transposes); training (loss and Adam on float32 master weights, the gather of per-level
weights) uses torch tensor operations and is not part of the inference path.
"""
from __future__ import annotations

import math

from . import (apr_convolve_mc, apr_convolve_mc_backward, apr_convolve_mc_relu_bf16, apr_mc_embed_bf16, apr_mc_readout,
               apr_mc_readout_backward_bf16, apr_mc_relu_backward_bf16, apr_mc_relu_bf16, apr_tree_restrict_bf16)

C = 16


def _level_index(layout, n_dist):
    """Weight row of every level l_min..l_max: min(l_max - l, n_dist - 1)."""
    return [min(layout.l_max - l, n_dist - 1) for l in range(layout.l_min, layout.l_max + 1)]


class AprCnn:
    def __init__(self, n_layers: int = 4, n_dist: int = 8, seed: int = 0, device="cuda"):
        import torch
        g = torch.Generator(device="cpu").manual_seed(seed)
        std = math.sqrt(2.0 / (C * 27))
        self.W = []
        for i in range(n_layers):
            w = torch.randn((n_dist, C, C, 27), generator=g) * std
            if i == n_layers - 1:
                w *= 0.1    # near-identity start through the residual
            self.W.append(w.to(device).contiguous())
        self.n_layers, self.n_dist = n_layers, n_dist
        self._saved = None

    def stack_weights(self, layout):
        """Per-layer bf16 weight stacks [L][16][16][27] for the levels of `layout`."""
        import torch
        idx = torch.as_tensor(_level_index(layout, self.n_dist), device=self.W[0].device)
        return [w.index_select(0, idx).to(torch.bfloat16).contiguous() for w in self.W]

    def forward(self, layout, x, scale: float, keep: bool = False, weights=None):
        """y = x + c_last[:, 0] / scale (float32 [N]); keep=True saves what backward needs."""
        Wb = self.stack_weights(layout) if weights is None else weights
        h = apr_mc_embed_bf16(x, scale)
        saved = []
        c = None
        for i in range(self.n_layers):
            tree = apr_tree_restrict_bf16(layout, h)
            if not keep and i + 1 < self.n_layers:
                h = apr_convolve_mc_relu_bf16(layout, h, tree, Wb[i])   # inference: ReLU fused into the write
                continue
            c = apr_convolve_mc(layout, h, tree, Wb[i])
            if keep:
                saved.append((h, tree, c))
            if i + 1 < self.n_layers:
                h = apr_mc_relu_bf16(c)
        if keep:
            self._saved = (layout, scale, Wb, saved)
        return apr_mc_readout(c, x, 1.0 / scale)

    def backward(self, grad_y):
        """float32 gradients of the per-level weight stacks of the last kept forward (one [L][16][16][27]
        tensor per layer) for dL/dy = grad_y."""
        layout, scale, Wb, saved = self._saved
        g = apr_mc_readout_backward_bf16(grad_y, 1.0 / scale)
        grads = [None] * self.n_layers
        for i in reversed(range(self.n_layers)):
            h, tree, _ = saved[i]
            gp, gw = apr_convolve_mc_backward(layout, h, tree, Wb[i], g, need_particles=i > 0)
            grads[i] = gw
            if i > 0:
                g = apr_mc_relu_backward_bf16(saved[i - 1][2], gp)
        return grads


def train(model: AprCnn, samples, steps: int, lr: float = 1e-3, log_every: int = 0):
    """Adam on the float32 master weights. samples: list of (layout, x, target, scale), float32
    device tensors; loss = mean((scale * (y - target))^2). Returns the loss history."""
    import torch
    params = [torch.nn.Parameter(w) for w in model.W]
    opt = torch.optim.Adam(params, lr=lr)
    hist = []
    for it in range(steps):
        layout, x, t, scale = samples[it % len(samples)]
        model.W = [p.data for p in params]
        y = model.forward(layout, x, scale, keep=True)
        d = (y - t) * scale
        loss = float((d * d).mean())
        gy = (2.0 * scale / d.numel()) * d
        grads = model.backward(gy.contiguous())
        idx = torch.as_tensor(_level_index(layout, model.n_dist), device=params[0].device)
        for p, gr in zip(params, grads):
            p.grad = torch.zeros_like(p).index_add_(0, idx, gr)
        opt.step()
        hist.append(loss)
        if log_every and it % log_every == 0:
            print(f"step {it} loss {loss:.6f}", flush=True)
    model.W = [p.data for p in params]
    return hist


def psnr(a, ref, weights=None):
    """Peak signal-to-noise ratio of a against ref (max |ref| as the peak), optionally weighted
    (e.g. by the pixels each particle covers)."""
    d = (a.double() - ref.double()) ** 2
    if weights is not None:
        mse = float((d * weights).sum() / weights.sum())
    else:
        mse = float(d.mean())
    peak = float(ref.double().abs().max())
    return 10.0 * math.log10(peak * peak / max(mse, 1e-300))
