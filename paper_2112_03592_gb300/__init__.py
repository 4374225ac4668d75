"""APR-native discrete convolution on GB300 (sm_103a): Python binding of libaprconv.so.

Method: Jonsson et al., "Parallel Discrete Convolutions on Adaptive Particle Representations of
Images" (arXiv 2112.03592). The C ABI is declared in include/apr.h; the functions here marshal
torch tensors (device memory, current stream) into it and do no arithmetic of their own. The
library must be built (``__graft_entry__.build()``); a missing library raises, never falls back.

Functions with the C names:
    apr_build_device(dims, l_min, l_max, row_ptr, y_idx, flags)   -> AprLayout
    apr_tree_restrict(layout, particles[, tree])                  -> tree      (Sec. 3.4)
    apr_convolve(layout, particles, tree, stencils, k[, bc, out]) -> out       (Sec. 4.1)
    apr_convolve_backward(layout, particles, tree, stencils, k, grad_out[, bc])
                                                                  -> (grad_particles, grad_stencils)
      = apr_convolve_adjoint + apr_tree_restrict_adjoint + apr_convolve_stencil_grad
    apr_richardson_lucy(layout, observed, stencils, k, n_iter[, bc, estimate])
                                                                  -> estimate  (Sec. 6.2)
    apr_tree_restrict_bf16(layout, particles[, tree])             -> tree      (bf16, 16 channels)
    apr_convolve_mc(layout, particles, tree, weights[, bc, out])  -> out       (16 -> 16 channels, k = 3)
    apr_convolve_mc_backward(layout, particles, tree, weights, grad_out[, bc])
                                                                  -> (grad_particles, grad_weights)
    apr_gradient_magnitude(layout, particles, tree, stencils3, k) -> |grad|    (Sec. 4.3, with sobel_stencils)
    apr_restrict_stencil(w, l_max, l_min)                         -> [L][k^3]  (Eq. restrict_stenc)
    apr_rescale_stencil(w, l_max, l_min)                          -> [L][k^3]  (Eq. adapt_grad)
plus ``AprConv`` (torch.autograd.Function): particles, stencils -> per-particle outputs.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import (APR_BC_REFLECT, APR_BC_ZERO, APR_HOST_ONLY, APR_REQUIRE_BALANCE, APR_SUBDOMAIN,  # noqa: F401
                   APR_VALIDATE, AprError)

__all__ = ["AprLayout", "AprConv", "apr_build_device", "apr_tree_restrict", "apr_convolve", "apr_convolve_auto",
           "apr_convolve_backward", "apr_convolve_adjoint", "apr_tree_restrict_adjoint",
           "apr_tree_restrict_adjoint_levels",
           "apr_convolve_stencil_grad", "apr_gradient_magnitude", "sobel_stencils", "apr_richardson_lucy", "apr_tree_restrict_bf16", "apr_convolve_mc", "apr_convolve_mc_relu_bf16", "apr_convolve_mc_backward",
           "apr_mc_embed_bf16", "apr_mc_relu_bf16", "apr_mc_relu_backward_bf16", "apr_mc_readout",
           "apr_mc_readout_backward_bf16", "apr_restrict_stencil", "apr_rescale_stencil", "apr_dense_convolve", "apr_convolve_tiles",
           "apr_convolve_adjoint_tiles", "AprError",
           "APR_BC_REFLECT", "APR_BC_ZERO", "APR_VALIDATE", "APR_REQUIRE_BALANCE", "APR_HOST_ONLY",
           "APR_SUBDOMAIN"]


def _stream_ptr(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t, name, numel=None, dtype=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, has {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _torch_allocator():
    """apr_allocator callbacks backed by torch's CUDA caching allocator (stream-ordered on the
    build stream). Returns (struct, keep-alive objects)."""
    import torch

    def alloc(nbytes, stream, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                          stream if stream else 0))
        except Exception:  # out of memory: the library reports APR_ERR_OOM
            return None

    def free(ptr, nbytes, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    fa, ff = _abi.ALLOC_FN(alloc), _abi.FREE_FN(free)
    return _abi.AprAllocator(fa, ff, None), (fa, ff)


class AprLayout:
    """Owns an apr_handle_t: the device-resident index of one APR (particles + APR tree).

    allocator: None (the library allocates stream-ordered with cudaMallocAsync) or "torch" (the
    index lives in torch's caching allocator, through apr_build_device_ex's callbacks)."""

    def __init__(self, dims, l_min, l_max, row_ptr, y_idx,
                 flags=APR_VALIDATE | APR_REQUIRE_BALANCE, allocator=None):
        lib = _abi.load()
        self._row_ptr = np.ascontiguousarray(np.asarray(row_ptr, np.int64))
        self._y_idx = np.ascontiguousarray(np.asarray(y_idx, np.int32))
        L = _abi.AprHostLayout()
        L.l_min, L.l_max = int(l_min), int(l_max)
        for a in range(3):
            L.dims[a] = int(dims[a])
        L.row_ptr = self._row_ptr.ctypes.data_as(ctypes.c_void_p)
        L.y_idx = self._y_idx.ctypes.data_as(ctypes.c_void_p)
        L.n_particles = int(self._y_idx.size)
        h = ctypes.c_void_p()
        stream = ctypes.c_void_p(0)
        if not (flags & APR_HOST_ONLY):
            stream = _stream_ptr()
        self._alloc_keep = None
        if allocator is None:
            _abi.check("apr_build_device", lib.apr_build_device(ctypes.byref(L), flags, stream, ctypes.byref(h)))
        elif allocator == "torch":
            al, self._alloc_keep = _torch_allocator()
            self._alloc_struct = al
            _abi.check("apr_build_device_ex",
                       lib.apr_build_device_ex(ctypes.byref(L), flags, stream, ctypes.byref(al), ctypes.byref(h)))
        else:
            raise ValueError("allocator must be None or 'torch'")
        self._h = h
        self._lib = lib
        self.dims = tuple(int(d) for d in dims)
        self.l_min, self.l_max = int(l_min), int(l_max)
        self.n_particles = int(lib.apr_num_particles(h))
        self.n_tree = int(lib.apr_num_tree(h))
        self.host_only = bool(flags & APR_HOST_ONLY)
        self._ws = {}

    @classmethod
    def from_apr(cls, apr, flags=APR_VALIDATE | APR_REQUIRE_BALANCE, allocator=None):
        """From any object with dims, l_min, l_max, row_ptr, y_idx (e.g. aprsynth.AprInput)."""
        return cls(apr.dims, apr.l_min, apr.l_max, apr.row_ptr, apr.y_idx, flags, allocator)

    @property
    def n_levels(self):
        return self.l_max - self.l_min + 1

    @property
    def handle(self):
        return self._h

    def layout_bytes(self) -> int:
        return int(self._lib.apr_layout_bytes(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.apr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- structure export (bit-exact checks)
    _EXPORT_DTYPES = {0: np.uint32, 1: np.uint16, 2: np.uint32, 3: np.uint16, 4: np.int32, 5: np.int32, 6: np.int32,
                      7: np.int32, 8: np.uint32, 9: np.uint32, 10: np.uint32, 11: np.uint32}

    def export(self, which: int) -> np.ndarray:
        nbytes = int(self._lib.apr_structure_bytes(self._h, which))
        dt = self._EXPORT_DTYPES[which]
        out = np.zeros(max(nbytes // np.dtype(dt).itemsize, 1), dt)
        _abi.check("apr_export_structure",
                   self._lib.apr_export_structure(self._h, which, out.ctypes.data_as(ctypes.c_void_p), nbytes))
        out = out[:nbytes // np.dtype(dt).itemsize]
        if which == 7:
            return out.reshape(-1, 8)
        if which >= 8:
            return out.reshape(-1, 2)
        return out.reshape(-1, 4) if which in (4, 5, 6) else out

    def workspace(self, k):
        import torch
        nbytes = int(self._lib.apr_backward_workspace_bytes(self._h, k))
        ws = self._ws.get(k)
        if ws is None or ws.numel() < nbytes:
            ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device="cuda")
            self._ws[k] = ws
        return ws, nbytes

    def sync_status(self, stream=None):
        _abi.check("apr_sync_status", self._lib.apr_sync_status(self._h, _stream_ptr(stream)))


# ------------------------------------------------------------------------------------------------
# functions named as in the C ABI
# ------------------------------------------------------------------------------------------------
def apr_build_device(dims, l_min, l_max, row_ptr, y_idx, flags=APR_VALIDATE | APR_REQUIRE_BALANCE) -> AprLayout:
    return AprLayout(dims, l_min, l_max, row_ptr, y_idx, flags)


def apr_tree_restrict(layout: AprLayout, particles, tree=None, stream=None):
    import torch
    C = 1 if particles.dim() == 1 else int(particles.shape[1])
    _dev_ptr(particles, "particles", layout.n_particles * C, torch.float32)
    if tree is None:
        tree = torch.empty((layout.n_tree,) if C == 1 else (layout.n_tree, C), dtype=torch.float32, device=particles.device)
    _dev_ptr(tree, "tree", layout.n_tree * C, torch.float32)
    _abi.check("apr_tree_restrict", layout._lib.apr_tree_restrict(
        layout.handle, ctypes.c_void_p(particles.data_ptr()), ctypes.c_void_p(tree.data_ptr()), C, _stream_ptr(stream)))
    return tree


def apr_convolve(layout: AprLayout, particles, tree, stencils, k, bc=APR_BC_REFLECT, out=None, stream=None):
    import torch
    _dev_ptr(particles, "particles", layout.n_particles, torch.float32)
    _dev_ptr(tree, "tree", layout.n_tree, torch.float32)
    _dev_ptr(stencils, "stencils", layout.n_levels * k ** 3, torch.float32)
    if out is None:
        out = torch.empty(layout.n_particles, dtype=torch.float32, device=particles.device)
    _dev_ptr(out, "out", layout.n_particles, torch.float32)
    _abi.check("apr_convolve", layout._lib.apr_convolve(
        layout.handle, ctypes.c_void_p(particles.data_ptr()), ctypes.c_void_p(tree.data_ptr()),
        ctypes.c_void_p(stencils.data_ptr()), int(k), int(bc), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def apr_convolve_auto(layout: AprLayout, particles, stencils, k, bc=APR_BC_REFLECT, out=None, workspace=None,
                      stream=None):
    """Tree restriction into a workspace, then apr_convolve, in one call (the paper's forward
    pipeline); the workspace (at least N_t float32) holds the tree values afterwards."""
    import torch
    _dev_ptr(particles, "particles", layout.n_particles, torch.float32)
    _dev_ptr(stencils, "stencils", layout.n_levels * k ** 3, torch.float32)
    if out is None:
        out = torch.empty(layout.n_particles, dtype=torch.float32, device=particles.device)
    _dev_ptr(out, "out", layout.n_particles, torch.float32)
    nbytes = int(layout._lib.apr_convolve_auto_workspace_bytes(layout.handle))
    if workspace is None:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=particles.device)
    _abi.check("apr_convolve_auto", layout._lib.apr_convolve_auto(
        layout.handle, ctypes.c_void_p(particles.data_ptr()), ctypes.c_void_p(stencils.data_ptr()), int(k), int(bc),
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(workspace.data_ptr()), ctypes.c_size_t(workspace.numel() *
                                                                                         workspace.element_size()),
        _stream_ptr(stream)))
    return out


def apr_gradient_magnitude(layout: AprLayout, particles, tree, stencils3, k, bc=APR_BC_REFLECT, out=None, stream=None):
    """sqrt of the sum of squares of three convolutions (stencils3 [3][L][k^3], e.g. level-rescaled
    Sobel filters along z, x, y; Sec. 4.3)."""
    import torch
    _dev_ptr(particles, "particles", layout.n_particles, torch.float32)
    _dev_ptr(tree, "tree", layout.n_tree, torch.float32)
    _dev_ptr(stencils3, "stencils3", 3 * layout.n_levels * k ** 3, torch.float32)
    if out is None:
        out = torch.empty(layout.n_particles, dtype=torch.float32, device=particles.device)
    _dev_ptr(out, "out", layout.n_particles, torch.float32)
    _abi.check("apr_gradient_magnitude", layout._lib.apr_gradient_magnitude(
        layout.handle, ctypes.c_void_p(particles.data_ptr()), ctypes.c_void_p(tree.data_ptr()),
        ctypes.c_void_p(stencils3.data_ptr()), int(k), int(bc), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def apr_convolve_tiles(layout: AprLayout, particles, tree, stencils, k, first_tile, n_tiles, bc=APR_BC_REFLECT,
                       out=None, stream=None):
    """apr_convolve over the forward work items [first_tile, first_tile + n_tiles) only (the other
    entries of out are left as they are)."""
    import torch
    _dev_ptr(particles, "particles", layout.n_particles, torch.float32)
    _dev_ptr(tree, "tree", layout.n_tree, torch.float32)
    _dev_ptr(stencils, "stencils", layout.n_levels * k ** 3, torch.float32)
    if out is None:
        out = torch.zeros_like(particles)
    _dev_ptr(out, "out", layout.n_particles, torch.float32)
    _abi.check("apr_convolve_tiles", layout._lib.apr_convolve_tiles(
        layout.handle, _dev_ptr(particles, "particles"), _dev_ptr(tree, "tree"), _dev_ptr(stencils, "stencils"),
        int(k), int(bc), _dev_ptr(out, "out"), int(first_tile), int(n_tiles), _stream_ptr(stream)))
    return out


def apr_convolve_adjoint_tiles(layout: AprLayout, stencils, k, grad_out, grad_particles, grad_tree, first_tile,
                               n_tiles, bc=APR_BC_REFLECT, stream=None):
    """apr_convolve_adjoint over the data-adjoint work items [first_tile, first_tile + n_tiles): adds
    into grad_particles, writes the tiles' tree-node gradients into grad_tree (nothing is cleared)."""
    import torch
    _dev_ptr(grad_out, "grad_out", layout.n_particles, torch.float32)
    _dev_ptr(stencils, "stencils", layout.n_levels * k ** 3, torch.float32)
    _dev_ptr(grad_particles, "grad_particles", layout.n_particles, torch.float32)
    _dev_ptr(grad_tree, "grad_tree", layout.n_tree, torch.float32)
    _abi.check("apr_convolve_adjoint_tiles", layout._lib.apr_convolve_adjoint_tiles(
        layout.handle, _dev_ptr(stencils, "stencils"), int(k), int(bc), _dev_ptr(grad_out, "grad_out"),
        _dev_ptr(grad_particles, "grad_particles"), _dev_ptr(grad_tree, "grad_tree"), int(first_tile), int(n_tiles),
        _stream_ptr(stream)))
    return grad_particles, grad_tree


def apr_dense_convolve(image, stencil, k, bc=APR_BC_REFLECT, out=None, stream=None):
    """Dense pixel-grid correlation of a [dz][dx][dy] float32 image with one k^3 stencil (the
    dense comparison; not part of the APR path)."""
    import torch
    if image.dim() != 3:
        raise ValueError("image must be [dz][dx][dy]")
    _dev_ptr(image, "image", dtype=torch.float32)
    _dev_ptr(stencil, "stencil", k ** 3, torch.float32)
    if out is None:
        out = torch.empty_like(image)
    _dev_ptr(out, "out", image.numel(), torch.float32)
    dz, dx, dy = (int(d) for d in image.shape)
    _abi.check("apr_dense_convolve", _abi.load().apr_dense_convolve(
        _dev_ptr(image, "image"), dz, dx, dy, _dev_ptr(stencil, "stencil"), int(k), int(bc),
        _dev_ptr(out, "out"), _stream_ptr(stream)))
    return out


def sobel_stencils(k=3):
    """Sobel derivative stencils [3][k][k][k] along z, x, y (apr_sobel_stencils: central difference
    along the axis, [1, 2, 1] / 4 smoothing across it, so a linear ramp of slope 1 gives 1)."""
    lib = _abi.load()
    out = np.zeros((3, k, k, k), np.float32)
    _abi.check("apr_sobel_stencils", lib.apr_sobel_stencils(int(k), out.ctypes.data_as(ctypes.c_void_p)))
    return out


def apr_convolve_backward(layout: AprLayout, particles, tree, stencils, k, grad_out, bc=APR_BC_REFLECT,
                          need_particles=True, need_stencils=True, grad_particles=None, grad_stencils=None,
                          stream=None):
    import torch
    _dev_ptr(grad_out, "grad_out", layout.n_particles, torch.float32)
    _dev_ptr(stencils, "stencils", layout.n_levels * k ** 3, torch.float32)
    gp_ptr = gw_ptr = ctypes.c_void_p(0)
    if need_particles:
        if grad_particles is None:
            grad_particles = torch.empty(layout.n_particles, dtype=torch.float32, device=grad_out.device)
        gp_ptr = _dev_ptr(grad_particles, "grad_particles", layout.n_particles, torch.float32)
    if need_stencils:
        _dev_ptr(particles, "particles", layout.n_particles, torch.float32)
        _dev_ptr(tree, "tree", layout.n_tree, torch.float32)
        if grad_stencils is None:
            grad_stencils = torch.empty((layout.n_levels, k ** 3), dtype=torch.float32, device=grad_out.device)
        gw_ptr = _dev_ptr(grad_stencils, "grad_stencils", layout.n_levels * k ** 3, torch.float32)
    ws, nbytes = layout.workspace(k)
    _abi.check("apr_convolve_backward", layout._lib.apr_convolve_backward(
        layout.handle, ctypes.c_void_p(particles.data_ptr() if particles is not None else 0),
        ctypes.c_void_p(tree.data_ptr() if tree is not None else 0), ctypes.c_void_p(stencils.data_ptr()),
        int(k), int(bc), ctypes.c_void_p(grad_out.data_ptr()), gp_ptr, gw_ptr,
        ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel()), _stream_ptr(stream)))
    return (grad_particles if need_particles else None), (grad_stencils if need_stencils else None)


def apr_convolve_adjoint(layout: AprLayout, stencils, k, grad_out, bc=APR_BC_REFLECT, grad_particles=None,
                         grad_tree=None, stream=None):
    """(grad_particles, grad_tree): transpose of apr_convolve w.r.t. particle and tree values."""
    import torch
    _dev_ptr(grad_out, "grad_out", layout.n_particles, torch.float32)
    _dev_ptr(stencils, "stencils", layout.n_levels * k ** 3, torch.float32)
    if grad_particles is None:
        grad_particles = torch.empty(layout.n_particles, dtype=torch.float32, device=grad_out.device)
    if grad_tree is None:
        grad_tree = torch.empty(layout.n_tree, dtype=torch.float32, device=grad_out.device)
    _abi.check("apr_convolve_adjoint", layout._lib.apr_convolve_adjoint(
        layout.handle, _dev_ptr(stencils, "stencils"), int(k), int(bc), _dev_ptr(grad_out, "grad_out"),
        _dev_ptr(grad_particles, "grad_particles", layout.n_particles, torch.float32),
        _dev_ptr(grad_tree, "grad_tree", layout.n_tree, torch.float32), _stream_ptr(stream)))
    return grad_particles, grad_tree


def apr_tree_restrict_adjoint(layout: AprLayout, grad_tree, grad_particles, stream=None):
    """Push tree gradients down to the particles (adds into grad_particles; grad_tree is updated)."""
    import torch
    _abi.check("apr_tree_restrict_adjoint", layout._lib.apr_tree_restrict_adjoint(
        layout.handle, _dev_ptr(grad_tree, "grad_tree", layout.n_tree, torch.float32),
        _dev_ptr(grad_particles, "grad_particles", layout.n_particles, torch.float32), _stream_ptr(stream)))
    return grad_particles


def apr_tree_restrict_adjoint_levels(layout: AprLayout, grad_tree, grad_particles, level_first, level_last,
                                     stream=None):
    """apr_tree_restrict_adjoint over the tree levels [level_first, level_last] only, coarsest first
    (after tree level t the particles of level t + 1 hold their final gradient)."""
    import torch
    _abi.check("apr_tree_restrict_adjoint_levels", layout._lib.apr_tree_restrict_adjoint_levels(
        layout.handle, _dev_ptr(grad_tree, "grad_tree", layout.n_tree, torch.float32),
        _dev_ptr(grad_particles, "grad_particles", layout.n_particles, torch.float32), int(level_first),
        int(level_last), _stream_ptr(stream)))
    return grad_particles


def apr_convolve_stencil_grad(layout: AprLayout, particles, tree, k, grad_out, bc=APR_BC_REFLECT,
                              grad_stencils=None, stream=None):
    """dL/d stencils [L][k^3] for dL/d out = grad_out."""
    import torch
    if grad_stencils is None:
        grad_stencils = torch.empty((layout.n_levels, k ** 3), dtype=torch.float32, device=grad_out.device)
    nbytes = int(layout._lib.apr_stencil_grad_workspace_bytes(layout.handle, k))
    key = ("sg", k)
    ws = layout._ws.get(key)
    if ws is None or ws.numel() < nbytes:
        ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=grad_out.device)
        layout._ws[key] = ws
    _abi.check("apr_convolve_stencil_grad", layout._lib.apr_convolve_stencil_grad(
        layout.handle, _dev_ptr(particles, "particles", layout.n_particles, torch.float32),
        _dev_ptr(tree, "tree", layout.n_tree, torch.float32), int(k), int(bc),
        _dev_ptr(grad_out, "grad_out", layout.n_particles, torch.float32),
        _dev_ptr(grad_stencils, "grad_stencils", layout.n_levels * k ** 3, torch.float32),
        ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel()), _stream_ptr(stream)))
    return grad_stencils


def apr_richardson_lucy(layout: AprLayout, observed, stencils, k, n_iter, bc=APR_BC_REFLECT, estimate=None,
                        stream=None):
    """n_iter Richardson-Lucy updates i <- i * ((u / (i conv w)) conv w_flip) (Sec. 6.2) on the APR;
    i_0 = observed unless `estimate` (updated in place) is given."""
    import torch
    _dev_ptr(observed, "observed", layout.n_particles, torch.float32)
    _dev_ptr(stencils, "stencils", layout.n_levels * k ** 3, torch.float32)
    if estimate is None:
        estimate = observed.clone()
    _dev_ptr(estimate, "estimate", layout.n_particles, torch.float32)
    nbytes = int(layout._lib.apr_rl_workspace_bytes(layout.handle))
    key = ("rl",)
    ws = layout._ws.get(key)
    if ws is None or ws.numel() < nbytes:
        ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=observed.device)
        layout._ws[key] = ws
    _abi.check("apr_richardson_lucy", layout._lib.apr_richardson_lucy(
        layout.handle, ctypes.c_void_p(observed.data_ptr()), ctypes.c_void_p(stencils.data_ptr()), int(k), int(bc),
        int(n_iter), ctypes.c_void_p(estimate.data_ptr()), ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel()),
        _stream_ptr(stream)))
    return estimate


# ---- multi-channel, bfloat16 features (16 channels, k = 3)
MC_CHANNELS = 16


def apr_tree_restrict_bf16(layout: AprLayout, particles, tree=None, stream=None):
    """BF16 tree [N_t][16] of particles [N_p][16] (FP32 averages rounded to bf16, level by level)."""
    import torch
    C = int(particles.shape[1])
    _dev_ptr(particles, "particles", layout.n_particles * C, torch.bfloat16)
    if tree is None:
        tree = torch.empty((layout.n_tree, C), dtype=torch.bfloat16, device=particles.device)
    _dev_ptr(tree, "tree", layout.n_tree * C, torch.bfloat16)
    _abi.check("apr_tree_restrict_bf16", layout._lib.apr_tree_restrict_bf16(
        layout.handle, ctypes.c_void_p(particles.data_ptr()), ctypes.c_void_p(tree.data_ptr()), C, _stream_ptr(stream)))
    return tree


def apr_convolve_mc(layout: AprLayout, particles, tree, weights, bc=APR_BC_REFLECT, out=None, stream=None):
    """out[p][co] (float32) = sum_ci sum_e weights[l][co][ci][e] * u_l(...)[ci]; bf16 inputs."""
    import torch
    C = MC_CHANNELS
    k = 3
    _dev_ptr(particles, "particles", layout.n_particles * C, torch.bfloat16)
    _dev_ptr(tree, "tree", layout.n_tree * C, torch.bfloat16)
    _dev_ptr(weights, "weights", layout.n_levels * C * C * k ** 3, torch.bfloat16)
    if out is None:
        out = torch.empty((layout.n_particles, C), dtype=torch.float32, device=particles.device)
    _dev_ptr(out, "out", layout.n_particles * C, torch.float32)
    _abi.check("apr_convolve_mc", layout._lib.apr_convolve_mc(
        layout.handle, ctypes.c_void_p(particles.data_ptr()), ctypes.c_void_p(tree.data_ptr()),
        ctypes.c_void_p(weights.data_ptr()), C, C, k, int(bc), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def apr_convolve_mc_relu_bf16(layout: AprLayout, particles, tree, weights, bc=APR_BC_REFLECT, out=None, stream=None):
    """bf16(max(apr_convolve_mc(...), 0)) [N_p][16]: a hidden CNN layer with the ReLU fused (inference)."""
    import torch
    C = MC_CHANNELS
    k = 3
    _dev_ptr(particles, "particles", layout.n_particles * C, torch.bfloat16)
    _dev_ptr(tree, "tree", layout.n_tree * C, torch.bfloat16)
    _dev_ptr(weights, "weights", layout.n_levels * C * C * k ** 3, torch.bfloat16)
    if out is None:
        out = torch.empty((layout.n_particles, C), dtype=torch.bfloat16, device=particles.device)
    _dev_ptr(out, "out", layout.n_particles * C, torch.bfloat16)
    _abi.check("apr_convolve_mc_relu_bf16", layout._lib.apr_convolve_mc_relu_bf16(
        layout.handle, ctypes.c_void_p(particles.data_ptr()), ctypes.c_void_p(tree.data_ptr()),
        ctypes.c_void_p(weights.data_ptr()), C, C, k, int(bc), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def apr_convolve_mc_backward(layout: AprLayout, particles, tree, weights, grad_out, bc=APR_BC_REFLECT,
                             need_particles=True, need_weights=True, grad_particles=None, grad_weights=None,
                             stream=None):
    """(grad_particles [N_p][16] float32, grad_weights [L][16][16][27] float32); grad_out is bf16."""
    import torch
    C = MC_CHANNELS
    k = 3
    _dev_ptr(grad_out, "grad_out", layout.n_particles * C, torch.bfloat16)
    _dev_ptr(weights, "weights", layout.n_levels * C * C * k ** 3, torch.bfloat16)
    gp_ptr = gw_ptr = ctypes.c_void_p(0)
    if need_particles:
        if grad_particles is None:
            grad_particles = torch.empty((layout.n_particles, C), dtype=torch.float32, device=grad_out.device)
        gp_ptr = _dev_ptr(grad_particles, "grad_particles", layout.n_particles * C, torch.float32)
    if need_weights:
        _dev_ptr(particles, "particles", layout.n_particles * C, torch.bfloat16)
        _dev_ptr(tree, "tree", layout.n_tree * C, torch.bfloat16)
        if grad_weights is None:
            grad_weights = torch.empty((layout.n_levels, C, C, k ** 3), dtype=torch.float32, device=grad_out.device)
        gw_ptr = _dev_ptr(grad_weights, "grad_weights", layout.n_levels * C * C * k ** 3, torch.float32)
    nbytes = int(layout._lib.apr_mc_backward_workspace_bytes(layout.handle, C, C, k))
    key = ("mc", k)
    ws = layout._ws.get(key)
    if ws is None or ws.numel() < nbytes:
        ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=grad_out.device)
        layout._ws[key] = ws
    _abi.check("apr_convolve_mc_backward", layout._lib.apr_convolve_mc_backward(
        layout.handle, ctypes.c_void_p(particles.data_ptr() if particles is not None else 0),
        ctypes.c_void_p(tree.data_ptr() if tree is not None else 0), ctypes.c_void_p(weights.data_ptr()),
        C, C, k, int(bc), ctypes.c_void_p(grad_out.data_ptr()), gp_ptr, gw_ptr,
        ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel()), _stream_ptr(stream)))
    return (grad_particles if need_particles else None), (grad_weights if need_weights else None)


# ---- element-wise layers of the APR CNN (16 channels)
def apr_mc_embed_bf16(x, scale, out=None, stream=None):
    import torch
    n = int(x.numel())
    _dev_ptr(x, "x", n, torch.float32)
    if out is None:
        out = torch.empty((n, MC_CHANNELS), dtype=torch.bfloat16, device=x.device)
    _dev_ptr(out, "out", n * MC_CHANNELS, torch.bfloat16)
    _abi.check("apr_mc_embed_bf16", _abi.load().apr_mc_embed_bf16(
        ctypes.c_void_p(x.data_ptr()), n, float(scale), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def apr_mc_relu_bf16(inp, out=None, stream=None):
    import torch
    n = int(inp.numel())
    _dev_ptr(inp, "in", n, torch.float32)
    if out is None:
        out = torch.empty(inp.shape, dtype=torch.bfloat16, device=inp.device)
    _dev_ptr(out, "out", n, torch.bfloat16)
    _abi.check("apr_mc_relu_bf16", _abi.load().apr_mc_relu_bf16(
        ctypes.c_void_p(inp.data_ptr()), n, ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def apr_mc_relu_backward_bf16(pre, grad_post, out=None, stream=None):
    import torch
    n = int(pre.numel())
    _dev_ptr(pre, "pre", n, torch.float32)
    _dev_ptr(grad_post, "grad_post", n, torch.float32)
    if out is None:
        out = torch.empty(pre.shape, dtype=torch.bfloat16, device=pre.device)
    _dev_ptr(out, "grad_pre", n, torch.bfloat16)
    _abi.check("apr_mc_relu_backward_bf16", _abi.load().apr_mc_relu_backward_bf16(
        ctypes.c_void_p(pre.data_ptr()), ctypes.c_void_p(grad_post.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
        _stream_ptr(stream)))
    return out


def apr_mc_readout(conv, x, inv_scale, out=None, stream=None):
    import torch
    n = int(x.numel())
    _dev_ptr(conv, "conv", n * MC_CHANNELS, torch.float32)
    _dev_ptr(x, "x", n, torch.float32)
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=x.device)
    _dev_ptr(out, "y", n, torch.float32)
    _abi.check("apr_mc_readout", _abi.load().apr_mc_readout(
        ctypes.c_void_p(conv.data_ptr()), ctypes.c_void_p(x.data_ptr()), n, float(inv_scale),
        ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def apr_mc_readout_backward_bf16(grad_y, inv_scale, out=None, stream=None):
    import torch
    n = int(grad_y.numel())
    _dev_ptr(grad_y, "grad_y", n, torch.float32)
    if out is None:
        out = torch.empty((n, MC_CHANNELS), dtype=torch.bfloat16, device=grad_y.device)
    _dev_ptr(out, "grad_conv", n * MC_CHANNELS, torch.bfloat16)
    _abi.check("apr_mc_readout_backward_bf16", _abi.load().apr_mc_readout_backward_bf16(
        ctypes.c_void_p(grad_y.data_ptr()), n, float(inv_scale), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def _stencil_stack(fn_name, w, l_max, l_min):
    lib = _abi.load()
    w = np.ascontiguousarray(np.asarray(w, np.float32))
    k = w.shape[0]
    if w.shape != (k, k, k):
        raise ValueError("stencil must be k x k x k")
    out = np.zeros((l_max - l_min + 1, k ** 3), np.float32)
    _abi.check(fn_name, getattr(lib, fn_name)(w.ctypes.data_as(ctypes.c_void_p), k, int(l_max), int(l_min),
                                              out.ctypes.data_as(ctypes.c_void_p)))
    return out


def apr_restrict_stencil(w, l_max, l_min) -> np.ndarray:
    return _stencil_stack("apr_restrict_stencil", w, l_max, l_min)


def apr_rescale_stencil(w, l_max, l_min) -> np.ndarray:
    return _stencil_stack("apr_rescale_stencil", w, l_max, l_min)


# ------------------------------------------------------------------------------------------------
# autograd
# ------------------------------------------------------------------------------------------------
def _autograd_function():
    import torch

    class _AprConv(torch.autograd.Function):
        """out = apr_convolve(restrict(particles), stencils); gradients through both (Sec. 6 outlook)."""

        @staticmethod
        def forward(ctx, particles, stencils, layout, k, bc):
            particles = particles.contiguous()
            stencils = stencils.contiguous()
            tree = apr_tree_restrict(layout, particles)
            out = apr_convolve(layout, particles, tree, stencils, k, bc)
            ctx.save_for_backward(particles, tree, stencils)
            ctx.layout, ctx.k, ctx.bc = layout, k, bc
            return out

        @staticmethod
        def backward(ctx, grad_out):
            particles, tree, stencils = ctx.saved_tensors
            gp, gw = apr_convolve_backward(ctx.layout, particles, tree, stencils, ctx.k, grad_out.contiguous(), ctx.bc,
                                           need_particles=ctx.needs_input_grad[0],
                                           need_stencils=ctx.needs_input_grad[1])
            if gw is not None:
                gw = gw.view_as(stencils)
            return gp, gw, None, None, None

    return _AprConv


class AprConv:
    """AprConv.apply(particles, stencils, layout, k, bc=APR_BC_REFLECT) -> per-particle outputs."""
    _fn = None

    @classmethod
    def apply(cls, particles, stencils, layout, k, bc=APR_BC_REFLECT):
        if cls._fn is None:
            cls._fn = _autograd_function()
        return cls._fn.apply(particles, stencils, layout, k, bc)
