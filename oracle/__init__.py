"""FP64 CPU oracle of APR-native convolution (arXiv 2112.03592) -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg may import this
package. The product (paper_2112_03592_gb300 and its CUDA library) never imports it, and this
package never imports the product: the two share no code. The only shared module is `aprsynth`,
which makes seeded inputs and holds none of the method's arithmetic.

Contents
  apr_oracle.c     the plain FP64 definition: APR tree (Sec. 3.4), isotropic patch values
                   (Sec. 3.5), APR convolution (Sec. 4.1), its transpose, and the coarse-fill
                   property the convolution relies on (Sec. 5.1 footnote).
  restrict_stencil the restricted stencils w_l of Eq. (restrict_stenc), K_{w_l} = R_l K_w P_l,
                   formed from explicit 1-D restriction / prolongation / shift matrices.

Every function is pinned by tests/test_oracle_*.py against brute force, closed forms, library
routines (scipy.ndimage) and hand-derived values under tests/golden/.
"""
from __future__ import annotations

import ctypes
import os
import pathlib
import subprocess

import numpy as np

_HERE = pathlib.Path(__file__).resolve().parent
_SO = _HERE / "_build" / "liboracle.so"
_lib = None


def build(force: bool = False) -> pathlib.Path:
    """Compile apr_oracle.c with the host C compiler (portable flags only)."""
    src = _HERE / "apr_oracle.c"
    if force or not _SO.exists() or _SO.stat().st_mtime < src.stat().st_mtime:
        _SO.parent.mkdir(parents=True, exist_ok=True)
        tmp = _SO.with_suffix(f".{os.getpid()}.tmp")
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-o", str(tmp), str(src), "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(str(_SO))
        P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        lib.ora_create.restype = P
        lib.ora_create.argtypes = [I32, I32, P, P, P, I64, P, I32]
        lib.ora_destroy.argtypes = [P]
        lib.ora_num_tree.restype = I64
        lib.ora_num_tree.argtypes = [P]
        lib.ora_error.restype = I32
        lib.ora_error.argtypes = [P]
        lib.ora_tree_coords.argtypes = [P, P]
        lib.ora_tree_layout.argtypes = [P, P, P]
        lib.ora_tree_fill.restype = I32
        lib.ora_tree_fill.argtypes = [P]
        lib.ora_get_tree.argtypes = [P, D]
        lib.ora_set_values.argtypes = [P, D]
        lib.ora_conv.restype = I32
        lib.ora_conv.argtypes = [P, D, I32, I32, I32, P, I64, D]
        lib.ora_conv_backward.restype = I32
        lib.ora_conv_backward.argtypes = [P, D, I32, I32, I32, D, P, I64, D, D]
        lib.ora_conv_backward_direct.restype = I32
        lib.ora_conv_backward_direct.argtypes = [P, D, I32, I32, I32, D, P, I64, D, D, D]
        lib.ora_tree_transpose.restype = I32
        lib.ora_tree_transpose.argtypes = [P, D, D]
        lib.ora_set_tree.argtypes = [P, D]
        lib.ora_check_coarse_fill.restype = I64
        lib.ora_check_coarse_fill.argtypes = [P, I32]
        lib.ora_tree_fill_bf16.restype = I32
        lib.ora_tree_fill_bf16.argtypes = [P]
        lib.ora_round_bf16.restype = ctypes.c_double
        lib.ora_round_bf16.argtypes = [ctypes.c_double]
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


BC_REFLECT, BC_ZERO = 0, 1


def round_bf16(v: float) -> float:
    """The oracle's bfloat16 rounding (nearest, ties to even) of one value."""
    return float(_load().ora_round_bf16(float(v)))


class Oracle:
    """The oracle's view of one APR: its own index, its own tree, FP64 values [N][C]."""

    def __init__(self, apr, values=None):
        lib = _load()
        self.apr = apr
        vals = apr.values if values is None else values
        vals = np.ascontiguousarray(np.asarray(vals, dtype=np.float64))
        if vals.ndim == 1:
            vals = vals[:, None]
        self.C = vals.shape[1]
        self._vals = vals
        self._keep = [np.ascontiguousarray(np.asarray(apr.dims, np.int64)),
                      np.ascontiguousarray(apr.row_ptr.astype(np.int64)),
                      np.ascontiguousarray(apr.y_idx.astype(np.int32))]
        self.h = lib.ora_create(apr.l_min, apr.l_max, _ptr(self._keep[0]), _ptr(self._keep[1]),
                                _ptr(self._keep[2]), apr.n_particles, _ptr(vals), self.C)
        if not self.h:
            raise ValueError("oracle: bad arguments")
        self.n_tree = int(lib.ora_num_tree(self.h))
        self._filled = False

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ora_destroy(self.h)
            self.h = None

    @property
    def error(self) -> int:
        return int(_load().ora_error(self.h))

    # ---- structure
    def tree_coords(self) -> np.ndarray:
        out = np.zeros((self.n_tree, 4), np.int32)
        _load().ora_tree_coords(self.h, _ptr(out))
        return out

    def tree_layout(self):
        """(row_ptr int64 [R_t+1], y_idx int32 [N_t]) of the tree, rows of levels l_min..l_max-1."""
        a = self.apr
        rows = sum(a.level_dims(l)[0] * a.level_dims(l)[1] for l in range(a.l_min, a.l_max))
        rp = np.zeros(rows + 1, np.int64)
        yi = np.zeros(max(self.n_tree, 1), np.int32)
        _load().ora_tree_layout(self.h, _ptr(rp), _ptr(yi))
        return rp, yi[:self.n_tree]

    # ---- values
    def set_values(self, values):
        v = np.ascontiguousarray(np.asarray(values, np.float64).reshape(self.apr.n_particles, self.C))
        _load().ora_set_values(self.h, _ptr(v))
        self._vals = v
        self._filled = False

    def tree(self) -> np.ndarray:
        """Tree values [N_t][C] (Sec. 3.4: average of children, finest level first)."""
        lib = _load()
        if not self._filled:
            rc = lib.ora_tree_fill(self.h)
            if rc:
                raise ValueError(f"oracle: invalid APR (tree fill error {rc})")
            self._filled = True
        out = np.zeros((max(self.n_tree, 1), self.C), np.float64)
        lib.ora_get_tree(self.h, _ptr(out))
        return out[:self.n_tree]

    def tree_bf16(self) -> np.ndarray:
        """Tree values [N_t][C] for bfloat16 features with FP32 accumulation: per node and channel,
        the FP32 sum of the in-grid children in (dz, dx, dy) order divided by their count in FP32,
        rounded to bfloat16 (nearest, ties to even) before the next coarser level uses it. The
        particle values must be bfloat16 numbers. Later conv() / conv_backward() calls use them."""
        lib = _load()
        v32 = self._vals.astype(np.float32)
        if not (np.all(v32.astype(np.float64) == self._vals) and np.all((v32.view(np.uint32) & 0xFFFF) == 0)):
            raise ValueError("oracle: tree_bf16 needs particle values that are bfloat16 numbers")
        rc = lib.ora_tree_fill_bf16(self.h)
        if rc:
            raise ValueError(f"oracle: invalid APR (tree fill error {rc})")
        self._filled = True
        out = np.zeros((max(self.n_tree, 1), self.C), np.float64)
        lib.ora_get_tree(self.h, _ptr(out))
        return out[:self.n_tree]

    def _stencils(self, stencils, k, C_out):
        L = self.apr.n_levels
        W = np.ascontiguousarray(np.asarray(stencils, np.float64).reshape(L, C_out, self.C, k ** 3))
        return W

    def conv(self, stencils, k, bc=BC_REFLECT, sample=None, C_out=1) -> np.ndarray:
        """APR convolution outputs [ns][C_out] (Sec. 4.1) for `sample` particle ids (all if None)."""
        self.tree()
        W = self._stencils(stencils, k, C_out)
        if sample is None:
            ns, sp = self.apr.n_particles, None
        else:
            s = np.ascontiguousarray(np.asarray(sample, np.int64))
            ns, sp = s.size, s
        out = np.zeros((max(ns, 1), C_out), np.float64)
        rc = _load().ora_conv(self.h, _ptr(W), k, C_out, bc, _ptr(sp) if sp is not None else None, ns, _ptr(out))
        if rc:
            raise ValueError(f"oracle: stencil tap without a source (code {rc})")
        return out[:ns]

    def conv_backward(self, stencils, k, grad_out, bc=BC_REFLECT, C_out=1, sample=None):
        """(dL/d particles [N][C], dL/d stencils [L][C_out][C][k^3]) for dL/d out = grad_out.

        With `sample`, only the listed outputs contribute (their grad_out rows are used)."""
        self.tree()
        W = self._stencils(stencils, k, C_out)
        G = np.ascontiguousarray(np.asarray(grad_out, np.float64).reshape(self.apr.n_particles, C_out))
        gp = np.zeros((max(self.apr.n_particles, 1), self.C), np.float64)
        gw = np.zeros(W.shape, np.float64)
        sp = None if sample is None else np.ascontiguousarray(np.asarray(sample, np.int64))
        rc = _load().ora_conv_backward(self.h, _ptr(W), k, C_out, bc, _ptr(G),
                                       _ptr(sp) if sp is not None else None, 0 if sp is None else sp.size,
                                       _ptr(gp), _ptr(gw))
        if rc:
            raise ValueError(f"oracle: invalid APR in backward (code {rc})")
        return gp[:self.apr.n_particles], gw

    def set_tree(self, tree):
        """Use the given tree values [N_t][C] (instead of filling them from the particles)."""
        t = np.ascontiguousarray(np.asarray(tree, np.float64).reshape(self.n_tree, self.C))
        if self.n_tree:
            _load().ora_set_tree(self.h, _ptr(t))
        self._filled = True

    def conv_backward_parts(self, stencils, k, grad_out, bc=BC_REFLECT, C_out=1, sample=None):
        """The backward's two linear parts: (dL/d particles through particle sources [N][C], dL/d tree
        nodes through tree sources [N_t][C], dL/d stencils). conv_backward adds
        tree_transpose(the second) to the first."""
        self.tree()
        W = self._stencils(stencils, k, C_out)
        G = np.ascontiguousarray(np.asarray(grad_out, np.float64).reshape(self.apr.n_particles, C_out))
        gp = np.zeros((max(self.apr.n_particles, 1), self.C), np.float64)
        gt = np.zeros((max(self.n_tree, 1), self.C), np.float64)
        gw = np.zeros(W.shape, np.float64)
        sp = None if sample is None else np.ascontiguousarray(np.asarray(sample, np.int64))
        rc = _load().ora_conv_backward_direct(self.h, _ptr(W), k, C_out, bc, _ptr(G),
                                              _ptr(sp) if sp is not None else None, 0 if sp is None else sp.size,
                                              _ptr(gp), _ptr(gt), _ptr(gw))
        if rc:
            raise ValueError(f"oracle: invalid APR in backward (code {rc})")
        return gp[:self.apr.n_particles], gt[:self.n_tree], gw

    def tree_transpose(self, grad_tree):
        """Particle shares [N][C] of a tree gradient [N_t][C] (transpose of the tree averages)."""
        gt = np.ascontiguousarray(np.asarray(grad_tree, np.float64).reshape(max(self.n_tree, 1), self.C))
        gp = np.zeros((max(self.apr.n_particles, 1), self.C), np.float64)
        rc = _load().ora_tree_transpose(self.h, _ptr(gt), _ptr(gp))
        if rc:
            raise ValueError(f"oracle: invalid APR in tree transpose (code {rc})")
        return gp[:self.apr.n_particles]

    def check_coarse_fill(self, r: int) -> int:
        return int(_load().ora_check_coarse_fill(self.h, r))


# --------------------------------------------------------------------------------------------
# restricted stencils, Eq. (restrict_stenc): K_{w_l} u_l = R_l K_w P_l u_l
# --------------------------------------------------------------------------------------------
def _shift_restrict_1d(s: int, d: int, n_c: int) -> np.ndarray:
    """(R S_d P) for a 1-D grid of n_c coarse cells of s fine cells each.

    P (n_f x n_c): piecewise-constant prolongation, P[i, j] = [i // s == j].
    S_d (n_f x n_f): shift, (S_d u)[i] = u[i + d] (zero outside).
    R (n_c x n_f): block average, R = P^T / s.
    """
    n_f = n_c * s
    P = np.zeros((n_f, n_c))
    P[np.arange(n_f), np.arange(n_f) // s] = 1.0
    SP = np.zeros_like(P)
    src = np.arange(n_f) + d
    ok = (src >= 0) & (src < n_f)
    SP[ok] = P[src[ok]]
    R = P.T / s
    return R @ SP


def restrict_stencil(w: np.ndarray, l_max: int, l_min: int) -> np.ndarray:
    """Per-level stencils [L][k][k][k] (level l_min first) with w_l = R_l K_w P_l (FP64).

    K_w = sum_d w[d] S_dz (x) S_dx (x) S_dy, and R, P act per axis, so
    R K_w P = sum_d w[d] (R S_dz P) (x) (R S_dx P) (x) (R S_dy P); the coarse stencil is the row of
    this Toeplitz operator at an interior coarse cell. Each 1-D factor is formed as an explicit
    matrix product on a small grid (no closed form is used).
    """
    w = np.asarray(w, np.float64)
    k = w.shape[0]
    r = k // 2
    out = np.zeros((l_max - l_min + 1, k, k, k))
    n_c = 2 * r + 3
    i0 = n_c // 2
    for l in range(l_min, l_max + 1):
        s = 1 << (l_max - l)
        row = np.zeros((k, k))  # row[d + r, e + r] = (R S_d P)[i0, i0 + e]
        for d in range(-r, r + 1):
            M = _shift_restrict_1d(s, d, n_c)
            for e in range(-r, r + 1):
                row[d + r, e + r] = M[i0, i0 + e]
        out[l - l_min] = np.einsum("abc,ai,bj,ck->ijk", w, row, row, row)
    return out


def richardson_lucy(apr, observed, stencils, k, n_iter, bc=BC_REFLECT, estimate=None) -> np.ndarray:
    """Richardson-Lucy on the APR (Sec. 6.2): i_{k+1} = i_k * ((u / (i_k (*) w)) (*) w_flip), with
    (*) the APR convolution of Sec. 4.1 using the per-level stencils [L][k^3] and w_flip every
    level's stencil with its taps reversed in each dimension. Division and multiplication are per
    particle; a ratio whose denominator is <= 0 is 0 (the paper divides without a guard).
    i_0 = observed unless `estimate` is given. FP64."""
    u = np.asarray(observed, np.float64).reshape(-1)
    i = u.copy() if estimate is None else np.asarray(estimate, np.float64).reshape(-1).copy()
    W = np.asarray(stencils, np.float64).reshape(apr.n_levels, k ** 3)
    W_flip = W[:, ::-1].copy()
    o = Oracle(apr, i)
    for _ in range(n_iter):
        o.set_values(i)
        c = o.conv(W, k, bc)[:, 0]
        ratio = np.where(c > 0, u / np.where(c > 0, c, 1.0), 0.0)
        o.set_values(ratio)
        i = i * o.conv(W_flip, k, bc)[:, 0]
    return i


def gradient_magnitude(apr, values, stencils3, k, bc=BC_REFLECT, sample=None) -> np.ndarray:
    """sqrt(sum_a (w_a (*) u)^2) per particle for three stencil stacks [3][L][k^3] (Sec. 4.3: gradient
    estimation with Sobel filters, level-rescaled by Eq. adapt_grad). FP64."""
    W = np.asarray(stencils3, np.float64).reshape(3, apr.n_levels, k ** 3)
    o = Oracle(apr, values)
    acc = None
    for a in range(3):
        c = o.conv(W[a], k, bc, sample=sample)[:, 0]
        acc = c * c if acc is None else acc + c * c
    return np.sqrt(acc)


def round_bf16_array(v) -> np.ndarray:
    """Element-wise bfloat16 rounding (to float32 first, then nearest-even on the upper 16 bits)."""
    f = np.asarray(v, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    finite = (u & 0x7F800000) != 0x7F800000
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    out = np.where(finite, r, u.astype(np.uint32)).astype(np.uint32).view(np.float32)
    return out.astype(np.float64)


def _cnn_layer_input(apr, h, rounding):
    """Oracle over the features h with its APR tree filled: the bf16 tree (tree_bf16) of the
    network, or, with rounding off, the FP64 tree of Sec. 3.4."""
    o = Oracle(apr, h)
    if rounding:
        o.tree_bf16()
    else:
        o.tree()
    return o


def cnn_forward(apr, x, weights, scale, rounding=True) -> np.ndarray:
    """APR CNN (Sec. 6 outlook: learned per-level filters) with 16 bfloat16 channels: h_0 = embed(x)
    (channel 0 = bf16(float32(scale) * x), others 0); for every layer i, c_i = 16 -> 16 APR
    convolution of h_i (Sec. 4.1, per-level 3^3 weights, tree of bf16 features as tree_bf16), and
    h_{i+1} = bf16(max(c_i, 0)) between layers; the output is y = x + c_last[:, 0] / scale. The
    convolutions are FP64 on the bf16 values; the bf16 rounding points are those of the layer.

    rounding=False (a test hook) removes every bf16 rounding (embedding, activations, tree): the
    same network in FP64, a piecewise-linear map whose derivative cnn_backward computes."""
    x = np.asarray(x, np.float64).reshape(-1)
    sc = np.float32(scale)
    rnd = round_bf16_array if rounding else (lambda a: np.asarray(a, np.float64))
    h = np.zeros((x.size, 16))
    h[:, 0] = rnd(np.float32(sc) * x.astype(np.float32)) if rounding else float(sc) * x
    c = None
    for i, W in enumerate(weights):
        o = _cnn_layer_input(apr, h, rounding)
        c = o.conv(np.asarray(W, np.float64), 3, C_out=16)
        if i + 1 < len(weights):
            h = rnd(np.maximum(c, 0.0))
    return x + c[:, 0] / float(sc)


def cnn_backward(apr, x, weights, scale, grad_y, rounding=True):
    """Weight gradients of cnn_forward for dL/dy = grad_y, every bf16 rounding taken as the identity
    (its derivative is not defined): the transposes of the read-out, of each 16 -> 16 convolution
    (conv_backward, through the tree) and of ReLU (mask c > 0: zero derivative at 0), from the last
    layer down. FP64. rounding=False: the activations are those of cnn_forward(rounding=False), so
    the result is the exact gradient of that piecewise-linear network."""
    x = np.asarray(x, np.float64).reshape(-1)
    sc = np.float32(scale)
    rnd = round_bf16_array if rounding else (lambda a: np.asarray(a, np.float64))
    h = np.zeros((x.size, 16))
    h[:, 0] = rnd(np.float32(sc) * x.astype(np.float32)) if rounding else float(sc) * x
    hs, cs = [], []
    for i, W in enumerate(weights):
        o = _cnn_layer_input(apr, h, rounding)
        c = o.conv(np.asarray(W, np.float64), 3, C_out=16)
        hs.append(h)
        cs.append(c)
        if i + 1 < len(weights):
            h = rnd(np.maximum(c, 0.0))
    g = np.zeros((x.size, 16))
    g[:, 0] = np.asarray(grad_y, np.float64).reshape(-1) / float(sc)
    grads = [None] * len(weights)
    for i in reversed(range(len(weights))):
        o = _cnn_layer_input(apr, hs[i], rounding)
        gp, gw = o.conv_backward(np.asarray(weights[i], np.float64), 3, g, C_out=16)
        grads[i] = gw
        if i > 0:
            g = gp * (cs[i - 1] > 0)
    return grads


def cnn_layers(apr, h, W, relu):
    """One layer of cnn_forward on given bf16 features h [N][16] (a test aid for layer-by-layer
    comparison): c = the 16 -> 16 APR convolution of h over the bf16 tree of h (FP64), returned as
    is (relu=False) or as bf16(max(c, 0)) (relu=True)."""
    o = _cnn_layer_input(apr, np.asarray(h, np.float64), True)
    c = o.conv(np.asarray(W, np.float64), 3, C_out=16)
    return round_bf16_array(np.maximum(c, 0.0)) if relu else c
