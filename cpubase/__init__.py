"""Multi-core FP32 CPU implementation of APR convolution: the CPU baseline that bench.py times.

This is a measurement baseline (the paper's OpenMP CPU comparison, Sec. 5.1: the rows of a level
processed in parallel), not part of the CUDA path and not the oracle: `apr_cpu.cpp` shares no code
with either. It computes the same step as the GPU path in FP32 on all host threads: tree
restriction (Sec. 3.4), convolution (Sec. 4.1), and the backward (data adjoint through the tree and
the stencil gradient).
"""
from __future__ import annotations

import ctypes
import os
import pathlib
import subprocess

import numpy as np

_HERE = pathlib.Path(__file__).resolve().parent
_SO = _HERE / "_build" / "libaprcpu.so"
_lib = None


def build(force: bool = False) -> pathlib.Path:
    """Compile apr_cpu.cpp with the host C++ compiler (portable flags only)."""
    src = _HERE / "apr_cpu.cpp"
    if force or not _SO.exists() or _SO.stat().st_mtime < src.stat().st_mtime:
        _SO.parent.mkdir(parents=True, exist_ok=True)
        tmp = _SO.with_suffix(f".{os.getpid()}.tmp")
        subprocess.check_call(["g++", "-O3", "-std=c++17", "-fPIC", "-shared", "-pthread", "-o", str(tmp), str(src)])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(str(_SO))
        P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.acpu_create.restype = P
        lib.acpu_create.argtypes = [I32, I32, P, P, P, I64]
        lib.acpu_destroy.argtypes = [P]
        lib.acpu_num_tree.restype = I64
        lib.acpu_num_tree.argtypes = [P]
        lib.acpu_tree_restrict.restype = I32
        lib.acpu_tree_restrict.argtypes = [P, P, P, I32]
        lib.acpu_convolve.restype = I32
        lib.acpu_convolve.argtypes = [P, P, P, P, I32, I32, P, I32]
        lib.acpu_convolve_backward.restype = I32
        lib.acpu_convolve_backward.argtypes = [P, P, P, P, I32, I32, P, P, P, I32]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def host_threads() -> int:
    """Threads the baseline uses by default: every CPU the process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


class CpuApr:
    """One APR (linear-access layout, Alg. 1) on the host, with its own APR tree."""

    def __init__(self, apr, threads: int | None = None):
        lib = _load()
        self.apr = apr
        self.threads = host_threads() if threads is None else int(threads)
        self._keep = [np.ascontiguousarray(np.asarray(apr.dims, np.int64)),
                      np.ascontiguousarray(apr.row_ptr.astype(np.int64)),
                      np.ascontiguousarray(apr.y_idx.astype(np.int32))]
        self.h = lib.acpu_create(apr.l_min, apr.l_max, _p(self._keep[0]), _p(self._keep[1]), _p(self._keep[2]),
                                 apr.n_particles)
        if not self.h:
            raise ValueError("cpubase: bad APR arguments")
        self.n_tree = int(lib.acpu_num_tree(self.h))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.acpu_destroy(self.h)
            self.h = None

    def tree_restrict(self, values) -> np.ndarray:
        v = np.ascontiguousarray(values, np.float32)
        t = np.zeros(max(self.n_tree, 1), np.float32)
        _load().acpu_tree_restrict(self.h, _p(v), _p(t), self.threads)
        return t[:self.n_tree]

    def convolve(self, values, tree, stencils, k, bc=0) -> np.ndarray:
        v = np.ascontiguousarray(values, np.float32)
        t = np.ascontiguousarray(tree if len(tree) else np.zeros(1), np.float32)
        st = np.ascontiguousarray(stencils, np.float32)
        out = np.zeros(max(self.apr.n_particles, 1), np.float32)
        rc = _load().acpu_convolve(self.h, _p(v), _p(t), _p(st), int(k), int(bc), _p(out), self.threads)
        if rc:
            raise ValueError(f"cpubase: convolve failed ({rc})")
        return out[:self.apr.n_particles]

    def backward(self, values, tree, stencils, k, grad_out, bc=0, particles=True, stencils_grad=True):
        v = np.ascontiguousarray(values, np.float32)
        t = np.ascontiguousarray(tree if len(tree) else np.zeros(1), np.float32)
        st = np.ascontiguousarray(stencils, np.float32)
        g = np.ascontiguousarray(grad_out, np.float32)
        gp = np.zeros(max(self.apr.n_particles, 1), np.float32) if particles else None
        gw = np.zeros(self.apr.n_levels * k ** 3, np.float32) if stencils_grad else None
        rc = _load().acpu_convolve_backward(self.h, _p(v), _p(t), _p(st), int(k), int(bc), _p(g), _p(gp), _p(gw),
                                            self.threads)
        if rc:
            raise ValueError(f"cpubase: backward failed ({rc})")
        return (gp[:self.apr.n_particles] if particles else None,
                gw.reshape(self.apr.n_levels, k ** 3) if stencils_grad else None)
