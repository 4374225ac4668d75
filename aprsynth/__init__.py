"""Seeded synthetic APR inputs: blob images turned into Adaptive Particle Representations.

This module only makes inputs. It is shared by the FP64 oracle, the CUDA library's tests and the
benchmark, and it holds none of the convolution or tree arithmetic of the method: it draws a
blob image, decides a resolution level per pixel, forms a 2:1-balanced partition of the image
into particle cells, and gives each particle the mean of its (Poisson-noisy) pixels.

Background (paper Sec. 2): an APR is a set of particle cells that partition the image domain,
each cell an element of the image pyramid at level l (edge 2^(l_max-l) pixels), stored level by
level in the linear order l -> z -> x -> y with sparse rows along y (Alg. 1, Alg. 2).
Particle values of coarse cells are averages of the pixels they cover (Sec. 2.3).

The level rule (our reading; the paper defers APR construction to its ref. [Cheeseman 2018]):
    L(x) = E * sigma_loc(x) / |grad lambda(x)|,    l_req(x) = clip(l_max - floor(log2 L), l_min, l_max)
with lambda the noise-free intensity, sigma_loc the largest amplitude of the blobs whose
3.5-sigma box covers x (floored), and E the relative error bound (Eq. 1). A cell at level l is
split when a pixel inside requires a finer level, or when one of its children touches (26-
neighbourhood) a split cell of the next finer level; this makes the particle levels of touching
cells differ by at most one (2:1 balance).

Noise: the value of a particle is Poisson(sum of lambda over its pixels) / (#pixels), which has
exactly the distribution of the mean of independently Poisson-noised pixels.
"""
from __future__ import annotations

import dataclasses
import hashlib
import math
import os
import pathlib

import numpy as np

__all__ = [
    "AprInput", "BlobImage", "CONFIGS", "make_config", "blob_image", "apr_from_levels",
    "apr_from_blobs", "uniform_level_apr", "random_balanced_apr", "validate_apr",
    "gaussian_stencil", "level_dims", "apr_from_particles", "paint_full",
]


# --------------------------------------------------------------------------------------------
# containers
# --------------------------------------------------------------------------------------------
@dataclasses.dataclass
class AprInput:
    """An APR in the linear-access layout of Alg. 1 (one row per (l, z, x), rows l -> z -> x).

    dims:     pixel image size (D_z, D_x, D_y); y is the contiguous (sparse) axis.
    l_min, l_max: levels present; l_max = ceil(log2(max(dims))).
    row_ptr:  int64 [R+1]; rows of level l start at sum_{l'<l} d_z(l') * d_x(l'); row r holds
              particles row_ptr[r] .. row_ptr[r+1]-1 (CSR form of xz_end).
    y_idx:    int32 [N_p], strictly increasing inside each row.
    values:   float32 [N_p], particle intensities in the same order.
    """
    dims: tuple
    l_min: int
    l_max: int
    row_ptr: np.ndarray
    y_idx: np.ndarray
    values: np.ndarray
    name: str = ""

    @property
    def n_particles(self) -> int:
        return int(self.y_idx.shape[0])

    @property
    def n_levels(self) -> int:
        return self.l_max - self.l_min + 1

    def level_dims(self, l: int) -> tuple:
        return level_dims(self.dims, self.l_max, l)

    def level_row_offset(self, l: int) -> int:
        off = 0
        for lv in range(self.l_min, l):
            dz, dx, _ = self.level_dims(lv)
            off += dz * dx
        return off

    def particle_coords(self):
        """(level, z, x, y) of every particle, by walking the rows in linear order (Alg. 2)."""
        lev = np.empty(self.n_particles, np.int32)
        zz = np.empty(self.n_particles, np.int32)
        xx = np.empty(self.n_particles, np.int32)
        for l in range(self.l_min, self.l_max + 1):
            dz, dx, _ = self.level_dims(l)
            r0 = self.level_row_offset(l)
            rp = self.row_ptr[r0:r0 + dz * dx + 1]
            counts = np.diff(rp)
            b, e = int(rp[0]), int(rp[-1])
            rows = np.repeat(np.arange(dz * dx, dtype=np.int64), counts)
            lev[b:e] = l
            zz[b:e] = rows // dx
            xx[b:e] = rows % dx
        return lev, zz, xx, self.y_idx.astype(np.int32)

    def nbytes_layout(self) -> int:
        return self.row_ptr.nbytes + self.y_idx.nbytes + self.values.nbytes


@dataclasses.dataclass
class BlobImage:
    dims: tuple
    centres: np.ndarray   # [n, 3] float64 (z, x, y) in pixels
    sigmas: np.ndarray    # [n]
    amps: np.ndarray      # [n]
    background: float


def level_dims(dims, l_max: int, l: int) -> tuple:
    """Grid size of level l: ceil(D / 2^(l_max - l)) per axis (Eq. 2: cells of edge |Omega|/2^l)."""
    s = 1 << (l_max - l)
    return tuple(int(-(-d // s)) for d in dims)


def l_max_for(dims) -> int:
    m = max(dims)
    return max(0, int(math.ceil(math.log2(m)))) if m > 1 else 0


# --------------------------------------------------------------------------------------------
# image
# --------------------------------------------------------------------------------------------
def blob_image(dims, n_blobs, sigma_range, amp_range=(200.0, 1000.0), background=100.0,
               seed=0) -> BlobImage:
    rng = np.random.default_rng(seed)
    dims = tuple(int(d) for d in dims)
    centres = rng.uniform(0.0, 1.0, size=(n_blobs, 3)) * np.array(dims, np.float64)
    sigmas = rng.uniform(sigma_range[0], sigma_range[1], size=n_blobs)
    amps = rng.uniform(amp_range[0], amp_range[1], size=n_blobs)
    return BlobImage(dims, centres, sigmas, amps, float(background))


def _blob_fields(img: BlobImage, trunc=3.5):
    """Noise-free intensity lambda (float32) and amplitude scale map (float32)."""
    dz, dx, dy = img.dims
    lam = np.full((dz, dx, dy), img.background, np.float32)
    amp = np.zeros((dz, dx, dy), np.float32)
    for c, s, a in zip(img.centres, img.sigmas, img.amps):
        h = int(math.ceil(trunc * s))
        lo = [max(0, int(math.floor(c[i])) - h) for i in range(3)]
        hi = [min(img.dims[i], int(math.floor(c[i])) + h + 1) for i in range(3)]
        if any(hi[i] <= lo[i] for i in range(3)):
            continue
        g = [np.exp(-0.5 * ((np.arange(lo[i], hi[i]) - c[i]) / s) ** 2).astype(np.float32)
             for i in range(3)]
        box = (slice(lo[0], hi[0]), slice(lo[1], hi[1]), slice(lo[2], hi[2]))
        gxy = np.multiply.outer(g[1] * np.float32(a), g[2])
        lam[box] += g[0][:, None, None] * gxy[None, :, :]
        np.maximum(amp[box], np.float32(a), out=amp[box])
    return lam, amp


def _grad_mag(lam: np.ndarray) -> np.ndarray:
    """|grad lambda| by central differences (one-sided at the image edges)."""
    out = np.zeros(lam.shape, np.float32)
    for ax in range(3):
        n = lam.shape[ax]
        if n < 2:
            continue
        d = np.empty(lam.shape, np.float32)
        sl = [slice(None)] * 3

        def S(a, b):
            s2 = list(sl)
            s2[ax] = slice(a, b)
            return tuple(s2)
        d[S(1, n - 1)] = 0.5 * (lam[S(2, n)] - lam[S(0, n - 2)])
        d[S(0, 1)] = lam[S(1, 2)] - lam[S(0, 1)]
        d[S(n - 1, n)] = lam[S(n - 1, n)] - lam[S(n - 2, n - 1)]
        np.multiply(d, d, out=d)
        out += d
    np.sqrt(out, out=out)
    return out


def required_levels(lam, amp, E, sigma_floor, l_min, l_max, sigma_scale=1.0) -> np.ndarray:
    g = _grad_mag(lam)
    sig = np.maximum(amp * np.float32(sigma_scale), np.float32(sigma_floor))
    with np.errstate(divide="ignore", invalid="ignore"):
        L = np.float32(E) * sig / g
    del g, sig
    # finest level whose cell edge 2^(l_max-l) does not exceed L; L=inf -> l_min
    with np.errstate(divide="ignore", invalid="ignore"):
        k = np.floor(np.log2(np.maximum(L, np.float32(1e-30))))
    del L
    k = np.nan_to_num(k, nan=0.0, posinf=64.0, neginf=0.0)
    lev = np.clip(l_max - k, l_min, l_max).astype(np.uint8)
    return lev


# --------------------------------------------------------------------------------------------
# pyramid helpers (ceil-sized levels; cells partly outside the image are padded)
# --------------------------------------------------------------------------------------------
def _pool2(a: np.ndarray, op, fill):
    pads = [(0, s % 2) for s in a.shape]
    if any(p[1] for p in pads):
        a = np.pad(a, pads, constant_values=fill)
    z, x, y = a.shape
    v = a.reshape(z // 2, 2, x // 2, 2, y // 2, 2)
    return op(op(op(v, axis=5), axis=3), axis=1)


def _dilate26(b: np.ndarray) -> np.ndarray:
    """Binary dilation with the 3x3x3 cube (26-neighbourhood plus self), cells outside = False."""
    out = b.copy()
    for ax in range(3):
        t = out.copy()
        sl_a = [slice(None)] * 3
        sl_b = [slice(None)] * 3
        sl_a[ax] = slice(1, None)
        sl_b[ax] = slice(None, -1)
        t[tuple(sl_a)] |= out[tuple(sl_b)]
        t[tuple(sl_b)] |= out[tuple(sl_a)]
        out = t
    return out


def _upsample2(b: np.ndarray, shape) -> np.ndarray:
    u = b.repeat(2, 0).repeat(2, 1).repeat(2, 2)
    return u[:shape[0], :shape[1], :shape[2]]


def apr_from_levels(lreq: np.ndarray, l_min: int, l_max: int, lam_sum_fn, rng, dims=None,
                    name="") -> AprInput:
    """Balanced particle partition from a per-pixel required level, values from lam_sum_fn.

    lam_sum_fn(level, z, x, y) -> (sum of lambda over the cell's in-image pixels, #pixels).
    """
    dims = tuple(lreq.shape) if dims is None else tuple(dims)
    need = {l_max: lreq}
    for l in range(l_max - 1, l_min - 1, -1):
        need[l] = _pool2(need[l + 1], np.max, 0)
        assert need[l].shape == level_dims(dims, l_max, l), (need[l].shape, l)
    split = {l_max: np.zeros(need[l_max].shape, bool)}
    for l in range(l_max - 1, l_min - 1, -1):
        s = need[l] > l
        if split[l + 1].any():
            s |= _pool2(_dilate26(split[l + 1]), np.max, False)
        split[l] = s
    exists = {l_min: np.ones(need[l_min].shape, bool)}
    for l in range(l_min + 1, l_max + 1):
        exists[l] = _upsample2(split[l - 1], need[l].shape)
    rows, ys, vals, means = [], [], [], []
    for l in range(l_min, l_max + 1):
        leaf = exists[l] & ~split[l]
        dz, dx, _ = leaf.shape
        rows.append(leaf.sum(axis=2, dtype=np.int64).reshape(-1))
        z, x, y = np.nonzero(leaf)
        ys.append(y.astype(np.int32))
        ssum, cnt = lam_sum_fn(l, z, x, y)
        v = rng.poisson(ssum).astype(np.float64) / cnt
        vals.append(v.astype(np.float32))
        means.append((np.asarray(ssum, np.float64) / cnt).astype(np.float32))
        del leaf
    counts = np.concatenate(rows)
    row_ptr = np.zeros(counts.size + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    apr = AprInput(dims, l_min, l_max, row_ptr, np.concatenate(ys), np.concatenate(vals), name)
    apr.values_clean = np.concatenate(means)  # the noise-free particle means (same particles)
    return apr


def _sum_pyramid(lam: np.ndarray, l_min, l_max):
    """Per-level pixel sums (float64) and pixel counts over each cell; level l_max is lam."""
    sums = {l_max: lam}
    cnts = {l_max: None}
    ones = np.ones(lam.shape, np.float32)
    prev_s, prev_c = lam.astype(np.float64), ones
    for l in range(l_max - 1, l_min - 1, -1):
        prev_s = _pool2(prev_s, np.sum, 0.0)
        prev_c = _pool2(prev_c, np.sum, 0.0)
        sums[l] = prev_s
        cnts[l] = prev_c
    return sums, cnts


class _Mean:
    """Stands in for the noise generator: returns the mean itself (noise-free particle values)."""
    @staticmethod
    def poisson(v):
        return v


def apr_from_blobs(img: BlobImage, E=0.1, sigma_floor=10.0, l_min=2, seed_noise=None,
                   name="", sigma_scale=1.0, clean=False) -> AprInput:
    lam, amp = _blob_fields(img)
    l_max = l_max_for(img.dims)
    lreq = required_levels(lam, amp, E, sigma_floor, l_min, l_max, sigma_scale)
    del amp
    sums, cnts = _sum_pyramid(lam, l_min, l_max)

    def lam_sum(l, z, x, y):
        if l == l_max:
            return sums[l][z, x, y].astype(np.float64), 1.0
        return sums[l][z, x, y], cnts[l][z, x, y].astype(np.float64)

    rng = np.random.default_rng(seed_noise if seed_noise is not None else 12345)
    apr = apr_from_levels(lreq, l_min, l_max, lam_sum, rng, img.dims, name)
    if clean:
        apr.values = apr.values_clean
    return apr


# --------------------------------------------------------------------------------------------
# small structured APRs for pins and edge cases
# --------------------------------------------------------------------------------------------
def uniform_level_apr(dims, level, values_fn=None, seed=0, l_min=None) -> AprInput:
    """Every particle at one level l (a uniform grid of cells of edge 2^(l_max-l))."""
    l_max = l_max_for(dims)
    l_min = level if l_min is None else l_min
    lreq = np.full(dims, level, np.uint8)
    rng = np.random.default_rng(seed)
    d = level_dims(dims, l_max, level)
    u = rng.uniform(50.0, 500.0, size=d) if values_fn is None else values_fn(d)

    def vals(l, z, x, y):
        return u[z, x, y], 1.0

    return apr_from_levels(lreq, l_min, l_max, vals, _Mean(), dims, f"uniform{level}")


def random_balanced_apr(dims, l_min, seed=0, p_fine=0.04, values="uniform", name="") -> AprInput:
    """Random balanced APR: random per-pixel level demands, values drawn per particle."""
    rng = np.random.default_rng(seed)
    l_max = l_max_for(dims)
    lreq = np.full(dims, l_min, np.uint8)
    n_seeds = max(1, int(p_fine * np.prod(dims)))
    idx = [rng.integers(0, d, n_seeds) for d in dims]
    lreq[idx[0], idx[1], idx[2]] = rng.integers(l_min, l_max + 1, n_seeds).astype(np.uint8)

    def vals(l, z, x, y):
        if values == "const":
            return np.full(z.shape, 7.25), 1.0
        return rng.uniform(10.0, 1000.0, size=z.shape), 1.0

    class _Det:
        @staticmethod
        def poisson(v):
            return v
    return apr_from_levels(lreq, l_min, l_max, vals, _Det(), dims, name or f"rand{seed}")


# --------------------------------------------------------------------------------------------
# validation of a layout (partition of the image + 2:1 balance); structure only
# --------------------------------------------------------------------------------------------
def validate_apr(apr: AprInput, check_balance=True) -> None:
    lev, zz, xx, yy = apr.particle_coords()
    l_max, l_min = apr.l_max, apr.l_min
    assert apr.row_ptr[0] == 0 and apr.row_ptr[-1] == apr.n_particles
    assert np.all(np.diff(apr.row_ptr) >= 0)
    # y strictly increasing within rows
    dy = np.diff(yy.astype(np.int64))
    starts = np.zeros(apr.n_particles, bool)
    starts[apr.row_ptr[:-1][np.diff(apr.row_ptr) > 0]] = True
    assert np.all(dy[~starts[1:]] > 0), "y not strictly increasing within a row"
    # paint the finest level with particle ids; every pixel exactly once
    cover = np.zeros(apr.dims, np.int32)
    for l in range(l_min, l_max + 1):
        s = 1 << (l_max - l)
        m = lev == l
        for z, x, y in zip(zz[m], xx[m], yy[m]):
            cover[z * s:(z + 1) * s, x * s:(x + 1) * s, y * s:(y + 1) * s] += 1
    assert cover.min() == 1 and cover.max() == 1, "particle cells do not partition the image"
    if check_balance:
        lvl = np.zeros(apr.dims, np.int8)
        for l in range(l_min, l_max + 1):
            s = 1 << (l_max - l)
            m = lev == l
            for z, x, y in zip(zz[m], xx[m], yy[m]):
                lvl[z * s:(z + 1) * s, x * s:(x + 1) * s, y * s:(y + 1) * s] = l
        for ax in range(3):
            for sh in (1,):
                a = np.swapaxes(lvl, 0, ax)
                d = np.abs(a[sh:].astype(np.int16) - a[:-sh])
                assert d.max(initial=0) <= 1, "2:1 balance violated (face)"
        # diagonal neighbours
        for oz in (-1, 0, 1):
            for ox in (-1, 0, 1):
                for oy in (-1, 0, 1):
                    a = lvl[max(0, oz):lvl.shape[0] + min(0, oz), max(0, ox):lvl.shape[1] + min(0, ox),
                            max(0, oy):lvl.shape[2] + min(0, oy)]
                    b = lvl[max(0, -oz):lvl.shape[0] + min(0, -oz), max(0, -ox):lvl.shape[1] + min(0, -ox),
                            max(0, -oy):lvl.shape[2] + min(0, -oy)]
                    assert np.abs(a.astype(np.int16) - b).max(initial=0) <= 1, "2:1 balance violated"


# --------------------------------------------------------------------------------------------
# stencils (inputs of the method)
# --------------------------------------------------------------------------------------------
def gaussian_stencil(k: int, sigma: float) -> np.ndarray:
    """Normalised k^3 Gaussian stencil [z][x][y], FP64 (rounded to FP32 by the caller)."""
    r = k // 2
    t = np.arange(-r, r + 1, dtype=np.float64)
    g = np.exp(-0.5 * (t / sigma) ** 2)
    w = g[:, None, None] * g[None, :, None] * g[None, None, :]
    return w / w.sum()


# --------------------------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------------------------
CONFIGS = {
    # 64^3, 20 blobs sigma 2-6, E=0.1, l_max 6; 3^3 Gaussian sigma=1, plain method
    "blob64": dict(dims=(64, 64, 64), n_blobs=20, sigma_range=(2.0, 6.0), seed=0, E=0.1,
                   sigma_floor=10.0, l_min=2, k=3, stencil_sigma=1.0, sigma_scale=3.0),
    # 1024x1024x512 (z=512), 2000 blobs sigma 2-20; 5^3 Gaussian sigma=1.5
    "blob1024": dict(dims=(512, 1024, 1024), n_blobs=2000, sigma_range=(2.0, 20.0), seed=1,
                     E=0.1, sigma_floor=10.0, l_min=3, k=5, stencil_sigma=1.5, sigma_scale=1.5),
    # 512^3 (Richardson-Lucy workload, ~2.9M particles), 256^3 (multi-channel, ~1.0M particles)
    "blob512": dict(dims=(512, 512, 512), n_blobs=200, sigma_range=(2.0, 20.0), seed=2,
                    E=0.1, sigma_floor=10.0, l_min=3, k=5, stencil_sigma=1.5, sigma_scale=1.0),
    "blob256": dict(dims=(256, 256, 256), n_blobs=400, sigma_range=(2.0, 12.0), seed=3,
                    E=0.1, sigma_floor=10.0, l_min=2, k=3, stencil_sigma=1.0, sigma_scale=1.5),
}


def _cache_dir():
    d = os.environ.get("APRSYNTH_CACHE")
    if d:
        return pathlib.Path(d)
    return pathlib.Path(os.environ.get("TMPDIR", "/tmp")) / "aprsynth_cache"


def make_config(name: str, use_cache=True, clean=False, **overrides) -> AprInput:
    """Build (or load from the on-disk cache) the APR of a named workload. clean=True: the same
    particles with noise-free values (the mean intensity over each particle's pixels)."""
    cfg = dict(CONFIGS[name])
    cfg.update(overrides)
    key = hashlib.sha1((repr(sorted(cfg.items())) + "+clean").encode()).hexdigest()[:12]
    path = _cache_dir() / f"{name}_{key}.npz"

    def pick(a, noisy, means):
        a.values_clean = means
        a.values = means if clean else noisy
        return a

    if use_cache and path.exists():
        z = np.load(path)
        a = AprInput(tuple(int(v) for v in z["dims"]), int(z["l_min"]), int(z["l_max"]),
                     z["row_ptr"], z["y_idx"], z["values"], name)
        return pick(a, z["values"], z["values_clean"])
    img = blob_image(cfg["dims"], cfg["n_blobs"], cfg["sigma_range"], seed=cfg["seed"])
    apr = apr_from_blobs(img, E=cfg["E"], sigma_floor=cfg["sigma_floor"], l_min=cfg["l_min"],
                         seed_noise=cfg["seed"] + 1000, name=name,
                         sigma_scale=cfg.get("sigma_scale", 1.0))
    if use_cache:
        try:
            path.parent.mkdir(parents=True, exist_ok=True)
            tmp = path.with_suffix(".tmp.npz")
            np.savez(tmp, dims=np.array(apr.dims), l_min=apr.l_min, l_max=apr.l_max,
                     row_ptr=apr.row_ptr, y_idx=apr.y_idx, values=apr.values, values_clean=apr.values_clean)
            os.replace(tmp, path)
        except OSError:
            pass
    return pick(apr, apr.values, apr.values_clean)


def apr_from_particles(dims, l_min, particles, name="") -> AprInput:
    """AprInput from an explicit list of (level, z, x, y, value) particles (any order)."""
    dims = tuple(int(d) for d in dims)
    l_max = l_max_for(dims)
    ps = sorted(particles, key=lambda p: (p[0], p[1], p[2], p[3]))
    counts = []
    for l in range(l_min, l_max + 1):
        dz, dx, _ = level_dims(dims, l_max, l)
        c = np.zeros(dz * dx, np.int64)
        for p in ps:
            if p[0] == l:
                c[p[1] * dx + p[2]] += 1
        counts.append(c)
    counts = np.concatenate(counts)
    row_ptr = np.zeros(counts.size + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    y = np.array([p[3] for p in ps], np.int32)
    v = np.array([p[4] for p in ps], np.float32)
    return AprInput(dims, l_min, l_max, row_ptr, y, v, name)


def paint_full(apr: AprInput, values=None) -> np.ndarray:
    """Piecewise-constant reconstruction at pixel resolution (Sec. 2.2), float64 [D_z, D_x, D_y]."""
    vals = apr.values if values is None else values
    out = np.zeros(apr.dims, np.float64)
    lev, zz, xx, yy = apr.particle_coords()
    for i in range(apr.n_particles):
        s = 1 << (apr.l_max - int(lev[i]))
        out[zz[i] * s:(zz[i] + 1) * s, xx[i] * s:(xx[i] + 1) * s, yy[i] * s:(yy[i] + 1) * s] = vals[i]
    return out
