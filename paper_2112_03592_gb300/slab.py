"""Z-slab decomposition of one APR across ranks with per-level halos (Sec. 5.1: the rows of a
level are independent; Sec. 4.1: a particle's output depends on its level-l patch only).

Plan. The z axis is cut into units of B pixels, B the largest power of two that leaves at least one
unit per rank; rank i owns the pixel rows [z0_i, z1_i) (whole units). A particle of level l (cells
of s_l = 2^(l_max-l) pixels) belongs to the rank whose slab holds its cell's first pixel row. Levels
with s_l <= B are sharded: every cell lies inside one slab. Coarser levels (s_l > B) hold few
particles and are replicated: every rank receives all of them.

What a rank needs for the outputs of its particles, and how it gets it:
  - particle values: its own, plus, per sharded level l, the level-l particles of the rows within
    r_l cells of its slab (reflected at the image edge) and the level-(l-1) particles under those
    rows, plus the replicated levels. One point-to-point message per rank pair (the exchange step).
  - tree values (Sec. 3.4): the tree average is linear in the particle values, so the whole tree is
    the sum over ranks of the tree each rank restricts from its own particles alone (zeros
    elsewhere): one all-reduce of the tree per convolution.
  - the convolution runs on the work items that hold its particles (one tile range per level).
The transpose runs the same plan backwards: the data adjoint of the rank's outputs over the tiles
that can receive their gradient, the tree gradients all-reduced and pushed down to the rank's own
particles, the particle gradients that landed on other ranks' particles sent to their owners (added
in rank order), and the stencil gradient all-reduced.

Every rank holds the index (row_ptr, y_idx) of the whole APR and full-length value arrays of which
only the entries above are valid; the per-rank particle data is the slab plus per-level halos of
r_l cells (e.g. under 1/4 of the particles per rank for 8 ranks on the 1024x1024x512 workload).
Communication uses torch.distributed (NCCL between GPUs, gloo between host processes).
"""
from __future__ import annotations

import numpy as np


def _level_dims(dims, l_max, l):
    s = 1 << (l_max - l)
    return tuple(-(-int(d) // s) for d in dims)


def _reflect(i, d):
    p = 2 * d
    m = np.mod(i, p)
    return np.where(m >= d, p - 1 - m, m)


class SlabPlan:
    """Slab bounds, particle ownership, needed particle sets and exchange lists for `world` ranks.

    radii: stencil radius per level index (a list of n_levels ints) or one int for all levels."""

    def __init__(self, apr, world: int, radii):
        dims, l_min, l_max = tuple(int(d) for d in apr.dims), int(apr.l_min), int(apr.l_max)
        rp = np.asarray(apr.row_ptr, np.int64)
        L = l_max - l_min + 1
        radii = [int(radii)] * L if np.isscalar(radii) else [int(r) for r in radii]
        Dz = dims[0]
        if world < 1 or world > Dz:
            raise ValueError(f"{world} ranks for {Dz} pixel rows")
        B = 1
        while B * 2 <= Dz and -(-Dz // (B * 2)) >= world:
            B *= 2
        U = -(-Dz // B)
        self.world, self.B, self.radii = world, B, radii
        self.bounds = [(min(Dz, (i * U // world) * B), min(Dz, ((i + 1) * U // world) * B)) for i in range(world)]
        starts = np.array([b[0] for b in self.bounds], np.int64)

        def rank_of(zpix):
            return np.searchsorted(starts, zpix, side="right") - 1

        self.levels = []  # per level: dict(l, s, dz, dx, row0, p0, p1, sharded)
        owner = np.empty(int(rp[-1]), np.int64)
        row0 = 0
        for l in range(l_min, l_max + 1):
            dz, dx, _ = _level_dims(dims, l_max, l)
            s = 1 << (l_max - l)
            p0, p1 = int(rp[row0]), int(rp[row0 + dz * dx])
            zc = np.repeat(np.arange(dz * dx) // dx, np.diff(rp[row0:row0 + dz * dx + 1]))
            owner[p0:p1] = rank_of(zc * s)
            self.levels.append(dict(l=l, s=s, dz=dz, dx=dx, row0=row0, p0=p0, p1=p1, sharded=s <= B))
            row0 += dz * dx
        self.owner = owner
        self.n_particles = int(rp[-1])
        self.n_levels = L
        self.owned = [np.nonzero(owner == i)[0] for i in range(world)]

        def rows_particles(li, zrows):
            """Particles of level index li in the z rows zrows (any order, unique)."""
            lv = self.levels[li]
            zrows = np.unique(zrows)
            if zrows.size == 0:
                return np.zeros(0, np.int64)
            a = rp[lv["row0"] + zrows * lv["dx"]]
            b = rp[lv["row0"] + (zrows + 1) * lv["dx"]]
            return np.concatenate([np.arange(x, y) for x, y in zip(a, b)]) if a.size else np.zeros(0, np.int64)

        self.needed = []
        for i, (z0, z1) in enumerate(self.bounds):
            parts = [self.owned[i]]
            for li, lv in enumerate(self.levels):
                if not lv["sharded"]:
                    parts.append(np.arange(lv["p0"], lv["p1"]))
                    continue
                s, r = lv["s"], radii[li]
                zc0, zc1 = -(-z0 // s), -(-z1 // s)
                if zc0 >= zc1:
                    continue
                zrows = _reflect(np.arange(zc0 - r, zc1 + r), lv["dz"])
                parts.append(rows_particles(li, zrows))
                if li > 0:
                    parts.append(rows_particles(li - 1, zrows // 2))
            self.needed.append(np.unique(np.concatenate(parts)))

    def held_fraction(self, i):
        """Share of all particles whose values rank i holds (owned and received)."""
        return self.needed[i].size / max(self.n_particles, 1)

    def transfer(self, src, dst):
        """Global indices of the particles owned by src that dst needs (sorted)."""
        n = self.needed[dst]
        return n[self.owner[n] == src] if src != dst else np.zeros(0, np.int64)

    def owned_z_cells(self, i, li):
        """Level li's z cells [zc0, zc1) whose first pixel row lies in rank i's slab."""
        z0, z1 = self.bounds[i]
        s = self.levels[li]["s"]
        return -(-z0 // s), -(-z1 // s)


class CudaLocal:
    """A rank's local work with this package's CUDA kernels on its GPU: the layout of the whole
    APR, tile ranges per level, full-length value arrays."""

    def __init__(self, apr, plan: SlabPlan, rank, stencils, k, bc=0):
        from . import APR_REQUIRE_BALANCE, APR_VALIDATE, AprLayout
        from ._abi import APR_STRUCT_BWD_ITEMS, APR_STRUCT_FWD_ITEMS
        self.lay = AprLayout.from_apr(apr, APR_VALIDATE | APR_REQUIRE_BALANCE)
        self.st, self.k, self.bc = stencils, k, bc
        self.fwd_ranges = self._ranges(plan, rank, self.lay.export(APR_STRUCT_FWD_ITEMS), 0)
        self.bwd_ranges = self._ranges(plan, rank, self.lay.export(APR_STRUCT_BWD_ITEMS), None)

    @staticmethod
    def _ranges(plan, rank, items, margin):
        """Per level, the contiguous run of work items (ordered l, tz, tx, yb) whose 8-cell z tile
        meets the rank's z cells widened by `margin` cells (None: the level's stencil radius)."""
        out = []
        for li, lv in enumerate(plan.levels):
            zc0, zc1 = plan.owned_z_cells(rank, li)
            if zc0 >= zc1:
                continue
            m = plan.radii[li] if margin is None else margin
            lev = np.nonzero(items[:, 0] == lv["l"])[0]
            if lev.size == 0:
                continue
            tz = items[lev, 1]
            a = np.searchsorted(tz, max(0, (zc0 - m) // 8), side="left")
            b = np.searchsorted(tz, (zc1 - 1 + m) // 8, side="right")
            if b > a:
                out.append((int(lev[0] + a), int(b - a)))
        return out

    def restrict(self, v):
        from . import apr_tree_restrict
        return apr_tree_restrict(self.lay, v)

    def convolve(self, v, tree, owned):
        import torch
        from . import apr_convolve_tiles
        out = torch.zeros_like(v)
        for first, n in self.fwd_ranges:
            apr_convolve_tiles(self.lay, v, tree, self.st, self.k, first, n, self.bc, out=out)
        return out

    def adjoint(self, v, tree, g, owned):
        import torch
        from . import apr_convolve_adjoint_tiles, apr_convolve_stencil_grad
        gp = torch.zeros_like(g)
        gt = torch.zeros(self.lay.n_tree, dtype=g.dtype, device=g.device)
        for first, n in self.bwd_ranges:
            apr_convolve_adjoint_tiles(self.lay, self.st, self.k, g, gp, gt, first, n, self.bc)
        gw = apr_convolve_stencil_grad(self.lay, v, tree, self.k, g, self.bc)
        return gp, gt, gw

    def tree_transpose(self, gt):
        import torch
        from . import apr_tree_restrict_adjoint
        gp = torch.zeros(self.lay.n_particles, dtype=gt.dtype, device=gt.device)
        return apr_tree_restrict_adjoint(self.lay, gt.clone(), gp)


class SlabConv:
    """One rank's part of a z-slab sharded APR convolution (forward and transpose).

    local: the rank's compute (CudaLocal by default) with restrict(v) -> tree, convolve(v, tree,
    owned) -> out, adjoint(v, tree, g, owned) -> (grad_particles, grad_tree, grad_stencils) and
    tree_transpose(grad_tree) -> grad_particles, on full-length 1-D tensors."""

    def __init__(self, apr, rank, world, k, stencils=None, bc=0, local=None, group=None, radii=None):
        self.plan = SlabPlan(apr, world, k // 2 if radii is None else radii)
        self.rank, self.world, self.k, self.bc, self.group = rank, world, k, bc, group
        self.local = local if local is not None else CudaLocal(apr, self.plan, rank, stencils, k, bc)
        self.own = self.plan.owned[rank]
        self.sends = {j: self.plan.transfer(rank, j) for j in range(world) if j != rank}
        self.recvs = {j: self.plan.transfer(j, rank) for j in range(world) if j != rank}

    # ---- exchange
    def _p2p(self, send, recv):
        """send: {peer: tensor}, recv: {peer: tensor} (filled in place). One message per pair."""
        import torch.distributed as dist
        reqs = []
        for j in sorted(set(send) | set(recv)):
            if j in recv and recv[j].numel():
                reqs.append(dist.irecv(recv[j], src=j, group=self.group))
            if j in send and send[j].numel():
                reqs.append(dist.isend(send[j].contiguous(), dst=j, group=self.group))
        for q in reqs:
            q.wait()

    def _ix(self, a, dev):
        import torch
        return torch.as_tensor(a, device=dev)

    def gather(self, owned_vals):
        """(values: own and needed particles filled, tree of the whole APR) from the owned values."""
        import torch
        import torch.distributed as dist
        dev, dt = owned_vals.device, owned_vals.dtype
        mine = torch.zeros(self.plan.n_particles, dtype=dt, device=dev)
        mine[self._ix(self.own, dev)] = owned_vals
        tree = self.local.restrict(mine)                 # this rank's share of every tree average
        dist.all_reduce(tree, group=self.group)
        v = mine.clone()
        send = {j: owned_vals[self._ix(np.searchsorted(self.own, ix), dev)] for j, ix in self.sends.items()}
        recv = {j: torch.empty(len(ix), dtype=dt, device=dev) for j, ix in self.recvs.items()}
        self._p2p(send, recv)
        for j, buf in recv.items():
            if buf.numel():
                v[self._ix(self.recvs[j], dev)] = buf
        return v, tree

    def forward(self, owned_vals):
        """Outputs of the owned particles (in global order) from the owned input values."""
        v, tree = self.gather(owned_vals)
        out = self.local.convolve(v, tree, self.own)
        return out[self._ix(self.own, out.device)]

    def backward(self, owned_vals, owned_grad_out):
        """(gradient w.r.t. the owned values, stencil gradient summed over ranks)."""
        import torch
        import torch.distributed as dist
        dev, dt = owned_grad_out.device, owned_grad_out.dtype
        v, tree = self.gather(owned_vals)
        g = torch.zeros(self.plan.n_particles, dtype=dt, device=dev)
        g[self._ix(self.own, dev)] = owned_grad_out      # only the owned outputs are this rank's
        gp, gt, gw = self.local.adjoint(v, tree, g, self.own)
        dist.all_reduce(gt, group=self.group)
        push = self.local.tree_transpose(gt)
        # shares of other ranks' particles back to their owners (the reverse of the forward exchange)
        send = {j: gp[self._ix(self.recvs[j], dev)] for j in self.recvs}
        recv = {j: torch.empty(len(self.sends[j]), dtype=dt, device=dev) for j in self.sends}
        self._p2p(send, recv)
        own_ix = self._ix(self.own, dev)
        g_own = gp[own_ix] + push[own_ix]
        for j in sorted(recv):
            if recv[j].numel():
                g_own.index_add_(0, self._ix(np.searchsorted(self.own, self.sends[j]), dev), recv[j])
        if gw is not None:
            gw = gw.clone()
            dist.all_reduce(gw, group=self.group)
        return g_own, gw
