"""Z-slab decomposition of one APR across ranks, with one halo exchange per convolution.

The particle order of the linear-access layout (Alg. 1) is level -> z -> x -> y, so a range of z
rows of one level is a contiguous range of particles. Rank i owns the particles whose cells start in
its slab [z0_i, z1_i) (pixels); slab bounds are multiples of the coarsest cell edge A = 2^(l_max -
l_min) so every cell of every level lies in exactly one slab. To convolve its particles, a rank
needs the values of every particle within the stencil reach r at the particle's level (at most
r * A pixels), the coarse fill of the next coarser level (inside the same aligned region) and the
tree nodes over that region (Sec. 3.4), whose subtrees lie inside the region because it is aligned
to coarsest cells. So each rank builds the index of the sub-APR covering
[z0 - r A, z1 + r A) (clipped to the image), receives the halo particles' values from their owners
(the exchange step), restricts the tree and convolves locally, and keeps the outputs of the
particles it owns. Outputs near a sub-domain edge that is not an image edge are not used (their
reflection differs from the whole image's); outputs of owned particles equal the whole-volume ones.

The transpose runs the same plan backwards: each rank back-propagates the gradient of the outputs
it owns through its local tree and convolution, sends the gradient that lands on halo particles to
their owners, and every owner adds the contributions it receives in rank order; stencil gradients
are summed over ranks with an all-reduce.

Every rank holds the index arrays (row_ptr, y_idx) of the whole APR (they are small next to the
feature values); the values are distributed. Communication uses torch.distributed point-to-point
calls (NCCL between GPUs, gloo between host processes).

The halo here is r A pixels for every level. The levels finer than the coarsest could use a halo
of r cells of their own level; the simplification costs extra halo work on coarse-heavy APRs, not
correctness.
"""
from __future__ import annotations

import numpy as np


class SubApr:
    """Index arrays of the sub-APR covering pixel rows [za, zb) of a larger APR (same levels)."""

    def __init__(self, dims, l_min, l_max, row_ptr, y_idx):
        self.dims = tuple(int(d) for d in dims)
        self.l_min, self.l_max = int(l_min), int(l_max)
        self.row_ptr = row_ptr
        self.y_idx = y_idx

    @property
    def n_particles(self):
        return int(self.y_idx.shape[0])

    @property
    def n_levels(self):
        return self.l_max - self.l_min + 1

    def level_dims(self, l):
        s = 1 << (self.l_max - l)
        return tuple(-(-d // s) for d in self.dims)


def _level_dims(dims, l_max, l):
    s = 1 << (l_max - l)
    return tuple(-(-int(d) // s) for d in dims)


class SlabPlan:
    """Slab bounds, local sub-APRs and exchange lists for `world` ranks and stencil radius r."""

    def __init__(self, apr, world: int, r: int):
        dims, l_min, l_max = tuple(int(d) for d in apr.dims), int(apr.l_min), int(apr.l_max)
        rp = np.asarray(apr.row_ptr, np.int64)
        yi = np.asarray(apr.y_idx, np.int32)
        A = 1 << (l_max - l_min)
        Dz = dims[0]
        ncz = -(-Dz // A)
        if world < 1 or world > ncz:
            raise ValueError(f"{world} ranks for {ncz} coarsest z cells")
        self.world, self.r, self.A = world, r, A
        self.bounds = [(min(Dz, (i * ncz // world) * A), min(Dz, ((i + 1) * ncz // world) * A)) for i in range(world)]
        H = r * A
        self.regions = [(max(0, z0 - H), min(Dz, z1 + H)) for z0, z1 in self.bounds]
        # per level: first row and particle range of z rows [a, b) (pixels, aligned)
        row0, lev = 0, {}
        for l in range(l_min, l_max + 1):
            dz, dx, _ = _level_dims(dims, l_max, l)
            lev[l] = (row0, dz, dx, 1 << (l_max - l))
            row0 += dz * dx

        def prange(l, za, zb):
            r0, dz, dx, s = lev[l]
            a, b = za // s, min(dz, -(-zb // s))
            return int(rp[r0 + a * dx]), int(rp[r0 + b * dx]), r0 + a * dx, r0 + b * dx

        self.owned = []      # per rank: list over levels of global particle ranges [a, b)
        self.local = []      # per rank: list over levels of global particle ranges of its region
        self.sub = []        # per rank: SubApr of its region
        for i in range(world):
            z0, z1 = self.bounds[i]
            za, zb = self.regions[i]
            own, loc, rows, ys = [], [], [np.zeros(1, np.int64)], []
            for l in range(l_min, l_max + 1):
                oa, ob, _, _ = prange(l, z0, z1)
                la, lb, ra, rb = prange(l, za, zb)
                own.append((oa, ob))
                loc.append((la, lb))
                base = rows[-1][-1]
                rows.append(rp[ra + 1:rb + 1] - rp[ra] + base)
                ys.append(yi[la:lb])
            self.owned.append(own)
            self.local.append(loc)
            self.sub.append(SubApr((zb - za, dims[1], dims[2]), l_min, l_max, np.concatenate(rows),
                                   np.concatenate(ys) if ys else np.zeros(0, np.int32)))
        self.n_levels = l_max - l_min + 1
        self.n_particles = int(yi.shape[0])

    # ---- index helpers (numpy int64 arrays of positions)
    def n_owned(self, i):
        return sum(b - a for a, b in self.owned[i])

    def owned_positions_global(self, i):
        return np.concatenate([np.arange(a, b) for a, b in self.owned[i]]) if self.owned[i] else np.zeros(0, np.int64)

    def _local_pos(self, i, l_idx, g0, g1):
        """Local positions (in rank i's sub-APR order) of global particles [g0, g1) of level index l_idx."""
        off = sum(b - a for a, b in self.local[i][:l_idx])
        la = self.local[i][l_idx][0]
        return np.arange(g0 - la + off, g1 - la + off)

    def own_local_positions(self, i):
        parts = [self._local_pos(i, li, a, b) for li, (a, b) in enumerate(self.owned[i])]
        return np.concatenate(parts) if parts else np.zeros(0, np.int64)

    def transfer(self, src, dst):
        """Particles owned by `src` inside `dst`'s region: (positions in src's owned vector,
        positions in dst's local vector)."""
        so, dl = [], []
        own_off = 0
        for li in range(self.n_levels):
            oa, ob = self.owned[src][li]
            la, lb = self.local[dst][li]
            a, b = max(oa, la), min(ob, lb)
            if a < b:
                so.append(np.arange(a - oa + own_off, b - oa + own_off))
                dl.append(self._local_pos(dst, li, a, b))
            own_off += ob - oa
        z = np.zeros(0, np.int64)
        return (np.concatenate(so) if so else z), (np.concatenate(dl) if dl else z)


class SlabConv:
    """One rank's part of a z-slab sharded APR convolution (forward and transpose).

    compute(sub_apr, local_values) -> local_outputs and
    compute_backward(sub_apr, local_values, local_grad_out) -> (local_grad_values, grad_stencils)
    run the local work; by default they are this package's CUDA kernels on the rank's GPU (tree
    restriction + apr_convolve, and apr_convolve_backward). Values are 1-D per-particle tensors.
    """

    def __init__(self, apr, rank, world, k, stencils=None, bc=0, compute=None, compute_backward=None, group=None):
        self.plan = SlabPlan(apr, world, k // 2)
        self.rank, self.world, self.k, self.bc, self.group = rank, world, k, bc, group
        self.sub = self.plan.sub[rank]
        self.own_loc = self.plan.own_local_positions(rank)
        self.sends = {j: self.plan.transfer(rank, j)[0] for j in range(world) if j != rank}
        self.recvs = {j: self.plan.transfer(j, rank)[1] for j in range(world) if j != rank}
        self.stencils = stencils
        self._compute, self._compute_bwd = compute, compute_backward
        self._layout = None

    # ---- default local work: CUDA kernels
    def _gpu_layout(self):
        if self._layout is None:
            from . import AprLayout, APR_VALIDATE, APR_REQUIRE_BALANCE, APR_SUBDOMAIN
            s = self.sub
            self._layout = AprLayout(s.dims, s.l_min, s.l_max, s.row_ptr, s.y_idx,
                                     APR_VALIDATE | APR_REQUIRE_BALANCE | APR_SUBDOMAIN)
        return self._layout

    def _local_forward(self, local_vals):
        if self._compute is not None:
            return self._compute(self.sub, local_vals)
        from . import apr_convolve, apr_tree_restrict
        lay = self._gpu_layout()
        tree = apr_tree_restrict(lay, local_vals)
        return apr_convolve(lay, local_vals, tree, self.stencils, self.k, self.bc)

    def _local_backward(self, local_vals, local_gout):
        if self._compute_bwd is not None:
            return self._compute_bwd(self.sub, local_vals, local_gout)
        from . import apr_convolve_backward, apr_tree_restrict
        lay = self._gpu_layout()
        tree = apr_tree_restrict(lay, local_vals)
        return apr_convolve_backward(lay, local_vals, tree, self.stencils, self.k, local_gout, self.bc)

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

    def gather_halo(self, owned_vals):
        """Local value vector of this rank's sub-APR from the owned values of every rank."""
        import torch
        dev, dt = owned_vals.device, owned_vals.dtype
        local = torch.zeros(self.sub.n_particles, dtype=dt, device=dev)
        local[torch.as_tensor(self.own_loc, device=dev)] = owned_vals
        send = {j: owned_vals[torch.as_tensor(ix, device=dev)] for j, ix in self.sends.items()}
        recv = {j: torch.empty(len(ix), dtype=dt, device=dev) for j, ix in self.recvs.items()}
        self._p2p(send, recv)
        for j, buf in recv.items():
            if buf.numel():
                local[torch.as_tensor(self.recvs[j], device=dev)] = buf
        return local

    def forward(self, owned_vals):
        """Outputs of the owned particles (in global order) from the owned input values."""
        import torch
        local = self.gather_halo(owned_vals)
        out = self._local_forward(local)
        return out[torch.as_tensor(self.own_loc, device=out.device)]

    def backward(self, owned_vals, owned_grad_out):
        """(gradient w.r.t. the owned values, stencil gradient summed over ranks)."""
        import torch
        import torch.distributed as dist
        dev = owned_grad_out.device
        local = self.gather_halo(owned_vals)
        gout = torch.zeros(self.sub.n_particles, dtype=owned_grad_out.dtype, device=dev)
        gout[torch.as_tensor(self.own_loc, device=dev)] = owned_grad_out   # only owned outputs are used
        gl, gw = self._local_backward(local, gout)
        # halo shares back to their owners: send[j] = my local grads at j's particles in my region
        send = {j: gl[torch.as_tensor(self.recvs[j], device=dev)] for j in self.recvs}
        recv = {j: torch.empty(len(self.sends[j]), dtype=gl.dtype, device=dev) for j in self.sends}
        self._p2p(send, recv)
        g_own = gl[torch.as_tensor(self.own_loc, device=dev)].clone()
        for j in sorted(recv):
            if recv[j].numel():
                g_own.index_add_(0, torch.as_tensor(self.sends[j], device=dev), recv[j])
        if gw is not None:
            gw = gw.clone()
            dist.all_reduce(gw, group=self.group)
        return g_own, gw
