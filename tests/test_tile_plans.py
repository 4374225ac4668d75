"""Tile plans (the per-tile source lists the convolution kernels stage from), on the host.

The plans of a host-only handle are decoded entry by entry and checked against the coordinates of the
particles (from the input rows) and of the tree nodes (from the oracle's own tree):
- forward: every listed element lands in the patch row and y window its entry names (reflected rows
  for patch rows outside the grid, 2 cells per level-(l-1) particle), no patch cell is covered twice,
  and every cell a target's (2R+1)^3 window reads inside the grid is covered exactly once (Sec. 3.5:
  the level-l particle, the level-l tree node or the level-(l-1) particle at that cell);
- data adjoint: the gradient rows list exactly the level-l particles of the in-grid patch rows, and
  the routing segments exactly the particles, tree nodes and level-(l-1) particles under the tile;
- the packet prefixes count the aligned 8-element packets of the entries before each one.
"""
import numpy as np
import pytest
from scipy import ndimage

import aprsynth as S
import oracle
import paper_2112_03592_gb300 as G
from paper_2112_03592_gb300 import _abi

HOST = G.APR_VALIDATE | G.APR_REQUIRE_BALANCE | G.APR_HOST_ONLY
T, B = _abi.APR_TILE_ZX, _abi.APR_BLOCK_Y
NIR = T * T


def reflect(i, d):
    p = 2 * d
    m = i % p
    return p - 1 - m if m >= d else m


def decode(ent):
    w0, w1 = int(ent[0]), int(ent[1])
    lo = w0 & 0x0FFFFFFF
    n = (w0 >> 28) | ((w1 >> 27) << 4)
    meta = (w1 >> 16) & 0x7FF
    pre = w1 & 0xFFFF
    return lo, n, meta, pre


def packets(lo, n):
    return ((lo + n + 7) >> 3) - (lo >> 3) if n > 0 else 0


class Coords:
    def __init__(self, apr):
        self.apr = apr
        self.pl, self.pz, self.px, self.py = apr.particle_coords()
        tc = oracle.Oracle(apr).tree_coords()
        self.tl, self.tz, self.tx, self.ty = (tc[:, i] for i in range(4))


def plans(lay, which, items_which):
    items = lay.export(items_which)
    raw = lay.export(which)
    return items, raw[:len(items)], raw[len(items):]


def check_forward(c, lay, R):
    apr = c.apr
    PZ = PX = T + 2 * R
    PY = B + 2 * R
    which = _abi.APR_STRUCT_FWD_PLAN_R1 if R == 1 else _abi.APR_STRUCT_FWD_PLAN_R2
    items, hdr, ent = plans(lay, which, _abi.APR_STRUCT_FWD_ITEMS)
    assert len(items) > 0
    for t, (l, a, b, yb) in enumerate(items.tolist()):
        first, count = int(hdr[t][0]), int(hdr[t][1])
        z0, x0, yw = a * T, b * T, yb * B - R
        dz, dx, dy = apr.level_dims(l)
        ylo, yhi = max(yw, 0), min(yw + PY, dy)
        cov = np.zeros((PZ, PX, PY), np.int32)
        total = 0
        for k in range(count):
            lo, n, meta, pre = decode(ent[first + k])
            assert pre == total and n > 0
            total += packets(lo, n)
            idx = np.arange(lo, lo + n)
            kind = (meta >> 8) & 3
            if kind == 3:
                rz0, rx0 = (meta & 15) - 1, ((meta >> 4) & 15) - 1
                assert (z0 - R + rz0) % 2 == 0 and (x0 - R + rx0) % 2 == 0
                cz, cx = (z0 - R + rz0) // 2, (x0 - R + rx0) // 2
                assert np.all(c.pl[idx] == l - 1) and np.all(c.pz[idx] == cz) and np.all(c.px[idx] == cx)
                rows = [(rz0 + i, rx0 + j) for i in range(2) for j in range(2)
                        if 0 <= rz0 + i < PZ and 0 <= rx0 + j < PX]
                for (rz, rx) in rows:   # once-staged rows: only away from the grid boundary
                    assert 0 <= z0 - R + rz < dz and 0 <= x0 - R + rx < dx
                cells = [(2 * int(y) + e) for y in c.py[idx] for e in range(2)]
                hit = [cy for cy in cells if ylo <= cy < yhi]
                assert len(hit) > 0
                for (rz, rx) in rows:
                    for cy in hit:
                        cov[rz, rx, cy - yw] += 1
                continue
            pr = meta & 255
            pz, px = divmod(pr, PX)
            z, x = z0 - R + pz, x0 - R + px
            inside = 0 <= z < dz and 0 <= x < dx
            assert bool(meta & 1024) == (not inside)
            zz, xx = reflect(z, dz), reflect(x, dx)
            if kind == 0:
                assert np.all(c.pl[idx] == l) and np.all(c.pz[idx] == zz) and np.all(c.px[idx] == xx)
                ys = c.py[idx].astype(np.int64)
            elif kind == 1:
                assert np.all(c.tl[idx] == l) and np.all(c.tz[idx] == zz) and np.all(c.tx[idx] == xx)
                ys = c.ty[idx].astype(np.int64)
            else:
                assert np.all(c.pl[idx] == l - 1)
                assert np.all(c.pz[idx] == zz // 2) and np.all(c.px[idx] == xx // 2)
                ys = np.concatenate([2 * c.py[idx].astype(np.int64), 2 * c.py[idx].astype(np.int64) + 1])
                ys = ys[(ys >= ylo) & (ys < yhi)]
                assert ys.size > 0
            assert np.all((ys >= ylo) & (ys < yhi))
            np.add.at(cov, (pz, px, ys - yw), 1)
        assert decode(ent[first + count])[3] == total
        assert cov.max() <= 1, f"item {t}: a patch cell listed twice"
        # every in-grid cell a target's window reads is covered exactly once
        sel = ((c.pl == l) & (c.pz >= z0) & (c.pz < z0 + T) & (c.px >= x0) & (c.px < x0 + T)
               & (c.py >= yb * B) & (c.py < yb * B + B))
        tgt = np.zeros((PZ, PX, PY), bool)
        tgt[c.pz[sel] - z0 + R, c.px[sel] - x0 + R, c.py[sel] - yw] = True
        assert tgt.any()
        need = ndimage.binary_dilation(tgt, structure=np.ones((2 * R + 1,) * 3, bool))
        ycol = np.arange(PY) + yw
        need &= ((ycol >= 0) & (ycol < dy))[None, None, :]
        assert np.all(cov[need] == 1), f"item {t}: a cell a target reads is not staged"


def check_adjoint(c, lay, R):
    apr = c.apr
    PZ = PX = T + 2 * R
    PY = B + 2 * R
    NROW = PZ * PX
    which = _abi.APR_STRUCT_BWD_PLAN_R1 if R == 1 else _abi.APR_STRUCT_BWD_PLAN_R2
    items, hdr, ent = plans(lay, which, _abi.APR_STRUCT_BWD_ITEMS)
    assert len(items) > 0
    for t, (l, a, b, yb) in enumerate(items.tolist()):
        first, cnt = int(hdr[t][0]), int(hdr[t][1])
        n1, n2 = cnt & 0xFFFF, cnt >> 16
        z0, x0, y0, yw = a * T, b * T, yb * B, yb * B - R
        dz, dx, dy = apr.level_dims(l)
        ylo, yhi = max(yw, 0), min(yw + PY, dy)
        got_grad, got_p, got_t, got_c = [], [], [], []
        total = 0
        for k in range(n1 + n2):
            lo, n, meta, pre = decode(ent[first + k])
            assert pre == total and n > 0
            total += packets(lo, n)
            idx = np.arange(lo, lo + n)
            if k < n1:
                assert meta < NROW
                pz, px = divmod(meta, PX)
                z, x = z0 - R + pz, x0 - R + px
                assert 0 <= z < dz and 0 <= x < dx
                assert np.all(c.pl[idx] == l) and np.all(c.pz[idx] == z) and np.all(c.px[idx] == x)
                got_grad += idx.tolist()
            elif meta < NIR:
                assert np.all(c.pl[idx] == l) and np.all(c.pz[idx] == z0 + meta // T)
                assert np.all(c.px[idx] == x0 + meta % T)
                got_p += idx.tolist()
            elif meta < 2 * NIR:
                r = meta - NIR
                assert np.all(c.tl[idx] == l) and np.all(c.tz[idx] == z0 + r // T) and np.all(c.tx[idx] == x0 + r % T)
                got_t += idx.tolist()
            else:
                r = meta - 2 * NIR
                assert np.all(c.pl[idx] == l - 1) and np.all(c.pz[idx] == z0 // 2 + r // (T // 2))
                assert np.all(c.px[idx] == x0 // 2 + r % (T // 2))
                got_c += idx.tolist()
        assert decode(ent[first + n1 + n2])[3] == total
        zr, xr = (c.pz >= z0 - R) & (c.pz < z0 + T + R), (c.px >= x0 - R) & (c.px < x0 + T + R)
        exp_grad = np.nonzero((c.pl == l) & zr & xr & (c.py >= ylo) & (c.py < yhi))[0]
        assert sorted(got_grad) == exp_grad.tolist()
        zi, xi, yi = (c.pz >= z0) & (c.pz < z0 + T), (c.px >= x0) & (c.px < x0 + T), (c.py >= y0) & (c.py < y0 + B)
        assert sorted(got_p) == np.nonzero((c.pl == l) & zi & xi & yi)[0].tolist()
        ti = ((c.tl == l) & (c.tz >= z0) & (c.tz < z0 + T) & (c.tx >= x0) & (c.tx < x0 + T)
              & (c.ty >= y0) & (c.ty < y0 + B))
        assert sorted(got_t) == np.nonzero(ti)[0].tolist()
        ci = ((c.pl == l - 1) & (c.pz >= z0 // 2) & (c.pz < z0 // 2 + T // 2) & (c.px >= x0 // 2)
              & (c.px < x0 // 2 + T // 2) & (c.py >= y0 // 2) & (c.py < y0 // 2 + B // 2))
        assert sorted(got_c) == np.nonzero(ci)[0].tolist()


MAKERS = {
    "blob64": lambda: S.make_config("blob64", use_cache=False),
    "rand_odd": lambda: S.random_balanced_apr((17, 33, 71), 1, seed=3, p_fine=0.05),
    "rand_thin": lambda: S.random_balanced_apr((9, 5, 70), 1, seed=2, p_fine=0.01),
    "two_wide": lambda: S.random_balanced_apr((2, 2, 40), 0, seed=22, p_fine=0.3),
}


@pytest.mark.parametrize("case", list(MAKERS))
@pytest.mark.parametrize("R", [1, 2])
def test_forward_plans_stage_every_cell_a_target_reads_once(case, R):
    apr = MAKERS[case]()
    lay = G.AprLayout.from_apr(apr, flags=HOST)
    check_forward(Coords(apr), lay, R)


@pytest.mark.parametrize("case", list(MAKERS))
@pytest.mark.parametrize("R", [1, 2])
def test_adjoint_plans_list_the_gradient_rows_and_sources_of_each_tile(case, R):
    apr = MAKERS[case]()
    lay = G.AprLayout.from_apr(apr, flags=HOST)
    check_adjoint(Coords(apr), lay, R)


def test_plan_export_holds_headers_then_entries():
    """The export of a host-only handle's plan: one header per work item, then the entries (at least
    the closing entry of every item)."""
    apr = MAKERS["rand_thin"]()
    lay = G.AprLayout.from_apr(apr, flags=HOST)
    assert lay.export(_abi.APR_STRUCT_FWD_PLAN_R2).shape[0] > len(lay.export(_abi.APR_STRUCT_FWD_ITEMS))
