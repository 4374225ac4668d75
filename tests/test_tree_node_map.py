"""Tree-node child maps (the index the tree restriction and push-down kernels read), on the host.

Each tree node (Sec. 3.4) averages the cells (2z + a, 2x + b, 2y + e) of the next finer level that lie
in the level grid, each of which is a particle or a tree node of that level. The library's map is
checked entry by entry against the children found independently from the input particle rows and
the oracle's own tree, and the average it encodes is checked against the oracle's tree values.
"""
import numpy as np
import pytest

import aprsynth as S
import oracle
import paper_2112_03592_gb300 as G
from paper_2112_03592_gb300 import _abi

HOST = G.APR_VALIDATE | G.APR_REQUIRE_BALANCE | G.APR_HOST_ONLY
INDEX = (1 << 30) - 1


def decode(words):
    """(kind, index) of the 8 children of one node in (a, b, e) order; kind 0 absent, 1 particle, 2 node."""
    out = []
    for k in range(4):
        pw, tw = int(words[k]) & 0xFFFFFFFF, int(words[4 + k]) & 0xFFFFFFFF
        pm, tm = pw >> 30, tw >> 30
        for e in range(2):
            if (pm >> e) & 1:
                out.append((1, (pw & INDEX) + (e and (pm & 1))))
            elif (tm >> e) & 1:
                out.append((2, (tw & INDEX) + (e and (tm & 1))))
            else:
                out.append((0, -1))
    return out


def expected_children(apr, o):
    """Children of every oracle tree node, from the particle rows of the input and the oracle's
    tree coordinates (no library code)."""
    tc = o.tree_coords()
    node_at = {tuple(r): i for i, r in enumerate(tc.tolist())}
    exp = []
    for (l, z, x, y) in tc.tolist():
        dz, dx, dy = apr.level_dims(l + 1)
        r0 = apr.level_row_offset(l + 1)
        kids = []
        for a in range(2):
            for b in range(2):
                cz, cx = 2 * z + a, 2 * x + b
                row = None
                if cz < dz and cx < dx:
                    r = r0 + cz * dx + cx
                    lo, hi = int(apr.row_ptr[r]), int(apr.row_ptr[r + 1])
                    row = (lo, apr.y_idx[lo:hi])
                for e in range(2):
                    cy = 2 * y + e
                    if row is None or cy >= dy:
                        kids.append((0, -1))
                        continue
                    lo, ys = row
                    j = int(np.searchsorted(ys, cy))
                    if j < len(ys) and int(ys[j]) == cy:
                        kids.append((1, lo + j))
                    elif (l + 1, cz, cx, cy) in node_at:
                        kids.append((2, node_at[(l + 1, cz, cx, cy)]))
                    else:
                        kids.append((0, -1))
        exp.append(kids)
    return exp


@pytest.mark.parametrize("maker", [
    lambda: S.make_config("blob64", use_cache=False),
    lambda: S.random_balanced_apr((12, 16, 10), 1, seed=1),
    lambda: S.random_balanced_apr((9, 5, 70), 1, seed=2, p_fine=0.01),
    lambda: S.random_balanced_apr((17, 33, 71), 1, seed=3, p_fine=0.05),
    lambda: S.random_balanced_apr((3, 1, 130), 0, seed=3),
    lambda: S.uniform_level_apr((16, 8, 8), 4),
    lambda: S.uniform_level_apr((16, 8, 8), 2, l_min=1),
])
def test_child_map_matches_the_children_of_every_node(maker):
    apr = maker()
    lay = G.AprLayout.from_apr(apr, flags=HOST)
    o = oracle.Oracle(apr)
    m = lay.export(_abi.APR_STRUCT_TREE_NODE_MAP)
    assert m.shape == (o.n_tree, 8)
    exp = expected_children(apr, o)
    got = [decode(m[t]) for t in range(o.n_tree)]
    assert got == exp
    # every in-grid child cell of a node of a complete APR is a particle or a node
    for (l, z, x, y), kids in zip(o.tree_coords().tolist(), got):
        dz, dx, dy = apr.level_dims(l + 1)
        n_in = sum(1 for a in range(2) for b in range(2) for e in range(2)
                   if 2 * z + a < dz and 2 * x + b < dx and 2 * y + e < dy)
        assert sum(1 for kind, _ in kids if kind) == n_in


def test_child_map_average_equals_oracle_tree_values():
    """The average the map encodes, level by level from the finest, equals the oracle's tree fill."""
    apr = S.random_balanced_apr((17, 33, 71), 1, seed=3, p_fine=0.05)
    rng = np.random.default_rng(7)
    v = rng.uniform(0.5, 2.0, apr.n_particles)
    lay = G.AprLayout.from_apr(apr, flags=HOST)
    o = oracle.Oracle(apr, v)
    ref = o.tree()[:, 0]
    m = lay.export(_abi.APR_STRUCT_TREE_NODE_MAP)
    tc = o.tree_coords()
    tree = np.zeros(o.n_tree)
    for l in sorted(set(tc[:, 0].tolist()), reverse=True):
        for t in np.nonzero(tc[:, 0] == l)[0]:
            vals = [v[i] if kind == 1 else tree[i] for kind, i in decode(m[t]) if kind]
            tree[t] = sum(vals) / len(vals)
    np.testing.assert_allclose(tree, ref, rtol=1e-12, atol=0)


def test_child_map_rejects_nothing_and_is_empty_without_a_tree():
    apr = S.uniform_level_apr((8, 8, 8), 3, l_min=3)
    lay = G.AprLayout.from_apr(apr, flags=HOST)
    assert lay.n_tree == 0
    assert lay.export(_abi.APR_STRUCT_TREE_NODE_MAP).shape == (0, 8)
