// Host construction of the device index: validation, the APR tree structure (Sec. 3.4), the
// per-block offsets of every row, and the work lists of non-empty tiles (Sec. 5.2, last paragraph:
// work is launched only where rows hold particles, and only over the y range they occupy).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "apr_internal.h"

namespace aprk {

namespace {

int ceil_log2(int64_t v) {
    int l = 0;
    while ((int64_t(1) << l) < v) ++l;
    return l;
}

// Block offsets of one sorted row: off[j] = #elements with y < j*BY, for j in [0, nb).
void row_block_offsets(const uint16_t *ys, int64_t n, int nb, uint16_t *off) {
    int64_t i = 0;
    for (int j = 0; j < nb; ++j) {
        const int64_t ystart = int64_t(j) * BY;
        while (i < n && ys[i] < ystart) ++i;
        off[j] = uint16_t(i);
    }
}

}  // namespace

apr_status_t build_index(const apr_host_layout &L, uint32_t flags, HostIndex &X, const char **msg) {
    *msg = "";
    if (!L.row_ptr || (L.n_particles > 0 && !L.y_idx)) { *msg = "null array"; return APR_ERR_INVALID_ARG; }
    if (L.n_particles < 0 || L.n_particles >= (int64_t(1) << 31)) { *msg = "n_particles out of range"; return APR_ERR_INVALID_ARG; }
    int64_t maxd = 1;
    for (int a = 0; a < 3; ++a) {
        if (L.dims[a] < 1 || L.dims[a] > 65536) { *msg = "dims must be in [1, 65536]"; return APR_ERR_INVALID_ARG; }
        maxd = std::max(maxd, L.dims[a]);
    }
    const int lmax = ceil_log2(maxd);
    if (L.l_max < lmax || (L.l_max != lmax && !(flags & APR_SUBDOMAIN))) {
        *msg = "l_max must equal ceil(log2(max dim)) (or exceed it for APR_SUBDOMAIN)";
        return APR_ERR_INVALID_LAYOUT;
    }
    if (L.l_min < 0 || L.l_min > L.l_max || L.l_max >= MAXL) { *msg = "bad level range"; return APR_ERR_INVALID_ARG; }

    X.l_min = L.l_min;
    X.l_max = L.l_max;
    for (int a = 0; a < 3; ++a) X.dims[a] = L.dims[a];
    X.np = L.n_particles;

    // ---- level geometry and row counts
    int64_t R = 0, Rt = 0, noff = 0, ntoff = 0;
    for (int l = L.l_min; l <= L.l_max; ++l) {
        LevelGeo &g = X.geo[l];
        g.dz = int32_t(level_cells(L.dims[0], L.l_max, l));
        g.dx = int32_t(level_cells(L.dims[1], L.l_max, l));
        g.dy = int32_t(level_cells(L.dims[2], L.l_max, l));
        g.nb = (g.dy + BY - 1) / BY;
        const int64_t rows = int64_t(g.dz) * g.dx;
        g.row0 = int32_t(R);
        g.off0 = int32_t(noff);
        R += rows;
        noff += rows * g.nb;
        if (l < L.l_max) {
            g.trow0 = int32_t(Rt);
            g.toff0 = int32_t(ntoff);
            Rt += rows;
            ntoff += rows * g.nb;
        }
        if (R >= (int64_t(1) << 31) || noff >= (int64_t(1) << 31)) { *msg = "too many rows"; return APR_ERR_UNSUPPORTED; }
    }
    X.R = R;
    X.Rt = Rt;
    X.noff = noff;
    X.ntoff = ntoff;

    // ---- particle rows: CSR consistency, y order and range (always checked: kernels index with them)
    const int64_t *rp = L.row_ptr;
    if (rp[0] != 0 || rp[R] != L.n_particles) { *msg = "row_ptr must start at 0 and end at n_particles"; return APR_ERR_INVALID_LAYOUT; }
    X.row_ptr.resize(size_t(R) + 1);
    X.y.resize(size_t(L.n_particles));
    X.off.resize(size_t(noff));
    for (int l = L.l_min; l <= L.l_max; ++l) {
        const LevelGeo &g = X.geo[l];
        for (int64_t rr = 0; rr < int64_t(g.dz) * g.dx; ++rr) {
            const int64_t r = g.row0 + rr;
            if (rp[r + 1] < rp[r]) { *msg = "row_ptr not monotone"; return APR_ERR_INVALID_LAYOUT; }
            for (int64_t i = rp[r]; i < rp[r + 1]; ++i) {
                const int32_t yv = L.y_idx[i];
                if (yv < 0 || yv >= g.dy) { *msg = "y index out of the level grid"; return APR_ERR_INVALID_LAYOUT; }
                if (i > rp[r] && yv <= L.y_idx[i - 1]) { *msg = "y not strictly increasing in a row"; return APR_ERR_INVALID_LAYOUT; }
                X.y[size_t(i)] = uint16_t(yv);
            }
            X.row_ptr[size_t(r)] = uint32_t(rp[r]);
            row_block_offsets(X.y.data() + rp[r], rp[r + 1] - rp[r], g.nb, X.off.data() + g.off0 + rr * g.nb);
        }
    }
    X.row_ptr[size_t(R)] = uint32_t(rp[R]);

    // ---- APR tree structure (Sec. 3.4): tree cells of level l = parents of the particles and tree
    // cells of level l+1, merged row by row from the 2x2 child rows, finest level first.
    // tree_rows[l][rr] lists the y of the tree nodes of row rr of level l.
    std::vector<std::vector<std::vector<uint16_t>>> tree_rows(size_t(L.l_max) + 1);
    std::vector<uint32_t> tmp;
    const bool validate = (flags & APR_VALIDATE) != 0;
    for (int l = L.l_max - 1; l >= L.l_min; --l) {
        const LevelGeo &g = X.geo[l], &gc = X.geo[l + 1];
        tree_rows[l].resize(size_t(g.dz) * g.dx);
        for (int32_t z = 0; z < g.dz; ++z)
            for (int32_t x = 0; x < g.dx; ++x) {
                tmp.clear();
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b) {
                        const int32_t cz = 2 * z + a, cx = 2 * x + b;
                        if (cz >= gc.dz || cx >= gc.dx) continue;
                        const int64_t crr = int64_t(cz) * gc.dx + cx;
                        const int64_t r = gc.row0 + crr;
                        for (int64_t i = rp[r]; i < rp[r + 1]; ++i) tmp.push_back(uint32_t(L.y_idx[i]) >> 1);
                        if (l + 1 < L.l_max)
                            for (uint16_t yv : tree_rows[l + 1][size_t(crr)]) tmp.push_back(uint32_t(yv) >> 1);
                    }
                if (tmp.empty()) continue;
                std::sort(tmp.begin(), tmp.end());
                auto &row = tree_rows[l][size_t(int64_t(z) * g.dx + x)];
                for (size_t i = 0; i < tmp.size();) {
                    size_t j = i;
                    while (j < tmp.size() && tmp[j] == tmp[i]) ++j;
                    row.push_back(uint16_t(tmp[i]));
                    if (validate) {
                        // every child inside the level-(l+1) grid must be a particle or a tree node
                        const int32_t yv = int32_t(tmp[i]);
                        const int n = (2 * z + 1 < gc.dz ? 2 : 1) * (2 * x + 1 < gc.dx ? 2 : 1) * (2 * yv + 1 < gc.dy ? 2 : 1);
                        if (int64_t(j - i) != n) { *msg = "particle cells do not cover a tree node's children"; return APR_ERR_INVALID_LAYOUT; }
                    }
                    i = j;
                }
                if (validate) {
                    // a particle cannot also be an interior node (the cells would overlap)
                    const int64_t r = g.row0 + int64_t(z) * g.dx + x;
                    size_t t = 0;
                    for (int64_t i = rp[r]; i < rp[r + 1]; ++i) {
                        while (t < row.size() && row[t] < L.y_idx[i]) ++t;
                        if (t < row.size() && row[t] == L.y_idx[i]) { *msg = "a particle cell overlaps finer particles"; return APR_ERR_INVALID_LAYOUT; }
                    }
                }
            }
    }
    if (validate) {
        // at the coarsest level every cell is a particle or a tree node
        const LevelGeo &g = X.geo[L.l_min];
        int64_t cover = 0;
        const int64_t r0 = g.row0;
        cover += rp[r0 + int64_t(g.dz) * g.dx] - rp[r0];
        if (L.l_min < L.l_max)
            for (const auto &row : tree_rows[L.l_min]) cover += int64_t(row.size());
        if (cover != int64_t(g.dz) * g.dx * g.dy) { *msg = "particle cells do not cover the coarsest level"; return APR_ERR_INVALID_LAYOUT; }
    }

    // ---- flatten the tree into its own linear-access layout
    X.trow_ptr.assign(size_t(Rt) + 1, 0);
    X.toff.assign(size_t(ntoff), 0);
    int64_t nt = 0;
    for (int l = L.l_min; l < L.l_max; ++l) {
        const LevelGeo &g = X.geo[l];
        for (int64_t rr = 0; rr < int64_t(g.dz) * g.dx; ++rr) {
            X.trow_ptr[size_t(g.trow0 + rr)] = uint32_t(nt);
            const auto &row = tree_rows[l][size_t(rr)];
            X.ty.insert(X.ty.end(), row.begin(), row.end());
            row_block_offsets(row.data(), int64_t(row.size()), g.nb, X.toff.data() + g.toff0 + rr * g.nb);
            nt += int64_t(row.size());
        }
    }
    X.trow_ptr[size_t(Rt)] = uint32_t(nt);
    X.nt = nt;
    if (nt >= (int64_t(1) << 31)) { *msg = "too many tree nodes"; return APR_ERR_UNSUPPORTED; }

    // ---- 2:1 balance: for every particle at level l > l_min, the parent of each of its 26
    // neighbours must be a node (particle or tree) of level l-1. This is what lets the convolution
    // fill a level-l patch from levels l and l-1 only (shown for stencil radius <= 2).
    if (flags & APR_REQUIRE_BALANCE) {
        std::vector<uint8_t> node;
        for (int l = L.l_min + 1; l <= L.l_max; ++l) {
            const LevelGeo &g = X.geo[l], &gp = X.geo[l - 1];
            node.assign(size_t(gp.dy), 0);
            int64_t cur = -1;
            for (int32_t z = 0; z < g.dz; ++z)
                for (int32_t x = 0; x < g.dx; ++x) {
                    const int64_t r = g.row0 + int64_t(z) * g.dx + x;
                    if (rp[r + 1] == rp[r]) continue;
                    for (int dz = -1; dz <= 1; ++dz)
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int32_t nz = z + dz, nx = x + dx;
                            if (nz < 0 || nx < 0 || nz >= g.dz || nx >= g.dx) continue;
                            const int64_t prr = int64_t(nz >> 1) * gp.dx + (nx >> 1);
                            if (prr != cur) {
                                std::fill(node.begin(), node.end(), 0);
                                const int64_t pr = gp.row0 + prr;
                                for (int64_t i = rp[pr]; i < rp[pr + 1]; ++i) node[size_t(L.y_idx[i])] = 1;
                                for (uint16_t yv : tree_rows[l - 1][size_t(prr)]) node[yv] = 1;
                                cur = prr;
                            }
                            for (int64_t i = rp[r]; i < rp[r + 1]; ++i)
                                for (int dy = -1; dy <= 1; ++dy) {
                                    const int32_t ny = L.y_idx[i] + dy;
                                    if (ny < 0 || ny >= g.dy) continue;
                                    if (!node[size_t(ny >> 1)]) { *msg = "APR is not 2:1 balanced"; return APR_ERR_INVALID_LAYOUT; }
                                }
                        }
                }
        }
    }

    // ---- work lists
    // forward: (l, tz, tx, yb) tiles holding at least one level-l particle
    // backward: tiles whose interior lies within kMaxRadius cells (Chebyshev) of a level-l particle:
    // every other tile receives no gradient (its staged window holds no nonzero dL/dout)
    constexpr int kMaxRadius = 2;
    X.fwd_items.clear();
    X.bwd_items.clear();
    std::vector<uint8_t> occ, near;
    for (int l = L.l_min; l <= L.l_max; ++l) {
        X.fwd_level_begin[l] = int64_t(X.fwd_items.size());
        X.bwd_level_begin[l] = int64_t(X.bwd_items.size());
        const LevelGeo &g = X.geo[l];
        const int32_t ntz = (g.dz + TZ - 1) / TZ, ntx = (g.dx + TX - 1) / TX;
        occ.assign(size_t(ntz) * ntx * g.nb, 0);
        near.assign(occ.size(), 0);
        auto fdiv = [](int32_t a, int32_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); };
        for (int32_t z = 0; z < g.dz; ++z)
            for (int32_t x = 0; x < g.dx; ++x) {
                const int64_t r = g.row0 + int64_t(z) * g.dx + x;
                for (int64_t i = rp[r]; i < rp[r + 1]; ++i) {
                    const int32_t y = L.y_idx[i];
                    occ[(size_t(z / TZ) * ntx + x / TX) * g.nb + y / BY] = 1;
                    for (int32_t a = std::max(0, fdiv(z - kMaxRadius, TZ)); a <= std::min(ntz - 1, (z + kMaxRadius) / TZ); ++a)
                        for (int32_t b = std::max(0, fdiv(x - kMaxRadius, TX)); b <= std::min(ntx - 1, (x + kMaxRadius) / TX); ++b)
                            for (int32_t j = std::max(0, fdiv(y - kMaxRadius, BY)); j <= std::min(g.nb - 1, (y + kMaxRadius) / BY); ++j)
                                near[(size_t(a) * ntx + b) * g.nb + j] = 1;
                }
            }
        for (int32_t a = 0; a < ntz; ++a)
            for (int32_t b = 0; b < ntx; ++b)
                for (int32_t j = 0; j < g.nb; ++j) {
                    const size_t k = (size_t(a) * ntx + b) * g.nb + j;
                    if (occ[k]) X.fwd_items.push_back(Item{l, a, b, j});
                    if (near[k]) X.bwd_items.push_back(Item{l, a, b, j});
                }
    }
    X.fwd_level_begin[L.l_max + 1] = int64_t(X.fwd_items.size());
    X.bwd_level_begin[L.l_max + 1] = int64_t(X.bwd_items.size());
    for (int l = L.l_max + 2; l <= MAXL; ++l) {
        X.fwd_level_begin[l] = X.fwd_level_begin[L.l_max + 1];
        X.bwd_level_begin[l] = X.bwd_level_begin[L.l_max + 1];
    }

    // tree bricks: (l, z, x, yb) holding at least one tree node
    X.tree_items.clear();
    for (int l = L.l_min; l <= L.l_max; ++l) {
        X.tree_level_begin[l] = int64_t(X.tree_items.size());
        if (l == L.l_max) continue;
        const LevelGeo &g = X.geo[l];
        for (int32_t z = 0; z < g.dz; ++z)
            for (int32_t x = 0; x < g.dx; ++x) {
                const auto &row = tree_rows[l][size_t(int64_t(z) * g.dx + x)];
                int32_t last = -1;
                for (uint16_t yv : row) {
                    const int32_t j = yv / BY;
                    if (j != last) { X.tree_items.push_back(Item{l, z, x, j}); last = j; }
                }
            }
    }
    X.tree_level_begin[L.l_max + 1] = int64_t(X.tree_items.size());
    for (int l = L.l_max + 2; l <= MAXL; ++l) X.tree_level_begin[l] = X.tree_level_begin[L.l_max + 1];
    return APR_OK;
}

}  // namespace aprk
