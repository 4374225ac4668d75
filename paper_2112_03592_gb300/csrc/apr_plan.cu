// Tile plans (host): for every forward and data-adjoint work item and both stencil radii, the
// non-empty source segments of the item's patch, listed once per APR so that the kernels read them
// with one coalesced load instead of evaluating every row's offsets (and a block scan) per call.
// The segments are those of fwd_segment / bwd_segment (apr_tile.cuh), evaluated here on the host
// copy of the index; forward entries carry the prefix of their 8-element packets. The multi-channel
// sub-tile plans come from build_mc_plans (apr_mc.cu).
#include <functional>
#include <thread>
#include <vector>

#include "apr_tile.cuh"

namespace aprk {

DevLayout host_layout_view(const HostIndex &X) {
    DevLayout L{};
    L.row_ptr = X.row_ptr.data();
    L.y = X.y.data();
    L.off = X.off.data();
    L.trow_ptr = X.trow_ptr.data();
    L.ty = X.ty.data();
    L.toff = X.toff.data();
    L.np = int32_t(X.np);
    L.nt = int32_t(X.nt);
    L.l_min = X.l_min;
    L.l_max = X.l_max;
    for (int l = 0; l < MAXL; ++l) L.geo[l] = X.geo[l];
    return L;
}

namespace {

using namespace dev;

// Narrows [lo, hi) of a sorted y range to the elements with y in [ya, yb).
void trim_y(const uint16_t *ys, int &lo, int &hi, int ya, int yb) {
    while (lo < hi && int(ys[lo]) < ya) ++lo;
    while (hi > lo && int(ys[hi - 1]) >= yb) --hi;
}

// Forward items: the non-empty segments with their packet prefixes; the entry after an item's
// segments holds its packet total. Totals above 65535 (not reachable: at most 3 (8 + 2R)^2
// segments of at most 2 BY + 2R elements, i.e. fewer than 10 000 packets) set `overflow`.
template <int R>
bool fwd_plan(const DevLayout &L, const std::vector<Item> &items, HostFPlan &P) {
    using G = Geo<R>;
    P.hdr.assign(items.size(), PlanHdr{0, 0});
    P.ent.clear();
    bool overflow = false;
    for (size_t t = 0; t < items.size(); ++t) {
        const Item &it = items[t];
        const bool bnd = fwd_tile_at_boundary<R>(L, it);
        const int first = int(P.ent.size());
        int total = 0;
        const LevelGeo &g = L.geo[it.l];
        const int yw = it.yb * BY - R, ylo = imax(yw, 0), yhi = imin(yw + G::PY, g.dy);
        for (int s = 0; s < G::NSEG; ++s) {
            int lo, hi, meta;
            fwd_segment<R>(L, it, bnd, s, lo, hi, meta);
            // exactly the elements whose cells lie in the patch window
            const int kind = meta_kind(meta);
            if (kind == 0) trim_y(L.y, lo, hi, ylo, yhi);
            else if (kind == 1) trim_y(L.ty, lo, hi, ylo, yhi);
            else trim_y(L.y, lo, hi, ylo >> 1, ((yhi - 1) >> 1) + 1);
            if (hi <= lo) continue;
            if (hi - lo > 255) overflow = true;
            const FPlanEnt e = fplan_encode(lo, hi - lo, meta, total);
            P.ent.push_back(uint2{e.w0, e.w1});
            total += packets_of(lo, hi - lo);
            if (total > 65535) overflow = true;
        }
        const FPlanEnt e = fplan_encode(0, 0, 0, total);
        P.ent.push_back(uint2{e.w0, e.w1});
        P.hdr[t] = PlanHdr{first, int(P.ent.size()) - 1 - first};
    }
    return !overflow;
}

// Adjoint items (bwd_segment): count = n1 | n2 << 16 (gradient rows, then routing segments); meta =
// the segment's index within its group (patch row, routing index q). Gradient rows are trimmed to
// the patch window and coarser-particle routing segments to the interior's parent cells, so every
// listed element lands in the tile.
template <int R>
bool bwd_plan(const DevLayout &L, const std::vector<Item> &items, HostFPlan &P) {
    using G = Geo<R>;
    P.hdr.assign(items.size(), PlanHdr{0, 0});
    P.ent.clear();
    bool overflow = false;
    for (size_t t = 0; t < items.size(); ++t) {
        const Item &it = items[t];
        const LevelGeo &g = L.geo[it.l];
        const int yw = it.yb * BY - R, y0 = it.yb * BY;
        const int first = int(P.ent.size());
        int total = 0, n1 = 0;
        for (int s = 0; s < G::NROW + G::NRSEG; ++s) {
            int lo, hi;
            bwd_segment<R>(L, it, s, lo, hi);
            const int q = s - G::NROW;
            if (s < G::NROW) {
                trim_y(L.y, lo, hi, imax(yw, 0), imin(yw + G::PY, g.dy));
            } else if (q >= 2 * NIR && it.l > L.l_min) {
                trim_y(L.y, lo, hi, y0 / 2, y0 / 2 + BY / 2);
            }
            if (hi <= lo) continue;
            if (hi - lo > 255) overflow = true;
            const FPlanEnt e = fplan_encode(lo, hi - lo, s < G::NROW ? s : q, total);
            P.ent.push_back(uint2{e.w0, e.w1});
            total += packets_of(lo, hi - lo);
            if (total > 65535) overflow = true;
            if (s < G::NROW) ++n1;
        }
        const FPlanEnt e = fplan_encode(0, 0, 0, total);
        P.ent.push_back(uint2{e.w0, e.w1});
        const int n = int(P.ent.size()) - 1 - first;
        P.hdr[t] = PlanHdr{first, n1 | ((n - n1) << 16)};
    }
    return !overflow;
}

}  // namespace

bool tree_node_plan(const DevLayout &L, const HostIndex &X, std::vector<TreeNodePlan> &P) {
    P.assign(size_t(X.nt), TreeNodePlan{});
    for (int l = L.l_min; l < L.l_max; ++l) {
        const LevelGeo g = L.geo[l], gc = L.geo[l + 1];
        const bool child_tree = l + 1 < L.l_max;
        for (int z = 0; z < g.dz; ++z)
            for (int x = 0; x < g.dx; ++x) {
                const int64_t rr = g.trow0 + int64_t(z) * g.dx + x;
                const int64_t n0 = L.trow_ptr[rr], n1 = L.trow_ptr[rr + 1];
                if (n0 == n1) continue;
                for (int k = 0; k < 4; ++k) {
                    const int cz = 2 * z + (k >> 1), cx = 2 * x + (k & 1);
                    const bool in_grid = cz < gc.dz && cx < gc.dx;
                    // the child row's particles [pa, pe) and tree nodes [ta, te), merged with the
                    // node row in y order (child cells 2y, 2y + 1 of consecutive nodes increase)
                    int64_t pa = 0, pe = 0, ta = 0, te = 0;
                    if (in_grid) {
                        const int64_t crr = int64_t(cz) * gc.dx + cx;
                        pa = L.row_ptr[gc.row0 + crr];
                        pe = L.row_ptr[gc.row0 + crr + 1];
                        if (child_tree) {
                            ta = L.trow_ptr[gc.trow0 + crr];
                            te = L.trow_ptr[gc.trow0 + crr + 1];
                        }
                    }
                    for (int64_t i = n0; i < n1; ++i) {
                        const int cy0 = 2 * int(L.ty[i]);
                        while (pa < pe && int(L.y[pa]) < cy0) ++pa;
                        while (ta < te && int(L.ty[ta]) < cy0) ++ta;
                        uint32_t pw = uint32_t(pa), tw = uint32_t(ta);
                        for (int e = 0; e < 2; ++e) {
                            const int cy = cy0 + e;
                            if (!in_grid || cy >= gc.dy) continue;
                            if (pa < pe && int(L.y[pa]) == cy) {
                                pw |= 1u << (30 + e);
                                ++pa;
                            } else if (ta < te && int(L.ty[ta]) == cy) {
                                tw |= 1u << (30 + e);
                                ++ta;
                            }
                            // else: neither (only in a sub-domain's partial index): the child is left
                            // out of the node's average and of its push-down
                        }
                        P[size_t(i)].p[k] = int32_t(pw);
                        P[size_t(i)].t[k] = int32_t(tw);
                    }
                }
            }
    }
    return true;
}

apr_status_t build_plans(HostIndex &X) {
    const DevLayout L = host_layout_view(X);
    if (X.np >= FPLAN_MAX_INDEX || X.nt >= FPLAN_MAX_INDEX) return APR_ERR_UNSUPPORTED;
    apr_status_t st[6] = {APR_OK, APR_OK, APR_OK, APR_OK, APR_OK, APR_OK};
    auto guarded = [&st](int i, auto f) {
        return [&st, i, f] {
            try {
                if (!f()) st[i] = APR_ERR_UNSUPPORTED;
            } catch (...) {  // host allocation failure
                st[i] = APR_ERR_OOM;
            }
        };
    };
    std::function<void()> jobs[6] = {guarded(0, [&] { return fwd_plan<1>(L, X.fwd_items, X.fplan[0]); }),
                                     guarded(1, [&] { return fwd_plan<2>(L, X.fwd_items, X.fplan[1]); }),
                                     guarded(2, [&] { return bwd_plan<1>(L, X.bwd_items, X.bplan[0]); }),
                                     guarded(3, [&] { return bwd_plan<2>(L, X.bwd_items, X.bplan[1]); }),
                                     guarded(4, [&] { return build_mc_plans(L, X, X.mcfplan, X.mcbplan); }),
                                     guarded(5, [&] { return tree_node_plan(L, X, X.tnplan); })};
    // one thread per plan; a job whose thread cannot be started runs here
    std::vector<std::thread> threads;
    try {
        threads.reserve(6);
    } catch (...) {  // the jobs then run here
    }
    for (auto &job : jobs) {
        try {
            threads.emplace_back(job);
        } catch (...) {
            job();
        }
    }
    for (auto &th : threads) th.join();
    for (apr_status_t s : st)
        if (s != APR_OK) return s;
    return APR_OK;
}

}  // namespace aprk
