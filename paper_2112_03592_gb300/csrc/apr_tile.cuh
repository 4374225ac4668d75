// Geometry of a convolution tile and the source segments of its staged patch. Shared by the kernels
// (apr_kernels.cu) and the host builder of the tile plans (apr_plan.cu): both sides use these
// definitions, so a plan lists exactly the segments a kernel would compute.
#pragma once

#include "apr_device.cuh"
#include "apr_internal.h"

namespace aprk {
namespace dev {

constexpr int WIN = 8;                 // y cells per compute window
constexpr int NWIN = BY / WIN;         // windows per interior row
constexpr int NIR = TZ * TX;           // interior rows of a tile
constexpr int NIW = NIR * NWIN;        // window slots of a tile
static_assert(NIW == 2 * NT, "window slots are scanned two per thread");

template <int R>
struct Geo {
    static constexpr int K = 2 * R + 1;
    static constexpr int K3 = K * K * K;
    static constexpr int NPAIR = K * K;                    // (dz, dx) pairs
    static constexpr int PZ = TZ + 2 * R, PX = TX + 2 * R, PY = BY + 2 * R;
    static constexpr int PYS = (PY + 3) / 4 * 4;           // row stride, 16-byte multiple
    static constexpr int NROW = PZ * PX;
    static constexpr int NSEG = 3 * NROW;                  // particle, tree, coarser-particle source per row
    static constexpr int NCZ = ((TZ + R - 1) >> 1) + ((R + 1) >> 1) + 1;  // level-(l-1) rows per axis under a patch
    static constexpr int NRSEG = 2 * NIR + NIR / 4;        // backward routing: particles, tree, coarser particles
    static_assert(WIN + 2 * R <= 12, "a window's taps must fit three 16-byte loads");
    static_assert((NWIN - 1) * WIN + 12 <= PYS, "window loads stay inside the row");
    static_assert(NSEG <= 2 * NT && NROW + NRSEG <= 2 * NT, "segments are scanned two per thread");
    static_assert(NCZ * NCZ <= NROW && PZ < 15 && PX < 15, "once-staged coarse rows: segment count, 4-bit row fields");
    static_assert(NROW < 256 && NIR < 127 && NROW + NRSEG < 65536, "meta fields: 8-bit patch row, 7-bit interior row");
};

// meta of a forward segment of kinds 0-2: patch row | kind << 8, plus META_REFL if the patch row lies
// outside the grid (the segment holds the reflected row; with zero boundary it is empty); kind 3:
// (first covered patch row z + 1) | (x + 1) << 4 | 3 << 8. These 11 bits are what a plan stores;
// with_trow adds (interior row + 1) << 11 for the particle segments of interior rows.
constexpr int META_REFL = 1 << 10;
__host__ __device__ __forceinline__ int meta_kind(int meta) { return (meta >> 8) & 3; }
__host__ __device__ __forceinline__ int meta_trow(int meta) { return ((meta >> 11) & 127) - 1; }

template <int R>
__host__ __device__ __forceinline__ int with_trow(const LevelGeo &g, const Item &it, int meta) {
    using G = Geo<R>;
    if (meta_kind(meta) != 0) return meta;
    const int pr = meta & 255;
    const int a = pr / G::PX - R, b = pr % G::PX - R;
    const bool target = a >= 0 && a < TZ && b >= 0 && b < TX && it.a * TZ + a < g.dz && it.b * TX + b < g.dx;
    return target ? meta | ((a * TX + b + 1) << 11) : meta;
}

// Forward tile plans: per work item and stencil radius, the non-empty segments of fwd_segment in
// segment order, each with the prefix of 8-element packets before it (the packets of segment
// [lo, lo + n) are the aligned groups lo >> 3 .. (lo + n - 1) >> 3). An item's entries are followed
// by one entry whose prefix is the item's packet total. Two 32-bit words:
//   w0 = lo (28 bits) | n[3:0] << 28,   w1 = packet prefix (16 bits) | meta (11 bits) << 16 | n[7:4] << 27.
struct FPlanEnt {
    uint32_t w0, w1;
};
constexpr int64_t FPLAN_MAX_INDEX = int64_t(1) << 28;  // particles and tree nodes an index may hold
__host__ __device__ __forceinline__ FPlanEnt fplan_encode(int lo, int n, int meta, int ppre) {
    return FPlanEnt{uint32_t(lo) | (uint32_t(n & 15) << 28),
                    uint32_t(ppre & 0xffff) | (uint32_t(meta & 0x7ff) << 16) | (uint32_t(n >> 4) << 27)};
}
__host__ __device__ __forceinline__ int fplan_lo(const FPlanEnt &e) { return int(e.w0 & 0x0fffffffu); }
__host__ __device__ __forceinline__ int fplan_n(const FPlanEnt &e) { return int(e.w0 >> 28) | int((e.w1 >> 27) << 4); }
__host__ __device__ __forceinline__ int fplan_meta(const FPlanEnt &e) { return int((e.w1 >> 16) & 0x7ffu); }
__host__ __device__ __forceinline__ int fplan_pre(const FPlanEnt &e) { return int(e.w1 & 0xffffu); }
__host__ __device__ __forceinline__ int packets_of(int lo, int n) { return n > 0 ? ((lo + n + 7) >> 3) - (lo >> 3) : 0; }

// Whether the forward patch of item it (rows z0-R .. z0+TZ+R, x likewise, y y0-R .. y0+BY+R) reaches
// outside the level grid.
template <int R>
__host__ __device__ inline bool fwd_tile_at_boundary(const DevLayout &L, const Item &it) {
    using G = Geo<R>;
    const LevelGeo &g = L.geo[it.l];
    const int z0 = it.a * TZ, x0 = it.b * TX, yw = it.yb * BY - R;
    return z0 - R < 0 || x0 - R < 0 || yw < 0 || z0 + TZ + R > g.dz || x0 + TX + R > g.dx || yw + G::PY > g.dy;
}

// Segment s of the forward patch of item it (Sec. 3.5: the sources of u_l), reflecting boundary.
// Segments [0, NROW): level-l particles of every patch row, [NROW, 2 NROW): level-l tree nodes,
// [2 NROW, 3 NROW): level-(l-1) particles. Away from the grid boundary each level-(l-1) row under the
// patch is one segment (the first NCZ^2, kind 3), written to the (up to 2 x 2) patch rows it covers;
// tiles reaching outside the grid take one level-(l-1) row per patch row (kind 2), which follows the
// reflection of every row. [lo, hi): index range holding the row's elements in y [y0-R, y0+BY+R)
// (row_range: possibly a few more).
template <int R>
__host__ __device__ inline void fwd_segment(const DevLayout &L, const Item &it, bool boundary, int s, int &lo,
                                            int &hi, int &meta) {
    using G = Geo<R>;
    const int l = it.l;
    const LevelGeo &g = L.geo[l];
    const int z0 = it.a * TZ, x0 = it.b * TX, yw = it.yb * BY - R;
    const int kind = s / G::NROW, pr = s % G::NROW;
    const int ylo = imax(yw, 0), yhi = imin(yw + G::PY, g.dy);
    lo = 0;
    hi = 0;
    meta = 0;
    if (kind == 2 && !boundary) {
        if (pr < G::NCZ * G::NCZ && l > L.l_min) {
            const LevelGeo &gp = L.geo[l - 1];
            const int cz = ((z0 - R) >> 1) + pr / G::NCZ, cx = ((x0 - R) >> 1) + pr % G::NCZ;
            if (cz < gp.dz && cx < gp.dx)
                row_range(L.row_ptr, L.off, gp.row0, gp.off0, gp.nb, cz * gp.dx + cx, ylo >> 1, ((yhi - 1) >> 1) + 1,
                          lo, hi);
            meta = (2 * cz - (z0 - R) + 1) | ((2 * cx - (x0 - R) + 1) << 4) | (3 << 8);
        }
        return;
    }
    int z = z0 - R + pr / G::PX, x = x0 - R + pr % G::PX;
    const bool inside = z >= 0 && z < g.dz && x >= 0 && x < g.dx;
    if (!inside) {
        z = reflect_idx(z, g.dz);
        x = reflect_idx(x, g.dx);
    }
    const int rr = z * g.dx + x;
    if (kind == 0) {
        row_range(L.row_ptr, L.off, g.row0, g.off0, g.nb, rr, ylo, yhi, lo, hi);
    } else if (kind == 1) {
        if (l < L.l_max) row_range(L.trow_ptr, L.toff, g.trow0, g.toff0, g.nb, rr, ylo, yhi, lo, hi);
    } else if (l > L.l_min) {
        const LevelGeo &gp = L.geo[l - 1];
        const int prr = (z >> 1) * gp.dx + (x >> 1);
        row_range(L.row_ptr, L.off, gp.row0, gp.off0, gp.nb, prr, ylo >> 1, ((yhi - 1) >> 1) + 1, lo, hi);
    }
    meta = pr | (kind << 8) | (inside ? 0 : META_REFL);
}

// Segment s of the data-adjoint tile of item it. [0, NROW): gradient rows, the level-l particles of
// every in-grid patch row (the gradient is zero outside the grid, so nothing is reflected);
// [NROW, NROW + NRSEG): the sources of the interior cells, q = s - NROW: particles (q < NIR) and tree
// nodes (q < 2 NIR) of interior row q mod NIR in y-block yb, then the level-(l-1) particles under the
// interior (TZ/2 x TX/2 parent rows, parent y in [y0/2, y0/2 + BY/2)).
template <int R>
__host__ __device__ inline void bwd_segment(const DevLayout &L, const Item &it, int s, int &lo, int &hi) {
    using G = Geo<R>;
    const int l = it.l;
    const LevelGeo &g = L.geo[l];
    const int z0 = it.a * TZ, x0 = it.b * TX, y0 = it.yb * BY, yw = y0 - R;
    lo = 0;
    hi = 0;
    if (s < G::NROW) {
        const int z = z0 - R + s / G::PX, x = x0 - R + s % G::PX;
        if (z >= 0 && z < g.dz && x >= 0 && x < g.dx)
            row_range(L.row_ptr, L.off, g.row0, g.off0, g.nb, z * g.dx + x, imax(yw, 0), imin(yw + G::PY, g.dy), lo, hi);
        return;
    }
    const int q = s - G::NROW;
    if (q < 2 * NIR) {
        const int r = q % NIR;
        const int z = z0 + r / TX, x = x0 + r % TX;
        if (z < g.dz && x < g.dx) {
            const int rr = z * g.dx + x;
            if (q < NIR) {
                lo = int(blk_start(L.row_ptr, L.off, g.row0, g.off0, g.nb, rr, it.yb));
                hi = int(blk_start(L.row_ptr, L.off, g.row0, g.off0, g.nb, rr, it.yb + 1));
            } else if (l < L.l_max) {
                lo = int(blk_start(L.trow_ptr, L.toff, g.trow0, g.toff0, g.nb, rr, it.yb));
                hi = int(blk_start(L.trow_ptr, L.toff, g.trow0, g.toff0, g.nb, rr, it.yb + 1));
            }
        }
    } else if (l > L.l_min) {
        const int r = q - 2 * NIR;
        const LevelGeo &gq = L.geo[l - 1];
        const int pz = z0 / 2 + r / (TX / 2), px = x0 / 2 + r % (TX / 2);
        if (pz < gq.dz && px < gq.dx)
            row_range(L.row_ptr, L.off, gq.row0, gq.off0, gq.nb, pz * gq.dx + px, y0 / 2, imin(y0 / 2 + BY / 2, gq.dy),
                      lo, hi);
    }
}

}  // namespace dev
}  // namespace aprk
