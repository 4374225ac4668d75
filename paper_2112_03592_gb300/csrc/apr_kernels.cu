// CUDA kernels (sm_103a) for APR-native convolution, its tree restriction and their adjoints.
//
// Data layout in device memory (built by apr_index.cpp, Sec. 3.1 Alg. 1 extended):
//   row_ptr[R+1] (uint32), y[N_p] (uint16), off[rows * nb] (uint16): for every row (l, z, x) and
//   y-block j of BY cells, the offset of the row's first particle with y >= j*BY. The tree has the
//   same three arrays. A work item names a tile of TZ x TX rows and one y-block of one level.
//
// Every kernel finds the particles of a tile's neighbourhood from block offsets (no searches), reads
// y indices and values with consecutive lanes on consecutive particles (coalesced), and stages an
// isotropic level-l patch in shared memory (Sec. 3.5): same-level particles directly, the
// coarser (level l-1) particle of each remaining cell piecewise-constant, and finer content through
// the level-l tree node (Sec. 4.1, Fig. treeconv).
#include <cuda_runtime.h>

#include <cstdint>

#include "apr_internal.h"

namespace aprk {

namespace {

constexpr int NT = 256;  // threads per block of every kernel below

__device__ __forceinline__ int reflect_idx(int i, int d) {
    // half-sample symmetric reflection into [0, d), repeated for grids smaller than the stencil
    const int p = 2 * d;
    int m = i % p;
    if (m < 0) m += p;
    return m >= d ? p - 1 - m : m;
}

// First particle of y-block j of row rr (level geometry g); j == nb gives the row end.
__device__ __forceinline__ uint32_t pblock(const DevLayout &L, const LevelGeo &g, int rr, int j) {
    if (j >= g.nb) return L.row_ptr[g.row0 + rr + 1];
    return L.row_ptr[g.row0 + rr] + L.off[g.off0 + rr * g.nb + j];
}

__device__ __forceinline__ uint32_t tblock(const DevLayout &L, const LevelGeo &g, int rr, int j) {
    if (j >= g.nb) return L.trow_ptr[g.trow0 + rr + 1];
    return L.trow_ptr[g.trow0 + rr] + L.toff[g.toff0 + rr * g.nb + j];
}

// Positions v in [-R, d + R) with reflect(v) == c: c itself and the out-of-grid positions that
// mirror onto it (at most 2R of them). Returns the count.
template <int R>
__device__ __forceinline__ int preimages(int c, int d, int *out) {
    int n = 0;
    out[n++] = c;
    for (int v = -R; v < 0; ++v)
        if (reflect_idx(v, d) == c) out[n++] = v;
    for (int v = d; v < d + R; ++v)
        if (reflect_idx(v, d) == c) out[n++] = v;
    return n;
}

template <int R>
struct Geo {
    static constexpr int K = 2 * R + 1;
    static constexpr int K3 = K * K * K;
    // forward patch: tile rows plus R halo rows; y-block plus R halo cells
    static constexpr int PZ = TZ + 2 * R, PX = TX + 2 * R, PY = BY + 2 * R, PYS = PY + 1;
    static constexpr int NROW = PZ * PX;
    static constexpr int NSEG = 3 * NROW;  // particle, tree and parent-level segment per patch row
    // backward gradient patch: halo 2R (taps of halo cells reach 2R)
    static constexpr int GZ = TZ + 4 * R, GX = TX + 4 * R, GY = BY + 4 * R, GYS = GY + 1;
    static constexpr int NGROW = GZ * GX;
};

// ------------------------------------------------------------------------------------------------
// Forward patch staging shared by the convolution and the stencil-gradient kernels.
// Fills patch[NROW][PYS] with the isotropic level-l values of cells
//   z in [tz*TZ - R, tz*TZ + TZ + R), x likewise, y in [yb*BY - R, yb*BY + BY + R)
// (rows outside the grid: reflected rows or zeros; cells outside in y: reflected cells or zeros).
// Also lists the tile's target particles (level-l particles of the TZ x TX interior rows inside
// y-block yb): tgt_lo[r], tgt_pre[r] (prefix counts, tgt_pre[TZ*TX] = total).
// ------------------------------------------------------------------------------------------------
template <int R>
__device__ void stage_forward_patch(const DevLayout &L, const Item &it, const float *__restrict__ vals,
                                    const float *__restrict__ tree, int bc, float *patch, int *seg_lo,
                                    int *seg_hi, int *row_valid, int *tgt_lo, int *tgt_pre) {
    using G = Geo<R>;
    const int tid = threadIdx.x;
    const int l = it.l;
    const LevelGeo g = L.geo[l];
    const int yw = it.yb * BY - R;  // level y of patch column 0

    for (int i = tid; i < G::NROW * G::PYS; i += NT) patch[i] = __int_as_float(0x7fc00000);  // NaN: unfilled
    if (tid < G::NSEG) {
        const int s = tid, kind = s / G::NROW, pr = s % G::NROW;
        const int a = pr / G::PX, b = pr % G::PX;
        int z = it.a * TZ - R + a, x = it.b * TX - R + b;
        const bool inside = z >= 0 && z < g.dz && x >= 0 && x < g.dx;
        const bool use = inside || bc == APR_BC_REFLECT;
        uint32_t lo = 0, hi = 0;
        if (use) {
            z = reflect_idx(z, g.dz);
            x = reflect_idx(x, g.dx);
            const int ylo = max(yw, 0), yhi = min(yw + G::PY, g.dy);  // in-grid y range of the patch
            const int rr = z * g.dx + x;
            if (kind == 0) {
                lo = pblock(L, g, rr, ylo / BY);
                hi = pblock(L, g, rr, (yhi - 1) / BY + 1);
            } else if (kind == 1) {
                if (l < L.l_max) {
                    lo = tblock(L, g, rr, ylo / BY);
                    hi = tblock(L, g, rr, (yhi - 1) / BY + 1);
                }
            } else if (l > L.l_min) {
                const LevelGeo gp = L.geo[l - 1];
                const int prr = (z >> 1) * gp.dx + (x >> 1);
                lo = pblock(L, gp, prr, (ylo >> 1) / BY);
                hi = pblock(L, gp, prr, ((yhi - 1) >> 1) / BY + 1);
            }
        }
        seg_lo[s] = int(lo);
        seg_hi[s] = int(hi);
        if (kind == 0) row_valid[pr] = use ? 1 : 0;
    }
    if (tid < TZ * TX) {
        const int z = it.a * TZ + tid / TX, x = it.b * TX + tid % TX;
        uint32_t lo = 0, hi = 0;
        if (z < g.dz && x < g.dx) {
            const int rr = z * g.dx + x;
            lo = pblock(L, g, rr, it.yb);
            hi = pblock(L, g, rr, it.yb + 1);
        }
        tgt_lo[tid] = int(lo);
        tgt_pre[tid + 1] = int(hi - lo);
    }
    __syncthreads();
    if (tid == 0) {
        tgt_pre[0] = 0;
        for (int r = 0; r < TZ * TX; ++r) tgt_pre[r + 1] += tgt_pre[r];
    }
    // fill: one warp per segment, consecutive lanes on consecutive particles
    const int warp = tid >> 5, lane = tid & 31;
    for (int s = warp; s < G::NSEG; s += NT / 32) {
        const int lo = seg_lo[s], hi = seg_hi[s];
        const int kind = s / G::NROW;
        float *prow = patch + (s % G::NROW) * G::PYS;
        if (kind < 2) {
            const uint16_t *ys = kind == 0 ? L.y : L.ty;
            const float *src = kind == 0 ? vals : tree;
            for (int i = lo + lane; i < hi; i += 32) {
                const int pos = int(ys[i]) - yw;
                const float v = src[i];
                if (pos >= 0 && pos < G::PY) prow[pos] = v;
            }
        } else {
            for (int i = lo + lane; i < hi; i += 32) {
                const int yy = 2 * int(L.y[i]);  // first level-l cell of the coarser particle
                const float v = vals[i];
                const int pos = yy - yw;
                if (pos >= 0 && pos < G::PY && yy < g.dy) prow[pos] = v;
                if (pos + 1 >= 0 && pos + 1 < G::PY && yy + 1 < g.dy) prow[pos + 1] = v;
            }
        }
    }
    __syncthreads();
    // cells outside the grid in y: mirror (reflect) or zero; rows outside with zero boundary: zero
    for (int i = tid; i < G::NROW * G::PY; i += NT) {
        const int pr = i / G::PY, pos = i % G::PY;
        float *prow = patch + pr * G::PYS;
        if (!row_valid[pr]) {
            prow[pos] = 0.f;
            continue;
        }
        const int yy = yw + pos;
        if (yy < 0 || yy >= g.dy) prow[pos] = bc == APR_BC_REFLECT ? prow[reflect_idx(yy, g.dy) - yw] : 0.f;
    }
    __syncthreads();
}

// ------------------------------------------------------------------------------------------------
// APR convolution, one block per work item (Sec. 4.1; Sec. 5.2 with a tile of TZ x TX rows and a
// y-block instead of the paper's 4x4 / 8x8 warp grid and sliding buffer).
// ------------------------------------------------------------------------------------------------
template <int R>
__global__ void __launch_bounds__(NT) conv_fwd_kernel(const DevLayout L, const Item *__restrict__ items,
                                                      const float *__restrict__ vals,
                                                      const float *__restrict__ tree,
                                                      const float *__restrict__ stencils, int bc,
                                                      float *__restrict__ out) {
    using G = Geo<R>;
    __shared__ float patch[G::NROW * G::PYS];
    __shared__ float w[G::K3];
    __shared__ int seg_lo[G::NSEG], seg_hi[G::NSEG], row_valid[G::NROW];
    __shared__ int tgt_lo[TZ * TX], tgt_pre[TZ * TX + 1];
    const Item it = items[blockIdx.x];
    for (int i = threadIdx.x; i < G::K3; i += NT) w[i] = stencils[(it.l - L.l_min) * G::K3 + i];
    stage_forward_patch<R>(L, it, vals, tree, bc, patch, seg_lo, seg_hi, row_valid, tgt_lo, tgt_pre);

    const int yw = it.yb * BY - R;
    const int total = tgt_pre[TZ * TX];
    for (int t = threadIdx.x; t < total; t += NT) {
        int r = 0;
        while (tgt_pre[r + 1] <= t) ++r;
        const int i = tgt_lo[r] + (t - tgt_pre[r]);
        const int pos = int(L.y[i]) - yw - R;  // patch column of tap dy = -R
        const int ia = r / TX, ib = r % TX;
        float acc = 0.f;
#pragma unroll
        for (int dz = 0; dz < G::K; ++dz)
#pragma unroll
            for (int dx = 0; dx < G::K; ++dx) {
                const float *prow = patch + ((ia + dz) * G::PX + (ib + dx)) * G::PYS + pos;
#pragma unroll
                for (int dy = 0; dy < G::K; ++dy) acc = fmaf(w[(dz * G::K + dx) * G::K + dy], prow[dy], acc);
            }
        out[i] = acc;
    }
}

// ------------------------------------------------------------------------------------------------
// APR tree restriction for one level l (Sec. 3.4): block per tree brick (l, z, x, yb). The children
// of the brick's nodes live in the 2x2 child rows of level l+1, y-blocks 2yb and 2yb+1; each child
// value goes to a slot (a, b, y&1) of its parent, then every node averages its in-grid slots in a
// fixed order.
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) tree_restrict_kernel(const DevLayout L, const Item *__restrict__ items,
                                                           const float *__restrict__ vals,
                                                           float *__restrict__ tree) {
    __shared__ float slot[8][BY];
    __shared__ int seg_lo[8], seg_hi[8];
    const Item it = items[blockIdx.x];
    const int l = it.l, tid = threadIdx.x;
    const LevelGeo g = L.geo[l], gc = L.geo[l + 1];
    const int y0 = it.yb * BY;
    if (tid < 8) {
        const int kind = tid >> 2, a = (tid >> 1) & 1, b = tid & 1;
        const int cz = 2 * it.a + a, cx = 2 * it.b + b;
        uint32_t lo = 0, hi = 0;
        if (cz < gc.dz && cx < gc.dx) {
            const int crr = cz * gc.dx + cx;
            const int j0 = 2 * it.yb, j1 = min(2 * it.yb + 2, gc.nb);
            if (kind == 0) {
                lo = pblock(L, gc, crr, j0);
                hi = pblock(L, gc, crr, j1);
            } else if (l + 1 < L.l_max) {
                lo = tblock(L, gc, crr, j0);
                hi = tblock(L, gc, crr, j1);
            }
        }
        seg_lo[tid] = int(lo);
        seg_hi[tid] = int(hi);
    }
    __syncthreads();
    {
        const int s = tid >> 5, lane = tid & 31;  // 8 warps, one per child segment
        const int kind = s >> 2, ab = s & 3;
        const uint16_t *ys = kind == 0 ? L.y : L.ty;
        const float *src = kind == 0 ? vals : tree;
        for (int i = seg_lo[s] + lane; i < seg_hi[s]; i += 32) {
            const int yv = ys[i];
            slot[ab * 2 + (yv & 1)][(yv >> 1) - y0] = src[i];
        }
    }
    __syncthreads();
    const int rr = it.a * g.dx + it.b;
    const int tlo = int(tblock(L, g, rr, it.yb)), thi = int(tblock(L, g, rr, it.yb + 1));
    for (int t = tlo + tid; t < thi; t += NT) {
        const int yv = L.ty[t];
        float s = 0.f;
        int n = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int a = c >> 2, b = (c >> 1) & 1, e = c & 1;
            if (2 * it.a + a < gc.dz && 2 * it.b + b < gc.dx && 2 * yv + e < gc.dy) {
                s += slot[(a * 2 + b) * 2 + e][yv - y0];
                ++n;
            }
        }
        tree[t] = s / float(n);
    }
}

// ------------------------------------------------------------------------------------------------
// Backward, data part: for every cell c of the tile interior that a target can reach,
//   H(c) = sum over preimages c' of c under the boundary reflection of sum_e w[e] g(c' - e),
// g being dL/dout at the level-l particles (zero elsewhere). H is then routed to the source that
// supplied cell c in the forward patch: the level-l particle (atomic add: it receives exactly one
// more term, from the next finer level), the level-l tree node (store), or the level-(l-1) particle
// containing c (sum over its cells in this tile, one atomic add).
// ------------------------------------------------------------------------------------------------
template <int R>
__global__ void __launch_bounds__(NT) conv_bwd_data_kernel(const DevLayout L, const Item *__restrict__ items,
                                                           const float *__restrict__ stencils, int bc,
                                                           const float *__restrict__ gout,
                                                           float *__restrict__ gp, float *__restrict__ gt) {
    using G = Geo<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *gpatch = reinterpret_cast<float *>(smem_raw);                   // [NGROW][GYS]
    float *H = gpatch + G::NGROW * G::GYS;                                 // [TZ*TX][BY]
    unsigned long long *tmask = reinterpret_cast<unsigned long long *>(H + TZ * TX * BY);  // [NGROW][2]
    unsigned long long *need = tmask + 2 * G::NGROW;                       // [TZ*TX]
    __shared__ float w[G::K3];
    __shared__ int seg_lo[3 * TZ * TX], seg_hi[3 * TZ * TX];
    __shared__ int gseg_lo[G::NGROW], gseg_hi[G::NGROW];

    const Item it = items[blockIdx.x];
    const int l = it.l, tid = threadIdx.x;
    const LevelGeo g = L.geo[l];
    const int y0 = it.yb * BY;
    const int gw0 = y0 - 2 * R;  // level y of gradient-patch column 0
    const int z0 = it.a * TZ, x0 = it.b * TX;

    for (int i = tid; i < G::K3; i += NT) w[i] = stencils[(l - L.l_min) * G::K3 + i];
    for (int i = tid; i < G::NGROW * G::GYS; i += NT) gpatch[i] = 0.f;
    for (int i = tid; i < 2 * G::NGROW; i += NT) tmask[i] = 0ull;
    for (int i = tid; i < G::NGROW; i += NT) {
        const int z = z0 - 2 * R + i / G::GX, x = x0 - 2 * R + i % G::GX;
        uint32_t lo = 0, hi = 0;
        if (z >= 0 && z < g.dz && x >= 0 && x < g.dx) {  // gradient is zero outside the grid
            const int rr = z * g.dx + x;
            const int ylo = max(gw0, 0), yhi = min(gw0 + G::GY, g.dy);
            if (yhi > ylo) {
                lo = pblock(L, g, rr, ylo / BY);
                hi = pblock(L, g, rr, (yhi - 1) / BY + 1);
            }
        }
        gseg_lo[i] = int(lo);
        gseg_hi[i] = int(hi);
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    for (int s = warp; s < G::NGROW; s += NT / 32) {
        for (int i = gseg_lo[s] + lane; i < gseg_hi[s]; i += 32) {
            const int pos = int(L.y[i]) - gw0;
            if (pos >= 0 && pos < G::GY) {
                gpatch[s * G::GYS + pos] = gout[i];
                atomicOr(&tmask[2 * s + (pos >> 6)], 1ull << (pos & 63));
            }
        }
    }
    __syncthreads();
    // cells of the interior that need H: within R (Chebyshev) of a target, or (reflect) close
    // enough to the grid boundary to receive a mirrored contribution
    if (tid < TZ * TX) {
        const int ia = tid / TX, ib = tid % TX;
        unsigned long long m = 0ull;
        for (int dz = -R; dz <= R; ++dz)
            for (int dx = -R; dx <= R; ++dx) {
                const int s = (ia + 2 * R + dz) * G::GX + (ib + 2 * R + dx);
                const unsigned long long m0 = tmask[2 * s], m1 = tmask[2 * s + 1];
                // window bits [2R, 2R + BY) of the 128-bit row mask, dilated by +-R
                for (int d = -R; d <= R; ++d) {
                    const int sh = 2 * R + d;  // bit of window cell 0 shifted by d
                    m |= (m0 >> sh) | (sh > 0 ? (m1 << (64 - sh)) : 0ull);
                }
            }
        const int z = z0 + ia, x = x0 + ib;
        if (z >= g.dz || x >= g.dx) m = 0ull;
        else if (bc == APR_BC_REFLECT) {
            // cells within R of the grid boundary have mirrored preimages; take them all
            if (z < R || z >= g.dz - R || x < R || x >= g.dx - R) {
                m = ~0ull;
            } else {
                for (int j = 0; j < BY; ++j) {
                    const int yy = y0 + j;
                    if (yy < R || yy >= g.dy - R) m |= 1ull << j;
                }
            }
        }
        // cells outside the grid in y are not interior cells
        const int nvalid = min(BY, g.dy - y0);
        if (nvalid < BY) m &= (nvalid <= 0) ? 0ull : ((1ull << nvalid) - 1ull);
        need[tid] = m;
    }
    __syncthreads();
    // H at needed interior cells
    for (int c = tid; c < TZ * TX * BY; c += NT) {
        const int r = c / BY, j = c % BY;
        float h = 0.f;
        if ((need[r] >> j) & 1ull) {
            const int ia = r / TX, ib = r % TX;
            const int z = z0 + ia, x = x0 + ib, yy = y0 + j;
            const bool mirror = bc == APR_BC_REFLECT &&
                                (z < R || z >= g.dz - R || x < R || x >= g.dx - R || yy < R || yy >= g.dy - R);
            if (!mirror) {
#pragma unroll
                for (int dz = 0; dz < G::K; ++dz)
#pragma unroll
                    for (int dx = 0; dx < G::K; ++dx) {
                        // cell (c - e): gradient row (ia + 2R - (dz - R)), column (j + 2R - (dy - R))
                        const float *grow = gpatch + ((ia + 3 * R - dz) * G::GX + (ib + 3 * R - dx)) * G::GYS + j + 3 * R;
#pragma unroll
                        for (int dy = 0; dy < G::K; ++dy) h = fmaf(w[(dz * G::K + dx) * G::K + dy], grow[-dy], h);
                    }
            } else {
                // preimages per axis: c itself and every out-of-grid position in [-R, d+R) that
                // reflects onto it
                int pz[2 * R + 1], px[2 * R + 1], py[2 * R + 1];
                const int nz = preimages<R>(z, g.dz, pz), nx = preimages<R>(x, g.dx, px),
                          ny = preimages<R>(yy, g.dy, py);
#pragma unroll 1
                for (int iz = 0; iz < nz; ++iz)
#pragma unroll 1
                    for (int ix = 0; ix < nx; ++ix)
#pragma unroll 1
                        for (int iy = 0; iy < ny; ++iy)
#pragma unroll 1
                            for (int dz = 0; dz < G::K; ++dz)
#pragma unroll 1
                                for (int dx = 0; dx < G::K; ++dx)
#pragma unroll 1
                                    for (int dy = 0; dy < G::K; ++dy) {
                                        const int sz = pz[iz] - (dz - R) - (z0 - 2 * R);
                                        const int sx = px[ix] - (dx - R) - (x0 - 2 * R);
                                        const int sy = py[iy] - (dy - R) - gw0;
                                        if (sz < 0 || sz >= G::GZ || sx < 0 || sx >= G::GX || sy < 0 || sy >= G::GY) continue;
                                        h = fmaf(w[(dz * G::K + dx) * G::K + dy], gpatch[(sz * G::GX + sx) * G::GYS + sy], h);
                                    }
            }
        }
        H[c] = h;
    }
    // segments of the sources of interior cells
    if (tid < 3 * TZ * TX) {
        const int kind = tid / (TZ * TX), r = tid % (TZ * TX);
        uint32_t lo = 0, hi = 0;
        if (kind < 2) {
            const int z = z0 + r / TX, x = x0 + r % TX;
            if (z < g.dz && x < g.dx) {
                const int rr = z * g.dx + x;
                if (kind == 0) {
                    lo = pblock(L, g, rr, it.yb);
                    hi = pblock(L, g, rr, it.yb + 1);
                } else if (l < L.l_max) {
                    lo = tblock(L, g, rr, it.yb);
                    hi = tblock(L, g, rr, it.yb + 1);
                }
            }
        } else if (l > L.l_min && r < (TZ / 2) * (TX / 2)) {
            const LevelGeo gq = L.geo[l - 1];
            const int pz = z0 / 2 + r / (TX / 2), px = x0 / 2 + r % (TX / 2);
            if (pz < gq.dz && px < gq.dx) {
                const int prr = pz * gq.dx + px;
                const int pj = (y0 / 2) / BY;
                lo = pblock(L, gq, prr, pj);
                hi = pblock(L, gq, prr, pj + 1);
            }
        }
        seg_lo[tid] = int(lo);
        seg_hi[tid] = int(hi);
    }
    __syncthreads();
    for (int s = warp; s < 3 * TZ * TX; s += NT / 32) {
        const int kind = s / (TZ * TX), r = s % (TZ * TX);
        for (int i = seg_lo[s] + lane; i < seg_hi[s]; i += 32) {
            if (kind == 0) {
                atomicAdd(&gp[i], H[r * BY + (int(L.y[i]) - y0)]);
            } else if (kind == 1) {
                gt[i] = H[r * BY + (int(L.ty[i]) - y0)];
            } else {
                const int py = int(L.y[i]);
                const int j0 = 2 * py - y0;  // first level-l cell column of the coarser particle
                if (j0 < 0 || j0 >= BY) continue;
                const int pa = r / (TX / 2), pb = r % (TX / 2);
                float s2 = 0.f;
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b)
                        for (int e = 0; e < 2; ++e) {
                            const int ia = 2 * pa + a, ib = 2 * pb + b;
                            if (z0 + ia < g.dz && x0 + ib < g.dx && y0 + j0 + e < g.dy)
                                s2 += H[(ia * TX + ib) * BY + j0 + e];
                        }
                atomicAdd(&gp[i], s2);
            }
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Backward, stencil part: per work item, partial[e][item] = sum over the item's targets p of
// g_p * u_l(p + e) (fixed order); the per-level sums follow in stencil_grad_reduce_kernel.
// ------------------------------------------------------------------------------------------------
template <int R>
__global__ void __launch_bounds__(NT) conv_bwd_stencil_kernel(const DevLayout L, const Item *__restrict__ items,
                                                              int n_items, const float *__restrict__ vals,
                                                              const float *__restrict__ tree, int bc,
                                                              const float *__restrict__ gout,
                                                              float *__restrict__ partial) {
    using G = Geo<R>;
    __shared__ float patch[G::NROW * G::PYS];
    __shared__ int seg_lo[G::NSEG], seg_hi[G::NSEG], row_valid[G::NROW];
    __shared__ int tgt_lo[TZ * TX], tgt_pre[TZ * TX + 1];
    __shared__ float half_sum[G::K3];
    const Item it = items[blockIdx.x];
    stage_forward_patch<R>(L, it, vals, tree, bc, patch, seg_lo, seg_hi, row_valid, tgt_lo, tgt_pre);
    const int yw = it.yb * BY - R;
    const int total = tgt_pre[TZ * TX];
    // two threads per stencil entry: targets of even / odd rank
    const int e = threadIdx.x % 128, half = threadIdx.x / 128;
    float acc = 0.f;
    if (e < G::K3) {
        const int dz = e / (G::K * G::K), dx = (e / G::K) % G::K, dy = e % G::K;
        int r = 0;
        for (int t = half; t < total; t += 2) {
            while (tgt_pre[r + 1] <= t) ++r;
            const int i = tgt_lo[r] + (t - tgt_pre[r]);
            const int pos = int(L.y[i]) - yw - R;
            const int ia = r / TX, ib = r % TX;
            acc = fmaf(gout[i], patch[((ia + dz) * G::PX + (ib + dx)) * G::PYS + pos + dy], acc);
        }
    }
    if (half == 1 && e < G::K3) half_sum[e] = acc;
    __syncthreads();
    if (half == 0 && e < G::K3) partial[size_t(e) * n_items + blockIdx.x] = acc + half_sum[e];
}

// grad_w[l][e] = sum over the level's items of partial[e][item], fixed-order block reduction.
__global__ void __launch_bounds__(NT) stencil_grad_reduce_kernel(const float *__restrict__ partial, int n_items,
                                                                 const int64_t *__restrict__ level_begin,
                                                                 int l_min, int K3, float *__restrict__ gw) {
    __shared__ float red[NT];
    const int l = l_min + blockIdx.y, e = blockIdx.x;
    const int64_t b = level_begin[l], en = level_begin[l + 1];
    float s = 0.f;
    for (int64_t i = b + threadIdx.x; i < en; i += NT) s += partial[size_t(e) * n_items + i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = NT / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) gw[size_t(blockIdx.y) * K3 + e] = red[0];
}

// ------------------------------------------------------------------------------------------------
// Backward through the tree averages, one level l (coarse to fine): each child (particle or tree
// node of level l+1) of a tree node t receives gt[t] / n_children(t).
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) tree_pushdown_kernel(const DevLayout L, const Item *__restrict__ items,
                                                           float *__restrict__ gp, float *__restrict__ gt) {
    __shared__ float share[BY];
    __shared__ int seg_lo[8], seg_hi[8];
    const Item it = items[blockIdx.x];
    const int l = it.l, tid = threadIdx.x;
    const LevelGeo g = L.geo[l], gc = L.geo[l + 1];
    const int y0 = it.yb * BY;
    const int rr = it.a * g.dx + it.b;
    const int tlo = int(tblock(L, g, rr, it.yb)), thi = int(tblock(L, g, rr, it.yb + 1));
    for (int t = tlo + tid; t < thi; t += NT) {
        const int yv = L.ty[t];
        const int n = (2 * it.a + 1 < gc.dz ? 2 : 1) * (2 * it.b + 1 < gc.dx ? 2 : 1) * (2 * yv + 1 < gc.dy ? 2 : 1);
        share[yv - y0] = gt[t] / float(n);
    }
    if (tid < 8) {
        const int kind = tid >> 2, a = (tid >> 1) & 1, b = tid & 1;
        const int cz = 2 * it.a + a, cx = 2 * it.b + b;
        uint32_t lo = 0, hi = 0;
        if (cz < gc.dz && cx < gc.dx) {
            const int crr = cz * gc.dx + cx;
            const int j0 = 2 * it.yb, j1 = min(2 * it.yb + 2, gc.nb);
            if (kind == 0) {
                lo = pblock(L, gc, crr, j0);
                hi = pblock(L, gc, crr, j1);
            } else if (l + 1 < L.l_max) {
                lo = tblock(L, gc, crr, j0);
                hi = tblock(L, gc, crr, j1);
            }
        }
        seg_lo[tid] = int(lo);
        seg_hi[tid] = int(hi);
    }
    __syncthreads();
    const int s = tid >> 5, lane = tid & 31;
    const int kind = s >> 2;
    const uint16_t *ys = kind == 0 ? L.y : L.ty;
    float *dst = kind == 0 ? gp : gt;
    for (int i = seg_lo[s] + lane; i < seg_hi[s]; i += 32) dst[i] += share[(int(ys[i]) >> 1) - y0];
}

template <int R>
size_t bwd_data_smem() {
    using G = Geo<R>;
    return sizeof(float) * (size_t(G::NGROW) * G::GYS + TZ * TX * BY) + sizeof(unsigned long long) * (2 * G::NGROW + TZ * TX);
}

template <int R>
cudaError_t launch_conv_fwd_t(const DevLayout &L, const Item *items, int n, const float *vals, const float *tree,
                              const float *st, int bc, float *out, cudaStream_t s) {
    if (n > 0) conv_fwd_kernel<R><<<n, NT, 0, s>>>(L, items, vals, tree, st, bc, out);
    return cudaGetLastError();
}

template <int R>
cudaError_t launch_bwd_data_t(const DevLayout &L, const Item *items, int n, const float *st, int bc,
                              const float *gout, float *gp, float *gt, cudaStream_t s) {
    const size_t sm = bwd_data_smem<R>();
    cudaError_t e = cudaFuncSetAttribute(conv_bwd_data_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    if (e != cudaSuccess) return e;
    if (n > 0) conv_bwd_data_kernel<R><<<n, NT, sm, s>>>(L, items, st, bc, gout, gp, gt);
    return cudaGetLastError();
}

template <int R>
cudaError_t launch_bwd_stencil_t(const DevLayout &L, const Item *items, int n, const float *vals,
                                 const float *tree, int bc, const float *gout, float *partial, cudaStream_t s) {
    if (n > 0) conv_bwd_stencil_kernel<R><<<n, NT, 0, s>>>(L, items, n, vals, tree, bc, gout, partial);
    return cudaGetLastError();
}

}  // namespace

// ---- launch entry points used by the C ABI (apr_api.cu)
cudaError_t launch_conv_fwd(int k, const DevLayout &L, const Item *items, int n, const float *vals,
                            const float *tree, const float *st, int bc, float *out, cudaStream_t s) {
    return k == 3 ? launch_conv_fwd_t<1>(L, items, n, vals, tree, st, bc, out, s)
                  : launch_conv_fwd_t<2>(L, items, n, vals, tree, st, bc, out, s);
}

cudaError_t launch_tree_restrict(const DevLayout &L, const Item *items, int n, const float *vals, float *tree,
                                 cudaStream_t s) {
    if (n > 0) tree_restrict_kernel<<<n, NT, 0, s>>>(L, items, vals, tree);
    return cudaGetLastError();
}

cudaError_t launch_bwd_data(int k, const DevLayout &L, const Item *items, int n, const float *st, int bc,
                            const float *gout, float *gp, float *gt, cudaStream_t s) {
    return k == 3 ? launch_bwd_data_t<1>(L, items, n, st, bc, gout, gp, gt, s)
                  : launch_bwd_data_t<2>(L, items, n, st, bc, gout, gp, gt, s);
}

cudaError_t launch_bwd_stencil(int k, const DevLayout &L, const Item *items, int n, const float *vals,
                               const float *tree, int bc, const float *gout, float *partial, cudaStream_t s) {
    return k == 3 ? launch_bwd_stencil_t<1>(L, items, n, vals, tree, bc, gout, partial, s)
                  : launch_bwd_stencil_t<2>(L, items, n, vals, tree, bc, gout, partial, s);
}

cudaError_t launch_stencil_reduce(const float *partial, int n_items, const int64_t *level_begin, int l_min,
                                  int n_levels, int K3, float *gw, cudaStream_t s) {
    if (n_levels > 0) stencil_grad_reduce_kernel<<<dim3(K3, n_levels), NT, 0, s>>>(partial, n_items, level_begin, l_min, K3, gw);
    return cudaGetLastError();
}

cudaError_t launch_tree_pushdown(const DevLayout &L, const Item *items, int n, float *gp, float *gt, cudaStream_t s) {
    if (n > 0) tree_pushdown_kernel<<<n, NT, 0, s>>>(L, items, gp, gt);
    return cudaGetLastError();
}

}  // namespace aprk
