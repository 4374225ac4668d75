// CUDA kernels (sm_103a) for APR-native convolution, its tree restriction and their adjoints.
//
// Data layout in device memory (built by apr_index.cpp, Sec. 3.1 Alg. 1 extended):
//   row_ptr[R+1] (uint32), y[N_p] (uint16), off[rows * nb] (uint16): for every row (l, z, x) and
//   y-block j of BY cells, the offset of the row's first particle with y >= j*BY. The tree has the
//   same three arrays. A work item names a tile of TZ x TX rows and one y-block of one level; its
//   tile plan (apr_plan.cu) lists the non-empty source segments of its patch.
//
// Convolution-type kernels stage an isotropic level-l patch (Sec. 3.5) of the tile plus an R-cell
// halo in shared memory: same-level particles directly, the level-(l-1) particle of each remaining
// cell piecewise-constant, and finer content through the level-l tree node (Sec. 4.1, Fig.
// treeconv). The source elements of all patch rows are loaded in one flattened, unrolled loop
// (consecutive lanes on consecutive particles, several loads in flight per thread), then the
// stencil is applied to 8-cell windows along y that hold target particles, two threads per window
// (one lane in each warp of a pair, each over half of the stencil rows), with 16-byte shared-memory
// loads. A 5^3 stack whose level has zero taps outside the central 3^3 is applied with radius 1.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "apr_device.cuh"
#include "apr_internal.h"
#include "apr_tile.cuh"

namespace aprk {

namespace {

using namespace dev;

// True on every thread if all taps of level l_idx of a 5^3 stack outside its central 3^3 are zero.
// Such a level is convolved with radius 1: a restricted 5^3 stencil (Eq. restrict_stenc) has support
// 2 ceil(2 / s) + 1 = 3 cells per axis at every level with cell edge s >= 2, i.e. below l_max. The
// result is the same linear map (the skipped products are 0 * u); only its FP32 summation order
// differs. Called by all threads of the block (a block barrier).
__device__ __forceinline__ bool outer_taps_zero5(const float *__restrict__ stencils, int l_idx) {
    const int t = threadIdx.x;
    bool nz = false;
    if (t < 125) {
        const int a = t / 25, b = (t / 5) % 5, c = t % 5;
        const bool outer = a == 0 || a == 4 || b == 0 || b == 4 || c == 0 || c == 4;
        nz = outer && stencils[l_idx * 125 + t] != 0.f;
    }
    return __syncthreads_or(nz) == 0;
}

// Bit i set: level l_idx0 + i of a 5^3 stack has a nonzero tap outside the central 3^3 (block-wide;
// uses the shared-memory word `word`, free again on return).
__device__ __forceinline__ unsigned levels_with_outer_taps(const float *__restrict__ stencils, int l_idx0, int n,
                                                           unsigned *word) {
    const int t = threadIdx.x;
    unsigned m = 0u;
    if (t < 125) {
        const int a = t / 25, b = (t / 5) % 5, c = t % 5;
        if (a == 0 || a == 4 || b == 0 || b == 4 || c == 0 || c == 4)
            for (int i = 0; i < n; ++i)
                if (stencils[(l_idx0 + i) * 125 + t] != 0.f) m |= 1u << i;
    }
    if (t == 0) *word = 0u;
    __syncthreads();
    if (m) atomicOr(word, m);
    __syncthreads();
    m = *word;
    __syncthreads();
    return m;
}

// The levels of lr selected by `sel` (bit i: level lr.l0 + i): their work-item count, and their j-th
// work item in level order.
__device__ __forceinline__ int selected_count(const LevelRanges &lr, unsigned sel) {
    int c = 0;
    for (int i = 0; i < lr.n; ++i)
        if ((sel >> i) & 1u) c += lr.begin[i + 1] - lr.begin[i];
    return c;
}
__device__ __forceinline__ int selected_item(const LevelRanges &lr, unsigned sel, int j) {
    for (int i = 0; i < lr.n; ++i) {
        if (!((sel >> i) & 1u)) continue;
        const int c = lr.begin[i + 1] - lr.begin[i];
        if (j < c) return lr.begin[i] + j;
        j -= c;
    }
    return -1;
}

// c itself (self) and, with reflection, the positions v in [-R, d + R) outside [0, d) that reflect
// onto it, each as (position - base) in 8 bits of one register word (base <= every position < base + 256);
// returns the count (at most 2R + 1). Registers only, no local array.
template <int R>
__device__ __forceinline__ int with_mirrors(int c, int d, int base, bool self, bool reflect, uint64_t &w) {
    uint64_t v = 0;
    int n = 0;
    if (self) v |= uint64_t(c - base) << (8 * n++);
    if (reflect) {
        if (d >= 2 * R) {
            if (c < R) v |= uint64_t(-c - 1 - base) << (8 * n++);
            if (c >= d - R) v |= uint64_t(2 * d - 1 - c - base) << (8 * n++);
        } else {
#pragma unroll
            for (int t = -R; t < 0; ++t)
                if (reflect_idx(t, d) == c) v |= uint64_t(t - base) << (8 * n++);
#pragma unroll
            for (int t = 0; t < R; ++t)
                if (reflect_idx(d + t, d) == c) v |= uint64_t(d + t - base) << (8 * n++);
        }
    }
    w = v;
    return n;
}
__device__ __forceinline__ int at8(uint64_t w, int i) { return int((w >> (8 * i)) & 255u); }

// Per-particle epilogue of the convolution: the plain output, or the element-wise division and
// multiplication of a Richardson-Lucy update (Sec. 6.2) fused into the write. aux may alias the
// output (each particle's entry is read, then written, by the same thread).
struct Epilogue {
    int mode;                  // EPI_PLAIN, EPI_DIVIDE (aux[p] / acc, 0 if acc <= 0), EPI_MULTIPLY (aux[p] * acc)
    bool flip;                 // taps in reversed order in every dimension (the flipped stencil)
    const float *aux;
    __device__ __forceinline__ float apply(int p, float acc) const {
        if (mode == EPI_DIVIDE) return acc > 0.f ? __fdiv_rn(aux[p], acc) : 0.f;
        if (mode == EPI_MULTIPLY) return aux[p] * acc;
        return acc;
    }
};

// ------------------------------------------------------------------------------------------------
// Staged forward patch (convolution, gradient magnitude, stencil gradient).
//
// The sources of every patch row (Sec. 3.5: level-l particles, level-l tree nodes, level-(l-1)
// particles) are index ranges [lo, lo + n) of the APR's arrays (fwd_segment). They are read as
// 8-element packets aligned to 8 elements: one 16-byte load of y and two of values per packet, with
// the elements outside the range masked (the y arrays are padded to a multiple of 8 elements; the
// last packet of a value array is read element by element up to the array's end). A packet ->
// segment table per chunk of packets replaces any per-element bookkeeping; the occupancy of the
// target rows is OR-ed per packet.
// ------------------------------------------------------------------------------------------------
constexpr int PCAP = 1024;  // packets per staging chunk

// Floats per stencil row in the paired-tap layout: taps (w0, w0, w1, w1, ...), padded to 16 bytes.
template <int R>
__host__ __device__ constexpr int w2_stride() {
    return ((2 * R + 1) + 1) / 2 * 4;
}

// Lanes per window: radius-1 windows (9 stencil rows) take one lane each, radius-2 windows (25 rows)
// two lanes over alternate rows.
template <int R>
__host__ __device__ constexpr int lanes_per_window() {
    return R == 1 ? 1 : 2;
}

// Offsets of the stencil rows (dz, dx) = pair in a staged patch: roff[pair] = (dz PX + dx) PYS.
template <int R>
__device__ __forceinline__ void fill_row_offsets(int *roff) {
    using G = Geo<R>;
    for (int i = threadIdx.x; i < G::NPAIR; i += NT) roff[i] = ((i / G::K) * G::PX + i % G::K) * G::PYS;
}

template <int R, int NS>
struct FwdSmem {
    using G = Geo<R>;
    float patch[G::NROW * G::PYS];             // first member: 16-byte aligned
    __align__(16) float w2[NS][G::NPAIR * w2_stride<R>()];  // paired taps of NS stencil stacks
    struct Staging {
        int seg_lo[G::NSEG];                    // first element of segment s
        unsigned seg_nm[G::NSEG];               // element count | segment meta << 8 (with_trow)
        int pre[G::NSEG + 1];                   // packet prefix over the segments
        unsigned short pseg[PCAP];              // segment of every packet of the current chunk
    };
    static constexpr int GWIN = int(sizeof(Staging) / 32);  // windows of dL/dout that fit in its place
    union {
        Staging st;                             // during staging
        float4 gwin[GWIN * 2];                  // after staging (stencil gradient): 8 dL/dout per window
    };
    int warp_tot[NWARP + 1];
    unsigned long long rmask[NIR];              // targets of interior row r: bit j = cell y0 + j
    int rfirst[NIR];                            // first target (particle index) of interior row r
    unsigned short act[NIW];                    // windows holding targets, in window order
    int roff[G::NPAIR];                         // stencil-row offsets in the patch (fill_row_offsets)
    int nact;
};

// Targets of window w (bit j = cell j of the window) and the particle index of its first target.
template <typename S>
__device__ __forceinline__ unsigned win_mask(const S &sm, int w) {
    return unsigned(sm.rmask[w / NWIN] >> ((w % NWIN) * WIN)) & 0xffu;
}
template <typename S>
__device__ __forceinline__ int win_first(const S &sm, int w) {
    const unsigned long long m = sm.rmask[w / NWIN];
    return sm.rfirst[w / NWIN] + __popcll(m & ((1ull << ((w % NWIN) * WIN)) - 1ull));
}

// Writes the valid elements of one packet (elements i0 .. i0+7; valid: lo <= i < lo + n) into the
// patch. Kinds 0, 1: one cell each (and, for level-l particles of interior rows, a target bit);
// kind 2: the two level-l cells of a level-(l-1) particle in its patch row; kind 3: its 2 x 2 x 2
// cells in the (up to) 2 x 2 patch rows of a once-staged level-(l-1) row.
template <int R, int NS>
__device__ __forceinline__ void place_packet(FwdSmem<R, NS> &S, int seg, int i0, const uint4 &yq, const float4 &va,
                                             const float4 &vb, int dy, int yw, int y0) {
    using G = Geo<R>;
    const int lo = S.st.seg_lo[seg];
    const unsigned nm = S.st.seg_nm[seg];
    const int n = int(nm & 255u), meta = int(nm >> 8);
    const int kind = meta_kind(meta);
    const int yv[8] = {int(yq.x & 0xffffu), int(yq.x >> 16), int(yq.y & 0xffffu), int(yq.y >> 16),
                       int(yq.z & 0xffffu), int(yq.z >> 16), int(yq.w & 0xffffu), int(yq.w >> 16)};
    const float vv[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
    if (kind < 2) {
        // the plan lists only elements whose cell lies in the patch window (0 <= y - yw < PY)
        float *prow = S.patch + (meta & 255) * G::PYS;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (unsigned(i0 + j - lo) < unsigned(n)) prow[yv[j] - yw] = vv[j];
        const int trow = meta_trow(meta);
        if (trow >= 0) {
            unsigned b0 = 0u, b1 = 0u;  // target bits of cells y0 .. y0+31 and y0+32 .. y0+63
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int yr = yv[j] - y0;
                if (unsigned(i0 + j - lo) < unsigned(n) && unsigned(yr) < unsigned(BY)) {
                    if (yr < 32) b0 |= 1u << yr;
                    else b1 |= 1u << (yr - 32);
                }
            }
            unsigned *rm = reinterpret_cast<unsigned *>(&S.rmask[trow]);
            if (b0) atomicOr(rm, b0);
            if (b1) atomicOr(rm + 1, b1);
        }
    } else if (kind == 2) {
        float *prow = S.patch + (meta & 255) * G::PYS;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (unsigned(i0 + j - lo) >= unsigned(n)) continue;
            const int yy = 2 * yv[j], pos = yy - yw;
            if (unsigned(pos) < unsigned(G::PY) && yy < dy) prow[pos] = vv[j];
            if (unsigned(pos + 1) < unsigned(G::PY) && yy + 1 < dy) prow[pos + 1] = vv[j];
        }
    } else {
        const int rz0 = (meta & 15) - 1, rx0 = ((meta >> 4) & 15) - 1;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (unsigned(i0 + j - lo) >= unsigned(n)) continue;
            const int yy = 2 * yv[j], pos = yy - yw;
            const bool c0 = unsigned(pos) < unsigned(G::PY) && yy < dy;
            const bool c1 = unsigned(pos + 1) < unsigned(G::PY) && yy + 1 < dy;
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const int rz = rz0 + a, rx = rx0 + b;
                    if (rz < 0 || rz >= G::PZ || rx < 0 || rx >= G::PX) continue;
                    float *q = S.patch + (rz * G::PX + rx) * G::PYS;
                    if constexpr (R % 2 == 0) {
                        // yw = y0 - R is even, so pos is even: both cells are one aligned float2
                        if (c0 && c1) {
                            *reinterpret_cast<float2 *>(q + pos) = make_float2(vv[j], vv[j]);
                            continue;
                        }
                    }
                    if (c0) q[pos] = vv[j];
                    if (c1) q[pos + 1] = vv[j];
                }
        }
    }
}

// Stage the forward patch of item `it` (Sec. 3.5): patch rows z in [z0-R, z0+TZ+R), x likewise, y in
// [y0-R, y0+BY+R); rows outside the grid hold the reflected rows (or zeros), cells outside the grid
// in y the reflected cells (or zeros); cells no source covers (possible only in layouts not checked
// for 2:1 balance) hold 0. Also records the target rows (rmask, rfirst) and lists the windows that
// hold targets (act, nact). Ends with a block barrier.
// A tile's plan header (loaded at kernel start, with the work item) and this thread's first entry
// (entry threadIdx.x, when the plan has it). count: the entries listed (the entry after them holds
// the packet total).
struct PlanPre {
    PlanHdr hd;
    uint2 e0;
};
__device__ __forceinline__ PlanHdr plan_hdr(const FPlanView &P, int tile) { return P.hdr[tile]; }
__device__ __forceinline__ PlanPre plan_pre(const FPlanView &P, const PlanHdr &hd, int count) {
    return PlanPre{hd, int(threadIdx.x) <= count ? P.ent[hd.first + threadIdx.x] : make_uint2(0u, 0u)};
}
__device__ __forceinline__ int bplan_count(const PlanHdr &hd) { return (hd.count & 0xffff) + (hd.count >> 16); }

template <int R, int NS>
__device__ void stage_fwd(const DevLayout &L, const Item &it, const PlanPre &pp, const float *__restrict__ vals,
                          const float *__restrict__ tree, int bc, FwdSmem<R, NS> &S) {
    using G = Geo<R>;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const LevelGeo g = L.geo[it.l];
    const int z0 = it.a * TZ, x0 = it.b * TX, y0 = it.yb * BY, yw = y0 - R;
    const bool boundary = fwd_tile_at_boundary<R>(L, it);
    const bool reflect = bc == APR_BC_REFLECT;

    fill_row_offsets<R>(S.roff);
    for (int i = tid; i < G::NROW * G::PYS / 4; i += NT)
        reinterpret_cast<float4 *>(S.patch)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (tid < NIR) {
        const int z = z0 + tid / TX, x = x0 + tid % TX;
        S.rmask[tid] = 0ull;
        S.rfirst[tid] = (z < g.dz && x < g.dx) ? int(pblock(L, g, z * g.dx + x, it.yb)) : 0;
    }
    // the tile's non-empty segments and their packet prefixes (fwd_segment, listed once per APR in
    // the tile plan); with zero boundary the segments of rows outside the grid are skipped (their
    // cells stay 0)
    const FPlanView FP = L.fplan[R - 1];
    const PlanHdr hd = pp.hd;
    const int nseg = hd.count;
    for (int k = tid; k <= nseg; k += NT) {
        const uint2 raw = k == tid ? pp.e0 : FP.ent[hd.first + k];
        const FPlanEnt e{raw.x, raw.y};
        if (k < nseg) {
            const int meta = fplan_meta(e);
            const bool drop = !reflect && (meta & META_REFL);
            S.st.seg_lo[k] = fplan_lo(e);
            S.st.seg_nm[k] = unsigned(drop ? 0 : fplan_n(e)) | (unsigned(with_trow<R>(g, it, meta)) << 8);
        }
        S.st.pre[k] = fplan_pre(e);
    }
    block_sync();

    const int P = S.st.pre[nseg];
    for (int c0 = 0; c0 < P; c0 += PCAP) {
        const int c1 = min(P, c0 + PCAP);
        for (int s = tid; s < nseg; s += NT) {
            const int a = max(S.st.pre[s], c0), b = min(S.st.pre[s + 1], c1);
            for (int p = a; p < b; ++p) S.st.pseg[p - c0] = (unsigned short)s;
        }
        block_sync();
        // two packets per thread and step: the loads of both are issued before either is placed
        for (int p0 = c0 + tid; p0 < c1; p0 += 2 * NT) {
            uint4 yq[2];
            float4 va[2], vb[2];
            int sg[2], i0[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int p = p0 + u * NT;
                sg[u] = -1;
                i0[u] = 0;
                if (p < c1) {
                    const int s = S.st.pseg[p - c0];
                    const bool t = meta_kind(int(S.st.seg_nm[s] >> 8)) == 1;
                    const int g8 = (S.st.seg_lo[s] >> 3) + (p - S.st.pre[s]);
                    const uint4 *yt = reinterpret_cast<const uint4 *>(t ? L.ty : L.y);
                    const float *vs = t ? tree : vals;
                    yq[u] = __ldg(yt + g8);
                    if (8 * g8 + 8 <= (t ? L.nt : L.np)) {
                        va[u] = __ldg(reinterpret_cast<const float4 *>(vs) + 2 * g8);
                        vb[u] = __ldg(reinterpret_cast<const float4 *>(vs) + 2 * g8 + 1);
                    } else {
                        float e[8];
                        const int nv = (t ? L.nt : L.np) - 8 * g8;
#pragma unroll
                        for (int j = 0; j < 8; ++j) e[j] = j < nv ? vs[8 * g8 + j] : 0.f;
                        va[u] = make_float4(e[0], e[1], e[2], e[3]);
                        vb[u] = make_float4(e[4], e[5], e[6], e[7]);
                    }
                    sg[u] = s;
                    i0[u] = 8 * g8;
                }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u)
                if (sg[u] >= 0) place_packet<R, NS>(S, sg[u], i0[u], yq[u], va[u], vb[u], g.dy, yw, y0);
        }
        block_sync();
    }
    if (boundary && reflect) {
        // cells outside the grid in y (the first max(0, -yw), the last from dy - yw on): mirrored from
        // the in-grid cells of the same row
        const int nlo = max(0, -yw), hi0 = min(G::PY, g.dy - yw), per = nlo + (G::PY - hi0);
        if (per > 0) {
            for (int task = tid; task < G::NROW * per; task += NT) {
                const int pr = task / per, q = task - pr * per;
                const int pos = q < nlo ? q : hi0 + (q - nlo);
                float *prow = S.patch + pr * G::PYS;
                prow[pos] = prow[reflect_idx(yw + pos, g.dy) - yw];
            }
            block_sync();
        }
    }
    // windows holding targets, in window order (rows of warps 0 and 1)
    if (tid < NIR) {
        const unsigned long long m = S.rmask[tid];
        unsigned am = 0u;
#pragma unroll
        for (int w = 0; w < NWIN; ++w) am |= ((m >> (w * WIN)) & 0xffull) ? (1u << w) : 0u;
        const int c = __popc(am);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) S.warp_tot[warp] = incl;
        pair_sync(0);
        int k = (warp == 1 ? S.warp_tot[0] : 0) + incl - c;
#pragma unroll
        for (int w = 0; w < NWIN; ++w)
            if ((am >> w) & 1u) S.act[k++] = (unsigned short)(tid * NWIN + w);
        if (tid == NIR - 1) S.nact = k;
    }
    block_sync();
}

// Stencil taps of level l_idx in the paired layout w2[pair][2t], w2[pair][2t+1] = w[pair][t],
// optionally flipped. The stack holds (2 RS + 1)^3 taps per level; with R < RS the central
// (2 R + 1)^3 of them are loaded.
template <int R, int RS = R>
__device__ void load_taps2(const float *__restrict__ stencils, int l_idx, bool flip, float *w2) {
    using G = Geo<R>;
    constexpr int KS = 2 * RS + 1, KS3 = KS * KS * KS, D = RS - R, WS = w2_stride<R>();
    for (int i = threadIdx.x; i < G::NPAIR * WS; i += NT) {
        const int pair = i / WS, t = (i % WS) / 2;
        float v = 0.f;
        if (t < G::K) {
            const int e = ((pair / G::K + D) * KS + (pair % G::K + D)) * KS + (t + D);
            v = stencils[l_idx * KS3 + (flip ? KS3 - 1 - e : e)];
        }
        w2[i] = v;
    }
}

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// One stencil row of a window: (acc_{2i}, acc_{2i+1}) += even taps x the aligned value pairs
// (v_{2i+t}, v_{2i+t+1}) in E, (o_{2m-1}, o_{2m}) += odd taps x (v_{2m-1+t}, v_{2m+t}) in O (also
// aligned pairs); paired FP32 FMAs.
template <int R>
__device__ __forceinline__ void window_row2(const float *src_row, const float *wrow, float2 E[4], float2 O[5]) {
    const float4 *src = reinterpret_cast<const float4 *>(src_row);
    const float4 q0 = src[0], q1 = src[1], q2 = src[2];
    const float2 V[6] = {make_float2(q0.x, q0.y), make_float2(q0.z, q0.w), make_float2(q1.x, q1.y),
                         make_float2(q1.z, q1.w), make_float2(q2.x, q2.y), make_float2(q2.z, q2.w)};
    const float4 *wq = reinterpret_cast<const float4 *>(wrow);
    const float4 wa = wq[0], wb = wq[1];
    const float2 W0 = make_float2(wa.x, wa.y), W1 = make_float2(wa.z, wa.w), W2 = make_float2(wb.x, wb.y);
#pragma unroll
    for (int i = 0; i < 4; ++i) E[i] = ffma2(W0, V[i], E[i]);
#pragma unroll
    for (int i = 0; i < 4; ++i) E[i] = ffma2(W2, V[i + 1], E[i]);
#pragma unroll
    for (int m = 0; m < 5; ++m) O[m] = ffma2(W1, V[m], O[m]);
    if constexpr (R == 2) {
        const float4 wc = wq[2];
        const float2 W3 = make_float2(wb.z, wb.w), W4 = make_float2(wc.x, wc.y);
#pragma unroll
        for (int i = 0; i < 4; ++i) E[i] = ffma2(W4, V[i + 2], E[i]);
#pragma unroll
        for (int m = 0; m < 5; ++m) O[m] = ffma2(W3, V[m + 1], O[m]);
    }
}

// Window sums over the stencil rows pair = sub, sub + LPW, ...: acc[j] = sum_rows sum_t
// w[row][t] * P[row][col + j + t], j < WIN (window_row2; o_{-1} and o_8 are unused). Radius 1:
// the 9 rows unrolled; radius 2: a loop over the row-offset table (not unrolled: it keeps the
// instruction cache warm).
template <int R>
__device__ __forceinline__ void window_part2(const float *patch, const float *w2, const int *roff, int w, int sub,
                                             float acc[WIN]) {
    using G = Geo<R>;
    constexpr int WS = w2_stride<R>(), LPW = lanes_per_window<R>();
    const int r = w / NWIN;
    const float *base = patch + ((r / TX) * G::PX + (r % TX)) * G::PYS + (w % NWIN) * WIN;
    float2 E[4], O[5];
#pragma unroll
    for (int i = 0; i < 4; ++i) E[i] = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 5; ++i) O[i] = make_float2(0.f, 0.f);
    if constexpr (LPW == 1) {
#pragma unroll
        for (int pair = 0; pair < G::NPAIR; ++pair)
            window_row2<R>(base + ((pair / G::K) * G::PX + pair % G::K) * G::PYS, w2 + pair * WS, E, O);
    } else {
#pragma unroll 1
        for (int pair = sub; pair < G::NPAIR; pair += LPW) window_row2<R>(base + roff[pair], w2 + pair * WS, E, O);
    }
    acc[0] = E[0].x + O[0].y;
    acc[1] = E[0].y + O[1].x;
    acc[2] = E[1].x + O[1].y;
    acc[3] = E[1].y + O[2].x;
    acc[4] = E[2].x + O[2].y;
    acc[5] = E[2].y + O[3].x;
    acc[6] = E[3].x + O[3].y;
    acc[7] = E[3].y + O[4].x;
}

// Window sums of the active windows act[0..nact). One lane per window (radius 1), or two adjacent
// lanes over alternate stencil rows followed by a reduce-scatter between them (lane 0 of the pair
// keeps outputs 0..3, lane 1 outputs 4..7; the sum of the two halves is commutative, so the result
// is deterministic). emit(w, j0, v, n) receives outputs j0 .. j0+n-1 of window w.
template <int R, typename Emit>
__device__ __forceinline__ void fwd_windows(const float *patch, const float *w2, const int *roff,
                                            const unsigned short *act, int nact, Emit emit) {
    constexpr int LPW = lanes_per_window<R>();
    const int sub = threadIdx.x % LPW;
    for (int base = 0; base < nact; base += NT / LPW) {
        const int a = base + threadIdx.x / LPW;
        const bool valid = a < nact;
        const int w = valid ? act[a] : 0;
        float acc[WIN];
        if (valid) {
            window_part2<R>(patch, w2, roff, w, sub, acc);
        } else {
#pragma unroll
            for (int j = 0; j < WIN; ++j) acc[j] = 0.f;
        }
        if constexpr (LPW == 1) {
            if (valid) emit(w, 0, acc, WIN);
        } else {
            float own[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float send = sub ? acc[k] : acc[4 + k];
                const float keep = sub ? acc[4 + k] : acc[k];
                own[k] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
            }
            if (valid) emit(w, 4 * sub, own, 4);
        }
    }
}

// ------------------------------------------------------------------------------------------------
// APR convolution (Sec. 4.1; Sec. 5.2 with 8x8-row tiles and 64-cell y-blocks instead of the
// paper's 4x4 / 8x8 warp grid with a sliding buffer).
// ------------------------------------------------------------------------------------------------
// One forward tile with stencil radius R from a stack of radius RS >= R.
template <int R, int RS>
__device__ __forceinline__ void conv_fwd_tile(const DevLayout &L, const Item &it, const PlanPre &pp, const float *__restrict__ vals,
                                              const float *__restrict__ tree, const float *__restrict__ stencils,
                                              int bc, float *out, const Epilogue &epi, unsigned char *smem_raw) {
    FwdSmem<R, 1> &S = *reinterpret_cast<FwdSmem<R, 1> *>(smem_raw);
    load_taps2<R, RS>(stencils, it.l - L.l_min, epi.flip, S.w2[0]);
    stage_fwd<R, 1>(L, it, pp, vals, tree, bc, S);
    fwd_windows<R>(S.patch, S.w2[0], S.roff, S.act, S.nact, [&](int w, int j0, const float *v, int n) {
        const unsigned m = win_mask(S, w);
        int p = win_first(S, w) + __popc(m & ((1u << j0) - 1u));
#pragma unroll
        for (int k = 0; k < n; ++k)
            if ((m >> (j0 + k)) & 1u) {
                out[p] = epi.apply(p, v[k]);
                ++p;
            }
    });
}

template <int R>
__global__ void __launch_bounds__(NT, R == 1 ? 5 : 4) conv_fwd_kernel(const DevLayout L, const Item *__restrict__ items,
                                                         int tile0, const float *__restrict__ vals,
                                                         const float *__restrict__ tree,
                                                         const float *__restrict__ stencils, int bc,
                                                         float *out, const Epilogue epi) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tile = tile0 + int(blockIdx.x);   // work items [tile0, tile0 + gridDim.x)
    const Item it = items[tile];
    // the plan headers of both radii the tile may take, loaded with the item (the radius follows
    // from the level's stencil; the entries are read only for the radius taken)
    const PlanHdr h1 = plan_hdr(L.fplan[0], tile);
    if constexpr (R == 2) {
        const PlanHdr h2 = plan_hdr(L.fplan[1], tile);
        if (outer_taps_zero5(stencils, it.l - L.l_min)) {
            conv_fwd_tile<1, 2>(L, it, plan_pre(L.fplan[0], h1, h1.count), vals, tree, stencils, bc, out, epi, smem_raw);
            return;
        }
        conv_fwd_tile<2, 2>(L, it, plan_pre(L.fplan[1], h2, h2.count), vals, tree, stencils, bc, out, epi, smem_raw);
    } else {
        conv_fwd_tile<R, R>(L, it, plan_pre(L.fplan[0], h1, h1.count), vals, tree, stencils, bc, out, epi, smem_raw);
    }
}

// A 5^3 convolution over the whole work list, split by radius. The levels below l_max of a
// restricted stack have no taps outside the central 3^3 (Eq. restrict_stenc); their tiles run in a
// launch of their own with radius-1 shared memory and registers, five blocks per SM instead of the
// radius-2 launch's four, beside the launch over the l_max tiles.
// First part: items [0, gridDim.x) (the levels below l_max) as radius-1 tiles. A tile of a level with
// outer taps returns at once; conv_fwd_r2_pool_kernel takes it.
__global__ void __launch_bounds__(NT, 5) conv_fwd_r1_kernel(const DevLayout L, const Item *__restrict__ items,
                                                            const float *__restrict__ vals,
                                                            const float *__restrict__ tree,
                                                            const float *__restrict__ stencils, int bc, float *out,
                                                            const Epilogue epi) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_trigger();   // the persistent radius-2 launch after this one is independent of it
    const int tile = int(blockIdx.x);
    const Item it = items[tile];
    if (!outer_taps_zero5(stencils, it.l - L.l_min)) return;
    const PlanHdr h1 = plan_hdr(L.fplan[0], tile);
    conv_fwd_tile<1, 2>(L, it, plan_pre(L.fplan[0], h1, h1.count), vals, tree, stencils, bc, out, epi, smem_raw);
}

// Second part: the tiles of the levels in lr (those below l_max) whose taps reach outside the
// central 3^3 (none for a restricted stack), as radius-2 tiles in a persistent grid, each block
// taking every gridDim.x-th of them. Block 0 records in *hint whether there were any.
__global__ void __launch_bounds__(NT, 4) conv_fwd_r2_pool_kernel(const DevLayout L, const Item *__restrict__ items,
                                                                 const LevelRanges lr, int *hint,
                                                                 const float *__restrict__ vals,
                                                                 const float *__restrict__ tree,
                                                                 const float *__restrict__ stencils, int bc,
                                                                 float *out, const Epilogue epi) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const unsigned sel = levels_with_outer_taps(stencils, lr.l0 - L.l_min, lr.n, reinterpret_cast<unsigned *>(smem_raw));
    if (blockIdx.x == 0 && threadIdx.x == 0) *hint = sel != 0u;
    const int total = selected_count(lr, sel);
#pragma unroll 1
    for (int j = int(blockIdx.x); j < total; j += int(gridDim.x)) {
        const int tile = selected_item(lr, sel, j);
        const Item it = items[tile];
        const PlanHdr h2 = plan_hdr(L.fplan[1], tile);
        conv_fwd_tile<2, 2>(L, it, plan_pre(L.fplan[1], h2, h2.count), vals, tree, stencils, bc, out, epi, smem_raw);
        __syncthreads();   // the next tile reuses the shared memory
    }
    pdl_wait();   // launched beside the radius-1 launch's tail: complete only after it
}

// Gradient magnitude (Sec. 4.3, Sobel filters with level-rescaled stencils, Eq. adapt_grad):
// out[p] = sqrt(sum_a (w_a (*) u)_p^2) for three stencil stacks w_a (a = z, x, y) on one staged
// patch; each window's three sums are taken by the same two lanes in turn.
template <int R>
__global__ void __launch_bounds__(NT, R == 1 ? 5 : 4) conv_gradmag_kernel(const DevLayout L, const Item *__restrict__ items,
                                                             const float *__restrict__ vals,
                                                             const float *__restrict__ tree,
                                                             const float *__restrict__ stencils, int bc,
                                                             float *__restrict__ out) {
    using G = Geo<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FwdSmem<R, 3> &S = *reinterpret_cast<FwdSmem<R, 3> *>(smem_raw);
    const Item it = items[blockIdx.x];
    const PlanHdr hd = plan_hdr(L.fplan[R - 1], blockIdx.x);
    const PlanPre pp = plan_pre(L.fplan[R - 1], hd, hd.count);
    const int n_levels = L.l_max - L.l_min + 1;
#pragma unroll 1
    for (int a = 0; a < 3; ++a) load_taps2<R>(stencils + size_t(a) * n_levels * G::K3, it.l - L.l_min, false, S.w2[a]);
    stage_fwd<R, 3>(L, it, pp, vals, tree, bc, S);
    constexpr int LPW = lanes_per_window<R>(), NO = WIN / LPW;  // outputs kept per lane
    const int sub = threadIdx.x % LPW;
    for (int base = 0; base < S.nact; base += NT / LPW) {
        const int ai = base + threadIdx.x / LPW;
        const bool valid = ai < S.nact;
        const int w = valid ? S.act[ai] : 0;
        float sq[NO];
#pragma unroll
        for (int k = 0; k < NO; ++k) sq[k] = 0.f;
#pragma unroll 1
        for (int a = 0; a < 3; ++a) {
            float acc[WIN];
            if (valid) {
                window_part2<R>(S.patch, S.w2[a], S.roff, w, sub, acc);
            } else {
#pragma unroll
                for (int j = 0; j < WIN; ++j) acc[j] = 0.f;
            }
            if constexpr (LPW == 1) {
#pragma unroll
                for (int k = 0; k < NO; ++k) sq[k] = fmaf(acc[k], acc[k], sq[k]);
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float send = sub ? acc[k] : acc[4 + k];
                    const float keep = sub ? acc[4 + k] : acc[k];
                    const float v = keep + __shfl_xor_sync(0xffffffffu, send, 1);
                    sq[k] = fmaf(v, v, sq[k]);
                }
            }
        }
        if (valid) {
            const unsigned m = win_mask(S, w);
            const int j0 = NO * sub;
            int p = win_first(S, w) + __popc(m & ((1u << j0) - 1u));
#pragma unroll
            for (int k = 0; k < NO; ++k)
                if ((m >> (j0 + k)) & 1u) {
                    out[p] = sqrtf(sq[k]);
                    ++p;
                }
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Backward, stencil part: per work item, partial[e][item] = sum over its targets p of g_p *
// u_l(p + e) (fixed order); stencil_grad_reduce_kernel then sums the items of every level.
// ------------------------------------------------------------------------------------------------
template <int R>
__global__ void __launch_bounds__(NT, R == 1 ? 5 : 4) conv_bwd_stencil_kernel(const DevLayout L, const Item *__restrict__ items,
                                                                 int n_items, const float *__restrict__ vals,
                                                                 const float *__restrict__ tree, int bc,
                                                                 const float *__restrict__ gout,
                                                                 float *__restrict__ partial) {
    using G = Geo<R>;
    using Smem = FwdSmem<R, 1>;
    constexpr int NGRP = NT / G::NPAIR;
    static_assert(NGRP * G::NPAIR * G::K <= G::NROW * G::PYS, "partials fit in the patch");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>(smem_raw);
    const Item it = items[blockIdx.x];
    const PlanHdr hd = plan_hdr(L.fplan[R - 1], blockIdx.x);
    stage_fwd<R, 1>(L, it, plan_pre(L.fplan[R - 1], hd, hd.count), vals, tree, bc, S);
    const int tid = threadIdx.x;
    const int pair = tid % G::NPAIR, grp = tid / G::NPAIR;
    // acc2[t] = (sum over even j, sum over odd j) of g_j * P[row][col + j + t]: taps t even pair
    // (g_{2i}, g_{2i+1}) with the aligned values (v_{2i+t}, v_{2i+1+t}), taps t odd pair
    // (g_{2i-1}, g_{2i}) with (v_{2i-1+t}, v_{2i+t}), also aligned (g_{-1} = g_8 = 0)
    float2 acc2[G::K];
#pragma unroll
    for (int t = 0; t < G::K; ++t) acc2[t] = make_float2(0.f, 0.f);
    const int roff = grp < NGRP ? S.roff[pair] : 0;
    // the windows in chunks: dL/dout of a chunk's windows (0 at cells without a target) are read
    // from global memory once into the place of the staging tables, then every stencil row uses them
    for (int c0 = 0; c0 < S.nact; c0 += Smem::GWIN) {
        const int nc = min(Smem::GWIN, S.nact - c0);
        float *gw = reinterpret_cast<float *>(S.gwin);
        for (int i = tid; i < nc * WIN; i += NT) {
            const int w = S.act[c0 + i / WIN], j = i % WIN;
            const unsigned m = win_mask(S, w);
            gw[i] = ((m >> j) & 1u) ? gout[win_first(S, w) + __popc(m & ((1u << j) - 1u))] : 0.f;
        }
        block_sync();
        if (grp < NGRP) {
            for (int a = grp; a < nc; a += NGRP) {
                const int w = S.act[c0 + a], r = w / NWIN;
                const float4 *src = reinterpret_cast<const float4 *>(
                    S.patch + ((r / TX) * G::PX + (r % TX)) * G::PYS + roff + (w % NWIN) * WIN);
                const float4 q0 = src[0], q1 = src[1], q2 = src[2];
                const float2 V[6] = {make_float2(q0.x, q0.y), make_float2(q0.z, q0.w), make_float2(q1.x, q1.y),
                                     make_float2(q1.z, q1.w), make_float2(q2.x, q2.y), make_float2(q2.z, q2.w)};
                const float4 ga = S.gwin[2 * a], gb = S.gwin[2 * a + 1];
                const float2 Ge[4] = {make_float2(ga.x, ga.y), make_float2(ga.z, ga.w), make_float2(gb.x, gb.y),
                                      make_float2(gb.z, gb.w)};
                const float2 Go[5] = {make_float2(0.f, ga.x), make_float2(ga.y, ga.z), make_float2(ga.w, gb.x),
                                      make_float2(gb.y, gb.z), make_float2(gb.w, 0.f)};
#pragma unroll
                for (int t = 0; t < G::K; ++t) {
                    if (t % 2 == 0) {
#pragma unroll
                        for (int i = 0; i < 4; ++i) acc2[t] = ffma2(Ge[i], V[i + t / 2], acc2[t]);
                    } else {
#pragma unroll
                        for (int i = 0; i < 5; ++i) acc2[t] = ffma2(Go[i], V[i + (t - 1) / 2], acc2[t]);
                    }
                }
            }
        }
        block_sync();   // the next chunk (or the partials) reuse shared memory
    }
    float *red = S.patch;
    if (grp < NGRP)
#pragma unroll
        for (int t = 0; t < G::K; ++t) red[(grp * G::NPAIR + pair) * G::K + t] = acc2[t].x + acc2[t].y;
    block_sync();
    if (tid < G::K3) {
        const int pr = tid / G::K, t = tid % G::K;
        float s = 0.f;
        for (int q = 0; q < NGRP; ++q) s += red[(q * G::NPAIR + pr) * G::K + t];
        partial[size_t(tid) * n_items + blockIdx.x] = s;
    }
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
    block_sync();
    for (int h = NT / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        block_sync();
    }
    if (threadIdx.x == 0) gw[size_t(blockIdx.y) * K3 + e] = red[0];
}

// ------------------------------------------------------------------------------------------------
// Backward, data part: for every interior cell c a target can reach,
//   H(c) = sum over preimages c' of c under the boundary reflection of sum_e w[e] g(c' - e),
// g = dL/dout at the level-l particles (zero elsewhere, and outside the grid). H is routed to the
// source that supplied cell c in the forward patch: the level-l particle (atomic add; it receives
// exactly one more term, from the next finer level, so the sum does not depend on order), the
// level-l tree node (store), or the level-(l-1) particle containing c (sum of its cells in this
// tile, then one atomic add).
// ------------------------------------------------------------------------------------------------
template <int R>
struct BwdSmem {
    using G = Geo<R>;
    static constexpr int NS = G::NROW + G::NRSEG;  // plan segments: gradient rows, routing
    float gpatch[G::NROW * G::PYS];
    __align__(16) float H[NIR * BY];
    __align__(16) float w2[G::NPAIR * w2_stride<R>()];  // flipped taps, paired layout
    unsigned occ[G::NROW * 3];                 // nonzero-gradient columns of every patch row (68 bits)
    unsigned long long dil[G::NROW];           // interior columns within R (in y) of a gradient column
    unsigned long long dilx[G::PZ * TX];       // dil OR-ed over patch rows x .. x + 2R of each z row
    unsigned long long need[NIR];
    int seg_lo[NS];
    unsigned seg_nm[NS];                       // element count | routing / patch-row index << 8
    int pre[NS + 1];                           // packet prefix
    int warp_tot[NWARP + 1];
    unsigned char wmir[NIW];                   // window has cells with mirrored preimages
    unsigned short act[NIW];
    unsigned short pseg[PCAP];
    int roff[G::NPAIR];                        // stencil-row offsets in the patch (fill_row_offsets)
    // routing packets whose y values are kept from the staging pass (radius 1: fewer, so that four
    // blocks share an SM)
    static constexpr int RCAP = R == 1 ? 150 : 320;
    uint4 rstash[RCAP];
    int nact;
};

// The packets of segments [s0, s0 + ns) (packet prefixes in pre[s0 .. s0 + ns]): loads y (from ty for
// segments with tree(seg), else from py) and, for segments with has_vals(seg), the values of 8
// elements per packet, then calls use(seg, p, i0, yq, va, vb, mask) with the packet index p and the
// packet's valid-element mask. Chunks of PCAP packets; ends with a block barrier (with a single
// chunk, pseg still maps every packet to its segment afterwards).
template <typename Tree, typename HasVals, typename Use>
__device__ __forceinline__ void for_each_packet(const int *seg_lo, const unsigned *seg_nm, const int *pre, int s0,
                                                int ns, unsigned short *pseg, const uint16_t *py, const uint16_t *ty,
                                                Tree tree, const float *vals, int nvals, HasVals has_vals, Use use) {
    const int tid = threadIdx.x;
    const int P0 = pre[s0], P1 = pre[s0 + ns];
    for (int c0 = P0; c0 < P1; c0 += PCAP) {
        const int c1 = min(P1, c0 + PCAP);
        for (int s = s0 + tid; s < s0 + ns; s += NT) {
            const int a = max(pre[s], c0), b = min(pre[s + 1], c1);
            for (int p = a; p < b; ++p) pseg[p - c0] = (unsigned short)s;
        }
        block_sync();
        for (int p0 = c0 + tid; p0 < c1; p0 += 2 * NT) {
            uint4 yq[2];
            float4 va[2], vb[2];
            int sg[2], i0[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int p = p0 + u * NT;
                sg[u] = -1;
                i0[u] = 0;
                va[u] = vb[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (p < c1) {
                    const int s = pseg[p - c0];
                    const int g8 = (seg_lo[s] >> 3) + (p - pre[s]);
                    yq[u] = __ldg(reinterpret_cast<const uint4 *>(tree(s) ? ty : py) + g8);
                    if (has_vals(s)) {
                        if (8 * g8 + 8 <= nvals) {
                            va[u] = __ldg(reinterpret_cast<const float4 *>(vals) + 2 * g8);
                            vb[u] = __ldg(reinterpret_cast<const float4 *>(vals) + 2 * g8 + 1);
                        } else {
                            float e[8];
                            const int nv = nvals - 8 * g8;
#pragma unroll
                            for (int j = 0; j < 8; ++j) e[j] = j < nv ? vals[8 * g8 + j] : 0.f;
                            va[u] = make_float4(e[0], e[1], e[2], e[3]);
                            vb[u] = make_float4(e[4], e[5], e[6], e[7]);
                        }
                    }
                    sg[u] = s;
                    i0[u] = 8 * g8;
                }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (sg[u] < 0) continue;
                const int lo = seg_lo[sg[u]], n = int(seg_nm[sg[u]] & 255u);
                unsigned m = 0u;
#pragma unroll
                for (int j = 0; j < 8; ++j) m |= (unsigned(i0[u] + j - lo) < unsigned(n) ? 1u : 0u) << j;
                use(sg[u], p0 + u * NT, i0[u], yq[u], va[u], vb[u], m);
            }
        }
        block_sync();
    }
}

__device__ __forceinline__ void unpack_y(const uint4 &q, int y[8]) {
    y[0] = int(q.x & 0xffffu), y[1] = int(q.x >> 16), y[2] = int(q.y & 0xffffu), y[3] = int(q.y >> 16);
    y[4] = int(q.z & 0xffffu), y[5] = int(q.z >> 16), y[6] = int(q.w & 0xffffu), y[7] = int(q.w >> 16);
}

// Like window_part2 over all stencil rows, one lane per window, for a window whose centre row (ia,
// ib) of the patch may lie outside the tile interior (a mirrored row): stencil rows outside the
// staged patch read zero. Boundary tiles only.
template <int R>
__device__ __forceinline__ void window_checked2(const float *patch, const float *w2, int ia, int ib, int col,
                                                float acc[WIN]) {
    using G = Geo<R>;
    constexpr int WS = w2_stride<R>();
#pragma unroll 1
    for (int pair = 0; pair < G::NPAIR; ++pair) {
        const int dz = pair / G::K, dx = pair % G::K;
        const int rz = ia + dz, rx = ib + dx;
        if (rz < 0 || rz >= G::PZ || rx < 0 || rx >= G::PX) continue;
        const float4 *src = reinterpret_cast<const float4 *>(patch + (rz * G::PX + rx) * G::PYS + col);
        const float4 a0 = src[0], a1 = src[1], a2 = src[2];
        const float v[12] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, a2.x, a2.y, a2.z, a2.w};
#pragma unroll
        for (int t = 0; t < G::K; ++t) {
            const float wt = w2[pair * WS + 2 * t];
#pragma unroll
            for (int j = 0; j < WIN; ++j) acc[j] = fmaf(wt, v[j + t], acc[j]);
        }
    }
}

// One data-adjoint tile with stencil radius R from a stack of radius RS >= R.
template <int R, int RS>
__device__ __forceinline__ void conv_bwd_data_tile(const DevLayout &L, const Item &it, const PlanPre &pp,
                                                   const float *__restrict__ stencils, int bc,
                                                   const float *__restrict__ gout, float *__restrict__ gp,
                                                   float *__restrict__ gt, unsigned char *smem_raw) {
    using G = Geo<R>;
    constexpr int WS = w2_stride<R>();
    BwdSmem<R> &S = *reinterpret_cast<BwdSmem<R> *>(smem_raw);
    const int l = it.l, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const LevelGeo g = L.geo[l];
    const int z0 = it.a * TZ, x0 = it.b * TX, y0 = it.yb * BY;
    const int yw = y0 - R;
    const bool reflect = bc == APR_BC_REFLECT;

    load_taps2<R, RS>(stencils, l - L.l_min, true, S.w2);
    fill_row_offsets<R>(S.roff);
    for (int i = tid; i < G::NROW * G::PYS / 4; i += NT) reinterpret_cast<float4 *>(S.gpatch)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = tid; i < NIR * BY / 4; i += NT) reinterpret_cast<float4 *>(S.H)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = tid; i < G::NROW * 3; i += NT) S.occ[i] = 0u;

    // the tile's non-empty segments (bwd_segment, listed once per APR in the tile plan): n1 gradient
    // rows (in-grid patch rows, trimmed to the patch window; no reflection: g is zero outside the
    // grid), then n2 sources of the interior cells (particles and tree nodes of the interior rows in
    // y-block yb, level-(l-1) particles over the interior)
    const FPlanView P = L.bplan[R - 1];
    const PlanHdr hd = pp.hd;
    const int n1 = hd.count & 0xffff, n2 = hd.count >> 16;
    for (int k = tid; k <= n1 + n2; k += NT) {
        const uint2 raw = k == tid ? pp.e0 : P.ent[hd.first + k];
        const FPlanEnt e{raw.x, raw.y};
        if (k < n1 + n2) {
            S.seg_lo[k] = fplan_lo(e);
            S.seg_nm[k] = unsigned(fplan_n(e)) | (unsigned(fplan_meta(e)) << 8);
        }
        S.pre[k] = fplan_pre(e);
    }
    block_sync();

    // gradient patch and its occupancy (the first n1 segments; one patch row per segment), in one pass
    // with the y values of the routing segments, which are kept in rstash for the routing at the end
    const auto is_tree = [&](int seg) {
        const int q = int(S.seg_nm[seg] >> 8);
        return seg >= n1 && q >= NIR && q < 2 * NIR;
    };
    const int P1 = S.pre[n1], P2 = S.pre[n1 + n2];
    for_each_packet(S.seg_lo, S.seg_nm, S.pre, 0, n1 + n2, S.pseg, L.y, L.ty, is_tree, gout, L.np,
                    [&](int seg) { return seg < n1; },
                    [&](int seg, int p, int, const uint4 &yq, const float4 &va, const float4 &vb, unsigned m) {
                        if (seg >= n1) {
                            if (p - P1 < BwdSmem<R>::RCAP) S.rstash[p - P1] = yq;
                            return;
                        }
                        const int row = int(S.seg_nm[seg] >> 8);
                        float *prow = S.gpatch + row * G::PYS;
                        int yv[8];
                        unpack_y(yq, yv);
                        const float vv[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
                        unsigned o[3] = {0u, 0u, 0u};
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            if (!((m >> j) & 1u)) continue;
                            const int pos = yv[j] - yw;
                            prow[pos] = vv[j];
                            o[pos >> 5] |= 1u << (pos & 31);
                        }
#pragma unroll
                        for (int wd = 0; wd < 3; ++wd)
                            if (o[wd]) atomicOr(&S.occ[row * 3 + wd], o[wd]);
                    });
    // y-dilation of every patch row: interior column j <-> patch column j + R, needed if any of the
    // patch columns j .. j + 2R holds a gradient; dilx: the same OR-ed over the 2R + 1 patch rows
    // x .. x + 2R of one patch z row, for the TX interior x columns (the dilation is separable)
    const auto ydil = [&](int row) {
        const unsigned long long lo64 = (unsigned long long)S.occ[row * 3] | ((unsigned long long)S.occ[row * 3 + 1] << 32);
        const unsigned long long hi64 = S.occ[row * 3 + 2];
        unsigned long long m = lo64;
#pragma unroll
        for (int d = 1; d <= 2 * R; ++d) m |= (lo64 >> d) | (hi64 << (64 - d));
        return m;
    };
    for (int row = tid; row < G::NROW; row += NT) S.dil[row] = ydil(row);
    for (int i = tid; i < G::PZ * TX; i += NT) {
        const int pz = i / TX, ib = i % TX;
        unsigned long long m = 0ull;
#pragma unroll
        for (int dx = 0; dx <= 2 * R; ++dx) m |= ydil(pz * G::PX + ib + dx);
        S.dilx[i] = m;
    }
    block_sync();

    // cells that need H: within R of a nonzero gradient, or (reflect) close enough to the grid
    // boundary to have mirrored preimages; windows with any such cell are active. Four threads per
    // interior row, each over a quarter of the stencil rows; bit j of need[r] = interior cell j.
    static_assert(NIR * 4 == NT, "four threads per interior row");
    {
        const int r = tid >> 2, q = tid & 3;
        const int z = z0 + r / TX, x = x0 + r % TX;
        const bool valid = z < g.dz && x < g.dx;
        unsigned long long m = 0ull;
        bool edge_zx = false;
        if (valid) {
            uint64_t wz, wx;  // rows and their mirrors, relative to the patch's first row (z0 - R)
            const int nz = with_mirrors<R>(z, g.dz, z0 - R, true, reflect, wz);
            const int nx = with_mirrors<R>(x, g.dx, x0 - R, true, reflect, wx);
            edge_zx = nz > 1 || nx > 1;
            if (!edge_zx) {
                // no mirrored rows: the patch rows (ia + dz, ib + dx), dz, dx in [0, 2R]
                for (int dz = q; dz <= 2 * R; dz += 4) m |= S.dilx[((r / TX) + dz) * TX + (r % TX)];
            } else {
                for (int iz = 0; iz < nz; ++iz)
                    for (int ix = 0; ix < nx; ++ix)
                        for (int pr = q; pr < G::NPAIR; pr += 4) {
                            const int rz = at8(wz, iz) - R + pr / G::K, rx = at8(wx, ix) - R + pr % G::K;  // patch row
                            if (rz < 0 || rz >= G::PZ || rx < 0 || rx >= G::PX) continue;
                            m |= S.dil[rz * G::PX + rx];
                        }
            }
        }
        const unsigned mlo = unsigned(m), mhi = unsigned(m >> 32);
        const unsigned olo = mlo | __shfl_xor_sync(0xffffffffu, mlo, 1), ohi = mhi | __shfl_xor_sync(0xffffffffu, mhi, 1);
        m = (unsigned long long)(olo | __shfl_xor_sync(0xffffffffu, olo, 2)) |
            ((unsigned long long)(ohi | __shfl_xor_sync(0xffffffffu, ohi, 2)) << 32);
        if (q == 0) {
            // cells inside the grid, and (reflect) cells within R of the y boundary of the grid
            const int nvalid = g.dy - y0;
            const unsigned long long vmask = nvalid >= BY ? ~0ull : (nvalid <= 0 ? 0ull : ((1ull << nvalid) - 1ull));
            const int jl = R - y0, jh = g.dy - R - y0;
            const unsigned long long ylow = jl <= 0 ? 0ull : (jl >= BY ? ~0ull : ((1ull << jl) - 1ull));
            const unsigned long long yhigh = jh <= 0 ? ~0ull : (jh >= BY ? 0ull : (~0ull << jh));
            const unsigned long long yedge = reflect && valid ? (ylow | yhigh) & vmask : 0ull;
            m = valid ? (m | yedge) & vmask : 0ull;
            // wmir: bit 0 = the row has mirrored rows (z or x), bit 1 = the window has cells within R
            // of the y boundary
#pragma unroll
            for (int w = 0; w < NWIN; ++w)
                S.wmir[r * NWIN + w] = (unsigned char)((reflect && valid && edge_zx ? 1 : 0) |
                                                       (((yedge >> (w * WIN)) & 0xffull) ? 2 : 0));
            S.need[r] = m;
        }
    }
    block_sync();
    // active windows, in window order (rows of warps 0 and 1)
    if (tid < NIR) {
        const unsigned long long m = S.need[tid];
        unsigned am = 0u;
#pragma unroll
        for (int w = 0; w < NWIN; ++w) am |= ((m >> (w * WIN)) & 0xffull) ? (1u << w) : 0u;
        const int c = __popc(am);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) S.warp_tot[warp] = incl;
        pair_sync(0);
        int k = (warp == 1 ? S.warp_tot[0] : 0) + incl - c;
#pragma unroll
        for (int w = 0; w < NWIN; ++w)
            if ((am >> w) & 1u) S.act[k++] = (unsigned short)(tid * NWIN + w);
        if (tid == NIR - 1) S.nact = k;
    }
    block_sync();

    // H = (flipped stencil) correlated with the gradient patch, at the active windows (c' = c term)
    fwd_windows<R>(S.gpatch, S.w2, S.roff, S.act, S.nact, [&](int w, int j0, const float *v, int n) {
        float4 *dst = reinterpret_cast<float4 *>(S.H + (w / NWIN) * BY + (w % NWIN) * WIN + j0);
#pragma unroll
        for (int k = 0; k < n; k += 4) dst[k / 4] = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
    });
    block_sync();
    // mirrored preimages (reflect only). Rows with mirrored z / x rows: one thread per active window
    // sums the windows of all mirrored row combinations (z', x') != (z, x) (same y cells); stencil
    // rows outside the staged patch read zero, as the gradient outside the grid is zero. Cells within
    // R of the y boundary then add the combinations whose y is mirrored.
    if (reflect) {
        for (int a = tid; a < S.nact; a += NT) {
            const int w = S.act[a];
            if (!(S.wmir[w] & 1)) continue;
            const int r = w / NWIN, col = (w % NWIN) * WIN;
            const int z = z0 + r / TX, x = x0 + r % TX;
            uint64_t wz, wx;
            const int nz = with_mirrors<R>(z, g.dz, z0 - R, true, true, wz);
            const int nx = with_mirrors<R>(x, g.dx, x0 - R, true, true, wx);
            float acc[WIN];
#pragma unroll
            for (int j = 0; j < WIN; ++j) acc[j] = 0.f;
            for (int iz = 0; iz < nz; ++iz)
                for (int ix = 0; ix < nx; ++ix)
                    if (iz != 0 || ix != 0) window_checked2<R>(S.gpatch, S.w2, at8(wz, iz) - R, at8(wx, ix) - R, col, acc);
            float *dst = S.H + r * BY + col;
#pragma unroll
            for (int j = 0; j < WIN; ++j) dst[j] += acc[j];
        }
        block_sync();
        // y-mirrored combinations: one thread per (interior row, cell within R of the y boundary)
        const int nlow = y0 == 0 ? min(R, g.dy) : 0;                       // cells 0 .. nlow-1
        const int hb = max(g.dy - R, max(y0, nlow));                        // cells hb .. min(dy, y0+BY)-1
        const int nhigh = max(0, min(g.dy, y0 + BY) - hb);
        const int per_row = nlow + nhigh;
        for (int task = tid; task < NIR * per_row; task += NT) {
            const int r = task / per_row, q = task % per_row;
            const int j = q < nlow ? q : hb - y0 + (q - nlow);
            const int z = z0 + r / TX, x = x0 + r % TX, yy = y0 + j;
            if (z >= g.dz || x >= g.dx) continue;
            if (!((S.need[r] >> j) & 1ull)) continue;
            uint64_t wz, wx, wy;
            const int nz = with_mirrors<R>(z, g.dz, z0 - R, true, true, wz);
            const int nx = with_mirrors<R>(x, g.dx, x0 - R, true, true, wx);
            const int ny = with_mirrors<R>(yy, g.dy, yw, false, true, wy);
            float h0 = 0.f, h1 = 0.f;
            for (int iz = 0; iz < nz; ++iz)
                for (int ix = 0; ix < nx; ++ix)
                    for (int iy = 0; iy < ny; ++iy) {
                        // taps e with c' - e inside the staged window (the rest reads zero gradient)
                        const int cz = at8(wz, iz), cx = at8(wx, ix), cy = at8(wy, iy);
                        const int ey0 = max(-R, cy - G::PY + 1), ey1 = min(R, cy);
#pragma unroll 1
                        for (int ez = -R; ez <= R; ++ez)
#pragma unroll 1
                            for (int ex = -R; ex <= R; ++ex) {
                                const int sz = cz - ez, sx = cx - ex;
                                if (sz < 0 || sz >= G::PZ || sx < 0 || sx >= G::PX) continue;
                                // unflipped tap w[ez][ex][ey] sits at flipped pair (R-ez, R-ex), slot R-ey
                                const float *wrow = S.w2 + ((R - ez) * G::K + (R - ex)) * WS + 2 * R;
                                const float *grow = S.gpatch + (sz * G::PX + sx) * G::PYS + cy;
                                for (int ey = ey0; ey <= ey1; ++ey) {
                                    if ((ey & 1) == 0) h0 = fmaf(wrow[-2 * ey], grow[-ey], h0);
                                    else h1 = fmaf(wrow[-2 * ey], grow[-ey], h1);
                                }
                            }
                    }
            S.H[r * BY + j] += h0 + h1;
        }
        block_sync();
    }
    // routing: the sources of the interior cells, plan segments n1 .. n1 + n2 (routing index q)
    const auto route = [&](int seg, int i0, const uint4 &yq, unsigned m) {
                        const int q = int(S.seg_nm[seg] >> 8);
                        int yv[8];
                        unpack_y(yq, yv);
                        if (q < NIR) {
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                if ((m >> j) & 1u) {
                                    const float h = S.H[q * BY + (yv[j] - y0)];
                                    if (h != 0.f) atomicAdd(&gp[i0 + j], h);
                                }
                        } else if (q < 2 * NIR) {
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                if ((m >> j) & 1u) gt[i0 + j] = S.H[(q - NIR) * BY + (yv[j] - y0)];
                        } else {
                            // a level-(l-1) particle: the sum of H over its (up to) 2 x 2 x 2 level-l cells,
                            // in (a, b, e) order; the two cells along y are one aligned float2 (y0, j0 even)
                            const int r = q - 2 * NIR;
                            const int ia = 2 * (r / (TX / 2)), ib = 2 * (r % (TX / 2));
                            const bool za = z0 + ia + 1 < g.dz, xb = x0 + ib + 1 < g.dx;  // second rows in the grid
                            const float *h0 = S.H + (ia * TX + ib) * BY;
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                if (!((m >> j) & 1u)) continue;
                                const int j0 = 2 * yv[j] - y0;  // first level-l cell column of the coarser particle
                                if (j0 < 0 || j0 >= BY) continue;
                                const bool ye = y0 + j0 + 1 < g.dy;
                                float sum = 0.f;
#pragma unroll
                                for (int a = 0; a < 2; ++a)
#pragma unroll
                                    for (int b = 0; b < 2; ++b) {
                                        if ((a && !za) || (b && !xb)) continue;
                                        const float2 h = *reinterpret_cast<const float2 *>(h0 + (a * TX + b) * BY + j0);
                                        sum += h.x;
                                        if (ye) sum += h.y;
                                    }
                                if (sum != 0.f) atomicAdd(&gp[i0 + j], sum);
                            }
                        }
    };
    if (P2 <= PCAP) {
        // one staging chunk: pseg still maps the routing packets to their segments, and their y
        // values are in rstash (the packets beyond its capacity are read again)
        for (int p = P1 + tid; p < P2; p += NT) {
            const int seg = S.pseg[p];
            const int lo = S.seg_lo[seg], n = int(S.seg_nm[seg] & 255u);
            const int g8 = (lo >> 3) + (p - S.pre[seg]);
            const uint4 yq = p - P1 < BwdSmem<R>::RCAP ? S.rstash[p - P1]
                                                       : __ldg(reinterpret_cast<const uint4 *>(is_tree(seg) ? L.ty : L.y) + g8);
            unsigned m = 0u;
#pragma unroll
            for (int j = 0; j < 8; ++j) m |= (unsigned(8 * g8 + j - lo) < unsigned(n) ? 1u : 0u) << j;
            route(seg, 8 * g8, yq, m);
        }
    } else {
        for_each_packet(S.seg_lo, S.seg_nm, S.pre, n1, n2, S.pseg, L.y, L.ty, is_tree, nullptr, 0,
                        [](int) { return false; },
                        [&](int seg, int, int i0, const uint4 &yq, const float4 &, const float4 &, unsigned m) {
                            route(seg, i0, yq, m);
                        });
    }
}

template <int R>
__global__ void __launch_bounds__(NT, R == 1 ? 4 : 3) conv_bwd_data_kernel(const DevLayout L, const Item *__restrict__ items,
                                                              int tile0, const float *__restrict__ stencils, int bc,
                                                              const float *__restrict__ gout,
                                                              float *__restrict__ gp, float *__restrict__ gt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tile = tile0 + int(blockIdx.x);   // work items [tile0, tile0 + gridDim.x)
    const Item it = items[tile];
    // the plan headers of both radii the tile may take, loaded with the item (the entries are read
    // only for the radius taken)
    const PlanHdr h1 = plan_hdr(L.bplan[0], tile);
    if constexpr (R == 2) {
        const PlanHdr h2 = plan_hdr(L.bplan[1], tile);
        if (outer_taps_zero5(stencils, it.l - L.l_min)) {
            conv_bwd_data_tile<1, 2>(L, it, plan_pre(L.bplan[0], h1, bplan_count(h1)), stencils, bc, gout, gp, gt, smem_raw);
            return;
        }
        conv_bwd_data_tile<2, 2>(L, it, plan_pre(L.bplan[1], h2, bplan_count(h2)), stencils, bc, gout, gp, gt, smem_raw);
    } else {
        conv_bwd_data_tile<R, R>(L, it, plan_pre(L.bplan[0], h1, bplan_count(h1)), stencils, bc, gout, gp, gt, smem_raw);
    }
}

// The data adjoint of a 5^3 stack over the whole work list, split by radius like the convolution:
// radius-1 tiles of the levels below l_max (items [0, gridDim.x)) with radius-1 shared memory, four
// blocks per SM instead of three; tiles of a level with outer taps return at once.
__global__ void __launch_bounds__(NT, 4) conv_bwd_data_r1_kernel(const DevLayout L, const Item *__restrict__ items,
                                                                 const float *__restrict__ stencils, int bc,
                                                                 const float *__restrict__ gout,
                                                                 float *__restrict__ gp, float *__restrict__ gt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_trigger();   // the persistent radius-2 launch after this one is independent of it
    const int tile = int(blockIdx.x);
    const Item it = items[tile];
    if (!outer_taps_zero5(stencils, it.l - L.l_min)) return;
    const PlanHdr h1 = plan_hdr(L.bplan[0], tile);
    conv_bwd_data_tile<1, 2>(L, it, plan_pre(L.bplan[0], h1, bplan_count(h1)), stencils, bc, gout, gp, gt, smem_raw);
}

// ... and the tiles of the levels in lr whose taps reach outside the central 3^3, as radius-2 tiles
// in a persistent grid (block 0 records in *hint whether there were any).
__global__ void __launch_bounds__(NT, 3) conv_bwd_data_r2_pool_kernel(const DevLayout L, const Item *__restrict__ items,
                                                                      const LevelRanges lr, int *hint,
                                                                      const float *__restrict__ stencils, int bc,
                                                                      const float *__restrict__ gout,
                                                                      float *__restrict__ gp, float *__restrict__ gt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const unsigned sel = levels_with_outer_taps(stencils, lr.l0 - L.l_min, lr.n, reinterpret_cast<unsigned *>(smem_raw));
    if (blockIdx.x == 0 && threadIdx.x == 0) *hint = sel != 0u;
    const int total = selected_count(lr, sel);
#pragma unroll 1
    for (int j = int(blockIdx.x); j < total; j += int(gridDim.x)) {
        const int tile = selected_item(lr, sel, j);
        const Item it = items[tile];
        const PlanHdr h2 = plan_hdr(L.bplan[1], tile);
        conv_bwd_data_tile<2, 2>(L, it, plan_pre(L.bplan[1], h2, bplan_count(h2)), stencils, bc, gout, gp, gt, smem_raw);
        __syncthreads();   // the next tile reuses the shared memory
    }
    pdl_wait();   // launched beside the radius-1 launch's tail: complete only after it
}

// Records in *hint whether a level in lr of a 5^3 stack has taps outside the central 3^3 (one block).
__global__ void __launch_bounds__(NT) radius_hint_kernel(const float *__restrict__ stencils, int l_idx0, int n,
                                                         int *hint) {
    __shared__ unsigned word;
    const unsigned sel = levels_with_outer_taps(stencils, l_idx0, n, &word);
    if (threadIdx.x == 0) *hint = sel != 0u;
}

// ------------------------------------------------------------------------------------------------
// Tree kernels, one launch per tree level, one thread per tree node. A node's children are the
// cells (2z + a, 2x + b, 2y + e) of level l+1, each a particle or a tree node of that level; the
// node's child map (TreeNodePlan, built once per APR) gives their indices, so a thread reads its map
// and then all eight children at once.
// ------------------------------------------------------------------------------------------------
// The children of one tree node from its child map (TreeNodePlan): child c = 2k + e (k = (a, b) the
// child row, e the child's y parity; (a, b, e) order) is a particle (kind 1) or a tree node (kind 2)
// at index ix[c], or not present (kind 0: outside the grid, or missing from a sub-domain's index).
struct NodeChildren {
    int ix[8];
    int kind[8];
    __device__ __forceinline__ NodeChildren(const int4 &pw, const int4 &tw) {
        const int pv[4] = {pw.x, pw.y, pw.z, pw.w}, tv[4] = {tw.x, tw.y, tw.z, tw.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned pm = unsigned(pv[k]) >> 30, tm = unsigned(tv[k]) >> 30;
            const int pi = int(unsigned(pv[k]) & TNP_INDEX), ti = int(unsigned(tv[k]) & TNP_INDEX);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                // the second child of a kind follows the first of that kind
                const int skip = e ? 1 : 0;
                const bool isp = (pm >> e) & 1u, ist = (tm >> e) & 1u;
                kind[2 * k + e] = isp ? 1 : (ist ? 2 : 0);
                ix[2 * k + e] = isp ? pi + (skip & int(pm & 1u)) : ti + (skip & int(tm & 1u));
            }
        }
    }
};

__device__ __forceinline__ void load_node_plan(const TreeNodePlan *np, int node, int4 &pw, int4 &tw) {
    const int4 *q = reinterpret_cast<const int4 *>(np + node);
    pw = __ldg(q);
    tw = __ldg(q + 1);
}

// APR tree restriction for one level l (Sec. 3.4), one thread per tree node of the level (nodes
// [node0, node0 + n)): the node's value is the average of its children (particles and tree nodes of
// level l+1), summed in (a, b, e) order. Channel ch of C channels-last values.
__global__ void __launch_bounds__(NT) tree_restrict_kernel(const TreeNodePlan *__restrict__ nplan, int node0, int n,
                                                           const float *__restrict__ vals, float *tree, int C,
                                                           int ch) {
    pdl_trigger();
    const int i = int(blockIdx.x) * NT + int(threadIdx.x);
    const bool live = i < n;
    // the child map is static: read before waiting for the finer level's restriction (the launch
    // before this one), whose node values this level reads
    int4 pw = make_int4(0, 0, 0, 0), tw = pw;
    if (live) load_node_plan(nplan, node0 + i, pw, tw);
    pdl_wait();
    if (!live) return;
    const NodeChildren ch8(pw, tw);
    float v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const size_t at = size_t(ch8.ix[c]) * C + ch;
        v[c] = ch8.kind[c] == 1 ? vals[at] : (ch8.kind[c] == 2 ? tree[at] : 0.f);
    }
    float s = 0.f;
    int cnt = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (ch8.kind[c]) {
            s += v[c];
            ++cnt;
        }
    tree[size_t(node0 + i) * C + ch] = cnt ? s / float(cnt) : 0.f;
}

// Backward through the tree averages, one level l (coarse to fine), one thread per tree node t of the
// level: each child (particle or tree node of level l+1) receives gt[t] / n_children(t). Every child
// has one parent, so each is written by one thread.
__global__ void __launch_bounds__(NT) tree_pushdown_kernel(const TreeNodePlan *__restrict__ nplan, int node0, int n,
                                                           float *gp, float *gt) {
    pdl_trigger();
    const int i = int(blockIdx.x) * NT + int(threadIdx.x);
    const bool live = i < n;
    // the child map is static: read before waiting for the coarser level's push-down (the launch
    // before this one), which writes this level's gt
    int4 pw = make_int4(0, 0, 0, 0), tw = pw;
    if (live) load_node_plan(nplan, node0 + i, pw, tw);
    pdl_wait();
    if (!live) return;
    const NodeChildren ch8(pw, tw);
    int cnt = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) cnt += ch8.kind[c] ? 1 : 0;
    const float share = gt[node0 + i] / float(cnt ? cnt : 1);
    float v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = ch8.kind[c] == 1 ? gp[ch8.ix[c]] : (ch8.kind[c] == 2 ? gt[ch8.ix[c]] : 0.f);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        if (ch8.kind[c] == 1) gp[ch8.ix[c]] = v[c] + share;
        else if (ch8.kind[c] == 2) gt[ch8.ix[c]] = v[c] + share;
    }
}

// Shared memory per block sets the blocks per SM (228 KB per SM, 1 KB reserved per block):
// forward 4, data adjoint 3.
static_assert(4 * (sizeof(FwdSmem<2, 1>) + 1024) <= 228 * 1024, "forward: four blocks per SM");
static_assert(4 * (sizeof(FwdSmem<2, 3>) + 1024) <= 228 * 1024, "gradient magnitude: four blocks per SM");
static_assert(3 * (sizeof(BwdSmem<2>) + 1024) <= 228 * 1024, "data adjoint: three blocks per SM");
static_assert(5 * (sizeof(FwdSmem<1, 1>) + 1024) <= 228 * 1024, "radius-1 forward: five blocks per SM");
static_assert(5 * (sizeof(FwdSmem<1, 3>) + 1024) <= 228 * 1024, "radius-1 gradient magnitude: five blocks per SM");
static_assert(4 * (sizeof(BwdSmem<1>) + 1024) <= 228 * 1024, "radius-1 data adjoint: four blocks per SM");
static_assert(sizeof(FwdSmem<1, 1>) <= sizeof(FwdSmem<2, 1>) && sizeof(BwdSmem<1>) <= sizeof(BwdSmem<2>),
              "radius-1 tiles run inside the radius-2 launch");

cudaError_t set_smem(const void *fn, size_t bytes) { return set_max_dynamic_smem(fn, bytes); }

template <int R>
cudaError_t launch_conv_fwd_t(const DevLayout &L, const Item *items, int tile0, int n, const float *vals,
                              const float *tree, const float *st, int bc, float *out, const Epilogue &epi,
                              cudaStream_t s) {
    const size_t sm = sizeof(FwdSmem<R, 1>);
    cudaError_t e = set_smem(reinterpret_cast<const void *>(conv_fwd_kernel<R>), sm);
    if (e != cudaSuccess) return e;
    if (n > 0) conv_fwd_kernel<R><<<n, NT, sm, s>>>(L, items, tile0, vals, tree, st, bc, out, epi);
    return cudaGetLastError();
}

template <int R>
cudaError_t launch_bwd_data_t(const DevLayout &L, const Item *items, int tile0, int n, const float *st, int bc,
                              const float *gout, float *gp, float *gt, cudaStream_t s) {
    const size_t sm = sizeof(BwdSmem<R>);
    cudaError_t e = set_smem(reinterpret_cast<const void *>(conv_bwd_data_kernel<R>), sm);
    if (e != cudaSuccess) return e;
    if (n > 0) conv_bwd_data_kernel<R><<<n, NT, sm, s>>>(L, items, tile0, st, bc, gout, gp, gt);
    return cudaGetLastError();
}

template <int R>
cudaError_t launch_bwd_stencil_t(const DevLayout &L, const Item *items, int n, const float *vals,
                                 const float *tree, int bc, const float *gout, float *partial, cudaStream_t s) {
    const size_t sm = sizeof(FwdSmem<R, 1>);
    cudaError_t e = set_smem(reinterpret_cast<const void *>(conv_bwd_stencil_kernel<R>), sm);
    if (e != cudaSuccess) return e;
    if (n > 0) conv_bwd_stencil_kernel<R><<<n, NT, sm, s>>>(L, items, n, vals, tree, bc, gout, partial);
    return cudaGetLastError();
}

// Streaming multiprocessors of the current device (the persistent grids take a multiple of it).
cudaError_t sm_count(int *n) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(n, cudaDevAttrMultiProcessorCount, dev);
    return e;
}

}  // namespace

// ---- launch entry points used by the C ABI (apr_api.cu)
cudaError_t launch_conv_fwd(int k, const DevLayout &L, const Item *items, int n, const float *vals,
                            const float *tree, const float *st, int bc, float *out, cudaStream_t s, int epi_mode,
                            bool flip, const float *aux, int tile0) {
    const Epilogue epi{epi_mode, flip, aux};
    return k == 3 ? launch_conv_fwd_t<1>(L, items, tile0, n, vals, tree, st, bc, out, epi, s)
                  : launch_conv_fwd_t<2>(L, items, tile0, n, vals, tree, st, bc, out, epi, s);
}

template <int R>
cudaError_t launch_gradmag_t(const DevLayout &L, const Item *items, int n, const float *vals, const float *tree,
                             const float *st, int bc, float *out, cudaStream_t s) {
    const size_t sm = sizeof(FwdSmem<R, 3>);
    cudaError_t e = set_smem(reinterpret_cast<const void *>(conv_gradmag_kernel<R>), sm);
    if (e != cudaSuccess) return e;
    if (n > 0) conv_gradmag_kernel<R><<<n, NT, sm, s>>>(L, items, vals, tree, st, bc, out);
    return cudaGetLastError();
}

cudaError_t launch_gradmag(int k, const DevLayout &L, const Item *items, int n, const float *vals, const float *tree,
                           const float *st, int bc, float *out, cudaStream_t s) {
    return k == 3 ? launch_gradmag_t<1>(L, items, n, vals, tree, st, bc, out, s)
                  : launch_gradmag_t<2>(L, items, n, vals, tree, st, bc, out, s);
}

cudaError_t launch_tree_restrict(const TreeNodePlan *np, int node0, int n, const float *vals, float *tree,
                                 cudaStream_t s, int C, int ch, bool pdl) {
    if (n <= 0) return cudaSuccess;
    return launch_pdl(tree_restrict_kernel, dim3((n + NT - 1) / NT), dim3(NT), 0, s, pdl, np, node0, n, vals, tree, C,
                      ch);
}

cudaError_t launch_bwd_data(int k, const DevLayout &L, const Item *items, int n, const float *st, int bc,
                            const float *gout, float *gp, float *gt, cudaStream_t s, int tile0) {
    return k == 3 ? launch_bwd_data_t<1>(L, items, tile0, n, st, bc, gout, gp, gt, s)
                  : launch_bwd_data_t<2>(L, items, tile0, n, st, bc, gout, gp, gt, s);
}

// The levels-below-l_max part of a 5^3 convolution (items [0, n_lo), level ranges lo), both launches
// on stream s: radius-1 tiles, then the persistent radius-2 launch for levels with outer taps, which
// writes *hint (see launch_radius_hint).
cudaError_t launch_conv_fwd_split(const DevLayout &L, const Item *items, int n_lo, const LevelRanges &lo, int *hint,
                                  const float *vals, const float *tree, const float *st, int bc, float *out,
                                  cudaStream_t s, int epi_mode, bool flip, const float *aux) {
    if (n_lo <= 0) return cudaSuccess;
    const Epilogue epi{epi_mode, flip, aux};
    const size_t sm1 = sizeof(FwdSmem<1, 1>), sm2 = sizeof(FwdSmem<2, 1>);
    cudaError_t e = set_smem(reinterpret_cast<const void *>(conv_fwd_r1_kernel), sm1);
    if (e == cudaSuccess) e = set_smem(reinterpret_cast<const void *>(conv_fwd_r2_pool_kernel), sm2);
    int nsm = 0;
    if (e == cudaSuccess) e = sm_count(&nsm);
    if (e != cudaSuccess) return e;
    conv_fwd_r1_kernel<<<n_lo, NT, sm1, s>>>(L, items, vals, tree, st, bc, out, epi);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_pdl(conv_fwd_r2_pool_kernel, dim3(std::min(n_lo, 4 * nsm)), dim3(NT), sm2, s, true, L, items, lo, hint,
                      vals, tree, st, bc, out, epi);
}

// The same for the data adjoint (items [0, n_lo) of the adjoint work list).
cudaError_t launch_bwd_data_split(const DevLayout &L, const Item *items, int n_lo, const LevelRanges &lo, int *hint,
                                  const float *st, int bc, const float *gout, float *gp, float *gt, cudaStream_t s) {
    if (n_lo <= 0) return cudaSuccess;
    const size_t sm1 = sizeof(BwdSmem<1>), sm2 = sizeof(BwdSmem<2>);
    cudaError_t e = set_smem(reinterpret_cast<const void *>(conv_bwd_data_r1_kernel), sm1);
    if (e == cudaSuccess) e = set_smem(reinterpret_cast<const void *>(conv_bwd_data_r2_pool_kernel), sm2);
    int nsm = 0;
    if (e == cudaSuccess) e = sm_count(&nsm);
    if (e != cudaSuccess) return e;
    conv_bwd_data_r1_kernel<<<n_lo, NT, sm1, s>>>(L, items, st, bc, gout, gp, gt);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_pdl(conv_bwd_data_r2_pool_kernel, dim3(std::min(n_lo, 3 * nsm)), dim3(NT), sm2, s, true, L, items, lo,
                      hint, st, bc, gout, gp, gt);
}

// *hint = whether a level of lo (a 5^3 stack) has taps outside the central 3^3: the radius split
// pays off only when none has, and the next call reads the hint to choose.
cudaError_t launch_radius_hint(const DevLayout &L, const LevelRanges &lo, const float *st, int *hint, cudaStream_t s) {
    radius_hint_kernel<<<1, NT, 0, s>>>(st, lo.l0 - L.l_min, lo.n, hint);
    return cudaGetLastError();
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

cudaError_t launch_tree_pushdown(const TreeNodePlan *np, int node0, int n, float *gp, float *gt, cudaStream_t s,
                                 bool pdl) {
    if (n <= 0) return cudaSuccess;
    return launch_pdl(tree_pushdown_kernel, dim3((n + NT - 1) / NT), dim3(NT), 0, s, pdl, np, node0, n, gp, gt);
}

}  // namespace aprk
