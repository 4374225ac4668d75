// Device helpers shared by the single-channel and multi-channel kernels: block barrier, reflection,
// per-block row offsets, block scan and the flattened element-staging loop.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "apr_internal.h"

namespace aprk {
namespace dev {

constexpr int NT = 256;                // threads per block of every kernel below
constexpr int NWARP = NT / 32;
constexpr int UNROLL = 4;              // element loads in flight per thread and staging step
static_assert(TZ % 2 == 0 && TX % 2 == 0, "tiles must be even-aligned (coarse cells)");

// Block barrier. The warp is reconverged first: threads of one warp may reach this point at
// different times after data-dependent loops, and the block barrier must be executed by converged
// warps.
__device__ __forceinline__ void block_sync() {
    __syncwarp();
    __syncthreads();
}

// Barrier of the two warps 2g and 2g+1 (named barrier 1 + g; barrier 0 is the block barrier).
__device__ __forceinline__ void pair_sync(int g) {
    __syncwarp();
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(64) : "memory");
}

__host__ __device__ __forceinline__ int imax(int a, int b) { return a > b ? a : b; }
__host__ __device__ __forceinline__ int imin(int a, int b) { return a < b ? a : b; }

__host__ __device__ __forceinline__ int reflect_idx(int i, int d) {
    // half-sample symmetric reflection into [0, d), repeated for grids smaller than the stencil
    const int p = 2 * d;
    int m = i % p;
    if (m < 0) m += p;
    return m >= d ? p - 1 - m : m;
}

// First element of y-block j of a row (particles or tree); j >= nb gives the row end.
__host__ __device__ __forceinline__ uint32_t blk_start(const uint32_t *rp, const uint16_t *off, int row0, int off0,
                                                       int nb, int rr, int j) {
    if (j >= nb) return rp[row0 + rr + 1];
    return rp[row0 + rr] + off[off0 + rr * nb + j];
}

__device__ __forceinline__ uint32_t pblock(const DevLayout &L, const LevelGeo &g, int rr, int j) {
    return blk_start(L.row_ptr, L.off, g.row0, g.off0, g.nb, rr, j);
}

// Index range [lo, hi) of a row containing every element with y in [ya, yb) (ya < yb), plus at
// most BY/2 extra elements on each side (callers filter by y). Uses the per-block offsets only:
// at most BY - ra elements of block ja lie at or after ya, at most rb elements of block jb before yb.
__host__ __device__ __forceinline__ void row_range(const uint32_t *rp, const uint16_t *off, int row0, int off0, int nb,
                                                   int rr, int ya, int yb, int &lo, int &hi) {
    const int rs = int(rp[row0 + rr]), re = int(rp[row0 + rr + 1]);
    const int ja = ya / BY, ra = ya - ja * BY;
    const int jb = yb / BY, rb = yb - jb * BY;
    int a = ra <= BY / 2 ? int(blk_start(rp, off, row0, off0, nb, rr, ja))
                         : int(blk_start(rp, off, row0, off0, nb, rr, ja + 1)) - (BY - ra);
    int b = rb <= BY / 2 ? int(blk_start(rp, off, row0, off0, nb, rr, jb)) + rb
                         : int(blk_start(rp, off, row0, off0, nb, rr, jb + 1));
    a = imax(a, rs);
    b = imin(b, re);
    lo = a;
    hi = imax(a, b);
}

// Block-wide exclusive scan of values held two per thread (entries 2t, 2t+1): writes pre[0..n]
// (pre[n] = total). n <= 2*NT. Starts and ends with a barrier.
__device__ inline void block_scan2(int c0, int c1, int n, int *pre, int *warp_tot) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s = c0 + c1;
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    block_sync();
    if (lane == 31) warp_tot[warp] = incl;
    block_sync();
    if (tid == 0) {
        int acc = 0;
        for (int w = 0; w < NWARP; ++w) {
            const int v = warp_tot[w];
            warp_tot[w] = acc;
            acc += v;
        }
        warp_tot[NWARP] = acc;
    }
    block_sync();
    const int excl = warp_tot[warp] + incl - s;
    if (2 * tid < n) pre[2 * tid] = excl;
    if (2 * tid + 1 < n) pre[2 * tid + 1] = excl + c0;
    if (tid == 0) pre[n] = warp_tot[NWARP];
    block_sync();
}

struct SlotYV {
    int y;
    float v;
};

// Loads y and value of element i of segment seg; segments [t0, t1) are tree segments.
struct YVLoader {
    using Slot = SlotYV;
    const uint16_t *py, *ty;
    const float *pv, *tv;
    int t0, t1;
    __device__ __forceinline__ void operator()(int seg, int i, Slot &s) const {
        const bool t = seg >= t0 && seg < t1;
        s.y = t ? int(ty[i]) : int(py[i]);
        s.v = t ? tv[i] : pv[i];
    }
};

// Programmatic dependent launch (launch_pdl): pdl_trigger lets the next kernel on the stream start
// (its blocks run their prologue while this kernel finishes); pdl_wait blocks until the kernel before
// this one on the stream has completed and its writes are visible. In a kernel launched without the
// attribute both are no-ops.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Flattened loop over the elements of nseg segments (segment s: global indices seg_lo[s] ..
// seg_lo[s] + pre[s+1] - pre[s]), in chunks of SEGID_CAP elements. For every chunk, the threads
// first write the segment id of each element into segid[] (one thread per segment), then the warps
// take groups of 32 consecutive elements in turn, each lane issuing the loads of UNROLL elements
// before any of them is used. Trip counts depend on the warp only (lanes stay converged).
// Ends with a block barrier.
constexpr int SEGID_CAP = 2048;

template <typename Load, typename Use>
__device__ __forceinline__ void for_each_element(const int *seg_lo, const int *pre, int nseg, unsigned short *segid,
                                                 const Load &load, Use use) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int E0 = pre[0], E1 = pre[nseg];
    for (int c0 = E0; c0 < E1; c0 += SEGID_CAP) {
        const int c1 = min(E1, c0 + SEGID_CAP);
        for (int sg = threadIdx.x; sg < nseg; sg += NT) {
            const int a = max(pre[sg], c0), b = min(pre[sg + 1], c1);
            for (int e = a; e < b; ++e) segid[e - c0] = (unsigned short)sg;
        }
        block_sync();
        // warp w takes the 32-element groups w, w + NWARP, w + 2 NWARP, ..., UNROLL groups per
        // step, so every warp gets a mix of the segment kinds (their per-element work differs)
        const int eb = c1;
        for (int base = c0 + warp * 32; base < eb; base += NWARP * 32 * UNROLL) {
            int sg[UNROLL], ix[UNROLL];
            typename Load::Slot slot[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                const int eu = base + lane + NWARP * 32 * u;
                sg[u] = -1;
                ix[u] = 0;
                if (eu < eb) {
                    const int sgu = segid[eu - c0];
                    sg[u] = sgu;
                    ix[u] = seg_lo[sgu] + (eu - pre[sgu]);
                    load(sgu, ix[u], slot[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < UNROLL; ++u)
                if (sg[u] >= 0) use(sg[u], ix[u], slot[u]);
        }
        block_sync();
    }
}

}  // namespace dev
}  // namespace aprk
