// Multi-channel APR convolution with bfloat16 features and weights on the fifth-generation tensor
// cores (tcgen05), FP32 accumulation: the per-level filters of an APR CNN layer (Sec. 6), with the
// isotropic patch of Sec. 3.5 and the per-level convolution of Sec. 4.1 applied per channel pair.
//
// Work decomposition: every convolution work item (an 8 x 8-row, 64-cell tile of one level) is cut
// into four 4 x 4-row sub-tiles; a CTA takes several consecutive sub-tiles of one item. For each it
// stages the patch (radius 1) with 16 channels per cell in shared memory from the segments its tile
// plan lists (built once per APR by build_mc_plans), lists the target cells, and runs the channel
// mixing as GEMMs:
//   forward      D[target][co] += sum_e A_e[target][ci] W_e[ci][co]     (A_e gathered per tap)
//   data adjoint D[row][ci]    += sum_e G(q_row - e)[co] W_e[co][ci]    (one row per pre-image q of a
//                                  destination; each destination sums its rows afterwards)
//   weights      D[(e,ci)][co] += sum_t U[t][(e,ci)] g_t[co]             (U: im2col of the targets)
// The gathered A operand of the first two is written to tensor memory with tcgen05.st (one lane
// per row, 8 columns per tap), B comes from shared memory, D lives in tensor memory. One thread
// issues the MMAs; completion is signalled through an mbarrier whose waits are bounded in time.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <mutex>

#include "apr_device.cuh"
#include "apr_internal.h"

namespace aprk {
namespace {

using namespace dev;

constexpr int MC = 16;                      // channels (c_in = c_out)
constexpr int SZ = 4, SX = 4, SY = BY;      // sub-tile rows (z, x) and cells (y)
constexpr int PZ = SZ + 2, PX = SX + 2, PY = SY + 2;
constexpr int NPROW = PZ * PX;              // patch rows
constexpr int NPC = NPROW * PY;             // patch cells
constexpr int NIROW = SZ * SX;              // interior rows
constexpr int MAXT = NIROW * SY;            // interior cells
constexpr int NSUB_ZX = (TZ / SZ) * (TX / SX);
constexpr int NSUB = NSUB_ZX * (BY / SY);   // sub-tiles per work item: (z, x) quarters, then y halves
constexpr int NWY = (PY + 31) / 32;         // 32-bit words of a patch row's cell mask
constexpr int SPC_F = 4, SPC_B = 2;         // sub-tiles per CTA: forward, data adjoint (measured best)
constexpr int NTAP = 27;
constexpr int WTAP = 512;                   // bytes of one tap's 16 x 16 bf16 weight block
constexpr uint32_t TMEM_COLS = 256;
constexpr uint32_t TM_A = 0;                // A operand: tap e in columns 8e .. 8e+7
constexpr uint32_t TM_D = 224;              // accumulator: 16 columns
constexpr int NSEG_F = 3 * NPROW;           // staging segments of the feature patch
constexpr int NCZM = ((SZ + 1) >> 1) + 2;   // level-(l-1) rows per axis under a patch (even sub-tile origin)
constexpr int WG_T = 16;                    // targets per weight-gradient GEMM step (one K step)
constexpr int WG_MG = 64;                   // M groups of 8 rows allocated (54 used: 27 taps x 2)
constexpr int WG_ROWS = NTAP * MC;          // 432 rows (e, ci) of the weight gradient
static_assert(TZ % SZ == 0 && TX % SX == 0 && BY % SY == 0, "sub-tiles must divide the work-item tile");
static_assert(MAXT % NT == 0, "whole interior cells per thread");
static_assert(NSUB % SPC_F == 0 && NSUB % SPC_B == 0, "whole sub-tile groups per work item");
static_assert(SZ % 2 == 0 && SX % 2 == 0, "sub-tiles must be even-aligned (coarse cells)");
static_assert(TM_A + 8 * NTAP <= TM_D && TM_D + 16 <= TMEM_COLS, "tensor-memory columns");
static_assert(NPC < 65536 && MAXT <= 1024, "16-bit cell ids");
static_assert(SZ == SX && NCZM * NCZM <= NPROW, "once-staged coarser rows fit the kind-2 segments");

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return uint32_t(__cvta_generic_to_shared(p)); }

// Shared-memory matrix descriptor, no swizzle: start address, leading-dimension byte offset (stride
// between core matrices along K) and stride-dimension byte offset (along M or N), version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return uint64_t((addr & 0x3FFFF) >> 4) | (uint64_t((lbo & 0x3FFFF) >> 4) << 16) |
           (uint64_t((sbo & 0x3FFFF) >> 4) << 32) | (uint64_t(1) << 46);
}

// Instruction descriptor of kind::f16: BF16 A and B, FP32 D, M x N, A/B K-major unless *_mn.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool a_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (a_mn ? (1u << 15) : 0u) | ((uint32_t(N) >> 3) << 17) |
           ((uint32_t(M) >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of the mbarrier; gives up after limit_ns nanoseconds (default one second)
// or 2^24 polls, whichever comes first.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns = 1000000000ull) {
    const uint32_t a = smem_u32(bar);
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 0; it < (1u << 24); ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (globaltimer() - t0 > limit_ns) return false;
    }
    return false;
}

// D (tensor memory) [+]= A (tensor memory) x B (shared memory descriptor)
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(d),
                 "r"(a), "l"(bdesc), "r"(idesc), "r"(acc)
                 : "memory");
}
// D (tensor memory) [+]= A (shared memory descriptor) x B (shared memory descriptor)
__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
                 "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
                 : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint4 &a, const uint4 &b) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr), "r"(a.x),
                 "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w)
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void red_add_v4(float *p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

// Bounded-wait outcome shared by the block: on a timeout every thread leaves through the same path;
// thread 0 records the error and waits once more (bounded) for the MMAs in flight.
__device__ __forceinline__ bool block_timed_out(bool ok, uint64_t *bar, uint32_t parity, unsigned *err) {
    const bool bad = __syncthreads_or(!ok) != 0;
    if (bad && threadIdx.x == 0) {
        atomicOr(err, ERR_TIMEOUT);
        mbar_wait(bar, parity);
    }
    return bad;
}

// Completion of the MMAs committed to `bar`: thread 0 (the issuing thread) waits on the mbarrier,
// the others at the block barrier that shares the outcome (so they spend no issue slots polling);
// tcgen05.fence::after_thread_sync after it orders their tensor-memory reads. True on a timeout.
__device__ __forceinline__ bool block_wait_mma(uint64_t *bar, uint32_t parity, unsigned *err) {
    const bool ok = threadIdx.x == 0 ? mbar_wait(bar, parity) : true;
    return block_timed_out(ok, bar, parity, err);
}

// Self-test of the bounded-wait path: one block waits on an mbarrier that nothing arrives at, gives up
// after limit_ns and records ERR_TIMEOUT, exactly as the tensor-core kernels do when their MMAs do
// not complete. Nothing faults; the context stays usable.
__global__ void bounded_wait_selftest_kernel(uint64_t limit_ns, unsigned *err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar);
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0, limit_ns);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(err, ERR_TIMEOUT);
}

// ---------------------------------------------------------------- geometry
__device__ __forceinline__ int tap_off(int e) {  // patch-cell offset of tap e = ((dz+1)*3 + dx+1)*3 + dy+1
    return (e / 9 - 1) * (PX * PY) + ((e / 3) % 3 - 1) * PY + (e % 3 - 1);
}

// A operand rows of taps E0 .. E1-1 (columns TM_A + 8e) for one row: the patch cells at
// (pz, px, py) + S_ * (tap offset), both 16-byte halves, zero outside the patch or for an invalid row
// (a warp-collective store, so every lane calls it). The tap offsets are compile-time constants;
// only rows on the patch edge test them against the patch.
template <int E0, int E1, int S_>
__device__ __forceinline__ void store_taps(const uint4 *p0, const uint4 *p1, int pz, int px, int py, bool valid,
                                           uint32_t taddr) {
    const bool inner = valid && pz >= 1 && pz <= PZ - 2 && px >= 1 && px <= PX - 2 && py >= 1 && py <= PY - 2;
    const int cell = (pz * PX + px) * PY + py;
#pragma unroll
    for (int e = E0; e < E1; ++e) {
        const int dz = S_ * (e / 9 - 1), dx = S_ * ((e / 3) % 3 - 1), dy = S_ * (e % 3 - 1);
        uint4 a = make_uint4(0, 0, 0, 0), b = a;
        if (inner || (valid && unsigned(pz + dz) < unsigned(PZ) && unsigned(px + dx) < unsigned(PX) &&
                      unsigned(py + dy) < unsigned(PY))) {
            const int c = cell + (dz * PX + dx) * PY + dy;
            a = p0[c];
            b = p1[c];
        }
        tmem_st8(taddr + TM_A + 8 * e, a, b);
    }
}

struct Sub {         // a sub-tile: level, interior origin, level grids
    int l, z0, x0, y0, yb;
    LevelGeo g, gc;  // level l and level l-1 (gc valid if l > l_min)
};

__host__ __device__ __forceinline__ bool sub_of(const DevLayout &L, const Item &it, int sub, Sub &s) {
    s.l = it.l;
    s.g = L.geo[it.l];
    s.gc = it.l > L.l_min ? L.geo[it.l - 1] : s.g;
    const int zx = sub % NSUB_ZX;
    s.z0 = it.a * TZ + (zx / (TX / SX)) * SZ;
    s.x0 = it.b * TX + (zx % (TX / SX)) * SX;
    s.yb = it.yb;
    s.y0 = it.yb * BY + (sub / NSUB_ZX) * SY;
    return s.z0 < s.g.dz && s.x0 < s.g.dx && s.y0 < s.g.dy;
}

// Patch row pr = (iz, ix) covers level cells (z0-1+iz, x0-1+ix). 0: never read, 1: staged from the
// (reflected) source row, 2: zero (outside the grid with zero boundary).
__host__ __device__ __forceinline__ int row_mode(const Sub &s, int pr, int bc, int &rz, int &rx) {
    const int z = s.z0 - 1 + pr / PX, x = s.x0 - 1 + pr % PX;
    if (z > s.g.dz || x > s.g.dx) return 0;
    const bool out = z < 0 || z >= s.g.dz || x < 0 || x >= s.g.dx;
    if (out && bc == APR_BC_ZERO) return 2;
    rz = reflect_idx(z, s.g.dz);
    rx = reflect_idx(x, s.g.dx);
    return 1;
}

// ---------------------------------------------------------------- feature patch staging
struct McSlot {
    int y;
    uint4 a, b;
};

// Loads y and the two 16-byte halves of element i of plan entry sg (segment og = meta & MC_SEG;
// tree segments: [NPROW, 2 NPROW)).
constexpr int MC_SEG = 255;           // plan meta: segment index; bit 8 = the patch row is outside the grid
constexpr int MC_REFL = 256;
struct FeatLoader {
    using Slot = McSlot;
    const uint16_t *py, *ty;
    const uint4 *pv, *tv;
    const unsigned short *meta;
    __device__ __forceinline__ void operator()(int sg, int i, Slot &sl) const {
        const int og = meta[sg] & MC_SEG;
        const bool t = og >= NPROW && og < 2 * NPROW;
        sl.y = t ? int(ty[i]) : int(py[i]);
        const uint4 *v = t ? tv : pv;
        sl.a = v[2 * size_t(i)];
        sl.b = v[2 * size_t(i) + 1];
    }
};

struct FeatStage {
    uint4 p0[NPC];  // channels 0-7 of every patch cell
    uint4 p1[NPC];  // channels 8-15
    int seg_lo[NSEG_F];
    int pre[NSEG_F + 1];
    unsigned short smeta[NSEG_F];  // plan meta of every entry
    int warp_tot[NWARP + 1];
    unsigned short segid[SEGID_CAP];
};

// Staging of the feature patch with u_l (Sec. 3.5) for the cells the sub-tile's targets read:
// level-l particles, level-l tree nodes and level-(l-1) particles (each covering two cells per
// axis), reflected or zero outside the grid. Segment s = kind * NPROW + patch row. All patch rows
// inside the grid: every coarser row is staged once (kind-2 segments then index the NCZM x NCZM
// level-(l-1) rows under the patch instead of the patch rows).
__host__ __device__ __forceinline__ bool sub_inner(const Sub &s) {
    return s.z0 >= 1 && s.x0 >= 1 && s.z0 + SZ + 1 <= s.g.dz && s.x0 + SX + 1 <= s.g.dx;
}

// Feature segment sg of sub-tile s with the reflecting boundary: index range [lo, hi) of one row's
// elements; refl: the patch row lies outside the grid (with zero boundary the segment is empty).
__host__ __device__ inline void feat_segment(const DevLayout &L, const Sub &s, int sg, int &lo, int &hi, bool &refl) {
    const int ylo = s.y0 - 1;
    const int ya = imax(ylo, 0), yb = imin(s.y0 + SY + 1, s.g.dy);
    const bool has_tree = s.l < L.l_max, has_coarse = s.l > L.l_min;
    const int kind = sg / NPROW, pr = sg - kind * NPROW;
    lo = 0;
    hi = 0;
    refl = false;
    if (kind == 2 && sub_inner(s)) {
        // a level-(l-1) row staged once for the (up to) 2 x 2 patch rows it covers
        if (pr < NCZM * NCZM && has_coarse) {
            const int cz = ((s.z0 - 1) >> 1) + pr / NCZM, cx = ((s.x0 - 1) >> 1) + pr % NCZM;
            const int cya = ya >> 1, cyb = imin((yb + 1) >> 1, s.gc.dy);
            if (cz < s.gc.dz && cx < s.gc.dx)
                row_range(L.row_ptr, L.off, s.gc.row0, s.gc.off0, s.gc.nb, cz * s.gc.dx + cx, cya, cyb, lo, hi);
        }
        return;
    }
    int rz = 0, rx = 0;
    if (row_mode(s, pr, APR_BC_REFLECT, rz, rx) != 1) return;
    const int z = s.z0 - 1 + pr / PX, x = s.x0 - 1 + pr % PX;
    refl = z < 0 || z >= s.g.dz || x < 0 || x >= s.g.dx;
    if (kind == 0) {
        row_range(L.row_ptr, L.off, s.g.row0, s.g.off0, s.g.nb, rz * s.g.dx + rx, ya, yb, lo, hi);
    } else if (kind == 1 && has_tree) {
        row_range(L.trow_ptr, L.toff, s.g.trow0, s.g.toff0, s.g.nb, rz * s.g.dx + rx, ya, yb, lo, hi);
    } else if (kind == 2 && has_coarse) {
        const int cya = ya >> 1, cyb = imin((yb + 1) >> 1, s.gc.dy);
        row_range(L.row_ptr, L.off, s.gc.row0, s.gc.off0, s.gc.nb, (rz >> 1) * s.gc.dx + (rx >> 1), cya, cyb, lo, hi);
    }
}

// Reads a sub-tile's plan (entries taken by threads t0, t0 + 1, ...; threads below t0 are free for
// other loads) into seg_lo / smeta / pre and returns the entry count. drop_refl (zero boundary on a
// sub-tile with rows outside the grid): the entries flagged MC_REFL are emptied and the counts
// rescanned by all threads. Ends with a block barrier.
__device__ __forceinline__ int load_mc_plan(const PlanView &P, int tile, int t0, bool drop_refl, int *seg_lo,
                                            unsigned short *smeta, int *pre, int *warp_tot) {
    const int tid = threadIdx.x;
    const PlanHdr hd = P.hdr[tile];
    const int n = hd.count;
    if (tid >= t0)
        for (int k = tid - t0; k <= n; k += NT - t0) {
            const PlanEnt e = P.ent[hd.first + k];
            if (k < n) {
                seg_lo[k] = e.lo;
                smeta[k] = e.meta;
            }
            if (!drop_refl) pre[k] = e.pre;
        }
    if (!drop_refl) {
        block_sync();
        return n;
    }
    int cnt[2] = {0, 0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k = 2 * tid + h;
        if (k < n) {
            const PlanEnt e = P.ent[hd.first + k];
            if (!(e.meta & MC_REFL)) cnt[h] = int(P.ent[hd.first + k + 1].pre) - int(e.pre);
        }
    }
    block_scan2(cnt[0], cnt[1], n, pre, warp_tot);
    return n;
}

// Target list of the sub-tile: the level-l particles of its interior, in particle order.
struct Targets {
    int idx[MAXT];
    unsigned short cell[MAXT];
    int row_lo[NIROW], row_base[NIROW + 1];
};

// Element loads and patch writes for the nseg plan entries in S (after load_mc_plan); ends with a
// block barrier. T (optional, its row offsets set): the targets (level-l particles of the in-grid
// interior rows with y in [y0, y0 + SY), all among the staged elements) are listed as they pass,
// target j of row r at T->row_base[r] + j.
__device__ void feature_elements(const DevLayout &L, const Sub &s, const uint4 *vals, const uint4 *tree, int bc,
                                 int nseg, FeatStage &S, Targets *T = nullptr) {
    const int tid = threadIdx.x;
    const int ylo = s.y0 - 1;
    const int ya = max(ylo, 0), yb = min(s.y0 + SY + 1, s.g.dy);
    const bool inner = sub_inner(s);
    const FeatLoader loader{L.y, L.ty, vals, tree, S.smeta};
    for_each_element(S.seg_lo, S.pre, nseg, S.segid, loader, [&](int sg, int i, const McSlot &sl) {
        const int og = S.smeta[sg] & MC_SEG;
        const int kind = og / NPROW, pr = og - kind * NPROW;
        if (kind < 2) {
            if (sl.y >= ya && sl.y < yb) {
                const int c = pr * PY + sl.y - ylo;
                S.p0[c] = sl.a;
                S.p1[c] = sl.b;
                if (T && kind == 0 && sl.y >= s.y0 && sl.y < s.y0 + SY) {
                    const int iz = pr / PX - 1, ix = pr % PX - 1;
                    if (unsigned(iz) < unsigned(SZ) && unsigned(ix) < unsigned(SX) && s.z0 + iz < s.g.dz &&
                        s.x0 + ix < s.g.dx) {
                        const int r = iz * SX + ix, slot = T->row_base[r] + (i - T->row_lo[r]);
                        T->idx[slot] = i;
                        T->cell[slot] = (unsigned short)c;
                    }
                }
            }
        } else if (!inner) {
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const int y = 2 * sl.y + f;
                if (y >= ya && y < yb) {
                    const int c = pr * PY + y - ylo;
                    S.p0[c] = sl.a;
                    S.p1[c] = sl.b;
                }
            }
        } else {
            const int rz0 = 2 * (((s.z0 - 1) >> 1) + pr / NCZM) - (s.z0 - 1);
            const int rx0 = 2 * (((s.x0 - 1) >> 1) + pr % NCZM) - (s.x0 - 1);
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const int y = 2 * sl.y + f;
                if (y < ya || y >= yb) continue;
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int b = 0; b < 2; ++b) {
                        const int pz = rz0 + a, px = rx0 + b;
                        if (pz < 0 || pz >= PZ || px < 0 || px >= PX) continue;
                        const int c = (pz * PX + px) * PY + y - ylo;
                        S.p0[c] = sl.a;
                        S.p1[c] = sl.b;
                    }
            }
        }
    });
    // cells outside the grid (none when the patch lies inside it): the cells y = -1 and y = dy of each
    // staged row mirror y = 0 and y = dy - 1 (zero with the zero boundary), and with the zero boundary
    // the rows outside the grid are zero
    const uint4 z4 = make_uint4(0, 0, 0, 0);
    if (!inner || ylo < 0 || s.y0 + SY >= s.g.dy) {
        for (int t = tid; t < 2 * NPROW; t += NT) {
            const int pr = t >> 1, y = (t & 1) ? s.g.dy : -1, py = y - ylo;
            int rz, rx;
            if (py < 0 || py >= PY || row_mode(s, pr, bc, rz, rx) != 1) continue;
            const int i = pr * PY + py;
            if (bc == APR_BC_ZERO) {
                S.p0[i] = z4;
                S.p1[i] = z4;
            } else {
                const int src = pr * PY + reflect_idx(y, s.g.dy) - ylo;  // y = -1 -> 0, y = dy -> dy-1
                S.p0[i] = S.p0[src];
                S.p1[i] = S.p1[src];
            }
        }
        if (bc == APR_BC_ZERO && !inner)
            for (int i = tid; i < NPROW * PY; i += NT) {
                int rz, rx;
                if (row_mode(s, i / PY, bc, rz, rx) == 2) {
                    S.p0[i] = z4;
                    S.p1[i] = z4;
                }
            }
    }
    block_sync();
}

// The whole staging of sub-tile `tile` (index into the feature plan: item * NSUB + sub).
__device__ void stage_features(const DevLayout &L, const Sub &s, int tile, const uint4 *vals, const uint4 *tree,
                               int bc, FeatStage &S, Targets *T = nullptr) {
    const int n = load_mc_plan(L.mcfplan, tile, 0, bc != APR_BC_REFLECT && !sub_inner(s), S.seg_lo, S.smeta, S.pre,
                               S.warp_tot);
    feature_elements(L, s, vals, tree, bc, n, S, T);
}

// Row offsets of the targets (warp 0; no barrier): the sub-tile spans whole y-blocks, so the block
// offsets give each interior row's level-l particles exactly.
__device__ __forceinline__ void target_rows(const DevLayout &L, const Sub &s, Targets &T) {
    static_assert(SY == BY, "sub-tiles span one y-block");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        int lo = 0, cnt = 0;
        if (lane < NIROW) {
            const int z = s.z0 + lane / SX, x = s.x0 + lane % SX;
            if (z < s.g.dz && x < s.g.dx) {
                const int rr = z * s.g.dx + x;
                lo = int(pblock(L, s.g, rr, s.yb));
                cnt = int(pblock(L, s.g, rr, s.yb + 1)) - lo;
            }
        }
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane < NIROW) {
            T.row_lo[lane] = lo;
            T.row_base[lane] = incl - cnt;
        }
        if (lane == NIROW - 1) T.row_base[NIROW] = incl;
    }
}

// Particle index of target j from the row offsets alone (before the list is filled).
__device__ __forceinline__ int target_index(const Targets &T, int j) {
    int r = 0;
#pragma unroll
    for (int k = 1; k < NIROW; ++k) r = T.row_base[k] <= j ? k : r;
    return T.row_lo[r] + (j - T.row_base[r]);
}

// Row offsets of the targets; returns their count (ends with a barrier).
__device__ int count_targets(const DevLayout &L, const Sub &s, Targets &T) {
    target_rows(L, s, T);
    block_sync();
    return T.row_base[NIROW];
}

// Weights of every level in the B-operand layout of each tap e: K-major core matrices of 8 rows x 16
// bytes, N-row group g and K chunk k at (2g + k) * 128 bytes (LBO 128, SBO 256). transpose = 0:
// N = co, K = ci (forward); transpose = 1: N = ci, K = co (data adjoint). One thread per destination
// element of out[lev][e * 256 + ...], read from W[lev][co][ci][e].
__global__ void mc_weight_layout_kernel(const uint16_t *__restrict__ W, int n_levels, int transpose,
                                        uint16_t *__restrict__ out) {
    constexpr int PER = MC * MC * NTAP;
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < n_levels * PER; d += gridDim.x * blockDim.x) {
        const int lev = d / PER, r = d % PER;
        const int e = r / (MC * MC), q = r % (MC * MC);
        const int cm = q / 64, row = (q % 64) / 8, col = q % 8;
        const int n = (cm >> 1) * 8 + row, k = (cm & 1) * 8 + col;
        const int co = transpose ? k : n, ci = transpose ? n : k;
        out[d] = W[((size_t(lev) * MC + co) * MC + ci) * NTAP + e];
    }
}

// One level's operand-layout weights (13 824 contiguous bytes) into shared memory, in two halves: the
// loads into registers (four 16-byte words per thread) early, the stores into shared memory later,
// so the loads' latency overlaps other work.
constexpr int WV = NTAP * WTAP / 16;  // 16-byte words of one level's weights
static_assert(WV <= 4 * NT, "four weight words per thread");

__device__ __forceinline__ void preload_weights(const uint16_t *wl, int lev, uint4 (&w)[4]) {
    const uint4 *src = reinterpret_cast<const uint4 *>(wl + size_t(lev) * MC * MC * NTAP);
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (threadIdx.x + k * NT < WV) w[k] = src[threadIdx.x + k * NT];
}

__device__ __forceinline__ void store_weights(const uint4 (&w)[4], unsigned char *wsm) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (threadIdx.x + k * NT < WV) reinterpret_cast<uint4 *>(wsm)[threadIdx.x + k * NT] = w[k];
    fence_async_smem();
}

// ---------------------------------------------------------------- BF16 tree restriction
// One level of the tree restriction for 16 bf16 channels, one thread per (tree node, 8-channel half):
// the node's children from its child map (TreeNodePlan, apr_internal.h), summed in FP32 in (a, b, e)
// order, divided by their count in FP32, rounded to bf16 (round to nearest even).
__global__ void __launch_bounds__(NT) mc_tree_restrict_kernel(const TreeNodePlan *__restrict__ nplan, int node0, int n,
                                                              const uint4 *__restrict__ vals, uint4 *tree) {
    pdl_trigger();
    const int q = int(blockIdx.x) * NT + int(threadIdx.x);
    const int i = q >> 1, half = q & 1;
    const bool live = i < n;
    // the child map is static: read before waiting for the finer level's restriction (the launch
    // before this one), whose node values this level reads
    int4 pw = make_int4(0, 0, 0, 0), tw = pw;
    if (live) {
        const int4 *m = reinterpret_cast<const int4 *>(nplan + node0 + i);
        pw = __ldg(m);
        tw = __ldg(m + 1);
    }
    pdl_wait();
    if (!live) return;
    const int pv[4] = {pw.x, pw.y, pw.z, pw.w}, tv[4] = {tw.x, tw.y, tw.z, tw.w};
    uint4 h[8];
    bool has[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const unsigned pm = unsigned(pv[k]) >> 30, tm = unsigned(tv[k]) >> 30;
        const int pi = int(unsigned(pv[k]) & TNP_INDEX), ti = int(unsigned(tv[k]) & TNP_INDEX);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            // the second child of a kind follows the first of that kind
            const bool isp = (pm >> e) & 1u, ist = (tm >> e) & 1u;
            const int ix = isp ? pi + (e ? int(pm & 1u) : 0) : ti + (e ? int(tm & 1u) : 0);
            has[2 * k + e] = isp || ist;
            h[2 * k + e] = isp ? vals[2 * size_t(ix) + half] : (ist ? tree[2 * size_t(ix) + half] : make_uint4(0u, 0u, 0u, 0u));
        }
    }
    float acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = 0.0f;
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (!has[k]) continue;
        ++cnt;
        const __nv_bfloat162 *p = reinterpret_cast<const __nv_bfloat162 *>(&h[k]);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float2 f = __bfloat1622float2(p[c]);
            acc[2 * c] = __fadd_rn(acc[2 * c], f.x);
            acc[2 * c + 1] = __fadd_rn(acc[2 * c + 1], f.y);
        }
    }
    const float nf = float(cnt ? cnt : 1);
    uint4 o;
    __nv_bfloat162 *r = reinterpret_cast<__nv_bfloat162 *>(&o);
#pragma unroll
    for (int c = 0; c < 4; ++c) r[c] = __floats2bfloat162_rn(__fdiv_rn(acc[2 * c], nf), __fdiv_rn(acc[2 * c + 1], nf));
    tree[2 * size_t(node0 + i) + half] = o;
}

// Transpose of the tree restriction for 16 FP32 gradient channels, one level (coarse to fine), one
// thread per (tree node, 4-channel group): every child (particle or tree node of level l+1) gets its
// parent's gradient / #children added. Every child has one parent, so each is written by one thread.
__global__ void __launch_bounds__(NT) mc_tree_pushdown_kernel(const TreeNodePlan *__restrict__ nplan, int node0, int n,
                                                              float4 *gp, float4 *gt) {
    pdl_trigger();
    const int q = int(blockIdx.x) * NT + int(threadIdx.x);
    const int i = q >> 2, cg = q & 3;
    const bool live = i < n;
    // the child map is static: read before waiting for the coarser level's push-down (the launch
    // before this one), which writes this level's gradients
    int4 pw = make_int4(0, 0, 0, 0), tw = pw;
    if (live) {
        const int4 *m = reinterpret_cast<const int4 *>(nplan + node0 + i);
        pw = __ldg(m);
        tw = __ldg(m + 1);
    }
    pdl_wait();
    if (!live) return;
    const int pv[4] = {pw.x, pw.y, pw.z, pw.w}, tv[4] = {tw.x, tw.y, tw.z, tw.w};
    float4 *dst[8];
    float4 v[8];
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const unsigned pm = unsigned(pv[k]) >> 30, tm = unsigned(tv[k]) >> 30;
        const int pi = int(unsigned(pv[k]) & TNP_INDEX), ti = int(unsigned(tv[k]) & TNP_INDEX);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const bool isp = (pm >> e) & 1u, ist = (tm >> e) & 1u;
            const int ix = isp ? pi + (e ? int(pm & 1u) : 0) : ti + (e ? int(tm & 1u) : 0);
            dst[2 * k + e] = isp ? gp + size_t(ix) * (MC / 4) + cg : (ist ? gt + size_t(ix) * (MC / 4) + cg : nullptr);
            cnt += (isp || ist) ? 1 : 0;
        }
    }
    const float4 g = gt[size_t(node0 + i) * (MC / 4) + cg];
    const float f = float(cnt ? cnt : 1);
    const float4 s = make_float4(g.x / f, g.y / f, g.z / f, g.w / f);
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = dst[k] ? *dst[k] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 8; ++k)
        if (dst[k]) *dst[k] = make_float4(v[k].x + s.x, v[k].y + s.y, v[k].z + s.z, v[k].w + s.w);
}

// ---------------------------------------------------------------- forward
struct FwdSmem {
    FeatStage st;
    alignas(16) unsigned char w[NTAP * WTAP];
    Targets tg;
    uint64_t bar;
    uint32_t tmem;
};

// out (float32 [N][16]) receives the convolution; if out_bf16 is given instead, it receives
// bf16(max(conv, 0)), the next layer's input in an APR CNN (the ReLU fused into the write).
// A CTA takes SPC_F consecutive sub-tiles of one work item (one level): the weights, the mbarrier and
// the tensor memory are set up once, at its first sub-tile with targets.
__global__ void __launch_bounds__(NT, 2) mc_fwd_kernel(const DevLayout L, const Item *__restrict__ items,
                                                       const uint4 *__restrict__ vals, const uint4 *__restrict__ tree,
                                                       const uint16_t *__restrict__ W, int bc, float *__restrict__ out,
                                                       uint4 *__restrict__ out_bf16) {
    extern __shared__ __align__(16) unsigned char smraw[];
    FwdSmem &S = *reinterpret_cast<FwdSmem *>(smraw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const Item it = items[blockIdx.x];
    // the level's weights are held in registers until the first patch is staged
    uint4 wreg[4];
    preload_weights(W, it.l - L.l_min, wreg);
    const int q = warp & 3;
    const uint32_t lane_base = uint32_t(32 * q) << 16;
    constexpr uint32_t idesc = idesc_bf16(128, 16, false);
    uint32_t phase = 0, tb = 0;
    bool ready = false, failed = false;  // block-uniform
    for (int k = 0; k < SPC_F && !failed; ++k) {
        const int sub = blockIdx.y * SPC_F + k;
        Sub s;
        if (!sub_of(L, it, sub, s)) continue;
        if (k > 0) block_sync();  // the previous sub-tile's readers of S.tg and S.st are done
        target_rows(L, s, S.tg);  // warp 0, while the other warps read the plan
        const int nseg = load_mc_plan(L.mcfplan, blockIdx.x * NSUB + sub, 32,
                                      bc != APR_BC_REFLECT && !sub_inner(s), S.st.seg_lo, S.st.smeta, S.st.pre,
                                      S.st.warp_tot);
        const int nt = S.tg.row_base[NIROW];
        if (nt == 0) continue;
        feature_elements(L, s, vals, tree, bc, nseg, S.st, &S.tg);
        if (!ready) {
            store_weights(wreg, S.w);
            if (tid == 0) mbar_init(&S.bar);
            if (warp == 0) tmem_alloc(smem_u32(&S.tmem), TMEM_COLS);
            ready = true;
        }
        fence_async_smem();
        tc_fence_before();
        block_sync();
        tc_fence_after();
        tb = S.tmem;
        for (int b0 = 0; b0 < nt; b0 += 128) {
            const int t = b0 + 32 * q + lane;
            const int cell = t < nt ? int(S.tg.cell[t]) : 0;
            const int cz = cell / (PX * PY), cx = (cell / PY) % PX, cy = cell % PY;
            // rows past the last target are never read back: a warp holding only such rows skips them
            if (b0 + 32 * q < nt) {
                if (warp < 4) store_taps<0, 14, 1>(S.st.p0, S.st.p1, cz, cx, cy, t < nt, tb + lane_base);
                else store_taps<14, NTAP, 1>(S.st.p0, S.st.p1, cz, cx, cy, t < nt, tb + lane_base);
            }
            tmem_wait_st();
            tc_fence_before();
            block_sync();
            tc_fence_after();
            if (tid == 0) {
                for (int e = 0; e < NTAP; ++e)
                    mma_ts(tb + TM_D, tb + TM_A + 8 * e, sdesc(smem_u32(S.w + e * WTAP), 128, 256), idesc, e > 0);
                mma_commit(&S.bar);
            }
            if (block_wait_mma(&S.bar, phase, L.err)) {
                failed = true;
                break;
            }
            phase ^= 1;
            tc_fence_after();
            if (warp < 4) {
                float v[16];
                tmem_ld16(tb + lane_base + TM_D, v);
                if (t < nt) {
                    if (out_bf16) {
                        uint4 r[2];
                        __nv_bfloat162 *b2 = reinterpret_cast<__nv_bfloat162 *>(r);
#pragma unroll
                        for (int c = 0; c < MC / 2; ++c) b2[c] = __floats2bfloat162_rn(fmaxf(v[2 * c], 0.f), fmaxf(v[2 * c + 1], 0.f));
                        out_bf16[2 * size_t(S.tg.idx[t])] = r[0];
                        out_bf16[2 * size_t(S.tg.idx[t]) + 1] = r[1];
                    } else {
                        float4 *o = reinterpret_cast<float4 *>(out + size_t(S.tg.idx[t]) * MC);
#pragma unroll
                        for (int c = 0; c < 4; ++c) o[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
                    }
                }
            }
            tc_fence_before();
            block_sync();
            tc_fence_after();
        }
    }
    if (ready) {
        tc_fence_before();
        block_sync();
        if (warp == 0) tmem_dealloc(tb, TMEM_COLS);
    }
}

// ---------------------------------------------------------------- data adjoint
constexpr int NSEG_B = NPROW + 3 * NIROW;  // gradient rows, then interior particle / tree / coarse rows
// Row groups of the data adjoint: a destination with q pre-images that a gradient reaches takes an
// aligned group of rows, one pre-image per row: class 0 (33..64 pre-images, 32 rows, two passes),
// class c = 1..6 (2^(6-c) rows for up to that many pre-images). Classes are laid out in order, so
// every group starts at a multiple of its size and stays inside one warp's 32 rows.
constexpr int NCLS = 7;
__device__ __forceinline__ int group_rows(int c) { return min(32, 64 >> c); }
__device__ __forceinline__ int group_class(int q) { return q > 32 ? 0 : 6 - (q > 1 ? 32 - __clz(q - 1) : 0); }
constexpr unsigned char SRC_NONE = 0xFF, SRC_P = 0, SRC_T = 1, SRC_C = 2;  // source kinds of a patch cell
static_assert(SRC_P == 0 && SRC_T == 1, "interior particle / tree segments store their kind index");

struct BwdSmem {
    uint4 g0[NPC];  // bf16 gradient of the targets, channels 0-7 (zero elsewhere)
    uint4 g1[NPC];
    alignas(16) unsigned char w[NTAP * WTAP];
    int srci[MAXT];                 // source of each interior cell: index ...
    unsigned char srck[MAXT];       // ... and kind (particle, tree, coarse particle)
    unsigned short dorder[MAXT];    // candidate cells, then the destinations grouped by row-group class in slot order
    unsigned tmask[NPROW][NWY];     // cells holding a target, per patch row (bits along y)
    unsigned hot[NPROW][NWY];       // cells within distance 1 of a target
    int seg_lo[NSEG_B];
    int pre[NSEG_B + 1];
    unsigned short smeta[NSEG_B];  // plan meta (segment index) of every entry
    int warp_tot[NWARP + 1];
    unsigned short segid[SEGID_CAP];
    int ccnt[NCLS];                 // destinations per row-group class
    int coff[NCLS + 1];             // first destination (in dorder) of each class
    int rbase[NCLS + 1];            // first row of each class
    uint64_t bar;
    uint32_t tmem;
};

// Segment sg of the data-adjoint sub-tile s: [0, NPROW) the targets of the patch rows (inside the
// grid only; y in the patch window), then per interior row the level-l particles, the level-l tree
// nodes and the level-(l-1) particles over the interior y range.
__host__ __device__ inline void adj_segment(const DevLayout &L, const Sub &s, int sg, int &lo, int &hi) {
    const int ylo = s.y0 - 1;
    const int ya = imax(ylo, 0), yb = imin(s.y0 + SY + 1, s.g.dy);
    const int yia = s.y0, yib = imin(s.y0 + SY, s.g.dy);
    const bool has_tree = s.l < L.l_max, has_coarse = s.l > L.l_min;
    lo = 0;
    hi = 0;
    if (sg < NPROW) {
        const int z = s.z0 - 1 + sg / PX, x = s.x0 - 1 + sg % PX;
        if (z >= 0 && z < s.g.dz && x >= 0 && x < s.g.dx)
            row_range(L.row_ptr, L.off, s.g.row0, s.g.off0, s.g.nb, z * s.g.dx + x, ya, yb, lo, hi);
        return;
    }
    const int k = (sg - NPROW) / NIROW, r = (sg - NPROW) % NIROW;
    const int z = s.z0 + r / SX, x = s.x0 + r % SX;
    if (z >= s.g.dz || x >= s.g.dx) return;
    if (k == 0)
        row_range(L.row_ptr, L.off, s.g.row0, s.g.off0, s.g.nb, z * s.g.dx + x, yia, yib, lo, hi);
    else if (k == 1 && has_tree)
        row_range(L.trow_ptr, L.toff, s.g.trow0, s.g.toff0, s.g.nb, z * s.g.dx + x, yia, yib, lo, hi);
    else if (k == 2 && has_coarse)
        row_range(L.row_ptr, L.off, s.gc.row0, s.gc.off0, s.gc.nb, (z >> 1) * s.gc.dx + (x >> 1), yia >> 1,
                  imin((yib + 1) >> 1, s.gc.dy), lo, hi);
}

__device__ __forceinline__ bool hot_at(const BwdSmem &S, int pz, int px, int py) {
    return (S.hot[pz * PX + px][py >> 5] >> (py & 31)) & 1u;
}

// Pre-images along one axis of a destination whose first fine coordinate is u: its in-grid fine
// cells (one, or two for a coarse particle) and the out-of-grid cells that reflect onto them, as
// patch coordinates (position - base, base = the patch's first position) packed 8 bits each into
// *w (registers, no local array). Returns the count (at most 4).
__device__ __forceinline__ int axis_pre(int u, bool coarse, int d, bool reflect, int base, uint32_t *w) {
    uint32_t v = uint32_t(u - base);
    int n = 1;
    if (coarse && u + 1 < d) v |= uint32_t(u + 1 - base) << (8 * n++);
    if (reflect) {
        if (u == 0) v |= uint32_t(-1 - base) << (8 * n++);
        if ((coarse ? min(u + 1, d - 1) : u) == d - 1) v |= uint32_t(d - base) << (8 * n++);
    }
    *w = v;
    return n;
}
__device__ __forceinline__ int pre_at(uint32_t w, int a) { return int((w >> (8 * a)) & 255u); }

__global__ void __launch_bounds__(NT, 2) mc_bwd_data_kernel(const DevLayout L, const Item *__restrict__ items,
                                                            const uint16_t *__restrict__ W, int bc,
                                                            const uint4 *__restrict__ gout, float *__restrict__ gp,
                                                            float *__restrict__ gt) {
    extern __shared__ __align__(16) unsigned char smraw[];
    BwdSmem &S = *reinterpret_cast<BwdSmem *>(smraw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const Item it = items[blockIdx.x];
    // the level's (transposed) weights are loaded now and held in registers until the first
    // destination list is known, so their latency overlaps the staging
    uint4 wreg[4];
    preload_weights(W, it.l - L.l_min, wreg);
    const bool reflect = bc == APR_BC_REFLECT;
    const int q = warp & 3;
    const uint32_t lane_base = uint32_t(32 * q) << 16;
    constexpr uint32_t idesc = idesc_bf16(128, 16, false);
    uint32_t phase = 0, tb = 0;
    bool ready = false, stop = false;  // block-uniform
    // SPC_B consecutive sub-tiles of the work item; the weights, the mbarrier and the tensor memory
    // are set up once, at the first sub-tile with destinations
    for (int kk = 0; kk < SPC_B && !stop; ++kk) {
        const int sub = blockIdx.y * SPC_B + kk;
        Sub s;
        if (!sub_of(L, it, sub, s)) continue;
        if (kk > 0) block_sync();  // the previous sub-tile's readers of the shared tables are done
        const int ylo = s.y0 - 1;
        const int ya = max(ylo, 0), yb = min(s.y0 + SY + 1, s.g.dy);  // gradient rows: y range of the patch
        const int yia = s.y0, yib = min(s.y0 + SY, s.g.dy);            // interior y range
        const uint4 z4 = make_uint4(0, 0, 0, 0);
        for (int i = tid; i < NPC; i += NT) {
            S.g0[i] = z4;
            S.g1[i] = z4;
        }
        for (int i = tid; i < MAXT; i += NT) S.srck[i] = SRC_NONE;
        for (int i = tid; i < NPROW * NWY; i += NT) (&S.tmask[0][0])[i] = 0;
        const int nseg = load_mc_plan(L.mcbplan, blockIdx.x * NSUB + sub, 0, false, S.seg_lo, S.smeta, S.pre,
                                      S.warp_tot);

        struct Loader {
            using Slot = McSlot;
            const DevLayout *L;
            const uint4 *gout;
            const unsigned short *meta;
            __device__ void operator()(int k, int i, Slot &sl) const {
                const int sg = meta[k];
                const bool t = sg >= NPROW + NIROW && sg < NPROW + 2 * NIROW;
                sl.y = t ? int(L->ty[i]) : int(L->y[i]);
                if (sg < NPROW) {
                    sl.a = gout[2 * size_t(i)];
                    sl.b = gout[2 * size_t(i) + 1];
                }
            }
        } loader{&L, gout, S.smeta};
        for_each_element(S.seg_lo, S.pre, nseg, S.segid, loader, [&](int ent, int i, const McSlot &sl) {
            const int sg = S.smeta[ent];
            if (sg < NPROW) {
                if (sl.y >= ya && sl.y < yb) {
                    const int py = sl.y - ylo;
                    S.g0[sg * PY + py] = sl.a;
                    S.g1[sg * PY + py] = sl.b;
                    atomicOr(&S.tmask[sg][py >> 5], 1u << (py & 31));
                }
                return;
            }
            const int k = (sg - NPROW) / NIROW, r = (sg - NPROW) % NIROW;
            if (k < 2) {
                if (sl.y >= yia && sl.y < yib) {
                    S.srck[r * SY + sl.y - s.y0] = (unsigned char)k;
                    S.srci[r * SY + sl.y - s.y0] = i;
                }
            } else {
#pragma unroll
                for (int f = 0; f < 2; ++f) {
                    const int y = 2 * sl.y + f;
                    if (y >= yia && y < yib) {
                        S.srck[r * SY + y - s.y0] = SRC_C;
                        S.srci[r * SY + y - s.y0] = i;
                    }
                }
            }
        });
        // cells within distance 1 of a target: y dilation of each row, OR over the 3 x 3 neighbour rows
        if (tid < NPROW) {
            const int pz = tid / PX, px = tid % PX;
            unsigned h[NWY] = {};
            for (int dz = -1; dz <= 1; ++dz)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int qz = pz + dz, qx = px + dx;
                    if (qz < 0 || qz >= PZ || qx < 0 || qx >= PX) continue;
                    const unsigned *m = S.tmask[qz * PX + qx];
#pragma unroll
                    for (int w = 0; w < NWY; ++w)
                        h[w] |= m[w] | (m[w] << 1) | (m[w] >> 1) | (w + 1 < NWY ? m[w + 1] << 31 : 0u) |
                                (w > 0 ? m[w - 1] >> 31 : 0u);
                }
#pragma unroll
            for (int w = 0; w < NWY; ++w) S.hot[tid][w] = h[w];
        }
        block_sync();
        // destinations: every particle / tree node of the interior, and every coarse particle (anchored
        // at its first fine cell), with q > 0 pre-images within distance 1 of a target (the others add
        // exact zeros). Each takes a slot in its row-group class. First the candidates (interior cells
        // holding a particle, a tree node or a coarse particle's first cell) are listed in cell order
        // (warp w: cells [w CPT 32, (w + 1) CPT 32)), in dorder's space; an uncovered cell next to a
        // target means an invalid layout.
        constexpr int CPT = MAXT / NT;  // interior cells per thread
        if (tid < NCLS) S.ccnt[tid] = 0;
        unsigned bal[CPT];
        int wcnt = 0;
#pragma unroll
        for (int u = 0; u < CPT; ++u) {
            const int ic = (warp * CPT + u) * 32 + lane;
            const int r = ic / SY, iy = ic % SY;
            const int z = s.z0 + r / SX, x = s.x0 + r % SX, y = s.y0 + iy;
            bool cand = false;
            if (z < s.g.dz && x < s.g.dx && y < s.g.dy) {
                const int k = S.srck[ic];
                if (k == SRC_NONE) {
                    if (hot_at(S, r / SX + 1, r % SX + 1, iy + 1)) atomicOr(L.err, ERR_DEVICE_CHECK);
                } else {
                    cand = k != SRC_C || !((z | x | y) & 1);
                }
            }
            bal[u] = __ballot_sync(0xffffffffu, cand);
            wcnt += __popc(bal[u]);
        }
        if (lane == 0) S.warp_tot[warp] = wcnt;
        block_sync();
        int ncand = 0, cbase = 0;
#pragma unroll
        for (int w = 0; w < NWARP; ++w) {
            cbase += w < warp ? S.warp_tot[w] : 0;
            ncand += S.warp_tot[w];
        }
        const unsigned below = (1u << lane) - 1u;
#pragma unroll
        for (int u = 0; u < CPT; ++u) {
            if ((bal[u] >> lane) & 1u) S.dorder[cbase + __popc(bal[u] & below)] = (unsigned short)((warp * CPT + u) * 32 + lane);
            cbase += __popc(bal[u]);
        }
        block_sync();
        // class of candidate cell ic as a destination (-1: no pre-image within reach of a target)
        auto dest_class = [&](int ic) -> int {
            const int r = ic / SY, iy = ic % SY;
            const int z = s.z0 + r / SX, x = s.x0 + r % SX, y = s.y0 + iy;
            const bool coarse = S.srck[ic] == SRC_C;
            uint32_t wz, wx, wy;
            const int nz = axis_pre(z, coarse, s.g.dz, reflect, s.z0 - 1, &wz);
            const int nx = axis_pre(x, coarse, s.g.dx, reflect, s.x0 - 1, &wx);
            const int ny = axis_pre(y, coarse, s.g.dy, reflect, ylo, &wy);
            int q = 0;
            for (int a = 0; a < nz; ++a)
                for (int b = 0; b < nx; ++b)
                    for (int c = 0; c < ny; ++c) q += hot_at(S, pre_at(wz, a), pre_at(wx, b), pre_at(wy, c));
            return q == 0 ? -1 : group_class(q);
        };
        int my_ic[CPT], my_c[CPT], my_slot[CPT];
#pragma unroll
        for (int u = 0; u < CPT; ++u) {
            const int jc = tid + u * NT;
            my_ic[u] = 0;
            my_c[u] = -1;
            my_slot[u] = 0;
            if (jc < ncand) {
                my_ic[u] = S.dorder[jc];
                my_c[u] = dest_class(my_ic[u]);
                if (my_c[u] >= 0) my_slot[u] = atomicAdd(&S.ccnt[my_c[u]], 1);
            }
        }
        block_sync();
        if (tid == 0) {
            int d = 0, rw = 0;
            for (int c = 0; c < NCLS; ++c) {
                S.coff[c] = d;
                S.rbase[c] = rw;
                d += S.ccnt[c];
                rw += S.ccnt[c] * group_rows(c);
            }
            S.coff[NCLS] = d;
            S.rbase[NCLS] = rw;
        }
        block_sync();
#pragma unroll
        for (int u = 0; u < CPT; ++u)
            if (my_c[u] >= 0) S.dorder[S.coff[my_c[u]] + my_slot[u]] = (unsigned short)my_ic[u];
        const int nrows = S.rbase[NCLS], rows2 = S.rbase[1];  // rows2: the two-pass rows come first
        if (nrows == 0) continue;
        if (!ready) {
            store_weights(wreg, S.w);
            if (tid == 0) mbar_init(&S.bar);
            if (warp == 0) tmem_alloc(smem_u32(&S.tmem), TMEM_COLS);
            ready = true;
        }
        fence_async_smem();
        tc_fence_before();
        block_sync();
        tc_fence_after();
        tb = S.tmem;
        for (int b0 = 0; b0 < nrows; b0 += 128) {
            // this thread's row: destination ic, its j-th pre-image (j + 32 in the second pass)
            const int row = b0 + 32 * q + lane;
            int ic = -1, j = 0, gr = 0;
            if (row < nrows) {
                int c = 0;
                while (row >= S.rbase[c + 1]) ++c;
                gr = group_rows(c);
                const int off = row - S.rbase[c];
                ic = S.dorder[S.coff[c] + off / gr];
                j = off % gr;
            }
            uint32_t wz = 0, wx = 0, wy = 0;
            int nz = 0, nx = 0, ny = 0;
            if (ic >= 0) {
                const int r = ic / SY;
                const bool coarse = S.srck[ic] == SRC_C;
                nz = axis_pre(s.z0 + r / SX, coarse, s.g.dz, reflect, s.z0 - 1, &wz);
                nx = axis_pre(s.x0 + r % SX, coarse, s.g.dx, reflect, s.x0 - 1, &wx);
                ny = axis_pre(s.y0 + ic % SY, coarse, s.g.dy, reflect, ylo, &wy);
            }
            const int npass = b0 < rows2 ? 2 : 1;
            bool failed = false;
            for (int pass = 0; pass < npass; ++pass) {
                // the (j + 32 pass)-th pre-image within distance 1 of a target, in (z, x, y) order
                int pz = -100, px = 0, py = 0, want = j + 32 * pass;
                for (int a = 0; a < nz && pz < -1; ++a)
                    for (int bb = 0; bb < nx && pz < -1; ++bb)
                        for (int c = 0; c < ny; ++c) {
                            const int tz = pre_at(wz, a), tx = pre_at(wx, bb), ty = pre_at(wy, c);
                            if (!hot_at(S, tz, tx, ty)) continue;
                            if (want-- == 0) {
                                pz = tz;
                                px = tx;
                                py = ty;
                                break;
                            }
                        }
                // rows past the last one are never read back: a warp holding only such rows skips them;
                // the adjoint reads G at q - e (the flipped stencil)
                if (b0 + 32 * q < nrows) {
                    if (warp < 4) store_taps<0, 14, -1>(S.g0, S.g1, pz, px, py, pz >= 0, tb + lane_base);
                    else store_taps<14, NTAP, -1>(S.g0, S.g1, pz, px, py, pz >= 0, tb + lane_base);
                }
                tmem_wait_st();
                tc_fence_before();
                block_sync();
                tc_fence_after();
                if (tid == 0) {
                    for (int e = 0; e < NTAP; ++e)
                        mma_ts(tb + TM_D, tb + TM_A + 8 * e, sdesc(smem_u32(S.w + e * WTAP), 128, 256),
                               idesc, (pass > 0 || e > 0) ? 1u : 0u);
                    mma_commit(&S.bar);
                }
                if (block_wait_mma(&S.bar, phase, L.err)) {
                    failed = true;
                    break;
                }
                phase ^= 1;
                tc_fence_after();
            }
            if (failed) {
                stop = true;
                break;
            }
            if (warp < 4) {
                float v[16];
                tmem_ld16(tb + lane_base + TM_D, v);
                // sum over the row group in a fixed butterfly order (every lane of a group gets the same sum)
                const int gmax = __reduce_max_sync(0xffffffffu, gr);
                for (int w = 1; w < gmax; w <<= 1) {
#pragma unroll
                    for (int c = 0; c < MC; ++c) {
                        const float o = __shfl_xor_sync(0xffffffffu, v[c], w);
                        if (w < gr) v[c] += o;
                    }
                }
                if (ic >= 0 && j == 0) {
                    const int k = S.srck[ic];
                    const size_t idx = size_t(S.srci[ic]);
                    if (k == SRC_T) {
                        float4 *o = reinterpret_cast<float4 *>(gt + idx * MC);
#pragma unroll
                        for (int c = 0; c < 4; ++c) o[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
                    } else {
#pragma unroll
                        for (int c = 0; c < 4; ++c) red_add_v4(gp + idx * MC + 4 * c, v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
                    }
                }
            }
            tc_fence_before();
            block_sync();
            tc_fence_after();
        }
    }
    if (ready) {
        tc_fence_before();
        block_sync();
        if (warp == 0) tmem_dealloc(tb, TMEM_COLS);
    }
}

// ---------------------------------------------------------------- weight gradient
struct WgradSmem {
    FeatStage st;
    Targets tg;
    alignas(16) unsigned char u[WG_MG * WG_T * 16];  // im2col of WG_T targets: group mg = 2e + h, target t at mg*256 + t*16
    alignas(16) unsigned char gtile[2 * (WG_T / 8) * 128];  // g^T: co group g, target chunk k at (2g + k) * 128
    uint64_t bar;
    uint32_t tmem;
};

struct WgradPlan {
    int first[MAXL], last[MAXL];  // CTAs whose unit range meets each level (inclusive), -1 if none
};

// Persistent: CTA i handles units [i*U/G, (i+1)*U/G) (unit = work item x sub-tile, ordered by level)
// and keeps one FP32 accumulator per level in tensor memory, flushed to partial[i + level index].
__global__ void __launch_bounds__(NT, 2) mc_wgrad_kernel(const DevLayout L, const Item *__restrict__ items, int n_units,
                                                         const uint4 *__restrict__ vals, const uint4 *__restrict__ tree,
                                                         int bc, const uint4 *__restrict__ gout,
                                                         float *__restrict__ partial) {
    extern __shared__ __align__(16) unsigned char smraw[];
    WgradSmem &S = *reinterpret_cast<WgradSmem *>(smraw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = gridDim.x;
    const int u0 = int((int64_t(blockIdx.x) * n_units) / G), u1 = int((int64_t(blockIdx.x + 1) * n_units) / G);
    if (u0 >= u1) return;
    if (tid == 0) mbar_init(&S.bar);
    for (int i = tid; i < int(sizeof(S.u) / 16); i += NT) reinterpret_cast<uint4 *>(S.u)[i] = make_uint4(0, 0, 0, 0);
    if (warp == 0) tmem_alloc(smem_u32(&S.tmem), TMEM_COLS);
    tc_fence_before();
    block_sync();
    tc_fence_after();
    const uint32_t tb = S.tmem;
    const int q = warp & 3;
    const uint32_t lane_base = uint32_t(32 * q) << 16;
    constexpr uint32_t idesc = idesc_bf16(128, 16, true);
    uint32_t phase = 0;
    // this thread's im2col share, the same in every K step: target it_t, taps ie0 and ie1 (both halves)
    static_assert(NT == WG_T * 16 && NTAP <= 32, "one target and two taps per thread");
    const int it_t = tid % WG_T, ie0 = tid / WG_T, ie1 = ie0 + 16;
    const int off0 = tap_off(ie0), off1 = ie1 < NTAP ? tap_off(ie1) : 0;
    int cur_l = items[u0 / NSUB].l;
    bool dirty = false, failed = false;
    // writes the level's accumulator (zeros if nothing was accumulated) to partial[cta + level index];
    // D block mb (rows 128 mb .. +127 of (e, ci)) lives in columns 16 mb .. 16 mb + 15
    auto flush = [&]() {
        if (warp < 4) {
            float *dst = partial + size_t(blockIdx.x + cur_l - L.l_min) * WG_ROWS * MC;
            for (int mb = 0; mb < 4; ++mb) {
                float v[16];
                tmem_ld16(tb + lane_base + 16 * mb, v);
                const int row = 128 * mb + 32 * q + lane;
                if (row < WG_ROWS) {
                    float4 *o = reinterpret_cast<float4 *>(dst + size_t(row) * MC);
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        o[c] = dirty ? make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3])
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        }
        tc_fence_before();
        block_sync();
        tc_fence_after();
    };
    for (int u = u0; u < u1 && !failed; ++u) {
        Sub s;
        const Item it = items[u / NSUB];
        if (it.l != cur_l) {
            flush();
            cur_l = it.l;
            dirty = false;
        }
        if (!sub_of(L, it, u % NSUB, s)) continue;
        const int nt = count_targets(L, s, S.tg);
        if (nt == 0) continue;
        // dL/dout of the first step's targets, loaded while the patch is staged; each step then loads
        // the next step's while its MMAs run (threads 0 .. 2 WG_T - 1: target tid / 2, half tid % 2)
        uint4 gnext = make_uint4(0, 0, 0, 0);
        if (tid < 2 * WG_T && (tid >> 1) < nt) gnext = gout[2 * size_t(target_index(S.tg, tid >> 1)) + (tid & 1)];
        stage_features(L, s, u, vals, tree, bc, S.st, &S.tg);
        for (int t0 = 0; t0 < nt; t0 += WG_T) {
            // im2col: entry (mg, t) = channels 8h .. 8h+7 of tap e = mg / 2 at target t0 + t; this
            // thread copies both halves of taps ie0 and ie1 for target it_t
            {
                const bool live = t0 + it_t < nt;
                const int cell = live ? int(S.tg.cell[t0 + it_t]) : 0;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int e = h ? ie1 : ie0;
                    if (e < NTAP) {
                        uint4 a = make_uint4(0, 0, 0, 0), b = a;
                        if (live) {
                            const int c = cell + (h ? off1 : off0);
                            a = S.st.p0[c];
                            b = S.st.p1[c];
                        }
                        *reinterpret_cast<uint4 *>(S.u + (2 * e) * (WG_T * 16) + it_t * 16) = a;
                        *reinterpret_cast<uint4 *>(S.u + (2 * e + 1) * (WG_T * 16) + it_t * 16) = b;
                    }
                }
            }
            // g^T (N = co rows, K = targets), K-major core matrices
            if (tid < 2 * WG_T) {
                const int tt = tid >> 1, h = tid & 1, tn = t0 + WG_T + tt;
                const uint4 v = gnext;
                gnext = tn < nt ? gout[2 * size_t(S.tg.idx[tn]) + h] : make_uint4(0, 0, 0, 0);
                const uint16_t *p = reinterpret_cast<const uint16_t *>(&v);
#pragma unroll
                for (int j = 0; j < 8; ++j)  // co = 8h + j
                    *reinterpret_cast<uint16_t *>(S.gtile + (h * (WG_T / 8) + (tt >> 3)) * 128 + j * 16 + (tt & 7) * 2) = p[j];
            }
            fence_async_smem();
            tc_fence_before();
            block_sync();
            tc_fence_after();
            if (tid == 0) {
                const uint64_t bd = sdesc(smem_u32(S.gtile), 128, (WG_T / 8) * 128);
                for (int mb = 0; mb < 4; ++mb) {
                    const uint64_t ad = sdesc(smem_u32(S.u + mb * 16 * (WG_T * 16)), 128, WG_T * 16);
                    mma_ss(tb + 16 * mb, ad, bd, idesc, dirty ? 1u : 0u);
                }
                mma_commit(&S.bar);
            }
            if (block_wait_mma(&S.bar, phase, L.err)) {
                failed = true;
                break;
            }
            phase ^= 1;
            dirty = true;
            tc_fence_after();
        }
    }
    if (!failed) flush();
    tc_fence_before();
    block_sync();
    if (warp == 0) tmem_dealloc(tb, TMEM_COLS);
}

// grad_weights[lev][co][ci][e] = sum over the level's CTAs (in order) of partial[cta + lev][16e + ci][co]
__global__ void mc_wgrad_reduce_kernel(const float *__restrict__ partial, WgradPlan plan, int n_levels,
                                       float *__restrict__ gw) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_levels * WG_ROWS * MC) return;
    const int lev = i / (WG_ROWS * MC), r = i % (WG_ROWS * MC);
    const int row = r / MC, co = r % MC;
    float acc = 0.0f;
    if (plan.first[lev] >= 0)
        for (int c = plan.first[lev]; c <= plan.last[lev]; ++c) acc += partial[(size_t(c) + lev) * WG_ROWS * MC + r];
    const int e = row / MC, ci = row % MC;
    gw[((size_t(lev) * MC + co) * MC + ci) * NTAP + e] = acc;
}

// Each CTA of the tensor-core kernels holds 256 of the SM's 512 tensor-memory columns, so their
// shared memory must admit exactly two CTAs per SM (228 KB per SM, 1 KB reserved per CTA).
constexpr size_t kTwoPerSmMin = 76 * 1024, kTwoPerSmMax = 112 * 1024;
static_assert(sizeof(FwdSmem) > kTwoPerSmMin && sizeof(FwdSmem) <= kTwoPerSmMax, "forward: two CTAs per SM");
static_assert(sizeof(BwdSmem) > kTwoPerSmMin && sizeof(BwdSmem) <= kTwoPerSmMax, "data adjoint: two CTAs per SM");
static_assert(sizeof(WgradSmem) > kTwoPerSmMin && sizeof(WgradSmem) <= kTwoPerSmMax, "weight gradient: two CTAs per SM");
// operands of tensor-core descriptors and 16-byte vector accesses start on 16-byte boundaries
static_assert(offsetof(FwdSmem, w) % 16 == 0 && offsetof(BwdSmem, w) % 16 == 0, "weights alignment");
static_assert(offsetof(WgradSmem, u) % 16 == 0 && offsetof(WgradSmem, gtile) % 16 == 0, "operand alignment");
static_assert(offsetof(BwdSmem, g1) % 16 == 0 && offsetof(FeatStage, p1) % 16 == 0, "patch alignment");
static_assert(offsetof(FwdSmem, bar) % 8 == 0 && offsetof(BwdSmem, bar) % 8 == 0 && offsetof(WgradSmem, bar) % 8 == 0,
              "mbarrier alignment");

cudaError_t set_smem(const void *fn, size_t bytes) { return set_max_dynamic_smem(fn, bytes); }

// CTAs of the weight-gradient kernel: 8 per SM (2 resident at a time), so each CTA accumulates a
// short chain of tensor-core MMAs (about 1/8 of an SM's share of the units) before its partial sum
// is written; the fixed-order reduction then adds the partials in FP32.
int wgrad_ctas(int n_units) {
    static int sms = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 152;
    });
    return std::max(1, std::min(n_units, 8 * sms));
}

bool mc_args_ok(int32_t c_in, int32_t c_out, int32_t k) { return c_in == MC && c_out == MC && k == 3; }
bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

// Multi-channel sub-tile plans (host): for every sub-tile (item * NSUB + sub) the non-empty feature
// segments (fwd_items; meta = segment index | MC_REFL for rows outside the grid) and the non-empty
// data-adjoint segments (bwd_items; meta = segment index). Entries as in the single-channel plans.
bool build_mc_plans(const DevLayout &L, const HostIndex &X, HostPlan &feat, HostPlan &adj) {
    bool ok = true;
    auto build = [&](const std::vector<Item> &items, HostPlan &P, bool features) {
        P.hdr.assign(items.size() * NSUB, PlanHdr{0, 0});
        P.ent.clear();
        for (size_t t = 0; t < items.size(); ++t)
            for (int sub = 0; sub < NSUB; ++sub) {
                const int first = int(P.ent.size());
                int total = 0;
                Sub s;
                if (sub_of(L, items[t], sub, s)) {
                    const int nseg = features ? NSEG_F : NSEG_B;
                    for (int sg = 0; sg < nseg; ++sg) {
                        int lo = 0, hi = 0;
                        bool refl = false;
                        if (features) feat_segment(L, s, sg, lo, hi, refl);
                        else adj_segment(L, s, sg, lo, hi);
                        if (hi <= lo) continue;
                        P.ent.push_back(PlanEnt{lo, uint16_t(sg | (refl ? MC_REFL : 0)), uint16_t(total)});
                        total += hi - lo;
                        if (total > 65535) ok = false;
                    }
                }
                P.hdr[t * NSUB + sub] = PlanHdr{first, int(P.ent.size()) - first};
                P.ent.push_back(PlanEnt{0, 0, uint16_t(total)});
            }
    };
    build(X.fwd_items, feat, true);
    build(X.bwd_items, adj, false);
    return ok;
}

}  // namespace aprk

using namespace aprk;

extern "C" {

apr_status_t apr_selftest_bounded_wait(apr_handle_t h, uint32_t limit_us, apr_stream_t stream) {
    if (!h || h->host_only || limit_us == 0 || limit_us > 2000000u) return APR_ERR_INVALID_ARG;
    bounded_wait_selftest_kernel<<<1, 32, 0, stream>>>(uint64_t(limit_us) * 1000ull, h->d_err);
    return cuda_status(cudaGetLastError());
}

apr_status_t apr_tree_restrict_bf16(apr_handle_t h, const uint16_t *particles, uint16_t *tree, int32_t channels,
                                    apr_stream_t stream) {
    if (!h || h->host_only) return APR_ERR_INVALID_ARG;
    if (channels != MC) return APR_ERR_UNSUPPORTED;
    const HostIndex &X = h->X;
    if ((X.np && !particles) || (X.nt && !tree) || !aligned16(particles) || !aligned16(tree)) return APR_ERR_INVALID_ARG;
    cudaError_t e = cudaSuccess;
    bool chained = false;   // the launches after the first start early (programmatic dependent launch)
    for (int l = X.l_max - 1; e == cudaSuccess && l >= X.l_min; --l) {
        int64_t b = 0, n = 0;
        tree_level_nodes(X, l, b, n);
        if (n > 0)
            e = launch_pdl(mc_tree_restrict_kernel, dim3(int((2 * n + NT - 1) / NT)), dim3(NT), 0, stream, chained,
                           h->d_tnplan, int(b), int(n), reinterpret_cast<const uint4 *>(particles),
                           reinterpret_cast<uint4 *>(tree));
        chained = chained || n > 0;
    }
    return cuda_status(e);
}

static apr_status_t convolve_mc(apr_handle_t h, const uint16_t *particles, const uint16_t *tree,
                                const uint16_t *weights, int32_t c_in, int32_t c_out, int32_t k, int32_t bc, float *out,
                                uint16_t *out_bf16, apr_stream_t stream) {
    if (!h || h->host_only) return APR_ERR_INVALID_ARG;
    if (!mc_args_ok(c_in, c_out, k)) return APR_ERR_UNSUPPORTED;
    if (bc != APR_BC_REFLECT && bc != APR_BC_ZERO) return APR_ERR_INVALID_ARG;
    const HostIndex &X = h->X;
    if (!weights || (X.np && (!particles || (!out && !out_bf16))) || (X.nt && !tree)) return APR_ERR_INVALID_ARG;
    if (!aligned16(particles) || !aligned16(tree) || !aligned16(out) || !aligned16(out_bf16)) return APR_ERR_INVALID_ARG;
    const size_t sm = sizeof(FwdSmem);
    cudaError_t e = set_smem(reinterpret_cast<const void *>(mc_fwd_kernel), sm);
    const int n = int(X.fwd_items.size());
    const int nl = X.l_max - X.l_min + 1;
    if (e == cudaSuccess && n > 0) {
        mc_weight_layout_kernel<<<(nl * MC * MC * NTAP + 255) / 256, 256, 0, stream>>>(weights, nl, 0, h->d_mcw);
        mc_fwd_kernel<<<dim3(n, NSUB / SPC_F), NT, sm, stream>>>(h->L, h->d_fwd, reinterpret_cast<const uint4 *>(particles),
                                                          reinterpret_cast<const uint4 *>(tree), h->d_mcw, bc, out,
                                                          reinterpret_cast<uint4 *>(out_bf16));
        e = cudaGetLastError();
    }
    return cuda_status(e);
}

apr_status_t apr_convolve_mc(apr_handle_t h, const uint16_t *particles, const uint16_t *tree, const uint16_t *weights,
                             int32_t c_in, int32_t c_out, int32_t k, int32_t bc, float *out, apr_stream_t stream) {
    if (!out && h && h->X.np) return APR_ERR_INVALID_ARG;
    return convolve_mc(h, particles, tree, weights, c_in, c_out, k, bc, out, nullptr, stream);
}

apr_status_t apr_convolve_mc_relu_bf16(apr_handle_t h, const uint16_t *particles, const uint16_t *tree,
                                       const uint16_t *weights, int32_t c_in, int32_t c_out, int32_t k, int32_t bc,
                                       uint16_t *out, apr_stream_t stream) {
    if (!out && h && h->X.np) return APR_ERR_INVALID_ARG;
    return convolve_mc(h, particles, tree, weights, c_in, c_out, k, bc, nullptr, out, stream);
}

size_t apr_mc_backward_workspace_bytes(apr_handle_t h, int32_t c_in, int32_t c_out, int32_t k) {
    if (!h || !mc_args_ok(c_in, c_out, k)) return 0;
    const int L = h->X.l_max - h->X.l_min + 1;
    const int units = int(h->X.fwd_items.size()) * NSUB;
    const size_t gt = (size_t(h->X.nt) * MC * sizeof(float) + 255) / 256 * 256;
    return gt + size_t(wgrad_ctas(units) + L) * WG_ROWS * MC * sizeof(float);
}

apr_status_t apr_convolve_mc_backward(apr_handle_t h, const uint16_t *particles, const uint16_t *tree,
                                      const uint16_t *weights, int32_t c_in, int32_t c_out, int32_t k, int32_t bc,
                                      const uint16_t *grad_out, float *grad_particles, float *grad_weights,
                                      void *workspace, size_t workspace_bytes, apr_stream_t stream) {
    if (!h || h->host_only) return APR_ERR_INVALID_ARG;
    if (!mc_args_ok(c_in, c_out, k)) return APR_ERR_UNSUPPORTED;
    if (bc != APR_BC_REFLECT && bc != APR_BC_ZERO) return APR_ERR_INVALID_ARG;
    const HostIndex &X = h->X;
    if (!weights || (X.np && !grad_out)) return APR_ERR_INVALID_ARG;
    if (grad_weights && ((X.np && !particles) || (X.nt && !tree))) return APR_ERR_INVALID_ARG;
    if (!aligned16(particles) || !aligned16(tree) || !aligned16(grad_out) || !aligned16(grad_particles) ||
        !aligned16(grad_weights))
        return APR_ERR_INVALID_ARG;
    const size_t need = apr_mc_backward_workspace_bytes(h, c_in, c_out, k);
    if (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) return APR_ERR_INVALID_ARG;
    const size_t gt_bytes = (size_t(X.nt) * MC * sizeof(float) + 255) / 256 * 256;
    float *gt = static_cast<float *>(workspace);
    float *partial = reinterpret_cast<float *>(static_cast<char *>(workspace) + gt_bytes);
    const int n_levels = X.l_max - X.l_min + 1;
    cudaError_t e = cudaSuccess;
    if (grad_particles) {
        if (X.np) e = cudaMemsetAsync(grad_particles, 0, size_t(X.np) * MC * sizeof(float), stream);
        if (e == cudaSuccess && X.nt) e = cudaMemsetAsync(gt, 0, size_t(X.nt) * MC * sizeof(float), stream);
        if (e == cudaSuccess) e = set_smem(reinterpret_cast<const void *>(mc_bwd_data_kernel), sizeof(BwdSmem));
        const int n = int(X.bwd_items.size());
        const uint16_t *wt = h->d_mcw + size_t(n_levels) * MC * MC * NTAP;
        if (e == cudaSuccess && n > 0) {
            mc_weight_layout_kernel<<<(n_levels * MC * MC * NTAP + 255) / 256, 256, 0, stream>>>(
                weights, n_levels, 1, h->d_mcw + size_t(n_levels) * MC * MC * NTAP);
            mc_bwd_data_kernel<<<dim3(n, NSUB / SPC_B), NT, sizeof(BwdSmem), stream>>>(
                h->L, h->d_bwd, wt, bc, reinterpret_cast<const uint4 *>(grad_out), grad_particles, gt);
            e = cudaGetLastError();
        }
        bool chained = false;   // the launches after the first start early (programmatic dependent launch)
        for (int l = X.l_min; e == cudaSuccess && l < X.l_max; ++l) {
            int64_t b = 0, nt = 0;
            tree_level_nodes(X, l, b, nt);
            if (nt > 0)
                e = launch_pdl(mc_tree_pushdown_kernel, dim3(int((4 * nt + NT - 1) / NT)), dim3(NT), 0, stream, chained,
                               h->d_tnplan, int(b), int(nt), reinterpret_cast<float4 *>(grad_particles),
                               reinterpret_cast<float4 *>(gt));
            chained = chained || nt > 0;
        }
    }
    if (e == cudaSuccess && grad_weights) {
        const int units = int(X.fwd_items.size()) * NSUB;
        const int G = wgrad_ctas(units);
        WgradPlan plan;
        for (int i = 0; i < MAXL; ++i) plan.first[i] = plan.last[i] = -1;
        auto cta_of = [&](int64_t u) {  // CTA c with c*units/G <= u < (c+1)*units/G
            int c = int((u * G) / units);
            while (c + 1 < G && (int64_t(c + 1) * units) / G <= u) ++c;
            while (c > 0 && (int64_t(c) * units) / G > u) --c;
            return c;
        };
        for (int lv = 0; lv < n_levels; ++lv) {
            const int64_t ua = X.fwd_level_begin[X.l_min + lv] * NSUB, ub = X.fwd_level_begin[X.l_min + lv + 1] * NSUB;
            if (ua >= ub) continue;
            plan.first[lv] = cta_of(ua);
            plan.last[lv] = cta_of(ub - 1);
        }
        e = set_smem(reinterpret_cast<const void *>(mc_wgrad_kernel), sizeof(WgradSmem));
        if (e == cudaSuccess && units > 0) {
            mc_wgrad_kernel<<<G, NT, sizeof(WgradSmem), stream>>>(h->L, h->d_fwd, units,
                                                                  reinterpret_cast<const uint4 *>(particles),
                                                                  reinterpret_cast<const uint4 *>(tree), bc,
                                                                  reinterpret_cast<const uint4 *>(grad_out), partial);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            const int tot = n_levels * WG_ROWS * MC;
            mc_wgrad_reduce_kernel<<<(tot + 255) / 256, 256, 0, stream>>>(partial, plan, n_levels, grad_weights);
            e = cudaGetLastError();
        }
    }
    return cuda_status(e);
}

}  // extern "C"
