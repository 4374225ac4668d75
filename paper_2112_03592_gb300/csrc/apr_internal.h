// Internal definitions shared by the host index builder, the C-ABI entry points and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "apr.h"

namespace aprk {

// y-block of the brick index and of every work item: rows are cut into blocks of BY cells along y,
// and each row stores, per block, the offset of its first element (a finer-grained xz_end).
constexpr int BY = 64;
// (z, x) rows per convolution tile at the tile's own level (APR_TILE_ZX in apr.h).
constexpr int TZ = APR_TILE_ZX;
constexpr int TX = APR_TILE_ZX;
static_assert(BY == APR_BLOCK_Y, "y-block must match apr.h");
constexpr int MAXL = 24;

// Geometry of one level, passed to kernels by value.
struct LevelGeo {
    int32_t dz, dx, dy;  // level grid size
    int32_t nb;          // ceil(dy / BY) blocks per row
    int32_t row0;        // index of the level's first particle row (into row_ptr)
    int32_t off0;        // index of the level's first entry in the particle block-offset array
    int32_t trow0;       // same for the tree (levels < l_max)
    int32_t toff0;
};

// Tile plans: per work item, the non-empty source segments of its staged patch (index range of one
// row's elements) in the kernels' segment order, built once per APR on the host. For each item,
// hdr = {first entry, count}; entries [first, first + count) hold {lo, meta, pre}, pre = the number
// of elements of the item's entries before this one; entry first + count holds the total in pre.
struct PlanHdr {
    int32_t first, count;
};
struct PlanEnt {
    int32_t lo;
    uint16_t meta, pre;
};
static_assert(sizeof(PlanEnt) == 8, "plan entries are 8-byte words");
// Child map of one tree node (built once per APR; one per node, in tree order): for each of the four
// child rows k = (a, b) = (k >> 1, k & 1) of level l+1 over the node, p[k] = index of its first
// particle child there and t[k] = index of its first tree child (bits 0..29), and in bits 30, 31 of
// p[k] (t[k]) whether child cell y = 2 y_node (bit 30) and 2 y_node + 1 (bit 31) is a particle (a
// tree node). A child cell with neither bit lies outside the grid (or, in a sub-domain's partial
// index, outside the sub-domain). The second child of a kind in a row follows the first at index + 1.
struct alignas(16) TreeNodePlan {
    int32_t p[4];
    int32_t t[4];
};
static_assert(sizeof(TreeNodePlan) == 32, "node plans are two 16-byte words");
constexpr uint32_t TNP_INDEX = (1u << 30) - 1u;
struct PlanView {
    const PlanHdr *hdr;
    const PlanEnt *ent;
};
struct HostPlan {
    std::vector<PlanHdr> hdr;
    std::vector<PlanEnt> ent;
};
struct FPlanView {     // forward tile plans (apr_tile.cuh: FPlanEnt)
    const PlanHdr *hdr;
    const uint2 *ent;
};
struct HostFPlan {
    std::vector<PlanHdr> hdr;
    std::vector<uint2> ent;
};

// Everything a kernel needs to walk the index (device pointers).
struct DevLayout {
    const uint32_t *row_ptr;   // [R+1]
    const uint16_t *y;         // [N_p]
    const uint16_t *off;       // [sum_l rows_l * nb_l]: first element of block j, relative to row start
    const uint32_t *trow_ptr;  // [R_t+1]
    const uint16_t *ty;        // [N_t]
    const uint16_t *toff;
    unsigned *err;
    int32_t np, nt;            // particles, tree nodes (value array lengths)
    int32_t l_min, l_max;
    LevelGeo geo[MAXL];
    FPlanView fplan[2];  // forward tiles (fwd_items), stencil radius 1 and 2
    FPlanView bplan[2];  // data-adjoint tiles (bwd_items), stencil radius 1 and 2
    PlanView mcfplan;    // multi-channel feature patches of the sub-tiles of fwd_items
    PlanView mcbplan;    // multi-channel data-adjoint sub-tiles of bwd_items
};

struct Item {  // a work item: level, tile (or row) coordinates, y block
    int32_t l, a, b, yb;
};

// Host-side index, built by build_index(); uploaded by apr_build_device.
struct HostIndex {
    int32_t l_min = 0, l_max = 0;
    int64_t dims[3] = {0, 0, 0};
    LevelGeo geo[MAXL] = {};
    int64_t np = 0, nt = 0, R = 0, Rt = 0, noff = 0, ntoff = 0;
    std::vector<uint32_t> row_ptr, trow_ptr;
    std::vector<uint16_t> y, ty, off, toff;
    std::vector<Item> fwd_items;              // non-empty (l, tz, tx, yb) tiles, by level
    std::vector<Item> bwd_items;              // tiles whose interior cells receive gradient
    std::vector<Item> tree_items;             // non-empty (l, z, x, yb) tree bricks, by level
    int64_t fwd_level_begin[MAXL + 1] = {};   // fwd_items of level l: [begin[l], begin[l+1])
    int64_t bwd_level_begin[MAXL + 1] = {};   // bwd_items of level l: [begin[l], begin[l+1])
    int64_t tree_level_begin[MAXL + 1] = {};
    HostFPlan fplan[2];                       // forward tile plans (build_plans), radius 1 and 2
    HostFPlan bplan[2];                       // data-adjoint tile plans (build_plans), radius 1 and 2
    HostPlan mcfplan, mcbplan;                // multi-channel sub-tile plans (build_mc_plans)
    std::vector<TreeNodePlan> tnplan;         // child maps of the tree nodes (tree_node_plan)
};

// The tree nodes of level l (l_min <= l < l_max): [b, b + n) in tree order.
inline void tree_level_nodes(const HostIndex &X, int l, int64_t &b, int64_t &n) {
    const LevelGeo &g = X.geo[l];
    b = X.trow_ptr[size_t(g.trow0)];
    n = int64_t(X.trow_ptr[size_t(g.trow0) + size_t(g.dz) * size_t(g.dx)]) - b;
}

// Work items of the consecutive levels l0 .. l0 + n - 1: level l0 + i owns items [begin[i], begin[i + 1])
// (passed to kernels by value).
struct LevelRanges {
    int32_t l0 = 0, n = 0;
    int32_t begin[MAXL + 1] = {};
};

// Builds and validates the index from the host layout. Returns APR_OK or an error code; `msg`
// receives a short reason on failure.
apr_status_t build_index(const apr_host_layout &L, uint32_t flags, HostIndex &out, const char **msg);

// Builds the tile plans of X's forward and data-adjoint work items (apr_plan.cu) and the
// multi-channel sub-tile plans. Returns APR_OK, APR_ERR_OOM (host allocation) or
// APR_ERR_UNSUPPORTED (a tile with 65536 or more staged elements).
apr_status_t build_plans(HostIndex &X);
// The multi-channel sub-tile plans (apr_mc.cu); true unless a tile overflows the 16-bit counts.
bool build_mc_plans(const DevLayout &L, const HostIndex &X, HostPlan &feat, HostPlan &adj);
// The child map of every tree node (TreeNodePlan), by one merge of each tree row with its child rows.
// In a complete index every in-grid child cell of a node is a particle or a node of the next level.
bool tree_node_plan(const DevLayout &L, const HostIndex &X, std::vector<TreeNodePlan> &P);
// apr_convolve_adjoint; split: a 5^3 stack's levels below l_max on the handle's split stream
apr_status_t convolve_adjoint(apr_handle_t h, const float *stencils, int32_t k, int32_t bc, const float *grad_out,
                              float *grad_particles, float *grad_tree, apr_stream_t stream, bool split);
// apr_convolve_backward; concurrent: the stencil gradient on the handle's second stream and the
// data adjoint split by radius
apr_status_t convolve_backward(apr_handle_t h, const float *particles, const float *tree, const float *stencils,
                               int32_t k, int32_t bc, const float *grad_out, float *grad_particles,
                               float *grad_stencils, void *workspace, size_t workspace_bytes, apr_stream_t stream,
                               bool concurrent);
// DevLayout over the host copy of X's index (for host code that walks it like a kernel).
DevLayout host_layout_view(const HostIndex &X);

// Record a short reason for the last failure on this thread (read by apr_last_error_message).
void set_last_message(const char *msg);

// Epilogues of the convolution kernel (launch_conv_fwd)
constexpr int EPI_PLAIN = 0, EPI_DIVIDE = 1, EPI_MULTIPLY = 2;

// Bits of the device error word (DevLayout::err), read and cleared by apr_sync_status.
constexpr unsigned ERR_DEVICE_CHECK = 1u;  // a device-side consistency check failed
constexpr unsigned ERR_TIMEOUT = 2u;       // a bounded wait (tensor-core completion) gave up

// Map a CUDA error to a status code, recording its message for apr_last_error_message.
apr_status_t cuda_status(cudaError_t e);

// Raise a kernel's dynamic shared-memory limit to `bytes` on the current device, once per (kernel,
// device): later calls make no CUDA call, so launches can be captured into CUDA graphs.
cudaError_t set_max_dynamic_smem(const void *fn, size_t bytes);

// kernel<<<grid, block, smem, s>>>(args...), with programmatic stream serialization when `pdl`: the
// kernel may then start while the kernel before it on s finishes, and waits for it with pdl_wait
// (apr_device.cuh) before it reads what that kernel writes.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                       Args &&...args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

inline int64_t level_cells(int64_t D, int l_max, int l) {
    int64_t s = int64_t(1) << (l_max - l);
    return (D + s - 1) / s;
}

}  // namespace aprk

// The object behind apr_handle_t: the host index and its device copy.
struct apr_handle_s {
    aprk::HostIndex X;
    bool host_only = false;
    aprk::DevLayout L{};
    aprk::Item *d_fwd = nullptr, *d_bwd = nullptr, *d_tree = nullptr;
    int64_t *d_fwd_level_begin = nullptr;
    uint32_t *d_row_ptr = nullptr, *d_trow_ptr = nullptr;
    uint16_t *d_y = nullptr, *d_ty = nullptr, *d_off = nullptr, *d_toff = nullptr;
    unsigned *d_err = nullptr;
    uint16_t *d_mcw = nullptr;   // multi-channel weights in the tensor-core operand layout, per level
    apr_stream_t stream = nullptr;                      // the build stream (uploads, stream-ordered allocation)
    apr_allocator alloc{};                              // the caller's allocator, if has_alloc
    bool has_alloc = false;
    std::vector<std::pair<void *, size_t>> blocks;      // every device block of the handle
    // tile plans: multi-channel feature, adjoint
    aprk::PlanHdr *d_plan_hdr[2] = {};
    aprk::PlanEnt *d_plan_ent[2] = {};
    aprk::TreeNodePlan *d_tnplan = nullptr;
    // host-only handles: tile plans built on the first apr_export_structure request for them
    std::mutex plan_mu;
    bool host_plans = false;
    aprk::PlanHdr *d_fplan_hdr[4] = {};   // forward radius 1, 2; adjoint radius 1, 2
    uint2 *d_fplan_ent[4] = {};
    size_t dev_bytes = 0;
    // apr_convolve_backward runs the stencil gradient on a second stream, forked from and joined back
    // to the caller's stream with these events (created on first use; side_mu orders the enqueues)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::mutex side_mu;
    // a 5^3 convolution or data adjoint over the whole work list runs its radius-1 tiles of the
    // levels below l_max on this stream, beside the l_max tiles on the caller's stream (split_mu
    // orders the enqueues; taken after side_mu where both are held)
    cudaStream_t split = nullptr;
    cudaEvent_t ev_split_fork = nullptr, ev_split_join = nullptr;
    std::mutex split_mu;
    // whether the last such call saw a level below l_max with taps outside the central 3^3 ([0]
    // convolution, [1] data adjoint): mapped host memory that the kernels write and the host reads to
    // choose the next call's launches (h_hint host view, d_hint device view)
    int *h_hint = nullptr, *d_hint = nullptr;
};
