/*
 * apr.h -- C ABI of the GB300 (sm_103a) library for discrete convolution evaluated natively on an
 * Adaptive Particle Representation (APR) of a 3-D image.
 *
 * Method: Jonsson, Cheeseman, Maddu, Gonciarz, Sbalzarini, "Parallel Discrete Convolutions on
 * Adaptive Particle Representations of Images" (arXiv 2112.03592). Section numbers below refer to it.
 *
 * Conventions shared by every call
 *   - Every call returns apr_status_t; nothing aborts or exits. apr_status_string() names a code.
 *   - Image axes are (z, x, y); y is the contiguous, sparsely stored axis (Sec. 3.1 footnote).
 *     l_max = ceil(log2(max(D_z, D_x, D_y))); level l has a grid of ceil(D / 2^(l_max-l)) cells
 *     per axis (Eq. 2, cells of edge 2^(l_max-l) pixels).
 *   - Particles are ordered l -> z -> x -> y (Alg. 2). Tree nodes (the APR tree, Sec. 3.4: every
 *     strict ancestor of a particle cell) use the same order over levels l_min .. l_max-1.
 *   - Value, output, gradient and stencil buffers are CALLER-OWNED DEVICE pointers (float32 unless
 *     stated), never freed or retained by the library. The opaque handle owns only the index
 *     structure it allocated in apr_build_device.
 *   - Work is enqueued asynchronously on the given stream (NULL = the legacy default stream); the
 *     caller synchronises. Launch failures return APR_ERR_CUDA. Device-side checks record into an
 *     error word read by apr_sync_status().
 *   - Not thread-safe per handle: calls on one handle must not run concurrently on different
 *     streams when they share output buffers or the handle's scratch.
 */
#ifndef APR_H
#define APR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    APR_OK = 0,
    APR_ERR_INVALID_ARG = 1,    /* NULL pointer, bad size, unknown flag or enum */
    APR_ERR_INVALID_LAYOUT = 2, /* the index arrays do not describe a (balanced) APR */
    APR_ERR_UNSUPPORTED = 3,    /* e.g. stencil size not 3 or 5, channel count not supported */
    APR_ERR_OOM = 4,            /* device or host allocation failed */
    APR_ERR_CUDA = 5,           /* a CUDA runtime call or kernel launch failed */
    APR_ERR_TIMEOUT = 6,        /* a bounded device wait gave up */
    APR_ERR_DEVICE = 7          /* a device-side check recorded an error (see apr_sync_status) */
} apr_status_t;

/* Same underlying type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *apr_stream_t;

typedef struct apr_handle_s *apr_handle_t;

/* Host description of an APR in the linear-access layout of Alg. 1 (LinearAccess).
 *   row_ptr: [R+1] int64, host memory. Rows are (l, z, x) for l = l_min..l_max, z, x in level grid
 *            order; row r holds particles row_ptr[r] .. row_ptr[r+1]-1 (CSR form of xz_end).
 *   y_idx:   [n_particles] int32, host memory, strictly increasing inside each row, < grid y size.
 * The library copies what it needs; the caller keeps ownership of both arrays. */
typedef struct {
    int32_t l_min;
    int32_t l_max;
    int64_t dims[3];          /* D_z, D_x, D_y in pixels, each >= 1 and <= 65536 */
    const int64_t *row_ptr;
    const int32_t *y_idx;
    int64_t n_particles;      /* < 2^31 */
} apr_host_layout;

/* apr_build_device flags */
#define APR_VALIDATE 1u          /* check that the particle cells partition the image exactly */
#define APR_REQUIRE_BALANCE 2u   /* check the 2:1 balance the 5^3 convolution relies on */
#define APR_HOST_ONLY 4u         /* build the index on the host only (no device memory): for
                                    inspecting the structure on machines without a GPU */
#define APR_SUBDOMAIN 8u         /* the APR covers a block of a larger image (e.g. one z-slab of a
                                    sharded APR): l_max may exceed ceil(log2(max dim)), the levels
                                    being those of the enclosing image */

/* Boundary modes of the convolution (the paper pads without naming a rule, Sec. 5.1) */
#define APR_BC_REFLECT 0         /* half-sample symmetric reflection at each level's grid */
#define APR_BC_ZERO 1            /* taps outside the level grid contribute zero */

/* Work-item geometry: a convolution work item is a tile of APR_TILE_ZX x APR_TILE_ZX rows (z, x)
 * of one level and one y-block of APR_BLOCK_Y cells; every row's particles are indexed per y-block. */
#define APR_TILE_ZX 8
#define APR_BLOCK_Y 64

/* apr_export_structure selectors (copy to host memory) */
#define APR_STRUCT_ROW_PTR 0       /* uint32 [R+1]    particle rows (CSR) */
#define APR_STRUCT_Y_IDX 1         /* uint16 [N_p]    particle y */
#define APR_STRUCT_TREE_ROW_PTR 2  /* uint32 [R_t+1]  tree rows, levels l_min..l_max-1 */
#define APR_STRUCT_TREE_Y_IDX 3    /* uint16 [N_t]    tree node y */
#define APR_STRUCT_FWD_ITEMS 4     /* int32 [n][4]    convolution work items (l, tz, tx, yb) */
#define APR_STRUCT_TREE_ITEMS 5    /* int32 [n][4]    tree work items (l, z, x, yb) */
#define APR_STRUCT_BWD_ITEMS 6     /* int32 [n][4]    data-adjoint work items (l, tz, tx, yb) */
/* int32 [N_t][8] child map of every tree node (what the tree kernels read): words k = 0..3 for the
 * child rows (2z + (k >> 1), 2x + (k & 1)) of level l+1, first the particle word, then (words 4..7)
 * the tree word: bits 0..29 the index of the row's first particle (tree node) child, bit 30 (31) set
 * when child cell y = 2 y_node (2 y_node + 1) is a particle (a tree node). Neither bit: the cell lies
 * outside the grid. A row's second child of a kind sits at the first one's index + 1. */
#define APR_STRUCT_TREE_NODE_MAP 7
/* Tile plans, host-only handles only (built on the first request; 0 bytes for a device handle):
 * uint32 [n_items][2] headers {first entry, count} for the items of APR_STRUCT_FWD_ITEMS (forward, stencil
 * radius 1 or 2) or APR_STRUCT_BWD_ITEMS (data adjoint: count = gradient rows | routing segments << 16),
 * then uint32 [n_entries][2] entries, one per non-empty source segment of an item's patch and one
 * after them holding the item's packet total: word 0 = first element (bits 0..27) | element count
 * bits 0..3 << 28, word 1 = prefix of 8-element packets (bits 0..15) | segment word (11 bits) << 16
 * | element count bits 4..7 << 27. */
#define APR_STRUCT_FWD_PLAN_R1 8
#define APR_STRUCT_FWD_PLAN_R2 9
#define APR_STRUCT_BWD_PLAN_R1 10
#define APR_STRUCT_BWD_PLAN_R2 11

/* Build the device-resident index of an APR (Sec. 3.1 LinearAccess for the particles, Sec. 3.4
 * APR tree structure, and the list of non-empty tiles the kernels are launched on, Sec. 5.2 last
 * paragraph). The tree structure (which nodes exist) is derived from the particle cells; its
 * values are computed later by apr_tree_restrict. y indices are stored as uint16. For every tile
 * the host also lists the non-empty source segments of its staged patch with the prefix of their
 * 8-element packets (tile plans, for stencil radius 1 and 2 and for the multi-channel sub-tiles),
 * so the convolution kernels never evaluate row offsets per call, and for every tree node the indices
 * of its children (32 bytes per node); on a 1024x1024x512 image with 8 M particles the handle holds
 * about 243 MB, plans included (the image itself would be 2.1 GB).
 * The index is allocated stream-ordered (cudaMallocAsync on `stream`) and uploaded on `stream`;
 * it is ready for work enqueued on `stream` (other streams synchronise with it first). The handle
 * also creates two streams and four events for the concurrent parts of later calls, and 8 bytes of
 * mapped pinned host memory (the radius hint of apr_convolve). Returns
 * APR_ERR_INVALID_LAYOUT when the arrays are inconsistent (row sizes, y order and range, and with
 * the flags the partition and the balance), APR_ERR_UNSUPPORTED for more than 2^28 particles or
 * tree nodes, APR_ERR_OOM on allocation failure. *out is NULL on error. */
apr_status_t apr_build_device(const apr_host_layout *layout, uint32_t flags, apr_stream_t stream,
                              apr_handle_t *out);

/* A caller allocator for the handle's device memory (e.g. a framework's caching allocator).
 * alloc(bytes, stream, ctx) returns device memory, 16-byte aligned at least (the kernels read the
 * index with 16-byte loads), usable in stream order on `stream` (NULL on
 * failure: the build returns APR_ERR_OOM); free(ptr, bytes, stream, ctx) releases it, called by
 * apr_destroy after the device has been synchronised. `stream` is the build stream; it must stay
 * valid until apr_destroy. */
typedef struct {
    void *(*alloc)(size_t bytes, apr_stream_t stream, void *ctx);
    void (*free)(void *ptr, size_t bytes, apr_stream_t stream, void *ctx);
    void *ctx;
} apr_allocator;

/* apr_build_device with the handle's device memory taken from `allocator` (NULL: stream-ordered
 * cudaMallocAsync, as apr_build_device). */
apr_status_t apr_build_device_ex(const apr_host_layout *layout, uint32_t flags, apr_stream_t stream,
                                 const apr_allocator *allocator, apr_handle_t *out);

/* Release the handle and its device memory (synchronises the device first). NULL is accepted. */
apr_status_t apr_destroy(apr_handle_t h);

int64_t apr_num_particles(apr_handle_t h);   /* -1 on NULL */
int64_t apr_num_tree(apr_handle_t h);        /* N_t, -1 on NULL */
apr_status_t apr_level_range(apr_handle_t h, int32_t *l_min, int32_t *l_max);
size_t apr_layout_bytes(apr_handle_t h);     /* device bytes owned by the handle (index, work lists, tile plans) */

/* Size in bytes of structure array `which`; 0 if not available. */
size_t apr_structure_bytes(apr_handle_t h, int32_t which);
/* Copy structure array `which` to host memory `dst` of `bytes` (>= apr_structure_bytes). */
apr_status_t apr_export_structure(apr_handle_t h, int32_t which, void *dst, size_t bytes);

/* APR tree restriction (Sec. 3.4, two-step fill, step 2; Sec. 5.2, GPU pipeline): for l = l_max-1 down to l_min, every
 * tree node gets the average of its children inside the level grid, each child being a particle of
 * level l+1 or a tree node of level l+1 (average downsampling, Sec. 2.3).
 *   particles: device [N_p][channels] float32 (channels-last), read only.
 *   tree:      device [N_t][channels] float32, written (every entry).
 * channels: 1 .. 64 (APR_ERR_INVALID_ARG otherwise); each channel is averaged on its own. */
apr_status_t apr_tree_restrict(apr_handle_t h, const float *particles, float *tree, int32_t channels,
                               apr_stream_t stream);

/* APR convolution (Sec. 4.1, per-level stencils Sec. 4.2-4.3; GPU design Sec. 5.2): for every particle
 * p at level l, out[p] = sum_{e in [-r,r]^3} stencils[l - l_min][e] * u_l(refl(i_p + e)), where u_l(c)
 * is the isotropic level-l patch value of cell c (Sec. 3.5): the level-l particle covering c, else
 * the level-l tree node at c, else the level-(l-1) particle containing c. Correlation form (no flip).
 *   particles: device [N_p] float32;  tree: device [N_t] float32 from apr_tree_restrict (required);
 *   stencils:  device [(l_max-l_min+1)][k][k][k] float32, level l_min first, [z][x][y] y fastest;
 *   k: 3 or 5;  bc: APR_BC_REFLECT or APR_BC_ZERO;  out: device [N_p] float32, overwritten.
 * Requires the 2:1 balance of the APR (checked by APR_REQUIRE_BALANCE at build).
 * A level whose 5^3 stencil is zero outside the central 3^3 (every level below l_max of a restricted
 * stack, Eq. restrict_stenc) is computed with radius 1. For k = 5 the tiles of the levels below l_max
 * run on a second stream that the handle owns, in a launch sized for radius 1, beside the l_max tiles
 * on `stream` (forked from and joined back to `stream` with events: the call stays ordered on
 * `stream` and can be captured into a CUDA graph). When the previous call's stack had taps outside
 * the central 3^3 below l_max (read from a hint that the kernels write, without waiting), one launch
 * over all tiles is taken instead. Either way every output is computed by the same code, so results
 * do not depend on the choice. */
apr_status_t apr_convolve(apr_handle_t h, const float *particles, const float *tree, const float *stencils,
                          int32_t k, int32_t bc, float *out, apr_stream_t stream);

/* apr_convolve restricted to the forward work items [first_tile, first_tile + n_tiles) of
 * APR_STRUCT_FWD_ITEMS (ordered by level, then tile z, tile x, y-block): only the outputs of the
 * targets of those tiles are written. For a rank of a z-sharded APR (Sec. 5.1 parallelisation over
 * rows), one range per level covers the tiles that hold its particles. */
apr_status_t apr_convolve_tiles(apr_handle_t h, const float *particles, const float *tree, const float *stencils,
                                int32_t k, int32_t bc, float *out, int64_t first_tile, int64_t n_tiles,
                                apr_stream_t stream);

/* apr_convolve_adjoint restricted to the data-adjoint work items [first_tile, first_tile + n_tiles)
 * of APR_STRUCT_BWD_ITEMS. Nothing is cleared: particle gradients are ADDED, the tree-node
 * gradients of the launched tiles' interior cells are written (each node belongs to one tile). */
apr_status_t apr_convolve_adjoint_tiles(apr_handle_t h, const float *stencils, int32_t k, int32_t bc,
                                        const float *grad_out, float *grad_particles, float *grad_tree,
                                        int64_t first_tile, int64_t n_tiles, apr_stream_t stream);

/* apr_tree_restrict into `workspace` followed by apr_convolve (the paper's pipeline: restriction,
 * then convolution, Sec. 5.2). workspace: caller-owned device memory of at least
 * apr_convolve_auto_workspace_bytes(h) bytes, 16-byte aligned; it holds the tree values [N_t]
 * afterwards. APR_ERR_INVALID_ARG if it is missing or too small; otherwise as the two calls, with the
 * same results. When the convolution is split by radius (see apr_convolve), its l_max tiles read no
 * tree node, so their launch runs on the handle's second stream beside the restriction. */
size_t apr_convolve_auto_workspace_bytes(apr_handle_t h);
apr_status_t apr_convolve_auto(apr_handle_t h, const float *particles, const float *stencils, int32_t k, int32_t bc,
                               float *out, void *workspace, size_t workspace_bytes, apr_stream_t stream);

/* Gradient magnitude on the APR (Sec. 4.3): out[p] = sqrt(sum_{a=0..2} (w_a (*) u)_p^2), where (*) is
 * apr_convolve with the a-th of three per-level stencil stacks (e.g. the Sobel derivative filters
 * along z, x and y, rescaled per level by Eq. adapt_grad with apr_rescale_stencil). The patch is
 * staged once for the three filters.
 *   stencils: device [3][(l_max-l_min+1)][k^3] float32; other arguments as apr_convolve. */
apr_status_t apr_gradient_magnitude(apr_handle_t h, const float *particles, const float *tree, const float *stencils,
                                    int32_t k, int32_t bc, float *out, apr_stream_t stream);

/* Scratch bytes apr_convolve_backward needs for stencil size k. */
size_t apr_backward_workspace_bytes(apr_handle_t h, int32_t k);

/* Adjoint of apr_tree_restrict followed by apr_convolve (the back-propagation through the
 * interpolation across levels that Sec. 6 proposes for APR CNNs). With g = grad_out:
 *   grad_particles[q] = sum over taps that read q (directly at q's level, or as the coarse fill of
 *                       the next finer level) of g_p * w[e], plus the tree share: every tree node's
 *                       gradient is passed to its children divided by its number of children,
 *                       from the coarsest level down;
 *   grad_stencils[l][e] = sum_{p at level l} g_p * u_l(refl(i_p + e)).
 * Inputs as in apr_convolve; grad_out device [N_p]. grad_particles (device [N_p]) and grad_stencils
 * (device [L][k^3]) are overwritten; either may be NULL to skip it. workspace: device scratch of at
 * least apr_backward_workspace_bytes(h, k) bytes, 256-byte aligned, contents ignored on entry.
 * Results are deterministic (fixed summation order).
 * When both gradients are requested, the stencil gradient runs on a second stream that the handle
 * owns, forked from `stream` and joined back to it with events, and the data adjoint takes its
 * launches as apr_convolve_adjoint does: the call stays ordered on `stream` (work enqueued after it
 * waits for both gradients) and can be captured into a CUDA graph from `stream`. Concurrent calls on
 * one handle are serialised while they enqueue. */
apr_status_t apr_convolve_backward(apr_handle_t h, const float *particles, const float *tree,
                                   const float *stencils, int32_t k, int32_t bc, const float *grad_out,
                                   float *grad_particles, float *grad_stencils, void *workspace,
                                   size_t workspace_bytes, apr_stream_t stream);

/* The three parts of apr_convolve_backward, callable on their own (each is the adjoint of one
 * forward piece; apr_convolve_backward runs them in this order).
 *
 * apr_convolve_adjoint: transpose of apr_convolve w.r.t. its value inputs (Sec. 4.1, 5.2): with
 * g = grad_out, grad_particles[q] = sum of g_p * w[e] over the taps that read particle q directly
 * (at q's level) or as the coarse fill of the next finer level; grad_tree[t] = the same for tree
 * node t. Both outputs are overwritten (device [N_p] and [N_t] float32). For k = 5 the launches are
 * chosen as in apr_convolve (the same results either way). */
apr_status_t apr_convolve_adjoint(apr_handle_t h, const float *stencils, int32_t k, int32_t bc, const float *grad_out,
                                  float *grad_particles, float *grad_tree, apr_stream_t stream);

/* apr_tree_restrict_adjoint: transpose of apr_tree_restrict (Sec. 3.4), from the coarsest level
 * down: every tree node's gradient is divided by its number of in-grid children and added to each
 * child (tree node or particle). grad_tree (device [N_t]) is updated in place to the accumulated tree
 * gradients; the particle shares are ADDED to grad_particles (device [N_p]). */
apr_status_t apr_tree_restrict_adjoint(apr_handle_t h, float *grad_tree, float *grad_particles, apr_stream_t stream);

/* apr_tree_restrict_adjoint over the tree levels [level_first, level_last] only (clipped to
 * [l_min, l_max - 1]), coarsest first. Calling it level by level from l_min up to l_max - 1 gives the
 * whole apr_tree_restrict_adjoint; after the call for tree level t the particles of level t + 1 hold
 * their final gradient (their parents are level-t tree nodes), so a caller can copy them out while
 * the finer levels still run. APR_ERR_INVALID_ARG if level_first > level_last. */
apr_status_t apr_tree_restrict_adjoint_levels(apr_handle_t h, float *grad_tree, float *grad_particles,
                                              int32_t level_first, int32_t level_last, apr_stream_t stream);

/* Scratch bytes of apr_convolve_stencil_grad for stencil size k (per-tile partial sums). */
size_t apr_stencil_grad_workspace_bytes(apr_handle_t h, int32_t k);

/* apr_convolve_stencil_grad: grad_stencils[l][e] = sum over particles p of level l of
 * grad_out[p] * u_l(refl(i_p + e)) (device [L][k^3], overwritten), summed in a fixed order.
 * workspace: device scratch of apr_stencil_grad_workspace_bytes(h, k) bytes, 256-byte aligned. */
apr_status_t apr_convolve_stencil_grad(apr_handle_t h, const float *particles, const float *tree, int32_t k, int32_t bc,
                                       const float *grad_out, float *grad_stencils, void *workspace,
                                       size_t workspace_bytes, apr_stream_t stream);

/* apr_convolve_backward for callers that cannot allocate device memory. The paper has no counterpart.
 * Some callers may not call cudaMalloc at all: code running inside a host callback or a framework
 * hook that must not allocate, a process whose device memory is reserved up front by another
 * allocator, or an embedded pipeline with a fixed memory budget. This entry point takes no workspace
 * and allocates nothing (no cudaMalloc, cudaFree or allocating library routine): its scratch is a
 * fixed 16 MiB (16777216-byte) device array inside the library, which every GPU that loads the
 * library holds until the process exits. The caller still passes inputs and outputs, as for
 * apr_convolve_backward, and gets the same results.
 *   - Returns APR_ERR_UNSUPPORTED when apr_backward_workspace_bytes(h, k) exceeds 16 MiB.
 *   - The first call on each device looks up the array's device address with that device current
 *     (cudaGetSymbolAddress). With CUDA's lazy module loading (the default) that first call is also
 *     when the device reserves the 16 MiB, so it can fail with APR_ERR_OOM if other allocators have
 *     taken the memory by then: make the first call at set-up, before other allocators reserve
 *     memory and before any stream capture on that device.
 *   - Every call shares the one array, which keeps the previous call's contents (the call clears what
 *     must start at zero itself). Calls that overlap on the GPU, from any handle or stream, race on it. */
apr_status_t apr_convolve_backward_noalloc(apr_handle_t h, const float *particles, const float *tree,
                                           const float *stencils, int32_t k, int32_t bc, const float *grad_out,
                                           float *grad_particles, float *grad_stencils, apr_stream_t stream);

/* Richardson-Lucy deconvolution on the APR (Sec. 6.2): n_iter iterations of
 *   i_{k+1} = i_k * ((u / (i_k (*) w)) (*) w_flip)
 * where (*) is apr_convolve with the per-level stencils `stencils` (pass the restricted stencils of
 * the PSF, apr_restrict_stencil, for the paper's scheme), w_flip is every level's stencil with its
 * taps reversed in each dimension, and division and multiplication are per particle (the division
 * gives 0 where the denominator is <= 0). Each iteration restricts the tree of i_k and of the ratio.
 * The division and the multiplication run inside the convolution kernel's output write; each
 * restriction and the convolution after it take their launches as apr_convolve_auto does.
 *   observed: device [N_p] float32 (u);  estimate: device [N_p] float32, in: i_0, out: i_n_iter;
 *   stencils: device [L][k^3] float32;  k: 3 or 5;  bc as apr_convolve;
 *   workspace: apr_rl_workspace_bytes(h) bytes, 256-byte aligned (a tree and a ratio buffer). */
size_t apr_rl_workspace_bytes(apr_handle_t h);
apr_status_t apr_richardson_lucy(apr_handle_t h, const float *observed, const float *stencils, int32_t k, int32_t bc,
                                 int32_t n_iter, float *estimate, void *workspace, size_t workspace_bytes,
                                 apr_stream_t stream);

/* ---- Multi-channel convolution with bfloat16 features and weights (the APR CNN layer that Sec. 6
 * proposes: several feature channels per particle, mixed by per-level learned filters). Features are
 * bfloat16 (stored as uint16 bit patterns), channels-last; products are exact and accumulate in FP32
 * on the tensor cores. Supported: channels = c_in = c_out = 16, k = 3. Pointers to features, weights,
 * gradients and outputs must be 16-byte aligned. */

/* BF16 tree restriction: as apr_tree_restrict, per channel, with the arithmetic of the BF16 layer:
 * a node's in-grid children are summed in FP32 in (dz, dx, dy) order, divided by their count in FP32,
 * and the quotient is rounded to bfloat16 (nearest, ties to even) before the next coarser level uses
 * it. particles: device [N_p][channels] bf16; tree: device [N_t][channels] bf16, every entry written.
 * Results are bit-exact. */
apr_status_t apr_tree_restrict_bf16(apr_handle_t h, const uint16_t *particles, uint16_t *tree, int32_t channels,
                                    apr_stream_t stream);

/* Multi-channel APR convolution (Sec. 4.1 per output channel, summed over input channels): for every
 * particle p at level l,
 *   out[p][co] = sum_{ci} sum_{e in [-1,1]^3} weights[l - l_min][co][ci][e] * u_l(refl(i_p + e))[ci],
 * with u_l and the boundary rule as in apr_convolve.
 *   particles: device [N_p][c_in] bf16;  tree: device [N_t][c_in] bf16 from apr_tree_restrict_bf16;
 *   weights:   device [(l_max-l_min+1)][c_out][c_in][k^3] bf16 ([z][x][y] taps, y fastest);
 *   out:       device [N_p][c_out] float32, overwritten.
 * Returns APR_ERR_UNSUPPORTED unless c_in = c_out = 16 and k = 3. A tensor-core wait that does not
 * finish in bounded time records APR_ERR_TIMEOUT for apr_sync_status. */
apr_status_t apr_convolve_mc(apr_handle_t h, const uint16_t *particles, const uint16_t *tree, const uint16_t *weights,
                             int32_t c_in, int32_t c_out, int32_t k, int32_t bc, float *out, apr_stream_t stream);

/* apr_convolve_mc with the hidden-layer activation of an APR CNN fused into the write:
 * out[p][co] = bf16(max(conv[p][co], 0)) (device [N_p][c_out] bf16), instead of the float32 result.
 * For inference (the backward needs the float32 pre-activation). */
apr_status_t apr_convolve_mc_relu_bf16(apr_handle_t h, const uint16_t *particles, const uint16_t *tree,
                                       const uint16_t *weights, int32_t c_in, int32_t c_out, int32_t k, int32_t bc,
                                       uint16_t *out, apr_stream_t stream);

/* Scratch bytes of apr_convolve_mc_backward (tree gradient and per-block weight-gradient partials). */
size_t apr_mc_backward_workspace_bytes(apr_handle_t h, int32_t c_in, int32_t c_out, int32_t k);

/* Adjoint of apr_tree_restrict_bf16 followed by apr_convolve_mc, with the rounding of the tree taken
 * as the identity (the derivative of the exact average). With g = grad_out:
 *   grad_particles[q][ci] = sum over taps that read q (directly, or as the coarse fill of the next
 *        finer level) of sum_co g_p[co] * weights[l][co][ci][e], plus the tree shares as in
 *        apr_convolve_backward;
 *   grad_weights[l][co][ci][e] = sum_{p at level l} g_p[co] * u_l(refl(i_p + e))[ci].
 * grad_out: device [N_p][c_out] bf16 (the caller rounds the incoming FP32 gradient). grad_particles
 * (device [N_p][c_in] float32) and grad_weights (device [L][c_out][c_in][k^3] float32) are
 * overwritten; either may be NULL. workspace: apr_mc_backward_workspace_bytes bytes, 256-byte
 * aligned. Results are deterministic (fixed summation order). */
apr_status_t apr_convolve_mc_backward(apr_handle_t h, const uint16_t *particles, const uint16_t *tree,
                                      const uint16_t *weights, int32_t c_in, int32_t c_out, int32_t k, int32_t bc,
                                      const uint16_t *grad_out, float *grad_particles, float *grad_weights,
                                      void *workspace, size_t workspace_bytes, apr_stream_t stream);

/* ---- Element-wise layers of an APR CNN (Sec. 6: learned per-level filters) around apr_convolve_mc,
 * on per-particle vectors of 16 channels (channels-last [n][16]). They need no handle; n is the
 * number of particles (n_values the number of channel values). All return APR_ERR_INVALID_ARG for
 * negative sizes or missing buffers. bf16 results are rounded to nearest, ties to even. */

/* Input embedding: out[p][0] = bf16(scale * x[p]) (product rounded to float first), out[p][1..15] = 0. */
apr_status_t apr_mc_embed_bf16(const float *x, int64_t n, float scale, uint16_t *out, apr_stream_t stream);

/* Hidden activation: out[i] = bf16(max(in[i], 0)). */
apr_status_t apr_mc_relu_bf16(const float *in, int64_t n_values, uint16_t *out, apr_stream_t stream);

/* Its transpose (the bf16 rounding taken as the identity): grad_pre[i] = bf16(pre[i] > 0 ? grad_post[i] : 0). */
apr_status_t apr_mc_relu_backward_bf16(const float *pre, const float *grad_post, int64_t n_values, uint16_t *grad_pre,
                                       apr_stream_t stream);

/* Residual read-out of the last layer: y[p] = x[p] + inv_scale * conv[p][0] (float32). */
apr_status_t apr_mc_readout(const float *conv, const float *x, int64_t n, float inv_scale, float *y, apr_stream_t stream);

/* Its transpose w.r.t. conv: grad_conv[p][0] = bf16(inv_scale * grad_y[p]), grad_conv[p][1..15] = 0. */
apr_status_t apr_mc_readout_backward_bf16(const float *grad_y, int64_t n, float inv_scale, uint16_t *grad_conv,
                                          apr_stream_t stream);

/* Restricted stencils (Eq. restrict_stenc, K_{w_l} = R_l K_w P_l with block-average R_l and
 * piecewise-constant P_l): out[l - l_min][e] = sum_d w[d] * prod_axes c_s(d_a, e_a), where
 * c_s(d, e) = (1/s) #{x in [0, s): floor((x + d) / s) = e} and s = 2^(l_max - l). Host memory in and
 * out: w [k^3], out [(l_max-l_min+1)][k^3] float32 (computed in double, rounded once). k: 3 or 5. */
apr_status_t apr_restrict_stencil(const float *w, int32_t k, int32_t l_max, int32_t l_min, float *out);

/* Level-rescaled stencils (Eq. adapt_grad): out[l - l_min] = 2^-(l_max - l) * w. Host memory. */
apr_status_t apr_rescale_stencil(const float *w, int32_t k, int32_t l_max, int32_t l_min, float *out);

/* Dense pixel-grid correlation (the dense comparison of the paper's results, Sec. 6.1: a pixel
 * image convolved with a stencil of the same size as the APR one; not part of the APR path):
 * out[z][x][y] = sum_e w[e] img[refl(z + ez)][refl(x + ex)][refl(y + ey)] (or zero outside the
 * image with APR_BC_ZERO), FP32.
 *   image, out: device [dz][dx][dy] float32 (y contiguous); stencil: device [k^3] float32; k: 3 or 5.
 * Returns APR_ERR_UNSUPPORTED for other k or grids of more than 65535 x 8 x columns or 65535 x 32
 * z planes. */
apr_status_t apr_dense_convolve(const float *image, int64_t dz, int64_t dx, int64_t dy, const float *stencil,
                                int32_t k, int32_t bc, float *out, apr_stream_t stream);

/* Host helper (no device): the Sobel derivative stencils of the gradient estimate (Sec. 4.3), out =
 * host [3][k^3] float32 along z, x, y: the central difference (-1/2, 0, 1/2) along the axis times
 * the smoothing (1/4, 1/2, 1/4) across it in both other axes, so a linear ramp of slope 1 gives 1.
 * Pass each through apr_rescale_stencil (Eq. adapt_grad) for apr_gradient_magnitude. k = 3 only
 * (APR_ERR_UNSUPPORTED otherwise). */
apr_status_t apr_sobel_stencils(int32_t k, float *out);

/* Self-test of the device error path (no paper counterpart): launches one block that waits on a
 * barrier nothing will complete, gives up after limit_us microseconds (1 .. 2 000 000) with the
 * same bounded wait the tensor-core kernels use, and records the timeout in the handle's error word,
 * so that the next apr_sync_status returns APR_ERR_TIMEOUT. No fault occurs; the handle and the
 * CUDA context stay usable. */
apr_status_t apr_selftest_bounded_wait(apr_handle_t h, uint32_t limit_us, apr_stream_t stream);

/* Wait for `stream`, then read and clear the handle's device error word. Returns APR_ERR_TIMEOUT if a
 * bounded device wait gave up since the last call, APR_ERR_DEVICE if another device-side check
 * failed, else APR_OK (or APR_ERR_CUDA). */
apr_status_t apr_sync_status(apr_handle_t h, apr_stream_t stream);

const char *apr_status_string(apr_status_t s);

#ifdef __cplusplus
}
#endif
#endif /* APR_H */
