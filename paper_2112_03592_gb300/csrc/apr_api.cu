// C ABI entry points (include/apr.h): handle lifetime, upload of the index, kernel launches.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "apr_internal.h"

namespace aprk {
cudaError_t launch_conv_fwd(int k, const DevLayout &L, const Item *items, int n, const float *vals,
                            const float *tree, const float *st, int bc, float *out, cudaStream_t s,
                            int epi_mode = EPI_PLAIN, bool flip = false, const float *aux = nullptr, int tile0 = 0);
cudaError_t launch_tree_restrict(const TreeNodePlan *np, int node0, int n, const float *vals, float *tree,
                                 cudaStream_t s, int C, int ch, bool pdl);
cudaError_t launch_gradmag(int k, const DevLayout &L, const Item *items, int n, const float *vals, const float *tree,
                           const float *st, int bc, float *out, cudaStream_t s);
cudaError_t launch_bwd_data(int k, const DevLayout &L, const Item *items, int n, const float *st, int bc,
                            const float *gout, float *gp, float *gt, cudaStream_t s, int tile0 = 0);
cudaError_t launch_bwd_stencil(int k, const DevLayout &L, const Item *items, int n, const float *vals,
                               const float *tree, int bc, const float *gout, float *partial, cudaStream_t s);
cudaError_t launch_stencil_reduce(const float *partial, int n_items, const int64_t *level_begin, int l_min,
                                  int n_levels, int K3, float *gw, cudaStream_t s);
cudaError_t launch_tree_pushdown(const TreeNodePlan *np, int node0, int n, float *gp, float *gt, cudaStream_t s,
                                 bool pdl);
cudaError_t launch_conv_fwd_split(const DevLayout &L, const Item *items, int n_lo, const LevelRanges &lo, int *hint,
                                  const float *vals, const float *tree, const float *st, int bc, float *out,
                                  cudaStream_t s, int epi_mode, bool flip, const float *aux);
cudaError_t launch_bwd_data_split(const DevLayout &L, const Item *items, int n_lo, const LevelRanges &lo, int *hint,
                                  const float *st, int bc, const float *gout, float *gp, float *gt, cudaStream_t s);
cudaError_t launch_radius_hint(const DevLayout &L, const LevelRanges &lo, const float *st, int *hint, cudaStream_t s);
}  // namespace aprk

using namespace aprk;

namespace {

thread_local char g_last_msg[256] = "";

// One device block of the handle: from the caller's allocator when one was given, else
// stream-ordered (cudaMallocAsync on the build stream). Every block is recorded for apr_destroy.
cudaError_t dev_alloc(apr_handle_s *h, void **p, size_t bytes) {
    *p = nullptr;
    if (h->has_alloc) {
        *p = h->alloc.alloc(bytes, h->stream, h->alloc.ctx);
        if (!*p) return cudaErrorMemoryAllocation;
        if (reinterpret_cast<uintptr_t>(*p) % 16 != 0) {  // the kernels read the index with 16-byte loads
            h->alloc.free(*p, bytes, h->stream, h->alloc.ctx);
            *p = nullptr;
            return cudaErrorMisalignedAddress;
        }
    } else {
        const cudaError_t e = cudaMallocAsync(p, bytes, reinterpret_cast<cudaStream_t>(h->stream));
        if (e != cudaSuccess) return e;
    }
    h->blocks.emplace_back(*p, bytes);
    h->dev_bytes += bytes;
    return cudaSuccess;
}

// Device copy of n elements on the build stream, the allocation rounded up to a multiple of `pad`
// elements (zeroed tail): the y arrays are read in aligned 8-element packets. The host arrays are
// pageable, so cudaMemcpyAsync has staged them when it returns; the caller may free them.
template <typename T>
cudaError_t upload(apr_handle_s *h, T **dst, const T *src, size_t n, size_t pad = 1) {
    *dst = nullptr;
    const size_t na = ((n ? n : 1) + pad - 1) / pad * pad;
    void *p = nullptr;
    cudaError_t e = dev_alloc(h, &p, na * sizeof(T));
    if (e != cudaSuccess) return e;
    *dst = static_cast<T *>(p);
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(h->stream);
    if (n) e = cudaMemcpyAsync(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && na > n) e = cudaMemsetAsync(*dst + n, 0, (na - n) * sizeof(T), s);
    return e;
}

// Staged value arrays (particles and tree values of the forward-type calls) are read in 16-byte
// vectors: their base addresses must be 16-byte aligned.
bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Releases every device block of the handle (the caller has synchronised the device).
void free_device(apr_handle_s *h) {
    for (const auto &b : h->blocks) {
        if (h->has_alloc) h->alloc.free(b.first, b.second, h->stream, h->alloc.ctx);
        else cudaFree(b.first);
    }
    h->blocks.clear();
}

bool stencil_k_ok(int32_t k) { return k == 3 || k == 5; }

// Work-item ranges of the levels below l_max (begin: fwd_level_begin or bwd_level_begin).
LevelRanges lower_levels(const HostIndex &X, const int64_t *begin) {
    LevelRanges r;
    r.l0 = X.l_min;
    r.n = X.l_max - X.l_min;
    for (int i = 0; i <= r.n; ++i) r.begin[i] = int32_t(begin[X.l_min + i]);
    return r;
}

// `side` enqueues work on the handle's split stream, `main` on the caller's stream s: the split
// stream is forked from s and joined back to it (also when a launch failed, so that a stream capture
// of s ends joined).
template <typename Side, typename Main>
cudaError_t fork_join(apr_handle_t h, cudaStream_t s, Side side, Main main) {
    std::lock_guard<std::mutex> lock(h->split_mu);
    cudaError_t e = cudaSuccess;
    if (!h->split) e = cudaStreamCreateWithFlags(&h->split, cudaStreamNonBlocking);
    if (e == cudaSuccess && !h->ev_split_fork) e = cudaEventCreateWithFlags(&h->ev_split_fork, cudaEventDisableTiming);
    if (e == cudaSuccess && !h->ev_split_join) e = cudaEventCreateWithFlags(&h->ev_split_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_split_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->split, h->ev_split_fork, 0);
    if (e != cudaSuccess) return e;
    const cudaError_t e_side = side(h->split);
    const cudaError_t e_main = main(s);
    e = cudaEventRecord(h->ev_split_join, h->split);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_split_join, 0);
    return e_side != cudaSuccess ? e_side : e_main != cudaSuccess ? e_main : e;
}

// Whether the last radius-split or hinted call of kind `which` (0 convolution, 1 data adjoint) saw a
// level below l_max with taps outside the central 3^3 (read without waiting: it may be older).
bool outer_taps_seen(apr_handle_t h, int which) {
    return static_cast<volatile const int *>(h->h_hint)[which] != 0;
}

// apr_convolve over the whole forward work list (with the Richardson-Lucy epilogues). For k = 5 the
// levels below l_max run split by radius on the split stream (launch_conv_fwd_split) beside the l_max
// tiles, unless the last call's stack had taps outside the central 3^3 below l_max: then one launch
// over all items, with the hint refreshed beside it. Either way every tile is computed the same way.
cudaError_t conv_fwd_all(apr_handle_t h, int k, const float *vals, const float *tree, const float *st, int bc,
                         float *out, cudaStream_t s, int epi_mode = EPI_PLAIN, bool flip = false,
                         const float *aux = nullptr) {
    const HostIndex &X = h->X;
    const int n = int(X.fwd_items.size()), n_lo = int(X.fwd_level_begin[X.l_max]);
    if (k != 5 || n_lo == 0)
        return launch_conv_fwd(k, h->L, h->d_fwd, n, vals, tree, st, bc, out, s, epi_mode, flip, aux);
    const LevelRanges lo = lower_levels(X, X.fwd_level_begin);
    if (outer_taps_seen(h, 0))
        return fork_join(
            h, s, [&](cudaStream_t side) { return launch_radius_hint(h->L, lo, st, h->d_hint, side); },
            [&](cudaStream_t main) { return launch_conv_fwd(k, h->L, h->d_fwd, n, vals, tree, st, bc, out, main, epi_mode, flip, aux); });
    return fork_join(
        h, s,
        [&](cudaStream_t side) {
            return launch_conv_fwd_split(h->L, h->d_fwd, n_lo, lo, h->d_hint, vals, tree, st, bc, out, side, epi_mode,
                                         flip, aux);
        },
        [&](cudaStream_t main) {
            return launch_conv_fwd(k, h->L, h->d_fwd, n - n_lo, vals, tree, st, bc, out, main, epi_mode, flip, aux, n_lo);
        });
}

// The paper's forward pipeline (Sec. 5.2): the tree restriction of `vals` into `tree`, then
// conv_fwd_all. When a 5^3 call is split by radius, its l_max tiles read no tree node (the tree ends
// at level l_max - 1): their launch starts on the split stream beside the restriction, and the
// levels below l_max follow the restriction on s.
apr_status_t restrict_then_conv(apr_handle_t h, int k, const float *vals, float *tree, const float *st, int bc,
                                float *out, cudaStream_t s, int epi_mode = EPI_PLAIN, bool flip = false,
                                const float *aux = nullptr) {
    const HostIndex &X = h->X;
    const int n = int(X.fwd_items.size()), n_lo = int(X.fwd_level_begin[X.l_max]);
    if (k != 5 || n_lo == 0 || n_lo == n || outer_taps_seen(h, 0)) {
        const apr_status_t r = apr_tree_restrict(h, vals, tree, 1, s);
        if (r != APR_OK) return r;
        return cuda_status(conv_fwd_all(h, k, vals, tree, st, bc, out, s, epi_mode, flip, aux));
    }
    const LevelRanges lo = lower_levels(X, X.fwd_level_begin);
    apr_status_t r = APR_OK;
    const cudaError_t e = fork_join(
        h, s,
        [&](cudaStream_t side) {
            return launch_conv_fwd(k, h->L, h->d_fwd, n - n_lo, vals, tree, st, bc, out, side, epi_mode, flip, aux, n_lo);
        },
        [&](cudaStream_t main) {
            r = apr_tree_restrict(h, vals, tree, 1, main);
            if (r != APR_OK) return cudaSuccess;
            return launch_conv_fwd_split(h->L, h->d_fwd, n_lo, lo, h->d_hint, vals, tree, st, bc, out, main, epi_mode,
                                         flip, aux);
        });
    if (r != APR_OK) return r;
    return cuda_status(e);
}

// The data adjoint over the whole adjoint work list; with `split`, k = 5 chooses its launches like
// conv_fwd_all.
cudaError_t bwd_data_all(apr_handle_t h, int k, const float *st, int bc, const float *gout, float *gp, float *gt,
                         cudaStream_t s, bool split) {
    const HostIndex &X = h->X;
    const int n = int(X.bwd_items.size()), n_lo = int(X.bwd_level_begin[X.l_max]);
    if (!split || k != 5 || n_lo == 0) return launch_bwd_data(k, h->L, h->d_bwd, n, st, bc, gout, gp, gt, s);
    const LevelRanges lo = lower_levels(X, X.bwd_level_begin);
    if (outer_taps_seen(h, 1))
        return fork_join(
            h, s, [&](cudaStream_t side) { return launch_radius_hint(h->L, lo, st, h->d_hint + 1, side); },
            [&](cudaStream_t main) { return launch_bwd_data(k, h->L, h->d_bwd, n, st, bc, gout, gp, gt, main); });
    return fork_join(
        h, s,
        [&](cudaStream_t side) {
            return launch_bwd_data_split(h->L, h->d_bwd, n_lo, lo, h->d_hint + 1, st, bc, gout, gp, gt, side);
        },
        [&](cudaStream_t main) { return launch_bwd_data(k, h->L, h->d_bwd, n - n_lo, st, bc, gout, gp, gt, main, n_lo); });
}

// The tree push-down (apr_tree_restrict_adjoint) of the tree levels [l0, l1] within [l_min, l_max - 1],
// coarsest first, one launch per level.
apr_status_t pushdown_levels(apr_handle_t h, float *grad_tree, float *grad_particles, int l0, int l1,
                             cudaStream_t s) {
    const HostIndex &X = h->X;
    if ((X.nt && !grad_tree) || (X.np && !grad_particles)) return APR_ERR_INVALID_ARG;
    if (l0 < X.l_min) l0 = X.l_min;
    if (l1 > X.l_max - 1) l1 = X.l_max - 1;
    cudaError_t e = cudaSuccess;
    bool chained = false;   // the launches after the first start early (programmatic dependent launch)
    for (int l = l0; e == cudaSuccess && l <= l1; ++l) {
        int64_t b = 0, n = 0;
        tree_level_nodes(X, l, b, n);
        e = launch_tree_pushdown(h->d_tnplan, int(b), int(n), grad_particles, grad_tree, s, chained);
        chained = chained || n > 0;
    }
    return cuda_status(e);
}

apr_status_t misaligned() {
    aprk::set_last_message("staged value arrays (particles, tree values) must be 16-byte aligned");
    return APR_ERR_INVALID_ARG;
}

}  // namespace

namespace aprk {
void set_last_message(const char *msg) { snprintf(g_last_msg, sizeof(g_last_msg), "%s", msg); }

cudaError_t set_max_dynamic_smem(const void *fn, size_t bytes) {
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    for (const auto &d : done)
        if (d.first == fn && d.second == dev) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e == cudaSuccess) done.emplace_back(fn, dev);
    return e;
}

apr_status_t cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return APR_OK;
    if (e == cudaErrorMemoryAllocation) return APR_ERR_OOM;
    snprintf(g_last_msg, sizeof(g_last_msg), "%s", cudaGetErrorString(e));
    return APR_ERR_CUDA;
}
}  // namespace aprk

extern "C" {

const char *apr_status_string(apr_status_t s) {
    switch (s) {
        case APR_OK: return "ok";
        case APR_ERR_INVALID_ARG: return "invalid argument";
        case APR_ERR_INVALID_LAYOUT: return "invalid APR layout";
        case APR_ERR_UNSUPPORTED: return "unsupported";
        case APR_ERR_OOM: return "out of memory";
        case APR_ERR_CUDA: return "CUDA error";
        case APR_ERR_TIMEOUT: return "device wait timed out";
        case APR_ERR_DEVICE: return "device-side check failed";
    }
    return "unknown status";
}

// Reason of the last failure on this thread (build errors, CUDA messages); not part of apr.h.
const char *apr_last_error_message(void) { return g_last_msg; }

apr_status_t apr_build_device(const apr_host_layout *layout, uint32_t flags, apr_stream_t stream, apr_handle_t *out) {
    return apr_build_device_ex(layout, flags, stream, nullptr, out);
}

apr_status_t apr_build_device_ex(const apr_host_layout *layout, uint32_t flags, apr_stream_t stream,
                                 const apr_allocator *allocator, apr_handle_t *out) {
    if (!out) return APR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!layout || (flags & ~(APR_VALIDATE | APR_REQUIRE_BALANCE | APR_HOST_ONLY | APR_SUBDOMAIN))) return APR_ERR_INVALID_ARG;
    if (allocator && (!allocator->alloc || !allocator->free)) return APR_ERR_INVALID_ARG;
    apr_handle_s *h = new (std::nothrow) apr_handle_s();
    if (!h) return APR_ERR_OOM;
    h->stream = stream;
    if (allocator) {
        h->alloc = *allocator;
        h->has_alloc = true;
    }
    const char *msg = "";
    apr_status_t st;
    try {
        st = build_index(*layout, flags, h->X, &msg);
    } catch (const std::bad_alloc &) {
        st = APR_ERR_OOM;
        msg = "host allocation failed";
    }
    if (st != APR_OK) {
        snprintf(g_last_msg, sizeof(g_last_msg), "%s", msg);
        delete h;
        return st;
    }
    h->host_only = (flags & APR_HOST_ONLY) != 0;
    if (h->host_only) {
        // the tree-node child maps, for apr_export_structure (a device handle builds them with its plans)
        try {
            tree_node_plan(host_layout_view(h->X), h->X, h->X.tnplan);
        } catch (const std::bad_alloc &) {
            snprintf(g_last_msg, sizeof(g_last_msg), "%s", "host allocation failed (tree-node child maps)");
            delete h;
            return APR_ERR_OOM;
        }
    }
    if (!h->host_only) {
        const apr_status_t pst = build_plans(h->X);
        if (pst != APR_OK) {
            snprintf(g_last_msg, sizeof(g_last_msg), "%s", pst == APR_ERR_OOM ? "host allocation failed (tile plans)"
                                                                                : "tile with too many staged elements, or more than 2^28 particles or tree nodes");
            delete h;
            return pst;
        }
        const HostIndex &X = h->X;
        cudaError_t e = cudaSuccess;
        if (e == cudaSuccess) e = upload(h, &h->d_row_ptr, X.row_ptr.data(), X.row_ptr.size());
        if (e == cudaSuccess) e = upload(h, &h->d_y, X.y.data(), X.y.size(), 8);
        if (e == cudaSuccess) e = upload(h, &h->d_off, X.off.data(), X.off.size());
        if (e == cudaSuccess) e = upload(h, &h->d_trow_ptr, X.trow_ptr.data(), X.trow_ptr.size());
        if (e == cudaSuccess) e = upload(h, &h->d_ty, X.ty.data(), X.ty.size(), 8);
        if (e == cudaSuccess) e = upload(h, &h->d_toff, X.toff.data(), X.toff.size());
        if (e == cudaSuccess) e = upload(h, &h->d_fwd, X.fwd_items.data(), X.fwd_items.size());
        if (e == cudaSuccess) e = upload(h, &h->d_bwd, X.bwd_items.data(), X.bwd_items.size());
        if (e == cudaSuccess) e = upload(h, &h->d_tree, X.tree_items.data(), X.tree_items.size());
        if (e == cudaSuccess) e = upload(h, &h->d_tnplan, X.tnplan.data(), X.tnplan.size());
        if (e == cudaSuccess) e = upload(h, &h->d_fwd_level_begin, X.fwd_level_begin, size_t(MAXL + 1));
        for (int i = 0; i < 4 && e == cudaSuccess; ++i) {
            const HostFPlan &P = i < 2 ? X.fplan[i] : X.bplan[i - 2];
            e = upload(h, &h->d_fplan_hdr[i], P.hdr.data(), P.hdr.size());
            if (e == cudaSuccess) e = upload(h, &h->d_fplan_ent[i], P.ent.data(), P.ent.size());
        }
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
            const HostPlan &P = i == 0 ? X.mcfplan : X.mcbplan;
            e = upload(h, &h->d_plan_hdr[i], P.hdr.data(), P.hdr.size());
            if (e == cudaSuccess) e = upload(h, &h->d_plan_ent[i], P.ent.data(), P.ent.size());
        }
        if (e == cudaSuccess) {
            void *p = nullptr;
            e = dev_alloc(h, &p, sizeof(unsigned));
            h->d_err = static_cast<unsigned *>(p);
            if (e == cudaSuccess) e = cudaMemsetAsync(h->d_err, 0, sizeof(unsigned), reinterpret_cast<cudaStream_t>(stream));
        }

        if (e == cudaSuccess) {
            // operand-layout copy of multi-channel weights: [2 (plain, transposed)][levels][27 * 16 * 16]
            const size_t nb = size_t(2) * size_t(X.l_max - X.l_min + 1) * 27 * 16 * 16 * sizeof(uint16_t);
            void *p = nullptr;
            e = dev_alloc(h, &p, nb);
            h->d_mcw = static_cast<uint16_t *>(p);
        }
        if (e != cudaSuccess) {
            st = cuda_status(e);
            cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
            free_device(h);
            delete h;
            return st;
        }
        DevLayout &L = h->L;
        L.row_ptr = h->d_row_ptr;
        L.y = h->d_y;
        L.off = h->d_off;
        L.trow_ptr = h->d_trow_ptr;
        L.ty = h->d_ty;
        L.toff = h->d_toff;
        L.err = h->d_err;
        L.np = int32_t(X.np);
        L.nt = int32_t(X.nt);
        L.l_min = X.l_min;
        L.l_max = X.l_max;
        for (int l = 0; l < MAXL; ++l) L.geo[l] = X.geo[l];
        for (int i = 0; i < 2; ++i) {
            L.fplan[i] = FPlanView{h->d_fplan_hdr[i], h->d_fplan_ent[i]};
            L.bplan[i] = FPlanView{h->d_fplan_hdr[2 + i], h->d_fplan_ent[2 + i]};
        }
        L.mcfplan = PlanView{h->d_plan_hdr[0], h->d_plan_ent[0]};
        L.mcbplan = PlanView{h->d_plan_hdr[1], h->d_plan_ent[1]};
        // the plans live on the device now; the host copies are not needed again
        for (int i = 0; i < 2; ++i) {
            h->X.fplan[i] = HostFPlan{};
            h->X.bplan[i] = HostFPlan{};
        }
        h->X.mcfplan = HostPlan{};
        h->X.mcbplan = HostPlan{};
        h->X.tnplan = std::vector<TreeNodePlan>{};
        // the second streams of apr_convolve_backward and of the radius split, and their events, are
        // made here, so that no later call creates them inside a stream capture
        e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->split, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_split_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_split_join, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&h->h_hint), 2 * sizeof(int), cudaHostAllocMapped);
        if (e == cudaSuccess) {
            h->h_hint[0] = h->h_hint[1] = 0;
            e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&h->d_hint), h->h_hint, 0);
        }
        if (e != cudaSuccess) {
            st = cuda_status(e);
            apr_destroy(h);
            return st;
        }
    }
    *out = h;
    return APR_OK;
}

apr_status_t apr_destroy(apr_handle_t h) {
    if (!h) return APR_OK;
    if (!h->host_only) {
        cudaDeviceSynchronize();
        free_device(h);
        if (h->ev_fork) cudaEventDestroy(h->ev_fork);
        if (h->ev_join) cudaEventDestroy(h->ev_join);
        if (h->side) cudaStreamDestroy(h->side);
        if (h->ev_split_fork) cudaEventDestroy(h->ev_split_fork);
        if (h->ev_split_join) cudaEventDestroy(h->ev_split_join);
        if (h->split) cudaStreamDestroy(h->split);
        if (h->h_hint) cudaFreeHost(h->h_hint);
    }
    delete h;
    return APR_OK;
}

int64_t apr_num_particles(apr_handle_t h) { return h ? h->X.np : -1; }
int64_t apr_num_tree(apr_handle_t h) { return h ? h->X.nt : -1; }

apr_status_t apr_level_range(apr_handle_t h, int32_t *l_min, int32_t *l_max) {
    if (!h || !l_min || !l_max) return APR_ERR_INVALID_ARG;
    *l_min = h->X.l_min;
    *l_max = h->X.l_max;
    return APR_OK;
}

size_t apr_layout_bytes(apr_handle_t h) { return h ? h->dev_bytes : 0; }

namespace {
// The tile plans of a host-only handle (built once, on request); nullptr for a device handle, whose
// plans live only on the device.
const HostFPlan *host_plan(apr_handle_t h, int32_t which) {
    if (!h->host_only || which < APR_STRUCT_FWD_PLAN_R1 || which > APR_STRUCT_BWD_PLAN_R2) return nullptr;
    std::lock_guard<std::mutex> lk(h->plan_mu);
    if (!h->host_plans) {
        if (build_plans(h->X) != APR_OK) return nullptr;
        h->host_plans = true;
    }
    const int i = which - APR_STRUCT_FWD_PLAN_R1;
    return i < 2 ? &h->X.fplan[i] : &h->X.bplan[i - 2];
}
}  // namespace

size_t apr_structure_bytes(apr_handle_t h, int32_t which) {
    if (!h) return 0;
    const HostIndex &X = h->X;
    if (which >= APR_STRUCT_FWD_PLAN_R1 && which <= APR_STRUCT_BWD_PLAN_R2) {
        const HostFPlan *P = host_plan(h, which);
        return P ? (P->hdr.size() + P->ent.size()) * sizeof(uint2) : 0;
    }
    switch (which) {
        case APR_STRUCT_ROW_PTR: return X.row_ptr.size() * sizeof(uint32_t);
        case APR_STRUCT_Y_IDX: return X.y.size() * sizeof(uint16_t);
        case APR_STRUCT_TREE_ROW_PTR: return X.trow_ptr.size() * sizeof(uint32_t);
        case APR_STRUCT_TREE_Y_IDX: return X.ty.size() * sizeof(uint16_t);
        case APR_STRUCT_FWD_ITEMS: return X.fwd_items.size() * sizeof(Item);
        case APR_STRUCT_TREE_ITEMS: return X.tree_items.size() * sizeof(Item);
        case APR_STRUCT_BWD_ITEMS: return X.bwd_items.size() * sizeof(Item);
        case APR_STRUCT_TREE_NODE_MAP: return size_t(X.nt) * sizeof(TreeNodePlan);
    }
    return 0;
}

apr_status_t apr_export_structure(apr_handle_t h, int32_t which, void *dst, size_t bytes) {
    if (!h || (!dst && bytes)) return APR_ERR_INVALID_ARG;
    const size_t need = apr_structure_bytes(h, which);
    if (which < APR_STRUCT_ROW_PTR || which > APR_STRUCT_BWD_PLAN_R2) return APR_ERR_INVALID_ARG;
    if (bytes < need) return APR_ERR_INVALID_ARG;
    if (need == 0) return APR_OK;
    if (which >= APR_STRUCT_FWD_PLAN_R1) {  // host-only handle (need > 0)
        const HostFPlan *P = host_plan(h, which);
        memcpy(dst, P->hdr.data(), P->hdr.size() * sizeof(PlanHdr));
        memcpy(static_cast<char *>(dst) + P->hdr.size() * sizeof(PlanHdr), P->ent.data(), P->ent.size() * sizeof(uint2));
        return APR_OK;
    }
    const HostIndex &X = h->X;
    const void *host_src = nullptr;
    const void *dev_src = nullptr;
    switch (which) {
        case APR_STRUCT_ROW_PTR: host_src = X.row_ptr.data(); dev_src = h->d_row_ptr; break;
        case APR_STRUCT_Y_IDX: host_src = X.y.data(); dev_src = h->d_y; break;
        case APR_STRUCT_TREE_ROW_PTR: host_src = X.trow_ptr.data(); dev_src = h->d_trow_ptr; break;
        case APR_STRUCT_TREE_Y_IDX: host_src = X.ty.data(); dev_src = h->d_ty; break;
        case APR_STRUCT_FWD_ITEMS: host_src = X.fwd_items.data(); dev_src = h->d_fwd; break;
        case APR_STRUCT_TREE_ITEMS: host_src = X.tree_items.data(); dev_src = h->d_tree; break;
        case APR_STRUCT_TREE_NODE_MAP: host_src = X.tnplan.data(); dev_src = h->d_tnplan; break;
        case APR_STRUCT_BWD_ITEMS: host_src = X.bwd_items.data(); dev_src = h->d_bwd; break;
    }
    if (h->host_only) {
        memcpy(dst, host_src, need);
        return APR_OK;
    }
    // the device copy is the one the kernels read (uploaded on the build stream)
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(h->stream));
    if (e == cudaSuccess) e = cudaMemcpy(dst, dev_src, need, cudaMemcpyDeviceToHost);
    return cuda_status(e);
}

apr_status_t apr_tree_restrict(apr_handle_t h, const float *particles, float *tree, int32_t channels,
                               apr_stream_t stream) {
    if (!h || h->host_only) return APR_ERR_INVALID_ARG;
    if (channels < 1 || channels > 64) return APR_ERR_INVALID_ARG;
    if ((!particles && h->X.np) || (!tree && h->X.nt)) return APR_ERR_INVALID_ARG;
    const HostIndex &X = h->X;
    bool chained = false;   // the launches after the first start early (programmatic dependent launch)
    for (int l = X.l_max - 1; l >= X.l_min; --l) {
        int64_t b = 0, n = 0;
        tree_level_nodes(X, l, b, n);
        for (int c = 0; c < channels; ++c) {  // channels-last values: one strided pass per channel
            cudaError_t e = launch_tree_restrict(h->d_tnplan, int(b), int(n), particles, tree, stream, channels, c,
                                                 chained);
            chained = chained || n > 0;
            if (e != cudaSuccess) return cuda_status(e);
        }
    }
    return APR_OK;
}

apr_status_t apr_convolve(apr_handle_t h, const float *particles, const float *tree, const float *stencils,
                          int32_t k, int32_t bc, float *out, apr_stream_t stream) {
    if (!h || h->host_only) return APR_ERR_INVALID_ARG;
    if (!stencil_k_ok(k)) return APR_ERR_UNSUPPORTED;
    if (bc != APR_BC_REFLECT && bc != APR_BC_ZERO) return APR_ERR_INVALID_ARG;
    if (!stencils || (h->X.np && (!particles || !out)) || (h->X.nt && !tree)) return APR_ERR_INVALID_ARG;
    if (!aligned16(particles) || !aligned16(tree)) return misaligned();
    return cuda_status(conv_fwd_all(h, k, particles, tree, stencils, bc, out, stream));
}

apr_status_t apr_convolve_tiles(apr_handle_t h, const float *particles, const float *tree, const float *stencils,
                                int32_t k, int32_t bc, float *out, int64_t first_tile, int64_t n_tiles,
                                apr_stream_t stream) {
    if (!h || h->host_only) return APR_ERR_INVALID_ARG;
    if (!stencil_k_ok(k)) return APR_ERR_UNSUPPORTED;
    if (bc != APR_BC_REFLECT && bc != APR_BC_ZERO) return APR_ERR_INVALID_ARG;
    const int64_t nt = int64_t(h->X.fwd_items.size());
    if (first_tile < 0 || n_tiles < 0 || first_tile + n_tiles > nt) return APR_ERR_INVALID_ARG;
    if (!stencils || (h->X.np && (!particles || !out)) || (h->X.nt && !tree)) return APR_ERR_INVALID_ARG;
    if (!aligned16(particles) || !aligned16(tree)) return misaligned();
    return cuda_status(launch_conv_fwd(k, h->L, h->d_fwd, int(n_tiles), particles, tree, stencils, bc, out, stream,
                                       EPI_PLAIN, false, nullptr, int(first_tile)));
}

apr_status_t apr_convolve_adjoint_tiles(apr_handle_t h, const float *stencils, int32_t k, int32_t bc,
                                        const float *grad_out, float *grad_particles, float *grad_tree,
                                        int64_t first_tile, int64_t n_tiles, apr_stream_t stream) {
    if (!h || h->host_only) return APR_ERR_INVALID_ARG;
    if (!stencil_k_ok(k)) return APR_ERR_UNSUPPORTED;
    if (bc != APR_BC_REFLECT && bc != APR_BC_ZERO) return APR_ERR_INVALID_ARG;
    const HostIndex &X = h->X;
    const int64_t nt = int64_t(X.bwd_items.size());
    if (first_tile < 0 || n_tiles < 0 || first_tile + n_tiles > nt) return APR_ERR_INVALID_ARG;
    if (!stencils || (X.np && (!grad_out || !grad_particles)) || (X.nt && !grad_tree)) return APR_ERR_INVALID_ARG;
    return cuda_status(launch_bwd_data(k, h->L, h->d_bwd, int(n_tiles), stencils, bc, grad_out, grad_particles,
                                       grad_tree, stream, int(first_tile)));
}

size_t apr_convolve_auto_workspace_bytes(apr_handle_t h) {
    return h ? size_t(h->X.nt > 0 ? h->X.nt : 1) * sizeof(float) : 0;
}

apr_status_t apr_convolve_auto(apr_handle_t h, const float *particles, const float *stencils, int32_t k, int32_t bc,
                               float *out, void *workspace, size_t workspace_bytes, apr_stream_t stream) {
    if (!h || h->host_only) return APR_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < apr_convolve_auto_workspace_bytes(h) ||
        !aligned16(workspace))
        return APR_ERR_INVALID_ARG;
    if (!stencil_k_ok(k)) return APR_ERR_UNSUPPORTED;
    if (bc != APR_BC_REFLECT && bc != APR_BC_ZERO) return APR_ERR_INVALID_ARG;
    if (!stencils || (h->X.np && (!particles || !out))) return APR_ERR_INVALID_ARG;
    if (!aligned16(particles)) return misaligned();
    return restrict_then_conv(h, k, particles, static_cast<float *>(workspace), stencils, bc, out, stream);
}

apr_status_t apr_gradient_magnitude(apr_handle_t h, const float *particles, const float *tree, const float *stencils,
                                    int32_t k, int32_t bc, float *out, apr_stream_t stream) {
    if (!h || h->host_only) return APR_ERR_INVALID_ARG;
    if (!stencil_k_ok(k)) return APR_ERR_UNSUPPORTED;
    if (bc != APR_BC_REFLECT && bc != APR_BC_ZERO) return APR_ERR_INVALID_ARG;
    if (!stencils || (h->X.np && (!particles || !out)) || (h->X.nt && !tree)) return APR_ERR_INVALID_ARG;
    if (!aligned16(particles) || !aligned16(tree)) return misaligned();
    const int n = int(h->X.fwd_items.size());
    return cuda_status(launch_gradmag(k, h->L, h->d_fwd, n, particles, tree, stencils, bc, out, stream));
}

size_t apr_backward_workspace_bytes(apr_handle_t h, int32_t k) {
    if (!h || !stencil_k_ok(k)) return 0;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    return al(size_t(h->X.nt) * sizeof(float)) + al(h->X.fwd_items.size() * size_t(k * k * k) * sizeof(float));
}

apr_status_t apr_convolve_adjoint(apr_handle_t h, const float *stencils, int32_t k, int32_t bc, const float *grad_out,
                                  float *grad_particles, float *grad_tree, apr_stream_t stream) {
    return aprk::convolve_adjoint(h, stencils, k, bc, grad_out, grad_particles, grad_tree, stream, true);
}

apr_status_t apr_tree_restrict_adjoint(apr_handle_t h, float *grad_tree, float *grad_particles, apr_stream_t stream) {
    if (!h || h->host_only) return APR_ERR_INVALID_ARG;
    return pushdown_levels(h, grad_tree, grad_particles, h->X.l_min, h->X.l_max - 1, stream);
}

apr_status_t apr_tree_restrict_adjoint_levels(apr_handle_t h, float *grad_tree, float *grad_particles,
                                              int32_t level_first, int32_t level_last, apr_stream_t stream) {
    if (!h || h->host_only || level_first > level_last) return APR_ERR_INVALID_ARG;
    return pushdown_levels(h, grad_tree, grad_particles, level_first, level_last, stream);
}

size_t apr_stencil_grad_workspace_bytes(apr_handle_t h, int32_t k) {
    if (!h || !stencil_k_ok(k)) return 0;
    return (h->X.fwd_items.size() * size_t(k * k * k) * sizeof(float) + 255) / 256 * 256;
}

apr_status_t apr_convolve_stencil_grad(apr_handle_t h, const float *particles, const float *tree, int32_t k, int32_t bc,
                                       const float *grad_out, float *grad_stencils, void *workspace,
                                       size_t workspace_bytes, apr_stream_t stream) {
    if (!h || h->host_only) return APR_ERR_INVALID_ARG;
    if (!stencil_k_ok(k)) return APR_ERR_UNSUPPORTED;
    if (bc != APR_BC_REFLECT && bc != APR_BC_ZERO) return APR_ERR_INVALID_ARG;
    const HostIndex &X = h->X;
    if (!grad_stencils || (X.np && (!particles || !grad_out)) || (X.nt && !tree)) return APR_ERR_INVALID_ARG;
    if (!aligned16(particles) || !aligned16(tree)) return misaligned();
    const size_t need = apr_stencil_grad_workspace_bytes(h, k);
    if (need && (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255))) return APR_ERR_INVALID_ARG;
    const int n = int(X.fwd_items.size());
    float *partial = static_cast<float *>(workspace);
    cudaError_t e = launch_bwd_stencil(k, h->L, h->d_fwd, n, particles, tree, bc, grad_out, partial, stream);
    if (e == cudaSuccess)
        e = launch_stencil_reduce(partial, n, h->d_fwd_level_begin, X.l_min, X.l_max - X.l_min + 1, k * k * k, grad_stencils, stream);
    return cuda_status(e);
}

}  // extern "C"

namespace aprk {
apr_status_t convolve_adjoint(apr_handle_t h, const float *stencils, int32_t k, int32_t bc, const float *grad_out,
                              float *grad_particles, float *grad_tree, apr_stream_t stream, bool split) {
    if (!h || h->host_only) return APR_ERR_INVALID_ARG;
    if (!stencil_k_ok(k)) return APR_ERR_UNSUPPORTED;
    if (bc != APR_BC_REFLECT && bc != APR_BC_ZERO) return APR_ERR_INVALID_ARG;
    const HostIndex &X = h->X;
    if (!stencils || (X.np && (!grad_out || !grad_particles)) || (X.nt && !grad_tree)) return APR_ERR_INVALID_ARG;
    cudaError_t e = cudaSuccess;
    if (X.np) e = cudaMemsetAsync(grad_particles, 0, size_t(X.np) * sizeof(float), stream);
    if (e == cudaSuccess && X.nt) e = cudaMemsetAsync(grad_tree, 0, size_t(X.nt) * sizeof(float), stream);
    if (e == cudaSuccess)
        e = bwd_data_all(h, k, stencils, bc, grad_out, grad_particles, grad_tree, stream, split);
    return cuda_status(e);
}

apr_status_t convolve_backward(apr_handle_t h, const float *particles, const float *tree, const float *stencils,
                               int32_t k, int32_t bc, const float *grad_out, float *grad_particles,
                               float *grad_stencils, void *workspace, size_t workspace_bytes, apr_stream_t stream,
                               bool concurrent) {
    if (!h || h->host_only) return APR_ERR_INVALID_ARG;
    if (!stencil_k_ok(k)) return APR_ERR_UNSUPPORTED;
    if (bc != APR_BC_REFLECT && bc != APR_BC_ZERO) return APR_ERR_INVALID_ARG;
    const HostIndex &X = h->X;
    if (!stencils || (X.np && !grad_out)) return APR_ERR_INVALID_ARG;
    if (grad_stencils && ((X.np && !particles) || (X.nt && !tree))) return APR_ERR_INVALID_ARG;
    const size_t need = apr_backward_workspace_bytes(h, k);
    if (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) return APR_ERR_INVALID_ARG;
    const size_t gt_bytes = (size_t(X.nt) * sizeof(float) + 255) / 256 * 256;
    float *gt = static_cast<float *>(workspace);
    void *partial = static_cast<char *>(workspace) + gt_bytes;
    apr_status_t st = APR_OK;
    if (concurrent && grad_particles && grad_stencils) {
        // the stencil gradient reads only the values, the tree and dL/dout: it runs on the handle's
        // second stream while the data adjoint and the tree adjoint run on the caller's (their
        // workspace regions are disjoint); the caller's stream then waits for it
        std::lock_guard<std::mutex> lock(h->side_mu);
        cudaError_t e = cudaSuccess;
        if (!h->side) e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
        if (e == cudaSuccess && !h->ev_fork) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess && !h->ev_join) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
        const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side, h->ev_fork, 0);
        if (e != cudaSuccess) return cuda_status(e);
        const apr_status_t sg = apr_convolve_stencil_grad(h, particles, tree, k, bc, grad_out, grad_stencils, partial,
                                                          workspace_bytes - gt_bytes, reinterpret_cast<apr_stream_t>(h->side));
        st = convolve_adjoint(h, stencils, k, bc, grad_out, grad_particles, gt, stream, true);
        if (st == APR_OK) st = apr_tree_restrict_adjoint(h, gt, grad_particles, stream);
        // always joined, so that a stream capture of the caller's stream ends joined
        e = cudaEventRecord(h->ev_join, h->side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_join, 0);
        if (st == APR_OK) st = sg;
        if (st == APR_OK && e != cudaSuccess) st = cuda_status(e);
        return st;
    }
    if (grad_particles) {
        st = convolve_adjoint(h, stencils, k, bc, grad_out, grad_particles, gt, stream, concurrent);
        if (st == APR_OK) st = apr_tree_restrict_adjoint(h, gt, grad_particles, stream);
    }
    if (st == APR_OK && grad_stencils)
        st = apr_convolve_stencil_grad(h, particles, tree, k, bc, grad_out, grad_stencils, partial,
                                       workspace_bytes - gt_bytes, stream);
    return st;
}
}  // namespace aprk

extern "C" {

apr_status_t apr_convolve_backward(apr_handle_t h, const float *particles, const float *tree, const float *stencils,
                                   int32_t k, int32_t bc, const float *grad_out, float *grad_particles,
                                   float *grad_stencils, void *workspace, size_t workspace_bytes,
                                   apr_stream_t stream) {
    return aprk::convolve_backward(h, particles, tree, stencils, k, bc, grad_out, grad_particles, grad_stencils,
                                   workspace, workspace_bytes, stream, true);
}

size_t apr_rl_workspace_bytes(apr_handle_t h) {
    if (!h) return 0;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    return al(size_t(h->X.nt) * sizeof(float)) + al(size_t(h->X.np) * sizeof(float));
}

apr_status_t apr_richardson_lucy(apr_handle_t h, const float *observed, const float *stencils, int32_t k, int32_t bc,
                                 int32_t n_iter, float *estimate, void *workspace, size_t workspace_bytes,
                                 apr_stream_t stream) {
    if (!h || h->host_only) return APR_ERR_INVALID_ARG;
    if (!stencil_k_ok(k)) return APR_ERR_UNSUPPORTED;
    if (bc != APR_BC_REFLECT && bc != APR_BC_ZERO) return APR_ERR_INVALID_ARG;
    const HostIndex &X = h->X;
    if (n_iter < 0 || !stencils || (X.np && (!observed || !estimate))) return APR_ERR_INVALID_ARG;
    if (!aligned16(estimate)) return misaligned();
    const size_t need = apr_rl_workspace_bytes(h);
    if (need && (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)))
        return APR_ERR_INVALID_ARG;
    float *tree = static_cast<float *>(workspace);
    float *ratio = reinterpret_cast<float *>(static_cast<char *>(workspace) + (size_t(X.nt) * sizeof(float) + 255) / 256 * 256);
    for (int it = 0; it < n_iter; ++it) {
        // ratio = u / (i_k conv w); i_{k+1} = i_k * (ratio conv w_flipped); each convolution with the
        // tree restriction of its input before it
        apr_status_t st = restrict_then_conv(h, k, estimate, tree, stencils, bc, ratio, stream, EPI_DIVIDE, false, observed);
        if (st != APR_OK) return st;
        st = restrict_then_conv(h, k, ratio, tree, stencils, bc, estimate, stream, EPI_MULTIPLY, true, estimate);
        if (st != APR_OK) return st;
    }
    return APR_OK;
}

apr_status_t apr_sync_status(apr_handle_t h, apr_stream_t stream) {
    if (!h) return APR_ERR_INVALID_ARG;
    if (h->host_only) return APR_OK;
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_status(e);
    unsigned v = 0;
    e = cudaMemcpy(&v, h->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    if (v) {
        cudaMemset(h->d_err, 0, sizeof(unsigned));
        return (v & ERR_TIMEOUT) ? APR_ERR_TIMEOUT : APR_ERR_DEVICE;
    }
    return APR_OK;
}

}  // extern "C"
