// Multi-core FP32 CPU implementation of APR-native convolution (arXiv 2112.03592), the CPU
// counterpart of the paper's OpenMP comparison (Sec. 5.1: rows of a level processed in parallel).
// It is a measurement baseline for bench.py: written independently of the FP64 oracle and of the
// CUDA library (no shared code), FP32 arithmetic (the stencil-gradient partial sums in FP64).
//
// Work is distributed over the host threads in chunks of rows taken from an atomic counter (the
// dynamic scheduling of an OpenMP loop over the rows of one level); std::thread keeps the build
// free of an OpenMP runtime.
//
// Definitions (the paper's, with the same readings as the GPU path):
//  - APR: particles per level l in rows (z, x) sorted by y (Alg. 1 linear access); level grids
//    d_l = ceil(D / 2^(l_max - l)).
//  - APR tree (Sec. 3.4): the parents of every particle and tree node of level l + 1, valued by the
//    mean of their in-grid children.
//  - û_l(c) (Sec. 3.5): the level-l particle at c, else the level-l tree node, else the level-(l-1)
//    particle containing c (2:1 balance).
//  - convolution (Sec. 4.1): o_p = sum_e w_l[e] û_l(refl(p + e)), correlation form, half-sample
//    reflection (or zero outside the grid).
//  - backward: transpose of the convolution through û and the tree average, and the stencil
//    gradient sum_p g_p û_l(refl(p + e)).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>
#include <thread>
#include <vector>

namespace {

struct Level {
    int64_t dz = 0, dx = 0, dy = 0;
    std::vector<int64_t> prow;   // particle row starts [dz*dx + 1] (global particle indices)
    std::vector<int64_t> trow;   // tree row starts [dz*dx + 1] (global tree indices), levels < l_max
};

struct Apr {
    int l_min = 0, l_max = 0;
    int64_t np = 0, nt = 0;
    std::vector<Level> lv;        // indexed by level
    std::vector<int32_t> py;      // particle y
    std::vector<int32_t> ty;      // tree y
    std::vector<int8_t> tnch;     // tree node: number of in-grid children
};

int64_t cells(int64_t D, int l_max, int l) {
    const int64_t s = int64_t(1) << (l_max - l);
    return (D + s - 1) / s;
}

int64_t refl(int64_t i, int64_t d) {
    const int64_t p = 2 * d;
    int64_t m = i % p;
    if (m < 0) m += p;
    return m >= d ? p - 1 - m : m;
}

// Runs f(row) for rows [0, n) on `threads` threads, chunks of `chunk` rows from a shared counter.
void parallel_rows(int64_t n, int threads, const std::function<void(int64_t, int)> &f, int64_t chunk = 8) {
    std::atomic<int64_t> next{0};
    auto work = [&](int tid) {
        for (;;) {
            const int64_t a = next.fetch_add(chunk);
            if (a >= n) break;
            const int64_t b = std::min(n, a + chunk);
            for (int64_t r = a; r < b; ++r) f(r, tid);
        }
    };
    if (threads <= 1) {
        work(0);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(size_t(threads));
    for (int t = 0; t < threads; ++t) th.emplace_back(work, t);
    for (auto &t : th) t.join();
}

// first index in [a, b) of the sorted ys with ys[i] >= y
int64_t lower(const std::vector<int32_t> &ys, int64_t a, int64_t b, int64_t y) {
    return std::lower_bound(ys.begin() + a, ys.begin() + b, int32_t(y)) - ys.begin();
}

// index of the element with y exactly, or -1
int64_t find_y(const std::vector<int32_t> &ys, int64_t a, int64_t b, int64_t y) {
    const int64_t i = lower(ys, a, b, y);
    return (i < b && ys[size_t(i)] == y) ? i : -1;
}

struct Ctx {
    const Apr &A;
    const float *vals;   // particle values
    const float *tree;   // tree values
};

// Dense line of û_l over level-l cells y in [y0, y0 + n) of row (z, x) (in-grid row and cells only;
// other entries are left as they are).
void fill_line(const Ctx &C, int l, int64_t z, int64_t x, int64_t y0, int64_t n, float *line) {
    const Apr &A = C.A;
    const Level &g = A.lv[size_t(l)];
    const int64_t ya = std::max<int64_t>(y0, 0), yb = std::min<int64_t>(y0 + n, g.dy);
    if (ya >= yb) return;
    const int64_t r = z * g.dx + x;
    for (int64_t i = lower(A.py, g.prow[size_t(r)], g.prow[size_t(r + 1)], ya); i < g.prow[size_t(r + 1)] && A.py[size_t(i)] < yb; ++i)
        line[A.py[size_t(i)] - y0] = C.vals[i];
    if (l < A.l_max)
        for (int64_t i = lower(A.ty, g.trow[size_t(r)], g.trow[size_t(r + 1)], ya); i < g.trow[size_t(r + 1)] && A.ty[size_t(i)] < yb; ++i)
            line[A.ty[size_t(i)] - y0] = C.tree[i];
    if (l > A.l_min) {
        const Level &q = A.lv[size_t(l - 1)];
        const int64_t rq = (z >> 1) * q.dx + (x >> 1);
        for (int64_t i = lower(A.py, q.prow[size_t(rq)], q.prow[size_t(rq + 1)], ya >> 1);
             i < q.prow[size_t(rq + 1)] && 2 * int64_t(A.py[size_t(i)]) < yb; ++i) {
            const int64_t c = 2 * int64_t(A.py[size_t(i)]);
            for (int64_t e = 0; e < 2; ++e)
                if (c + e >= ya && c + e < yb) line[c + e - y0] = C.vals[i];
        }
    }
}

// Line of û_l for patch row (z, x) (possibly outside the grid) over cells [y0, y0 + n), with the
// boundary rule applied to the row and to the cells outside [0, dy).
void patch_line(const Ctx &C, int l, int64_t z, int64_t x, int64_t y0, int64_t n, bool reflect, float *line) {
    const Level &g = C.A.lv[size_t(l)];
    std::fill(line, line + n, 0.f);
    const bool in = z >= 0 && z < g.dz && x >= 0 && x < g.dx;
    if (!in && !reflect) return;
    fill_line(C, l, refl(z, g.dz), refl(x, g.dx), y0, n, line);
    if (!reflect) return;
    for (int64_t j = 0; j < n; ++j) {
        const int64_t y = y0 + j;
        if (y < 0 || y >= g.dy) {
            const int64_t m = refl(y, g.dy);
            if (m >= y0 && m < y0 + n) {
                line[j] = line[m - y0];
            } else {
                float v = 0.f;
                fill_line(C, l, refl(z, g.dz), refl(x, g.dx), m, 1, &v);
                line[j] = v;
            }
        }
    }
}

// Calls f(y0, i0, i1) for consecutive runs [i0, i1) of the sorted ys[a, b) that fit in a window
// [y0, y0 + span) starting at their first element: rows are processed in windows of bounded length,
// so a sparse row costs per window, not per cell of the row.
template <typename F>
void windows_of(const std::vector<int32_t> &ys, int64_t a, int64_t b, int64_t span, F f) {
    int64_t i = a;
    while (i < b) {
        const int64_t y0 = ys[size_t(i)];
        int64_t j = i + 1;
        while (j < b && ys[size_t(j)] < y0 + span) ++j;
        f(y0, i, j);
        i = j;
    }
}

constexpr int64_t SPAN = 64;  // window length in cells

// Line of dL/dout at the level-l particles of in-grid row (z, x) over cells [y0, y0 + n) (0 at every
// other cell and outside the grid).
void grad_line(const Apr &A, int l, int64_t z, int64_t x, int64_t y0, int64_t n, const float *gout, float *line) {
    const Level &g = A.lv[size_t(l)];
    std::fill(line, line + n, 0.f);
    if (z < 0 || z >= g.dz || x < 0 || x >= g.dx) return;
    const int64_t r = z * g.dx + x;
    for (int64_t i = lower(A.py, g.prow[size_t(r)], g.prow[size_t(r + 1)], y0); i < g.prow[size_t(r + 1)] && A.py[size_t(i)] < y0 + n; ++i)
        line[A.py[size_t(i)] - y0] = gout[i];
}

// Radius of level l_idx's stencil: 1 if a 5^3 stencil has zero taps outside its central 3^3.
int level_radius(const float *st, int k) {
    if (k == 3) return 1;
    for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b)
            for (int c = 0; c < 5; ++c)
                if ((a == 0 || a == 4 || b == 0 || b == 4 || c == 0 || c == 4) && st[(a * 5 + b) * 5 + c] != 0.f) return 2;
    return 1;
}

}  // namespace

extern "C" {

void *acpu_create(int l_min, int l_max, const int64_t *dims, const int64_t *row_ptr, const int32_t *y, int64_t np) {
    if (l_min < 0 || l_max < l_min || l_max > 20 || !dims || !row_ptr || (np && !y)) return nullptr;
    Apr *A = new Apr();
    A->l_min = l_min;
    A->l_max = l_max;
    A->np = np;
    A->lv.resize(size_t(l_max) + 1);
    int64_t row = 0;
    for (int l = l_min; l <= l_max; ++l) {
        Level &g = A->lv[size_t(l)];
        g.dz = cells(dims[0], l_max, l);
        g.dx = cells(dims[1], l_max, l);
        g.dy = cells(dims[2], l_max, l);
        g.prow.assign(row_ptr + row, row_ptr + row + g.dz * g.dx + 1);
        row += g.dz * g.dx;
    }
    A->py.assign(y, y + np);
    // tree levels l_max - 1 .. l_min: sorted unique parents of the next finer level's particles
    // and tree nodes, row by row
    std::vector<std::vector<std::vector<int32_t>>> rows(size_t(l_max) + 1);
    for (int l = l_max - 1; l >= l_min; --l) {
        const Level &g = A->lv[size_t(l)], &f = A->lv[size_t(l + 1)];
        auto &R = rows[size_t(l)];
        R.assign(size_t(g.dz * g.dx), {});
        for (int64_t z = 0; z < f.dz; ++z)
            for (int64_t x = 0; x < f.dx; ++x) {
                auto &dst = R[size_t((z >> 1) * g.dx + (x >> 1))];
                const int64_t r = z * f.dx + x;
                for (int64_t i = f.prow[size_t(r)]; i < f.prow[size_t(r + 1)]; ++i) dst.push_back(A->py[size_t(i)] >> 1);
                if (l + 1 < l_max)
                    for (int32_t yy : rows[size_t(l + 1)][size_t(r)]) dst.push_back(yy >> 1);
            }
        for (auto &v : R) {
            std::sort(v.begin(), v.end());
            v.erase(std::unique(v.begin(), v.end()), v.end());
        }
    }
    int64_t nt = 0;
    for (int l = l_min; l < l_max; ++l) {
        Level &g = A->lv[size_t(l)];
        const Level &f = A->lv[size_t(l + 1)];
        g.trow.assign(size_t(g.dz * g.dx + 1), 0);
        for (int64_t r = 0; r < g.dz * g.dx; ++r) {
            g.trow[size_t(r)] = nt;
            const int64_t z = r / g.dx, x = r % g.dx;
            for (int32_t yy : rows[size_t(l)][size_t(r)]) {
                A->ty.push_back(yy);
                const int n = (2 * z + 1 < f.dz ? 2 : 1) * (2 * x + 1 < f.dx ? 2 : 1) * (2 * int64_t(yy) + 1 < f.dy ? 2 : 1);
                A->tnch.push_back(int8_t(n));
                ++nt;
            }
        }
        g.trow[size_t(g.dz * g.dx)] = nt;
    }
    A->nt = nt;
    return A;
}

void acpu_destroy(void *h) { delete static_cast<Apr *>(h); }
int64_t acpu_num_tree(void *h) { return h ? static_cast<Apr *>(h)->nt : -1; }

// Tree values, finest level first (Sec. 3.4): each node is the mean of its in-grid children. Rows
// of a level in parallel.
int acpu_tree_restrict(void *h, const float *vals, float *tree, int threads) {
    const Apr &A = *static_cast<Apr *>(h);
    for (int l = A.l_max - 1; l >= A.l_min; --l) {
        const Level &g = A.lv[size_t(l)], &f = A.lv[size_t(l + 1)];
        parallel_rows(g.dz * g.dx, threads, [&](int64_t r, int) {
            const int64_t t0 = g.trow[size_t(r)], t1 = g.trow[size_t(r + 1)];
            if (t0 == t1) return;
            const int64_t z = r / g.dx, x = r % g.dx;
            for (int64_t t = t0; t < t1; ++t) tree[t] = 0.f;
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) {
                    const int64_t cz = 2 * z + a, cx = 2 * x + b;
                    if (cz >= f.dz || cx >= f.dx) continue;
                    const int64_t cr = cz * f.dx + cx;
                    // children of this row's nodes, merged by y (both lists are sorted)
                    int64_t t = t0;
                    for (int64_t i = f.prow[size_t(cr)]; i < f.prow[size_t(cr + 1)]; ++i) {
                        const int32_t py = A.py[size_t(i)] >> 1;
                        while (A.ty[size_t(t)] < py) ++t;
                        tree[t] += vals[i];
                    }
                    if (l + 1 < A.l_max) {
                        t = t0;
                        for (int64_t i = f.trow[size_t(cr)]; i < f.trow[size_t(cr + 1)]; ++i) {
                            const int32_t py = A.ty[size_t(i)] >> 1;
                            while (A.ty[size_t(t)] < py) ++t;
                            tree[t] += tree[i];
                        }
                    }
                }
            for (int64_t t = t0; t < t1; ++t) tree[t] /= float(A.tnch[size_t(t)]);
        });
    }
    return 0;
}

// APR convolution (Sec. 4.1), FP32: per level, rows in parallel; for each row the (2r+1)^2 patch
// lines of û_l over the row's y range are built, then every particle of the row takes its taps.
int acpu_convolve(void *h, const float *vals, const float *tree, const float *stencils, int k, int bc, float *out,
                  int threads) {
    const Apr &A = *static_cast<Apr *>(h);
    if (k != 3 && k != 5) return 1;
    const Ctx C{A, vals, tree};
    const bool reflect = bc == 0;
    const int K3 = k * k * k;
    for (int l = A.l_min; l <= A.l_max; ++l) {
        const Level &g = A.lv[size_t(l)];
        const float *w = stencils + size_t(l - A.l_min) * K3;
        const int R = level_radius(w, k), K = 2 * R + 1, D = k / 2 - R;
        std::vector<std::vector<float>> buf(size_t(std::max(threads, 1)));
        parallel_rows(g.dz * g.dx, threads, [&](int64_t r, int tid) {
            const int64_t z = r / g.dx, x = r % g.dx;
            std::vector<float> &L = buf[size_t(tid)];
            windows_of(A.py, g.prow[size_t(r)], g.prow[size_t(r + 1)], SPAN, [&](int64_t ys, int64_t p0, int64_t p1) {
                const int64_t y0 = ys - R, n = SPAN + 2 * R;
                L.resize(size_t(K * K * n));
                for (int a = 0; a < K; ++a)
                    for (int b = 0; b < K; ++b)
                        patch_line(C, l, z - R + a, x - R + b, y0, n, reflect, L.data() + size_t(a * K + b) * n);
                for (int64_t p = p0; p < p1; ++p) {
                    const int64_t j = A.py[size_t(p)] - R - y0;
                    float acc = 0.f;
                    for (int a = 0; a < K; ++a)
                        for (int b = 0; b < K; ++b) {
                            const float *line = L.data() + size_t(a * K + b) * n + j;
                            const float *wr = w + ((a + D) * k + (b + D)) * k + D;
                            for (int c = 0; c < K; ++c) acc += wr[c] * line[c];
                        }
                    out[p] = acc;
                }
            });
        });
    }
    return 0;
}

// Backward of the convolution layer (FP32): grad_particles (through û and the tree average) and
// grad_stencils [levels][k^3]; either may be null.
//   Data part, gather form: H_l(c) = sum over the preimages c' of c under the boundary rule of
//   sum_e w_l[e] g_l(c' - e), g_l = dL/dout at the level-l particles (0 elsewhere). Level-l
//   particles receive H_l at their cell, level-l tree nodes likewise (then pushed down the tree,
//   coarse to fine, divided by the child count), level-(l-1) particles the sum of H_l over their
//   2 x 2 x 2 cells. The preimage c' = c is evaluated from windowed lines of g; the other preimages
//   (cells within R of the grid boundary, reflecting boundary) tap by tap.
int acpu_convolve_backward(void *h, const float *vals, const float *tree, const float *stencils, int k, int bc,
                           const float *gout, float *gpart, float *gsten, int threads) {
    const Apr &A = *static_cast<Apr *>(h);
    if (k != 3 && k != 5) return 1;
    const bool reflect = bc == 0;
    const int K3 = k * k * k, nl = A.l_max - A.l_min + 1;
    const int nth = std::max(threads, 1);
    if (gpart) {
        std::vector<float> gtree(size_t(std::max<int64_t>(A.nt, 1)), 0.f);
        std::fill(gpart, gpart + A.np, 0.f);
        std::vector<std::vector<float>> buf(static_cast<size_t>(nth));
        for (int l = A.l_min; l <= A.l_max; ++l) {
            const Level &g = A.lv[size_t(l)];
            const float *w = stencils + size_t(l - A.l_min) * K3;
            const int R = level_radius(w, k), K = 2 * R + 1, D = k / 2 - R;
            auto tap = [&](int ez, int ex, int ey) { return w[((ez + R + D) * k + (ex + R + D)) * k + (ey + R + D)]; };
            auto g_at = [&](int64_t z, int64_t x, int64_t y) -> float {
                if (z < 0 || z >= g.dz || x < 0 || x >= g.dx || y < 0 || y >= g.dy) return 0.f;
                const int64_t r = z * g.dx + x;
                const int64_t i = find_y(A.py, g.prow[size_t(r)], g.prow[size_t(r + 1)], y);
                return i >= 0 ? gout[i] : 0.f;
            };
            auto preimages = [&](int64_t c, int64_t d, int64_t *o) {
                int n = 0;
                o[n++] = c;
                if (!reflect) return n;
                for (int64_t v = -R; v < 0; ++v)
                    if (refl(v, d) == c) o[n++] = v;
                for (int64_t v = d; v < d + R; ++v)
                    if (refl(v, d) == c) o[n++] = v;
                return n;
            };
            // terms of the preimages other than c itself
            auto H_mirror = [&](int64_t z, int64_t x, int64_t y) {
                int64_t pz[5], px[5], py[5];
                const int nz = preimages(z, g.dz, pz), nx = preimages(x, g.dx, px), ny = preimages(y, g.dy, py);
                float acc = 0.f;
                for (int iz = 0; iz < nz; ++iz)
                    for (int ix = 0; ix < nx; ++ix)
                        for (int iy = 0; iy < ny; ++iy) {
                            if (iz == 0 && ix == 0 && iy == 0) continue;
                            for (int a = -R; a <= R; ++a)
                                for (int b = -R; b <= R; ++b)
                                    for (int c = -R; c <= R; ++c) {
                                        const float gv = g_at(pz[iz] - a, px[ix] - b, py[iy] - c);
                                        if (gv != 0.f) acc += tap(a, b, c) * gv;
                                    }
                        }
                return acc;
            };
            const auto near_edge = [&](int64_t z, int64_t x, int64_t y) {
                return reflect && (z < R || z >= g.dz - R || x < R || x >= g.dx - R || y < R || y >= g.dy - R);
            };
            // H at the cells ys[i0, i1) (sorted, inside [y_s, y_s + SPAN)) of in-grid row (z, x)
            auto H_window = [&](int64_t z, int64_t x, const int32_t *ys, int64_t m, int64_t y_s, std::vector<float> &L,
                                float *hv) {
                const int64_t n = SPAN + 2 * R, y0 = y_s - R;
                L.resize(size_t(K * K * n));
                for (int a = 0; a < K; ++a)
                    for (int b = 0; b < K; ++b)
                        grad_line(A, l, z - (a - R), x - (b - R), y0, n, gout, L.data() + size_t(a * K + b) * n);
                for (int64_t j = 0; j < m; ++j) {
                    const int64_t y = ys[j];
                    float acc = 0.f;
                    for (int a = 0; a < K; ++a)
                        for (int b = 0; b < K; ++b) {
                            const float *line = L.data() + size_t(a * K + b) * n + (y - y0 + R);
                            for (int c = 0; c < K; ++c) acc += tap(a - R, b - R, c - R) * line[-c];
                        }
                    if (near_edge(z, x, y)) acc += H_mirror(z, x, y);
                    hv[j] = acc;
                }
            };
            // pass A: level-l particles and tree nodes, one row at a time
            parallel_rows(g.dz * g.dx, threads, [&](int64_t r, int tid) {
                const int64_t z = r / g.dx, x = r % g.dx;
                std::vector<float> &L = buf[size_t(tid)];
                float hv[SPAN];
                windows_of(A.py, g.prow[size_t(r)], g.prow[size_t(r + 1)], SPAN, [&](int64_t ys, int64_t i0, int64_t i1) {
                    H_window(z, x, A.py.data() + i0, i1 - i0, ys, L, hv);
                    for (int64_t i = i0; i < i1; ++i) gpart[i] += hv[i - i0];
                });
                if (l < A.l_max)
                    windows_of(A.ty, g.trow[size_t(r)], g.trow[size_t(r + 1)], SPAN, [&](int64_t ys, int64_t i0, int64_t i1) {
                        H_window(z, x, A.ty.data() + i0, i1 - i0, ys, L, hv);
                        for (int64_t i = i0; i < i1; ++i) gtree[size_t(i)] = hv[i - i0];
                    });
            });
            // pass B: level-(l-1) particles, the sum of H_l over their level-l cells, one parent row at a time
            if (l > A.l_min) {
                const Level &q = A.lv[size_t(l - 1)];
                parallel_rows(q.dz * q.dx, threads, [&](int64_t r, int tid) {
                    const int64_t q0 = q.prow[size_t(r)], q1 = q.prow[size_t(r + 1)];
                    if (q0 == q1) return;
                    const int64_t Z = r / q.dx, X = r % q.dx;
                    std::vector<float> &L = buf[size_t(tid)];
                    std::vector<float> sum(size_t(q1 - q0), 0.f);
                    std::vector<int32_t> cy;
                    std::vector<int64_t> owner;
                    for (int64_t i = q0; i < q1; ++i)
                        for (int e = 0; e < 2; ++e) {
                            const int64_t y = 2 * int64_t(A.py[size_t(i)]) + e;
                            if (y < g.dy) {
                                cy.push_back(int32_t(y));
                                owner.push_back(i - q0);
                            }
                        }
                    float hv[SPAN];
                    for (int a = 0; a < 2; ++a)
                        for (int b = 0; b < 2; ++b) {
                            const int64_t z = 2 * Z + a, x = 2 * X + b;
                            if (z >= g.dz || x >= g.dx) continue;
                            windows_of(cy, 0, int64_t(cy.size()), SPAN, [&](int64_t ys, int64_t i0, int64_t i1) {
                                H_window(z, x, cy.data() + i0, i1 - i0, ys, L, hv);
                                for (int64_t i = i0; i < i1; ++i) sum[size_t(owner[size_t(i)])] += hv[i - i0];
                            });
                        }
                    for (int64_t i = q0; i < q1; ++i) gpart[i] += sum[size_t(i - q0)];
                });
            }
        }
        // tree transpose, coarse to fine: every child of level l + 1 gets its parent's gradient / count
        for (int l = A.l_min; l < A.l_max; ++l) {
            const Level &g = A.lv[size_t(l)], &f = A.lv[size_t(l + 1)];
            parallel_rows(f.dz * f.dx, threads, [&](int64_t r, int) {
                const int64_t z = r / f.dx, x = r % f.dx;
                const int64_t pr = (z >> 1) * g.dx + (x >> 1);
                const int64_t t0 = g.trow[size_t(pr)], t1 = g.trow[size_t(pr + 1)];
                for (int64_t i = f.prow[size_t(r)]; i < f.prow[size_t(r + 1)]; ++i) {
                    const int64_t t = find_y(A.ty, t0, t1, A.py[size_t(i)] >> 1);
                    if (t >= 0) gpart[i] += gtree[size_t(t)] / float(A.tnch[size_t(t)]);
                }
                if (l + 1 < A.l_max)
                    for (int64_t i = f.trow[size_t(r)]; i < f.trow[size_t(r + 1)]; ++i) {
                        const int64_t t = find_y(A.ty, t0, t1, A.ty[size_t(i)] >> 1);
                        if (t >= 0) gtree[size_t(i)] += gtree[size_t(t)] / float(A.tnch[size_t(t)]);
                    }
            });
        }
    }
    if (gsten) {
        // sum_p g_p û_l(refl(p + e)) over windowed patch lines; per thread FP64 partials, summed in
        // thread order
        const Ctx C{A, vals, tree};
        std::vector<double> part(size_t(nth) * size_t(nl) * size_t(K3), 0.0);
        std::vector<std::vector<float>> buf(static_cast<size_t>(nth));
        const int R = k / 2, K = k;
        for (int l = A.l_min; l <= A.l_max; ++l) {
            const Level &g = A.lv[size_t(l)];
            parallel_rows(g.dz * g.dx, threads, [&](int64_t r, int tid) {
                const int64_t z = r / g.dx, x = r % g.dx;
                std::vector<float> &L = buf[size_t(tid)];
                double *acc = part.data() + (size_t(tid) * size_t(nl) + size_t(l - A.l_min)) * size_t(K3);
                windows_of(A.py, g.prow[size_t(r)], g.prow[size_t(r + 1)], SPAN, [&](int64_t ys, int64_t p0, int64_t p1) {
                    const int64_t y0 = ys - R, n = SPAN + 2 * R;
                    L.resize(size_t(K * K * n));
                    for (int a = 0; a < K; ++a)
                        for (int b = 0; b < K; ++b)
                            patch_line(C, l, z - R + a, x - R + b, y0, n, reflect, L.data() + size_t(a * K + b) * n);
                    for (int a = 0; a < K; ++a)
                        for (int b = 0; b < K; ++b) {
                            const float *line = L.data() + size_t(a * K + b) * n;
                            for (int c = 0; c < K; ++c) {
                                float s = 0.f;
                                for (int64_t p = p0; p < p1; ++p) s += gout[p] * line[A.py[size_t(p)] - R - y0 + c];
                                acc[(a * K + b) * K + c] += double(s);
                            }
                        }
                });
            });
        }
        for (int i = 0; i < nl * K3; ++i) {
            double s = 0.0;
            for (int t = 0; t < nth; ++t) s += part[size_t(t) * size_t(nl) * size_t(K3) + size_t(i)];
            gsten[i] = float(s);
        }
    }
    return 0;
}

}  // extern "C"
