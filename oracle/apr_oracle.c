/*
 * FP64 CPU oracle for APR-native discrete convolution
 * (Jonsson, Cheeseman, Maddu, Gonciarz, Sbalzarini: "Parallel Discrete Convolutions on Adaptive
 * Particle Representations of Images", arXiv 2112.03592).
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg
 * load this file's library. The product path (the CUDA library and its binding) never does.
 *
 * This is the plain, slow definition of the method, in double precision, single threaded. It shares
 * no code with the CUDA library: it builds its own index (sorted keys + binary search), its own APR
 * tree (ancestor marking, level by level), and evaluates every output by looking up every stencil
 * tap one at a time.
 *
 *   - Particle layout (Sec. 3.1, Alg. 1): rows (l, z, x), CSR offsets, y index per particle, particles
 *     ordered l -> z -> x -> y (Alg. 2). Level grid size d_l = ceil(D / 2^(l_max - l)).
 *   - APR tree (Sec. 3.4): the interior nodes of the pruned pyramid = all strict ancestors of
 *     particle cells. A tree node's value is the average of its children (particles or tree nodes),
 *     computed level by level from the finest level (Sec. 3.4, two-step fill; Sec. 2.3: average
 *     downsampling). At image edges only the children inside the level grid are averaged.
 *   - Isotropic patch value (Sec. 3.5): the value of level-l grid cell c is the particle at level l
 *     covering c, else the tree node at (l, c), else the particle at a coarser level containing c.
 *   - APR convolution (Sec. 4.1): o_p = sum_e w_{l_p}[e] * u_{l_p}(refl(i_p + e)), one output per
 *     particle at its own level, positions fixed; e in [-r, r]^3 ordered [z][x][y], y fastest.
 *     Reading: correlation (no flip), half-sample symmetric reflection at the level-l grid, or zeros.
 *   - Backward: the transpose of the above linear map (the paper's future-work CNN, Sec. 6).
 *
 * Multi-channel: values [N][C] channels-last; stencils [L][C_out][C_in][k^3].
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORA_MAXL 32

enum { SRC_NONE = 0, SRC_PARTICLE = 1, SRC_TREE = 2 };

typedef struct {
    uint64_t *key;   /* sorted (z * d_x + x) * d_y + y */
    int64_t *idx;    /* particle index, or tree index */
    int64_t n;
} keyset;

typedef struct {
    int l_min, l_max, C;
    int64_t dims[3];
    int64_t ld[ORA_MAXL][3];
    int64_t np, nt;
    int32_t *pl, *pz, *px, *py;  /* per particle: level and level coordinates */
    keyset P[ORA_MAXL];          /* particles per level */
    keyset T[ORA_MAXL];          /* tree nodes per level (idx = global tree index) */
    int64_t t_off[ORA_MAXL + 1]; /* tree index of the first node of each level */
    int32_t *tl, *tz, *tx, *ty;  /* per tree node */
    double *pval;                /* [np][C] */
    double *tval;                /* [nt][C] */
    int error;                   /* nonzero: the layout is not a valid APR */
} ora_t;

/* ---------------------------------------------------------------- small helpers */
static uint64_t cell_key(const ora_t *o, int l, int64_t z, int64_t x, int64_t y) {
    return ((uint64_t)z * (uint64_t)o->ld[l][1] + (uint64_t)x) * (uint64_t)o->ld[l][2] + (uint64_t)y;
}

static void key_cell(const ora_t *o, int l, uint64_t k, int64_t *z, int64_t *x, int64_t *y) {
    *y = (int64_t)(k % (uint64_t)o->ld[l][2]);
    k /= (uint64_t)o->ld[l][2];
    *x = (int64_t)(k % (uint64_t)o->ld[l][1]);
    *z = (int64_t)(k / (uint64_t)o->ld[l][1]);
}

static int64_t find(const keyset *s, uint64_t k) {
    int64_t lo = 0, hi = s->n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (s->key[mid] < k) lo = mid + 1; else hi = mid;
    }
    return (lo < s->n && s->key[lo] == k) ? s->idx[lo] : -1;
}

typedef struct { uint64_t k; int64_t i; } kv;
static int kv_cmp(const void *a, const void *b) {
    uint64_t x = ((const kv *)a)->k, y = ((const kv *)b)->k;
    return x < y ? -1 : (x > y ? 1 : 0);
}
static int u64_cmp(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* half-sample symmetric reflection into [0, d): ... 1 0 | 0 1 ... d-1 | d-1 d-2 ... */
static int64_t reflect(int64_t i, int64_t d) {
    int64_t m = i % (2 * d);
    if (m < 0) m += 2 * d;
    return m >= d ? 2 * d - 1 - m : m;
}

/* ---------------------------------------------------------------- construction */
void ora_destroy(ora_t *o);

/* Build the oracle's own view of an APR from the linear-access layout (Alg. 1).
 * row_ptr: [R+1] (rows l -> z -> x), y_idx: [np], values: [np][C]. */
ora_t *ora_create(int l_min, int l_max, const int64_t *dims, const int64_t *row_ptr,
                  const int32_t *y_idx, int64_t np, const double *values, int C) {
    ora_t *o = (ora_t *)calloc(1, sizeof(ora_t));
    if (!o || l_max >= ORA_MAXL || l_min < 0 || l_min > l_max || C < 1) { free(o); return NULL; }
    o->l_min = l_min; o->l_max = l_max; o->C = C; o->np = np;
    for (int a = 0; a < 3; ++a) o->dims[a] = dims[a];
    for (int l = l_min; l <= l_max; ++l) {
        int64_t s = (int64_t)1 << (l_max - l);
        for (int a = 0; a < 3; ++a) o->ld[l][a] = (dims[a] + s - 1) / s;
    }
    o->pl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(np ? np : 1));
    o->pz = (int32_t *)malloc(sizeof(int32_t) * (size_t)(np ? np : 1));
    o->px = (int32_t *)malloc(sizeof(int32_t) * (size_t)(np ? np : 1));
    o->py = (int32_t *)malloc(sizeof(int32_t) * (size_t)(np ? np : 1));
    o->pval = (double *)malloc(sizeof(double) * (size_t)(np ? np : 1) * (size_t)C);
    if (np) memcpy(o->pval, values, sizeof(double) * (size_t)np * (size_t)C);

    /* linear iteration over rows (Alg. 2): l -> z -> x -> particles of the row */
    int64_t row = 0;
    for (int l = l_min; l <= l_max; ++l) {
        int64_t cnt = 0;
        int64_t first = row_ptr[row];
        for (int64_t z = 0; z < o->ld[l][0]; ++z)
            for (int64_t x = 0; x < o->ld[l][1]; ++x, ++row)
                for (int64_t i = row_ptr[row]; i < row_ptr[row + 1]; ++i) {
                    o->pl[i] = l; o->pz[i] = (int32_t)z; o->px[i] = (int32_t)x; o->py[i] = y_idx[i];
                    if (y_idx[i] < 0 || y_idx[i] >= o->ld[l][2]) o->error = 1;
                    ++cnt;
                }
        kv *tmp = (kv *)malloc(sizeof(kv) * (size_t)(cnt ? cnt : 1));
        for (int64_t j = 0; j < cnt; ++j) {
            int64_t i = first + j;
            tmp[j].k = cell_key(o, l, o->pz[i], o->px[i], o->py[i]);
            tmp[j].i = i;
        }
        qsort(tmp, (size_t)cnt, sizeof(kv), kv_cmp);
        o->P[l].n = cnt;
        o->P[l].key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(cnt ? cnt : 1));
        o->P[l].idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(cnt ? cnt : 1));
        for (int64_t j = 0; j < cnt; ++j) {
            o->P[l].key[j] = tmp[j].k; o->P[l].idx[j] = tmp[j].i;
            if (j && tmp[j].k == tmp[j - 1].k) o->error = 1;  /* duplicate particle */
        }
        free(tmp);
    }

    /* APR tree (Sec. 3.4): the strict ancestors of all particles. Level by level from the finest:
     * the tree cells of level l are the parents of the particles and tree cells of level l+1. */
    for (int l = l_max - 1; l >= l_min; --l) {
        int64_t n = o->P[l + 1].n + o->T[l + 1].n;
        uint64_t *par = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n ? n : 1));
        int64_t m = 0;
        for (int src = 0; src < 2; ++src) {
            const keyset *s = src == 0 ? &o->P[l + 1] : &o->T[l + 1];
            for (int64_t j = 0; j < s->n; ++j) {
                int64_t z, x, y;
                key_cell(o, l + 1, s->key[j], &z, &x, &y);
                par[m++] = cell_key(o, l, z / 2, x / 2, y / 2);
            }
        }
        qsort(par, (size_t)m, sizeof(uint64_t), u64_cmp);
        int64_t u = 0;
        for (int64_t j = 0; j < m; ++j)
            if (u == 0 || par[j] != par[u - 1]) par[u++] = par[j];
        o->T[l].n = u;
        o->T[l].key = par;
        o->T[l].idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(u ? u : 1));
    }
    /* global tree order: l_min .. l_max-1, then z, x, y */
    int64_t nt = 0;
    for (int l = l_min; l <= l_max; ++l) {
        o->t_off[l] = nt;
        for (int64_t j = 0; j < o->T[l].n; ++j) o->T[l].idx[j] = nt + j;
        nt += o->T[l].n;
    }
    o->t_off[l_max + 1] = nt;
    o->nt = nt;
    o->tl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nt ? nt : 1));
    o->tz = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nt ? nt : 1));
    o->tx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nt ? nt : 1));
    o->ty = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nt ? nt : 1));
    for (int l = l_min; l < l_max; ++l)
        for (int64_t j = 0; j < o->T[l].n; ++j) {
            int64_t z, x, y, t = o->t_off[l] + j;
            key_cell(o, l, o->T[l].key[j], &z, &x, &y);
            o->tl[t] = l; o->tz[t] = (int32_t)z; o->tx[t] = (int32_t)x; o->ty[t] = (int32_t)y;
            /* a cell cannot be both a particle (leaf) and a tree node (interior) */
            if (find(&o->P[l], o->T[l].key[j]) >= 0) o->error = 1;
        }
    o->tval = (double *)calloc((size_t)(nt ? nt : 1) * (size_t)C, sizeof(double));
    return o;
}

void ora_destroy(ora_t *o) {
    if (!o) return;
    for (int l = 0; l < ORA_MAXL; ++l) {
        free(o->P[l].key); free(o->P[l].idx); free(o->T[l].key); free(o->T[l].idx);
    }
    free(o->pl); free(o->pz); free(o->px); free(o->py);
    free(o->tl); free(o->tz); free(o->tx); free(o->ty);
    free(o->pval); free(o->tval); free(o);
}

int64_t ora_num_tree(const ora_t *o) { return o->nt; }
int ora_error(const ora_t *o) { return o->error; }

/* Tree node coordinates in the global tree order: out[t] = (l, z, x, y). */
void ora_tree_coords(const ora_t *o, int32_t *out) {
    for (int64_t t = 0; t < o->nt; ++t) {
        out[4 * t] = o->tl[t]; out[4 * t + 1] = o->tz[t]; out[4 * t + 2] = o->tx[t]; out[4 * t + 3] = o->ty[t];
    }
}

/* Tree structure in the linear-access form (Alg. 1) of the tree: per-row CSR over the rows
 * (l, z, x) of levels l_min .. l_max-1, and the y index of every node. */
void ora_tree_layout(const ora_t *o, int64_t *row_ptr, int32_t *y_idx) {
    int64_t row = 0, t = 0;
    row_ptr[0] = 0;
    for (int l = o->l_min; l < o->l_max; ++l)
        for (int64_t z = 0; z < o->ld[l][0]; ++z)
            for (int64_t x = 0; x < o->ld[l][1]; ++x) {
                while (t < o->nt && o->tl[t] == l && o->tz[t] == z && o->tx[t] == x) { y_idx[t] = o->ty[t]; ++t; }
                row_ptr[++row] = t;
            }
}

/* ---------------------------------------------------------------- tree values */
/* Number of children of level-l cell (z, x, y) that lie inside the level-(l+1) grid. */
static int n_children_in_grid(const ora_t *o, int l, int64_t z, int64_t x, int64_t y) {
    int n = 1;
    int64_t c[3] = {z, x, y};
    for (int a = 0; a < 3; ++a) n *= (2 * c[a] + 1 < o->ld[l + 1][a]) ? 2 : 1;
    return n;
}

/* T(l, c) = (1 / n_c) * sum over children ch of c inside the grid of v(l+1, ch), for l from l_max-1
 * down to l_min, v = particle value if ch is a particle, else the tree value (Sec. 3.4). */
int ora_tree_fill(ora_t *o) {
    const int C = o->C;
    for (int l = o->l_max - 1; l >= o->l_min; --l)
        for (int64_t j = 0; j < o->T[l].n; ++j) {
            int64_t t = o->t_off[l] + j;
            int64_t z = o->tz[t], x = o->tx[t], y = o->ty[t];
            double *acc = &o->tval[t * C];
            for (int c = 0; c < C; ++c) acc[c] = 0.0;
            int n = 0;
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b)
                    for (int e = 0; e < 2; ++e) {
                        int64_t cz = 2 * z + a, cx = 2 * x + b, cy = 2 * y + e;
                        if (cz >= o->ld[l + 1][0] || cx >= o->ld[l + 1][1] || cy >= o->ld[l + 1][2]) continue;
                        uint64_t k = cell_key(o, l + 1, cz, cx, cy);
                        int64_t i = find(&o->P[l + 1], k);
                        const double *v;
                        if (i >= 0) v = &o->pval[i * C];
                        else {
                            int64_t ti = find(&o->T[l + 1], k);
                            if (ti < 0) { o->error = 2; return 2; }  /* a hole: not a partition */
                            v = &o->tval[ti * C];
                        }
                        for (int c = 0; c < C; ++c) acc[c] += v[c];
                        ++n;
                    }
            if (n != n_children_in_grid(o, l, z, x, y)) { o->error = 2; return 2; }
            for (int c = 0; c < C; ++c) acc[c] /= (double)n;
        }
    return 0;
}

/* Round a double to the nearest bfloat16 (ties to even) and return it as a double. The value is
 * first rounded to float (round-to-nearest), then the low 16 bits of the float are rounded away. */
static double round_bf16(double v) {
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (double)f;  /* inf / nan unchanged */
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    u &= 0xffff0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

double ora_round_bf16(double v) { return round_bf16(v); }

/* Tree fill for bfloat16 features: the same average of children (Sec. 3.4), each node's value
 * rounded to bfloat16 before it is used by the next coarser level. */
int ora_tree_fill_bf16(ora_t *o) {
    /* BF16 tree of the multi-channel path (BF16 activations, FP32 accumulation): per node and
     * channel, the in-grid children are summed in FP32 in (dz, dx, dy) order starting from 0, the
     * sum is divided by their count in FP32, and the quotient is rounded to BF16. Levels are filled
     * finest first, each from the rounded values of the level below. */
    const int C = o->C;
    float acc[64];
    if (C > 64) return 1;
    for (int l = o->l_max - 1; l >= o->l_min; --l)
        for (int64_t j = 0; j < o->T[l].n; ++j) {
            int64_t t = o->t_off[l] + j;
            int64_t z = o->tz[t], x = o->tx[t], y = o->ty[t];
            for (int c = 0; c < C; ++c) acc[c] = 0.0f;
            int n = 0;
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b)
                    for (int e = 0; e < 2; ++e) {
                        int64_t cz = 2 * z + a, cx = 2 * x + b, cy = 2 * y + e;
                        if (cz >= o->ld[l + 1][0] || cx >= o->ld[l + 1][1] || cy >= o->ld[l + 1][2]) continue;
                        uint64_t k = cell_key(o, l + 1, cz, cx, cy);
                        int64_t i = find(&o->P[l + 1], k);
                        const double *v;
                        if (i >= 0) v = &o->pval[i * C];
                        else {
                            int64_t ti = find(&o->T[l + 1], k);
                            if (ti < 0) { o->error = 2; return 2; }
                            v = &o->tval[ti * C];
                        }
                        for (int c = 0; c < C; ++c) acc[c] = acc[c] + (float)v[c];
                        ++n;
                    }
            for (int c = 0; c < C; ++c) o->tval[t * C + c] = round_bf16((double)(acc[c] / (float)n));
        }
    return 0;
}

void ora_get_tree(const ora_t *o, double *out) { memcpy(out, o->tval, sizeof(double) * (size_t)o->nt * (size_t)o->C); }
void ora_set_values(ora_t *o, const double *values) { memcpy(o->pval, values, sizeof(double) * (size_t)o->np * (size_t)o->C); }

/* ---------------------------------------------------------------- patch value lookup */
/* Source of the value of level-l grid cell (z, x, y) (Sec. 3.5): a particle at level l, a tree node
 * at level l, or the particle at the first coarser level whose cell contains it. */
static int resolve(const ora_t *o, int l, int64_t z, int64_t x, int64_t y, int64_t *index) {
    int64_t i = find(&o->P[l], cell_key(o, l, z, x, y));
    if (i >= 0) { *index = i; return SRC_PARTICLE; }
    if (l < o->l_max) {
        i = find(&o->T[l], cell_key(o, l, z, x, y));
        if (i >= 0) { *index = i; return SRC_TREE; }
    }
    for (int lc = l - 1; lc >= o->l_min; --lc) {
        int sh = l - lc;
        i = find(&o->P[lc], cell_key(o, lc, z >> sh, x >> sh, y >> sh));
        if (i >= 0) { *index = i; return SRC_PARTICLE; }
    }
    return SRC_NONE;
}

/* map a stencil tap to a level-l cell; returns 0 if the tap falls outside with zero boundary */
static int tap_cell(const ora_t *o, int l, int bc, int64_t z, int64_t x, int64_t y, int64_t *c) {
    int64_t v[3] = {z, x, y};
    for (int a = 0; a < 3; ++a) {
        if (v[a] < 0 || v[a] >= o->ld[l][a]) {
            if (bc == 1) return 0;
            v[a] = reflect(v[a], o->ld[l][a]);
        }
        c[a] = v[a];
    }
    return 1;
}

/* ---------------------------------------------------------------- convolution */
/* o[p][co] = sum_{dz,dx,dy} sum_ci W[l_p - l_min][co][ci][dz+r][dx+r][dy+r] * u_{l_p}[ci](refl(.))
 * for the particles listed in `sample` (all if sample == NULL). W is FP64 (the caller upcasts
 * FP32 stencils). out is [ns][C_out]. Returns 0, or 3 when a tap has no source. */
int ora_conv(const ora_t *o, const double *W, int k, int C_out, int bc, const int64_t *sample,
             int64_t ns, double *out) {
    const int r = k / 2, C = o->C, k3 = k * k * k;
    if (!sample) ns = o->np;
    for (int64_t s = 0; s < ns; ++s) {
        int64_t p = sample ? sample[s] : s;
        int l = o->pl[p];
        const double *Wl = W + (size_t)(l - o->l_min) * C_out * C * k3;
        for (int co = 0; co < C_out; ++co) out[s * C_out + co] = 0.0;
        for (int dz = -r; dz <= r; ++dz)
            for (int dx = -r; dx <= r; ++dx)
                for (int dy = -r; dy <= r; ++dy) {
                    int64_t c[3], idx;
                    if (!tap_cell(o, l, bc, o->pz[p] + dz, o->px[p] + dx, o->py[p] + dy, c)) continue;
                    int src = resolve(o, l, c[0], c[1], c[2], &idx);
                    if (src == SRC_NONE) return 3;
                    const double *u = src == SRC_PARTICLE ? &o->pval[idx * C] : &o->tval[idx * C];
                    int e = ((dz + r) * k + (dx + r)) * k + (dy + r);
                    for (int co = 0; co < C_out; ++co)
                        for (int ci = 0; ci < C; ++ci)
                            out[s * C_out + co] += Wl[((size_t)co * C + ci) * k3 + e] * u[ci];
                }
    }
    return 0;
}

/* ---------------------------------------------------------------- backward (adjoint) */
/* Given G = dL/do [np][C_out]:
 *   grad_p [np][C] = dL/d(particle values) through both the direct taps and the tree averages,
 *   grad_w [L][C_out][C][k^3] = dL/dW,
 * (only the outputs listed in `sample` contribute when it is not NULL), as the explicit transpose of ora_tree_fill + ora_conv: every tap scatters G*w to the source of
 * its cell; tree gradients are then pushed from coarse to fine, each child receiving its parent's
 * gradient divided by the parent's number of children. Returns 0 or 3 (tap without source). */
/* The backward in its two linear parts. Part 1 (transpose of the convolution through the patch
 * sources): grad_p receives the terms whose source is a particle, gt those whose source is a tree
 * node, grad_w the stencil gradient. Part 2 (transpose of the tree averages): ora_tree_transpose. */
static int conv_backward_direct(const ora_t *o, const double *W, int k, int C_out, int bc, const double *G,
                                const int64_t *sample, int64_t ns, double *grad_p, double *gt, double *grad_w) {
    const int r = k / 2, C = o->C, k3 = k * k * k, L = o->l_max - o->l_min + 1;
    memset(grad_p, 0, sizeof(double) * (size_t)o->np * C);
    memset(gt, 0, sizeof(double) * (size_t)(o->nt ? o->nt : 1) * C);
    if (grad_w) memset(grad_w, 0, sizeof(double) * (size_t)L * C_out * C * k3);
    if (!sample) ns = o->np;
    for (int64_t s = 0; s < ns; ++s) {
        int64_t p = sample ? sample[s] : s;
        int l = o->pl[p];
        const double *Wl = W + (size_t)(l - o->l_min) * C_out * C * k3;
        double *gWl = grad_w ? grad_w + (size_t)(l - o->l_min) * C_out * C * k3 : NULL;
        for (int dz = -r; dz <= r; ++dz)
            for (int dx = -r; dx <= r; ++dx)
                for (int dy = -r; dy <= r; ++dy) {
                    int64_t c[3], idx;
                    if (!tap_cell(o, l, bc, o->pz[p] + dz, o->px[p] + dx, o->py[p] + dy, c)) continue;
                    int src = resolve(o, l, c[0], c[1], c[2], &idx);
                    if (src == SRC_NONE) return 3;
                    double *g = src == SRC_PARTICLE ? &grad_p[idx * C] : &gt[idx * C];
                    const double *u = src == SRC_PARTICLE ? &o->pval[idx * C] : &o->tval[idx * C];
                    int e = ((dz + r) * k + (dx + r)) * k + (dy + r);
                    for (int co = 0; co < C_out; ++co) {
                        double gp = G[p * C_out + co];
                        for (int ci = 0; ci < C; ++ci) {
                            g[ci] += gp * Wl[((size_t)co * C + ci) * k3 + e];
                            if (gWl) gWl[((size_t)co * C + ci) * k3 + e] += gp * u[ci];
                        }
                    }
                }
    }
    return 0;
}

/* Transpose of the tree averages (Sec. 3.4), coarse to fine: every child of a tree node (a particle
 * or a tree node of the next finer level) receives the node's gradient / (its in-grid children).
 * gt [N_t][C] is updated in place (tree nodes pass on what they received); the particle shares are
 * added to grad_p. */
static int tree_transpose(const ora_t *o, double *gt, double *grad_p) {
    const int C = o->C;
    for (int l = o->l_min; l < o->l_max; ++l)
        for (int64_t j = 0; j < o->T[l].n; ++j) {
            int64_t t = o->t_off[l] + j;
            int64_t z = o->tz[t], x = o->tx[t], y = o->ty[t];
            int n = n_children_in_grid(o, l, z, x, y);
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b)
                    for (int e = 0; e < 2; ++e) {
                        int64_t cz = 2 * z + a, cx = 2 * x + b, cy = 2 * y + e;
                        if (cz >= o->ld[l + 1][0] || cx >= o->ld[l + 1][1] || cy >= o->ld[l + 1][2]) continue;
                        uint64_t kk = cell_key(o, l + 1, cz, cx, cy);
                        int64_t i = find(&o->P[l + 1], kk);
                        double *dst;
                        if (i >= 0) dst = &grad_p[i * C];
                        else {
                            int64_t ti = find(&o->T[l + 1], kk);
                            if (ti < 0) return 2;
                            dst = &gt[ti * C];
                        }
                        for (int c = 0; c < C; ++c) dst[c] += gt[t * C + c] / (double)n;
                    }
        }
    return 0;
}

int ora_conv_backward(const ora_t *o, const double *W, int k, int C_out, int bc, const double *G,
                      const int64_t *sample, int64_t ns, double *grad_p, double *grad_w) {
    double *gt = (double *)calloc((size_t)(o->nt ? o->nt : 1) * o->C, sizeof(double));
    if (!gt) return 4;
    int rc = conv_backward_direct(o, W, k, C_out, bc, G, sample, ns, grad_p, gt, grad_w);
    if (rc == 0) rc = tree_transpose(o, gt, grad_p);
    free(gt);
    return rc;
}

/* Part 1 alone: grad_p (particle sources), grad_tree (tree-node sources), grad_w (nullable). */
int ora_conv_backward_direct(const ora_t *o, const double *W, int k, int C_out, int bc, const double *G,
                             const int64_t *sample, int64_t ns, double *grad_p, double *grad_tree, double *grad_w) {
    return conv_backward_direct(o, W, k, C_out, bc, G, sample, ns, grad_p, grad_tree, grad_w);
}

/* Part 2 alone: grad_p = the particle shares of the tree gradient grad_tree (copied, not changed). */
int ora_tree_transpose(const ora_t *o, const double *grad_tree, double *grad_p) {
    double *gt = (double *)malloc(sizeof(double) * (size_t)(o->nt ? o->nt : 1) * o->C);
    if (!gt) return 4;
    memcpy(gt, grad_tree, sizeof(double) * (size_t)o->nt * o->C);
    memset(grad_p, 0, sizeof(double) * (size_t)o->np * o->C);
    const int rc = tree_transpose(o, gt, grad_p);
    free(gt);
    return rc;
}

/* Replace the tree values (e.g. tree values assembled elsewhere); later convolutions use them. */
void ora_set_tree(ora_t *o, const double *tval) {
    memcpy(o->tval, tval, sizeof(double) * (size_t)o->nt * (size_t)o->C);
}

/* ---------------------------------------------------------------- balance check */
/* The property the convolution relies on (Sec. 4.2 footnote on neighbouring levels): every level-l
 * cell within Chebyshev distance r of a level-l particle is a particle at l, a tree node at l, or
 * lies inside a particle of level l-1. Returns the number of violations. */
int64_t ora_check_coarse_fill(const ora_t *o, int r) {
    int64_t bad = 0;
    for (int64_t p = 0; p < o->np; ++p) {
        int l = o->pl[p];
        for (int dz = -r; dz <= r; ++dz)
            for (int dx = -r; dx <= r; ++dx)
                for (int dy = -r; dy <= r; ++dy) {
                    int64_t c[3] = {o->pz[p] + dz, o->px[p] + dx, o->py[p] + dy};
                    int in = 1;
                    for (int a = 0; a < 3; ++a) in &= (c[a] >= 0 && c[a] < o->ld[l][a]);
                    if (!in) continue;
                    if (find(&o->P[l], cell_key(o, l, c[0], c[1], c[2])) >= 0) continue;
                    if (l < o->l_max && find(&o->T[l], cell_key(o, l, c[0], c[1], c[2])) >= 0) continue;
                    if (l > o->l_min && find(&o->P[l - 1], cell_key(o, l - 1, c[0] / 2, c[1] / 2, c[2] / 2)) >= 0) continue;
                    ++bad;
                }
    }
    return bad;
}
