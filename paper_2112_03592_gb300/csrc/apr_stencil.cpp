// Host helpers that build per-level stencil stacks (Sec. 4.2 and 4.3).
#include <cmath>
#include <vector>

#include "apr.h"

namespace {

// c_s(d, e) = (1/s) * #{x in [0, s) : floor((x + d) / s) == e}: the share of a fine tap d that lands on
// coarse offset e when the fine stencil is applied at every position inside a coarse cell of s pixels
// (block-average restriction after piecewise-constant prolongation, R_l P_l = I).
double coarse_share(int s, int d, int e) {
    int n = 0;
    for (int x = 0; x < s; ++x) {
        const int v = x + d;
        const int q = v >= 0 ? v / s : -((-v + s - 1) / s);  // floor division
        if (q == e) ++n;
    }
    return double(n) / double(s);
}

}  // namespace

extern "C" {

apr_status_t apr_restrict_stencil(const float *w, int32_t k, int32_t l_max, int32_t l_min, float *out) {
    if (!w || !out) return APR_ERR_INVALID_ARG;
    if (k != 3 && k != 5) return APR_ERR_UNSUPPORTED;
    if (l_min < 0 || l_max < l_min || l_max - l_min > 30) return APR_ERR_INVALID_ARG;
    const int r = k / 2, k3 = k * k * k;
    std::vector<double> share(size_t(k) * k);
    for (int l = l_min; l <= l_max; ++l) {
        const int s = 1 << (l_max - l);
        for (int d = -r; d <= r; ++d)
            for (int e = -r; e <= r; ++e) share[size_t(d + r) * k + (e + r)] = coarse_share(s, d, e);
        float *o = out + size_t(l - l_min) * k3;
        for (int ez = 0; ez < k; ++ez)
            for (int ex = 0; ex < k; ++ex)
                for (int ey = 0; ey < k; ++ey) {
                    double acc = 0.0;
                    for (int dz = 0; dz < k; ++dz) {
                        const double cz = share[size_t(dz) * k + ez];
                        if (cz == 0.0) continue;
                        for (int dx = 0; dx < k; ++dx) {
                            const double cx = share[size_t(dx) * k + ex];
                            if (cx == 0.0) continue;
                            for (int dy = 0; dy < k; ++dy) {
                                const double cy = share[size_t(dy) * k + ey];
                                if (cy == 0.0) continue;
                                acc += double(w[(dz * k + dx) * k + dy]) * cz * cx * cy;
                            }
                        }
                    }
                    o[(ez * k + ex) * k + ey] = float(acc);
                }
    }
    return APR_OK;
}

apr_status_t apr_rescale_stencil(const float *w, int32_t k, int32_t l_max, int32_t l_min, float *out) {
    if (!w || !out) return APR_ERR_INVALID_ARG;
    if (k != 3 && k != 5) return APR_ERR_UNSUPPORTED;
    if (l_min < 0 || l_max < l_min || l_max - l_min > 30) return APR_ERR_INVALID_ARG;
    const int k3 = k * k * k;
    for (int l = l_min; l <= l_max; ++l) {
        const double f = std::ldexp(1.0, -(l_max - l));
        for (int i = 0; i < k3; ++i) out[size_t(l - l_min) * k3 + i] = float(double(w[i]) * f);
    }
    return APR_OK;
}

apr_status_t apr_sobel_stencils(int32_t k, float *out) {
    if (!out) return APR_ERR_INVALID_ARG;
    if (k != 3) return APR_ERR_UNSUPPORTED;
    const double d[3] = {-0.5, 0.0, 0.5}, sm[3] = {0.25, 0.5, 0.25};
    for (int a = 0; a < 3; ++a)           // derivative axis: z, x, y
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int m = 0; m < 3; ++m) {
                    const double fz = a == 0 ? d[i] : sm[i], fx = a == 1 ? d[j] : sm[j], fy = a == 2 ? d[m] : sm[m];
                    out[((a * 3 + i) * 3 + j) * 3 + m] = float(fz * fx * fy);
                }
    return APR_OK;
}

}  // extern "C"
