// Dense pixel-grid correlation with one k^3 stencil (k = 3 or 5), FP32: the dense comparison of
// the paper's results (a pixel-image convolution of the same size as the APR one, Sec. 6.1).
// 2.5-D blocking: a block owns a (TX x TY) tile of (x, y) columns and ZC consecutive z planes; the
// input planes z0 - R .. z0 + ZC + R - 1 pass through shared memory one at a time (double
// buffered), and every thread keeps the running sums of the k output planes an input plane feeds
// in a register ring, writing each output plane once it is complete.
#include <cuda_runtime.h>

#include <cstdint>

#include "apr_internal.h"

namespace aprk {
namespace {

constexpr int DTY = 64, DTX = 8, DZC = 32;  // tile: 64 y x 8 x columns, 32 z planes per block

__device__ __forceinline__ int64_t dense_reflect(int64_t i, int64_t d) {
    const int64_t p = 2 * d;
    int64_t m = i % p;
    if (m < 0) m += p;
    return m >= d ? p - 1 - m : m;
}

template <int R>
__global__ void __launch_bounds__(DTY * DTX) dense_conv_kernel(const float *__restrict__ img, int64_t dz, int64_t dx,
                                                               int64_t dy, const float *__restrict__ w, int bc,
                                                               float *__restrict__ out) {
    constexpr int K = 2 * R + 1, PXD = DTX + 2 * R, PYD = DTY + 2 * R;
    __shared__ float plane[2][PXD][PYD + 1];
    __shared__ float ws[K * K * K];
    const int ty = threadIdx.x, tx = threadIdx.y, tid = tx * DTY + ty;
    const int64_t y0 = int64_t(blockIdx.x) * DTY, x0 = int64_t(blockIdx.y) * DTX, z0 = int64_t(blockIdx.z) * DZC;
    for (int i = tid; i < K * K * K; i += DTY * DTX) ws[i] = w[i];
    const bool reflect = bc == APR_BC_REFLECT;
    // stage input plane z (reflected, or zero outside the image) into buffer b
    auto stage = [&](int64_t z, int b) {
        const bool zin = z >= 0 && z < dz;
        const int64_t zr = zin ? z : dense_reflect(z, dz);
        for (int i = tid; i < PXD * PYD; i += DTY * DTX) {
            const int a = i / PYD, c = i % PYD;
            int64_t x = x0 - R + a, y = y0 - R + c;
            const bool in = zin && x >= 0 && x < dx && y >= 0 && y < dy;
            float v = 0.f;
            if (in || reflect) {
                x = dense_reflect(x, dx);
                y = dense_reflect(y, dy);
                v = img[(zr * dx + x) * dy + y];
            }
            plane[b][a][c] = v;
        }
    };
    float acc[K];
#pragma unroll
    for (int i = 0; i < K; ++i) acc[i] = 0.f;
    const int64_t x = x0 + tx, y = y0 + ty;
    const bool mine = x < dx && y < dy;
    const int64_t zend = z0 + DZC < dz ? z0 + DZC : dz;
    stage(z0 - R, 0);
    __syncthreads();
    // input plane zi feeds output planes zi - R .. zi + R with tap (zi - zo) + R along z; the ring
    // slot of output plane zo is (zo - z0 + R) mod K... kept in acc[] by rotation after each plane
    for (int64_t zi = z0 - R; zi < zend + R; ++zi) {
        const int b = int((zi - (z0 - R)) & 1);
        if (zi + 1 < zend + R) stage(zi + 1, b ^ 1);
        // acc[j] accumulates output plane zo = zi - R + j ... tap along z: zi - zo + R = 2R - j
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const float *wz = ws + (2 * R - j) * K * K;
            float s = acc[j];
#pragma unroll
            for (int a = 0; a < K; ++a)
#pragma unroll
                for (int c = 0; c < K; ++c) s = fmaf(wz[a * K + c], plane[b][tx + a][ty + c], s);
            acc[j] = s;
        }
        // output plane zi - R is complete
        const int64_t zo = zi - R;
        if (mine && zo >= z0 && zo < zend) out[(zo * dx + x) * dy + y] = acc[0];
#pragma unroll
        for (int j = 0; j < K - 1; ++j) acc[j] = acc[j + 1];
        acc[K - 1] = 0.f;
        __syncthreads();
    }
}

}  // namespace
}  // namespace aprk

extern "C" apr_status_t apr_dense_convolve(const float *image, int64_t dz, int64_t dx, int64_t dy, const float *stencil,
                                           int32_t k, int32_t bc, float *out, apr_stream_t stream) {
    using namespace aprk;
    if (k != 3 && k != 5) return APR_ERR_UNSUPPORTED;
    if (bc != APR_BC_REFLECT && bc != APR_BC_ZERO) return APR_ERR_INVALID_ARG;
    if (dz < 1 || dx < 1 || dy < 1 || !image || !stencil || !out) return APR_ERR_INVALID_ARG;
    const dim3 grid(unsigned((dy + DTY - 1) / DTY), unsigned((dx + DTX - 1) / DTX), unsigned((dz + DZC - 1) / DZC));
    if (grid.y > 65535 || grid.z > 65535) return APR_ERR_UNSUPPORTED;
    const dim3 block(DTY, DTX);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (k == 3) dense_conv_kernel<1><<<grid, block, 0, s>>>(image, dz, dx, dy, stencil, bc, out);
    else dense_conv_kernel<2><<<grid, block, 0, s>>>(image, dz, dx, dy, stencil, bc, out);
    return cuda_status(cudaGetLastError());
}
