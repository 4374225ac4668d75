// Element-wise layers of the APR-native CNN (the learned per-level filters Sec. 6 proposes): the
// input embedding into 16 bfloat16 channels, ReLU with rounding to bfloat16 between convolution
// layers, the residual read-out, and their transposes. One thread per value, grid-stride loops.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>

#include "apr_internal.h"

namespace aprk {
namespace {

constexpr int CH = 16;       // channels per particle
constexpr int EW_NT = 256;   // threads per block of the element-wise kernels

__device__ __forceinline__ uint16_t to_bf16_bits(float v) {
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    return *reinterpret_cast<const uint16_t *>(&b);
}

int ew_blocks(int64_t n) {
    const int64_t b = (n + EW_NT - 1) / EW_NT;
    return int(b < 1 ? 1 : (b > 65535 * 4 ? 65535 * 4 : b));
}

__global__ void embed_kernel(const float *__restrict__ x, int64_t n, float scale, uint16_t *__restrict__ out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n * CH; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = (i % CH == 0) ? to_bf16_bits(__fmul_rn(scale, x[i / CH])) : uint16_t(0);
}

__global__ void relu_kernel(const float *__restrict__ in, int64_t n, uint16_t *__restrict__ out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = to_bf16_bits(fmaxf(in[i], 0.f));
}

__global__ void relu_backward_kernel(const float *__restrict__ pre, const float *__restrict__ gpost, int64_t n,
                                     uint16_t *__restrict__ gpre) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        gpre[i] = to_bf16_bits(pre[i] > 0.f ? gpost[i] : 0.f);
}

__global__ void readout_kernel(const float *__restrict__ conv, const float *__restrict__ x, int64_t n, float inv_scale,
                               float *__restrict__ y) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[i] = __fadd_rn(x[i], __fmul_rn(inv_scale, conv[i * CH]));
}

__global__ void readout_backward_kernel(const float *__restrict__ gy, int64_t n, float inv_scale,
                                        uint16_t *__restrict__ gconv) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n * CH; i += int64_t(gridDim.x) * blockDim.x)
        gconv[i] = (i % CH == 0) ? to_bf16_bits(__fmul_rn(inv_scale, gy[i / CH])) : uint16_t(0);
}

}  // namespace
}  // namespace aprk

using namespace aprk;

extern "C" {

apr_status_t apr_mc_embed_bf16(const float *x, int64_t n, float scale, uint16_t *out, apr_stream_t stream) {
    if (n < 0 || (n && (!x || !out))) return APR_ERR_INVALID_ARG;
    if (n) embed_kernel<<<ew_blocks(n * CH), EW_NT, 0, stream>>>(x, n, scale, out);
    return cuda_status(cudaGetLastError());
}

apr_status_t apr_mc_relu_bf16(const float *in, int64_t n_values, uint16_t *out, apr_stream_t stream) {
    if (n_values < 0 || (n_values && (!in || !out))) return APR_ERR_INVALID_ARG;
    if (n_values) relu_kernel<<<ew_blocks(n_values), EW_NT, 0, stream>>>(in, n_values, out);
    return cuda_status(cudaGetLastError());
}

apr_status_t apr_mc_relu_backward_bf16(const float *pre, const float *grad_post, int64_t n_values, uint16_t *grad_pre,
                                       apr_stream_t stream) {
    if (n_values < 0 || (n_values && (!pre || !grad_post || !grad_pre))) return APR_ERR_INVALID_ARG;
    if (n_values) relu_backward_kernel<<<ew_blocks(n_values), EW_NT, 0, stream>>>(pre, grad_post, n_values, grad_pre);
    return cuda_status(cudaGetLastError());
}

apr_status_t apr_mc_readout(const float *conv, const float *x, int64_t n, float inv_scale, float *y, apr_stream_t stream) {
    if (n < 0 || (n && (!conv || !x || !y))) return APR_ERR_INVALID_ARG;
    if (n) readout_kernel<<<ew_blocks(n), EW_NT, 0, stream>>>(conv, x, n, inv_scale, y);
    return cuda_status(cudaGetLastError());
}

apr_status_t apr_mc_readout_backward_bf16(const float *grad_y, int64_t n, float inv_scale, uint16_t *grad_conv,
                                          apr_stream_t stream) {
    if (n < 0 || (n && (!grad_y || !grad_conv))) return APR_ERR_INVALID_ARG;
    if (n) readout_backward_kernel<<<ew_blocks(n * CH), EW_NT, 0, stream>>>(grad_y, n, inv_scale, grad_conv);
    return cuda_status(cudaGetLastError());
}

}  // extern "C"
