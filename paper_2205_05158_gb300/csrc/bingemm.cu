// Dispatch of the per-subcarrier contractions (bingemm.cuh) by operand storage, and
// the 16-bit copies of H and W.
#include "bingemm.cuh"

namespace fdk {

cudaError_t bin_expand(const Geo &g, int mode, int S, const void *A, int a_kind, const float *alpha, const c32 *B,
                       c32 *out, cudaStream_t st) {
    if (a_kind == OUT_BF16) return bin_expand_bf16(g, mode, S, A, alpha, B, out, st);
    if (a_kind == OUT_F16) return bin_expand_f16(g, mode, S, A, alpha, B, out, st);
    return bin_expand_f32(g, mode, S, A, alpha, B, out, st);
}

cudaError_t bin_reduce(const Geo &g, int mode, int S, const void *A, int a_kind, const float *alpha, const c32 *B,
                       c32 *out, const c32 *s_ref, c32 *gy, double *metrics, double inv_count, cudaStream_t st) {
    if (a_kind == OUT_BF16) return bin_reduce_bf16(g, mode, S, A, alpha, B, out, s_ref, gy, metrics, inv_count, st);
    if (a_kind == OUT_F16) return bin_reduce_f16(g, mode, S, A, alpha, B, out, s_ref, gy, metrics, inv_count, st);
    return bin_reduce_f32(g, mode, S, A, alpha, B, out, s_ref, gy, metrics, inv_count, st);
}

// 16-bit copies of H [R][N_d][K][M] and W [R][N_d][M][K] (same layouts)
template <typename T>
__global__ void convert16_kernel(long n, const c32 *__restrict__ in, T *__restrict__ out) {
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x)
        out[j] = Operand<T>::from(in[j]);
}

cudaError_t to_16bit(long n, const c32 *in, void *out, int kind, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const long b = (n + 255) / 256;
    const unsigned blocks = (unsigned)(b < 152 * 32 ? b : 152 * 32);
    if (kind == OUT_BF16) convert16_kernel<<<blocks, 256, 0, st>>>(n, in, (cbf16 *)out);
    else convert16_kernel<<<blocks, 256, 0, st>>>(n, in, (cf16 *)out);
    return cudaGetLastError();
}

}  // namespace fdk
