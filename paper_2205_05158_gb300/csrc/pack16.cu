// 16-bit operand preparation for the tensor-core dense layer: BF16 activations from
// the convolution, interleaved-row (n' = 2 i + c) and transposed copies of fc_w, and
// tiled transposes (32 x 32 tiles through shared memory, coalesced on both sides).
#include "common.cuh"
#include "kernels.h"
#include "tc_gemm.h"

namespace fdk {

// out[n'][f] = bf16(fc_w[pi(n')][f])
__global__ void pack_fcw_kernel(Geo g, const float *__restrict__ fw, __nv_bfloat16 *__restrict__ out, long ld) {
    const long n = blockIdx.y;
    const long src = (n & 1) * g.N_d + (n >> 1);
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < g.F; f += gridDim.x * blockDim.x)
        out[n * ld + f] = __float2bfloat16_rn(fw[src * g.F + f]);
}

cudaError_t pack_fcw(const Geo &g, const float *theta, __nv_bfloat16 *out, long ld_out, cudaStream_t st) {
    dim3 grid((g.F + 255) / 256, 2 * g.N_d);
    pack_fcw_kernel<<<grid, 256, 0, st>>>(g, theta + g.off_fw, out, ld_out);
    return cudaGetLastError();
}

// Tiled transpose: out[c][r] = in(r, c); in(r, c) = in[rowmap(r) * ld_in + c]
template <typename Tin, bool PERM>
__global__ void transpose_kernel(const Tin *__restrict__ in, long rows, long cols, long ld_in, int Nd,
                                 __nv_bfloat16 *__restrict__ out, long ld_out) {
    __shared__ float tile[32][33];
    const long r0 = (long)blockIdx.y * 32, c0 = (long)blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    for (int k = ty; k < 32; k += 8) {
        const long r = r0 + k, c = c0 + tx;
        float v = 0.f;
        if (r < rows && c < cols) {
            const long rr = PERM ? ((r & 1) * Nd + (r >> 1)) : r;
            if constexpr (sizeof(Tin) == 4) v = (float)in[rr * ld_in + c];
            else v = __bfloat162float(in[rr * ld_in + c]);
        }
        tile[k][tx] = v;
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const long c = c0 + k, r = r0 + tx;
        if (c < cols && r < rows) out[c * ld_out + r] = __float2bfloat16_rn(tile[tx][k]);
    }
}

template <typename Tin, bool PERM>
static cudaError_t run_transpose(const Tin *in, long rows, long cols, long ld_in, int Nd, __nv_bfloat16 *out,
                                 long ld_out, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    transpose_kernel<Tin, PERM><<<grid, dim3(32, 8), 0, st>>>(in, rows, cols, ld_in, Nd, out, ld_out);
    return cudaGetLastError();
}

cudaError_t pack_fcw_t(const Geo &g, const float *theta, __nv_bfloat16 *out, long ld_out, cudaStream_t st) {
    // rows n' (interleaved), cols f  ->  out[f][n']
    return run_transpose<float, true>(theta + g.off_fw, 2L * g.N_d, g.F, g.F, g.N_d, out, ld_out, st);
}

cudaError_t transpose_bf16(const float *in, long rows, long cols, long ld_in, __nv_bfloat16 *out, long ld_out,
                           cudaStream_t st) {
    return run_transpose<float, false>(in, rows, cols, ld_in, 0, out, ld_out, st);
}

cudaError_t transpose_bf16(const __nv_bfloat16 *in, long rows, long cols, long ld_in, __nv_bfloat16 *out, long ld_out,
                           cudaStream_t st) {
    return run_transpose<__nv_bfloat16, false>(in, rows, cols, ld_in, 0, out, ld_out, st);
}

__global__ void to_bf16_kernel(const float *__restrict__ in, long rows, long cols, long ld_in,
                               __nv_bfloat16 *__restrict__ out, long ld_out) {
    const long r = blockIdx.y;
    for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < cols; c += (long)gridDim.x * blockDim.x)
        out[r * ld_out + c] = __float2bfloat16_rn(in[r * ld_in + c]);
}

cudaError_t to_bf16(const float *in, long rows, long cols, long ld_in, __nv_bfloat16 *out, long ld_out,
                    cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const long bx = (cols + 255) / 256;
    dim3 grid((unsigned)(bx < 64 ? bx : 64), (unsigned)rows);
    to_bf16_kernel<<<grid, 256, 0, st>>>(in, rows, cols, ld_in, out, ld_out);
    return cudaGetLastError();
}

}  // namespace fdk
