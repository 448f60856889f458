// 16-bit operand preparation for the tensor-core dense layer: BF16 activations from
// the convolution, interleaved-row (n' = 2 i + c) and transposed copies of fc_w, and
// tiled transposes (32 x 32 tiles through shared memory, coalesced on both sides).
#include "common.cuh"
#include "kernels.h"
#include "tc_gemm.h"

namespace fdk {

// out[n'][f] = bf16(fc_w[pi(n')][f])
__global__ void pack_fcw_kernel(Geo g, const float *__restrict__ fw, const float *__restrict__ fb,
                                __nv_bfloat16 *__restrict__ out, long ld, float *__restrict__ fbi) {
    const long n = blockIdx.y;
    const long src = (n & 1) * g.N_d + (n >> 1);
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < g.F; f += gridDim.x * blockDim.x)
        out[n * ld + f] = __float2bfloat16_rn(fw[src * g.F + f]);
    if (blockIdx.x == 0 && threadIdx.x == 0) fbi[n] = fb[src];
}

cudaError_t pack_fcw(const Geo &g, const float *theta, __nv_bfloat16 *out, long ld_out, float *fbi, cudaStream_t st) {
    dim3 grid((g.F + 255) / 256, 2 * g.N_d);
    pack_fcw_kernel<<<grid, 256, 0, st>>>(g, theta + g.off_fw, theta + g.off_fb, out, ld_out, fbi);
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

// BF16 to BF16 transpose in 64 x 64 tiles, two elements per 4-byte access on both sides
// (a warp reads and writes 128 contiguous bytes); needs even leading dimensions and
// 4-byte aligned bases
__global__ void __launch_bounds__(256) transpose16_kernel(const __nv_bfloat16 *__restrict__ in, long rows, long cols,
                                                          long ld_in, __nv_bfloat16 *__restrict__ out, long ld_out) {
    __shared__ __nv_bfloat16 tile[64][66];   // [column][row], padded
    const long r0 = (long)blockIdx.y * 64, c0 = (long)blockIdx.x * 64;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 column pairs x 8 rows
    for (int k = ty; k < 64; k += 8) {
        const long r = r0 + k, c = c0 + 2 * tx;
        __nv_bfloat162 b = __floats2bfloat162_rn(0.f, 0.f);
        if (r < rows) {
            if (c + 1 < cols) b = *reinterpret_cast<const __nv_bfloat162 *>(in + r * ld_in + c);
            else if (c < cols) b.x = in[r * ld_in + c];
        }
        tile[2 * tx][k] = b.x;
        tile[2 * tx + 1][k] = b.y;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * 32; e += 256) {   // 64 columns x 32 row pairs
        const int cc = e >> 5, rp = e & 31;
        const long c = c0 + cc, r = r0 + 2 * rp;
        if (c >= cols || r >= rows) continue;
        if (r + 1 < rows) {
            __nv_bfloat162 b;
            b.x = tile[cc][2 * rp];
            b.y = tile[cc][2 * rp + 1];
            *reinterpret_cast<__nv_bfloat162 *>(out + c * ld_out + r) = b;
        } else {
            out[c * ld_out + r] = tile[cc][2 * rp];
        }
    }
}

cudaError_t transpose_bf16(const __nv_bfloat16 *in, long rows, long cols, long ld_in, __nv_bfloat16 *out, long ld_out,
                           cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    if ((ld_in | ld_out) & 1 || (reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 3)
        return run_transpose<__nv_bfloat16, false>(in, rows, cols, ld_in, 0, out, ld_out, st);
    dim3 grid((unsigned)((cols + 63) / 64), (unsigned)((rows + 63) / 64));
    transpose16_kernel<<<grid, 256, 0, st>>>(in, rows, cols, ld_in, out, ld_out);
    return cudaGetLastError();
}

// One pass over an FP32 matrix in[rows][ld_in] (cols valid) writing both its BF16 copy
// out[rows][ld_out] and its BF16 transpose outT[cols][ld_t]: 32 x 64 tiles, pairs of
// elements (8-byte loads, 4-byte stores) on both sides, the transpose through shared memory.
__global__ void __launch_bounds__(256) bf16_and_transpose_kernel(const float *__restrict__ in, long rows, long cols,
                                                                 long ld_in, __nv_bfloat16 *__restrict__ out,
                                                                 long ld_out, __nv_bfloat16 *__restrict__ outT,
                                                                 long ld_t) {
    __shared__ __nv_bfloat16 tile[64][34];   // [column][row], padded
    const long r0 = (long)blockIdx.y * 32, c0 = (long)blockIdx.x * 64;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 column pairs x 8 rows
    for (int k = ty; k < 32; k += 8) {
        const long r = r0 + k, c = c0 + 2 * tx;
        float2 v = make_float2(0.f, 0.f);
        if (r < rows) {
            if (c + 1 < cols) v = *reinterpret_cast<const float2 *>(in + r * ld_in + c);
            else if (c < cols) v.x = in[r * ld_in + c];
        }
        const __nv_bfloat162 b = __floats2bfloat162_rn(v.x, v.y);
        if (r < rows && c + 1 < cols) *reinterpret_cast<__nv_bfloat162 *>(out + r * ld_out + c) = b;
        else if (r < rows && c < cols) out[r * ld_out + c] = b.x;
        tile[2 * tx][k] = b.x;
        tile[2 * tx + 1][k] = b.y;
    }
    __syncthreads();
    // transpose: 64 columns x 16 row pairs
    for (int e = threadIdx.x; e < 64 * 16; e += 256) {
        const int cc = e >> 4, rp = e & 15;
        const long c = c0 + cc, r = r0 + 2 * rp;
        if (c >= cols || r >= rows) continue;
        if (r + 1 < rows) {
            __nv_bfloat162 b;
            b.x = tile[cc][2 * rp];
            b.y = tile[cc][2 * rp + 1];
            *reinterpret_cast<__nv_bfloat162 *>(outT + c * ld_t + r) = b;
        } else {
            outT[c * ld_t + r] = tile[cc][2 * rp];
        }
    }
}

cudaError_t bf16_and_transpose(const float *in, long rows, long cols, long ld_in, __nv_bfloat16 *out, long ld_out,
                               __nv_bfloat16 *outT, long ld_t, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    // pairs must stay 4-byte aligned: even leading dimensions and bases
    if ((ld_in & 1) || (ld_out & 1) || (ld_t & 1) || (reinterpret_cast<uintptr_t>(in) & 7) ||
        (reinterpret_cast<uintptr_t>(out) & 3) || (reinterpret_cast<uintptr_t>(outT) & 3)) {
        cudaError_t e = to_bf16(in, rows, cols, ld_in, out, ld_out, st);
        return e == cudaSuccess ? transpose_bf16(in, rows, cols, ld_in, outT, ld_t, st) : e;
    }
    dim3 grid((unsigned)((cols + 63) / 64), (unsigned)((rows + 31) / 32));
    bf16_and_transpose_kernel<<<grid, 256, 0, st>>>(in, rows, cols, ld_in, out, ld_out, outT, ld_t);
    return cudaGetLastError();
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
