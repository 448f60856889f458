// Tensor-core (tcgen05) GEMM launchers: C[m][n] = sum_k A[m][k] B[n][k], 16-bit operands,
// both row-major with k contiguous (leading dimensions in elements, multiples of 8).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace fdk {

struct GemmArgs {
    const void *A;   // [M][lda]
    const void *B;   // [N][ldb]
    int M, N, K;
    long lda, ldb;
    int ab_type;     // 1 = BF16, 0 = FP16
    int splits;      // K slices (partial sums are added by the epilogue)
};

cudaError_t tc_gemm_store(const GemmArgs &g, float *C, long ldc, int *err, cudaStream_t st);
// fbi: fc_b in the output's interleaved order [2 N_d] (as pack_fcw writes it)
// output row m is chain column m row_mul + row_add of s and s_tilde (per-user passes: K, u)
cudaError_t tc_fc_forward(const GemmArgs &g, float *st_out, const float *s, const float *fbi, int Nd, int residual,
                          int *err, cudaStream_t st, int row_mul = 1, int row_add = 0);
// gpre [rows][ld_g] FP32 (ld_g a multiple of 8 for whole-sector stores)
cudaError_t tc_fc_backward_data(const GemmArgs &g, float *gpre, long ld_g, const __nv_bfloat16 *act, long ld_act,
                                int *err, cudaStream_t st);
cudaError_t tc_fc_backward_weight(const GemmArgs &g, float *gfw, int Nd, int F, int *err, cudaStream_t st);

// 16-bit operand preparation (pack16.cu)
cudaError_t conv_forward_bf16(const struct Geo &g, int S, const float2 *s, const float *theta, __nv_bfloat16 *act,
                              long ld, cudaStream_t st, int user = -1);
// fc_w rows in interleaved order: out[n'][f] = bf16(fc_w[pi(n')][f]), ld_out; and the
// bias in the same order, fbi[n'] = fc_b[pi(n')] (FP32)
cudaError_t pack_fcw(const struct Geo &g, const float *theta, __nv_bfloat16 *out, long ld_out, float *fbi,
                     cudaStream_t st);
// transposed: out[f][n'] = bf16(fc_w[pi(n')][f]), ld_out
cudaError_t pack_fcw_t(const struct Geo &g, const float *theta, __nv_bfloat16 *out, long ld_out, cudaStream_t st);
// out[r][c] = bf16(in[r][c]) for a float matrix
// bf16 copy and bf16 transpose of an FP32 matrix in one pass
cudaError_t bf16_and_transpose(const float *in, long rows, long cols, long ld_in, __nv_bfloat16 *out, long ld_out,
                               __nv_bfloat16 *outT, long ld_t, cudaStream_t st);
cudaError_t to_bf16(const float *in, long rows, long cols, long ld_in, __nv_bfloat16 *out, long ld_out,
                    cudaStream_t st);
// out[c][r] = in[r][c] (float or bf16 input)
cudaError_t transpose_bf16(const float *in, long rows, long cols, long ld_in, __nv_bfloat16 *out, long ld_out,
                           cudaStream_t st);
cudaError_t transpose_bf16(const __nv_bfloat16 *in, long rows, long cols, long ld_in, __nv_bfloat16 *out, long ld_out,
                           cudaStream_t st);

}  // namespace fdk
