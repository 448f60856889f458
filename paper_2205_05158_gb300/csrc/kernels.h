// Internal launch interface between the C-ABI layer (api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "common.cuh"

namespace fdk {

enum OutKind { OUT_F32 = 0, OUT_BF16 = 1, OUT_F16 = 2 };

// Every size a kernel needs, derived once at plan creation.
struct Geo {
    int M, K, N, N_d, first_bin, S_per_real, log2N;
    int n_orders, orders[8], L;
    int pa_G;                // PA cross-term length of Eq. 9 (0: memory polynomial)
    int in_all;              // the forward row kernel reads x_hat rows of all N bins (FD-NN chain)
    int row_ctas;            // CTAs per SM of the row kernels' persistent grids (0: as many as fit)
    int bin_ctas;            // CTAs per SM of the tensor-core contractions' grids (0: two, the most that fit)
    int bin_half;            // the generic tensor-core contractions take items of half the subcarriers
    int G, Go, L_U, Cin, K_C, K_S, pad, N_conv, F, residual;
    int n_convw;             // N_conv * Cin * K_C * K_C
    long off_cb, off_fw, off_fb, theta_len;
    double P_T;
};

// BF16 activation planes read by the tensor-core antenna -> user reductions (the FFT-PA
// outputs X and g_xhat of BF16 plans): [realisation][subcarrier / 4][symbol of the
// realisation][antenna][subcarrier % 4] of complex BF16, so that one reduction item -- 4
// subcarriers of one realisation, all its symbols and antennas -- is one contiguous block.
// The other planes (x_hat, g_X) keep rows [symbol][antenna][subcarrier].
struct BlkPlane {
    long per_group;   // elements of one subcarrier group: S_per_real x M x 4
    long per_real;    // elements of one realisation
    FD_HD explicit BlkPlane(const Geo &g)
        : per_group((long)g.S_per_real * g.M * 4), per_real((long)((g.N_d + 3) >> 2) * g.S_per_real * g.M * 4) {}
    // element of (symbol s, antenna m) at subcarrier 0 ...
    FD_HD long row(const Geo &g, long s, int m) const {
        return (s / g.S_per_real) * per_real + ((s % g.S_per_real) * g.M + m) * 4;
    }
    // ... plus this for subcarrier i
    FD_HD long sub(int i) const { return (long)(i >> 2) * per_group + (i & 3); }
    // first element of item (realisation r, subcarriers 4 j ..), then (slot t, antenna m) at 4 (t M + m)
    FD_HD long item(long r, int j) const { return r * per_real + (long)j * per_group; }
};
inline size_t blk_plane_bytes(const Geo &g, long S) {
    const long R = (S + g.S_per_real - 1) / g.S_per_real;
    return (size_t)R * BlkPlane(g).per_real * 4;
}

// zero-forcing precoder (Eq. 6): FP32 Gram, Cholesky + triangular inverse (FP64), W = H^H G^{-1}
size_t zf_scratch_bytes(const Geo &g, long nbins);
// H16 / W16 (optional, kind OUT_BF16 / OUT_F16): 16-bit copies of H and W written on the way
cudaError_t zf_build(const Geo &g, int R, const c32 *H, c32 *W, float *alpha, int *status, void *scratch,
                     void *H16, void *W16, int kind, cudaStream_t st);
// one of the three ZF kernels: 0 = Gram, 1 = factor / inverse, 2 = W (-1: all three).
// tc: W on the tensor cores when kind is 16-bit and M <= 128, K <= 16 (err: timeout word)
// keep_w32 = false: with the tensor-core apply, only the 16-bit copy of W is written
// fp64: Cholesky and triangular inverse in FP64 (else FP32; FP32 kinds always FP64)
// HH16 (16-bit kinds, may be null): the Gram phase also writes H^H in W's layout [bin][m][u]
cudaError_t zf_phase(int phase, const Geo &g, int R, const c32 *H, c32 *W, float *alpha, int *status, void *scratch,
                     void *H16, void *W16, int kind, bool tc, bool fp64, int *err, cudaStream_t st,
                     bool keep_w32 = true, void *HH16 = nullptr);
// out = Z X per (symbol, subcarrier) of S symbols, Z = G^{-1} = Y^H Y from the factor's Y
// in `scratch` (the realisations of those symbols, from the first); X, out [S][K][N_d]
cudaError_t zf_zmul(const Geo &g, int S, const void *scratch, const c32 *X, c32 *out, cudaStream_t st);
// W = H^H Z, Z = G^{-1} = Y^H Y formed in FP32 from the factor's Y = L^{-1} (lower triangle
// in its scratch layout), with BF16 hi / lo operand splits on the tensor cores; W16 of the
// given 16-bit kind beside it
cudaError_t zf_apply_tc(const Geo &g, long nbins, const c32 *H, const c32 *Zs, const float *alpha, c32 *W, void *W16,
                        int kind, int *err, cudaStream_t st);
// the tensor-core contractions: M <= 256 antennas, K <= 32 users
bool tc_bin_supported(const Geo &g);
// the tensor-core ZF apply (W = H^H Z): M <= 128, K <= 16
bool tc_apply_supported(const Geo &g);

// symbol errors at the users: counts[0] += errors, counts[1] += symbols compared
// wrong (may be null): per (symbol, user, subcarrier) 1 = error, 0 = correct, 2 = not compared
cudaError_t ser_count(const Geo &g, int S, const c32 *y, const c32 *s, const float *alpha, int Q, float N0,
                      unsigned long long seed, unsigned long long *counts, cudaStream_t st,
                      unsigned char *wrong = nullptr);
// a wait on an mbarrier nothing arrives at, bounded by limit_ns: sets err bit 2 when it gives up
cudaError_t wait_probe(unsigned long long limit_ns, int *err, cudaStream_t st);

// FD-CNN.  `user` < 0: the shared network over all S K columns (chain order, column
// t K + u); user u >= 0: user u's own pass over its S columns, FD-CNN column t reading
// and writing chain column t K + u of s, s_tilde and their gradients (the activations
// act / gact are that pass's own [S][.] block; theta / grad point at user u's set)
cudaError_t conv_forward(const Geo &g, int S, const c32 *s, const float *theta, float *act, cudaStream_t st,
                         int user = -1);
// gact: gradient at the pre-activations, [cols][ldg] FP32
cudaError_t conv_backward(const Geo &g, int S, const c32 *s, const float *gact, long ldg, float *partials,
                          cudaStream_t st, int user = -1);
// grad[conv_w, conv_b] = (accumulate ? grad + : ) the sum of the partial rows (cols: the
// columns of the conv_backward call)
cudaError_t conv_reduce(const Geo &g, int cols, const float *partials, float *grad, bool accumulate, cudaStream_t st);
cudaError_t colsum_fcb(const Geo &g, int cols, const float *gd, float *grad, cudaStream_t st, int user = -1);

// FP32 GEMM with the FD-CNN dense-layer layouts (rows of fc_w interleaved Re/Im)
cudaError_t fc_forward_f32(const Geo &g, int cols, const float *act, const float *theta, const c32 *s, c32 *st,
                           cudaStream_t stm, int user = -1);
cudaError_t fc_backward_data_f32(const Geo &g, int cols, const float *gd, const float *theta, const float *act,
                                 float *gpre, cudaStream_t stm, int user = -1);
cudaError_t fc_backward_weight_f32(const Geo &g, int cols, const float *gd, const float *act, float *grad,
                                   bool accumulate, cudaStream_t stm, int user = -1);

// per-subcarrier complex contractions (FP32 operands)
// With the precoder kept as its ZF factors (the 16-bit copies are H and H^H):
// ADJ_PRECODE_F: the adjoint of precoding, alpha H g (the A operand is H's own copy, read
// as in COMBINE; Z is applied afterwards); ADJ_COMBINE_F: the adjoint of combining,
// H^H g / alpha (the A operand is the H^H copy, read as in PRECODE)
enum BinMode { PRECODE = 0, ADJ_COMBINE = 1, COMBINE = 2, ADJ_PRECODE = 3, ADJ_PRECODE_F = 4, ADJ_COMBINE_F = 5 };
// A is FP32 (a_kind OUT_F32) or the 16-bit copy (OUT_BF16 / OUT_F16) of W or H
cudaError_t bin_expand(const Geo &g, int mode, int S, const void *A, int a_kind, const float *alpha, const c32 *B,
                       c32 *out, cudaStream_t st);
cudaError_t bin_reduce(const Geo &g, int mode, int S, const void *A, int a_kind, const float *alpha, const c32 *B,
                       c32 *out, const c32 *s_ref, c32 *gy, double *metrics, double inv_count, cudaStream_t st);
// tcgen05 versions for 16-bit H / W copies (M <= 128, K <= 16); err: sticky timeout word
// act_kind: storage of the antenna-side activations (the expand's output, the reduce's
// input): OUT_F32, or OUT_BF16 in BF16 plans (then b_scale must be 1)
cudaError_t tc_bin_expand(const Geo &g, int mode, int S, const void *A, int a_kind, const float *alpha, const c32 *B,
                          void *out, int act_kind, float b_scale, int *err, cudaStream_t st);
cudaError_t tc_bin_reduce(const Geo &g, int mode, int S, const void *A, int a_kind, const float *alpha, const void *B,
                          int act_kind, c32 *out, const c32 *s_ref, c32 *gy, double *metrics, double inv_count,
                          float b_scale, int *err, cudaStream_t st);
cudaError_t to_16bit(long n, const c32 *in, void *out, int kind, cudaStream_t st);

// OFDM + PA rows
size_t fftpa_smem_bytes(const Geo &g, bool adjoint);
// xt (BF16 planes only, may be null): the forward stores the time-domain PA input there
// [rows][N], and the adjoint reads it instead of transforming x_hat again.  With BF16
// planes, X (forward) and gxh (adjoint) are written in the blocked layout (BlkPlane);
// x_hat and gX are rows, so gxh may not alias gX then.
cudaError_t fftpa_forward(const Geo &g, int rows, const c32 *xh, const c32 *pa, const c32 *tw, void *X, int out_kind,
                          double *metrics, void *xt, cudaStream_t st);
cudaError_t fftpa_adjoint(const Geo &g, int rows, const c32 *xh, const c32 *pa, const c32 *tw, const void *gX, void *gxh,
                          int act_kind, const void *xt, cudaStream_t st);

// FP64 check of H_k W_k = I on every `every`-th of nbins subcarriers: *out (device) =
// max over them of max_ij |(H_k W_k - I)_ij|
cudaError_t zf_residual(const Geo &g, long nbins, long every, const c32 *H, const c32 *W, double *out,
                        cudaStream_t st);
// FMA-loop peak of the FP32 (kind 0 scalar, 1 packed pairs) or FP64 (kind 2) pipe, TFLOP/s
cudaError_t alu_peak(int kind, double *tflops, cudaStream_t st);

// FD-NN comparison workload (Sec. III-C), FP32: per-user IDFT of the data bins into
// t [S K][N]; the time-domain network at every sample into o [S K][N]; the per-user DFT
// of o in place (every bin); alpha of the data bins from the all-bins alpha
struct FdnnDesc {
    int L4, D, layers, residual;
};
cudaError_t fdnn_user_rows(const Geo &g, long rows, bool inverse, const c32 *in, c32 *out, const c32 *tw,
                           cudaStream_t st);
cudaError_t fdnn_mlp(const Geo &g, const FdnnDesc &nn, int S, const float *theta, const c32 *t, c32 *o,
                     cudaStream_t st);
cudaError_t fdnn_alpha_data(const Geo &g, int R, const float *alpha_all, float *alpha, cudaStream_t st);
long fdnn_theta_len(const Geo &g, const FdnnDesc &nn);

// parameter updates and bookkeeping
// gscale multiplies the gradient (1: the library's own steps)
cudaError_t sgd_step(long n, float *theta, const float *grad, float lr, cudaStream_t st, float gscale = 1.0f);
cudaError_t adam_step(long n, float *theta, const float *grad, float *m, float *v, float lr, float c1, float c2,
                      cudaStream_t st, float gscale = 1.0f);
cudaError_t finalize_metrics(double *metrics, double inv_count, cudaStream_t st);
cudaError_t twiddles(int N, c32 *tw, cudaStream_t st);
cudaError_t pass_twiddles(int log2N, c32 *tw, cudaStream_t st);

}  // namespace fdk
