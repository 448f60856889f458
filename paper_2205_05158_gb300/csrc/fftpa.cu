// Dispatch of the OFDM + PA row kernels (fftpa.cuh) by transform size, and the
// per-pass twiddle tables.
#include "fftpa.cuh"

namespace fdk {

// Twiddle tables of the radix-16 passes: entry [tw_off(i) + (r - 1) Ns + k] =
// exp(-j 2 pi r k / (16 Ns)) for the pass of span Ns (Ns = R0, 16 R0, ... < N).
__global__ void pass_twiddle_kernel(int log2N, c32 *out) {
    const int N = 1 << log2N;
    const int R0 = 1 << (log2N % 4 == 0 ? 4 : log2N % 4);
    int off = 0;
    for (int Ns = R0; Ns < N; Ns *= 16) {
        for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < 15 * Ns; e += blockDim.x * gridDim.x) {
            const int r = e / Ns + 1, k = e % Ns;
            double s, c;
            sincospi(-2.0 * (double)(r * k) / (double)(16 * Ns), &s, &c);
            out[off + e] = make_float2((float)c, (float)s);
        }
        off += 15 * Ns;
    }
}

size_t fftpa_smem_bytes(const Geo &g, bool /*adjoint*/) { return fftpa_smem_bytes_(g); }

cudaError_t fftpa_forward(const Geo &g, int rows, const c32 *xh, const c32 *pa, const c32 *twp, void *X, int out_kind,
                          double *metrics, void *xt_out, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    if (out_kind != OUT_F32 && out_kind != OUT_BF16) return cudaErrorInvalidValue;
    if (xt_out && out_kind != OUT_BF16) return cudaErrorInvalidValue;
    cbf16 *xt = static_cast<cbf16 *>(xt_out);
    const bool a16 = out_kind == OUT_BF16;
    switch (g.log2N) {
        case 6: return a16 ? fftpa_fwd16_6(g, rows, xh, pa, twp, static_cast<cbf16 *>(X), metrics, xt, st)
                     : fftpa_fwd_6(g, rows, xh, pa, twp, static_cast<c32 *>(X), metrics, st);
        case 7: return a16 ? fftpa_fwd16_7(g, rows, xh, pa, twp, static_cast<cbf16 *>(X), metrics, xt, st)
                     : fftpa_fwd_7(g, rows, xh, pa, twp, static_cast<c32 *>(X), metrics, st);
        case 8: return a16 ? fftpa_fwd16_8(g, rows, xh, pa, twp, static_cast<cbf16 *>(X), metrics, xt, st)
                     : fftpa_fwd_8(g, rows, xh, pa, twp, static_cast<c32 *>(X), metrics, st);
        case 9: return a16 ? fftpa_fwd16_9(g, rows, xh, pa, twp, static_cast<cbf16 *>(X), metrics, xt, st)
                     : fftpa_fwd_9(g, rows, xh, pa, twp, static_cast<c32 *>(X), metrics, st);
        case 10: return a16 ? fftpa_fwd16_10(g, rows, xh, pa, twp, static_cast<cbf16 *>(X), metrics, xt, st)
                     : fftpa_fwd_10(g, rows, xh, pa, twp, static_cast<c32 *>(X), metrics, st);
        case 11: return a16 ? fftpa_fwd16_11(g, rows, xh, pa, twp, static_cast<cbf16 *>(X), metrics, xt, st)
                     : fftpa_fwd_11(g, rows, xh, pa, twp, static_cast<c32 *>(X), metrics, st);
        case 12: return a16 ? fftpa_fwd16_12(g, rows, xh, pa, twp, static_cast<cbf16 *>(X), metrics, xt, st)
                     : fftpa_fwd_12(g, rows, xh, pa, twp, static_cast<c32 *>(X), metrics, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t fftpa_adjoint(const Geo &g, int rows, const c32 *xh, const c32 *pa, const c32 *twp, const void *gX,
                          void *gxh, int act_kind, const void *xt_in, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    if (act_kind != OUT_F32 && act_kind != OUT_BF16) return cudaErrorInvalidValue;
    if (xt_in && act_kind != OUT_BF16) return cudaErrorInvalidValue;
    const cbf16 *xt = static_cast<const cbf16 *>(xt_in);
    const bool a16 = act_kind == OUT_BF16;
    if (a16 && gX == gxh) return cudaErrorInvalidValue;   // rows in, blocked plane out
    switch (g.log2N) {
        case 6:
            return a16 ? fftpa_adj16_6(g, rows, xh, pa, twp, static_cast<const cbf16 *>(gX), static_cast<cbf16 *>(gxh), xt, st)
                       : fftpa_adj_6(g, rows, xh, pa, twp, static_cast<const c32 *>(gX), static_cast<c32 *>(gxh), st);
        case 7:
            return a16 ? fftpa_adj16_7(g, rows, xh, pa, twp, static_cast<const cbf16 *>(gX), static_cast<cbf16 *>(gxh), xt, st)
                       : fftpa_adj_7(g, rows, xh, pa, twp, static_cast<const c32 *>(gX), static_cast<c32 *>(gxh), st);
        case 8:
            return a16 ? fftpa_adj16_8(g, rows, xh, pa, twp, static_cast<const cbf16 *>(gX), static_cast<cbf16 *>(gxh), xt, st)
                       : fftpa_adj_8(g, rows, xh, pa, twp, static_cast<const c32 *>(gX), static_cast<c32 *>(gxh), st);
        case 9:
            return a16 ? fftpa_adj16_9(g, rows, xh, pa, twp, static_cast<const cbf16 *>(gX), static_cast<cbf16 *>(gxh), xt, st)
                       : fftpa_adj_9(g, rows, xh, pa, twp, static_cast<const c32 *>(gX), static_cast<c32 *>(gxh), st);
        case 10:
            return a16 ? fftpa_adj16_10(g, rows, xh, pa, twp, static_cast<const cbf16 *>(gX), static_cast<cbf16 *>(gxh), xt, st)
                       : fftpa_adj_10(g, rows, xh, pa, twp, static_cast<const c32 *>(gX), static_cast<c32 *>(gxh), st);
        case 11:
            return a16 ? fftpa_adj16_11(g, rows, xh, pa, twp, static_cast<const cbf16 *>(gX), static_cast<cbf16 *>(gxh), xt, st)
                       : fftpa_adj_11(g, rows, xh, pa, twp, static_cast<const c32 *>(gX), static_cast<c32 *>(gxh), st);
        case 12:
            return a16 ? fftpa_adj16_12(g, rows, xh, pa, twp, static_cast<const cbf16 *>(gX), static_cast<cbf16 *>(gxh), xt, st)
                       : fftpa_adj_12(g, rows, xh, pa, twp, static_cast<const c32 *>(gX), static_cast<c32 *>(gxh), st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t pass_twiddles(int log2N, c32 *out, cudaStream_t st) {
    pass_twiddle_kernel<<<8, 256, 0, st>>>(log2N, out);
    return cudaGetLastError();
}

}  // namespace fdk
