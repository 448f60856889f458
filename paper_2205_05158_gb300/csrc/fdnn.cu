// The FD-NN comparison DPD of Sec. III-C (the frequency-domain NN of the paper's
// complexity comparison), FP32:
//   t_u = IDFT_N(s_u)                        one unitary transform per (symbol, user) row,
//                                            the guard bins zero
//   o_u[n] = [t_u[n]] + NN(t_0[n..n-L_4], ..., t_{U-1}[n..n-L_4])     at every sample n
//   s_dpd_u = DFT_N(o_u)                     every bin: the guard bins are no longer empty,
//                                            so the precoder covers all N of them
// NN: fully connected, 2U(L_4+1) real inputs (the real parts of s_u[n-l], u major, l
// minor, then the imaginary parts), K^NN hidden layers of D ReLU neurons, 2U outputs (the
// real parts of the U predistorted samples, then the imaginary parts); taps circular in n
// (a cyclic prefix of at least L_4 samples).  The transforms are the radix-16 row
// transforms of the PA row kernels; the network runs one thread per (symbol, sample) with
// its parameters in shared memory and the first layer accumulated while the tap inputs
// stream in (coalesced across the samples of a warp).
#include "fftpa.cuh"

namespace fdk {

long fdnn_theta_len(const Geo &g, const FdnnDesc &nn) {
    const long U = g.K, L1 = nn.L4 + 1, D = nn.D;
    return D * 2 * U * L1 + D + (nn.layers - 1) * (D * D + D) + 2 * U * D + 2 * U;
}

template <int LOG2N, bool INV>
static cudaError_t user_rows_t(const Geo &g, long rows, const c32 *in, c32 *out, const c32 *tw, cudaStream_t st) {
    using F = Fft<LOG2N>;
    const size_t sm = sizeof(c32) * ((size_t)F::N + 2 * (size_t)rows_per_cta_t<LOG2N>() * F::PADN);
    long blocks = 0;
    cudaError_t e = persistent_blocks(user_rows_kernel<LOG2N, INV>, F::N, rows, 256, sm, blocks);
    if (e != cudaSuccess) return e;
    user_rows_kernel<LOG2N, INV><<<(unsigned)blocks, 256, sm, st>>>(g, rows, in, out, tw);
    return cudaGetLastError();
}

template <bool INV>
static cudaError_t user_rows_n(const Geo &g, long rows, const c32 *in, c32 *out, const c32 *tw, cudaStream_t st) {
    switch (g.log2N) {
        case 6: return user_rows_t<6, INV>(g, rows, in, out, tw, st);
        case 7: return user_rows_t<7, INV>(g, rows, in, out, tw, st);
        case 8: return user_rows_t<8, INV>(g, rows, in, out, tw, st);
        case 9: return user_rows_t<9, INV>(g, rows, in, out, tw, st);
        case 10: return user_rows_t<10, INV>(g, rows, in, out, tw, st);
        case 11: return user_rows_t<11, INV>(g, rows, in, out, tw, st);
        case 12: return user_rows_t<12, INV>(g, rows, in, out, tw, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t fdnn_user_rows(const Geo &g, long rows, bool inverse, const c32 *in, c32 *out, const c32 *tw,
                           cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    return inverse ? user_rows_n<true>(g, rows, in, out, tw, st) : user_rows_n<false>(g, rows, in, out, tw, st);
}

constexpr int NN_DMAX = 32;       // neurons per hidden layer (the paper's network has 15)
constexpr int NN_SMEM_FLOATS = 12288;

__global__ void __launch_bounds__(256) fdnn_mlp_kernel(Geo g, FdnnDesc nn, int S, const float *__restrict__ theta,
                                                       long n_theta, const c32 *__restrict__ t,
                                                       c32 *__restrict__ o) {
    extern __shared__ float sth[];
    for (long i = threadIdx.x; i < n_theta; i += blockDim.x) sth[i] = theta[i];
    __syncthreads();
    const int U = g.K, N = g.N, L1 = nn.L4 + 1, D = nn.D, nin = 2 * U * L1;
    const float *W0 = sth, *b0 = W0 + (long)D * nin, *hid = b0 + D;
    const float *Wo = hid + (long)(nn.layers - 1) * (D * D + D), *bo = Wo + 2 * U * D;
    const long total = (long)S * N;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const long s = idx / N;
        const int n = (int)(idx - s * N);
        const c32 *ts = t + s * U * N;
        float h[NN_DMAX];
#pragma unroll
        for (int a = 0; a < NN_DMAX; ++a) h[a] = a < D ? b0[a] : 0.f;
        for (int u = 0; u < U; ++u)
            for (int l = 0; l < L1; ++l) {
                const c32 v = ts[(long)u * N + ((n - l) & (N - 1))];
                const int jr = u * L1 + l, ji = U * L1 + jr;
#pragma unroll
                for (int a = 0; a < NN_DMAX; ++a)
                    if (a < D) h[a] = fmaf(W0[a * nin + jr], v.x, fmaf(W0[a * nin + ji], v.y, h[a]));
            }
#pragma unroll
        for (int a = 0; a < NN_DMAX; ++a) h[a] = fmaxf(h[a], 0.f);
        for (int k = 1; k < nn.layers; ++k) {
            const float *Wk = hid + (long)(k - 1) * (D * D + D), *bk = Wk + D * D;
            float h2[NN_DMAX];
#pragma unroll
            for (int a = 0; a < NN_DMAX; ++a) {
                float acc = a < D ? bk[a] : 0.f;
                if (a < D)
                    for (int j = 0; j < D; ++j) acc = fmaf(Wk[a * D + j], h[j], acc);
                h2[a] = fmaxf(acc, 0.f);
            }
#pragma unroll
            for (int a = 0; a < NN_DMAX; ++a) h[a] = h2[a];
        }
        c32 *os = o + s * U * N + n;
        for (int u = 0; u < U; ++u) {
            float re = bo[u], im = bo[U + u];
#pragma unroll
            for (int a = 0; a < NN_DMAX; ++a)
                if (a < D) {
                    re = fmaf(Wo[u * D + a], h[a], re);
                    im = fmaf(Wo[(U + u) * D + a], h[a], im);
                }
            if (nn.residual) {
                const c32 v = ts[(long)u * N + n];
                re += v.x;
                im += v.y;
            }
            os[(long)u * N] = make_float2(re, im);
        }
    }
}

cudaError_t fdnn_mlp(const Geo &g, const FdnnDesc &nn, int S, const float *theta, const c32 *t, c32 *o,
                     cudaStream_t st) {
    const long n_theta = fdnn_theta_len(g, nn);
    if (nn.D < 1 || nn.D > NN_DMAX || n_theta > NN_SMEM_FLOATS) return cudaErrorInvalidValue;
    if (S <= 0) return cudaSuccess;
    const size_t sm = sizeof(float) * (size_t)n_theta;
    cudaError_t e = cudaFuncSetAttribute(fdnn_mlp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long need = ((long)S * g.N + 255) / 256;
    long blocks = (long)resident_ctas(fdnn_mlp_kernel, 256, sm) * (sms > 0 ? sms : 1);
    if (blocks > need) blocks = need;
    fdnn_mlp_kernel<<<(unsigned)blocks, 256, sm, st>>>(g, nn, S, theta, n_theta, t, o);
    return cudaGetLastError();
}

__global__ void fdnn_alpha_kernel(Geo g, long n, const float *__restrict__ alpha_all, float *__restrict__ alpha) {
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        const long r = j / g.N_d;
        const int i = (int)(j - r * g.N_d);
        alpha[j] = alpha_all[r * g.N + (g.first_bin + i) % g.N];
    }
}

cudaError_t fdnn_alpha_data(const Geo &g, int R, const float *alpha_all, float *alpha, cudaStream_t st) {
    const long n = (long)R * g.N_d;
    if (n <= 0) return cudaSuccess;
    const long b = (n + 255) / 256;
    fdnn_alpha_kernel<<<(unsigned)(b < 4096 ? b : 4096), 256, 0, st>>>(g, n, alpha_all, alpha);
    return cudaGetLastError();
}

}  // namespace fdk
