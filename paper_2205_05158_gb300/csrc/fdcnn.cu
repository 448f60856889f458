// FD-CNN of Sec. IV-A and its adjoint.
//
// Input (Eq. 13): for user u the N_d data symbols of users u, u+1, ..., u+L_U-1 (mod K)
// fill G x G grids row by row in increasing frequency, zero padded; their real and
// imaginary parts are 2 L_U channels.  N_conv kernels of size K_C, stride K_S, zero
// "same" padding (pad = K_C / 2), bias, ReLU; flatten (kernel-major) to F values; a
// dense layer to 2 N_d outputs, rows 0..N_d-1 real and N_d..2N_d-1 imaginary parts.
// The predistorted symbols are s_tilde = s + out (residual) or out.
//
// The dense layer is a GEMM over all (symbol, user) columns.  Internally its output
// rows are taken in interleaved order n' = 2 i + c (c = 0 real, 1 imaginary), i.e.
// row pi(n') = c N_d + i of fc_w, so that the GEMM output of one column is directly
// the complex vector s_tilde and its adjoint input is the complex gradient vector.
#include "common.cuh"
#include "kernels.h"

namespace fdk {

// ---------------------------------------------------------------------------
// conv + ReLU forward: one CTA per (symbol, user) column
// ---------------------------------------------------------------------------
FD_D void load_grid(const Geo &g, const c32 *s, long t, int u, float *X) {
    const int GG = g.G * g.G;
    for (int l = 0; l < g.L_U; ++l) {
        const int v = (u + l) % g.K;
        const c32 *sv = s + (t * g.K + v) * g.N_d;
        for (int idx = threadIdx.x; idx < GG; idx += blockDim.x) {
            const c32 val = idx < g.N_d ? sv[idx] : make_float2(0.f, 0.f);
            X[(2 * l) * GG + idx] = val.x;
            X[(2 * l + 1) * GG + idx] = val.y;
        }
    }
}

__global__ void conv_fwd_kernel(Geo g, const c32 *__restrict__ s, const float *__restrict__ theta,
                                float *__restrict__ act) {
    extern __shared__ float smf[];
    float *X = smf;                                  // Cin * G * G
    float *w = X + g.Cin * g.G * g.G;                // n_convw + N_conv
    const long col = blockIdx.x;
    const long t = col / g.K;
    const int u = (int)(col % g.K);
    for (int i = threadIdx.x; i < g.n_convw + g.N_conv; i += blockDim.x) w[i] = theta[i];
    load_grid(g, s, t, u, X);
    __syncthreads();
    const int GoGo = g.Go * g.Go, KC = g.K_C;
    const float *bias = w + g.n_convw;
    for (int f = threadIdx.x; f < g.F; f += blockDim.x) {
        const int o = f / GoGo, rem = f % GoGo, i = rem / g.Go, j = rem % g.Go;
        float acc = bias[o];
        for (int c = 0; c < g.Cin; ++c) {
            const float *Xc = X + c * g.G * g.G;
            const float *wc = w + (o * g.Cin + c) * KC * KC;
            for (int a = 0; a < KC; ++a) {
                const int r = i * g.K_S + a - g.pad;
                if (r < 0 || r >= g.G) continue;
                for (int b = 0; b < KC; ++b) {
                    const int q = j * g.K_S + b - g.pad;
                    if (q < 0 || q >= g.G) continue;
                    acc = fmaf(wc[a * KC + b], Xc[r * g.G + q], acc);
                }
            }
        }
        act[col * g.F + f] = fmaxf(acc, 0.0f);
    }
}

cudaError_t conv_forward(const Geo &g, int S, const c32 *s, const float *theta, float *act, cudaStream_t st) {
    const long cols = (long)S * g.K;
    if (!cols) return cudaSuccess;
    const size_t sm = sizeof(float) * ((size_t)g.Cin * g.G * g.G + g.n_convw + g.N_conv);
    conv_fwd_kernel<<<(unsigned)cols, 256, sm, st>>>(g, s, theta, act);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// conv backward: per-column partial gradients of conv_w and conv_b from the
// masked activation gradient gpre, then a column reduction.
// ---------------------------------------------------------------------------
__global__ void conv_bwd_kernel(Geo g, const c32 *__restrict__ s, const float *__restrict__ gpre,
                                float *__restrict__ partials) {
    extern __shared__ float smf[];
    float *X = smf;
    float *gp = X + g.Cin * g.G * g.G;
    const long col = blockIdx.x;
    const long t = col / g.K;
    const int u = (int)(col % g.K);
    load_grid(g, s, t, u, X);
    for (int f = threadIdx.x; f < g.F; f += blockDim.x) gp[f] = gpre[col * g.F + f];
    __syncthreads();
    const int GoGo = g.Go * g.Go, KC = g.K_C, nw = g.n_convw + g.N_conv;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int widx = warp; widx < nw; widx += nwarps) {
        float acc = 0.f;
        if (widx < g.n_convw) {
            const int b = widx % KC, a = (widx / KC) % KC, c = (widx / (KC * KC)) % g.Cin, o = widx / (KC * KC * g.Cin);
            const float *Xc = X + c * g.G * g.G;
            const float *go = gp + o * GoGo;
            for (int p = lane; p < GoGo; p += 32) {
                const int i = p / g.Go, j = p % g.Go;
                const int r = i * g.K_S + a - g.pad, q = j * g.K_S + b - g.pad;
                if (r >= 0 && r < g.G && q >= 0 && q < g.G) acc = fmaf(go[p], Xc[r * g.G + q], acc);
            }
        } else {
            const float *go = gp + (widx - g.n_convw) * GoGo;
            for (int p = lane; p < GoGo; p += 32) acc += go[p];
        }
        acc = warp_sum(acc);
        if (lane == 0) partials[col * nw + widx] = acc;
    }
}

cudaError_t conv_backward(const Geo &g, int S, const c32 *s, const float *gpre, const float * /*act*/,
                          float *partials, cudaStream_t st) {
    const long cols = (long)S * g.K;
    if (!cols) return cudaSuccess;
    const size_t sm = sizeof(float) * ((size_t)g.Cin * g.G * g.G + g.F);
    cudaError_t e = cudaFuncSetAttribute(conv_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    conv_bwd_kernel<<<(unsigned)cols, 256, sm, st>>>(g, s, gpre, partials);
    return cudaGetLastError();
}

__global__ void conv_reduce_kernel(int cols, int nw, const float *__restrict__ partials, float *__restrict__ out) {
    __shared__ double red[32];
    const int w = blockIdx.x;
    double acc = 0;
    for (int c = threadIdx.x; c < cols; c += blockDim.x) acc += partials[(long)c * nw + w];
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) out[w] = (float)acc;
}

cudaError_t conv_reduce(const Geo &g, int cols, const float *partials, float *grad, cudaStream_t st) {
    const int nw = g.n_convw + g.N_conv;
    conv_reduce_kernel<<<nw, 256, 0, st>>>(cols, nw, partials, grad);   // conv_w then conv_b: contiguous in theta
    return cudaGetLastError();
}

// fc_b gradient: column sums of gd [cols][2 N_d] (interleaved rows) -> grad[off_fb + pi(n')]
__global__ void colsum_fcb_kernel(Geo g, int cols, int chunk, const float *__restrict__ gd, float *__restrict__ gfb) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int W2 = 2 * g.N_d;
    if (n >= W2) return;
    const long c0 = (long)blockIdx.y * chunk, c1 = min((long)cols, c0 + chunk);
    float acc = 0.f;
    for (long c = c0; c < c1; ++c) acc += gd[c * W2 + n];
    const int row = (n & 1) * g.N_d + (n >> 1);
    atomicAdd(gfb + row, acc);
}

cudaError_t colsum_fcb(const Geo &g, int cols, const float *gd, float *grad, cudaStream_t st) {
    const int W2 = 2 * g.N_d, chunk = 256;
    dim3 grid((W2 + 255) / 256, (cols + chunk - 1) / chunk);
    if (!cols) return cudaSuccess;
    colsum_fcb_kernel<<<grid, 256, 0, st>>>(g, cols, chunk, gd, grad + g.off_fb);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP32 GEMM  C[m][n] = sum_k A(m, k) B(n, k), 64 x 64 tiles, 4 x 4 per thread.
// A_K / B_K: the operand is contiguous along k (else along m / n).
// ---------------------------------------------------------------------------
struct FcFwd {   // A = act [cols][F]; B(n', f) = fc_w[pi(n')][f]; C -> s_tilde (interleaved floats)
    const float *act, *fw, *fb;
    const float *s;
    float *st;
    int F, Nd, residual;
    FD_D float a(long m, long k) const { return act[m * F + k]; }
    FD_D float b(long n, long k) const { return fw[(long)((n & 1) * Nd + (n >> 1)) * F + k]; }
    FD_D void store(long m, long n, float v) const {
        const long idx = m * 2 * Nd + n;
        st[idx] = v + fb[(n & 1) * Nd + (n >> 1)] + (residual ? s[idx] : 0.f);
    }
};
struct FcBwdData {   // A = gd [cols][2N_d]; B(f, n') = fc_w[pi(n')][f]; C -> gpre (ReLU mask)
    const float *gd, *fw, *act;
    float *gpre;
    int F, Nd;
    FD_D float a(long m, long k) const { return gd[m * 2 * Nd + k]; }
    FD_D float b(long n, long k) const { return fw[(long)((k & 1) * Nd + (k >> 1)) * F + n]; }
    FD_D void store(long m, long n, float v) const {
        const long idx = m * F + n;
        gpre[idx] = act[idx] > 0.f ? v : 0.f;
    }
};
struct FcBwdWeight {   // A(n', c) = gd[c][n']; B(f, c) = act[c][f]; C -> grad fc_w[pi(n')][f]
    const float *gd, *act;
    float *gfw;
    int F, Nd;
    FD_D float a(long m, long k) const { return gd[k * 2 * Nd + m]; }
    FD_D float b(long n, long k) const { return act[k * F + n]; }
    FD_D void store(long m, long n, float v) const { gfw[(long)((m & 1) * Nd + (m >> 1)) * F + n] = v; }
};

template <class Op, bool A_K, bool B_K>
__global__ void __launch_bounds__(256) sgemm_kernel(Op op, long Mdim, long Ndim, long Kdim) {
    __shared__ float As[16][68];
    __shared__ float Bs[16][68];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const long m0 = (long)blockIdx.y * 64, n0 = (long)blockIdx.x * 64;
    float acc[4][4] = {};
    for (long k0 = 0; k0 < Kdim; k0 += 16) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q;
            int r, k;
            if (A_K) { r = e >> 4; k = e & 15; } else { r = e & 63; k = e >> 6; }
            const long gm = m0 + r, gk = k0 + k;
            As[k][r] = (gm < Mdim && gk < Kdim) ? op.a(gm, gk) : 0.f;
            if (B_K) { r = e >> 4; k = e & 15; } else { r = e & 63; k = e >> 6; }
            const long gn = n0 + r, gk2 = k0 + k;
            Bs[k][r] = (gn < Ndim && gk2 < Kdim) ? op.b(gn, gk2) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float4 av = *reinterpret_cast<const float4 *>(&As[k][ty * 4]);
            const float4 bv = *reinterpret_cast<const float4 *>(&Bs[k][tx * 4]);
            const float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(ar[i], br[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
            if (gm < Mdim && gn < Ndim) op.store(gm, gn, acc[i][j]);
        }
}

template <class Op, bool A_K, bool B_K>
static cudaError_t run_sgemm(const Op &op, long Mdim, long Ndim, long Kdim, cudaStream_t st) {
    if (Mdim <= 0 || Ndim <= 0) return cudaSuccess;
    dim3 grid((unsigned)((Ndim + 63) / 64), (unsigned)((Mdim + 63) / 64));
    sgemm_kernel<Op, A_K, B_K><<<grid, 256, 0, st>>>(op, Mdim, Ndim, Kdim);
    return cudaGetLastError();
}

cudaError_t fc_forward_f32(const Geo &g, int cols, const float *act, const float *theta, const c32 *s, c32 *st,
                           cudaStream_t stm) {
    FcFwd op{act, theta + g.off_fw, theta + g.off_fb, reinterpret_cast<const float *>(s),
             reinterpret_cast<float *>(st), g.F, g.N_d, g.residual};
    return run_sgemm<FcFwd, true, true>(op, cols, 2L * g.N_d, g.F, stm);
}

cudaError_t fc_backward_data_f32(const Geo &g, int cols, const float *gd, const float *theta, const float *act,
                                 float *gpre, cudaStream_t stm) {
    FcBwdData op{gd, theta + g.off_fw, act, gpre, g.F, g.N_d};
    return run_sgemm<FcBwdData, true, false>(op, cols, g.F, 2L * g.N_d, stm);
}

cudaError_t fc_backward_weight_f32(const Geo &g, int cols, const float *gd, const float *act, float *grad,
                                   cudaStream_t stm) {
    FcBwdWeight op{gd, act, grad + g.off_fw, g.F, g.N_d};
    return run_sgemm<FcBwdWeight, false, false>(op, 2L * g.N_d, g.F, cols, stm);
}

}  // namespace fdk
