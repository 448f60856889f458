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

// FD-CNN column -> (symbol, user) of the chain's [S][K] order.  A shared network runs over
// every column c = t K + u; per-user parameters run one pass per user u over that user's
// own column block, FD-CNN column t being chain column t K + u.
struct ColMap {
    int K, u;   // u < 0: all columns of the chain
    FD_HD long chain(long c) const { return u < 0 ? c : c * K + u; }
    FD_HD long sym(long c) const { return u < 0 ? c / K : c; }
    FD_HD int user(long c) const { return u < 0 ? (int)(c % K) : u; }
};

// ---------------------------------------------------------------------------
// conv + ReLU forward and the conv parameter gradient.  The input grids sit in
// shared memory zero padded to Gp = (Go - 1) K_S + K_C per side (data at offset pad),
// so no tap needs a bounds test; KC > 0 fixes the kernel size at compile time.
// ---------------------------------------------------------------------------
FD_HD int padded_side(const Geo &g) { return (g.Go - 1) * g.K_S + g.K_C; }

FD_D void load_padded(const Geo &g, const c32 *s, long t, int u, float *Xp) {
    const int Gp = padded_side(g), GpGp = Gp * Gp;
    for (int idx = threadIdx.x; idx < g.Cin * GpGp; idx += blockDim.x) Xp[idx] = 0.f;
    __syncthreads();
    for (int l = 0; l < g.L_U; ++l) {
        const int v = (u + l) % g.K;
        const c32 *sv = s + (t * g.K + v) * g.N_d;
        for (int idx = threadIdx.x; idx < g.N_d; idx += blockDim.x) {
            const c32 val = sv[idx];
            const int r = idx / g.G + g.pad, q = idx % g.G + g.pad;
            Xp[(2 * l) * GpGp + r * Gp + q] = val.x;
            Xp[(2 * l + 1) * GpGp + r * Gp + q] = val.y;
        }
    }
}

template <int KC, typename TOut>
__global__ void __launch_bounds__(256) conv_fwd_kernel(Geo g, ColMap cm, int cols_per_cta, long cols,
                                                       const c32 *__restrict__ s, const float *__restrict__ theta,
                                                       TOut *__restrict__ act, long ld) {
    extern __shared__ float Xp[];
    const int kc = KC > 0 ? KC : g.K_C;
    const int Gp = padded_side(g), GpGp = Gp * Gp, GoGo = g.Go * g.Go;
    const long c0 = (long)blockIdx.x * cols_per_cta;
    for (long col = c0; col < min(cols, c0 + cols_per_cta); ++col) {
        __syncthreads();
        load_padded(g, s, cm.sym(col), cm.user(col), Xp);
        __syncthreads();
        for (int f = threadIdx.x; f < g.F; f += blockDim.x) {
            const int o = f / GoGo, rem = f % GoGo, i = rem / g.Go, j = rem % g.Go;
            float acc = theta[g.off_cb + o];
            const float *x0 = Xp + (i * g.K_S) * Gp + j * g.K_S;
            for (int c = 0; c < g.Cin; ++c) {
                const float *w = theta + ((o * g.Cin + c) * kc) * kc;
                const float *x = x0 + c * GpGp;
#pragma unroll
                for (int a = 0; a < (KC > 0 ? KC : 1); ++a)
#pragma unroll
                    for (int b = 0; b < (KC > 0 ? KC : 1); ++b) acc = fmaf(__ldg(w + a * kc + b), x[a * Gp + b], acc);
                if (KC == 0)
                    for (int a = 0; a < kc; ++a)
                        for (int b = 0; b < kc; ++b)
                            if (a | b) acc = fmaf(__ldg(w + a * kc + b), x[a * Gp + b], acc);
            }
            acc = fmaxf(acc, 0.0f);
            if constexpr (sizeof(TOut) == 4) act[col * ld + f] = acc;
            else act[col * ld + f] = __float2bfloat16_rn(acc);
        }
    }
}

// ---------------------------------------------------------------------------
// The benchmark's network (3 x 3 kernels, stride 1, 2 input channels -- the real and
// imaginary parts of one user's symbols -- and 2 output channels) without a staged grid:
// a thread owns output positions p = tid + 256 k for every column, whose 9-tap validity
// masks (inside the G x G grid and below N_d) and base offsets are computed once; a tap
// is one 8-byte complex load from the column's symbol row, which stays in L1, and the
// weights live in registers.
constexpr int CF_PPT = 5;   // positions per thread: G^2 <= 256 * 5

FD_HD bool conv_fast(const Geo &g) {
    return g.K_C == 3 && g.K_S == 1 && g.N_conv == 2 && g.Cin == 2 && g.pad == 1 && g.G * g.G <= 256 * CF_PPT;
}

// L1 warm-up of the next column's symbol row: one 128-byte line per thread
FD_D void prefetch_row_l1(const c32 *row, int n) {
    const int lines = (n * (int)sizeof(c32) + 127) / 128;
    if ((int)threadIdx.x < lines)
        asm volatile("prefetch.global.L1 [%0];" ::"l"(reinterpret_cast<const char *>(row) + 128 * threadIdx.x));
}

struct ConvPos {
    int base[CF_PPT];    // symbol index of tap (0, 0)
    int mask[CF_PPT];    // bit 3a + b: tap (a, b) inside the grid and the data
};
FD_D ConvPos conv_positions(const Geo &g) {
    ConvPos cp;
    const int G = g.G, GG = G * G;
#pragma unroll
    for (int k = 0; k < CF_PPT; ++k) {
        const int p = threadIdx.x + 256 * k;
        const int i = p / G, j = p % G;
        int m = 0;
        if (p < GG) {
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const int r = i + a - 1, q = j + b - 1;
                    if (r >= 0 && r < G && q >= 0 && q < G && r * G + q < g.N_d) m |= 1 << (3 * a + b);
                }
        }
        cp.base[k] = (i - 1) * G + (j - 1);
        cp.mask[k] = m;
    }
    return cp;
}

template <typename TOut, bool PU>   // PU: a per-user pass (column map t -> t K + u)
__global__ void __launch_bounds__(256) conv_fwd_fast_kernel(Geo g, ColMap cm, long cols, const c32 *__restrict__ s,
                                                            const float *__restrict__ theta, TOut *__restrict__ act,
                                                            long ld) {
    const int G = g.G, GG = G * G;
    float w[2][2][9], bias[2];
#pragma unroll
    for (int o = 0; o < 2; ++o) {
        bias[o] = theta[g.off_cb + o];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int k = 0; k < 9; ++k) w[o][c][k] = theta[(o * 2 + c) * 9 + k];   // conv_w at the start of theta
    }
    const ConvPos cp = conv_positions(g);
    for (long col = blockIdx.x; col < cols; col += gridDim.x) {
        const c32 *row = s + (PU ? cm.chain(col) : col) * g.N_d;   // L_U = 1: the column's own user
        TOut *out = act + col * ld;
        if (col + gridDim.x < cols) prefetch_row_l1(s + (PU ? cm.chain(col + gridDim.x) : col + gridDim.x) * g.N_d, g.N_d);
#pragma unroll
        for (int k = 0; k < CF_PPT; ++k) {
            const int p = threadIdx.x + 256 * k;
            if (p >= GG) break;
            float a0 = bias[0], a1 = bias[1];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const int tap = 3 * a + b;
                    if (cp.mask[k] >> tap & 1) {
                        const c32 v = __ldg(row + cp.base[k] + a * G + b);
                        a0 = fmaf(w[0][0][tap], v.x, fmaf(w[0][1][tap], v.y, a0));
                        a1 = fmaf(w[1][0][tap], v.x, fmaf(w[1][1][tap], v.y, a1));
                    }
                }
            a0 = fmaxf(a0, 0.f);
            a1 = fmaxf(a1, 0.f);
            if constexpr (sizeof(TOut) == 4) {
                out[p] = a0;
                out[GG + p] = a1;
            } else {
                out[p] = __float2bfloat16_rn(a0);
                out[GG + p] = __float2bfloat16_rn(a1);
            }
        }
    }
}

// parameter gradient: every thread accumulates the 36 weight and 2 bias partial sums of
// its positions over the CTA's columns; one block reduction per CTA
template <bool PU>
__global__ void __launch_bounds__(256) conv_bwd_fast_kernel(Geo g, ColMap cm, long cols, const c32 *__restrict__ s,
                                                            const float *__restrict__ gpre, long ldg,
                                                            float *__restrict__ partials) {
    constexpr int NW = 2 * 2 * 9 + 2;
    const int G = g.G, GG = G * G;
    float acc[2][2][9], accb[2] = {0.f, 0.f};
#pragma unroll
    for (int o = 0; o < 2; ++o)
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int k = 0; k < 9; ++k) acc[o][c][k] = 0.f;
    const ConvPos cp = conv_positions(g);
    // this thread's gradient values of the next column, loaded one column ahead
    float gn[2][CF_PPT];
    auto load_g = [&](long col) {
        const float *gp = gpre + col * ldg;
#pragma unroll
        for (int k = 0; k < CF_PPT; ++k) {
            const int p = threadIdx.x + 256 * k;
            const bool ok = col < cols && p < GG;
            gn[0][k] = ok ? gp[p] : 0.f;
            gn[1][k] = ok ? gp[GG + p] : 0.f;
        }
    };
    load_g(blockIdx.x);
    for (long col = blockIdx.x; col < cols; col += gridDim.x) {
        const c32 *row = s + (PU ? cm.chain(col) : col) * g.N_d;
        float gc[2][CF_PPT];
#pragma unroll
        for (int k = 0; k < CF_PPT; ++k) {
            gc[0][k] = gn[0][k];
            gc[1][k] = gn[1][k];
        }
        load_g(col + gridDim.x);
        if (col + gridDim.x < cols) prefetch_row_l1(s + (PU ? cm.chain(col + gridDim.x) : col + gridDim.x) * g.N_d, g.N_d);
#pragma unroll
        for (int k = 0; k < CF_PPT; ++k) {
            const int p = threadIdx.x + 256 * k;
            if (p >= GG) break;
            const float g0 = gc[0][k], g1 = gc[1][k];
            accb[0] += g0;
            accb[1] += g1;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const int tap = 3 * a + b;
                    if (cp.mask[k] >> tap & 1) {
                        const c32 v = __ldg(row + cp.base[k] + a * G + b);
                        acc[0][0][tap] = fmaf(g0, v.x, acc[0][0][tap]);
                        acc[0][1][tap] = fmaf(g0, v.y, acc[0][1][tap]);
                        acc[1][0][tap] = fmaf(g1, v.x, acc[1][0][tap]);
                        acc[1][1][tap] = fmaf(g1, v.y, acc[1][1][tap]);
                    }
                }
        }
    }
    __shared__ float red[8][NW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 0; o < 2; ++o)
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const float v = warp_sum(acc[o][c][k]);
                if (lane == 0) red[warp][(o * 2 + c) * 9 + k] = v;
            }
#pragma unroll
    for (int o = 0; o < 2; ++o) {
        const float v = warp_sum(accb[o]);
        if (lane == 0) red[warp][36 + o] = v;
    }
    __syncthreads();
    for (int wi = threadIdx.x; wi < NW; wi += blockDim.x) {
        float t = 0.f;
        for (int k = 0; k < 8; ++k) t += red[k][wi];
        partials[(long)blockIdx.x * NW + wi] = t;
    }
}

static long conv_fast_blocks(long cols) { return cols < 152L * 8 ? cols : 152L * 8; }

static int conv_cols_per_cta(long cols) { return cols >= 152 * 64 ? 8 : 1; }

template <typename TOut>
static cudaError_t conv_fwd_launch(const Geo &g, int S, const c32 *s, const float *theta, TOut *act, long ld,
                                   cudaStream_t st, int user) {
    const ColMap cm{g.K, user};
    const long cols = user < 0 ? (long)S * g.K : S;
    if (!cols) return cudaSuccess;
    const int Gp = padded_side(g);
    const size_t sm = sizeof(float) * (size_t)g.Cin * Gp * Gp;
    if (conv_fast(g) && g.L_U == 1) {
        if (user < 0)
            conv_fwd_fast_kernel<TOut, false><<<(unsigned)conv_fast_blocks(cols), 256, 0, st>>>(g, cm, cols, s, theta,
                                                                                                 act, ld);
        else
            conv_fwd_fast_kernel<TOut, true><<<(unsigned)conv_fast_blocks(cols), 256, 0, st>>>(g, cm, cols, s, theta,
                                                                                                act, ld);
        return cudaGetLastError();
    }
    const int cpc = conv_cols_per_cta(cols);
    const unsigned blocks = (unsigned)((cols + cpc - 1) / cpc);
    if (g.K_C == 3) conv_fwd_kernel<3, TOut><<<blocks, 256, sm, st>>>(g, cm, cpc, cols, s, theta, act, ld);
    else conv_fwd_kernel<0, TOut><<<blocks, 256, sm, st>>>(g, cm, cpc, cols, s, theta, act, ld);
    return cudaGetLastError();
}

cudaError_t conv_forward(const Geo &g, int S, const c32 *s, const float *theta, float *act, cudaStream_t st,
                         int user) {
    return conv_fwd_launch(g, S, s, theta, act, g.F, st, user);
}

cudaError_t conv_forward_bf16(const Geo &g, int S, const c32 *s, const float *theta, __nv_bfloat16 *act, long ld,
                              cudaStream_t st, int user) {
    return conv_fwd_launch(g, S, s, theta, act, ld, st, user);
}

// Parameter gradient: thread owns output positions (o-independent) and, for a batch of
// columns, accumulates every (o, c, a, b) product and the bias sums in registers; one
// block reduction per CTA writes the CTA's partial sums.
template <int KC, int NCONV, int CIN>
__global__ void __launch_bounds__(256) conv_bwd_kernel(Geo g, ColMap cm, int cols_per_cta, long cols,
                                                       const c32 *__restrict__ s, const float *__restrict__ gpre,
                                                       long ldg, float *__restrict__ partials) {
    extern __shared__ float smf[];
    constexpr int NW = NCONV * CIN * KC * KC + NCONV;
    const int Gp = padded_side(g), GpGp = Gp * Gp, GoGo = g.Go * g.Go;
    float *Xp = smf;
    float *gp = Xp + CIN * GpGp;
    float acc[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) acc[w] = 0.f;
    const long c0 = (long)blockIdx.x * cols_per_cta;
    for (long col = c0; col < min(cols, c0 + cols_per_cta); ++col) {
        __syncthreads();
        load_padded(g, s, cm.sym(col), cm.user(col), Xp);
        for (int f = threadIdx.x; f < g.F; f += blockDim.x) gp[f] = gpre[col * ldg + f];
        __syncthreads();
        for (int p = threadIdx.x; p < GoGo; p += blockDim.x) {
            const int i = p / g.Go, j = p % g.Go;
            const float *x0 = Xp + (i * g.K_S) * Gp + j * g.K_S;
            float gv[NCONV];
#pragma unroll
            for (int o = 0; o < NCONV; ++o) {
                gv[o] = gp[o * GoGo + p];
                acc[NCONV * CIN * KC * KC + o] += gv[o];
            }
#pragma unroll
            for (int c = 0; c < CIN; ++c)
#pragma unroll
                for (int a = 0; a < KC; ++a)
#pragma unroll
                    for (int b = 0; b < KC; ++b) {
                        const float x = x0[c * GpGp + a * Gp + b];
#pragma unroll
                        for (int o = 0; o < NCONV; ++o) acc[((o * CIN + c) * KC + a) * KC + b] = fmaf(gv[o], x, acc[((o * CIN + c) * KC + a) * KC + b]);
                    }
        }
    }
    __shared__ float red[8][NW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const float v = warp_sum(acc[w]);
        if (lane == 0) red[warp][w] = v;
    }
    __syncthreads();
    for (int w = threadIdx.x; w < NW; w += blockDim.x) {
        float t = 0.f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k][w];
        partials[(long)blockIdx.x * NW + w] = t;
    }
}

// generic fallback (any kernel size / channel count): one warp per parameter, lanes
// over positions, one column per CTA
__global__ void conv_bwd_generic_kernel(Geo g, ColMap cm, const c32 *__restrict__ s, const float *__restrict__ gpre,
                                        long ldg, float *__restrict__ partials) {
    extern __shared__ float smf[];
    const int Gp = padded_side(g), GpGp = Gp * Gp, GoGo = g.Go * g.Go, KC = g.K_C;
    float *Xp = smf;
    float *gp = Xp + g.Cin * GpGp;
    const long col = blockIdx.x;
    load_padded(g, s, cm.sym(col), cm.user(col), Xp);
    for (int f = threadIdx.x; f < g.F; f += blockDim.x) gp[f] = gpre[col * ldg + f];
    __syncthreads();
    const int nw = g.n_convw + g.N_conv;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int widx = warp; widx < nw; widx += nwarps) {
        float acc = 0.f;
        if (widx < g.n_convw) {
            const int b = widx % KC, a = (widx / KC) % KC, c = (widx / (KC * KC)) % g.Cin, o = widx / (KC * KC * g.Cin);
            for (int p = lane; p < GoGo; p += 32) {
                const int i = p / g.Go, j = p % g.Go;
                acc = fmaf(gp[o * GoGo + p], Xp[c * GpGp + (i * g.K_S + a) * Gp + j * g.K_S + b], acc);
            }
        } else {
            for (int p = lane; p < GoGo; p += 32) acc += gp[(widx - g.n_convw) * GoGo + p];
        }
        acc = warp_sum(acc);
        if (lane == 0) partials[col * nw + widx] = acc;
    }
}

static bool conv_bwd_fast(const Geo &g) { return g.K_C == 3 && g.N_conv == 2 && g.Cin == 2; }
static const int kConvColsPerCta = 16;
// rows of `partials` written by conv_backward for `cols` columns
static long conv_partial_rows(const Geo &g, long cols) {
    if (conv_fast(g) && g.L_U == 1) return conv_fast_blocks(cols);
    return conv_bwd_fast(g) ? (cols + kConvColsPerCta - 1) / kConvColsPerCta : cols;
}

cudaError_t conv_backward(const Geo &g, int S, const c32 *s, const float *gpre, long ldg, float *partials,
                          cudaStream_t st, int user) {
    const ColMap cm{g.K, user};
    const long cols = user < 0 ? (long)S * g.K : S;
    if (!cols) return cudaSuccess;
    const int Gp = padded_side(g);
    const size_t sm = sizeof(float) * ((size_t)g.Cin * Gp * Gp + g.F);
    cudaError_t e;
    if (conv_fast(g) && g.L_U == 1) {
        if (user < 0)
            conv_bwd_fast_kernel<false><<<(unsigned)conv_partial_rows(g, cols), 256, 0, st>>>(g, cm, cols, s, gpre, ldg,
                                                                                             partials);
        else
            conv_bwd_fast_kernel<true><<<(unsigned)conv_partial_rows(g, cols), 256, 0, st>>>(g, cm, cols, s, gpre, ldg,
                                                                                            partials);
        return cudaGetLastError();
    }
    if (conv_bwd_fast(g)) {
        const int cpc = kConvColsPerCta;
        const unsigned blocks = (unsigned)conv_partial_rows(g, cols);
        e = cudaFuncSetAttribute(conv_bwd_kernel<3, 2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        conv_bwd_kernel<3, 2, 2><<<blocks, 256, sm, st>>>(g, cm, cpc, cols, s, gpre, ldg, partials);
    } else {
        e = cudaFuncSetAttribute(conv_bwd_generic_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        conv_bwd_generic_kernel<<<(unsigned)cols, 256, sm, st>>>(g, cm, s, gpre, ldg, partials);
    }
    return cudaGetLastError();
}

__global__ void conv_reduce_kernel(int rows, int nw, const float *__restrict__ partials, float *__restrict__ out,
                                   int accumulate) {
    __shared__ double red[32];
    const int w = blockIdx.x;
    double acc = 0;
    for (int c = threadIdx.x; c < rows; c += blockDim.x) acc += partials[(long)c * nw + w];
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) out[w] = accumulate ? out[w] + (float)acc : (float)acc;
}

cudaError_t conv_reduce(const Geo &g, int cols, const float *partials, float *grad, bool accumulate, cudaStream_t st) {
    const int nw = g.n_convw + g.N_conv;
    conv_reduce_kernel<<<nw, 256, 0, st>>>((int)conv_partial_rows(g, cols), nw, partials, grad,
                                           accumulate ? 1 : 0);   // conv_w, conv_b
    return cudaGetLastError();
}

// fc_b gradient: column sums of gd [cols][2 N_d] (interleaved rows) -> grad[off_fb + pi(n')]
__global__ void colsum_fcb_kernel(Geo g, ColMap cm, int cols, int chunk, const float *__restrict__ gd,
                                  float *__restrict__ gfb) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int W2 = 2 * g.N_d;
    if (n >= W2) return;
    const long c0 = (long)blockIdx.y * chunk, c1 = min((long)cols, c0 + chunk);
    float acc = 0.f;
    for (long c = c0; c < c1; ++c) acc += gd[cm.chain(c) * W2 + n];
    const int row = (n & 1) * g.N_d + (n >> 1);
    atomicAdd(gfb + row, acc);
}

cudaError_t colsum_fcb(const Geo &g, int cols, const float *gd, float *grad, cudaStream_t st, int user) {
    const int W2 = 2 * g.N_d, chunk = 256;
    dim3 grid((W2 + 255) / 256, (cols + chunk - 1) / chunk);
    if (!cols) return cudaSuccess;
    colsum_fcb_kernel<<<grid, 256, 0, st>>>(g, ColMap{g.K, user}, cols, chunk, gd, grad + g.off_fb);
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
    ColMap cm;      // s and s_tilde in the chain's column order
    FD_D float a(long m, long k) const { return act[m * F + k]; }
    FD_D float b(long n, long k) const { return fw[(long)((n & 1) * Nd + (n >> 1)) * F + k]; }
    FD_D void store(long m, long n, float v) const {
        const long idx = cm.chain(m) * 2 * Nd + n;
        st[idx] = v + fb[(n & 1) * Nd + (n >> 1)] + (residual ? s[idx] : 0.f);
    }
};
struct FcBwdData {   // A = gd [cols][2N_d]; B(f, n') = fc_w[pi(n')][f]; C -> gpre (ReLU mask)
    const float *gd, *fw, *act;
    float *gpre;
    int F, Nd;
    ColMap cm;         // gd in the chain's column order
    FD_D float a(long m, long k) const { return gd[cm.chain(m) * 2 * Nd + k]; }
    FD_D float b(long n, long k) const { return fw[(long)((k & 1) * Nd + (k >> 1)) * F + n]; }
    FD_D void store(long m, long n, float v) const {
        const long idx = m * F + n;
        gpre[idx] = act[idx] > 0.f ? v : 0.f;
    }
};
struct FcBwdWeight {   // A(n', c) = gd[c][n']; B(f, c) = act[c][f]; C -> grad fc_w[pi(n')][f] (= or +=)
    const float *gd, *act;
    float *gfw;
    int F, Nd, accumulate;
    ColMap cm;           // gd in the chain's column order
    FD_D float a(long m, long k) const { return gd[cm.chain(k) * 2 * Nd + m]; }
    FD_D float b(long n, long k) const { return act[k * F + n]; }
    FD_D void store(long m, long n, float v) const {
        float *dst = gfw + (long)((m & 1) * Nd + (m >> 1)) * F + n;
        *dst = accumulate ? *dst + v : v;
    }
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
                           cudaStream_t stm, int user) {
    FcFwd op{act, theta + g.off_fw, theta + g.off_fb, reinterpret_cast<const float *>(s),
             reinterpret_cast<float *>(st), g.F, g.N_d, g.residual, ColMap{g.K, user}};
    return run_sgemm<FcFwd, true, true>(op, cols, 2L * g.N_d, g.F, stm);
}

cudaError_t fc_backward_data_f32(const Geo &g, int cols, const float *gd, const float *theta, const float *act,
                                 float *gpre, cudaStream_t stm, int user) {
    FcBwdData op{gd, theta + g.off_fw, act, gpre, g.F, g.N_d, ColMap{g.K, user}};
    return run_sgemm<FcBwdData, true, false>(op, cols, g.F, 2L * g.N_d, stm);
}

cudaError_t fc_backward_weight_f32(const Geo &g, int cols, const float *gd, const float *act, float *grad,
                                   bool accumulate, cudaStream_t stm, int user) {
    FcBwdWeight op{gd, act, grad + g.off_fw, g.F, g.N_d, accumulate ? 1 : 0, ColMap{g.K, user}};
    return run_sgemm<FcBwdWeight, false, false>(op, 2L * g.N_d, g.F, cols, stm);
}

}  // namespace fdk
