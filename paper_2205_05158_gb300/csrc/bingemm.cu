// Per-subcarrier complex contractions of the downlink, FP32 operands on CUDA cores.
//
//   expand (users -> antennas), out[t][m][i] = scale_i sum_u A_i[m][u] B[t][u][i]
//     PRECODE     : A = W_i,           scale = alpha_i     (Eq. 1, x_hat = alpha W s_tilde)
//     ADJ_COMBINE : A = H_i^H,         scale = 1 / alpha_i (adjoint of y = H X / alpha)
//   reduce (antennas -> users), out[t][u][i] = scale_i sum_m A_i[u][m] B[t][m][i]
//     COMBINE     : A = H_i,           scale = 1 / alpha_i (Eq. 5 then equalisation), with
//                   the loss terms |y - s|^2, |s|^2 and the loss gradient 2 (y - s) / count
//     ADJ_PRECODE : A = W_i^H,         scale = alpha_i     (adjoint of the precoder)
// i runs over data subcarriers, t over the symbols of realisation r = t / S_per_real.
// A CTA owns 32 consecutive subcarriers (one per lane, so every global access along
// i is coalesced) of one realisation, and stages the B operand of a symbol chunk in
// shared memory.
#include "common.cuh"
#include "kernels.h"

namespace fdk {

static constexpr int EXP_SC = 16;   // symbols per chunk (expand)
static constexpr int RED_SC = 8;    // symbols per chunk (reduce)
static constexpr int RED_MC = 16;   // antennas per chunk (reduce)

template <int KM>
__global__ void __launch_bounds__(256) expand_kernel(Geo g, int mode, int S, const c32 *__restrict__ A,
                                                     const float *__restrict__ alpha, const c32 *__restrict__ B,
                                                     c32 *__restrict__ out) {
    extern __shared__ __align__(16) c32 sB[];   // [EXP_SC][K][32]
    const int K = g.K, M = g.M, Nd = g.N_d;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int r = blockIdx.y, i = blockIdx.x * 32 + lane;
    const bool valid = i < Nd;
    const long t0 = (long)r * g.S_per_real;
    const int nsym = (int)min((long)g.S_per_real, (long)S - t0);
    const long bin = (long)r * Nd + (valid ? i : 0);
    const float al = alpha[bin];
    const float scale = valid ? (mode == PRECODE ? al : 1.0f / al) : 0.f;
    const int mper = (M + nwarps - 1) / nwarps, mlo = warp * mper, mhi = min(M, mlo + mper);

    for (int s0 = 0; s0 < nsym; s0 += EXP_SC) {
        const int ns = min(EXP_SC, nsym - s0);
        __syncthreads();
        for (int e = warp; e < ns * K; e += nwarps) {
            const int s = e / K, u = e % K;
            sB[(s * K + u) * 32 + lane] = valid ? B[((t0 + s0 + s) * K + u) * Nd + i] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int m = mlo; m < mhi; ++m) {
            c32 a[KM];
#pragma unroll
            for (int u = 0; u < KM; ++u) {
                if (u < K && valid) {
                    if (mode == PRECODE) a[u] = A[(bin * M + m) * K + u];
                    else a[u] = cconj(A[(bin * K + u) * M + m]);
                } else {
                    a[u] = make_float2(0.f, 0.f);
                }
            }
            for (int s = 0; s < ns; ++s) {
                c32 acc = make_float2(0.f, 0.f);
                const c32 *bs = sB + s * K * 32 + lane;
#pragma unroll
                for (int u = 0; u < KM; ++u)
                    if (u < K) acc = cfma(a[u], bs[u * 32], acc);
                if (valid) out[((t0 + s0 + s) * M + m) * Nd + i] = cscale(acc, scale);
            }
        }
    }
}

template <int UPW>
__global__ void __launch_bounds__(256) reduce_kernel(Geo g, int mode, int S, const c32 *__restrict__ A,
                                                     const float *__restrict__ alpha, const c32 *__restrict__ B,
                                                     c32 *__restrict__ out, const c32 *__restrict__ s_ref,
                                                     c32 *__restrict__ gy, double *metrics, double inv_count) {
    __shared__ __align__(16) c32 sB[RED_SC * RED_MC * 32];
    __shared__ double red[32];
    const int K = g.K, M = g.M, Nd = g.N_d;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int r = blockIdx.y, i = blockIdx.x * 32 + lane;
    const bool valid = i < Nd;
    const long t0 = (long)r * g.S_per_real;
    const int nsym = (int)min((long)g.S_per_real, (long)S - t0);
    const long bin = (long)r * Nd + (valid ? i : 0);
    const float al = alpha[bin];
    const float scale = valid ? (mode == COMBINE ? 1.0f / al : al) : 0.f;
    double err = 0, sig = 0;

    for (int s0 = 0; s0 < nsym; s0 += RED_SC) {
        const int ns = min(RED_SC, nsym - s0);
        c32 acc[UPW][RED_SC];
#pragma unroll
        for (int uu = 0; uu < UPW; ++uu)
#pragma unroll
            for (int s = 0; s < RED_SC; ++s) acc[uu][s] = make_float2(0.f, 0.f);
        for (int m0 = 0; m0 < M; m0 += RED_MC) {
            const int nm = min(RED_MC, M - m0);
            __syncthreads();
            for (int e = warp; e < RED_SC * RED_MC; e += nwarps) {
                const int s = e / RED_MC, mm = e % RED_MC;
                sB[e * 32 + lane] = (valid && s < ns && mm < nm) ? B[((t0 + s0 + s) * M + m0 + mm) * Nd + i]
                                                                  : make_float2(0.f, 0.f);
            }
            __syncthreads();
            for (int mm = 0; mm < nm; ++mm) {
                const int m = m0 + mm;
#pragma unroll
                for (int uu = 0; uu < UPW; ++uu) {
                    const int u = warp + uu * nwarps;
                    c32 a = make_float2(0.f, 0.f);
                    if (u < K && valid) a = (mode == COMBINE) ? A[(bin * K + u) * M + m] : cconj(A[(bin * M + m) * K + u]);
#pragma unroll
                    for (int s = 0; s < RED_SC; ++s) acc[uu][s] = cfma(a, sB[(s * RED_MC + mm) * 32 + lane], acc[uu][s]);
                }
            }
        }
#pragma unroll
        for (int uu = 0; uu < UPW; ++uu) {
            const int u = warp + uu * nwarps;
            if (u >= K || !valid) continue;
#pragma unroll
            for (int s = 0; s < RED_SC; ++s) {
                if (s >= ns) continue;
                const long idx = ((t0 + s0 + s) * K + u) * Nd + i;
                const c32 v = cscale(acc[uu][s], scale);
                if (mode == COMBINE) {
                    const c32 sr = s_ref[idx];
                    const c32 e = csub(v, sr);
                    err += cabs2(e);
                    sig += cabs2(sr);
                    if (out) out[idx] = v;
                    if (gy) gy[idx] = cscale(e, (float)(2.0 * inv_count));
                } else {
                    out[idx] = v;
                }
            }
        }
    }
    if (mode == COMBINE && metrics) {
        const double es = block_sum(err, red);
        const double ss = block_sum(sig, red);
        if (threadIdx.x == 0) {
            atomicAdd(metrics + 1, es);
            atomicAdd(metrics + 2, ss);
        }
    }
}

cudaError_t bin_expand(const Geo &g, int mode, int S, const c32 *A, const float *alpha, const c32 *B, c32 *out,
                       cudaStream_t st) {
    const int R = (S + g.S_per_real - 1) / g.S_per_real;
    if (R == 0) return cudaSuccess;
    dim3 grid((g.N_d + 31) / 32, R);
    const size_t sm = sizeof(c32) * EXP_SC * g.K * 32;
    cudaError_t e;
#define FD_EXPAND(KM)                                                                                       \
    e = cudaFuncSetAttribute(expand_kernel<KM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);       \
    if (e != cudaSuccess) return e;                                                                         \
    expand_kernel<KM><<<grid, 256, sm, st>>>(g, mode, S, A, alpha, B, out);
    if (g.K <= 4) { FD_EXPAND(4) }
    else if (g.K <= 8) { FD_EXPAND(8) }
    else if (g.K <= 16) { FD_EXPAND(16) }
    else { FD_EXPAND(32) }
#undef FD_EXPAND
    return cudaGetLastError();
}

cudaError_t bin_reduce(const Geo &g, int mode, int S, const c32 *A, const float *alpha, const c32 *B, c32 *out,
                       const c32 *s_ref, c32 *gy, double *metrics, double inv_count, cudaStream_t st) {
    const int R = (S + g.S_per_real - 1) / g.S_per_real;
    if (R == 0) return cudaSuccess;
    dim3 grid((g.N_d + 31) / 32, R);
    const int nwarps = g.K < 8 ? g.K : 8;
    const int upw = (g.K + nwarps - 1) / nwarps;
    const int threads = 32 * nwarps;
    if (upw <= 1) reduce_kernel<1><<<grid, threads, 0, st>>>(g, mode, S, A, alpha, B, out, s_ref, gy, metrics, inv_count);
    else if (upw <= 2) reduce_kernel<2><<<grid, threads, 0, st>>>(g, mode, S, A, alpha, B, out, s_ref, gy, metrics, inv_count);
    else reduce_kernel<4><<<grid, threads, 0, st>>>(g, mode, S, A, alpha, B, out, s_ref, gy, metrics, inv_count);
    return cudaGetLastError();
}

}  // namespace fdk
