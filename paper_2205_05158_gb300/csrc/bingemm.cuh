// Per-subcarrier complex contractions of the downlink on CUDA cores (FP32 accumulate).
//
//   expand (users -> antennas), out[t][m][i] = scale_i sum_u A_i[m][u] B[t][u][i]
//     PRECODE     : A = W_i,           scale = alpha_i     (Eq. 1, x_hat = alpha W s_tilde)
//     ADJ_COMBINE : A = H_i^H,         scale = 1 / alpha_i (adjoint of y = H X / alpha)
//   reduce (antennas -> users), out[t][u][i] = scale_i sum_m A_i[u][m] B[t][m][i]
//     COMBINE     : A = H_i,           scale = 1 / alpha_i (Eq. 5 then equalisation), with
//                   the loss terms |y - s|^2, |s|^2 and the loss gradient 2 (y - s) / count
//     ADJ_PRECODE : A = W_i^H,         scale = alpha_i     (adjoint of the precoder)
// i runs over data subcarriers, t over the symbols of realisation r = t / S_per_real.
//
// A CTA owns 32 consecutive subcarriers of one realisation: lane = subcarrier, so every
// access to the [t][.][i] planes is coalesced.  The B operand of a symbol chunk is staged
// in shared memory; each thread accumulates TWO rows (antennas m, m+1 for expand, users
// u, u+1 for reduce) for every symbol of the chunk, so one shared load feeds two complex
// multiply-adds.  A (W or H) is read straight from global memory, as FP32 or as the
// 16-bit copy a 16-bit plan keeps (TA = cbf16 / cf16).
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace fdk {

constexpr int RMC = 16;   // antennas per shared chunk (reduce)

template <typename TA> FD_D c32 ld(const TA *p) { return Operand<TA>::load(p); }

// ---------------------------------------------------------------------------
template <typename TA, int SC>
__global__ void __launch_bounds__(256, 2) expand2_kernel(Geo g, int mode, int S, const TA *__restrict__ A,
                                                      const float *__restrict__ alpha, const c32 *__restrict__ B,
                                                      c32 *__restrict__ out) {
    extern __shared__ __align__(16) c32 sB[];   // [SC][K][32]
    const int K = g.K, M = g.M, Nd = g.N_d;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int r = blockIdx.y, i = blockIdx.x * 32 + lane;
    const bool valid = i < Nd;
    const long t0 = (long)r * g.S_per_real;
    const int nsym = (int)min((long)g.S_per_real, (long)S - t0);
    const long bin = (long)r * Nd + (valid ? i : 0);
    const float al = alpha[bin];
    const float scale = valid ? (mode == PRECODE ? al : 1.0f / al) : 0.f;
    const int npairs = (M + 1) / 2;

    for (int s0 = 0; s0 < nsym; s0 += SC) {
        const int ns = min(SC, nsym - s0);
        __syncthreads();
        for (int e = warp; e < SC * K; e += nwarps) {
            const int s = e / K, u = e % K;
            sB[e * 32 + lane] = (valid && s < ns) ? B[((t0 + s0 + s) * K + u) * Nd + i] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int pr = warp; pr < npairs; pr += nwarps) {
            const int m0 = 2 * pr, m1 = m0 + 1;
            const bool has1 = m1 < M;
            c32 acc0[SC], acc1[SC];
#pragma unroll
            for (int s = 0; s < SC; ++s) acc0[s] = acc1[s] = make_float2(0.f, 0.f);
            for (int u0 = 0; u0 < K; u0 += 4) {
                c32 a0[4], a1[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {   // four users' loads in flight together
                    const int u = u0 + j;
                    a0[j] = a1[j] = make_float2(0.f, 0.f);
                    if (valid && u < K) {
                        if (mode == PRECODE) {
                            a0[j] = ld(A + (bin * M + m0) * K + u);
                            if (has1) a1[j] = ld(A + (bin * M + m1) * K + u);
                        } else {
                            a0[j] = cconj(ld(A + (bin * K + u) * M + m0));
                            if (has1) a1[j] = cconj(ld(A + (bin * K + u) * M + m1));
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (u0 + j >= K) break;
                    const c32 *bs = sB + (u0 + j) * 32 + lane;
#pragma unroll
                    for (int s = 0; s < SC; ++s) {
                        const c32 b = bs[s * K * 32];
                        acc0[s] = cfma(a0[j], b, acc0[s]);
                        acc1[s] = cfma(a1[j], b, acc1[s]);
                    }
                }
            }
            if (valid) {
#pragma unroll
                for (int s = 0; s < SC; ++s) {
                    if (s < ns) {
                        out[((t0 + s0 + s) * M + m0) * Nd + i] = cscale(acc0[s], scale);
                        if (has1) out[((t0 + s0 + s) * M + m1) * Nd + i] = cscale(acc1[s], scale);
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
template <typename TA, int PPW, int SC>
__global__ void __launch_bounds__(256, 2) reduce2_kernel(Geo g, int mode, int S, const TA *__restrict__ A,
                                                      const float *__restrict__ alpha, const c32 *__restrict__ B,
                                                      c32 *__restrict__ out, const c32 *__restrict__ s_ref,
                                                      c32 *__restrict__ gy, double *metrics, double inv_count) {
    extern __shared__ __align__(16) c32 sB[];   // [SC][RMC][32]
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
    const int npairs = (K + 1) / 2;
    double err = 0, sig = 0;

    for (int s0 = 0; s0 < nsym; s0 += SC) {
        const int ns = min(SC, nsym - s0);
        // each warp owns user pairs pr = warp, warp + nwarps, ...; at most 2 pairs per warp
        c32 acc[PPW][2][SC];
#pragma unroll
        for (int a = 0; a < PPW; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int s = 0; s < SC; ++s) acc[a][b][s] = make_float2(0.f, 0.f);
        for (int m0 = 0; m0 < M; m0 += RMC) {
            const int nm = min(RMC, M - m0);
            __syncthreads();
            for (int e = warp; e < SC * RMC; e += nwarps) {
                const int s = e / RMC, mm = e % RMC;
                sB[e * 32 + lane] = (valid && s < ns && mm < nm) ? B[((t0 + s0 + s) * M + m0 + mm) * Nd + i]
                                                                  : make_float2(0.f, 0.f);
            }
            __syncthreads();
#pragma unroll
            for (int pp = 0; pp < PPW; ++pp) {
                const int pr = warp + pp * nwarps;
                if (pr >= npairs) break;
                const int u0 = 2 * pr, u1 = u0 + 1;
                const bool has1 = u1 < K;
                for (int mb = 0; mb < nm; mb += 4) {
                    c32 a0[4], a1[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {   // four antennas' loads in flight together
                        const int m = m0 + mb + j;
                        a0[j] = a1[j] = make_float2(0.f, 0.f);
                        if (valid && mb + j < nm) {
                            if (mode == COMBINE) {
                                a0[j] = ld(A + (bin * K + u0) * M + m);
                                if (has1) a1[j] = ld(A + (bin * K + u1) * M + m);
                            } else {
                                a0[j] = cconj(ld(A + (bin * M + m) * K + u0));
                                if (has1) a1[j] = cconj(ld(A + (bin * M + m) * K + u1));
                            }
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (mb + j >= nm) break;
                        const c32 *bs = sB + (mb + j) * 32 + lane;
#pragma unroll
                        for (int s = 0; s < SC; ++s) {
                            const c32 b = bs[s * RMC * 32];
                            acc[pp][0][s] = cfma(a0[j], b, acc[pp][0][s]);
                            acc[pp][1][s] = cfma(a1[j], b, acc[pp][1][s]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int pp = 0; pp < PPW; ++pp) {
            const int pr = warp + pp * nwarps;
            if (pr >= npairs || !valid) continue;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int u = 2 * pr + h;
                if (u >= K) continue;
#pragma unroll
                for (int s = 0; s < SC; ++s) {
                    if (s >= ns) continue;
                    const long idx = ((t0 + s0 + s) * K + u) * Nd + i;
                    const c32 v = cscale(acc[pp][h][s], scale);
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

// symbols per chunk: the realisation length when it is 14 (one slot), else 8 or 16
inline int chunk_symbols(int S_per_real) { return S_per_real <= 8 ? 8 : (S_per_real % 14 == 0 ? 14 : 16); }

template <typename TA, int SC>
inline cudaError_t expand_sc(const Geo &g, int mode, int S, const TA *A, const float *alpha, const c32 *B, c32 *out,
                             cudaStream_t st) {
    const int R = (S + g.S_per_real - 1) / g.S_per_real;
    if (R == 0) return cudaSuccess;
    dim3 grid((g.N_d + 31) / 32, R);
    const size_t sm = sizeof(c32) * SC * g.K * 32;
    cudaError_t e = cudaFuncSetAttribute(expand2_kernel<TA, SC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    expand2_kernel<TA, SC><<<grid, 256, sm, st>>>(g, mode, S, A, alpha, B, out);
    return cudaGetLastError();
}

template <typename TA>
inline cudaError_t expand_t(const Geo &g, int mode, int S, const TA *A, const float *alpha, const c32 *B, c32 *out,
                            cudaStream_t st) {
    switch (chunk_symbols(g.S_per_real)) {
        case 8: return expand_sc<TA, 8>(g, mode, S, A, alpha, B, out, st);
        case 14: return expand_sc<TA, 14>(g, mode, S, A, alpha, B, out, st);
        default: return expand_sc<TA, 16>(g, mode, S, A, alpha, B, out, st);
    }
}

template <typename TA, int SC>
inline cudaError_t reduce_sc(const Geo &g, int mode, int S, const TA *A, const float *alpha, const c32 *B, c32 *out,
                             const c32 *s_ref, c32 *gy, double *metrics, double inv_count, cudaStream_t st) {
    const int R = (S + g.S_per_real - 1) / g.S_per_real;
    if (R == 0) return cudaSuccess;
    dim3 grid((g.N_d + 31) / 32, R);
    const int npairs = (g.K + 1) / 2;
    const int nwarps = npairs < 8 ? npairs : 8;    // <= 2 user pairs per warp (K <= 32)
    const size_t sm = sizeof(c32) * SC * RMC * 32;
    if (npairs > nwarps && SC != 8) return reduce_sc<TA, 8>(g, mode, S, A, alpha, B, out, s_ref, gy, metrics, inv_count, st);
    if (npairs <= nwarps) {
        cudaError_t e = cudaFuncSetAttribute(reduce2_kernel<TA, 1, SC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        reduce2_kernel<TA, 1, SC><<<grid, 32 * nwarps, sm, st>>>(g, mode, S, A, alpha, B, out, s_ref, gy, metrics, inv_count);
    } else {
        cudaError_t e = cudaFuncSetAttribute(reduce2_kernel<TA, 2, SC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        reduce2_kernel<TA, 2, SC><<<grid, 32 * nwarps, sm, st>>>(g, mode, S, A, alpha, B, out, s_ref, gy, metrics, inv_count);
    }
    return cudaGetLastError();
}

template <typename TA>
inline cudaError_t reduce_t(const Geo &g, int mode, int S, const TA *A, const float *alpha, const c32 *B, c32 *out,
                            const c32 *s_ref, c32 *gy, double *metrics, double inv_count, cudaStream_t st) {
    switch (chunk_symbols(g.S_per_real)) {
        case 8: return reduce_sc<TA, 8>(g, mode, S, A, alpha, B, out, s_ref, gy, metrics, inv_count, st);
        case 14: return reduce_sc<TA, 14>(g, mode, S, A, alpha, B, out, s_ref, gy, metrics, inv_count, st);
        default: return reduce_sc<TA, 16>(g, mode, S, A, alpha, B, out, s_ref, gy, metrics, inv_count, st);
    }
}

// One translation unit per operand storage type instantiates these.
#define FD_BIN_TYPE(NAME, TA)                                                                                    \
    cudaError_t bin_expand_##NAME(const Geo &g, int mode, int S, const void *A, const float *alpha, const c32 *B, \
                                  c32 *out, cudaStream_t st) {                                                  \
        return expand_t(g, mode, S, (const TA *)A, alpha, B, out, st);                                          \
    }                                                                                                           \
    cudaError_t bin_reduce_##NAME(const Geo &g, int mode, int S, const void *A, const float *alpha, const c32 *B, \
                                  c32 *out, const c32 *s_ref, c32 *gy, double *metrics, double inv_count,       \
                                  cudaStream_t st) {                                                            \
        return reduce_t(g, mode, S, (const TA *)A, alpha, B, out, s_ref, gy, metrics, inv_count, st);           \
    }
#define FD_BIN_DECL(NAME)                                                                                        \
    cudaError_t bin_expand_##NAME(const Geo &g, int mode, int S, const void *A, const float *alpha, const c32 *B, \
                                  c32 *out, cudaStream_t st);                                                   \
    cudaError_t bin_reduce_##NAME(const Geo &g, int mode, int S, const void *A, const float *alpha, const c32 *B, \
                                  c32 *out, const c32 *s_ref, c32 *gy, double *metrics, double inv_count,       \
                                  cudaStream_t st);
FD_BIN_DECL(f32) FD_BIN_DECL(bf16) FD_BIN_DECL(f16)

}  // namespace fdk
