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

constexpr int RMC = 8;    // antennas per shared chunk (reduce)

template <typename TA> FD_D c32 ld(const TA *p) { return Operand<TA>::load(p); }

// ---------------------------------------------------------------------------
template <typename TA> FD_D TA zero_op() { return Operand<TA>::from(make_float2(0.f, 0.f)); }

// expand: each warp walks (antenna pair, 8-user chunk) items; the A operands of the
// next item load into registers while the current one is multiplied.
template <typename TA, int SC>
__global__ void __launch_bounds__(256, 2) expand2_kernel(Geo g, int mode, int S, const TA *__restrict__ A,
                                                         const float *__restrict__ alpha, const c32 *__restrict__ B,
                                                         c32 *__restrict__ out) {
    constexpr int KB = 8;
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
    const int nuc = (K + KB - 1) / KB;
    const int my_pairs = warp < npairs ? (npairs - warp + nwarps - 1) / nwarps : 0;
    const int nitems = my_pairs * nuc;

    auto load_item = [&](int it, TA (&x0)[KB], TA (&x1)[KB]) {
        const int pr = warp + (it / nuc) * nwarps, uc = it % nuc;
        const int m0 = 2 * pr, m1 = m0 + 1;
#pragma unroll
        for (int j = 0; j < KB; ++j) {
            const int u = uc * KB + j;
            const bool ok = valid && u < K;
            if (mode == PRECODE) {
                x0[j] = ok ? A[(bin * M + m0) * K + u] : zero_op<TA>();
                x1[j] = (ok && m1 < M) ? A[(bin * M + m1) * K + u] : zero_op<TA>();
            } else {
                x0[j] = ok ? A[(bin * K + u) * M + m0] : zero_op<TA>();
                x1[j] = (ok && m1 < M) ? A[(bin * K + u) * M + m1] : zero_op<TA>();
            }
        }
    };

    for (int s0 = 0; s0 < nsym; s0 += SC) {
        const int ns = min(SC, nsym - s0);
        __syncthreads();
        for (int e = warp; e < SC * K; e += nwarps) {
            const int s = e / K, u = e % K;
            sB[e * 32 + lane] = (valid && s < ns) ? B[((t0 + s0 + s) * K + u) * Nd + i] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        TA n0[KB], n1[KB];
        if (nitems > 0) load_item(0, n0, n1);
        c32 acc0[SC], acc1[SC];
        for (int it = 0; it < nitems; ++it) {
            const int pr = warp + (it / nuc) * nwarps, uc = it % nuc;
            TA c0[KB], c1[KB];
#pragma unroll
            for (int j = 0; j < KB; ++j) {
                c0[j] = n0[j];
                c1[j] = n1[j];
            }
            if (it + 1 < nitems) load_item(it + 1, n0, n1);
            if (uc == 0) {
#pragma unroll
                for (int s = 0; s < SC; ++s) acc0[s] = acc1[s] = make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int j = 0; j < KB; ++j) {
                const int u = uc * KB + j;
                if (u >= K) break;
                c32 a0 = Operand<TA>::load(&c0[j]), a1 = Operand<TA>::load(&c1[j]);
                if (mode != PRECODE) {
                    a0 = cconj(a0);
                    a1 = cconj(a1);
                }
                const c32 *bs = sB + u * 32 + lane;
#pragma unroll
                for (int s = 0; s < SC; ++s) {
                    const c32 b = bs[s * K * 32];
                    acc0[s] = cfma(a0, b, acc0[s]);
                    acc1[s] = cfma(a1, b, acc1[s]);
                }
            }
            if (uc == nuc - 1 && valid) {
                const int m0 = 2 * pr, m1 = m0 + 1;
#pragma unroll
                for (int s = 0; s < SC; ++s) {
                    if (s < ns) {
                        out[((t0 + s0 + s) * M + m0) * Nd + i] = cscale(acc0[s], scale);
                        if (m1 < M) out[((t0 + s0 + s) * M + m1) * Nd + i] = cscale(acc1[s], scale);
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
FD_D void cp_async8(void *dst, const void *src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
FD_D void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> FD_D void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// reduce: B chunks of RMC antennas stream into a double buffer with cp.async while the
// previous chunk is consumed; the A operands of a chunk are issued as one batch.
template <typename TA, int PPW, int SC>
__global__ void __launch_bounds__(256, 2) reduce2_kernel(Geo g, int mode, int S, const TA *__restrict__ A,
                                                         const float *__restrict__ alpha, const c32 *__restrict__ B,
                                                         c32 *__restrict__ out, const c32 *__restrict__ s_ref,
                                                         c32 *__restrict__ gy, double *metrics, double inv_count) {
    extern __shared__ __align__(16) c32 sB[];   // [2][SC][RMC][32]
    __shared__ double red[32];
    const int K = g.K, M = g.M, Nd = g.N_d;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int r = blockIdx.y, i0 = blockIdx.x * 32, i = i0 + lane;
    const bool valid = i < Nd;
    const long t0 = (long)r * g.S_per_real;
    const int nsym = (int)min((long)g.S_per_real, (long)S - t0);
    const long bin = (long)r * Nd + (valid ? i : 0);
    const float al = alpha[bin];
    const float scale = valid ? (mode == COMBINE ? 1.0f / al : al) : 0.f;
    const int npairs = (K + 1) / 2;
    const int nchunks = (M + RMC - 1) / RMC;
    constexpr int CH = SC * RMC * 32;   // complex per buffer
    float err = 0.f, sig = 0.f;

    for (int s0 = 0; s0 < nsym; s0 += SC) {
        const int ns = min(SC, nsym - s0);
        auto issue = [&](int c) {
            c32 *dst = sB + (c & 1) * CH;
            for (int e = threadIdx.x; e < CH; e += blockDim.x) {
                const int s = e / (RMC * 32), mm = (e / 32) % RMC, l = e % 32;
                const int m = c * RMC + mm, ii = i0 + l;
                const bool ok = s < ns && m < M && ii < Nd;
                const c32 *src = ok ? B + ((t0 + s0 + s) * M + m) * Nd + ii : B;
                cp_async8(dst + e, src, ok);
            }
            cp_async_commit();
        };
        c32 acc[PPW][2][SC];
#pragma unroll
        for (int a = 0; a < PPW; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int s = 0; s < SC; ++s) acc[a][b][s] = make_float2(0.f, 0.f);
        __syncthreads();   // the previous symbol chunk is done with both buffers
        issue(0);
        for (int c = 0; c < nchunks; ++c) {
            if (c + 1 < nchunks) issue(c + 1);
            // A operands of this chunk, both pairs of the warp, as one batch of loads
            TA a0[PPW][RMC], a1[PPW][RMC];
#pragma unroll
            for (int pp = 0; pp < PPW; ++pp) {
                const int pr = warp + pp * nwarps;
                const int u0 = 2 * pr, u1 = u0 + 1;
#pragma unroll
                for (int mm = 0; mm < RMC; ++mm) {
                    const int m = c * RMC + mm;
                    const bool ok = valid && pr < npairs && m < M;
                    if (mode == COMBINE) {
                        a0[pp][mm] = ok ? A[(bin * K + u0) * M + m] : zero_op<TA>();
                        a1[pp][mm] = (ok && u1 < K) ? A[(bin * K + u1) * M + m] : zero_op<TA>();
                    } else {
                        a0[pp][mm] = ok ? A[(bin * M + m) * K + u0] : zero_op<TA>();
                        a1[pp][mm] = (ok && u1 < K) ? A[(bin * M + m) * K + u1] : zero_op<TA>();
                    }
                }
            }
            if (c + 1 < nchunks) cp_async_wait<1>();
            else cp_async_wait<0>();
            __syncthreads();
            const c32 *buf = sB + (c & 1) * CH;
#pragma unroll
            for (int pp = 0; pp < PPW; ++pp) {
                if (warp + pp * nwarps >= npairs) break;
#pragma unroll
                for (int mm = 0; mm < RMC; ++mm) {
                    c32 x0 = Operand<TA>::load(&a0[pp][mm]), x1 = Operand<TA>::load(&a1[pp][mm]);
                    if (mode != COMBINE) {
                        x0 = cconj(x0);
                        x1 = cconj(x1);
                    }
                    const c32 *bs = buf + mm * 32 + lane;
#pragma unroll
                    for (int s = 0; s < SC; ++s) {
                        const c32 b = bs[s * RMC * 32];
                        acc[pp][0][s] = cfma(x0, b, acc[pp][0][s]);
                        acc[pp][1][s] = cfma(x1, b, acc[pp][1][s]);
                    }
                }
            }
            __syncthreads();   // buffer (c & 1) is refilled by issue(c + 2)
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
        const double es = block_sum((double)err, red);
        const double ss = block_sum((double)sig, red);
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
    const size_t sm = sizeof(c32) * 2 * SC * RMC * 32;
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
