// Zero-forcing precoder, Eq. (6): W_k = H_k^H (H_k H_k^H)^{-1} and the per-subcarrier
// normalisation alpha_k = sqrt(P_T / tr((H_k H_k^H)^{-1})), so that the precoded
// vector alpha_k W_k s has E||.||^2 = P_T for unit-power symbols.
//
// Three kernels over all (realisation, data subcarrier) pairs ("bins"):
//   gram   : one warp per bin, G = H H^H from FP32 products and FP32 sums; each lane a
//            4 x 2 block of G (6 shared loads per 8 complex multiply-adds).  The lower
//            triangle goes to a scratch array laid out [bin / 32][entry][bin % 32].
//   factor : one bin per LANE, so every FP64 instruction is a full-warp instruction:
//            Cholesky G = L L^H (left-looking) and the in-place triangular inverse
//            Y = L^{-1} in FP64; tr(G^{-1}) = ||Y||_F^2 in FP64.  1/sqrt(d) starts from
//            the FP32 rsqrtf and takes two Newton-Raphson steps y <- y (3 - d y^2) / 2
//            in FP64.  Y (FP32) and alpha go out; a pivot <= 1e-9 of its Gram diagonal
//            marks the bin singular (alpha = 0, W = 0, status bit 0).
//   apply  : one warp per bin, W^H = Y^H (Y H) in FP32 (one antenna per lane), staged
//            through shared memory for coalesced stores.
#include "common.cuh"
#include "kernels.h"

namespace fdk {

static constexpr int ZF_WARPS = 8;

__host__ __device__ static inline size_t al16(size_t b) { return (b + 15) & ~size_t(15); }
__host__ __device__ static inline int tri(int K) { return K * (K + 1) / 2; }
FD_HD long soa(long b, int e, int T) { return (b >> 5) * (long)T * 32 + (long)e * 32 + (b & 31); }

size_t zf_scratch_bytes(const Geo &g, long nbins) {
    const long nb32 = (nbins + 31) / 32 * 32;
    return 2 * al16(sizeof(c32) * (size_t)nb32 * tri(g.K)) + 256;
}

FD_D void load_h(const c32 *__restrict__ Hb, c32 *sH, int K, int M, int ld, bool vec4, int lane) {
    if (vec4) {
        const float4 *Hb4 = reinterpret_cast<const float4 *>(Hb);
        for (int e = lane; e < K * M / 2; e += 32) {
            const float4 v = Hb4[e];
            const int idx = 2 * e, u = idx / M, m = idx % M;
            sH[u * ld + m] = make_float2(v.x, v.y);
            sH[u * ld + m + 1] = make_float2(v.z, v.w);
        }
    } else {
        for (int e = lane; e < K * M; e += 32) sH[(e / M) * ld + e % M] = Hb[e];
    }
}

// ---------------------------------------------------------------------------
template <typename T16>
__global__ void __launch_bounds__(32 * ZF_WARPS) zf_gram_kernel(Geo g, long nbins, const c32 *__restrict__ H,
                                                                c32 *__restrict__ Gs, T16 *__restrict__ H16) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int K = g.K, M = g.M, ld = M + 1, T = tri(K);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    c32 *sH = reinterpret_cast<c32 *>(sm) + (size_t)warp * K * ld;
    const bool vec4 = !(M & 1) && !(reinterpret_cast<uintptr_t>(H) & 15);
    const int nib = (K + 3) / 4, njb = (K + 1) / 2;
    for (long b = (long)blockIdx.x * nwarps + warp; b < nbins; b += (long)gridDim.x * nwarps) {
        load_h(H + b * K * M, sH, K, M, ld, vec4, lane);
        __syncwarp();
        if (H16)
            for (int e = lane; e < K * M; e += 32) H16[b * K * M + e] = Operand<T16>::from(sH[(e / M) * ld + e % M]);
        for (int blk = lane; blk < nib * njb; blk += 32) {
            const int i0 = (blk / njb) * 4, j0 = (blk % njb) * 2;
            if (j0 > i0 + 3) continue;   // block entirely above the diagonal
            const int ni = min(4, K - i0), nj = min(2, K - j0);
            c32 acc[4][2];
#pragma unroll
            for (int a = 0; a < 4; ++a) acc[a][0] = acc[a][1] = make_float2(0.f, 0.f);
            for (int m = 0; m < M; ++m) {
                c32 hi[4], hj[2];
#pragma unroll
                for (int a = 0; a < 4; ++a) hi[a] = a < ni ? sH[(i0 + a) * ld + m] : make_float2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < 2; ++c) hj[c] = c < nj ? cconj(sH[(j0 + c) * ld + m]) : make_float2(0.f, 0.f);
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 2; ++c) acc[a][c] = cfma(hi[a], hj[c], acc[a][c]);
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int i = i0 + a, j = j0 + c;
                    if (a < ni && c < nj && j <= i) Gs[soa(b, tri(i) + j, T)] = acc[a][c];
                }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
FD_D double rsqrt_f64(double d) {
    double y = (double)rsqrtf((float)d);
#pragma unroll
    for (int it = 0; it < 2; ++it) y = y * (1.5 - 0.5 * d * y * y);
    return y;
}

__global__ void __launch_bounds__(32) zf_factor_kernel(Geo g, long nbins, const c32 *__restrict__ Gs,
                                                       c32 *__restrict__ Ys, float *__restrict__ alpha, int *status) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int K = g.K, T = tri(K);
    const int lane = threadIdx.x, NB = blockDim.x;          // NB bins per CTA, one per thread
    double2 *A = reinterpret_cast<double2 *>(sm);          // [T][NB]: lower triangle, becomes L, then Y
    double *inv = reinterpret_cast<double *>(A + (size_t)T * NB);   // [K][NB]
    const long b = (long)blockIdx.x * NB + lane;
    const bool live = b < nbins;
    const long bb = live ? b : 0;
    for (int e = 0; e < T; ++e) {
        const c32 v = Gs[soa(bb, e, T)];
        A[e * NB + lane] = make_double2(v.x, v.y);
    }
    bool bad = false;
    // Cholesky, left-looking: column j from the columns left of it
    for (int j = 0; j < K; ++j) {
        const int dj = tri(j) + j;
        double d = A[dj * NB + lane].x;
        const double g0 = d;
        for (int k = 0; k < j; ++k) {
            const double2 l = A[(tri(j) + k) * NB + lane];
            d = fma(-l.x, l.x, d);
            d = fma(-l.y, l.y, d);
        }
        const bool ok = d > 1e-9 * g0;
        bad |= !ok;
        const double r = ok ? rsqrt_f64(d) : 1.0;
        A[dj * NB + lane] = make_double2(ok ? d * r : 1.0, 0.0);
        inv[j * NB + lane] = r;
        for (int i = j + 1; i < K; ++i) {
            double2 s = A[(tri(i) + j) * NB + lane];
            for (int k = 0; k < j; ++k) {     // s -= L[i][k] conj(L[j][k])
                const double2 a = A[(tri(i) + k) * NB + lane], c = A[(tri(j) + k) * NB + lane];
                s.x = fma(-a.x, c.x, s.x);
                s.x = fma(-a.y, c.y, s.x);
                s.y = fma(-a.y, c.x, s.y);
                s.y = fma(a.x, c.y, s.y);
            }
            A[(tri(i) + j) * NB + lane] = make_double2(s.x * r, s.y * r);
        }
    }
    // in-place inverse: for j = K-1..0, Y[j][j] = 1/L[j][j], and for i = K-1..j+1
    // Y[i][j] = -(1/L[j][j]) sum_{k=j+1}^{i} Y[i][k] L[k][j]  (L[k][j], k <= i, not yet overwritten)
    double tr = 0.0;
    for (int j = K - 1; j >= 0; --j) {
        const double r = inv[j * NB + lane];
        for (int i = K - 1; i > j; --i) {
            double2 s = make_double2(0.0, 0.0);
            for (int k = j + 1; k <= i; ++k) {
                const double2 y = A[(tri(i) + k) * NB + lane], l = A[(tri(k) + j) * NB + lane];
                s.x = fma(y.x, l.x, s.x);
                s.x = fma(-y.y, l.y, s.x);
                s.y = fma(y.x, l.y, s.y);
                s.y = fma(y.y, l.x, s.y);
            }
            const double2 v = make_double2(-s.x * r, -s.y * r);
            A[(tri(i) + j) * NB + lane] = v;
            tr = fma(v.x, v.x, tr);
            tr = fma(v.y, v.y, tr);
        }
        A[(tri(j) + j) * NB + lane] = make_double2(r, 0.0);
        tr = fma(r, r, tr);
    }
    if (live) {
        for (int e = 0; e < T; ++e) {
            const double2 v = A[e * NB + lane];
            Ys[soa(b, e, T)] = make_float2((float)v.x, (float)v.y);
        }
        alpha[b] = bad ? 0.0f : (float)sqrt(g.P_T / tr);
    }
    if (live && bad) atomicOr(status, 1);
}

// ---------------------------------------------------------------------------
template <int KM, typename T16>
__global__ void __launch_bounds__(32 * ZF_WARPS, 2) zf_apply_kernel(Geo g, long nbins, const c32 *__restrict__ H,
                                                                 const c32 *__restrict__ Ys,
                                                                 const float *__restrict__ alpha,
                                                                 c32 *__restrict__ W, T16 *__restrict__ W16) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int K = g.K, M = g.M, T = tri(K);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const size_t per_warp = al16(sizeof(c32) * K * K) + al16(sizeof(c32) * 32 * (K + 1));
    unsigned char *base = sm + warp * per_warp;
    c32 *sY = reinterpret_cast<c32 *>(base);
    c32 *sW = reinterpret_cast<c32 *>(base + al16(sizeof(c32) * K * K));
    for (long b = (long)blockIdx.x * nwarps + warp; b < nbins; b += (long)gridDim.x * nwarps) {
        for (int p = lane; p < K * K; p += 32) {
            const int i = p / K, k = p % K;
            sY[p] = k <= i ? Ys[soa(b, tri(i) + k, T)] : make_float2(0.f, 0.f);
        }
        const bool bad = alpha[b] == 0.0f;
        __syncwarp();
        const c32 *Hb = H + b * K * M;
        c32 *Wb = W + b * M * K;
        for (int m0 = 0; m0 < M; m0 += 32) {
            const int m = m0 + lane;
            if (m < M) {
                // h = H[:, m], then in place q = Y h (descending, q[i] needs h[k <= i])
                c32 q[KM];
#pragma unroll
                for (int k = 0; k < KM; ++k) q[k] = k < K ? Hb[(long)k * M + m] : make_float2(0.f, 0.f);
#pragma unroll
                for (int i = KM - 1; i >= 0; --i) {
                    if (i < K) {
                        c32 acc = make_float2(0.f, 0.f);
#pragma unroll
                        for (int k = 0; k <= i; ++k) acc = cfma(sY[i * K + k], q[k], acc);
                        q[i] = acc;
                    }
                }
#pragma unroll
                for (int u = 0; u < KM; ++u) {
                    if (u < K) {
                        c32 acc = make_float2(0.f, 0.f);
#pragma unroll
                        for (int i = u; i < KM; ++i)
                            if (i < K) acc = cfma(sY[i * K + u], cconj(q[i]), acc);
                        sW[lane * (K + 1) + u] = bad ? make_float2(0.f, 0.f) : acc;
                    }
                }
            }
            __syncwarp();
            const int nm = min(32, M - m0);
            for (int e = lane; e < nm * K; e += 32) {
                const c32 w = sW[(e / K) * (K + 1) + e % K];
                Wb[(long)m0 * K + e] = w;
                if (W16) W16[b * M * K + (long)m0 * K + e] = Operand<T16>::from(w);
            }
            __syncwarp();
        }
    }
}

static int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

template <class Kern>
static cudaError_t persistent_launch_dims(Kern k, int threads, size_t smem, long work_items, int items_per_cta,
                                          long &blocks) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
    if (e != cudaSuccess) return e;
    blocks = (long)(per_sm > 0 ? per_sm : 1) * sm_count();
    const long need = (work_items + items_per_cta - 1) / items_per_cta;
    if (blocks > need) blocks = need;
    return cudaSuccess;
}

template <int KM, typename T16>
static cudaError_t launch_apply(const Geo &g, long nbins, const c32 *H, const c32 *Ys, const float *alpha, c32 *W,
                                T16 *W16, cudaStream_t st) {
    const size_t per_warp = al16(sizeof(c32) * g.K * g.K) + al16(sizeof(c32) * 32 * (g.K + 1));
    int nw = (int)((200 * 1024) / per_warp);
    nw = nw > ZF_WARPS ? ZF_WARPS : nw;
    if (nw < 1) return cudaErrorInvalidConfiguration;
    long blocks = 0;
    cudaError_t e = persistent_launch_dims(zf_apply_kernel<KM, T16>, 32 * nw, nw * per_warp, nbins, nw, blocks);
    if (e != cudaSuccess) return e;
    zf_apply_kernel<KM, T16><<<(unsigned)blocks, 32 * nw, nw * per_warp, st>>>(g, nbins, H, Ys, alpha, W, W16);
    return cudaGetLastError();
}

// phase 0 = gram, 1 = factor, 2 = apply, -1 = all three in order
template <typename T16>
static cudaError_t zf_build_t(const Geo &g, int R, const c32 *H, c32 *W, float *alpha, int *status, void *scratch,
                              T16 *H16, T16 *W16, int phase, cudaStream_t st) {
    const long nbins = (long)R * g.N_d;
    if (nbins == 0) return cudaSuccess;
    const int T = tri(g.K);
    const long nb32 = (nbins + 31) / 32 * 32;
    c32 *Gs = reinterpret_cast<c32 *>(scratch);
    c32 *Ys = reinterpret_cast<c32 *>(reinterpret_cast<char *>(scratch) + al16(sizeof(c32) * (size_t)nb32 * T));
    // gram
    if (phase < 0 || phase == 0) {
        const size_t per_warp = sizeof(c32) * g.K * (g.M + 1);
        int nw = (int)((200 * 1024) / per_warp);
        nw = nw > ZF_WARPS ? ZF_WARPS : nw;
        if (nw < 1) return cudaErrorInvalidConfiguration;
        long blocks = 0;
        cudaError_t e = persistent_launch_dims(zf_gram_kernel<T16>, 32 * nw, nw * per_warp, nbins, nw, blocks);
        if (e != cudaSuccess) return e;
        zf_gram_kernel<T16><<<(unsigned)blocks, 32 * nw, nw * per_warp, st>>>(g, nbins, H, Gs, H16);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // factor
    if (phase < 0 || phase == 1) {
        int NB = 32;
        size_t smem = (sizeof(double2) * T + sizeof(double) * g.K) * NB;
        if (smem > 200 * 1024) {
            NB = 16;
            smem = (sizeof(double2) * T + sizeof(double) * g.K) * NB;
        }
        cudaError_t e = cudaFuncSetAttribute(zf_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        zf_factor_kernel<<<(unsigned)((nbins + NB - 1) / NB), NB, smem, st>>>(g, nbins, Gs, Ys, alpha, status);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // apply
    if (phase >= 0 && phase != 2) return cudaSuccess;
    if (g.K <= 4) return launch_apply<4>(g, nbins, H, Ys, alpha, W, W16, st);
    if (g.K <= 8) return launch_apply<8>(g, nbins, H, Ys, alpha, W, W16, st);
    if (g.K <= 16) return launch_apply<16>(g, nbins, H, Ys, alpha, W, W16, st);
    return launch_apply<32>(g, nbins, H, Ys, alpha, W, W16, st);
}

cudaError_t zf_phase(int phase, const Geo &g, int R, const c32 *H, c32 *W, float *alpha, int *status, void *scratch,
                     void *H16, void *W16, int kind, cudaStream_t st) {
    if (kind == OUT_F16) return zf_build_t(g, R, H, W, alpha, status, scratch, (cf16 *)H16, (cf16 *)W16, phase, st);
    return zf_build_t(g, R, H, W, alpha, status, scratch, (cbf16 *)H16, (cbf16 *)W16, phase, st);
}

cudaError_t zf_build(const Geo &g, int R, const c32 *H, c32 *W, float *alpha, int *status, void *scratch,
                     void *H16, void *W16, int kind, cudaStream_t st) {
    return zf_phase(-1, g, R, H, W, alpha, status, scratch, H16, W16, kind, st);
}

}  // namespace fdk
