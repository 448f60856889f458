// Zero-forcing precoder, Eq. (6): W_k = H_k^H (H_k H_k^H)^{-1} and the per-subcarrier
// normalisation alpha_k = sqrt(P_T / tr((H_k H_k^H)^{-1})), so that the precoded
// vector alpha_k W_k s has E||.||^2 = P_T for unit-power symbols.
//
// One CTA per (realisation, data subcarrier):
//   1. G = H H^H (lower triangle) from FP32 products and FP32 accumulation;
//   2. Cholesky G = L L^H and the triangular inverse Y = L^{-1} in FP64 by one warp
//      (lane i owns row i of L, then column i of Y); tr(G^{-1}) = ||Y||_F^2 in FP64;
//   3. W^H = Y^H (Y H): Q = Y H and W[m][u] = sum_{i>=u} Y[i][u] conj(Q[i][m]) in FP32,
//      one thread per antenna.
// A non-positive pivot (relative to its diagonal) flags the subcarrier as singular:
// its W and alpha are written as zero and the status word is set.
#include "common.cuh"
#include "kernels.h"

namespace fdk {

static constexpr int ZF_THREADS = 128;

__host__ __device__ static inline size_t zf_align(size_t b) { return (b + 15) & ~size_t(15); }

template <int KM>
__global__ void __launch_bounds__(ZF_THREADS) zf_kernel(Geo g, const c32 *__restrict__ H, c32 *__restrict__ W,
                                                        float *__restrict__ alpha, int *status) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int K = g.K, M = g.M, ld = M + 1;
    const long b = blockIdx.x;
    c32 *sH = reinterpret_cast<c32 *>(sm);
    double2 *sG = reinterpret_cast<double2 *>(sm + zf_align(sizeof(c32) * K * ld));   // G, then Y = L^{-1}
    double2 *sL = sG + K * K;
    c32 *sY = reinterpret_cast<c32 *>(sL + K * K);
    __shared__ int bad;
    __shared__ double trace;

    const c32 *Hb = H + b * K * M;
    for (int idx = threadIdx.x; idx < K * M; idx += blockDim.x) sH[(idx / M) * ld + idx % M] = Hb[idx];
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();

    for (int p = threadIdx.x; p < K * K; p += blockDim.x) {
        const int i = p / K, j = p % K;
        if (j > i) continue;
        c32 acc = make_float2(0.f, 0.f);
        const c32 *hi = sH + i * ld, *hj = sH + j * ld;
        for (int m = 0; m < M; ++m) acc = cfma(hi[m], cconj(hj[m]), acc);
        sG[i * K + j] = make_double2(acc.x, acc.y);
    }
    __syncthreads();

    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int j = 0; j < K; ++j) {
            if (lane == j) {
                const double g0 = sG[j * K + j].x;
                double d = g0;
                for (int k = 0; k < j; ++k) {
                    const double2 l = sL[j * K + k];
                    d -= l.x * l.x + l.y * l.y;
                }
                if (!(d > 1e-9 * g0)) {
                    bad = 1;
                    d = 1.0;
                }
                sL[j * K + j] = make_double2(sqrt(d), 0.0);
            }
            __syncwarp();
            if (lane > j && lane < K) {
                double2 s = sG[lane * K + j];
                for (int k = 0; k < j; ++k) {
                    const double2 a = sL[lane * K + k], c = sL[j * K + k];   // s -= a conj(c)
                    s.x -= a.x * c.x + a.y * c.y;
                    s.y -= a.y * c.x - a.x * c.y;
                }
                const double inv = 1.0 / sL[j * K + j].x;
                sL[lane * K + j] = make_double2(s.x * inv, s.y * inv);
            }
            __syncwarp();
        }
        // Y = L^{-1}: lane c solves L y = e_c; Y kept in sG (no longer needed)
        double tr = 0.0;
        if (lane < K) {
            const int c = lane;
            for (int i = 0; i < c; ++i) sG[i * K + c] = make_double2(0.0, 0.0);
            const double y0 = 1.0 / sL[c * K + c].x;
            sG[c * K + c] = make_double2(y0, 0.0);
            tr = y0 * y0;
            for (int i = c + 1; i < K; ++i) {
                double2 s = make_double2(0.0, 0.0);
                for (int k = c; k < i; ++k) {
                    const double2 a = sL[i * K + k], y = sG[k * K + c];
                    s.x += a.x * y.x - a.y * y.y;
                    s.y += a.x * y.y + a.y * y.x;
                }
                const double inv = -1.0 / sL[i * K + i].x;
                const double2 yi = make_double2(s.x * inv, s.y * inv);
                sG[i * K + c] = yi;
                tr += yi.x * yi.x + yi.y * yi.y;
            }
        }
        __syncwarp();
        tr = warp_sum(tr);
        if (lane == 0) trace = tr;
        for (int p = lane; p < K * K; p += 32) sY[p] = make_float2((float)sG[p].x, (float)sG[p].y);
    }
    __syncthreads();

    const bool singular = bad != 0;
    if (threadIdx.x == 0) {
        alpha[b] = singular ? 0.0f : (float)sqrt(g.P_T / trace);
        if (singular) atomicOr(status, 1);
    }
    c32 *Wb = W + b * M * K;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        c32 q[KM];
#pragma unroll
        for (int i = 0; i < KM; ++i) {
            c32 acc = make_float2(0.f, 0.f);
            if (i < K) {
#pragma unroll
                for (int k = 0; k <= i; ++k) acc = cfma(sY[i * K + k], sH[k * ld + m], acc);
            }
            q[i] = acc;
        }
#pragma unroll
        for (int u = 0; u < KM; ++u) {
            if (u < K) {
                c32 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = u; i < KM; ++i)
                    if (i < K) acc = cfma(sY[i * K + u], cconj(q[i]), acc);
                Wb[m * K + u] = singular ? make_float2(0.f, 0.f) : acc;
            }
        }
    }
}

template <int KM>
static cudaError_t launch_zf(const Geo &g, int R, const c32 *H, c32 *W, float *alpha, int *status, cudaStream_t st) {
    const size_t smem = zf_align(sizeof(c32) * g.K * (g.M + 1)) + 2 * sizeof(double2) * g.K * g.K +
                        sizeof(c32) * g.K * g.K;
    cudaError_t e = cudaFuncSetAttribute(zf_kernel<KM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long blocks = (long)R * g.N_d;
    if (blocks == 0) return cudaSuccess;
    zf_kernel<KM><<<(unsigned)blocks, ZF_THREADS, smem, st>>>(g, H, W, alpha, status);
    return cudaGetLastError();
}

cudaError_t zf_build(const Geo &g, int R, const c32 *H, c32 *W, float *alpha, int *status, cudaStream_t st) {
    if (g.K <= 4) return launch_zf<4>(g, R, H, W, alpha, status, st);
    if (g.K <= 8) return launch_zf<8>(g, R, H, W, alpha, status, st);
    if (g.K <= 16) return launch_zf<16>(g, R, H, W, alpha, status, st);
    return launch_zf<32>(g, R, H, W, alpha, status, st);
}

}  // namespace fdk
