// Measurements and checks that sit beside the chain.
//
//   zf_residual : the FP64 check of the zero-forcing identity of Eq. (6), H_k W_k = I_K,
//                 on the precoders a plan produced: max over the checked subcarriers of
//                 max_{i,j} |(H_k W_k - I)_{ij}|, every product and sum in FP64 (the
//                 FP32 H and W are widened exactly).  One CTA per checked subcarrier;
//                 H_k and W_k pass through shared memory in 64-antenna chunks and each
//                 thread owns a few (i, j) entries of the K x K product.
//   alu_peak    : the arithmetic peak of this GPU's FP32 and FP64 pipes, measured with an
//                 FMA loop (16 independent dependency chains per thread, a grid of
//                 resident CTAs on every SM), timed with CUDA events.  It is the
//                 denominator of the ALU rooflines; the paper has no counterpart.
//   wait_probe  : the bounded-wait failure path of the tensor-core kernels, made to run out.
#include <cstdint>

#include "fddpd.h"
#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace fdk {

static constexpr int RES_THREADS = 256;
static constexpr int RES_CHUNK = 64;

// max of non-negative doubles: their bit patterns order like the values
FD_D void atomic_max_nonneg(double *dst, double v) {
    atomicMax(reinterpret_cast<unsigned long long *>(dst), (unsigned long long)__double_as_longlong(v));
}

__global__ void __launch_bounds__(RES_THREADS) zf_residual_kernel(int M, int K, long nbins, long every,
                                                                   const c32 *__restrict__ H,
                                                                   const c32 *__restrict__ W, double *out) {
    __shared__ c32 sH[32 * RES_CHUNK];   // [K][chunk]
    __shared__ c32 sW[RES_CHUNK * 32];   // [chunk][K]
    __shared__ double red[RES_THREADS / 32];
    const long nchk = (nbins + every - 1) / every;
    const int KK = K * K;
    for (long c = blockIdx.x; c < nchk; c += gridDim.x) {
        const long b = c * every;
        const c32 *Hb = H + b * K * M;
        const c32 *Wb = W + b * M * K;
        double2 acc[4];   // entries e = threadIdx.x + q RES_THREADS, K^2 <= 1024
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = make_double2(0.0, 0.0);
        for (int m0 = 0; m0 < M; m0 += RES_CHUNK) {
            const int nm = min(RES_CHUNK, M - m0);
            __syncthreads();
            for (int e = threadIdx.x; e < K * nm; e += RES_THREADS) {
                const int k = e / nm, m = e % nm;
                sH[k * RES_CHUNK + m] = Hb[(long)k * M + m0 + m];
            }
            for (int e = threadIdx.x; e < nm * K; e += RES_THREADS) sW[e] = Wb[(long)m0 * K + e];
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e = threadIdx.x + q * RES_THREADS;
                if (e >= KK) break;
                const int i = e / K, j = e % K;
                double2 s = acc[q];
                for (int m = 0; m < nm; ++m) {
                    const c32 h = sH[i * RES_CHUNK + m], w = sW[m * K + j];
                    const double hr = h.x, hi = h.y, wr = w.x, wi = w.y;
                    s.x = fma(hr, wr, s.x);
                    s.x = fma(-hi, wi, s.x);
                    s.y = fma(hr, wi, s.y);
                    s.y = fma(hi, wr, s.y);
                }
                acc[q] = s;
            }
        }
        double mx = 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = threadIdx.x + q * RES_THREADS;
            if (e >= KK) break;
            const double re = acc[q].x - ((e / K) == (e % K) ? 1.0 : 0.0), im = acc[q].y;
            mx = fmax(mx, sqrt(re * re + im * im));
        }
        for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
        __syncthreads();
        if (threadIdx.x == 0) {
            double v = 0.0;
            for (int w = 0; w < RES_THREADS / 32; ++w) v = fmax(v, red[w]);
            atomic_max_nonneg(out, v);
        }
    }
}

cudaError_t zf_residual(const Geo &g, long nbins, long every, const c32 *H, const c32 *W, double *out,
                        cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), st);
    if (e != cudaSuccess || nbins <= 0) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long nchk = (nbins + every - 1) / every;
    long blocks = (long)(sms > 0 ? sms : 1) * 8;
    if (blocks > nchk) blocks = nchk;
    zf_residual_kernel<<<(unsigned)blocks, RES_THREADS, 0, st>>>(g.M, g.K, nbins, every, H, W, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The bounded-wait failure path of the tensor-core kernels, run on purpose: one thread
// waits on an mbarrier that nothing arrives at (no copy or MMA is in flight), gives up
// after limit_ns, sets the error word as a real timeout does, and the kernel returns.
__global__ void wait_probe_kernel(unsigned long long limit_ns, int *err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tc::mbar_wait_for(&bar, 0, err, limit_ns);
    }
}

cudaError_t wait_probe(unsigned long long limit_ns, int *err, cudaStream_t st) {
    wait_probe_kernel<<<1, 32, 0, st>>>(limit_ns, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FMA-loop peaks
static __device__ float g_sink_f;
static __device__ double g_sink_d;

static constexpr int PK_CHAINS = 16;

FD_D unsigned long long ffma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// kind 0: scalar FP32 FMA, 1: packed FP32-pair FMA (fma.rn.f32x2), 2: FP64 FMA
template <int KIND>
__global__ void __launch_bounds__(256) alu_peak_kernel(int iters, float b, float c) {
    if constexpr (KIND == 0) {
        float a[PK_CHAINS];
#pragma unroll
        for (int i = 0; i < PK_CHAINS; ++i) a[i] = (float)(threadIdx.x + i) * 1e-3f;
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int i = 0; i < PK_CHAINS; ++i) a[i] = fmaf(a[i], b, c);
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < PK_CHAINS; ++i) s += a[i];
        if (s == -1.0f) g_sink_f = s;
    } else if constexpr (KIND == 1) {
        unsigned long long a[PK_CHAINS];
        const unsigned long long bb = ((unsigned long long)__float_as_uint(b) << 32) | __float_as_uint(b);
        const unsigned long long cc = ((unsigned long long)__float_as_uint(c) << 32) | __float_as_uint(c);
#pragma unroll
        for (int i = 0; i < PK_CHAINS; ++i) {
            const float v = (float)(threadIdx.x + i) * 1e-3f;
            a[i] = ((unsigned long long)__float_as_uint(v) << 32) | __float_as_uint(v + 1.0f);
        }
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int i = 0; i < PK_CHAINS; ++i) a[i] = ffma2(a[i], bb, cc);
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < PK_CHAINS; ++i) s += __uint_as_float((unsigned)a[i]) + __uint_as_float((unsigned)(a[i] >> 32));
        if (s == -1.0f) g_sink_f = s;
    } else {
        double a[PK_CHAINS];
        const double bd = b, cd = c;
#pragma unroll
        for (int i = 0; i < PK_CHAINS; ++i) a[i] = (double)(threadIdx.x + i) * 1e-3;
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int i = 0; i < PK_CHAINS; ++i) a[i] = fma(a[i], bd, cd);
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < PK_CHAINS; ++i) s += a[i];
        if (s == -1.0) g_sink_d = s;
    }
}

template <int KIND>
static cudaError_t time_peak(int iters, int reps, cudaStream_t st, double *tflops) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, alu_peak_kernel<KIND>, 256, 0);
    if (e != cudaSuccess) return e;
    const long blocks = (long)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    alu_peak_kernel<KIND><<<(unsigned)blocks, 256, 0, st>>>(iters, 0.999999f, 1e-7f);   // warm-up
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        alu_peak_kernel<KIND><<<(unsigned)blocks, 256, 0, st>>>(iters, 0.999999f, 1e-7f);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    const double fmas = (double)blocks * 256 * PK_CHAINS * (double)iters * reps * (KIND == 1 ? 2 : 1);
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    return cudaSuccess;
}

cudaError_t alu_peak(int kind, double *tflops, cudaStream_t st) {
    switch (kind) {
        case 0: return time_peak<0>(1 << 16, 4, st, tflops);
        case 1: return time_peak<1>(1 << 15, 4, st, tflops);
        case 2: return time_peak<2>(1 << 10, 4, st, tflops);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fdk
