// Shared device helpers of the fddpd library (complex FP32 arithmetic, 16-bit
// operand conversion, block reductions).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#define FD_HD __host__ __device__ __forceinline__
#define FD_D __device__ __forceinline__

typedef float2 c32;

FD_HD c32 cmk(float r, float i) { return make_float2(r, i); }
FD_HD c32 cadd(c32 a, c32 b) { return make_float2(a.x + b.x, a.y + b.y); }
FD_HD c32 csub(c32 a, c32 b) { return make_float2(a.x - b.x, a.y - b.y); }
FD_HD c32 cscale(c32 a, float s) { return make_float2(a.x * s, a.y * s); }
FD_HD c32 cconj(c32 a) { return make_float2(a.x, -a.y); }
FD_HD c32 cmul(c32 a, c32 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// a * conj(b)
FD_HD c32 cmulc(c32 a, c32 b) { return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }
// acc += a * b
FD_HD c32 cfma(c32 a, c32 b, c32 acc) {
    acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(a.y, b.x, acc.y);
    return acc;
}
// acc += conj(a) * b
FD_HD c32 cfmac(c32 a, c32 b, c32 acc) {
    acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(-a.y, b.x, acc.y);
    return acc;
}
FD_HD float cabs2(c32 a) { return fmaf(a.x, a.x, a.y * a.y); }

// 16-bit complex operand storage: (re, im) pair of bf16 or fp16.
struct cbf16 { __nv_bfloat162 v; };
struct cf16 { __half2 v; };

template <typename T> struct Operand;
template <> struct Operand<c32> {
    static FD_D c32 load(const c32 *p) { return *p; }
    static FD_D c32 from(c32 a) { return a; }
};
template <> struct Operand<cbf16> {
    static FD_D c32 load(const cbf16 *p) { return __bfloat1622float2(p->v); }
    static FD_D cbf16 from(c32 a) { cbf16 r; r.v = __float22bfloat162_rn(a); return r; }
};
template <> struct Operand<cf16> {
    static FD_D c32 load(const cf16 *p) { return __half22float2(p->v); }
    static FD_D cf16 from(c32 a) { cf16 r; r.v = __float22half2_rn(a); return r; }
};

FD_D float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
FD_D double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block (blockDim.x a multiple of 32, <= 1024); result valid in thread 0.
template <typename T>
FD_D T block_sum(T v, T *scratch /* >= 32 entries */) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) scratch[w] = v;
    __syncthreads();
    T r = 0;
    if (w == 0) {
        r = (l < (int)(blockDim.x >> 5)) ? scratch[l] : T(0);
        r = warp_sum(r);
    }
    return r;
}

// Index of data subcarrier for FFT bin k, or -1 for a guard bin.
// CTAs of kernel k that fit on one SM at once: the register / thread limit from the
// occupancy query (asked without dynamic shared memory, which it counts against a smaller
// carveout than the one launches get), and the shared memory against the SM's capacity at
// the largest carveout, which is requested here.
template <class Kern> inline int resident_ctas(Kern k, int threads, size_t dyn_smem) {
    int dev = 0, cap = 0, resv = 0, by_regs = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, k);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&by_regs, k, threads, 0) != cudaSuccess || by_regs < 1) by_regs = 1;
    const size_t per = dyn_smem + fa.sharedSizeBytes + (size_t)resv;
    const int by_smem = cap > 0 ? (int)((size_t)cap / per) : 1;
    const int n = by_regs < by_smem ? by_regs : by_smem;
    return n > 0 ? n : 1;
}

FD_HD int data_index(int k, int first_bin, int N, int N_d) {
    int i = (k - first_bin) & (N - 1);  // N is a power of two
    return i < N_d ? i : -1;
}
