// Symbol error counting at the users (Sec. V-B, the Fig. 3 setting).  The received
// frequency-domain symbol of Eq. (5) carries the noise term w_k ~ CN(0, N0) of Eq. (4)
// (unitary DFT: the per-subcarrier noise keeps the variance N0); the user equalises by
// 1 / alpha_k (Eq. 6), so the decided value is z = y + w / alpha_k, with y the noiseless
// equalised symbol the forward chain produces.  z is decided to the nearest point of the
// unit-power square Q-QAM constellation, per component, and compared with the sent s.
//
// The noise is drawn by the method, so it comes from a counter-based generator written
// from its published definition: Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with
// key = the 64-bit seed and counter = (flat index of (symbol, user, subcarrier), 0, 0);
// its first two outputs become u = (x + 1/2) 2^-32 and the Box-Muller transform gives
// w = sqrt(N0) sqrt(-ln u1) (cos 2 pi u2 + j sin 2 pi u2).
#include "common.cuh"
#include "kernels.h"

namespace fdk {

FD_D uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// index of the nearest level of the side-point PAM (levels (2 i - side + 1) / scale)
FD_D int pam_index(float v, float inv_step, int side) {
    const float x = v * inv_step + 0.5f * (float)(side - 1);   // level i sits at x = i
    int i = __float2int_rn(x);
    return i < 0 ? 0 : (i > side - 1 ? side - 1 : i);
}

// IDX: 32-bit index arithmetic when every flat index fits (the divisions by K N_d, N_d
// and S_per_real are then 32-bit), else 64-bit
template <typename IDX>
__global__ void __launch_bounds__(256) ser_kernel(Geo g, IDX n, const c32 *__restrict__ y,
                                                  const c32 *__restrict__ s, const float *__restrict__ alpha,
                                                  int side, float inv_step, float sigma, uint2 key,
                                                  unsigned long long *__restrict__ counts,
                                                  unsigned char *__restrict__ wrong_out) {
    const IDX per_sym = (IDX)g.K * (IDX)g.N_d, nd = (IDX)g.N_d, spr = (IDX)g.S_per_real;
    unsigned errors = 0, compared = 0;
    for (IDX e = blockIdx.x * (IDX)blockDim.x + threadIdx.x; e < n; e += (IDX)gridDim.x * blockDim.x) {
        const IDX t = e / per_sym;
        const IDX i = e % nd;
        const float al = alpha[(long)(t / spr) * g.N_d + (long)i];
        if (!(al > 0.f)) {   // a singular subcarrier carries no symbol
            if (wrong_out) wrong_out[e] = 2;
            continue;
        }
        c32 z = y[e];
        if (sigma > 0.f) {
            const uint4 r = philox4x32_10(make_uint4((uint32_t)e, (uint32_t)((unsigned long long)e >> 32), 0u, 0u), key);
            const float u1 = ((float)r.x + 0.5f) * 2.3283064365386963e-10f;   // 2^-32
            const float u2 = ((float)r.y + 0.5f) * 2.3283064365386963e-10f;
            const float rad = sigma * sqrtf(-logf(u1)) / al;
            float sn, cs;
            sincospif(2.0f * u2, &sn, &cs);
            z.x += rad * cs;
            z.y += rad * sn;
        }
        const c32 sv = s[e];
        const bool wrong = pam_index(z.x, inv_step, side) != pam_index(sv.x, inv_step, side) ||
                           pam_index(z.y, inv_step, side) != pam_index(sv.y, inv_step, side);
        errors += wrong ? 1u : 0u;
        ++compared;
        if (wrong_out) wrong_out[e] = wrong ? 1 : 0;
    }
    __shared__ unsigned red[2][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        errors += __shfl_xor_sync(0xffffffffu, errors, o);
        compared += __shfl_xor_sync(0xffffffffu, compared, o);
    }
    if (lane == 0) {
        red[0][warp] = errors;
        red[1][warp] = compared;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long es = 0, cs = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            es += red[0][w];
            cs += red[1][w];
        }
        atomicAdd(counts, es);
        atomicAdd(counts + 1, cs);
    }
}

cudaError_t ser_count(const Geo &g, int S, const c32 *y, const c32 *s, const float *alpha, int Q, float N0,
                      unsigned long long seed, unsigned long long *counts, cudaStream_t st, unsigned char *wrong) {
    const long n = (long)S * g.K * g.N_d;
    if (n == 0) return cudaSuccess;
    int side = 1;
    while (side * side < Q) ++side;
    // levels (2 i - side + 1) / sqrt(2 (Q - 1) / 3): a step of 2 / that scale between levels
    const float inv_step = (float)(sqrt(2.0 * (Q - 1) / 3.0) / 2.0);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long blocks = (n + 255) / 256;
    const long cap = 8L * (sms > 0 ? sms : 1);
    if (blocks > cap) blocks = cap;
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    if (n + 256L * blocks < 0xFFFFFFFFL)   // no flat index (nor its grid-stride successor) wraps
        ser_kernel<uint32_t><<<(unsigned)blocks, 256, 0, st>>>(g, (uint32_t)n, y, s, alpha, side, inv_step, sqrtf(N0),
                                                              key, counts, wrong);
    else
        ser_kernel<unsigned long long><<<(unsigned)blocks, 256, 0, st>>>(g, (unsigned long long)n, y, s, alpha, side,
                                                                        inv_step, sqrtf(N0), key, counts, wrong);
    return cudaGetLastError();
}

}  // namespace fdk
