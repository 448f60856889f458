// Zero-forcing precoder matrix W_i = H_i^H Z_i, Z_i = (H_i H_i^H)^{-1} (Eq. 6), on the
// 5th-generation tensor cores, for 16-bit plans (K <= 16, M <= 128).  The factor kernel
// leaves Y = L^{-1} (lower triangle, FP32) in its scratch layout [bin / 32][entry][bin % 32],
// and Z = Y^H Y is formed here in FP32 while the operands are staged.
//
// W[m][u] = sum_i conj(H[i][m]) Z[i][u] is an expand-shaped contraction: A = H^T with
// antenna rows m and k = (i, c) interleaved (re, im) pairs, B = the conjugate real form
// of Z (row 2u = (Zr, Zi), row 2u + 1 = (Zi, -Zr) over k = (i, c)), so D[m][2u + c] is
// component c of W[m][u].  W is an output in FP32, so each operand is split into BF16
// high and low parts (x = hi + lo, lo = bf16(x - hi)), and hi.hi + lo.hi + hi.lo goes
// into the same FP32 accumulator: the dropped lo.lo term and the rounding of lo leave a
// relative error near 2^-16, far below the 16-bit rounding the plan's copy of W
// undergoes.  BF16 keeps the FP32 exponent range, so FP16 plans use it here too.
//
// An item is 4 consecutive subcarriers; each MMA is M = 128 (antennas), N = 32 (16 users
// x re / im), K = 2 x 16, three per K step.  The epilogue writes W [bin][m][u] in FP32
// (unless W is null: only the copy is wanted) and the plan's 16-bit copy; singular
// subcarriers (alpha = 0) get W = 0.
#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace fdk {
namespace tczf {
using namespace tc;

constexpr int NBI = 4;
// A hi / lo: 2 pair tiles of [128 rows][128 B] each; B hi / lo: 2 pair tiles of [32][128 B]
constexpr int A_BYTES = 2 * 16384, B_BYTES = 2 * 4096;

FD_HD int tri(int K) { return K * (K + 1) / 2; }
FD_HD long soa(long b, int e, int T) { return (b >> 5) * (long)T * 32 + (long)e * 32 + (b & 31); }

FD_D uint32_t bf2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}
// hi / lo BF16 pairs of a complex value
FD_D void split(c32 v, uint32_t &hi, uint32_t &lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
    const float2 hf = __bfloat1622float2(h);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = bf2(v.x - hf.x, v.y - hf.y);
}

// One CTA of 512 threads per SM walks its items with two raw stages.
// While item j is converted, multiplied and written out, cp.async brings item j + 1's
// H block (4 subcarriers are contiguous in H), its Y lower triangles (4 subcarriers are
// contiguous per entry in the scratch layout) and its alpha into the other stage, so the
// loads are never on the item's critical path.  16 warps: warp w reads TMEM lane quarter
// w % 4 (antennas) of subcarrier w / 4.
constexpr int PT = 512;
constexpr int RAW_H = NBI * 16 * 128 * 8;            // H of 4 subcarriers, [b][u][m]
constexpr int RAW_Z = NBI * 136 * 8;                  // Y entries [e][b]
constexpr int STAGE = RAW_H + RAW_Z + 16;             // + alpha of the 4 subcarriers
constexpr int SMEM = 2 * A_BYTES + 2 * B_BYTES + 2 * STAGE + 1024;

FD_D void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

template <typename T16>
__global__ void __launch_bounds__(PT, 1)
    apply_kernel(Geo g, long nbins, const c32 *__restrict__ H, const c32 *__restrict__ Zs,
                      const float *__restrict__ alpha, c32 *__restrict__ W, T16 *__restrict__ W16, int vec, int h16,
                      int *err) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *aHi = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *aLo = aHi + A_BYTES;
    uint8_t *bHi = aLo + A_BYTES;
    uint8_t *bLo = bHi + B_BYTES;
    uint8_t *stg0 = bLo + B_BYTES;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int M = g.M, K = g.K, T = tri(K);
    const long nitems = (nbins + NBI - 1) / NBI;
    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&tmem_slot, 128);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = instr_desc(1, 128, 32);
    const int nks = K > 8 ? 2 : 1;
    uint32_t phase = 0;
    bool alive = true;

    // raw stage s: H [b][u][m] (RAW_H bytes), Z [e][b] (RAW_Z), alpha [b]
    auto issue = [&](long item, int s) {
        if (item < nitems) {
            uint8_t *dst = stg0 + (size_t)s * STAGE;
            const long b0 = item * NBI;
            const int n = (int)min((long)NBI, nbins - b0);
            const char *src = reinterpret_cast<const char *>(H + b0 * K * M);
            const int bytes = n * K * M * 8;
            if (h16) {
                for (int o = 16 * tid; o < bytes; o += 16 * PT) cp_async16(dst + o, src + o, true);
            } else {
                for (int o = 8 * tid; o < bytes; o += 8 * PT) cp_async8(dst + o, src + o);
            }
            // bins past nbins in the last item read scratch padding (never used)
            for (int c = tid; c < 2 * T; c += PT)
                cp_async16(dst + RAW_H + 16 * c, reinterpret_cast<const char *>(Zs + soa(b0, c >> 1, T)) + 16 * (c & 1),
                           true);
            if (tid < n) cp_async4(dst + RAW_H + RAW_Z + 4 * tid, alpha + b0 + tid, true);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    issue(blockIdx.x, 0);
    int s = 0;
    for (long item = blockIdx.x; item < nitems && alive; item += gridDim.x, s ^= 1) {
        const long bin0 = item * NBI;
        const int nb = (int)min((long)NBI, nbins - bin0);
        issue(item + gridDim.x, s ^ 1);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncthreads();
        const uint8_t *stg = stg0 + (size_t)s * STAGE;
        const c32 *rH = reinterpret_cast<const c32 *>(stg);
        const c32 *rZ = reinterpret_cast<const c32 *>(stg + RAW_H);
        const float *rA = reinterpret_cast<const float *>(stg + RAW_H + RAW_Z);
        // A: chunk (pair tile p, antenna m, 16-byte chunk ch) = users 4 (ch & 3) .. + 3 of
        // subcarrier 2p + (ch >> 2), split into BF16 hi / lo
        for (int c = tid; c < 2 * 128 * 8; c += PT) {
            const int m = c & 127, ch = (c >> 7) & 7, b = 2 * (c >> 10) + (ch >> 2), u0 = 4 * (ch & 3);
            const bool ok = b < nb && m < M;
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const c32 v = (ok && u0 + j < K) ? rH[(b * K + u0 + j) * M + m] : make_float2(0.f, 0.f);
                split(v, hi[j], lo[j]);
            }
            const uint32_t off = (c >> 10) * 16384 + sw128_offset(m, ch * 8);
            *reinterpret_cast<uint4 *>(aHi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4 *>(aLo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
        // B: element (i, u, subcarrier b) = Z[i][u] = sum_{k >= max(i, u)} conj(Y[k][i]) Y[k][u]
        // (FP32, from the factor's lower-triangular Y = L^{-1}); rows 2u and 2u + 1 of pair
        // tile b >> 1 at k = 32 (b & 1) + 2i
        for (int e = tid; e < 16 * 16 * NBI; e += PT) {
            const int b = e & 3, u = (e >> 2) & 15, i = e >> 6;
            c32 z = make_float2(0.f, 0.f);
            if (b < nb && i < K && u < K)
                for (int k = i > u ? i : u; k < K; ++k) {
                    const c32 yi = rZ[(tri(k) + i) * 4 + b], yu = rZ[(tri(k) + u) * 4 + b];
                    z.x = fmaf(yi.x, yu.x, fmaf(yi.y, yu.y, z.x));
                    z.y = fmaf(yi.x, yu.y, fmaf(-yi.y, yu.x, z.y));
                }
            uint32_t h0, l0, h1, l1;
            split(z, h0, l0);                                  // (Zr, Zi)
            split(make_float2(z.y, -z.x), h1, l1);             // (Zi, -Zr)
            const int k = 32 * (b & 1) + 2 * i;
            const uint32_t o0 = (b >> 1) * 4096 + sw128_offset(2 * u, k);
            const uint32_t o1 = (b >> 1) * 4096 + sw128_offset(2 * u + 1, k);
            *reinterpret_cast<uint32_t *>(bHi + o0) = h0;
            *reinterpret_cast<uint32_t *>(bLo + o0) = l0;
            *reinterpret_cast<uint32_t *>(bHi + o1) = h1;
            *reinterpret_cast<uint32_t *>(bLo + o1) = l1;
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            fence_after();
            for (int b = 0; b < nb; ++b)
                for (int ks = 0; ks < nks; ++ks) {
                    const uint32_t ao = (b >> 1) * 16384 + (b & 1) * 64 + ks * 32;
                    const uint32_t bo = (b >> 1) * 4096 + (b & 1) * 64 + ks * 32;
                    const uint32_t d = tmem + 32 * b;
                    mma_f16(d, smem_desc(aHi + ao), smem_desc(bHi + bo), idesc, ks ? 1u : 0u);
                    mma_f16(d, smem_desc(aLo + ao), smem_desc(bHi + bo), idesc, 1u);
                    mma_f16(d, smem_desc(aHi + ao), smem_desc(bLo + bo), idesc, 1u);
                }
            mma_commit(&bar);
        }
        const bool ok = tid == 0 ? mbar_wait(&bar, phase, err) : true;   // one thread polls
        phase ^= 1u;
        alive = __syncthreads_and(ok) != 0;
        fence_after();
        if (alive) {
            const int q = warp & 3, b = warp >> 2, m = 32 * q + lane;
            const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16);
            float v0[16], v1[16];
            tmem_ld16(trow + 32 * b, v0);
            tmem_ld16(trow + 32 * b + 16, v1);
            if (b < nb && m < M) {
                float v[32];
#pragma unroll
                for (int x = 0; x < 16; ++x) {
                    v[x] = v0[x];
                    v[16 + x] = v1[x];
                }
                const long bin = bin0 + b;
                const bool zero = rA[b] == 0.0f;
                c32 *Wr = W ? W + (bin * M + m) * K : nullptr;
                T16 *W16r = W16 + (bin * M + m) * K;
                if (vec) {
                    uint32_t w16[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const c32 w = zero ? make_float2(0.f, 0.f) : make_float2(v[2 * u], v[2 * u + 1]);
                        const T16 q16 = Operand<T16>::from(w);
                        w16[u] = *reinterpret_cast<const uint32_t *>(&q16);
                        if (zero) v[2 * u] = v[2 * u + 1] = 0.f;
                    }
                    if (Wr) {
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            st_global_v8(Wr + 4 * u, v[8 * u], v[8 * u + 1], v[8 * u + 2], v[8 * u + 3], v[8 * u + 4],
                                         v[8 * u + 5], v[8 * u + 6], v[8 * u + 7]);
                    }
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        uint32_t w8[8];
#pragma unroll
                        for (int x = 0; x < 8; ++x) w8[x] = w16[8 * u + x];
                        st_global_v8(W16r + 8 * u, w8);
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        if (u >= K) break;
                        const c32 w = zero ? make_float2(0.f, 0.f) : make_float2(v[2 * u], v[2 * u + 1]);
                        if (Wr) Wr[u] = w;
                        W16r[u] = Operand<T16>::from(w);
                    }
                }
            }
        }
        fence_before();
        __syncthreads();
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (!alive && tid == 0) mbar_wait(&bar, phase ^ 1u, err);
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        tmem_dealloc(tmem, 128);
    }
}

static int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

template <typename T16>
static cudaError_t launch(const Geo &g, long nbins, const c32 *H, const c32 *Zs, const float *alpha, c32 *W, T16 *W16,
                          int *err, cudaStream_t st) {
    const long items = (nbins + NBI - 1) / NBI;
    if (items == 0) return cudaSuccess;
    // whole-sector stores need K = 16 and 32-byte aligned rows; W is the caller's array
    const int vec = g.K == 16 && !((reinterpret_cast<uintptr_t>(W) | reinterpret_cast<uintptr_t>(W16)) & 31);
    // H rows of 16 bytes when H and every subcarrier's block are 16-byte aligned
    const int h16 = !(reinterpret_cast<uintptr_t>(H) & 15) && !((g.K * g.M) & 1);
    cudaError_t e = cudaFuncSetAttribute(apply_kernel<T16>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e != cudaSuccess) return e;
    long blocks = sm_count();   // one CTA per SM
    if (blocks > items) blocks = items;
    apply_kernel<T16><<<(unsigned)blocks, PT, SMEM, st>>>(g, nbins, H, Zs, alpha, W, W16, vec, h16, err);
    return cudaGetLastError();
}

}  // namespace tczf

cudaError_t zf_apply_tc(const Geo &g, long nbins, const c32 *H, const c32 *Zs, const float *alpha, c32 *W, void *W16,
                        int kind, int *err, cudaStream_t st) {
    if (!tc_apply_supported(g) || !W16) return cudaErrorInvalidValue;
    if (kind == OUT_F16) return tczf::launch(g, nbins, H, Zs, alpha, W, (cf16 *)W16, err, st);
    return tczf::launch(g, nbins, H, Zs, alpha, W, (cbf16 *)W16, err, st);
}

}  // namespace fdk
