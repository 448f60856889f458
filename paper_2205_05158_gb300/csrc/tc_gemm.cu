// 5th-generation tensor-core GEMM for sm_103a: C[m][n] = sum_k A[m][k] B[n][k]
// with 16-bit A, B (both K-major, row-major in global memory) and FP32 accumulation
// in tensor memory.  Used for the FD-CNN dense layer (forward, data gradient and
// weight gradient) in 16-bit plans.
//
// A persistent CTA per SM walks 128 x BN output tiles (optionally K slices of them,
// split-K), n fastest:
//   warp 0 lane 0 : TMA producer, 128-byte-swizzled 128 x 64 / BN x 64 tiles into a
//                   STAGES-deep shared-memory ring (mbarrier full / empty pairs) that
//                   runs on across tiles;
//   warp 1 lane 0 : issues tcgen05.mma (M = 128, N = BN, K = 16) into one of two TMEM
//                   accumulators of BN columns (tile j uses buffer j & 1), commits each
//                   stage back to its producer barrier and the tile to tfull;
//   warps 2..9    : epilogue of tile j while tile j + 1 accumulates: two warps per TMEM
//                   lane quarter (warp w reads lanes 32 (w % 4) .. + 31), each taking half
//                   of the tile's columns -- tcgen05.ld, a caller-supplied functor, then
//                   tempty.  Each lane owns one output row, so the operands the functor
//                   reads are strided by rows; two warps per quarter halve each tile's
//                   serial chain of prefetch latencies and double the loads in flight.
// Every mbarrier wait is bounded (about 2 s of %globaltimer); a timeout sets the
// error word, the waiting role stops, the MMA warp still drains its commits, and
// TMEM is freed before the CTA exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_gemm.h"
#include "tc_ptx.cuh"

namespace fdk {
namespace tc {

constexpr int BM = 128, BK = 64, STAGES = 4, EPI_WARPS = 8, THREADS = 64 + 32 * EPI_WARPS;

template <int BN>
struct Smem {
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int BYTES = STAGES * STAGE + 1024;   // + alignment slack
    static constexpr int TMEM_COLS = BN < 32 ? 32 : BN;   // per accumulator buffer (two are allocated)
};

template <int BN, class Epi>
__global__ void __launch_bounds__(THREADS, 1) gemm_kernel(const __grid_constant__ CUtensorMap ta,
                                                          const __grid_constant__ CUtensorMap tb, int Mdim, int Ndim,
                                                          int Kdim, int k_per_split, int ntn, int ntiles, int ab_type,
                                                          Epi epi, int *err) {
    using L = Smem<BN>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], tfull[2], tempty[2];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntm = (Mdim + BM - 1) / BM;
    // tile t of this CTA: n fastest, so neighbouring CTAs share the A rows in L2
    auto tile_of = [&](int t, int &m0, int &n0, int &kbeg, int &nkb) {
        const int tn = t % ntn, tm = (t / ntn) % ntm, ks = t / (ntn * ntm);
        m0 = tm * BM;
        n0 = tn * BN;
        kbeg = ks * k_per_split;
        const int kend = min(Kdim, kbeg + k_per_split);
        nkb = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 32 * EPI_WARPS);   // every epilogue thread
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(2 * L::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // producer: one ring of STAGES stages across all of this CTA's tiles
            int g = 0;   // k-blocks issued so far
            for (int t = blockIdx.x; t < ntiles && !abort_flag; t += gridDim.x) {
                int m0, n0, kbeg, nkb;
                tile_of(t, m0, n0, kbeg, nkb);
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int s = g % STAGES;
                    const uint32_t use = g / STAGES;
                    if (g >= STAGES && !mbar_wait(&empty[s], (use & 1) ^ 1, err)) {
                        abort_flag = 1;
                        break;
                    }
                    uint8_t *sa = base + s * L::STAGE;
                    uint8_t *sb = sa + L::A_BYTES;
                    mbar_expect_tx(&full[s], L::STAGE);
                    const int kx = kbeg + kb * BK;
                    tma_load_2d(sa, &ta, &full[s], kx, m0);
                    tma_load_2d(sb, &tb, &full[s], kx, n0);
                }
            }
            // no copy may still be landing in shared memory when the CTA exits
            for (int s = 0; s < STAGES && s < g; ++s) {
                const int last = s + ((g - 1 - s) / STAGES) * STAGES;
                mbar_wait(&full[s], (uint32_t)(last / STAGES) & 1, err);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA: tile j of this CTA accumulates into TMEM buffer j & 1
            const uint32_t idesc = instr_desc(ab_type, BM, BN);
            int g = 0, j = 0;
            for (int t = blockIdx.x; t < ntiles && !abort_flag; t += gridDim.x, ++j) {
                int m0, n0, kbeg, nkb;
                tile_of(t, m0, n0, kbeg, nkb);
                const int buf = j & 1;
                if (j >= 2 && !mbar_wait(&tempty[buf], (uint32_t)((j >> 1) - 1) & 1, err)) {
                    abort_flag = 1;
                    break;
                }
                fence_after();
                const uint32_t d = tmem + (uint32_t)(buf * L::TMEM_COLS);
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int s = g % STAGES;
                    const uint32_t use = g / STAGES;
                    if (!mbar_wait(&full[s], use & 1, err)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint64_t ad = smem_desc(base + s * L::STAGE);
                    const uint64_t bd = smem_desc(base + s * L::STAGE + L::A_BYTES);
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k) mma_f16(d, ad + 2 * k, bd + 2 * k, idesc, (kb | k) ? 1u : 0u);
                    mma_commit(&empty[s]);
                }
                mma_commit(&tfull[buf]);   // arrives once this tile's MMAs have completed
                if (!ok) {
                    abort_flag = 1;
                    break;
                }
            }
        }
    } else {
        // epilogue: tile j from TMEM buffer j & 1; the operands the functor reads besides
        // the accumulator (residual, activation) are fetched PRE chunks ahead, the first
        // ones while the tile's MMAs run
        constexpr int PRE = 4, NCH = BN / 16;
        constexpr int NH = NCH >= 2 ? 2 : 1, HCH = NCH / NH;   // column halves per tile, chunks per half
        const int q = warp & 3, half = NH > 1 ? (warp - 2) / 4 : 0;
        const bool idle = warp - 2 >= 4 * NH;                    // one warp per quarter when BN = 16
        int j = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
            int m0, n0, kbeg, nkb;
            tile_of(t, m0, n0, kbeg, nkb);
            const int buf = j & 1;
            const int row = m0 + 32 * q + lane;
            const bool rok = row < Mdim;
            const int nh = n0 + 16 * HCH * half;   // first column of this warp's half
            typename Epi::Pre pre[PRE];
#pragma unroll
            for (int c = 0; c < PRE; ++c)
                if (!idle && c < HCH && rok && nh + 16 * c + 16 <= Ndim) epi.prefetch(row, nh + 16 * c, pre[c]);
            if (!mbar_wait(&tfull[buf], (uint32_t)(j >> 1) & 1, err)) break;
            fence_after();
            const bool ok = nkb > 0 && !abort_flag && !idle;
            const uint32_t trow =
                tmem + (uint32_t)(buf * L::TMEM_COLS + 16 * HCH * half) + ((uint32_t)(32 * q) << 16);
#pragma unroll
            for (int c = 0; c < HCH; ++c) {
                float v[16];
                tmem_ld16(trow + (uint32_t)(16 * c), v);
                const int n = nh + 16 * c;
                if (ok && rok && n < Ndim) {
                    if (n + 16 <= Ndim) {
                        epi.chunk(row, n, v, pre[c % PRE]);   // 16 contiguous columns of the row
                    } else {
#pragma unroll
                        for (int jj = 0; jj < 16; ++jj)
                            if (n + jj < Ndim) epi(row, n + jj, v[jj]);
                    }
                }
                if (!idle && c + PRE < HCH && rok && n + 16 * PRE + 16 <= Ndim)
                    epi.prefetch(row, n + 16 * PRE, pre[c % PRE]);
            }
            fence_before();
            mbar_arrive(&tempty[buf]);
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * L::TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D map over a [rows][ld] 16-bit array whose first `cols` entries of each row are valid;
// box = 64 x box_rows with 128-byte swizzle; out-of-range reads return zero.
static cudaError_t make_map(CUtensorMap *map, const void *ptr, long rows, long cols, long ld, int box_rows, int ab_type) {
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    if ((reinterpret_cast<uintptr_t>(ptr) & 15) || ((ld * 2) & 15)) return cudaErrorMisalignedAddress;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, ab_type ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                    const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BN, class Epi>
static cudaError_t launch(const GemmArgs &g, const Epi &epi, int *err, cudaStream_t st) {
    if (g.M <= 0 || g.N <= 0 || g.K <= 0) return cudaSuccess;
    CUtensorMap ta, tb;
    cudaError_t e = make_map(&ta, g.A, g.M, g.K, g.lda, BM, g.ab_type);
    if (e != cudaSuccess) return e;
    e = make_map(&tb, g.B, g.N, g.K, g.ldb, BN, g.ab_type);
    if (e != cudaSuccess) return e;
    int splits = g.splits < 1 ? 1 : g.splits;
    int kps = (g.K + splits - 1) / splits;
    kps = (kps + BK - 1) / BK * BK;
    splits = (g.K + kps - 1) / kps;          // every split gets at least one k-block
    const int smem = Smem<BN>::BYTES;
    e = cudaFuncSetAttribute(gemm_kernel<BN, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int ntn = (g.N + BN - 1) / BN, ntm = (g.M + BM - 1) / BM, ntiles = ntn * ntm * splits;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = ntiles < sms ? ntiles : sms;   // persistent: one CTA per SM
    gemm_kernel<BN, Epi><<<grid, THREADS, smem, st>>>(ta, tb, g.M, g.N, g.K, kps, ntn, ntiles, g.ab_type, epi, err);
    return cudaGetLastError();
}

// --- epilogues --------------------------------------------------------------
// operator()(m, n, v): one element; chunk(m, n, v[16], pre): columns n .. n + 15 of row m,
// n a multiple of 16 -- whole 32-byte sectors where the row layout allows (vec) -- with
// what prefetch(m, n, pre) loaded for those columns beforehand
struct NoPre {};
struct EpiStore {          // C[m][n] = acc (plain GEMM, ldc)
    using Pre = NoPre;
    float *C;
    long ldc;
    FD_D void operator()(int m, int n, float v) const { C[(long)m * ldc + n] = v; }
    FD_D void prefetch(int, int, Pre &) const {}
    FD_D void chunk(int m, int n, const float (&v)[16], const Pre &) const {
#pragma unroll
        for (int j = 0; j < 16; ++j) (*this)(m, n + j, v[j]);
    }
};
struct EpiAdd {            // C[m][n] += acc (split-K partial sums)
    using Pre = NoPre;
    float *C;
    long ldc;
    FD_D void operator()(int m, int n, float v) const { atomicAdd(C + (long)m * ldc + n, v); }
    FD_D void prefetch(int, int, Pre &) const {}
    FD_D void chunk(int m, int n, const float (&v)[16], const Pre &) const {
#pragma unroll
        for (int j = 0; j < 16; ++j) (*this)(m, n + j, v[j]);
    }
};
struct EpiFcFwd {          // s_tilde (interleaved floats) = acc + fc_b[pi(n)] + residual * s
    struct Pre {
        float4 r[4];
    };
    float *st;
    const float *s, *fbi;   // fbi: the bias in output order
    int Nd, residual, vec;  // vec: st and s rows 32-byte aligned, fbi 16-byte aligned
    int row_mul, row_add;   // output row m is chain column m row_mul + row_add
    FD_D long col(int m) const { return (long)m * row_mul + row_add; }
    FD_D void operator()(int m, int n, float v) const {
        const long idx = col(m) * 2 * Nd + n;
        st[idx] = v + fbi[n] + (residual ? s[idx] : 0.f);
    }
    FD_D void prefetch(int m, int n, Pre &p) const {
        if (!vec) return;
        if (residual) {
            const float4 *s4 = reinterpret_cast<const float4 *>(s + col(m) * 2 * Nd + n);
#pragma unroll
            for (int h = 0; h < 4; ++h) p.r[h] = s4[h];
        }
    }
    FD_D void chunk(int m, int n, const float (&v)[16], const Pre &p) const {
        if (!vec) {
#pragma unroll
            for (int j = 0; j < 16; ++j) (*this)(m, n + j, v[j]);
            return;
        }
        const long idx = col(m) * 2 * Nd + n;
        float o[16];
        const float4 *b4 = reinterpret_cast<const float4 *>(fbi + n);   // the same for every row
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const float4 b = b4[h];
            o[4 * h] = v[4 * h] + b.x;
            o[4 * h + 1] = v[4 * h + 1] + b.y;
            o[4 * h + 2] = v[4 * h + 2] + b.z;
            o[4 * h + 3] = v[4 * h + 3] + b.w;
        }
        if (residual) {
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                o[4 * h] += p.r[h].x;
                o[4 * h + 1] += p.r[h].y;
                o[4 * h + 2] += p.r[h].z;
                o[4 * h + 3] += p.r[h].w;
            }
        }
        st_global_v8(st + idx, o[0], o[1], o[2], o[3], o[4], o[5], o[6], o[7]);
        st_global_v8(st + idx + 8, o[8], o[9], o[10], o[11], o[12], o[13], o[14], o[15]);
    }
};
struct EpiFcBwdData {      // gpre[m][f] = acc where act > 0
    struct Pre {
        uint4 a[2];
    };
    float *gpre;
    const __nv_bfloat16 *act;
    long ld_g, ld_act;
    int vec;                // vec: gpre rows 32-byte and act rows 16-byte aligned
    FD_D void operator()(int m, int n, float v) const {
        gpre[(long)m * ld_g + n] = __bfloat162float(act[(long)m * ld_act + n]) > 0.f ? v : 0.f;
    }
    FD_D void prefetch(int m, int n, Pre &p) const {
        if (vec) {
            const uint4 *a4 = reinterpret_cast<const uint4 *>(act + (long)m * ld_act + n);
            p.a[0] = a4[0];
            p.a[1] = a4[1];
        }
    }
    FD_D void chunk(int m, int n, const float (&v)[16], const Pre &p) const {
        if (!vec) {
#pragma unroll
            for (int j = 0; j < 16; ++j) (*this)(m, n + j, v[j]);
            return;
        }
        float o[16];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t w[4] = {p.a[h].x, p.a[h].y, p.a[h].z, p.a[h].w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const __nv_bfloat162 b2 = *reinterpret_cast<const __nv_bfloat162 *>(&w[k]);
                const float2 f2 = __bfloat1622float2(b2);
                o[8 * h + 2 * k] = f2.x > 0.f ? v[8 * h + 2 * k] : 0.f;
                o[8 * h + 2 * k + 1] = f2.y > 0.f ? v[8 * h + 2 * k + 1] : 0.f;
            }
        }
        float *g = gpre + (long)m * ld_g + n;
        st_global_v8(g, o[0], o[1], o[2], o[3], o[4], o[5], o[6], o[7]);
        st_global_v8(g + 8, o[8], o[9], o[10], o[11], o[12], o[13], o[14], o[15]);
    }
};
struct EpiFcBwdWeight {    // grad fc_w[pi(n')][f] += acc (split-K partial sums)
    using Pre = NoPre;
    float *gfw;
    int Nd, F;
    FD_D void operator()(int m, int n, float v) const {
        atomicAdd(gfw + (long)((m & 1) * Nd + (m >> 1)) * F + n, v);
    }
    FD_D void prefetch(int, int, Pre &) const {}
    FD_D void chunk(int m, int n, const float (&v)[16], const Pre &) const {
#pragma unroll
        for (int j = 0; j < 16; ++j) (*this)(m, n + j, v[j]);
    }
};

}  // namespace tc

cudaError_t tc_gemm_store(const GemmArgs &g, float *C, long ldc, int *err, cudaStream_t st) {
    if (g.splits > 1) return tc::launch<256>(g, tc::EpiAdd{C, ldc}, err, st);
    return tc::launch<256>(g, tc::EpiStore{C, ldc}, err, st);
}

static bool al(const void *p, int b) { return !(reinterpret_cast<uintptr_t>(p) & (uintptr_t)(b - 1)); }

cudaError_t tc_fc_forward(const GemmArgs &g, float *st_out, const float *s, const float *fbi, int Nd, int residual,
                          int *err, cudaStream_t st, int row_mul, int row_add) {
    // rows of 2 N_d floats: whole sectors when that is a multiple of 8 and both bases align
    const int vec = (2 * Nd) % 8 == 0 && al(st_out, 32) && (!residual || al(s, 16)) && al(fbi, 16);
    return tc::launch<256>(g, tc::EpiFcFwd{st_out, s, fbi, Nd, residual, vec, row_mul, row_add}, err, st);
}

cudaError_t tc_fc_backward_data(const GemmArgs &g, float *gpre, long ld_g, const __nv_bfloat16 *act, long ld_act,
                                int *err, cudaStream_t st) {
    const int vec = ld_g % 8 == 0 && ld_act % 8 == 0 && al(gpre, 32) && al(act, 16);
    return tc::launch<256>(g, tc::EpiFcBwdData{gpre, act, ld_g, ld_act, vec}, err, st);
}

cudaError_t tc_fc_backward_weight(const GemmArgs &g, float *gfw, int Nd, int F, int *err, cudaStream_t st) {
    return tc::launch<256>(g, tc::EpiFcBwdWeight{gfw, Nd, F}, err, st);
}

}  // namespace fdk
