// Per-subcarrier contractions of the downlink on the 5th-generation tensor cores, for
// plans that keep H and W as 16-bit copies (BF16 or FP16 operands, FP32 accumulation in
// tensor memory).  Same operations as the CUDA-core kernels of bingemm.cuh:
//   expand (users -> antennas)   PRECODE      x = alpha_i W_i s~           (Eq. 1)
//                                ADJ_COMBINE  g_x = H_i^H g_y / alpha_i
//                                ADJ_COMBINE_F  the same from the H^H copy (precoder kept
//                                             as its factors): PRECODE's form over 1 / alpha
//   reduce (antennas -> users)   COMBINE      y = H_i x / alpha_i and the loss terms (Eq. 5)
//                                ADJ_PRECODE  g_s = alpha_i W_i^H g_x
//                                ADJ_PRECODE_F  alpha_i H_i g_x (W^H = Z H with the ZF factor's
//                                             Z applied afterwards: COMBINE's form, times alpha)
// i runs over data subcarriers; every realisation's symbols share its H_i and W_i.
//
// Complex products as real MMAs.  An A row holds complex entries a_j as interleaved
// (re, im) pairs along k = 2j + c, which is how the 16-bit copies store them, so A needs
// no arithmetic.  The B operand gets two real rows per symbol t, built from the FP32
// activations b_j(t):
//   plain      sum_j a_j b_j        row 2t = (br, -bi), row 2t+1 = (bi,  br)
//   conjugate  sum_j conj(a_j) b_j  row 2t = (br,  bi), row 2t+1 = (bi, -br)
// so that D[row][2t] and D[row][2t+1] are the real and imaginary parts of the result (in
// the reduce, where the activations are the A operand, D[2t][row] and D[2t+1][row]).
// Symbols go 16 at a time: N = 32 real columns per MMA.
//
// expand: an item is 8 consecutive subcarriers of one realisation.  A_i = [m][(u, c)]
//   (antenna rows, 16 user slots = 32 k), two subcarriers side by side in each 128-byte
//   row of a swizzled tile; MMA i (M = 128, N = 32, K = 2 x 16) accumulates into TMEM
//   columns 32 i .. 32 i + 31, and the epilogue reads antenna m from lane m.  (Generic
//   form: 4 subcarriers of 32 user slots each, one per tile row, with K > 16; the
//   antennas in items of 128.)
// reduce: an item is 4 subcarriers, computed transposed (y^T = x^T H^T): A holds the real
//   form of all 4 subcarriers' activations (rows (b, t, c'), 128), B their 4 x 16 user
//   rows of H (or W^H), so one MMA (M = 128, N = 64) per K step covers the item and the
//   diagonal blocks b = b' of its result are kept.  The discarded blocks cost tensor-core
//   time, which this HBM-bound contraction has to spare.
//
// The threads write every operand tile (the 16-bit conversion and the real-form signs
// are needed anyway) in the K-major, 128-byte-swizzled layout, make the writes visible
// to the tensor core with fence.proxy.async, and one thread issues tcgen05.mma and
// tcgen05.commit onto an mbarrier; every wait on it is bounded (about 2 s), after which
// the error word is set, the CTA stops, and its tensor memory is freed.  Two CTAs share
// an SM, so one builds operands while the other's MMAs and epilogue run.
#include <type_traits>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace fdk {
namespace tcb {
using namespace tc;

constexpr int THREADS = 256;
constexpr int TS = 16;            // symbols per MMA
constexpr int EXB = 8, RDB = 4;   // subcarriers per item: expand, reduce

// expand: A [4 pair tiles][128 rows][128 B], B [4 pair tiles][32 rows][128 B]
constexpr int EX_A = 4 * 128 * 128, EX_B = 4 * 32 * 128;
constexpr int EX_SMEM = EX_A + EX_B + 1024;
// reduce: A (activations) [4 k-blocks][128 rows][128 B], B (H or W^H) [4 k-blocks][64
// rows][128 B], then the staging of the results [16 t][16 u][4 subcarriers]
// result staging: symbol rows of 16 users x 4 subcarriers x (re, im) floats, padded to
// 130 floats so the 16 symbols of a warp's write land in different banks
constexpr int RD_YT = 16 * RDB * 2 + 2;
constexpr int RD_A = 4 * 128 * 128, RD_B = 4 * 64 * 128, RD_Y = TS * RD_YT * 4;
constexpr int RD_SMEM = RD_A + RD_B + RD_Y + 1024;

template <typename T16> struct Pk;
template <> struct Pk<cbf16> {
    static constexpr int type = 1;
    FD_D static uint32_t two(float lo, float hi) {
        __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<uint32_t *>(&v);
    }
};
template <> struct Pk<cf16> {
    static constexpr int type = 0;
    FD_D static uint32_t two(float lo, float hi) {
        __half2 v = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<uint32_t *>(&v);
    }
};

template <typename T16, bool CONJ> FD_D void real_rows(float br, float bi, uint32_t &w0, uint32_t &w1) {
    if (CONJ) {
        w0 = Pk<T16>::two(br, bi);
        w1 = Pk<T16>::two(bi, -br);
    } else {
        w0 = Pk<T16>::two(br, -bi);
        w1 = Pk<T16>::two(bi, br);
    }
}

// the same rows from a BF16 (re, im) pair already packed as stored (low half = re): the
// sign flips and the swap are bit operations
template <bool CONJ> FD_D void real_rows_packed(uint32_t w, uint32_t &w0, uint32_t &w1) {
    const uint32_t sw = __byte_perm(w, 0u, 0x1032u);   // (im, re)
    if (CONJ) {
        w0 = w;
        w1 = sw ^ 0x80000000u;
    } else {
        w0 = w ^ 0x80000000u;
        w1 = sw;
    }
}
FD_D uint32_t pack_bf16(float re, float im) {
    __nv_bfloat162 v = __floats2bfloat162_rn(re, im);
    return *reinterpret_cast<uint32_t *>(&v);
}

FD_D void st32(uint8_t *p, uint32_t v) { *reinterpret_cast<uint32_t *>(p) = v; }
FD_D void st128(uint8_t *p, uint4 v) { *reinterpret_cast<uint4 *>(p) = v; }
FD_D uint8_t *align1024(uint8_t *p) {
    return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// Setup shared by both kernels: the mbarrier and `cols` columns of tensor memory.
FD_D uint32_t setup(uint64_t *bar, uint32_t *slot, uint32_t cols) {
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((threadIdx.x >> 5) == 0) tmem_alloc(slot, cols);
    fence_before();
    __syncthreads();
    fence_after();
    return *slot;
}

// Waits for the MMAs of this round (one thread polls, the CTA meets it at the barrier);
// false in every thread of the CTA if the wait timed out.
FD_D bool wait_mma(uint64_t *bar, uint32_t &phase, int *err) {
    const bool ok = threadIdx.x == 0 ? mbar_wait(bar, phase, err) : true;
    phase ^= 1u;
    const bool all = __syncthreads_and(ok) != 0;
    fence_after();
    return all;
}

FD_D void teardown(uint64_t *bar, uint32_t phase, bool alive, uint32_t tmem, uint32_t cols, int *err) {
    // after a timeout, give the outstanding commit one more bounded wait before the
    // tensor memory it targets is released
    if (!alive && threadIdx.x == 0) mbar_wait(bar, phase ^ 1u, err);
    fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        fence_after();
        tmem_dealloc(tmem, cols);
    }
}

// ---------------------------------------------------------------------------
// expand.  AT = false: A = W16 [bin][m][u] (rows m, PRECODE); AT = true: A = H16
// [bin][u][m] read transposed (ADJ_COMBINE).  out[t][m][i] = scale_i D / b_scale, stored
// as TO (c32, or cbf16 for the BF16 activation planes).
// Up to 256 antennas and 32 users: an item covers 128 antennas (M > 128: two items per
// subcarrier group, antennas 128 h ..); with K > 16 a subcarrier's 32 user slots fill a
// whole 128-byte tile row (one subcarrier per tile, 4 per item, 4 MMA K steps) instead
// of two subcarriers side by side.
template <typename T16, bool CONJ, bool AT, typename TO>
__global__ void __launch_bounds__(THREADS, 2)
    expand_kernel(Geo g, int S, const uint32_t *__restrict__ A, const float *__restrict__ alpha,
                  const c32 *__restrict__ B, TO *__restrict__ out, int inv_alpha, float b_scale, int vec_ok,
                  int *err) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *sA = align1024(smem_raw);
    uint8_t *sB = sA + EX_A;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int M = g.M, K = g.K, Nd = g.N_d;
    const int spt = K > 16 ? 1 : 2;        // subcarriers per tile (per 128-byte row)
    const int exb = (4 * spt) >> (g.bin_half ? 1 : 0);   // subcarriers per item (half items: the
                                                         // rest of the tiles stay zero)
    const int MH = (M + 127) >> 7;         // 128-antenna parts, one item each
    const int ngroups = (Nd + exb - 1) / exb;
    const int R = (S + g.S_per_real - 1) / g.S_per_real;
    const long nitems = (long)R * ngroups * MH;
    const uint32_t tmem = setup(&bar, &tmem_slot, 256);
    const uint32_t idesc = instr_desc(Pk<T16>::type, 128, 32);
    const int nks = K > 16 ? 4 : K > 8 ? 2 : 1;
    uint32_t phase = 0;
    bool alive = true;

    for (long item = blockIdx.x; item < nitems && alive; item += gridDim.x) {
        const int m0 = 128 * (int)(item % MH);
        const long grp = item / MH;
        const int r = (int)(grp / ngroups), i0 = (int)(grp % ngroups) * exb;
        const long t0 = (long)r * g.S_per_real;
        const int nsym = (int)min((long)g.S_per_real, (long)S - t0);
        const long bin0 = (long)r * Nd + i0;
        const int nb = min(exb, Nd - i0);
        // the subcarrier scales, loaded before they are needed
        float sc[EXB];
#pragma unroll
        for (int j = 0; j < EXB; ++j) {
            const float al = j < nb ? alpha[bin0 + j] : 0.f;
            sc[j] = (inv_alpha ? 1.0f / al : al) / b_scale;
        }

        // A: chunk (tile p, row m, 16-byte chunk ch) = users u0 .. u0 + 3 of subcarrier b at
        // antenna m0 + m -- b = 2p + (ch >> 2), u0 = 4 (ch & 3) with two subcarriers a tile,
        // b = p, u0 = 4 ch with one -- copied with cp.async (zero outside)
        if (!AT) {
            if (!(K & 3)) {   // whole 16-byte runs of 4 users
                for (int c = tid; c < 4 * 128 * 8; c += THREADS) {
                    const int ch = c & 7, m = (c >> 3) & 127, p = c >> 10;
                    const int b = spt == 2 ? 2 * p + (ch >> 2) : p, u0 = spt == 2 ? 4 * (ch & 3) : 4 * ch;
                    const bool ok = b < nb && m0 + m < M && u0 < K;
                    const uint32_t *src = ok ? A + ((bin0 + b) * M + m0 + m) * K + u0 : A;
                    cp_async16(sA + p * 16384 + sw128_offset(m, ch * 8), src, ok);
                }
            } else {
                for (int c = tid; c < 4 * 128 * 8; c += THREADS) {
                    const int ch = c & 7, m = (c >> 3) & 127, p = c >> 10;
                    const int b = spt == 2 ? 2 * p + (ch >> 2) : p, u0 = spt == 2 ? 4 * (ch & 3) : 4 * ch;
                    uint8_t *dst = sA + p * 16384 + sw128_offset(m, ch * 8);
                    const bool ok = b < nb && m0 + m < M;
                    const uint32_t *src = ok ? A + ((bin0 + b) * M + m0 + m) * K : A;
#pragma unroll
                    for (int j = 0; j < 4; ++j) cp_async4(dst + 4 * j, ok && u0 + j < K ? src + u0 + j : A, ok && u0 + j < K);
                }
            }
        } else {
            // transposed: the four users of a chunk are M entries apart; lanes run along m
            for (int c = tid; c < 4 * 128 * 8; c += THREADS) {
                const int m = c & 127, ch = (c >> 7) & 7, p = c >> 10;
                const int b = spt == 2 ? 2 * p + (ch >> 2) : p, u0 = spt == 2 ? 4 * (ch & 3) : 4 * ch;
                uint8_t *dst = sA + p * 16384 + sw128_offset(m, ch * 8);
                const bool ok = b < nb && m0 + m < M;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const bool okj = ok && u0 + j < K;
                    cp_async4(dst + 4 * j, okj ? A + ((bin0 + b) * K + u0 + j) * M + m0 + m : A, okj);
                }
            }
        }

        for (int s0 = 0; s0 < nsym && alive; s0 += TS) {
            const int ns = min(TS, nsym - s0);
            // B: element (t, u, subcarrier b), b fastest (16 user slots x 8 subcarriers, or
            // 32 x 4); rows 2t and 2t + 1 of tile b / spt, k = 32 (b % spt) + 2u
            for (int e0 = tid; e0 < TS * 16 * EXB; e0 += 8 * THREADS) {
                c32 v[8];
#pragma unroll
                for (int h = 0; h < 8; ++h) {
                    const int e = e0 + h * THREADS, t = e >> 7;
                    const int b = spt == 2 ? e & 7 : e & 3, u = spt == 2 ? (e >> 3) & 15 : (e >> 2) & 31;
                    v[h] = (t < ns && u < K && b < nb) ? B[((t0 + s0 + t) * K + u) * Nd + i0 + b]
                                                       : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int h = 0; h < 8; ++h) {
                    const int e = e0 + h * THREADS, t = e >> 7;
                    const int b = spt == 2 ? e & 7 : e & 3, u = spt == 2 ? (e >> 3) & 15 : (e >> 2) & 31;
                    uint32_t w0, w1;
                    real_rows<T16, CONJ>(v[h].x * b_scale, v[h].y * b_scale, w0, w1);
                    uint8_t *tile = sB + (spt == 2 ? b >> 1 : b) * 4096;
                    const int k = (spt == 2 ? 32 * (b & 1) : 0) + 2 * u;
                    st32(tile + sw128_offset(2 * t, k), w0);
                    st32(tile + sw128_offset(2 * t + 1, k), w1);
                }
            }
            cp_async_wait_all();
            fence_proxy_async();
            __syncthreads();
            if (tid == 0) {
                fence_after();
                for (int b = 0; b < nb; ++b)
                    for (int ks = 0; ks < nks; ++ks) {
                        const int p = spt == 2 ? b >> 1 : b;
                        const uint32_t off = (spt == 2 ? (b & 1) * 64 : 0) + ks * 32;
                        mma_f16(tmem + 32 * b, smem_desc(sA + p * 16384 + off), smem_desc(sB + p * 4096 + off),
                                idesc, ks ? 1u : 0u);
                    }
                mma_commit(&bar);
            }
            alive = wait_mma(&bar, phase, err);
            if (alive) {
                const int q = warp & 3, m = m0 + 32 * q + lane;
                const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16);
                if constexpr (std::is_same<TO, c32>::value) {
                    // warp w: antennas 32 (w & 3) .., subcarriers 4 (w >> 2) .. + 3: one
                    // 32-byte sector of out[t][m][i0 + 4 (w >> 2) ..] per symbol
                    const int hb = 4 * (warp >> 2);
                    const bool vec = vec_ok && hb + 4 <= nb;
                    float sch[4];   // this warp's 4 scales, without indexing sc at run time
#pragma unroll
                    for (int j = 0; j < 4; ++j) sch[j] = hb ? sc[4 + j] : sc[j];
                    for (int tb = 0; 4 * tb < ns; ++tb) {
                        float v[4][8];
#pragma unroll
                        for (int j = 0; j < 4; ++j) tmem_ld8(trow + 32 * (hb + j) + 8 * tb, v[j]);
                        if (m < M) {
#pragma unroll
                            for (int tt = 0; tt < 4; ++tt) {
                                const int t = 4 * tb + tt;
                                if (t >= ns) break;
                                c32 *dst = out + ((t0 + s0 + t) * M + m) * Nd + i0 + hb;
                                if (vec) {
                                    st_global_v8(dst, v[0][2 * tt] * sch[0], v[0][2 * tt + 1] * sch[0],
                                                 v[1][2 * tt] * sch[1], v[1][2 * tt + 1] * sch[1], v[2][2 * tt] * sch[2],
                                                 v[2][2 * tt + 1] * sch[2], v[3][2 * tt] * sch[3],
                                                 v[3][2 * tt + 1] * sch[3]);
                                } else {
#pragma unroll
                                    for (int j = 0; j < 4; ++j)
                                        if (hb + j < nb)
                                            dst[j] = make_float2(v[j][2 * tt] * sch[j], v[j][2 * tt + 1] * sch[j]);
                                }
                            }
                        }
                    }
                } else {
                    // BF16 planes: warp w: antennas 32 (w & 3) .., symbol blocks tb with
                    // tb % 2 = w >> 2, all 8 subcarriers = one 32-byte sector per symbol
                    const bool vec = vec_ok && nb == EXB;
                    for (int tb = warp >> 2; 4 * tb < ns; tb += 2) {
                        uint32_t w[4][EXB];
#pragma unroll
                        for (int b = 0; b < EXB; ++b) {
                            float v[8];
                            tmem_ld8(trow + 32 * b + 8 * tb, v);
#pragma unroll
                            for (int tt = 0; tt < 4; ++tt) w[tt][b] = pack_bf16(v[2 * tt] * sc[b], v[2 * tt + 1] * sc[b]);
                        }
                        if (m < M) {
#pragma unroll
                            for (int tt = 0; tt < 4; ++tt) {
                                const int t = 4 * tb + tt;
                                if (t >= ns) break;
                                uint32_t *dst = reinterpret_cast<uint32_t *>(out + ((t0 + s0 + t) * M + m) * Nd + i0);
                                if (vec) {
                                    st_global_v8(dst, w[tt]);
                                } else {
#pragma unroll
                                    for (int b = 0; b < EXB; ++b)
                                        if (b < nb) dst[b] = w[tt][b];
                                }
                            }
                        }
                    }
                }
            }
            fence_before();
            __syncthreads();
        }
    }
    teardown(&bar, phase, alive, tmem, 256, err);
}

// ---------------------------------------------------------------------------
// reduce, transposed: y_i^T[t][u] = sum_m x_i^T[t][m] H_i^T[m][u].  A = the real form of
// the activations of 4 subcarriers, rows (b, t, c') = 32 b + 2 t + c' over k = (m, c);
// B = the 16 user rows of all 4 subcarriers, (b', u) = 16 b' + u over k = (m, c), as the
// 16-bit copies store them (AT = false: H16 [bin][u][m], COMBINE) or read transposed
// (AT = true: W16 [bin][m][u], ADJ_PRECODE).  One MMA per K step (M = 128, N = 64) gives
// every cross product of the 4 subcarriers; the diagonal blocks b = b' are kept: warp b
// reads TMEM lanes 32 b .. (its subcarrier's symbols) at columns 16 b .. 16 b + 15.
// FULL: M = 128 antennas and K = 16 users as compile-time constants, so the index
// arithmetic of the tile builds and the epilogue is shifts and masks.
// Up to 256 antennas and 32 users: the antennas go in parts of 128 (A and B rebuilt per
// part, the MMAs accumulating in TMEM), the users in halves of 16 (TMEM columns 64 h ..,
// B rebuilt per half); then one epilogue pass per user half.
template <typename T16, bool CONJ, bool AT, bool COMB, typename TX, bool FULL>
__global__ void __launch_bounds__(THREADS, 2)
    reduce_kernel(Geo g, int S, const uint32_t *__restrict__ Wt, const float *__restrict__ alpha,
                  const TX *__restrict__ X, c32 *__restrict__ out, const c32 *__restrict__ s_ref,
                  c32 *__restrict__ gy, double *metrics, double inv_count, int inv_alpha, float b_scale, int vec_ok,
                  int *err) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *sA = align1024(smem_raw);          // activations [4 k-blocks][128 rows][128 B]
    uint8_t *sB = sA + RD_A;                    // H / W^H     [4 k-blocks][64 rows][128 B]
    float *sY = reinterpret_cast<float *>(sB + RD_B);   // [t][u][b][re, im], rows of RD_YT floats
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    __shared__ double red[32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int M = FULL ? 128 : g.M, K = FULL ? 16 : g.K, Nd = g.N_d;
    const int MH = FULL ? 1 : (M + 127) >> 7;   // 128-antenna parts
    const int UH = FULL ? 1 : (K + 15) >> 4;    // 16-user halves
    const bool one_b = MH == 1 && UH == 1;      // B loaded once per item
    const int rdb = g.bin_half ? RDB / 2 : RDB;   // subcarriers per item (half items: 2 of the 4 blocks)
    const int ngroups = (Nd + rdb - 1) / rdb;
    const int R = (S + g.S_per_real - 1) / g.S_per_real;
    const long nitems = (long)R * ngroups;
    const uint32_t tcols = UH > 1 ? 128 : 64;
    const uint32_t tmem = setup(&bar, &tmem_slot, tcols);
    const uint32_t idesc = instr_desc(Pk<T16>::type, 128, 64);
    const float gscale = (float)(2.0 * inv_count);
    uint32_t phase = 0;
    bool alive = true;
    float err_acc = 0.f, sig_acc = 0.f;

    for (long item = blockIdx.x; item < nitems && alive; item += gridDim.x) {
        const int r = (int)(item / ngroups), i0 = (int)(item % ngroups) * rdb;
        const long t0 = (long)r * g.S_per_real;
        const int nsym = (int)min((long)g.S_per_real, (long)S - t0);
        const long bin0 = (long)r * Nd + i0;
        const int nb = min(rdb, Nd - i0);
        // scale of the subcarrier whose TMEM lanes this warp reads, loaded early
        float sc = 0.f;
        if (warp < nb) {
            const float al = alpha[bin0 + warp];
            sc = (inv_alpha ? 1.0f / al : al) / b_scale;
        }

        // B rows 16 b + u' (user u = 16 uh + u' < K) of antenna part mh, k-block (m - 128 mh)
        // / 32, copied with cp.async; antennas past the part's last are zero
        auto load_b = [&](int mh, int uh) {
            const int Mp = min(128, M - 128 * mh), Kh = min(16, K - 16 * uh), MC = ((Mp + 7) & ~7) / 4;
            const int ma = 128 * mh, ua = 16 * uh;
            if (!AT) {
                const int n = RDB * Kh * MC;
                for (int c = tid; c < n; c += THREADS) {
                    const int mc = c % MC, bu = c / MC, u = bu % Kh, b = bu / Kh;
                    uint8_t *dst = sB + (mc >> 3) * 8192 + sw128_offset(16 * b + u, (mc & 7) * 8);
                    const uint32_t *src = Wt + ((bin0 + (b < nb ? b : 0)) * K + ua + u) * M + ma + 4 * mc;
                    if (!(M & 3)) {
                        const bool ok = b < nb && 4 * mc < Mp;
                        cp_async16(dst, ok ? src : Wt, ok);
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const bool ok = b < nb && 4 * mc + j < Mp;
                            cp_async4(dst + 4 * j, ok ? src + j : Wt, ok);
                        }
                    }
                }
            } else {
                // transposed: a 16-byte run of W16 (4 users at antenna m) feeds 4 rows
                const int MPp = (Mp + 7) & ~7, UQ = (Kh + 3) / 4, n = RDB * MPp * UQ;
                for (int c = tid; c < n; c += THREADS) {
                    const int uq = c % UQ, bm = c / UQ, m = bm % MPp, b = bm / MPp;
                    const bool ok = b < nb && m < Mp;
                    const uint32_t *src = ok ? Wt + ((bin0 + b) * M + ma + m) * K + ua + 4 * uq : Wt;
                    uint8_t *dst = sB + (m >> 5) * 8192;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int u = 4 * uq + j;
                        if (u < Kh) cp_async4(dst + sw128_offset(16 * b + u, 2 * (m & 31)), ok ? src + j : Wt, ok);
                    }
                }
            }
        };
        if (one_b) load_b(0, 0);

        for (int s0 = 0; s0 < nsym && alive; s0 += TS) {
            const int ns = min(TS, nsym - s0);
            const bool vec = vec_ok && nb == RDB;
            // outputs (t, u, b) of user half 0, b fastest (4 subcarriers = 32 contiguous
            // bytes): at most 16 x 16 x 4 = 4 per thread; its reference symbols loaded ahead
            c32 sref[4];
            auto load_sref = [&](int uh) {
                const int Kh = min(16, K - 16 * uh), nout = ns * Kh * RDB;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int e = tid + k * THREADS;
                    const int b = e & (RDB - 1), tu = e / RDB, u = 16 * uh + tu % Kh, t = tu / Kh;
                    sref[k] = (COMB && e < nout && b < nb) ? s_ref[((t0 + s0 + t) * K + u) * Nd + i0 + b]
                                                           : make_float2(0.f, 0.f);
                }
            };
            load_sref(0);
            for (int mh = 0; mh < MH && alive; ++mh) {
                const int ma = 128 * mh, Mp = FULL ? 128 : min(128, M - ma);
                const int MP = FULL ? 128 : (Mp + 7) & ~7;   // antennas padded to one K step (8 complex)
                const int nks = MP / 8;
                // A: (t, m) pairs of antennas ma + m, m fastest, all 4 subcarriers (32
                // contiguous bytes of FP32, 16 of BF16) each; rows 32 b + 2t and 32 b + 2t + 1
                // of k-block m / 32
                if constexpr (std::is_same<TX, c32>::value) {
                    for (int e0 = tid; e0 < TS * MP; e0 += 4 * THREADS) {
                        c32 v[4][RDB];
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            const int e = e0 + h * THREADS, m = e % MP, t = e / MP;
                            const bool ok = e < TS * MP && t < ns && m < Mp;
                            const c32 *src = X + ((t0 + s0 + (ok ? t : 0)) * M + ma + (ok ? m : 0)) * Nd + i0;
                            if (ok && vec) {
                                const float4 lo = reinterpret_cast<const float4 *>(src)[0];
                                const float4 hi = reinterpret_cast<const float4 *>(src)[1];
                                v[h][0] = make_float2(lo.x, lo.y);
                                v[h][1] = make_float2(lo.z, lo.w);
                                v[h][2] = make_float2(hi.x, hi.y);
                                v[h][3] = make_float2(hi.z, hi.w);
                            } else {
#pragma unroll
                                for (int b = 0; b < RDB; ++b) v[h][b] = (ok && b < nb) ? src[b] : make_float2(0.f, 0.f);
                            }
                        }
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            const int e = e0 + h * THREADS, m = e % MP, t = e / MP;
                            if (e >= TS * MP) break;
                            uint8_t *tile = sA + (m >> 5) * 16384;
                            const int k = 2 * (m & 31);
#pragma unroll
                            for (int b = 0; b < RDB; ++b) {
                                uint32_t w0, w1;
                                real_rows<T16, CONJ>(v[h][b].x * b_scale, v[h][b].y * b_scale, w0, w1);
                                st32(tile + sw128_offset(32 * b + 2 * t, k), w0);
                                st32(tile + sw128_offset(32 * b + 2 * t + 1, k), w1);
                            }
                        }
                    }
                } else {
                    // BF16 planes (BF16 plans, b_scale 1): every load of the unit in flight at once;
                    // subcarriers past N_d in the last group are padding, read as zero
                    constexpr int PER = TS * 128 / THREADS;
                    const bool b1 = nb > 1, b2 = nb > 2, b3 = nb > 3;
                    uint32_t w[PER][RDB];
#pragma unroll
                    for (int h = 0; h < PER; ++h) {
                        const int e = tid + h * THREADS, m = e % MP, t = e / MP;
                        const bool ok = e < TS * MP && t < ns && m < Mp;
                        // the blocked plane: the 4 subcarriers of group i0 / 4 at (slot, antenna) are 16
                        // bytes; a half item starts at subcarrier i0 % 4 of them
                        const uint32_t *src = reinterpret_cast<const uint32_t *>(
                            X + BlkPlane(g).item(r, i0 / RDB) + ((long)(s0 + (ok ? t : 0)) * M + ma + (ok ? m : 0)) * RDB) +
                            (i0 & (RDB - 1));
                        if (ok && vec_ok && !(i0 & (RDB - 1))) {
                            const uint4 q4 = *reinterpret_cast<const uint4 *>(src);
                            w[h][0] = q4.x;
                            w[h][1] = b1 ? q4.y : 0u;
                            w[h][2] = b2 ? q4.z : 0u;
                            w[h][3] = b3 ? q4.w : 0u;
                        } else {
#pragma unroll
                            for (int b = 0; b < RDB; ++b) w[h][b] = (ok && b < nb) ? src[b] : 0u;
                        }
                    }
#pragma unroll
                    for (int h = 0; h < PER; ++h) {
                        const int e = tid + h * THREADS, m = e % MP, t = e / MP;
                        if (e >= TS * MP) break;
                        uint8_t *tile = sA + (m >> 5) * 16384;
                        const int k = 2 * (m & 31);
#pragma unroll
                        for (int b = 0; b < RDB; ++b) {
                            uint32_t w0, w1;
                            real_rows_packed<CONJ>(w[h][b], w0, w1);
                            st32(tile + sw128_offset(32 * b + 2 * t, k), w0);
                            st32(tile + sw128_offset(32 * b + 2 * t + 1, k), w1);
                        }
                    }
                }
                for (int uh = 0; uh < UH && alive; ++uh) {
                    if (!one_b) load_b(mh, uh);   // into the B tile the previous round's MMAs are done with
                    cp_async_wait_all();
                    fence_proxy_async();
                    __syncthreads();
                    if (tid == 0) {
                        fence_after();
                        for (int ks = 0; ks < nks; ++ks)
                            mma_f16(tmem + 64 * uh, smem_desc(sA + (ks >> 2) * 16384 + (ks & 3) * 32),
                                    smem_desc(sB + (ks >> 2) * 8192 + (ks & 3) * 32), idesc, (mh || ks) ? 1u : 0u);
                        mma_commit(&bar);
                    }
                    alive = wait_mma(&bar, phase, err);
                }
            }
            for (int uh = 0; uh < UH && alive; ++uh) {
                const int Kh = min(16, K - 16 * uh), nout = ns * Kh * RDB;
                if (uh) load_sref(uh);
                if (warp < RDB) {
                    // lane = (t, c') of subcarrier b = warp; columns 64 uh + 16 b + u'
                    const int b = warp, t = lane >> 1, c = lane & 1;
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + 64 * uh + 16 * b, v);
                    if (b < nb && t < ns) {
#pragma unroll
                        for (int u = 0; u < 16; ++u)
                            if (u < Kh) sY[t * RD_YT + (u * RDB + b) * 2 + c] = v[u] * sc;
                    }
                }
                __syncthreads();
                const c32 *sYc = reinterpret_cast<const c32 *>(sY);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int e = tid + k * THREADS;
                    const int b = e & (RDB - 1), tu = e / RDB, u = tu % Kh, t = tu / Kh;
                    if (e >= nout || b >= nb) continue;
                    const c32 v = sYc[(t * RD_YT + (u * RDB + b) * 2) / 2];
                    const long idx = ((t0 + s0 + t) * K + 16 * uh + u) * Nd + i0 + b;
                    if (COMB) {
                        const c32 sr = sref[k];
                        const c32 d = csub(v, sr);
                        err_acc += cabs2(d);
                        sig_acc += cabs2(sr);
                        if (out) out[idx] = v;
                        if (gy) gy[idx] = cscale(d, gscale);
                    } else {
                        out[idx] = v;
                    }
                }
                __syncthreads();   // sY is read before the next half writes it
            }
            fence_before();
            __syncthreads();
        }
    }
    teardown(&bar, phase, alive, tmem, tcols, err);
    if (COMB && metrics) {
        const double es = block_sum((double)err_acc, red);
        const double ss = block_sum((double)sig_acc, red);
        if (tid == 0) {
            atomicAdd(metrics + 1, es);
            atomicAdd(metrics + 2, ss);
        }
    }
}

// ---------------------------------------------------------------------------
// The expand for the benchmark shape -- BF16 plans, M = 128, K = 16, one 16-symbol block
// per realisation -- software-pipelined: as soon as an item's MMAs are complete, the next
// item's A tile (cp.async) and activations (registers) go in flight, during this item's
// store-heavy epilogue.
template <bool CONJ, bool AT, typename TO>
__global__ void __launch_bounds__(THREADS, 2)
    expand_pipe_kernel(Geo g, int S, const uint32_t *__restrict__ A, const float *__restrict__ alpha,
                       const c32 *__restrict__ B, TO *__restrict__ out, int inv_alpha, int vec_ok, int *err) {
    constexpr int M = 128, K = 16, PER = TS * 16 * EXB / THREADS;   // B elements per thread
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *sA = align1024(smem_raw);
    uint8_t *sB = sA + EX_A;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Nd = g.N_d;
    const int ngroups = (Nd + EXB - 1) / EXB;
    const int R = (S + g.S_per_real - 1) / g.S_per_real;
    const long nitems = (long)R * ngroups;
    const uint32_t tmem = setup(&bar, &tmem_slot, 256);
    const uint32_t idesc = instr_desc(1, 128, 32);
    uint32_t phase = 0;
    bool alive = true;

    struct It {
        long t0, bin0;
        int i0, ns, nb;
    };
    auto info = [&](long item) {
        It u;
        const int r = (int)(item / ngroups);
        u.i0 = (int)(item % ngroups) * EXB;
        u.t0 = (long)r * g.S_per_real;
        u.ns = (int)min((long)g.S_per_real, (long)S - u.t0);
        u.bin0 = (long)r * Nd + u.i0;
        u.nb = min(EXB, Nd - u.i0);
        return u;
    };
    c32 bv[PER];   // the activations of the item being prepared
    auto issue = [&](const It &u) {
        // A by cp.async: direct (W16 rows m) or transposed (H16, lanes along m)
        for (int c = tid; c < 4 * 128 * 8; c += THREADS) {
            if (!AT) {
                const int ch = c & 7, m = (c >> 3) & 127, b = 2 * (c >> 10) + (ch >> 2);
                const bool ok = b < u.nb;
                cp_async16(sA + (c >> 10) * 16384 + sw128_offset(m, ch * 8),
                           ok ? A + ((u.bin0 + b) * M + m) * K + 4 * (ch & 3) : A, ok);
            } else {
                const int m = c & 127, ch = (c >> 7) & 7, b = 2 * (c >> 10) + (ch >> 2);
                const int u0 = 4 * (ch & 3);
                uint8_t *dst = sA + (c >> 10) * 16384 + sw128_offset(m, ch * 8);
                const bool ok = b < u.nb;
#pragma unroll
                for (int j = 0; j < 4; ++j) cp_async4(dst + 4 * j, ok ? A + ((u.bin0 + b) * K + u0 + j) * M + m : A, ok);
            }
        }
#pragma unroll
        for (int h = 0; h < PER; ++h) {
            const int e = tid + h * THREADS, b = e & 7, uu = (e >> 3) & 15, t = e >> 7;
            bv[h] = (t < u.ns && b < u.nb) ? B[((u.t0 + t) * K + uu) * Nd + u.i0 + b] : make_float2(0.f, 0.f);
        }
    };
    if (blockIdx.x < nitems) issue(info(blockIdx.x));

    for (long item = blockIdx.x; item < nitems && alive; item += gridDim.x) {
        const It u = info(item);
        float sc[EXB];
#pragma unroll
        for (int j = 0; j < EXB; ++j) {
            const float al = j < u.nb ? alpha[u.bin0 + j] : 0.f;
            sc[j] = inv_alpha ? 1.0f / al : al;
        }
        // B: rows 2t and 2t + 1 of pair tile b >> 1 at k = 32 (b & 1) + 2u
#pragma unroll
        for (int h = 0; h < PER; ++h) {
            const int e = tid + h * THREADS, b = e & 7, uu = (e >> 3) & 15, t = e >> 7;
            uint32_t w0, w1;
            real_rows<cbf16, CONJ>(bv[h].x, bv[h].y, w0, w1);
            uint8_t *tile = sB + (b >> 1) * 4096;
            const int k = 32 * (b & 1) + 2 * uu;
            st32(tile + sw128_offset(2 * t, k), w0);
            st32(tile + sw128_offset(2 * t + 1, k), w1);
        }
        cp_async_wait_all();
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            fence_after();
            for (int b = 0; b < u.nb; ++b)
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    const uint32_t off = (b & 1) * 64 + ks * 32;
                    mma_f16(tmem + 32 * b, smem_desc(sA + (b >> 1) * 16384 + off),
                            smem_desc(sB + (b >> 1) * 4096 + off), idesc, ks ? 1u : 0u);
                }
            mma_commit(&bar);
        }
        alive = wait_mma(&bar, phase, err);
        if (!alive) break;
        // the operands are consumed: the next item's go in flight during this epilogue
        if (item + gridDim.x < nitems) issue(info(item + gridDim.x));
        const int q = warp & 3, m = 32 * q + lane;
        const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16);
        if constexpr (std::is_same<TO, c32>::value) {
            const int hb = 4 * (warp >> 2);
            const bool vec = vec_ok && hb + 4 <= u.nb;
            float sch[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) sch[j] = hb ? sc[4 + j] : sc[j];
            for (int tb = 0; 4 * tb < u.ns; ++tb) {
                float v[4][8];
#pragma unroll
                for (int j = 0; j < 4; ++j) tmem_ld8(trow + 32 * (hb + j) + 8 * tb, v[j]);
#pragma unroll
                for (int tt = 0; tt < 4; ++tt) {
                    const int t = 4 * tb + tt;
                    if (t >= u.ns) break;
                    c32 *dst = out + ((u.t0 + t) * M + m) * Nd + u.i0 + hb;
                    if (vec) {
                        st_global_v8(dst, v[0][2 * tt] * sch[0], v[0][2 * tt + 1] * sch[0], v[1][2 * tt] * sch[1],
                                     v[1][2 * tt + 1] * sch[1], v[2][2 * tt] * sch[2], v[2][2 * tt + 1] * sch[2],
                                     v[3][2 * tt] * sch[3], v[3][2 * tt + 1] * sch[3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (hb + j < u.nb) dst[j] = make_float2(v[j][2 * tt] * sch[j], v[j][2 * tt + 1] * sch[j]);
                    }
                }
            }
        } else {
            const bool vec = vec_ok && u.nb == EXB;
            for (int tb = warp >> 2; 4 * tb < u.ns; tb += 2) {
                uint32_t w[4][EXB];
#pragma unroll
                for (int b = 0; b < EXB; ++b) {
                    float v[8];
                    tmem_ld8(trow + 32 * b + 8 * tb, v);
#pragma unroll
                    for (int tt = 0; tt < 4; ++tt) w[tt][b] = pack_bf16(v[2 * tt] * sc[b], v[2 * tt + 1] * sc[b]);
                }
#pragma unroll
                for (int tt = 0; tt < 4; ++tt) {
                    const int t = 4 * tb + tt;
                    if (t >= u.ns) break;
                    uint32_t *dst = reinterpret_cast<uint32_t *>(out + ((u.t0 + t) * M + m) * Nd + u.i0);
                    if (vec) {
                        st_global_v8(dst, w[tt]);
                    } else {
#pragma unroll
                        for (int b = 0; b < EXB; ++b)
                            if (b < u.nb) dst[b] = w[tt][b];
                    }
                }
            }
        }
        fence_before();
        __syncthreads();
    }
    teardown(&bar, phase, alive, tmem, 256, err);
}

// ---------------------------------------------------------------------------
// The reduce for the benchmark shape -- BF16 activation planes, M = 128, K = 16, one
// 16-symbol block per realisation -- software-pipelined: right after an item's A tile is
// built, the activation loads of the CTA's next item are issued into the registers it
// freed, so they are in flight during this item's MMAs and epilogue.
template <bool CONJ, bool AT, bool COMB>
__global__ void __launch_bounds__(THREADS, 2)
    reduce_pipe_kernel(Geo g, int S, const uint32_t *__restrict__ Wt, const float *__restrict__ alpha,
                       const cbf16 *__restrict__ X, c32 *__restrict__ out, const c32 *__restrict__ s_ref,
                       c32 *__restrict__ gy, double *metrics, double inv_count, int inv_alpha, int vec_ok, int *err) {
    constexpr int M = 128, K = 16, PER = TS * 128 / THREADS;   // (t, m) pairs per thread
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *sA = align1024(smem_raw);
    uint8_t *sB = sA + RD_A;
    float *sY = reinterpret_cast<float *>(sB + RD_B);
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    __shared__ double red[32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Nd = g.N_d;
    const int ngroups = (Nd + RDB - 1) / RDB;
    const int R = (S + g.S_per_real - 1) / g.S_per_real;
    const long nitems = (long)R * ngroups;
    const uint32_t tmem = setup(&bar, &tmem_slot, 64);
    const uint32_t idesc = instr_desc(1, 128, 64);
    const float gscale = (float)(2.0 * inv_count);
    uint32_t phase = 0;
    bool alive = true;
    float err_acc = 0.f, sig_acc = 0.f;

    struct It {
        long t0, bin0, x0;
        int i0, ns, nb;
    };
    const BlkPlane bp(g);
    auto info = [&](long item) {
        It u;
        const int r = (int)(item / ngroups), j = (int)(item % ngroups);
        u.i0 = j * RDB;
        u.t0 = (long)r * g.S_per_real;
        u.ns = (int)min((long)g.S_per_real, (long)S - u.t0);
        u.bin0 = (long)r * Nd + u.i0;
        u.nb = min(RDB, Nd - u.i0);
        u.x0 = bp.item(r, j);
        return u;
    };
    uint32_t w[PER][RDB];   // the activations of the item being prepared
    // from the blocked plane: (slot t, antenna m) = element x0 + 4 (128 t + m), one 16-byte
    // load each, consecutive across the CTA; padding subcarriers past N_d read as zero
    auto load_acts = [&](const It &u) {
#pragma unroll
        for (int h = 0; h < PER; ++h) {
            const int e = tid + h * THREADS, t = e >> 7;
            const bool ok = t < u.ns;
            const uint32_t *src = reinterpret_cast<const uint32_t *>(X + u.x0 + (long)(ok ? e : 0) * RDB);
            if (ok && vec_ok) {
                const uint4 q4 = *reinterpret_cast<const uint4 *>(src);
                w[h][0] = q4.x;
                w[h][1] = u.nb > 1 ? q4.y : 0u;
                w[h][2] = u.nb > 2 ? q4.z : 0u;
                w[h][3] = u.nb > 3 ? q4.w : 0u;
            } else {
#pragma unroll
                for (int b = 0; b < RDB; ++b) w[h][b] = (ok && b < u.nb) ? src[b] : 0u;
            }
        }
    };
    // B rows 16 b + u of an item by cp.async (into a tile no MMA is reading)
    auto issue_b = [&](const It &u) {
        if (!AT) {
            for (int c = tid; c < RDB * K * 32; c += THREADS) {
                const int mc = c & 31, uu = (c >> 5) & 15, b = c >> 9;
                const bool ok = b < u.nb;
                cp_async16(sB + (mc >> 3) * 8192 + sw128_offset(16 * b + uu, (mc & 7) * 8),
                           ok ? Wt + ((u.bin0 + b) * K + uu) * M + 4 * mc : Wt, ok);
            }
        } else {
            for (int c = tid; c < RDB * M * 4; c += THREADS) {
                const int uq = c & 3, m = (c >> 2) & 127, b = c >> 9;
                const bool ok = b < u.nb;
                const uint32_t *src = ok ? Wt + ((u.bin0 + b) * M + m) * K + 4 * uq : Wt;
                uint8_t *dst = sB + (m >> 5) * 8192;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    cp_async4(dst + sw128_offset(16 * b + 4 * uq + j, 2 * (m & 31)), ok ? src + j : Wt, ok);
            }
        }
    };
    if (blockIdx.x < nitems) {
        load_acts(info(blockIdx.x));
        issue_b(info(blockIdx.x));
    }

    for (long item = blockIdx.x; item < nitems && alive; item += gridDim.x) {
        const It u = info(item);
        float sc = 0.f;
        if (warp < u.nb) {
            const float al = alpha[u.bin0 + warp];
            sc = inv_alpha ? 1.0f / al : al;
        }
        // the reference symbols of the epilogue, in flight from the start of the item
        const int nout = u.ns * K * RDB;
        c32 sref[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e = tid + k * THREADS;
            const int b = e & (RDB - 1), uu = (e >> 2) & 15, t = e >> 6;
            sref[k] = (COMB && e < nout && b < u.nb) ? s_ref[((u.t0 + t) * K + uu) * Nd + u.i0 + b]
                                                     : make_float2(0.f, 0.f);
        }
        // A: the real form of this item's activations (loaded during the previous item)
#pragma unroll
        for (int h = 0; h < PER; ++h) {
            const int e = tid + h * THREADS, m = e & 127, t = e >> 7;
            uint8_t *tile = sA + (m >> 5) * 16384;
            const int k = 2 * (m & 31);
#pragma unroll
            for (int b = 0; b < RDB; ++b) {
                uint32_t w0, w1;
                real_rows_packed<CONJ>(w[h][b], w0, w1);
                st32(tile + sw128_offset(32 * b + 2 * t, k), w0);
                st32(tile + sw128_offset(32 * b + 2 * t + 1, k), w1);
            }
        }
        // the next item's activations go in flight now
        if (item + gridDim.x < nitems) load_acts(info(item + gridDim.x));
        cp_async_wait_all();
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            fence_after();
#pragma unroll
            for (int ks = 0; ks < 16; ++ks)
                mma_f16(tmem, smem_desc(sA + (ks >> 2) * 16384 + (ks & 3) * 32),
                        smem_desc(sB + (ks >> 2) * 8192 + (ks & 3) * 32), idesc, ks ? 1u : 0u);
            mma_commit(&bar);
        }
        alive = wait_mma(&bar, phase, err);
        // the tiles are consumed: the next item's B goes in flight during this epilogue
        if (alive && item + gridDim.x < nitems) issue_b(info(item + gridDim.x));
        if (alive) {
            if (warp < RDB) {
                const int b = warp, t = lane >> 1, c = lane & 1;
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + 16 * b, v);
                if (b < u.nb && t < u.ns) {
#pragma unroll
                    for (int uu = 0; uu < 16; ++uu) sY[t * RD_YT + (uu * RDB + b) * 2 + c] = v[uu] * sc;
                }
            }
            __syncthreads();
            const c32 *sYc = reinterpret_cast<const c32 *>(sY);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int e = tid + k * THREADS;
                const int b = e & (RDB - 1), uu = (e >> 2) & 15, t = e >> 6;
                if (e >= nout || b >= u.nb) continue;
                const c32 v = sYc[(t * RD_YT + (uu * RDB + b) * 2) / 2];
                const long idx = ((u.t0 + t) * K + uu) * Nd + u.i0 + b;
                if (COMB) {
                    const c32 d = csub(v, sref[k]);
                    err_acc += cabs2(d);
                    sig_acc += cabs2(sref[k]);
                    if (out) out[idx] = v;
                    if (gy) gy[idx] = cscale(d, gscale);
                } else {
                    out[idx] = v;
                }
            }
        }
        fence_before();
        __syncthreads();
    }
    teardown(&bar, phase, alive, tmem, 64, err);
    if (COMB && metrics) {
        const double es = block_sum((double)err_acc, red);
        const double ss = block_sum((double)sig_acc, red);
        if (tid == 0) {
            atomicAdd(metrics + 1, es);
            atomicAdd(metrics + 2, ss);
        }
    }
}

// ---------------------------------------------------------------------------
static int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// Two CTAs per SM only fit with the largest shared-memory carveout; the occupancy query
// assumes the function's preferred carveout, so it is set first.
// Two CTAs per SM (both kernels are sized for it: shared memory below half the SM's, at
// most 128 registers a thread, at most 256 TMEM columns each) with the largest carveout,
// or one (Geo::bin_ctas = 1: room for other plans' kernels running beside these).
template <class Kern> static cudaError_t grid_for(const Geo &g, Kern k, int smem, long items, unsigned &blocks) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    long b = (g.bin_ctas == 1 ? 1L : 2L) * sm_count();
    if (b > items) b = items;
    blocks = (unsigned)(b > 0 ? b : 1);
    return cudaSuccess;
}

static bool aligned32(const void *p) { return !(reinterpret_cast<uintptr_t>(p) & 31); }
static bool aligned16(const void *p) { return !(reinterpret_cast<uintptr_t>(p) & 15); }

template <typename T16, typename TO>
static cudaError_t expand_t(const Geo &g, int mode, int S, const void *A, const float *alpha, const c32 *B, TO *out,
                            float b_scale, int *err, cudaStream_t st) {
    const int R = (S + g.S_per_real - 1) / g.S_per_real;
    const int exb = (g.K > 16 ? EXB / 2 : EXB) >> (g.bin_half ? 1 : 0);
    const long items = (long)R * ((g.N_d + exb - 1) / exb) * ((g.M + 127) / 128);
    if (items == 0) return cudaSuccess;
    // one 32-byte sector = 4 FP32 or 8 BF16 subcarriers
    const int vec_ok = !(g.N_d & (std::is_same<TO, c32>::value ? 3 : 7)) && aligned32(out);
    const uint32_t *a = static_cast<const uint32_t *>(A);
    unsigned blocks = 0;
    cudaError_t e;
    if constexpr (std::is_same<T16, cbf16>::value) {
        if (g.M == 128 && g.K == 16 && g.S_per_real <= TS && b_scale == 1.0f && !g.bin_half) {
            if (mode == PRECODE || mode == ADJ_COMBINE_F) {
                auto k = expand_pipe_kernel<false, false, TO>;
                if ((e = grid_for(g, k, EX_SMEM, items, blocks)) != cudaSuccess) return e;
                k<<<blocks, THREADS, EX_SMEM, st>>>(g, S, a, alpha, B, out, mode == ADJ_COMBINE_F, vec_ok, err);
            } else {
                auto k = expand_pipe_kernel<true, true, TO>;
                if ((e = grid_for(g, k, EX_SMEM, items, blocks)) != cudaSuccess) return e;
                k<<<blocks, THREADS, EX_SMEM, st>>>(g, S, a, alpha, B, out, 1, vec_ok, err);
            }
            return cudaGetLastError();
        }
    }
    if (mode == PRECODE || mode == ADJ_COMBINE_F) {
        auto k = expand_kernel<T16, false, false, TO>;
        if ((e = grid_for(g, k, EX_SMEM, items, blocks)) != cudaSuccess) return e;
        k<<<blocks, THREADS, EX_SMEM, st>>>(g, S, a, alpha, B, out, mode == ADJ_COMBINE_F, b_scale, vec_ok, err);
    } else {
        auto k = expand_kernel<T16, true, true, TO>;
        if ((e = grid_for(g, k, EX_SMEM, items, blocks)) != cudaSuccess) return e;
        k<<<blocks, THREADS, EX_SMEM, st>>>(g, S, a, alpha, B, out, 1, b_scale, vec_ok, err);
    }
    return cudaGetLastError();
}

template <typename T16, typename TX>
static cudaError_t reduce_t(const Geo &g, int mode, int S, const void *A, const float *alpha, const TX *B, c32 *out,
                            const c32 *s_ref, c32 *gy, double *metrics, double inv_count, float b_scale, int *err,
                            cudaStream_t st) {
    const int R = (S + g.S_per_real - 1) / g.S_per_real;
    const int rdb = g.bin_half ? RDB / 2 : RDB;
    const long items = (long)R * ((g.N_d + rdb - 1) / rdb);
    if (items == 0) return cudaSuccess;
    // 4 subcarriers: two 16-byte FP32 loads from rows, or one of BF16 from the blocked plane
    const int vec_ok = (std::is_same<TX, c32>::value ? !(g.N_d & 1) : 1) && aligned16(B);
    const uint32_t *a = static_cast<const uint32_t *>(A);
    unsigned blocks = 0;
    cudaError_t e;
    const bool full = g.M == 128 && g.K == 16;
    if constexpr (std::is_same<TX, cbf16>::value && std::is_same<T16, cbf16>::value) {
        if (full && g.S_per_real <= TS && b_scale == 1.0f && !g.bin_half) {
            if (mode == COMBINE) {
                auto k = reduce_pipe_kernel<false, false, true>;
                if ((e = grid_for(g, k, RD_SMEM, items, blocks)) != cudaSuccess) return e;
                k<<<blocks, THREADS, RD_SMEM, st>>>(g, S, a, alpha, B, out, s_ref, gy, metrics, inv_count, 1, vec_ok, err);
            } else if (mode == ADJ_PRECODE_F) {
                auto k = reduce_pipe_kernel<false, false, false>;
                if ((e = grid_for(g, k, RD_SMEM, items, blocks)) != cudaSuccess) return e;
                k<<<blocks, THREADS, RD_SMEM, st>>>(g, S, a, alpha, B, out, nullptr, nullptr, nullptr, 0.0, 0, vec_ok, err);
            } else {
                auto k = reduce_pipe_kernel<true, true, false>;
                if ((e = grid_for(g, k, RD_SMEM, items, blocks)) != cudaSuccess) return e;
                k<<<blocks, THREADS, RD_SMEM, st>>>(g, S, a, alpha, B, out, nullptr, nullptr, nullptr, 0.0, 0, vec_ok, err);
            }
            return cudaGetLastError();
        }
    }
    if (mode == COMBINE) {
        auto k = full ? reduce_kernel<T16, false, false, true, TX, true> : reduce_kernel<T16, false, false, true, TX, false>;
        if ((e = grid_for(g, k, RD_SMEM, items, blocks)) != cudaSuccess) return e;
        k<<<blocks, THREADS, RD_SMEM, st>>>(g, S, a, alpha, B, out, s_ref, gy, metrics, inv_count, 1, b_scale, vec_ok,
                                            err);
    } else if (mode == ADJ_PRECODE_F) {
        auto k = full ? reduce_kernel<T16, false, false, false, TX, true> : reduce_kernel<T16, false, false, false, TX, false>;
        if ((e = grid_for(g, k, RD_SMEM, items, blocks)) != cudaSuccess) return e;
        k<<<blocks, THREADS, RD_SMEM, st>>>(g, S, a, alpha, B, out, nullptr, nullptr, nullptr, 0.0, 0, b_scale, vec_ok,
                                            err);
    } else {
        auto k = full ? reduce_kernel<T16, true, true, false, TX, true> : reduce_kernel<T16, true, true, false, TX, false>;
        if ((e = grid_for(g, k, RD_SMEM, items, blocks)) != cudaSuccess) return e;
        k<<<blocks, THREADS, RD_SMEM, st>>>(g, S, a, alpha, B, out, nullptr, nullptr, nullptr, 0.0, 0, b_scale,
                                            vec_ok, err);
    }
    return cudaGetLastError();
}

}  // namespace tcb

bool tc_bin_supported(const Geo &g) { return g.M >= 1 && g.M <= 256 && g.K >= 1 && g.K <= 32; }
bool tc_apply_supported(const Geo &g) { return g.M >= 1 && g.M <= 128 && g.K >= 1 && g.K <= 16; }

cudaError_t tc_bin_expand(const Geo &g, int mode, int S, const void *A, int a_kind, const float *alpha, const c32 *B,
                          void *out, int act_kind, float b_scale, int *err, cudaStream_t st) {
    if (!tc_bin_supported(g) || (mode != PRECODE && mode != ADJ_COMBINE && mode != ADJ_COMBINE_F))
        return cudaErrorInvalidValue;
    if (act_kind == OUT_BF16) {
        if (a_kind != OUT_BF16 || b_scale != 1.0f) return cudaErrorInvalidValue;
        return tcb::expand_t<cbf16>(g, mode, S, A, alpha, B, static_cast<cbf16 *>(out), b_scale, err, st);
    }
    if (act_kind != OUT_F32) return cudaErrorInvalidValue;
    c32 *o = static_cast<c32 *>(out);
    if (a_kind == OUT_BF16) return tcb::expand_t<cbf16>(g, mode, S, A, alpha, B, o, b_scale, err, st);
    if (a_kind == OUT_F16) return tcb::expand_t<cf16>(g, mode, S, A, alpha, B, o, b_scale, err, st);
    return cudaErrorInvalidValue;
}

cudaError_t tc_bin_reduce(const Geo &g, int mode, int S, const void *A, int a_kind, const float *alpha, const void *B,
                          int act_kind, c32 *out, const c32 *s_ref, c32 *gy, double *metrics, double inv_count,
                          float b_scale, int *err, cudaStream_t st) {
    if (!tc_bin_supported(g) || (mode != COMBINE && mode != ADJ_PRECODE && mode != ADJ_PRECODE_F))
        return cudaErrorInvalidValue;
    if (act_kind == OUT_BF16) {
        if (a_kind != OUT_BF16 || b_scale != 1.0f) return cudaErrorInvalidValue;
        return tcb::reduce_t<cbf16>(g, mode, S, A, alpha, static_cast<const cbf16 *>(B), out, s_ref, gy, metrics,
                                    inv_count, b_scale, err, st);
    }
    if (act_kind != OUT_F32) return cudaErrorInvalidValue;
    const c32 *x = static_cast<const c32 *>(B);
    if (a_kind == OUT_BF16)
        return tcb::reduce_t<cbf16>(g, mode, S, A, alpha, x, out, s_ref, gy, metrics, inv_count, b_scale, err, st);
    if (a_kind == OUT_F16)
        return tcb::reduce_t<cf16>(g, mode, S, A, alpha, x, out, s_ref, gy, metrics, inv_count, b_scale, err, st);
    return cudaErrorInvalidValue;
}

}  // namespace fdk
