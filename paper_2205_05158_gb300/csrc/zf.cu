// Zero-forcing precoder, Eq. (6): W_k = H_k^H (H_k H_k^H)^{-1} and the per-subcarrier
// normalisation alpha_k = sqrt(P_T / tr((H_k H_k^H)^{-1})), so that the precoded
// vector alpha_k W_k s has E||.||^2 = P_T for unit-power symbols.
//
// Three kernels over all (realisation, data subcarrier) pairs ("bins"):
//   gram   : one warp per bin, G = H H^H from FP32 products and FP32 sums; each lane a
//            4 x 4 block of the lower triangle over one group of antennas (8 shared
//            loads per 16 complex multiply-adds).  The lower triangle goes to a scratch
//            array laid out [bin / 32][entry][bin % 32].
//   factor : one bin per LANE, so every instruction is a full-warp instruction:
//            Cholesky G = L L^H (left-looking) and the in-place triangular inverse
//            Y = L^{-1}; tr(G^{-1}) = ||Y||_F^2.  FP64 (1/sqrt(d) from the FP32
//            rsqrtf and two Newton-Raphson steps y <- y (3 - d y^2) / 2 in FP64), or
//            FP32 in 16-bit plans that select it (one Newton step).  Y (FP32) and alpha go out;
//            a pivot <= 1e-9 (FP64) or 1e-5 (FP32) of its Gram diagonal marks the bin
//            singular (alpha = 0, W = 0, status bit 0).
//   apply  : one warp per bin, W^H = Y^H (Y H) in FP32 (one antenna per lane), staged
//            through shared memory for coalesced stores.
#include <type_traits>

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

// ---------------------------------------------------------------------------
// Gram G = H H^H, one warp per subcarrier.  The lower triangle is tiled into 4 x 4 blocks
// (10 for K = 16) and the antennas of each 32-antenna chunk into ng groups, one (block,
// group) task per lane (30 of 32 lanes for K = 16): per antenna a lane loads 4 + 4
// entries for 16 complex multiply-adds.  Partial sums of the groups meet in shared memory
// at the end.  A warp streams its (subcarrier, chunk) sequence through two chunk buffers
// ([K][33] complex, 4.2 KB for K = 16) with cp.async, so the next chunk -- also the next
// subcarrier's first -- is in flight while the current one is multiplied.
constexpr int GR_CHUNK = 32, GR_LD = GR_CHUNK + 1;

FD_HD int gram_tasks(int K, int &nbt, int &ng) {
    const int nblk = (K + 3) / 4;
    nbt = nblk * (nblk + 1) / 2;
    ng = 32 / nbt;
    if (ng < 1) ng = 1;
    if (ng > GR_CHUNK) ng = GR_CHUNK;
    return nbt * ng;
}
// one of the two per-warp buffers: a chunk, or the partial sums of the tasks
size_t gram_buf_bytes(int K) {
    int nbt, ng;
    const int tasks = gram_tasks(K, nbt, ng);
    const size_t chunk = sizeof(c32) * K * GR_LD, red = sizeof(c32) * 16 * tasks;
    return al16(chunk > red ? chunk : red);
}

FD_D void cp_async8z(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(valid ? 8 : 0)
                 : "memory");
}
FD_D void cp_async16(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}

template <typename T16, int NT>   // NT: tasks per lane (2 when K > 28)
__global__ void __launch_bounds__(32 * ZF_WARPS, NT == 1 ? 3 : 1) zf_gram_kernel(Geo g, long nbins, const c32 *__restrict__ H,
                                                                c32 *__restrict__ Gs, T16 *__restrict__ H16,
                                                                T16 *__restrict__ HH16, int buf_bytes) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int K = g.K, M = g.M, T = tri(K);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    unsigned char *wbuf = sm + (size_t)(2 * warp) * buf_bytes;   // this warp's two buffers
    auto buf = [&](long it) { return reinterpret_cast<c32 *>(wbuf + (it & 1) * (size_t)buf_bytes); };
    int nbt, ng;
    const int tasks = gram_tasks(K, nbt, ng);
    // this lane's tasks: task = group * nbt + block
    int bi[NT], bj[NT], glo[NT], ghi[NT], ntask = 0;
    for (int t = lane; t < tasks && ntask < NT; t += 32, ++ntask) {
        int blk = t % nbt, r = 0;
        while (blk > r) { blk -= r + 1; ++r; }
        bi[ntask] = r;
        bj[ntask] = blk;
        const int grp = t / nbt;
        glo[ntask] = grp * GR_CHUNK / ng;
        ghi[ntask] = (grp + 1) * GR_CHUNK / ng;
    }
    const int nch = (M + GR_CHUNK - 1) / GR_CHUNK;
    const long b0 = (long)blockIdx.x * nwarps + warp, bstep = (long)gridDim.x * nwarps;
    const long nmine = b0 < nbins ? (nbins - 1 - b0) / bstep + 1 : 0;
    const long nitems = nmine * nch;   // (subcarrier, chunk) pairs of this warp, in order
    auto issue = [&](long it) {
        const long b = b0 + (it / nch) * bstep;
        const int m = (int)(it % nch) * GR_CHUNK + lane;
        c32 *dst = buf(it);
        for (int u = 0; u < K; ++u)
            cp_async8z(dst + u * GR_LD + lane, m < M ? H + (b * K + u) * M + m : H, m < M);
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    c32 acc[NT][4][4];
    if (nitems > 0) issue(0);
    for (long it = 0; it < nitems; ++it) {
        const long b = b0 + (it / nch) * bstep;
        const int ch = (int)(it % nch), m0 = ch * GR_CHUNK;
        c32 *sH = buf(it);
        if (it + 1 < nitems) {
            issue(it + 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncwarp();
        if (ch == 0) {
#pragma unroll
            for (int q = 0; q < NT; ++q)
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[q][a][c] = make_float2(0.f, 0.f);
        }
        if (H16 && m0 + lane < M)
            for (int u = 0; u < K; ++u) H16[(b * K + u) * M + m0 + lane] = Operand<T16>::from(sH[u * GR_LD + lane]);
        if (HH16 && m0 + lane < M)   // H^H in W's layout [b][m][u]
            for (int u = 0; u < K; ++u)
                HH16[(b * M + m0 + lane) * K + u] = Operand<T16>::from(cconj(sH[u * GR_LD + lane]));
#pragma unroll
        for (int q = 0; q < NT; ++q) {
            if (q >= ntask) break;
            const int ri = 4 * bi[q], rj = 4 * bj[q];
            for (int mm = glo[q]; mm < ghi[q]; ++mm) {
                c32 hi[4], hj[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    hi[a] = ri + a < K ? sH[(ri + a) * GR_LD + mm] : make_float2(0.f, 0.f);
                    hj[a] = rj + a < K ? cconj(sH[(rj + a) * GR_LD + mm]) : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[q][a][c] = cfma(hi[a], hj[c], acc[q][a][c]);
            }
        }
        __syncwarp();
        if (ch == nch - 1) {
            // sum the antenna groups of each block in this (now free) buffer: partials
            // [task][16]; the other buffer may already hold the next subcarrier's chunk
            c32 *red = sH;
#pragma unroll
            for (int q = 0; q < NT; ++q) {
                if (q >= ntask) break;
                const int t = lane + 32 * q;
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) red[t * 16 + a * 4 + c] = acc[q][a][c];
            }
            __syncwarp();
            for (int idx = lane; idx < nbt * 16; idx += 32) {
                int blk = idx >> 4, r = 0;
                while (blk > r) { blk -= r + 1; ++r; }
                const int i = 4 * r + ((idx >> 2) & 3), j = 4 * blk + (idx & 3);
                if (i < K && j <= i) {
                    c32 sum = make_float2(0.f, 0.f);
                    for (int grp = 0; grp < ng; ++grp) {
                        const c32 v = red[(grp * nbt + (idx >> 4)) * 16 + (idx & 15)];
                        sum.x += v.x;
                        sum.y += v.y;
                    }
                    Gs[soa(b, tri(i) + j, T)] = sum;
                }
            }
            __syncwarp();
        }
    }
}

// K = 16 with M a multiple of 32 (the massive-MIMO shapes): the same warp-per-subcarrier
// product with every index a compile-time constant.  Lane l < 30 takes block l % 10 over
// antenna group l / 10 of each chunk: columns 11 g .. 11 g + 10, where the third group's
// last column is the zero padding column 32 of the chunk buffer, so all three run the
// same 11 steps.  The three groups' partial sums meet by warp shuffles.
template <typename T16>
__global__ void __launch_bounds__(32 * ZF_WARPS, 3)
    zf_gram16_kernel(Geo g, long nbins, const c32 *__restrict__ H, c32 *__restrict__ Gs, T16 *__restrict__ H16,
                     T16 *__restrict__ HH16) {
    constexpr int K = 16, T = 136, LD = GR_LD, BUF = K * LD;
    extern __shared__ __align__(16) unsigned char sm[];
    const int M = g.M;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    c32 *wbuf = reinterpret_cast<c32 *>(sm) + (size_t)warp * 2 * BUF;
    wbuf[(lane >> 4) * BUF + (lane & 15) * LD + GR_CHUNK] = make_float2(0.f, 0.f);   // padding columns
    const int blk = lane % 10, grp = lane < 30 ? lane / 10 : 2;
    const int bi = blk < 1 ? 0 : blk < 3 ? 1 : blk < 6 ? 2 : 3;
    const int bj = blk - bi * (bi + 1) / 2;
    const int ri = 4 * bi, rj = 4 * bj, col0 = 11 * grp;
    const int nch = M / GR_CHUNK;
    const long bstep = (long)gridDim.x * ZF_WARPS;
    // chunk (b, ch) into buffer p: H rows u = 0..15, antennas 32 ch + lane
    auto issue = [&](long b, int ch, int p) {
        const c32 *src = H + b * K * M + ch * GR_CHUNK + lane;
        c32 *dst = wbuf + p * BUF + lane;
#pragma unroll
        for (int u = 0; u < K; ++u) cp_async8z(dst + u * LD, src + (long)u * M, true);
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    __syncwarp();
    long b = (long)blockIdx.x * ZF_WARPS + warp;
    if (b < nbins) issue(b, 0, 0);
    int p = 0;
    for (; b < nbins; b += bstep) {
        c32 acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][c] = make_float2(0.f, 0.f);
        for (int ch = 0; ch < nch; ++ch, p ^= 1) {
            const c32 *sH = wbuf + p * BUF;
            // the next chunk -- of this subcarrier, else of the next one -- goes in flight
            const long bn = ch + 1 < nch ? b : b + bstep;
            if (bn < nbins) {
                issue(bn, ch + 1 < nch ? ch + 1 : 0, p ^ 1);
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            } else {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            }
            __syncwarp();
            if (H16 || HH16) {   // one shared read of antenna 32 ch + lane's users for both copies,
                                 // eight users at a time
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    c32 hv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) hv[u] = sH[(8 * h + u) * LD + lane];
                    if (H16) {
                        T16 *dst = H16 + b * K * M + ch * GR_CHUNK + lane;
#pragma unroll
                        for (int u = 0; u < 8; ++u) dst[(long)(8 * h + u) * M] = Operand<T16>::from(hv[u]);
                    }
                    if (HH16) {   // H^H in W's layout: antenna row m = 32 ch + lane, 16 users (64 bytes)
                        uint4 *dst = reinterpret_cast<uint4 *>(HH16 + (b * M + ch * GR_CHUNK + lane) * K);
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            uint32_t w[4];
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const T16 v = Operand<T16>::from(cconj(hv[4 * q + j]));
                                w[j] = *reinterpret_cast<const uint32_t *>(&v);
                            }
                            dst[2 * h + q] = make_uint4(w[0], w[1], w[2], w[3]);
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 11; ++k) {
                c32 hi[4], hj[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    hi[a] = sH[(ri + a) * LD + col0 + k];
                    hj[a] = sH[(rj + a) * LD + col0 + k];
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[a][c] = cfmac(hj[c], hi[a], acc[a][c]);   // h_i conj(h_j)
            }
            __syncwarp();   // this buffer is free for the chunk after next
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                c32 v = acc[a][c];
                const float x1 = __shfl_down_sync(0xffffffffu, v.x, 10), y1 = __shfl_down_sync(0xffffffffu, v.y, 10);
                const float x2 = __shfl_down_sync(0xffffffffu, v.x, 20), y2 = __shfl_down_sync(0xffffffffu, v.y, 20);
                v.x = (v.x + x1) + x2;
                v.y = (v.y + y1) + y2;
                const int i = ri + a, j = rj + c;
                if (lane < 10 && j <= i) Gs[soa(b, tri(i) + j, T)] = v;
            }
    }
}

// ---------------------------------------------------------------------------
// Scalar type of the factor: FP64; or FP32 where a 16-bit plan selects it, since its W is
// rounded to 16 bits afterwards (the FP32 factor's relative error, about the Gram
// condition number times 2^-24, stays far below that rounding).
template <typename Real> struct Fac;
template <> struct Fac<double> {
    using C = double2;
    static constexpr double kPivot = 1e-9;   // singular below this fraction of the Gram diagonal
    FD_D static double rsqrt(double d) {     // FP32 estimate, two Newton-Raphson steps in FP64
        double y = (double)rsqrtf((float)d);
#pragma unroll
        for (int it = 0; it < 2; ++it) y = y * (1.5 - 0.5 * d * y * y);
        return y;
    }
};
template <> struct Fac<float> {
    using C = float2;
    static constexpr float kPivot = 1e-5f;   // a pivot this small is lost in FP32 rounding
    FD_D static float rsqrt(float d) {
        const float y = rsqrtf(d);
        return y * (1.5f - 0.5f * d * y * y);
    }
};

// LPB lanes per bin: the bin's Cholesky rows (and the partial sums of its pivots) and
// its triangular-inverse rows are dealt round-robin to the LPB lanes, which sit BPW =
// 32 / LPB lanes apart in one warp (so a shared-memory phase of 8 lanes reads 8 bins,
// conflict free).  FP64 runs 4 lanes per bin in 4-warp CTAs, so that every SM
// sub-partition holds warps of the slow FP64 pipe's work; FP32 one lane per bin.
template <typename Real, int LPB>
__global__ void __launch_bounds__(128) zf_factor_kernel(Geo g, long nbins, const c32 *__restrict__ Gs,
                                                        c32 *__restrict__ Ys, float *__restrict__ alpha, int *status) {
    using F = Fac<Real>;
    using C = typename F::C;
    constexpr int BPW = 32 / LPB, RMAX = LPB > 1 ? (32 + LPB - 1) / LPB : 1;   // bins per warp, rows per lane
    extern __shared__ __align__(16) unsigned char sm[];
    const int K = g.K, T = tri(K);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int part = lane / BPW, lb = warp * BPW + lane % BPW;
    const int NB = (int)(blockDim.x >> 5) * BPW;             // bins per CTA
    C *A = reinterpret_cast<C *>(sm);                        // [T][NB]: lower triangle, becomes L, then Y
    Real *inv = reinterpret_cast<Real *>(A + (size_t)T * NB);   // [K][NB]
    const long b = (long)blockIdx.x * NB + lb;
    const bool live = b < nbins;
    const long bb = live ? b : 0;
    for (int e = part; e < T; e += LPB) {
        const c32 v = Gs[soa(bb, e, T)];
        A[e * NB + lb] = C{(Real)v.x, (Real)v.y};
    }
    __syncwarp();
    bool bad = false;
    // Cholesky, left-looking: column j from the columns left of it
    for (int j = 0; j < K; ++j) {
        const int dj = tri(j) + j;
        Real q = 0;
        for (int k = part; k < j; k += LPB) {
            const C l = A[(tri(j) + k) * NB + lb];
            q = fma(l.x, l.x, q);
            q = fma(l.y, l.y, q);
        }
        for (int o = BPW; o < 32; o <<= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
        const Real g0 = A[dj * NB + lb].x;
        const Real d = g0 - q;
        const bool ok = d > F::kPivot * g0;
        bad |= !ok;
        const Real r = ok ? F::rsqrt(d) : Real(1);
        // rows i > j: each row's sum over k < j on one lane (rows dealt to the lanes), or --
        // where that leaves lanes idle, for few long rows -- every row's sum split over
        // the lanes by k and combined by shuffles.  The choice depends on j alone and
        // counts the FP64 instructions a lane issues for the column either way: dealt
        // rows, ceil(nr / LPB) rows of j multiply-adds (4 each) and a scaling (2); split
        // sums, nr rows of ceil(j / LPB) multiply-adds, the shuffle reduction's adds
        // (2 per halving step) and the subtract-and-scale (4)
        const int nr = K - 1 - j;
        const int lg = LPB >= 4 ? 2 : LPB == 2 ? 1 : 0;
        const bool ksplit = LPB > 1 && nr * (4 * ((j + LPB - 1) / LPB) + 2 * lg + 4) <
                                           ((nr + LPB - 1) / LPB) * (4 * j + 2);
        if (ksplit) {
            for (int i = j + 1; i < K; ++i) {
                C s = C{Real(0), Real(0)};
                for (int k = part; k < j; k += LPB) {   // s += L[i][k] conj(L[j][k])
                    const C a = A[(tri(i) + k) * NB + lb], c = A[(tri(j) + k) * NB + lb];
                    s.x = fma(a.x, c.x, s.x);
                    s.x = fma(a.y, c.y, s.x);
                    s.y = fma(a.y, c.x, s.y);
                    s.y = fma(-a.x, c.y, s.y);
                }
                for (int o = BPW; o < 32; o <<= 1) {
                    s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
                    s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
                }
                if (part == (i & (LPB - 1))) {
                    const C a = A[(tri(i) + j) * NB + lb];
                    A[(tri(i) + j) * NB + lb] = C{(a.x - s.x) * r, (a.y - s.y) * r};
                }
            }
        } else {
            for (int i = j + 1 + part; i < K; i += LPB) {
                C s = A[(tri(i) + j) * NB + lb];
                for (int k = 0; k < j; ++k) {     // s -= L[i][k] conj(L[j][k])
                    const C a = A[(tri(i) + k) * NB + lb], c = A[(tri(j) + k) * NB + lb];
                    s.x = fma(-a.x, c.x, s.x);
                    s.x = fma(-a.y, c.y, s.x);
                    s.y = fma(-a.y, c.x, s.y);
                    s.y = fma(a.x, c.y, s.y);
                }
                A[(tri(i) + j) * NB + lb] = C{s.x * r, s.y * r};
            }
        }
        if (part == 0) {
            A[dj * NB + lb] = C{ok ? d * r : Real(1), Real(0)};
            inv[j * NB + lb] = r;
        }
        __syncwarp();
    }
    // in-place inverse: for j = K-1..0, Y[j][j] = 1/L[j][j], and for i = K-1..j+1
    // Y[i][j] = -(1/L[j][j]) sum_{k=j+1}^{i} Y[i][k] L[k][j]; a column's new values are
    // held until every lane has read its L entries
    Real tr = 0;
    for (int j = K - 1; j >= 0 && LPB == 1; --j) {   // one lane per bin: rows in descending order, in place
        const Real r = inv[j * NB + lb];
        for (int i = K - 1; i > j; --i) {
            C s = C{Real(0), Real(0)};
            for (int k = j + 1; k <= i; ++k) {
                const C y = A[(tri(i) + k) * NB + lb], l = A[(tri(k) + j) * NB + lb];
                s.x = fma(y.x, l.x, s.x);
                s.x = fma(-y.y, l.y, s.x);
                s.y = fma(y.x, l.y, s.y);
                s.y = fma(y.y, l.x, s.y);
            }
            const C v = C{-s.x * r, -s.y * r};
            A[(tri(i) + j) * NB + lb] = v;
            tr = fma(v.x, v.x, tr);
            tr = fma(v.y, v.y, tr);
        }
        A[(tri(j) + j) * NB + lb] = C{r, Real(0)};
        tr = fma(r, r, tr);
    }
    for (int j = K - 1; j >= 0 && LPB > 1; --j) {
        const Real r = inv[j * NB + lb];
        C out[RMAX];
        // rows dealt in snake order (K-1 .. K-LPB to lanes 0..LPB-1, the next LPB rows back
        // from lane LPB-1), which evens out the rows' unequal lengths i - j
#pragma unroll
        for (int t = 0; t < RMAX; ++t) {
            const int i = K - 1 - t * LPB - ((t & 1) ? LPB - 1 - part : part);
            if (i > j) {
                C s = C{Real(0), Real(0)};
                for (int k = j + 1; k <= i; ++k) {
                    const C y = A[(tri(i) + k) * NB + lb], l = A[(tri(k) + j) * NB + lb];
                    s.x = fma(y.x, l.x, s.x);
                    s.x = fma(-y.y, l.y, s.x);
                    s.y = fma(y.x, l.y, s.y);
                    s.y = fma(y.y, l.x, s.y);
                }
                out[t] = C{-s.x * r, -s.y * r};
            }
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < RMAX; ++t) {
            const int i = K - 1 - t * LPB - ((t & 1) ? LPB - 1 - part : part);
            if (i > j) {
                A[(tri(i) + j) * NB + lb] = out[t];
                tr = fma(out[t].x, out[t].x, tr);
                tr = fma(out[t].y, out[t].y, tr);
            }
        }
        if (part == 0) {
            A[(tri(j) + j) * NB + lb] = C{r, Real(0)};
            tr = fma(r, r, tr);
        }
        __syncwarp();
    }
    for (int o = BPW; o < 32; o <<= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    if (live) {
        for (int e = part; e < T; e += LPB) {
            const C v = A[e * NB + lb];
            Ys[soa(b, e, T)] = make_float2((float)v.x, (float)v.y);
        }
        if (part == 0) alpha[b] = bad ? 0.0f : (float)sqrt(g.P_T / (double)tr);
    }
    if (live && bad && part == 0) atomicOr(status, 1);
}

template <typename Real>
static cudaError_t launch_factor(const Geo &g, long nbins, const c32 *Gs, c32 *Ys, float *alpha, int *status,
                                 cudaStream_t st) {
    using C = typename Fac<Real>::C;
    constexpr int LPB = sizeof(Real) == 8 ? 4 : 1;
    const int T = tri(g.K);
    int threads = sizeof(Real) == 8 ? 128 : 32;
    auto bytes = [&](int thr) { return (sizeof(C) * T + sizeof(Real) * g.K) * (size_t)(thr / LPB); };
    while (bytes(threads) > 200 * 1024 && threads > 32) threads /= 2;
    if (bytes(threads) > 200 * 1024) return cudaErrorInvalidConfiguration;
    const int NB = threads / LPB;
    const size_t smem = bytes(threads);
    cudaError_t e = cudaFuncSetAttribute(zf_factor_kernel<Real, LPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    zf_factor_kernel<Real, LPB><<<(unsigned)((nbins + NB - 1) / NB), threads, smem, st>>>(g, nbins, Gs, Ys, alpha,
                                                                                        status);
    return cudaGetLastError();
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
    blocks = (long)resident_ctas(k, threads, smem) * sm_count();
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
                              T16 *H16, T16 *W16, int phase, bool fp64_factor, bool tc_apply, int *err,
                              cudaStream_t st, T16 *HH16) {
    const long nbins = (long)R * g.N_d;
    if (nbins == 0) return cudaSuccess;
    const int T = tri(g.K);
    const long nb32 = (nbins + 31) / 32 * 32;
    c32 *Gs = reinterpret_cast<c32 *>(scratch);
    c32 *Ys = reinterpret_cast<c32 *>(reinterpret_cast<char *>(scratch) + al16(sizeof(c32) * (size_t)nb32 * T));
    // gram
    if (phase < 0 || phase == 0) {
        const int per_buf = (int)gram_buf_bytes(g.K);
        const size_t smem = (size_t)ZF_WARPS * 2 * per_buf;
        long blocks = 0;
        cudaError_t e;
        if (g.K == 16 && g.M % GR_CHUNK == 0 && !(reinterpret_cast<uintptr_t>(HH16) & 15)) {
            const size_t smem16 = (size_t)ZF_WARPS * 2 * 16 * GR_LD * sizeof(c32);
            e = persistent_launch_dims(zf_gram16_kernel<T16>, 32 * ZF_WARPS, smem16, nbins, ZF_WARPS, blocks);
            if (e != cudaSuccess) return e;
            zf_gram16_kernel<T16><<<(unsigned)blocks, 32 * ZF_WARPS, smem16, st>>>(g, nbins, H, Gs, H16, HH16);
        } else if (g.K <= 28) {
            e = persistent_launch_dims(zf_gram_kernel<T16, 1>, 32 * ZF_WARPS, smem, nbins, ZF_WARPS, blocks);
            if (e != cudaSuccess) return e;
            zf_gram_kernel<T16, 1><<<(unsigned)blocks, 32 * ZF_WARPS, smem, st>>>(g, nbins, H, Gs, H16, HH16, per_buf);
        } else {
            e = persistent_launch_dims(zf_gram_kernel<T16, 2>, 32 * ZF_WARPS, smem, nbins, ZF_WARPS, blocks);
            if (e != cudaSuccess) return e;
            zf_gram_kernel<T16, 2><<<(unsigned)blocks, 32 * ZF_WARPS, smem, st>>>(g, nbins, H, Gs, H16, HH16, per_buf);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // factor
    if (phase < 0 || phase == 1) {
        cudaError_t e = fp64_factor ? launch_factor<double>(g, nbins, Gs, Ys, alpha, status, st)
                                    : launch_factor<float>(g, nbins, Gs, Ys, alpha, status, st);
        if (e != cudaSuccess) return e;
    }
    // apply
    if (phase >= 0 && phase != 2) return cudaSuccess;
    if (tc_apply)
        return zf_apply_tc(g, nbins, H, Ys, alpha, W, W16, std::is_same<T16, cbf16>::value ? OUT_BF16 : OUT_F16, err,
                           st);
    if (g.K <= 4) return launch_apply<4>(g, nbins, H, Ys, alpha, W, W16, st);
    if (g.K <= 8) return launch_apply<8>(g, nbins, H, Ys, alpha, W, W16, st);
    if (g.K <= 16) return launch_apply<16>(g, nbins, H, Ys, alpha, W, W16, st);
    return launch_apply<32>(g, nbins, H, Ys, alpha, W, W16, st);
}

cudaError_t zf_phase(int phase, const Geo &g, int R, const c32 *H, c32 *W, float *alpha, int *status, void *scratch,
                     void *H16, void *W16, int kind, bool tc, bool fp64, int *err, cudaStream_t st, bool keep_w32,
                     void *HH16) {
    // the tensor-core apply needs the 16-bit copy it writes beside W, and K <= 16, M <= 128;
    // it may leave the FP32 W out when only the copy is wanted
    const bool tc_apply = tc && kind != OUT_F32 && W16 && tc_apply_supported(g);
    if (tc_apply && !keep_w32) W = nullptr;
    if (kind == OUT_F16)
        return zf_build_t(g, R, H, W, alpha, status, scratch, (cf16 *)H16, (cf16 *)W16, phase, fp64, tc_apply, err,
                          st, (cf16 *)HH16);
    return zf_build_t(g, R, H, W, alpha, status, scratch, (cbf16 *)H16, (cbf16 *)W16, phase, fp64 || kind == OUT_F32,
                      tc_apply, err, st, (cbf16 *)HH16);
}

// ---------------------------------------------------------------------------
// out = Z X per (symbol, subcarrier), Z = G^{-1} = Y^H Y from the factor's lower-triangular
// Y = L^{-1} (FP32 scratch, [bin / 32][entry][bin % 32]): the precoder applied through its
// factors, W s = H^H (Z s) (Eq. 6 by associativity), and the adjoint side Z (H g).
// X, out [S][K][N_d].
//
// A CTA takes a 32-bin block: Y's block (contiguous, 16-byte cp.async) and the block's
// symbol vectors -- up to sc symbols of each bin's realisation at a time, one 8-byte
// cp.async per (symbol, user, bin), so blocks that straddle two realisations need no
// special case -- are staged in shared memory, then one thread per (bin, symbol) forms
// u = Y^H (Y x) row by row: row k of Y goes into registers once, gives
// w_k = sum_{j <= k} Y_kj x_j and is reused for u_j += conj(Y_kj) w_k, j <= k.  Lanes run
// along the bins, so every shared load of a warp is 32 consecutive entries and every
// store 32 consecutive subcarriers.  Up to K = 16 two CTAs share an SM: one stages while
// the other computes.
constexpr int ZM_SC = 14;   // symbols staged per pass at most (the benchmark's 14 per realisation)

// KM: the unrolled bound on K; EX: K == KM, compiled in (the run-time K otherwise costs
// every unrolled product a predicate: 12 % of the kernel's time at K = 16)
template <int KM, bool EX>
__global__ void __launch_bounds__(256, KM > 16 ? 1 : 2)
    zmul_kernel(Geo g, int S, long nbins, int sc_max, const c32 *__restrict__ Ys, const c32 *__restrict__ X,
                c32 *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int K = EX ? KM : g.K, T = tri(K), Nd = g.N_d, Sr = g.S_per_real;
    c32 *sY = reinterpret_cast<c32 *>(sm);   // [T][32]
    c32 *sX = sY + T * 32;                   // [sc_max][K][32]
    const long nblk = (nbins + 31) / 32;
    // blockDim is whole warps, so a thread's staged entries and tasks all belong to bin
    // (block, lane): its realisation and subcarrier are found once per block
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        __syncthreads();   // the previous block's shared reads are done
        const c32 *src = Ys + blk * (long)T * 32;
        for (int c = threadIdx.x; c < T * 16; c += blockDim.x) cp_async16(sY + 2 * c, src + 2 * c, true);
        const long b = blk * 32 + lane;
        const bool bok = b < nbins;
        const long r = bok ? b / Nd : 0;
        const int i = (int)(b - r * Nd);
        const long s0 = r * Sr;   // the realisation's first symbol
        for (int t0 = 0; t0 < Sr; t0 += sc_max) {
            const int sc = min(sc_max, Sr - t0);
            if (t0) __syncthreads();   // the previous symbols' shared reads are done
            // entry (t, u, lane) of the staged block: warp wid takes rows tu = wid, wid + nw, ...
            int t = wid / K, u = wid - (wid / K) * K;
            for (int tu = wid; tu < sc * K; tu += nw) {
                const long s = s0 + t0 + t;
                const bool ok = bok && s < S;
                cp_async8z(sX + tu * 32 + lane, ok ? X + (s * K + u) * Nd + i : X, ok);
                u += nw;
                while (u >= K) {
                    u -= K;
                    ++t;
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncthreads();
            for (int tt = wid; tt < sc; tt += nw) {   // task (lane's bin, symbol t0 + tt)
                const long s = s0 + t0 + tt;
                if (!bok || s >= S) continue;
                const c32 *xs = sX + tt * K * 32 + lane;
                c32 x[KM], uacc[KM];
#pragma unroll
                for (int j = 0; j < KM; ++j) {
                    x[j] = j < K ? xs[j * 32] : make_float2(0.f, 0.f);
                    uacc[j] = make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int k = 0; k < KM; ++k) {
                    if (k < K) {
                        c32 y[KM];
                        c32 w = make_float2(0.f, 0.f);
#pragma unroll
                        for (int j = 0; j <= k; ++j) {
                            y[j] = sY[(tri(k) + j) * 32 + lane];
                            w = cfma(y[j], x[j], w);
                        }
#pragma unroll
                        for (int j = 0; j <= k; ++j) uacc[j] = cfma(cconj(y[j]), w, uacc[j]);
                    }
                }
                c32 *os = out + s * K * Nd + i;
#pragma unroll
                for (int j = 0; j < KM; ++j)
                    if (j < K) os[(long)j * Nd] = uacc[j];
            }
        }
    }
}

template <int KM>
static cudaError_t launch_zmul(const Geo &g, int S, long nbins, const c32 *Ys, const c32 *X, c32 *out,
                               cudaStream_t st) {
    // symbols per pass: as many as fit beside Y in half (K <= 16) or all of the SM's shared memory
    const long budget = KM > 16 ? 200 * 1024 : 100 * 1024, ybytes = (long)sizeof(c32) * tri(g.K) * 32;
    int sc = (int)((budget - ybytes) / ((long)sizeof(c32) * g.K * 32));
    sc = sc < 1 ? 1 : sc > ZM_SC ? ZM_SC : sc;
    if (sc > g.S_per_real) sc = g.S_per_real;
    const size_t smem = (size_t)ybytes + sizeof(c32) * (size_t)sc * g.K * 32;
    const bool ex = g.K == KM;
    cudaError_t e = cudaFuncSetAttribute(zmul_kernel<KM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(zmul_kernel<KM, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // one thread per (bin, staged symbol) in as few rounds of at most 256 threads as fit,
    // whole warps (14 symbols: 224 threads, two rounds)
    const int rounds = (32 * sc + 255) / 256, threads = 32 * ((sc + rounds - 1) / rounds);
    long blocks = (long)resident_ctas(zmul_kernel<KM, false>, threads, smem) * sm_count();
    const long nblk = (nbins + 31) / 32;
    if (blocks > nblk) blocks = nblk;
    if (blocks < 1) blocks = 1;
    if (ex)
        zmul_kernel<KM, true><<<(unsigned)blocks, threads, smem, st>>>(g, S, nbins, sc, Ys, X, out);
    else
        zmul_kernel<KM, false><<<(unsigned)blocks, threads, smem, st>>>(g, S, nbins, sc, Ys, X, out);
    return cudaGetLastError();
}

cudaError_t zf_zmul(const Geo &g, int S, const void *scratch, const c32 *X, c32 *out, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    const long R = (S + g.S_per_real - 1) / g.S_per_real, nbins = R * g.N_d;
    const long nb32 = (nbins + 31) / 32 * 32;
    const c32 *Ys = reinterpret_cast<const c32 *>(reinterpret_cast<const char *>(scratch) +
                                                  al16(sizeof(c32) * (size_t)nb32 * tri(g.K)));
    if (g.K <= 4) return launch_zmul<4>(g, S, nbins, Ys, X, out, st);
    if (g.K <= 8) return launch_zmul<8>(g, S, nbins, Ys, X, out, st);
    if (g.K <= 16) return launch_zmul<16>(g, S, nbins, Ys, X, out, st);
    return launch_zmul<32>(g, S, nbins, Ys, X, out, st);
}

cudaError_t zf_build(const Geo &g, int R, const c32 *H, c32 *W, float *alpha, int *status, void *scratch,
                     void *H16, void *W16, int kind, cudaStream_t st) {
    return zf_phase(-1, g, R, H, W, alpha, status, scratch, H16, W16, kind, false, true, nullptr, st, true, nullptr);
}

}  // namespace fdk
