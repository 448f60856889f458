// Per-antenna OFDM modulation, PA and demodulation for every (symbol, antenna) row.
//
//   forward : x = IDFT_N(x_hat)  (Eq. 2, unitary, guard bins zero)
//             x^PA = PA_b(x)     (Eq. 7 with the memory polynomial of Eq. 9, G = 0,
//                                 taps circular in the N-sample symbol)
//             X = DFT_N(x^PA)    (unitary), keep the N_d data bins; accumulate the
//                                 guard- and data-bin power of X for the ACPR.
//   adjoint : g   = IDFT_N(gX)   (adjoint of the unitary DFT; guard bins of gX zero)
//             x   = IDFT_N(x_hat) recomputed, never stored
//             gx_n = sum_l A_l(x_n) g_{n+l} + B_l(x_n) conj(g_{n+l}),
//                    A_l = sum_p a_p(x) conj(c_{p,l}),  B_l = sum_p b_p(x) c_{p,l},
//                    a_p = (p+1)/2 |x|^{p-1}, b_p = (p-1)/2 x^2 |x|^{p-3}  (Wirtinger)
//             g_xhat = DFT_N(gx) on the data bins (adjoint of the unitary IDFT).
//
// A row is transformed by T = N/8 threads holding 8 points each: one radix-2/4 pass
// (when log2 N is not a multiple of 3) and radix-8 Stockham passes, ping-ponging
// between two padded shared buffers (one barrier per pass).  The pass structure is a
// template parameter, so every index is a compile-time expression, and each radix-8
// pass with span Ns reads its twiddles from its own table laid out [r][k] (k = the
// thread's position in the span), which consecutive threads read without bank
// conflicts.  The last pass of an inverse transform leaves thread t with samples
// t + q T (q = 0..7) -- the inputs of its first-pass butterflies of the next forward
// transform -- so the time-domain row stays in registers: the PA (or its adjoint) is
// applied there, its memory taps (samples n - l, or n + l for the adjoint) come from
// neighbouring lanes by warp shuffles and, across warp boundaries, from a small
// shared array.  CTAs are persistent.  All arithmetic is FP32.
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace fdk {

static constexpr float kSqrtHalf = 0.70710678118654752f;

FD_HD int pidx(int i) { return i + (i >> 3); }   // one pad word per 8 entries

template <bool INV> FD_D c32 mul_mi(c32 a) {      // a * (-i) forward, a * (+i) inverse
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
template <bool INV> FD_D c32 twmul(c32 v, c32 w) { return INV ? cmulc(v, w) : cmul(v, w); }

template <bool INV> FD_D void dft2(c32 *v) {
    c32 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}
template <bool INV> FD_D void dft4(c32 *v) {
    c32 a0 = cadd(v[0], v[2]), a2 = csub(v[0], v[2]);
    c32 a1 = cadd(v[1], v[3]), a3 = mul_mi<INV>(csub(v[1], v[3]));
    v[0] = cadd(a0, a1);
    v[2] = csub(a0, a1);
    v[1] = cadd(a2, a3);
    v[3] = csub(a2, a3);
}
template <bool INV> FD_D void dft8(c32 *v) {
    c32 e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    dft4<INV>(e);
    dft4<INV>(o);
    // W8^1 = (1 -/+ i)/sqrt2, W8^2 = -/+ i, W8^3 = (-1 -/+ i)/sqrt2
    c32 o1 = INV ? make_float2((o[1].x - o[1].y) * kSqrtHalf, (o[1].x + o[1].y) * kSqrtHalf)
                 : make_float2((o[1].x + o[1].y) * kSqrtHalf, (o[1].y - o[1].x) * kSqrtHalf);
    c32 o2 = mul_mi<INV>(o[2]);
    c32 o3 = INV ? make_float2(-(o[3].x + o[3].y) * kSqrtHalf, (o[3].x - o[3].y) * kSqrtHalf)
                 : make_float2((o[3].y - o[3].x) * kSqrtHalf, -(o[3].x + o[3].y) * kSqrtHalf);
    v[0] = cadd(e[0], o[0]); v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);   v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);   v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);   v[7] = csub(e[3], o3);
}

// Compile-time pass structure of an N = 2^LOG2N transform.
template <int LOG2N>
struct Fft {
    static constexpr int N = 1 << LOG2N, T = N / 8, PADN = N + N / 8;
    static constexpr int R0 = LOG2N % 3 == 0 ? 8 : (LOG2N % 3 == 1 ? 2 : 4);   // first pass radix
    static constexpr int LOGR0 = R0 == 8 ? 3 : (R0 == 2 ? 1 : 2);
    static constexpr int NP8 = (LOG2N - LOGR0) / 3;                           // radix-8 passes after it
    static constexpr int ns(int i) { return i == 0 ? 1 : R0 << (3 * (i - 1)); }   // span of pass i (1..NP8)
    static constexpr int tw_off(int i) {                                          // table offset of pass i >= 1
        int o = 0;
        for (int j = 1; j < i; ++j) o += 7 * ns(j);
        return o;
    }
    static constexpr int TW = tw_off(NP8 + 1);                                   // table entries
    static constexpr int pos(int b, int r) { return R0 == 8 ? r : (R0 == 4 ? b + 2 * r : b + 4 * r); }
};

// One transform.  in[q] holds input sample t + q T; on return out[q] holds output
// t + q T scaled by `scale`.  Uses bufA, bufB; returns after a barrier that lets the
// caller reuse both buffers only after its own next barrier (the last pass reads
// bufX without a trailing barrier).
template <int LOG2N, bool INV>
FD_D void transform(const c32 (&in)[8], c32 (&out)[8], c32 *bufA, c32 *bufB, const c32 *twp, int t, float scale) {
    using F = Fft<LOG2N>;
    c32 v[8];
    // ---- first pass, radix R0, span 1 (no twiddles) ----
    constexpr int B0 = 8 / F::R0;
#pragma unroll
    for (int b = 0; b < B0; ++b) {
#pragma unroll
        for (int r = 0; r < F::R0; ++r) v[b * F::R0 + r] = in[F::pos(b, r)];
        if (F::R0 == 2) dft2<INV>(v + 2 * b);
        else if (F::R0 == 4) dft4<INV>(v + 4 * b);
        else dft8<INV>(v);
        const int j = t + b * F::T;   // span 1: k = 0, base = j R0
#pragma unroll
        for (int q = 0; q < F::R0; ++q) bufA[pidx(j * F::R0 + q)] = v[b * F::R0 + q];
    }
    __syncthreads();
    c32 *src = bufA, *dst = bufB;
    // ---- radix-8 passes; the last one stays in registers ----
#pragma unroll
    for (int i = 1; i <= F::NP8; ++i) {
        const int Ns = F::ns(i);
        const int k = t & (Ns - 1);
#pragma unroll
        for (int r = 0; r < 8; ++r) v[r] = src[pidx(t + r * F::T)];
        const c32 *tw = twp + F::tw_off(i);
#pragma unroll
        for (int r = 1; r < 8; ++r) v[r] = twmul<INV>(v[r], tw[(r - 1) * Ns + k]);
        dft8<INV>(v);
        if (i == F::NP8) {   // Ns = N/8, k = t: outputs t + q T
#pragma unroll
            for (int q = 0; q < 8; ++q) out[q] = cscale(v[q], scale);
        } else {
            const int base = (t - k) * 8 + k;
#pragma unroll
            for (int q = 0; q < 8; ++q) dst[pidx(base + q * Ns)] = v[q];
            __syncthreads();
            c32 *tmp = src; src = dst; dst = tmp;
        }
    }
}

struct TapCtx {      // where the neighbours of thread t (row-local index) live
    int T, lane, t, wrow, nwarps_row, wbase;   // wbase: CTA warp index of the row's first warp
};

FD_D TapCtx tap_ctx(int T, int t, int grp) {
    TapCtx c;
    c.T = T;
    c.t = t;
    c.lane = threadIdx.x & 31;
    c.nwarps_row = T >= 32 ? T / 32 : 1;
    c.wrow = T >= 32 ? t / 32 : 0;
    c.wbase = T >= 32 ? grp * c.nwarps_row : 0;
    return c;
}

// Publish what other warps of the row need: for d < 0 the last D lanes of each warp,
// for d > 0 the first D lanes.  pub: [CTA warp][D][8] complex.
template <bool NEXT>
FD_D void publish(const TapCtx &c, const c32 (&v)[8], int D, c32 *pub) {
    if (c.T < 32 || D == 0) return;
    const int slot = NEXT ? c.lane : c.lane - (32 - D);
    if (slot >= 0 && slot < D) {
        const int w = c.wbase + c.wrow;
#pragma unroll
        for (int q = 0; q < 8; ++q) pub[(w * D + slot) * 8 + q] = v[q];
    }
}

// out[q] = v at sample (t + q T) + d of the same row (circular), |d| <= D.
// Every lane of the warp must call this with the same d.
FD_D void neighbour(const TapCtx &c, const c32 (&v)[8], int d, int D, const c32 *pub, c32 (&out)[8]) {
    int st = c.t + d, dq = 0;
    if (st < 0) { st += c.T; dq = -1; }
    else if (st >= c.T) { st -= c.T; dq = 1; }
    int src_lane;
    bool in_warp;
    if (c.T < 32) {
        src_lane = (c.lane - c.t) + st;
        in_warp = true;
    } else {
        src_lane = c.lane + d;
        in_warp = src_lane >= 0 && src_lane < 32;
    }
    const int sl = src_lane & 31;
    c32 tmp[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        tmp[q].x = __shfl_sync(0xffffffffu, v[q].x, sl);
        tmp[q].y = __shfl_sync(0xffffffffu, v[q].y, sl);
    }
    if (in_warp) {
#pragma unroll
        for (int q = 0; q < 8; ++q) out[q] = dq == 0 ? tmp[q] : (dq < 0 ? tmp[(q + 7) & 7] : tmp[(q + 1) & 7]);
    } else {
        const int wsrc = c.wbase + (d < 0 ? (c.wrow + c.nwarps_row - 1) % c.nwarps_row : (c.wrow + 1) % c.nwarps_row);
        const int slot = d < 0 ? (src_lane + 32) - (32 - D) : src_lane - 32;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int qs = dq == 0 ? q : (dq < 0 ? ((q + 7) & 7) : ((q + 1) & 7));
            out[q] = pub[(wsrc * D + slot) * 8 + qs];
        }
    }
}

// |x|^e from r2 = |x|^2 and mag = |x|
FD_D float powabs(float r2, float mag, int e) {
    float w = 1.0f;
    for (int q = 0; q + 1 < e; q += 2) w *= r2;
    if (e & 1) w *= mag;
    return w;
}

// PA shape: P_ > 0 means orders 1, 3, ..., 2 P_ - 1 and memory L_ (compile time);
// P_ == 0 is the general case (orders and memory from Geo at run time).
template <int P_, int L_>
struct PaShape {
    static constexpr bool fixed = P_ > 0;
};

template <int LOG2N, int P_, int L_>
struct FwdRow {
    // y_n = sum_l sum_p c_{p,l} x_{n-l} |x_{n-l}|^{p-1}
    static FD_D void pa(const Geo &g, const TapCtx &tc, const c32 (&x)[8], const c32 *cp, const c32 *pub, int D,
                        bool any_even, c32 (&y)[8]) {
        const int P = P_ > 0 ? P_ : g.n_orders;
        const int L = P_ > 0 ? L_ : g.L;
        const int L1 = L + 1;
#pragma unroll
        for (int q = 0; q < 8; ++q) y[q] = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l <= (P_ > 0 ? L_ : 7); ++l) {
            if (l > L) break;
            c32 xl[8];
            if (l == 0) {
#pragma unroll
                for (int q = 0; q < 8; ++q) xl[q] = x[q];
            } else {
                neighbour(tc, x, -l, D, pub, xl);
            }
            if (P_ > 0) {
                c32 c[P_ > 0 ? P_ : 1];
#pragma unroll
                for (int p = 0; p < P_; ++p) c[p] = cp[p * L1 + l];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float r2 = cabs2(xl[q]);
                    c32 phi = xl[q];
                    y[q] = cfma(c[0], phi, y[q]);
#pragma unroll
                    for (int p = 1; p < P_; ++p) {
                        phi = cscale(phi, r2);
                        y[q] = cfma(c[p], phi, y[q]);
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float r2 = cabs2(xl[q]);
                    const float mg = any_even ? sqrtf(r2) : 0.f;
                    for (int p = 0; p < P; ++p)
                        y[q] = cfma(cp[p * L1 + l], cscale(xl[q], powabs(r2, mg, g.orders[p] - 1)), y[q]);
                }
            }
        }
    }
    // gx_n = sum_l A_l g_{n+l} + B_l conj(g_{n+l})
    static FD_D void pa_adjoint(const Geo &g, const TapCtx &tc, const c32 (&x)[8], const c32 (&gv)[8],
                                const c32 *cp, const c32 *pub, int D, c32 (&gx)[8]) {
        const int P = P_ > 0 ? P_ : g.n_orders;
        const int L = P_ > 0 ? L_ : g.L;
        const int L1 = L + 1;
#pragma unroll
        for (int q = 0; q < 8; ++q) gx[q] = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l <= (P_ > 0 ? L_ : 7); ++l) {
            if (l > L) break;
            c32 gl[8];
            if (l == 0) {
#pragma unroll
                for (int q = 0; q < 8; ++q) gl[q] = gv[q];
            } else {
                neighbour(tc, gv, l, D, pub, gl);
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float r2 = cabs2(x[q]);
                const c32 xx = cmul(x[q], x[q]);
                c32 A = make_float2(0.f, 0.f), B = make_float2(0.f, 0.f);
                if (P_ > 0) {
                    // order 2k+1: a = (k+1) r2^k, b = k x^2 r2^(k-1)
                    float rk = 1.0f, rk1 = 0.0f;
#pragma unroll
                    for (int k = 0; k < P_; ++k) {
                        const c32 c = cp[k * L1 + l];
                        A = cadd(A, cscale(cconj(c), (float)(k + 1) * rk));
                        if (k >= 1) B = cfma(cscale(xx, (float)k * rk1), c, B);
                        rk1 = rk;
                        rk *= r2;
                    }
                } else {
                    const float mag = sqrtf(r2);
                    for (int p = 0; p < P; ++p) {
                        const int e = g.orders[p] - 1;
                        const float w = powabs(r2, mag, e);
                        const c32 c = cp[p * L1 + l];
                        A = cadd(A, cscale(cconj(c), 0.5f * (float)(e + 2) * w));
                        if (e >= 1 && mag > 0.0f) B = cfma(cscale(xx, 0.5f * (float)e * w / r2), c, B);
                    }
                }
                gx[q] = cfma(A, gl[q], gx[q]);
                gx[q] = cfma(B, cconj(gl[q]), gx[q]);
            }
        }
    }
};

template <int LOG2N>
FD_HD constexpr int rows_per_cta_t() { return LOG2N >= 11 ? 1 : (1 << (11 - LOG2N)); }

inline int rows_per_cta(int N) { return N >= 2048 ? 1 : 2048 / N; }

// smem: per-pass twiddles, 2 buffers per row, coefficients per row, boundary array
inline size_t fftpa_smem_bytes_(const Geo &g) {
    const int N = g.N, padN = N + (N >> 3), r = rows_per_cta(N);
    const int T = N >> 3, nw = (r * T + 31) / 32, D = g.L > 0 ? g.L : 1;
    return sizeof(c32) * ((size_t)N + 2 * (size_t)r * padN + (size_t)r * g.n_orders * (g.L + 1) + (size_t)nw * D * 8);
}

template <int LOG2N, int P_, int L_, typename TOut>
__global__ void __launch_bounds__(LOG2N == 12 ? 512 : 256, LOG2N == 12 ? 1 : 2) fftpa_forward_kernel(
    Geo g, long rows, const c32 *__restrict__ xh, const c32 *__restrict__ pa, const c32 *__restrict__ twp_g,
    TOut *__restrict__ Xout, double *__restrict__ metrics) {
    using F = Fft<LOG2N>;
    constexpr int RPC = rows_per_cta_t<LOG2N>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int grp = threadIdx.x / F::T, t = threadIdx.x % F::T;
    const int P = P_ > 0 ? P_ : g.n_orders, L = P_ > 0 ? L_ : g.L, PL = P * (L + 1), D = L > 0 ? L : 1;
    c32 *twp = reinterpret_cast<c32 *>(smem_raw);
    c32 *bufA = twp + F::N + grp * 2 * F::PADN;
    c32 *bufB = bufA + F::PADN;
    c32 *coef = twp + F::N + RPC * 2 * F::PADN;
    c32 *pub = coef + RPC * PL;
    __shared__ double red[32];
    for (int i = threadIdx.x; i < F::TW; i += blockDim.x) twp[i] = twp_g[i];
    const TapCtx tc = tap_ctx(F::T, t, grp);
    bool any_even = false;
    for (int p = 0; p < P; ++p) any_even |= !(g.orders[p] & 1);
    const float rs = rsqrtf((float)F::N);
    double gpow = 0, dpow = 0;
    const long ngroups = (rows + RPC - 1) / RPC;

    for (long grp0 = blockIdx.x; grp0 < ngroups; grp0 += gridDim.x) {
        const long row = grp0 * RPC + grp;
        const bool active = row < rows;
        const long rowc = active ? row : 0;
        const int m = (int)(rowc % g.M);
        __syncthreads();   // the previous row is done with coef, pub and both buffers
        c32 *cp = coef + grp * PL;
        for (int i = t; i < PL; i += F::T) cp[i] = pa[(long)m * PL + i];
        const c32 *xrow = xh + rowc * g.N_d;
        c32 in[8], x[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = data_index(t + q * F::T, g.first_bin, F::N, g.N_d);
            in[q] = (active && i >= 0) ? xrow[i] : make_float2(0.f, 0.f);
        }
        transform<LOG2N, true>(in, x, bufA, bufB, twp, t, rs);
        publish<false>(tc, x, D, pub);
        __syncthreads();
        c32 y[8];
        FwdRow<LOG2N, P_, L_>::pa(g, tc, x, cp, pub, D, any_even, y);
        c32 v[8];
        transform<LOG2N, false>(y, v, bufA, bufB, twp, t, rs);
        TOut *orow = Xout + rowc * g.N_d;
        float gp = 0.f, dp = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = data_index(t + q * F::T, g.first_bin, F::N, g.N_d);
            const float p2 = cabs2(v[q]);
            if (i >= 0) {
                dp += p2;
                if (active) orow[i] = Operand<TOut>::from(v[q]);
            } else {
                gp += p2;
            }
        }
        if (active) {
            gpow += gp;
            dpow += dp;
        }
    }
    if (metrics) {
        const double gs = block_sum(gpow, red);
        const double ds = block_sum(dpow, red);
        if (threadIdx.x == 0) {
            atomicAdd(metrics + 3, gs);
            atomicAdd(metrics + 4, ds);
        }
    }
}

template <int LOG2N, int P_, int L_, typename TIn>
__global__ void __launch_bounds__(LOG2N == 12 ? 512 : 256, LOG2N == 12 ? 1 : 2) fftpa_adjoint_kernel(
    Geo g, long rows, const c32 *__restrict__ xh, const c32 *__restrict__ pa, const c32 *__restrict__ twp_g,
    const TIn *gX, c32 *gxh) {
    using F = Fft<LOG2N>;
    constexpr int RPC = rows_per_cta_t<LOG2N>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int grp = threadIdx.x / F::T, t = threadIdx.x % F::T;
    const int P = P_ > 0 ? P_ : g.n_orders, L = P_ > 0 ? L_ : g.L, PL = P * (L + 1), D = L > 0 ? L : 1;
    c32 *twp = reinterpret_cast<c32 *>(smem_raw);
    c32 *bufA = twp + F::N + grp * 2 * F::PADN;
    c32 *bufB = bufA + F::PADN;
    c32 *coef = twp + F::N + RPC * 2 * F::PADN;
    c32 *pub = coef + RPC * PL;
    for (int i = threadIdx.x; i < F::TW; i += blockDim.x) twp[i] = twp_g[i];
    const TapCtx tc = tap_ctx(F::T, t, grp);
    const float rs = rsqrtf((float)F::N);
    const long ngroups = (rows + RPC - 1) / RPC;

    for (long grp0 = blockIdx.x; grp0 < ngroups; grp0 += gridDim.x) {
        const long row = grp0 * RPC + grp;
        const bool active = row < rows;
        const long rowc = active ? row : 0;
        const int m = (int)(rowc % g.M);
        __syncthreads();
        c32 *cp = coef + grp * PL;
        for (int i = t; i < PL; i += F::T) cp[i] = pa[(long)m * PL + i];
        const c32 *xrow = xh + rowc * g.N_d;
        const TIn *grow = gX + rowc * g.N_d;
        c32 in[8], x[8], gv[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = data_index(t + q * F::T, g.first_bin, F::N, g.N_d);
            in[q] = (active && i >= 0) ? xrow[i] : make_float2(0.f, 0.f);
        }
        transform<LOG2N, true>(in, x, bufA, bufB, twp, t, rs);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = data_index(t + q * F::T, g.first_bin, F::N, g.N_d);
            in[q] = (active && i >= 0) ? Operand<TIn>::load(grow + i) : make_float2(0.f, 0.f);
        }
        __syncthreads();   // the first transform's last pass has read its buffer
        transform<LOG2N, true>(in, gv, bufA, bufB, twp, t, rs);
        publish<true>(tc, gv, D, pub);
        __syncthreads();
        c32 gx[8];
        FwdRow<LOG2N, P_, L_>::pa_adjoint(g, tc, x, gv, cp, pub, D, gx);
        c32 v[8];
        transform<LOG2N, false>(gx, v, bufA, bufB, twp, t, rs);
        if (active) {
            c32 *orow = gxh + row * g.N_d;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int i = data_index(t + q * F::T, g.first_bin, F::N, g.N_d);
                if (i >= 0) orow[i] = v[q];
            }
        }
    }
}

template <class Kern>
inline cudaError_t persistent_blocks(Kern k, int N, long rows, int threads, size_t sm, long &blocks) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, sm);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int r = rows_per_cta(N);
    const long groups = (rows + r - 1) / r;
    blocks = (long)(per_sm > 0 ? per_sm : 1) * sms;
    if (blocks > groups) blocks = groups;
    return cudaSuccess;
}

template <int LOG2N, int P_, int L_, typename TOut>
inline cudaError_t fwd_t(const Geo &g, long rows, const c32 *xh, const c32 *pa, const c32 *twp, TOut *X,
                         double *metrics, cudaStream_t st) {
    const int threads = rows_per_cta(g.N) * (g.N >> 3);
    const size_t sm = fftpa_smem_bytes_(g);
    long blocks = 0;
    cudaError_t e = persistent_blocks(fftpa_forward_kernel<LOG2N, P_, L_, TOut>, g.N, rows, threads, sm, blocks);
    if (e != cudaSuccess) return e;
    fftpa_forward_kernel<LOG2N, P_, L_, TOut><<<(unsigned)blocks, threads, sm, st>>>(g, rows, xh, pa, twp, X, metrics);
    return cudaGetLastError();
}

template <int LOG2N, int P_, int L_>
inline cudaError_t adj_t(const Geo &g, long rows, const c32 *xh, const c32 *pa, const c32 *twp, const c32 *gX,
                         c32 *gxh, cudaStream_t st) {
    const int threads = rows_per_cta(g.N) * (g.N >> 3);
    const size_t sm = fftpa_smem_bytes_(g);
    long blocks = 0;
    cudaError_t e = persistent_blocks(fftpa_adjoint_kernel<LOG2N, P_, L_, c32>, g.N, rows, threads, sm, blocks);
    if (e != cudaSuccess) return e;
    fftpa_adjoint_kernel<LOG2N, P_, L_, c32><<<(unsigned)blocks, threads, sm, st>>>(g, rows, xh, pa, twp, gX, gxh);
    return cudaGetLastError();
}

// PA shapes with a compiled fast path: orders 1,3,5 with taps 0..3, orders 1,3 with
// taps 0..3, and the memoryless 1,3.  Anything else takes the general path.
inline int pa_shape(const Geo &g) {
    for (int p = 0; p < g.n_orders; ++p)
        if (g.orders[p] != 2 * p + 1) return 0;
    if (g.n_orders == 3 && g.L == 3) return 1;
    if (g.n_orders == 2 && g.L == 3) return 2;
    if (g.n_orders == 2 && g.L == 0) return 3;
    return 0;
}

template <int LOG2N, typename TOut>
inline cudaError_t fwd_n(const Geo &g, long rows, const c32 *xh, const c32 *pa, const c32 *twp, TOut *X,
                         double *metrics, cudaStream_t st) {
    switch (pa_shape(g)) {
        case 1: return fwd_t<LOG2N, 3, 3>(g, rows, xh, pa, twp, X, metrics, st);
        case 2: return fwd_t<LOG2N, 2, 3>(g, rows, xh, pa, twp, X, metrics, st);
        case 3: return fwd_t<LOG2N, 2, 0>(g, rows, xh, pa, twp, X, metrics, st);
        default: return fwd_t<LOG2N, 0, 0>(g, rows, xh, pa, twp, X, metrics, st);
    }
}

template <int LOG2N>
inline cudaError_t adj_n(const Geo &g, long rows, const c32 *xh, const c32 *pa, const c32 *twp, const c32 *gX,
                         c32 *gxh, cudaStream_t st) {
    switch (pa_shape(g)) {
        case 1: return adj_t<LOG2N, 3, 3>(g, rows, xh, pa, twp, gX, gxh, st);
        case 2: return adj_t<LOG2N, 2, 3>(g, rows, xh, pa, twp, gX, gxh, st);
        case 3: return adj_t<LOG2N, 2, 0>(g, rows, xh, pa, twp, gX, gxh, st);
        default: return adj_t<LOG2N, 0, 0>(g, rows, xh, pa, twp, gX, gxh, st);
    }
}


// One translation unit per transform size instantiates these.
#define FD_FFTPA_SIZE(LOG2N)                                                                                      \
    cudaError_t fftpa_fwd_##LOG2N(const Geo &g, long rows, const c32 *xh, const c32 *pa, const c32 *twp, c32 *X, \
                                  double *metrics, cudaStream_t st) {                                            \
        return fwd_n<LOG2N>(g, rows, xh, pa, twp, X, metrics, st);                                               \
    }                                                                                                            \
    cudaError_t fftpa_adj_##LOG2N(const Geo &g, long rows, const c32 *xh, const c32 *pa, const c32 *twp,         \
                                  const c32 *gX, c32 *gxh, cudaStream_t st) {                                    \
        return adj_n<LOG2N>(g, rows, xh, pa, twp, gX, gxh, st);                                                  \
    }

#define FD_FFTPA_DECL(LOG2N)                                                                                      \
    cudaError_t fftpa_fwd_##LOG2N(const Geo &g, long rows, const c32 *xh, const c32 *pa, const c32 *twp, c32 *X, \
                                  double *metrics, cudaStream_t st);                                             \
    cudaError_t fftpa_adj_##LOG2N(const Geo &g, long rows, const c32 *xh, const c32 *pa, const c32 *twp,         \
                                  const c32 *gX, c32 *gxh, cudaStream_t st);
FD_FFTPA_DECL(6) FD_FFTPA_DECL(7) FD_FFTPA_DECL(8) FD_FFTPA_DECL(9) FD_FFTPA_DECL(10) FD_FFTPA_DECL(11) FD_FFTPA_DECL(12)

}  // namespace fdk
