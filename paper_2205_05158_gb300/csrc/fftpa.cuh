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
// A row is transformed by T = N/16 threads holding 16 points each: one radix-2/4/8/16
// pass (absorbing log2 N mod 4) and radix-16 Stockham passes (a 16-point DFT is two
// radix-4 layers in registers), ping-ponging between two shared buffers indexed
// i + i/16, which keeps every store pattern of N = 256..4096 free of bank conflicts.
// The pass structure is a template parameter; each radix-16 pass with span Ns reads its
// twiddles from its own table laid out [r][k].  The last pass of an inverse transform
// leaves thread t with samples t + q T (q = 0..15) -- exactly the inputs of its first-pass
// butterflies of the next forward transform -- so the row is transformed back in
// registers after the PA.  The PA (or its adjoint) reads the memory taps (samples n - l,
// or n + l) from a natural-order copy of the row in shared memory.  CTAs are persistent.
// All arithmetic is FP32.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace fdk {

static constexpr float kSqrtHalf = 0.70710678118654752f;
static constexpr float kCos8 = 0.92387953251128676f;   // cos(pi/8)
static constexpr float kSin8 = 0.38268343236508977f;   // sin(pi/8)

FD_HD int pidx(int i) { return i + (i >> 4); }   // one pad word per 16 entries

// cp.async of 4, 8 or 16 bytes (the row inputs of the next row group, staged in shared memory)
template <int BYTES> FD_D void cp_async_n(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src),
                 "n"(BYTES)
                 : "memory");
}
FD_D void cp_async_commit_all() { asm volatile("cp.async.commit_group;" ::: "memory"); }
FD_D void cp_async_wait_none() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Sum and difference of complex values as one packed FP32-pair instruction each
// (add / sub .f32x2, sm_100 and later): the same IEEE results as two scalar adds.
FD_D c32 padd(c32 a, c32 b) {
    c32 r;
    asm("{.reg .b64 x, y, z;\n\tmov.b64 x, {%2, %3};\n\tmov.b64 y, {%4, %5};\n\tadd.rn.f32x2 z, x, y;\n\t"
        "mov.b64 {%0, %1}, z;}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
FD_D c32 psub(c32 a, c32 b) {
    c32 r;
    asm("{.reg .b64 x, y, z;\n\tmov.b64 x, {%2, %3};\n\tmov.b64 y, {%4, %5};\n\tsub.rn.f32x2 z, x, y;\n\t"
        "mov.b64 {%0, %1}, z;}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

template <bool INV> FD_D c32 mul_mi(c32 a) {      // a * (-i) forward, a * (+i) inverse
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
template <bool INV> FD_D c32 twmul(c32 v, c32 w) { return INV ? cmulc(v, w) : cmul(v, w); }

// a * W16^m, W16 = exp(-/+ j 2 pi / 16), for the constant m used inside dft16
template <bool INV, int MM> FD_D c32 w16(c32 a) {
    constexpr int m = MM & 15;
    if (m == 0) return a;
    if (m == 4) return mul_mi<INV>(a);
    if (m == 8) return make_float2(-a.x, -a.y);
    const float sg = INV ? 1.f : -1.f;   // exp(sg j pi m / 8)
    float c, s;
    switch (m) {
        case 1: c = kCos8; s = kSin8; break;
        case 2: c = kSqrtHalf; s = kSqrtHalf; break;
        case 3: c = kSin8; s = kCos8; break;
        case 6: c = -kSqrtHalf; s = kSqrtHalf; break;
        case 9: c = -kCos8; s = -kSin8; break;
        default: c = 1.f; s = 0.f; break;
    }
    s *= sg;
    return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
}

template <bool INV> FD_D void dft2(c32 *v) {
    c32 a = v[0], b = v[1];
    v[0] = padd(a, b);
    v[1] = psub(a, b);
}
template <bool INV> FD_D void dft4s(c32 &x0, c32 &x1, c32 &x2, c32 &x3) {
    c32 a0 = padd(x0, x2), a2 = psub(x0, x2);
    c32 a1 = padd(x1, x3), a3 = mul_mi<INV>(psub(x1, x3));
    x0 = padd(a0, a1);
    x2 = psub(a0, a1);
    x1 = cadd(a2, a3);   // a3 is a swapped pair: two scalar adds
    x3 = csub(a2, a3);
}
template <bool INV> FD_D void dft4(c32 *v) { dft4s<INV>(v[0], v[1], v[2], v[3]); }
template <bool INV> FD_D void dft8(c32 *v) {
    c32 e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    dft4<INV>(e);
    dft4<INV>(o);
    c32 o1 = w16<INV, 2>(o[1]), o2 = w16<INV, 4>(o[2]), o3 = w16<INV, 6>(o[3]);
    v[0] = padd(e[0], o[0]); v[4] = psub(e[0], o[0]);
    v[1] = padd(e[1], o1);   v[5] = psub(e[1], o1);
    v[2] = padd(e[2], o2);   v[6] = psub(e[2], o2);
    v[3] = padd(e[3], o3);   v[7] = psub(e[3], o3);
}
// 16-point DFT, natural order in and out: n = 4 n1 + n2, k = k1 + 4 k2.
template <bool INV> FD_D void dft16(c32 *v) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4s<INV>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);   // over n1 -> k1
    // v[4 k1 + n2] now holds A[n2][k1]; twiddle W16^(n2 k1)
    v[5] = w16<INV, 1>(v[5]);   v[6] = w16<INV, 2>(v[6]);   v[7] = w16<INV, 3>(v[7]);
    v[9] = w16<INV, 2>(v[9]);   v[10] = w16<INV, 4>(v[10]); v[11] = w16<INV, 6>(v[11]);
    v[13] = w16<INV, 3>(v[13]); v[14] = w16<INV, 6>(v[14]); v[15] = w16<INV, 9>(v[15]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4s<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);   // over n2 -> k2
    // v[4 k1 + k2] holds X[k1 + 4 k2]: transpose the 4 x 4 block into natural order
    c32 t[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) t[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = t[i];
}

template <int R, bool INV> FD_D void dftR(c32 *v) {
    if (R == 2) dft2<INV>(v);
    else if (R == 4) dft4<INV>(v);
    else if (R == 8) dft8<INV>(v);
    else dft16<INV>(v);
}

// Compile-time pass structure of an N = 2^LOG2N transform.
template <int LOG2N>
struct Fft {
    static constexpr int N = 1 << LOG2N, T = N / 16, PADN = N + N / 16;
    static constexpr int LOGR0 = LOG2N % 4 == 0 ? 4 : LOG2N % 4;
    static constexpr int R0 = 1 << LOGR0;                      // first pass radix
    static constexpr int NP = (LOG2N - LOGR0) / 4;             // radix-16 passes after it
    static constexpr int ns(int i) { return R0 << (4 * (i - 1)); }   // span of pass i (1..NP)
    static constexpr int tw_off(int i) {
        int o = 0;
        for (int j = 1; j < i; ++j) o += 15 * ns(j);
        return o;
    }
    static constexpr int TW = tw_off(NP + 1);
    // first pass: butterfly b (0..16/R0-1) input r holds sample t + pos(b, r) T
    static constexpr int pos(int b, int r) { return b + r * (16 / R0); }
};

// One transform in place: x[q] is input sample t + q T; on return output t + q T,
// scaled.  The last pass reads a buffer with no barrier after it: the caller must
// barrier before either buffer is written again.
template <int LOG2N, bool INV>
FD_D void transform(c32 (&x)[16], c32 *bufA, c32 *bufB, const c32 *twp, int t, float scale) {
    using F = Fft<LOG2N>;
    constexpr int B0 = 16 / F::R0;
    c32 v[16];
#pragma unroll
    for (int b = 0; b < B0; ++b) {
#pragma unroll
        for (int r = 0; r < F::R0; ++r) v[b * F::R0 + r] = x[F::pos(b, r)];
        dftR<F::R0, INV>(v + b * F::R0);
        const int j = t + b * F::T;   // span 1: outputs j R0 + q
#pragma unroll
        for (int q = 0; q < F::R0; ++q) bufA[pidx(j * F::R0 + q)] = v[b * F::R0 + q];
    }
    __syncthreads();
    c32 *src = bufA, *dst = bufB;
#pragma unroll
    for (int i = 1; i <= F::NP; ++i) {
        const int Ns = F::ns(i);
        const int k = t & (Ns - 1);
        if constexpr ((F::T & 15) == 0) {   // pidx(t + r T) = pidx(t) + r (T + T / 16)
            const c32 *s0 = src + pidx(t);
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = s0[r * (F::T + F::T / 16)];
        } else {
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = src[pidx(t + r * F::T)];
        }
        const c32 *tw = twp + F::tw_off(i);
#pragma unroll
        for (int r = 1; r < 16; ++r) v[r] = twmul<INV>(v[r], tw[(r - 1) * Ns + k]);
        dft16<INV>(v);
        if (i == F::NP) {   // Ns = N/16, k = t: outputs t + q T
#pragma unroll
            for (int q = 0; q < 16; ++q) x[q] = cscale(v[q], scale);
        } else {
            const int base = (t - k) * 16 + k;
#pragma unroll
            for (int q = 0; q < 16; ++q) dst[pidx(base + q * Ns)] = v[q];
            __syncthreads();
            c32 *tmp = src; src = dst; dst = tmp;
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
struct RowPa {
    // y_n = sum_l sum_p c_{p,l} x_{n-l} |x_{n-l}|^{p-1}; xs holds the row in natural order.
    // With odd orders 2k+1 each tap is x * poly_l(|x|^2), poly_l(r) = sum_k c_{k,l} r^k,
    // evaluated by Horner's rule in the real variable r.
    static FD_D void forward(const Geo &g, int N, int T, int t, const c32 (&x)[16], const c32 *xs, const c32 *cp,
                             bool any_even, c32 (&y)[16]) {
        const int P = P_ > 0 ? P_ : g.n_orders;
        const int L = P_ > 0 ? L_ : g.L;
        const int L1 = L + 1;
#pragma unroll
        for (int q = 0; q < 16; ++q) y[q] = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l <= (P_ > 0 ? L_ : 7); ++l) {
            if (l > L) break;
            c32 c[P_ > 0 ? P_ : 1];
            if (P_ > 0) {
#pragma unroll
                for (int p = 0; p < (P_ > 0 ? P_ : 1); ++p) c[p] = cp[p * L1 + l];
            }
            // tap n - l of sample n = t + q T: with T a multiple of 16, pidx(i + q T) =
            // pidx(i) + q (T + T / 16), so one base per tap and constant offsets; only q = 0
            // can wrap around the row
            const int stepq = T + (T >> 4);
            const c32 *tap_q1 = xs + pidx(t - l + T) - stepq;   // + q stepq for q >= 1
            const c32 *tap_q0 = xs + pidx((t - l) & (N - 1));
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const c32 xl = l == 0 ? x[q]
                                      : ((T & 15) == 0 ? (q == 0 ? *tap_q0 : tap_q1[q * stepq])
                                                       : xs[pidx((t + q * T - l) & (N - 1))]);
                const float r2 = cabs2(xl);
                if (P_ > 0) {
                    c32 poly = c[(P_ > 0 ? P_ : 1) - 1];
#pragma unroll
                    for (int p = (P_ > 0 ? P_ : 1) - 2; p >= 0; --p)
                        poly = make_float2(fmaf(poly.x, r2, c[p].x), fmaf(poly.y, r2, c[p].y));
                    y[q] = cfma(xl, poly, y[q]);
                } else if (g.orders[0] == 0) {   // linear clipping (L = 0): x min(1, A / |x|), A = Re c
                    const float A = cp[0].x, mg = sqrtf(r2);
                    y[q] = mg > A ? cscale(xl, A / mg) : xl;
                } else {
                    const float mg = any_even ? sqrtf(r2) : 0.f;
                    for (int p = 0; p < P; ++p)
                        y[q] = cfma(cp[p * L1 + l], cscale(xl, powabs(r2, mg, g.orders[p] - 1)), y[q]);
                    // cross terms of Eq. 9 (P_ < 0 only): x_{n-l} times the envelope of
                    // x_{n-l-g} (lagging, b) and of x_{n-l+g} (leading, c), orders p >= 2
                    const int Gx = P_ < 0 ? g.pa_G : 0, PL1 = P * L1;
                    for (int gg = 1; gg <= Gx; ++gg) {
                        const int n = t + q * T;
                        const c32 xa = xs[pidx((n - l - gg) & (N - 1))], xb = xs[pidx((n - l + gg) & (N - 1))];
                        const float ra = cabs2(xa), rb = cabs2(xb), ma = sqrtf(ra), mb = sqrtf(rb);
                        c32 env = make_float2(0.f, 0.f);
                        for (int p = 0; p < P; ++p) {
                            const int e = g.orders[p] - 1;
                            if (e < 1) continue;
                            const int k = (p * L1 + l) * Gx + gg - 1;
                            env = cfma(cp[PL1 + k], make_float2(powabs(ra, ma, e), 0.f), env);
                            env = cfma(cp[PL1 + PL1 * Gx + k], make_float2(powabs(rb, mb, e), 0.f), env);
                        }
                        y[q] = cfma(xl, env, y[q]);
                    }
                }
            }
        }
    }
    // gx_n = sum_l A_l(x_n) g_{n+l} + B_l(x_n) conj(g_{n+l}); gs holds g in natural order
    // and gx the thread's own samples of g on entry (tap 0 of the compiled shapes), the
    // gradient on return; xs: x in natural order (read by the cross terms of the general
    // path only)
    static FD_D void adjoint(const Geo &g, int N, int T, int t, const c32 (&x)[16], const c32 *gs, const c32 *cp,
                             c32 (&gx)[16], const c32 *xs) {
        if constexpr (P_ > 0) {
            // odd orders 2k+1, k < P_, r = |x_n|^2:
            //   sum_l A_l g_{n+l} = sum_k (k+1) r^k G_k(n),  G_k(n) = sum_l conj(c_{k,l}) g_{n+l}
            //   sum_l B_l conj(g_{n+l}) = x_n^2 sum_{k>=1} k r^(k-1) conj(G_k(n))
            // (the B sums are the conjugates of the same tap sums), so each sample takes
            // P_ four-tap filters of g and two Horner evaluations in r
            constexpr int L1 = L_ + 1;
            c32 cc[P_][L1];   // conj(c_{k,l})
#pragma unroll
            for (int k = 0; k < P_; ++k)
#pragma unroll
                for (int l = 0; l < L1; ++l) cc[k][l] = cconj(cp[k * L1 + l]);
            // sample n + l of n = t + q T: one base per tap (T a multiple of 16), only q = 15
            // can wrap around the row
            const int stepq = T + (T >> 4);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                c32 G[P_];   // tap l = 0 is this thread's own sample, gx[q] on entry
#pragma unroll
                for (int k = 0; k < P_; ++k) G[k] = cmul(cc[k][0], gx[q]);
#pragma unroll
                for (int l = 1; l < L1; ++l) {
                    const c32 gl = ((T & 15) == 0 && q < 15) ? gs[pidx(t + l) + q * stepq]
                                                             : gs[pidx((t + q * T + l) & (N - 1))];
#pragma unroll
                    for (int k = 0; k < P_; ++k) G[k] = cfma(cc[k][l], gl, G[k]);
                }
                const float r2 = cabs2(x[q]);
                c32 A = cscale(G[P_ - 1], (float)P_);
#pragma unroll
                for (int k = P_ - 2; k >= 0; --k)
                    A = make_float2(fmaf(A.x, r2, (float)(k + 1) * G[k].x), fmaf(A.y, r2, (float)(k + 1) * G[k].y));
                if (P_ >= 2) {
                    c32 Bs = cscale(cconj(G[P_ - 1]), (float)(P_ - 1));
#pragma unroll
                    for (int k = P_ - 2; k >= 1; --k)
                        Bs = make_float2(fmaf(Bs.x, r2, (float)k * G[k].x), fmaf(Bs.y, r2, -(float)k * G[k].y));
                    A = cfma(cmul(x[q], x[q]), Bs, A);
                }
                gx[q] = A;
            }
        } else if (g.orders[0] == 0) {
            // linear clipping: above A, d y / d x = A / (2 |x|), d y / d x* = -A x^2 / (2 |x|^3)
            const float A = cp[0].x;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const c32 gl = gs[pidx((t + q * T) & (N - 1))];
                const float r2 = cabs2(x[q]), mg = sqrtf(r2);
                gx[q] = mg > A ? cfma(cscale(cmul(x[q], x[q]), -A / (2.0f * mg * r2)), cconj(gl), cscale(gl, A / (2.0f * mg)))
                               : gl;
            }
        } else {
            const int P = g.n_orders, L = g.L, L1 = L + 1;
#pragma unroll
            for (int q = 0; q < 16; ++q) gx[q] = make_float2(0.f, 0.f);
            for (int l = 0; l <= L; ++l) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const c32 gl = gs[pidx((t + q * T + l) & (N - 1))];
                    const float r2 = cabs2(x[q]);
                    const c32 xx = cmul(x[q], x[q]);
                    c32 A = make_float2(0.f, 0.f), B = make_float2(0.f, 0.f);
                    const float mag = sqrtf(r2);
                    for (int p = 0; p < P; ++p) {
                        const int e = g.orders[p] - 1;
                        const float w = powabs(r2, mag, e);
                        const c32 c = cp[p * L1 + l];
                        A = cadd(A, cscale(cconj(c), 0.5f * (float)(e + 2) * w));
                        if (e >= 1 && mag > 0.0f) B = cfma(cscale(xx, 0.5f * (float)e * w / r2), c, B);
                    }
                    gx[q] = cfma(A, gl, gx[q]);
                    gx[q] = cfma(B, cconj(gl), gx[q]);
                }
            }
            // cross terms T = b x_j e(x_i), e = |x_i|^E, i = j -+ g (lagging b, leading c):
            // as the signal x_j (output j + l): conj(b e(x_i)) g; as the envelope sample x_i
            // (de/dx = E/2 |x|^{E-2} x*): E/2 |x_i|^{E-2} (conj(b x_j) x_i g + b x_j x_i conj(g))
            if constexpr (P_ < 0) {
            const int Gx = g.pa_G, PL1 = P * L1;
            for (int gg = 1; gg <= Gx; ++gg)
                for (int l = 0; l <= L; ++l)
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int n = t + q * T;
                        const c32 xn = x[q];
                        const float rn = cabs2(xn), mn = sqrtf(rn);
                        const c32 g0 = gs[pidx((n + l) & (N - 1))];               // n as the signal sample
                        const c32 xa = xs[pidx((n - gg) & (N - 1))], xb = xs[pidx((n + gg) & (N - 1))];
                        const float ra = cabs2(xa), rb = cabs2(xb), ma = sqrtf(ra), mb = sqrtf(rb);
                        const c32 xj1 = xs[pidx((n + gg) & (N - 1))], g1 = gs[pidx((n + gg + l) & (N - 1))];
                        const c32 xj2 = xs[pidx((n - gg) & (N - 1))], g2 = gs[pidx((n - gg + l) & (N - 1))];
                        for (int p = 0; p < P; ++p) {
                            const int e = g.orders[p] - 1;
                            if (e < 1) continue;
                            const int k = (p * L1 + l) * Gx + gg - 1;
                            const c32 b = cp[PL1 + k], c = cp[PL1 + PL1 * Gx + k];
                            // signal: envelopes at n - g (b) and n + g (c)
                            gx[q] = cfma(cconj(cadd(cscale(b, powabs(ra, ma, e)), cscale(c, powabs(rb, mb, e)))), g0,
                                         gx[q]);
                            if (mn > 0.f) {
                                const float h = 0.5f * (float)e * powabs(rn, mn, e) / rn;   // E/2 |x_n|^{E-2}
                                // envelope of the lagging term of signal j = n + g (output n + g + l)
                                const c32 bx1 = cmul(b, xj1), cx2 = cmul(c, xj2);
                                gx[q] = cfma(cscale(cmul(cconj(bx1), xn), h), g1, gx[q]);
                                gx[q] = cfma(cscale(cmul(bx1, xn), h), cconj(g1), gx[q]);
                                // envelope of the leading term of signal j = n - g (output n - g + l)
                                gx[q] = cfma(cscale(cmul(cconj(cx2), xn), h), g2, gx[q]);
                                gx[q] = cfma(cscale(cmul(cx2, xn), h), cconj(g2), gx[q]);
                            }
                        }
                    }
            }
        }
    }
};

template <int LOG2N>
FD_HD constexpr int rows_per_cta_t() { return LOG2N >= 12 ? 1 : (1 << (12 - LOG2N)); }

FD_HD int rows_per_cta(int N) { return N >= 4096 ? 1 : 4096 / N; }

// PA coefficients of one antenna: the memory polynomial [P][L+1], then with cross terms
// (Eq. 9) the lagging [P][L+1][G] and the leading [P][L+1][G]
FD_HD int pa_coef_count(const Geo &g) { return g.n_orders * (g.L + 1) * (1 + 2 * g.pa_G); }

// smem: per-pass twiddles, 2 buffers per row, two sets of coefficients per row (this row
// group's and the next one's, in flight), then the staging of the next row group's inputs
// (stage_bytes per row)
FD_HD size_t fftpa_smem_base_(const Geo &g) {
    const int N = g.N, padN = N + (N >> 4), r = rows_per_cta(N);
    const size_t b = sizeof(c32) * ((size_t)N + 2 * (size_t)r * padN + 2 * (size_t)r * pa_coef_count(g));
    return (b + 15) & ~size_t(15);
}
// x_hat row: the N_d data bins, or every bin (in_all: the precoded rows of the FD-NN chain)
FD_HD int fwd_in_len(const Geo &g) { return g.in_all ? g.N : g.N_d; }
inline size_t fwd_stage_bytes(const Geo &g) { return sizeof(c32) * (size_t)((fwd_in_len(g) + 1) & ~1); }
inline size_t adj_stage_bytes(const Geo &g) { return 4 * (size_t)(g.N + ((g.N_d + 3) & ~3)); }    // x(t), gX rows
inline size_t fftpa_smem_bytes_(const Geo &g) {
    return fftpa_smem_base_(g) + (size_t)rows_per_cta(g.N) * fwd_stage_bytes(g);
}

// BF16 outputs go to the blocked plane (BlkPlane): after a row group's last transform each
// row's values are staged as BF16 in its (now free) buffer, and the CTA then writes 16-byte
// pieces (4 subcarriers of one row), rows of the group fastest, so that the pieces of the
// group's adjacent antennas land side by side.  Padding subcarriers past N_d are zero.
// rbase[rr]: row rr's first element in the plane (BlkPlane::row), or -1 past the last row;
// written once per group by one thread of the row, so the pieces need no division.
template <int RPC>
FD_D void store_blk_rows(const Geo &g, const long *rbase, const uint32_t *stage, int stride, cbf16 *out) {
    const long per_group = BlkPlane(g).per_group;   // sub(4 j) = j per_group
    const int ng4 = (g.N_d + 3) >> 2;
    for (int idx = threadIdx.x; idx < RPC * ng4; idx += blockDim.x) {
        const int rr = idx % RPC, j = idx / RPC;
        const long b = rbase[rr];
        if (b < 0) continue;
        const uint4 v = *reinterpret_cast<const uint4 *>(stage + rr * stride + 4 * j);
        *reinterpret_cast<uint4 *>(out + b + (long)j * per_group) = v;
    }
}

template <int LOG2N, int P_, int L_, typename TOut>
__global__ void __launch_bounds__(256, 2) fftpa_forward_kernel(Geo g, long rows, const c32 *__restrict__ xh,
                                                               const c32 *__restrict__ pa,
                                                               const c32 *__restrict__ twp_g, TOut *__restrict__ Xout,
                                                               double *__restrict__ metrics, cbf16 *__restrict__ xt) {
    using F = Fft<LOG2N>;
    constexpr int RPC = rows_per_cta_t<LOG2N>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int grp = threadIdx.x / F::T, t = threadIdx.x % F::T;
    // coefficients per antenna: compile-time for the fixed shapes (which have no cross terms)
    const int P = P_ > 0 ? P_ : g.n_orders, L = P_ > 0 ? L_ : g.L;
    const int PL = P_ > 0 ? P_ * (L_ + 1) : pa_coef_count(g);
    c32 *twp = reinterpret_cast<c32 *>(smem_raw);
    c32 *bufA = twp + F::N + grp * 2 * F::PADN;
    c32 *bufB = bufA + F::PADN;
    c32 *coef = twp + F::N + RPC * 2 * F::PADN;   // [2][RPC][PL]: this group's and the next one's
    // x_hat rows of the next row group, in flight while this one is transformed
    const int in_nd = fwd_in_len(g);
    c32 *stage = reinterpret_cast<c32 *>(smem_raw + fftpa_smem_base_(g)) + grp * ((in_nd + 1) & ~1);
    __shared__ double red[32];
    __shared__ long rbase[RPC];   // blocked-plane start of each row of the group (BF16 X)
    for (int i = threadIdx.x; i < F::TW; i += blockDim.x) twp[i] = twp_g[i];
    bool any_even = false;
    for (int p = 0; p < P; ++p) any_even |= !(g.orders[p] & 1);
    const float rs = rsqrtf((float)F::N);
    float gpow = 0.f, dpow = 0.f;
    const long ngroups = (rows + RPC - 1) / RPC;
    // group gg's x_hat rows and PA coefficients (antenna r mod M; antenna 0 past the last
    // row) into coefficient set pb
    auto prefetch = [&](long gg, int pb) {
        const long r = gg * RPC + grp;
        if (gg < ngroups && r < rows) {
            if (!(in_nd & 1)) {   // rows start on 16 bytes: two subcarriers a copy
                for (int i = t; i < (in_nd >> 1); i += F::T) cp_async_n<16>(stage + 2 * i, xh + r * in_nd + 2 * i);
            } else {
                for (int i = t; i < in_nd; i += F::T) cp_async_n<8>(stage + i, xh + r * in_nd + i);
            }
        }
        if (gg < ngroups) {
            const c32 *src = pa + (long)((unsigned)(r < rows ? r : 0) % (unsigned)g.M) * PL;
            c32 *dst = coef + (pb * RPC + grp) * PL;
            for (int i = t; i < PL; i += F::T) cp_async_n<8>(dst + i, src + i);
        }
        cp_async_commit_all();
    };
    prefetch(blockIdx.x, 0);

    int pb = 0;   // coefficient set of this group
    for (long grp0 = blockIdx.x; grp0 < ngroups; grp0 += gridDim.x, pb ^= 1) {
        const long row = grp0 * RPC + grp;
        const bool active = row < rows;
        const long rowc = active ? row : 0;
        const long sym = (long)((unsigned)rowc / (unsigned)g.M);   // rows < 2^31 (an int on the host)
        const int m = (int)(rowc - sym * g.M);
        cp_async_wait_none();
        __syncthreads();   // this group's rows and coefficients are staged; the previous group is done with the buffers
        if (std::is_same<TOut, cbf16>::value && t == 0) rbase[grp] = active ? BlkPlane(g).row(g, sym, m) : -1;
        const c32 *cp = coef + (pb * RPC + grp) * PL;
        c32 x[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int i = g.in_all ? t + q * F::T : data_index(t + q * F::T, g.first_bin, F::N, g.N_d);
            x[q] = (active && i >= 0) ? stage[i] : make_float2(0.f, 0.f);
        }
        __syncthreads();   // the staged rows are read
        prefetch(grp0 + gridDim.x, pb ^ 1);
        transform<LOG2N, true>(x, bufA, bufB, twp, t, rs);
        if (xt && active) {   // the time-domain PA input, kept (BF16) for the adjoint
            cbf16 *xrow_t = xt + row * F::N;
#pragma unroll
            for (int q = 0; q < 16; ++q) xrow_t[t + q * F::T] = Operand<cbf16>::from(x[q]);
        }
        __syncthreads();   // the last pass has read its buffer
#pragma unroll
        for (int q = 0; q < 16; ++q) bufB[pidx(t + q * F::T)] = x[q];
        __syncthreads();
        c32 y[16];
        RowPa<P_, L_>::forward(g, F::N, F::T, t, x, bufB, cp, any_even, y);
        __syncthreads();   // taps read; bufA / bufB are free
        transform<LOG2N, false>(y, bufA, bufB, twp, t, rs);
        constexpr bool BLK = std::is_same<TOut, cbf16>::value;   // BF16: the blocked plane
        uint32_t *so = reinterpret_cast<uint32_t *>(bufA);   // this row's BF16 values, by subcarrier
        if (BLK) __syncthreads();   // the last pass has read bufA
        TOut *orow = Xout + rowc * g.N_d;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int i = data_index(t + q * F::T, g.first_bin, F::N, g.N_d);
            const float p2 = active ? cabs2(y[q]) : 0.f;
            if (i >= 0) {
                dpow += p2;
                if (BLK) {
                    const cbf16 v = Operand<cbf16>::from(y[q]);
                    so[i] = *reinterpret_cast<const uint32_t *>(&v);
                } else if (active) {
                    orow[i] = Operand<TOut>::from(y[q]);
                }
            } else {
                gpow += p2;
            }
        }
        if constexpr (BLK) {
            for (int i = g.N_d + t; i < 4 * ((g.N_d + 3) >> 2); i += F::T) so[i] = 0u;
            __syncthreads();
            store_blk_rows<RPC>(g, rbase, reinterpret_cast<uint32_t *>(twp + F::N), 4 * F::PADN,
                                reinterpret_cast<cbf16 *>(Xout));
        }
    }
    if (metrics) {
        const double gs = block_sum((double)gpow, red);
        const double ds = block_sum((double)dpow, red);
        if (threadIdx.x == 0) {
            atomicAdd(metrics + 3, gs);
            atomicAdd(metrics + 4, ds);
        }
    }
}

template <int LOG2N, int P_, int L_, typename TIn, typename TOut>
__global__ void __launch_bounds__(256, 2) fftpa_adjoint_kernel(Geo g, long rows, const c32 *__restrict__ xh,
                                                               const c32 *__restrict__ pa,
                                                               const c32 *__restrict__ twp_g, const TIn *gX, TOut *gxh,
                                                               const cbf16 *__restrict__ xt) {
    using F = Fft<LOG2N>;
    constexpr int RPC = rows_per_cta_t<LOG2N>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int grp = threadIdx.x / F::T, t = threadIdx.x % F::T;
    // coefficients per antenna: compile-time for the fixed shapes (which have no cross terms)
    const int P = P_ > 0 ? P_ : g.n_orders, L = P_ > 0 ? L_ : g.L;
    const int PL = P_ > 0 ? P_ * (L_ + 1) : pa_coef_count(g);
    c32 *twp = reinterpret_cast<c32 *>(smem_raw);
    c32 *bufA = twp + F::N + grp * 2 * F::PADN;
    c32 *bufB = bufA + F::PADN;
    c32 *coef = twp + F::N + RPC * 2 * F::PADN;   // [2][RPC][PL]: this group's and the next one's
    // the next row group's inputs, in flight while this one is transformed: with a kept x(t)
    // and BF16 gX both rows ([N] then [N_d rounded to 4] 4-byte words per row); with x(t)
    // recomputed the x_hat row ([N_d rounded to 2] complex values; gX is read directly)
    constexpr bool STAGE = std::is_same<TIn, cbf16>::value;
    const int ndp = (g.N_d + 3) & ~3;
    uint32_t *sx = reinterpret_cast<uint32_t *>(smem_raw + fftpa_smem_base_(g)) + grp * (F::N + ndp);
    uint32_t *sg = sx + F::N;
    c32 *sxh = reinterpret_cast<c32 *>(smem_raw + fftpa_smem_base_(g)) + grp * ((g.N_d + 1) & ~1);
    const bool stage_xh = !xt;
    __shared__ long rbase[RPC];   // blocked-plane start of each row of the group (BF16 g_xhat)
    for (int i = threadIdx.x; i < F::TW; i += blockDim.x) twp[i] = twp_g[i];
    const float rs = rsqrtf((float)F::N);
    const long ngroups = (rows + RPC - 1) / RPC;
    // group gg's staged rows (where this form stages them) and PA coefficients (antenna
    // r mod M; antenna 0 past the last row) into coefficient set pb
    auto prefetch = [&](long gg, int pb) {
        const long r = gg * RPC + grp;
        if (gg < ngroups && r < rows && stage_xh && !(g.N_d & 1)) {   // 16-byte rows: two subcarriers a copy
            for (int i = t; i < (g.N_d >> 1); i += F::T) cp_async_n<16>(sxh + 2 * i, xh + r * g.N_d + 2 * i);
        } else if (gg < ngroups && r < rows && stage_xh) {
            for (int i = t; i < g.N_d; i += F::T) cp_async_n<8>(sxh + i, xh + r * g.N_d + i);
        } else if (gg < ngroups && r < rows && STAGE && xt) {
            const uint4 *srcx = reinterpret_cast<const uint4 *>(xt + r * F::N);
            for (int c = t; c < F::N / 4; c += F::T) cp_async_n<16>(sx + 4 * c, srcx + c);
            const uint32_t *srcg = reinterpret_cast<const uint32_t *>(gX + r * g.N_d);
            for (int i = t; i < g.N_d; i += F::T) cp_async_n<4>(sg + i, srcg + i);
        }
        if (gg < ngroups) {
            const c32 *src = pa + (long)((unsigned)(r < rows ? r : 0) % (unsigned)g.M) * PL;
            c32 *dst = coef + (pb * RPC + grp) * PL;
            for (int i = t; i < PL; i += F::T) cp_async_n<8>(dst + i, src + i);
        }
        cp_async_commit_all();
    };
    prefetch(blockIdx.x, 0);

    int pb = 0;   // coefficient set of this group
    for (long grp0 = blockIdx.x; grp0 < ngroups; grp0 += gridDim.x, pb ^= 1) {
        const long row = grp0 * RPC + grp;
        const bool active = row < rows;
        const long rowc = active ? row : 0;
        const long sym = (long)((unsigned)rowc / (unsigned)g.M);   // rows < 2^31 (an int on the host)
        const int m = (int)(rowc - sym * g.M);
        cp_async_wait_none();
        __syncthreads();   // this group's staged rows and coefficients are in; the previous group is done
        if (std::is_same<TOut, cbf16>::value && t == 0) rbase[grp] = active ? BlkPlane(g).row(g, sym, m) : -1;
        const c32 *cp = coef + (pb * RPC + grp) * PL;
        const TIn *grow = gX + rowc * g.N_d;
        c32 x[16], gv[16];
        if (STAGE && xt) {   // the forward kept the time-domain PA input; both rows staged
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int i = data_index(t + q * F::T, g.first_bin, F::N, g.N_d);
                x[q] = active ? Operand<cbf16>::load(reinterpret_cast<const cbf16 *>(sx + t + q * F::T))
                              : make_float2(0.f, 0.f);
                gv[q] = (active && i >= 0) ? Operand<cbf16>::load(reinterpret_cast<const cbf16 *>(sg + i))
                                           : make_float2(0.f, 0.f);
            }
            __syncthreads();   // the staged rows are read
            prefetch(grp0 + gridDim.x, pb ^ 1);
        } else if (xt) {
            const cbf16 *xrow_t = xt + rowc * F::N;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int i = data_index(t + q * F::T, g.first_bin, F::N, g.N_d);
                x[q] = active ? Operand<cbf16>::load(xrow_t + t + q * F::T) : make_float2(0.f, 0.f);
                gv[q] = (active && i >= 0) ? Operand<TIn>::load(grow + i) : make_float2(0.f, 0.f);
            }
            prefetch(grp0 + gridDim.x, pb ^ 1);   // the next group's coefficients
        } else {   // x(t) recomputed from the staged x_hat row
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int i = data_index(t + q * F::T, g.first_bin, F::N, g.N_d);
                x[q] = (active && i >= 0) ? sxh[i] : make_float2(0.f, 0.f);
                gv[q] = (active && i >= 0) ? Operand<TIn>::load(grow + i) : make_float2(0.f, 0.f);
            }
            __syncthreads();   // the staged rows are read
            prefetch(grp0 + gridDim.x, pb ^ 1);
            transform<LOG2N, true>(x, bufA, bufB, twp, t, rs);
            __syncthreads();
        }
        transform<LOG2N, true>(gv, bufA, bufB, twp, t, rs);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 16; ++q) bufB[pidx(t + q * F::T)] = gv[q];
        if (P_ < 0) {   // the cross terms read x's neighbours
#pragma unroll
            for (int q = 0; q < 16; ++q) bufA[pidx(t + q * F::T)] = x[q];
        }
        __syncthreads();
        RowPa<P_, L_>::adjoint(g, F::N, F::T, t, x, bufB, cp, gv, bufA);
        __syncthreads();
        transform<LOG2N, false>(gv, bufA, bufB, twp, t, rs);
        constexpr bool BLK = std::is_same<TOut, cbf16>::value;   // BF16: the blocked plane (never gX's rows)
        if constexpr (BLK) {
            uint32_t *so = reinterpret_cast<uint32_t *>(bufA);   // this row's BF16 values, by subcarrier
            __syncthreads();   // the last pass has read bufA
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int i = data_index(t + q * F::T, g.first_bin, F::N, g.N_d);
                if (i >= 0) {
                    const cbf16 v = Operand<cbf16>::from(gv[q]);
                    so[i] = *reinterpret_cast<const uint32_t *>(&v);
                }
            }
            for (int i = g.N_d + t; i < 4 * ((g.N_d + 3) >> 2); i += F::T) so[i] = 0u;
            __syncthreads();
            store_blk_rows<RPC>(g, rbase, reinterpret_cast<uint32_t *>(twp + F::N), 4 * F::PADN,
                                reinterpret_cast<cbf16 *>(gxh));
        } else if (active) {
            TOut *orow = gxh + row * g.N_d;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int i = data_index(t + q * F::T, g.first_bin, F::N, g.N_d);
                if (i >= 0) orow[i] = Operand<TOut>::from(gv[q]);
            }
        }
    }
}

// Plain unitary transforms of user rows (the FD-NN comparison workload of Sec. III-C):
// INV: [rows][N_d] data bins (guard bins zero) -> [rows][N] time samples (the IDFT of
// the users' symbols); !INV: [rows][N] time samples -> [rows][N] every bin (the DFT of
// the predistorted streams).  Rows of RPC per CTA as in the PA row kernels; in place
// allowed (a row is read whole before it is written).
template <int LOG2N, bool INV>
__global__ void __launch_bounds__(256, 2) user_rows_kernel(Geo g, long rows, const c32 *in, c32 *out,
                                                           const c32 *__restrict__ twp_g) {
    using F = Fft<LOG2N>;
    constexpr int RPC = rows_per_cta_t<LOG2N>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int grp = threadIdx.x / F::T, t = threadIdx.x % F::T;
    c32 *twp = reinterpret_cast<c32 *>(smem_raw);
    c32 *bufA = twp + F::N + grp * 2 * F::PADN;
    c32 *bufB = bufA + F::PADN;
    for (int i = threadIdx.x; i < F::TW; i += blockDim.x) twp[i] = twp_g[i];
    __syncthreads();
    const float rs = rsqrtf((float)F::N);
    const long ngroups = (rows + RPC - 1) / RPC;
    for (long grp0 = blockIdx.x; grp0 < ngroups; grp0 += gridDim.x) {
        const long row = grp0 * RPC + grp;
        const bool active = row < rows;
        c32 x[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int n = t + q * F::T;
            if (INV) {
                const int i = data_index(n, g.first_bin, F::N, g.N_d);
                x[q] = (active && i >= 0) ? in[row * g.N_d + i] : make_float2(0.f, 0.f);
            } else {
                x[q] = active ? in[row * F::N + n] : make_float2(0.f, 0.f);
            }
        }
        transform<LOG2N, INV>(x, bufA, bufB, twp, t, rs);
        if (active) {
#pragma unroll
            for (int q = 0; q < 16; ++q) out[row * F::N + t + q * F::T] = x[q];
        }
        __syncthreads();   // the last pass has read its buffer
    }
}

template <class Kern>
inline cudaError_t persistent_blocks(Kern k, int N, long rows, int threads, size_t sm, long &blocks, int cap = 0) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int per_sm = resident_ctas(k, threads, sm);
    if (cap > 0 && cap < per_sm) per_sm = cap;
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
                         double *metrics, cbf16 *xt, cudaStream_t st) {
    const int threads = 256;
    const size_t sm = fftpa_smem_bytes_(g);
    long blocks = 0;
    cudaError_t e =
        persistent_blocks(fftpa_forward_kernel<LOG2N, P_, L_, TOut>, g.N, rows, threads, sm, blocks, g.row_ctas);
    if (e != cudaSuccess) return e;
    fftpa_forward_kernel<LOG2N, P_, L_, TOut><<<(unsigned)blocks, threads, sm, st>>>(g, rows, xh, pa, twp, X, metrics,
                                                                                     xt);
    return cudaGetLastError();
}

template <int LOG2N, int P_, int L_, typename TA>
inline cudaError_t adj_t(const Geo &g, long rows, const c32 *xh, const c32 *pa, const c32 *twp, const TA *gX,
                         TA *gxh, const cbf16 *xt, cudaStream_t st) {
    const int threads = 256;
    const size_t sm = fftpa_smem_base_(g) + (size_t)rows_per_cta(g.N) *
                                                (std::is_same<TA, cbf16>::value && xt ? adj_stage_bytes(g)
                                                                                      : fwd_stage_bytes(g));
    long blocks = 0;
    cudaError_t e =
        persistent_blocks(fftpa_adjoint_kernel<LOG2N, P_, L_, TA, TA>, g.N, rows, threads, sm, blocks, g.row_ctas);
    if (e != cudaSuccess) return e;
    fftpa_adjoint_kernel<LOG2N, P_, L_, TA, TA><<<(unsigned)blocks, threads, sm, st>>>(g, rows, xh, pa, twp, gX, gxh,
                                                                                       xt);
    return cudaGetLastError();
}

// PA shapes with a compiled fast path: orders 1,3,5 with taps 0..3, orders 1,3 with
// taps 0..3, and the memoryless 1,3.  Anything else takes the general path.
inline int pa_shape(const Geo &g) {
    if (g.pa_G > 0) return 4;   // cross terms: the general path with the GMP terms compiled in
    for (int p = 0; p < g.n_orders; ++p)
        if (g.orders[p] != 2 * p + 1) return 0;
    if (g.n_orders == 3 && g.L == 3) return 1;
    if (g.n_orders == 2 && g.L == 3) return 2;
    if (g.n_orders == 2 && g.L == 0) return 3;
    return 0;
}

template <int LOG2N, typename TOut>
inline cudaError_t fwd_n(const Geo &g, long rows, const c32 *xh, const c32 *pa, const c32 *twp, TOut *X,
                         double *metrics, cbf16 *xt, cudaStream_t st) {
    switch (pa_shape(g)) {
        case 1: return fwd_t<LOG2N, 3, 3>(g, rows, xh, pa, twp, X, metrics, xt, st);
        case 2: return fwd_t<LOG2N, 2, 3>(g, rows, xh, pa, twp, X, metrics, xt, st);
        case 3: return fwd_t<LOG2N, 2, 0>(g, rows, xh, pa, twp, X, metrics, xt, st);
        case 4: return fwd_t<LOG2N, -1, 0>(g, rows, xh, pa, twp, X, metrics, xt, st);
        default: return fwd_t<LOG2N, 0, 0>(g, rows, xh, pa, twp, X, metrics, xt, st);
    }
}

template <int LOG2N, typename TA>
inline cudaError_t adj_n(const Geo &g, long rows, const c32 *xh, const c32 *pa, const c32 *twp, const TA *gX, TA *gxh,
                         const cbf16 *xt, cudaStream_t st) {
    switch (pa_shape(g)) {
        case 1: return adj_t<LOG2N, 3, 3>(g, rows, xh, pa, twp, gX, gxh, xt, st);
        case 2: return adj_t<LOG2N, 2, 3>(g, rows, xh, pa, twp, gX, gxh, xt, st);
        case 3: return adj_t<LOG2N, 2, 0>(g, rows, xh, pa, twp, gX, gxh, xt, st);
        case 4: return adj_t<LOG2N, -1, 0>(g, rows, xh, pa, twp, gX, gxh, xt, st);
        default: return adj_t<LOG2N, 0, 0>(g, rows, xh, pa, twp, gX, gxh, xt, st);
    }
}

// Translation units per transform size instantiate these, the FP32-plane variants
// (FD_FFTPA_SIZE) and the BF16-plane ones (FD_FFTPA_SIZE16: X out of the forward, gX in
// and g_xhat out of the adjoint in BF16; xt, when given, is the BF16 time-domain PA input
// the forward keeps and the adjoint reads instead of transforming x_hat again) separately,
// so they compile in parallel.
#define FD_FFTPA_SIZE(LOG2N)                                                                                      \
    cudaError_t fftpa_fwd_##LOG2N(const Geo &g, long rows, const c32 *xh, const c32 *pa, const c32 *twp, c32 *X,  \
                                  double *metrics, cudaStream_t st) {                                            \
        return fwd_n<LOG2N>(g, rows, xh, pa, twp, X, metrics, nullptr, st);                                      \
    }                                                                                                            \
    cudaError_t fftpa_adj_##LOG2N(const Geo &g, long rows, const c32 *xh, const c32 *pa, const c32 *twp,         \
                                  const c32 *gX, c32 *gxh, cudaStream_t st) {                                    \
        return adj_n<LOG2N>(g, rows, xh, pa, twp, gX, gxh, nullptr, st);                                         \
    }
#define FD_FFTPA_SIZE16(LOG2N)                                                                                    \
    cudaError_t fftpa_fwd16_##LOG2N(const Geo &g, long rows, const c32 *xh, const c32 *pa, const c32 *twp,       \
                                    cbf16 *X, double *metrics, cbf16 *xt, cudaStream_t st) {                     \
        return fwd_n<LOG2N>(g, rows, xh, pa, twp, X, metrics, xt, st);                                           \
    }                                                                                                            \
    cudaError_t fftpa_adj16_##LOG2N(const Geo &g, long rows, const c32 *xh, const c32 *pa, const c32 *twp,       \
                                    const cbf16 *gX, cbf16 *gxh, const cbf16 *xt, cudaStream_t st) {             \
        return adj_n<LOG2N>(g, rows, xh, pa, twp, gX, gxh, xt, st);                                              \
    }

#define FD_FFTPA_DECL(LOG2N)                                                                                      \
    cudaError_t fftpa_fwd_##LOG2N(const Geo &g, long rows, const c32 *xh, const c32 *pa, const c32 *twp, c32 *X,  \
                                  double *metrics, cudaStream_t st);                                             \
    cudaError_t fftpa_adj_##LOG2N(const Geo &g, long rows, const c32 *xh, const c32 *pa, const c32 *twp,         \
                                  const c32 *gX, c32 *gxh, cudaStream_t st);                                     \
    cudaError_t fftpa_fwd16_##LOG2N(const Geo &g, long rows, const c32 *xh, const c32 *pa, const c32 *twp,       \
                                    cbf16 *X, double *metrics, cbf16 *xt, cudaStream_t st);                      \
    cudaError_t fftpa_adj16_##LOG2N(const Geo &g, long rows, const c32 *xh, const c32 *pa, const c32 *twp,       \
                                    const cbf16 *gX, cbf16 *gxh, const cbf16 *xt, cudaStream_t st);
FD_FFTPA_DECL(6) FD_FFTPA_DECL(7) FD_FFTPA_DECL(8) FD_FFTPA_DECL(9) FD_FFTPA_DECL(10) FD_FFTPA_DECL(11) FD_FFTPA_DECL(12)

}  // namespace fdk
