// Per-antenna OFDM modulation, PA and demodulation for every (symbol, antenna) row.
//
//   forward : x = IDFT_N(x_hat)  (Eq. 2, unitary, guard bins zero)
//             x^PA = PA_b(x)     (Eq. 7 with the memory polynomial of Eq. 9, G = 0,
//                                 taps circular in the N-sample symbol)
//             X = DFT_N(x^PA)    (unitary), keep the N_d data bins; accumulate the
//                                 guard- and data-bin power of X for the ACPR.
//   adjoint : g   = IDFT_N(gX)   (adjoint of the unitary DFT; guard bins of gX zero)
//             x   = IDFT_N(x_hat) recomputed, never stored
//             gx_n = sum_p a_p(x_n) h_{p,n} + b_p(x_n) conj(h_{p,n}),
//                    h_{p,n} = sum_l conj(c_{p,l}) g_{n+l}
//                    a_p = (p+1)/2 |x|^{p-1}, b_p = (p-1)/2 x^2 |x|^{p-3}  (Wirtinger)
//             g_xhat = DFT_N(gx) on the data bins (adjoint of the unitary IDFT).
//
// One row is transformed by N/8 threads, each holding 8 points in registers, with
// Stockham autosort radix-8 passes (one radix-2 or radix-4 pass first when log2 N is
// not a multiple of 3) exchanged through padded shared memory.  The PA (or its
// adjoint) is evaluated while loading the first pass of the final transform, so the
// time-domain signal never leaves shared memory.  All arithmetic is FP32.
#include "common.cuh"
#include "kernels.h"

namespace fdk {

static constexpr float kSqrtHalf = 0.70710678118654752f;

FD_D int pidx(int i) { return i + (i >> 3); }   // one pad word per 8 entries

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
template <int R, bool INV> FD_D void dftR(c32 *v) {
    if (R == 2) dft2<INV>(v);
    else if (R == 4) dft4<INV>(v);
    else dft8<INV>(v);
}

// Twiddle, butterfly and Stockham store of one pass whose inputs v were loaded from
// positions j + r N/R (j = t + b N/8).  Writes buf at (j - k) R + k + q Ns.
template <int R, bool INV>
FD_D void pass_compute_store(c32 *v, c32 *buf, int N, int Ns, int t, const c32 *tw, float scale) {
    constexpr int B = 8 / R;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = t + b * (N >> 3);
        const int k = j & (Ns - 1);
        if (Ns > 1) {
            const int step = N / (Ns * R);
#pragma unroll
            for (int r = 1; r < R; ++r) v[b * R + r] = twmul<INV>(v[b * R + r], tw[r * k * step]);
        }
        dftR<R, INV>(v + b * R);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) buf[pidx(base + q * Ns)] = cscale(v[b * R + q], scale);
    }
}

template <int R>
FD_D void pass_load(c32 *v, const c32 *buf, int N, int t) {
    constexpr int B = 8 / R;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = t + b * (N >> 3);
#pragma unroll
        for (int r = 0; r < R; ++r) v[b * R + r] = buf[pidx(j + r * (N / R))];
    }
}

// The first pass loads through `src(n)`; the remaining passes run in buf.  The last
// pass of a transform whose output goes to global memory is left to the caller:
// `stop_before_last` returns with the final radix-8 inputs loaded in v.
template <bool INV, class Src>
FD_D void fft_run(c32 *buf, int N, int log2N, int t, const c32 *tw, Src src, float last_scale,
                  bool stop_before_last, c32 (&v)[8], int &Ns_out) {
    const int r0 = log2N % 3;
    int Ns = 1;
    // ---- first pass ----
    if (r0 == 1) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = t + b * (N >> 3);
            v[2 * b] = src(j);
            v[2 * b + 1] = src(j + N / 2);
        }
        __syncthreads();
        pass_compute_store<2, INV>(v, buf, N, 1, t, tw, 1.0f);
        Ns = 2;
    } else if (r0 == 2) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int j = t + b * (N >> 3);
#pragma unroll
            for (int r = 0; r < 4; ++r) v[4 * b + r] = src(j + r * (N / 4));
        }
        __syncthreads();
        pass_compute_store<4, INV>(v, buf, N, 1, t, tw, 1.0f);
        Ns = 4;
    } else {
#pragma unroll
        for (int r = 0; r < 8; ++r) v[r] = src(t + r * (N / 8));
        __syncthreads();
        const bool last = (Ns * 8 == N);
        if (last && stop_before_last) { Ns_out = Ns; return; }
        pass_compute_store<8, INV>(v, buf, N, 1, t, tw, last ? last_scale : 1.0f);
        Ns = 8;
    }
    __syncthreads();
    // ---- radix-8 passes ----
    while (Ns < N) {
        pass_load<8>(v, buf, N, t);
        __syncthreads();
        const bool last = (Ns * 8 == N);
        if (last && stop_before_last) { Ns_out = Ns; return; }
        pass_compute_store<8, INV>(v, buf, N, Ns, t, tw, last ? last_scale : 1.0f);
        __syncthreads();
        Ns *= 8;
    }
    Ns_out = Ns;
}

// Finish the last radix-8 pass in registers: returns outputs and their bins.
template <bool INV>
FD_D void last_pass_regs(c32 (&v)[8], int (&bin)[8], int N, int Ns, int t, const c32 *tw, float scale) {
    const int j = t, k = j & (Ns - 1);
    if (Ns > 1) {
        const int step = N / (Ns * 8);
#pragma unroll
        for (int r = 1; r < 8; ++r) v[r] = twmul<INV>(v[r], tw[r * k * step]);
    }
    dft8<INV>(v);
    const int base = (j - k) * 8 + k;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        v[q] = cscale(v[q], scale);
        bin[q] = base + q * Ns;
    }
}

struct PaCoef {
    int P, L1;
    int orders[8];
};

// sum_p c_p(l) x |x|^{p-1} for one sample (cp: [P][L1] at tap l)
FD_D c32 pa_basis_sum(c32 x, const c32 *cp, int P, int L1, int l, const int *orders, bool any_even) {
    const float r2 = cabs2(x);
    const float mag = any_even ? sqrtf(r2) : 0.0f;
    c32 acc = make_float2(0.f, 0.f);
    for (int p = 0; p < P; ++p) {
        const int e = orders[p] - 1;  // power of |x|
        float w = 1.0f;
        for (int q = 0; q + 1 < e; q += 2) w *= r2;
        if (e & 1) w *= mag;
        acc = cfma(cp[p * L1 + l], cscale(x, w), acc);
    }
    return acc;
}

// ---------------------------------------------------------------------------
// forward: one CTA runs rows_per_cta rows, N/8 threads each
// ---------------------------------------------------------------------------
template <typename TOut>
__global__ void __launch_bounds__(512) fftpa_forward_kernel(Geo g, int rows, const c32 *__restrict__ xh,
                                                            const c32 *__restrict__ pa, const c32 *__restrict__ tw_g,
                                                            TOut *__restrict__ Xout, double *__restrict__ metrics) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = g.N, T = N >> 3, log2N = g.log2N;
    const int grp = threadIdx.x / T, t = threadIdx.x % T;
    const int rows_per_cta = blockDim.x / T;
    const int padN = N + (N >> 3);
    c32 *tw = reinterpret_cast<c32 *>(smem_raw);                       // N
    c32 *buf = tw + N + grp * padN;                                    // padN per row
    c32 *coef = tw + N + rows_per_cta * padN;                          // rows_per_cta * P * L1
    __shared__ double red[32];
    __shared__ int orders_s[8];

    const int P = g.n_orders, L1 = g.L + 1, PL = P * L1;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
    if (threadIdx.x < 8) orders_s[threadIdx.x] = g.orders[threadIdx.x];
    const long row = (long)blockIdx.x * rows_per_cta + grp;
    const bool active = row < rows;
    const int m = (int)(row % g.M);
    c32 *cp = coef + grp * PL;
    if (active)
        for (int i = t; i < PL; i += T) cp[i] = pa[(long)m * PL + i];
    __syncthreads();

    const float rs = rsqrtf((float)N);
    const c32 *xrow = xh + row * g.N_d;
    c32 v[8];
    int Ns;
    // IDFT of the spectrum with x_hat at the data bins
    auto src_spec = [&](int k) -> c32 {
        const int i = data_index(k, g.first_bin, N, g.N_d);
        return (active && i >= 0) ? xrow[i] : make_float2(0.f, 0.f);
    };
    fft_run<true>(buf, N, log2N, t, tw, src_spec, rs, false, v, Ns);
    // DFT of PA(x): the PA is evaluated while loading the first pass
    bool any_even = false;
    for (int p = 0; p < P; ++p) any_even |= !(orders_s[p] & 1);
    auto src_pa = [&](int n) -> c32 {
        c32 acc = make_float2(0.f, 0.f);
        for (int l = 0; l < L1; ++l) {
            const c32 x = buf[pidx((n - l) & (N - 1))];
            acc = cadd(acc, pa_basis_sum(x, cp, P, L1, l, orders_s, any_even));
        }
        return acc;
    };
    fft_run<false>(buf, N, log2N, t, tw, src_pa, rs, true, v, Ns);
    int bin[8];
    last_pass_regs<false>(v, bin, N, Ns, t, tw, rs);
    double gpow = 0, dpow = 0;
    TOut *orow = Xout + row * g.N_d;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int i = data_index(bin[q], g.first_bin, N, g.N_d);
        const float p2 = cabs2(v[q]);
        if (i >= 0) {
            dpow += p2;
            if (active) orow[i] = Operand<TOut>::from(v[q]);
        } else {
            gpow += p2;
        }
    }
    if (!active) gpow = dpow = 0;
    if (metrics) {
        double gs = block_sum(gpow, red);
        double ds = block_sum(dpow, red);
        if (threadIdx.x == 0) {
            atomicAdd(metrics + 3, gs);
            atomicAdd(metrics + 4, ds);
        }
    }
}

// ---------------------------------------------------------------------------
// adjoint: gX (data bins) -> g_xhat (data bins), in place; x recomputed from x_hat
// ---------------------------------------------------------------------------
template <typename TIn>
__global__ void __launch_bounds__(512) fftpa_adjoint_kernel(Geo g, int rows, const c32 *__restrict__ xh,
                                                            const c32 *__restrict__ pa, const c32 *__restrict__ tw_g,
                                                            const TIn *gX, c32 *gxh) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = g.N, T = N >> 3, log2N = g.log2N;
    const int grp = threadIdx.x / T, t = threadIdx.x % T;
    const int rows_per_cta = blockDim.x / T;
    const int padN = N + (N >> 3);
    c32 *tw = reinterpret_cast<c32 *>(smem_raw);
    c32 *bufx = tw + N + grp * 2 * padN;
    c32 *bufg = bufx + padN;
    c32 *coef = tw + N + rows_per_cta * 2 * padN;
    __shared__ int orders_s[8];

    const int P = g.n_orders, L1 = g.L + 1, PL = P * L1;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
    if (threadIdx.x < 8) orders_s[threadIdx.x] = g.orders[threadIdx.x];
    const long row = (long)blockIdx.x * rows_per_cta + grp;
    const bool active = row < rows;
    const int m = (int)(row % g.M);
    c32 *cp = coef + grp * PL;
    if (active)
        for (int i = t; i < PL; i += T) cp[i] = pa[(long)m * PL + i];
    __syncthreads();

    const float rs = rsqrtf((float)N);
    const c32 *xrow = xh + row * g.N_d;
    const TIn *grow = gX + row * g.N_d;
    c32 v[8];
    int Ns;
    auto src_x = [&](int k) -> c32 {
        const int i = data_index(k, g.first_bin, N, g.N_d);
        return (active && i >= 0) ? xrow[i] : make_float2(0.f, 0.f);
    };
    auto src_g = [&](int k) -> c32 {
        const int i = data_index(k, g.first_bin, N, g.N_d);
        return (active && i >= 0) ? Operand<TIn>::load(grow + i) : make_float2(0.f, 0.f);
    };
    fft_run<true>(bufx, N, log2N, t, tw, src_x, rs, false, v, Ns);
    fft_run<true>(bufg, N, log2N, t, tw, src_g, rs, false, v, Ns);
    auto src_adj = [&](int n) -> c32 {
        const c32 x = bufx[pidx(n)];
        const float r2 = cabs2(x);
        const float mag = sqrtf(r2);
        c32 acc = make_float2(0.f, 0.f);
        for (int p = 0; p < P; ++p) {
            c32 h = make_float2(0.f, 0.f);
            for (int l = 0; l < L1; ++l) h = cfmac(cp[p * L1 + l], bufg[pidx((n + l) & (N - 1))], h);
            const int e = orders_s[p] - 1;
            float w = 1.0f;   // |x|^{p-1}
            for (int q = 0; q + 1 < e; q += 2) w *= r2;
            if (e & 1) w *= mag;
            const float a = 0.5f * (float)(e + 2) * w;
            acc = cadd(acc, cscale(h, a));
            if (e >= 1 && mag > 0.0f) {
                // b = (p-1)/2 x^2 |x|^{p-3} = (p-1)/2 x^2 w / r2
                const float bs = 0.5f * (float)e * w / r2;
                const c32 b = cscale(cmul(x, x), bs);
                acc = cfma(b, cconj(h), acc);
            }
        }
        return acc;
    };
    fft_run<false>(bufx, N, log2N, t, tw, src_adj, rs, true, v, Ns);
    int bin[8];
    last_pass_regs<false>(v, bin, N, Ns, t, tw, rs);
    __syncthreads();  // every thread has read its gX row entries before any is overwritten
    if (active) {
        c32 *orow = gxh + row * g.N_d;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = data_index(bin[q], g.first_bin, N, g.N_d);
            if (i >= 0) orow[i] = v[q];
        }
    }
}

static int rows_per_cta(int N) { return N >= 2048 ? 1 : 2048 / N; }

size_t fftpa_smem_bytes(const Geo &g, bool adjoint) {
    const int N = g.N, padN = N + (N >> 3), r = rows_per_cta(N);
    return sizeof(c32) * ((size_t)N + (size_t)r * padN * (adjoint ? 2 : 1) + (size_t)r * g.n_orders * (g.L + 1));
}

template <typename TOut>
static cudaError_t launch_fwd(const Geo &g, int rows, const c32 *xh, const c32 *pa, const c32 *tw, TOut *X,
                              double *metrics, cudaStream_t st) {
    const int r = rows_per_cta(g.N), threads = r * (g.N >> 3);
    const size_t sm = fftpa_smem_bytes(g, false);
    cudaError_t e = cudaFuncSetAttribute(fftpa_forward_kernel<TOut>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int blocks = (rows + r - 1) / r;
    fftpa_forward_kernel<TOut><<<blocks, threads, sm, st>>>(g, rows, xh, pa, tw, X, metrics);
    return cudaGetLastError();
}

cudaError_t fftpa_forward(const Geo &g, int rows, const c32 *xh, const c32 *pa, const c32 *tw, void *X, int out_kind,
                          double *metrics, cudaStream_t st) {
    if (out_kind == OUT_BF16) return launch_fwd(g, rows, xh, pa, tw, (cbf16 *)X, metrics, st);
    if (out_kind == OUT_F16) return launch_fwd(g, rows, xh, pa, tw, (cf16 *)X, metrics, st);
    return launch_fwd(g, rows, xh, pa, tw, (c32 *)X, metrics, st);
}

cudaError_t fftpa_adjoint(const Geo &g, int rows, const c32 *xh, const c32 *pa, const c32 *tw, const c32 *gX,
                          c32 *gxh, cudaStream_t st) {
    const int r = rows_per_cta(g.N), threads = r * (g.N >> 3);
    const size_t sm = fftpa_smem_bytes(g, true);
    cudaError_t e = cudaFuncSetAttribute(fftpa_adjoint_kernel<c32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int blocks = (rows + r - 1) / r;
    fftpa_adjoint_kernel<c32><<<blocks, threads, sm, st>>>(g, rows, xh, pa, tw, gX, gxh);
    return cudaGetLastError();
}

}  // namespace fdk
