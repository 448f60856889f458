// C-ABI of the fddpd library: plan life cycle, argument checks, workspace layout and
// the order in which the stage kernels run on the plan's stream.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <climits>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>

#include "fddpd.h"
#include "kernels.h"
#include "tc_gemm.h"

using fdk::Geo;

static constexpr int kMaxRec = 4096;
static constexpr int kCopyChunks = 16;   // most chunks of fddpd_update_host

struct fddpd_plan {
    fddpd_dims d;
    fddpd_pa_desc pa;
    fddpd_dpd_desc dpd;
    Geo g;
    cudaStream_t stream;
    int R_max;
    void *base;
    size_t bytes;
    c32 *st, *gy, *gst, *xh, *Xpa, *tw;
    void *zf_scratch;
    float *act, *gpre, *partials, *grad, *adam_m, *adam_v;
    double *met;
    int *status;        // [0] singular subcarriers of the last precode, [1] sticky device timeouts
    int *status_host;
    // 16-bit plans: dense-layer operands (leading dimensions in elements)
    bool p16;
    long ldF, ld2N, ldC;
    __nv_bfloat16 *act16, *actT16, *gd16, *gdT16, *fcw16, *fcwT16;
    float *fbi;                    // fc_b in the dense layer's interleaved output order
    int kind16;                    // OUT_BF16 or OUT_F16: storage of the H / W copies
    bool tc_bin;                   // per-subcarrier contractions on the tensor cores
    bool keep_xt;                  // BF16 planes: the forward keeps x(t) for the adjoint (FDDPD_OPT_KEEP_PA_INPUT)
    bool fp64_factor;              // Cholesky + triangular inverse in FP64 (FDDPD_OPT_FACTOR_FP64)
    void *H16, *W16;               // [R_max][N_d][K][M] and [R_max][N_d][M][K]
    void *xt16;                    // kept time-domain PA input [S][M][N] (BF16), allocated by the option
    size_t gxh_off;                // BF16 planes, recomputed x(t): g_xhat's offset in the X^PA buffer
    const void *pk_H, *pk_W;       // the FP32 arrays the copies were made from
    int pk_R;
    bool wfree;                    // W16 holds H^H and the ZF scratch Y = L^{-1} of pk_H (fddpd_precode, W = NULL)
    // FD-NN comparison plans (fddpd_fdnn_plan_create)
    bool nn;
    fdk::FdnnDesc nnd;
    c32 *nn_t, *nn_o;              // user streams in time [S K][N]; network output, then its DFT
    float *nn_al;                  // alpha of the data bins [R_max][N_d]
    long adam_t;
    // stage tracing
    int prof;
    int nrec;
    cudaEvent_t *ev;          // 2 * kMaxRec events, created on first enable
    int rec_stage[4096];
    long long launches;
    // device staging of fddpd_update_host
    void *stage_base;
    c32 *hs, *hH, *hW, *hpa;
    float *hal, *htheta;
    double *hmet;
    int host_chunks;                             // chunks of fddpd_update_host (FDDPD_OPT_HOST_CHUNKS)
    cudaStream_t cstream;                        // host-to-device copies, beside p->stream
    cudaEvent_t cev[kCopyChunks + 2];            // [0] staging free, [1..kCopyChunks] H chunks, last: s, pa, theta
    char err[512];
};

static const char *kStageNames[FDDPD_N_STAGES] = {
    "zf_gram", "zf_factor", "zf_apply", "conv_fwd", "fc_fwd", "precode", "fftpa_fwd", "combine", "adj_combine", "fftpa_adj",
    "adj_precode", "fc_bwd_w", "fc_bwd_b", "fc_bwd_d", "conv_bwd", "step", "pack", "zmul", "fdnn_rows", "fdnn_mlp"};

static int stage_begin(fddpd_plan *p, int stage) {
    if (!p->prof || p->nrec >= kMaxRec) return -1;
    const int slot = p->nrec++;
    p->rec_stage[slot] = stage;
    cudaEventRecord(p->ev[2 * slot], p->stream);
    return slot;
}
static void stage_end(fddpd_plan *p, int slot) {
    if (slot >= 0) cudaEventRecord(p->ev[2 * slot + 1], p->stream);
}

static thread_local char g_create_err[512] = "";

static int set_err(fddpd_plan *p, int code, const char *fmt, ...) {
    char *dst = p ? p->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return code;
}

#define FD_CK(p, expr)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (expr);                                                                \
        if (e_ != cudaSuccess) return set_err(p, FDDPD_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

// Run one stage: `nk` kernels launched by `expr`, bracketed by events when tracing.
#define FD_STAGE(p, stage, nk, expr)                 \
    do {                                             \
        const int slot_ = stage_begin(p, stage);     \
        FD_CK(p, expr);                              \
        stage_end(p, slot_);                         \
        (p)->launches += (nk);                       \
    } while (0)

static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// Device allocations of the library; fddpd_debug_fail_allocs(n) makes the next n of them
// fail (host-side fault injection: the failure paths run without exhausting the GPU).
static std::atomic<int> g_fail_allocs{0};
static cudaError_t dev_alloc(void **ptr, size_t bytes) {
    int n = g_fail_allocs.load();
    while (n > 0)
        if (g_fail_allocs.compare_exchange_weak(n, n - 1)) return cudaErrorMemoryAllocation;
    return cudaMalloc(ptr, bytes);
}
extern "C" int fddpd_debug_fail_allocs(int n) {
    if (n < 0) return FDDPD_ERR_ARG;
    g_fail_allocs.store(n);
    return FDDPD_OK;
}
static bool aligned(const void *ptr, size_t a) { return (reinterpret_cast<uintptr_t>(ptr) % a) == 0; }

static int validate(const fddpd_dims *d, const fddpd_pa_desc *pa, const fddpd_dpd_desc *dpd) {
    if (!d || !pa || !dpd) return set_err(nullptr, FDDPD_ERR_ARG, "null descriptor");
    if (d->M < 1 || d->M > 512) return set_err(nullptr, FDDPD_ERR_ARG, "M=%d outside 1..512", d->M);
    if (d->K < 1 || d->K > 32 || d->K > d->M) return set_err(nullptr, FDDPD_ERR_ARG, "K=%d outside 1..min(32,M)", d->K);
    if (!is_pow2(d->N) || d->N < 64 || d->N > 4096) return set_err(nullptr, FDDPD_ERR_UNSUPPORTED, "N=%d is not a power of two in 64..4096", d->N);
    if (d->N_d < 1 || d->N_d > d->N) return set_err(nullptr, FDDPD_ERR_ARG, "N_d=%d outside 1..N", d->N_d);
    if (d->first_bin < -1 || d->first_bin >= d->N) return set_err(nullptr, FDDPD_ERR_ARG, "first_bin=%d", d->first_bin);
    if (d->S_per_real < 1 || d->max_symbols < 1) return set_err(nullptr, FDDPD_ERR_ARG, "S_per_real / max_symbols < 1");
    // symbol x antenna rows and symbol x user columns are counted in 32 bits by the launchers
    if ((long)d->max_symbols * d->M > INT_MAX)
        return set_err(nullptr, FDDPD_ERR_ARG, "max_symbols x M above 2^31 - 1");
    if (d->precision != FDDPD_FP32 && d->precision != FDDPD_BF16 && d->precision != FDDPD_FP16)
        return set_err(nullptr, FDDPD_ERR_ARG, "precision=%d", d->precision);
    if (!(d->P_T > 0)) return set_err(nullptr, FDDPD_ERR_ARG, "P_T must be positive");
    if (pa->n_orders < 1 || pa->n_orders > 8 || pa->L < 0 || pa->L > 7 || pa->G < 0 || pa->G > 2)
        return set_err(nullptr, FDDPD_ERR_ARG, "PA orders / memory / cross-term length out of range");
    if (pa->G > 0 && pa->orders[0] == 0) return set_err(nullptr, FDDPD_ERR_ARG, "the clipping PA has no cross terms");
    for (int i = 0; i < pa->n_orders; ++i)
        if (pa->orders[i] < 0 || pa->orders[i] > 15 || (pa->orders[i] == 0 && (pa->n_orders != 1 || pa->L != 0)))
            return set_err(nullptr, FDDPD_ERR_ARG, "PA order %d: 1..15, or 0 (linear clipping) alone with L = 0",
                           pa->orders[i]);
    if (dpd->G < 1 || dpd->G * dpd->G < d->N_d || dpd->G > 128) return set_err(nullptr, FDDPD_ERR_ARG, "grid G=%d cannot hold N_d", dpd->G);
    if (dpd->L_U < 1 || dpd->L_U > d->K) return set_err(nullptr, FDDPD_ERR_ARG, "L_U=%d outside 1..K", dpd->L_U);
    if (dpd->K_C < 1 || !(dpd->K_C & 1) || dpd->K_C > 15) return set_err(nullptr, FDDPD_ERR_ARG, "K_C=%d must be odd in 1..15", dpd->K_C);
    if (dpd->K_S < 1 || dpd->K_S > dpd->G) return set_err(nullptr, FDDPD_ERR_ARG, "K_S=%d", dpd->K_S);
    if (dpd->N_conv < 1 || dpd->N_conv > 64) return set_err(nullptr, FDDPD_ERR_ARG, "N_conv=%d outside 1..64", dpd->N_conv);
    if (dpd->residual != 0 && dpd->residual != 1) return set_err(nullptr, FDDPD_ERR_ARG, "residual must be 0 or 1");
    if (dpd->per_user != 0 && dpd->per_user != 1) return set_err(nullptr, FDDPD_ERR_ARG, "per_user must be 0 or 1");
    return FDDPD_OK;
}

static Geo make_geo(const fddpd_dims *d, const fddpd_pa_desc *pa, const fddpd_dpd_desc *dpd) {
    Geo g;
    memset(&g, 0, sizeof g);
    g.M = d->M; g.K = d->K; g.N = d->N; g.N_d = d->N_d;
    g.first_bin = d->first_bin < 0 ? d->N - d->N_d / 2 : d->first_bin;
    g.S_per_real = d->S_per_real;
    g.log2N = 0;
    while ((1 << g.log2N) < d->N) ++g.log2N;
    g.n_orders = pa->n_orders;
    for (int i = 0; i < 8; ++i) g.orders[i] = i < pa->n_orders ? pa->orders[i] : 0;
    g.L = pa->L;
    g.pa_G = pa->G;
    g.G = dpd->G; g.K_S = dpd->K_S; g.Go = (dpd->G + dpd->K_S - 1) / dpd->K_S;
    g.L_U = dpd->L_U; g.Cin = 2 * dpd->L_U; g.K_C = dpd->K_C; g.pad = dpd->K_C / 2;
    g.N_conv = dpd->N_conv; g.F = dpd->N_conv * g.Go * g.Go; g.residual = dpd->residual;
    g.n_convw = g.N_conv * g.Cin * g.K_C * g.K_C;
    g.off_cb = g.n_convw;
    g.off_fw = g.off_cb + g.N_conv;
    g.off_fb = g.off_fw + 2L * g.N_d * g.F;
    g.theta_len = (g.off_fb + 2L * g.N_d) * (dpd->per_user ? g.K : 1);   // per user: K sets stacked by user
    g.P_T = d->P_T;
    return g;
}

extern "C" int fddpd_plan_create(fddpd_plan **out, const fddpd_dims *d, const fddpd_pa_desc *pa,
                                 const fddpd_dpd_desc *dpd, void *stream) {
    if (!out) return set_err(nullptr, FDDPD_ERR_ARG, "out is null");
    *out = nullptr;
    int rc = validate(d, pa, dpd);
    if (rc) return rc;
    fddpd_plan *p = new (std::nothrow) fddpd_plan;
    if (!p) return set_err(nullptr, FDDPD_ERR_NOMEM, "host allocation failed");
    memset(p, 0, sizeof *p);
    p->d = *d; p->pa = *pa; p->dpd = *dpd;
    p->g = make_geo(d, pa, dpd);
    p->stream = static_cast<cudaStream_t>(stream);
    const Geo &g = p->g;
    const long S = d->max_symbols, cols = S * g.K;
    p->R_max = (int)((S + g.S_per_real - 1) / g.S_per_real);

    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
    // rows of the dense layer's 16-bit operands (and of its FP32 pre-activation gradient)
    // start on 128-byte boundaries, so every 64-element TMA box row is whole 32-byte sectors
    auto r64 = [](long v) { return (v + 63) / 64 * 64; };
    const size_t o_st = take(sizeof(c32) * cols * g.N_d), o_gy = take(sizeof(c32) * cols * g.N_d),
                 o_gst = take(sizeof(c32) * cols * g.N_d), o_xh = take(std::max(sizeof(c32) * S * g.M * g.N_d, fdk::blk_plane_bytes(g, S))),
                 // X^PA buffer: the FP32 plane, or (BF16 planes) the blocked X^PA, or the BF16 rows
                 // of g_X followed by the blocked g_xhat of an adjoint that recomputes x(t)
                 gxh_off = (4 * (size_t)S * g.M * g.N_d + 255) & ~size_t(255),
                 o_X = take(std::max(sizeof(c32) * S * g.M * g.N_d, gxh_off + fdk::blk_plane_bytes(g, S))),
                 o_tw = take(sizeof(c32) * g.N),
                 o_act = take(sizeof(float) * cols * g.F), o_gpre = take(sizeof(float) * cols * r64(g.F)),
                 o_part = take(sizeof(float) * cols * (g.n_convw + g.N_conv)),
                 o_grad = take(sizeof(float) * g.theta_len), o_met = take(sizeof(double) * 8),
                 o_stat = take(2 * sizeof(int));
    const size_t o_zf = take(fdk::zf_scratch_bytes(g, (long)p->R_max * g.N_d));
    p->p16 = d->precision != FDDPD_FP32;
    p->tc_bin = true;
    p->keep_xt = false;
    p->fp64_factor = true;
    p->gxh_off = gxh_off;
    p->host_chunks = 7;
    p->ldF = r64(g.F);
    p->ld2N = r64(2L * g.N_d);
    p->ldC = r64(cols);
    size_t o_a16 = 0, o_aT = 0, o_g16 = 0, o_gT = 0, o_w16 = 0, o_wT = 0, o_fbi = 0;
    if (p->p16) {
        o_a16 = take(2 * (size_t)cols * p->ldF);
        o_aT = take(2 * (size_t)g.F * p->ldC);
        o_g16 = take(2 * (size_t)cols * p->ld2N);
        o_gT = take(2 * (size_t)2 * g.N_d * p->ldC);
        o_w16 = take(2 * (size_t)2 * g.N_d * p->ldF);
        o_wT = take(2 * (size_t)g.F * p->ld2N);
        o_fbi = take(sizeof(float) * 2 * (size_t)g.N_d);
    }
    size_t o_h16 = 0, o_wq16 = 0;
    if (p->p16) {
        o_h16 = take(4 * (size_t)p->R_max * g.N_d * g.K * g.M);
        o_wq16 = take(4 * (size_t)p->R_max * g.N_d * g.K * g.M);
    }
    p->bytes = off;
    cudaError_t e = dev_alloc(&p->base, off);
    if (e != cudaSuccess) {
        delete p;
        cudaGetLastError();
        return set_err(nullptr, FDDPD_ERR_NOMEM, "cudaMalloc(%zu): %s", off, cudaGetErrorString(e));
    }
    char *b = static_cast<char *>(p->base);
    p->st = (c32 *)(b + o_st); p->gy = (c32 *)(b + o_gy); p->gst = (c32 *)(b + o_gst);
    p->xh = (c32 *)(b + o_xh); p->Xpa = (c32 *)(b + o_X); p->tw = (c32 *)(b + o_tw);
    p->act = (float *)(b + o_act); p->gpre = (float *)(b + o_gpre); p->partials = (float *)(b + o_part);
    p->grad = (float *)(b + o_grad);   // the Adam moments are allocated by the first Adam step
    p->met = (double *)(b + o_met); p->status = (int *)(b + o_stat);
    p->zf_scratch = b + o_zf;
    if (p->p16) {
        p->act16 = (__nv_bfloat16 *)(b + o_a16); p->actT16 = (__nv_bfloat16 *)(b + o_aT);
        p->gd16 = (__nv_bfloat16 *)(b + o_g16); p->gdT16 = (__nv_bfloat16 *)(b + o_gT);
        p->fcw16 = (__nv_bfloat16 *)(b + o_w16); p->fcwT16 = (__nv_bfloat16 *)(b + o_wT);
        p->fbi = (float *)(b + o_fbi);
        p->H16 = b + o_h16;
        p->W16 = b + o_wq16;
        p->kind16 = d->precision == FDDPD_FP16 ? fdk::OUT_F16 : fdk::OUT_BF16;
    }
    e = cudaMallocHost(&p->status_host, 2 * sizeof(int));
    if (e == cudaSuccess) e = fdk::pass_twiddles(g.log2N, p->tw, p->stream);
    p->launches = 1;
    if (e == cudaSuccess) e = cudaMemsetAsync(p->status, 0, 2 * sizeof(int), p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) {
        set_err(nullptr, FDDPD_ERR_CUDA, "plan set-up: %s", cudaGetErrorString(e));
        fddpd_plan_destroy(p);
        return FDDPD_ERR_CUDA;
    }
    *out = p;
    return FDDPD_OK;
}

// The Adam moments [theta_len] each, zeroed, allocated the first time they are needed (a
// plan that only runs forward passes, or GD, never holds them).
static int ensure_adam(fddpd_plan *p) {
    if (p->adam_m) return FDDPD_OK;
    const size_t n = sizeof(float) * (size_t)p->g.theta_len;
    void *m = nullptr;
    if (dev_alloc(&m, 2 * n) != cudaSuccess) {
        cudaGetLastError();
        return set_err(p, FDDPD_ERR_NOMEM, "Adam moments (%zu bytes)", 2 * n);
    }
    FD_CK(p, cudaMemsetAsync(m, 0, 2 * n, p->stream));
    p->adam_m = static_cast<float *>(m);
    p->adam_v = p->adam_m + p->g.theta_len;
    return FDDPD_OK;
}

// Every subcarrier as a data bin in FFT bin order: the geometry of the FD-NN chain's
// precoder, which covers the guard bins too.
static Geo all_bins(const Geo &g) {
    Geo a = g;
    a.N_d = g.N;
    a.first_bin = 0;
    return a;
}

extern "C" int fddpd_fdnn_plan_create(fddpd_plan **out, const fddpd_dims *d, const fddpd_pa_desc *pa,
                                      const fddpd_fdnn_desc *nn, void *stream) {
    if (!out) return set_err(nullptr, FDDPD_ERR_ARG, "out is null");
    *out = nullptr;
    if (!d || !nn) return set_err(nullptr, FDDPD_ERR_ARG, "null descriptor");
    fddpd_dpd_desc dummy{};
    dummy.G = 1;
    while (dummy.G * dummy.G < d->N_d) ++dummy.G;
    dummy.L_U = 1; dummy.K_C = 1; dummy.K_S = 1; dummy.N_conv = 1; dummy.residual = 1;
    int rc = validate(d, pa, &dummy);
    if (rc) return rc;
    if (d->precision != FDDPD_FP32) return set_err(nullptr, FDDPD_ERR_UNSUPPORTED, "FD-NN plans are FP32");
    if (nn->L4 < 0 || nn->L4 > 15 || nn->D < 1 || nn->D > 32 || nn->layers < 1 || nn->layers > 4 ||
        (nn->residual != 0 && nn->residual != 1))
        return set_err(nullptr, FDDPD_ERR_ARG, "FD-NN: L4 0..15, D 1..32, layers 1..4, residual 0 or 1");
    fddpd_plan *p = new (std::nothrow) fddpd_plan;
    if (!p) return set_err(nullptr, FDDPD_ERR_NOMEM, "host allocation failed");
    memset(p, 0, sizeof *p);
    p->d = *d; p->pa = *pa; p->dpd = dummy;
    p->g = make_geo(d, pa, &dummy);
    p->nn = true;
    p->nnd = fdk::FdnnDesc{nn->L4, nn->D, nn->layers, nn->residual};
    p->g.theta_len = fdk::fdnn_theta_len(p->g, p->nnd);
    if (p->g.theta_len > 12288) {
        delete p;
        return set_err(nullptr, FDDPD_ERR_UNSUPPORTED, "FD-NN with more than 12288 parameters");
    }
    p->stream = static_cast<cudaStream_t>(stream);
    p->fp64_factor = true;
    const Geo &g = p->g;
    const long S = d->max_symbols;
    p->R_max = (int)((S + g.S_per_real - 1) / g.S_per_real);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
    const size_t o_t = take(sizeof(c32) * S * g.K * g.N), o_o = take(sizeof(c32) * S * g.K * g.N),
                 o_xh = take(sizeof(c32) * S * g.M * g.N), o_X = take(sizeof(c32) * S * g.M * g.N_d),
                 o_al = take(sizeof(float) * (size_t)p->R_max * g.N_d), o_tw = take(sizeof(c32) * g.N),
                 o_met = take(sizeof(double) * 8), o_stat = take(2 * sizeof(int)),
                 o_zf = take(fdk::zf_scratch_bytes(g, (long)p->R_max * g.N));
    p->bytes = off;
    cudaError_t e = dev_alloc(&p->base, off);
    if (e != cudaSuccess) {
        delete p;
        cudaGetLastError();
        return set_err(nullptr, FDDPD_ERR_NOMEM, "cudaMalloc(%zu): %s", off, cudaGetErrorString(e));
    }
    char *b = static_cast<char *>(p->base);
    p->nn_t = (c32 *)(b + o_t); p->nn_o = (c32 *)(b + o_o); p->xh = (c32 *)(b + o_xh); p->Xpa = (c32 *)(b + o_X);
    p->nn_al = (float *)(b + o_al); p->tw = (c32 *)(b + o_tw); p->met = (double *)(b + o_met);
    p->status = (int *)(b + o_stat); p->zf_scratch = b + o_zf;
    e = cudaMallocHost(&p->status_host, 2 * sizeof(int));
    if (e == cudaSuccess) e = fdk::pass_twiddles(g.log2N, p->tw, p->stream);
    p->launches = 1;
    if (e == cudaSuccess) e = cudaMemsetAsync(p->status, 0, 2 * sizeof(int), p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) {
        set_err(nullptr, FDDPD_ERR_CUDA, "plan set-up: %s", cudaGetErrorString(e));
        fddpd_plan_destroy(p);
        return FDDPD_ERR_CUDA;
    }
    *out = p;
    return FDDPD_OK;
}

extern "C" int fddpd_plan_destroy(fddpd_plan *p) {
    if (!p) return FDDPD_OK;
    if (p->base) cudaFree(p->base);
    if (p->xt16) cudaFree(p->xt16);
    if (p->adam_m) cudaFree(p->adam_m);
    if (p->stage_base) cudaFree(p->stage_base);
    if (p->cstream) {
        cudaStreamDestroy(p->cstream);
        for (int i = 0; i < kCopyChunks + 2; ++i) cudaEventDestroy(p->cev[i]);
    }
    if (p->status_host) cudaFreeHost(p->status_host);
    if (p->ev) {
        for (int i = 0; i < 2 * kMaxRec; ++i) cudaEventDestroy(p->ev[i]);
        delete[] p->ev;
    }
    delete p;
    return FDDPD_OK;
}

extern "C" const char *fddpd_last_error(const fddpd_plan *p) { return p ? p->err : g_create_err; }
extern "C" size_t fddpd_theta_len(const fddpd_plan *p) { return p ? (size_t)p->g.theta_len : 0; }
extern "C" size_t fddpd_workspace_bytes(const fddpd_plan *p) { return p ? p->bytes : 0; }

extern "C" int fddpd_set_stream(fddpd_plan *p, void *stream) {
    if (!p) return FDDPD_ERR_ARG;
    p->stream = static_cast<cudaStream_t>(stream);
    return FDDPD_OK;
}

extern "C" int fddpd_set_option(fddpd_plan *p, int option, int value) {
    if (!p) return FDDPD_ERR_ARG;
    if (option == FDDPD_OPT_TENSOR_CONTRACTIONS && (value == 0 || value == 1)) {
        p->tc_bin = value != 0;
        return FDDPD_OK;
    }
    if (option == FDDPD_OPT_HOST_CHUNKS && value >= 1 && value <= kCopyChunks) {
        p->host_chunks = value;
        return FDDPD_OK;
    }
    if (option == FDDPD_OPT_KEEP_PA_INPUT && (value == 0 || value == 1)) {
        // BF16 plans only: the BF16 copy of x(t), [max_symbols][M][N], allocated once
        if (value && p->d.precision == FDDPD_BF16 && !p->xt16) {
            const size_t n = 4 * (size_t)p->d.max_symbols * p->g.M * p->g.N;
            if (dev_alloc(&p->xt16, n) != cudaSuccess) {
                cudaGetLastError();
                p->xt16 = nullptr;
                return set_err(p, FDDPD_ERR_NOMEM, "kept PA input (%zu bytes)", n);
            }
        }
        p->keep_xt = value != 0;
        return FDDPD_OK;
    }
    if (option == FDDPD_OPT_FACTOR_FP64 && (value == 0 || value == 1)) {
        p->fp64_factor = value != 0 || !p->p16;   // FP32 plans always factor in FP64
        return FDDPD_OK;
    }
    if (option == FDDPD_OPT_ROW_CTAS && value >= 0 && value <= 8) {
        p->g.row_ctas = value;
        return FDDPD_OK;
    }
    if (option == FDDPD_OPT_CONTRACTION_CTAS && value >= 0 && value <= 2) {
        p->g.bin_ctas = value == 1 ? 1 : 0;
        return FDDPD_OK;
    }
    if (option == FDDPD_OPT_CONTRACTION_ITEM && (value == 0 || value == 1)) {
        p->g.bin_half = value;
        return FDDPD_OK;
    }
    return set_err(p, FDDPD_ERR_ARG, "fddpd_set_option: unknown option or value");
}

extern "C" int fddpd_get_option(const fddpd_plan *p, int option, int *value) {
    if (!p || !value) return FDDPD_ERR_ARG;
    switch (option) {
        case FDDPD_OPT_TENSOR_CONTRACTIONS: *value = p->tc_bin ? 1 : 0; return FDDPD_OK;
        case FDDPD_OPT_HOST_CHUNKS: *value = p->host_chunks; return FDDPD_OK;
        case FDDPD_OPT_KEEP_PA_INPUT: *value = p->keep_xt ? 1 : 0; return FDDPD_OK;
        case FDDPD_OPT_FACTOR_FP64: *value = p->fp64_factor ? 1 : 0; return FDDPD_OK;
        case FDDPD_OPT_ROW_CTAS: *value = p->g.row_ctas; return FDDPD_OK;
        case FDDPD_OPT_CONTRACTION_CTAS: *value = p->g.bin_ctas == 1 ? 1 : 2; return FDDPD_OK;
        case FDDPD_OPT_CONTRACTION_ITEM: *value = p->g.bin_half; return FDDPD_OK;
        default: return FDDPD_ERR_ARG;
    }
}

extern "C" int fddpd_set_power(fddpd_plan *p, double P_T) {
    if (!p) return FDDPD_ERR_ARG;
    if (!(P_T > 0) || !std::isfinite(P_T)) return set_err(p, FDDPD_ERR_ARG, "P_T must be positive and finite");
    p->d.P_T = P_T;
    p->g.P_T = P_T;
    return FDDPD_OK;
}

extern "C" int fddpd_invalidate_operands(fddpd_plan *p) {
    if (!p) return FDDPD_ERR_ARG;
    p->pk_H = nullptr;
    p->pk_W = nullptr;
    p->pk_R = 0;
    p->wfree = false;
    return FDDPD_OK;
}

extern "C" int fddpd_reset_optimizer(fddpd_plan *p) {
    if (!p) return FDDPD_ERR_ARG;
    p->adam_t = 0;
    if (p->adam_m) FD_CK(p, cudaMemsetAsync(p->adam_m, 0, 2 * sizeof(float) * p->g.theta_len, p->stream));
    return FDDPD_OK;
}

extern "C" int fddpd_get_optimizer_state(fddpd_plan *p, float *m, float *v, long long *t) {
    if (!p) return FDDPD_ERR_ARG;
    if (!m || !v || !t) return set_err(p, FDDPD_ERR_ARG, "null pointer");
    if (!aligned(m, 4) || !aligned(v, 4)) return set_err(p, FDDPD_ERR_LAYOUT, "misaligned pointer");
    const int rc = ensure_adam(p);
    if (rc) return rc;
    const size_t n = sizeof(float) * (size_t)p->g.theta_len;
    FD_CK(p, cudaMemcpyAsync(m, p->adam_m, n, cudaMemcpyDefault, p->stream));
    FD_CK(p, cudaMemcpyAsync(v, p->adam_v, n, cudaMemcpyDefault, p->stream));
    FD_CK(p, cudaStreamSynchronize(p->stream));
    *t = p->adam_t;
    return FDDPD_OK;
}

extern "C" int fddpd_set_optimizer_state(fddpd_plan *p, const float *m, const float *v, long long t) {
    if (!p) return FDDPD_ERR_ARG;
    if (!m || !v || t < 0) return set_err(p, FDDPD_ERR_ARG, "null pointer or negative step count");
    if (!aligned(m, 4) || !aligned(v, 4)) return set_err(p, FDDPD_ERR_LAYOUT, "misaligned pointer");
    const int rc = ensure_adam(p);
    if (rc) return rc;
    const size_t n = sizeof(float) * (size_t)p->g.theta_len;
    FD_CK(p, cudaMemcpyAsync(p->adam_m, m, n, cudaMemcpyDefault, p->stream));
    FD_CK(p, cudaMemcpyAsync(p->adam_v, v, n, cudaMemcpyDefault, p->stream));
    FD_CK(p, cudaStreamSynchronize(p->stream));
    p->adam_t = (long)t;
    return FDDPD_OK;
}

extern "C" int fddpd_precode(fddpd_plan *p, int R, const fddpd_c32 *H, fddpd_c32 *W, float *alpha) {
    if (!p) return FDDPD_ERR_ARG;
    if (R < 0 || R > p->R_max) return set_err(p, FDDPD_ERR_ARG, "R=%d outside 0..%d", R, p->R_max);
    if (R == 0) return FDDPD_OK;
    if (!H || !alpha) return set_err(p, FDDPD_ERR_ARG, "null pointer");
    if (p->nn) {   // the FD-NN chain precodes every bin: ZF of all N subcarriers
        if (!W) return set_err(p, FDDPD_ERR_ARG, "FD-NN plans need W");
        if (!aligned(H, 8) || !aligned(W, 8) || !aligned(alpha, 4)) return set_err(p, FDDPD_ERR_LAYOUT, "misaligned pointer");
        const Geo ga = all_bins(p->g);
        FD_CK(p, cudaMemsetAsync(p->status, 0, sizeof(int), p->stream));
        for (int ph = 0; ph < 3; ++ph)
            FD_STAGE(p, FDDPD_STAGE_ZF_GRAM + ph, 1,
                     fdk::zf_phase(ph, ga, R, reinterpret_cast<const c32 *>(H), reinterpret_cast<c32 *>(W), alpha,
                                   p->status, p->zf_scratch, nullptr, nullptr, fdk::OUT_F32, false, true,
                                   p->status + 1, p->stream));
        FD_CK(p, cudaMemcpyAsync(p->status_host, p->status, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
        FD_CK(p, cudaStreamSynchronize(p->stream));
        if (p->status_host[0]) return set_err(p, FDDPD_ERR_SINGULAR, "a Gram matrix H_k H_k^H is not positive definite");
        return FDDPD_OK;
    }
    if (!W && !p->p16) return set_err(p, FDDPD_ERR_UNSUPPORTED, "W = NULL (precoder kept as its factors) needs a 16-bit plan");
    if (!aligned(H, 8) || (W && !aligned(W, 8)) || !aligned(alpha, 4)) return set_err(p, FDDPD_ERR_LAYOUT, "misaligned pointer");
    cudaStream_t st = p->stream;
    FD_CK(p, cudaMemsetAsync(p->status, 0, sizeof(int), st));
    // W = NULL: the Gram kernel writes the 16-bit H^H beside H's copy and the factor's Y
    // stays in the scratch; the chain then applies W s = H^H (Z s) and no W is formed
    const int nph = W ? 3 : 2;
    for (int ph = 0; ph < nph; ++ph)
        FD_STAGE(p, FDDPD_STAGE_ZF_GRAM + ph, 1,
                 fdk::zf_phase(ph, p->g, R, reinterpret_cast<const c32 *>(H), reinterpret_cast<c32 *>(W), alpha,
                               p->status, p->zf_scratch, p->p16 ? p->H16 : nullptr, p->p16 && W ? p->W16 : nullptr,
                               p->kind16, p->tc_bin, p->fp64_factor, p->status + 1, st, true,
                               W ? nullptr : p->W16));
    if (p->p16) {
        p->pk_H = H;
        p->pk_W = W;
        p->pk_R = R;
        p->wfree = !W;
    }
    FD_CK(p, cudaMemcpyAsync(p->status_host, p->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    FD_CK(p, cudaStreamSynchronize(st));
    if (p->status_host[0]) return set_err(p, FDDPD_ERR_SINGULAR, "a Gram matrix H_k H_k^H is not positive definite");
    return FDDPD_OK;
}

static int check_chain(fddpd_plan *p, int S, const void *s, const void *H, const void *W, const void *alpha,
                       const void *pa, const void *theta) {
    if (S < 1 || S > p->d.max_symbols) return set_err(p, FDDPD_ERR_ARG, "S=%d outside 1..%d", S, p->d.max_symbols);
    if (!s || !H || !alpha || !pa || !theta) return set_err(p, FDDPD_ERR_ARG, "null pointer");
    if (!W) {   // the precoder kept as its factors by fddpd_precode(H, NULL, alpha)
        const int R = (S + p->g.S_per_real - 1) / p->g.S_per_real;
        if (!p->wfree || p->pk_H != H || p->pk_R < R)
            return set_err(p, FDDPD_ERR_ARG, "W is null but no factor of this H is kept (fddpd_precode with W = NULL first)");
    }
    if (!aligned(s, 8) || !aligned(H, 8) || (W && !aligned(W, 8)) || !aligned(pa, 8) || !aligned(alpha, 4) ||
        !aligned(theta, 4))
        return set_err(p, FDDPD_ERR_LAYOUT, "misaligned pointer");
    return FDDPD_OK;
}

// Precode / combine operands: FP32 H and W, or the plan's 16-bit copies (made by
// fddpd_precode, or here when the caller passes arrays they were not made from).
struct BinOps {
    const void *H, *W;
    int kind;
    const void *W_or_H(int mode) const {
        return (mode == fdk::PRECODE || mode == fdk::ADJ_PRECODE || mode == fdk::ADJ_COMBINE_F) ? W : H;
    }
};
static int bin_operands(fddpd_plan *p, int S, const c32 *H, const c32 *W, BinOps &o) {
    if (!p->p16) {
        o = BinOps{H, W, fdk::OUT_F32};
        return FDDPD_OK;
    }
    const Geo &g = p->g;
    const int R = (S + g.S_per_real - 1) / g.S_per_real;
    if (!W) {   // checked by check_chain: the copies of H and H^H of the kept factor
        o = BinOps{p->H16, p->W16, p->kind16};
        return FDDPD_OK;
    }
    if (p->pk_H != H || p->pk_W != W || p->pk_R < R) {
        const long n = (long)R * g.N_d * g.K * g.M;
        FD_STAGE(p, FDDPD_STAGE_PACK, 2,
                 fdk::to_16bit(n, H, p->H16, p->kind16, p->stream) == cudaSuccess
                     ? fdk::to_16bit(n, W, p->W16, p->kind16, p->stream)
                     : cudaGetLastError());
        p->pk_H = H;
        p->pk_W = W;
        p->pk_R = R;
        p->wfree = false;
    }
    o = BinOps{p->H16, p->W16, p->kind16};
    return FDDPD_OK;
}

// Per-subcarrier contractions: tensor cores in 16-bit plans where supported, else CUDA
// cores.  b_scale multiplies the activations before their 16-bit rounding (and divides
// the results): a power of two that lifts the loss gradients, O(1 / count), out of the
// FP16 subnormal range (BF16 has the FP32 range and needs none).
static bool use_tc_bin(const fddpd_plan *p) { return p->p16 && p->tc_bin && fdk::tc_bin_supported(p->g); }
// BF16 plans on the tensor-core path keep the antenna-side frequency-domain planes (X^PA,
// its gradient and the gradient of x_hat) in BF16: the MMAs round them to BF16 anyway.
static int act_kind(const fddpd_plan *p) {
    return use_tc_bin(p) && p->kind16 == fdk::OUT_BF16 ? fdk::OUT_BF16 : fdk::OUT_F32;
}
static cudaError_t expand_op(fddpd_plan *p, int mode, int S, const BinOps &o, const float *alpha, const c32 *B,
                             void *out, float b_scale) {
    if (use_tc_bin(p))
        return fdk::tc_bin_expand(p->g, mode, S, o.W_or_H(mode), o.kind, alpha, B, out,
                                  mode == fdk::PRECODE ? fdk::OUT_F32 : act_kind(p), b_scale, p->status + 1, p->stream);
    return fdk::bin_expand(p->g, mode, S, o.W_or_H(mode), o.kind, alpha, B, static_cast<c32 *>(out), p->stream);
}
static cudaError_t reduce_op(fddpd_plan *p, int mode, int S, const BinOps &o, const float *alpha, const void *B,
                             c32 *out, const c32 *s_ref, c32 *gy, double *metrics, double inv_count, float b_scale) {
    if (use_tc_bin(p))
        return fdk::tc_bin_reduce(p->g, mode, S, o.W_or_H(mode), o.kind, alpha, B, act_kind(p), out, s_ref, gy, metrics,
                                  inv_count, b_scale, p->status + 1, p->stream);
    return fdk::bin_reduce(p->g, mode, S, o.W_or_H(mode), o.kind, alpha, static_cast<const c32 *>(B), out, s_ref, gy,
                           metrics, inv_count, p->stream);
}
// BF16 planes with FDDPD_OPT_KEEP_PA_INPUT: the forward of a training pass stores x(t)
static bool keeps_xt(const fddpd_plan *p) { return p->keep_xt && p->xt16 && act_kind(p) == fdk::OUT_BF16; }
static float grad_scale(const fddpd_plan *p, double inv_count) {
    return p->kind16 == fdk::OUT_F16 ? exp2f(rintf(log2f((float)(0.5 / inv_count)))) : 1.0f;
}

// Forward chain; gy (loss gradient at y) is written when non-null.
// One pass of the chain over S symbols that may be part of a larger batch: the loss is
// normalised by the whole batch (inv_count), the metric sums are cleared by the first
// part and finalised by the last, parameter gradients are accumulated after the first,
// and the plan's 16-bit H / W copies are read from realisation r0 on (the caller made
// them for the whole batch).  A null Pass is a whole batch on its own.
struct Pass {
    double inv_count;
    bool first, last;
    int r0;
};

static int pass_operands(fddpd_plan *p, int S, const c32 *H, const c32 *W, const Pass *ps, BinOps &o) {
    if (!ps || !p->p16) return bin_operands(p, S, H, W, o);
    const size_t real16 = (size_t)p->g.N_d * p->g.K * p->g.M * 4;   // one realisation of a 16-bit copy
    o = BinOps{(const char *)p->H16 + ps->r0 * real16, (const char *)p->W16 + ps->r0 * real16, p->kind16};
    return FDDPD_OK;
}

static int run_forward(fddpd_plan *p, int S, const c32 *s, const c32 *H, const c32 *W, const float *alpha,
                       const c32 *pa, const float *theta, c32 *y, c32 *gy, const Pass *ps = nullptr) {
    const Geo &g = p->g;
    cudaStream_t st = p->stream;
    const long cols = (long)S * g.K;
    const double inv_count = ps ? ps->inv_count : 1.0 / ((double)cols * g.N_d);
    const bool first = !ps || ps->first, last = !ps || ps->last;
    BinOps ops;
    int rc0 = pass_operands(p, S, H, W, ps, ops);
    if (rc0) return rc0;
    if (first) FD_CK(p, cudaMemsetAsync(p->met, 0, sizeof(double) * 8, st));
    if (p->dpd.per_user) {
        // user u's own network theta_u over its column block (FD-CNN column t is chain column
        // t K + u): the shared network's kernels once per user, s and s_tilde addressed in place
        const long len1 = g.theta_len / g.K;
        for (int u = 0; u < g.K; ++u) {
            const float *th = theta + u * len1;
            if (p->p16) {
                __nv_bfloat16 *a16 = p->act16 + (long)u * S * p->ldF;
                FD_STAGE(p, FDDPD_STAGE_CONV_FWD, 1, fdk::conv_forward_bf16(g, S, s, th, a16, p->ldF, st, u));
                FD_STAGE(p, FDDPD_STAGE_PACK, 1, fdk::pack_fcw(g, th, p->fcw16, p->ldF, p->fbi, st));
                const fdk::GemmArgs ga{a16, p->fcw16, S, 2 * g.N_d, g.F, p->ldF, p->ldF, 1, 1};
                FD_STAGE(p, FDDPD_STAGE_FC_FWD, 1,
                         fdk::tc_fc_forward(ga, reinterpret_cast<float *>(p->st), reinterpret_cast<const float *>(s),
                                            p->fbi, g.N_d, g.residual, p->status + 1, st, g.K, u));
            } else {
                float *act = p->act + (long)u * S * g.F;
                FD_STAGE(p, FDDPD_STAGE_CONV_FWD, 1, fdk::conv_forward(g, S, s, th, act, st, u));
                FD_STAGE(p, FDDPD_STAGE_FC_FWD, 1, fdk::fc_forward_f32(g, S, act, th, s, p->st, st, u));
            }
        }
    } else if (p->p16) {
        FD_STAGE(p, FDDPD_STAGE_CONV_FWD, 1, fdk::conv_forward_bf16(g, S, s, theta, p->act16, p->ldF, st));
        if (first) FD_STAGE(p, FDDPD_STAGE_PACK, 1, fdk::pack_fcw(g, theta, p->fcw16, p->ldF, p->fbi, st));
        const fdk::GemmArgs ga{p->act16, p->fcw16, (int)cols, 2 * g.N_d, g.F, p->ldF, p->ldF, 1, 1};
        FD_STAGE(p, FDDPD_STAGE_FC_FWD, 1,
                 fdk::tc_fc_forward(ga, reinterpret_cast<float *>(p->st), reinterpret_cast<const float *>(s),
                                    p->fbi, g.N_d, g.residual, p->status + 1, st));
    } else {
        FD_STAGE(p, FDDPD_STAGE_CONV_FWD, 1, fdk::conv_forward(g, S, s, theta, p->act, st));
        FD_STAGE(p, FDDPD_STAGE_FC_FWD, 1, fdk::fc_forward_f32(g, (int)cols, p->act, theta, s, p->st, st));
    }
    if (W) {
        FD_STAGE(p, FDDPD_STAGE_PRECODE, 1, expand_op(p, fdk::PRECODE, S, ops, alpha, p->st, p->xh, 1.0f));
    } else {   // x_hat = alpha H^H (Z s_tilde): Z s_tilde into gst (free until the adjoint)
        FD_STAGE(p, FDDPD_STAGE_ZMUL, 1, fdk::zf_zmul(g, S, p->zf_scratch, p->st, p->gst, st));
        FD_STAGE(p, FDDPD_STAGE_PRECODE, 1, expand_op(p, fdk::PRECODE, S, ops, alpha, p->gst, p->xh, 1.0f));
    }
    // a backward follows when gy is wanted: keep the time-domain PA input for its adjoint
    // when the plan is set to (FDDPD_OPT_KEEP_PA_INPUT); by default the adjoint recomputes it
    void *xt = keeps_xt(p) && gy ? p->xt16 : nullptr;
    FD_STAGE(p, FDDPD_STAGE_FFTPA_FWD, 1,
             fdk::fftpa_forward(g, S * g.M, p->xh, pa, p->tw, p->Xpa, act_kind(p), p->met, xt, st));
    FD_STAGE(p, FDDPD_STAGE_COMBINE, 1,
             reduce_op(p, fdk::COMBINE, S, ops, alpha, p->Xpa, y, s, gy, p->met, inv_count, 1.0f));
    if (last) {
        FD_CK(p, fdk::finalize_metrics(p->met, inv_count, st));
        p->launches += 1;
    }
    return FDDPD_OK;
}

static int run_backward(fddpd_plan *p, int S, const c32 *s, const c32 *H, const c32 *W, const float *alpha,
                        const c32 *pa, const float *theta, float *grad, const Pass *ps = nullptr) {
    const Geo &g = p->g;
    cudaStream_t st = p->stream;
    const int cols = S * g.K;
    const bool first = !ps || ps->first;
    int rc = run_forward(p, S, s, H, W, alpha, pa, theta, nullptr, p->gy, ps);
    if (rc) return rc;
    BinOps ops;
    rc = pass_operands(p, S, H, W, ps, ops);
    if (rc) return rc;
    const float gsc = grad_scale(p, ps ? ps->inv_count : 1.0 / ((double)cols * g.N_d));
    // with the precoder kept as its factors the 16-bit W slot holds H^H: the tensor-core form
    // reads it with direct row loads
    const int acm = (!W && use_tc_bin(p)) ? fdk::ADJ_COMBINE_F : fdk::ADJ_COMBINE;
    FD_STAGE(p, FDDPD_STAGE_ADJ_COMBINE, 1, expand_op(p, acm, S, ops, alpha, p->gy, p->Xpa, gsc));
    // BF16 planes: g_xhat goes to a blocked plane -- in x_hat's buffer when the adjoint
    // reads the kept x(t), else behind the rows of g_X (x_hat is read to recompute x(t));
    // FP32 planes: in place over g_X
    const bool a16 = act_kind(p) == fdk::OUT_BF16, kept = keeps_xt(p);
    void *gxh = !a16 ? (void *)p->Xpa : kept ? (void *)p->xh : (void *)((char *)p->Xpa + p->gxh_off);
    FD_STAGE(p, FDDPD_STAGE_FFTPA_ADJ, 1,
             fdk::fftpa_adjoint(g, S * g.M, p->xh, pa, p->tw, p->Xpa, gxh, act_kind(p), kept ? p->xt16 : nullptr, st));
    if (W) {
        FD_STAGE(p, FDDPD_STAGE_ADJ_PRECODE, 1,
                 reduce_op(p, fdk::ADJ_PRECODE, S, ops, alpha, gxh, p->gst, nullptr, nullptr, nullptr, 0.0, gsc));
    } else {   // g_s_tilde = Z (alpha H g_xhat): the reduction into gy (read by the adjoint of combine, now free);
               // the tensor-core form reads H's own copy with direct row loads
        const int mode = use_tc_bin(p) ? fdk::ADJ_PRECODE_F : fdk::ADJ_PRECODE;
        FD_STAGE(p, FDDPD_STAGE_ADJ_PRECODE, 1,
                 reduce_op(p, mode, S, ops, alpha, gxh, p->gy, nullptr, nullptr, nullptr, 0.0, gsc));
        FD_STAGE(p, FDDPD_STAGE_ZMUL, 1, fdk::zf_zmul(g, S, p->zf_scratch, p->gy, p->gst, st));
    }
    const float *gd = reinterpret_cast<const float *>(p->gst);
    if (p->dpd.per_user) {
        // user u's pass over its column block with theta_u and its slice of grad (gd, s in
        // the chain's column order; the dense layer's 16-bit operands one block at a time)
        const long len1 = g.theta_len / g.K, W2 = 2L * g.N_d, ldCu = (S + 63) / 64 * 64;
        for (int u = 0; u < g.K; ++u) {
            const float *th = theta + u * len1;
            float *gr = grad + u * len1;
            if (first) FD_CK(p, cudaMemsetAsync(gr + g.off_fb, 0, sizeof(float) * W2, st));
            if (p->p16) {
                __nv_bfloat16 *a16 = p->act16 + (long)u * S * p->ldF, *g16 = p->gd16 + (long)u * S * p->ld2N;
                float *gpre = p->gpre + (long)u * S * p->ldF;
                FD_STAGE(p, FDDPD_STAGE_PACK, 2,
                         fdk::bf16_and_transpose(gd + u * W2, S, W2, g.K * W2, g16, p->ld2N, p->gdT16, ldCu, st) ==
                                 cudaSuccess
                             ? fdk::transpose_bf16(a16, S, g.F, p->ldF, p->actT16, ldCu, st)
                             : cudaGetLastError());
                if (first) FD_CK(p, cudaMemsetAsync(gr + g.off_fw, 0, sizeof(float) * W2 * g.F, st));
                const fdk::GemmArgs gw{p->gdT16, p->actT16, (int)W2, g.F, S, ldCu, ldCu, 1, 2};
                FD_STAGE(p, FDDPD_STAGE_FC_BWD_W, 1,
                         fdk::tc_fc_backward_weight(gw, gr + g.off_fw, g.N_d, g.F, p->status + 1, st));
                FD_STAGE(p, FDDPD_STAGE_FC_BWD_B, 1, fdk::colsum_fcb(g, S, gd, gr, st, u));
                FD_STAGE(p, FDDPD_STAGE_PACK, 1, fdk::pack_fcw_t(g, th, p->fcwT16, p->ld2N, st));
                const fdk::GemmArgs gdx{g16, p->fcwT16, S, g.F, (int)W2, p->ld2N, p->ld2N, 1, 1};
                FD_STAGE(p, FDDPD_STAGE_FC_BWD_D, 1,
                         fdk::tc_fc_backward_data(gdx, gpre, p->ldF, a16, p->ldF, p->status + 1, st));
                FD_STAGE(p, FDDPD_STAGE_CONV_BWD, 2, fdk::conv_backward(g, S, s, gpre, p->ldF, p->partials, st, u));
            } else {
                const float *act = p->act + (long)u * S * g.F;
                float *gpre = p->gpre + (long)u * S * g.F;
                FD_STAGE(p, FDDPD_STAGE_FC_BWD_W, 1, fdk::fc_backward_weight_f32(g, S, gd, act, gr, !first, st, u));
                FD_STAGE(p, FDDPD_STAGE_FC_BWD_B, 1, fdk::colsum_fcb(g, S, gd, gr, st, u));
                FD_STAGE(p, FDDPD_STAGE_FC_BWD_D, 1, fdk::fc_backward_data_f32(g, S, gd, th, act, gpre, st, u));
                FD_STAGE(p, FDDPD_STAGE_CONV_BWD, 2, fdk::conv_backward(g, S, s, gpre, g.F, p->partials, st, u));
            }
            FD_CK(p, fdk::conv_reduce(g, S, p->partials, gr, !first, st));
        }
        // the shared network's tail below (convolution gradient and its reduction) is done
        // per user inside the loop above: a change to that tail belongs in both places
        return FDDPD_OK;
    }
    if (first) FD_CK(p, cudaMemsetAsync(grad + g.off_fb, 0, sizeof(float) * 2 * g.N_d, st));
    if (p->p16) {
        const long W2 = 2L * g.N_d;
        FD_STAGE(p, FDDPD_STAGE_PACK, 2,
                 fdk::bf16_and_transpose(gd, cols, W2, W2, p->gd16, p->ld2N, p->gdT16, p->ldC, st) == cudaSuccess
                     ? fdk::transpose_bf16(p->act16, cols, g.F, p->ldF, p->actT16, p->ldC, st)
                     : cudaGetLastError());
        if (first) {
            FD_STAGE(p, FDDPD_STAGE_PACK, 1, fdk::pack_fcw_t(g, theta, p->fcwT16, p->ld2N, st));
            FD_CK(p, cudaMemsetAsync(grad + g.off_fw, 0, sizeof(float) * W2 * g.F, st));
        }
        // split-K partial sums are added into grad: enough splits to fill the GPU
        const int splits = cols >= 16384 ? 4 : 2;
        const fdk::GemmArgs gw{p->gdT16, p->actT16, (int)W2, g.F, cols, p->ldC, p->ldC, 1, splits};
        FD_STAGE(p, FDDPD_STAGE_FC_BWD_W, 1, fdk::tc_fc_backward_weight(gw, grad + g.off_fw, g.N_d, g.F, p->status + 1, st));
        FD_STAGE(p, FDDPD_STAGE_FC_BWD_B, 1, fdk::colsum_fcb(g, cols, gd, grad, st));
        const fdk::GemmArgs gdx{p->gd16, p->fcwT16, cols, g.F, (int)W2, p->ld2N, p->ld2N, 1, 1};
        FD_STAGE(p, FDDPD_STAGE_FC_BWD_D, 1, fdk::tc_fc_backward_data(gdx, p->gpre, p->ldF, p->act16, p->ldF, p->status + 1, st));
    } else {
        FD_STAGE(p, FDDPD_STAGE_FC_BWD_W, 1, fdk::fc_backward_weight_f32(g, cols, gd, p->act, grad, !first, st));
        FD_STAGE(p, FDDPD_STAGE_FC_BWD_B, 1, fdk::colsum_fcb(g, cols, gd, grad, st));
        FD_STAGE(p, FDDPD_STAGE_FC_BWD_D, 1, fdk::fc_backward_data_f32(g, cols, gd, theta, p->act, p->gpre, st));
    }
    FD_STAGE(p, FDDPD_STAGE_CONV_BWD, 2, fdk::conv_backward(g, S, s, p->gpre, p->p16 ? p->ldF : g.F, p->partials, st));
    FD_CK(p, fdk::conv_reduce(g, cols, p->partials, grad, !first, st));
    return FDDPD_OK;
}

// The FD-NN chain (Sec. III-C): per-user IDFT, the time-domain network, per-user DFT onto
// every bin, precoding of every bin (W, alpha over all N), IDFT / PA / DFT, combining at
// the data bins (H of the data bins, alpha gathered at them).
static int run_fdnn_forward(fddpd_plan *p, int S, const c32 *s, const c32 *H, const c32 *W, const float *alpha,
                            const c32 *pa, const float *theta, c32 *y) {
    const Geo &g = p->g;
    cudaStream_t st = p->stream;
    const long rows = (long)S * g.K;
    const double inv_count = 1.0 / ((double)rows * g.N_d);
    Geo gi = g;
    gi.in_all = 1;
    FD_CK(p, cudaMemsetAsync(p->met, 0, sizeof(double) * 8, st));
    FD_STAGE(p, FDDPD_STAGE_FDNN_ROWS, 1, fdk::fdnn_user_rows(g, rows, true, s, p->nn_t, p->tw, st));
    FD_STAGE(p, FDDPD_STAGE_FDNN_MLP, 1, fdk::fdnn_mlp(g, p->nnd, S, theta, p->nn_t, p->nn_o, st));
    FD_STAGE(p, FDDPD_STAGE_FDNN_ROWS, 1, fdk::fdnn_user_rows(g, rows, false, p->nn_o, p->nn_o, p->tw, st));
    FD_STAGE(p, FDDPD_STAGE_PRECODE, 1,
             fdk::bin_expand(all_bins(g), fdk::PRECODE, S, W, fdk::OUT_F32, alpha, p->nn_o, p->xh, st));
    FD_STAGE(p, FDDPD_STAGE_FFTPA_FWD, 1,
             fdk::fftpa_forward(gi, S * g.M, p->xh, pa, p->tw, p->Xpa, fdk::OUT_F32, p->met, nullptr, st));
    FD_CK(p, fdk::fdnn_alpha_data(g, (S + g.S_per_real - 1) / g.S_per_real, alpha, p->nn_al, st));
    FD_STAGE(p, FDDPD_STAGE_COMBINE, 1,
             fdk::bin_reduce(g, fdk::COMBINE, S, H, fdk::OUT_F32, p->nn_al, p->Xpa, y, s, nullptr, p->met, inv_count,
                             st));
    FD_CK(p, fdk::finalize_metrics(p->met, inv_count, st));
    p->launches += 2;
    return FDDPD_OK;
}

extern "C" int fddpd_distort(fddpd_plan *p, int S, const fddpd_c32 *s, const fddpd_c32 *H, const fddpd_c32 *W,
                             const float *alpha, const fddpd_c32 *pa_coef, const float *theta, fddpd_c32 *y,
                             double *metrics) {
    if (!p) return FDDPD_ERR_ARG;
    if (p->nn) {
        if (!W) return set_err(p, FDDPD_ERR_ARG, "FD-NN plans need W");
        int rc = check_chain(p, S, s, H, W, alpha, pa_coef, theta);
        if (rc) return rc;
        if ((y && !aligned(y, 8)) || (metrics && !aligned(metrics, 8))) return set_err(p, FDDPD_ERR_LAYOUT, "misaligned output");
        rc = run_fdnn_forward(p, S, (const c32 *)s, (const c32 *)H, (const c32 *)W, alpha, (const c32 *)pa_coef, theta,
                              (c32 *)y);
        if (rc) return rc;
        if (metrics) FD_CK(p, cudaMemcpyAsync(metrics, p->met, sizeof(double) * 5, cudaMemcpyDeviceToDevice, p->stream));
        return FDDPD_OK;
    }
    int rc = check_chain(p, S, s, H, W, alpha, pa_coef, theta);
    if (rc) return rc;
    if ((y && !aligned(y, 8)) || (metrics && !aligned(metrics, 8))) return set_err(p, FDDPD_ERR_LAYOUT, "misaligned output");
    rc = run_forward(p, S, (const c32 *)s, (const c32 *)H, (const c32 *)W, alpha, (const c32 *)pa_coef, theta,
                     (c32 *)y, nullptr);
    if (rc) return rc;
    if (metrics) FD_CK(p, cudaMemcpyAsync(metrics, p->met, sizeof(double) * 5, cudaMemcpyDeviceToDevice, p->stream));
    return FDDPD_OK;
}

extern "C" int fddpd_backward(fddpd_plan *p, int S, const fddpd_c32 *s, const fddpd_c32 *H, const fddpd_c32 *W,
                              const float *alpha, const fddpd_c32 *pa_coef, const float *theta, float *grad,
                              double *metrics) {
    if (!p) return FDDPD_ERR_ARG;
    if (p->nn) return set_err(p, FDDPD_ERR_UNSUPPORTED, "FD-NN plans run the forward chain only");
    int rc = check_chain(p, S, s, H, W, alpha, pa_coef, theta);
    if (rc) return rc;
    if (!grad) return set_err(p, FDDPD_ERR_ARG, "grad is null");
    if (!aligned(grad, 4) || (metrics && !aligned(metrics, 8))) return set_err(p, FDDPD_ERR_LAYOUT, "misaligned output");
    rc = run_backward(p, S, (const c32 *)s, (const c32 *)H, (const c32 *)W, alpha, (const c32 *)pa_coef, theta, grad);
    if (rc) return rc;
    if (metrics) FD_CK(p, cudaMemcpyAsync(metrics, p->met, sizeof(double) * 5, cudaMemcpyDeviceToDevice, p->stream));
    return FDDPD_OK;
}

static int opt_step(fddpd_plan *p, float *theta, float lr, int optimizer, const float *grad = nullptr,
                    float gscale = 1.0f) {
    if (!grad) grad = p->grad;
    if (optimizer == FDDPD_GD) {
        FD_STAGE(p, FDDPD_STAGE_STEP, 1, fdk::sgd_step(p->g.theta_len, theta, grad, lr, p->stream, gscale));
    } else {
        const int rc = ensure_adam(p);
        if (rc) return rc;
        const long t = ++p->adam_t;
        const float c1 = (float)(1.0 - pow(0.9, (double)t)), c2 = (float)(1.0 - pow(0.999, (double)t));
        FD_STAGE(p, FDDPD_STAGE_STEP, 1,
                 fdk::adam_step(p->g.theta_len, theta, grad, p->adam_m, p->adam_v, lr, c1, c2, p->stream, gscale));
    }
    return FDDPD_OK;
}

extern "C" int fddpd_apply_gradient(fddpd_plan *p, float *theta, const float *grad, float scale, float lr,
                                    int optimizer) {
    if (!p) return FDDPD_ERR_ARG;
    if (p->nn) return set_err(p, FDDPD_ERR_UNSUPPORTED, "FD-NN plans run the forward chain only");
    if (!theta || !grad) return set_err(p, FDDPD_ERR_ARG, "null theta or grad");
    if (!aligned(theta, 4) || !aligned(grad, 4)) return set_err(p, FDDPD_ERR_LAYOUT, "misaligned theta or grad");
    if (!std::isfinite(scale) || !std::isfinite(lr)) return set_err(p, FDDPD_ERR_ARG, "scale and lr must be finite");
    if (optimizer != FDDPD_GD && optimizer != FDDPD_ADAM) return set_err(p, FDDPD_ERR_ARG, "optimizer=%d", optimizer);
    return opt_step(p, theta, lr, optimizer, grad, scale);
}

extern "C" int fddpd_update(fddpd_plan *p, int S, const fddpd_c32 *s, const fddpd_c32 *H, const fddpd_c32 *W,
                            const float *alpha, const fddpd_c32 *pa_coef, float *theta, float lr, int iters,
                            int optimizer, double *metrics) {
    if (!p) return FDDPD_ERR_ARG;
    if (p->nn) return set_err(p, FDDPD_ERR_UNSUPPORTED, "FD-NN plans run the forward chain only");
    int rc = check_chain(p, S, s, H, W, alpha, pa_coef, theta);
    if (rc) return rc;
    if (iters < 0) return set_err(p, FDDPD_ERR_ARG, "iters < 0");
    if (optimizer != FDDPD_GD && optimizer != FDDPD_ADAM) return set_err(p, FDDPD_ERR_ARG, "optimizer=%d", optimizer);
    if (metrics && !aligned(metrics, 8)) return set_err(p, FDDPD_ERR_LAYOUT, "misaligned metrics");
    for (int it = 0; it < iters; ++it) {
        rc = run_backward(p, S, (const c32 *)s, (const c32 *)H, (const c32 *)W, alpha, (const c32 *)pa_coef, theta,
                          p->grad);
        if (rc) return rc;
        rc = opt_step(p, theta, lr, optimizer);
        if (rc) return rc;
    }
    if (metrics && iters > 0)
        FD_CK(p, cudaMemcpyAsync(metrics, p->met, sizeof(double) * 5, cudaMemcpyDeviceToDevice, p->stream));
    return FDDPD_OK;
}

extern "C" int fddpd_profile_enable(fddpd_plan *p, int enable) {
    if (!p) return FDDPD_ERR_ARG;
    if (enable && !p->ev) {
        p->ev = new (std::nothrow) cudaEvent_t[2 * kMaxRec];
        if (!p->ev) return set_err(p, FDDPD_ERR_NOMEM, "event pool");
        for (int i = 0; i < 2 * kMaxRec; ++i) FD_CK(p, cudaEventCreate(&p->ev[i]));
    }
    p->prof = enable ? 1 : 0;
    return FDDPD_OK;
}

extern "C" int fddpd_profile_read(fddpd_plan *p, double *ms, long long *count) {
    if (!p) return FDDPD_ERR_ARG;
    FD_CK(p, cudaStreamSynchronize(p->stream));
    double acc[FDDPD_N_STAGES] = {0};
    long long cnt[FDDPD_N_STAGES] = {0};
    for (int i = 0; i < p->nrec; ++i) {
        float t = 0.f;
        FD_CK(p, cudaEventElapsedTime(&t, p->ev[2 * i], p->ev[2 * i + 1]));
        acc[p->rec_stage[i]] += t;
        cnt[p->rec_stage[i]] += 1;
    }
    p->nrec = 0;
    for (int k = 0; k < FDDPD_N_STAGES; ++k) {
        if (ms) ms[k] = acc[k];
        if (count) count[k] = cnt[k];
    }
    return FDDPD_OK;
}

extern "C" const char *fddpd_stage_name(int stage) {
    return (stage >= 0 && stage < FDDPD_N_STAGES) ? kStageNames[stage] : nullptr;
}

extern "C" long long fddpd_launch_count(const fddpd_plan *p) { return p ? p->launches : 0; }

static int update_host_impl(fddpd_plan *p, int S, const fddpd_c32 *s, const fddpd_c32 *H,
                            const fddpd_c32 *pa_coef, float *theta, float lr, int iters, int optimizer,
                            double *metrics) {
    if (S < 1 || S > p->d.max_symbols) return set_err(p, FDDPD_ERR_ARG, "S=%d outside 1..%d", S, p->d.max_symbols);
    if (!s || !H || !pa_coef || !theta) return set_err(p, FDDPD_ERR_ARG, "null pointer");
    if (iters < 0) return set_err(p, FDDPD_ERR_ARG, "iters < 0");
    if (optimizer != FDDPD_GD && optimizer != FDDPD_ADAM) return set_err(p, FDDPD_ERR_ARG, "optimizer=%d", optimizer);
    const Geo &g = p->g;
    const long R = (S + g.S_per_real - 1) / g.S_per_real;
    const size_t n_s = sizeof(c32) * (size_t)p->d.max_symbols * g.K * g.N_d,
                 n_H = sizeof(c32) * (size_t)p->R_max * g.N_d * g.K * g.M,
                 n_al = sizeof(float) * (size_t)p->R_max * g.N_d,
                 n_pa = sizeof(c32) * (size_t)g.M * g.n_orders * (g.L + 1) * (1 + 2 * g.pa_G),
                 n_th = sizeof(float) * (size_t)g.theta_len;
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    if (!p->stage_base) {
        const size_t tot = up(n_s) + 2 * up(n_H) + up(n_al) + up(n_pa) + up(n_th) + up(8 * sizeof(double));
        if (dev_alloc(&p->stage_base, tot) != cudaSuccess) {
            cudaGetLastError();
            p->stage_base = nullptr;
            return set_err(p, FDDPD_ERR_NOMEM, "staging buffers (%zu bytes)", tot);
        }
        char *b = static_cast<char *>(p->stage_base);
        p->hs = (c32 *)b; b += up(n_s);
        p->hH = (c32 *)b; b += up(n_H);
        p->hW = (c32 *)b; b += up(n_H);
        p->hal = (float *)b; b += up(n_al);
        p->hpa = (c32 *)b; b += up(n_pa);
        p->htheta = (float *)b; b += up(n_th);
        p->hmet = (double *)b;
    }
    if (!p->cstream) {
        FD_CK(p, cudaStreamCreateWithFlags(&p->cstream, cudaStreamNonBlocking));
        for (int i = 0; i < kCopyChunks + 2; ++i) FD_CK(p, cudaEventCreateWithFlags(&p->cev[i], cudaEventDisableTiming));
    }
    // The batch crosses in chunks of whole realisations on the copy stream.  On the plan's
    // stream each chunk's ZF, forward and adjoint run as soon as its H and s have landed,
    // under the copy of the next chunk; the loss is normalised by the whole batch and the
    // gradient accumulates over the chunks.  The step itself waits for the last chunk and
    // for the check that every Gram matrix was positive definite.
    cudaStream_t st = p->stream, cs = p->cstream;
    const size_t h_real = sizeof(c32) * (size_t)g.N_d * g.K * g.M;   // one realisation of H (and of W)
    const size_t s_sym = sizeof(c32) * (size_t)g.K * g.N_d;          // one symbol of s
    // chunk c holds realisations [rb[c], rb[c + 1]): the first is half the size of the
    // others, so the step starts after a short copy; the rest split the remainder evenly
    long rb[kCopyChunks + 1];
    int nch = (int)std::min<long>(p->host_chunks, R);
    rb[0] = 0;
    if (nch > 1) {
        const long first = std::max<long>(1, R / (2 * nch - 1));
        rb[1] = first;
        for (int c = 2; c <= nch; ++c) rb[c] = first + (R - first) * (c - 1) / (nch - 1);
    } else {
        rb[1] = R;
    }
    const double inv_count = 1.0 / ((double)S * g.K * g.N_d);
    FD_CK(p, cudaEventRecord(p->cev[0], st));
    FD_CK(p, cudaStreamWaitEvent(cs, p->cev[0], 0));
    FD_CK(p, cudaMemcpyAsync(p->hpa, pa_coef, n_pa, cudaMemcpyHostToDevice, cs));
    FD_CK(p, cudaMemcpyAsync(p->htheta, theta, n_th, cudaMemcpyHostToDevice, cs));
    for (int c = 0; c < nch; ++c) {
        const long r0 = rb[c], r1 = rb[c + 1];
        const long t0 = r0 * g.S_per_real, t1 = r1 * g.S_per_real < S ? r1 * g.S_per_real : S;
        FD_CK(p, cudaMemcpyAsync((char *)p->hH + r0 * h_real, (const char *)H + r0 * h_real, (r1 - r0) * h_real,
                                 cudaMemcpyHostToDevice, cs));
        FD_CK(p, cudaMemcpyAsync((char *)p->hs + t0 * s_sym, (const char *)s + t0 * s_sym, (t1 - t0) * s_sym,
                                 cudaMemcpyHostToDevice, cs));
        FD_CK(p, cudaEventRecord(p->cev[1 + c], cs));
    }
    FD_CK(p, cudaMemsetAsync(p->status, 0, sizeof(int), st));
    const size_t h16_real = h_real / 2;
    // one iteration in a 16-bit plan: each chunk's precoder stays as its factors (H^H and the
    // chunk's Y, used right after by its own pass), so no W is formed at all
    const bool wfree = p->p16 && iters == 1;
    for (int c = 0; c < nch; ++c) {
        const long r0 = rb[c], r1 = rb[c + 1];
        const long t0 = r0 * g.S_per_real, t1 = r1 * g.S_per_real < S ? r1 * g.S_per_real : S;
        const c32 *Hc = (const c32 *)((const char *)p->hH + r0 * h_real);
        c32 *Wc = (c32 *)((char *)p->hW + r0 * h_real);
        float *alc = p->hal + r0 * g.N_d;
        FD_CK(p, cudaStreamWaitEvent(st, p->cev[1 + c], 0));
        void *W16c = p->p16 ? (char *)p->W16 + r0 * h16_real : nullptr;
        for (int ph = 0; ph < (wfree ? 2 : 3); ++ph)
            FD_STAGE(p, FDDPD_STAGE_ZF_GRAM + ph, 1,
                     fdk::zf_phase(ph, g, (int)(r1 - r0), Hc, Wc, alc, p->status, p->zf_scratch,
                                   p->p16 ? (char *)p->H16 + r0 * h16_real : nullptr, wfree ? nullptr : W16c,
                                   p->kind16, p->tc_bin, p->fp64_factor, p->status + 1, st,
                                   !p->p16,                        // 16-bit plans read only W's copy
                                   wfree ? W16c : nullptr));
        if (iters > 0) {
            const Pass ps{inv_count, c == 0, c == nch - 1, (int)r0};
            int rc1 = run_backward(p, (int)(t1 - t0), (const c32 *)((const char *)p->hs + t0 * s_sym), Hc,
                                   wfree ? nullptr : Wc, alc, p->hpa, p->htheta, p->grad, &ps);
            if (rc1) return rc1;
        }
    }
    if (p->p16) {   // the scratch holds only the last chunk's factor: no kept factor after this call
        p->pk_H = wfree ? nullptr : p->hH;
        p->pk_W = wfree ? nullptr : p->hW;
        p->pk_R = wfree ? 0 : (int)R;
        p->wfree = false;
    }
    // a singular Gram matrix fails the call before the step, leaving theta as it was
    FD_CK(p, cudaMemcpyAsync(p->status_host, p->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    FD_CK(p, cudaStreamSynchronize(st));
    if (p->status_host[0]) return set_err(p, FDDPD_ERR_SINGULAR, "a Gram matrix H_k H_k^H is not positive definite");
    if (iters > 0) {
        int rc2 = opt_step(p, p->htheta, lr, optimizer);
        if (rc2) return rc2;
        if (metrics) FD_CK(p, cudaMemcpyAsync(p->hmet, p->met, 5 * sizeof(double), cudaMemcpyDeviceToDevice, st));
        // further iterations over the batch, now resident
        rc2 = fddpd_update(p, S, (const fddpd_c32 *)p->hs, (const fddpd_c32 *)p->hH, (const fddpd_c32 *)p->hW,
                           p->hal, (const fddpd_c32 *)p->hpa, p->htheta, lr, iters - 1, optimizer, p->hmet);
        if (rc2) return rc2;
    }
    FD_CK(p, cudaMemcpyAsync(theta, p->htheta, n_th, cudaMemcpyDeviceToHost, st));
    if (metrics && iters > 0)
        FD_CK(p, cudaMemcpyAsync(metrics, p->hmet, 5 * sizeof(double), cudaMemcpyDeviceToHost, st));
    return fddpd_sync(p);
}

extern "C" int fddpd_update_host(fddpd_plan *p, int S, const fddpd_c32 *s, const fddpd_c32 *H,
                                 const fddpd_c32 *pa_coef, float *theta, float lr, int iters, int optimizer,
                                 double *metrics) {
    if (!p) return FDDPD_ERR_ARG;
    if (p->nn) return set_err(p, FDDPD_ERR_UNSUPPORTED, "FD-NN plans run the forward chain only");
    const int rc = update_host_impl(p, S, s, H, pa_coef, theta, lr, iters, optimizer, metrics);
    // a call that fails part-way may have copies of the caller's host arrays in flight:
    // they end before the call returns, so the caller may reuse or free the arrays (a
    // stream being recorded into a graph runs nothing, and is left alone)
    auto drain = [](cudaStream_t q) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(q, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone)
            cudaStreamSynchronize(q);
    };
    if (rc != FDDPD_OK) {
        if (p->cstream) drain(p->cstream);
        drain(p->stream);
    }
    return rc;
}

static int ser_impl(fddpd_plan *p, int S, const fddpd_c32 *y, const fddpd_c32 *s, const float *alpha, int Q, float N0,
                    unsigned long long seed, unsigned long long *counts, unsigned char *wrong) {
    if (!p) return FDDPD_ERR_ARG;
    if (S < 1 || S > p->d.max_symbols) return set_err(p, FDDPD_ERR_ARG, "S=%d outside 1..%d", S, p->d.max_symbols);
    if (!y || !s || !alpha || !counts) return set_err(p, FDDPD_ERR_ARG, "null pointer");
    if (Q != 4 && Q != 16 && Q != 64 && Q != 256 && Q != 1024) return set_err(p, FDDPD_ERR_ARG, "Q=%d", Q);
    if (!(N0 >= 0.0f)) return set_err(p, FDDPD_ERR_ARG, "N0 must be >= 0");
    if (!aligned(y, 8) || !aligned(s, 8) || !aligned(alpha, 4) || !aligned(counts, 8))
        return set_err(p, FDDPD_ERR_LAYOUT, "misaligned pointer");
    FD_CK(p, fdk::ser_count(p->g, S, reinterpret_cast<const c32 *>(y), reinterpret_cast<const c32 *>(s), alpha, Q, N0,
                            seed, counts, p->stream, wrong));
    p->launches += 1;
    return FDDPD_OK;
}

extern "C" int fddpd_ser(fddpd_plan *p, int S, const fddpd_c32 *y, const fddpd_c32 *s, const float *alpha, int Q,
                         float N0, unsigned long long seed, unsigned long long *counts) {
    return ser_impl(p, S, y, s, alpha, Q, N0, seed, counts, nullptr);
}

extern "C" int fddpd_ser_decisions(fddpd_plan *p, int S, const fddpd_c32 *y, const fddpd_c32 *s, const float *alpha,
                                   int Q, float N0, unsigned long long seed, unsigned long long *counts,
                                   unsigned char *wrong) {
    if (!p) return FDDPD_ERR_ARG;
    if (!wrong) return set_err(p, FDDPD_ERR_ARG, "wrong is null");
    return ser_impl(p, S, y, s, alpha, Q, N0, seed, counts, wrong);
}

extern "C" int fddpd_selftest_wait(fddpd_plan *p, int limit_us) {
    if (!p) return FDDPD_ERR_ARG;
    if (limit_us < 1 || limit_us > 1000000) return set_err(p, FDDPD_ERR_ARG, "limit_us outside 1..1000000");
    FD_CK(p, fdk::wait_probe(1000ull * (unsigned long long)limit_us, p->status + 1, p->stream));
    p->launches += 1;
    return FDDPD_OK;
}

// Choices of fddpd_autotune per shape: a plan of a shape met before takes the stored
// choice without timing (many instances of a few shapes in one batched launch).
struct TuneKey {
    int M, K, N, N_d, S_per_real, precision, n_orders, L, pa_G, per_user, L_U, G, S;
    bool operator<(const TuneKey &o) const {
        return std::tie(M, K, N, N_d, S_per_real, precision, n_orders, L, pa_G, per_user, L_U, G, S) <
               std::tie(o.M, o.K, o.N, o.N_d, o.S_per_real, o.precision, o.n_orders, o.L, o.pa_G, o.per_user, o.L_U,
                        o.G, o.S);
    }
};
struct TuneChoice {
    bool tc;
    int row_ctas, bin_ctas, bin_half;
    float ms[2];
};
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneChoice> g_tune_cache;

extern "C" int fddpd_autotune(fddpd_plan *p, int S, const fddpd_c32 *s, const fddpd_c32 *H, const fddpd_c32 *W,
                              const float *alpha, const fddpd_c32 *pa_coef, const float *theta, int reps,
                              float *ms) {
    if (!p) return FDDPD_ERR_ARG;
    if (p->nn) return set_err(p, FDDPD_ERR_UNSUPPORTED, "FD-NN plans have one implementation");
    if (reps < 1) return set_err(p, FDDPD_ERR_ARG, "reps < 1");
    const TuneKey key{p->g.M, p->g.K, p->g.N, p->g.N_d, p->g.S_per_real, p->d.precision, p->g.n_orders, p->g.L,
                      p->g.pa_G, p->dpd.per_user, p->dpd.L_U, p->dpd.G, S};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            p->tc_bin = it->second.tc;
            p->g.row_ctas = it->second.row_ctas;
            p->g.bin_ctas = it->second.bin_ctas;
            p->g.bin_half = it->second.bin_half;
            if (ms) {
                ms[0] = it->second.ms[0];
                ms[1] = it->second.ms[1];
            }
            return FDDPD_OK;
        }
    }
    // candidates: the contraction implementations the shape admits (tcgen05 in 16-bit plans
    // with M <= 256, K <= 32, at two or one CTAs per SM, with whole or half items; CUDA
    // cores) x the row kernels' CTAs per SM (as many as fit; one)
    float t[2][2][2][2];
    for (int a = 0; a < 16; ++a) (&t[0][0][0][0])[a] = -1.0f;
    const bool was_tc = p->tc_bin;
    const int was_rc = p->g.row_ctas, was_bc = p->g.bin_ctas, was_bh = p->g.bin_half;
    const bool tc_ok = p->p16 && fdk::tc_bin_supported(p->g);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    FD_CK(p, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return set_err(p, FDDPD_ERR_CUDA, "event creation failed");
    }
    int rc = FDDPD_OK;
    for (int v = 0; v < 2 && rc == FDDPD_OK; ++v) {
        if (v == 0 && !tc_ok) continue;
        for (int c = 0; c < 8 && rc == FDDPD_OK; ++c) {
            const int rcta = c & 1, bcta = (c >> 1) & 1, bhalf = c >> 2;
            if (v == 1 && (bcta || bhalf)) continue;   // the CUDA-core contractions have one form
            p->tc_bin = v == 0;
            p->g.row_ctas = rcta;
            p->g.bin_ctas = bcta;
            p->g.bin_half = bhalf;
            rc = fddpd_distort(p, S, s, H, W, alpha, pa_coef, theta, nullptr, nullptr);   // warm-up (and re-pack)
            if (rc) break;
            if (cudaEventRecord(e0, p->stream) != cudaSuccess) { rc = set_err(p, FDDPD_ERR_CUDA, "event record"); break; }
            for (int r = 0; r < reps && rc == FDDPD_OK; ++r)
                rc = fddpd_distort(p, S, s, H, W, alpha, pa_coef, theta, nullptr, nullptr);
            if (rc) break;
            float el = 0.0f;
            if (cudaEventRecord(e1, p->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&el, e0, e1) != cudaSuccess) {
                rc = set_err(p, FDDPD_ERR_CUDA, "event timing");
                break;
            }
            t[v][rcta][bcta][bhalf] = el / reps;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        p->tc_bin = was_tc;
        p->g.row_ctas = was_rc;
        p->g.bin_ctas = was_bc;
        p->g.bin_half = was_bh;
        return rc;
    }
    int bv = -1, br = 0, bb = 0, bh = 0;
    for (int v = 0; v < 2; ++v)
        for (int r = 0; r < 2; ++r)
            for (int b = 0; b < 2; ++b)
                for (int h = 0; h < 2; ++h)
                    if (t[v][r][b][h] >= 0 && (bv < 0 || t[v][r][b][h] < t[bv][br][bb][bh])) {
                        bv = v; br = r; bb = b; bh = h;
                    }
    p->tc_bin = bv == 0;
    p->g.row_ctas = br;
    p->g.bin_ctas = bb;
    p->g.bin_half = bh;
    TuneChoice ch{p->tc_bin, p->g.row_ctas, p->g.bin_ctas, p->g.bin_half, {-1.0f, -1.0f}};
    for (int v = 0; v < 2; ++v)
        for (int r = 0; r < 2; ++r)
            for (int b = 0; b < 2; ++b)
                for (int h = 0; h < 2; ++h)
                    if (t[v][r][b][h] >= 0 && (ch.ms[v] < 0 || t[v][r][b][h] < ch.ms[v])) ch.ms[v] = t[v][r][b][h];
    if (ms) {
        ms[0] = ch.ms[0];
        ms[1] = ch.ms[1];
    }
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = ch;
    }
    return fddpd_sync(p);
}

extern "C" int fddpd_autotune_forget(void) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache.clear();
    return FDDPD_OK;
}

// ---------------------------------------------------------------------------
// CUDA graphs over recorded calls of many plans (batched uneven workloads)
struct fddpd_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int lanes;
    cudaStream_t lane[FDDPD_GRAPH_MAX_LANES];
};

// Lanes of a recording in progress on this host thread: side streams forked from the
// recording stream at fddpd_graph_begin_lanes and joined back at fddpd_graph_end.
struct LaneSet {
    cudaStream_t main;
    int n;
    cudaStream_t lane[FDDPD_GRAPH_MAX_LANES];
    cudaEvent_t fork, join[FDDPD_GRAPH_MAX_LANES];
};
static thread_local LaneSet g_lanes{};

static void release_lanes(LaneSet &ls, bool streams) {
    if (ls.fork) cudaEventDestroy(ls.fork);
    for (int i = 0; i < ls.n; ++i) {
        if (ls.join[i]) cudaEventDestroy(ls.join[i]);
        if (streams && ls.lane[i]) cudaStreamDestroy(ls.lane[i]);
    }
    ls = LaneSet{};
}

extern "C" int fddpd_graph_begin_lanes(void *stream, int lanes, void **lane_streams) {
    if (!stream || !lane_streams || lanes < 1 || lanes > FDDPD_GRAPH_MAX_LANES)
        return set_err(nullptr, FDDPD_ERR_ARG, "fddpd_graph_begin_lanes: a stream, 1..%d lanes", FDDPD_GRAPH_MAX_LANES);
    if (g_lanes.n) return set_err(nullptr, FDDPD_ERR_ARG, "fddpd_graph_begin_lanes: a recording is in progress");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LaneSet ls{};
    ls.main = st;
    cudaError_t e = cudaEventCreateWithFlags(&ls.fork, cudaEventDisableTiming);
    for (int i = 0; i < lanes && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&ls.lane[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ls.join[i], cudaEventDisableTiming);
        ls.n = i + 1;
    }
    if (e == cudaSuccess) e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    bool capturing = e == cudaSuccess;
    if (e == cudaSuccess) e = cudaEventRecord(ls.fork, st);
    for (int i = 0; i < lanes && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(ls.lane[i], ls.fork, 0);
    if (e != cudaSuccess) {
        if (capturing) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(st, &g);
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();
        release_lanes(ls, true);
        return set_err(nullptr, FDDPD_ERR_CUDA, "fddpd_graph_begin_lanes: %s", cudaGetErrorString(e));
    }
    for (int i = 0; i < lanes; ++i) lane_streams[i] = ls.lane[i];
    g_lanes = ls;
    return FDDPD_OK;
}

extern "C" int fddpd_graph_begin(void *stream) {
    if (!stream) return set_err(nullptr, FDDPD_ERR_ARG, "fddpd_graph_begin: the default stream cannot record");
    const cudaError_t e = cudaStreamBeginCapture(static_cast<cudaStream_t>(stream), cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return set_err(nullptr, FDDPD_ERR_CUDA, "fddpd_graph_begin: %s", cudaGetErrorString(e));
    return FDDPD_OK;
}

extern "C" int fddpd_graph_end(void *stream, fddpd_graph **out) {
    if (!stream || !out) return set_err(nullptr, FDDPD_ERR_ARG, "fddpd_graph_end: null argument");
    *out = nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LaneSet ls{};
    if (g_lanes.n && g_lanes.main == st) {   // join the lanes back into the recording stream
        ls = g_lanes;
        g_lanes = LaneSet{};
        for (int i = 0; i < ls.n; ++i) {
            cudaEventRecord(ls.join[i], ls.lane[i]);
            cudaStreamWaitEvent(st, ls.join[i], 0);
        }
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        release_lanes(ls, true);
        return set_err(nullptr, FDDPD_ERR_CUDA, "fddpd_graph_end: %s", cudaGetErrorString(e));
    }
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        release_lanes(ls, true);
        return set_err(nullptr, FDDPD_ERR_CUDA, "fddpd_graph_end: instantiate: %s", cudaGetErrorString(e));
    }
    fddpd_graph *r = new (std::nothrow) fddpd_graph{};
    if (!r) {
        cudaGraphExecDestroy(x);
        cudaGraphDestroy(g);
        release_lanes(ls, true);
        return set_err(nullptr, FDDPD_ERR_NOMEM, "fddpd_graph_end: host allocation failed");
    }
    r->graph = g;
    r->exec = x;
    r->lanes = ls.n;   // the lane streams live as long as the graph (plans may still name them)
    for (int i = 0; i < ls.n; ++i) r->lane[i] = ls.lane[i];
    release_lanes(ls, false);
    *out = r;
    return FDDPD_OK;
}

extern "C" int fddpd_graph_launch(fddpd_graph *graph, void *stream) {
    if (!graph) return set_err(nullptr, FDDPD_ERR_ARG, "fddpd_graph_launch: null graph");
    const cudaError_t e = cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return set_err(nullptr, FDDPD_ERR_CUDA, "fddpd_graph_launch: %s", cudaGetErrorString(e));
    return FDDPD_OK;
}

extern "C" int fddpd_graph_destroy(fddpd_graph *graph) {
    if (!graph) return FDDPD_OK;
    cudaGraphExecDestroy(graph->exec);
    cudaGraphDestroy(graph->graph);
    for (int i = 0; i < graph->lanes; ++i) cudaStreamDestroy(graph->lane[i]);
    delete graph;
    return FDDPD_OK;
}

extern "C" int fddpd_sync(fddpd_plan *p) {
    if (!p) return FDDPD_ERR_ARG;
    FD_CK(p, cudaMemcpyAsync(p->status_host, p->status, 2 * sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    FD_CK(p, cudaStreamSynchronize(p->stream));
    if (p->status_host[1]) {
        FD_CK(p, cudaMemsetAsync(p->status + 1, 0, sizeof(int), p->stream));
        return set_err(p, FDDPD_ERR_TIMEOUT, "a bounded wait in a tensor-core kernel timed out");
    }
    return FDDPD_OK;
}

extern "C" int fddpd_tc_gemm(int M, int N, int K, const void *A, int lda, const void *B, int ldb, float *C, int ldc,
                             int ab_type, int splits, void *stream) {
    if (M < 0 || N < 0 || K < 0 || !A || !B || !C || lda < K || ldb < K || ldc < N || splits < 1 ||
        (ab_type != 0 && ab_type != 1))
        return set_err(nullptr, FDDPD_ERR_ARG, "fddpd_tc_gemm: bad argument");
    if ((lda % 8) || (ldb % 8) || !aligned(A, 16) || !aligned(B, 16) || !aligned(C, 4))
        return set_err(nullptr, FDDPD_ERR_LAYOUT, "fddpd_tc_gemm: A/B need 16-byte rows and alignment");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int *err = nullptr;
    int herr = 0;
    cudaError_t e = cudaMalloc(&err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
    const fdk::GemmArgs g{A, B, M, N, K, lda, ldb, ab_type, splits};
    if (e == cudaSuccess) e = fdk::tc_gemm_store(g, C, ldc, err, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (err) cudaFree(err);
    if (e != cudaSuccess) return set_err(nullptr, FDDPD_ERR_CUDA, "fddpd_tc_gemm: %s", cudaGetErrorString(e));
    if (herr) return set_err(nullptr, FDDPD_ERR_TIMEOUT, "fddpd_tc_gemm: bounded wait timed out");
    return FDDPD_OK;
}

extern "C" int fddpd_zf_residual(fddpd_plan *p, int R, const fddpd_c32 *H, const fddpd_c32 *W, int every,
                                 double *out) {
    if (!p) return FDDPD_ERR_ARG;
    if (R < 0 || R > p->R_max) return set_err(p, FDDPD_ERR_ARG, "R=%d outside 0..%d", R, p->R_max);
    if (every < 1) return set_err(p, FDDPD_ERR_ARG, "every=%d < 1", every);
    if (!H || !W || !out) return set_err(p, FDDPD_ERR_ARG, "null pointer");
    if (!aligned(H, 8) || !aligned(W, 8) || !aligned(out, 8)) return set_err(p, FDDPD_ERR_LAYOUT, "misaligned pointer");
    FD_CK(p, fdk::zf_residual(p->g, (long)R * p->g.N_d, every, reinterpret_cast<const c32 *>(H),
                              reinterpret_cast<const c32 *>(W), out, p->stream));
    p->launches += 1;
    return FDDPD_OK;
}

extern "C" int fddpd_alu_peak(int kind, double *tflops, void *stream) {
    if (kind < 0 || kind > 2 || !tflops) return set_err(nullptr, FDDPD_ERR_ARG, "fddpd_alu_peak: bad argument");
    const cudaError_t e = fdk::alu_peak(kind, tflops, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return set_err(nullptr, FDDPD_ERR_CUDA, "fddpd_alu_peak: %s", cudaGetErrorString(e));
    return FDDPD_OK;
}

// Error text for entry points that have no plan (see fddpd_last_error(NULL)).
void fddpd_internal_set_error(const char *msg) { set_err(nullptr, FDDPD_ERR_ARG, "%s", msg); }
