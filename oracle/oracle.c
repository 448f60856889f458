/*
 * FP64 CPU oracle of the frequency-domain DPD downlink chain (arxiv 2205.05158).
 *
 * TEST INFRASTRUCTURE ONLY: the plain definition the CUDA path is checked
 * against.  Nothing in the library links or calls it.  Direct O(N^2) DFTs,
 * an explicit Gauss-Jordan inverse of the Gram matrix, direct loops for the
 * PA, the convolution and the dense layer, and a hand-derived adjoint.  Each
 * function names the passage of the paper it follows.  Where the paper is
 * silent the readings used are:
 *   - both DFTs are unitary (1/sqrt(N)), as Eq. (2) and Sec. III-C state;
 *   - data subcarrier i sits at FFT bin (first_bin + i) mod N;
 *   - alpha is per subcarrier, alpha_k = sqrt(P_T / tr((H_k H_k^H)^{-1})),
 *     and the receiver equalises y_k / alpha_k;
 *   - PA memory taps wrap around the N-sample symbol (cyclic prefix >= L);
 *   - the FD-CNN output is added to its input (residual form) unless
 *     residual == 0, conv is a cross-correlation with zero "same" padding,
 *     and the loss is the mean of |y/alpha - s|^2 over the data bins.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Eq. (2): x_n = N^{-1/2} sum_k X_k e^{+j 2 pi k n / N}  (inverse = 1), and */
/* the unitary forward transform with e^{-j 2 pi k n / N} (inverse = 0).     */
/* ------------------------------------------------------------------------ */
void orc_dft(int N, const cplx *in, cplx *out, int inverse)
{
    cplx *tw = malloc(sizeof(cplx) * (size_t)N);
    cplx *tmp = malloc(sizeof(cplx) * (size_t)N);
    const double sgn = inverse ? 1.0 : -1.0;
    for (int m = 0; m < N; ++m) {
        double ang = sgn * 2.0 * M_PI * (double)m / (double)N;
        tw[m] = cos(ang) + I * sin(ang);
    }
    const double sc = 1.0 / sqrt((double)N);
    for (int k = 0; k < N; ++k) {
        cplx acc = 0;
        for (int n = 0; n < N; ++n) acc += in[n] * tw[((long)k * n) % N];
        tmp[k] = acc * sc;
    }
    memcpy(out, tmp, sizeof(cplx) * (size_t)N);
    free(tw);
    free(tmp);
}

/* Gauss-Jordan inverse with partial pivoting; A is overwritten. */
static int gj_inverse(int n, cplx *A, cplx *Ainv)
{
    double amax = 0;
    for (int i = 0; i < n * n; ++i) amax = fmax(amax, cabs(A[i]));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Ainv[i * n + j] = (i == j);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (cabs(A[r * n + c]) > cabs(A[piv * n + c])) piv = r;
        if (!(cabs(A[piv * n + c]) > 1e-13 * amax)) return -1;
        if (piv != c)
            for (int j = 0; j < n; ++j) {
                cplx t = A[c * n + j]; A[c * n + j] = A[piv * n + j]; A[piv * n + j] = t;
                t = Ainv[c * n + j]; Ainv[c * n + j] = Ainv[piv * n + j]; Ainv[piv * n + j] = t;
            }
        cplx p = 1.0 / A[c * n + c];
        for (int j = 0; j < n; ++j) { A[c * n + j] *= p; Ainv[c * n + j] *= p; }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            cplx f = A[r * n + c];
            if (f == 0) continue;
            for (int j = 0; j < n; ++j) {
                A[r * n + j] -= f * A[c * n + j];
                Ainv[r * n + j] -= f * Ainv[c * n + j];
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. (6): P_k = alpha H_k^H (H_k H_k^H)^{-1}.  Returns W = H^H (H H^H)^{-1} */
/* [M][K] and alpha_k = sqrt(P_T / tr((H H^H)^{-1})), so that                 */
/* E||alpha W s||^2 = P_T for unit-power symbols.                             */
/* ------------------------------------------------------------------------ */
int orc_zf(int K, int M, const cplx *Hk, double P_T, cplx *Wk, double *alpha)
{
    cplx *Gm = malloc(sizeof(cplx) * (size_t)K * K);
    cplx *Gi = malloc(sizeof(cplx) * (size_t)K * K);
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) {
            cplx acc = 0;
            for (int m = 0; m < M; ++m) acc += Hk[i * M + m] * conj(Hk[j * M + m]);
            Gm[i * K + j] = acc;
        }
    int rc = gj_inverse(K, Gm, Gi);
    if (rc == 0) {
        double tr = 0;
        for (int i = 0; i < K; ++i) tr += creal(Gi[i * K + i]);
        for (int m = 0; m < M; ++m)
            for (int u = 0; u < K; ++u) {
                cplx acc = 0;
                for (int v = 0; v < K; ++v) acc += conj(Hk[v * M + m]) * Gi[v * K + u];
                Wk[m * K + u] = acc;
            }
        *alpha = sqrt(P_T / tr);
    }
    free(Gm);
    free(Gi);
    return rc;
}

/* Eq. (6) for every data subcarrier of R realisations; nonzero if any is singular. */
int orc_precode_all(const orc_dims *d, int R, const cplx *H, cplx *W, double *alpha)
{
    const long nb = (long)R * d->N_d;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (long b = 0; b < nb; ++b)
        bad |= (orc_zf(d->K, d->M, H + b * d->K * d->M, d->P_T, W + b * d->M * d->K, alpha + b) != 0);
    return bad ? -3 : 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. (7) with the GMP of Eq. (9) restricted to its diagonal terms (G = 0):  */
/* y_n = sum_p sum_{l=0}^{L} c_{p,l} x_{n-l} |x_{n-l}|^{p-1}, taps circular.  */
/* c is [n_orders][L+1].                                                      */
/* ------------------------------------------------------------------------ */
void orc_pa(int N, const cplx *x, int n_orders, const int *orders, int L, const cplx *c, cplx *y)
{
    if (n_orders == 1 && orders[0] == 0) {   /* ideal linear-clipping PA (Sec. V-B), A = Re c */
        const double A = creal(c[0]);
        for (int n = 0; n < N; ++n) {
            const double r = cabs(x[n]);
            y[n] = r > A ? x[n] * (A / r) : x[n];
        }
        return;
    }
    for (int n = 0; n < N; ++n) {
        cplx acc = 0;
        for (int pi = 0; pi < n_orders; ++pi)
            for (int l = 0; l <= L; ++l) {
                cplx v = x[((n - l) % N + N) % N];
                acc += c[pi * (L + 1) + l] * v * pow(cabs(v), orders[pi] - 1);
            }
        y[n] = acc;
    }
}

/* Eq. (9) with its cross terms (the GMP): the lagging and leading envelope    */
/* |x_{n-l-+g}|^{p-1} multiplies x_{n-l}, for orders p >= 2 and g = 1..Gx.     */
static int wrapi(int i, int N) { return ((i % N) + N) % N; }

void orc_pa_gmp(int N, const cplx *x, int n_orders, const int *orders, int L, int Gx, const cplx *c, cplx *y)
{
    const int L1 = L + 1, PL = n_orders * L1;
    orc_pa(N, x, n_orders, orders, L, c, y);
    if (Gx <= 0) return;
    const cplx *cb = c + PL, *cc = c + PL + (long)PL * Gx;    /* b [P][L1][Gx], c [P][L1][Gx] */
    for (int n = 0; n < N; ++n)
        for (int pi = 0; pi < n_orders; ++pi) {
            const int e = orders[pi] - 1;
            if (e < 1) continue;
            for (int l = 0; l <= L; ++l)
                for (int g = 1; g <= Gx; ++g) {
                    const int k = (pi * L1 + l) * Gx + (g - 1);
                    const cplx v = x[wrapi(n - l, N)];
                    y[n] += cb[k] * v * pow(cabs(x[wrapi(n - l - g, N)]), e)
                          + cc[k] * v * pow(cabs(x[wrapi(n - l + g, N)]), e);
                }
        }
}

/* Wirtinger derivatives of phi_p(x) = x |x|^{p-1}:                          */
/* d phi / dx = (p+1)/2 |x|^{p-1},  d phi / dx* = (p-1)/2 x^2 |x|^{p-3}.      */
static void phi_derivs(int p, cplx x, double *a, cplx *b)
{
    double r = cabs(x);
    *a = 0.5 * (p + 1) * pow(r, p - 1);
    *b = (p == 1 || r == 0.0) ? 0.0 : 0.5 * (p - 1) * x * x * pow(r, p - 3);
}

/* ------------------------------------------------------------------------ */
/* FD-CNN (Sec. IV-A): each user's N_d data symbols fill a G x G grid row by  */
/* row (zero padded); L_U users (u, u+1, ... mod K) give 2 L_U real channels; */
/* N_conv kernels K_C x K_C with stride K_S and zero "same" padding, ReLU,    */
/* then a dense layer to 2 N_d outputs (Re rows then Im rows).               */
/* ------------------------------------------------------------------------ */
typedef struct { int G, Go, pad, Cin, F; long o_cb, o_fw, o_fb; } cnn_geo;

static cnn_geo geometry(const orc_dims *d)
{
    cnn_geo g;
    g.G = d->G;
    g.Go = (d->G + d->K_S - 1) / d->K_S;
    g.pad = d->K_C / 2;
    g.Cin = 2 * d->L_U;
    g.F = d->N_conv * g.Go * g.Go;
    g.o_cb = (long)d->N_conv * g.Cin * d->K_C * d->K_C;
    g.o_fw = g.o_cb + d->N_conv;
    g.o_fb = g.o_fw + 2L * d->N_d * g.F;
    return g;
}

static void cnn_input(const orc_dims *d, const cnn_geo *g, const cplx *s_sym, int u, double *X)
{
    const int GG = g->G * g->G;
    memset(X, 0, sizeof(double) * (size_t)g->Cin * GG);
    for (int l = 0; l < d->L_U; ++l) {
        int v = (u + l) % d->K;
        for (int i = 0; i < d->N_d; ++i) {
            X[(2 * l) * GG + i] = creal(s_sym[v * d->N_d + i]);
            X[(2 * l + 1) * GG + i] = cimag(s_sym[v * d->N_d + i]);
        }
    }
}

/* Sec. IV-A: the FD-CNN of one symbol for every user (pre / act: the conv layer). */
void orc_fdcnn(const orc_dims *d, const cplx *s_sym, const double *theta, cplx *s_tilde,
               double *pre, double *act)
{
    cnn_geo g = geometry(d);
    double *X = malloc(sizeof(double) * (size_t)g.Cin * g.G * g.G);
    double *a = malloc(sizeof(double) * (size_t)g.F);
    double *dd = malloc(sizeof(double) * 2 * (size_t)d->N_d);
    for (int u = 0; u < d->K; ++u) {
        /* one parameter set for all users, or user u's own (theta_u, stacked by user) */
        const double *th = theta + (d->per_user ? (long)u * (g.o_fb + 2L * d->N_d) : 0);
        const double *cw = th, *cb = th + g.o_cb, *fw = th + g.o_fw, *fb = th + g.o_fb;
        cnn_input(d, &g, s_sym, u, X);
        for (int o = 0; o < d->N_conv; ++o)
            for (int i = 0; i < g.Go; ++i)
                for (int j = 0; j < g.Go; ++j) {
                    double acc = cb[o];
                    for (int c = 0; c < g.Cin; ++c)
                        for (int p = 0; p < d->K_C; ++p)
                            for (int q = 0; q < d->K_C; ++q) {
                                int r = i * d->K_S + p - g.pad, t = j * d->K_S + q - g.pad;
                                if (r < 0 || r >= g.G || t < 0 || t >= g.G) continue;
                                acc += cw[((o * g.Cin + c) * d->K_C + p) * d->K_C + q] * X[(c * g.G + r) * g.G + t];
                            }
                    int f = (o * g.Go + i) * g.Go + j;
                    if (pre) pre[(long)u * g.F + f] = acc;
                    a[f] = acc > 0 ? acc : 0;
                    if (act) act[(long)u * g.F + f] = a[f];
                }
        for (int r = 0; r < 2 * d->N_d; ++r) {
            double acc = fb[r];
            const double *row = fw + (long)r * g.F;
            for (int f = 0; f < g.F; ++f) acc += row[f] * a[f];
            dd[r] = acc;
        }
        for (int i = 0; i < d->N_d; ++i)
            s_tilde[u * d->N_d + i] = (d->residual ? s_sym[u * d->N_d + i] : 0) + dd[i] + I * dd[d->N_d + i];
    }
    free(X);
    free(a);
    free(dd);
}

/* ------------------------------------------------------------------------ */
/* One OFDM symbol through Eq. (1) precoding, Eq. (2) IDFT, Eq. (7)/(9) PAs,  */
/* the unitary DFT and Eq. (5) combining by H_k (noise-free), followed by     */
/* equalisation y_k / alpha_k.                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    cplx *st;          /* [K][N_d]   predistorted symbols           */
    double *pre, *act; /* [K][F]     conv pre-activation, activation */
    cplx *x;           /* [M][N]     time-domain PA input           */
    cplx *yb;          /* [K][N_d]   equalised received symbols     */
} fwd_store;

static int bin_of(const orc_dims *d, int i) { return (d->first_bin + i) % d->N; }

static void forward_symbol(const orc_dims *d, const cplx *s_sym, const cplx *Hr, const cplx *Wr,
                           const double *al, const cplx *pa, const double *theta,
                           fwd_store *st, double *met)
{
    const int M = d->M, K = d->K, N = d->N, Nd = d->N_d, P = d->n_orders, L1 = d->L + 1;
    orc_fdcnn(d, s_sym, theta, st->st, st->pre, st->act);
    cplx *X = malloc(sizeof(cplx) * (size_t)M * N);
    double *gp = calloc((size_t)M, sizeof(double)), *dp = calloc((size_t)M, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int m = 0; m < M; ++m) {
        cplx *xh = calloc((size_t)N, sizeof(cplx));
        cplx *xpa = malloc(sizeof(cplx) * (size_t)N);
        for (int i = 0; i < Nd; ++i) {
            cplx acc = 0;
            for (int u = 0; u < K; ++u) acc += Wr[((long)i * M + m) * K + u] * st->st[u * Nd + i];
            xh[bin_of(d, i)] = al[i] * acc;
        }
        orc_dft(N, xh, st->x + (long)m * N, 1);
        orc_pa_gmp(N, st->x + (long)m * N, P, d->orders, d->L, d->Gx,
                   pa + (long)m * P * L1 * (1 + 2 * (d->Gx > 0 ? d->Gx : 0)), xpa);
        orc_dft(N, xpa, X + (long)m * N, 0);
        double gsum = 0, dat = 0;
        for (int k = 0; k < N; ++k) {
            cplx v = X[(long)m * N + k];
            if (((k - d->first_bin) % N + N) % N < Nd) dat += creal(v * conj(v));
            else gsum += creal(v * conj(v));
        }
        gp[m] = gsum;
        dp[m] = dat;
        free(xh);
        free(xpa);
    }
    for (int m = 0; m < M; ++m) { met[3] += gp[m]; met[4] += dp[m]; }
    for (int u = 0; u < K; ++u)
        for (int i = 0; i < Nd; ++i) {
            cplx acc = 0;
            for (int m = 0; m < M; ++m) acc += Hr[((long)i * K + u) * M + m] * X[(long)m * N + bin_of(d, i)];
            cplx yb = acc / al[i];
            cplx e = yb - s_sym[u * Nd + i];
            st->yb[u * Nd + i] = yb;
            met[1] += creal(e * conj(e));
            met[2] += creal(s_sym[u * Nd + i] * conj(s_sym[u * Nd + i]));
        }
    free(X);
    free(gp);
    free(dp);
}

static void store_alloc(const orc_dims *d, fwd_store *st)
{
    cnn_geo g = geometry(d);
    st->st = malloc(sizeof(cplx) * (size_t)d->K * d->N_d);
    st->pre = malloc(sizeof(double) * (size_t)d->K * g.F);
    st->act = malloc(sizeof(double) * (size_t)d->K * g.F);
    st->x = malloc(sizeof(cplx) * (size_t)d->M * d->N);
    st->yb = malloc(sizeof(cplx) * (size_t)d->K * d->N_d);
}

static void store_free(fwd_store *st)
{
    free(st->st); free(st->pre); free(st->act); free(st->x); free(st->yb);
}

static int check_dims(const orc_dims *d)
{
    if (d->M < 1 || d->K < 1 || d->N < 2 || d->N_d < 1 || d->N_d > d->N || d->S_per_real < 1) return -1;
    if (d->n_orders < 1 || d->n_orders > 8 || d->L < 0 || d->G * d->G < d->N_d) return -1;
    if (d->K_C < 1 || (d->K_C & 1) == 0 || d->K_S < 1 || d->N_conv < 1 || d->L_U < 1 || d->L_U > d->K) return -1;
    return 0;
}

/* The forward chain above over S symbols (symbol t on realisation t / S_per_real). */
int orc_distort(const orc_dims *d, int S, const cplx *s, const cplx *H, const cplx *W,
                const double *alpha, const cplx *pa, const double *theta, cplx *y, double *metrics)
{
    if (check_dims(d)) return -1;
    const long symN = (long)d->K * d->N_d, realN = (long)d->N_d * d->K * d->M;
    double met[5] = {0, 0, 0, 0, 0};
    fwd_store st;
    store_alloc(d, &st);
    for (int t = 0; t < S; ++t) {
        int r = t / d->S_per_real;
        forward_symbol(d, s + t * symN, H + r * realN, W + r * realN, alpha + (long)r * d->N_d,
                       pa, theta, &st, met);
        if (y) memcpy(y + t * symN, st.yb, sizeof(cplx) * (size_t)symN);
    }
    store_free(&st);
    met[0] = met[1] / ((double)S * symN);
    if (metrics) memcpy(metrics, met, sizeof met);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. III-C: the FD-NN comparison DPD (see oracle.h for the parameter and    */
/* input order).  Step by step: U IDFTs, the network at every time sample,     */
/* U DFTs.                                                                     */
/* ------------------------------------------------------------------------ */
void orc_fdnn(const orc_dims *d, const cplx *s_sym, const double *theta, cplx *s_dpd)
{
    const int U = d->K, N = d->N, Nd = d->N_d, L1 = d->nn_L4 + 1, D = d->nn_D, NL = d->nn_layers;
    const int nin = 2 * U * L1;
    cplx *t = malloc(sizeof(cplx) * (size_t)U * N);     /* time-domain user streams */
    cplx *o = malloc(sizeof(cplx) * (size_t)U * N);     /* predistorted streams     */
    cplx *fd = calloc((size_t)N, sizeof(cplx));
    for (int u = 0; u < U; ++u) {
        for (int k = 0; k < N; ++k) fd[k] = 0;
        for (int i = 0; i < Nd; ++i) fd[bin_of(d, i)] = s_sym[u * Nd + i];
        orc_dft(N, fd, t + (long)u * N, 1);
    }
    const double *W0 = theta, *b0 = W0 + (long)D * nin;
    const double *hid = b0 + D;                          /* (W_k, b_k), k = 1..NL-1 */
    const double *Wo = hid + (long)(NL - 1) * (D * D + D), *bo = Wo + (long)2 * U * D;
#pragma omp parallel for schedule(static)
    for (int n = 0; n < N; ++n) {
        double *in = malloc(sizeof(double) * (size_t)nin);
        double *h = malloc(sizeof(double) * (size_t)D), *h2 = malloc(sizeof(double) * (size_t)D);
        for (int u = 0; u < U; ++u)
            for (int l = 0; l < L1; ++l) {
                const cplx v = t[(long)u * N + wrapi(n - l, N)];
                in[u * L1 + l] = creal(v);
                in[U * L1 + u * L1 + l] = cimag(v);
            }
        for (int a = 0; a < D; ++a) {
            double acc = b0[a];
            for (int j = 0; j < nin; ++j) acc += W0[(long)a * nin + j] * in[j];
            h[a] = acc > 0 ? acc : 0;
        }
        for (int k = 1; k < NL; ++k) {
            const double *Wk = hid + (long)(k - 1) * (D * D + D), *bk = Wk + (long)D * D;
            for (int a = 0; a < D; ++a) {
                double acc = bk[a];
                for (int j = 0; j < D; ++j) acc += Wk[a * D + j] * h[j];
                h2[a] = acc > 0 ? acc : 0;
            }
            memcpy(h, h2, sizeof(double) * (size_t)D);
        }
        for (int u = 0; u < U; ++u) {
            double re = bo[u], im = bo[U + u];
            for (int a = 0; a < D; ++a) {
                re += Wo[(long)u * D + a] * h[a];
                im += Wo[(long)(U + u) * D + a] * h[a];
            }
            o[(long)u * N + n] = (d->residual ? t[(long)u * N + n] : 0) + re + I * im;
        }
        free(in); free(h); free(h2);
    }
    for (int u = 0; u < U; ++u) orc_dft(N, o + (long)u * N, s_dpd + (long)u * N, 0);
    free(t); free(o); free(fd);
}

int orc_fdnn_distort(const orc_dims *d, int S, const cplx *s, const cplx *H, const cplx *W_all,
                     const double *alpha_all, const cplx *pa, const double *theta, cplx *y, double *metrics)
{
    if (d->M < 1 || d->K < 1 || d->N < 2 || d->N_d < 1 || d->N_d > d->N || d->S_per_real < 1) return -1;
    if (d->nn_L4 < 0 || d->nn_D < 1 || d->nn_layers < 1 || d->n_orders < 1 || d->L < 0) return -1;
    const int M = d->M, K = d->K, N = d->N, Nd = d->N_d, P = d->n_orders, L1 = d->L + 1;
    const long symN = (long)K * Nd;
    double met[5] = {0, 0, 0, 0, 0};
    cplx *sd = malloc(sizeof(cplx) * (size_t)K * N);
    cplx *X = malloc(sizeof(cplx) * (size_t)M * N);
    double *gp = malloc(sizeof(double) * (size_t)M), *dp = malloc(sizeof(double) * (size_t)M);
    for (int t = 0; t < S; ++t) {
        const int r = t / d->S_per_real;
        const cplx *Wr = W_all + (long)r * N * M * K, *Hr = H + (long)r * Nd * K * M;
        const double *al = alpha_all + (long)r * N;
        const cplx *s_sym = s + t * symN;
        orc_fdnn(d, s_sym, theta, sd);
#pragma omp parallel for schedule(static)
        for (int m = 0; m < M; ++m) {
            cplx *xh = malloc(sizeof(cplx) * (size_t)N), *x = malloc(sizeof(cplx) * (size_t)N);
            cplx *xpa = malloc(sizeof(cplx) * (size_t)N);
            for (int k = 0; k < N; ++k) {          /* every bin is precoded (Sec. III-C) */
                cplx acc = 0;
                for (int u = 0; u < K; ++u) acc += Wr[((long)k * M + m) * K + u] * sd[(long)u * N + k];
                xh[k] = al[k] * acc;
            }
            orc_dft(N, xh, x, 1);
            orc_pa_gmp(N, x, P, d->orders, d->L, d->Gx, pa + (long)m * P * L1 * (1 + 2 * (d->Gx > 0 ? d->Gx : 0)), xpa);
            orc_dft(N, xpa, X + (long)m * N, 0);
            double gsum = 0, dat = 0;
            for (int k = 0; k < N; ++k) {
                const cplx v = X[(long)m * N + k];
                if (((k - d->first_bin) % N + N) % N < Nd) dat += creal(v * conj(v));
                else gsum += creal(v * conj(v));
            }
            gp[m] = gsum;
            dp[m] = dat;
            free(xh); free(x); free(xpa);
        }
        for (int m = 0; m < M; ++m) { met[3] += gp[m]; met[4] += dp[m]; }
        for (int u = 0; u < K; ++u)
            for (int i = 0; i < Nd; ++i) {
                const int k = bin_of(d, i);
                cplx acc = 0;
                for (int m = 0; m < M; ++m) acc += Hr[((long)i * K + u) * M + m] * X[(long)m * N + k];
                const cplx yb = acc / al[k], e = yb - s_sym[u * Nd + i];
                if (y) y[t * symN + u * Nd + i] = yb;
                met[1] += creal(e * conj(e));
                met[2] += creal(s_sym[u * Nd + i] * conj(s_sym[u * Nd + i]));
            }
    }
    free(sd); free(X); free(gp); free(dp);
    met[0] = met[1] / ((double)S * symN);
    if (metrics) memcpy(metrics, met, sizeof met);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the whole chain for L = mean |y/alpha - s|^2 (Sec. V-A training */
/* criterion).  Gradients of a real L w.r.t. a complex z are carried as       */
/* g(z) = dL/dRe z + j dL/dIm z; a complex-linear map A has adjoint A^H, and  */
/* w = f(z, z*) gives g(z) = conj(df/dz) g(w) + (df/dz*) conj(g(w)).         */
/* The time-domain PA input is recomputed by the forward, as the GPU does.    */
/* ------------------------------------------------------------------------ */
static void backward_symbol(const orc_dims *d, const cplx *s_sym, const cplx *Hr, const cplx *Wr,
                            const double *al, const cplx *pa, const double *theta, const fwd_store *st,
                            double inv_count, double *grad)
{
    const int M = d->M, K = d->K, N = d->N, Nd = d->N_d, P = d->n_orders, L1 = d->L + 1;
    cnn_geo g = geometry(d);
    cplx *gy = malloc(sizeof(cplx) * (size_t)K * Nd);
    for (int j = 0; j < K * Nd; ++j) gy[j] = 2.0 * (st->yb[j] - s_sym[j]) * inv_count;
    cplx *gxh = malloc(sizeof(cplx) * (size_t)M * N);
#pragma omp parallel for schedule(static)
    for (int m = 0; m < M; ++m) {
        cplx *gX = calloc((size_t)N, sizeof(cplx));
        cplx *gpa = malloc(sizeof(cplx) * (size_t)N);
        cplx *gx = malloc(sizeof(cplx) * (size_t)N);
        for (int i = 0; i < Nd; ++i) {          /* adjoint of y = H X / alpha      */
            cplx acc = 0;
            for (int u = 0; u < K; ++u) acc += conj(Hr[((long)i * K + u) * M + m]) * gy[u * Nd + i];
            gX[bin_of(d, i)] = acc / al[i];
        }
        orc_dft(N, gX, gpa, 1);                 /* adjoint of the unitary DFT      */
        const cplx *x = st->x + (long)m * N;
        const int Gx = d->Gx > 0 ? d->Gx : 0;
        const cplx *c = pa + (long)m * P * L1 * (1 + 2 * Gx);
        const int clip = P == 1 && d->orders[0] == 0;
        for (int n = 0; n < N && clip; ++n) {   /* adjoint of the clipping PA:      */
            const double A = creal(c[0]), r = cabs(x[n]);   /* above A, df/dx = A/(2r),  */
            gx[n] = r > A ? (A / (2 * r)) * gpa[n]          /* df/dx* = -A x^2/(2 r^3)  */
                              - (A / (2 * r * r * r)) * x[n] * x[n] * conj(gpa[n])
                          : gpa[n];
        }
        for (int n = 0; n < N && !clip; ++n) {  /* adjoint of the PA               */
            cplx acc = 0;
            for (int pi = 0; pi < P; ++pi) {
                cplx h = 0;
                for (int l = 0; l <= d->L; ++l) h += conj(c[pi * L1 + l]) * gpa[(n + l) % N];
                double a; cplx b;
                phi_derivs(d->orders[pi], x[n], &a, &b);
                acc += a * h + b * conj(h);
            }
            gx[n] = acc;
        }
        /* adjoint of the cross terms T = b x_j e(x_i), e = |x_i|^E, i = j -+ g, j = n - l:
         * to x_j: conj(b e(x_i)) g_n; to x_i (de/dx = E/2 |x|^{E-2} x*, de/dx* = E/2 |x|^{E-2} x):
         * E/2 |x_i|^{E-2} (conj(b x_j) x_i g_n + b x_j x_i conj(g_n))                       */
        const cplx *cb = c + P * L1, *cc = c + P * L1 + (long)P * L1 * Gx;
        for (int n = 0; n < N && Gx > 0; ++n)
            for (int pi = 0; pi < P; ++pi) {
                const int E = d->orders[pi] - 1;
                if (E < 1) continue;
                for (int l = 0; l <= d->L; ++l)
                    for (int gg = 1; gg <= Gx; ++gg)
                        for (int side = 0; side < 2; ++side) {
                            const cplx b = side ? cc[(pi * L1 + l) * Gx + gg - 1] : cb[(pi * L1 + l) * Gx + gg - 1];
                            const int j = wrapi(n - l, N), i = wrapi(side ? n - l + gg : n - l - gg, N);
                            const double r = cabs(x[i]);
                            gx[j] += conj(b * pow(r, E)) * gpa[n];
                            if (r > 0.0)
                                gx[i] += 0.5 * E * pow(r, E - 2) *
                                         (conj(b * x[j]) * x[i] * gpa[n] + b * x[j] * x[i] * conj(gpa[n]));
                        }
            }
        orc_dft(N, gx, gxh + (long)m * N, 0);   /* adjoint of the unitary IDFT     */
        free(gX); free(gpa); free(gx);
    }
    /* adjoint of x_hat = alpha W s_tilde, then of the FD-CNN */
    double *gd = malloc(sizeof(double) * 2 * (size_t)Nd);
    double *ga = malloc(sizeof(double) * (size_t)g.F);
    double *X = malloc(sizeof(double) * (size_t)g.Cin * g.G * g.G);
    const long len1 = g.o_fb + 2L * Nd;   /* one parameter set */
    for (int u = 0; u < K; ++u) {
        const long off = d->per_user ? (long)u * len1 : 0;
        double *gcw = grad + off, *gcb = grad + off + g.o_cb, *gfw = grad + off + g.o_fw, *gfb = grad + off + g.o_fb;
        const double *fw = theta + off + g.o_fw;
        for (int i = 0; i < Nd; ++i) {
            cplx acc = 0;
            for (int m = 0; m < M; ++m) acc += conj(Wr[((long)i * M + m) * K + u]) * gxh[(long)m * N + bin_of(d, i)];
            acc *= al[i];
            gd[i] = creal(acc);
            gd[Nd + i] = cimag(acc);
        }
        const double *a = st->act + (long)u * g.F, *pre = st->pre + (long)u * g.F;
        for (int r = 0; r < 2 * Nd; ++r) {
            gfb[r] += gd[r];
            double *grow = gfw + (long)r * g.F;
            for (int f = 0; f < g.F; ++f) grow[f] += gd[r] * a[f];
        }
        for (int f = 0; f < g.F; ++f) {
            double acc = 0;
            for (int r = 0; r < 2 * Nd; ++r) acc += fw[(long)r * g.F + f] * gd[r];
            ga[f] = pre[f] > 0 ? acc : 0;
        }
        cnn_input(d, &g, s_sym, u, X);
        for (int o = 0; o < d->N_conv; ++o)
            for (int i = 0; i < g.Go; ++i)
                for (int j = 0; j < g.Go; ++j) {
                    double gv = ga[(o * g.Go + i) * g.Go + j];
                    if (gv == 0) continue;
                    gcb[o] += gv;
                    for (int c = 0; c < g.Cin; ++c)
                        for (int p = 0; p < d->K_C; ++p)
                            for (int q = 0; q < d->K_C; ++q) {
                                int r = i * d->K_S + p - g.pad, t = j * d->K_S + q - g.pad;
                                if (r < 0 || r >= g.G || t < 0 || t >= g.G) continue;
                                gcw[((o * g.Cin + c) * d->K_C + p) * d->K_C + q] += gv * X[(c * g.G + r) * g.G + t];
                            }
                }
    }
    free(gd); free(ga); free(X); free(gy); free(gxh);
}

static long theta_len(const orc_dims *d)
{
    cnn_geo g = geometry(d);
    return (g.o_fb + 2L * d->N_d) * (d->per_user ? d->K : 1);
}

/* Sec. V-A: gradient of the symbol MSE over S symbols by the adjoint above.     */
int orc_backward(const orc_dims *d, int S, const cplx *s, const cplx *H, const cplx *W,
                 const double *alpha, const cplx *pa, const double *theta, double *grad, double *metrics)
{
    if (check_dims(d)) return -1;
    const long symN = (long)d->K * d->N_d, realN = (long)d->N_d * d->K * d->M;
    memset(grad, 0, sizeof(double) * (size_t)theta_len(d));
    double met[5] = {0, 0, 0, 0, 0};
    const double inv_count = 1.0 / ((double)S * symN);
    fwd_store st;
    store_alloc(d, &st);
    for (int t = 0; t < S; ++t) {
        int r = t / d->S_per_real;
        const cplx *Hr = H + r * realN, *Wr = W + r * realN;
        const double *al = alpha + (long)r * d->N_d;
        forward_symbol(d, s + t * symN, Hr, Wr, al, pa, theta, &st, met);
        backward_symbol(d, s + t * symN, Hr, Wr, al, pa, theta, &st, inv_count, grad);
    }
    store_free(&st);
    met[0] = met[1] * inv_count;
    if (metrics) memcpy(metrics, met, sizeof met);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Parameter update (Sec. V-A): plain gradient descent, or Adam (Kingma & Ba) */
/* with beta1 = 0.9, beta2 = 0.999, eps = 1e-8; one iteration = forward,      */
/* adjoint and one step over the S symbols.                                   */
/* ------------------------------------------------------------------------ */
int orc_update(const orc_dims *d, int S, const cplx *s, const cplx *H, const cplx *W,
               const double *alpha, const cplx *pa, double *theta, double lr, int iters, int adam,
               double *m1, double *m2, int *t_adam, double *metrics)
{
    const long n = theta_len(d);
    double *g = malloc(sizeof(double) * (size_t)n);
    for (int it = 0; it < iters; ++it) {
        int rc = orc_backward(d, S, s, H, W, alpha, pa, theta, g, metrics);
        if (rc) { free(g); return rc; }
        if (!adam) {
            for (long j = 0; j < n; ++j) theta[j] -= lr * g[j];
        } else {
            const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
            int t = ++(*t_adam);
            double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
            for (long j = 0; j < n; ++j) {
                m1[j] = b1 * m1[j] + (1 - b1) * g[j];
                m2[j] = b2 * m2[j] + (1 - b2) * g[j] * g[j];
                theta[j] -= lr * (m1[j] / c1) / (sqrt(m2[j] / c2) + eps);
            }
        }
    }
    free(g);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11): ten rounds; each multiplies counter words 0 and  */
/* 2 by 0xD2511F53 and 0xCD9E8D57 (64-bit products), XORs the high halves     */
/* with words 1 and 3 and the key, and permutes; the key is bumped by the     */
/* Weyl constants 0x9E3779B9 and 0xBB67AE85 between rounds.                   */
void orc_philox4x32_10(const unsigned int ctr[4], const unsigned int key[2], unsigned int out[4])
{
    unsigned long long c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    unsigned int k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = 0xD2511F53ull * c0, p1 = 0xCD9E8D57ull * c2;
        const unsigned long long n0 = (p1 >> 32) ^ c1 ^ k0, n1 = p1 & 0xFFFFFFFFull;
        const unsigned long long n2 = (p0 >> 32) ^ c3 ^ k1, n3 = p0 & 0xFFFFFFFFull;
        c0 = n0 & 0xFFFFFFFFull; c1 = n1; c2 = n2 & 0xFFFFFFFFull; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = (unsigned int)c0; out[1] = (unsigned int)c1; out[2] = (unsigned int)c2; out[3] = (unsigned int)c3;
}

/* nearest level index of the side-point PAM with levels (2 i - side + 1) / scale */
static int pam_nearest(double v, double scale, int side)
{
    int best = 0;
    double bd = INFINITY;
    for (int i = 0; i < side; ++i) {
        const double d = fabs(v - (2.0 * i - side + 1) / scale);
        if (d < bd) { bd = d; best = i; }
    }
    return best;
}

/* Sec. V-B (SER at the users) with the noise of Eq. (4)-(5) under the unitary DFT:  */
/* the per-subcarrier noise is CN(0, N0), and the user equalises by 1 / alpha_k.    */
int orc_ser(const orc_dims *d, int S, const cplx *y, const cplx *s, const double *alpha, int Q, double N0,
            unsigned long long seed, cplx *z, int *wrong, long long *counts)
{
    int side = 1;
    while (side * side < Q) ++side;
    if (side * side != Q || S < 0) return -1;
    const double scale = sqrt(2.0 * (Q - 1) / 3.0);          /* unit mean power */
    const unsigned int key[2] = {(unsigned int)seed, (unsigned int)(seed >> 32)};
    const long long n = (long long)S * d->K * d->N_d;
    long long errors = 0, compared = 0;
    for (long long e = 0; e < n; ++e) {
        const long long t = e / ((long long)d->K * d->N_d);
        const int i = (int)(e % d->N_d);
        const double al = alpha[(t / d->S_per_real) * d->N_d + i];
        if (wrong) wrong[e] = 0;
        if (!(al > 0.0)) {
            if (z) z[e] = y[e];
            continue;
        }
        cplx w = 0.0;
        if (N0 > 0.0) {
            const unsigned int ctr[4] = {(unsigned int)e, (unsigned int)((unsigned long long)e >> 32), 0u, 0u};
            unsigned int r[4];
            orc_philox4x32_10(ctr, key, r);
            const double u1 = ((double)r[0] + 0.5) / 4294967296.0, u2 = ((double)r[1] + 0.5) / 4294967296.0;
            w = sqrt(N0) * sqrt(-log(u1)) * (cos(2.0 * M_PI * u2) + I * sin(2.0 * M_PI * u2));
        }
        const cplx zz = y[e] + w / al;
        if (z) z[e] = zz;
        const int bad = pam_nearest(creal(zz), scale, side) != pam_nearest(creal(s[e]), scale, side) ||
                        pam_nearest(cimag(zz), scale, side) != pam_nearest(cimag(s[e]), scale, side);
        if (wrong) wrong[e] = bad;
        errors += bad;
        ++compared;
    }
    counts[0] = errors;
    counts[1] = compared;
    return 0;
}
