/*
 * FP64 CPU oracle of the frequency-domain DPD downlink chain (arxiv 2205.05158).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, obviously correct
 * definition the CUDA path is checked against.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the library never
 * does.  It shares no code, header or table with the CUDA path.
 *
 * Complex numbers are C99 `double complex`; all arrays are row-major.
 *   s      [S][K][N_d]          user symbols (data bins, increasing frequency)
 *   H      [R][N_d][K][M]       per-subcarrier channel, R = ceil(S / S_per_real)
 *   W      [R][N_d][M][K]       unnormalised ZF precoder H^H (H H^H)^{-1}
 *   alpha  [R][N_d]             per-subcarrier power normalisation
 *   pa     [M][P][L+1]          memory-polynomial coefficients c^b_{p,l} when Gx = 0;
 *                               with Gx > 0 each antenna holds a [P][L+1], then the lagging
 *                               b [P][L+1][Gx] and the leading c [P][L+1][Gx] of Eq. (9)
 *                               (order-1 cross slots unused); orders = {0}
 *                               with L = 0 is the ideal linear-clipping PA of clipping
 *                               amplitude A = Re c^b_{0,0}
 *   theta  flat: conv_w[N_conv][2L_U][K_C][K_C], conv_b[N_conv],
 *                fc_w[2N_d][N_conv*Go*Go], fc_b[2N_d]   (Go = ceil(G/K_S))
 * metrics[5] = { loss, sum|y/alpha - s|^2, sum|s|^2, guard-bin power, data-bin power }
 */
#ifndef FDDPD_ORACLE_H
#define FDDPD_ORACLE_H
#include <complex.h>

typedef struct {
    int M, K, N, N_d, first_bin;
    int S_per_real;
    int n_orders, orders[8], L;
    int G, L_U, K_C, K_S, N_conv, residual;
    double P_T;
    int Gx;   /* PA cross-term length (Eq. 9): 0 = memory polynomial */
    int per_user;  /* 1: every user u has its own FD-CNN parameters theta_u (Sec. IV-A) */
    /* FD-NN of Sec. III-C (the comparison workload): memory length L_4, D neurons per hidden
     * layer, K^NN hidden layers; its residual form follows `residual` above               */
    int nn_L4, nn_D, nn_layers;
} orc_dims;

int  orc_num_threads(void);
void orc_dft(int N, const double complex *in, double complex *out, int inverse);
int  orc_zf(int K, int M, const double complex *Hk, double P_T, double complex *Wk, double *alpha);
int  orc_precode_all(const orc_dims *d, int R, const double complex *H, double complex *W, double *alpha);
void orc_pa(int N, const double complex *x, int n_orders, const int *orders, int L,
            const double complex *c, double complex *y);
/* Eq. (9) with cross terms: y_n = sum_p sum_l a_{p,l} x_{n-l} |x_{n-l}|^{p-1}
 *   + sum_{p>=2} sum_l sum_{g=1..Gx} (b_{p,l,g} x_{n-l} |x_{n-l-g}|^{p-1} + c_{p,l,g} x_{n-l} |x_{n-l+g}|^{p-1}),
 * indices circular in n; coefficients as described for pa above.                 */
void orc_pa_gmp(int N, const double complex *x, int n_orders, const int *orders, int L, int Gx,
                const double complex *c, double complex *y);
void orc_fdcnn(const orc_dims *d, const double complex *s_sym, const double *theta,
               double complex *s_tilde, double *pre, double *act);
int  orc_distort(const orc_dims *d, int S, const double complex *s, const double complex *H,
                 const double complex *W, const double *alpha, const double complex *pa,
                 const double *theta, double complex *y, double *metrics);
int  orc_backward(const orc_dims *d, int S, const double complex *s, const double complex *H,
                  const double complex *W, const double *alpha, const double complex *pa,
                  const double *theta, double *grad, double *metrics);
int  orc_update(const orc_dims *d, int S, const double complex *s, const double complex *H,
                const double complex *W, const double *alpha, const double complex *pa,
                double *theta, double lr, int iters, int adam, double *adam_m, double *adam_v,
                int *adam_t, double *metrics);
/* FD-NN of Sec. III-C for one OFDM symbol: each user's symbols (data bins, guard bins
 * zero) go to the time domain by the unitary IDFT; at every sample n a fully connected
 * network with K^NN ReLU hidden layers of D neurons maps the real and imaginary parts of
 * s_u[n], s_u[n-1], ..., s_u[n-L_4] of all users (taps circular in n) to 2U outputs, the
 * predistorted time-domain sample of every user (added to s_u[n] when residual = 1);
 * the unitary DFT takes each user back to all N bins.
 *   s_sym [K][N_d] in, s_dpd [K][N] out (every bin, natural order)
 *   theta: W_0 [D][2U(L_4+1)], b_0 [D], (W_k [D][D], b_k [D]) for k = 1..K^NN-1,
 *          W_o [2U][D], b_o [2U]; input j < U(L_4+1) is Re s_u[n-l] at j = u(L_4+1) + l,
 *          the imaginary parts follow; output u is the real part, U + u the imaginary. */
void orc_fdnn(const orc_dims *d, const double complex *s_sym, const double *theta, double complex *s_dpd);
/* The FD-NN chain over S symbols: FD-NN, ZF precoding of EVERY subcarrier (guard bins
 * too, with W_all [R][N][M][K], alpha_all [R][N] indexed by FFT bin), IDFT, PA, DFT,
 * combining at the data bins with H [R][N_d][K][M], equalised by alpha_all at the data
 * bins; metrics as orc_distort.                                                      */
int  orc_fdnn_distort(const orc_dims *d, int S, const double complex *s, const double complex *H,
                      const double complex *W_all, const double *alpha_all, const double complex *pa,
                      const double *theta, double complex *y, double *metrics);
/* Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ctr[4], key[2] -> out[4]. */
void orc_philox4x32_10(const unsigned int ctr[4], const unsigned int key[2], unsigned int out[4]);
/* Symbol errors at the users (Sec. V-B; noise of Eq. 4-5): z = y + w / alpha with
 * w ~ CN(0, N0) drawn by Philox-4x32-10 (key = seed, counter = (flat index, 0, 0), first
 * two outputs u = (x + 1/2) 2^-32, w = sqrt(N0) sqrt(-ln u1) e^{j 2 pi u2}), decided to the
 * nearest unit-power square Q-QAM point.  Subcarriers with alpha <= 0 are skipped.
 *   z [S][K][N_d] out (may be NULL), wrong [S][K][N_d] out 0/1 (may be NULL)
 *   counts[2] out: errors, symbols compared                                       */
int  orc_ser(const orc_dims *d, int S, const double complex *y, const double complex *s,
             const double *alpha, int Q, double N0, unsigned long long seed, double complex *z,
             int *wrong, long long *counts);
#endif
