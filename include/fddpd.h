/*
 * fddpd — frequency-domain digital predistortion for the massive MU-MIMO-OFDM
 * downlink (arxiv 2205.05158), as a C-ABI library for one sm_103a GPU.
 *
 * Per OFDM symbol the library computes, on the GPU:
 *   s_tilde = s + FD-CNN_theta(s)            (Sec. IV-A; residual form, see residual)
 *   x_hat_k = alpha_k W_k s_tilde_k          (Eq. 1 with the ZF precoder of Eq. 6)
 *   x_b     = IDFT_N(x_hat_{.,b})            (Eq. 2, unitary; guard bins zero)
 *   x^PA_b  = PA_b(x_b)                      (Eq. 7: the GMP of Eq. 9, or the clipping PA)
 *   y_k     = H_k DFT_N(x^PA)_k / alpha_k    (Eq. 4-5, noise free, then equalised)
 *   loss    = mean |y - s|^2                 (training criterion, Sec. V-A)
 * and its adjoint with respect to theta, and gradient-descent / Adam updates.
 *
 * Conventions shared by every entry point
 *   - Complex values are interleaved (re, im) FP32 (fddpd_c32).  All arrays are
 *     row-major, densely packed, 8-byte aligned device memory unless stated.
 *   - Data subcarrier i (0 <= i < N_d) is FFT bin (first_bin + i) mod N; the other
 *     N - N_d bins are guard bins (precoder zero there, Sec. II-A).
 *   - Symbol t uses channel realisation t / S_per_real.
 *   - theta is one flat FP32 vector:
 *       conv_w [N_conv][2 L_U][K_C][K_C], conv_b [N_conv],
 *       fc_w   [2 N_d][N_conv Go Go],     fc_b   [2 N_d]        (Go = ceil(G / K_S));
 *     fc rows 0..N_d-1 give the real parts, rows N_d..2N_d-1 the imaginary parts;
 *     with per-user parameters (fddpd_dpd_desc.per_user) K such vectors, user 0 first.
 *   - metrics (device, double[5]) receive { loss, sum |y - s|^2, sum |s|^2,
 *     guard-bin power of DFT(x^PA), data-bin power of DFT(x^PA) } summed over the call.
 *   - Ownership: the caller owns every data pointer; the plan owns its workspace.
 *   - Every call is asynchronous and ordered on the plan's stream; read results
 *     after synchronising that stream.  Calls on one plan must not overlap.
 *   - Return value: FDDPD_OK or a negative fddpd_status; fddpd_last_error()
 *     describes the last failure.  No call aborts or throws.
 */
#ifndef FDDPD_H
#define FDDPD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { float re, im; } fddpd_c32;
typedef struct fddpd_plan fddpd_plan;

enum fddpd_status {
    FDDPD_OK = 0,
    FDDPD_ERR_ARG = -1,          /* a null pointer, a size out of range, S > max_symbols    */
    FDDPD_ERR_LAYOUT = -2,       /* a pointer not aligned as the layout requires            */
    FDDPD_ERR_SINGULAR = -3,     /* a Gram matrix H_k H_k^H not positive definite          */
    FDDPD_ERR_CUDA = -4,         /* a CUDA runtime error (launch, allocation on create)     */
    FDDPD_ERR_TIMEOUT = -5,      /* a bounded device-side wait gave up                      */
    FDDPD_ERR_UNSUPPORTED = -6,  /* a configuration the library does not implement          */
    FDDPD_ERR_NOMEM = -7         /* workspace allocation failed                             */
};

enum fddpd_precision {
    FDDPD_FP32 = 0,   /* every stage in FP32 on CUDA cores                                 */
    FDDPD_BF16 = 1,   /* FD-CNN dense layer, precoding and combining with BF16 operands,   */
    FDDPD_FP16 = 2    /* or FP16 operands, FP32 accumulation; FFT and PA stay FP32         */
};

enum fddpd_optimizer { FDDPD_GD = 0, FDDPD_ADAM = 1 };

typedef struct {
    int M;            /* BS antennas (paper: B), 1..512                                  */
    int K;            /* users (paper: U), 1..32, K <= M                                 */
    int N;            /* OFDM size, a power of two in 64..4096                           */
    int N_d;          /* data subcarriers, 1..N                                          */
    int first_bin;    /* FFT bin of data subcarrier 0; -1 selects N - N_d/2 (DC-centred) */
    int S_per_real;   /* OFDM symbols per channel realisation, >= 1                      */
    int max_symbols;  /* the largest S any call passes (sizes the workspace); x M < 2^31 */
    int precision;    /* enum fddpd_precision                                            */
    double P_T;       /* transmit power of the ZF normalisation, E||x_hat_k||^2 = P_T    */
} fddpd_dims;

typedef struct {
    int n_orders;     /* 1..8                                                            */
    int orders[8];    /* nonlinear orders p >= 1 of the basis x |x|^{p-1} (e.g. 1, 3, 5); */
                      /* or {0} with n_orders = 1, L = 0: the ideal linear-clipping PA of  */
                      /* Sec. V-B, y = x for |x| <= A, A x / |x| above, A = Re c^b_{0,0}   */
    int L;            /* memory: taps l = 0..L, 0..7                                     */
    int G;            /* cross-term length of Eq. (9), 0..2: with G > 0 each antenna's   */
                      /* coefficients are a [n_orders][L+1] (the memory polynomial), then */
                      /* the lagging b [n_orders][L+1][G] of x_{n-l} |x_{n-l-g}|^{p-1} and */
                      /* the leading c [n_orders][L+1][G] of x_{n-l} |x_{n-l+g}|^{p-1}     */
                      /* (order-1 slots unused), n_orders (L+1)(1+2G) values per antenna */
} fddpd_pa_desc;

typedef struct {
    int G;            /* grid side, G*G >= N_d, <= 128 (the paper's ceil(sqrt(N_d)))     */
    int L_U;          /* users per FD-CNN input, 1..K (users u, u+1, ... mod K)          */
    int K_C;          /* kernel size, odd, 1..15                                         */
    int K_S;          /* stride, 1..G                                                    */
    int N_conv;       /* number of kernels, 1..64                                        */
    int residual;     /* 1: s_tilde = s + FC(.); 0: s_tilde = FC(.) as printed           */
    int per_user;     /* 0: one theta for all users; 1: user u has its own theta_u (the  */
                      /* K sets stacked by user; every precision and L_U)                */
} fddpd_dpd_desc;

/* The FD-NN of Sec. III-C, the frequency-domain NN DPD the paper compares the FD-CNN with:
 * every user's symbols go to the time domain (unitary IDFT of the data bins, guard bins
 * zero); at every sample n a fully connected network maps the real and imaginary parts of
 * s_u[n], s_u[n-1], ..., s_u[n-L4] of all K users (taps circular in n) through `layers`
 * ReLU layers of D neurons to 2K outputs, the predistorted samples (added to s_u[n] when
 * residual = 1, the form in which zero output weights are the identity); the unitary DFT
 * takes each user back to all N bins, so the precoder must cover the guard bins too.
 * theta: W_0 [D][2K(L4+1)] (input j < K(L4+1) is Re s_u[n-l] at j = u(L4+1) + l, the
 * imaginary parts follow), b_0 [D], then (W_k [D][D], b_k [D]) per further layer, W_o
 * [2K][D] (row u the real part of user u, K + u the imaginary part), b_o [2K].       */
typedef struct {
    int L4;           /* memory length of the tapped delay lines, 0..15                  */
    int D;            /* neurons per hidden layer, 1..32                                 */
    int layers;       /* hidden layers K^NN, 1..4                                        */
    int residual;     /* 1: output added to s_u[n]; 0: the network output alone          */
} fddpd_fdnn_desc;

/* Create an FD-NN plan (FP32 only; at most 12288 parameters): the running mode of the
 * comparison workload.  On such a plan
 *   fddpd_precode(plan, R, H_all [R][N][K][M], W_all [R][N][M][K], alpha_all [R][N]) builds
 *       the ZF precoder of Eq. (6) on every one of the N bins (FFT bin order);
 *   fddpd_distort(plan, S, s [S][K][N_d], H [R][N_d][K][M] (the data bins, for combining),
 *       W_all, alpha_all, pa, theta, y, metrics) runs FD-NN, precoding of every bin, IDFT,
 *       PA, DFT and the combining of the data bins (metrics as for the FD-CNN chain);
 *   backward / update / update_host / autotune return FDDPD_ERR_UNSUPPORTED.
 * Errors: ARG, UNSUPPORTED (precision, parameter count), NOMEM, CUDA.              */
int fddpd_fdnn_plan_create(fddpd_plan **out, const fddpd_dims *dims, const fddpd_pa_desc *pa,
                           const fddpd_fdnn_desc *nn, void *stream);

/* Create a plan on `stream` (a cudaStream_t; NULL = legacy default stream).  Validates
 * the sizes, selects the kernels and allocates the workspace for max_symbols symbols.
 * *out receives the plan, or NULL on failure.  Errors: ARG, UNSUPPORTED, NOMEM, CUDA. */
int fddpd_plan_create(fddpd_plan **out, const fddpd_dims *dims, const fddpd_pa_desc *pa,
                      const fddpd_dpd_desc *dpd, void *stream);

/* Release the plan and its workspace (after its stream has finished).  NULL is a no-op. */
int fddpd_plan_destroy(fddpd_plan *plan);

/* Text of the last error on this plan (or of the last failed create when plan is NULL). */
const char *fddpd_last_error(const fddpd_plan *plan);

/* Number of FP32 entries of theta for this plan. */
size_t fddpd_theta_len(const fddpd_plan *plan);

/* Device bytes the plan holds. */
size_t fddpd_workspace_bytes(const fddpd_plan *plan);

/* Re-bind the plan to another stream. */
int fddpd_set_stream(fddpd_plan *plan, void *stream);

/* Plan options (no counterpart in the paper; they select among implementations of the
 * same arithmetic).
 *   FDDPD_OPT_TENSOR_CONTRACTIONS  1 (default): in 16-bit plans with M <= 256 and
 *       K <= 32, the four per-subcarrier contractions (precode, combine and their
 *       adjoints) run as tcgen05 MMAs with 16-bit B operands (the activations rounded
 *       to the plan's 16-bit type), and, with M <= 128 and K <= 16, the ZF matrix
 *       W = H^H (H H^H)^{-1} as tcgen05 MMAs on BF16 high / low splits of H and
 *       (H H^H)^{-1} (relative error near 2^-16); 0: CUDA-core contractions on the same
 *       16-bit copies of H and W with FP32 activations, and W computed on CUDA cores in
 *       FP32 before its rounding.
 *       Ignored by FP32 plans.
 *   FDDPD_OPT_HOST_CHUNKS  1..16 (default 7): the number of realisation chunks in which
 *       fddpd_update_host moves a batch and overlaps its copies with the step; 1 copies
 *       everything first.  The result does not depend on it beyond the order of FP32
 *       sums over symbols.
 *   FDDPD_OPT_KEEP_PA_INPUT  0 (default): the adjoint recomputes the time-domain PA input
 *       x(t) = IDFT(x_hat) in FP32 from x_hat, so the PA derivative is evaluated at the
 *       FP32 signal and nothing time-domain is stored between the passes; 1: BF16 plans
 *       on the tensor-core path keep x(t) from the forward of a training pass as BF16
 *       [max_symbols][M][N] (allocated by this call; NOMEM if that fails) and the
 *       adjoint reads it instead of a third transform (faster; the PA derivative then
 *       sees x rounded to 8 significant bits).  Ignored by FP32 and FP16 plans.
 *   FDDPD_OPT_FACTOR_FP64  1 (default): the Cholesky factor and triangular inverse of
 *       every Gram matrix run in FP64; 0: in FP32 in 16-bit plans (whose W is rounded to
 *       16 bits afterwards; faster).  FP32 plans always factor in FP64.
 *   FDDPD_OPT_ROW_CTAS  0 (default): the IFFT / PA / FFT row kernels' persistent grids
 *       hold as many CTAs per SM as fit; 1..8: at most that many (fewer leave room for
 *       the kernels of other plans recorded on other lanes of one graph).
 *   FDDPD_OPT_CONTRACTION_CTAS  0 or 2 (default): the tensor-core per-subcarrier
 *       contractions' persistent grids hold two CTAs per SM; 1: one (fddpd_get_option
 *       reads 2 or 1).  The arithmetic does not depend on it.
 *   FDDPD_OPT_CONTRACTION_ITEM  0 (default): the tensor-core contractions' work items
 *       span 8 subcarriers (expand; 4 with K > 16) and 4 (reduce); 1: half as many
 *       (more, smaller items for small plans; the benchmark shape's pipelined kernels
 *       then give way to the generic ones).  The arithmetic does not depend on it.
 * Returns FDDPD_ERR_ARG for an unknown option or value.  fddpd_get_option reads one
 * back (*value; ARG for an unknown option).                                          */
enum { FDDPD_OPT_TENSOR_CONTRACTIONS = 1, FDDPD_OPT_HOST_CHUNKS = 2, FDDPD_OPT_KEEP_PA_INPUT = 3,
       FDDPD_OPT_FACTOR_FP64 = 4, FDDPD_OPT_ROW_CTAS = 5, FDDPD_OPT_CONTRACTION_CTAS = 6,
       FDDPD_OPT_CONTRACTION_ITEM = 7 };
int fddpd_set_option(fddpd_plan *plan, int option, int value);
int fddpd_get_option(const fddpd_plan *plan, int option, int *value);

/* Transmit power P_T of Eq. (6) for the plan's next fddpd_precode / fddpd_update_host
 * calls (the ZF normalisation alpha_k = sqrt(P_T / tr((H_k H_k^H)^{-1})); W does not
 * depend on it).  The PA drive level of an SER-versus-power sweep (Sec. V-B, Fig. 3):
 * the PA sees alpha W s, so P_T sets its input back-off.  Host-side only; it changes no
 * array already produced.  Errors: ARG unless 0 < P_T < inf.                     */
int fddpd_set_power(fddpd_plan *plan, double P_T);

/* Drops a 16-bit plan's copies of H and W (see fddpd_precode), so that the next
 * distort / backward / update call re-packs them from the FP32 arrays it is given: for
 * H or W rewritten in place under the same pointers (fddpd_precode_noalloc, a copy).
 * Host-side only; no effect on FP32 plans.  Errors: ARG for a null plan.           */
int fddpd_invalidate_operands(fddpd_plan *plan);

/* Eq. (6): zero-forcing precoder for R channel realisations (Sec. II-A).
 *   H     [R][N_d][K][M]  in : per-subcarrier channel of the data bins
 *   W     [R][N_d][M][K]  out: H_k^H (H_k H_k^H)^{-1}
 *   alpha [R][N_d]        out: sqrt(P_T / tr((H_k H_k^H)^{-1}))
 * The Gram matrix is accumulated in FP32 and factorised (Cholesky) and inverted in
 * FP64 (in FP32 in 16-bit plans set so by FDDPD_OPT_FACTOR_FP64 = 0).  16-bit plans also
 * keep 16-bit copies of W and H for the next distort /
 * backward / update calls with these same H and W pointers (calls with other pointers
 * re-pack from the FP32 arrays; after H or W is rewritten in place by other means than
 * this call, call fddpd_invalidate_operands).  R <= ceil(max_symbols /
 * S_per_real).
 * W = NULL (16-bit plans): no W is formed.  The plan keeps the precoder as its factors --
 * the 16-bit copies of H and H^H and Y = L^{-1} of the Cholesky factor G = L L^H -- and
 * distort / backward / update calls given these same H and alpha with W = NULL apply
 * alpha W s = alpha H^H (Z s), Z = Y^H Y = G^{-1} (Eq. 6 by associativity), until the
 * next fddpd_precode or fddpd_invalidate_operands.  FP32 plans: UNSUPPORTED.
 * Errors: ARG, LAYOUT, UNSUPPORTED, SINGULAR (reported after the kernel completes:
 * this call synchronises the stream once to read the status word).              */
int fddpd_precode(fddpd_plan *plan, int R, const fddpd_c32 *H, fddpd_c32 *W, float *alpha);

/* FP64 check of the zero-forcing identity of Eq. (6) on precoders already produced:
 *   out (device double, 8-byte aligned) = max over the subcarriers b = 0, every,
 *   2 every, ... of the R N_d ones of max_{i,j} |(H_b W_b - I_K)_{ij}|,
 * with H, W laid out as for fddpd_precode and every product and sum in FP64.  About
 * K^2 M complex FP64 multiply-adds per checked subcarrier (the final check of a run,
 * not a per-step stage).  Asynchronous on the plan's stream.  Errors: ARG, LAYOUT.  */
int fddpd_zf_residual(fddpd_plan *plan, int R, const fddpd_c32 *H, const fddpd_c32 *W, int every, double *out);

/* Forward chain over S symbols (running mode of the FD-DPD, Sec. III-A and IV).
 *   s       [S][K][N_d]       in : unit-power QAM symbols of the data bins
 *   H, W, alpha               in : as produced for realisations 0..ceil(S/S_per_real)-1 (W may
 *                                    be NULL after fddpd_precode(H, NULL, alpha) on this plan)
 *   pa_coef [M][n_orders][L+1] in: per-antenna PA coefficients c^b_{p,l} (with cross
 *           terms, G > 0: [M][n_orders (L+1) (1 + 2G)] as fddpd_pa_desc describes)
 *   theta                     in : FD-CNN parameters (layout above)
 *   y       [S][K][N_d]       out: equalised received symbols y_k / alpha_k (may be NULL)
 *   metrics double[5]         out: see above (may be NULL)                         */
int fddpd_distort(fddpd_plan *plan, int S, const fddpd_c32 *s, const fddpd_c32 *H,
                  const fddpd_c32 *W, const float *alpha, const fddpd_c32 *pa_coef,
                  const float *theta, fddpd_c32 *y, double *metrics);

/* Gradient of the loss over the S symbols with respect to theta (Sec. V-A), by the
 * hand-written adjoint of the whole chain, after a forward pass of its own; the
 * time-domain PA inputs of the adjoint are recomputed from x_hat (or, in BF16 plans set
 * so by FDDPD_OPT_KEEP_PA_INPUT, kept by that forward pass in BF16).
 * grad [theta_len] out (overwritten).  metrics as distort.                        */
int fddpd_backward(fddpd_plan *plan, int S, const fddpd_c32 *s, const fddpd_c32 *H,
                   const fddpd_c32 *W, const float *alpha, const fddpd_c32 *pa_coef,
                   const float *theta, float *grad, double *metrics);

/* `iters` training iterations over the S symbols (Sec. V-A): each runs forward, the
 * adjoint and one step theta -= lr * grad (FDDPD_GD), or one Adam step with
 * beta1 = 0.9, beta2 = 0.999, eps = 1e-8 (FDDPD_ADAM; the moments live in the plan
 * and persist across calls until fddpd_reset_optimizer; the plan's first Adam step
 * allocates them -- NOMEM if that fails -- so make one before recording Adam steps into
 * a graph).  theta is updated in place.
 * metrics: those of the last iteration's forward pass (before its step).          */
int fddpd_update(fddpd_plan *plan, int S, const fddpd_c32 *s, const fddpd_c32 *H,
                 const fddpd_c32 *W, const float *alpha, const fddpd_c32 *pa_coef,
                 float *theta, float lr, int iters, int optimizer, double *metrics);

/* One optimizer step from a gradient the caller supplies (the step of fddpd_update, Sec.
 * V-A), for training loops that combine gradients themselves -- data-parallel training
 * runs fddpd_backward on each GPU's own symbols, sums the gradients across the GPUs (an
 * all-reduce) and applies the same step on every GPU with scale = 1 / GPUs:
 *   theta -= lr * scale * grad (FDDPD_GD), or one Adam step on g = scale * grad with the
 *   plan's moments and step counter (FDDPD_ADAM, as fddpd_update; the plan's first Adam
 *   step allocates the moments -- NOMEM if that fails).
 * theta [theta_len] in/out and grad [theta_len] in: device FP32, 4-byte aligned, caller
 * owned; stream-ordered on the plan's stream.  Errors: ARG (null pointer, scale or lr
 * not finite, unknown optimizer), LAYOUT, UNSUPPORTED (FD-NN plans), NOMEM, CUDA.   */
int fddpd_apply_gradient(fddpd_plan *plan, float *theta, const float *grad, float scale, float lr, int optimizer);

/* Zero the Adam moments and step counter. */
int fddpd_reset_optimizer(fddpd_plan *plan);

/* Checkpoint / resume of a training run (Sec. V-A trains theta over many steps): the
 * Adam first and second moments m, v [theta_len] FP32 and the step counter t.  theta
 * itself is the caller's array.  m, v may be host or device memory (any pointer the CUDA
 * runtime can address); both calls synchronise the plan's stream.  Restoring a state
 * and continuing gives the steps an uninterrupted run would take (up to the order of
 * FP32 sums).  Errors: ARG (null pointer, t < 0), LAYOUT, CUDA.                      */
int fddpd_get_optimizer_state(fddpd_plan *plan, float *m, float *v, long long *t);
int fddpd_set_optimizer_state(fddpd_plan *plan, const float *m, const float *v, long long t);

/* One training step from HOST memory (Sec. V-A with a new channel per mini-batch):
 * copies s [S][K][N_d], H [R][N_d][K][M] (R = ceil(S / S_per_real)), pa_coef and theta
 * to plan-owned device buffers (allocated on the first call) and copies theta and
 * metrics[5] back; the result is that of fddpd_precode followed by fddpd_update(iters)
 * up to the order of FP32 sums over symbols.  The first iteration is pipelined: the
 * batch crosses in chunks of whole realisations (FDDPD_OPT_HOST_CHUNKS of them, the
 * first half the size of the others) on a second, plan-owned stream, and each chunk's
 * ZF, forward chain and adjoint run on the plan's stream while the next chunk is
 * copied (the loss stays normalised by the whole batch; the gradient is summed over
 * the chunks).  16-bit plans keep only the 16-bit copy of W here.  Further iterations
 * run on the resident batch.  Host buffers should be page-locked for full copy
 * bandwidth.  Blocks until the step is complete.  A singular Gram matrix anywhere in the batch returns FDDPD_ERR_SINGULAR
 * before any step, with theta untouched.  iters = 0 only computes the precoders.
 * Other errors as fddpd_precode / fddpd_update, NOMEM if the staging buffers cannot
 * be allocated; a failed call still waits for its copies, so the host arrays are free
 * for reuse whenever it returns.                                                  */
int fddpd_update_host(fddpd_plan *plan, int S, const fddpd_c32 *s, const fddpd_c32 *H,
                      const fddpd_c32 *pa_coef, float *theta, float lr, int iters, int optimizer,
                      double *metrics);

/* Symbol errors at the users (Sec. V-B, the setting of Fig. 3).  To the equalised
 * symbols y of fddpd_distort it adds the receiver noise of Eq. (4)-(5) -- w ~ CN(0, N0)
 * per (symbol, user, data subcarrier); the unitary DFT keeps the variance N0 -- scaled
 * by the user's equaliser, z = y + w / alpha_k, decides z to the nearest point of the
 * unit-power square Q-QAM constellation (per component) and compares with s.
 *   y, s   [S][K][N_d]  in (device)   alpha [R][N_d] in (device), R = ceil(S / S_per_real)
 *   Q      4, 16, 64, 256 or 1024      N0 >= 0 (0: no noise)
 *   counts [2] (device, 8-byte aligned): errors and symbols compared are ADDED to it
 *          (subcarriers with alpha <= 0, i.e. singular, are not compared)
 * Noise: Philox-4x32-10 (Salmon et al., SC'11) with key = seed (low word first) and
 * counter = (flat index s K N_d + k N_d + i, low word first, 0, 0); its first two
 * outputs x1, x2 give u = (x + 1/2) 2^-32 and w = sqrt(N0) sqrt(-ln u1) e^{j 2 pi u2}.
 * Imperfect CSI (Sec. II-A) is the caller's choice of the H given to fddpd_precode.
 * Asynchronous on the plan's stream.  Errors: ARG, LAYOUT.                         */
int fddpd_ser(fddpd_plan *plan, int S, const fddpd_c32 *y, const fddpd_c32 *s, const float *alpha, int Q,
              float N0, unsigned long long seed, unsigned long long *counts);

/* fddpd_ser, and per symbol: wrong [S][K][N_d] (device bytes) receives 1 for an error, 0
 * for a correct decision and 2 where the subcarrier is singular (not compared), so that
 * decisions can be compared symbol by symbol.  Errors as fddpd_ser, ARG for a null wrong. */
int fddpd_ser_decisions(fddpd_plan *plan, int S, const fddpd_c32 *y, const fddpd_c32 *s, const float *alpha, int Q,
                        float N0, unsigned long long seed, unsigned long long *counts, unsigned char *wrong);

/* Per-shape launch choice (for batches of uneven plans): times `reps` forward passes
 * (fddpd_distort) of every candidate -- the per-subcarrier contraction implementations
 * the plan's shape admits (tcgen05 in 16-bit plans with M <= 256, K <= 32, with their
 * grid at two or one CTAs per SM, FDDPD_OPT_CONTRACTION_CTAS, and whole or half work
 * items, FDDPD_OPT_CONTRACTION_ITEM; CUDA cores) times the row
 * kernels' grid (FDDPD_OPT_ROW_CTAS 0 or 1) -- with CUDA events on the
 * plan's stream, and keeps the fastest.  The choice is stored per shape (M, K, N, N_d,
 * S_per_real, precision, PA shape, FD-CNN shape, S) in the process: a later plan of a
 * stored shape takes it without timing (fddpd_autotune_forget clears the store).  ms[2]
 * (host, may be NULL) receives the best time of each contraction implementation
 * (tensor-core first; -1 where not admitted).  Synchronises, so it cannot be recorded
 * into a graph (call it before fddpd_graph_begin).  On an error the previous choice is
 * kept.  No counterpart in the paper.  Errors as fddpd_distort, ARG for reps < 1.    */
int fddpd_autotune(fddpd_plan *plan, int S, const fddpd_c32 *s, const fddpd_c32 *H, const fddpd_c32 *W,
                   const float *alpha, const fddpd_c32 *pa_coef, const float *theta, int reps, float *ms);
int fddpd_autotune_forget(void);

/* Batched launch of many plans (uneven M, K, N) as one CUDA graph.  Between
 * fddpd_graph_begin and fddpd_graph_end every fddpd_distort / fddpd_backward /
 * fddpd_update / fddpd_ser call of plans whose stream is `stream` (fddpd_set_stream) is
 * recorded instead of run; fddpd_graph_launch then runs the whole recorded sequence as
 * one graph launch on `stream`, as often as wanted, with the pointers and sizes given at
 * recording time (the data behind them may change between launches).  fddpd_precode,
 * fddpd_update_host, fddpd_autotune and fddpd_sync synchronise and cannot be recorded
 * (they fail with FDDPD_ERR_CUDA).
 * fddpd_graph_begin_lanes records on `stream` and `lanes` side streams forked from it
 * (created by the call, returned in lane_streams[lanes]); plans bound to the lanes
 * (fddpd_set_stream) run concurrently inside the one launch, and fddpd_graph_end joins
 * the lanes back.  The lane streams live until fddpd_graph_destroy; rebind the plans
 * to other streams before calling them outside the graph.  One recording per host
 * thread at a time.
 * Errors: ARG, CUDA (a call that cannot be recorded ends the recording).            */
#define FDDPD_GRAPH_MAX_LANES 32
typedef struct fddpd_graph fddpd_graph;
int fddpd_graph_begin(void *stream);
int fddpd_graph_begin_lanes(void *stream, int lanes, void **lane_streams);
int fddpd_graph_end(void *stream, fddpd_graph **out);
int fddpd_graph_launch(fddpd_graph *graph, void *stream);
int fddpd_graph_destroy(fddpd_graph *graph);

/* Stage tracing.  Stages of the chain, in execution order. */
enum fddpd_stage {
    FDDPD_STAGE_ZF_GRAM = 0, FDDPD_STAGE_ZF_FACTOR, FDDPD_STAGE_ZF_APPLY, FDDPD_STAGE_CONV_FWD, FDDPD_STAGE_FC_FWD, FDDPD_STAGE_PRECODE,
    FDDPD_STAGE_FFTPA_FWD, FDDPD_STAGE_COMBINE, FDDPD_STAGE_ADJ_COMBINE, FDDPD_STAGE_FFTPA_ADJ,
    FDDPD_STAGE_ADJ_PRECODE, FDDPD_STAGE_FC_BWD_W, FDDPD_STAGE_FC_BWD_B, FDDPD_STAGE_FC_BWD_D,
    FDDPD_STAGE_CONV_BWD, FDDPD_STAGE_STEP, FDDPD_STAGE_PACK, FDDPD_STAGE_ZMUL, FDDPD_STAGE_FDNN_ROWS,
    FDDPD_STAGE_FDNN_MLP, FDDPD_N_STAGES
};

/* While enabled, every stage's kernels are bracketed by CUDA events on the plan's
 * stream (at most 4096 brackets between reads; later ones are not timed). */
int fddpd_profile_enable(fddpd_plan *plan, int enable);

/* Synchronise the plan's stream, then write per stage the summed device time in ms
 * (ms[FDDPD_N_STAGES]) and the number of timed brackets (count[FDDPD_N_STAGES]) since
 * the last read, and clear them.  Either pointer may be NULL.                        */
int fddpd_profile_read(fddpd_plan *plan, double *ms, long long *count);

/* Name of a stage ("zf_gram", "fc_fwd", "fftpa_adj", ...), or NULL. */
const char *fddpd_stage_name(int stage);

/* Number of kernels this plan has launched since it was created. */
long long fddpd_launch_count(const fddpd_plan *plan);

/* Synchronise the plan's stream and report device-side failures recorded since the
 * last report: FDDPD_ERR_TIMEOUT when a bounded wait inside a tensor-core kernel gave
 * up (its results are then invalid).  Clears the record.                           */
int fddpd_sync(fddpd_plan *plan);

/* Failure paths on purpose, without a GPU fault (no counterpart in the paper).
 * fddpd_selftest_wait runs, on the plan's stream, one bounded wait on an mbarrier that
 * nothing arrives at (no copy or MMA in flight); after limit_us (1..1000000) it gives up
 * and records the timeout as the tensor-core kernels do, so the next fddpd_sync returns
 * FDDPD_ERR_TIMEOUT (and clears it).  fddpd_debug_fail_allocs(n): the library's next n
 * device allocations fail as if the GPU were out of memory (plan creation, staging,
 * Adam moments, kept PA input): the callers get FDDPD_ERR_NOMEM.                      */
int fddpd_selftest_wait(fddpd_plan *plan, int limit_us);
int fddpd_debug_fail_allocs(int n);

/* The library's tensor-core GEMM on its own (used to validate it):
 *   C[m][n] (+)= sum_k A[m][k] B[n][k],  A [M][lda], B [N][ldb] 16-bit (ab_type 1 = BF16,
 *   0 = FP16), K-major, lda / ldb multiples of 8, 16-byte aligned; C [M][ldc] FP32.
 * splits > 1 slices K and adds the partial sums into C (which the caller zeroes).
 * Runs on `stream` and synchronises it.  Errors: ARG, LAYOUT, CUDA, TIMEOUT.  No
 * counterpart in the paper: a building block of the dense layer of Sec. IV-A.      */
int fddpd_tc_gemm(int M, int N, int K, const void *A, int lda, const void *B, int ldb, float *C, int ldc,
                  int ab_type, int splits, void *stream);

/* Arithmetic peak of this GPU's FP32 or FP64 pipe in TFLOP/s (*tflops, host), measured by
 * an FMA loop over a grid of resident CTAs on every SM and timed with CUDA events on
 * `stream` (synchronised): kind 0 scalar FP32 fma, 1 packed FP32-pair fma (fma.rn.f32x2),
 * 2 FP64 fma.  Each measurement runs for some tens of milliseconds.  No counterpart in
 * the paper: the denominator of the FP32 / FP64 rooflines.  Errors: ARG, CUDA.       */
int fddpd_alu_peak(int kind, double *tflops, void *stream);

/* Zero-forcing precoder (same result as fddpd_precode) for callers that cannot allocate
 * device memory, e.g. a real-time baseband pipeline that reserves all device memory up
 * front and forbids cudaMalloc on its processing path.  The paper has no counterpart.
 *   H [R][N_d][K][M] in, W [R][N_d][M][K] out, alpha [R][N_d] out: device memory owned by
 *   the caller, as for fddpd_precode (data subcarriers only; no plan is needed).
 * No device memory is allocated: the scratch of the ZF kernels is one static device
 * array of FDDPD_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * exit.  It fits R * N_d * K * (K + 1) * 8 + 512 bytes or less (about 15,400 subcarriers
 * at K = 16); larger requests return FDDPD_ERR_UNSUPPORTED before any work.  The first
 * call on each device looks up the array's device address (with that device current),
 * so that call should come before any stream capture.  All calls share the array:
 * calls whose work overlaps on the GPU race.  Runs on `stream` and synchronises it to
 * read the singular-matrix flag.  Errors: ARG, LAYOUT, UNSUPPORTED, SINGULAR, CUDA
 * (text via fddpd_last_error(NULL)).                                                  */
#define FDDPD_NOALLOC_SCRATCH_BYTES (32u << 20)
int fddpd_precode_noalloc(int M, int K, int N_d, int R, double P_T, const fddpd_c32 *H, fddpd_c32 *W,
                          float *alpha, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FDDPD_H */
