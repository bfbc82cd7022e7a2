/*
 * neno6.h — C ABI of the NENO6 Euler right-hand side on one GB300 (sm_103a).
 *
 * NENO6 (Li, Fu & Adams, arXiv 2207.08500) is a six-point finite-difference
 * reconstruction in which a small MLP decides which of four candidate
 * stencils of incremental width enter the convex combination.  This library
 * evaluates, for every cell face of a uniform 1D or 2D grid, the
 * Roe-averaged characteristic projection, the local Lax-Friedrichs
 * (Rusanov) flux split, the MLP stencil classification, the renormalised
 * convex combination and the back-projection (Sec. 4.4, Algorithm 2), then
 * the conservative difference (Eq. (approximateEq)) and the third-order SSP
 * Runge-Kutta update (Sec. 4.4).
 *
 * Conventions for every entry point
 *  - All array arguments are DEVICE pointers owned by the caller, unless a
 *    comment says otherwise; the library never frees them.  They must be
 *    8-byte aligned (16-byte for U / dUdt).
 *  - States are float64 structure-of-arrays [nv][ny][nx], x fastest, with
 *    nv = 3 conserved variables (rho, rho*u, E) in 1D and nv = 4
 *    (rho, rho*u, rho*v, E) in 2D; ny = 1 in 1D.  Ghost cells are handled
 *    inside the library (periodic wrap or zero-gradient copy per axis).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  All work is enqueued on it; no call synchronises the host
 *    except neno6_status, neno6_guard_count, neno6_step_host (whose state
 *    lives in host memory) and neno6_create/destroy.
 *  - Every call returns NENO6_OK (0) or a negative NENO6_ERR_* code and
 *    never throws or aborts; neno6_last_error gives a one-line message.
 *    Conditions found on the device (a non-physical state) are latched in a
 *    status word read by neno6_status; kernels never trap.
 *  - A handle may be used from one host thread at a time.
 */
#ifndef NENO6_H
#define NENO6_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define NENO6_OK 0
#define NENO6_ERR_ARG (-1)         /* null pointer, bad enum, bad number   */
#define NENO6_ERR_SHAPE (-2)       /* grid or batch size out of range      */
#define NENO6_ERR_ALIGN (-3)       /* misaligned device pointer            */
#define NENO6_ERR_WEIGHTS (-4)     /* weights file unreadable or corrupt   */
#define NENO6_ERR_CUDA (-5)        /* a CUDA runtime call failed           */
#define NENO6_ERR_NONPHYSICAL (-6) /* rho <= 0, p <= 0 or c^2 <= 0 seen    */
#define NENO6_ERR_TIMEOUT (-7)     /* a bounded device wait gave up        */
#define NENO6_ERR_UNSUPPORTED (-8) /* option not available for this handle */

/* device status bits (neno6_status) */
#define NENO6_STATUS_NONPHYSICAL_CELL 1 /* rho <= 0 or p <= 0 (or NaN)   */
#define NENO6_STATUS_NONPHYSICAL_ROE 2  /* Roe-averaged c^2 <= 0         */
#define NENO6_STATUS_TIMEOUT 4          /* a tensor-core wait gave up    */
#define NENO6_STATUS_BAD_SAMPLE 8       /* mlp_train: index out of range; datagen: draw outside [0, 1) */

/* neno6_config.precision */
#define NENO6_FP64 0        /* everything in binary64 (bit-exact masks)    */
#define NENO6_MIXED_BF16 1  /* classifier in bf16 on tensor cores (layer
                               1's weights as two bf16 terms), FP32
                               reconstruction, FP64 Roe eigenvectors,
                               back-projection, difference and RK3         */
#define NENO6_MIXED_FP16 2  /* same with fp16 classifier operands          */

/* neno6_config.bc[axis] */
#define NENO6_BC_PERIODIC 0
#define NENO6_BC_TRANSMISSIVE 1 /* zero-gradient ghost cells */

/* neno6_config.linear_weights */
#define NENO6_W_PAPER_OPT 0 /* d_k printed in Sec. 2.2 (fourth order)      */
#define NENO6_W_SIXTH 1     /* (9/20, 3/10, 1/20, 1/5): sixth-order test   */

/* neno6_config.mask_mode */
#define NENO6_MASK_MLP 0        /* the classifier decides (the method)     */
#define NENO6_MASK_ALL_SMOOTH 1 /* keep every stencil: the linear scheme   */
#define NENO6_MASK_ALL_ROUGH 2  /* discard all: first-order upwind fallback */
/* TENO6-opt stencil selection of Sec. 2.1-2.2 (Eqs. (measureTENO),
 * (taukTENO), (normalize), (cut-off); C = 1, q = 6, eps = 1e-40, C_T = 1e-6,
 * smoothness indicators from the Jiang-Shu definition) on the split
 * characteristic fluxes, in place of the classifier: the paper's comparison
 * scheme on the same path.  FP64 handles only (neno6_create refuses it for
 * the mixed precisions with NENO6_ERR_UNSUPPORTED). */
#define NENO6_MASK_TENO6 3

typedef struct neno6_config {
  int ndim;           /* 1 or 2                                            */
  int nx, ny;         /* interior cells, nx >= 1, ny >= 1 (ny = 1 in 1D)   */
  double dx, dy;      /* cell sizes (> 0; dy unused in 1D)                 */
  double gamma;       /* ratio of specific heats (> 1)                     */
  int bc[2];          /* NENO6_BC_* for x and y                            */
  int precision;      /* NENO6_FP64 | NENO6_MIXED_BF16 | NENO6_MIXED_FP16  */
  int linear_weights; /* NENO6_W_*                                         */
  int mask_mode;      /* NENO6_MASK_*                                      */
  double guard_tau;   /* mixed precision: a row whose |logit_k| < guard_tau
                         for some k is re-evaluated in FP32 (0 = off)       */
} neno6_config;

typedef struct neno6_handle neno6_handle;

/*
 * neno6_create — validate the configuration, read the classifier weights
 * and prepare device state on the current CUDA device.
 *   cfg           host pointer, copied.
 *   weights_path  host string: weights file (magic "NENO6W01", int32 layer
 *                 count L, int32 widths[L+1], per layer W[out][in] then
 *                 b[out] as float64 little-endian, uint64 FNV-1a hash of the
 *                 payload).  The parameters (w^l, b^l) of Sec. 3.1,
 *                 Eq. (reconstuction).  Widths must be 6-64-32-16-8-4,
 *                 or 6-32-32-32-4 (the width study's network): a handle
 *                 holding the latter serves neno6_classify (and the calls
 *                 that use no network: neno6_datagen, neno6_status,
 *                 neno6_guard_count, neno6_mask_bytes, neno6_last_error,
 *                 neno6_destroy); the right-hand-side, step, adjoint,
 *                 backward, training and scalar-law calls return UNSUPPORTED
 *                 on it.
 *   out           receives the handle (host pointer).
 * Allocates device memory for the weights and the status word; the RK3
 * stage buffers are allocated on the first neno6_step.
 * Errors: ARG, SHAPE, WEIGHTS, UNSUPPORTED, CUDA.
 */
int neno6_create(const neno6_config* cfg, const char* weights_path, neno6_handle** out);

/* neno6_destroy — free the handle and its device memory (synchronises the
 * device first).  NULL is accepted. */
int neno6_destroy(neno6_handle* h);

/* neno6_mask_bytes — size in bytes of a classifier mask array for this grid:
 * x faces [nv][ny][nx+1] followed (2D) by y faces [nv][ny+1][nx]; face f of
 * a line sits between cells f-1 and f.  One byte per (face, field): bits 0-3
 * the "+" side's eta_0..eta_3, bits 4-7 the "-" side's (eta_k = 1: stencil
 * S_k discarded).  Returns a negative code for a bad handle. */
int64_t neno6_mask_bytes(const neno6_handle* h);

/*
 * neno6_rhs — semi-discrete right-hand side dU/dt = L(U).
 * Sec. 4.4: x sweep then y sweep; per face the Roe characteristic
 * projection, LLF split, classifier (Sec. 3.1), candidates and renormalised
 * combination (Eqs. (convex), (TENOweight_renormalize), Algorithm 2), back-
 * projection; then -(F_{i+1/2}-F_{i-1/2})/dx - (G_{j+1/2}-G_{j-1/2})/dy.
 *   U         [nv][ny][nx] float64 in.
 *   dUdt      [nv][ny][nx] float64 out (must not alias U).
 *   mask_in   nullable; if given, the classifier is not run and these bits
 *             (layout of neno6_mask_bytes) are used instead (frozen mask).
 *   mask_out  nullable; receives the bits used.
 * Errors: ARG, ALIGN, CUDA.  Non-physical states set the status word.
 */
int neno6_rhs(neno6_handle* h, const double* U, double* dUdt, const uint8_t* mask_in,
              uint8_t* mask_out, void* stream);

/*
 * neno6_step — one third-order SSP Runge-Kutta step in place (Sec. 4.4):
 *   U1 = U + dt L(U);  U2 = 3/4 U + 1/4 (U1 + dt L(U1));
 *   U  = 1/3 U + 2/3 (U2 + dt L(U2)),
 * with dt = cfl / (max(|u|+c)/dx + max(|v|+c)/dy) computed on the device
 * from U at the start of the step, clipped so that t + dt <= t_end when
 * t_end > 0.
 *   U      [nv][ny][nx] float64 in/out.
 *   t_dev  nullable device float64 scalar holding t; advanced by dt.  When
 *          NULL an internal time starting at 0 is used.
 *   dt_dev nullable device float64 scalar receiving dt.
 * Uses two library-owned stage buffers (allocated on first use).
 * Errors: ARG, ALIGN, CUDA.
 */
int neno6_step(neno6_handle* h, double* U, double cfl, double t_end, double* t_dev,
               double* dt_dev, void* stream);

/*
 * neno6_step_host — the same SSP-RK3 step (Sec. 4.4) on a state held in
 * HOST memory: copies U_in to a library-owned device state, runs neno6_step
 * on it, copies the result to U_out and synchronises the stream before
 * returning.
 *   U_in   [nv][ny][nx] float64 host array (pinned memory makes the copies
 *          asynchronous DMA; pageable memory works too, more slowly).
 *   U_out  [nv][ny][nx] float64 host array; may be U_in.
 *   t_io   nullable host float64: t in, t + dt out (t_end clips as in
 *          neno6_step).  When NULL the handle's internal time is used.
 * The device state (nv * nx * ny doubles) is allocated on the first call and
 * kept by the handle.  Device-side conditions (non-physical states) are
 * latched in the status word as for neno6_step.
 * Mixed-precision handles overlap the copies with compute: the state goes in
 * and out in row bands (multiples of 16 rows, at most eight: from 1024 rows a
 * 128-row first and last band around six equal ones, from 256 rows eight
 * equal bands, else -- and in 1D -- one band) on a second stream owned by the
 * handle,
 * the first stage's face fluxes and wave-speed maxima start on the bands
 * that have arrived, and the last stage runs band by band, each band copied
 * out as it finishes.  The result is bit for bit that of neno6_step.  U_out
 * is written while the step runs; U_out == U_in is allowed (every band is in
 * before any band is written).
 * Errors: ARG, CUDA.
 */
int neno6_step_host(neno6_handle* h, const double* U_in, double* U_out, double cfl, double t_end,
                    double* t_io, void* stream);

/*
 * neno6_classify — the classifier alone on a batch of stencils: Eq.
 * (normalizainput) then Eqs. (reconstuction), (activationfunction); eta_k =
 * [logit_k > 0] (sigmoid > 1/2, Sec. 3.1).
 *   X        [n][6] float64 raw stencil values f_{i-2..i+3} (normalised here).
 *   n        number of stencils, 0 <= n < 2^31.
 *   eta_out  [n] uint8, bits 0-3 = eta_0..eta_3.
 *   logits   nullable [n][4] float64.
 * Errors: ARG, SHAPE, ALIGN, CUDA.
 */
int neno6_classify(neno6_handle* h, const double* X, int64_t n, uint8_t* eta_out,
                   double* logits, void* stream);

/*
 * neno6_rhs_vjp — adjoint of neno6_rhs with the classifier mask frozen:
 * grad_U = J^T lambda, J = dL(U)/dU with the stencil-selection bits and the
 * LLF alpha argmax (first index on ties) held at their values for U.  Not in
 * the paper: the derivative of the scheme where the mask is locally
 * constant.  Evaluated in FP64 for every precision; each face is recomputed
 * from U (no stored intermediates) and differentiated exactly with
 * forward-mode dual numbers; each cell gathers the contributions of the faces
 * whose stencils contain it (no atomics, deterministic).
 *   U       [nv][ny][nx] float64 state.
 *   lambda  [nv][ny][nx] float64 cotangent of dU/dt.
 *   mask    nullable; the frozen mask (layout of neno6_mask_bytes).  NULL:
 *           recomputed from U by the FP64 classifier (bit-identical to
 *           neno6_rhs of an FP64 handle).
 *   grad_U  [nv][ny][nx] float64 out (must not alias U or lambda).
 * Errors: ARG, ALIGN, CUDA.
 */
int neno6_rhs_vjp(neno6_handle* h, const double* U, const double* lambda, const uint8_t* mask,
                  double* grad_U, void* stream);

/*
 * neno6_mlp_bwd — gradient of the classifier's training loss for retraining:
 * the mean binary cross entropy of Eq. (Crossentropy) (mean over the n
 * samples and the S = 4 outputs, sigmoid outputs of Sec. 3.1) with respect
 * to every parameter of the handle's network; the stencils are normalised as
 * in Eq. (normalizainput) first.  Deterministic (fixed-order reductions).
 * An FP64 handle computes it in FP32 on the CUDA cores; a mixed-precision
 * handle on the tensor cores (its bf16 / fp16 operands: the network's
 * weights, activations and deltas rounded to 16 bits, FP32 accumulation).
 *   X        [n][6] float64 stencil values.
 *   labels   [n] uint8, bit k = eta_k (1: stencil S_k discarded).
 *   n        1 <= n < 2^31.
 *   grad     [3228] float32 out, weights-file order (per layer W[out][in]
 *            then b[out]).
 *   loss     nullable float32 scalar out: the loss itself.
 * Errors: ARG, SHAPE, ALIGN, CUDA.
 */
int neno6_mlp_bwd(neno6_handle* h, const double* X, const uint8_t* labels, int64_t n, float* grad,
                  float* loss, void* stream);

/* scalar laws (neno6_scalar_rhs / neno6_scalar_solve) */
#define NENO6_LAW_ADVECTION 0 /* f(u) = u       (Sec. 4.1) */
#define NENO6_LAW_BURGERS 1   /* f(u) = u^2 / 2 (Sec. 4.2) */

/*
 * neno6_scalar_rhs — du/dt of a scalar conservation law u_t + f(u)_x = 0 on
 * the handle's 1D grid with the same reconstruction as the Euler path (Sec.
 * 4.1-4.2, Algorithm 2): local Lax-Friedrichs split with alpha = max over the
 * six stencil cells of |f'(u)|, the "-" side mirrored about the face, the
 * handle's classifier / mask mode / linear weights, the conservative
 * difference of Eq. (approximateEq).  FP64, bit-identical to the oracle.
 *   law       NENO6_LAW_ADVECTION or NENO6_LAW_BURGERS.
 *   u, dudt   [nx] float64 (device).
 *   mask_out  nullable [nx + 1] uint8: face f (between cells f-1 and f) has
 *             the "+" side's eta bits in bits 0-3, the "-" side's in 4-7.
 * The handle must be 1D and FP64 (else UNSUPPORTED).
 * Errors: ARG, ALIGN, UNSUPPORTED, CUDA.
 */
int neno6_scalar_rhs(neno6_handle* h, int law, const double* u, double* dudt, uint8_t* mask_out, void* stream);

/*
 * neno6_scalar_solve — advance u (in place) to t_end with SSP-RK3 at the fixed
 * step dt = cfl * dx / max_i |f'(u_i)| of the initial data (the scalar cases
 * of Sec. 4.1-4.2), the last step clipped to end exactly at t_end.
 * Synchronises `stream` once to read the initial wave speed.
 *   nsteps_out  nullable: number of steps taken.
 * Errors: ARG, ALIGN, UNSUPPORTED, CUDA.
 */
int neno6_scalar_solve(neno6_handle* h, int law, double* u, double cfl, double t_end, int64_t* nsteps_out,
                       void* stream);

/*
 * neno6_mlp_train — retrain the classifier on the GPU: mini-batch Adam on the
 * mean binary cross entropy of Eq. (Crossentropy) as Sec. 3.3 and Table 2
 * prescribe (Adam of Kingma & Ba with beta1 = 0.9, beta2 = 0.999, epsilon =
 * 1e-8; the caller supplies batch 175, the per-epoch learning rate of the
 * schedule and a fresh permutation each epoch).  Runs ceil(n_perm / batch)
 * steps in order: step s takes the samples perm[s*batch ..], normalises them
 * as in Eq. (normalizainput), and updates every parameter once.  FP32
 * arithmetic, deterministic.  The handle's own network is not used or changed.
 *   X        [n][6] float64 stencil values;  labels [n] uint8 (bit k = eta_k).
 *   perm     [n_perm] int32 sample indices (device); an index outside [0, n)
 *            skips that sample and sets NENO6_STATUS_BAD_SAMPLE.
 *   batch    1 <= batch <= 192 (the last batch may be shorter).
 *   params   [3228] float32 in/out, weights-file order.
 *   adam_m, adam_v  [3228] float32 in/out Adam moments (zero to start).
 *   adam_t0  Adam steps already taken with these moments (bias correction).
 *   lr       learning rate of these steps.
 *   loss_sum nullable float64 scalar out: the sum over the steps of each
 *            batch's mean loss (before its update).
 * Errors: ARG, SHAPE, ALIGN, CUDA.
 */
int neno6_mlp_train(neno6_handle* h, const double* X, const uint8_t* labels, int64_t n, const int32_t* perm,
                    int64_t n_perm, int batch, float* params, float* adam_m, float* adam_v, int64_t adam_t0,
                    double lr, double* loss_sum, void* stream);

/*
 * neno6_pipe_peak — measured fused multiply-add rate of this GPU, a
 * measurement aid for roofline figures (no counterpart in the paper): eight
 * independent FMA chains per thread, 8 CTAs of 256 threads per SM, timed with
 * CUDA events on `stream` (synchronises it).  which = 0: FP64 (DFMA), 1: FP32
 * (FFMA).  *flops_per_s receives 2 x FMAs / s for the whole GPU.  Needs no
 * handle.  Errors: ARG, CUDA.
 */
int neno6_pipe_peak(int which, double* flops_per_s, void* stream);

/*
 * neno6_datagen — training samples of the classifier (Algorithm 1, Table 9,
 * Sec. 3.2) generated on the device from caller-given uniform draws, one
 * sample per row of u:
 *   column 0  grid N in {50, 100, 200} (40 / 40 / 20 %) on [-1, 1];
 *   column 1  function family 1..9 of Table 9, equally likely;
 *   column 2  the interface x_{i+1/2}, i uniform in 2..N-4;
 *   3..7      the family's parameters over Table 9's ranges;
 *   column 8  sign (the sample is negated when u < 1/2).
 * Labels: families 1-3 smooth (0); 4-8 eta_k = 1 iff a kink or jump lies
 * strictly between the outermost cell centres of S_k; family 9 by the
 * TENO6-opt selection (Eqs. (measureTENO)-(cut-off)).  Values are normalised
 * by Eq. (normalizainput), as neno6_mlp_train and neno6_classify expect.
 *   u       [n][NENO6_DATAGEN_DRAWS] float64 device array, values in [0, 1).
 *   X       [n][6] float64 device array (out).
 *   labels  [n] uint8 device array (out): eta_k in bit k.
 *   family  nullable [n] uint8 device array (out): 1..9.
 * A row with a draw outside [0, 1) is written as zeros (family 0) and sets
 * NENO6_STATUS_BAD_SAMPLE.  Errors: ARG, SHAPE, ALIGN, CUDA.
 */
#define NENO6_DATAGEN_DRAWS 9
int neno6_datagen(neno6_handle* h, const double* u, int64_t n, double* X, uint8_t* labels, uint8_t* family,
                  void* stream);

/*
 * neno6_status — synchronise `stream`, return the latched device status bits
 * (NENO6_STATUS_*) in *device_status and clear them.  Returns
 * NENO6_ERR_NONPHYSICAL when any bit was set, NENO6_ERR_CUDA when the stream
 * reported an error, else NENO6_OK.
 */
int neno6_status(neno6_handle* h, int* device_status, void* stream);

/*
 * neno6_guard_count — synchronise `stream` and return in *count the number
 * of classifier rows (face, field, side) that the mixed-precision forms
 * re-evaluated in FP32 on the CUDA cores because some logit fell within
 * guard_tau of 0 (the 16-bit tensor-core result was not trusted to decide
 * the sign, Sec. 3.1's 1/2 threshold), summed over the interior faces of every
 * neno6_rhs / neno6_step evaluation since the handle was created or last
 * reset; reset != 0 clears the counter afterwards.  One RHS evaluates
 * 2 * neno6_mask_bytes(h) rows.  FP64 handles report 0.  Not in the paper: an
 * accuracy diagnostic of the mixed-precision forms.
 * Errors: ARG, CUDA.
 */
int neno6_guard_count(neno6_handle* h, uint64_t* count, int reset, void* stream);

/* neno6_last_error — message of the last failed call on this handle (never
 * NULL; "" when none).  With h == NULL: the last create failure. */
const char* neno6_last_error(const neno6_handle* h);

/*
 * neno6_step_noalloc — the SSP-RK3 step of neno6_step, for callers that must
 * not allocate device memory.  (No counterpart in the paper: an interface
 * choice of this library.)
 *
 * Who needs it: code that runs inside a host application which has reserved
 * the GPU's memory up front for its own pool, or that runs under a fixed
 * device-memory budget, cannot call cudaMalloc mid-run (the call may fail or
 * take memory the owner accounted for), and a cudaMalloc / cudaFree also
 * synchronises the device, stalling the other streams of a latency-critical
 * loop.  neno6_create allocates (weights, status word, and neno6_step's
 * stage buffers on first use); this entry point needs no handle and calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *
 * Scratch: one file-scope static device array holding two stage states of at
 * most NENO6_NOALLOC_MAX_STATE_ELEMS float64 values each (4 MiB each) plus a
 * few words; every GPU that loads the library holds it (8 MiB) until the
 * process exits.  Every call shares it and it keeps the previous call's
 * contents; the call clears what must start at zero.  Calls whose work
 * overlaps on the GPU (different streams, or different host threads) race on
 * it and must be serialised by the caller.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress, with that device
 * current); make that first call before any stream capture.  The address is
 * kept per device together with the id of the context it was taken in; after
 * a device reset (or a release of the primary context) the next call sees a
 * new context id and looks the address up again, so that call too should
 * come before any stream capture.
 *
 *   cfg          host pointer: grid and scheme (precision must be NENO6_FP64);
 *                nv * nx * ny must not exceed NENO6_NOALLOC_MAX_STATE_ELEMS.
 *   net_params   host pointer: the 3228 classifier parameters in the weights
 *                file's order (per layer W[out][in] then b[out]); n_params
 *                must be 3228.
 *   U            [nv][ny][nx] float64 device state, advanced in place.
 *   cfl, t_end   as in neno6_step.
 *   t_dev        nullable device float64 time, advanced by dt; NULL: the step
 *                starts from t = 0.
 *   dt_dev       nullable device float64 receiving dt.
 *   status_dev   nullable device int; NENO6_STATUS_* bits are OR-ed into it
 *                (NULL: they are dropped).
 * Returns NENO6_OK or ARG, SHAPE (state larger than the static scratch),
 * ALIGN, WEIGHTS (n_params), UNSUPPORTED, CUDA; no message is recorded.
 */
#define NENO6_NOALLOC_MAX_STATE_ELEMS (1u << 19)
int neno6_step_noalloc(const neno6_config* cfg, const double* net_params, int64_t n_params,
                       double* U, double cfl, double t_end, double* t_dev, double* dt_dev,
                       int* status_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NENO6_H */
