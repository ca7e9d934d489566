/*
 * ws.h - C-ABI of the B300 Whittaker-Henderson smoother library (libws_b300.so).
 *
 * For every pixel time series (x, w, lambda) on a regular daily grid the library
 * solves the banded symmetric positive-definite system
 *
 *     (W + D^T Lambda D) z = W x                                    (Eq. 3)
 *
 * where W = diag(w) holds observation weights (0 for cloudy or missing days),
 * D in R^{(T-d) x T} is the order-d difference operator (the paper's order k+1)
 * with rows c_0..c_d = (-1)^(d-i) C(d, i) at columns k..k+d (Section 2), and
 * Lambda = diag(lambda_0 .. lambda_{T-d-1}) weights the rows of D (Section 2.2).
 * A scalar lambda gives the homoscedastic smoother of Eq. 2. Several spectral
 * bands share w and lambda and are solved as right-hand sides against one factor
 * (Section 2, "batched multivariate"). The reverse-mode derivatives of Eqs. 4-5
 * (Section 2.3) make the solve a differentiable layer. The *_dates entry points keep each
 * series on its own unevenly spaced sample times instead of the daily grid (the difference
 * operator for uneven spacing that Section 2 adopts); ws_posterior gives the credibility
 * intervals of Fig. 4, ws_weight_grad the gradient in soft weights, ws_gcv_smooth a lambda
 * per series, the ws_plan_* calls ragged batches and the ws_tcn_* calls the lambda network.
 *
 * Conventions shared by every entry point
 *   - Pointers named x, w, lam, t, z, factor, gz, gx, glam, gw, diag, sigma2, sd, status,
 *     workspace are DEVICE pointers owned by the caller. The library never allocates memory on
 *     a call path; callers size `workspace` with ws_workspace_size().
 *   - `stream` is a cudaStream_t passed as void*. Every call only enqueues work
 *     on that stream and never synchronises it (except ws_sync_status).
 *   - Return value: WS_OK (0) or a negative WS_E* code; ws_last_error() gives the
 *     text of the last error on the calling thread.
 *   - Numerical failures are reported per series in the optional `status` array
 *     (uint8, one per series) and do not make the call fail:
 *       WS_SERIES_OK        0
 *       WS_SERIES_NOT_PD    1  Omega singular: fewer than min(d, T) positive
 *                              weights; outputs of the series are zero-filled
 *       WS_SERIES_NONFINITE 2  a non-finite value (e.g. NaN x on a weighted day)
 *                              reached the output
 *       WS_SERIES_BADARG    3  some lambda_k (k < T-d) not > 0 and finite, or
 *                              some w_t not >= 0 and finite; outputs zero-filled
 *   - Where w_t == 0 the observation x_t is never read into the arithmetic (a NaN
 *     in a gap is harmless).
 *
 * Tile layout (WS_LAYOUT_TILE): time-major, pixel-interleaved, pixel fastest:
 *     x[(t*B + b)*P + p], z likewise, w[t*P + p],
 *     lam[t*P + p] (WS_LAM_PER_DAY: entry k weights difference row k, which spans
 *     days k..k+d; entries T-d..T-1 are ignored) or lam[p] (WS_LAM_SCALAR),
 *     factor[(t*(d+1) + j)*P + p] (see ws_factor).
 * Element type: float (WS_F32) or double (WS_F64) for every floating array of a call.
 */
#ifndef WS_B300_H
#define WS_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define WS_OK 0
#define WS_EINVAL (-1)        /* invalid argument (null pointer, size, alignment, enum) */
#define WS_ENOMEM_WS (-2)     /* workspace smaller than ws_workspace_size() */
#define WS_ECUDA (-3)         /* a CUDA runtime call failed (launch, attribute, ...) */
#define WS_ETIMEOUT (-4)      /* a device-side wait gave up (reported by ws_sync_status) */
#define WS_EUNSUPPORTED (-5)  /* valid request the library does not implement (e.g. an instantiation left out) */

/* per-series status codes */
#define WS_SERIES_OK 0
#define WS_SERIES_NOT_PD 1
#define WS_SERIES_NONFINITE 2
#define WS_SERIES_BADARG 3

/* enums */
#define WS_LAYOUT_TILE 0
#define WS_F32 0
#define WS_F64 1
#define WS_LAM_PER_DAY 0
#define WS_LAM_SCALAR 1

/* flags */
#define WS_GRAD_LOGLAM 0x1u   /* ws_solve_adjoint: glam = lambda * dL/dlambda (d/dlog lambda) */
#define WS_REFINE 0x2u        /* ws_smooth_batch: one step of iterative refinement */
#define WS_GCV 0x8u           /* ws_workspace_size: size for ws_gcv_smooth */
#define WS_REFINE_ADJOINT 0x4u /* ws_solve_adjoint: one step of iterative refinement of g */
#define WS_POSTERIOR 0x10u     /* ws_workspace_size: size for ws_posterior */
#define WS_DATES 0x40u         /* ws_workspace_size: size for ws_smooth_dates */
#define WS_PARTITIONED 0x80u   /* ws_workspace_size: size for ws_smooth_partitioned */
#define WS_ADJ_RAW_G 0x20u     /* ws_solve_adjoint: gx receives g = Omega^{-1} gz itself (not W g),
                                  the input of ws_weight_grad */

typedef struct ws_problem {
  int64_t n_series; /* P >= 0: number of series (pixels) */
  int32_t T;        /* days per series, >= 0 */
  int32_t d;        /* difference order, 1..4 */
  int32_t n_bands;  /* B >= 1: right-hand sides sharing w and lambda */
  int32_t layout;   /* WS_LAYOUT_TILE */
  int32_t dtype;    /* WS_F32 | WS_F64 */
  int32_t lam_mode; /* WS_LAM_PER_DAY | WS_LAM_SCALAR */
} ws_problem;

/* Bytes of device scratch the calls below need for `pb` (checkpoints of the
 * forward sweep plus a 256-byte header holding the device error word; with
 * flags & WS_REFINE also the residual, T*B*P elements; with WS_REFINE_ADJOINT two
 * such arrays). The first
 * 256 bytes must be zero before the first call that uses the workspace (e.g.
 * cudaMemset once after allocation); ws_sync_status() clears the word again.
 * Returns 0 for an invalid problem. */
size_t ws_workspace_size(const ws_problem* pb, uint32_t flags);

/* Smoothing, Eq. 3 (Eq. 2 with WS_LAM_SCALAR): z = (W + D^T Lambda D)^{-1} W x for
 * every series and band. x, w, lam: inputs in the tile layout; z: output (may not
 * alias x). factor_out: optional (NULL or the ws_factor layout) receives the
 * factor of Omega. status: optional per-series codes. flags: 0 or WS_REFINE: after
 * the solve, the residual r = W x - Omega z is formed with double-word (FP64-level)
 * accumulation, Omega d = r is solved with the same factorisation and z += d; this
 * needs the larger workspace ws_workspace_size(pb, WS_REFINE). The factor is the
 * Cholesky factor of Omega (Section 3.1) computed by plane rotations on the
 * stacked square-root system [sqrt(W); sqrt(Lambda) D]; two sweeps over time
 * (forward elimination, backward substitution). */
int ws_smooth_batch(const ws_problem* pb, const void* x, const void* w, const void* lam, void* z,
                    void* factor_out, uint8_t* status, uint32_t flags, void* workspace,
                    size_t ws_bytes, void* stream);

/* Smoothing with lambda chosen per series by generalized cross-validation over a grid.
 * The paper names the selection problem but defines no criterion; this is the
 * Craven-Wahba score: for each grid value lam_g, z = Omega^{-1} W x (Eq. 2, scalar lambda),
 * RSS = sum_t w_t (x_t - z_t)^2, tr H = sum_t w_t (Omega^{-1})_tt with H = Omega^{-1} W
 * (diagonal of the inverse by the banded selected-inverse recursion on the same factor),
 * n = sum_t w_t, V_g = n RSS / (n - tr H)^2. The smallest V wins, ties to the smaller
 * lambda; z is then the smoothing at that lambda (ws_smooth_batch, WS_REFINE allowed).
 * pb: FP32, one band, tile layout; pb->lam_mode is ignored (the final smooth uses one
 * lambda per series). lam_grid: HOST array of n_grid (1..16) finite positive values.
 * x, w, z: device, [T][P]. lam_best: device, P floats (output). scores: optional device
 * [n_grid][P] (V per grid value; NaN where the series is not positive definite or has
 * invalid weights). status: optional per-series codes of the final smooth.
 * Workspace: ws_workspace_size(pb, WS_GCV | flags). Errors as ws_smooth_batch;
 * WS_EUNSUPPORTED for FP64 or several bands. */
int ws_gcv_smooth(const ws_problem* pb, const void* x, const void* w, const float* lam_grid, int n_grid,
                  void* z, float* lam_best, float* scores, uint8_t* status, uint32_t flags,
                  void* workspace, size_t ws_bytes, void* stream);

/* Smoothing on unevenly spaced sample times (Section 2): each series stays on its own
 * acquisition dates t_0 < ... < t_{T-1} (e.g. day numbers) instead of a padded daily grid,
 * and D is the discrete derivative for uneven spacing that the paper adopts: row k is d!
 * times the weights of the divided difference f[t_k, ..., t_{k+d}], c_{k,j} = d! /
 * prod_{m != j} (t_{k+j} - t_{k+m}); on t = 0, 1, 2, ... it is the daily grid's binomial
 * difference, so z matches ws_smooth_batch there. z = (W + D^T Lambda D)^{-1} W x per series
 * and band. t: device [T][P] in pb->dtype (per-series dates); x, z: [T][B][P]; w: [T][P];
 * lam: [T][P] (entry k weights row k; the last d unused) or [P] (WS_LAM_SCALAR). Dates that
 * are not strictly increasing or not finite give the series status WS_SERIES_BADARG; the
 * other codes as ws_smooth_batch (zeros where not WS_SERIES_OK). flags: 0 or WS_REFINE: one
 * step of iterative refinement as for ws_smooth_batch (residual W x - Omega z with D z and
 * D^T (Lambda D z) as nested divided differences and the cancelling combination rounded
 * once, then Omega d = r with the same rotations, z += d). Workspace:
 * ws_workspace_size(pb, WS_DATES | flags), 256-byte aligned. One launch per band group
 * on `stream` (plus the residual and the correction with WS_REFINE). */
int ws_smooth_dates(const ws_problem* pb, const void* t, const void* x, const void* w, const void* lam, void* z,
                    uint8_t* status, uint32_t flags, void* workspace, size_t ws_bytes, void* stream);

/* Reverse-mode derivatives of ws_smooth_dates (Section 2.3 on sample times): g = Omega^{-1}
 * gz with the uneven-spacing Omega, gx = W g (Eq. 5, transposed), glam_k = -sum_b (D g_b)_k
 * (D z_b)_k (Eq. 4) for k < T-d and 0 after (WS_LAM_SCALAR: the sum over k), times lambda_k
 * with WS_GRAD_LOGLAM; (D f)_k as nested divided differences. t, w, lam, z (the forward
 * output), gz: inputs as for ws_smooth_dates; gx: [T][B][P] output (required); glam:
 * optional. Series that are not positive definite or have invalid inputs get zeros and their
 * status code. Workspace: ws_workspace_size(pb, WS_DATES). One launch per band group (up to
 * 4 bands in FP32, 2 in FP64). */
int ws_smooth_dates_adjoint(const ws_problem* pb, const void* t, const void* w, const void* lam, const void* z,
                            const void* gz, void* gx, void* glam, uint32_t flags, uint8_t* status, void* workspace,
                            size_t ws_bytes, void* stream);

/* Gradient with respect to the observation weights (soft weights): the weights of the
 * objective (Eq. 1) taken as parameters. From Omega z = W x, dz/dw_t = Omega^{-1} e_t
 * (x_t - z_t), so dL/dw_t = sum_b g_tb (x_tb - z_tb) with g = Omega^{-1} dL/dz, the solution
 * of the adjoint system (Section 2.3); a day with w_t = 0 contributes x_t = 0 (its value is
 * ignored, selected away rather than multiplied). g: device [T][B][P], the output of
 * ws_solve_adjoint with WS_ADJ_RAW_G. gw: device [T][P] output. gx: NULL, or g itself (then
 * overwritten in place), or a separate [T][B][P] array: receives dL/dx = W g. x, w, z: the
 * smoothing's inputs and output (tile layout). Series that failed in the adjoint have
 * g = 0 and so gw = 0. Outputs may not overlap the inputs (WS_EINVAL); one kernel launch
 * on `stream`, no workspace. */
int ws_weight_grad(const ws_problem* pb, const void* x, const void* w, const void* z, void* g, void* gx,
                   void* gw, void* stream);

/* Posterior spread of the smooth: the pointwise credibility intervals drawn in Fig. 4.
 * The paper plots them and borrows their formula from the Bayesian reading of the smoother
 * it cites; this call computes that reading. z = Omega^{-1} W x (Eq. 3) is the posterior
 * mean of a signal whose observations on days with w_t > 0 have precision w_t / sigma^2 and
 * whose improper prior has precision D^T Lambda D / sigma^2; the posterior covariance is
 * sigma^2 Omega^{-1}, with sigma^2 estimated per band by RSS_b / (n - tr H), RSS_b =
 * sum_t w_t (x_tb - z_tb)^2 over days with w_t > 0, n = sum_t w_t, tr H = sum_t w_t
 * (Omega^{-1})_tt. Outputs (device, caller-owned, tile layout):
 *   diag   [T][P]     (Omega^{-1})_tt, by the banded selected-inverse recursion on the
 *                     rotation factor of the solve (double-word window in FP32);
 *   sigma2 [B][P]     the residual variance per band (NaN where n - tr H <= 1e-4 n in
 *                     FP32, 1e-10 n in FP64: the smoother interpolates the observations
 *                     and the residual degrees of freedom are within rounding of zero);
 *   sd     [T][B][P]  optional (NULL to skip): sqrt(sigma2_b diag_t); the interval at level
 *                     q is z +- q sd.
 * Inputs: x, w, lam as for ws_smooth_batch (FP32 or FP64, per-day or scalar lambda), z the
 * smooth of x (normally ws_smooth_batch's output; any z is accepted and enters RSS only).
 * Series whose Omega is not positive definite (status WS_SERIES_NOT_PD) or with invalid
 * w/lambda (WS_SERIES_BADARG) get zeros in all three outputs; WS_SERIES_NONFINITE marks a
 * non-finite diagonal or an undetermined sigma2 (NaN). Outputs may not overlap the inputs or each other
 * (WS_EINVAL). Workspace: ws_workspace_size(pb, WS_POSTERIOR), 256-byte aligned (its
 * error header is not used). Two kernel launches on `stream`; no allocation, no
 * synchronisation. T = 0: sigma2 is zeroed and every status is WS_SERIES_NOT_PD. */
int ws_posterior(const ws_problem* pb, const void* x, const void* w, const void* lam, const void* z,
                 void* diag, void* sigma2, void* sd, uint8_t* status, void* workspace, size_t ws_bytes,
                 void* stream);

/* ws_posterior on unevenly spaced sample times: Omega = W + D^T Lambda D with D the
 * uneven-spacing operator of ws_smooth_dates (rows from t [T][P], each series' strictly
 * increasing dates); z is the smooth on those dates. Same outputs, codes (dates that do not
 * increase: WS_SERIES_BADARG) and workspace (ws_workspace_size(pb, WS_POSTERIOR)). */
int ws_posterior_dates(const ws_problem* pb, const void* t, const void* x, const void* w, const void* lam,
                       const void* z, void* diag, void* sigma2, void* sd, uint8_t* status, void* workspace,
                       size_t ws_bytes, void* stream);

/* ws_gcv_smooth on unevenly spaced sample times: the grid search and the final smooth use
 * the uneven-spacing operator of ws_smooth_dates (rows from t [T][P], each series' strictly
 * increasing dates). Same arguments otherwise; workspace ws_workspace_size(pb, WS_GCV |
 * WS_DATES | flags) (pb->lam_mode is ignored, as for ws_gcv_smooth). */
int ws_gcv_smooth_dates(const ws_problem* pb, const void* t, const void* x, const void* w, const float* lam_grid,
                        int n_grid, void* z, float* lam_best, float* scores, uint8_t* status, uint32_t flags,
                        void* workspace, size_t ws_bytes, void* stream);

/* ---- Learned lambda: temporal convolution network g_theta (Section 4.2 names a network
 * with a sigmoid output range; this one is a 4-layer 1-D convolution net) ----
 * Per series, per day: (x_t [w_t > 0], w_t) -> conv(2->64, k=9) -> ReLU -> conv(64->64) ->
 * ReLU -> conv(64->64) -> ReLU -> conv(64->1) = o_t; log lambda_t = Lmin + sigmoid(o_t)
 * (Lmax - Lmin). "Same" zero padding per series. BF16 weights and activations, FP32
 * accumulation; the two 64->64 layers and their data gradients run on the tensor cores
 * (tcgen05), the 2->64 and 64->1 layers and the weight gradients on CUDA cores.
 * Parameters: an FP32 master vector of WS_TCN_PARAMS values, PyTorch conv1d layouts
 * concatenated: W1 [64][2][9], b1 [64], W2 [64][64][9], b2, W3 [64][64][9], b3, W4 [1][64][9],
 * b4 [1]. ws_tcn_pack writes the BF16 copy (WS_TCN_PACKED_BYTES) the kernels read; biases are
 * read from the master. All pointers are device pointers. */
#define WS_TCN_PARAMS 75649
#define WS_TCN_PACKED_BYTES 304512
typedef struct ws_tcn_batch {
  int32_t T;            /* days per series */
  int32_t n_series;     /* P: series of the [T][P] inputs */
  float log_lam_min;    /* Lmin, natural log */
  float log_lam_max;    /* Lmax > Lmin */
} ws_tcn_batch;

/* Scratch bytes for ws_tcn_forward (training = 0: inference; 1: keeps the activations the
 * backward pass needs) and ws_tcn_backward (training = 1). 0 on invalid input. */
size_t ws_tcn_scratch_size(const ws_tcn_batch* b, int training);
int ws_tcn_pack(const float* master, void* packed, void* stream);
/* lam, loglam (optional): [T][P] FP32 outputs. x, w: [T][P] FP32 inputs. */
int ws_tcn_forward(const ws_tcn_batch* b, const void* packed, const float* master, const float* x, const float* w,
                   float* lam, float* loglam, void* scratch, size_t scratch_bytes, int training, void* stream);
/* grad (FP32, WS_TCN_PARAMS) += dL/dtheta given g_loglam = dL/dlog lambda ([T][P]), using the
 * activations the last training forward left in scratch. */
int ws_tcn_backward(const ws_tcn_batch* b, const void* packed, const float* g_loglam, float* grad, void* scratch,
                    size_t scratch_bytes, void* stream);
/* One 64 -> 64 layer over `rows` stream rows (series of T days each followed by 4 gap rows):
 * out[r][co] = relu(bias[co] + sum_{k,ci} W[k][ci][co] in[r + k - 4][ci]) with zeros on gap
 * rows (mode 0), or the data gradient form out[r][co] = [mask[r][co] > 0] sum_{k,ci} ... (mode
 * 1). in, mask, out: BF16 [rows][64]; wplanes: BF16 [9 taps][8 ci chunks][64 co][8 ci] (73,728
 * bytes, the layout ws_tcn_pack writes); err_word: a device word set if a wait gives up. */
int ws_tcn_conv64(const void* in, const void* wplanes, const float* bias, const void* mask, void* out, int64_t rows,
                  int32_t T, int32_t mode, void* err_word, void* stream);
/* Adam with bias correction (step >= 1); grad is cleared after the update. */
int ws_adam_step(float* params, float* m, float* v, float* grad, int64_t n, int32_t step, float lr, float beta1,
                 float beta2, float eps, void* stream);
/* gz = scale (z - target); *loss_sum += scale/2 sum (z - target)^2 (loss_sum may be NULL). */
int ws_mse_grad(const float* z, const float* target, float* gz, float* loss_sum, int64_t n, float scale,
                void* stream);

/* ws_smooth_batch without a caller-provided workspace (the paper has no counterpart:
 * this is an interface for callers that cannot allocate device memory where they
 * smooth, e.g. under a framework's caching allocator that already holds the memory, or
 * where the device-wide synchronisation of cudaFree must be avoided). Same arguments,
 * results and per-series status as ws_smooth_batch, whose kernels it runs; the scratch
 * is a file-scope device array of WS_NOALLOC_MAX_BYTES per device.
 *   - Problems with ws_workspace_size(pb, flags) > WS_NOALLOC_MAX_BYTES (64 MiB)
 *     return WS_ENOMEM_WS before anything is launched. That size is the checkpoints of
 *     the persistent grid (up to grid x ceil(T/C) x (d(d+1) + B d) x 128 elements, C the
 *     planned chunk) plus, with WS_REFINE, a T x B x P residual: 4096 FP64 series of
 *     T = 365, d = 2, one band, with WS_REFINE fit (about 35 MiB).
 *   - No cudaMalloc, cudaFree or allocating library routine is called.
 *   - The first call on each device does the set-up with that device current
 *     (cudaGetSymbolAddress, then a synchronous cudaMemset clearing the error word):
 *     make that first call before any stream capture.
 *   - Calls on the same device share the array: calls that overlap in time (host
 *     threads, or streams without ordering between them) race on it.
 *   - A device-side wait that gives up sets the array's error word, which this entry
 *     point does not report; use ws_smooth_batch and ws_sync_status for that report. */
#define WS_NOALLOC_MAX_BYTES (64u << 20)
int ws_smooth_batch_noalloc(const ws_problem* pb, const void* x, const void* w, const void* lam, void* z,
                            void* factor_out, uint8_t* status, uint32_t flags, void* stream);

/* One step of iterative refinement of a smoothing result z, in place:
 *     r = W x - Omega z        (double-word accumulation: FP64-level accuracy from
 *                               error-free transformations of the working precision)
 *     z <- z + Omega^{-1} r    (same rotation factorisation, recomputed)
 * x, w, lam: the inputs z was computed from. Needs ws_workspace_size(pb, WS_REFINE).
 * The paper (Section 3) solves in one pass; this step restores the accuracy FP32 loses
 * on ill-conditioned series (large lambda, few valid days, d >= 3). */
int ws_refine(const ws_problem* pb, const void* x, const void* w, const void* lam, void* z,
              void* workspace, size_t ws_bytes, void* stream);

/* Factor only (Section 3.1): writes, per day t, factor[(t*(d+1) + 0)*P + p] = 1/D_t and
 * factor[(t*(d+1) + j)*P + p] = L[t+j][t] (j = 1..d) of Omega = L diag(D) L^T with L
 * unit lower triangular banded (entries that would fall past T are 0). One forward
 * sweep (the same plane rotations as ws_smooth_batch); workspace unused (may be NULL).
 * Series that fail (status != 0) get a zero factor. */
int ws_factor(const ws_problem* pb, const void* w, const void* lam, void* factor, uint8_t* status,
              void* workspace, size_t ws_bytes, void* stream);

/* Solve with a stored factor: z = Omega^{-1} W x, Omega given by `factor` (ws_factor
 * layout) and w; z is used as scratch between the two sweeps. flags: 0; workspace
 * unused (may be NULL). */
int ws_solve(const ws_problem* pb, const void* factor, const void* w, const void* x, void* z,
             uint32_t flags, void* workspace, size_t ws_bytes, void* stream);

/* Reverse-mode derivatives through z = Omega^{-1} W x (Section 2.3, Eqs. 4-5).
 * Given z (the forward output) and gz = dL/dz (tile layout, B bands):
 *     g_b = Omega^{-1} gz_b                 (Omega symmetric)
 *     gx_b = W g_b                          (Eq. 5; the vector-Jacobian product)
 *     glam_k = -sum_b (D g_b)_k (D z_b)_k   (Eq. 4), k < T-d; glam_k = 0 for k >= T-d
 * With WS_LAM_SCALAR, glam[p] is the sum over k. With WS_GRAD_LOGLAM, glam is
 * multiplied by lambda (the derivative with respect to log lambda). With
 * WS_REFINE_ADJOINT, g gets one step of iterative refinement (residual gz - Omega g with
 * double-word accumulation) before the epilogue; needs ws_workspace_size(pb,
 * WS_REFINE_ADJOINT). (D g)_k and (D z)_k are formed as nested first differences.
 * factor_or_null: a stored factor (ws_factor layout), or NULL to recompute it from
 * (w, lam) inside the sweeps (less memory). With a stored factor the workspace must be
 * ws_workspace_size(pb, WS_REFINE) bytes (g is held there) and `status` is not written.
 * gx and glam are each optional (NULL). With WS_ADJ_RAW_G, gx receives g itself instead of
 * W g (the input of ws_weight_grad). */
int ws_solve_adjoint(const ws_problem* pb, const void* factor_or_null, const void* w,
                     const void* lam, const void* z, const void* gz, void* gx, void* glam,
                     uint32_t flags, uint8_t* status, void* workspace, size_t ws_bytes,
                     void* stream);

/* z = Omega^{-1} W x (Eq. 3) by a partitioned parallel-in-time solve, for few long series
 * (Section 2.3's cost argument: with one series per thread, a handful of series keep a
 * handful of threads busy). Each series' days are cut into domains of 16, 32 or 64 days
 * (the largest that still gives the GPU about 9,500 threads; one domain if T <= 64); the
 * last d days of each domain but the last are a separator. One thread per (series,
 * domain) factors its interior band (LDL^T of Omega assembled from w and lambda) and forms
 * its Schur-complement pieces; one thread per series factors the separators'
 * block-tridiagonal Schur complement and one per (series, band) solves it; one per
 * (series, domain) then finishes its interior. Arithmetic: double-float (hi + lo FP32
 * pairs, about 48 bits) for FP32 data, FP64 for FP64 data, so no refinement step is
 * needed. Same layout, arguments, status codes and zero-filled outputs as ws_smooth_batch
 * (flags: none). workspace: ws_workspace_size(pb, WS_PARTITIONED) bytes, 256-byte aligned
 * (else WS_EINVAL / WS_ENOMEM_WS before any launch); contents need no initialisation.
 * Per series it moves a few hundred bytes of scratch per day, so it suits up to a few
 * thousand series; beyond that ws_smooth_batch is faster. Accuracy: elimination on Omega
 * (not the rotation factor of ws_smooth_batch) has an error of order eps * cond(Omega)
 * (eps about 3.6e-15 in double-float), against eps * sqrt(cond(Omega)) for the rotations:
 * within 1e-4 up to cond(Omega) of about 1e10 (the heteroscedastic and homoscedastic
 * workloads); for worse-conditioned series (d = 3 with unsmoothed lambda up to 1e5 and
 * sparse weights reaches 1e13) use ws_smooth_batch with WS_REFINE or the ragged plan's
 * refinement, whose double-float re-solve uses the rotations. */
int ws_smooth_partitioned(const ws_problem* pb, const void* x, const void* w, const void* lam, void* z,
                          uint8_t* status, void* workspace, size_t ws_bytes, void* stream);

/* The adjoint of Section 4.3's training loss with the loss fused into its sweeps: the
 * masked mean squared error of the smooth z against held-out targets,
 *   L_p = scale/2 * sum_{t,b} m_tp (z_tbp - target_tbp)^2,
 * whose gradient gz = scale * m * (z - target) is formed per day inside the kernel (never
 * stored), then Eqs. 4-5 as ws_solve_adjoint (recomputed factor): gx = W Omega^{-1} gz,
 * glam_k = -sum_b (D g_b)_k (D z_b)_k (times lambda_k with WS_GRAD_LOGLAM). With
 * scale = 2 / (number of held-out entries) the sum of L over the series is their mean.
 * target: [T][B][P] like x (read only where m > 0, so NaN elsewhere is harmless); mask:
 * [T][P] non-negative day weights shared by the bands (1 on held-out days), or NULL for all
 * ones; z: the forward output. loss: optional [P] output (L_p), gx / glam optional as in
 * ws_solve_adjoint. flags: WS_GRAD_LOGLAM, WS_ADJ_RAW_G. workspace: ws_workspace_size(pb, 0).
 * Outputs must not overlap the inputs or each other (WS_EINVAL). status as ws_solve_adjoint. */
int ws_solve_adjoint_mse(const ws_problem* pb, const void* w, const void* lam, const void* z,
                         const void* target, const void* mask, double scale, void* gx, void* glam,
                         void* loss, uint32_t flags, uint8_t* status, void* workspace, size_t ws_bytes,
                         void* stream);

/* Tuning knobs of the tile kernels, process-wide (0 = automatic): the number of CTAs
 * (of the pixels per CTA in force) to fit on one SM, 1..32, which sets the shared memory per CTA, and
 * an upper bound on the days per staged chunk, 1..255. The chunk is the largest that
 * fits; registers may allow fewer CTAs than requested. ws_workspace_size() reflects the
 * current setting. Returns WS_EINVAL for out-of-range values. */
int ws_tune_set(int32_t ctas_per_sm, int32_t chunk_days);

/* Tuning of the tile kernels (no counterpart in the paper): pixel series per CTA, 0
 * (automatic), 128 or 64 (FP32 only; FP64 always uses 128). 64-pixel CTAs give each
 * pixel twice the shared memory at the same CTAs per SM, so chunks twice as deep and half
 * the checkpoint traffic; ws_tune_set's ctas_per_sm then counts 64-pixel CTAs.
 * ws_workspace_size() reflects the current setting. Returns WS_EINVAL for other values. */
int ws_tune_pixels_per_cta(int32_t pixels);

/* Tuning of the tile kernels (no counterpart in the paper): chunks per checkpoint of the
 * forward sweep, 0 (automatic: 2), 1 or 2. With 2 the backward sweep recomputes both
 * chunks resident in the two-stage ring from one checkpoint, halving the checkpoint words
 * written and read; with 1 every chunk has its own checkpoint and the next chunk's input
 * loads while the current one is computed. Results are identical. Returns WS_EINVAL for
 * other values. */
int ws_tune_checkpoint_group(int32_t chunks);

/* ---------------------------------------------------------------------------------
 * Ragged batches: series of different lengths (and orders) packed back to back.
 * Band b of series i occupies x[b*N + offsets[i] + t], t < T_i = offsets[i+1] - offsets[i],
 * N = offsets[n_series]; w, z likewise (w one band); lam per day packed like w
 * (WS_LAM_PER_DAY) or one value per series (WS_LAM_SCALAR). FP32.
 * A plan sorts the series by (order, length) into work items of 32 series (one per
 * lane of a warp); a persistent grid pulls items from an atomic counter, each warp
 * running the same two-sweep rotation solve as ws_smooth_batch (Section 3.1: O(T_i d)
 * storage per series).
 * Set-up and call path: ws_plan_create is set-up. It reads offsets and orders back to the
 * host (it synchronises `stream`), allocates the plan's device tables (item lists,
 * length-class tables, two error/counter words) and creates the length classes' 32
 * streams and events; ws_plan_destroy frees them. ws_plan_execute is the call path: it
 * allocates no device memory and never synchronises (except the autotuner's first run,
 * which times candidates with events). Its scratch (checkpoints, the length-class tiles
 * and their tile-kernel workspaces, the refinement state) is the caller's `workspace`,
 * sized by ws_plan_workspace_size for the same flags. Without WS_PLAN_AUTOTUNE and
 * WS_PLAN_GRAPH an execute can itself be captured into the caller's CUDA graph. */
typedef struct ws_ragged {
  int64_t n_series;            /* n >= 0 */
  const int64_t* offsets;      /* device, n + 1 entries, offsets[0] = 0, non-decreasing */
  const int8_t* d_per_series;  /* device, n orders in 1..4, or NULL: every series uses d_uniform */
  int32_t d_uniform;           /* 1..4 when d_per_series is NULL */
  int32_t n_bands;             /* B >= 1 */
  int32_t dtype;               /* WS_F32 */
  int32_t lam_mode;            /* WS_LAM_PER_DAY | WS_LAM_SCALAR */
} ws_ragged;

typedef struct ws_plan ws_plan;

typedef struct ws_plan_stats {
  int32_t n_items;        /* work items (warps of 32 series) */
  int32_t chunk_days;     /* days staged per chunk */
  int32_t warps_per_cta;
  int32_t grid;           /* persistent CTAs */
  int32_t tuned;          /* the autotuner has run */
  int32_t graph;          /* a CUDA graph is instantiated */
  float tuned_ms;         /* best time the autotuner measured */
  int32_t hp_series;      /* series of band 0 re-solved in double-float by the last refined
                             execute (reading it synchronises the device) */
  int32_t tiles;          /* WS_PLAN_TILES is honoured: 0 once the autotuner found the
                             per-lane kernel faster on this plan */
} ws_plan_stats;

#define WS_PLAN_AUTOTUNE 0x1u  /* ws_plan_execute: time the (chunk, warps/CTA) candidates once;
                                  with WS_PLAN_TILES also the length-class tiles against the
                                  best per-lane configuration, keeping them only if faster */
#define WS_PLAN_GRAPH 0x2u     /* ws_plan_execute: replay a captured CUDA graph (one band) */
#define WS_PLAN_TILES 0x8u     /* ws_plan_execute: series of at least 64 days (one band) are
                                  solved as length-class tiles by the tile kernels: padded
                                  with zero weights to a multiple of 32 days, which leaves
                                  the solution unchanged; the workspace holds four float
                                  arrays of the padded size and 32 tile workspaces */
#define WS_PLAN_REFINE 0x4u    /* ws_plan_execute: iterative refinement (the paper
                                  fixes no precision): up to three FP32 steps, r = W x - Omega z
                                  with a double-word combination, z += Omega^{-1} r; a series
                                  leaves the steps once its correction is <= 3e-6 max|z| (the
                                  others are regrouped into fresh items for the next step);
                                  series whose first correction exceeds 1e-4 max|z| (FP32
                                  too close to its conditioning limit for the corrections to
                                  measure the error), and series whose last correction is
                                  still > 3e-5 max|z| or more than half the step before it
                                  (a slowly contracting step), are solved again in
                                  double-float arithmetic (hi + lo FP32 pairs,
                                  about 48 bits). The workspace holds N floats, about 30
                                  bytes per series, (1 + largest d) x 8 bytes per day of the
                                  longest series for each thread of the re-solve (5 x 128 per SM)
                                  (9.97 GB at T = 3288, d <= 3), and with WS_PLAN_TILES a
                                  fifth tile array (the residual of the length classes' first
                                  step, which runs on their tiles). */

int ws_plan_create(const ws_ragged* rg, ws_plan** out, void* stream);

/* Bytes of device scratch ws_plan_execute needs with these flags (0 on error): the
 * per-lane kernel's checkpoints (with WS_PLAN_AUTOTUNE before the autotuner has run, the
 * largest candidate's), plus the length-class tiles with WS_PLAN_TILES, plus the
 * refinement state with WS_PLAN_REFINE. Its contents need no initialisation. */
size_t ws_plan_workspace_size(const ws_plan* plan, uint32_t flags);

/* z = Omega^{-1} W x for every series of the plan (Eq. 3 with each series' own T_i and d).
 * status: optional per-series codes. flags: WS_PLAN_AUTOTUNE, WS_PLAN_GRAPH, WS_PLAN_REFINE,
 * WS_PLAN_TILES. workspace: device, 256-byte aligned, ws_bytes >=
 * ws_plan_workspace_size(plan, flags), else WS_EINVAL / WS_ENOMEM_WS before any launch;
 * it must stay allocated while the call runs (and while ws_plan_info may read the re-solve
 * count of the last refined execute from it); calls that overlap in time need different
 * workspaces. With WS_PLAN_AUTOTUNE the first call times the candidates (running the solve
 * several times on these buffers) and keeps the fastest; with WS_PLAN_GRAPH the launch is
 * captured once (again when the workspace or configuration changes) and later calls update
 * its arguments and replay it. */
int ws_plan_execute(ws_plan* plan, const void* x, const void* w, const void* lam, void* z, uint8_t* status,
                    uint32_t flags, void* workspace, size_t ws_bytes, void* stream);

int ws_plan_info(const ws_plan* plan, ws_plan_stats* out);

void ws_plan_destroy(ws_plan* plan);

/* Synchronises `stream`, reads and clears the device error word in `workspace`.
 * Returns WS_OK, WS_ETIMEOUT (a device-side wait gave up: its outputs are invalid)
 * or WS_ECUDA. */
int ws_sync_status(void* workspace, size_t ws_bytes, void* stream);

/* Diagnostic of the bounded device-side waits: launches one CTA that waits on an mbarrier no
 * thread ever arrives at, with the bounded wait of the staging pipelines; after the wait
 * limit (about one second) it gives up, records the timeout in the workspace's error word
 * (the first 256 bytes, as ws_smooth_batch's) and returns. A following ws_sync_status
 * returns WS_ETIMEOUT and clears the word; the context stays usable. workspace: device,
 * 256-byte aligned, at least 256 bytes. No counterpart in the paper. */
int ws_selftest_wait(void* workspace, size_t ws_bytes, void* stream);

/* Copies the text of the last error on the calling thread into buf (NUL-terminated,
 * truncated to n bytes). Returns the code of that error (WS_OK if none). */
int ws_last_error(char* buf, size_t n);

/* Library version string, e.g. "ws_b300 0.1 sm_103a". */
const char* ws_version(void);

#ifdef __cplusplus
}
#endif

#endif /* WS_B300_H */
