/*
 * lamp.h — C ABI of the GB300 (sm_103a) implementation of Log-Averaged Mirror
 * Prox (LAMP, arXiv 2511.11359) for discrete optimal transport
 *
 *     min_{X in Pi(r,c)} <C, X>                      (Eq. prob:primal_ot)
 *
 * through the l1-penalised saddle problem (Eq. prob:spp), solved by Alg. 2:
 * a dual-only mirror-prox iteration whose primal coupling
 *
 *     X = diag(r) p^{eta_t}(nu),   p^{eta}(nu)_ij = exp(-(C_ij + 2K nu_j)/eta) / Z_i
 *
 * (Eq. def:dual_to_primal, K = ||C||_inf) is never stored: every iteration
 * makes one fused pass that computes the row log-normalisers log Z_i and the
 * column marginals col(X) of the two couplings the iteration needs
 * (Section 4.1), in O(n + m) memory.
 *
 * Conventions for every entry point
 *   - Return value: LAMP_OK (0) or one of the LAMP_E_* codes below.  On error
 *     lamp_last_error(ctx) returns a one-line description (ctx may be NULL for
 *     errors raised before a context exists; the message is then thread-local).
 *   - Device pointers are CUDA global-memory pointers of the device that is
 *     current when lamp_create is called.  Host pointers are ordinary memory.
 *   - Input buffers are borrowed: the caller keeps them alive and unchanged
 *     for the lifetime of the context.  The library never copies or stores C
 *     and never forms X.
 *   - All device work goes to the CUDA stream given to lamp_create (NULL = the
 *     legacy default stream).  Entry points that return results to host memory
 *     synchronise that stream before returning.
 *   - Floating point: costs and points are float32; marginals, potentials and
 *     all reported scalars are float64.  The inner loops run in float32 with a
 *     compensated exponent; row/column sums are combined in float64.
 *   - Not thread-safe per context; distinct contexts may be used concurrently.
 */
#ifndef LAMP_H_
#define LAMP_H_

#include <stdint.h>

#if defined(__GNUC__)
#define LAMP_API __attribute__((visibility("default")))
#else
#define LAMP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LAMP_OK 0
#define LAMP_E_INVALID 1        /* bad argument: sizes, pointers, parameters, marginals */
#define LAMP_E_CUDA 2           /* a CUDA runtime call failed (message holds its text)  */
#define LAMP_E_NOMEM 3          /* device allocation failed                             */
#define LAMP_E_NOT_CONVERGED 4  /* lamp_solve hit max_iter; the result is still valid    */
#define LAMP_E_NUMERIC 5        /* a non-finite or out-of-range sum appeared            */
#define LAMP_E_TIMEOUT 6        /* a device-side wait ran out of its iteration budget   */
#define LAMP_E_UNSUPPORTED 7    /* valid request this build does not implement          */

typedef struct lamp_ctx lamp_ctx;

/* How the cost matrix is given. */
typedef enum {
  LAMP_COST_DENSE = 0,    /* stored n x m float32 matrix C, row-major with leading dimension ldc */
  LAMP_COST_SQEUCLID = 1, /* C_ij = cost_scale * |x_i - y_j|^2 generated on the fly from points */
  LAMP_COST_L1 = 2,       /* C_ij = cost_scale * sum_k |x_ik - y_jk|  (App. E.2 metric comparison) */
  LAMP_COST_LINF = 3,     /* C_ij = cost_scale * max_k |x_ik - y_jk|  (App. E.2 metric comparison) */
  LAMP_COST_COSINE = 4    /* C_ij = cost_scale * (1 - x_i.y_j / (|x_i| |y_j|))  (App. E.2 cell omics);
                             points must be nonzero.  Evaluated as cost_scale * |u_i - v_j|^2 with
                             u = x / (sqrt 2 |x|), v = y / (sqrt 2 |y|): the SQEUCLID machinery on
                             normalised copies the context owns */
} lamp_cost_kind;

/* Arithmetic of the cost generation for LAMP_COST_SQEUCLID. */
typedef enum {
  LAMP_PREC_FP32 = 0,     /* x.y in float32 on CUDA cores                                  */
  LAMP_PREC_BF16_TC = 1   /* x.y with bf16-rounded points on tcgen05 tensor cores, float32
                             accumulation; the problem solved is the one of the rounded points */
} lamp_precision;

/*
 * Problem data (Section 2.1).  All pointers are DEVICE pointers and borrowed.
 *   n, m      number of source / target supports, n >= 1, m >= 1, n*m < 2^62.
 *   d         point dimension of the point-cloud kinds (1 <= d <= 64); ignored for DENSE.
 *   kind      lamp_cost_kind.
 *   C, ldc    DENSE: row-major n x m float32, entry (i,j) at C[i*ldc + j], ldc >= m,
 *             entries >= 0 and finite (C in R_+^{n x m}, Alg. 2).  With C 16-byte
 *             aligned and ldc a multiple of 4 the sweeps stream C by tensor (TMA)
 *             copies; otherwise by plain loads (same results up to rounding).
 *   x, y      point-cloud kinds: row-major n x d and m x d float32 point coordinates.
 *   r, c      float64 marginals, entries > 0, each summing to 1 within 1e-9
 *             (r in Delta^n, c in Delta^m with full support, Lemma l1_prob_equiv).
 *   cost_scale  multiplier s of a point-cloud cost: s > 0 uses s as given; s = 0
 *             means 1; s < 0 means 1 / max_ij of the unscaled cost (normalised to max 1).
 * LAMP_PREC_BF16_TC applies to SQEUCLID and COSINE; L1 and LINF use the float32 direct
 * form (packed f32x2 sweeps for d <= 8).  lamp_grad needs SQEUCLID.
 */
typedef struct {
  int64_t n, m, d;
  int32_t kind;
  int32_t _pad0;
  const float* C;
  int64_t ldc;
  const float* x;
  const float* y;
  const double* r;
  const double* c;
  double cost_scale;
} lamp_problem;

/*
 * Alg. 2 parameters.  lamp_params_default fills the paper's experimental
 * settings (App. E.2): eta = 0, tau1 = tau2 = 1/(2K), alpha = 0.01, beta = 1.1.
 *   eta        entropic coefficient >= 0, in cost units (Eq. prob:primal_eot); tau1*eta <= 1.
 *   tau1, tau2 primal / dual step sizes; 0 means 1/(2K).
 *   alpha      dual-entropy smoothing, c^alpha = c + alpha/m (Section 3.1), > 0.
 *   beta       clip level of tclip (Section 3.1), > 0.
 *   tol        L1 infeasibility target of lamp_solve: stop at the first t with
 *              ||col(X^t) - c||_1 + ||row(X^t) - r||_1 <= tol (App. E.2).
 *   max_iter   lamp_solve stops at iteration index t = max_iter at the latest.
 *   check_every how many iterations run on the device between host polls (>= 1).
 *   prec       lamp_precision (SQEUCLID only).
 *   infeas_only for eta > 0: 0 (default) stops on infeasibility only once also
 *              1 - kappa_t eta <= tol (X^t then solves the eta problem, not the eta_t one);
 *              1 stops on infeasibility alone.  Ignored for eta = 0.
 *   K          0: ||C||_inf computed on the device from the cost the kernels use;
 *              > 0: use this value for K.
 *   gap_tol    > 0: lamp_solve also stops at the first evaluated X^t whose primal-dual
 *              gap P^eta(X^t) - max(D(theta^t), D(nu^t)) of the saddle problem is <= gap_tol
 *              (App. B duals, App. E.2 termination); 0: no gap test.
 *   gap_every  iterations between gap evaluations (0 means check_every); each costs one
 *              evaluation pass and the dual sweeps of lamp_dual.
 */
typedef struct {
  double eta, tau1, tau2, alpha, beta, tol;
  int64_t max_iter, check_every;
  int32_t prec;
  int32_t infeas_only;
  double K;
  double gap_tol;
  int64_t gap_every;
} lamp_params;

/* Summary of the current state (all host values).
 *   iters    iteration index t of the state (number of updates applied).
 *   infeas   ||col(X^t) - c||_1 + ||row(X^t) - r||_1 (float64 sums).
 *   obj_CX   <C, X^t>.
 *   kappa    1/eta_t.   K  the ||C||_inf in use.   status  LAMP_OK, LAMP_E_NOT_CONVERGED or LAMP_E_NUMERIC.
 *   stop     why lamp_solve stopped: LAMP_STOP_INFEAS, LAMP_STOP_GAP or LAMP_STOP_MAX_ITER (0 otherwise).
 *   gap      the last evaluated primal-dual gap (gap_tol > 0), else NaN. */
#define LAMP_STOP_INFEAS 1
#define LAMP_STOP_GAP 2
#define LAMP_STOP_MAX_ITER 3
typedef struct {
  int64_t iters;
  double infeas, obj_CX, kappa, K;
  int32_t status;
  int32_t stop;
  double gap;
} lamp_result;

/* Fill *p with the defaults listed above (tol = 1e-6, max_iter = 100000, check_every = 50). */
LAMP_API int lamp_params_default(lamp_params* p);

/* Validate the problem and parameters, allocate the O(n + m) device workspace,
 * compute K (unless given) and the cost scale, and set the Alg. 2 start
 * (theta = nu = 0, eta_0 = infinity).  stream: a cudaStream_t, or NULL.
 * Errors: LAMP_E_INVALID (nothing allocated), LAMP_E_NOMEM, LAMP_E_CUDA. */
LAMP_API int lamp_create(lamp_ctx** out, const lamp_problem* prob, const lamp_params* params, void* stream);

/* Run Alg. 2 from the current state until the infeasibility of X^t is <= tol
 * (for eta > 0 see infeas_only), or, with gap_tol > 0, until an evaluated X^t has a
 * primal-dual gap <= gap_tol, or t reaches max_iter (App. E.2 termination, checked on
 * X^t before the iteration's updates).  The state left in the context is that X^t's
 * state.  Returns LAMP_OK, LAMP_E_NOT_CONVERGED (max_iter reached; *out is valid),
 * LAMP_E_NUMERIC or LAMP_E_CUDA.  out may be NULL. */
LAMP_API int lamp_solve(lamp_ctx* ctx, lamp_result* out);

/* Apply exactly `iters` iterations of Alg. 2 to the current state with no
 * termination test (iters >= 0).  Asynchronous on the context's stream. */
LAMP_API int lamp_iterate(lamp_ctx* ctx, int64_t iters);

/* Evaluate the current state t: one fused pass computing col(X^t), log Z and
 * the objective quantities, written to host memory (synchronises):
 *   out[0] <C, X^t>             out[1] ||col(X^t) - c||_1   out[2] ||row(X^t) - r||_1
 *   out[3] H(X^t)               (entropy identity of App. D, from O(n+m) values)
 *   out[4] P^eta(X^t)           (Eq. prob:l1_ot_primal)
 *   out[5] certificate RHS 4K||col-c||_1 + 2K log m / t (Prop. infeas_bound (a); eta = 0, t >= 1, else NaN)
 *   out[6] saddle dual max(D(theta^t), D(nu^t)), as lamp_dual (two or four extra sweeps)
 *   out[7] K
 *   out[8] L = <C, X^t> - eta H(X^t), the entropic objective of Eq. prob:primal_eot at X^t (the
 *          loss the autograd form returns; its gradient is lamp_grad's)
 *   out[9] primal-dual gap out[4] - out[6] of the saddle problem (App. B, App. E.2), >= 0 up to
 *          rounding by weak duality
 * out must hold LAMP_OBJECTIVE_SLOTS doubles. */
#define LAMP_OBJECTIVE_SLOTS 10
LAMP_API int lamp_objective(lamp_ctx* ctx, double out[LAMP_OBJECTIVE_SLOTS]);

/* Transport-map application (App. E, colour transfer): with the current
 * X^t = diag(r) p^{eta_t}(nu^t) and p row-stochastic,
 *   side 0: out = p V      (V: device m x k float32 row-major; out: device n x k)
 *   side 1: out = p^T U    (U: device n x k float32 row-major; out: device m x k)
 * 1 <= k <= 8 value columns (colour channels, coordinates: p y is the barycentric map).
 * One evaluation pass, then one recompute sweep of X^t over all n m entries with
 * float32 exponents as in the iteration and float64 accumulation across tiles.
 * The first call with k larger than the context's partial-sum width (3, or d for
 * |x - y|^2 with d <= 8) widens two O(k (n + m) splits) buffers (LAMP_E_NOMEM if that
 * fails).  Asynchronous on the context's stream after the evaluation pass. */
LAMP_API int lamp_apply_map(lamp_ctx* ctx, const float* V, int64_t k, float* out, int side);

/* Dual function of the saddle problem (App. B, Eqs. def:dual_spp, def:dual_spp_e)
 *   D(phi)     = sum_i r_i min_j (C_ij + 2K phi_j) - 2K <c, phi>                       (eta = 0)
 *   D^eta(phi) = sum_i r_i softmin^eta_j (C_ij + 2K phi_j) - 2K <c, phi> - eta H(r)     (eta > 0)
 * at phi = theta^t (out[0]) and phi = nu^t (out[1]); host memory, synchronises.  For
 * any phi in [-1, 1]^m it is a lower bound on the optimal value of the penalised problem
 * (weak duality).  eta = 0: two row-max sweeps per phi at a large kappa, the second with
 * the row shifts of the first and the sub-grid remainders of the column offsets
 * subtracted, so the row minima of the kernels' float32 cost come out to about 1e-12 K
 * (the float32 cost itself differs from an exact one by its own rounding; a
 * LAMP_PREC_BF16_TC context runs both sweeps on the tensor cores, so its bound is on the
 * cost its iteration uses, x.y of the bf16 points accumulated in float32); eta > 0: a
 * row-max and a row-sum sweep per phi at kappa = 1/eta (relative error of the row sums
 * about 2^-22, i.e. about 2^-22 eta in the softmin).  The state is not changed. */
LAMP_API int lamp_dual(lamp_ctx* ctx, double out[2]);

/* Round (Alg. 3, Altschuler et al.) of the current X^t, returned in factored form
 *   Round(X^t) = X^t diag(y) + delta_r delta_c^T / ||delta_r||_1,
 * with y_j = min(c_j / col(X^t)_j, 1), delta_c = c - col(X^t diag(y)) = max(c - col(X^t), 0)
 * and delta_r = r - row(X^t diag(y)) >= 0 (Step 1 is the identity: row(X^t) = r by
 * construction).  Round(X^t) is in Pi(r, c).  out (host, synchronises):
 *   out[0] <C, Round(X^t)>   (the left side of Prop. infeas_bound (a) plus <C, X*>)
 *   out[1] ||delta_r||_1      out[2] ||delta_c||_1      out[3] <C, X^t diag(y)>
 * y (m), delta_r (n), delta_c (m): device float64 buffers, each may be NULL.
 * Cost: one evaluation pass, one row sweep and O(n + m) work (|x - y|^2), or one more
 * pass over the stored C (LAMP_COST_DENSE).  The state is not changed. */
LAMP_API int lamp_round(lamp_ctx* ctx, double out[4], double* y, double* delta_r, double* delta_c);

/* Gradient of L = <C, X> - eta H(X) at the current state's X^t with respect
 * to the points (envelope theorem): dL/dx_i = sum_j X_ij dC_ij/dx_i and
 * dL/dy_j = sum_i X_ij dC_ij/dy_j, with dC_ij/dx_i = 2 s (x_i - y_j).
 * dx: device n x d float32, dy: device m x d float32 (either may be NULL).
 * One evaluation pass (skipped when the state's X^t was the last one evaluated, e.g. after
 * lamp_solve or lamp_objective), then per side one recompute pass (X never stored):
 *   LAMP_PREC_FP32: ceil(d / 8) float32 sweeps per side (chunks of 8 coordinates);
 *   LAMP_PREC_BF16_TC: one tensor-core pass per side on the bf16-rounded points the
 *   context solves with: S = x.y^T by tcgen05, the coupling's entries formed in the
 *   epilogue and split into two bf16 parts (16 significant bits), sum_j X_ij y_j by a
 *   second tcgen05 MMA with float32 accumulation; the first call allocates transposed
 *   bf16 copies of the points (O((n + m) 64)) and float32 partial sums (O((n + m) 64)
 *   per inner split), and a second stream of its own: with both dx and dy requested the
 *   dy side runs on it, forked from and joined back into the context's stream, so work
 *   queued later on the context's stream sees both results.
 * SQEUCLID only (LAMP_E_UNSUPPORTED otherwise).  Asynchronous. */
LAMP_API int lamp_grad(lamp_ctx* ctx, float* dx, float* dy);

/* Copy the state to host memory (synchronises).  nu, theta: m doubles; logZ:
 * n doubles, the natural-log row normalisers of X^t (valid after lamp_solve or
 * lamp_objective; NaN-filled otherwise); kappa, t: scalars; row_shifts: 2n
 * floats, the per-row exponent shifts the next iteration will use (with them a
 * restored run repeats the original bit for bit).  Any pointer may be NULL. */
LAMP_API int lamp_get_state(lamp_ctx* ctx, double* nu, double* theta, double* logZ, double* kappa, int64_t* t,
                            float* row_shifts);

/* Replace the state by (nu, theta, kappa, t) from host memory (checkpoint
 * restore): |nu_j| < 1, |theta_j| < 1, kappa >= 0, t >= 0.  row_shifts: the 2n
 * floats from lamp_get_state, or NULL to recompute them with a row-max pass. */
LAMP_API int lamp_set_state(lamp_ctx* ctx, const double* nu, const double* theta, double kappa, int64_t t,
                            const float* row_shifts);

/* Host-buffer variant used for end-to-end timing: copy x, y (SQEUCLID) or C
 * (DENSE) and r, c from HOST memory into device buffers the context owns, run
 * `iters` iterations, and copy the infeasibility of the last evaluated X^t and
 * nu (m doubles, may be NULL) back to host memory.  The context must have been
 * created with lamp_create_owned, and the uploaded data must describe the same
 * problem (K and the squared norms are not recomputed).  Synchronises. */
LAMP_API int lamp_step_host(lamp_ctx* ctx, const float* C_or_x, const float* y, const double* r, const double* c,
                   int64_t iters, double* infeas_out, double* nu_out);

/* Like lamp_create, but the context allocates and owns device copies of the
 * inputs; prob's pointers are HOST pointers and are copied once here. */
LAMP_API int lamp_create_owned(lamp_ctx** out, const lamp_problem* host_prob, const lamp_params* params, void* stream);

/* Apply iters + 1 iterations (as lamp_iterate) launched one kernel at a time, the
 * last `iters` of them with CUDA events between consecutive kernels on the context's
 * stream and one synchronisation at the end, and return the mean device time in
 * milliseconds of each kernel of an iteration in ms_out[0..3]: [0] row sweep, [1] row
 * finalize, [2] column sweep, [3] column finalize.  Synchronises.  1 <= iters <= 1000. */
LAMP_API int lamp_time_kernels(lamp_ctx* ctx, int64_t iters, double* ms_out);

/* Measurement helper with no counterpart in the paper: the sustained MUFU ex2
 * rate of the current device in results per SM per clock (dependent chains of
 * ex2.approx.ftz.f32 on every SM, timed with the SMs' cycle counters).  It is
 * the denominator of the roofline of the tensor-core sweeps.  Allocates and
 * frees two small device buffers; synchronises. */
LAMP_API int lamp_measure_ex2_rate(double* ex2_per_clk_per_sm);

/* Self-test of failure detection on the GPU: launches one thread that waits, with the
 * bounded mbarrier wait of the tensor-core sweeps limited to `polls` polls (1..2^30;
 * a poll suspends for up to 20 us, and every wait also gives up after 4 s), on a
 * barrier that nothing arrives on.  The wait gives up, records LAMP_E_TIMEOUT in a
 * device status word and the kernel returns normally; *status receives that word
 * (LAMP_E_TIMEOUT expected).  Returns LAMP_OK, or LAMP_E_INVALID / LAMP_E_NOMEM /
 * LAMP_E_CUDA.  The device stays usable afterwards.  Synchronises. */
LAMP_API int lamp_selftest_wait_timeout(int64_t polls, int* status);

/* Number of kernel launches one iteration issues (for launch accounting). */
LAMP_API int64_t lamp_launches_per_iteration(const lamp_ctx* ctx);

LAMP_API const char* lamp_last_error(const lamp_ctx* ctx);

/* Allocation-free evaluation of one coupling's marginals.  The paper has no
 * counterpart: it exists for callers that may not call cudaMalloc where they
 * run, such as plugins whose host framework owns every byte of device memory
 * through its own pool, or latency-bound loops that cannot afford the device
 * synchronisation cudaMalloc/cudaFree can cause.  No context is created.
 *
 * For X = diag(r) p^{1/kappa}(nu) it writes log Z (n doubles, natural log) to
 * logZ_out, col(X) (m doubles) to col_out and <C, X> (one double, NaN if a row
 * sum left the representable range; may be NULL) to cost_out.  prob holds
 * DEVICE pointers (DENSE, or SQEUCLID with d <= 8 and an explicit cost_scale > 0);
 * K > 0 is the ||C||_inf to use; kappa >= 0; nu: m doubles on the device.
 * Work is enqueued on `stream`; the call returns without synchronising.
 *
 * Scratch comes from a 16 MiB array compiled into the library (each GPU that
 * loads the library keeps it until the process exits).  Requests whose
 * workspace does not fit (about 136 n + 168 m bytes) return LAMP_E_INVALID.
 * The first call on a device looks up the array's device address (and looks it
 * up again when it finds a different CUDA context current on that device, e.g.
 * after cudaDeviceReset); make that call before starting any stream capture.  All calls on a device share the array:
 * calls whose GPU work overlaps (other streams, other threads) race and
 * corrupt each other, so issue them one after another on one stream.  The
 * array keeps the previous call's contents; the call clears what must start
 * at zero.  Errors: LAMP_E_INVALID, LAMP_E_UNSUPPORTED (d > 8), LAMP_E_CUDA;
 * the message is in lamp_last_error(NULL). */
LAMP_API int lamp_marginals_noalloc(const lamp_problem* prob, double K, double kappa, const double* nu,
                                    double* logZ_out, double* col_out, double* cost_out, void* stream);

/* Release everything the context owns (NULL is a no-op). */
LAMP_API void lamp_destroy(lamp_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LAMP_H_ */
