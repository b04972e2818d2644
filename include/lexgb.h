/*
 * lexgb.h -- C ABI of the GB300 (sm_103a) Leja exponential-integrator engine.
 *
 * The engine computes phi_l(hA)v, the action of the matrix exponential
 * (l = 0) and of the phi_l functions on a vector, by Newton interpolation at
 * real Leja points, and the exponential Rosenbrock-Euler and EXPRB32 steps
 * built on it.  Citations refer to Deka, Moriggl, Einkemmer, "LeXInt:
 * GPU-accelerated exponential integrators package" (arXiv 2310.08344).
 *
 * Conventions shared by every entry point
 *  - Grid: periodic unit square, nx x ny points x_i = i/nx, y_j = j/ny; a
 *    field is a contiguous array of nx*ny doubles, index j*nx + i (x fastest).
 *    Contiguous data is what the paper's RHS functors require (Sec. 2).
 *  - Operators (second-order central differences, periodic):
 *      LX_ADVDIFF  A v = nu (v_xx + v_yy) + a (v_x + v_y)        (Sec. 3, Eq. 3)
 *      LX_BURGERS  f(u) = nu (u_xx + u_yy) - u (u_x + u_y); the Jacobian
 *                  action J(u)v = nu Lap v - v (u_x+u_y) - u (v_x+v_y) is the
 *                  exact linearisation (the paper's finite-difference action,
 *                  Sec. 2.3, is replaced by it).
 *  - The paper's own discretisation (Sec. 3): periodic [-1,1)^2 (spacing
 *    2/nx, 2/ny), the Laplacian by second-order central differences and the
 *    gradient by the third-order upwind-biased scheme -- for a term +a v_x,
 *    a > 0: (-v_{i+2} + 6 v_{i+1} - 3 v_i - 2 v_{i-1}) / (6 dx), mirrored for
 *    a < 0:
 *      LX_ADVDIFF_UP3  A v = nu (v_xx + v_yy) + a (v_x + v_y)  (Problems I, II
 *                      with nu = 1, a = 10)
 *      LX_BURGERS_UP3  f(u) = nu (u_xx + u_yy) + (a/2) ((u^2)_x + (u^2)_y)
 *                      (Problem III with nu = 1, a = 10), J(u) v = nu Lap v +
 *                      a ((u v)_x + (u v)_y); the upwind side follows the sign
 *                      of a (the paper's state stays positive).
 *    LX_DF64 with LX_BURGERS_UP3 needs nx % 128 == 0 (as LX_BURGERS); batches
 *    and the allocation-free entry point take the central operators only.
 *  - Norms: ||x|| = ||x||_2 / sqrt(N) (Sec. 2.2).
 *  - Device pointers ("_dev") are CUDA global-memory pointers of the current
 *    device; host pointers ("_host") are ordinary CPU memory.  The caller
 *    allocates and owns every input and output buffer (Sec. 2.2, Listing 4);
 *    the context owns its auxiliary vectors from setup to destroy (Sec. 2.3,
 *    Listing 10).
 *  - Streams: all device work of a context runs on the stream passed at setup
 *    (NULL = the legacy default stream).  Every call synchronises that stream
 *    once before it returns, so the scalars it reports (iters, err, rho) are
 *    valid on return.  Calls on one context must not run concurrently.
 *  - Errors: every call returns an lx_status.  On an error other than
 *    LX_E_NOCONV the contents of the output buffers are unspecified; on
 *    LX_E_NOCONV they hold the last partial sum of the Newton series, which
 *    is not converged and must not be used as a result.
 */
#ifndef LEXGB_H
#define LEXGB_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LX_OK = 0,
  LX_E_INVAL = 1,     /* invalid argument (sizes, NULL, aliasing, gamma == 0) */
  LX_E_NOMEM = 2,     /* device or host allocation failed */
  LX_E_CUDA = 3,      /* a CUDA runtime call failed (see lx_last_cuda_error) */
  LX_E_NOCONV = 4,    /* Leja series not converged within the point table */
  LX_E_NONFINITE = 5, /* a NaN or Inf appeared in a norm */
  LX_E_TIMEOUT = 6,   /* a bounded device-side wait gave up */
  LX_E_CALLBACK = 7   /* a caller's right-hand side function reported an error */
} lx_status;

enum { LX_ADVDIFF = 0, LX_BURGERS = 1, LX_ADVDIFF_UP3 = 2, LX_BURGERS_UP3 = 3 }; /* lx_problem.kind */
enum { LX_FP64 = 0, LX_MIXED = 1, LX_DF64 = 2 }; /* lx_problem.precision */
enum { LX_ROS_EU = 0, LX_EXPRB32 = 1, LX_EPIRK4S3A = 2 }; /* integrator */

typedef struct {
  int nx, ny;     /* grid points per direction, each >= 1 */
  double nu;      /* diffusion coefficient */
  double a;       /* advection speed (LX_ADVDIFF, LX_ADVDIFF_UP3); flux
                     coefficient (LX_BURGERS_UP3); unused by LX_BURGERS */
  int kind;       /* LX_ADVDIFF, LX_BURGERS, LX_ADVDIFF_UP3, LX_BURGERS_UP3 */
  int precision;  /* LX_FP64: all arithmetic in double (FP64 pipe).
                     LX_MIXED: the Newton basis y_m and its stencil in float;
                     the coefficients, the polynomial p and both stopping
                     norms in double.
                     LX_DF64: FP64-accurate float-float ("double-float",
                     48-bit significand) arithmetic on the FP32 pipe for the
                     basis, the stencil and the polynomial; double inputs and
                     outputs; norms accumulated in float-float from the
                     leading float of each value.  The Burgers kinds
                     need nx % 128 == 0 in this form. */
} lx_problem;

typedef struct lx_ctx lx_ctx;

/* Human-readable name of a status code (static storage). */
const char* lx_status_str(lx_status s);

/* Message of the last CUDA error seen by this library on the calling thread
 * ("" if none). */
const char* lx_last_cuda_error(void);

/* ---------------------------------------------------------------------------
 * Host numerics (no GPU needed)
 * ------------------------------------------------------------------------- */

/* The first K greedy Leja points on [-2, 2] (Sec. 2.1: xi_j maximises
 * prod_{k<j} |x - xi_k|; |xi_0| is maximal).  Readings: xi_0 = +2; ties in
 * the maximum (1e-12 relative in the log-product) go to the larger point.
 * xi_out: host array of K doubles, written.  Computed once per process and
 * cached.  LX_E_INVAL if K <= 0 or xi_out is NULL. */
lx_status lx_leja_points(int K, double* xi_out);

/* Newton coefficients d_j = f[xi_0, ..., xi_j], j < K, of
 * f(xi) = phi_l(h (c + gamma xi)) at the points xi (Sec. 2.1, Eq. 2 with exp
 * replaced by phi_l).  FP64, by Opitz' theorem with scaled Taylor sub-steps.
 * xi: host array of K points; d_out: host array of K doubles, written.
 * LX_E_INVAL for l < 0, K <= 0, NULL pointers, gamma == 0 or non-finite
 * h*c, h*gamma; LX_E_NONFINITE if a coefficient overflows. */
lx_status lx_leja_coeffs(int l, double h, double c, double gamma, const double* xi, int K, double* d_out);

/* Number of Newton coefficients the engine computes and uses for (h, c,
 * gamma) with a table of K points: the first J with the bound
 * (2 h|gamma|)^J / J! * e^{max(0, h (c + 2|gamma|))} below 1e-40, plus 8, at
 * most K (the factor 2 covers the geometric growth of the Newton basis when
 * the spectrum reaches off the real focal interval).  The Leja loop stops
 * with LX_E_NOCONV after J - 1 iterations. */
int lx_leja_coeff_count(double h, double c, double gamma, int K);

/* Focal interval of the real Leja points from a spectral-radius estimate
 * (Sec. 2.2, Listing 7: the largest eigenvalue magnitude rho, enlarged by
 * 5 %, gives lambda = -1.05 rho, and the interpolation interval [lambda, 0]
 * has centre c = lambda / 2 and quarter-width gamma = -lambda / 4).
 *   rho       spectral-radius estimate (power_bound), finite and > 0
 *   c, gamma  host doubles, written on success
 * LX_E_INVAL for NULL outputs or rho not finite and positive (a zero
 * operator has no interval: gamma would be 0). */
lx_status lx_spectral_interval(double rho, double* c, double* gamma);

/* ---------------------------------------------------------------------------
 * Context (the paper's struct Leja, Sec. 2.3 Listing 10)
 * ------------------------------------------------------------------------- */

/* Create a context for one problem: uploads the Leja point table, allocates
 * the auxiliary vectors (two basis vectors, stage vectors of the integrator,
 * reduction scratch) and builds the CUDA graph of the Leja loop.
 *   prob        problem description (copied)
 *   integrator  LX_ROS_EU or LX_EXPRB32 (the integrator expint_step runs)
 *   max_leja    size K of the Leja point table, 16 <= K <= 4096 (0: 1000)
 *   cuda_stream a cudaStream_t of the current device, or NULL
 *   out         receives the context
 * Errors: LX_E_INVAL (bad sizes/kind/precision), LX_E_NOMEM, LX_E_CUDA. */
lx_status leja_setup(const lx_problem* prob, int integrator, int max_leja, void* cuda_stream, lx_ctx** out);

/* Free the context and its device memory.  NULL is accepted. */
void leja_destroy(lx_ctx* ctx);

/* Spectral bound by power iteration (Sec. 2, Listing 7: the dominant
 * eigenvalue gives c = lambda/2, gamma = -lambda/4 with lambda = -1.05 rho).
 *   u_dev      linearisation point (Burgers kinds: J(u); diffusion-advection: ignored,
 *              may be NULL)
 *   v0_dev     start vector, N doubles, not modified (must not be constant:
 *              constants are in the null space of the periodic operators)
 *   max_iters  1..64 matrix-vector products
 *   rho        receives the estimate ||A v_k|| / ||v_k|| of the last pass
 *   iters      receives the number of passes (may be NULL)
 * Stops after max_iters passes or when |rho_k - rho_{k-1}| <= 1e-2 rho_k. */
lx_status power_bound(lx_ctx* ctx, const double* u_dev, const double* v0_dev, int max_iters, double* rho,
                      int* iters);

/* phi_l(h Op) w by Leja interpolation (Sec. 2.2 Listings 2-3, Sec. 2.3
 * Listings 8, 9, 11: real_Leja_exp for l = 0, real_Leja_phi_nl /
 * real_Leja_phi otherwise).  Op is A (diffusion-advection kinds) or J(u) (Burgers kinds).
 *   l          0..8
 *   u_dev      linearisation point (Burgers kinds), else ignored / NULL
 *   w_dev      input vector (N doubles), not modified
 *   out_dev    output p (N doubles); must not alias w_dev or u_dev
 *   c, gamma   centre and quarter-width of the focal interval [c-2g, c+2g]
 *   h          step size
 *   rtol, atol stop when |d_m| ||y_m|| <= rtol ||p_m|| + atol
 *   iters      receives the number of Leja iterations (matrix-vector
 *              products) m at the stop (may be NULL)
 * The loop runs as a CUDA graph whose while-node is ended by the device: no
 * host synchronisation per iteration. */
lx_status phi_l_apply(lx_ctx* ctx, int l, const double* u_dev, const double* w_dev, double* out_dev, double c,
                      double gamma, double h, double rtol, double atol, int* iters);

/* "Vertical" interpolation (Sec. 2.3, real_Leja_phi with several integrator
 * coefficients): out[j] = phi_l(alpha[j] h J) w for j < nc (1..4) from ONE
 * Newton basis at the same Leja points, shift cc and scale gamma -- only the
 * divided differences (of phi_l(alpha_j h (cc + gamma xi))) differ per j, so
 * one fused launch per iteration moves y once and the nc polynomials once.
 * The loop stops at the first iteration at which every polynomial passes its
 * own test |d^(j)_{m+1}| ||y_{m+1}|| <= rtol ||p^(j)|| + atol (the paper
 * states no rule for several polynomials; this is the reading used), so
 * *iters is at least the largest single-alpha count.
 *   alpha: host array of nc step fractions, each > 0 (typically <= 1; the
 *          table length follows the largest one);
 *   out:   host array of nc distinct device pointers (nx*ny doubles each, not
 *          aliasing u or w);
 *   u, w, cc, gamma, h, rtol, atol: as in phi_l_apply.
 * LX_DF64 contexts of the central operators need nx % 128 == 0 and a 16-byte
 * aligned w (else LX_E_INVAL); the upwind kinds run one thread per point
 * and take any layout.  Buffers for the nc polynomials are allocated on
 * first use and kept until leja_destroy. */
lx_status phi_l_apply_vertical(lx_ctx* ctx, int l, int nc, const double* alpha, const double* u,
                               const double* w, double* const* out, double cc, double gamma, double h,
                               double rtol, double atol, int* iters);

/* One step of the context's integrator (Sec. 2.2 Listings 5-6; Sec. 2.3
 * Listings 12-13; EPIRK4s3A of Sec. 3, Table 2):
 *   LX_ROS_EU   u_high = u + phi_1(h J(u)) h f(u); u_low unused (may be
 *               NULL); err = 0.
 *   LX_EXPRB32  u_low  = a = u + phi_1(h J(u)) h f(u)
 *               u_high = a + 2 phi_3(h J(u)) R,  R = h (F(a) - F(u)),
 *               F(k) = f(k) - J(u) k;  err = ||2 phi_3(h J(u)) R||.
 *               (For the quadratic Burgers f, R = -h p (p_x + p_y) with
 *               p = a - u, which is how the engine evaluates it.)
 *   LX_EPIRK4S3A  fourth order, with the coefficients the stiff order
 *               conditions fix for the stage nodes 1/2 and 2/3 (the paper
 *               names the scheme, not its coefficients):
 *               P_i = phi_1(c_i h J) h f(u) for c = 1/2, 2/3, 1 from one
 *               vertical loop, R_i = h (F(u + c_i P_i) - F(u)),
 *               u_low  = u + P_1 + phi_3(h J)(32 R_2 - 27/2 R_3) (third order)
 *               u_high = u_low + phi_4(h J)(-144 R_2 + 81 R_3) (fourth order),
 *               err = ||u_high - u_low||.  Needs nx % 128 == 0 with LX_DF64
 *               and the central operators (vertical interpolation).
 * u_dev is not modified; u_low_dev and u_high_dev must not alias u_dev or
 * each other.  iters receives the total Leja iterations of the step. */
lx_status expint_step(lx_ctx* ctx, const double* u_dev, double* u_low_dev, double* u_high_dev, double c,
                      double gamma, double h, double rtol, double atol, double* err, int* iters);

/* expint_step on HOST buffers: copies u_host to the device, runs the step
 * and copies the results back (context-owned staging buffers; nothing is
 * allocated per call).  For page-locked host memory the copies are
 * asynchronous DMA transfers.  u_low_host may be NULL. */
lx_status expint_step_host(lx_ctx* ctx, const double* u_host, double* u_low_host, double* u_high_host, double c,
                           double gamma, double h, double rtol, double atol, double* err, int* iters);

/* Time-independent source term S (Sec. 3, Eq. 4, the diffusion-advection problem
 * with sources; any kind): after this call expint_step, expint_step_host
 * and lx_integrate integrate u' = f(u) + S, i.e. the right-hand side of
 * every step is h (f(u) + S); the Jacobian, the spectral bound and the
 * EXPRB32 remainder R = h (F(a) - F(u)) are unchanged (S cancels in R).
 * For a linear f this makes the Rosenbrock-Euler step
 * u + h phi_1(h A) (A u + S), the exact solution of the affine problem.
 * s_dev: device vector of nx*ny doubles, borrowed (it must stay valid and
 * unchanged while steps run); NULL removes the source.  phi_l_apply is not
 * affected. */
lx_status lx_ctx_set_source(lx_ctx* ctx, const double* s_dev);

/* Classical step-size controller for the embedded third-order pair (Sec.
 * 2.2 mentions that the EXPRB32 error estimate can steer the step size but
 * gives no controller):
 *   h_new = h * min(2, max(0.2, 0.9 (tol/err)^(1/3)))   (factor 2 if err = 0).
 * Host arithmetic only. */
double lx_controller_classical(double h, double err, double tol);

typedef struct {
  double t;             /* in: start time; out: time reached */
  double h;             /* in: first trial step (> 0); out: next proposed step */
  int steps;            /* out: accepted steps */
  int rejected;         /* out: rejected attempts */
  long long leja_iters; /* out: Leja iterations of all attempts */
  double last_err;      /* out: error estimate of the last attempt */
  int power_iters;      /* in: power-iteration passes per attempt (0: 10) */
} lx_integrate_info;

/* Adaptive EXPRB32 integration of the context's problem from info->t to
 * t_final (Listing 7's time loop with step control): every attempt takes a
 * power-iteration bound at the current state from v0_dev (c, gamma from
 * lambda = -1.05 rho), one expint_step with Leja tolerance leja_tol (rtol =
 * atol), accepts the step when err <= tol and sets the next step size with
 * lx_controller_classical.  u_dev (N doubles) holds the state and is updated
 * in place.  Requires a context set up with LX_EXPRB32.  At most
 * max_attempts attempts; info->t < t_final on return means the budget ran
 * out.  The context's staging vectors are allocated on the first call. */
lx_status lx_integrate(lx_ctx* ctx, double* u_dev, const double* v0_dev, double t_final, double tol,
                       double leja_tol, int max_attempts, lx_integrate_info* info);

/* Forward declaration of the controller network (see mlp_setup below). */
typedef struct lx_mlp lx_mlp;

/* lx_integrate with the learned controller: after every accepted step the
 * network proposes the next step size from the attempt's features
 * (log(rho h), log(h / dt_ref), iters / 100, log10(err / tol), ||u||); the
 * factor is clipped to [0.2, 16] (the classical controller grows by at most
 * 2 per step; the network, trained on steps up to 16 times the current one,
 * may jump further, e.g. from a cautious first step).  Rejections, and
 * non-finite proposals, fall
 * back to lx_controller_classical.  The embedded error test (err <= tol)
 * still accepts or rejects every step.  dt_ref > 0 is the explicit CFL step
 * used in the features. */
lx_status lx_integrate_learned(lx_ctx* ctx, double* u_dev, const double* v0_dev, double t_final, double tol,
                               double leja_tol, int max_attempts, lx_mlp* model, double dt_ref,
                               lx_integrate_info* info);

/* Timing of the Leja loops run by this context since the last reset: the
 * summed CUDA-event time of the loop graphs (milliseconds, measured on the
 * context stream) and the number of Leja iterations they ran.  The average
 * duration of one fused Leja-iteration launch is loop_ms / iterations. */
typedef struct {
  double loop_ms;             /* CUDA-event time of the Leja loops */
  long long loop_iterations;  /* fused-iteration launches that did work */
  long long loop_launches;    /* Leja loops run */
  double power_ms;            /* CUDA-event time of power_bound calls */
  long long kernels;          /* kernel launches of this library on the context's stream */
} lx_stats;
lx_status lx_ctx_stats(lx_ctx* ctx, lx_stats* out, int reset);

/* Loop launch mode: 0 (default) runs each Leja loop as one CUDA graph with a
 * device-ended while node; 1 launches the iteration kernels from the host in
 * batches of 8 with a status read-back per batch, for profilers that cannot
 * see kernels inside conditional graphs.  The environment variable
 * LEXGB_STREAM_LOOP=1 selects mode 1 at setup. */
lx_status lx_ctx_set_loop_mode(lx_ctx* ctx, int stream_loop);

/* Graph loop unrolling: the while body of each loop graph holds `unroll`
 * (1..8, default 4) chained launches of the fused iteration, so the loop
 * condition is evaluated once per `unroll` iterations; launches that start
 * after the device-side stop return without work (at most unroll - 1 per
 * loop).  Results are identical for every value.  Rebuilds the context's
 * loop graphs with their selected kernels. */
lx_status lx_ctx_set_graph_unroll(lx_ctx* ctx, int unroll);

/* Autotuner of the fused Leja iteration (a tile-shape search).  Times every
 * candidate kernel of the context's (kind, precision) -- for LX_DF64 the
 * shared-memory-pipelined kernel at 2, 3 and 4 resident blocks per SM, the
 * register-window kernel and the two-step (two Leja iterations per pass
 * over memory) pipelined kernel; for the upwind kinds the one- and two-step
 * pipelined kernels, the point-wise kernel and, for LX_BURGERS_UP3, the
 * product-form and point-weight forms -- at strip heights 8..128 rows and, for the
 * pipelined kernels, strip height 0 (one balanced contiguous row range per
 * warp), each for
 * `iters` launches (1..50) on the context's own buffers, and selects the
 * fastest per Leja iteration for the vector-access ("wide") class.  cache_path (may be NULL) is
 * a text file of lines "<device|SMs|nx x ny|kind|precision> <kernel> <strip
 * height> <us>": a matching line is applied without timing, and a new
 * result is appended.  report (may be NULL) receives a JSON summary.  The
 * context's auxiliary vectors are overwritten (with zeros). */
lx_status lx_ctx_autotune(lx_ctx* ctx, int iters, const char* cache_path, char* report, int len);

/* Select a fused-iteration kernel by name (as reported by the autotuner or
 * lx_ctx_kernel_name) and strip height (>= 1 rows, or 0 for balanced row
 * ranges, pipelined kernels only; LX_E_INVAL otherwise). */
lx_status lx_ctx_select_kernel(lx_ctx* ctx, const char* name, int strip_h);

/* Kernel selection of the context (for diagnostics): writes a short name of
 * the fused Leja-iteration kernel into buf (NUL-terminated, at most len). */
lx_status lx_ctx_kernel_name(lx_ctx* ctx, char* buf, int len);

/* Leja iterations per launch of the selected fused-iteration kernel: 1, or 2
 * for the two-step (temporally blocked) kernels; 0 before any selection. */
int lx_ctx_iters_per_launch(lx_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Batched instances.  Not in the paper: many independent problems of uneven
 * grid sizes advance through the Leja loop together -- one fused launch per
 * iteration (LX_FP64) or per two iterations (LX_DF64, with the stopping
 * test after each) covers every instance that has not converged, each
 * instance has its own coefficients, weights, stopping test and status, and
 * one CUDA graph runs the whole loop (with LEXGB_STREAM_LOOP=1 in the
 * environment at setup, the host launches the same kernel instead, for
 * profilers that cannot see kernels inside a conditional graph).
 * ------------------------------------------------------------------------- */

typedef struct lx_batch lx_batch;

/* Set up a batch of `count` diffusion-advection problems (kind LX_ADVDIFF),
 * all of precision LX_FP64, or all LX_DF64 with nx % 128 == 0 (float-float
 * batches then also need 16-byte aligned w and out in batch_step, else
 * LX_E_INVAL there).  Allocates the per-instance basis vectors (and, for
 * LX_DF64, polynomials) and the strip table.  max_leja as in leja_setup. */
lx_status batch_setup(int count, const lx_problem* probs, int max_leja, void* cuda_stream, lx_batch** out);

/* phi_l(h_i A_i) w_i for every instance i (Sec. 2.1 Eq. 2 per instance).
 *   w_dev, out_dev   host arrays of `count` device pointers (inputs are not
 *                    modified; out_dev[i] must not alias w_dev[i])
 *   c, gamma, h      host arrays of `count` doubles
 *   rtol, atol       stopping test, shared
 *   iters, status    host arrays of `count` ints (may be NULL): Leja
 *                    iterations and lx_status of each instance
 * Returns LX_OK, a call-level error, or the first non-OK instance status. */
lx_status batch_step(lx_batch* b, int l, const double* const* w_dev, double* const* out_dev, const double* c,
                     const double* gamma, const double* h, double rtol, double atol, int* iters, int* status);

/* Loop timing of the batch (as lx_ctx_stats; loop_iterations counts launches
 * of the fused batch kernel). */
lx_status batch_stats(lx_batch* b, lx_stats* out, int reset);

void batch_destroy(lx_batch* b);

/* ---------------------------------------------------------------------------
 * Learned step-size controller (not in the paper): a 5 -> 64 -> 64 -> 64 -> 2
 * ReLU MLP, BF16 weights and activations with FP32 accumulation on the tensor
 * cores.  Inputs (per attempted step): log(rho h), log(h / dt_CFL),
 * iters / 100, log10(err / tol), ||u||; outputs: log(h_next / h) and
 * log(iters predicted).  It only proposes step sizes: the embedded error
 * test still accepts or rejects every step.
 * Parameter vector (FP32, mlp_param_count() floats): W1[5][64], b1[64],
 * W2[64][64], b2[64], W3[64][64], b3[64], W4[64][2], b4[2] (W[i][j] joins
 * input i to output j).  Normalisation vector (14 floats): mean_x[5],
 * std_x[5], mean_y[2], std_y[2]; the network works on normalised values.
 * ------------------------------------------------------------------------- */

int mlp_param_count(void);

/* Create a model for batches of up to batch_max rows from host weights and
 * normalisation (both copied). */
lx_status mlp_setup(int batch_max, const float* w_host, const float* norm_host, void* cuda_stream, lx_mlp** out);

/* Current FP32 master weights to the host. */
lx_status mlp_get_weights(lx_mlp* m, float* w_host);

/* y[B][2] = net(x[B][5]), device row-major arrays. */
lx_status mlp_forward(lx_mlp* m, const float* x_dev, float* y_dev, int B);

/* The same for host arrays, B <= 64 (inference inside a time loop). */
lx_status mlp_forward_host(lx_mlp* m, const float* x_host, float* y_host, int B);

/* One training step on device arrays x[B][5], targets t[B][2]: the loss
 * sum_rows sum_outputs (y_n - t_n)^2 / (2 B) on normalised values, its
 * gradient (forward and backward on the tensor cores, per-CTA partials added
 * in a fixed order), and with adam = 1 an Adam step (lr, beta 0.9 / 0.999,
 * eps 1e-8) on the FP32 masters.  grad_host (may be NULL) receives the
 * gradient, loss (may be NULL) the loss before the step.  B <= batch_max. */
lx_status mlp_train_step(lx_mlp* m, const float* x_dev, const float* t_dev, int B, int adam, float lr,
                         float* grad_host, float* loss);

void mlp_destroy(lx_mlp* m);

/* ---------------------------------------------------------------------------
 * Allocation-free entry point.  The paper has no counterpart: it exists for
 * callers that cannot allocate device memory at the point of the call --
 * applications whose own memory pool owns the device (and plug-ins loaded
 * into them), and time-critical loops that cannot afford the implicit device
 * synchronisation of cudaMalloc/cudaFree.
 * ------------------------------------------------------------------------- */

#define LX_NOALLOC_MAX_POINTS 262144 /* largest nx * ny (512 x 512) */
#define LX_NOALLOC_MAX_LEJA 1000     /* Leja points / coefficients used at most */

/* phi_l(hA)w for LX_ADVDIFF with LX_FP64 -- the same fused Leja-iteration
 * kernel and stopping test as phi_l_apply -- without a context and without
 * allocating memory.  Its scratch (two basis vectors, reduction partials,
 * loop state, Leja points and coefficients; about 4.2 MB) is one fixed
 * __device__ array inside the library, resident on every GPU that loads the
 * library until the process exits.
 *   prob         problem (kind LX_ADVDIFF, precision LX_FP64), nx*ny <=
 *                LX_NOALLOC_MAX_POINTS; otherwise LX_E_INVAL with a message
 *                in lx_last_cuda_error()
 *   l, w_dev, out_dev, c, gamma, h, rtol, atol, iters: as in phi_l_apply
 *                (out_dev must not alias w_dev)
 *   cuda_stream  stream of the current device for all work (NULL: default);
 *                the call synchronises it before returning
 * Every call shares the scratch array and leaves its contents behind; each
 * call clears what must start at zero.  Calls whose GPU work overlaps (other
 * streams, other host threads) race on the array: serialise them.  The call
 * is driven from the host: it launches the fused iteration in batches of 8
 * and reads the loop state back, synchronising the stream, after each batch.
 * Set-up: the first call in the process computes the table of
 * LX_NOALLOC_MAX_LEJA Leja points on the host (its one host allocation),
 * and the first call on each device, with that device current, resolves the
 * array's device address (cudaGetSymbolAddress) and uploads the table with a
 * synchronous copy; make that first call before any stream capture starts.
 * Later calls allocate nothing.  The host side uses about 56 KB of stack. */
lx_status phi_l_apply_noalloc(const lx_problem* prob, int l, const double* w_dev, double* out_dev, double c,
                              double gamma, double h, double rtol, double atol, void* cuda_stream, int* iters);

/* ---------------------------------------------------------------------------
 * Unfused form: a caller's right-hand side and a finite-difference Jacobian
 * (Sec. 2: the user supplies f as a function of an input and an output
 * pointer to contiguous data, with its parameters held by a functor;
 * Sec. 2.3: the action of the Jacobian is taken by finite differences).
 *
 * The engine cannot fuse an arbitrary f into its stencil kernels, so every
 * Jacobian product costs two calls of f plus two passes of the engine's
 * own kernels (the perturbed states, then the Newton update with its
 * stopping norms).  Reading of the difference quotient (the paper gives no
 * formula): the central quotient
 *     J(u) v = [f(u + e v) - f(u - e v)] / (2 e),  e = eps0 (1 + ||u||) / ||v||,
 * second-order in e and exact up to rounding for f of degree <= 2; J(u) 0 = 0.
 * FP64 throughout.  Everything else (Leja points, coefficients, stopping
 * test, integrator stages in the order of Sec. 2.3 Listings 12-13) is as in
 * the fused entry points.
 * ------------------------------------------------------------------------- */

/* Right-hand side: out_dev = f(in_dev) for n doubles (device pointers, never
 * aliasing), enqueued on cuda_stream (the context's stream; the engine's
 * kernels that follow run on the same stream, so the function may return
 * before its work completes).  user: the pointer given at setup (the
 * functor's parameters).  Return 0 on success; any other value makes the
 * calling entry point stop and return LX_E_CALLBACK. */
typedef int (*lx_rhs_fn)(const double* in_dev, double* out_dev, void* user, void* cuda_stream);

/* The engine's own right-hand side of a problem, in lx_rhs_fn form: user is
 * a const lx_problem* (kinds LX_ADVDIFF .. LX_BURGERS_UP3; the precision
 * field is ignored, the arithmetic is FP64).  f is A u for the
 * diffusion-advection kinds and the Burgers right-hand side otherwise.
 * Returns 0, or 1 for an invalid problem or a failed launch. */
int lx_rhs_builtin(const double* in_dev, double* out_dev, void* user, void* cuda_stream);

typedef struct lx_rhs_ctx lx_rhs_ctx;

/* Context of the unfused form (the paper's struct Leja with its RHS
 * functor): the Leja point table, the basis and stage vectors (about 11 n
 * doubles for LX_EXPRB32, 8 n for LX_ROS_EU) and the reduction scratch.
 *   n           number of unknowns, 1 <= n <= 2^31
 *   f, user     the right-hand side (kept; called from the calling thread)
 *   eps0        relative difference step, > 0; 0 selects 2^-18 (about the
 *               cube root of the unit roundoff, which balances the O(e^2)
 *               truncation against the rounding of f amplified by 1/e)
 *   integrator, max_leja, cuda_stream, out: as in leja_setup
 * Errors: LX_E_INVAL, LX_E_NOMEM, LX_E_CUDA. */
lx_status leja_setup_rhs(long long n, lx_rhs_fn f, void* user, double eps0, int integrator, int max_leja,
                         void* cuda_stream, lx_rhs_ctx** out);

void leja_destroy_rhs(lx_rhs_ctx* ctx);

/* power_bound with J(u) by differences (u_dev NULL: u = 0, i.e. the
 * operator of a linear f).  Arguments and stopping rule as power_bound. */
lx_status power_bound_rhs(lx_rhs_ctx* ctx, const double* u_dev, const double* v0_dev, int max_iters,
                          double* rho, int* iters);

/* phi_l(h J(u)) w with J(u) by differences (u_dev NULL: u = 0).  Arguments,
 * stopping test and iteration count as phi_l_apply.  The loop is driven
 * from the host (f cannot run inside a device-ended graph loop); the host
 * reads the device's stop flag one iteration behind, so at most one
 * further pair of f calls runs after the stop, on unchanged buffers. */
lx_status phi_l_apply_rhs(lx_rhs_ctx* ctx, int l, const double* u_dev, const double* w_dev, double* out_dev,
                          double c, double gamma, double h, double rtol, double atol, int* iters);

/* One step of the context's integrator, as expint_step, with f from the
 * callback and J(u) by differences; EXPRB32 evaluates
 * R = h (F(a) - F(u)), F(k) = f(k) - J(u) k, as written (no simplification
 * for a particular f). */
lx_status expint_step_rhs(lx_rhs_ctx* ctx, const double* u_dev, double* u_low_dev, double* u_high_dev, double c,
                          double gamma, double h, double rtol, double atol, double* err, int* iters);

/* Counters of the context: Leja iterations, right-hand-side calls and
 * engine kernel launches since the last reset. */
typedef struct {
  long long leja_iterations;
  long long rhs_calls;
  long long kernels;
} lx_rhs_stats;
lx_status lx_rhs_ctx_stats(lx_rhs_ctx* ctx, lx_rhs_stats* out, int reset);

#ifdef __cplusplus
}
#endif

#endif /* LEXGB_H */
