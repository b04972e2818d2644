/*
 * CPU oracle for the Leja exponential-integrator hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  The product
 * (the CUDA library under paper_2310_08344_gb300/) never calls it, shares no
 * code, header, table or constant with it, and fails if its own extension is
 * missing.
 *
 * Plain, slow, obviously correct: loops in the order the paper states the
 * algorithm, fp64 for vectors, IEEE binary128 for the scalar
 * phi functions and the Newton divided differences.  Each function names the
 * passage of Deka, Moriggl, Einkemmer, "LeXInt: GPU-accelerated exponential
 * integrators package" (arXiv 2310.08344) that it follows.
 *
 * Readings where the paper is silent (stated again at each use):
 *  - Leja points on [-2,2]: xi_0 = +2; later near-ties (log-products within
 *    1e-12 relative) are broken toward the larger point.
 *  - The interpolated function is f(xi) = phi_l(h (c + gamma xi)); the Newton
 *    basis uses (A - c)/gamma - xi_m, which carries no h.
 *  - Error estimate e_m = |d_m| * ||y_m||, stop when e_m <= rtol ||p_m|| + atol,
 *    iters = m at the stop; ||x|| = ||x||_2 / sqrt(N).
 *  - Iteration cap: K - 1 iterations for a table of K points, then NOCONV.
 *  - Power iteration: w = Av, rho_k = ||w||/||v||, v <- w/||w||, stop at
 *    max_iters or when |rho_k - rho_{k-1}| <= 1e-2 rho_k.
 *  - The Jacobian action is the analytic linearisation of the stencil; the
 *    "_fd" entry points instead take it by finite differences of f (Sec. 2.3),
 *    read as the central quotient J(u)v = [f(u + e v) - f(u - e v)] / (2e)
 *    with e = eps0 (1 + ||u||) / ||v|| (J(u)0 = 0; a NULL u is u = 0), and
 *    f either the problem kind's own or a caller's function (Sec. 2: the
 *    right-hand side takes an input and an output pointer).
 */
/*
 * Threads: the parity build (oracle/_oracle.so) is single-threaded, so every
 * sum runs in index order.  The same source compiled with -fopenmp
 * (oracle/_oracle_omp.so) splits the grid loops and norms over the host's
 * cores; that build only times the CPU baseline of the benchmark.
 */
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#if LDBL_MANT_DIG == 113
typedef long double qreal; /* IEEE binary128 on aarch64 Linux */
#define QEXP expl
#define QFABS fabsl
#else
#include <quadmath.h>
typedef __float128 qreal; /* libquadmath on x86-64 */
#define QEXP expq
#define QFABS fabsq
#endif

enum { OR_OK = 0, OR_E_INVAL = 1, OR_E_NOMEM = 2, OR_E_NOCONV = 4, OR_E_NONFINITE = 5 };
enum { OR_ADVDIFF = 0, OR_BURGERS = 1, OR_ADVDIFF_UP3 = 2, OR_BURGERS_UP3 = 3 };

#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads the grid loops use (1 in the parity build). */
int or_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int or_qreal_mant_dig(void) {
#if LDBL_MANT_DIG == 113
  return LDBL_MANT_DIG;
#else
  return FLT128_MANT_DIG;
#endif
}

/* ------------------------------------------------------------------------ */
/* Leja points on [-2, 2]  (Sec. 2.1: the recursive Leja definition, with    */
/* |z_0| the maximum modulus on the set; points are precomputed on [-2,2]).  */
/* ------------------------------------------------------------------------ */

static int cmp_double(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return (x > y) - (x < y);
}

/* The maximiser of sum_k log|x - xi_k| inside the open interval (lo, hi)
 * between two consecutive nodes.  It is the unique root of the derivative
 * g(x) = sum_k 1/(x - xi_k), which falls from +inf to -inf on the interval.
 * Newton steps, replaced by bisection whenever they leave the bracket. */
static double interval_maximiser(const double* xi, int j, double lo, double hi) {
  double x = 0.5 * (lo + hi);
  for (int it = 0; it < 400; ++it) {
    double g = 0.0, gp = 0.0;
    for (int k = 0; k < j; ++k) {
      double r = 1.0 / (x - xi[k]);
      g += r;
      gp -= r * r;
    }
    if (g == 0.0) break; /* exact critical point */
    if (g > 0.0) lo = x; else hi = x;
    double xn = x - g / gp;
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    if (fabs(xn - x) <= 2.0 * DBL_EPSILON * fabs(x) || hi - lo <= 4.0 * DBL_EPSILON * fabs(x)) {
      x = xn;
      break;
    }
    x = xn;
  }
  return x;
}

static double log_product(const double* xi, int j, double x) {
  double s = 0.0;
  for (int k = 0; k < j; ++k) s += log(fabs(x - xi[k]));
  return s;
}

/* Greedy Leja sequence: xi_j maximises prod_{k<j} |x - xi_k| over [-2, 2].
 * xi_0 = +2 (both ends have maximal modulus; the sign is a reading).
 * xi_1 = -2 (|x - 2| is largest at the other end).  For j >= 2 both ends are
 * nodes, so the maximum lies inside one of the intervals between consecutive
 * nodes; every interval is searched.  Ties within 1e-12 (relative, in the
 * log-product) go to the larger point.  Returns 0 on success. */
int or_leja_points(int K, double* xi) {
  if (K <= 0 || !xi) return OR_E_INVAL;
  xi[0] = 2.0;
  if (K > 1) xi[1] = -2.0;
  if (K <= 2) return OR_OK;
  double* sorted = (double*)malloc(sizeof(double) * (size_t)K);
  double* cx = (double*)malloc(sizeof(double) * (size_t)K);
  double* cl = (double*)malloc(sizeof(double) * (size_t)K);
  if (!sorted || !cx || !cl) {
    free(sorted); free(cx); free(cl);
    return OR_E_NOMEM;
  }
  for (int j = 2; j < K; ++j) {
    memcpy(sorted, xi, sizeof(double) * (size_t)j);
    qsort(sorted, (size_t)j, sizeof(double), cmp_double);
    double best = -INFINITY;
    for (int q = 0; q + 1 < j; ++q) {
      cx[q] = interval_maximiser(xi, j, sorted[q], sorted[q + 1]);
      cl[q] = log_product(xi, j, cx[q]);
      if (cl[q] > best) best = cl[q];
    }
    double tie = 1e-12 * fmax(1.0, fabs(best));
    double pick = -INFINITY;
    for (int q = 0; q + 1 < j; ++q)
      if (cl[q] >= best - tie && cx[q] > pick) pick = cx[q];
    xi[j] = pick;
  }
  free(sorted); free(cx); free(cl);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* phi functions (Sec. 1): phi_0 = exp, phi_{l+1}(z) = (phi_l(z) - 1/l!)/z.  */
/* ------------------------------------------------------------------------ */

static qreal q_factorial(int n) {
  qreal f = 1;
  for (int k = 2; k <= n; ++k) f *= (qreal)k;
  return f;
}

/* phi_l(z) in binary128.  |z| < 1: the power series sum_k z^k/(k+l)!, which
 * is the recursion solved for small z.  Otherwise the recursion itself,
 * starting from exp(z). */
static qreal q_phi(int l, qreal z) {
  if (QFABS(z) < 1) {
    qreal term = 1 / q_factorial(l), sum = term;
    for (int k = 1; k < 400; ++k) {
      term *= z / (qreal)(k + l);
      sum += term;
      if (QFABS(term) <= (qreal)1e-40 * QFABS(sum)) break;
    }
    return sum;
  }
  qreal phi = QEXP(z);
  qreal inv_fact = 1; /* 1/k! */
  for (int k = 0; k < l; ++k) {
    phi = (phi - inv_fact) / z;
    inv_fact /= (qreal)(k + 1);
  }
  return phi;
}

double or_phi(int l, double z) { return (double)q_phi(l, (qreal)z); }

/* ------------------------------------------------------------------------ */
/* Newton divided differences (Sec. 2.1, Eq. 2: the coefficients d_m of the  */
/* Newton form at the Leja points).  Row-wise recursion in binary128:        */
/* d_j <- f_j, then d_j <- (d_j - d_k)/(x_j - x_k) for k = 0..j-1.           */
/* ------------------------------------------------------------------------ */

static void q_divdiff(int n, const qreal* x, qreal* d) {
  for (int j = 1; j < n; ++j)
    for (int k = 0; k < j; ++k) d[j] = (d[j] - d[k]) / (x[j] - x[k]);
}

/* Divided differences of given values f at nodes x (both double). */
int or_divdiff_values(int n, const double* x, const double* f, double* d) {
  if (n <= 0) return OR_E_INVAL;
  qreal* qx = (qreal*)malloc(sizeof(qreal) * (size_t)n);
  qreal* qd = (qreal*)malloc(sizeof(qreal) * (size_t)n);
  if (!qx || !qd) { free(qx); free(qd); return OR_E_NOMEM; }
  for (int j = 0; j < n; ++j) { qx[j] = x[j]; qd[j] = f[j]; }
  q_divdiff(n, qx, qd);
  for (int j = 0; j < n; ++j) d[j] = (double)qd[j];
  free(qx); free(qd);
  return OR_OK;
}

/* d_j = f[xi_0, ..., xi_j] for f(xi) = phi_l(h (c + gamma xi))  (Eq. 2 with
 * exp replaced by phi_l; the interpolation variable is xi in [-2, 2]). */
int or_leja_coeffs(int l, double h, double c, double gamma, const double* xi, int K, double* d) {
  if (K <= 0 || l < 0) return OR_E_INVAL;
  qreal* qx = (qreal*)malloc(sizeof(qreal) * (size_t)K);
  qreal* qd = (qreal*)malloc(sizeof(qreal) * (size_t)K);
  if (!qx || !qd) { free(qx); free(qd); return OR_E_NOMEM; }
  for (int j = 0; j < K; ++j) {
    qx[j] = xi[j];
    qd[j] = q_phi(l, (qreal)h * ((qreal)c + (qreal)gamma * qx[j]));
  }
  q_divdiff(K, qx, qd);
  for (int j = 0; j < K; ++j) d[j] = (double)qd[j];
  free(qx); free(qd);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Operators on the periodic grid x_i = i/nx, y_j = j/ny, index j*nx + i.    */
/* Second-order central differences for both the Laplacian and the gradient. */
/* ------------------------------------------------------------------------ */

static long idx(int nx, int i, int j) { return (long)j * nx + i; }
static int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

/* A v = nu (v_xx + v_yy) + a (v_x + v_y)   (the linear diffusion-advection
 * operator of Sec. 3, Problem I, with this build's coefficients). */
void or_apply_advdiff(int nx, int ny, double nu, double a, const double* v, double* out) {
  double dx = 1.0 / nx, dy = 1.0 / ny;
#pragma omp parallel for
  for (int j = 0; j < ny; ++j) {
    int jn = wrap(j + 1, ny), js = wrap(j - 1, ny);
    for (int i = 0; i < nx; ++i) {
      int ie = wrap(i + 1, nx), iw = wrap(i - 1, nx);
      double vc = v[idx(nx, i, j)];
      double ve = v[idx(nx, ie, j)], vw = v[idx(nx, iw, j)];
      double vn = v[idx(nx, i, jn)], vs = v[idx(nx, i, js)];
      double lap = (ve - 2.0 * vc + vw) / (dx * dx) + (vn - 2.0 * vc + vs) / (dy * dy);
      double grad = (ve - vw) / (2.0 * dx) + (vn - vs) / (2.0 * dy);
      out[idx(nx, i, j)] = nu * lap + a * grad;
    }
  }
}

/* D v = v_x + v_y by central differences. */
static void central_sum_grad(int nx, int ny, const double* v, double* out) {
  double dx = 1.0 / nx, dy = 1.0 / ny;
  for (int j = 0; j < ny; ++j) {
    int jn = wrap(j + 1, ny), js = wrap(j - 1, ny);
    for (int i = 0; i < nx; ++i) {
      int ie = wrap(i + 1, nx), iw = wrap(i - 1, nx);
      out[idx(nx, i, j)] = (v[idx(nx, ie, j)] - v[idx(nx, iw, j)]) / (2.0 * dx) +
                           (v[idx(nx, i, jn)] - v[idx(nx, i, js)]) / (2.0 * dy);
    }
  }
}

/* f(u) = nu (u_xx + u_yy) - u (u_x + u_y)   (viscous Burgers). */
void or_burgers_f(int nx, int ny, double nu, const double* u, double* out) {
  long n = (long)nx * ny;
  double* du = (double*)malloc(sizeof(double) * (size_t)n);
  or_apply_advdiff(nx, ny, nu, 0.0, u, out);
  central_sum_grad(nx, ny, u, du);
  for (long k = 0; k < n; ++k) out[k] = out[k] - u[k] * du[k];
  free(du);
}

/* J(u) v = nu (v_xx + v_yy) - v (u_x + u_y) - u (v_x + v_y): the exact
 * derivative of or_burgers_f at u applied to v (the paper uses finite
 * differences for this action, Sec. 2.3; the analytic form is the reading). */
void or_burgers_J(int nx, int ny, double nu, const double* u, const double* v, double* out) {
  long n = (long)nx * ny;
  double* du = (double*)malloc(sizeof(double) * (size_t)n);
  double* dv = (double*)malloc(sizeof(double) * (size_t)n);
  or_apply_advdiff(nx, ny, nu, 0.0, v, out);
  central_sum_grad(nx, ny, u, du);
  central_sum_grad(nx, ny, v, dv);
  for (long k = 0; k < n; ++k) out[k] = out[k] - v[k] * du[k] - u[k] * dv[k];
  free(du);
  free(dv);
}

/* ------------------------------------------------------------------------ */
/* The paper's own discretisation (Sec. 3): periodic [-1,1]^2 (spacing       */
/* 2/nx, 2/ny), the Laplacian by second-order central differences and the    */
/* gradient by the third-order upwind-biased scheme.  For a term +a v_x with */
/* a > 0 the characteristics run toward -x, so the upwind side is +x:        */
/*   (D v)_i = (-v_{i+2} + 6 v_{i+1} - 3 v_i - 2 v_{i-1}) / (6 dx);          */
/* for a < 0 the mirror image (2 v_{i+1} + 3 v_i - 6 v_{i-1} + v_{i-2})/(6dx).*/
/* ------------------------------------------------------------------------ */

/* Periodic index for any offset. */
static int wrapm(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

/* out = (D_x + D_y) v with the upwind side given by the sign s (+1 / -1). */
static void up3_sum_grad(int nx, int ny, int s, const double* v, double* out) {
  double dx = 2.0 / nx, dy = 2.0 / ny;
  for (int j = 0; j < ny; ++j) {
    for (int i = 0; i < nx; ++i) {
      double gx, gy;
      const double* row = v + (long)j * nx;
      if (s > 0) {
        gx = (-row[wrapm(i + 2, nx)] + 6.0 * row[wrapm(i + 1, nx)] - 3.0 * row[i] - 2.0 * row[wrapm(i - 1, nx)]) /
             (6.0 * dx);
        gy = (-v[idx(nx, i, wrapm(j + 2, ny))] + 6.0 * v[idx(nx, i, wrapm(j + 1, ny))] - 3.0 * row[i] -
              2.0 * v[idx(nx, i, wrapm(j - 1, ny))]) / (6.0 * dy);
      } else {
        gx = (2.0 * row[wrapm(i + 1, nx)] + 3.0 * row[i] - 6.0 * row[wrapm(i - 1, nx)] + row[wrapm(i - 2, nx)]) /
             (6.0 * dx);
        gy = (2.0 * v[idx(nx, i, wrapm(j + 1, ny))] + 3.0 * row[i] - 6.0 * v[idx(nx, i, wrapm(j - 1, ny))] +
              v[idx(nx, i, wrapm(j - 2, ny))]) / (6.0 * dy);
      }
      out[idx(nx, i, j)] = gx + gy;
    }
  }
}

/* out = nu (v_xx + v_yy) by central differences on [-1,1]^2. */
static void lap_pm1(int nx, int ny, double nu, const double* v, double* out) {
  double dx = 2.0 / nx, dy = 2.0 / ny;
  for (int j = 0; j < ny; ++j) {
    int jn = wrap(j + 1, ny), js = wrap(j - 1, ny);
    for (int i = 0; i < nx; ++i) {
      int ie = wrap(i + 1, nx), iw = wrap(i - 1, nx);
      double vc = v[idx(nx, i, j)];
      out[idx(nx, i, j)] = nu * ((v[idx(nx, ie, j)] - 2.0 * vc + v[idx(nx, iw, j)]) / (dx * dx) +
                                 (v[idx(nx, i, jn)] - 2.0 * vc + v[idx(nx, i, js)]) / (dy * dy));
    }
  }
}

/* A v = nu (v_xx + v_yy) + a (v_x + v_y), upwind gradient (Problem I, Sec. 3, Eq. 3,
 * with nu the diffusion and a the advection coefficient). */
void or_apply_advdiff_up3(int nx, int ny, double nu, double a, const double* v, double* out) {
  long n = (long)nx * ny;
  double* g = (double*)malloc(sizeof(double) * (size_t)n);
  lap_pm1(nx, ny, nu, v, out);
  if (a != 0.0) {
    up3_sum_grad(nx, ny, a > 0.0 ? 1 : -1, v, g);
    for (long k = 0; k < n; ++k) out[k] = out[k] + a * g[k];
  }
  free(g);
}

/* f(u) = nu (u_xx + u_yy) + (a/2) ((u^2)_x + (u^2)_y)   (Problem III, Sec. 3, Eq. 5,
 * the flux form; the upwind side follows the sign of a, i.e. the reading
 * takes u > 0 as in the paper's initial state). */
void or_burgers_up3_f(int nx, int ny, double nu, double a, const double* u, double* out) {
  long n = (long)nx * ny;
  double* u2 = (double*)malloc(sizeof(double) * (size_t)n);
  double* g = (double*)malloc(sizeof(double) * (size_t)n);
  lap_pm1(nx, ny, nu, u, out);
  for (long k = 0; k < n; ++k) u2[k] = u[k] * u[k];
  up3_sum_grad(nx, ny, a >= 0.0 ? 1 : -1, u2, g);
  for (long k = 0; k < n; ++k) out[k] = out[k] + 0.5 * a * g[k];
  free(u2);
  free(g);
}

/* J(u) v = nu (v_xx + v_yy) + a ((u v)_x + (u v)_y): the exact derivative of
 * or_burgers_up3_f (the difference operator is linear). */
void or_burgers_up3_J(int nx, int ny, double nu, double a, const double* u, const double* v, double* out) {
  long n = (long)nx * ny;
  double* uv = (double*)malloc(sizeof(double) * (size_t)n);
  double* g = (double*)malloc(sizeof(double) * (size_t)n);
  lap_pm1(nx, ny, nu, v, out);
  for (long k = 0; k < n; ++k) uv[k] = u[k] * v[k];
  up3_sum_grad(nx, ny, a >= 0.0 ? 1 : -1, uv, g);
  for (long k = 0; k < n; ++k) out[k] = out[k] + a * g[k];
  free(uv);
  free(g);
}

/* The operator the Leja basis multiplies by: A for diffusion-advection,
 * J(u) for Burgers.  S (may be NULL): a time-independent source added to
 * the right-hand side (Problem II of Sec. 3, Eq. 4); it does not enter J. */
typedef void (*or_rhs_fn)(const double* in, double* out, void* user);

typedef struct {
  int kind, nx, ny;
  double nu, a;
  const double* u;
  const double* S;
  or_rhs_fn f;   /* caller's right-hand side, or NULL for the kind's own */
  void* user;    /* passed to f */
  double eps0;   /* > 0: Jacobian action by central finite differences */
  int regroup;   /* 1: the diffusion-advection operator with its terms grouped
                    per neighbour (same operator, other rounding) */
} or_op;

static void op_rhs(const or_op* op, const double* u, double* out);
static double nrm(const double* x, long n);

/* J(u) v by the central difference quotient of f (Sec. 2.3: the action of
 * the Jacobian is taken numerically), e = eps0 (1 + ||u||) / ||v||. */
static void op_apply_fd(const or_op* op, const double* v, double* out) {
  long n = (long)op->nx * op->ny;
  double vn = nrm(v, n);
  if (vn == 0.0) {
    for (long q = 0; q < n; ++q) out[q] = 0.0;
    return;
  }
  double un = op->u ? nrm(op->u, n) : 0.0;
  double e = op->eps0 * (1.0 + un) / vn;
  double* x = (double*)malloc(sizeof(double) * (size_t)n);
  double* fp = (double*)malloc(sizeof(double) * (size_t)n);
  if (!x || !fp) {
    free(x);
    free(fp);
    for (long q = 0; q < n; ++q) out[q] = NAN;
    return;
  }
  for (long q = 0; q < n; ++q) x[q] = (op->u ? op->u[q] : 0.0) + e * v[q];
  op_rhs(op, x, fp);
  for (long q = 0; q < n; ++q) x[q] = (op->u ? op->u[q] : 0.0) - e * v[q];
  op_rhs(op, x, out);
  for (long q = 0; q < n; ++q) out[q] = (fp[q] - out[q]) / (2.0 * e);
  free(x);
  free(fp);
}

/* A v for the diffusion-advection operator with one weight per neighbour,
 *   (A v)_ij = wE v_E + wW v_W + wN v_N + wS v_S + wC v_ij,
 *   wE = nu/dx^2 + a/(2dx), wW = nu/dx^2 - a/(2dx), wC = -2nu/dx^2 - 2nu/dy^2
 * (wN, wS likewise in y): the same operator as or_apply_advdiff in another
 * evaluation order.  The difference of a Leja run in the two orders shows
 * how strongly a problem amplifies rounding (the Newton basis grows where
 * the spectrum reaches far off the real focal interval). */
static void apply_advdiff_per_neighbour(int nx, int ny, double nu, double a, const double* v, double* out) {
  double dx = 1.0 / nx, dy = 1.0 / ny;
  double wE = nu / (dx * dx) + a / (2.0 * dx), wW = nu / (dx * dx) - a / (2.0 * dx);
  double wN = nu / (dy * dy) + a / (2.0 * dy), wS = nu / (dy * dy) - a / (2.0 * dy);
  double wC = -2.0 * nu / (dx * dx) - 2.0 * nu / (dy * dy);
#pragma omp parallel for
  for (int j = 0; j < ny; ++j) {
    int jn = wrap(j + 1, ny), js = wrap(j - 1, ny);
    for (int i = 0; i < nx; ++i) {
      int ie = wrap(i + 1, nx), iw = wrap(i - 1, nx);
      out[idx(nx, i, j)] = wE * v[idx(nx, ie, j)] + wW * v[idx(nx, iw, j)] + wN * v[idx(nx, i, jn)] +
                           wS * v[idx(nx, i, js)] + wC * v[idx(nx, i, j)];
    }
  }
}

static void op_apply(const or_op* op, const double* v, double* out) {
  if (op->regroup && op->kind == OR_ADVDIFF)
    apply_advdiff_per_neighbour(op->nx, op->ny, op->nu, op->a, v, out);
  else if (op->eps0 > 0.0)
    op_apply_fd(op, v, out);
  else if (op->kind == OR_BURGERS)
    or_burgers_J(op->nx, op->ny, op->nu, op->u, v, out);
  else if (op->kind == OR_ADVDIFF_UP3)
    or_apply_advdiff_up3(op->nx, op->ny, op->nu, op->a, v, out);
  else if (op->kind == OR_BURGERS_UP3)
    or_burgers_up3_J(op->nx, op->ny, op->nu, op->a, op->u, v, out);
  else
    or_apply_advdiff(op->nx, op->ny, op->nu, op->a, v, out);
}

/* f(u): A u for diffusion-advection, the Burgers right-hand side otherwise,
 * plus the source S when there is one. */
static void op_rhs(const or_op* op, const double* u, double* out) {
  if (op->f)
    op->f(u, out, op->user);
  else if (op->kind == OR_BURGERS)
    or_burgers_f(op->nx, op->ny, op->nu, u, out);
  else if (op->kind == OR_ADVDIFF_UP3)
    or_apply_advdiff_up3(op->nx, op->ny, op->nu, op->a, u, out);
  else if (op->kind == OR_BURGERS_UP3)
    or_burgers_up3_f(op->nx, op->ny, op->nu, op->a, u, out);
  else
    or_apply_advdiff(op->nx, op->ny, op->nu, op->a, u, out);
  if (op->S) {
    long n = (long)op->nx * op->ny;
    for (long q = 0; q < n; ++q) out[q] = out[q] + op->S[q];
  }
}

/* ||x|| = ||x||_2 / sqrt(N) (Sec. 2.2: the l2 norm scaled by 1/sqrt(N)). */
static double nrm(const double* x, long n) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s)
  for (long k = 0; k < n; ++k) s += x[k] * x[k];
  return sqrt(s / (double)n);
}

/* ------------------------------------------------------------------------ */
/* Power iteration for the dominant eigenvalue modulus (Sec. 2, Listing 7).  */
/* ------------------------------------------------------------------------ */

static int power_core(const or_op* opp, const double* v0, int max_iters, double* rho_out, int* iters_out) {
  const or_op op = *opp;
  long n = (long)op.nx * op.ny;
  double* v = (double*)malloc(sizeof(double) * (size_t)n);
  double* w = (double*)malloc(sizeof(double) * (size_t)n);
  if (!v || !w) { free(v); free(w); return OR_E_NOMEM; }
  memcpy(v, v0, sizeof(double) * (size_t)n);
  double rho = 0.0, rho_prev = 0.0;
  int k;
  for (k = 1; k <= max_iters; ++k) {
    op_apply(&op, v, w);
    double nw = nrm(w, n), nv = nrm(v, n);
    rho = nw / nv;
#pragma omp parallel for
    for (long q = 0; q < n; ++q) v[q] = w[q] / nw;
    if (k > 1 && fabs(rho - rho_prev) <= 1e-2 * rho) break;
    rho_prev = rho;
  }
  if (k > max_iters) k = max_iters;
  *rho_out = rho;
  if (iters_out) *iters_out = k;
  free(v);
  free(w);
  return isfinite(rho) ? OR_OK : OR_E_NONFINITE;
}

int or_power_iteration(int kind, int nx, int ny, double nu, double a, const double* u,
                       const double* v0, int max_iters, double* rho_out, int* iters_out) {
  if (nx <= 0 || ny <= 0 || max_iters <= 0) return OR_E_INVAL;
  or_op op = {kind, nx, ny, nu, a, u};
  return power_core(&op, v0, max_iters, rho_out, iters_out);
}

/* ------------------------------------------------------------------------ */
/* Leja interpolation of phi_l(h Op) w  (Sec. 2.1 Eq. 2; Sec. 2.2 and 2.3,   */
/* the real_Leja_exp / real_Leja_phi_nl / real_Leja_phi interfaces).         */
/*   y_0 = w, p_0 = d_0 w;                                                   */
/*   y_{m+1} = ((Op - c)/gamma - xi_m) y_m,  p_{m+1} = p_m + d_{m+1} y_{m+1}; */
/*   stop when |d_{m+1}| ||y_{m+1}|| <= rtol ||p_{m+1}|| + atol.             */
/* ------------------------------------------------------------------------ */

/* The loop itself, for Newton coefficients d[0..K) already formed.
 * growth (may be NULL): receives max_m ||y_m|| / ||y_0||, the growth of the
 * Newton basis, which sets how far rounding in the recursion is amplified. */
static int leja_loop_core(const or_op* op, const double* w, double c, double gamma, double rtol, double atol,
                          const double* xi, const double* d, int K, double* out, int* iters, double* growth) {
  long n = (long)op->nx * op->ny;
  if (K < 2) return OR_E_INVAL;
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  double* t = (double*)malloc(sizeof(double) * (size_t)n);
  if (!y || !t) { free(y); free(t); return OR_E_NOMEM; }
#pragma omp parallel for
  for (long q = 0; q < n; ++q) {
    y[q] = w[q];
    out[q] = d[0] * w[q];
  }
  int status = OR_E_NOCONV;
  *iters = K - 1;
  const double y0n = nrm(w, n);
  double ymax = y0n;
  for (int m = 0; m + 1 < K; ++m) {
    op_apply(op, y, t);
#pragma omp parallel for
    for (long q = 0; q < n; ++q) y[q] = (t[q] - c * y[q]) / gamma - xi[m] * y[q];
#pragma omp parallel for
    for (long q = 0; q < n; ++q) out[q] = out[q] + d[m + 1] * y[q];
    const double yn = nrm(y, n);
    if (yn > ymax) ymax = yn;
    double e = fabs(d[m + 1]) * yn;
    double pn = nrm(out, n);
    if (!isfinite(e) || !isfinite(pn)) {
      *iters = m + 1;
      status = OR_E_NONFINITE;
      break;
    }
    if (e <= rtol * pn + atol) {
      *iters = m + 1;
      status = OR_OK;
      break;
    }
  }
  if (growth) *growth = y0n > 0.0 ? ymax / y0n : 1.0;
  free(y);
  free(t);
  return status;
}

static int leja_phi_core(const or_op* op, int l, const double* w, double c, double gamma,
                         double h, double rtol, double atol, const double* xi, int K,
                         double* out, int* iters) {
  if (K < 2) return OR_E_INVAL;
  double* d = (double*)malloc(sizeof(double) * (size_t)K);
  if (!d) return OR_E_NOMEM;
  or_leja_coeffs(l, h, c, gamma, xi, K, d);
  int st = leja_loop_core(op, w, c, gamma, rtol, atol, xi, d, K, out, iters, NULL);
  free(d);
  return st;
}

int or_leja_phi(int kind, int nx, int ny, double nu, double a, const double* u, int l,
                const double* w, double c, double gamma, double h, double rtol, double atol,
                const double* xi, int K, double* out, int* iters) {
  if (nx <= 0 || ny <= 0 || l < 0 || gamma == 0.0) return OR_E_INVAL;
  or_op op = {kind, nx, ny, nu, a, u};
  return leja_phi_core(&op, l, w, c, gamma, h, rtol, atol, xi, K, out, iters);
}

/* The same loop with caller-supplied coefficients d[0..K) of
 * f(xi) = phi_l(h (c + gamma xi)) at the points xi, e.g. divided differences
 * formed by the same recursion at a precision above binary128, for the
 * regime where binary128 reaches its rounding floor before the series
 * converges.  Stops with OR_E_NOCONV after K - 1 iterations; growth (may be
 * NULL) receives max_m ||y_m|| / ||y_0||; regroup = 1 evaluates the
 * diffusion-advection operator per neighbour (apply_advdiff_per_neighbour). */
int or_leja_phi_given(int kind, int nx, int ny, double nu, double a, const double* u, const double* w,
                      double c, double gamma, double rtol, double atol, const double* xi, const double* d, int K,
                      double* out, int* iters, double* growth, int regroup) {
  if (nx <= 0 || ny <= 0 || gamma == 0.0 || !d) return OR_E_INVAL;
  or_op op = {kind, nx, ny, nu, a, u};
  op.regroup = regroup;
  return leja_loop_core(&op, w, c, gamma, rtol, atol, xi, d, K, out, iters, growth);
}

/* ------------------------------------------------------------------------ */
/* "Vertical" interpolation (Sec. 2.3, real_Leja_phi with several integrator */
/* coefficients): phi_l(alpha_j h Op) w for nc step fractions alpha_j from   */
/* one Newton basis.  The nodes, the shift c and the scale gamma are shared, */
/* so y_m is the same for every j; only the divided differences differ:      */
/*   d^(j)_k = f_j[xi_0..xi_k],  f_j(xi) = phi_l(alpha_j h (c + gamma xi)),  */
/*   p^(j)_{m+1} = p^(j)_m + d^(j)_{m+1} y_{m+1}.                            */
/* The paper does not state the stop rule; the reading is that the loop     */
/* stops at the first m at which every polynomial passes its own test        */
/* |d^(j)_{m+1}| ||y_{m+1}|| <= rtol ||p^(j)_{m+1}|| + atol.                 */
/* out: nc vectors of n values, polynomial j at out + j n.                   */
/* ------------------------------------------------------------------------ */

int or_leja_phi_vertical(int kind, int nx, int ny, double nu, double a, const double* u, int l, int nc,
                         const double* alpha, const double* w, double c, double gamma, double h,
                         double rtol, double atol, const double* xi, int K, double* out, int* iters) {
  if (nx <= 0 || ny <= 0 || l < 0 || gamma == 0.0 || nc < 1 || K < 2) return OR_E_INVAL;
  or_op op = {kind, nx, ny, nu, a, u};
  long n = (long)nx * ny;
  double* d = (double*)malloc(sizeof(double) * (size_t)K * (size_t)nc);
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  double* t = (double*)malloc(sizeof(double) * (size_t)n);
  if (!d || !y || !t) { free(d); free(y); free(t); return OR_E_NOMEM; }
  for (int j = 0; j < nc; ++j) or_leja_coeffs(l, alpha[j] * h, c, gamma, xi, K, d + (size_t)j * K);
  for (long q = 0; q < n; ++q) y[q] = w[q];
  for (int j = 0; j < nc; ++j)
    for (long q = 0; q < n; ++q) out[(size_t)j * n + q] = d[(size_t)j * K] * w[q];
  int status = OR_E_NOCONV;
  *iters = K - 1;
  for (int m = 0; m + 1 < K; ++m) {
    op_apply(&op, y, t);
    for (long q = 0; q < n; ++q) y[q] = (t[q] - c * y[q]) / gamma - xi[m] * y[q];
    double yn = nrm(y, n);
    int all_pass = 1, finite = isfinite(yn);
    for (int j = 0; j < nc; ++j) {
      double* p = out + (size_t)j * n;
      double dj = d[(size_t)j * K + m + 1];
      for (long q = 0; q < n; ++q) p[q] = p[q] + dj * y[q];
      double e = fabs(dj) * yn;
      double pn = nrm(p, n);
      if (!isfinite(e) || !isfinite(pn)) finite = 0;
      if (!(e <= rtol * pn + atol)) all_pass = 0;
    }
    if (!finite) {
      *iters = m + 1;
      status = OR_E_NONFINITE;
      break;
    }
    if (all_pass) {
      *iters = m + 1;
      status = OR_OK;
      break;
    }
  }
  free(d);
  free(y);
  free(t);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Exponential Rosenbrock-Euler (Sec. 2.3, Listing 12):                      */
/*   u+ = u + phi_1(h J(u)) h f(u).                                          */
/* ------------------------------------------------------------------------ */

/* With a source (Problem II, Sec. 3, Eq. 4): f(u) = A u + S, so the step is
 * u+ = u + phi_1(h A) h (A u + S). */
static int ros_eu_core(const or_op* opp, const double* u, double c, double gamma, double h, double rtol,
                       double atol, const double* xi, int K, double* u_out, int* iters) {
  const or_op op = *opp;
  long n = (long)op.nx * op.ny;
  double* f_u = (double*)malloc(sizeof(double) * (size_t)n);
  double* p = (double*)malloc(sizeof(double) * (size_t)n);
  if (!f_u || !p) { free(f_u); free(p); return OR_E_NOMEM; }
  op_rhs(&op, u, f_u);
#pragma omp parallel for
  for (long q = 0; q < n; ++q) f_u[q] = h * f_u[q];
  int st = leja_phi_core(&op, 1, f_u, c, gamma, h, rtol, atol, xi, K, p, iters);
#pragma omp parallel for
  for (long q = 0; q < n; ++q) u_out[q] = u[q] + p[q];
  free(f_u);
  free(p);
  return st;
}

int or_ros_eu_src(int kind, int nx, int ny, double nu, double a, const double* u, const double* S,
                  double c, double gamma, double h, double rtol, double atol, const double* xi, int K,
                  double* u_out, int* iters) {
  if (nx <= 0 || ny <= 0) return OR_E_INVAL;
  or_op op = {kind, nx, ny, nu, a, u, S};
  return ros_eu_core(&op, u, c, gamma, h, rtol, atol, xi, K, u_out, iters);
}

int or_ros_eu(int kind, int nx, int ny, double nu, double a, const double* u, double c,
              double gamma, double h, double rtol, double atol, const double* xi, int K,
              double* u_out, int* iters) {
  return or_ros_eu_src(kind, nx, ny, nu, a, u, NULL, c, gamma, h, rtol, atol, xi, K, u_out, iters);
}

/* ------------------------------------------------------------------------ */
/* EXPRB32 (Sec. 2.3, Listing 13), in the listing's stage order:             */
/*   a   = u + phi_1(h J(u)) h f(u)                       (lower order)      */
/*   R   = h (F(a) - F(u)),  F(k) = f(k) - J(u) k                            */
/*   u3  = a + 2 phi_3(h J(u)) R                          (higher order)     */
/*   err = ||2 phi_3(h J(u)) R||                                             */
/* ------------------------------------------------------------------------ */

static int exprb32_core(const or_op* opp, const double* u, double c, double gamma, double h, double rtol,
                        double atol, const double* xi, int K, double* u_low, double* u_high, double* err,
                        int* iters) {
  const or_op op = *opp;
  long n = (long)op.nx * op.ny;
  double* f_u = (double*)malloc(sizeof(double) * (size_t)n);
  double* p1 = (double*)malloc(sizeof(double) * (size_t)n);
  double* t1 = (double*)malloc(sizeof(double) * (size_t)n);
  double* t2 = (double*)malloc(sizeof(double) * (size_t)n);
  double* nl_u = (double*)malloc(sizeof(double) * (size_t)n);
  double* nl_a = (double*)malloc(sizeof(double) * (size_t)n);
  double* p3 = (double*)malloc(sizeof(double) * (size_t)n);
  if (!f_u || !p1 || !t1 || !t2 || !nl_u || !nl_a || !p3) {
    free(f_u); free(p1); free(t1); free(t2); free(nl_u); free(nl_a); free(p3);
    return OR_E_NOMEM;
  }
  int it1 = 0, it2 = 0;
  op_rhs(&op, u, f_u);
  for (long q = 0; q < n; ++q) f_u[q] = h * f_u[q];
  int st = leja_phi_core(&op, 1, f_u, c, gamma, h, rtol, atol, xi, K, p1, &it1);
  for (long q = 0; q < n; ++q) u_low[q] = u[q] + p1[q];
  /* F(u) = f(u) - J(u) u */
  op_rhs(&op, u, t1);
  op_apply(&op, u, t2);
  for (long q = 0; q < n; ++q) nl_u[q] = t1[q] - t2[q];
  /* F(a) = f(a) - J(u) a */
  op_rhs(&op, u_low, t1);
  op_apply(&op, u_low, t2);
  for (long q = 0; q < n; ++q) nl_a[q] = t1[q] - t2[q];
  /* R = h (F(a) - F(u)) */
  for (long q = 0; q < n; ++q) t1[q] = h * nl_a[q] - h * nl_u[q];
  int st2 = OR_OK;
  if (st == OR_OK) st2 = leja_phi_core(&op, 3, t1, c, gamma, h, rtol, atol, xi, K, p3, &it2);
  else memset(p3, 0, sizeof(double) * (size_t)n);
  for (long q = 0; q < n; ++q) {
    p3[q] = 2.0 * p3[q];
    u_high[q] = u_low[q] + p3[q];
  }
  *err = nrm(p3, n);
  *iters = it1 + it2;
  free(f_u); free(p1); free(t1); free(t2); free(nl_u); free(nl_a); free(p3);
  return st != OR_OK ? st : st2;
}

int or_exprb32_src(int kind, int nx, int ny, double nu, double a, const double* u, const double* S,
                   double c, double gamma, double h, double rtol, double atol, const double* xi, int K,
                   double* u_low, double* u_high, double* err, int* iters) {
  if (nx <= 0 || ny <= 0) return OR_E_INVAL;
  or_op op = {kind, nx, ny, nu, a, u, S};
  return exprb32_core(&op, u, c, gamma, h, rtol, atol, xi, K, u_low, u_high, err, iters);
}

int or_exprb32(int kind, int nx, int ny, double nu, double a, const double* u, double c,
               double gamma, double h, double rtol, double atol, const double* xi, int K,
               double* u_low, double* u_high, double* err, int* iters) {
  return or_exprb32_src(kind, nx, ny, nu, a, u, NULL, c, gamma, h, rtol, atol, xi, K, u_low, u_high, err,
                        iters);
}

/* ------------------------------------------------------------------------ */
/* EPIRK4s3A (a fourth-order exponential integrator of the paper's Table 2;  */
/* Sec. 2.3: the phi_1 stages by "vertical" interpolation).  The paper names */
/* the scheme without its coefficients; they are the ones the stiff order    */
/* conditions of exponential Rosenbrock methods fix for the stage nodes      */
/* c2 = 1/2, c3 = 2/3 (Hochbruck, Ostermann, Schweitzer 2009):               */
/*   U_i = u + phi_1(c_i h J) c_i h f(u),   R_i = h (F(U_i) - F(u)),         */
/*   u4  = u + phi_1(h J) h f(u) + phi_3(h J) W3 + phi_4(h J) W4,            */
/* with W3 = b2 R_2 + b3 R_3, W4 = e2 R_2 + e3 R_3 solving                   */
/*   b2 c2^2 + b3 c3^2 = 2, b2 c2^3 + b3 c3^3 = 0   (sum b_i(z) c_i^2 = 2 phi_3) */
/*   e2 c2^2 + e3 c3^2 = 0, e2 c2^3 + e3 c3^3 = 6   (sum b_i(z) c_i^3 = 6 phi_4) */
/* i.e. (b2, b3) = (32, -27/2), (e2, e3) = (-144, 81).  The embedded         */
/* third-order solution drops the phi_4 term (it meets the first condition  */
/* only): u3 = u4 - phi_4(h J) W4, err = ||phi_4(h J) W4||.  The three phi_1 */
/* stages come from one vertical loop (alpha = 1/2, 2/3, 1).                 */
/* ------------------------------------------------------------------------ */

static int epirk4s3a_core(const or_op* opp, const double* u, double c, double gamma, double h, double rtol,
                          double atol, const double* xi, int K, double* u_low, double* u_high, double* err,
                          int* iters) {
  const or_op op = *opp;
  long n = (long)op.nx * op.ny;
  const double c2 = 0.5, c3 = 2.0 / 3.0;
  /* the 2x2 systems above, solved by Cramer's rule */
  const double det = c2 * c2 * c3 * c3 * c3 - c3 * c3 * c2 * c2 * c2;
  const double b2 = (2.0 * c3 * c3 * c3) / det, b3 = (-2.0 * c2 * c2 * c2) / det;
  const double e2 = (-6.0 * c3 * c3) / det, e3 = (6.0 * c2 * c2) / det;
  double* f_u = (double*)malloc(sizeof(double) * (size_t)n);
  double* P = (double*)malloc(sizeof(double) * (size_t)n * 3);
  double* U = (double*)malloc(sizeof(double) * (size_t)n);
  double* t1 = (double*)malloc(sizeof(double) * (size_t)n);
  double* t2 = (double*)malloc(sizeof(double) * (size_t)n);
  double* nl_u = (double*)malloc(sizeof(double) * (size_t)n);
  double* R2 = (double*)malloc(sizeof(double) * (size_t)n);
  double* R3 = (double*)malloc(sizeof(double) * (size_t)n);
  double* q3 = (double*)malloc(sizeof(double) * (size_t)n);
  double* q4 = (double*)malloc(sizeof(double) * (size_t)n);
  if (!f_u || !P || !U || !t1 || !t2 || !nl_u || !R2 || !R3 || !q3 || !q4) {
    free(f_u); free(P); free(U); free(t1); free(t2); free(nl_u); free(R2); free(R3); free(q3); free(q4);
    return OR_E_NOMEM;
  }
  int it_v = 0, it3 = 0, it4 = 0;
  op_rhs(&op, u, f_u);
  for (long q = 0; q < n; ++q) f_u[q] = h * f_u[q];
  /* P_j = phi_1(alpha_j h J) h f(u), alpha = (c2, c3, 1), one Newton basis */
  const double alpha[3] = {c2, c3, 1.0};
  int st = or_leja_phi_vertical(op.kind, op.nx, op.ny, op.nu, op.a, op.u, 1, 3, alpha, f_u, c, gamma, h, rtol,
                                atol, xi, K, P, &it_v);
  /* F(u) = f(u) - J(u) u */
  op_rhs(&op, u, t1);
  op_apply(&op, u, t2);
  for (long q = 0; q < n; ++q) nl_u[q] = t1[q] - t2[q];
  /* U_i = u + c_i P_i (phi_1(c_i h J) c_i h f(u)), R_i = h (F(U_i) - F(u)) */
  for (int i = 0; i < 2; ++i) {
    const double ci = alpha[i];
    double* R = i == 0 ? R2 : R3;
    for (long q = 0; q < n; ++q) U[q] = u[q] + ci * P[(size_t)i * n + q];
    op_rhs(&op, U, t1);
    op_apply(&op, U, t2);
    for (long q = 0; q < n; ++q) R[q] = h * (t1[q] - t2[q]) - h * nl_u[q];
  }
  /* W3, W4 into t1, t2 */
  for (long q = 0; q < n; ++q) {
    t1[q] = b2 * R2[q] + b3 * R3[q];
    t2[q] = e2 * R2[q] + e3 * R3[q];
  }
  int st3 = OR_OK, st4 = OR_OK;
  if (st == OR_OK) st3 = leja_phi_core(&op, 3, t1, c, gamma, h, rtol, atol, xi, K, q3, &it3);
  if (st == OR_OK && st3 == OR_OK) st4 = leja_phi_core(&op, 4, t2, c, gamma, h, rtol, atol, xi, K, q4, &it4);
  if (st != OR_OK || st3 != OR_OK) memset(q4, 0, sizeof(double) * (size_t)n);
  if (st != OR_OK) memset(q3, 0, sizeof(double) * (size_t)n);
  for (long q = 0; q < n; ++q) {
    u_low[q] = u[q] + P[2 * (size_t)n + q] + q3[q];
    u_high[q] = u_low[q] + q4[q];
  }
  *err = nrm(q4, n);
  *iters = it_v + it3 + it4;
  free(f_u); free(P); free(U); free(t1); free(t2); free(nl_u); free(R2); free(R3); free(q3); free(q4);
  return st != OR_OK ? st : (st3 != OR_OK ? st3 : st4);
}

int or_epirk4s3a_src(int kind, int nx, int ny, double nu, double a, const double* u, const double* S, double c,
                     double gamma, double h, double rtol, double atol, const double* xi, int K, double* u_low,
                     double* u_high, double* err, int* iters) {
  if (nx <= 0 || ny <= 0 || gamma == 0.0) return OR_E_INVAL;
  or_op op = {kind, nx, ny, nu, a, u, S};
  return epirk4s3a_core(&op, u, c, gamma, h, rtol, atol, xi, K, u_low, u_high, err, iters);
}

/* ------------------------------------------------------------------------ */
/* Step-size control with the embedded error (Sec. 2.2 mentions that the    */
/* EXPRB32 error estimate can steer the step size).  The paper gives no     */
/* controller; the reading is the classical one for a third-order pair:     */
/* accept when err <= tol, and h_new = h * min(2, max(0.2,                  */
/* 0.9 (tol/err)^(1/3))) after every attempt (factor 2 when err = 0).       */
/* Every attempt first takes 10 power-iteration passes from v0 at the       */
/* current state for the spectral interval (Sec. 2.2, Listing 7).           */
/* ------------------------------------------------------------------------ */

double or_controller(double h, double err, double tol) {
  double f;
  if (!(err > 0.0)) f = 2.0;
  else {
    f = 0.9 * pow(tol / err, 1.0 / 3.0);
    if (f > 2.0) f = 2.0;
    if (f < 0.2) f = 0.2;
  }
  return h * f;
}

/* The adaptive run.  log (may be NULL): per attempt, four doubles (t at
 * the attempt, step tried, error estimate, 1 if accepted else 0), at most
 * log_cap attempts recorded. */
int or_integrate_exprb32_log(int kind, int nx, int ny, double nu, double a, double* u, const double* v0,
                             double t_final, double h0, double tol, double leja_tol, const double* xi, int K,
                             int max_attempts, int* steps_out, int* rejected_out, long long* iters_out,
                             double* h_out, double* t_out, double* log, int log_cap) {
  long n = (long)nx * ny;
  double* lo = (double*)malloc(sizeof(double) * (size_t)n);
  double* hi = (double*)malloc(sizeof(double) * (size_t)n);
  if (!lo || !hi) { free(lo); free(hi); return OR_E_NOMEM; }
  double t = 0.0, h = h0;
  int steps = 0, rejected = 0, status = OR_OK;
  long long iters_total = 0;
  for (int att = 0; att < max_attempts && t < t_final; ++att) {
    double hh = h < t_final - t ? h : t_final - t;
    double rho;
    int pit;
    int st = or_power_iteration(kind, nx, ny, nu, a, u, v0, 10, &rho, &pit);
    if (st != OR_OK) { status = st; break; }
    double lam = -1.05 * rho, c = lam / 2.0, gamma = -lam / 4.0;
    double err;
    int it;
    st = or_exprb32(kind, nx, ny, nu, a, u, c, gamma, hh, leja_tol, leja_tol, xi, K, lo, hi, &err, &it);
    iters_total += it;
    if (st != OR_OK) { status = st; break; }
    if (log && att < log_cap) {
      log[4 * att] = t;
      log[4 * att + 1] = hh;
      log[4 * att + 2] = err;
      log[4 * att + 3] = err <= tol ? 1.0 : 0.0;
    }
    if (err <= tol) {
      memcpy(u, hi, sizeof(double) * (size_t)n);
      t += hh;
      ++steps;
    } else {
      ++rejected;
    }
    h = or_controller(hh, err, tol);
  }
  *steps_out = steps;
  *rejected_out = rejected;
  *iters_out = iters_total;
  *h_out = h;
  *t_out = t;
  free(lo);
  free(hi);
  return status;
}

int or_integrate_exprb32(int kind, int nx, int ny, double nu, double a, double* u, const double* v0,
                         double t_final, double h0, double tol, double leja_tol, const double* xi, int K,
                         int max_attempts, int* steps_out, int* rejected_out, long long* iters_out,
                         double* h_out, double* t_out) {
  return or_integrate_exprb32_log(kind, nx, ny, nu, a, u, v0, t_final, h0, tol, leja_tol, xi, K, max_attempts,
                                  steps_out, rejected_out, iters_out, h_out, t_out, NULL, 0);
}

/* ------------------------------------------------------------------------ */
/* The unfused form with a finite-difference Jacobian action (Sec. 2.3) and  */
/* a caller's right-hand side (Sec. 2).  f: NULL for the kind's own f (nu,   */
/* a, nx, ny as in the fused entry points), else f(in, out, user) over       */
/* nx*ny values.  eps0 > 0: the relative difference step (see the header).   */
/* ------------------------------------------------------------------------ */

static int fd_op(int kind, int nx, int ny, double nu, double a, or_rhs_fn f, void* user, double eps0,
                 const double* u, or_op* op) {
  if (nx <= 0 || ny <= 0 || !(eps0 > 0.0)) return OR_E_INVAL;
  or_op o = {kind, nx, ny, nu, a, u, NULL, f, user, eps0};
  *op = o;
  return OR_OK;
}

int or_fd_jv(int kind, int nx, int ny, double nu, double a, or_rhs_fn f, void* user, double eps0,
             const double* u, const double* v, double* out) {
  or_op op;
  int st = fd_op(kind, nx, ny, nu, a, f, user, eps0, u, &op);
  if (st != OR_OK) return st;
  op_apply(&op, v, out);
  return OR_OK;
}

int or_power_iteration_fd(int kind, int nx, int ny, double nu, double a, or_rhs_fn f, void* user, double eps0,
                          const double* u, const double* v0, int max_iters, double* rho_out, int* iters_out) {
  or_op op;
  int st = fd_op(kind, nx, ny, nu, a, f, user, eps0, u, &op);
  if (st != OR_OK || max_iters <= 0) return OR_E_INVAL;
  return power_core(&op, v0, max_iters, rho_out, iters_out);
}

int or_leja_phi_fd(int kind, int nx, int ny, double nu, double a, or_rhs_fn f, void* user, double eps0,
                   const double* u, int l, const double* w, double c, double gamma, double h, double rtol,
                   double atol, const double* xi, int K, double* out, int* iters) {
  or_op op;
  int st = fd_op(kind, nx, ny, nu, a, f, user, eps0, u, &op);
  if (st != OR_OK || l < 0 || gamma == 0.0) return OR_E_INVAL;
  return leja_phi_core(&op, l, w, c, gamma, h, rtol, atol, xi, K, out, iters);
}

int or_ros_eu_fd(int kind, int nx, int ny, double nu, double a, or_rhs_fn f, void* user, double eps0,
                 const double* u, double c, double gamma, double h, double rtol, double atol, const double* xi,
                 int K, double* u_out, int* iters) {
  or_op op;
  int st = fd_op(kind, nx, ny, nu, a, f, user, eps0, u, &op);
  if (st != OR_OK) return st;
  return ros_eu_core(&op, u, c, gamma, h, rtol, atol, xi, K, u_out, iters);
}

int or_exprb32_fd(int kind, int nx, int ny, double nu, double a, or_rhs_fn f, void* user, double eps0,
                  const double* u, double c, double gamma, double h, double rtol, double atol, const double* xi,
                  int K, double* u_low, double* u_high, double* err, int* iters) {
  or_op op;
  int st = fd_op(kind, nx, ny, nu, a, f, user, eps0, u, &op);
  if (st != OR_OK) return st;
  return exprb32_core(&op, u, c, gamma, h, rtol, atol, xi, K, u_low, u_high, err, iters);
}
