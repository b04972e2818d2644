// Unfused Leja engine for a caller's right-hand side f (Sec. 2: f maps an
// input pointer to an output pointer over contiguous data, its parameters
// held by a functor) with the Jacobian action by central finite differences
// of f (Sec. 2.3).
//
// One Leja iteration (Sec. 2.1, Eq. 2, with Op = J(u)) is
//   fd_perturb_kernel   x+ = u + e y_m,  x- = u - e y_m             one pass
//   f(x+), f(x-)                                                    the caller's
//   fd_update_kernel    t = (f(x+) - f(x-)) / (2e)
//                       y_{m+1} = (t - c y_m)/gamma - xi_m y_m
//                       p_{m+1} = p_m + d_{m+1} y_{m+1}
//                       sum y^2, sum p^2 -> stopping test (Sec. 2.2)   one pass
// with e = eps0 (1 + ||u||) / ||y_m||.  ||y_m|| comes out of the previous
// update's reduction, so e, the iteration index and the stop flag live on
// the device (FdState) and the host never waits inside an iteration; it
// reads the stop flag one iteration behind.  The perturbation is formed with
// separately rounded products and sums (no contraction), as a plain
// sequential evaluation would; the update folds 1/(2e) and 1/gamma into one
// factor, y_{m+1} = (f(x+) - f(x-)) (1/(2e gamma)) - (c/gamma + xi_m) y_m,
// which leaves three FP64 operations per point (the FP64 pipe, not memory,
// bounds these kernels on GB300).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "leja_kernels.cuh"
#include "lexgb.h"
#include "lexgb_internal.h"

namespace lexgb {
namespace {

constexpr double kDefaultEps0 = 3.814697265625e-06;  // 2^-18
constexpr int kMaxPowerPasses = 64;

struct FdState {
  int m;        // Leja iterations done in the current loop
  int done;     // 1 once the loop stopped
  int status;   // lx_status of the loop
  int pk;       // power iteration: passes done
  int pdone;    // power iteration: stopped
  int pmax;     // power iteration: pass limit
  double eps;   // difference step e of the next Jacobian product (0: the vector is zero)
  double unorm; // ||u|| of the linearisation point
  double vnorm; // ||v|| of the power iteration's current vector
  double ynorm, pnorm, err;
  double rho, rho_prev;
  double red;   // ||x|| from fd_final_kernel
};

__device__ __forceinline__ long long gtid() { return blockIdx.x * (long long)blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long gstride() { return (long long)gridDim.x * blockDim.x; }

__device__ __forceinline__ double fd_step(double eps0, double unorm, double vnorm) {
  return vnorm > 0.0 ? eps0 * (1.0 + unorm) / vnorm : 0.0;
}

// Start of a Leja loop: y_0 = w, p_0 = d_0 w; ||u|| and ||w|| give the first
// step; the loop state is reset.
__global__ void __launch_bounds__(kThreadsPerBlock)
    fd_init_kernel(long long n, const double* __restrict__ u, const double* __restrict__ w,
                   const double* __restrict__ d, double* __restrict__ y0, double* __restrict__ p, FdState* st,
                   double eps0, double* __restrict__ partials, unsigned int* __restrict__ ticket) {
  const double d0 = d[0];
  double su = 0.0, sw = 0.0;
  for (long long q = gtid(); q < n; q += gstride()) {
    const double wq = w[q];
    y0[q] = wq;
    p[q] = __dmul_rn(d0, wq);
    sw += wq * wq;
    if (u) su += u[q] * u[q];
  }
  if (last_block_total2(su, sw, partials, ticket) && threadIdx.x == 0) {
    const double un = sqrt(su / double(n)), wn = sqrt(sw / double(n));
    st->m = 0;
    st->done = 0;
    st->status = 0;
    st->unorm = un;
    st->eps = fd_step(eps0, un, wn);
  }
}

// x+ = u + e v, x- = u - e v (u NULL: 0).  gate 1: skip once the Leja loop
// has stopped; 2: once the power iteration has; 0: always run.
__global__ void __launch_bounds__(kThreadsPerBlock)
    fd_perturb_kernel(long long n, const double* __restrict__ u, const double* __restrict__ v,
                      double* __restrict__ xp, double* __restrict__ xm, const FdState* st, int gate) {
  if ((gate == 1 && st->done) || (gate == 2 && st->pdone)) return;
  const double e = st->eps;
  for (long long q = gtid(); q < n; q += gstride()) {
    const double uq = u ? u[q] : 0.0;
    const double ev = __dmul_rn(e, v[q]);
    xp[q] = __dadd_rn(uq, ev);
    xm[q] = __dsub_rn(uq, ev);
  }
}

// 1 / (2 e) once per thread (0 for a zero vector, whose product is 0).
__device__ __forceinline__ double fd_inv2e(double e) { return e > 0.0 ? 1.0 / (2.0 * e) : 0.0; }

// The Newton update from the difference quotient, the stopping norms and the
// stopping test (thread 0 of the last block), then the next step e.
__global__ void __launch_bounds__(kThreadsPerBlock)
    fd_update_kernel(long long n, const double* __restrict__ y, double* __restrict__ ynew, double* __restrict__ p,
                     const double* __restrict__ fp, const double* __restrict__ fm, const double* __restrict__ xi,
                     const double* __restrict__ d, double cc, double gamma, double rtol, double atol, int kmax,
                     double eps0, FdState* st, double* __restrict__ partials, unsigned int* __restrict__ ticket) {
  if (st->done) return;
  const int m = st->m;
  const double xm = xi[m], dm1 = d[m + 1];
  const double sq = fd_inv2e(st->eps) / gamma;  // 1 / (2 e gamma)
  const double sc = -(cc / gamma + xm);         // -(c/gamma + xi_m)
  double sy = 0.0, sp = 0.0;
  for (long long q = gtid(); q < n; q += gstride()) {
    const double yn = fma(fp[q] - fm[q], sq, sc * y[q]);
    const double pn = fma(dm1, yn, p[q]);
    ynew[q] = yn;
    p[q] = pn;
    sy = fma(yn, yn, sy);
    sp = fma(pn, pn, sp);
  }
  if (last_block_total2(sy, sp, partials, ticket) && threadIdx.x == 0) {
    const double ynorm = sqrt(sy / double(n)), pnorm = sqrt(sp / double(n));
    const double err = fabs(dm1) * ynorm;
    const int m1 = m + 1;
    int status = 0;
    bool stop = false;
    if (!isfinite(err) || !isfinite(pnorm)) {
      status = 5;  // LX_E_NONFINITE
      stop = true;
    } else if (err <= rtol * pnorm + atol) {
      stop = true;
    } else if (m1 >= kmax) {
      status = 4;  // LX_E_NOCONV
      stop = true;
    }
    st->m = m1;
    st->ynorm = ynorm;
    st->pnorm = pnorm;
    st->err = err;
    st->eps = fd_step(eps0, st->unorm, ynorm);
    if (stop) {
      st->status = status;
      st->done = 1;
    }
  }
}

// Norms of u and v and the step of one Jacobian product J(u) v (outside the
// Leja loop), or the start of a power iteration (power: v0 copied to vbuf,
// pass state reset).
__global__ void __launch_bounds__(kThreadsPerBlock)
    fd_norms_kernel(long long n, const double* __restrict__ u, const double* __restrict__ v,
                    double* __restrict__ vbuf, FdState* st, double eps0, int power_max,
                    double* __restrict__ partials, unsigned int* __restrict__ ticket) {
  double su = 0.0, sv = 0.0;
  for (long long q = gtid(); q < n; q += gstride()) {
    const double vq = v[q];
    if (vbuf) vbuf[q] = vq;
    sv += vq * vq;
    if (u) su += u[q] * u[q];
  }
  if (last_block_total2(su, sv, partials, ticket) && threadIdx.x == 0) {
    const double un = sqrt(su / double(n)), vn = sqrt(sv / double(n));
    st->unorm = un;
    st->vnorm = vn;
    st->eps = fd_step(eps0, un, vn);
    if (power_max > 0) {
      st->pk = 0;
      st->pdone = 0;
      st->pmax = power_max;
      st->rho = 0.0;
      st->rho_prev = 0.0;
    }
  }
}

// out = J(u) v from the two right-hand-side values.
__global__ void __launch_bounds__(kThreadsPerBlock)
    fd_jv_kernel(long long n, const double* __restrict__ fp, const double* __restrict__ fm, double* __restrict__ out,
                 const FdState* st) {
  const double ie = fd_inv2e(st->eps);
  for (long long q = gtid(); q < n; q += gstride()) out[q] = (fp[q] - fm[q]) * ie;
}

// One power-iteration pass (Sec. 2, Listing 7) after the two right-hand-side
// calls: w = J(u) v, rho_k = ||w|| / ||v||, stop test; the next kernel
// normalises v = w / ||w||.
__global__ void __launch_bounds__(kThreadsPerBlock)
    fd_power_kernel(long long n, const double* __restrict__ fp, const double* __restrict__ fm,
                    double* __restrict__ w, FdState* st, double* __restrict__ partials,
                    unsigned int* __restrict__ ticket) {
  if (st->pdone) return;
  const double ie = fd_inv2e(st->eps);
  double sw = 0.0, unused = 0.0;
  for (long long q = gtid(); q < n; q += gstride()) {
    const double t = (fp[q] - fm[q]) * ie;
    w[q] = t;
    sw += t * t;
  }
  if (last_block_total2(sw, unused, partials, ticket) && threadIdx.x == 0) {
    const double nw = sqrt(sw / double(n));
    const double rho = nw / st->vnorm;
    const int k = st->pk + 1;
    st->pk = k;
    st->rho = rho;
    st->red = nw;
    bool stop = k >= st->pmax || !isfinite(rho);
    if (k > 1 && fabs(rho - st->rho_prev) <= 1e-2 * rho) stop = true;
    st->rho_prev = rho;
    if (stop) st->pdone = 1;
  }
}

__global__ void __launch_bounds__(kThreadsPerBlock)
    fd_power_scale_kernel(long long n, const double* __restrict__ w, double* __restrict__ v, FdState* st,
                          double eps0, double* __restrict__ partials, unsigned int* __restrict__ ticket) {
  if (st->pdone) return;
  const double nw = st->red;
  double sv = 0.0, unused = 0.0;
  for (long long q = gtid(); q < n; q += gstride()) {
    const double t = w[q] / nw;
    v[q] = t;
    sv += t * t;
  }
  if (last_block_total2(sv, unused, partials, ticket) && threadIdx.x == 0) {
    const double vn = sqrt(sv / double(n));
    st->vnorm = vn;
    st->eps = fd_step(eps0, st->unorm, vn);
  }
}

// Element-wise stage arithmetic of the integrators (Sec. 2.3, Listings 12, 13).
enum { kScale = 0, kAdd = 1, kSub = 2, kRemainder = 3 };

// kScale: y = s x;  kAdd: y = x + z;  kSub: y = x - z;
// kRemainder: y = s x - s z  (R = h nl_a - h nl_u).
__global__ void __launch_bounds__(kThreadsPerBlock)
    fd_axpy_kernel(int op, long long n, double s, const double* __restrict__ x, const double* __restrict__ z,
                   double* y) {
  for (long long q = gtid(); q < n; q += gstride()) {
    double r;
    if (op == kScale)
      r = __dmul_rn(s, x[q]);
    else if (op == kAdd)
      r = __dadd_rn(x[q], z[q]);
    else if (op == kSub)
      r = __dsub_rn(x[q], z[q]);
    else
      r = __dsub_rn(__dmul_rn(s, x[q]), __dmul_rn(s, z[q]));
    y[q] = r;
  }
}

// EXPRB32 output: p3 = 2 p3, u_high = u_low + p3, ||p3|| into st->red.
__global__ void __launch_bounds__(kThreadsPerBlock)
    fd_final_kernel(long long n, const double* __restrict__ u_low, double* __restrict__ p3,
                    double* __restrict__ u_high, FdState* st, double* __restrict__ partials,
                    unsigned int* __restrict__ ticket) {
  double s = 0.0, unused = 0.0;
  for (long long q = gtid(); q < n; q += gstride()) {
    const double t = __dmul_rn(2.0, p3[q]);
    p3[q] = t;
    u_high[q] = __dadd_rn(u_low[q], t);
    s += t * t;
  }
  if (last_block_total2(s, unused, partials, ticket) && threadIdx.x == 0) st->red = sqrt(s / double(n));
}

// ---------------------------------------------------------------------------
// The engine's own right-hand sides in lx_rhs_fn form (FP64, one thread per
// point, periodic).  Central kinds on the unit square (spacing 1/n): A u =
// nu Lap u + a (u_x + u_y); Burgers f = nu Lap u - u (u_x + u_y).  Upwind
// kinds on [-1,1)^2 (spacing 2/n): the third-order upwind-biased gradient,
// for a term +a v_x with side s = sign(a): |a| (-v_{i+2s} + 6 v_{i+s} - 3 v_i
// - 2 v_{i-s}) / (6 dx); Burgers flux form nu Lap u + (a/2) D(u^2) (Sec. 3, Eq. 5).
// ---------------------------------------------------------------------------

struct BuiltinRhs {
  int nx, ny, kind, s;
  long long n;
  double nu, a, cxx, cyy, gx, gy;
  double we, ww, wn, ws, wc;  // central kinds: neighbour weights of A, centre weight of the Laplacian
};

// periodic index for any offset (grids down to one point per direction)
__device__ __forceinline__ int wrapi(int i, int n) {
  const int r = i % n;
  return r < 0 ? r + n : r;
}

__global__ void __launch_bounds__(kThreadsPerBlock) builtin_rhs_kernel(BuiltinRhs B, const double* __restrict__ u,
                                                                     double* __restrict__ f) {
  for (long long q = gtid(); q < B.n; q += gstride()) {
    // q < 2^31: 32-bit index arithmetic
    const unsigned uq = (unsigned)q, unx = (unsigned)B.nx;
    const int j = (int)(uq / unx), i = (int)(uq - (unsigned)j * unx);
    const long long row = (long long)j * B.nx;
    const int ie = i + 1 == B.nx ? 0 : i + 1, iw = i == 0 ? B.nx - 1 : i - 1;
    const int jn = j + 1 == B.ny ? 0 : j + 1, js = j == 0 ? B.ny - 1 : j - 1;
    const double uc = u[q];
    const double ue = u[row + ie], uw = u[row + iw];
    const double un = u[(long long)jn * B.nx + i], us = u[(long long)js * B.nx + i];
    double r;
    if (B.kind == LX_ADVDIFF) {
      // one weight per neighbour: nu / dx^2 +- a / (2 dx), ...
      r = fma(B.we, ue, fma(B.ww, uw, fma(B.wn, un, fma(B.ws, us, B.wc * uc))));
    } else if (B.kind == LX_BURGERS) {
      const double lap = fma(B.cxx, ue + uw, fma(B.cyy, un + us, B.wc * uc));
      const double grad = fma(B.gx, ue - uw, B.gy * (un - us));
      r = fma(-uc, grad, lap);
    } else {
      const double lap = B.cxx * (ue - 2.0 * uc + uw) + B.cyy * (un - 2.0 * uc + us);
      const int s = B.s;
      const bool sq = B.kind == LX_BURGERS_UP3;
      auto val = [&](long long k) {
        const double v = u[k];
        return sq ? v * v : v;
      };
      const double x2 = val(row + wrapi(i + 2 * s, B.nx)), x1 = val(row + wrapi(i + s, B.nx)),
                   x0 = val(q), xm1 = val(row + wrapi(i - s, B.nx));
      const double y2 = val((long long)wrapi(j + 2 * s, B.ny) * B.nx + i),
                   y1 = val((long long)wrapi(j + s, B.ny) * B.nx + i),
                   ym1 = val((long long)wrapi(j - s, B.ny) * B.nx + i);
      const double dgrad = B.gx * (-x2 + 6.0 * x1 - 3.0 * x0 - 2.0 * xm1) + B.gy * (-y2 + 6.0 * y1 - 3.0 * x0 - 2.0 * ym1);
      r = lap + (sq ? 0.5 * dgrad : dgrad);
    }
    f[q] = r;
  }
}

std::string cuda_msg(cudaError_t e, const char* what) { return std::string(what) + ": " + cudaGetErrorString(e); }

}  // namespace
}  // namespace lexgb

using namespace lexgb;

struct lx_rhs_ctx {
  long long n = 0;
  lx_rhs_fn f = nullptr;
  void* user = nullptr;
  double eps0 = kDefaultEps0;
  int integrator = LX_ROS_EU;
  int K = 1000;
  cudaStream_t stream = nullptr;
  int grid = 1;
  std::vector<double> xi;
  double* d_xi = nullptr;
  struct Slot {
    bool valid = false;
    int l = -1, count = 0;
    double h = 0, c = 0, gamma = 0;
    double* dev = nullptr;
    std::vector<double> host;
  } coef[2];
  double* d_y[2] = {nullptr, nullptr};
  double *d_xp = nullptr, *d_xm = nullptr, *d_fp = nullptr, *d_fm = nullptr, *d_fu = nullptr;
  double *d_p1 = nullptr, *d_t1 = nullptr, *d_t2 = nullptr, *d_p3 = nullptr;
  double* d_partials = nullptr;
  unsigned int* d_ticket = nullptr;
  FdState* d_state = nullptr;
  FdState* h_state = nullptr;  // pinned
  int* h_flag = nullptr;       // pinned, two slots
  cudaEvent_t ev[2] = {};
  lx_rhs_stats stats{};
};

namespace {

#define FD_CUDA(call)                                       \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) {                                \
      lexgb::set_last_error(cuda_msg(e_, #call).c_str());   \
      return LX_E_CUDA;                                     \
    }                                                       \
  } while (0)

lx_status launched(lx_rhs_ctx* c) {
  ++c->stats.kernels;
  FD_CUDA(cudaGetLastError());
  return LX_OK;
}

lx_status call_f(lx_rhs_ctx* c, const double* in, double* out) {
  ++c->stats.rhs_calls;
  const int rc = c->f(in, out, c->user, reinterpret_cast<void*>(c->stream));
  if (rc != 0) {
    cudaStreamSynchronize(c->stream);
    lexgb::set_last_error("the right-hand side function returned an error");
    return LX_E_CALLBACK;
  }
  return LX_OK;
}

#define FD_TRY(expr)             \
  do {                           \
    lx_status s_ = (expr);       \
    if (s_ != LX_OK) return s_;  \
  } while (0)

lx_status ensure_coeffs(lx_rhs_ctx* c, int slot, int l, double h, double cc, double gamma) {
  auto& S = c->coef[slot];
  if (S.valid && S.l == l && S.h == h && S.c == cc && S.gamma == gamma) return LX_OK;
  const int count = leja_coeff_count(h, cc, gamma, c->K);
  S.host.assign(count, 0.0);
  const int st = leja_coeffs(l, h, cc, gamma, c->xi.data(), count, S.host.data());
  if (st != LX_OK) return (lx_status)st;
  // the previous table may still be read by queued kernels
  FD_CUDA(cudaStreamSynchronize(c->stream));
  FD_CUDA(cudaMemcpy(S.dev, S.host.data(), sizeof(double) * count, cudaMemcpyHostToDevice));
  S.valid = true;
  S.l = l;
  S.h = h;
  S.c = cc;
  S.gamma = gamma;
  S.count = count;
  return LX_OK;
}

// Enqueue the stop-flag copy of the current iteration and test the previous
// one's; true once the device has stopped.
lx_status poll_stop(lx_rhs_ctx* c, int k, const int* dev_flag, bool* stopped) {
  FD_CUDA(cudaMemcpyAsync(c->h_flag + (k & 1), dev_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  FD_CUDA(cudaEventRecord(c->ev[k & 1], c->stream));
  *stopped = false;
  if (k >= 1) {
    FD_CUDA(cudaEventSynchronize(c->ev[(k - 1) & 1]));
    *stopped = c->h_flag[(k - 1) & 1] != 0;
  }
  return LX_OK;
}

lx_status fetch_state(lx_rhs_ctx* c) {
  FD_CUDA(cudaMemcpyAsync(c->h_state, c->d_state, sizeof(FdState), cudaMemcpyDeviceToHost, c->stream));
  FD_CUDA(cudaStreamSynchronize(c->stream));
  return LX_OK;
}

// phi_l(h J(u)) w into p (Sec. 2.2-2.3: real_Leja_phi with the Jacobian by
// differences).  Synchronises; iters and status from the device state.
lx_status leja_loop(lx_rhs_ctx* c, int slot, int l, const double* u, const double* w, double* p, double cc,
                    double gamma, double h, double rtol, double atol, int* iters) {
  FD_TRY(ensure_coeffs(c, slot, l, h, cc, gamma));
  const auto& S = c->coef[slot];
  const int kmax = S.count - 1;
  const long long n = c->n;
  fd_init_kernel<<<c->grid, kThreadsPerBlock, 0, c->stream>>>(n, u, w, S.dev, c->d_y[0], p, c->d_state, c->eps0,
                                                              c->d_partials, c->d_ticket);
  FD_TRY(launched(c));
  int cur = 0;
  for (int m = 0; m < kmax; ++m) {
    fd_perturb_kernel<<<c->grid, kThreadsPerBlock, 0, c->stream>>>(n, u, c->d_y[cur], c->d_xp, c->d_xm, c->d_state,
                                                                   1);
    FD_TRY(launched(c));
    FD_TRY(call_f(c, c->d_xp, c->d_fp));
    FD_TRY(call_f(c, c->d_xm, c->d_fm));
    fd_update_kernel<<<c->grid, kThreadsPerBlock, 0, c->stream>>>(
        n, c->d_y[cur], c->d_y[cur ^ 1], p, c->d_fp, c->d_fm, c->d_xi, S.dev, cc, gamma, rtol, atol, kmax, c->eps0,
        c->d_state, c->d_partials, c->d_ticket);
    FD_TRY(launched(c));
    cur ^= 1;
    bool stopped = false;
    FD_TRY(poll_stop(c, m, &c->d_state->done, &stopped));
    if (stopped) break;
  }
  FD_TRY(fetch_state(c));
  if (iters) *iters = c->h_state->m;
  c->stats.leja_iterations += c->h_state->m;
  return (lx_status)c->h_state->status;
}

// out = J(u) v by the central quotient (st->eps set for v).
lx_status jv(lx_rhs_ctx* c, const double* u, const double* v, double* out) {
  fd_norms_kernel<<<c->grid, kThreadsPerBlock, 0, c->stream>>>(c->n, u, v, nullptr, c->d_state, c->eps0, 0,
                                                               c->d_partials, c->d_ticket);
  FD_TRY(launched(c));
  fd_perturb_kernel<<<c->grid, kThreadsPerBlock, 0, c->stream>>>(c->n, u, v, c->d_xp, c->d_xm, c->d_state, 0);
  FD_TRY(launched(c));
  FD_TRY(call_f(c, c->d_xp, c->d_fp));
  FD_TRY(call_f(c, c->d_xm, c->d_fm));
  fd_jv_kernel<<<c->grid, kThreadsPerBlock, 0, c->stream>>>(c->n, c->d_fp, c->d_fm, out, c->d_state);
  return launched(c);
}

lx_status axpy(lx_rhs_ctx* c, int op, double s, const double* x, const double* z, double* y) {
  fd_axpy_kernel<<<c->grid, kThreadsPerBlock, 0, c->stream>>>(op, c->n, s, x, z, y);
  return launched(c);
}

void free_ctx(lx_rhs_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  cudaFree(c->d_xi);
  for (auto& S : c->coef) cudaFree(S.dev);
  for (double* p : {c->d_y[0], c->d_y[1], c->d_xp, c->d_xm, c->d_fp, c->d_fm, c->d_fu, c->d_p1, c->d_t1, c->d_t2,
                    c->d_p3, c->d_partials})
    cudaFree(p);
  cudaFree(c->d_ticket);
  cudaFree(c->d_state);
  cudaFreeHost(c->h_state);
  cudaFreeHost(c->h_flag);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  delete c;
}

}  // namespace

extern "C" {

int lx_rhs_builtin(const double* in, double* out, void* user, void* cuda_stream) {
  const lx_problem* P = static_cast<const lx_problem*>(user);
  if (!P || !in || !out || P->nx < 1 || P->ny < 1 || P->kind < LX_ADVDIFF || P->kind > LX_BURGERS_UP3) return 1;
  BuiltinRhs B{};
  B.nx = P->nx;
  B.ny = P->ny;
  B.kind = P->kind;
  B.n = (long long)P->nx * P->ny;
  B.nu = P->nu;
  B.a = P->a;
  if (P->kind == LX_ADVDIFF || P->kind == LX_BURGERS) {
    const double dx = 1.0 / P->nx, dy = 1.0 / P->ny;
    B.cxx = P->nu / (dx * dx);
    B.cyy = P->nu / (dy * dy);
    B.gx = 1.0 / (2 * dx);
    B.gy = 1.0 / (2 * dy);
    B.s = 1;
    B.we = B.cxx + P->a * B.gx;
    B.ww = B.cxx - P->a * B.gx;
    B.wn = B.cyy + P->a * B.gy;
    B.ws = B.cyy - P->a * B.gy;
    B.wc = -2.0 * (B.cxx + B.cyy);
  } else {
    const double dx = 2.0 / P->nx, dy = 2.0 / P->ny;
    B.cxx = P->nu / (dx * dx);
    B.cyy = P->nu / (dy * dy);
    B.gx = std::fabs(P->a) / (6.0 * dx);
    B.gy = std::fabs(P->a) / (6.0 * dy);
    B.s = P->a >= 0.0 ? 1 : -1;
  }
  const long long want = (B.n + kThreadsPerBlock - 1) / kThreadsPerBlock;
  const int grid = (int)std::max<long long>(1, std::min<long long>(want, 4096));
  builtin_rhs_kernel<<<grid, kThreadsPerBlock, 0, reinterpret_cast<cudaStream_t>(cuda_stream)>>>(B, in, out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    lexgb::set_last_error(cuda_msg(e, "builtin_rhs_kernel").c_str());
    return 1;
  }
  return 0;
}

lx_status leja_setup_rhs(long long n, lx_rhs_fn f, void* user, double eps0, int integrator, int max_leja,
                         void* cuda_stream, lx_rhs_ctx** out) {
  if (!out) return LX_E_INVAL;
  *out = nullptr;
  if (n < 1 || n > (1LL << 31) || !f) return LX_E_INVAL;
  if (integrator != LX_ROS_EU && integrator != LX_EXPRB32) return LX_E_INVAL;
  if (eps0 == 0.0) eps0 = kDefaultEps0;
  if (!(eps0 > 0.0) || !std::isfinite(eps0)) return LX_E_INVAL;
  if (max_leja == 0) max_leja = 1000;
  if (max_leja < 16 || max_leja > 4096) return LX_E_INVAL;
  lx_rhs_ctx* c = new (std::nothrow) lx_rhs_ctx();
  if (!c) return LX_E_NOMEM;
  c->n = n;
  c->f = f;
  c->user = user;
  c->eps0 = eps0;
  c->integrator = integrator;
  c->K = max_leja;
  c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  auto fail = [&](lx_status s, cudaError_t e, const char* what) {
    if (e != cudaSuccess) lexgb::set_last_error(cuda_msg(e, what).c_str());
    free_ctx(c);
    return s;
  };
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(LX_E_CUDA, e, "cudaGetDevice");
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(LX_E_CUDA, e, "sm count");
  const long long want = (n + kThreadsPerBlock - 1) / kThreadsPerBlock;
  c->grid = (int)std::max<long long>(1, std::min<long long>(want, 4LL * sms));
  c->xi.assign(c->K, 0.0);
  if (leja_points(c->K, c->xi.data()) != LX_OK) return fail(LX_E_INVAL, cudaSuccess, "");
  const size_t nb = sizeof(double) * (size_t)n;
  auto dm = [&](void** p, size_t bytes) { return cudaMalloc(p, bytes); };
  if ((e = dm((void**)&c->d_xi, sizeof(double) * c->K)) != cudaSuccess) return fail(LX_E_NOMEM, e, "cudaMalloc");
  for (auto& S : c->coef)
    if ((e = dm((void**)&S.dev, sizeof(double) * c->K)) != cudaSuccess) return fail(LX_E_NOMEM, e, "cudaMalloc");
  std::vector<double**> bufs = {&c->d_y[0], &c->d_y[1], &c->d_xp, &c->d_xm, &c->d_fp, &c->d_fm, &c->d_fu};
  if (integrator == LX_EXPRB32) {
    bufs.push_back(&c->d_p1);
    bufs.push_back(&c->d_t1);
    bufs.push_back(&c->d_t2);
    bufs.push_back(&c->d_p3);
  }
  for (double** b : bufs)
    if ((e = dm((void**)b, nb)) != cudaSuccess) return fail(LX_E_NOMEM, e, "cudaMalloc");
  if ((e = dm((void**)&c->d_partials, sizeof(double) * 2 * c->grid)) != cudaSuccess)
    return fail(LX_E_NOMEM, e, "cudaMalloc");
  if ((e = dm((void**)&c->d_ticket, sizeof(unsigned int))) != cudaSuccess) return fail(LX_E_NOMEM, e, "cudaMalloc");
  if ((e = dm((void**)&c->d_state, sizeof(FdState))) != cudaSuccess) return fail(LX_E_NOMEM, e, "cudaMalloc");
  if ((e = cudaMallocHost((void**)&c->h_state, sizeof(FdState))) != cudaSuccess)
    return fail(LX_E_NOMEM, e, "cudaMallocHost");
  if ((e = cudaMallocHost((void**)&c->h_flag, 2 * sizeof(int))) != cudaSuccess)
    return fail(LX_E_NOMEM, e, "cudaMallocHost");
  for (auto& ev : c->ev)
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
      return fail(LX_E_CUDA, e, "cudaEventCreate");
  if ((e = cudaMemsetAsync(c->d_ticket, 0, sizeof(unsigned int), c->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->d_state, 0, sizeof(FdState), c->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(c->d_xi, c->xi.data(), sizeof(double) * c->K, cudaMemcpyHostToDevice, c->stream)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return fail(LX_E_CUDA, e, "setup");
  *out = c;
  return LX_OK;
}

void leja_destroy_rhs(lx_rhs_ctx* c) { free_ctx(c); }

lx_status power_bound_rhs(lx_rhs_ctx* c, const double* u, const double* v0, int max_iters, double* rho, int* iters) {
  if (!c || !v0 || !rho || max_iters < 1 || max_iters > kMaxPowerPasses) return LX_E_INVAL;
  // v lives in d_y[0], w in d_y[1]
  fd_norms_kernel<<<c->grid, kThreadsPerBlock, 0, c->stream>>>(c->n, u, v0, c->d_y[0], c->d_state, c->eps0,
                                                               max_iters, c->d_partials, c->d_ticket);
  FD_TRY(launched(c));
  for (int k = 0; k < max_iters; ++k) {
    fd_perturb_kernel<<<c->grid, kThreadsPerBlock, 0, c->stream>>>(c->n, u, c->d_y[0], c->d_xp, c->d_xm,
                                                                   c->d_state, 2);
    FD_TRY(launched(c));
    FD_TRY(call_f(c, c->d_xp, c->d_fp));
    FD_TRY(call_f(c, c->d_xm, c->d_fm));
    fd_power_kernel<<<c->grid, kThreadsPerBlock, 0, c->stream>>>(c->n, c->d_fp, c->d_fm, c->d_y[1], c->d_state,
                                                                 c->d_partials, c->d_ticket);
    FD_TRY(launched(c));
    fd_power_scale_kernel<<<c->grid, kThreadsPerBlock, 0, c->stream>>>(c->n, c->d_y[1], c->d_y[0], c->d_state,
                                                                       c->eps0, c->d_partials, c->d_ticket);
    FD_TRY(launched(c));
    bool stopped = false;
    FD_TRY(poll_stop(c, k, &c->d_state->pdone, &stopped));
    if (stopped) break;
  }
  FD_TRY(fetch_state(c));
  *rho = c->h_state->rho;
  if (iters) *iters = c->h_state->pk;
  return std::isfinite(*rho) ? LX_OK : LX_E_NONFINITE;
}

lx_status phi_l_apply_rhs(lx_rhs_ctx* c, int l, const double* u, const double* w, double* out, double cc,
                          double gamma, double h, double rtol, double atol, int* iters) {
  if (!c || !w || !out || l < 0 || l > 8 || gamma == 0.0 || !std::isfinite(h)) return LX_E_INVAL;
  if (out == w || (u && out == u)) return LX_E_INVAL;
  return leja_loop(c, l == 3 ? 1 : 0, l, u, w, out, cc, gamma, h, rtol, atol, iters);
}

lx_status expint_step_rhs(lx_rhs_ctx* c, const double* u, double* u_low, double* u_high, double cc, double gamma,
                          double h, double rtol, double atol, double* err, int* iters) {
  if (!c || !u || !u_high || gamma == 0.0 || !std::isfinite(h)) return LX_E_INVAL;
  if (u_high == u || (u_low && (u_low == u || u_low == u_high))) return LX_E_INVAL;
  if (c->integrator == LX_EXPRB32 && !u_low) return LX_E_INVAL;
  int it1 = 0, it2 = 0;
  // h f(u)
  FD_TRY(call_f(c, u, c->d_fu));
  FD_TRY(axpy(c, kScale, h, c->d_fu, nullptr, c->d_fu));
  if (c->integrator == LX_ROS_EU) {
    // u_high = u + phi_1(h J(u)) h f(u)   (Sec. 2.3, Listing 12)
    const lx_status st = leja_loop(c, 0, 1, u, c->d_fu, u_high, cc, gamma, h, rtol, atol, &it1);
    FD_TRY(axpy(c, kAdd, 0.0, u, u_high, u_high));
    FD_CUDA(cudaStreamSynchronize(c->stream));
    if (err) *err = 0.0;
    if (iters) *iters = it1;
    return st;
  }
  // EXPRB32 in the order of Sec. 2.3, Listing 13
  const lx_status st1 = leja_loop(c, 0, 1, u, c->d_fu, c->d_p1, cc, gamma, h, rtol, atol, &it1);
  FD_TRY(axpy(c, kAdd, 0.0, u, c->d_p1, u_low));
  // nl_u = f(u) - J(u) u  (into d_fu, whose h f(u) is no longer needed)
  FD_TRY(call_f(c, u, c->d_t1));
  FD_TRY(jv(c, u, u, c->d_t2));
  FD_TRY(axpy(c, kSub, 0.0, c->d_t1, c->d_t2, c->d_fu));
  // nl_a = f(a) - J(u) a  (into d_t1)
  FD_TRY(call_f(c, u_low, c->d_t1));
  FD_TRY(jv(c, u, u_low, c->d_t2));
  FD_TRY(axpy(c, kSub, 0.0, c->d_t1, c->d_t2, c->d_t1));
  // R = h nl_a - h nl_u  (into d_t2)
  FD_TRY(axpy(c, kRemainder, h, c->d_t1, c->d_fu, c->d_t2));
  lx_status st2 = LX_OK;
  if (st1 == LX_OK) {
    st2 = leja_loop(c, 1, 3, u, c->d_t2, c->d_p3, cc, gamma, h, rtol, atol, &it2);
  } else {
    FD_CUDA(cudaMemsetAsync(c->d_p3, 0, sizeof(double) * (size_t)c->n, c->stream));
  }
  fd_final_kernel<<<c->grid, kThreadsPerBlock, 0, c->stream>>>(c->n, u_low, c->d_p3, u_high, c->d_state,
                                                               c->d_partials, c->d_ticket);
  FD_TRY(launched(c));
  FD_TRY(fetch_state(c));
  if (err) *err = c->h_state->red;
  if (iters) *iters = it1 + it2;
  return st1 != LX_OK ? st1 : st2;
}

lx_status lx_rhs_ctx_stats(lx_rhs_ctx* c, lx_rhs_stats* out, int reset) {
  if (!c || !out) return LX_E_INVAL;
  *out = c->stats;
  if (reset) c->stats = lx_rhs_stats{};
  return LX_OK;
}

}  // extern "C"
