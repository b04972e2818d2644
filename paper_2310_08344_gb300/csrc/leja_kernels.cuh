// Device code of the Leja engine (sm_103a).
//
// The hot kernel is one fused Leja iteration (Sec. 2.1, Eq. 2):
//     y_{m+1} = ((Op - c)/gamma - xi_m) y_m            (5-point stencil)
//     p_{m+1} = p_m + d_{m+1} y_{m+1}                  (Newton term)
//     sum y_{m+1}^2, sum p_{m+1}^2                     (stopping norms)
// followed, in the last block to finish, by the stopping test of Sec. 2.2
// (|d_{m+1}| ||y_{m+1}|| <= rtol ||p_{m+1}|| + atol) which ends the CUDA
// graph's while-loop from the device.  The grid reduction is deterministic:
// every block writes its partial sums, and the last block adds them in block
// order.
//
// Work decomposition: a warp owns a strip of 32*VEC columns by H rows and
// walks down its rows with a three-row register window (rows j-1, j, j+1),
// so every y value is loaded from memory once per strip; x-neighbours come
// from the neighbouring lanes by warp shuffles, and only the two strip-edge
// columns are loaded separately.  VEC = 2 uses 16-byte (double) or 8-byte
// (float) vector accesses and needs nx % 64 == 0 and 16-byte aligned
// vectors; VEC = 1 handles any nx.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace lexgb {

constexpr int kWarpsPerBlock = 8;
constexpr int kThreadsPerBlock = kWarpsPerBlock * 32;

// Constants of the upwind operators on periodic [-1,1)^2 (see leja_upwind.cuh).
struct Up3Op {
  int nx, ny;
  long long n;
  int s;            // upwind side along both axes: +1 (a >= 0) or -1
  double cxx, cyy;  // nu / dx^2, nu / dy^2
  double gx, gy;    // |a| / (6 dx), |a| / (6 dy)
};

// Device-resident arguments of one Leja loop, written by set_loop_args before
// each graph launch so that the graph itself never changes.
struct LoopArgs {
  int nx, ny;
  long long n;
  int strip_h;
  int kmax;           // last allowed iteration index m+1 (NOCONV beyond)
  const double* w;    // y_0 (caller's input, double)
  void* y0;           // basis ping-pong buffers (double or float)
  void* y1;
  double* p;          // polynomial (caller's output)
  const double* u;    // linearisation point (Burgers)
  const double* s;    // u_x + u_y at the linearisation point (Burgers)
  const double* xi;   // Leja points
  const double* d;    // Newton coefficients
  // diffusion-advection: y' = wxp yE + wxm yW + wyp yN + wym yS + (wc0 - xi_m) yC
  double wxp, wxm, wyp, wym, wc0;
  // Burgers: y' = lx (yE + yW) + ly (yN + yS) + (wc0 - xi_m - s/gamma) yC
  //               - u (gx (yE - yW) + gy (yN - yS))
  double lx, ly, gx, gy, inv_gamma;
  double rtol, atol;
  float wf[8];        // df64 form: hi/lo float parts of wxp, wxm, wyp, wym
  float2* pdf;        // df64 form: the polynomial as float pairs
  int use_cond;       // 1: end the graph's while-loop from the device
  // df64 Burgers form: per-point q = u / (2 dx gamma) and
  // r = (-2 nu/dx^2 - 2 nu/dy^2 - c)/gamma - (u_x + u_y)/gamma as float pairs,
  // and hi/lo of lx = nu/(dx^2 gamma), ly = nu/(dy^2 gamma), dx/dy
  const float2* bq;
  const float2* br;
  float bl[6];
  // upwind operators: constants and the shift c of the spectral interval
  Up3Op up;
  double up_c;
  // mixed Burgers form: u and u_x + u_y as floats (converted once per loop)
  const float* uf;
  const float* sf;
};

// Device-resident loop and reduction state.
struct LoopState {
  int m;            // Leja iterations done in the current loop
  int status;       // lx_status of the current loop
  int done;         // 1 once the current loop has stopped
  int iters_total;  // Leja iterations summed over the loops of one call
  int status_total; // first non-OK loop status of the call
  int pk;           // power iteration: passes done
  int pdone;        // power iteration: stopped
  int pstatus;
  double ynorm, pnorm, err;  // last stopping-test values
  double sigma;              // power iteration: 1/||v_k||
  double rho, rho_prev;      // power iteration estimates
  double red;                // result of a reduction kernel (e.g. the step error)
  double red2;               // ||u|| from vec_norm_kernel
  int pmax;                  // power iteration: pass limit
  int wexp;                  // df64 form: largest biased exponent of |w|
  int kscale;                // df64 form: w is scaled by 2^-kscale
  int sig;                   // df64 form: the stored basis is y_m 2^-sig
  int dlt;                   // df64 form: extra scaling 2^-dlt of the next step
  int launches;              // fused-iteration launches of the call (incl. ones that found done)
  int fix;                   // two-step loops that stopped at an odd count: p holds one more term,
  int fix_buf;               //   fix_d * (basis buffer fix_buf), to be subtracted by the output pass
  double fix_d;
};

// One thread per launch records it (launches of one loop are stream-ordered).
__device__ __forceinline__ void count_launch(LoopState* st) {
  if (blockIdx.x == 0 && threadIdx.x == 0) st->launches += 1;
}

__device__ __forceinline__ int wrap_up(int i, int n) { return i + 1 == n ? 0 : i + 1; }
__device__ __forceinline__ int wrap_dn(int i, int n) { return i == 0 ? n - 1 : i - 1; }

// float -> double without the conversion unit (which issues at the FP64
// rate on GB300): for a normal float the double's bits are its sign, its
// exponent rebiased by 1023 - 127 and its 23 mantissa bits; zeros,
// subnormals, infinities and NaNs take the ordinary conversion.  Exact.
__device__ __forceinline__ double f2d_int(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return (double)f;
  const unsigned hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(b << 29));
}
__device__ __forceinline__ double to_double(float f) { return f2d_int(f); }
__device__ __forceinline__ double to_double(double d) { return d; }

template <typename S, int VEC>
__device__ __forceinline__ void load_vec(const S* __restrict__ row, int c, int nx, S (&v)[VEC]) {
  if constexpr (VEC == 2) {
    if constexpr (sizeof(S) == 8) {
      double2 t = __ldg(reinterpret_cast<const double2*>(row + c));
      v[0] = t.x;
      v[1] = t.y;
    } else {
      float2 t = __ldg(reinterpret_cast<const float2*>(row + c));
      v[0] = t.x;
      v[1] = t.y;
    }
  } else {
    v[0] = (c < nx) ? __ldg(row + c) : S(0);
  }
}

template <int VEC>
__device__ __forceinline__ void load_p(const double* __restrict__ row, int c, int nx, double (&v)[VEC]) {
  if constexpr (VEC == 2) {
    double2 t = *reinterpret_cast<const double2*>(row + c);
    v[0] = t.x;
    v[1] = t.y;
  } else {
    v[0] = (c < nx) ? row[c] : 0.0;
  }
}

template <int VEC>
__device__ __forceinline__ void store_p(double* __restrict__ row, int c, int nx, const double (&v)[VEC]) {
  if constexpr (VEC == 2) {
    *reinterpret_cast<double2*>(row + c) = make_double2(v[0], v[1]);
  } else {
    if (c < nx) row[c] = v[0];
  }
}

template <typename T, int VEC>
__device__ __forceinline__ void store_y(T* __restrict__ row, int c, int nx, const T (&v)[VEC]) {
  if constexpr (VEC == 2) {
    if constexpr (sizeof(T) == 8)
      *reinterpret_cast<double2*>(row + c) = make_double2(v[0], v[1]);
    else
      *reinterpret_cast<float2*>(row + c) = make_float2(v[0], v[1]);
  } else {
    if (c < nx) row[c] = v[0];
  }
}

// One strip: rows [r0, r1) of the columns [col0, col0 + 32*VEC).
// KIND: 0 diffusion-advection, 1 Burgers.  T: arithmetic / storage type of
// the basis.  S: type of the source vector (double for y_0 = w).  FIRST:
// the m = 0 iteration, where p_0 = d_0 y_0 is formed instead of loaded.
template <int KIND, typename T, int VEC, typename S, bool FIRST>
__device__ __forceinline__ void leja_strip(const LoopArgs& A, const S* __restrict__ src, T* __restrict__ dst,
                                           double* __restrict__ p, int col0, int r0, int r1, T wcm, double d0,
                                           double dm1, double& sy, double& sp) {
  const int lane = threadIdx.x & 31;
  const int nx = A.nx, ny = A.ny;
  const int c = col0 + lane * VEC;
  const int cl = c + VEC - 1;
  const bool active = c < nx;
  const int cw = col0 == 0 ? nx - 1 : col0 - 1;
  const int ce = (cl + 1 >= nx) ? 0 : cl + 1;
  const bool need_e = active && (lane == 31 || cl + 1 >= nx);

  S ys[VEC], yc[VEC], yn[VEC];
  load_vec<S, VEC>(src + (size_t)wrap_dn(r0, ny) * nx, c, nx, ys);
  load_vec<S, VEC>(src + (size_t)r0 * nx, c, nx, yc);
  for (int r = r0; r < r1; ++r) {
    const size_t ro = (size_t)r * nx;
    load_vec<S, VEC>(src + (size_t)wrap_up(r, ny) * nx, c, nx, yn);
    S xw = __shfl_up_sync(0xffffffffu, yc[VEC - 1], 1);
    S xe = __shfl_down_sync(0xffffffffu, yc[0], 1);
    if (lane == 0) xw = __ldg(src + ro + cw);
    if (need_e) xe = __ldg(src + ro + ce);
    double pold[VEC];
    if constexpr (!FIRST) load_p<VEC>(p + ro, c, nx, pold);
    T uu[VEC], ss[VEC];
    if constexpr (KIND == 1) {
#pragma unroll
      for (int k = 0; k < VEC; ++k) {
        if constexpr (std::is_same<T, float>::value) {
          uu[k] = active ? __ldg(A.uf + ro + c + k) : 0.f;
          ss[k] = active ? __ldg(A.sf + ro + c + k) : 0.f;
        } else {
          uu[k] = active ? __ldg(A.u + ro + c + k) : 0.0;
          ss[k] = active ? __ldg(A.s + ro + c + k) : 0.0;
        }
      }
    }
    T ynew[VEC];
    double pnew[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      const T e = T(k == VEC - 1 ? xe : yc[k + 1]);
      const T w = T(k == 0 ? xw : yc[k - 1]);
      const T nn = T(yn[k]), sv = T(ys[k]), cc = T(yc[k]);
      T v;
      if constexpr (KIND == 0) {
        v = T(A.wxp) * e;
        v = fma(T(A.wxm), w, v);
        v = fma(T(A.wyp), nn, v);
        v = fma(T(A.wym), sv, v);
        v = fma(wcm, cc, v);
      } else {
        const T gxy = fma(T(A.gx), e - w, T(A.gy) * (nn - sv));
        v = T(A.lx) * (e + w);
        v = fma(T(A.ly), nn + sv, v);
        v = fma(fma(-T(ss[k]), T(A.inv_gamma), wcm), cc, v);
        v = fma(-T(uu[k]), gxy, v);
      }
      ynew[k] = v;
      const double vd = to_double(v);
      const double po = FIRST ? d0 * double(yc[k]) : pold[k];
      pnew[k] = fma(dm1, vd, po);
      if (active) {
        sy = fma(vd, vd, sy);
        sp = fma(pnew[k], pnew[k], sp);
      }
    }
    if (active) {
      store_y<T, VEC>(dst + ro, c, nx, ynew);
      store_p<VEC>(p + ro, c, nx, pnew);
    }
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      ys[k] = yc[k];
      yc[k] = yn[k];
    }
  }
}

// Sum (a, b) over the block; returns the totals in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[32], sb[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sa[warp] = a;
    sb[warp] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    const int nw = (int)(blockDim.x >> 5);
    for (int w = 0; w < nw; ++w) {
      x += sa[w];
      y += sb[w];
    }
    a = x;
    b = y;
  }
  __syncthreads();
}

// Publish this block's partials and report whether it is the last block to
// arrive; the last block then holds the fixed-order totals in thread 0.
__device__ __forceinline__ bool last_block_total2(double& a, double& b, double* __restrict__ partials,
                                                  unsigned int* __restrict__ ticket) {
  __shared__ int am_last;
  block_sum2(a, b);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double x = 0.0, y = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    x += __ldcg(partials + 2 * i);
    y += __ldcg(partials + 2 * i + 1);
  }
  block_sum2(x, y);
  a = x;
  b = y;
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// Stopping test of one Leja iteration (thread 0 of the last block):
// converged when |d_{m+1}| ||y_{m+1}|| <= rtol ||p_{m+1}|| + atol (Sec. 2.2),
// with ||x|| = sqrt(sum x^2 / N); nscale undoes an input scaling.
__device__ __forceinline__ void leja_finalize(const LoopArgs& A, LoopState* st, int m, double dm1, double sy,
                                              double sp, double yscale, double pscale,
                                              cudaGraphConditionalHandle cond) {
  const double inv_n = 1.0 / double(A.n);
  const double ynorm = sqrt(sy * inv_n) * yscale, pnorm = sqrt(sp * inv_n) * pscale;
  const double e = fabs(dm1) * ynorm;
  const int m1 = m + 1;
  int status = 0;
  bool done = false;
  if (!isfinite(e) || !isfinite(pnorm)) {
    status = 5;  // LX_E_NONFINITE
    done = true;
  } else if (e <= A.rtol * pnorm + A.atol) {
    done = true;
  } else if (m1 >= A.kmax) {
    status = 4;  // LX_E_NOCONV
    done = true;
  }
  st->m = m1;
  st->ynorm = ynorm;
  st->pnorm = pnorm;
  st->err = e;
  if (done) {
    st->status = status;
    st->done = 1;
    st->iters_total += m1;
    if (st->status_total == 0) st->status_total = status;
    if (A.use_cond) cudaGraphSetConditional(cond, 0);
  }
}

template <int KIND, typename T, int VEC>
static __global__ void __launch_bounds__(kThreadsPerBlock)
    leja_iter_kernel(const LoopArgs* __restrict__ Ap, LoopState* __restrict__ st, double* __restrict__ partials,
                     unsigned int* __restrict__ ticket, cudaGraphConditionalHandle cond) {
  const LoopArgs& A = *Ap;
  const int m = __ldcg(&st->m);
  count_launch(st);
  if (__ldcg(&st->done)) return;
  const int nx = A.nx, ny = A.ny;
  const int H = A.strip_h;
  const int ncs = (nx + 32 * VEC - 1) / (32 * VEC);
  const int nstrips = ncs * ((ny + H - 1) / H);
  const double xim = __ldg(A.xi + m);
  const double dm1 = __ldg(A.d + m + 1);
  const double d0 = __ldg(A.d);
  const T wcm = T(A.wc0 - xim);
  T* dst = reinterpret_cast<T*>((m & 1) ? A.y1 : A.y0);
  double sy = 0.0, sp = 0.0;
  const int warp = threadIdx.x >> 5;
  for (int s = blockIdx.x * kWarpsPerBlock + warp; s < nstrips; s += gridDim.x * kWarpsPerBlock) {
    const int col0 = (s % ncs) * 32 * VEC;
    const int r0 = (s / ncs) * H;
    const int r1 = min(r0 + H, ny);
    if (m == 0) {
      leja_strip<KIND, T, VEC, double, true>(A, A.w, dst, A.p, col0, r0, r1, wcm, d0, dm1, sy, sp);
    } else {
      const T* src = reinterpret_cast<const T*>(((m - 1) & 1) ? A.y1 : A.y0);
      leja_strip<KIND, T, VEC, T, false>(A, src, dst, A.p, col0, r0, r1, wcm, d0, dm1, sy, sp);
    }
  }
  if (!last_block_total2(sy, sp, partials, ticket)) return;
  if (threadIdx.x == 0) leja_finalize(A, st, m, dm1, sy, sp, 1.0, 1.0, cond);
}

// Writes the loop arguments and resets the per-loop state (one thread).
static __global__ void set_loop_args_kernel(LoopArgs args, LoopArgs* dst, LoopState* st, unsigned int* ticket,
                                           int reset_wexp = 1) {
  *dst = args;
  st->m = 0;
  st->status = 0;
  st->done = 0;
  st->fix = 0;
  if (reset_wexp) st->wexp = 0;
  st->kscale = 0;
  st->sig = 0;
  st->dlt = 0;
  *ticket = 0u;
}

// Resets the per-call totals (one thread).
static __global__ void reset_call_kernel(LoopState* st, unsigned int* ticket) {
  st->wexp = 0;
  st->iters_total = 0;
  st->status_total = 0;
  st->launches = 0;
  st->red = 0.0;
  *ticket = 0u;
}

// Point-wise stencil helpers for the non-hot kernels (one thread per point).
struct Geo {
  int nx, ny;
  long long n;
  double idx2, idy2, i2dx, i2dy;  // 1/dx^2, 1/dy^2, 1/(2dx), 1/(2dy)
};

__device__ __forceinline__ void neighbours(const Geo& g, long long q, long long& e, long long& w, long long& nn,
                                           long long& s) {
  const int i = int(q % g.nx), j = int(q / g.nx);
  const long long row = (long long)j * g.nx;
  e = row + (i + 1 == g.nx ? 0 : i + 1);
  w = row + (i == 0 ? g.nx - 1 : i - 1);
  nn = (long long)(j + 1 == g.ny ? 0 : j + 1) * g.nx + i;
  s = (long long)(j == 0 ? g.ny - 1 : j - 1) * g.nx + i;
}

// h f(u) into f_out; for Burgers also (u_x + u_y) into s_out.  f_out may be
// NULL (only s is wanted).  src (may be NULL): a time-independent source
// added to f (the diffusion-advection problem with sources, Sec. 3, Eq. 4).
template <int KIND>
__global__ void rhs_kernel(Geo g, double nu, double a, double h, const double* __restrict__ u,
                           double* __restrict__ f_out, double* __restrict__ s_out,
                           const double* __restrict__ src = nullptr) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < g.n; q += (long long)gridDim.x * blockDim.x) {
    long long e, w, nn, s;
    neighbours(g, q, e, w, nn, s);
    const double uc = u[q], ue = u[e], uw = u[w], un = u[nn], us = u[s];
    const double lap = (ue - 2.0 * uc + uw) * g.idx2 + (un - 2.0 * uc + us) * g.idy2;
    const double grad = (ue - uw) * g.i2dx + (un - us) * g.i2dy;
    const double sq = src ? src[q] : 0.0;
    if (KIND == 0) {
      if (f_out) f_out[q] = h * (nu * lap + a * grad + sq);
    } else {
      if (f_out) f_out[q] = h * (nu * lap - uc * grad + sq);
      s_out[q] = grad;
    }
  }
}

// Float copy of a double vector (the mixed Burgers form's u and u_x + u_y).
static __global__ void to_float_kernel(long long n, const double* __restrict__ x, float* __restrict__ y) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    y[q] = (float)x[q];
}

// out = x + y (in place allowed on y).
static __global__ void add_kernel(long long n, const double* __restrict__ x, double* y) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    y[q] = x[q] + y[q];
}

// EXPRB32 middle stage: R = h (F(a) - F(u)) = -h p1 (D p1) for the quadratic
// Burgers term with p1 = a - u (R = 0 for the linear operator).  p1 is only
// read: a = u + p1 is formed later, by the final pass.
template <int KIND>
__global__ void exprb32_stage_kernel(Geo g, double h, const double* __restrict__ p1, double* __restrict__ R) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < g.n; q += (long long)gridDim.x * blockDim.x) {
    if (KIND == 1) {
      long long e, w, nn, s;
      neighbours(g, q, e, w, nn, s);
      const double dp = (p1[e] - p1[w]) * g.i2dx + (p1[nn] - p1[s]) * g.i2dy;
      R[q] = -h * p1[q] * dp;
    } else {
      R[q] = 0.0;
    }
  }
}

// The EXPRB32 final pass: a = u + p1 (in place of p1, which the remainder's
// stencil has read unmodified), u_high = a + 2 p3 and err = ||2 p3||
// (last-block reduction into st->red).
static __global__ void __launch_bounds__(kThreadsPerBlock)
    exprb32_final_kernel(long long n, const double* __restrict__ u, double* __restrict__ p1_a,
                         const double* __restrict__ p3, double* __restrict__ u_high, double* __restrict__ partials,
                         unsigned int* __restrict__ ticket, LoopState* st) {
  double s = 0.0, dummy = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const double e = 2.0 * p3[q];
    const double a = u[q] + p1_a[q];
    p1_a[q] = a;
    u_high[q] = a + e;
    s = fma(e, e, s);
  }
  if (!last_block_total2(s, dummy, partials, ticket)) return;
  if (threadIdx.x == 0) st->red = sqrt(s / double(n));
}

// EPIRK4s3A: out = c_i P_i (the stage increment U_i - u from phi_1(c_i h J)
// h f(u)), read by the remainder kernels.
static __global__ void scale_kernel(long long n, double s, const double* __restrict__ x, double* __restrict__ y) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    y[q] = s * x[q];
}

// EPIRK4s3A: W3 = b2 R2 + b3 R3 and W4 = e2 R2 + e3 R3, the inputs of the
// phi_3 and phi_4 loops.
static __global__ void epirk_combine_kernel(long long n, const double* __restrict__ R2,
                                            const double* __restrict__ R3, double b2, double b3, double e2,
                                            double e3, double* __restrict__ W3, double* __restrict__ W4) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const double r2 = R2[q], r3 = R3[q];
    W3[q] = b2 * r2 + b3 * r3;
    W4[q] = e2 * r2 + e3 * r3;
  }
}

// EPIRK4s3A final pass: u_low = u + p1 + q3 (in place of p1), u_high =
// u_low + q4 and err = ||q4|| (last-block reduction into st->red).
static __global__ void __launch_bounds__(kThreadsPerBlock)
    epirk_final_kernel(long long n, const double* __restrict__ u, double* __restrict__ p1_low,
                       const double* __restrict__ q3, const double* __restrict__ q4, double* __restrict__ u_high,
                       double* __restrict__ partials, unsigned int* __restrict__ ticket, LoopState* st) {
  double s = 0.0, dummy = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const double e = q4[q];
    const double lo = u[q] + p1_low[q] + q3[q];
    p1_low[q] = lo;
    u_high[q] = lo + e;
    s = fma(e, e, s);
  }
  if (!last_block_total2(s, dummy, partials, ticket)) return;
  if (threadIdx.x == 0) st->red = sqrt(s / double(n));
}

// ||v|| = sqrt(sum v^2 / n) into st->red2 (last-block reduction).
static __global__ void __launch_bounds__(kThreadsPerBlock)
    vec_norm_kernel(long long n, const double* __restrict__ v, double* __restrict__ partials,
                    unsigned int* __restrict__ ticket, LoopState* st) {
  double s = 0.0, dummy = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    s = fma(v[q], v[q], s);
  if (!last_block_total2(s, dummy, partials, ticket)) return;
  if (threadIdx.x == 0) st->red2 = sqrt(s / double(n));
}

// sigma = 1/||v0|| and reset of the power-iteration state.
static __global__ void __launch_bounds__(kThreadsPerBlock)
    power_start_kernel(long long n, const double* __restrict__ v, int pmax, double* __restrict__ partials,
                       unsigned int* __restrict__ ticket, LoopState* st) {
  double s = 0.0, dummy = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    s = fma(v[q], v[q], s);
  if (!last_block_total2(s, dummy, partials, ticket)) return;
  if (threadIdx.x == 0) {
    const double nv = sqrt(s / double(n));
    st->sigma = 1.0 / nv;
    st->pk = 0;
    st->pmax = pmax;
    st->rho = 0.0;
    st->rho_prev = 0.0;
    st->pstatus = 0;
    st->pdone = 0;
    if (!(nv > 0.0) || !isfinite(nv)) {
      st->pstatus = 5;
      st->pdone = 1;
    }
  }
}

// One power-iteration pass: w = Op(v) / ||v||, rho_k = ||w||, stop test
// |rho_k - rho_{k-1}| <= 1e-2 rho_k or k = pmax.
template <int KIND>
static __global__ void __launch_bounds__(kThreadsPerBlock)
    power_pass_kernel(Geo g, double nu, double a, const double* __restrict__ u, const double* __restrict__ sgrad,
                      const double* __restrict__ v, double* __restrict__ w, double* __restrict__ partials,
                      unsigned int* __restrict__ ticket, LoopState* st) {
  if (__ldcg(&st->pdone)) return;
  const double sigma = __ldcg(&st->sigma);
  double s = 0.0, dummy = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < g.n; q += (long long)gridDim.x * blockDim.x) {
    long long e, ww, nn, ss;
    neighbours(g, q, e, ww, nn, ss);
    const double vc = v[q], ve = v[e], vw = v[ww], vn = v[nn], vs = v[ss];
    const double lap = (ve - 2.0 * vc + vw) * g.idx2 + (vn - 2.0 * vc + vs) * g.idy2;
    const double grad = (ve - vw) * g.i2dx + (vn - vs) * g.i2dy;
    double r;
    if (KIND == 0)
      r = nu * lap + a * grad;
    else
      r = nu * lap - vc * sgrad[q] - u[q] * grad;
    r *= sigma;
    w[q] = r;
    s = fma(r, r, s);
  }
  if (!last_block_total2(s, dummy, partials, ticket)) return;
  if (threadIdx.x == 0) {
    const double rho = sqrt(s / double(g.n));
    const int k = st->pk + 1;
    st->pk = k;
    st->rho = rho;
    if (!isfinite(rho) || !(rho > 0.0)) {
      st->pstatus = 5;
      st->pdone = 1;
    } else {
      if ((k >= 2 && fabs(rho - st->rho_prev) <= 1e-2 * rho) || k >= st->pmax) st->pdone = 1;
      st->rho_prev = rho;
      st->sigma = 1.0 / rho;
    }
  }
}

// End of a power-iteration pass (thread 0 of the last block): s = sum w^2
// over the n points of w = Op(v) / ||v||.
__device__ __forceinline__ void power_pass_finish(LoopState* st, double s, long long n) {
  const double rho = sqrt(s / double(n));
  const int k = st->pk + 1;
  st->pk = k;
  st->rho = rho;
  if (!isfinite(rho) || !(rho > 0.0)) {
    st->pstatus = 5;
    st->pdone = 1;
  } else {
    if ((k >= 2 && fabs(rho - st->rho_prev) <= 1e-2 * rho) || k >= st->pmax) st->pdone = 1;
    st->rho_prev = rho;
    st->sigma = 1.0 / rho;
  }
}

}  // namespace lexgb
