// The paper's own discretisation (Sec. 3): periodic [-1,1)^2 with spacing
// 2/nx, 2/ny, the Laplacian by second-order central differences and the
// gradient by the third-order upwind-biased scheme.  Along one axis, for a
// term +a v_x with a > 0 (characteristics toward -x, upwind side +x):
//   (D v)_i = (-v_{i+2} + 6 v_{i+1} - 3 v_i - 2 v_{i-1}) / (6 dx),
// and its mirror image for a < 0.  Writing s = sign(a) and the offsets o s
// (o = -1, 0, 1, 2), a D v_i = |a| / (6 dx) * sum_o k_o v_{i + o s} with
// k = (-2, -3, 6, -1): one stencil of seven points (the centre shared by
// both axes).
//   LX_ADVDIFF_UP3:  A v  = nu lap v + a (D_x + D_y) v
//   LX_BURGERS_UP3:  f(u) = nu lap u + (a/2) (D_x + D_y) (u^2)   (flux form)
//                    J(u) v = nu lap v + a (D_x + D_y) (u v)
// The kernels here are point-wise (one thread per point, neighbours through
// the caches).
#pragma once

#include "leja_df64_2step.cuh"

namespace lexgb {

// k_o of the upwind stencil for o = -1, 0, 1, 2 (scalars: usable in device code)
constexpr double kUp3Km = -2.0, kUp3K0 = -3.0, kUp3K1 = 6.0, kUp3K2 = -1.0;

__device__ __forceinline__ int up3_wrap(int i, int n) {
  // offsets are within [-2, 2]; n >= 1
  while (i < 0) i += n;
  while (i >= n) i -= n;
  return i;
}

// Indices of the seven stencil points of (i, j): [C, X(-s), X(s), X(2s),
// Y(-s), Y(s), Y(2s)].
__device__ __forceinline__ void up3_points(const Up3Op& o, int i, int j, long long (&q)[7]) {
  const int s = o.s;
  const long long row = (long long)j * o.nx;
  q[0] = row + i;
  q[1] = row + up3_wrap(i - s, o.nx);
  q[2] = row + up3_wrap(i + s, o.nx);
  q[3] = row + up3_wrap(i + 2 * s, o.nx);
  q[4] = (long long)up3_wrap(j - s, o.ny) * o.nx + i;
  q[5] = (long long)up3_wrap(j + s, o.ny) * o.nx + i;
  q[6] = (long long)up3_wrap(j + 2 * s, o.ny) * o.nx + i;
}

// Constant weights of A (diffusion-advection) at the seven points.
__device__ __forceinline__ void up3_weights(const Up3Op& o, double (&w)[7]) {
  w[0] = -2.0 * o.cxx - 2.0 * o.cyy + kUp3K0 * (o.gx + o.gy);
  w[1] = o.cxx + kUp3Km * o.gx;
  w[2] = o.cxx + kUp3K1 * o.gx;
  w[3] = kUp3K2 * o.gx;
  w[4] = o.cyy + kUp3Km * o.gy;
  w[5] = o.cyy + kUp3K1 * o.gy;
  w[6] = kUp3K2 * o.gy;
}

// Op(v) at one point: A v (BURGERS = false) or J(u) v (BURGERS = true); for
// the right-hand side of Burgers pass v = u and half = true, which gives
// nu lap u + (a/2) D(u^2).
template <bool BURGERS, typename T, typename V>
__device__ __forceinline__ T up3_apply(const Up3Op& o, const double* __restrict__ u, const V* __restrict__ v,
                                       const long long (&q)[7], bool half = false) {
  T vv[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) vv[k] = T(v[q[k]]);
  const T lap = T(o.cxx) * (vv[1] + vv[2] - T(2) * vv[0]) + T(o.cyy) * (vv[4] + vv[5] - T(2) * vv[0]);
  T dx, dy;
  if constexpr (BURGERS) {
    T uu[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) uu[k] = T(u[q[k]]);
    const T f = half ? T(0.5) : T(1);
    dx = T(kUp3Km) * uu[1] * vv[1] + T(kUp3K0) * uu[0] * vv[0] + T(kUp3K1) * uu[2] * vv[2] +
         T(kUp3K2) * uu[3] * vv[3];
    dy = T(kUp3Km) * uu[4] * vv[4] + T(kUp3K0) * uu[0] * vv[0] + T(kUp3K1) * uu[5] * vv[5] +
         T(kUp3K2) * uu[6] * vv[6];
    return lap + f * (T(o.gx) * dx + T(o.gy) * dy);
  } else {
    dx = T(kUp3Km) * vv[1] + T(kUp3K0) * vv[0] + T(kUp3K1) * vv[2] + T(kUp3K2) * vv[3];
    dy = T(kUp3Km) * vv[4] + T(kUp3K0) * vv[0] + T(kUp3K1) * vv[5] + T(kUp3K2) * vv[6];
    return lap + T(o.gx) * dx + T(o.gy) * dy;
  }
}

// Point (i, j) of flat index q for q < 2^31 (checked at setup).
__device__ __forceinline__ void up3_ij(const Up3Op& o, long long q, int& i, int& j) {
  const unsigned qq = (unsigned)q;
  j = (int)(qq / (unsigned)o.nx);
  i = (int)(qq - (unsigned)j * (unsigned)o.nx);
}

// One fused Leja iteration on the upwind operators (FP64 / mixed basis):
// y_{m+1} = (Op y_m - c y_m)/gamma - xi_m y_m, p_{m+1} = p_m + d_{m+1} y_{m+1},
// the two norms, and the stop test in the last block.
template <bool BURGERS, typename T>
static __global__ void __launch_bounds__(kThreadsPerBlock)
    leja_iter_up3_kernel(const LoopArgs* __restrict__ Ap, LoopState* __restrict__ st, double* __restrict__ partials,
                         unsigned int* __restrict__ ticket, cudaGraphConditionalHandle cond) {
  const LoopArgs& A = *Ap;
  const int m = __ldcg(&st->m);
  count_launch(st);
  if (__ldcg(&st->done)) return;
  const Up3Op o = A.up;
  const double xim = __ldg(A.xi + m);
  const double dm1 = __ldg(A.d + m + 1);
  const double d0 = __ldg(A.d);
  const T ig = T(A.inv_gamma);
  const T cs = T(-A.up_c * A.inv_gamma - xim);  // -c/gamma - xi_m
  T* dst = reinterpret_cast<T*>((m & 1) ? A.y1 : A.y0);
  const T* src = reinterpret_cast<const T*>(((m - 1) & 1) ? A.y1 : A.y0);
  double sy = 0.0, sp = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < o.n; q += (long long)gridDim.x * blockDim.x) {
    int i, j;
    up3_ij(o, q, i, j);
    long long pts[7];
    up3_points(o, i, j, pts);
    T v, yc;
    if (m == 0) {
      v = up3_apply<BURGERS, T, double>(o, A.u, A.w, pts);
      yc = T(__ldg(A.w + q));
    } else {
      v = up3_apply<BURGERS, T, T>(o, A.u, src, pts);
      yc = src[q];
    }
    v = ig * v + cs * yc;
    dst[q] = v;
    const double vd = to_double(v);
    const double po = m == 0 ? d0 * double(yc) : A.p[q];
    const double pn = fma(dm1, vd, po);
    A.p[q] = pn;
    sy = fma(vd, vd, sy);
    sp = fma(pn, pn, sp);
  }
  if (!last_block_total2(sy, sp, partials, ticket)) return;
  if (threadIdx.x == 0) leja_finalize(A, st, m, dm1, sy, sp, 1.0, 1.0, cond);
}

// Float-float form of the upwind diffusion-advection iteration (constant
// weights, Dot2 over the seven points; storage scaling as the other df64
// kernels: stored y_m = y_m 2^-sig, p in 2^-kscale units, the new basis
// vector renormalised by 2^-dlt).  The final renormalisation is Fast2Sum:
// exact when |s| >= |c|; otherwise s has cancelled below the correction c,
// itself of order u sum |w_k y_k|, and the pair misses s + c by at most a
// unit roundoff of |c| -- the order of Dot2's own bound u^2 sum |w_k y_k|.
__device__ __forceinline__ dfv df_dot7(const float (&wh)[7], const float (&wl)[7], const dfv (&y)[7]) {
  float s, c, p, e, t;
  two_prod(wh[0], y[0].h, s, c);
#pragma unroll
  for (int k = 1; k < 7; ++k) {
    two_prod(wh[k], y[k].h, p, e);
    two_sum(s, p, s, t);
    c = __fadd_rn(c, __fadd_rn(t, e));
  }
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    c = __fmaf_rn(wh[k], y[k].l, c);
    c = __fmaf_rn(wl[k], y[k].h, c);
  }
  dfv r;
  fast_two_sum(s, c, r.h, r.l);
  return r;
}

static __global__ void __launch_bounds__(kThreadsPerBlock)
    leja_iter_df_up3_kernel(const LoopArgs* __restrict__ Ap, LoopState* __restrict__ st,
                            double* __restrict__ partials, unsigned int* __restrict__ ticket,
                            cudaGraphConditionalHandle cond) {
  const LoopArgs& A = *Ap;
  const int m = __ldcg(&st->m);
  count_launch(st);
  if (__ldcg(&st->done)) return;
  const int kexp = __ldcg(&st->kscale);
  const int sig = __ldcg(&st->sig);
  const int dlt = __ldcg(&st->dlt);
  const Up3Op o = A.up;
  const double xim = __ldg(A.xi + m);
  const double dm1d = __ldg(A.d + m + 1);
  const dfv dm1 = df_from_double(dm1d * pow2(sig + dlt - kexp));
  const dfv d0 = df_from_double(__ldg(A.d));
  const double sw = pow2(-dlt);
  double wd[7];
  up3_weights(o, wd);
  float wh[7], wl[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    double wk = wd[k] * A.inv_gamma;
    if (k == 0) wk += -A.up_c * A.inv_gamma - xim;
    const dfv t = df_from_double(wk * sw);
    wh[k] = t.h;
    wl[k] = t.l;
  }
  float2* dst = reinterpret_cast<float2*>((m & 1) ? A.y1 : A.y0);
  const float2* src = reinterpret_cast<const float2*>(((m - 1) & 1) ? A.y1 : A.y0);
  dfv accy = {0.f, 0.f}, accp = {0.f, 0.f};
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < o.n; q += (long long)gridDim.x * blockDim.x) {
    int i, j;
    up3_ij(o, q, i, j);
    long long pts[7];
    up3_points(o, i, j, pts);
    dfv t[7];
    if (m == 0) {
#pragma unroll
      for (int k = 0; k < 7; ++k) t[k] = df_split_scaled(__ldg(A.w + pts[k]), kexp);
    } else {
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        const float2 f = __ldg(src + pts[k]);
        t[k] = {f.x, f.y};
      }
    }
    const dfv v = df_dot7(wh, wl, t);
    dst[q] = make_float2(v.h, v.l);
    dfv po;
    if (m == 0) {
      po = df_mul(d0, t[0]);
    } else {
      const float2 f = A.pdf[q];
      po = {f.x, f.y};
    }
    const dfv pn = df_axpy(dm1, v, po);
    A.pdf[q] = make_float2(pn.h, pn.l);
    df_acc(accy, __fmul_rn(v.h, v.h));
    df_acc(accp, __fmul_rn(pn.h, pn.h));
  }
  double sy = df_to_double(accy), sp = df_to_double(accp);
  if (!last_block_total2(sy, sp, partials, ticket)) return;
  if (threadIdx.x == 0) {
    leja_finalize(A, st, m, dm1d, sy, sp, pow2(sig + dlt), pow2(kexp), cond);
    const double rms = sqrt(sy / double(A.n));
    int e = 0;
    if (rms > 0.0 && isfinite(rms)) e = ilogb(rms);
    st->sig = sig + dlt;
    st->dlt = max(-100, min(100, e));
  }
}

// h (f(u) + S) for the upwind operators.
template <bool BURGERS>
static __global__ void __launch_bounds__(kThreadsPerBlock)
    rhs_up3_kernel(Up3Op o, double h, const double* __restrict__ u, const double* __restrict__ src,
                   double* __restrict__ f_out) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < o.n; q += (long long)gridDim.x * blockDim.x) {
    int i, j;
    up3_ij(o, q, i, j);
    long long pts[7];
    up3_points(o, i, j, pts);
    double f = up3_apply<BURGERS, double, double>(o, u, u, pts, true);
    if (src) f += src[q];
    f_out[q] = h * f;
  }
}

// h (A u + S) for the upwind diffusion-advection operator on the FP32 pipe:
// float-float Dot2 over the seven points with the weights h w_k, rounded to
// double, plus h S in double; records the largest exponent of the result for
// the Leja loop's input scaling.  Points whose neighbours lie outside the
// float-float range (|u| beyond 2^+-100) take the FP64 formula.
static __global__ void __launch_bounds__(kThreadsPerBlock)
    rhs_df_up3_kernel(Up3Op o, double h, const double* __restrict__ u, const double* __restrict__ src,
                      double* __restrict__ f_out, LoopState* st) {
  double wd[7];
  up3_weights(o, wd);
  float wh[7], wl[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    wd[k] *= h;
    const dfv t = df_from_double(wd[k]);
    wh[k] = t.h;
    wl[k] = t.l;
  }
  int emax = 0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < o.n; q += (long long)gridDim.x * blockDim.x) {
    int i, j;
    up3_ij(o, q, i, j);
    long long pts[7];
    up3_points(o, i, j, pts);
    double v[7];
    bool in_range = true;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      v[k] = __ldg(u + pts[k]);
      const int ex = (int)((__double_as_longlong(v[k]) >> 52) & 0x7ff);
      in_range = in_range && (ex == 0 || (ex > 1023 - 100 && ex < 1023 + 100));
    }
    double r;
    if (in_range) {
      dfv t[7];
#pragma unroll
      for (int k = 0; k < 7; ++k) t[k] = df_split_scaled(v[k], 0);
      const dfv d = df_dot7(wh, wl, t);
      r = f2d_scaled(d.h, 0) + f2d_scaled(d.l, 0);
    } else {
      r = 0.0;
#pragma unroll
      for (int k = 0; k < 7; ++k) r = fma(wd[k], v[k], r);
    }
    if (src) r = r + h * __ldg(src + q);
    f_out[q] = r;
    emax = max(emax, (int)((__double2hiint(r) >> 20) & 0x7ff));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, off));
  if ((threadIdx.x & 31) == 0) atomicMax(&st->wexp, emax);
}

// EXPRB32 remainder for the upwind Burgers operator: with p1 = a - u,
// F(a) - F(u) = (a/2) D(p1^2) exactly (quadratic flux), so R = h (a/2) D(p1^2);
// R = 0 for the linear operator.
template <bool BURGERS>
static __global__ void __launch_bounds__(kThreadsPerBlock)
    exprb32_stage_up3_kernel(Up3Op o, double h, const double* __restrict__ p1, double* __restrict__ R) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < o.n; q += (long long)gridDim.x * blockDim.x) {
    if constexpr (BURGERS) {
      int i, j;
      up3_ij(o, q, i, j);
      long long pts[7];
      up3_points(o, i, j, pts);
      double sq[7];
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        const double v = p1[pts[k]];
        sq[k] = v * v;
      }
      const double dx = kUp3Km * sq[1] + kUp3K0 * sq[0] + kUp3K1 * sq[2] + kUp3K2 * sq[3];
      const double dy = kUp3Km * sq[4] + kUp3K0 * sq[0] + kUp3K1 * sq[5] + kUp3K2 * sq[6];
      R[q] = h * 0.5 * (o.gx * dx + o.gy * dy);
    } else {
      R[q] = 0.0;
    }
  }
}

// One power-iteration pass on the upwind operators: w = Op(v) / ||v||.
template <bool BURGERS>
static __global__ void __launch_bounds__(kThreadsPerBlock)
    power_pass_up3_kernel(Up3Op o, const double* __restrict__ u, const double* __restrict__ v, double* __restrict__ w,
                          double* __restrict__ partials, unsigned int* __restrict__ ticket, LoopState* st) {
  if (__ldcg(&st->pdone)) return;
  const double sigma = __ldcg(&st->sigma);
  double s = 0.0, dummy = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < o.n; q += (long long)gridDim.x * blockDim.x) {
    int i, j;
    up3_ij(o, q, i, j);
    long long pts[7];
    up3_points(o, i, j, pts);
    const double r = up3_apply<BURGERS, double, double>(o, u, v, pts) * sigma;
    w[q] = r;
    s = fma(r, r, s);
  }
  if (!last_block_total2(s, dummy, partials, ticket)) return;
  if (threadIdx.x == 0) power_pass_finish(st, s, o.n);
}

}  // namespace lexgb

namespace lexgb {

// ---------------------------------------------------------------------------
// Pipelined float-float iteration for the upwind diffusion-advection
// operator (nx % 128 == 0): the same warp-per-row-range layout as the
// central-difference pipelined kernel.  Rows r0-2 .. r1+1 stream through a
// shared-memory ring (two-point column halos); each lane keeps its four
// points of five consecutive rows in registers, so the seven-point stencil
// takes its y-neighbours from the register window and its x-neighbours from
// the centre row (shuffles, and the ring's halo for lanes 0 and 31).
// ---------------------------------------------------------------------------
constexpr int kUpStages = 7;  // ring slots per warp (two rows in flight)
constexpr int kUpSmemBytes = kPipeWarps * kUpStages * kSlotElems2 * 8;

// SG: the upwind side (+1 or -1), a template parameter so that the choice
// of the stencil points costs no per-point selects.  POWER: one
// power-iteration pass instead (w = A v * sg, no polynomial, sum w^2 to
// double accuracy in accy and *small).
template <typename S, bool FIRST, int SG, bool POWER = false>
__device__ __forceinline__ void df_strip_up3(const LoopArgs& A, const S* __restrict__ src, float2* __restrict__ dst,
                                             float2* __restrict__ p, unsigned long long* ring, int col0, int r0,
                                             int r1, const float (&wh)[7], const float (&wl)[7], dfv d0, dfv dm1,
                                             int sc, dfv& accy, dfv& accp, dfv sg = dfv{0.f, 0.f},
                                             float* small = nullptr) {
  constexpr int s = SG;
  const int lane = threadIdx.x & 31;
  const int nx = A.nx, ny = A.ny;
  const int c = col0 + lane * 4;
  const int cw = col0 == 0 ? nx - 2 : col0 - 2;
  const int ce = (col0 + kPipeRow >= nx) ? 0 : col0 + kPipeRow;
  const int nrows = r1 - r0;
  const int last_q = nrows + 3;  // rows q = 0 .. nrows+3 are r0-2 .. r1+1
  auto slot = [&](int q) { return ring + (size_t)(q % kUpStages) * kSlotElems2; };
  auto issue = [&](int q) {
    if (q <= last_q) {
      const int ry = wrap_row(r0 - 2 + q, ny);
      unsigned long long* sl = slot(q);
      const S* row = src + (size_t)ry * nx;
      cp_async16(sl + 2 + lane * 4, row + c);
      cp_async16(sl + 4 + lane * 4, row + c + 2);
      if (lane == 0) cp_async16(sl, row + cw);
      if (lane == 31) cp_async16(sl + 2 + kPipeRow, row + ce);
      if constexpr (!FIRST && !POWER) {
        if (q >= 4) {  // p of output row r0 + q - 4 arrives with y row r0 + q - 2
          const float2* prow = p + (size_t)(r0 + q - 4) * nx;
          cp_async16(sl + kY2Slot + lane * 4, prow + c);
          cp_async16(sl + kY2Slot + lane * 4 + 2, prow + c + 2);
        }
      }
    }
    cp_commit();
  };
  // window rows: w0..w4 = grid rows r-2 .. r+2 of output row r
  dfv w0[4], w1[4], w2[4], w3[4], w4[4];
  for (int q = 0; q < kUpStages - 1; ++q) issue(q);
  cp_wait<kUpStages - 5>();  // rows 0..3 complete
  __syncwarp();
  df_from_raw4<S>(slot(0) + 2 + lane * 4, sc, w0);
  df_from_raw4<S>(slot(1) + 2 + lane * 4, sc, w1);
  df_from_raw4<S>(slot(2) + 2 + lane * 4, sc, w2);
  df_from_raw4<S>(slot(3) + 2 + lane * 4, sc, w3);
  for (int a = 0; a < nrows; ++a) {
    issue(a + kUpStages - 1);
    cp_wait<kUpStages - 5>();  // row a+4 complete
    __syncwarp();
    const unsigned long long* sn = slot(a + 4);
    const unsigned long long* sc2 = slot(a + 2);  // centre row: halo points
    df_from_raw4<S>(sn + 2 + lane * 4, sc, w4);
    dfv pold[4];
    if constexpr (!FIRST && !POWER) df_from_raw4<float2>(sn + kY2Slot + lane * 4, 0, pold);
    // x-neighbours of the centre row
    const dfv u3 = shfl_up_df(w2[3]), u2 = shfl_up_df(w2[2]);
    const dfv d0n = shfl_down_df(w2[0]), d1n = shfl_down_df(w2[1]);
    // (lane 0 / lane 31 read their halo from the ring; the selects keep the
    // shuffles above outside any divergent branch)
    const dfv hw1 = df_from_raw<S>(sc2 + 1, sc), hw2 = df_from_raw<S>(sc2 + 0, sc);
    const dfv he1 = df_from_raw<S>(sc2 + 2 + kPipeRow, sc), he2 = df_from_raw<S>(sc2 + 3 + kPipeRow, sc);
    const dfv wm1 = lane == 0 ? hw1 : u3, wm2 = lane == 0 ? hw2 : u2;  // columns c-1, c-2
    const dfv ep1 = lane == 31 ? he1 : d0n, ep2 = lane == 31 ? he2 : d1n;  // columns c+4, c+5
    const dfv xm1[4] = {wm1, w2[0], w2[1], w2[2]};
    const dfv xm2[4] = {wm2, wm1, w2[0], w2[1]};
    const dfv xp1[4] = {w2[1], w2[2], w2[3], ep1};
    const dfv xp2[4] = {w2[2], w2[3], ep1, ep2};
    dfv ynew[4], pnew[4];
    float fy = 0.f, fp = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      // [C, X(-s), X(s), X(2s), Y(-s), Y(s), Y(2s)]
      const dfv t[7] = {w2[k],
                        s > 0 ? xm1[k] : xp1[k],
                        s > 0 ? xp1[k] : xm1[k],
                        s > 0 ? xp2[k] : xm2[k],
                        s > 0 ? w1[k] : w3[k],
                        s > 0 ? w3[k] : w1[k],
                        s > 0 ? w4[k] : w0[k]};
      ynew[k] = df_dot7(wh, wl, t);
      if constexpr (POWER) {
        ynew[k] = df_mul(sg, ynew[k]);
        float sq, se;
        two_prod(ynew[k].h, ynew[k].h, sq, se);
        df_acc(accy, sq);
        *small = __fmaf_rn(2.f * ynew[k].h, ynew[k].l, __fadd_rn(*small, se));
      } else {
        const dfv po = FIRST ? df_mul(d0, w2[k]) : pold[k];
        pnew[k] = df_axpy(dm1, ynew[k], po);
        fy = __fmaf_rn(ynew[k].h, ynew[k].h, fy);
        fp = __fmaf_rn(pnew[k].h, pnew[k].h, fp);
      }
    }
    const size_t ro = (size_t)(r0 + a) * nx;
    df_store_row<4>(dst + ro, c, nx, ynew);
    if constexpr (!POWER) {
      df_acc(accy, fy);
      df_acc(accp, fp);
      df_store_row<4>(p + ro, c, nx, pnew);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      w0[k] = w1[k];
      w1[k] = w2[k];
      w2[k] = w3[k];
      w3[k] = w4[k];
    }
    __syncwarp();
  }
  cp_wait<0>();
  __syncwarp();
}

template <int MINB>
__global__ void __launch_bounds__(kPipeThreads, MINB)
    leja_iter_df_pipe_up3_kernel(const LoopArgs* __restrict__ Ap, LoopState* __restrict__ st,
                                 double* __restrict__ partials, unsigned int* __restrict__ ticket,
                                 cudaGraphConditionalHandle cond) {
  extern __shared__ __align__(16) unsigned long long up3_smem[];
  const LoopArgs& A = *Ap;
  const int m = __ldcg(&st->m);
  count_launch(st);
  if (__ldcg(&st->done)) return;
  const int kexp = __ldcg(&st->kscale);
  const int sig = __ldcg(&st->sig);
  const int dlt = __ldcg(&st->dlt);
  const Up3Op o = A.up;
  const double xim = __ldg(A.xi + m);
  const double dm1d = __ldg(A.d + m + 1);
  const dfv dm1 = df_from_double(dm1d * pow2(sig + dlt - kexp));
  const dfv d0 = df_from_double(__ldg(A.d));
  const double sw = pow2(-dlt);
  double wd[7];
  up3_weights(o, wd);
  float wh[7], wl[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    double wk = wd[k] * A.inv_gamma;
    if (k == 0) wk += -A.up_c * A.inv_gamma - xim;
    const dfv t = df_from_double(wk * sw);
    wh[k] = t.h;
    wl[k] = t.l;
  }
  float2* dst = reinterpret_cast<float2*>((m & 1) ? A.y1 : A.y0);
  const float2* src = reinterpret_cast<const float2*>(((m - 1) & 1) ? A.y1 : A.y0);
  dfv accy = {0.f, 0.f}, accp = {0.f, 0.f};
  const int warp = threadIdx.x >> 5;
  unsigned long long* ring = up3_smem + (size_t)warp * kUpStages * kSlotElems2;
  for_each_segment(o.nx, o.ny, A.strip_h, blockIdx.x * kPipeWarps + warp, gridDim.x * kPipeWarps,
                   [&](int col0, int r0, int r1) {
    if (m == 0) {
      if (o.s > 0)
        df_strip_up3<double, true, 1>(A, A.w, dst, A.pdf, ring, col0, r0, r1, wh, wl, d0, dm1, kexp, accy, accp);
      else
        df_strip_up3<double, true, -1>(A, A.w, dst, A.pdf, ring, col0, r0, r1, wh, wl, d0, dm1, kexp, accy, accp);
    } else {
      if (o.s > 0)
        df_strip_up3<float2, false, 1>(A, src, dst, A.pdf, ring, col0, r0, r1, wh, wl, d0, dm1, kexp, accy, accp);
      else
        df_strip_up3<float2, false, -1>(A, src, dst, A.pdf, ring, col0, r0, r1, wh, wl, d0, dm1, kexp, accy, accp);
    }
  });
  double sy = df_to_double(accy), sp = df_to_double(accp);
  if (!last_block_total2(sy, sp, partials, ticket)) return;
  if (threadIdx.x == 0) {
    leja_finalize(A, st, m, dm1d, sy, sp, pow2(sig + dlt), pow2(kexp), cond);
    const double rms = sqrt(sy / double(A.n));
    int e = 0;
    if (rms > 0.0 && isfinite(rms)) e = ilogb(rms);
    st->sig = sig + dlt;
    st->dlt = max(-100, min(100, e));
  }
}

}  // namespace lexgb

namespace lexgb {

// ---------------------------------------------------------------------------
// Pipelined float-float iteration for the upwind Burgers Jacobian
// J(u) v = nu lap v + a (D_x + D_y)(u v)  (nx % 128 == 0).  With
// q = u |a| / (6 dx gamma) as float pairs (prepared once per Leja loop) and
// rat = dx/dy, the weight of v at the point o s of the x stencil is
// lx [o = +-1] + k_o q (and lap centre terms at o = 0), on the y stencil
// ly [o = +-1] + k_o rat q, so each point needs q on the same seven points
// as y: q streams through the ring beside y with the same two-point halos.
// ---------------------------------------------------------------------------
constexpr int kSlotElemsUB = 2 * kY2Slot + kPipeRow;  // y (halo 2), q (halo 2), p
constexpr int kUpSmemBytesB = kPipeWarps * kUpStages * kSlotElemsUB * 8;

// q = u * scale as float pairs.
static __global__ void __launch_bounds__(kThreadsPerBlock)
    up3_df_prep_kernel(long long n, const double* __restrict__ u, double scale, float2* __restrict__ q) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const dfv a = df_split_scaled(u[i] * scale, 0);
    q[i] = make_float2(a.h, a.l);
  }
}

__device__ __forceinline__ dfv df_scale_f(dfv a, float k) {  // a * k, k a small integer
  float p, e;
  two_prod(a.h, k, p, e);
  e = __fmaf_rn(a.l, k, e);
  dfv r;
  fast_two_sum(p, e, r.h, r.l);
  return r;
}

template <typename S, bool FIRST, int SG>
__device__ __forceinline__ void df_strip_burgers_up3(const LoopArgs& A, const S* __restrict__ src,
                                                     float2* __restrict__ dst, float2* __restrict__ p,
                                                     unsigned long long* ring, int col0, int r0, int r1, dfv cc0,
                                                     dfv lxs, dfv lys, dfv rat, bool square, float swf, dfv d0,
                                                     dfv dm1, int sc, dfv& accy, dfv& accp) {
  constexpr int s = SG;
  const int lane = threadIdx.x & 31;
  const int nx = A.nx, ny = A.ny;
  const int c = col0 + lane * 4;
  const int cw = col0 == 0 ? nx - 2 : col0 - 2;
  const int ce = (col0 + kPipeRow >= nx) ? 0 : col0 + kPipeRow;
  const int nrows = r1 - r0;
  const int last_q = nrows + 3;
  auto slot = [&](int q) { return ring + (size_t)(q % kUpStages) * kSlotElemsUB; };
  auto issue = [&](int q) {
    if (q <= last_q) {
      const int ry = wrap_row(r0 - 2 + q, ny);
      unsigned long long* sl = slot(q);
      const S* row = src + (size_t)ry * nx;
      cp_async16(sl + 2 + lane * 4, row + c);
      cp_async16(sl + 4 + lane * 4, row + c + 2);
      if (lane == 0) cp_async16(sl, row + cw);
      if (lane == 31) cp_async16(sl + 2 + kPipeRow, row + ce);
      const float2* qrow = A.bq + (size_t)ry * nx;
      unsigned long long* sq = sl + kY2Slot;
      cp_async16(sq + 2 + lane * 4, qrow + c);
      cp_async16(sq + 4 + lane * 4, qrow + c + 2);
      if (lane == 0) cp_async16(sq, qrow + cw);
      if (lane == 31) cp_async16(sq + 2 + kPipeRow, qrow + ce);
      if constexpr (!FIRST) {
        if (q >= 4) {
          const float2* prow = p + (size_t)(r0 + q - 4) * nx;
          unsigned long long* sp = sl + 2 * kY2Slot;
          cp_async16(sp + lane * 4, prow + c);
          cp_async16(sp + lane * 4 + 2, prow + c + 2);
        }
      }
    }
    cp_commit();
  };
  dfv w0[4], w1[4], w2[4], w3[4], w4[4];   // y rows r-2 .. r+2
  dfv g0[4], g1[4], g2[4], g3[4], g4[4];   // q rows r-2 .. r+2
  for (int q = 0; q < kUpStages - 1; ++q) issue(q);
  cp_wait<kUpStages - 5>();
  __syncwarp();
  df_from_raw4<S>(slot(0) + 2 + lane * 4, sc, w0);
  df_from_raw4<S>(slot(1) + 2 + lane * 4, sc, w1);
  df_from_raw4<S>(slot(2) + 2 + lane * 4, sc, w2);
  df_from_raw4<S>(slot(3) + 2 + lane * 4, sc, w3);
  df_from_raw4<float2>(slot(0) + kY2Slot + 2 + lane * 4, 0, g0);
  df_from_raw4<float2>(slot(1) + kY2Slot + 2 + lane * 4, 0, g1);
  df_from_raw4<float2>(slot(2) + kY2Slot + 2 + lane * 4, 0, g2);
  df_from_raw4<float2>(slot(3) + kY2Slot + 2 + lane * 4, 0, g3);
  for (int a = 0; a < nrows; ++a) {
    issue(a + kUpStages - 1);
    cp_wait<kUpStages - 5>();
    __syncwarp();
    const unsigned long long* sn = slot(a + 4);
    const unsigned long long* sc2 = slot(a + 2);
    df_from_raw4<S>(sn + 2 + lane * 4, sc, w4);
    df_from_raw4<float2>(sn + kY2Slot + 2 + lane * 4, 0, g4);
    dfv pold[4];
    if constexpr (!FIRST) df_from_raw4<float2>(sn + 2 * kY2Slot + lane * 4, 0, pold);
    // x-neighbours of the centre row, of y and of q (shuffles outside any
    // divergent branch; lanes 0 and 31 take the ring's halo)
    const dfv yu3 = shfl_up_df(w2[3]), yu2 = shfl_up_df(w2[2]);
    const dfv yd0 = shfl_down_df(w2[0]), yd1 = shfl_down_df(w2[1]);
    const dfv qu3 = shfl_up_df(g2[3]), qu2 = shfl_up_df(g2[2]);
    const dfv qd0 = shfl_down_df(g2[0]), qd1 = shfl_down_df(g2[1]);
    const unsigned long long* hq = sc2 + kY2Slot;
    const dfv ym1 = lane == 0 ? df_from_raw<S>(sc2 + 1, sc) : yu3, ym2 = lane == 0 ? df_from_raw<S>(sc2, sc) : yu2;
    const dfv yp1 = lane == 31 ? df_from_raw<S>(sc2 + 2 + kPipeRow, sc) : yd0;
    const dfv yp2 = lane == 31 ? df_from_raw<S>(sc2 + 3 + kPipeRow, sc) : yd1;
    const dfv qm1 = lane == 0 ? df_from_raw<float2>(hq + 1, 0) : qu3, qm2 = lane == 0 ? df_from_raw<float2>(hq, 0) : qu2;
    const dfv qp1 = lane == 31 ? df_from_raw<float2>(hq + 2 + kPipeRow, 0) : qd0;
    const dfv qp2 = lane == 31 ? df_from_raw<float2>(hq + 3 + kPipeRow, 0) : qd1;
    const dfv yxm1[4] = {ym1, w2[0], w2[1], w2[2]}, yxm2[4] = {ym2, ym1, w2[0], w2[1]};
    const dfv yxp1[4] = {w2[1], w2[2], w2[3], yp1}, yxp2[4] = {w2[2], w2[3], yp1, yp2};
    const dfv qxm1[4] = {qm1, g2[0], g2[1], g2[2]}, qxm2[4] = {qm2, qm1, g2[0], g2[1]};
    const dfv qxp1[4] = {g2[1], g2[2], g2[3], qp1}, qxp2[4] = {g2[2], g2[3], qp1, qp2};
    dfv ynew[4], pnew[4];
    float fy = 0.f, fp = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      // stencil points [C, X(-s), X(s), X(2s), Y(-s), Y(s), Y(2s)] of y and q
      const dfv yv[7] = {w2[k], s > 0 ? yxm1[k] : yxp1[k], s > 0 ? yxp1[k] : yxm1[k], s > 0 ? yxp2[k] : yxm2[k],
                         s > 0 ? w1[k] : w3[k], s > 0 ? w3[k] : w1[k], s > 0 ? w4[k] : w0[k]};
      const dfv qv[7] = {g2[k], s > 0 ? qxm1[k] : qxp1[k], s > 0 ? qxp1[k] : qxm1[k], s > 0 ? qxp2[k] : qxm2[k],
                         s > 0 ? g1[k] : g3[k], s > 0 ? g3[k] : g1[k], s > 0 ? g4[k] : g0[k]};
      dfv qy[7];
#pragma unroll
      for (int j = 4; j < 7; ++j) qy[j] = square ? qv[j] : df_mul(qv[j], rat);
      const dfv qcy = square ? qv[0] : df_mul(qv[0], rat);
      dfv wv[7];
      wv[0] = df_add(cc0, df_scale_f(df_add(qv[0], qcy), (float)kUp3K0));
      wv[1] = df_add(lxs, df_scale_f(qv[1], (float)kUp3Km));
      wv[2] = df_add(lxs, df_scale_f(qv[2], (float)kUp3K1));
      wv[3] = df_scale_f(qv[3], (float)kUp3K2);
      wv[4] = df_add(lys, df_scale_f(qy[4], (float)kUp3Km));
      wv[5] = df_add(lys, df_scale_f(qy[5], (float)kUp3K1));
      wv[6] = df_scale_f(qy[6], (float)kUp3K2);
      float wh[7], wl[7];
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        wh[j] = wv[j].h;
        wl[j] = wv[j].l;
      }
      dfv v = df_dot7(wh, wl, yv);
      v.h *= swf;
      v.l *= swf;
      ynew[k] = v;
      const dfv po = FIRST ? df_mul(d0, w2[k]) : pold[k];
      pnew[k] = df_axpy(dm1, v, po);
      fy = __fmaf_rn(v.h, v.h, fy);
      fp = __fmaf_rn(pnew[k].h, pnew[k].h, fp);
    }
    df_acc(accy, fy);
    df_acc(accp, fp);
    const size_t ro = (size_t)(r0 + a) * nx;
    df_store_row<4>(dst + ro, c, nx, ynew);
    df_store_row<4>(p + ro, c, nx, pnew);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      w0[k] = w1[k];
      w1[k] = w2[k];
      w2[k] = w3[k];
      w3[k] = w4[k];
      g0[k] = g1[k];
      g1[k] = g2[k];
      g2[k] = g3[k];
      g3[k] = g4[k];
    }
    __syncwarp();
  }
  cp_wait<0>();
  __syncwarp();
}

template <int MINB>
__global__ void __launch_bounds__(kPipeThreads, MINB)
    leja_iter_df_pipe_burgers_up3_kernel(const LoopArgs* __restrict__ Ap, LoopState* __restrict__ st,
                                         double* __restrict__ partials, unsigned int* __restrict__ ticket,
                                         cudaGraphConditionalHandle cond) {
  extern __shared__ __align__(16) unsigned long long up3b_smem[];
  const LoopArgs& A = *Ap;
  const int m = __ldcg(&st->m);
  count_launch(st);
  if (__ldcg(&st->done)) return;
  const int kexp = __ldcg(&st->kscale);
  const int sig = __ldcg(&st->sig);
  const int dlt = __ldcg(&st->dlt);
  const Up3Op o = A.up;
  const double xim = __ldg(A.xi + m);
  const double dm1d = __ldg(A.d + m + 1);
  const dfv dm1 = df_from_double(dm1d * pow2(sig + dlt - kexp));
  const dfv d0 = df_from_double(__ldg(A.d));
  const float swf = (float)pow2(-dlt);
  const double ig = A.inv_gamma;
  const dfv cc0 = df_from_double((-2.0 * o.cxx - 2.0 * o.cyy - A.up_c) * ig - xim);
  const dfv lxs = df_from_double(o.cxx * ig), lys = df_from_double(o.cyy * ig);
  const dfv rat = df_from_double(o.gy / o.gx);
  const bool square = o.gx == o.gy;
  float2* dst = reinterpret_cast<float2*>((m & 1) ? A.y1 : A.y0);
  const float2* src = reinterpret_cast<const float2*>(((m - 1) & 1) ? A.y1 : A.y0);
  dfv accy = {0.f, 0.f}, accp = {0.f, 0.f};
  const int warp = threadIdx.x >> 5;
  unsigned long long* ring = up3b_smem + (size_t)warp * kUpStages * kSlotElemsUB;
  for_each_segment(o.nx, o.ny, A.strip_h, blockIdx.x * kPipeWarps + warp, gridDim.x * kPipeWarps,
                   [&](int col0, int r0, int r1) {
    if (m == 0) {
      if (o.s > 0)
        df_strip_burgers_up3<double, true, 1>(A, A.w, dst, A.pdf, ring, col0, r0, r1, cc0, lxs, lys, rat, square,
                                              swf, d0, dm1, kexp, accy, accp);
      else
        df_strip_burgers_up3<double, true, -1>(A, A.w, dst, A.pdf, ring, col0, r0, r1, cc0, lxs, lys, rat, square,
                                               swf, d0, dm1, kexp, accy, accp);
    } else {
      if (o.s > 0)
        df_strip_burgers_up3<float2, false, 1>(A, src, dst, A.pdf, ring, col0, r0, r1, cc0, lxs, lys, rat, square,
                                               swf, d0, dm1, kexp, accy, accp);
      else
        df_strip_burgers_up3<float2, false, -1>(A, src, dst, A.pdf, ring, col0, r0, r1, cc0, lxs, lys, rat, square,
                                                swf, d0, dm1, kexp, accy, accp);
    }
  });
  double sy = df_to_double(accy), sp = df_to_double(accp);
  if (!last_block_total2(sy, sp, partials, ticket)) return;
  if (threadIdx.x == 0) {
    leja_finalize(A, st, m, dm1d, sy, sp, pow2(sig + dlt), pow2(kexp), cond);
    const double rms = sqrt(sy / double(A.n));
    int e = 0;
    if (rms > 0.0 && isfinite(rms)) e = ilogb(rms);
    st->sig = sig + dlt;
    st->dlt = max(-100, min(100, e));
  }
}

}  // namespace lexgb

namespace lexgb {

// One power-iteration pass on the upwind operators in float-float (one
// thread per point): w = Op(v) / ||v|| with v the caller's doubles on the
// first pass and float pairs afterwards.  Op = A (constant weights) or J(u)
// (weights from q = u |a| / (6 dx) as float pairs).  The squares of w are
// accumulated exactly enough for a double-accurate rho, as in the central
// float-float pass.
template <bool BURGERS>
static __global__ void __launch_bounds__(kThreadsPerBlock)
    power_pass_df_up3_kernel(Up3Op o, const void* __restrict__ vin, int vin_double, float2* __restrict__ w,
                             const float2* __restrict__ q, double* __restrict__ partials,
                             unsigned int* __restrict__ ticket, LoopState* st) {
  if (__ldcg(&st->pdone)) return;
  const dfv sg = df_from_double(__ldcg(&st->sigma));
  const double* vd = reinterpret_cast<const double*>(vin);
  const float2* vf = reinterpret_cast<const float2*>(vin);
  auto ld = [&](long long i) -> dfv {
    if (vin_double) return df_split_scaled(__ldg(vd + i), 0);
    const float2 t = __ldg(vf + i);
    return {t.x, t.y};
  };
  double wd[7];
  up3_weights(o, wd);
  const dfv lxs = df_from_double(o.cxx), lys = df_from_double(o.cyy), rat = df_from_double(o.gy / o.gx);
  const dfv cc0 = df_from_double(-2.0 * o.cxx - 2.0 * o.cyy);
  float ch[7], cl[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const dfv t = df_from_double(wd[k]);
    ch[k] = t.h;
    cl[k] = t.l;
  }
  dfv acc = {0.f, 0.f};
  float small = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < o.n; i += (long long)gridDim.x * blockDim.x) {
    int pi, pj;
    up3_ij(o, i, pi, pj);
    long long pts[7];
    up3_points(o, pi, pj, pts);
    dfv t[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) t[k] = ld(pts[k]);
    dfv y;
    if constexpr (BURGERS) {
      dfv qv[7];
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        const float2 f = __ldg(q + pts[k]);
        qv[k] = {f.x, f.y};
      }
      dfv wv[7];
      wv[0] = df_add(cc0, df_scale_f(df_add(qv[0], df_mul(qv[0], rat)), (float)kUp3K0));
      wv[1] = df_add(lxs, df_scale_f(qv[1], (float)kUp3Km));
      wv[2] = df_add(lxs, df_scale_f(qv[2], (float)kUp3K1));
      wv[3] = df_scale_f(qv[3], (float)kUp3K2);
      wv[4] = df_add(lys, df_scale_f(df_mul(qv[4], rat), (float)kUp3Km));
      wv[5] = df_add(lys, df_scale_f(df_mul(qv[5], rat), (float)kUp3K1));
      wv[6] = df_scale_f(df_mul(qv[6], rat), (float)kUp3K2);
      float wh[7], wl[7];
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        wh[k] = wv[k].h;
        wl[k] = wv[k].l;
      }
      y = df_mul(sg, df_dot7(wh, wl, t));
    } else {
      y = df_mul(sg, df_dot7(ch, cl, t));
    }
    w[i] = make_float2(y.h, y.l);
    float sq, se;
    two_prod(y.h, y.h, sq, se);
    df_acc(acc, sq);
    small = __fmaf_rn(2.f * y.h, y.l, __fadd_rn(small, se));
  }
  double s = df_to_double(acc) + (double)small, dummy = 0.0;
  if (!last_block_total2(s, dummy, partials, ticket)) return;
  if (threadIdx.x == 0) power_pass_finish(st, s, o.n);
}

}  // namespace lexgb

namespace lexgb {

// sum_{k<N} w_k y_k (Dot2, the final renormalisation as df_dot7's).
template <int N>
__device__ __forceinline__ dfv df_dot_n(const float (&wh)[N], const float (&wl)[N], const dfv (&y)[N]) {
  float s, c, p, e, t;
  two_prod(wh[0], y[0].h, s, c);
#pragma unroll
  for (int k = 1; k < N; ++k) {
    two_prod(wh[k], y[k].h, p, e);
    two_sum(s, p, s, t);
    c = __fadd_rn(c, __fadd_rn(t, e));
  }
#pragma unroll
  for (int k = 0; k < N; ++k) {
    c = __fmaf_rn(wh[k], y[k].l, c);
    c = __fmaf_rn(wl[k], y[k].h, c);
  }
  dfv r;
  fast_two_sum(s, c, r.h, r.l);
  return r;
}

template <int STAGES>
constexpr int up3z_smem_bytes() {
  return kPipeWarps * STAGES * kSlotElemsUB * 8;
}

// One power-iteration pass on the upwind diffusion-advection operator in the
// pipelined form (nx % 128 == 0, 16-byte aligned vectors): w = A v / ||v||,
// rho_k = ||w||, the stop test of power_pass_finish; v is the caller's
// doubles on the first pass (vin_double), float pairs after.
template <int MINB>
__global__ void __launch_bounds__(kPipeThreads, MINB)
    power_pass_df_pipe_up3_kernel(Up3Op o, const void* __restrict__ vin, int vin_double, float2* __restrict__ w,
                                  double* __restrict__ partials, unsigned int* __restrict__ ticket, LoopState* st) {
  extern __shared__ __align__(16) unsigned long long up3p_smem[];
  if (__ldcg(&st->pdone)) return;
  const dfv sg = df_from_double(__ldcg(&st->sigma));
  double wd[7];
  up3_weights(o, wd);
  float wh[7], wl[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const dfv t = df_from_double(wd[k]);
    wh[k] = t.h;
    wl[k] = t.l;
  }
  LoopArgs A;
  A.nx = o.nx;
  A.ny = o.ny;
  dfv acc = {0.f, 0.f}, unused = {0.f, 0.f};
  float small = 0.f;
  const dfv zero = {0.f, 0.f};
  const int warp = threadIdx.x >> 5;
  unsigned long long* ring = up3p_smem + (size_t)warp * kUpStages * kSlotElems2;
  const double* vd = reinterpret_cast<const double*>(vin);
  const float2* vf = reinterpret_cast<const float2*>(vin);
  for_each_segment(o.nx, o.ny, 0, blockIdx.x * kPipeWarps + warp, gridDim.x * kPipeWarps,
                   [&](int col0, int r0, int r1) {
    if (vin_double) {
      if (o.s > 0)
        df_strip_up3<double, true, 1, true>(A, vd, w, nullptr, ring, col0, r0, r1, wh, wl, zero, zero, 0, acc,
                                            unused, sg, &small);
      else
        df_strip_up3<double, true, -1, true>(A, vd, w, nullptr, ring, col0, r0, r1, wh, wl, zero, zero, 0, acc,
                                             unused, sg, &small);
    } else {
      if (o.s > 0)
        df_strip_up3<float2, false, 1, true>(A, vf, w, nullptr, ring, col0, r0, r1, wh, wl, zero, zero, 0, acc,
                                             unused, sg, &small);
      else
        df_strip_up3<float2, false, -1, true>(A, vf, w, nullptr, ring, col0, r0, r1, wh, wl, zero, zero, 0, acc,
                                              unused, sg, &small);
    }
  });
  double s = df_to_double(acc) + (double)small, dummy = 0.0;
  if (!last_block_total2(s, dummy, partials, ticket)) return;
  if (threadIdx.x == 0) power_pass_finish(st, s, o.n);
}

// The quadratic upwind Burgers parts on the FP32 pipe (float-float, one
// thread per point): RHS = true gives h (nu lap u + (a/2) D(u^2) + S) (the
// step's right-hand side, recording the largest exponent of the result for
// the Leja loop's input scaling), RHS = false the EXPRB32 remainder
// h (a/2) D(p1^2).  The squares are float-float products.  A point takes the
// FP64 formula when a neighbour lies outside [2^-50, 2^e) (e <= 50, chosen so
// that weight times square stays below 2^118 in float), zero excepted.
template <bool RHS>
static __global__ void __launch_bounds__(kThreadsPerBlock)
    burgers_up3_df_kernel(Up3Op o, double h, const double* __restrict__ x, const double* __restrict__ src,
                          double* __restrict__ out, LoopState* st) {
  // weights of [x_C, x_X(-s), x_X(s), x_Y(-s), x_Y(s)] (RHS) and of the squares
  // at [C, X(-s), X(s), X(2s), Y(-s), Y(s), Y(2s)]
  const double hx = 0.5 * h * o.gx, hy = 0.5 * h * o.gy;
  const double wd[12] = {RHS ? h * (-2.0 * o.cxx - 2.0 * o.cyy) : 0.0, RHS ? h * o.cxx : 0.0, RHS ? h * o.cxx : 0.0,
                         RHS ? h * o.cyy : 0.0, RHS ? h * o.cyy : 0.0, kUp3K0 * (hx + hy), kUp3Km * hx,
                         kUp3K1 * hx, kUp3K2 * hx, kUp3Km * hy, kUp3K1 * hy, kUp3K2 * hy};
  float wh[12], wl[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const dfv t = df_from_double(wd[k]);
    wh[k] = t.h;
    wl[k] = t.l;
  }
  double wmax = 0.0;
#pragma unroll
  for (int k = 0; k < 12; ++k) wmax = fmax(wmax, fabs(wd[k]));
  const int ew = (wmax > 0.0 && isfinite(wmax)) ? ilogb(wmax) : 0;
  const int ehi = 1023 + min(50, (118 - ew) / 2);  // biased exponents below ehi qualify
  int emax = 0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < o.n; q += (long long)gridDim.x * blockDim.x) {
    int i, j;
    up3_ij(o, q, i, j);
    long long pts[7];
    up3_points(o, i, j, pts);
    double v[7];
    bool in_range = true;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      v[k] = __ldg(x + pts[k]);
      const int ex = (int)((__double_as_longlong(v[k]) >> 52) & 0x7ff);
      in_range = in_range && (ex == 0 || (ex >= 1023 - 50 && ex < ehi));
    }
    double r;
    if (in_range) {
      dfv t[12];
      dfv a[7];
#pragma unroll
      for (int k = 0; k < 7; ++k) a[k] = df_split_scaled(v[k], 0);
      t[0] = a[0];
      t[1] = a[1];
      t[2] = a[2];
      t[3] = a[4];
      t[4] = a[5];
#pragma unroll
      for (int k = 0; k < 7; ++k) t[5 + k] = df_mul(a[k], a[k]);
      const dfv d = df_dot_n<12>(wh, wl, t);
      r = f2d_scaled(d.h, 0) + f2d_scaled(d.l, 0);
    } else {
      r = wd[0] * v[0] + wd[1] * v[1] + wd[2] * v[2] + wd[3] * v[4] + wd[4] * v[5];
#pragma unroll
      for (int k = 0; k < 7; ++k) r = fma(wd[5 + k], v[k] * v[k], r);
    }
    if constexpr (RHS) {
      if (src) r = r + h * __ldg(src + q);
      emax = max(emax, (int)((__double2hiint(r) >> 20) & 0x7ff));
    }
    out[q] = r;
  }
  if constexpr (RHS) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, off));
    if ((threadIdx.x & 31) == 0) atomicMax(&st->wexp, emax);
  }
}

}  // namespace lexgb
