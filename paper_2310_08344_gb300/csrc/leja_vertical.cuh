// "Vertical" Leja interpolation (Sec. 2.3, real_Leja_phi with several
// integrator coefficients): phi_l(alpha_j h J) w for NP step fractions
// alpha_j at once.  The Leja nodes, the shift c and the scale gamma are the
// same for every alpha_j, so the Newton basis y_m is shared and only the
// divided differences differ:
//   p^(j)_{m+1} = p^(j)_m + d^(j)_{m+1} y_{m+1},
//   d^(j) = divided differences of phi_l(alpha_j h (c + gamma xi)).
// One fused launch per iteration computes y_{m+1}, updates the NP
// polynomials and reduces ||y_{m+1}|| and every ||p^(j)_{m+1}||; the last
// block stops the loop once every polynomial passes its own test
// |d^(j)_{m+1}| ||y_{m+1}|| <= rtol ||p^(j)_{m+1}|| + atol (the paper does
// not state the rule for several polynomials; this is the reading used).
// Traffic per point and iteration: y read + write and NP polynomials read +
// write, against NP separate loops that each move y and one polynomial.
#pragma once

#include "leja_upwind.cuh"
#include "lexgb_vertical.h"

namespace lexgb {

// Stopping test of a vertical loop (thread 0 of the last block).  sy:
// sum y^2; sp[j]: sum p_j^2; dm1[j]: d^(j)_{m+1} (unscaled); yscale and
// pscale undo the df64 storage scaling.
template <int NP>
__device__ __forceinline__ void leja_finalize_vertical(const LoopArgs& A, LoopState* st, int m, const double (&dm1)[NP],
                                                       double sy, const double (&sp)[NP], double yscale, double pscale,
                                                       cudaGraphConditionalHandle cond) {
  const double inv_n = 1.0 / double(A.n);
  const double ynorm = sqrt(sy * inv_n) * yscale;
  bool finite = isfinite(ynorm), pass = true;
  double emax = 0.0, pmin = 0.0;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const double pn = sqrt(sp[j] * inv_n) * pscale;
    const double e = fabs(dm1[j]) * ynorm;
    finite = finite && isfinite(e) && isfinite(pn);
    pass = pass && (e <= A.rtol * pn + A.atol);
    if (e > emax) emax = e;
    if (j == 0 || pn < pmin) pmin = pn;
  }
  const int m1 = m + 1;
  int status = 0;
  bool done = false;
  if (!finite) {
    status = 5;  // LX_E_NONFINITE
    done = true;
  } else if (pass) {
    done = true;
  } else if (m1 >= A.kmax) {
    status = 4;  // LX_E_NOCONV
    done = true;
  }
  st->m = m1;
  st->ynorm = ynorm;
  st->pnorm = pmin;
  st->err = emax;
  if (done) {
    st->status = status;
    st->done = 1;
    st->iters_total += m1;
    if (st->status_total == 0) st->status_total = status;
    if (A.use_cond) cudaGraphSetConditional(cond, 0);
  }
}

// FP64 / mixed strip (rows [r0, r1) of the columns [col0, col0 + 32 VEC)),
// the vertical counterpart of leja_strip.
template <int KIND, typename T, int VEC, typename S, bool FIRST, int NP>
__device__ __forceinline__ void leja_strip_vertical(const LoopArgs& A, const VertArgs& V, const S* __restrict__ src,
                                                    T* __restrict__ dst, int col0, int r0, int r1, T wcm,
                                                    const double (&d0)[NP], const double (&dm1)[NP], double& sy,
                                                    double (&sp)[NP]) {
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
    double pold[NP][VEC];
#pragma unroll
    for (int j = 0; j < NP; ++j)
      if constexpr (!FIRST) load_p<VEC>(V.p[j] + ro, c, nx, pold[j]);
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
    double pnew[NP][VEC];
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
      if (active) sy = fma(vd, vd, sy);
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const double po = FIRST ? d0[j] * double(yc[k]) : pold[j][k];
        pnew[j][k] = fma(dm1[j], vd, po);
        if (active) sp[j] = fma(pnew[j][k], pnew[j][k], sp[j]);
      }
    }
    if (active) {
      store_y<T, VEC>(dst + ro, c, nx, ynew);
#pragma unroll
      for (int j = 0; j < NP; ++j) store_p<VEC>(V.p[j] + ro, c, nx, pnew[j]);
    }
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      ys[k] = yc[k];
      yc[k] = yn[k];
    }
  }
}

template <int KIND, typename T, int VEC, int NP>
static __global__ void __launch_bounds__(kThreadsPerBlock)
    leja_iter_vertical_kernel(const LoopArgs* __restrict__ Ap, const VertArgs* __restrict__ Vp,
                              LoopState* __restrict__ st, double* __restrict__ partials,
                              unsigned int* __restrict__ ticket, cudaGraphConditionalHandle cond) {
  const LoopArgs& A = *Ap;
  const VertArgs& V = *Vp;
  const int m = __ldcg(&st->m);
  count_launch(st);
  if (__ldcg(&st->done)) return;
  const int nx = A.nx, ny = A.ny;
  const int H = A.strip_h;
  const int ncs = (nx + 32 * VEC - 1) / (32 * VEC);
  const int nstrips = ncs * ((ny + H - 1) / H);
  const double xim = __ldg(A.xi + m);
  double d0[NP], dm1[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    d0[j] = __ldg(V.d[j]);
    dm1[j] = __ldg(V.d[j] + m + 1);
  }
  const T wcm = T(A.wc0 - xim);
  T* dst = reinterpret_cast<T*>((m & 1) ? A.y1 : A.y0);
  double sums[1 + NP];
  double sy = 0.0, sp[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) sp[j] = 0.0;
  const int warp = threadIdx.x >> 5;
  for (int s = blockIdx.x * kWarpsPerBlock + warp; s < nstrips; s += gridDim.x * kWarpsPerBlock) {
    const int col0 = (s % ncs) * 32 * VEC;
    const int r0 = (s / ncs) * H;
    const int r1 = min(r0 + H, ny);
    if (m == 0) {
      leja_strip_vertical<KIND, T, VEC, double, true, NP>(A, V, A.w, dst, col0, r0, r1, wcm, d0, dm1, sy, sp);
    } else {
      const T* src = reinterpret_cast<const T*>(((m - 1) & 1) ? A.y1 : A.y0);
      leja_strip_vertical<KIND, T, VEC, T, false, NP>(A, V, src, dst, col0, r0, r1, wcm, d0, dm1, sy, sp);
    }
  }
  sums[0] = sy;
#pragma unroll
  for (int j = 0; j < NP; ++j) sums[1 + j] = sp[j];
  if (!last_block_total_n<1 + NP>(sums, partials, ticket)) return;
  if (threadIdx.x == 0) {
    double tp[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) tp[j] = sums[1 + j];
    leja_finalize_vertical<NP>(A, st, m, dm1, sums[0], tp, 1.0, 1.0, cond);
  }
}

// ---------------------------------------------------------------------------
// Float-float (df64) form, both operators, register window of three rows
// (4 points per lane, nx % 128 == 0).  Same storage scaling as the one-step
// df64 kernels: stored y_m = y_m 2^-sig, polynomials in 2^-kscale units, the
// new basis vector renormalised by 2^-dlt.
// ---------------------------------------------------------------------------
template <int KIND, bool FIRST, int NP, typename S>
__device__ __forceinline__ void df_strip_vertical(const LoopArgs& A, const VertArgs& V, const S* __restrict__ src,
                                                  float2* __restrict__ dst, int col0, int r0, int r1,
                                                  const float (&wh)[5], const float (&wl)[5], dfv xim, float swf,
                                                  const dfv (&d0)[NP], const dfv (&dm1)[NP], int sc, dfv& accy,
                                                  dfv (&accp)[NP]) {
  const int lane = threadIdx.x & 31;
  const int nx = A.nx, ny = A.ny;
  const int c = col0 + lane * 4;
  const int cw = col0 == 0 ? nx - 1 : col0 - 1;
  const int ce = (col0 + kPipeRow >= nx) ? 0 : col0 + kPipeRow;
  auto load = [&](int r, dfv (&v)[4]) {
    r = r < 0 ? r + ny : (r >= ny ? r - ny : r);
    if constexpr (FIRST)
      df_load_row<4>(reinterpret_cast<const double*>(src) + (size_t)r * nx, c, nx, sc, v);
    else
      df_load_row<4>(reinterpret_cast<const float2*>(src) + (size_t)r * nx, c, nx, v);
  };
  auto point = [&](int r, int col) -> dfv {
    if constexpr (FIRST)
      return df_point(reinterpret_cast<const double*>(src), (size_t)r * nx + col, sc);
    else
      return df_point(reinterpret_cast<const float2*>(src), (size_t)r * nx + col, sc);
  };
  const dfv lx = {A.bl[0], A.bl[1]}, ly = {A.bl[2], A.bl[3]}, rat = {A.bl[4], A.bl[5]};
  dfv ys[4], yc[4], yn[4];
  load(r0 - 1, ys);
  load(r0, yc);
  for (int r = r0; r < r1; ++r) {
    load(r + 1, yn);
    dfv xw = shfl_up_df(yc[3]);
    dfv xe = shfl_down_df(yc[0]);
    if (lane == 0) xw = point(r, cw);
    if (lane == 31) xe = point(r, ce);
    const size_t ro = (size_t)r * nx;
    dfv pold[NP][4];
    if constexpr (!FIRST) {
#pragma unroll
      for (int j = 0; j < NP; ++j) df_load_p<4>(V.pdf[j] + ro, c, nx, pold[j]);
    }
    dfv qv[4], rv[4];
    if constexpr (KIND == 1) {
      df_load_p<4>(A.bq + ro, c, nx, qv);
      df_load_p<4>(A.br + ro, c, nx, rv);
    }
    dfv ynew[4], pnew[NP][4];
    float fy = 0.f, fp[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) fp[j] = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const dfv t[5] = {k == 3 ? xe : yc[k + 1], k == 0 ? xw : yc[k - 1], yn[k], ys[k], yc[k]};
      dfv v;
      if constexpr (KIND == 0) {
        v = df_dot5(wh, wl, t);
      } else {
        const dfv qy = df_mul(qv[k], rat);
        const dfv wE = df_add(lx, df_neg(qv[k])), wW = df_add(lx, qv[k]);
        const dfv wN = df_add(ly, df_neg(qy)), wS = df_add(ly, qy);
        const dfv wC = df_add(rv[k], xim);
        const float bh[5] = {wE.h, wW.h, wN.h, wS.h, wC.h};
        const float bl[5] = {wE.l, wW.l, wN.l, wS.l, wC.l};
        v = df_dot5(bh, bl, t);
        v.h *= swf;
        v.l *= swf;
      }
      ynew[k] = v;
      fy = __fmaf_rn(v.h, v.h, fy);
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const dfv po = FIRST ? df_mul(d0[j], yc[k]) : pold[j][k];
        pnew[j][k] = df_axpy(dm1[j], v, po);
        fp[j] = __fmaf_rn(pnew[j][k].h, pnew[j][k].h, fp[j]);
      }
    }
    df_acc(accy, fy);
#pragma unroll
    for (int j = 0; j < NP; ++j) df_acc(accp[j], fp[j]);
    df_store_row<4>(dst + ro, c, nx, ynew);
#pragma unroll
    for (int j = 0; j < NP; ++j) df_store_row<4>(V.pdf[j] + ro, c, nx, pnew[j]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ys[k] = yc[k];
      yc[k] = yn[k];
    }
  }
}

template <int KIND, int NP>
static __global__ void __launch_bounds__(kThreadsPerBlock)
    leja_iter_df_vertical_kernel(const LoopArgs* __restrict__ Ap, const VertArgs* __restrict__ Vp,
                                 LoopState* __restrict__ st, double* __restrict__ partials,
                                 unsigned int* __restrict__ ticket, cudaGraphConditionalHandle cond) {
  const LoopArgs& A = *Ap;
  const VertArgs& V = *Vp;
  const int m = __ldcg(&st->m);
  count_launch(st);
  if (__ldcg(&st->done)) return;
  const int kexp = __ldcg(&st->kscale);
  const int sig = __ldcg(&st->sig);
  const int dlt = __ldcg(&st->dlt);
  const int nx = A.nx, ny = A.ny;
  const double xim_d = __ldg(A.xi + m);
  const double ysc = pow2(sig + dlt - kexp);
  double dm1d[NP];
  dfv d0[NP], dm1[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    dm1d[j] = __ldg(V.d[j] + m + 1);
    dm1[j] = df_from_double(dm1d[j] * ysc);
    d0[j] = df_from_double(__ldg(V.d[j]));
  }
  const double sw = pow2(-dlt);
  const float swf = (float)sw;
  float wh[5], wl[5];
  dfv xim = {0.f, 0.f};
  if constexpr (KIND == 0) {
    const dfv wc = df_from_double((A.wc0 - xim_d) * sw);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      wh[k] = A.wf[2 * k] * swf;
      wl[k] = A.wf[2 * k + 1] * swf;
    }
    wh[4] = wc.h;
    wl[4] = wc.l;
  } else {
    xim = df_from_double(-xim_d);
#pragma unroll
    for (int k = 0; k < 5; ++k) wh[k] = wl[k] = 0.f;
  }
  float2* dst = reinterpret_cast<float2*>((m & 1) ? A.y1 : A.y0);
  const float2* src = reinterpret_cast<const float2*>(((m - 1) & 1) ? A.y1 : A.y0);
  dfv accy = {0.f, 0.f}, accp[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) accp[j] = dfv{0.f, 0.f};
  const int warp = threadIdx.x >> 5;
  for_each_segment(nx, ny, A.strip_h, blockIdx.x * kWarpsPerBlock + warp, gridDim.x * kWarpsPerBlock,
                   [&](int col0, int r0, int r1) {
    if (m == 0)
      df_strip_vertical<KIND, true, NP>(A, V, A.w, dst, col0, r0, r1, wh, wl, xim, swf, d0, dm1, kexp, accy, accp);
    else
      df_strip_vertical<KIND, false, NP>(A, V, src, dst, col0, r0, r1, wh, wl, xim, swf, d0, dm1, kexp, accy, accp);
  });
  double sums[1 + NP];
  sums[0] = df_to_double(accy);
#pragma unroll
  for (int j = 0; j < NP; ++j) sums[1 + j] = df_to_double(accp[j]);
  if (!last_block_total_n<1 + NP>(sums, partials, ticket)) return;
  if (threadIdx.x == 0) {
    double tp[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) tp[j] = sums[1 + j];
    leja_finalize_vertical<NP>(A, st, m, dm1d, sums[0], tp, pow2(sig + dlt), pow2(kexp), cond);
    const double rms = sqrt(sums[0] / double(A.n));
    int e = 0;
    if (rms > 0.0 && isfinite(rms)) e = ilogb(rms);
    st->sig = sig + dlt;
    st->dlt = max(-100, min(100, e));
  }
}

// ---------------------------------------------------------------------------
// Vertical loops on the paper's upwind operators (periodic [-1,1)^2, Sec. 3),
// one thread per point with the seven stencil points through the caches, as
// the one-polynomial point-wise kernels: FP64 / mixed basis (T), and
// float-float with both operators (Burgers: the seven point weights from
// q = u |a| / (6 dx gamma)).
// ---------------------------------------------------------------------------
template <bool BURGERS, typename T, int NP>
static __global__ void __launch_bounds__(kThreadsPerBlock)
    leja_iter_up3_vertical_kernel(const LoopArgs* __restrict__ Ap, const VertArgs* __restrict__ Vp,
                                  LoopState* __restrict__ st, double* __restrict__ partials,
                                  unsigned int* __restrict__ ticket, cudaGraphConditionalHandle cond) {
  const LoopArgs& A = *Ap;
  const VertArgs& V = *Vp;
  const int m = __ldcg(&st->m);
  count_launch(st);
  if (__ldcg(&st->done)) return;
  const Up3Op o = A.up;
  const double xim = __ldg(A.xi + m);
  double d0[NP], dm1[NP], sp[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    d0[j] = __ldg(V.d[j]);
    dm1[j] = __ldg(V.d[j] + m + 1);
    sp[j] = 0.0;
  }
  const T ig = T(A.inv_gamma);
  const T cs = T(-A.up_c * A.inv_gamma - xim);  // -c/gamma - xi_m
  T* dst = reinterpret_cast<T*>((m & 1) ? A.y1 : A.y0);
  const T* src = reinterpret_cast<const T*>(((m - 1) & 1) ? A.y1 : A.y0);
  double sy = 0.0;
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
    sy = fma(vd, vd, sy);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const double po = m == 0 ? d0[k] * double(yc) : V.p[k][q];
      const double pn = fma(dm1[k], vd, po);
      V.p[k][q] = pn;
      sp[k] = fma(pn, pn, sp[k]);
    }
  }
  double sums[1 + NP];
  sums[0] = sy;
#pragma unroll
  for (int k = 0; k < NP; ++k) sums[1 + k] = sp[k];
  if (!last_block_total_n<1 + NP>(sums, partials, ticket)) return;
  if (threadIdx.x == 0) {
    double tp[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) tp[k] = sums[1 + k];
    leja_finalize_vertical<NP>(A, st, m, dm1, sums[0], tp, 1.0, 1.0, cond);
  }
}

template <bool BURGERS, int NP>
static __global__ void __launch_bounds__(kThreadsPerBlock)
    leja_iter_df_up3_vertical_kernel(const LoopArgs* __restrict__ Ap, const VertArgs* __restrict__ Vp,
                                     LoopState* __restrict__ st, double* __restrict__ partials,
                                     unsigned int* __restrict__ ticket, cudaGraphConditionalHandle cond) {
  const LoopArgs& A = *Ap;
  const VertArgs& V = *Vp;
  const int m = __ldcg(&st->m);
  count_launch(st);
  if (__ldcg(&st->done)) return;
  const int kexp = __ldcg(&st->kscale);
  const int sig = __ldcg(&st->sig);
  const int dlt = __ldcg(&st->dlt);
  const Up3Op o = A.up;
  const double xim = __ldg(A.xi + m);
  const double ysc = pow2(sig + dlt - kexp);
  double dm1d[NP];
  dfv d0[NP], dm1[NP], accp[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    dm1d[k] = __ldg(V.d[k] + m + 1);
    dm1[k] = df_from_double(dm1d[k] * ysc);
    d0[k] = df_from_double(__ldg(V.d[k]));
    accp[k] = dfv{0.f, 0.f};
  }
  const double sw = pow2(-dlt);
  const float swf = (float)sw;
  const double ig = A.inv_gamma;
  // diffusion-advection: the seven constant weights (shift and 2^-dlt folded in)
  float wh[7], wl[7];
  {
    double wd[7];
    up3_weights(o, wd);
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      double wk = wd[k] * ig;
      if (k == 0) wk += -A.up_c * ig - xim;
      const dfv t = df_from_double(wk * sw);
      wh[k] = t.h;
      wl[k] = t.l;
    }
  }
  // Burgers: the constant parts of the point weights
  const dfv cc0 = df_from_double((-2.0 * o.cxx - 2.0 * o.cyy - A.up_c) * ig - xim);
  const dfv lxs = df_from_double(o.cxx * ig), lys = df_from_double(o.cyy * ig);
  const dfv rat = df_from_double(o.gy / o.gx);
  float2* dst = reinterpret_cast<float2*>((m & 1) ? A.y1 : A.y0);
  const float2* src = reinterpret_cast<const float2*>(((m - 1) & 1) ? A.y1 : A.y0);
  dfv accy = {0.f, 0.f};
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
    dfv v;
    if constexpr (BURGERS) {
      dfv qv[7];
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        const float2 f = __ldg(A.bq + pts[k]);
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
      float bh[7], bl[7];
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        bh[k] = wv[k].h;
        bl[k] = wv[k].l;
      }
      v = df_dot7(bh, bl, t);
      v.h *= swf;
      v.l *= swf;
    } else {
      v = df_dot7(wh, wl, t);
    }
    dst[q] = make_float2(v.h, v.l);
    df_acc(accy, __fmul_rn(v.h, v.h));
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      dfv po;
      if (m == 0) {
        po = df_mul(d0[k], t[0]);
      } else {
        const float2 f = V.pdf[k][q];
        po = {f.x, f.y};
      }
      const dfv pn = df_axpy(dm1[k], v, po);
      V.pdf[k][q] = make_float2(pn.h, pn.l);
      df_acc(accp[k], __fmul_rn(pn.h, pn.h));
    }
  }
  double sums[1 + NP];
  sums[0] = df_to_double(accy);
#pragma unroll
  for (int k = 0; k < NP; ++k) sums[1 + k] = df_to_double(accp[k]);
  if (!last_block_total_n<1 + NP>(sums, partials, ticket)) return;
  if (threadIdx.x == 0) {
    double tp[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) tp[k] = sums[1 + k];
    leja_finalize_vertical<NP>(A, st, m, dm1d, sums[0], tp, pow2(sig + dlt), pow2(kexp), cond);
    const double rms = sqrt(sums[0] / double(A.n));
    int e = 0;
    if (rms > 0.0 && isfinite(rms)) e = ilogb(rms);
    st->sig = sig + dlt;
    st->dlt = max(-100, min(100, e));
  }
}

}  // namespace lexgb
