// Double-float ("df64") form of the fused Leja iteration for GB300.
//
// GB300 issues FP64 fused multiply-adds at about 1/58 of its FP32 rate
// (measured: ~0.6 T DFMA/s against ~35 T FFMA/s), so a stencil iteration
// written in native double is bound by the FP64 pipe at about a third of the
// HBM bandwidth.  This form keeps every vector value as an unevaluated sum of
// two floats (hi + lo, 48 significant bits, relative rounding ~2^-48) and
// does all per-point arithmetic on the FP32 pipe with error-free
// transformations:
//   TwoSum (Knuth), FastTwoSum (Dekker), TwoProduct by FMA, and the
//   compensated dot product Dot2 of Ogita, Rump and Oishi (2005) for the
//   five-point stencil.
// The basis y_m and the polynomial p_m live in context buffers as float2
// (8 bytes per point, the same traffic as double); the first iteration reads
// the caller's double input and the loop ends with one conversion pass into
// the caller's double output.  Inputs are scaled by an exact power of two so
// that max|w| is in [1, 2), and the stored basis is renormalised every
// iteration by a power of two 2^-dlt (folded exactly into the five stencil
// weights and the Newton coefficient, so it costs nothing per point): the
// stored vectors stay near unit norm even when the Newton basis itself grows
// or decays by many orders of magnitude, and the float exponent range always
// covers them.
#pragma once

#include "leja_kernels.cuh"

namespace lexgb {

struct dfv {
  float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// 2^k; 0 below the normal range, +inf above it (a vanished or overflowed basis).
__device__ __forceinline__ double pow2(int k) {
  if (k < -1022) return 0.0;
  if (k > 1023) return __longlong_as_double(0x7ff0000000000000LL);
  return __hiloint2double((k + 1023) << 20, 0);
}

// Split a double into hi + lo floats (exact up to the 48-bit precision).
__device__ __forceinline__ dfv df_from_double(double x) {
  dfv r;
  r.h = __double2float_rn(x);
  r.l = __double2float_rn(x - (double)r.h);
  return r;
}

__device__ __forceinline__ double df_to_double(dfv a) { return (double)a.h + (double)a.l; }

// x * 2^-k split into hi + lo floats with integer operations only (no FP64
// pipe work): hi keeps the leading 24 significant bits (truncated), lo the
// next 24 of the remaining 29 (rounded).  Values whose scaled magnitude is
// below 2^-126 become 0; above the float range, +-inf; NaN stays NaN.  lo is
// scaled in two steps, by 2^-29 and then by 2^(ef - 23), so that it stays
// exact down to a scaled magnitude of 2^-103 (a one-step scale by
// 2^(ef - 52) is not a normal float below 2^-74, which would leave the
// value with its leading 24 bits only).
__device__ __forceinline__ dfv df_split_scaled(double x, int k) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ffu);
  if (e == 0x7ff) return {__int_as_float((int)(sign | 0x7f800000u | (unsigned)((b & 0xfffffffffffffULL) ? 1 : 0))), 0.f};
  const int ef = e - 1023 - k;  // unbiased exponent of the scaled value
  if (e == 0 || ef < -126) return {__int_as_float((int)sign), 0.f};
  if (ef > 127) return {__int_as_float((int)(sign | 0x7f800000u)), 0.f};
  const unsigned long long mant = b & 0xfffffffffffffULL;
  dfv r;
  r.h = __int_as_float((int)(sign | ((unsigned)(ef + 127) << 23) | (unsigned)(mant >> 29)));
  const unsigned rest = (unsigned)(mant & 0x1fffffffULL);  // value rest * 2^(ef - 52)
  const int el = ef - 23 + 127;
  const float scale = el >= 1 ? __int_as_float((int)(sign | ((unsigned)el << 23))) : 0.f;
  r.l = (__uint2float_rn(rest) * 0x1p-29f) * scale;
  return r;
}

// Rare path of f2d_scaled, kept out of line so that the compiler branches
// around it instead of evaluating it (on the FP64 pipe) for every value.
static __device__ __noinline__ double f2d_scaled_slow(float f, int k) { return (double)f * pow2(k); }

// Exact float -> double by integer operations (zero -> 0; subnormals,
// infinities and NaN through the conversion instruction), then scaled by 2^k
// through the exponent field when that stays in range.  Subnormals matter
// where results are small without scaling (the low float of a value below
// about 2^-102 is one).
__device__ __forceinline__ double f2d_scaled(float f, int k) {
  const unsigned b = __float_as_uint(f);
  const int e = (int)((b >> 23) & 0xffu);
  if (e == 0) return (b & 0x7fffffu) ? f2d_scaled_slow(f, k) : 0.0;
  const int ed = e + 896 + k;
  if (e == 0xff || ed < 1 || ed > 2046) return f2d_scaled_slow(f, k);
  const unsigned long long db = ((unsigned long long)(b & 0x80000000u) << 32) | ((unsigned long long)ed << 52) |
                                ((unsigned long long)(b & 0x7fffffu) << 29);
  return __longlong_as_double((long long)db);
}

// sum_{k<5} w_k y_k with w_k = wh_k + wl_k, y_k = y_k.h + y_k.l (Dot2).
__device__ __forceinline__ dfv df_dot5(const float (&wh)[5], const float (&wl)[5], const dfv (&y)[5]) {
  float s, c, p, e, t;
  two_prod(wh[0], y[0].h, s, c);
#pragma unroll
  for (int k = 1; k < 5; ++k) {
    two_prod(wh[k], y[k].h, p, e);
    two_sum(s, p, s, t);
    c = __fadd_rn(c, __fadd_rn(t, e));
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    c = __fmaf_rn(wh[k], y[k].l, c);
    c = __fmaf_rn(wl[k], y[k].h, c);
  }
  dfv r;
  two_sum(s, c, r.h, r.l);
  return r;
}

// sum_{k<3} w_k y_k, the same compensated scheme as df_dot5.
__device__ __forceinline__ dfv df_dot3(const float (&wh)[3], const float (&wl)[3], const dfv (&y)[3]) {
  float s, c, p, e, t;
  two_prod(wh[0], y[0].h, s, c);
#pragma unroll
  for (int k = 1; k < 3; ++k) {
    two_prod(wh[k], y[k].h, p, e);
    two_sum(s, p, s, t);
    c = __fadd_rn(c, __fadd_rn(t, e));
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    c = __fmaf_rn(wh[k], y[k].l, c);
    c = __fmaf_rn(wl[k], y[k].h, c);
  }
  dfv r;
  two_sum(s, c, r.h, r.l);
  return r;
}

// a + b as an unnormalised float pair: the rounded sum of the leading parts
// and, in the low part, its exact rounding error plus both low parts.
__device__ __forceinline__ dfv df_add_loose(dfv a, dfv b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return {s, __fadd_rn(e, __fadd_rn(a.l, b.l))};
}

// sum_{k<3} w_k y_k as df_dot3, with the final renormalisation by Fast2Sum:
// when |s| >= |c| it is exact; otherwise s has cancelled below the
// correction c, and the pair misses s + c by at most a unit roundoff of |c|,
// where |c| is itself of order u sum |w_k y_k| (the products' rounding
// errors and low parts) -- the order of Dot2's own error bound, u^2 sum
// |w_k y_k|, so the accuracy class is unchanged.
__device__ __forceinline__ dfv df_dot3_f2s(const float (&wh)[3], const float (&wl)[3], const dfv (&y)[3]) {
  float s, c, p, e, t;
  two_prod(wh[0], y[0].h, s, c);
#pragma unroll
  for (int k = 1; k < 3; ++k) {
    two_prod(wh[k], y[k].h, p, e);
    two_sum(s, p, s, t);
    c = __fadd_rn(c, __fadd_rn(t, e));
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    c = __fmaf_rn(wh[k], y[k].l, c);
    c = __fmaf_rn(wl[k], y[k].h, c);
  }
  dfv r;
  fast_two_sum(s, c, r.h, r.l);
  return r;
}

// p + d * y
__device__ __forceinline__ dfv df_axpy(dfv d, dfv y, dfv p) {
  float q, qe, s, t;
  two_prod(d.h, y.h, q, qe);
  qe = __fmaf_rn(d.h, y.l, qe);
  qe = __fmaf_rn(d.l, y.h, qe);
  two_sum(p.h, q, s, t);
  t = __fadd_rn(t, __fadd_rn(p.l, qe));
  dfv r;
  fast_two_sum(s, t, r.h, r.l);
  return r;
}

// d * y
__device__ __forceinline__ dfv df_mul(dfv d, dfv y) {
  float q, qe;
  two_prod(d.h, y.h, q, qe);
  qe = __fmaf_rn(d.h, y.l, qe);
  qe = __fmaf_rn(d.l, y.h, qe);
  dfv r;
  fast_two_sum(q, qe, r.h, r.l);
  return r;
}

// acc += x (x a float partial sum of squares)
__device__ __forceinline__ void df_acc(dfv& acc, float x) {
  float s, e;
  two_sum(acc.h, x, s, e);
  acc.h = s;
  acc.l = __fadd_rn(acc.l, e);
}


template <int VEC>
__device__ __forceinline__ void df_load_row(const float2* __restrict__ row, int c, int nx, dfv (&v)[VEC]) {
  if constexpr (VEC == 4) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(row + c));
    const float4 b = __ldg(reinterpret_cast<const float4*>(row + c + 2));
    v[0] = {a.x, a.y};
    v[1] = {a.z, a.w};
    v[2] = {b.x, b.y};
    v[3] = {b.z, b.w};
  } else {
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      const float2 t = (c + k < nx) ? __ldg(row + c + k) : make_float2(0.f, 0.f);
      v[k] = {t.x, t.y};
    }
  }
}

// First iteration: the caller's double vector, scaled by 2^-ks, split to df.
template <int VEC>
__device__ __forceinline__ void df_load_row(const double* __restrict__ row, int c, int nx, int ks, dfv (&v)[VEC]) {
  if constexpr (VEC == 4) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(row + c));
    const double2 b = __ldg(reinterpret_cast<const double2*>(row + c + 2));
    v[0] = df_split_scaled(a.x, ks);
    v[1] = df_split_scaled(a.y, ks);
    v[2] = df_split_scaled(b.x, ks);
    v[3] = df_split_scaled(b.y, ks);
  } else {
#pragma unroll
    for (int k = 0; k < VEC; ++k) v[k] = df_split_scaled((c + k < nx) ? __ldg(row + c + k) : 0.0, ks);
  }
}

template <int VEC>
__device__ __forceinline__ void df_store_row(float2* __restrict__ row, int c, int nx, const dfv (&v)[VEC]) {
  if constexpr (VEC == 4) {
    *reinterpret_cast<float4*>(row + c) = make_float4(v[0].h, v[0].l, v[1].h, v[1].l);
    *reinterpret_cast<float4*>(row + c + 2) = make_float4(v[2].h, v[2].l, v[3].h, v[3].l);
  } else {
#pragma unroll
    for (int k = 0; k < VEC; ++k)
      if (c + k < nx) row[c + k] = make_float2(v[k].h, v[k].l);
  }
}

template <int VEC>
__device__ __forceinline__ void df_load_p(const float2* __restrict__ row, int c, int nx, dfv (&v)[VEC]) {
  if constexpr (VEC == 4) {
    const float4 a = *reinterpret_cast<const float4*>(row + c);
    const float4 b = *reinterpret_cast<const float4*>(row + c + 2);
    v[0] = {a.x, a.y};
    v[1] = {a.z, a.w};
    v[2] = {b.x, b.y};
    v[3] = {b.z, b.w};
  } else {
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      const float2 t = (c + k < nx) ? row[c + k] : make_float2(0.f, 0.f);
      v[k] = {t.x, t.y};
    }
  }
}

__device__ __forceinline__ dfv shfl_up_df(dfv v) {
  return {__shfl_up_sync(0xffffffffu, v.h, 1), __shfl_up_sync(0xffffffffu, v.l, 1)};
}
__device__ __forceinline__ dfv shfl_down_df(dfv v) {
  return {__shfl_down_sync(0xffffffffu, v.h, 1), __shfl_down_sync(0xffffffffu, v.l, 1)};
}

// Halo value of the row as df (the first iteration reads doubles).
__device__ __forceinline__ dfv df_point(const float2* __restrict__ src, size_t q, int) {
  const float2 t = __ldg(src + q);
  return {t.x, t.y};
}
__device__ __forceinline__ dfv df_point(const double* __restrict__ src, size_t q, int ks) {
  return df_split_scaled(__ldg(src + q), ks);
}

// One strip of the diffusion-advection iteration in df arithmetic.
// S = double (first iteration, caller's w) or float2 (basis buffer).
template <int VEC, typename S, bool FIRST>
__device__ __forceinline__ void df_strip_advdiff(const LoopArgs& A, const S* __restrict__ src, float2* __restrict__ dst,
                                                 float2* __restrict__ p, int col0, int r0, int r1,
                                                 const float (&wh)[5], const float (&wl)[5], dfv d0, dfv dm1,
                                                 int sc, dfv& accy, dfv& accp) {
  const int lane = threadIdx.x & 31;
  const int nx = A.nx, ny = A.ny;
  const int c = col0 + lane * VEC;
  const int cl = c + VEC - 1;
  const bool active = c < nx;
  const int cw = col0 == 0 ? nx - 1 : col0 - 1;
  const int ce = (cl + 1 >= nx) ? 0 : cl + 1;
  const bool need_e = active && (lane == 31 || cl + 1 >= nx);

  dfv ys[VEC], yc[VEC], yn[VEC];
  if constexpr (FIRST) {
    df_load_row<VEC>(src + (size_t)wrap_dn(r0, ny) * nx, c, nx, sc, ys);
    df_load_row<VEC>(src + (size_t)r0 * nx, c, nx, sc, yc);
  } else {
    df_load_row<VEC>(src + (size_t)wrap_dn(r0, ny) * nx, c, nx, ys);
    df_load_row<VEC>(src + (size_t)r0 * nx, c, nx, yc);
  }
  for (int r = r0; r < r1; ++r) {
    const size_t ro = (size_t)r * nx;
    if constexpr (FIRST)
      df_load_row<VEC>(src + (size_t)wrap_up(r, ny) * nx, c, nx, sc, yn);
    else
      df_load_row<VEC>(src + (size_t)wrap_up(r, ny) * nx, c, nx, yn);
    dfv pold[VEC];
    if constexpr (!FIRST) df_load_p<VEC>(p + ro, c, nx, pold);
    dfv xw = shfl_up_df(yc[VEC - 1]);
    dfv xe = shfl_down_df(yc[0]);
    if (lane == 0) xw = df_point(src, ro + cw, sc);
    if (need_e) xe = df_point(src, ro + ce, sc);
    dfv ynew[VEC], pnew[VEC];
    float fy = 0.f, fp = 0.f;
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      // terms ordered E, W, N, S, C to match the weights
      const dfv t[5] = {k == VEC - 1 ? xe : yc[(k + 1) % VEC], k == 0 ? xw : yc[(k + VEC - 1) % VEC], yn[k], ys[k],
                        yc[k]};
      ynew[k] = df_dot5(wh, wl, t);
      const dfv po = FIRST ? df_mul(d0, yc[k]) : pold[k];
      pnew[k] = df_axpy(dm1, ynew[k], po);
      if (c + k < nx) {
        fy = __fmaf_rn(ynew[k].h, ynew[k].h, fy);
        fp = __fmaf_rn(pnew[k].h, pnew[k].h, fp);
      }
    }
    df_acc(accy, fy);
    df_acc(accp, fp);
    if (active) {
      df_store_row<VEC>(dst + ro, c, nx, ynew);
      df_store_row<VEC>(p + ro, c, nx, pnew);
    }
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      ys[k] = yc[k];
      yc[k] = yn[k];
    }
  }
}

template <int VEC>
__global__ void __launch_bounds__(kThreadsPerBlock)
    leja_iter_df_advdiff_kernel(const LoopArgs* __restrict__ Ap, LoopState* __restrict__ st,
                                double* __restrict__ partials, unsigned int* __restrict__ ticket,
                                cudaGraphConditionalHandle cond) {
  const LoopArgs& A = *Ap;
  const int m = __ldcg(&st->m);
  count_launch(st);
  if (__ldcg(&st->done)) return;
  const int kexp = __ldcg(&st->kscale);
  const int sig = __ldcg(&st->sig);  // stored y_m = y_m 2^-sig
  const int dlt = __ldcg(&st->dlt);  // stored y_{m+1} = y_{m+1} 2^-(sig + dlt)
  const int sc = kexp;
  const int nx = A.nx, ny = A.ny;
  const int H = A.strip_h;
  const int ncs = (nx + 32 * VEC - 1) / (32 * VEC);
  const int nstrips = ncs * ((ny + H - 1) / H);
  const double xim = __ldg(A.xi + m);
  const double dm1d = __ldg(A.d + m + 1);
  // p (stored as p 2^-kexp) += d_{m+1} y_{m+1} = d_{m+1} 2^(sig+dlt-kexp) * stored y_{m+1}
  const dfv dm1 = df_from_double(dm1d * pow2(sig + dlt - kexp));
  const dfv d0 = df_from_double(__ldg(A.d));
  const double sw = pow2(-dlt);
  const float swf = (float)sw;
  const dfv wc = df_from_double((A.wc0 - xim) * sw);
  const float wh[5] = {A.wf[0] * swf, A.wf[2] * swf, A.wf[4] * swf, A.wf[6] * swf, wc.h};
  const float wl[5] = {A.wf[1] * swf, A.wf[3] * swf, A.wf[5] * swf, A.wf[7] * swf, wc.l};
  float2* dst = reinterpret_cast<float2*>((m & 1) ? A.y1 : A.y0);
  float2* p = A.pdf;
  dfv accy = {0.f, 0.f}, accp = {0.f, 0.f};
  const int warp = threadIdx.x >> 5;
  for (int s = blockIdx.x * kWarpsPerBlock + warp; s < nstrips; s += gridDim.x * kWarpsPerBlock) {
    const int col0 = (s % ncs) * 32 * VEC;
    const int r0 = (s / ncs) * H;
    const int r1 = min(r0 + H, ny);
    if (m == 0) {
      df_strip_advdiff<VEC, double, true>(A, A.w, dst, p, col0, r0, r1, wh, wl, d0, dm1, sc, accy, accp);
    } else {
      const float2* src = reinterpret_cast<const float2*>(((m - 1) & 1) ? A.y1 : A.y0);
      df_strip_advdiff<VEC, float2, false>(A, src, dst, p, col0, r0, r1, wh, wl, d0, dm1, sc, accy, accp);
    }
  }
  double sy = df_to_double(accy), sp = df_to_double(accp);
  if (!last_block_total2(sy, sp, partials, ticket)) return;
  if (threadIdx.x == 0) {
    leja_finalize(A, st, m, dm1d, sy, sp, pow2(sig + dlt), pow2(kexp), cond);
    // next renormalisation: bring the stored basis back to unit norm
    const double rms = sqrt(sy / double(A.n));
    int e = 0;
    if (rms > 0.0 && isfinite(rms)) e = ilogb(rms);
    st->sig = sig + dlt;
    st->dlt = max(-100, min(100, e));
  }
}

// max over |w| of the binary exponent, to choose the power-of-two scaling.
static __global__ void __launch_bounds__(kThreadsPerBlock) df_scale_kernel(long long n, const double* __restrict__ w,
                                                                    LoopState* st) {
  int e = 0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    e = max(e, (int)((__double2hiint(w[q]) >> 20) & 0x7ff));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&st->wexp, e);
}

// kscale from the maximal exponent (one thread).
static __global__ void df_scale_finish_kernel(LoopState* st) {
  int e = st->wexp;  // biased; 0 for an all-zero (or subnormal) vector
  int k = (e == 0) ? 0 : (e == 2047 ? 0 : e - 1023);
  st->kscale = max(-1000, min(1000, k));
  st->sig = st->kscale;
  st->dlt = 0;
}

// out = base + (p.h + p.l) 2^k  (base may be NULL): the loop's conversion
// pass, fused with the Rosenbrock-Euler update u + p when base = u.
static __global__ void df_output_kernel(long long n, const float2* __restrict__ pdf, const double* __restrict__ base,
                                        double* __restrict__ out, const LoopState* st, const float2* __restrict__ y0,
                                        const float2* __restrict__ y1) {
  const int k = __ldcg(&st->kscale);
  const int fix = __ldcg(&st->fix);
  const dfv fd = df_from_double(-__ldcg(&st->fix_d));
  const float2* yb = __ldcg(&st->fix_buf) ? y1 : y0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const float2 t = pdf[q];
    dfv pv = {t.x, t.y};
    if (fix) {  // a two-step loop that stopped after its first step
      const float2 y = yb[q];
      pv = df_axpy(fd, dfv{y.x, y.y}, pv);
    }
    const double v = f2d_scaled(pv.h, k) + f2d_scaled(pv.l, k);
    out[q] = base ? base[q] + v : v;
  }
}

// h A u for the diffusion-advection operator in df arithmetic (Dot2 over the
// five stencil points), written as double; also records max exponent of the
// result for the scaling of the Leja loop that follows.  wf: hi/lo of the
// five weights h*(wE, wW, wN, wS, wC).  Points whose inputs are outside the
// float range use double arithmetic.  src (may be NULL): a time-independent
// source, added as h * src in double (problem with sources, Sec. 3, Eq. 4).
struct RhsWeights {
  float wf[10];   // hi/lo of h*(wE, wW, wN, wS, wC)
  double wd[5];   // the same weights in double
};

static __global__ void __launch_bounds__(kThreadsPerBlock)
    rhs_df_advdiff_kernel(Geo g, const double* __restrict__ u, RhsWeights W, double* __restrict__ f_out,
                          LoopState* st, const double* __restrict__ src = nullptr, double h = 0.0) {
  float wh[5], wl[5];
  const double* wd = W.wd;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    wh[k] = W.wf[2 * k];
    wl[k] = W.wf[2 * k + 1];
  }
  int emax = 0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < g.n; q += (long long)gridDim.x * blockDim.x) {
    long long e, w, nn, s;
    neighbours(g, q, e, w, nn, s);
    const double v[5] = {__ldg(u + e), __ldg(u + w), __ldg(u + nn), __ldg(u + s), __ldg(u + q)};
    bool in_range = true;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const int ex = (int)((__double_as_longlong(v[k]) >> 52) & 0x7ff);
      in_range = in_range && (ex == 0 || (ex > 1023 - 100 && ex < 1023 + 100));
    }
    double r;
    if (in_range) {
      const dfv t[5] = {df_split_scaled(v[0], 0), df_split_scaled(v[1], 0), df_split_scaled(v[2], 0),
                        df_split_scaled(v[3], 0), df_split_scaled(v[4], 0)};
      const dfv d = df_dot5(wh, wl, t);
      r = f2d_scaled(d.h, 0) + f2d_scaled(d.l, 0);
    } else {
      r = wd[0] * v[0] + wd[1] * v[1] + wd[2] * v[2] + wd[3] * v[3] + wd[4] * v[4];
    }
    if (src) r = r + h * __ldg(src + q);
    f_out[q] = r;
    emax = max(emax, (int)((__double2hiint(r) >> 20) & 0x7ff));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&st->wexp, emax);
}

}  // namespace lexgb

namespace lexgb {

// ---------------------------------------------------------------------------
// Pipelined df64 iteration (nx % 128 == 0): each warp stages the rows it is
// about to need -- y with its two x-halo points, and p -- into a private
// shared-memory ring with asynchronous copies (cp.async), kPipeAhead rows
// ahead of the row it computes.  The bytes in flight then no longer occupy
// registers, so a resident warp keeps several rows of loads outstanding.
// ---------------------------------------------------------------------------

constexpr int kPipeWarps = 4;
constexpr int kPipeThreads = kPipeWarps * 32;
constexpr int kPipeStages = 5;            // ring slots per warp
constexpr int kPipeAhead = kPipeStages - 3;
constexpr int kPipeRow = 128;             // points per warp row (4 per lane)
constexpr int kYSlot = kPipeRow + 4;      // [pad][west halo][128 points][east halo][pad]
constexpr int kPSlot = kPipeRow;
constexpr int kSlotElems = kYSlot + kPSlot;
constexpr int kPipeSmemBytes = kPipeWarps * kPipeStages * kSlotElems * 8;
constexpr int kPipeSmemBytes8 = kPipeWarps * 8 * kSlotElems * 8;  // the 8-stage variant

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Rows a warp processes, as segments (col0, r0, r1) of one warp-row column
// strip: strips of H rows dealt round-robin over the nw warps (H > 0), or
// one contiguous, evenly sized range of the ncs * ny (column strip, row)
// lines per warp (H == 0), which balances the warps and reads each halo row
// only twice per warp instead of once per strip.
template <typename F>
__device__ __forceinline__ void for_each_segment(int nx, int ny, int H, int wid, int nw, F&& f) {
  const int ncs = nx / kPipeRow;
  if (H > 0) {
    const int nstrips = ncs * ((ny + H - 1) / H);
    for (int s = wid; s < nstrips; s += nw) {
      const int r0 = (s / ncs) * H;
      f((s % ncs) * kPipeRow, r0, min(r0 + H, ny));
    }
  } else {
    const long long T = (long long)ncs * ny;
    long long t = T * wid / nw;
    const long long t1 = T * (wid + 1) / nw;
    while (t < t1) {
      const int cs = (int)(t / ny), r0 = (int)(t % ny);
      const int r1 = (int)min((long long)ny, (long long)r0 + (t1 - t));
      f(cs * kPipeRow, r0, r1);
      t += r1 - r0;
    }
  }
}

template <typename S>
__device__ __forceinline__ dfv df_from_raw(const unsigned long long* e, int sc) {
  if constexpr (sizeof(S) == 8 && !std::is_same<S, float2>::value) {
    return df_split_scaled(__longlong_as_double((long long)*e), sc);
  } else {
    const float2 t = *reinterpret_cast<const float2*>(e);
    return {t.x, t.y};
  }
}

template <typename S>
__device__ __forceinline__ void df_from_raw4(const unsigned long long* e, int sc, dfv (&v)[4]) {
  if constexpr (!std::is_same<S, float2>::value) {
    const double2 a = *reinterpret_cast<const double2*>(e);
    const double2 b = *reinterpret_cast<const double2*>(e + 2);
    v[0] = df_split_scaled(a.x, sc);
    v[1] = df_split_scaled(a.y, sc);
    v[2] = df_split_scaled(b.x, sc);
    v[3] = df_split_scaled(b.y, sc);
  } else {
    const float4 a = *reinterpret_cast<const float4*>(e);
    const float4 b = *reinterpret_cast<const float4*>(e + 2);
    v[0] = {a.x, a.y};
    v[1] = {a.z, a.w};
    v[2] = {b.x, b.y};
    v[3] = {b.z, b.w};
  }
}

template <int STAGES, typename S, bool FIRST>
__device__ __forceinline__ void df_strip_pipe(const LoopArgs& A, const S* __restrict__ src, float2* __restrict__ dst,
                                              float2* __restrict__ p, unsigned long long* ring, int col0, int r0,
                                              int r1, const float (&wh)[5], const float (&wl)[5], dfv d0, dfv dm1,
                                              int sc, dfv& accy, dfv& accp) {
  const int lane = threadIdx.x & 31;
  const int nx = A.nx, ny = A.ny;
  const int c = col0 + lane * 4;
  const int cw = col0 == 0 ? nx - 1 : col0 - 1;
  const int ce = (col0 + kPipeRow >= nx) ? 0 : col0 + kPipeRow;
  const int nrows = r1 - r0;           // rows computed
  const int last_q = nrows + 1;        // y rows q = 0 .. nrows+1 (r0-1 .. r1)
  auto slot = [&](int q) { return ring + (size_t)(q % STAGES) * kSlotElems; };
  auto issue = [&](int q) {
    if (q <= last_q) {
      int ry = r0 - 1 + q;
      ry = ry < 0 ? ry + ny : (ry >= ny ? ry - ny : ry);
      unsigned long long* s = slot(q);
      const S* row = src + (size_t)ry * nx;
      cp_async16(s + 2 + lane * 4, row + c);
      cp_async16(s + 4 + lane * 4, row + c + 2);
      if (lane == 0) cp_async8(s + 1, row + cw);
      if (lane == 31) cp_async8(s + 2 + kPipeRow, row + ce);
      if constexpr (!FIRST) {
        if (q >= 1 && q <= nrows) {
          const float2* prow = p + (size_t)(r0 - 1 + q) * nx;
          cp_async16(s + kYSlot + lane * 4, prow + c);
          cp_async16(s + kYSlot + lane * 4 + 2, prow + c + 2);
        }
      }
    }
    cp_commit();
  };
  for (int q = 0; q < STAGES - 1; ++q) issue(q);
  cp_wait<STAGES - 3>();
  __syncwarp();
  dfv ys[4], yc[4], yn[4];
  df_from_raw4<S>(slot(0) + 2 + lane * 4, sc, ys);
  df_from_raw4<S>(slot(1) + 2 + lane * 4, sc, yc);
  for (int qc = 1; qc <= nrows; ++qc) {
    issue(qc + STAGES - 2);
    cp_wait<STAGES - 3>();
    __syncwarp();
    const unsigned long long* sn = slot(qc + 1);
    const unsigned long long* scn = slot(qc);
    df_from_raw4<S>(sn + 2 + lane * 4, sc, yn);
    dfv pold[4];
    if constexpr (!FIRST) df_from_raw4<float2>(scn + kYSlot + lane * 4, sc, pold);
    dfv xw = shfl_up_df(yc[3]);
    dfv xe = shfl_down_df(yc[0]);
    if (lane == 0) xw = df_from_raw<S>(scn + 1, sc);
    if (lane == 31) xe = df_from_raw<S>(scn + 2 + kPipeRow, sc);
    dfv ynew[4], pnew[4];
    float fy = 0.f, fp = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const dfv t[5] = {k == 3 ? xe : yc[k + 1], k == 0 ? xw : yc[k - 1], yn[k], ys[k], yc[k]};
      ynew[k] = df_dot5(wh, wl, t);
      const dfv po = FIRST ? df_mul(d0, yc[k]) : pold[k];
      pnew[k] = df_axpy(dm1, ynew[k], po);
      fy = __fmaf_rn(ynew[k].h, ynew[k].h, fy);
      fp = __fmaf_rn(pnew[k].h, pnew[k].h, fp);
    }
    df_acc(accy, fy);
    df_acc(accp, fp);
    const size_t ro = (size_t)(r0 - 1 + qc) * nx;
    df_store_row<4>(dst + ro, c, nx, ynew);
    df_store_row<4>(p + ro, c, nx, pnew);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ys[k] = yc[k];
      yc[k] = yn[k];
    }
    __syncwarp();
  }
  cp_wait<0>();
  __syncwarp();
}

// Split for the right-hand side's float-float rows, without branches or
// conversion instructions: x with |x| in [2^-99, 2^100), or zero (a
// subnormal counts as zero); ok reports whether x is one of them (a value
// outside gives an unspecified pair, and its row is computed in double).
// hi: the leading 24 bits (truncated), from the bits shifted left by 3 with
// the exponent rebased modulo 2^9 (exact over the range); lo: the remaining
// 29 bits rounded to 23, as the float whose bits are those of
// M = +-2^(e-23) plus the rounded bits, minus M (exact: the two lie within a
// factor of 2).  |x - hi - lo| <= 2^-47 |x|.
__device__ __forceinline__ dfv df_split_rhs(double x, bool& ok) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned a = hi & 0x7ff00000u;
  ok = a == 0u || (a - (924u << 20)) < (199u << 20);
  const unsigned t = __funnelshift_l(lo, hi, 3);
  const unsigned sign = hi & 0x80000000u;
  const unsigned mb = ((t & 0xff800000u) - (407u << 23)) | sign;
  const unsigned r = ((lo & 0x1fffffffu) + 32u) >> 6;
  const float l = __fsub_rn(__uint_as_float(mb + r), __uint_as_float(mb));
  dfv v;
  v.h = __uint_as_float(a ? ((t - 0xC0000000u) | sign) : sign);
  v.l = a ? l : 0.f;
  return v;
}

// h A u (+ h S) for the diffusion-advection operator when nx % 128 == 0 and
// u, f_out, src are 16-byte aligned: warps take balanced row ranges of
// 128-column strips; the input rows are staged into shared memory by
// cp.async STAGES - 3 rows ahead of use (a per-warp ring of raw double rows
// with a one-point halo per side), so that loads overlap the float-float
// arithmetic.  Each lane keeps the float-float splits of its four points of
// the centre and north rows in registers (every value is split once); a row
// whose inputs include a value outside the float-float range is computed in
// double by the whole warp from the input re-read in global memory.  Records
// the largest exponent of the result like rhs_df_advdiff_kernel.
// SQ (square grids with the east and north weights equal, and the west and
// south ones): the paired stencil w_E (y_E + y_N) + w_W (y_W + y_S) +
// w_C y_C; the (W,S) sums at columns c+1 .. c+3 are the (E,N) sums of the
// row before at c .. c+2 (the same two operands, so the same values), which
// are formed on every row, so that the carry stays valid across rows
// computed in double (a row on the float-float path has all its inputs, and
// so those of the carried sums, in range).  Four warps per block; dynamic
// shared memory rhs_ring_smem_bytes<STAGES>().
constexpr int kRhsSlot = kPipeRow + 4;  // [pad][w1][128 points][e1][pad]
template <int STAGES>
constexpr int rhs_ring_smem_bytes() {
  return kPipeWarps * STAGES * kRhsSlot * 8;
}

template <int STAGES, bool SQ>
static __global__ void __launch_bounds__(kPipeThreads)
    rhs_df_advdiff_ring_kernel(int nx, int ny, const double* __restrict__ u, RhsWeights W,
                               double* __restrict__ f_out, LoopState* st, const double* __restrict__ src, double h) {
  extern __shared__ __align__(16) unsigned long long rhs_ring[];
  float wh[5], wl[5];
  const double* wd = W.wd;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    wh[k] = W.wf[2 * k];
    wl[k] = W.wf[2 * k + 1];
  }
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  unsigned long long* ring = rhs_ring + (size_t)warp * STAGES * kRhsSlot;
  int emax = 0;
  const float h3[3] = {wh[0], wh[1], wh[4]}, l3[3] = {wl[0], wl[1], wl[4]};
  for_each_segment(nx, ny, 0, blockIdx.x * kPipeWarps + warp, gridDim.x * kPipeWarps, [&](int col0, int r0, int r1) {
    const int c = col0 + lane * 4;
    const int cw = col0 == 0 ? nx - 1 : col0 - 1;
    const int ce = (col0 + kPipeRow >= nx) ? 0 : col0 + kPipeRow;
    const int last_q = r1 - r0 + 1;  // rows q = 0 .. last_q are grid rows r0 - 1 .. r1
    auto slot = [&](int q) { return ring + (size_t)(q % STAGES) * kRhsSlot; };
    auto issue = [&](int q) {
      if (q <= last_q) {
        int r = r0 - 1 + q;
        r = r < 0 ? r + ny : (r >= ny ? r - ny : r);
        const double* row = u + (size_t)r * nx;
        unsigned long long* s = slot(q);
        cp_async16(s + 2 + lane * 4, row + c);
        cp_async16(s + 4 + lane * 4, row + c + 2);
        if (lane == 0) cp_async8(s + 1, row + cw);
        if (lane == 31) cp_async8(s + 2 + kPipeRow, row + ce);
      }
      cp_commit();
    };
    // the lane's four values of staged row q, split; whether all are in range
    auto load = [&](int q, dfv(&f)[4]) {
      const unsigned long long* s = slot(q);
      const double2 a = *reinterpret_cast<const double2*>(s + 2 + lane * 4);
      const double2 b = *reinterpret_cast<const double2*>(s + 4 + lane * 4);
      const double v[4] = {a.x, a.y, b.x, b.y};
      bool ok = true;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        bool okk;
        f[k] = df_split_rhs(v[k], okk);
        ok = ok && okk;
      }
      return ok;
    };
    for (int q = 0; q < STAGES; ++q) issue(q);
    cp_wait<STAGES - 3>();
    __syncwarp();
    dfv S[4], C[4], N[4];  // SQ: only S[0] is kept after the first row
    bool okS = load(0, S), okC = load(1, C), okN = load(2, N);
    dfv qa[3];  // SQ: the (E,N) sums of the previous row at columns c .. c+2
    if constexpr (SQ) {
#pragma unroll
      for (int k = 0; k < 3; ++k) qa[k] = df_add_loose(S[k + 1], C[k]);
    }
    for (int r = r0; r < r1; ++r) {
      const int i = r - r0;
      issue(i + STAGES);  // into the slot of row q = i, whose values are in registers
      cp_wait<STAGES - 3>();
      __syncwarp();
      // the strip's halo value of row r: lane 0 west, lane 31 east (each
      // reads only the word its own copy wrote)
      const unsigned long long* scn = slot(i + 1);
      const double hx = lane == 0 ? __longlong_as_double((long long)scn[1])
                                  : (lane == 31 ? __longlong_as_double((long long)scn[2 + kPipeRow]) : 0.0);
      bool okH;
      const dfv dh = df_split_rhs(hx, okH);
      dfv sen[4];
      if constexpr (SQ) {
#pragma unroll
        for (int k = 0; k < 3; ++k) sen[k] = df_add_loose(C[k + 1], N[k]);
      }
      double res[4];
      if (__all_sync(0xffffffffu, okS && okC && okN && okH)) {
        const dfv sw = shfl_up_df(C[3]);
        const dfv se = shfl_down_df(C[0]);
        const dfv dw = lane == 0 ? dh : sw;
        const dfv de = lane == 31 ? dh : se;
        if constexpr (SQ) {
          sen[3] = df_add_loose(de, N[3]);
          const dfv sws0 = df_add_loose(dw, S[0]);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const dfv t[3] = {sen[k], k == 0 ? sws0 : qa[k - 1], C[k]};
            const dfv d = df_dot3_f2s(h3, l3, t);
            res[k] = f2d_scaled(d.h, 0) + f2d_scaled(d.l, 0);
          }
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const dfv t[5] = {k == 3 ? de : C[k + 1], k == 0 ? dw : C[k - 1], N[k], S[k], C[k]};
            const dfv d = df_dot5(wh, wl, t);
            res[k] = f2d_scaled(d.h, 0) + f2d_scaled(d.l, 0);
          }
        }
      } else {
        // in double, from the input rows r - 1, r, r + 1 in global memory
        const int rs = r == 0 ? ny - 1 : r - 1, rn = r + 1 == ny ? 0 : r + 1;
        const double* rowC = u + (size_t)r * nx;
        const double* rowS = u + (size_t)rs * nx;
        const double* rowN = u + (size_t)rn * nx;
        double vc[6];
        vc[0] = __ldg(rowC + (lane == 0 ? cw : c - 1));
        vc[5] = __ldg(rowC + (lane == 31 ? ce : c + 4));
#pragma unroll
        for (int k = 0; k < 4; ++k) vc[k + 1] = __ldg(rowC + c + k);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          res[k] = wd[0] * vc[k + 2] + wd[1] * vc[k] + wd[2] * __ldg(rowN + c + k) + wd[3] * __ldg(rowS + c + k) +
                   wd[4] * vc[k + 1];
      }
      const size_t ro = (size_t)r * nx + c;
      if (src) {
        const double2 s0 = __ldg(reinterpret_cast<const double2*>(src + ro));
        const double2 s1 = __ldg(reinterpret_cast<const double2*>(src + ro + 2));
        res[0] = res[0] + h * s0.x;
        res[1] = res[1] + h * s0.y;
        res[2] = res[2] + h * s1.x;
        res[3] = res[3] + h * s1.y;
      }
      *reinterpret_cast<double2*>(f_out + ro) = make_double2(res[0], res[1]);
      *reinterpret_cast<double2*>(f_out + ro + 2) = make_double2(res[2], res[3]);
#pragma unroll
      for (int k = 0; k < 4; ++k) emax = max(emax, (int)((__double2hiint(res[k]) >> 20) & 0x7ff));
      // next row: S <- C, C <- N, N <- staged row q = i + 3 (complete since
      // this row's wait)
      if constexpr (SQ) {
#pragma unroll
        for (int k = 0; k < 3; ++k) qa[k] = sen[k];
        S[0] = C[0];
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) S[k] = C[k];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) C[k] = N[k];
      okS = okC;
      okC = okN;
      if (r + 1 < r1) okN = load(i + 3, N);
    }
    cp_wait<0>();
    __syncwarp();
  });
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  if (lane == 0) atomicMax(&st->wexp, emax);
}

// p as float pairs -> double (times 2^kscale), plus base when given; two
// points per step with 16-byte accesses (n even, base and out 16-byte
// aligned).  Same semantics as df_output_kernel, including the correction of
// a two-step loop that stopped after its first iteration.
static __global__ void __launch_bounds__(kThreadsPerBlock)
    df_output2_kernel(long long n2, const float4* __restrict__ pdf, const double2* __restrict__ base,
                      double2* __restrict__ out, const LoopState* st, const float4* __restrict__ y0,
                      const float4* __restrict__ y1) {
  const int k = __ldcg(&st->kscale);
  const int fix = __ldcg(&st->fix);
  const dfv fd = df_from_double(-__ldcg(&st->fix_d));
  const float4* yb = __ldcg(&st->fix_buf) ? y1 : y0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n2; q += (long long)gridDim.x * blockDim.x) {
    const float4 t = pdf[q];
    dfv a = {t.x, t.y}, b = {t.z, t.w};
    if (fix) {
      const float4 y = yb[q];
      a = df_axpy(fd, dfv{y.x, y.y}, a);
      b = df_axpy(fd, dfv{y.z, y.w}, b);
    }
    double2 r = make_double2(f2d_scaled(a.h, k) + f2d_scaled(a.l, k), f2d_scaled(b.h, k) + f2d_scaled(b.l, k));
    if (base) {
      const double2 bb = base[q];
      r.x = bb.x + r.x;
      r.y = bb.y + r.y;
    }
    out[q] = r;
  }
}

template <int MINB, int STAGES = kPipeStages>
__global__ void __launch_bounds__(kPipeThreads, MINB)
    leja_iter_df_pipe_kernel(const LoopArgs* __restrict__ Ap, LoopState* __restrict__ st,
                             double* __restrict__ partials, unsigned int* __restrict__ ticket,
                             cudaGraphConditionalHandle cond) {
  extern __shared__ __align__(16) unsigned long long pipe_smem[];
  const LoopArgs& A = *Ap;
  const int m = __ldcg(&st->m);
  count_launch(st);
  if (__ldcg(&st->done)) return;
  const int kexp = __ldcg(&st->kscale);
  const int sig = __ldcg(&st->sig);
  const int dlt = __ldcg(&st->dlt);
  const int sc = kexp;
  const int nx = A.nx, ny = A.ny;
  const int H = A.strip_h;
  const double xim = __ldg(A.xi + m);
  const double dm1d = __ldg(A.d + m + 1);
  const dfv dm1 = df_from_double(dm1d * pow2(sig + dlt - kexp));
  const dfv d0 = df_from_double(__ldg(A.d));
  const double sw = pow2(-dlt);
  const float swf = (float)sw;
  const dfv wc = df_from_double((A.wc0 - xim) * sw);
  const float wh[5] = {A.wf[0] * swf, A.wf[2] * swf, A.wf[4] * swf, A.wf[6] * swf, wc.h};
  const float wl[5] = {A.wf[1] * swf, A.wf[3] * swf, A.wf[5] * swf, A.wf[7] * swf, wc.l};
  float2* dst = reinterpret_cast<float2*>((m & 1) ? A.y1 : A.y0);
  dfv accy = {0.f, 0.f}, accp = {0.f, 0.f};
  const int warp = threadIdx.x >> 5;
  unsigned long long* ring = pipe_smem + (size_t)warp * STAGES * kSlotElems;
  const float2* src = reinterpret_cast<const float2*>(((m - 1) & 1) ? A.y1 : A.y0);
  for_each_segment(nx, ny, H, blockIdx.x * kPipeWarps + warp, gridDim.x * kPipeWarps, [&](int col0, int r0, int r1) {
    if (m == 0)
      df_strip_pipe<STAGES, double, true>(A, A.w, dst, A.pdf, ring, col0, r0, r1, wh, wl, d0, dm1, sc, accy, accp);
    else
      df_strip_pipe<STAGES, float2, false>(A, src, dst, A.pdf, ring, col0, r0, r1, wh, wl, d0, dm1, sc, accy,
                                           accp);
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
// df64 Burgers: the Jacobian J(u) has point-wise weights
//   wE = lx - q, wW = lx + q, wN = ly - q dx/dy, wS = ly + q dx/dy, wC = r - xi_m
// with the per-point float pairs q and r prepared once per Leja loop.
// ---------------------------------------------------------------------------

constexpr int kSlotElemsB = kYSlot + 3 * kPipeRow;  // y (+halo), p, q, r
constexpr int kPipeSmemBytesB = kPipeWarps * kPipeStages * kSlotElemsB * 8;
constexpr int kPipeSmemBytesB4 = kPipeWarps * 4 * kSlotElemsB * 8;  // the 4-stage variant (3 blocks/SM)

__device__ __forceinline__ dfv df_add(dfv a, dfv b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  dfv r;
  fast_two_sum(s, e, r.h, r.l);
  return r;
}

__device__ __forceinline__ dfv df_neg(dfv a) { return {-a.h, -a.l}; }

// q = u gx and r = wc0 - s ig as float pairs (gx = 1/(2 dx gamma), ig = 1/gamma).
static __global__ void burgers_df_prep_kernel(long long n, const double* __restrict__ u, const double* __restrict__ s,
                                              double gx, double ig, double wc0, float2* __restrict__ q,
                                              float2* __restrict__ r) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const dfv a = df_split_scaled(u[i] * gx, 0);
    const dfv b = df_split_scaled(fma(-s[i], ig, wc0), 0);
    q[i] = make_float2(a.h, a.l);
    r[i] = make_float2(b.h, b.l);
  }
}

template <typename S, bool FIRST, int STAGES = kPipeStages>
__device__ __forceinline__ void df_strip_pipe_burgers(const LoopArgs& A, const S* __restrict__ src,
                                                      float2* __restrict__ dst, float2* __restrict__ p,
                                                      unsigned long long* ring, int col0, int r0, int r1, dfv xim,
                                                      float swf, dfv d0, dfv dm1, int sc, dfv& accy, dfv& accp) {
  const int lane = threadIdx.x & 31;
  const int nx = A.nx, ny = A.ny;
  const int c = col0 + lane * 4;
  const int cw = col0 == 0 ? nx - 1 : col0 - 1;
  const int ce = (col0 + kPipeRow >= nx) ? 0 : col0 + kPipeRow;
  const int nrows = r1 - r0;
  const int last_q = nrows + 1;
  const dfv lx = {A.bl[0], A.bl[1]}, ly = {A.bl[2], A.bl[3]}, rat = {A.bl[4], A.bl[5]};
  const bool square = A.bl[4] == 1.0f && A.bl[5] == 0.0f && A.bl[0] == A.bl[2] && A.bl[1] == A.bl[3];
  auto slot = [&](int q) { return ring + (size_t)(q % STAGES) * kSlotElemsB; };
  auto issue = [&](int q) {
    if (q <= last_q) {
      int ry = r0 - 1 + q;
      ry = ry < 0 ? ry + ny : (ry >= ny ? ry - ny : ry);
      unsigned long long* s = slot(q);
      const S* row = src + (size_t)ry * nx;
      cp_async16(s + 2 + lane * 4, row + c);
      cp_async16(s + 4 + lane * 4, row + c + 2);
      if (lane == 0) cp_async8(s + 1, row + cw);
      if (lane == 31) cp_async8(s + 2 + kPipeRow, row + ce);
      if (q >= 1 && q <= nrows) {
        const size_t ro = (size_t)(r0 - 1 + q) * nx;
        if constexpr (!FIRST) {
          cp_async16(s + kYSlot + lane * 4, p + ro + c);
          cp_async16(s + kYSlot + lane * 4 + 2, p + ro + c + 2);
        }
        cp_async16(s + kYSlot + kPipeRow + lane * 4, A.bq + ro + c);
        cp_async16(s + kYSlot + kPipeRow + lane * 4 + 2, A.bq + ro + c + 2);
        cp_async16(s + kYSlot + 2 * kPipeRow + lane * 4, A.br + ro + c);
        cp_async16(s + kYSlot + 2 * kPipeRow + lane * 4 + 2, A.br + ro + c + 2);
      }
    }
    cp_commit();
  };
  for (int q = 0; q < STAGES - 1; ++q) issue(q);
  cp_wait<STAGES - 3>();
  __syncwarp();
  dfv ys[4], yc[4], yn[4];
  df_from_raw4<S>(slot(0) + 2 + lane * 4, sc, ys);
  df_from_raw4<S>(slot(1) + 2 + lane * 4, sc, yc);
  for (int qc = 1; qc <= nrows; ++qc) {
    issue(qc + STAGES - 2);
    cp_wait<STAGES - 3>();
    __syncwarp();
    const unsigned long long* sn = slot(qc + 1);
    const unsigned long long* scn = slot(qc);
    df_from_raw4<S>(sn + 2 + lane * 4, sc, yn);
    dfv pold[4], qv[4], rv[4];
    if constexpr (!FIRST) df_from_raw4<float2>(scn + kYSlot + lane * 4, sc, pold);
    df_from_raw4<float2>(scn + kYSlot + kPipeRow + lane * 4, sc, qv);
    df_from_raw4<float2>(scn + kYSlot + 2 * kPipeRow + lane * 4, sc, rv);
    dfv xw = shfl_up_df(yc[3]);
    dfv xe = shfl_down_df(yc[0]);
    if (lane == 0) xw = df_from_raw<S>(scn + 1, sc);
    if (lane == 31) xe = df_from_raw<S>(scn + 2 + kPipeRow, sc);
    dfv ynew[4], pnew[4];
    float fy = 0.f, fp = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const dfv ye = k == 3 ? xe : yc[k + 1], yw = k == 0 ? xw : yc[k - 1];
      const dfv wE = df_add(lx, df_neg(qv[k])), wW = df_add(lx, qv[k]);
      const dfv wC = df_add(rv[k], xim);
      dfv v;
      if (square) {
        // nx == ny: the north and south weights equal the east and west ones,
        // so J y = wE (yE + yN) + wW (yW + yS) + wC yC (three products)
        const float wh[3] = {wE.h, wW.h, wC.h};
        const float wl[3] = {wE.l, wW.l, wC.l};
        const dfv t[3] = {df_add(ye, yn[k]), df_add(yw, ys[k]), yc[k]};
        v = df_dot3(wh, wl, t);
      } else {
        const dfv qy = df_mul(qv[k], rat);
        const dfv wN = df_add(ly, df_neg(qy)), wS = df_add(ly, qy);
        const float wh[5] = {wE.h, wW.h, wN.h, wS.h, wC.h};
        const float wl[5] = {wE.l, wW.l, wN.l, wS.l, wC.l};
        const dfv t[5] = {ye, yw, yn[k], ys[k], yc[k]};
        v = df_dot5(wh, wl, t);
      }
      v.h *= swf;
      v.l *= swf;
      ynew[k] = v;
      const dfv po = FIRST ? df_mul(d0, yc[k]) : pold[k];
      pnew[k] = df_axpy(dm1, ynew[k], po);
      fy = __fmaf_rn(ynew[k].h, ynew[k].h, fy);
      fp = __fmaf_rn(pnew[k].h, pnew[k].h, fp);
    }
    df_acc(accy, fy);
    df_acc(accp, fp);
    const size_t ro = (size_t)(r0 - 1 + qc) * nx;
    df_store_row<4>(dst + ro, c, nx, ynew);
    df_store_row<4>(p + ro, c, nx, pnew);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ys[k] = yc[k];
      yc[k] = yn[k];
    }
    __syncwarp();
  }
  cp_wait<0>();
  __syncwarp();
}

template <int MINB, int STAGES = kPipeStages>
__global__ void __launch_bounds__(kPipeThreads, MINB)
    leja_iter_df_pipe_burgers_kernel(const LoopArgs* __restrict__ Ap, LoopState* __restrict__ st,
                                     double* __restrict__ partials, unsigned int* __restrict__ ticket,
                                     cudaGraphConditionalHandle cond) {
  extern __shared__ __align__(16) unsigned long long pipe_smem_b[];
  const LoopArgs& A = *Ap;
  const int m = __ldcg(&st->m);
  count_launch(st);
  if (__ldcg(&st->done)) return;
  const int kexp = __ldcg(&st->kscale);
  const int sig = __ldcg(&st->sig);
  const int dlt = __ldcg(&st->dlt);
  const int nx = A.nx, ny = A.ny;
  const int H = A.strip_h;
  const double xim_d = __ldg(A.xi + m);
  const double dm1d = __ldg(A.d + m + 1);
  const dfv dm1 = df_from_double(dm1d * pow2(sig + dlt - kexp));
  const dfv d0 = df_from_double(__ldg(A.d));
  const dfv xim = df_from_double(-xim_d);
  const float swf = (float)pow2(-dlt);
  float2* dst = reinterpret_cast<float2*>((m & 1) ? A.y1 : A.y0);
  dfv accy = {0.f, 0.f}, accp = {0.f, 0.f};
  const int warp = threadIdx.x >> 5;
  unsigned long long* ring = pipe_smem_b + (size_t)warp * STAGES * kSlotElemsB;
  const float2* src = reinterpret_cast<const float2*>(((m - 1) & 1) ? A.y1 : A.y0);
  for_each_segment(nx, ny, H, blockIdx.x * kPipeWarps + warp, gridDim.x * kPipeWarps, [&](int col0, int r0, int r1) {
    if (m == 0)
      df_strip_pipe_burgers<double, true, STAGES>(A, A.w, dst, A.pdf, ring, col0, r0, r1, xim, swf, d0, dm1, kexp, accy,
                                          accp);
    else
      df_strip_pipe_burgers<float2, false, STAGES>(A, src, dst, A.pdf, ring, col0, r0, r1, xim, swf, d0, dm1, kexp, accy,
                                           accp);
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

// ---------------------------------------------------------------------------
// df64 power-iteration pass: w = Op(v) / ||v|| with Op = A (KIND 0, constant
// weights W) or J(u) (KIND 1, point-wise weights from q = u/(2dx),
// r = -2nu/dx^2 - 2nu/dy^2 - (u_x+u_y)); v is the caller's double start
// vector on the first pass (vin_double = 1), float pairs afterwards.
// ---------------------------------------------------------------------------
struct PowWeights {
  float w[10];   // KIND 0: hi/lo of wE, wW, wN, wS, wC
  float bl[6];   // KIND 1: hi/lo of lx = nu/dx^2, ly = nu/dy^2, dx/dy
};

template <int KIND>
static __global__ void __launch_bounds__(kThreadsPerBlock)
    power_pass_df_kernel(Geo g, const void* __restrict__ vin, int vin_double, float2* __restrict__ w,
                         const float2* __restrict__ q, const float2* __restrict__ r, PowWeights W,
                         double* __restrict__ partials, unsigned int* __restrict__ ticket, LoopState* st) {
  if (__ldcg(&st->pdone)) return;
  const dfv sg = df_from_double(__ldcg(&st->sigma));
  dfv acc = {0.f, 0.f};
  float small = 0.f;
  const double* vd = reinterpret_cast<const double*>(vin);
  const float2* vf = reinterpret_cast<const float2*>(vin);
  auto ld = [&](long long i) -> dfv {
    if (vin_double) return df_split_scaled(__ldg(vd + i), 0);
    const float2 t = __ldg(vf + i);
    return {t.x, t.y};
  };
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.n; i += (long long)gridDim.x * blockDim.x) {
    long long e, ww, nn, ss;
    neighbours(g, i, e, ww, nn, ss);
    const dfv t[5] = {ld(e), ld(ww), ld(nn), ld(ss), ld(i)};
    float wh[5], wl[5];
    if (KIND == 0) {
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        wh[k] = W.w[2 * k];
        wl[k] = W.w[2 * k + 1];
      }
    } else {
      const float2 qq = __ldg(q + i), rr = __ldg(r + i);
      const dfv qx = {qq.x, qq.y}, rv = {rr.x, rr.y};
      const dfv lx = {W.bl[0], W.bl[1]}, ly = {W.bl[2], W.bl[3]}, rat = {W.bl[4], W.bl[5]};
      const dfv qy = df_mul(qx, rat);
      const dfv wE = df_add(lx, df_neg(qx)), wW = df_add(lx, qx), wN = df_add(ly, df_neg(qy)), wS = df_add(ly, qy);
      wh[0] = wE.h; wl[0] = wE.l;
      wh[1] = wW.h; wl[1] = wW.l;
      wh[2] = wN.h; wl[2] = wN.l;
      wh[3] = wS.h; wl[3] = wS.l;
      wh[4] = rv.h; wl[4] = rv.l;
    }
    const dfv y = df_mul(sg, df_dot5(wh, wl, t));
    w[i] = make_float2(y.h, y.l);
    // exact square of the leading float plus the cross term 2 h l: the
    // power estimate rho = ||w|| must carry double accuracy
    float sq, se;
    two_prod(y.h, y.h, sq, se);
    df_acc(acc, sq);
    small = __fmaf_rn(2.f * y.h, y.l, __fadd_rn(small, se));
  }
  double s = df_to_double(acc) + (double)small, dummy = 0.0;
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

// The same power-iteration pass in row-strip form (nx % 128 == 0, 16-byte
// aligned vectors): warps take balanced row ranges of 128-column strips,
// each lane four consecutive points; the rows of v (one-point halo per side)
// and, for J(u), of q and r arrive in a per-warp cp.async ring STAGES - 3
// rows ahead of use, so loads overlap the arithmetic, and v is split once
// per row.  ||w||^2 is accumulated with exact squares of the leading floats
// (float-float) plus the cross terms in float, as in power_pass_df_kernel.
template <int KIND>
__host__ __device__ constexpr int pow_slot_elems() {
  return kRhsSlot + (KIND == 1 ? 2 * kPipeRow : 0);
}
template <int KIND, int STAGES>
constexpr int pow_rows_smem_bytes() {
  return kPipeWarps * STAGES * pow_slot_elems<KIND>() * 8;
}

template <int KIND, int STAGES, typename S>
__device__ __forceinline__ void pow_strip(int nx, int ny, const S* __restrict__ v, float2* __restrict__ w,
                                          const float2* __restrict__ q, const float2* __restrict__ r,
                                          const PowWeights& W, unsigned long long* ring, int col0, int r0, int r1,
                                          dfv sg, dfv& acc, float& small) {
  const int lane = threadIdx.x & 31;
  const int c = col0 + lane * 4;
  const int cw = col0 == 0 ? nx - 1 : col0 - 1;
  const int ce = (col0 + kPipeRow >= nx) ? 0 : col0 + kPipeRow;
  const int last_q = r1 - r0 + 1;  // rows q = 0 .. last_q are grid rows r0 - 1 .. r1
  constexpr int kSlot = pow_slot_elems<KIND>();
  auto slot = [&](int qq) { return ring + (size_t)(qq % STAGES) * kSlot; };
  auto issue = [&](int qq) {
    if (qq <= last_q) {
      int ry = r0 - 1 + qq;
      ry = ry < 0 ? ry + ny : (ry >= ny ? ry - ny : ry);
      const S* row = v + (size_t)ry * nx;
      unsigned long long* sl = slot(qq);
      cp_async16(sl + 2 + lane * 4, row + c);
      cp_async16(sl + 4 + lane * 4, row + c + 2);
      if (lane == 0) cp_async8(sl + 1, row + cw);
      if (lane == 31) cp_async8(sl + 2 + kPipeRow, row + ce);
      if constexpr (KIND == 1) {
        // the point weights of this row, used when it is the centre row
        const size_t o = (size_t)ry * nx + c;
        cp_async16(sl + kRhsSlot + lane * 4, q + o);
        cp_async16(sl + kRhsSlot + lane * 4 + 2, q + o + 2);
        cp_async16(sl + kRhsSlot + kPipeRow + lane * 4, r + o);
        cp_async16(sl + kRhsSlot + kPipeRow + lane * 4 + 2, r + o + 2);
      }
    }
    cp_commit();
  };
  for (int qq = 0; qq < STAGES - 1; ++qq) issue(qq);
  cp_wait<STAGES - 3>();
  __syncwarp();
  dfv ys[4], yc[4], yn[4];
  df_from_raw4<S>(slot(0) + 2 + lane * 4, 0, ys);
  df_from_raw4<S>(slot(1) + 2 + lane * 4, 0, yc);
  float wh[5], wl[5];
  if constexpr (KIND == 0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      wh[k] = W.w[2 * k];
      wl[k] = W.w[2 * k + 1];
    }
  }
  for (int qc = 1; qc < last_q; ++qc) {
    issue(qc + STAGES - 2);
    cp_wait<STAGES - 3>();
    __syncwarp();
    const unsigned long long* sn = slot(qc + 1);
    const unsigned long long* scn = slot(qc);
    df_from_raw4<S>(sn + 2 + lane * 4, 0, yn);
    dfv xw = shfl_up_df(yc[3]);
    dfv xe = shfl_down_df(yc[0]);
    if (lane == 0) xw = df_from_raw<S>(scn + 1, 0);
    if (lane == 31) xe = df_from_raw<S>(scn + 2 + kPipeRow, 0);
    dfv qv[4], rv[4];
    if constexpr (KIND == 1) {
      df_from_raw4<float2>(scn + kRhsSlot + lane * 4, 0, qv);
      df_from_raw4<float2>(scn + kRhsSlot + kPipeRow + lane * 4, 0, rv);
    }
    dfv out[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if constexpr (KIND == 1) {
        const dfv lx = {W.bl[0], W.bl[1]}, ly = {W.bl[2], W.bl[3]}, rat = {W.bl[4], W.bl[5]};
        const dfv qy = df_mul(qv[k], rat);
        const dfv wE = df_add(lx, df_neg(qv[k])), wW = df_add(lx, qv[k]), wN = df_add(ly, df_neg(qy)),
                  wS = df_add(ly, qy);
        wh[0] = wE.h;
        wl[0] = wE.l;
        wh[1] = wW.h;
        wl[1] = wW.l;
        wh[2] = wN.h;
        wl[2] = wN.l;
        wh[3] = wS.h;
        wl[3] = wS.l;
        wh[4] = rv[k].h;
        wl[4] = rv[k].l;
      }
      const dfv t[5] = {k == 3 ? xe : yc[k + 1], k == 0 ? xw : yc[k - 1], yn[k], ys[k], yc[k]};
      out[k] = df_mul(sg, df_dot5(wh, wl, t));
      float sq, se;
      two_prod(out[k].h, out[k].h, sq, se);
      df_acc(acc, sq);
      small = __fmaf_rn(2.f * out[k].h, out[k].l, __fadd_rn(small, se));
    }
    df_store_row<4>(w + (size_t)(r0 - 1 + qc) * nx, c, nx, out);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ys[k] = yc[k];
      yc[k] = yn[k];
    }
    __syncwarp();
  }
  cp_wait<0>();
  __syncwarp();
}

template <int KIND, int STAGES>
static __global__ void __launch_bounds__(kPipeThreads)
    power_pass_df_rows_kernel(int nx, int ny, long long n, const void* __restrict__ vin, int vin_double,
                              float2* __restrict__ w, const float2* __restrict__ q, const float2* __restrict__ r,
                              PowWeights W, double* __restrict__ partials, unsigned int* __restrict__ ticket,
                              LoopState* st) {
  extern __shared__ __align__(16) unsigned long long pow_ring[];
  if (__ldcg(&st->pdone)) return;
  const dfv sg = df_from_double(__ldcg(&st->sigma));
  dfv acc = {0.f, 0.f};
  float small = 0.f;
  const int warp = threadIdx.x >> 5;
  unsigned long long* ring = pow_ring + (size_t)warp * STAGES * pow_slot_elems<KIND>();
  for_each_segment(nx, ny, 0, blockIdx.x * kPipeWarps + warp, gridDim.x * kPipeWarps, [&](int col0, int r0, int r1) {
    if (vin_double)
      pow_strip<KIND, STAGES, double>(nx, ny, reinterpret_cast<const double*>(vin), w, q, r, W, ring, col0, r0, r1,
                                      sg, acc, small);
    else
      pow_strip<KIND, STAGES, float2>(nx, ny, reinterpret_cast<const float2*>(vin), w, q, r, W, ring, col0, r0, r1,
                                      sg, acc, small);
  });
  double s = df_to_double(acc) + (double)small, dummy = 0.0;
  if (!last_block_total2(s, dummy, partials, ticket)) return;
  if (threadIdx.x == 0) power_pass_finish(st, s, n);
}

}  // namespace lexgb

