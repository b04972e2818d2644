// Two Leja iterations per pass (temporal blocking) for the paper's upwind
// diffusion-advection operator, float-float form (Problems I and II of
// Sec. 3; the stencil and its weights are those of leja_upwind.cuh).
//
// One launch reads y_m and p_m once and writes y_{m+2} and p_{m+2}; y_{m+1}
// is recomputed on the rows and columns the second step needs and never
// stored.  The seven-point stencil reaches one point against the upwind side
// s and two along it, in both directions, so:
//   * rows are walked along s (ascending for s = +1, descending for s = -1):
//     in walk order every stencil takes the previous, the current and the
//     next two rows, whichever the side;
//   * y_{m+1} is needed on the output rows, one walk row before them and two
//     after, and y_m on one more before and two more after (nrows + 6 rows);
//   * across the warp's 128 columns y_{m+1} needs three halo points (one on
//     the -s side, two on the +s side), each computed from y_m with a
//     four-point ring halo on both sides (lane 0 computes the west pair,
//     lane 31 the east pair, the others a pair they do not use, so that no
//     branch diverges).
// The stopping test runs after every iteration exactly as in the central
// two-step kernel (four partial sums; an odd stop is undone by the output
// pass with p_{m+1} = p_{m+2} - d_{m+2} y_{m+2}).
#pragma once

#include "leja_upwind.cuh"

namespace lexgb {

constexpr int kY4Slot = kPipeRow + 8;  // [w4 w3 w2 w1][128 points][e1 e2 e3 e4]
constexpr int kSlotElemsU2 = kY4Slot + kPipeRow;  // y_m row, then the p_m row
template <int STAGES>
constexpr int up3_2step_smem_bytes() {
  return kPipeWarps * STAGES * kSlotElemsU2 * 8;
}

// Row r wrapped into [0, ny) (r within a few rows of the grid).
__device__ __forceinline__ int wrap_row_any(int r, int ny) {
  r %= ny;
  return r < 0 ? r + ny : r;
}

// Seven-point value at one point from [C, X(-s), X(s), X(2s), Y(-s), Y(s), Y(2s)].
__device__ __forceinline__ dfv up3_point(const float (&wh)[7], const float (&wl)[7], dfv c, dfv xm, dfv xp, dfv xp2,
                                         dfv ym, dfv yp, dfv yp2) {
  const dfv t[7] = {c, xm, xp, xp2, ym, yp, yp2};
  return df_dot7(wh, wl, t);
}

// One segment (rows r0..r1-1 of one 128-column strip).  S = double on the
// first launch (the caller's w, scaled by 2^-sc), else float2.  wa: weights
// of step m (with 2^-dlt folded in), wb: of step m+1.  acc: sums of
// y_{m+1}^2, p_{m+1}^2, y_{m+2}^2, p_{m+2}^2 over the output rows.
template <int STAGES, typename S, bool FIRST, int SG>
__device__ __forceinline__ void df2_strip_up3(const LoopArgs& A, const S* __restrict__ src, float2* __restrict__ dst,
                                              float2* __restrict__ p, unsigned long long* ring, int col0, int r0,
                                              int r1, const float (&wah)[7], const float (&wal)[7],
                                              const float (&wbh)[7], const float (&wbl)[7], dfv d0, dfv dm1, dfv dm2,
                                              int sc, dfv (&acc)[4]) {
  constexpr int s = SG;
  constexpr int AHEAD = STAGES - 4;
  static_assert(AHEAD >= 1, "four live rows plus at least one in flight");
  const int lane = threadIdx.x & 31;
  const int nx = A.nx, ny = A.ny;
  const int c = col0 + lane * 4;
  const int cw = col0 == 0 ? nx - 4 : col0 - 4;                  // first of the four west halo points
  const int ce = (col0 + kPipeRow >= nx) ? 0 : col0 + kPipeRow;  // first of the four east halo points
  const int nrows = r1 - r0;
  const int last_t = nrows + 5;  // walk rows t = 0 .. nrows+5
  // grid row of walk row t: r0-2+t ascending (s = +1), r1+1-t descending (s = -1)
  auto grow = [&](int t) { return s > 0 ? r0 - 2 + t : r1 + 1 - t; };
  auto slot = [&](int t) { return ring + (size_t)(t % STAGES) * kSlotElemsU2; };
  auto issue = [&](int t) {
    if (t <= last_t) {
      const int ry = wrap_row_any(grow(t), ny);
      unsigned long long* sl = slot(t);
      const S* row = src + (size_t)ry * nx;
      cp_async16(sl + 4 + lane * 4, row + c);
      cp_async16(sl + 6 + lane * 4, row + c + 2);
      if (lane == 0) {
        cp_async16(sl, row + cw);
        cp_async16(sl + 2, row + cw + 2);
      }
      if (lane == 31) {
        cp_async16(sl + 4 + kPipeRow, row + ce);
        cp_async16(sl + 6 + kPipeRow, row + ce + 2);
      }
      if constexpr (!FIRST) {
        // slot t also carries p_m of the output walk row t - 4
        if (t >= 6) {
          const float2* prow = p + (size_t)grow(t - 4) * nx;
          cp_async16(sl + kY4Slot + lane * 4, prow + c);
          cp_async16(sl + kY4Slot + lane * 4 + 2, prow + c + 2);
        }
      }
    }
    cp_commit();
  };
  // halo columns of this lane in a slot (index 4 + x for column col0 + x):
  // lane 0 the west pair (col0-1, col0-2), the others the east pair
  // (col0+128, col0+129; used by lane 31)
  const int hi1 = lane == 0 ? 3 : 4 + kPipeRow;
  const int hi2 = lane == 0 ? 2 : 5 + kPipeRow;
  // y_m at walk rows t-3 .. t (m0 .. m3), y_{m+1} at walk rows t-5 .. t-2
  // (b0 .. b3), and the y_{m+1} halo pairs of walk rows t-4 .. t-2
  dfv m0[4], m1[4], m2[4], m3[4];
  dfv b0[4], b1[4], b2[4], b3[4];
  dfv g1[2], g2[2], g3[2];
#pragma unroll
  for (int k = 0; k < 4; ++k) m0[k] = m1[k] = m2[k] = m3[k] = b0[k] = b1[k] = b2[k] = b3[k] = dfv{0.f, 0.f};
  g1[0] = g1[1] = g2[0] = g2[1] = g3[0] = g3[1] = dfv{0.f, 0.f};
  for (int t = 0; t < AHEAD; ++t) issue(t);
  for (int t = 0; t <= last_t; ++t) {
    issue(t + AHEAD);  // into the slot of walk row t - 4
    cp_wait<AHEAD>();  // walk row t complete
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      m0[k] = m1[k];
      m1[k] = m2[k];
      m2[k] = m3[k];
    }
    df_from_raw4<S>(slot(t) + 4 + lane * 4, sc, m3);
    if (t >= 3) {
      // step m: y_{m+1} on walk row t-2 (centre m1) and its halo pair
      const unsigned long long* sp = slot(t - 3);
      const unsigned long long* sc1 = slot(t - 2);
      const unsigned long long* sn = slot(t - 1);
      const unsigned long long* sn2 = slot(t);
      const dfv u3 = shfl_up_df(m1[3]), u2 = shfl_up_df(m1[2]);
      const dfv d0n = shfl_down_df(m1[0]), d1n = shfl_down_df(m1[1]);
      const dfv hw1 = df_from_raw<S>(sc1 + 3, sc), hw2 = df_from_raw<S>(sc1 + 2, sc);
      const dfv he1 = df_from_raw<S>(sc1 + 4 + kPipeRow, sc), he2 = df_from_raw<S>(sc1 + 5 + kPipeRow, sc);
      const dfv wm1 = lane == 0 ? hw1 : u3, wm2 = lane == 0 ? hw2 : u2;    // columns c-1, c-2
      const dfv ep1 = lane == 31 ? he1 : d0n, ep2 = lane == 31 ? he2 : d1n;  // columns c+4, c+5
      const dfv xm1[4] = {wm1, m1[0], m1[1], m1[2]};
      const dfv xm2[4] = {wm2, wm1, m1[0], m1[1]};
      const dfv xp1[4] = {m1[1], m1[2], m1[3], ep1};
      const dfv xp2[4] = {m1[2], m1[3], ep1, ep2};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        b0[k] = b1[k];
        b1[k] = b2[k];
        b2[k] = b3[k];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
        b3[k] = up3_point(wah, wal, m1[k], s > 0 ? xm1[k] : xp1[k], s > 0 ? xp1[k] : xm1[k],
                          s > 0 ? xp2[k] : xm2[k], m0[k], m2[k], m3[k]);
      // the halo pair: columns at slot indices hi1, hi2 of walk row t-2
      g1[0] = g2[0];
      g1[1] = g2[1];
      g2[0] = g3[0];
      g2[1] = g3[1];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int hi = q == 0 ? hi1 : hi2;
        g3[q] = up3_point(wah, wal, df_from_raw<S>(sc1 + hi, sc), df_from_raw<S>(sc1 + hi - s, sc),
                          df_from_raw<S>(sc1 + hi + s, sc), df_from_raw<S>(sc1 + hi + 2 * s, sc),
                          df_from_raw<S>(sp + hi, sc), df_from_raw<S>(sn + hi, sc), df_from_raw<S>(sn2 + hi, sc));
      }
    }
    if (t >= 6) {
      // step m+1: y_{m+2} on walk row t-4 (centre b1) from y_{m+1} rows t-5 .. t-2
      const dfv u3 = shfl_up_df(b1[3]), u2 = shfl_up_df(b1[2]);
      const dfv d0n = shfl_down_df(b1[0]), d1n = shfl_down_df(b1[1]);
      const dfv wm1 = lane == 0 ? g1[0] : u3, wm2 = lane == 0 ? g1[1] : u2;
      const dfv ep1 = lane == 31 ? g1[0] : d0n, ep2 = lane == 31 ? g1[1] : d1n;
      const dfv xm1[4] = {wm1, b1[0], b1[1], b1[2]};
      const dfv xm2[4] = {wm2, wm1, b1[0], b1[1]};
      const dfv xp1[4] = {b1[1], b1[2], b1[3], ep1};
      const dfv xp2[4] = {b1[2], b1[3], ep1, ep2};
      const int orow = grow(t - 4);
      const size_t ro = (size_t)orow * nx;
      dfv pold[4];
      if constexpr (FIRST) {
        // p_0 = d_0 y_0 on the output row (y_0: the caller's doubles)
        dfv y0[4];
        df_load_row<4>(reinterpret_cast<const double*>(src) + ro, c, nx, sc, y0);
#pragma unroll
        for (int k = 0; k < 4; ++k) pold[k] = df_mul(d0, y0[k]);
      } else {
        df_from_raw4<float2>(slot(t) + kY4Slot + lane * 4, 0, pold);
      }
      dfv yb[4], pb[4];
      float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const dfv p1 = df_axpy(dm1, b1[k], pold[k]);
        yb[k] = up3_point(wbh, wbl, b1[k], s > 0 ? xm1[k] : xp1[k], s > 0 ? xp1[k] : xm1[k], s > 0 ? xp2[k] : xm2[k],
                          b0[k], b2[k], b3[k]);
        pb[k] = df_axpy(dm2, yb[k], p1);
        f0 = __fmaf_rn(b1[k].h, b1[k].h, f0);
        f1 = __fmaf_rn(p1.h, p1.h, f1);
        f2 = __fmaf_rn(yb[k].h, yb[k].h, f2);
        f3 = __fmaf_rn(pb[k].h, pb[k].h, f3);
      }
      df_acc(acc[0], f0);
      df_acc(acc[1], f1);
      df_acc(acc[2], f2);
      df_acc(acc[3], f3);
      df_store_row<4>(dst + ro, c, nx, yb);
      df_store_row<4>(p + ro, c, nx, pb);
    }
    __syncwarp();
  }
  cp_wait<0>();
  __syncwarp();
}

// Launch m (even) of the two-step loop: y_m, p_m -> y_{m+2}, p_{m+2}.
template <int MINB, int STAGES>
__global__ void __launch_bounds__(kPipeThreads, MINB)
    leja_iter_df_pipe2_up3_kernel(const LoopArgs* __restrict__ Ap, LoopState* __restrict__ st,
                                  double* __restrict__ partials, unsigned int* __restrict__ ticket,
                                  cudaGraphConditionalHandle cond) {
  extern __shared__ __align__(16) unsigned long long up3b2_smem[];
  const LoopArgs& A = *Ap;
  const int m = __ldcg(&st->m);
  count_launch(st);
  if (__ldcg(&st->done)) return;
  const int kexp = __ldcg(&st->kscale);
  const int sig = __ldcg(&st->sig);
  const int dlt = __ldcg(&st->dlt);
  const Up3Op o = A.up;
  const double xa = __ldg(A.xi + m);
  const double xb = __ldg(A.xi + m + 1);
  const double dm1d = __ldg(A.d + m + 1);
  const double dm2d = __ldg(A.d + min(m + 2, A.kmax));  // unused when the loop ends at m+1 = kmax
  const double ys = pow2(sig + dlt - kexp);
  const dfv dm1 = df_from_double(dm1d * ys);
  const dfv dm2 = df_from_double(dm2d * ys);
  const dfv d0 = df_from_double(__ldg(A.d));
  const double sw = pow2(-dlt);
  double wd[7];
  up3_weights(o, wd);
  float wah[7], wal[7], wbh[7], wbl[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const double base = wd[k] * A.inv_gamma + (k == 0 ? -A.up_c * A.inv_gamma : 0.0);
    const dfv ta = df_from_double((base - (k == 0 ? xa : 0.0)) * sw);
    const dfv tb = df_from_double(base - (k == 0 ? xb : 0.0));
    wah[k] = ta.h;
    wal[k] = ta.l;
    wbh[k] = tb.h;
    wbl[k] = tb.l;
  }
  const int pass = m >> 1;
  float2* dst = reinterpret_cast<float2*>((pass & 1) ? A.y1 : A.y0);
  const float2* src = reinterpret_cast<const float2*>((pass & 1) ? A.y0 : A.y1);
  dfv acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  const int warp = threadIdx.x >> 5;
  unsigned long long* ring = up3b2_smem + (size_t)warp * STAGES * kSlotElemsU2;
  for_each_segment(o.nx, o.ny, A.strip_h, blockIdx.x * kPipeWarps + warp, gridDim.x * kPipeWarps,
                   [&](int col0, int r0, int r1) {
    if (m == 0) {
      if (o.s > 0)
        df2_strip_up3<STAGES, double, true, 1>(A, A.w, dst, A.pdf, ring, col0, r0, r1, wah, wal, wbh, wbl, d0, dm1,
                                               dm2, kexp, acc);
      else
        df2_strip_up3<STAGES, double, true, -1>(A, A.w, dst, A.pdf, ring, col0, r0, r1, wah, wal, wbh, wbl, d0, dm1,
                                                dm2, kexp, acc);
    } else {
      if (o.s > 0)
        df2_strip_up3<STAGES, float2, false, 1>(A, src, dst, A.pdf, ring, col0, r0, r1, wah, wal, wbh, wbl, d0, dm1,
                                                dm2, kexp, acc);
      else
        df2_strip_up3<STAGES, float2, false, -1>(A, src, dst, A.pdf, ring, col0, r0, r1, wah, wal, wbh, wbl, d0,
                                                 dm1, dm2, kexp, acc);
    }
  });
  double v[4] = {df_to_double(acc[0]), df_to_double(acc[1]), df_to_double(acc[2]), df_to_double(acc[3])};
  if (!last_block_total_n<4>(v, partials, ticket)) return;
  if (threadIdx.x == 0) {
    const double yscale = pow2(sig + dlt), pscale = pow2(kexp);
    leja_finalize(A, st, m, dm1d, v[0], v[1], yscale, pscale, cond);
    if (!st->done) {
      leja_finalize(A, st, m + 1, dm2d, v[2], v[3], yscale, pscale, cond);
    } else {
      st->fix = 1;  // p holds p_{m+2}: the output pass subtracts d_{m+2} y_{m+2}
      st->fix_d = dm2d * ys;
      st->fix_buf = pass & 1;
    }
    const double rms = sqrt(v[2] / double(A.n));
    int e = 0;
    if (rms > 0.0 && isfinite(rms)) e = ilogb(rms);
    st->sig = sig + dlt;
    st->dlt = max(-100, min(100, e));
  }
}

}  // namespace lexgb
