// Two Leja iterations per pass over memory for the paper's upwind
// diffusion-advection operator, float-float form (Problems I and II of
// Sec. 3): the issue-lean variant of leja_iter_df_pipe2_up3_kernel, built
// the way leja_iter_df_pipe2x_kernel is built for the central operator.
//
// The arithmetic is that of the two-step kernel (Sec. 2.1, Eq. 2, applied
// twice per launch; the seven-point stencil [C, X(-s), X(s), X(2s), Y(-s),
// Y(s), Y(2s)] of up3_weights, rows walked along the upwind side s).  Against
// the first form:
//  * square grids with equal x and y coefficients (the x and y weights at
//    each offset coincide) take the pair sums P(o) = X(o) + Y(o) for
//    o = -s, s, 2s and a four-term compensated dot product; P(-s) at
//    (g, i) is P(s) at (g - s, i - s), the previous walk row one column
//    over (the same two operands, so the same value), so it is carried;
//  * the values of y_{m+1} at the strip's three halo columns (one on the
//    -s side, two on the s side) are computed for 16 output rows at a time,
//    two stencils per lane, from their seven inputs each, copied into shared
//    memory with cp.async half a chunk ahead -- instead of two stencils by
//    every lane on every row;
//  * final renormalisations by Fast2Sum; the two Newton updates of p as one
//    compensated three-term sum; sums of squares in float over 16 rows.
#pragma once

#include "leja_df64_2step_x.cuh"
#include "leja_upwind_2step.cuh"

namespace lexgb {

constexpr int kHaloU2x = 14;  // per lane: two halo tasks of seven inputs

template <int STAGES>
constexpr int pipe2x_up3_smem_bytes() {
  return kPipeWarps * STAGES * kSlotElems2 * 8 + kPipeWarps * 32 * kHaloU2x * 8;
}

// One point of the square form from its centre and pair sums (weights in
// the order C, X(-s), X(s), X(2s); the Y weights equal them).
__device__ __forceinline__ dfv up3_point_sq(const float (&wh)[7], const float (&wl)[7], dfv c, dfv pms, dfv ps,
                                            dfv p2s) {
  const float h4[4] = {wh[0], wh[1], wh[2], wh[3]};
  const float l4[4] = {wl[0], wl[1], wl[2], wl[3]};
  const dfv t[4] = {c, pms, ps, p2s};
  return df_dot_n<4>(h4, l4, t);
}

// One point from the seven values in the order of up3_weights.
template <bool SQ>
__device__ __forceinline__ dfv up3x_point(const float (&wh)[7], const float (&wl)[7], dfv c, dfv xms, dfv xs,
                                          dfv x2s, dfv yms, dfv ys, dfv y2s) {
  if constexpr (SQ)
    return up3_point_sq(wh, wl, c, df_add_loose(xms, yms), df_add_loose(xs, ys), df_add_loose(x2s, y2s));
  else
    return up3_point(wh, wl, c, xms, xs, x2s, yms, ys, y2s);
}

// Halo task tau (0..47) of the chunk at output rows o_base .. o_base + 15:
// row o_base + (tau & 15) (rows past the last repeat it), column tau >> 4 of
// {the -s side's first, the s side's first, the s side's second}.
template <int SG>
__device__ __forceinline__ int up3x_halo_col(int col0, int nx, int ci) {
  const int w1 = col0 == 0 ? nx - 1 : col0 - 1;
  const int w2 = col0 == 0 ? nx - 2 : col0 - 2;  // col0 >= 128 otherwise
  const int e1 = col0 + kPipeRow >= nx ? 0 : col0 + kPipeRow;
  const int e2 = e1 + 1;
  if constexpr (SG > 0)
    return ci == 0 ? w1 : (ci == 1 ? e1 : e2);
  else
    return ci == 0 ? e1 : (ci == 1 ? w1 : w2);
}

// Copies the seven inputs (y_m at C, X(-s), X(s), X(2s), Y(-s), Y(s), Y(2s))
// of this lane's halo tasks into its hbuf entries.  grow(j): grid row of
// output index j (the walk maps output index j to walk row j + 2).
template <typename S, int SG, typename GR>
__device__ __forceinline__ void up3x_halo_issue(const S* __restrict__ src, int nx, int ny, int col0, int o_base,
                                                int nrows, GR grow, unsigned long long* hbuf) {
  constexpr int s = SG;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int tau = lane + 32 * q;
    if (tau < 48) {
      const int o = min(o_base + (tau & 15), nrows - 1);
      const int g = grow(o + 2);
      const int x = up3x_halo_col<SG>(col0, nx, tau >> 4);
      const int xm = x - s < 0 ? x - s + nx : (x - s >= nx ? x - s - nx : x - s);
      const int xp = x + s < 0 ? x + s + nx : (x + s >= nx ? x + s - nx : x + s);
      const int xp2 = x + 2 * s < 0 ? x + 2 * s + nx : (x + 2 * s >= nx ? x + 2 * s - nx : x + 2 * s);
      const size_t rg = (size_t)g * nx;
      const size_t rm = (size_t)wrap_row_any(g - s, ny) * nx;
      const size_t rp = (size_t)wrap_row_any(g + s, ny) * nx;
      const size_t rp2 = (size_t)wrap_row_any(g + 2 * s, ny) * nx;
      unsigned long long* h = hbuf + lane * kHaloU2x + 7 * q;
      cp_async8(h + 0, src + rg + x);
      cp_async8(h + 1, src + rg + xm);
      cp_async8(h + 2, src + rg + xp);
      cp_async8(h + 3, src + rg + xp2);
      cp_async8(h + 4, src + rm + x);
      cp_async8(h + 5, src + rp + x);
      cp_async8(h + 6, src + rp2 + x);
    }
  }
}

// y_{m+1} (step-m weights) at this lane's two halo tasks.
template <typename S, bool SQ>
__device__ __forceinline__ void up3x_halo_compute(const unsigned long long* hbuf, int sc, const float (&wh)[7],
                                                  const float (&wl)[7], dfv& hv0, dfv& hv1) {
  const int lane = threadIdx.x & 31;
  const unsigned long long* h = hbuf + lane * kHaloU2x;
  hv0 = up3x_point<SQ>(wh, wl, df_from_raw<S>(h + 0, sc), df_from_raw<S>(h + 1, sc), df_from_raw<S>(h + 2, sc),
                       df_from_raw<S>(h + 3, sc), df_from_raw<S>(h + 4, sc), df_from_raw<S>(h + 5, sc),
                       df_from_raw<S>(h + 6, sc));
  if (lane < 16) {
    h += 7;
    hv1 = up3x_point<SQ>(wh, wl, df_from_raw<S>(h + 0, sc), df_from_raw<S>(h + 1, sc), df_from_raw<S>(h + 2, sc),
                         df_from_raw<S>(h + 3, sc), df_from_raw<S>(h + 4, sc), df_from_raw<S>(h + 5, sc),
                         df_from_raw<S>(h + 6, sc));
  }
}

// The X neighbours X(-s), X(s), X(2s) of a lane's four points k of one row v
// (two-point halos lw1, lw2 west and le1, le2 east at lanes 0 and 31; the
// other lanes' halo arguments are unused).
template <int SG>
__device__ __forceinline__ void up3x_xnb(const dfv (&v)[4], dfv lw1, dfv lw2, dfv le1, dfv le2, dfv (&xms)[4],
                                         dfv (&xs)[4], dfv (&x2s)[4]) {
  const int lane = threadIdx.x & 31;
  if constexpr (SG > 0) {
    dfv u3 = shfl_up_df(v[3]);
    dfv d0 = shfl_down_df(v[0]), d1 = shfl_down_df(v[1]);
    if (lane == 0) u3 = lw1;
    if (lane == 31) {
      d0 = le1;
      d1 = le2;
    }
    xms[0] = u3;
    xms[1] = v[0];
    xms[2] = v[1];
    xms[3] = v[2];
    xs[0] = v[1];
    xs[1] = v[2];
    xs[2] = v[3];
    xs[3] = d0;
    x2s[0] = v[2];
    x2s[1] = v[3];
    x2s[2] = d0;
    x2s[3] = d1;
  } else {
    dfv d0 = shfl_down_df(v[0]);
    dfv u3 = shfl_up_df(v[3]), u2 = shfl_up_df(v[2]);
    if (lane == 31) d0 = le1;
    if (lane == 0) {
      u3 = lw1;
      u2 = lw2;
    }
    xms[0] = v[1];
    xms[1] = v[2];
    xms[2] = v[3];
    xms[3] = d0;
    xs[0] = u3;
    xs[1] = v[0];
    xs[2] = v[1];
    xs[3] = v[2];
    x2s[0] = u2;
    x2s[1] = u3;
    x2s[2] = v[0];
    x2s[3] = v[1];
  }
}

// One segment (rows r0..r1-1 of one 128-column strip), rows walked along s:
// walk row j is grid row r0 - 2 + j (s = +1) or r1 + 1 - j (s = -1); y_m is
// read on walk rows 0 .. nrows+5, y_{m+1} formed on walk rows 1 .. nrows+3,
// y_{m+2} on the output walk rows 2 .. nrows+1.  S = double on the first
// launch (the caller's w, scaled by 2^-sc), else float2.  wa: weights of
// step m (with 2^-dlt folded in), wb: of step m+1.  acc: sums of
// y_{m+1}^2, p_{m+1}^2, y_{m+2}^2, p_{m+2}^2 over the output rows.
template <int STAGES, typename S, bool FIRST, int SG, bool SQ>
__device__ __forceinline__ void up3x_strip(const LoopArgs& A, const S* __restrict__ src, float2* __restrict__ dst,
                                           float2* __restrict__ p, unsigned long long* ring,
                                           unsigned long long* hbuf, int col0, int r0, int r1,
                                           const float (&wah)[7], const float (&wal)[7], const float (&wbh)[7],
                                           const float (&wbl)[7], dfv d0, dfv dm1, dfv dm2, int sc,
                                           dfv (&acc)[4]) {
  constexpr int s = SG;
  constexpr int AHEAD = STAGES - 4;
  static_assert(AHEAD >= 1 && AHEAD <= 8, "four live rows plus rows in flight; halo inputs 8 rows ahead");
  constexpr int KE = s > 0 ? 0 : 3;  // the lane's point whose (-s) pair is not carried
  const int lane = threadIdx.x & 31;
  const int nx = A.nx, ny = A.ny;
  const int c = col0 + lane * 4;
  const int cw = col0 == 0 ? nx - 2 : col0 - 2;                  // first of the two west halo points
  const int ce = (col0 + kPipeRow >= nx) ? 0 : col0 + kPipeRow;  // first of the two east halo points
  const int nrows = r1 - r0;
  const int last_t = nrows + 5;
  auto grow = [&](int j) { return s > 0 ? r0 - 2 + j : r1 + 1 - j; };
  auto slot = [&](int t) { return ring + (size_t)((unsigned)t % STAGES) * kSlotElems2; };
  auto issue = [&](int t) {
    // halo inputs of the next 16 output rows, 8 rows before they are needed
    // (output index o is formed at walk row o + 6)
    const int oq = t - AHEAD - 6;
    if (oq >= 0 && (oq & 15) == 8 && oq + 8 < nrows)
      up3x_halo_issue<S, SG>(src, nx, ny, col0, oq + 8, nrows, [&](int j) { return wrap_row_any(grow(j), ny); },
                             hbuf);
    if (t <= last_t) {
      const int ry = wrap_row_any(grow(t), ny);
      unsigned long long* sl = slot(t);
      const S* row = src + (size_t)ry * nx;
      cp_async16(sl + 2 + lane * 4, row + c);
      cp_async16(sl + 4 + lane * 4, row + c + 2);
      if (lane == 0) cp_async16(sl, row + cw);
      if (lane == 31) cp_async16(sl + 2 + kPipeRow, row + ce);
      if constexpr (!FIRST) {
        // slot t also carries p_m of the output walk row t - 4
        if (t >= 6) {
          const float2* prow = p + (size_t)grow(t - 4) * nx;
          cp_async16(sl + kY2Slot + lane * 4, prow + c);
          cp_async16(sl + kY2Slot + lane * 4 + 2, prow + c + 2);
        }
      }
    }
    cp_commit();
  };
  // y_m at walk rows t-3 .. t (M0 .. M3), y_{m+1} at walk rows t-5 .. t-2
  // (B0 .. B3); qa / qb: the s-pairs of the previous y_m / y_{m+1} row
  // (indices k - s of the next row's carried -s pairs)
  dfv M0[4], M1[4], M2[4], M3[4], B0[4], B1[4], B2[4], B3[4];
  dfv qa[4], qb[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    M0[k] = M1[k] = M2[k] = M3[k] = B0[k] = B1[k] = B2[k] = B3[k] = dfv{0.f, 0.f};
    qa[k] = qb[k] = dfv{0.f, 0.f};
  }
  dfv hv0 = {0.f, 0.f}, hv1 = {0.f, 0.f};  // this lane's halo values of the current 16-row chunk
  float fs[4] = {0.f, 0.f, 0.f, 0.f};
  up3x_halo_issue<S, SG>(src, nx, ny, col0, 0, nrows, [&](int j) { return wrap_row_any(grow(j), ny); },
                         hbuf);  // chunk 0, in the first commit group
  for (int t = 0; t < AHEAD; ++t) issue(t);
  for (int t = 0; t <= last_t; ++t) {
    issue(t + AHEAD);  // into the slot of walk row t - 4
    cp_wait<AHEAD>();  // walk row t complete
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      M0[k] = M1[k];
      M1[k] = M2[k];
      M2[k] = M3[k];
    }
    df_from_raw4<S>(slot(t) + 2 + lane * 4, sc, M3);
    if (t >= 3) {
      // step m: y_{m+1} on walk row t-2 (centre M1)
      const unsigned long long* sc1 = slot(t - 2);
      dfv xms[4], xs[4], x2s[4];
      up3x_xnb<SG>(M1, df_from_raw<S>(sc1 + 1, sc), df_from_raw<S>(sc1 + 0, sc), df_from_raw<S>(sc1 + 2 + kPipeRow, sc),
                   df_from_raw<S>(sc1 + 3 + kPipeRow, sc), xms, xs, x2s);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        B0[k] = B1[k];
        B1[k] = B2[k];
        B2[k] = B3[k];
      }
      if constexpr (SQ) {
        if (t == 3) {
          // the s-pairs of walk row 0 (M0), for walk row 1's carried pairs
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int kx = k + s;  // X(s) of M0 at k, within the lane where it is used
            if (kx >= 0 && kx < 4) qa[k] = df_add_loose(M0[kx], M1[k]);
          }
        }
        dfv ps[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) ps[k] = df_add_loose(xs[k], M2[k]);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const dfv pms = k == KE ? df_add_loose(xms[k], M0[k]) : qa[k - s];
          B3[k] = up3_point_sq(wah, wal, M1[k], pms, ps[k], df_add_loose(x2s[k], M3[k]));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) qa[k] = ps[k];
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) B3[k] = up3_point(wah, wal, M1[k], xms[k], xs[k], x2s[k], M0[k], M2[k], M3[k]);
      }
    }
    if (t >= 6) {
      // step m+1: y_{m+2} on walk row t-4 = output index o (centre B1)
      const int o = t - 6;
      if ((o & 15) == 0) {
        // a new chunk of 16 output rows: its halo values of y_{m+1} (the
        // inputs arrived with the ring's copies at least 8 rows earlier)
        df_flush4(acc, fs);
        up3x_halo_compute<S, SQ>(hbuf, sc, wah, wal, hv0, hv1);
      }
      const int r = o & 15;
      // lane 0 and lane 31 take their halo values: the -s side's first is
      // task r (hv0 of lane r), the s side's first task 16 + r (hv0 of lane
      // 16 + r), the s side's second task 32 + r (hv1 of lane r)
      const int src_a = (s > 0) == (lane == 0) ? r : 16 + r;
      const dfv ha = {__shfl_sync(0xffffffffu, hv0.h, src_a), __shfl_sync(0xffffffffu, hv0.l, src_a)};
      const dfv hb = {__shfl_sync(0xffffffffu, hv1.h, r), __shfl_sync(0xffffffffu, hv1.l, r)};
      // west halo (lw1, lw2) and east halo (le1, le2) of y_{m+1} on this row
      const dfv lw1 = ha, lw2 = hb, le1 = ha, le2 = hb;
      dfv xms[4], xs[4], x2s[4];
      up3x_xnb<SG>(B1, lw1, lw2, le1, le2, xms, xs, x2s);
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
        df_from_raw4<float2>(slot(t) + kY2Slot + lane * 4, 0, pold);
      }
      dfv yb[4], pb[4];
      if constexpr (SQ) {
        if (t == 6) {
          // the s-pairs of walk row 1 (B0), for walk row 2's carried pairs
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int kx = k + s;
            if (kx >= 0 && kx < 4) qb[k] = df_add_loose(B0[kx], B1[k]);
          }
        }
        dfv ps[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) ps[k] = df_add_loose(xs[k], B2[k]);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const dfv pms = k == KE ? df_add_loose(xms[k], B0[k]) : qb[k - s];
          yb[k] = up3_point_sq(wbh, wbl, B1[k], pms, ps[k], df_add_loose(x2s[k], B3[k]));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) qb[k] = ps[k];
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) yb[k] = up3_point(wbh, wbl, B1[k], xms[k], xs[k], x2s[k], B0[k], B2[k], B3[k]);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        pb[k] = df_axpy2(dm1, B1[k], dm2, yb[k], pold[k]);
        const float p1h = __fmaf_rn(dm1.h, B1[k].h, pold[k].h);  // leading float of p_{m+1}
        fs[0] = __fmaf_rn(B1[k].h, B1[k].h, fs[0]);
        fs[1] = __fmaf_rn(p1h, p1h, fs[1]);
        fs[2] = __fmaf_rn(yb[k].h, yb[k].h, fs[2]);
        fs[3] = __fmaf_rn(pb[k].h, pb[k].h, fs[3]);
      }
      df_store_row<4>(dst + ro, c, nx, yb);
      df_store_row<4>(p + ro, c, nx, pb);
    }
    __syncwarp();
  }
  df_flush4(acc, fs);
  cp_wait<0>();
  __syncwarp();
}

// Launch m (even) of the two-step loop: y_m, p_m -> y_{m+2}, p_{m+2}; the
// launch protocol, buffers, scaling and stopping logic of
// leja_iter_df_pipe2_up3_kernel.  SQ: the paired stencil, for square grids
// with equal x and y coefficients only (the host offers these instances
// only then).
template <int MINB, int STAGES, bool SQ>
__global__ void __launch_bounds__(kPipeThreads, MINB)
    leja_iter_df_pipe2x_up3_kernel(const LoopArgs* __restrict__ Ap, LoopState* __restrict__ st,
                                   double* __restrict__ partials, unsigned int* __restrict__ ticket,
                                   cudaGraphConditionalHandle cond) {
  extern __shared__ __align__(16) unsigned long long up3x_smem[];
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
  unsigned long long* ring = up3x_smem + (size_t)warp * STAGES * kSlotElems2;
  unsigned long long* hbuf = up3x_smem + (size_t)kPipeWarps * STAGES * kSlotElems2 + (size_t)warp * 32 * kHaloU2x;
  for_each_segment(o.nx, o.ny, A.strip_h, blockIdx.x * kPipeWarps + warp, gridDim.x * kPipeWarps,
                   [&](int col0, int r0, int r1) {
    if (m == 0) {
      if (o.s > 0)
        up3x_strip<STAGES, double, true, 1, SQ>(A, A.w, dst, A.pdf, ring, hbuf, col0, r0, r1, wah, wal, wbh, wbl, d0,
                                                dm1, dm2, kexp, acc);
      else
        up3x_strip<STAGES, double, true, -1, SQ>(A, A.w, dst, A.pdf, ring, hbuf, col0, r0, r1, wah, wal, wbh, wbl, d0,
                                                 dm1, dm2, kexp, acc);
    } else {
      if (o.s > 0)
        up3x_strip<STAGES, float2, false, 1, SQ>(A, src, dst, A.pdf, ring, hbuf, col0, r0, r1, wah, wal, wbh, wbl, d0,
                                                 dm1, dm2, kexp, acc);
      else
        up3x_strip<STAGES, float2, false, -1, SQ>(A, src, dst, A.pdf, ring, hbuf, col0, r0, r1, wah, wal, wbh, wbl,
                                                  d0, dm1, dm2, kexp, acc);
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
