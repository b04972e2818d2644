// Two Leja iterations per pass over memory, float-float form, diffusion-
// advection operator: the issue-lean variant of leja_iter_df_pipe2_kernel.
//
// The arithmetic is that of the two-step kernel (Sec. 2.1, Eq. 2, applied
// twice per launch: y_m -> y_{m+1} -> y_{m+2}, p_m -> p_{m+2}, stopping
// test after each iteration), at the same float-float accuracy, with fewer
// issued instructions per point:
//  * square grids (nx == ny: the east and north weights coincide, and so do
//    west and south) form (y_E + y_N) and (y_W + y_S) with one error-free
//    addition each and take a three-term compensated dot product instead of
//    a five-term one;
//  * the two Newton updates of p are one compensated three-term sum
//    p_m + d_{m+1} y_{m+1} + d_{m+2} y_{m+2} (the norm of p_{m+1} needs only
//    its leading float);
//  * the values of y_{m+1} at the strip's two halo columns, which the
//    second step needs on every output row, are computed for 16 rows at a
//    time, one row and side per lane, from the halo's inputs copied into
//    shared memory with cp.async half a chunk ahead (instead of one
//    full-warp five-point product per row for the two lanes at the edges);
//  * sums of squares accumulate in float per lane over 16 rows, then in
//    float-float;
//  * the stencil's and the Newton update's final renormalisations are
//    Fast2Sum instead of TwoSum (the error bound argued at df_dot3_f2s;
//    139 -> 134 us per launch at 4096^2);
//  * on square grids, three of each lane's four (W,S) pair sums are the
//    (E,N) sums of the row before, one column over (same operands, same
//    values): one error-free addition per point and step instead of two;
//  * the row loop rotates its register windows by copying: unrolling it
//    three times to rotate them by renaming made it instruction-cache bound
//    (170 against 139 us per launch at 4096^2), and moving the chunk work
//    out of the row loop into an outer loop over 16-row chunks cost 5 %.
#pragma once

#include "leja_df64_2step.cuh"

namespace lexgb {

// p + d1 y1 + d2 y2 as one compensated sum (exact products, error-free
// additions of the leading parts, the remaining terms accumulated in float;
// the final renormalisation by Fast2Sum, as in df_dot3_f2s).
__device__ __forceinline__ dfv df_axpy2(dfv d1, dfv y1, dfv d2, dfv y2, dfv p) {
  float q1, e1, q2, e2, s, t1, t2;
  two_prod(d1.h, y1.h, q1, e1);
  e1 = __fmaf_rn(d1.h, y1.l, e1);
  e1 = __fmaf_rn(d1.l, y1.h, e1);
  two_prod(d2.h, y2.h, q2, e2);
  e2 = __fmaf_rn(d2.h, y2.l, e2);
  e2 = __fmaf_rn(d2.l, y2.h, e2);
  two_sum(p.h, q1, s, t1);
  two_sum(s, q2, s, t2);
  const float c = __fadd_rn(__fadd_rn(p.l, e1), __fadd_rn(__fadd_rn(e2, t1), t2));
  dfv r;
  fast_two_sum(s, c, r.h, r.l);
  return r;
}

// One application of the folded stencil w_E y_E + w_W y_W + w_N y_N +
// w_S y_S + w_C y_C (weights in the order E, W, N, S, C).  SQ: w_N = w_E and
// w_S = w_W.
// Square grids: w_E (y_E + y_N) + w_W (y_W + y_S) + w_C y_C from the two
// pair sums sen = y_E + y_N and sws = y_W + y_S.
__device__ __forceinline__ dfv df_stencil_sq(const float (&wh)[5], const float (&wl)[5], dfv sen, dfv sws, dfv c) {
  const float h3[3] = {wh[0], wh[1], wh[4]};
  const float l3[3] = {wl[0], wl[1], wl[4]};
  const dfv t[3] = {sen, sws, c};
  return df_dot3_f2s(h3, l3, t);
}

template <bool SQ>
__device__ __forceinline__ dfv df_stencil(const float (&wh)[5], const float (&wl)[5], dfv e, dfv w, dfv n, dfv s,
                                          dfv c) {
  if constexpr (SQ) {
    return df_stencil_sq(wh, wl, df_add_loose(e, n), df_add_loose(w, s), c);
  } else {
    const dfv t[5] = {e, w, n, s, c};
    return df_dot5(wh, wl, t);
  }
}

// y_{m+1} at the halo columns for 16 output rows r_base .. r_base + 15 of
// the strip at col0: lane j computes row r_base + (j & 15) on the west
// (j < 16, column col0 - 1) or east (column col0 + 128) side.  Rows past the
// segment's last row r1 - 1 repeat that row.  The five stencil inputs of
// each lane are copied into hbuf (5 values per lane) with cp.async ahead of
// use (df2x_halo_issue, in the ring's commit groups) and combined by
// df2x_halo_compute once they have arrived.
template <typename S>
__device__ __forceinline__ void df2x_halo_issue(const LoopArgs& A, const S* __restrict__ src, int col0, int r_base,
                                                int r1, unsigned long long* hbuf) {
  const int lane = threadIdx.x & 31;
  const int nx = A.nx, ny = A.ny;
  const int cx = lane < 16 ? (col0 == 0 ? nx - 1 : col0 - 1) : (col0 + kPipeRow >= nx ? 0 : col0 + kPipeRow);
  const int ce = cx + 1 == nx ? 0 : cx + 1;
  const int cw = cx == 0 ? nx - 1 : cx - 1;
  const int r = min(r_base + (lane & 15), r1 - 1);
  const int rn = wrap_row(r + 1, ny), rs = wrap_row(r - 1, ny);
  const S* row = src + (size_t)r * nx;
  unsigned long long* h = hbuf + lane * 5;
  cp_async8(h + 0, row + ce);
  cp_async8(h + 1, row + cw);
  cp_async8(h + 2, src + (size_t)rn * nx + cx);
  cp_async8(h + 3, src + (size_t)rs * nx + cx);
  cp_async8(h + 4, row + cx);
}

template <typename S, bool SQ>
__device__ __forceinline__ dfv df2x_halo_compute(const unsigned long long* hbuf, int sc, const float (&wh)[5],
                                                 const float (&wl)[5]) {
  const unsigned long long* h = hbuf + (threadIdx.x & 31) * 5;
  return df_stencil<SQ>(wh, wl, df_from_raw<S>(h + 0, sc), df_from_raw<S>(h + 1, sc), df_from_raw<S>(h + 2, sc),
                        df_from_raw<S>(h + 3, sc), df_from_raw<S>(h + 4, sc));
}

__device__ __forceinline__ void df_flush4(dfv (&acc)[4], float (&fs)[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    df_acc(acc[i], fs[i]);
    fs[i] = 0.f;
  }
}

// One segment (rows r0..r1-1 of one 128-point column strip); as df2_strip.
template <int STAGES, typename S, bool FIRST, bool SQ>
__device__ __forceinline__ void df2x_strip(const LoopArgs& A, const S* __restrict__ src, float2* __restrict__ dst,
                                           float2* __restrict__ p, unsigned long long* ring,
                                           unsigned long long* hbuf, int col0, int r0, int r1,
                                           const float (&wah)[5], const float (&wal)[5], const float (&wbh)[5],
                                           const float (&wbl)[5], dfv d0, dfv dm1, dfv dm2, int sc, dfv (&acc)[4]) {
  const int lane = threadIdx.x & 31;
  const int nx = A.nx, ny = A.ny;
  const int c = col0 + lane * 4;
  const int cw = col0 == 0 ? nx - 2 : col0 - 2;                // first of the two west halo points
  const int ce = (col0 + kPipeRow >= nx) ? 0 : col0 + kPipeRow;  // first of the two east halo points
  const int nrows = r1 - r0;
  const int last_q = nrows + 3;  // y_m rows q = 0 .. nrows+3 are rows r0-2 .. r1+1
  auto slot = [&](int q) { return ring + (size_t)((unsigned)q % STAGES) * kSlotElems2; };
  auto issue = [&](int q) {
    // halo inputs of the next 16-row chunk, 8 rows before it is needed
    // (row q is issued at a = q - STAGES + 1, output row t = a - 2)
    const int tq = q - STAGES - 1;
    if ((tq & 15) == 8 && tq + 8 < nrows) df2x_halo_issue<S>(A, src, col0, r0 + tq + 8, r1, hbuf);
    if (q <= last_q) {
      const int ry = wrap_row(r0 - 2 + q, ny);
      unsigned long long* s = slot(q);
      const S* row = src + (size_t)ry * nx;
      cp_async16(s + 2 + lane * 4, row + c);
      cp_async16(s + 4 + lane * 4, row + c + 2);
      if (lane == 0) cp_async16(s, row + cw);
      if (lane == 31) cp_async16(s + 2 + kPipeRow, row + ce);
      if constexpr (!FIRST) {
        // slot q also carries p_m of row r0 + q - 4
        if (q >= 4) {
          const float2* prow = p + (size_t)(r0 + q - 4) * nx;
          cp_async16(s + kY2Slot + lane * 4, prow + c);
          cp_async16(s + kY2Slot + lane * 4 + 2, prow + c + 2);
        }
      }
    }
    cp_commit();
  };
  df2x_halo_issue<S>(A, src, col0, r0, r1, hbuf);  // chunk 0, in the first commit group
  for (int q = 0; q < STAGES - 1; ++q) issue(q);
  cp_wait<STAGES - 3>();
  __syncwarp();
  // rolling windows: y_m rows (ms, mc, mn) and y_{m+1} rows (bs, bc, ya)
  dfv M0[4], M1[4], M2[4], B0[4], B1[4], B2[4];
  df_from_raw4<S>(slot(0) + 2 + lane * 4, sc, M0);
  df_from_raw4<S>(slot(1) + 2 + lane * 4, sc, M1);
#pragma unroll
  for (int k = 0; k < 4; ++k) B0[k] = B1[k] = dfv{0.f, 0.f};
  // square grids: y_W + y_S at (r, i) is the sum y_E + y_N at (r-1, i-1),
  // so each row takes three of its four (W,S) sums from the (E,N) sums of
  // the row before, one column to the left (the same two operands, so the
  // same values); only the lane's first column forms its own.  qa, qb:
  // the (E,N) sums of the previous y_m and y_{m+1} rows at columns c .. c+2.
  dfv qa[3], qb[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    qa[k] = df_add_loose(M0[k + 1], M1[k]);  // y_m row 0
    qb[k] = dfv{0.f, 0.f};
  }
  dfv hwin = {0.f, 0.f};  // this lane's halo value of the current 16-row chunk
  float fs[4] = {0.f, 0.f, 0.f, 0.f};
  const int sl_base = lane == 0 ? 0 : 16;
  // one row of the walk: step m on y_m row a+1, and (a >= 2) step m+1 on
  // output row r0 + a - 2
  auto row = [&](int a, dfv(&ms)[4], dfv(&mc)[4], dfv(&mn)[4], dfv(&bs)[4], dfv(&bc)[4], dfv(&ya)[4]) {
    issue(a + STAGES - 1);
    cp_wait<STAGES - 3>();
    __syncwarp();
    const unsigned long long* s1 = slot(a + 1);
    const unsigned long long* s2 = slot(a + 2);
    df_from_raw4<S>(s2 + 2 + lane * 4, sc, mn);
    // step m: y_{m+1} on y_m row a+1 (grid row r0 - 1 + a)
    dfv xw = shfl_up_df(mc[3]);
    dfv xe = shfl_down_df(mc[0]);
    if (lane == 0) xw = df_from_raw<S>(s1 + 1, sc);
    if (lane == 31) xe = df_from_raw<S>(s1 + 2 + kPipeRow, sc);
    if constexpr (SQ) {
      dfv sen[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) sen[k] = df_add_loose(k == 3 ? xe : mc[k + 1], mn[k]);
      const dfv sws0 = df_add_loose(xw, ms[0]);
#pragma unroll
      for (int k = 0; k < 4; ++k) ya[k] = df_stencil_sq(wah, wal, sen[k], k == 0 ? sws0 : qa[k - 1], mc[k]);
#pragma unroll
      for (int k = 0; k < 3; ++k) qa[k] = sen[k];
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        ya[k] = df_stencil<SQ>(wah, wal, k == 3 ? xe : mc[k + 1], k == 0 ? xw : mc[k - 1], mn[k], ms[k], mc[k]);
    }
    // square grids: the (E,N) sums of y_{m+1} row a at columns c .. c+2
    // (for the next row's step m+1; at a = 0 not yet meaningful)
    dfv senb[3];
    if constexpr (SQ) {
#pragma unroll
      for (int k = 0; k < 3; ++k) senb[k] = df_add_loose(bc[k + 1], ya[k]);
    }
    if (a >= 2) {
      // step m+1: y_{m+2} on output row r0 + t from y_{m+1} rows t-1 .. t+1
      const int t = a - 2;
      if ((t & 15) == 0) {
        // a new chunk of 16 output rows: its halo values of y_{m+1} (the
        // inputs arrived with the ring's copies at least 8 rows earlier)
        df_flush4(acc, fs);
        hwin = df2x_halo_compute<S, SQ>(hbuf, sc, wah, wal);
      }
      const int sl = sl_base + (t & 15);
      const dfv hv = {__shfl_sync(0xffffffffu, hwin.h, sl), __shfl_sync(0xffffffffu, hwin.l, sl)};
      dfv bw = shfl_up_df(bc[3]);
      dfv be = shfl_down_df(bc[0]);
      if (lane == 0) bw = hv;
      if (lane == 31) be = hv;
      dfv pold[4];
      if constexpr (FIRST) {
#pragma unroll
        for (int k = 0; k < 4; ++k) pold[k] = df_mul(d0, ms[k]);  // p_0 = d_0 y_0 on that row
      } else {
        df_from_raw4<float2>(s2 + kY2Slot + lane * 4, sc, pold);
      }
      dfv yb[4], pb[4];
      dfv senb3, swsb0;
      if constexpr (SQ) {
        senb3 = df_add_loose(be, ya[3]);
        swsb0 = df_add_loose(bw, bs[0]);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if constexpr (SQ)
          yb[k] = df_stencil_sq(wbh, wbl, k == 3 ? senb3 : senb[k], k == 0 ? swsb0 : qb[k - 1], bc[k]);
        else
          yb[k] = df_stencil<SQ>(wbh, wbl, k == 3 ? be : bc[k + 1], k == 0 ? bw : bc[k - 1], ya[k], bs[k], bc[k]);
        pb[k] = df_axpy2(dm1, bc[k], dm2, yb[k], pold[k]);
        const float p1h = __fmaf_rn(dm1.h, bc[k].h, pold[k].h);  // leading float of p_{m+1}
        fs[0] = __fmaf_rn(bc[k].h, bc[k].h, fs[0]);
        fs[1] = __fmaf_rn(p1h, p1h, fs[1]);
        fs[2] = __fmaf_rn(yb[k].h, yb[k].h, fs[2]);
        fs[3] = __fmaf_rn(pb[k].h, pb[k].h, fs[3]);
      }
      const size_t ro = (size_t)(r0 + t) * nx;
      df_store_row<4>(dst + ro, c, nx, yb);
      df_store_row<4>(p + ro, c, nx, pb);
    }
    if constexpr (SQ) {
#pragma unroll
      for (int k = 0; k < 3; ++k) qb[k] = senb[k];
    }
    // no barrier here: the next row's copies go to the slot last read two
    // rows ago, before the barrier at the start of this row
  };
  auto rotate = [&]() {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      M0[k] = M1[k];
      M1[k] = M2[k];
      B0[k] = B1[k];
      B1[k] = B2[k];
    }
  };
  const int alast = nrows + 1;
  for (int a = 0; a <= alast; ++a) {
    row(a, M0, M1, M2, B0, B1, B2);
    rotate();
  }
  df_flush4(acc, fs);
  cp_wait<0>();
  __syncwarp();
}

// Launch m (even) of the two-step loop: y_m, p_m -> y_{m+2}, p_{m+2}; the
// same launch protocol, buffers and stopping logic as
// leja_iter_df_pipe2_kernel.  SQ: the paired stencil, for square grids only
// (the host offers these instances only when nx == ny).
template <int MINB, int STAGES, bool SQ>
__global__ void __launch_bounds__(kPipeThreads, MINB)
    leja_iter_df_pipe2x_kernel(const LoopArgs* __restrict__ Ap, LoopState* __restrict__ st,
                               double* __restrict__ partials, unsigned int* __restrict__ ticket,
                               cudaGraphConditionalHandle cond) {
  extern __shared__ __align__(16) unsigned long long pipe2x_smem[];
  const LoopArgs& A = *Ap;
  const int m = __ldcg(&st->m);
  count_launch(st);
  if (__ldcg(&st->done)) return;
  const int kexp = __ldcg(&st->kscale);
  const int sig = __ldcg(&st->sig);
  const int dlt = __ldcg(&st->dlt);
  const int nx = A.nx, ny = A.ny;
  const int H = A.strip_h;
  const double xa = __ldg(A.xi + m);
  const double xb = __ldg(A.xi + m + 1);
  const double dm1d = __ldg(A.d + m + 1);
  const double dm2d = __ldg(A.d + min(m + 2, A.kmax));  // unused when the loop ends at m+1 = kmax
  const double ys = pow2(sig + dlt - kexp);
  const dfv dm1 = df_from_double(dm1d * ys);
  const dfv dm2 = df_from_double(dm2d * ys);
  const dfv d0 = df_from_double(__ldg(A.d));
  const double sw = pow2(-dlt);
  const float swf = (float)sw;
  const dfv wca = df_from_double((A.wc0 - xa) * sw);
  const dfv wcb = df_from_double(A.wc0 - xb);
  const float wah[5] = {A.wf[0] * swf, A.wf[2] * swf, A.wf[4] * swf, A.wf[6] * swf, wca.h};
  const float wal[5] = {A.wf[1] * swf, A.wf[3] * swf, A.wf[5] * swf, A.wf[7] * swf, wca.l};
  const float wbh[5] = {A.wf[0], A.wf[2], A.wf[4], A.wf[6], wcb.h};
  const float wbl[5] = {A.wf[1], A.wf[3], A.wf[5], A.wf[7], wcb.l};
  const int pass = m >> 1;
  float2* dst = reinterpret_cast<float2*>((pass & 1) ? A.y1 : A.y0);
  const float2* src = reinterpret_cast<const float2*>((pass & 1) ? A.y0 : A.y1);
  dfv acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  const int warp = threadIdx.x >> 5;
  unsigned long long* ring = pipe2x_smem + (size_t)warp * STAGES * kSlotElems2;
  unsigned long long* hbuf = pipe2x_smem + (size_t)kPipeWarps * STAGES * kSlotElems2 + (size_t)warp * 32 * 5;
  for_each_segment(nx, ny, H, blockIdx.x * kPipeWarps + warp, gridDim.x * kPipeWarps, [&](int col0, int r0, int r1) {
    if (m == 0)
      df2x_strip<STAGES, double, true, SQ>(A, A.w, dst, A.pdf, ring, hbuf, col0, r0, r1, wah, wal, wbh, wbl, d0, dm1,
                                           dm2, kexp, acc);
    else
      df2x_strip<STAGES, float2, false, SQ>(A, src, dst, A.pdf, ring, hbuf, col0, r0, r1, wah, wal, wbh, wbl, d0, dm1,
                                            dm2, kexp, acc);
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

// Dynamic shared memory of leja_iter_df_pipe2x_kernel: the rings and, per
// warp, 5 halo inputs per lane.
template <int STAGES>
constexpr int pipe2x_smem_bytes() {
  return pipe2_smem_bytes<STAGES>() + kPipeWarps * 32 * 5 * 8;
}

}  // namespace lexgb
