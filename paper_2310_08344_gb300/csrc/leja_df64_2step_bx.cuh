// Two Leja iterations per pass over memory, float-float form, Jacobian of
// the viscous Burgers right-hand side (central differences): the issue-lean
// variant of leja_iter_df_pipe2_burgers_kernel, built the way
// leja_iter_df_pipe2x_kernel is built for the constant-coefficient operator.
//
// The arithmetic is that of the two-step kernel (Sec. 2.1, Eq. 2, applied
// twice per launch).  J(u) y at a point is w_E y_E + w_W y_W + w_N y_N +
// w_S y_S + w_C y_C with the point weights w_E = lx - q, w_W = lx + q,
// w_N = ly - q dx/dy, w_S = ly + q dx/dy, w_C = r - xi_m, where q = u/(2 dx
// gamma) and r (the centre term with -(u_x + u_y)/gamma) are float pairs per
// point that stream through the ring with y.  Against the first form:
//  * square grids (lx = ly, dx = dy, so w_N = w_E and w_S = w_W) form
//    y_E + y_N with one error-free addition, take y_W + y_S from the
//    previous row's (E,N) sum one column over (the same two operands, so the
//    same value; the pair sums do not depend on the point weights), and
//    evaluate a three-term compensated dot product;
//  * the point weights are unnormalised error-free additions, the final
//    renormalisations Fast2Sum (the bound argued at df_dot3_f2s);
//  * the two Newton updates of p are one compensated three-term sum;
//  * the values of y_{m+1} at the strip's two halo columns are computed for
//    16 rows at a time, one row and side per lane, from their inputs (five
//    values of y_m, q and r) copied into shared memory with cp.async half a
//    chunk ahead, instead of by the whole warp on every row;
//  * sums of squares accumulate in float per lane over 16 rows.
#pragma once

#include "leja_df64_2step_x.cuh"

namespace lexgb {

// Ring slot: y_m row with a two-point halo per side, then the p_m row of the
// output row that the slot serves (see df2x_strip), the q row and the r row.
constexpr int kQBx = kY2Slot + kPipeRow;
constexpr int kRBx = kQBx + kPipeRow;
constexpr int kSlotElemsBx = kRBx + kPipeRow;
constexpr int kHaloBx = 7;  // halo inputs per lane: y_E, y_W, y_N, y_S, y_C, q, r

template <int STAGES>
constexpr int pipe2bx_smem_bytes() {
  return kPipeWarps * STAGES * kSlotElemsBx * 8 + kPipeWarps * 32 * kHaloBx * 8;
}

__device__ __forceinline__ dfv df_negv(dfv a) { return {-a.h, -a.l}; }

// J(u) y at one point of a square grid from the pair sums sen = y_E + y_N
// and sws = y_W + y_S.  xim = -xi_m.
__device__ __forceinline__ dfv bx_point_sq(dfv lx, dfv q, dfv r, dfv xim, dfv sen, dfv sws, dfv c) {
  const dfv wE = df_add_loose(lx, df_negv(q));
  const dfv wW = df_add_loose(lx, q);
  const dfv wC = df_add_loose(r, xim);
  const float wh[3] = {wE.h, wW.h, wC.h};
  const float wl[3] = {wE.l, wW.l, wC.l};
  const dfv t[3] = {sen, sws, c};
  return df_dot3_f2s(wh, wl, t);
}

// J(u) y at one point of any grid (five terms); rat = dx/dy.
__device__ __forceinline__ dfv bx_point5(dfv lx, dfv ly, dfv rat, dfv q, dfv r, dfv xim, dfv e, dfv w, dfv n, dfv s,
                                         dfv c) {
  const dfv qy = df_mul(q, rat);
  const dfv wE = df_add_loose(lx, df_negv(q));
  const dfv wW = df_add_loose(lx, q);
  const dfv wN = df_add_loose(ly, df_negv(qy));
  const dfv wS = df_add_loose(ly, qy);
  const dfv wC = df_add_loose(r, xim);
  const float wh[5] = {wE.h, wW.h, wN.h, wS.h, wC.h};
  const float wl[5] = {wE.l, wW.l, wN.l, wS.l, wC.l};
  const dfv t[5] = {e, w, n, s, c};
  return df_dot5(wh, wl, t);
}

// Inputs of the halo values for output rows r_base .. r_base + 15: lane j
// takes row r_base + (j & 15) (rows past r1 - 1 repeat that row) on the west
// (j < 16, column col0 - 1) or east (column col0 + 128) side: y_m at the
// point and its four neighbours, and q, r at the point.
template <typename S>
__device__ __forceinline__ void bx_halo_issue(const LoopArgs& A, const S* __restrict__ src, int col0, int r_base,
                                              int r1, unsigned long long* hbuf) {
  const int lane = threadIdx.x & 31;
  const int nx = A.nx, ny = A.ny;
  const int cx = lane < 16 ? (col0 == 0 ? nx - 1 : col0 - 1) : (col0 + kPipeRow >= nx ? 0 : col0 + kPipeRow);
  const int ce = cx + 1 == nx ? 0 : cx + 1;
  const int cw = cx == 0 ? nx - 1 : cx - 1;
  const int r = min(r_base + (lane & 15), r1 - 1);
  const int rn = wrap_row(r + 1, ny), rs = wrap_row(r - 1, ny);
  const size_t o = (size_t)r * nx;
  const S* row = src + o;
  unsigned long long* h = hbuf + lane * kHaloBx;
  cp_async8(h + 0, row + ce);
  cp_async8(h + 1, row + cw);
  cp_async8(h + 2, src + (size_t)rn * nx + cx);
  cp_async8(h + 3, src + (size_t)rs * nx + cx);
  cp_async8(h + 4, row + cx);
  cp_async8(h + 5, A.bq + o + cx);
  cp_async8(h + 6, A.br + o + cx);
}

template <typename S, bool SQ>
__device__ __forceinline__ dfv bx_halo_compute(const unsigned long long* hbuf, int sc, dfv lx, dfv ly, dfv rat,
                                               dfv xim) {
  const unsigned long long* h = hbuf + (threadIdx.x & 31) * kHaloBx;
  const dfv e = df_from_raw<S>(h + 0, sc), w = df_from_raw<S>(h + 1, sc), n = df_from_raw<S>(h + 2, sc);
  const dfv s = df_from_raw<S>(h + 3, sc), c = df_from_raw<S>(h + 4, sc);
  const dfv q = df_from_raw<float2>(h + 5, 0), r = df_from_raw<float2>(h + 6, 0);
  if constexpr (SQ)
    return bx_point_sq(lx, q, r, xim, df_add_loose(e, n), df_add_loose(w, s), c);
  else
    return bx_point5(lx, ly, rat, q, r, xim, e, w, n, s, c);
}

// One segment (rows r0..r1-1 of one 128-point column strip); the walk of
// df2x_strip.  xa = -xi_m, xb = -xi_{m+1}; y_{m+1} is scaled by swf.
template <int STAGES, typename S, bool FIRST, bool SQ>
__device__ __forceinline__ void bx_strip(const LoopArgs& A, const S* __restrict__ src, float2* __restrict__ dst,
                                         float2* __restrict__ p, unsigned long long* ring, unsigned long long* hbuf,
                                         int col0, int r0, int r1, dfv lx, dfv ly, dfv rat, dfv xa, dfv xb, float swf,
                                         dfv d0, dfv dm1, dfv dm2, int sc, dfv (&acc)[4]) {
  const int lane = threadIdx.x & 31;
  const int nx = A.nx, ny = A.ny;
  const int c = col0 + lane * 4;
  const int cw = col0 == 0 ? nx - 2 : col0 - 2;                // first of the two west halo points
  const int ce = (col0 + kPipeRow >= nx) ? 0 : col0 + kPipeRow;  // first of the two east halo points
  const int nrows = r1 - r0;
  const int last_q = nrows + 3;  // y_m rows q = 0 .. nrows+3 are rows r0-2 .. r1+1
  auto slot = [&](int q) { return ring + (size_t)((unsigned)q % STAGES) * kSlotElemsBx; };
  auto issue = [&](int q) {
    // halo inputs of the next 16-row chunk, 8 rows before it is needed
    const int tq = q - STAGES - 1;
    if ((tq & 15) == 8 && tq + 8 < nrows) bx_halo_issue<S>(A, src, col0, r0 + tq + 8, r1, hbuf);
    if (q <= last_q) {
      const int ry = wrap_row(r0 - 2 + q, ny);
      unsigned long long* s = slot(q);
      const size_t ro = (size_t)ry * nx;
      const S* row = src + ro;
      cp_async16(s + 2 + lane * 4, row + c);
      cp_async16(s + 4 + lane * 4, row + c + 2);
      if (lane == 0) cp_async16(s, row + cw);
      if (lane == 31) cp_async16(s + 2 + kPipeRow, row + ce);
      cp_async16(s + kQBx + lane * 4, A.bq + ro + c);
      cp_async16(s + kQBx + lane * 4 + 2, A.bq + ro + c + 2);
      cp_async16(s + kRBx + lane * 4, A.br + ro + c);
      cp_async16(s + kRBx + lane * 4 + 2, A.br + ro + c + 2);
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
  bx_halo_issue<S>(A, src, col0, r0, r1, hbuf);  // chunk 0, in the first commit group
  for (int q = 0; q < STAGES - 1; ++q) issue(q);
  cp_wait<STAGES - 3>();
  __syncwarp();
  // rolling windows: y_m rows (ms, mc, mn) and y_{m+1} rows (bs, bc, ya)
  dfv M0[4], M1[4], M2[4], B0[4], B1[4], B2[4];
  df_from_raw4<S>(slot(0) + 2 + lane * 4, sc, M0);
  df_from_raw4<S>(slot(1) + 2 + lane * 4, sc, M1);
#pragma unroll
  for (int k = 0; k < 4; ++k) B0[k] = B1[k] = dfv{0.f, 0.f};
  // square grids: the (E,N) pair sums of the previous y_m and y_{m+1} rows
  // at columns c .. c+2 (the next row's (W,S) sums one column over)
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
    const unsigned long long* s0 = slot(a);
    const unsigned long long* s1 = slot(a + 1);
    const unsigned long long* s2 = slot(a + 2);
    df_from_raw4<S>(s2 + 2 + lane * 4, sc, mn);
    // step m: y_{m+1} on y_m row a+1 (grid row r0 - 1 + a), q and r of that row
    {
      dfv qv[4], rv[4];
      df_from_raw4<float2>(s1 + kQBx + lane * 4, 0, qv);
      df_from_raw4<float2>(s1 + kRBx + lane * 4, 0, rv);
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
        for (int k = 0; k < 4; ++k) {
          const dfv v = bx_point_sq(lx, qv[k], rv[k], xa, sen[k], k == 0 ? sws0 : qa[k - 1], mc[k]);
          ya[k] = {v.h * swf, v.l * swf};
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) qa[k] = sen[k];
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const dfv v = bx_point5(lx, ly, rat, qv[k], rv[k], xa, k == 3 ? xe : mc[k + 1], k == 0 ? xw : mc[k - 1],
                                  mn[k], ms[k], mc[k]);
          ya[k] = {v.h * swf, v.l * swf};
        }
      }
    }
    // square grids: the (E,N) sums of y_{m+1} row a at columns c .. c+2
    // (for the next row's step m+1; at a = 0 not yet meaningful)
    dfv senb[3];
    if constexpr (SQ) {
#pragma unroll
      for (int k = 0; k < 3; ++k) senb[k] = df_add_loose(bc[k + 1], ya[k]);
    }
    if (a >= 2) {
      // step m+1: y_{m+2} on output row r0 + t from y_{m+1} rows t-1 .. t+1,
      // q and r of that row (y_m slot a)
      const int t = a - 2;
      if ((t & 15) == 0) {
        // a new chunk of 16 output rows: its halo values of y_{m+1} (the
        // inputs arrived with the ring's copies at least 8 rows earlier)
        df_flush4(acc, fs);
        const dfv hv0 = bx_halo_compute<S, SQ>(hbuf, sc, lx, ly, rat, xa);
        hwin = {hv0.h * swf, hv0.l * swf};
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
      dfv q0[4], r0v[4];
      df_from_raw4<float2>(s0 + kQBx + lane * 4, 0, q0);
      df_from_raw4<float2>(s0 + kRBx + lane * 4, 0, r0v);
      dfv senb3, swsb0;
      if constexpr (SQ) {
        senb3 = df_add_loose(be, ya[3]);
        swsb0 = df_add_loose(bw, bs[0]);
      }
      dfv yb[4], pb[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if constexpr (SQ)
          yb[k] = bx_point_sq(lx, q0[k], r0v[k], xb, k == 3 ? senb3 : senb[k], k == 0 ? swsb0 : qb[k - 1], bc[k]);
        else
          yb[k] = bx_point5(lx, ly, rat, q0[k], r0v[k], xb, k == 3 ? be : bc[k + 1], k == 0 ? bw : bc[k - 1], ya[k],
                            bs[k], bc[k]);
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
    // rows ago (slot a - 1), before the barrier at the start of this row
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

// One power-iteration pass (Sec. 2, Listing 7) on the Burgers Jacobian of a
// square grid: the row-strip walk and ring of pow_strip (leja_df64.cuh; v
// with a one-point halo, q = u/(2 dx) and r = the centre term per row), with
// the lean point form of bx_strip -- the (E,N) pair sum by one error-free
// addition, the (W,S) pair carried from the previous row one column over,
// the weights lx -+ q by unnormalised additions, a three-term Dot2 -- then
// w = J(u) v / ||v|| and ||w||^2 to double accuracy as in pow_strip.
template <int STAGES, typename S>
__device__ __forceinline__ void pow_bx_strip(int nx, int ny, const S* __restrict__ v, float2* __restrict__ w,
                                             const float2* __restrict__ q, const float2* __restrict__ r, dfv lx,
                                             unsigned long long* ring, int col0, int r0, int r1, dfv sg, dfv& acc,
                                             float& small) {
  const int lane = threadIdx.x & 31;
  const int c = col0 + lane * 4;
  const int cw = col0 == 0 ? nx - 1 : col0 - 1;
  const int ce = (col0 + kPipeRow >= nx) ? 0 : col0 + kPipeRow;
  const int last_q = r1 - r0 + 1;  // rows q = 0 .. last_q are grid rows r0 - 1 .. r1
  constexpr int kSlot = pow_slot_elems<1>();
  auto slot = [&](int qq) { return ring + (size_t)((unsigned)qq % STAGES) * kSlot; };
  auto issue = [&](int qq) {
    if (qq <= last_q) {
      const int ry = wrap_row(r0 - 1 + qq, ny);
      const S* row = v + (size_t)ry * nx;
      unsigned long long* sl = slot(qq);
      cp_async16(sl + 2 + lane * 4, row + c);
      cp_async16(sl + 4 + lane * 4, row + c + 2);
      if (lane == 0) cp_async8(sl + 1, row + cw);
      if (lane == 31) cp_async8(sl + 2 + kPipeRow, row + ce);
      const size_t o = (size_t)ry * nx + c;
      cp_async16(sl + kRhsSlot + lane * 4, q + o);
      cp_async16(sl + kRhsSlot + lane * 4 + 2, q + o + 2);
      cp_async16(sl + kRhsSlot + kPipeRow + lane * 4, r + o);
      cp_async16(sl + kRhsSlot + kPipeRow + lane * 4 + 2, r + o + 2);
    }
    cp_commit();
  };
  for (int qq = 0; qq < STAGES - 1; ++qq) issue(qq);
  cp_wait<STAGES - 3>();
  __syncwarp();
  dfv ys[4], yc[4], yn[4], qa[3];
  df_from_raw4<S>(slot(0) + 2 + lane * 4, 0, ys);
  df_from_raw4<S>(slot(1) + 2 + lane * 4, 0, yc);
#pragma unroll
  for (int k = 0; k < 3; ++k) qa[k] = df_add_loose(ys[k + 1], yc[k]);  // row r0 - 1
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
    dfv qv[4], rv[4], sen[4];
    df_from_raw4<float2>(scn + kRhsSlot + lane * 4, 0, qv);
    df_from_raw4<float2>(scn + kRhsSlot + kPipeRow + lane * 4, 0, rv);
#pragma unroll
    for (int k = 0; k < 4; ++k) sen[k] = df_add_loose(k == 3 ? xe : yc[k + 1], yn[k]);
    const dfv sws0 = df_add_loose(xw, ys[0]);
    dfv out[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const dfv wE = df_add_loose(lx, df_negv(qv[k]));
      const dfv wW = df_add_loose(lx, qv[k]);
      const float wh[3] = {wE.h, wW.h, rv[k].h};
      const float wl[3] = {wE.l, wW.l, rv[k].l};
      const dfv t[3] = {sen[k], k == 0 ? sws0 : qa[k - 1], yc[k]};
      out[k] = df_mul(sg, df_dot3_f2s(wh, wl, t));
      float sq, se;
      two_prod(out[k].h, out[k].h, sq, se);
      df_acc(acc, sq);
      small = __fmaf_rn(2.f * out[k].h, out[k].l, __fadd_rn(small, se));
    }
    df_store_row<4>(w + (size_t)(r0 - 1 + qc) * nx, c, nx, out);
#pragma unroll
    for (int k = 0; k < 3; ++k) qa[k] = sen[k];
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

// power_pass_df_rows_kernel<1, STAGES> (the same arguments, shared memory
// and stopping test) with pow_bx_strip: square grids only (lx = ly, dx = dy).
template <int STAGES>
__global__ void __launch_bounds__(kPipeThreads)
    power_pass_df_bx_kernel(int nx, int ny, long long n, const void* __restrict__ vin, int vin_double,
                            float2* __restrict__ w, const float2* __restrict__ q, const float2* __restrict__ r,
                            PowWeights W, double* __restrict__ partials, unsigned int* __restrict__ ticket,
                            LoopState* st) {
  extern __shared__ __align__(16) unsigned long long powbx_ring[];
  if (__ldcg(&st->pdone)) return;
  const dfv sg = df_from_double(__ldcg(&st->sigma));
  const dfv lx = {W.bl[0], W.bl[1]};
  dfv acc = {0.f, 0.f};
  float small = 0.f;
  const int warp = threadIdx.x >> 5;
  unsigned long long* ring = powbx_ring + (size_t)warp * STAGES * pow_slot_elems<1>();
  for_each_segment(nx, ny, 0, blockIdx.x * kPipeWarps + warp, gridDim.x * kPipeWarps, [&](int col0, int r0, int r1) {
    if (vin_double)
      pow_bx_strip<STAGES, double>(nx, ny, reinterpret_cast<const double*>(vin), w, q, r, lx, ring, col0, r0, r1, sg,
                                   acc, small);
    else
      pow_bx_strip<STAGES, float2>(nx, ny, reinterpret_cast<const float2*>(vin), w, q, r, lx, ring, col0, r0, r1, sg,
                                   acc, small);
  });
  double s = df_to_double(acc) + (double)small, dummy = 0.0;
  if (!last_block_total2(s, dummy, partials, ticket)) return;
  if (threadIdx.x == 0) power_pass_finish(st, s, n);
}

// The point weights of J(u) as float pairs, from u alone: q = u gx and
// r = wc0 - (u_x + u_y) ig with u_x + u_y = (u_E - u_W) / (2 dx) +
// (u_N - u_S) / (2 dy) (central differences, as the FP64 right-hand side
// forms it) -- the float-float counterpart of the FP64 gradient followed by
// burgers_df_prep_kernel.  Row strips with balanced row ranges, u rows (one-
// point halo) through a per-warp cp.async ring, each value split once
// (nx % 128 == 0, u 16-byte aligned).  cst: gx, ig, wc0, 1/(2 dx), 1/(2 dy)
// as float pairs.
struct BxWeights {
  float c[10];
};

template <int STAGES>
__global__ void __launch_bounds__(kPipeThreads)
    burgers_weights_df_kernel(int nx, int ny, const double* __restrict__ u, BxWeights W, float2* __restrict__ q,
                              float2* __restrict__ r) {
  extern __shared__ __align__(16) unsigned long long bw_ring[];
  const dfv gx = {W.c[0], W.c[1]}, ig = {W.c[2], W.c[3]}, wc0 = {W.c[4], W.c[5]};
  const dfv i2dx = {W.c[6], W.c[7]}, i2dy = {W.c[8], W.c[9]};
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  unsigned long long* ring = bw_ring + (size_t)warp * STAGES * kRhsSlot;
  for_each_segment(nx, ny, 0, blockIdx.x * kPipeWarps + warp, gridDim.x * kPipeWarps, [&](int col0, int r0, int r1) {
    const int c = col0 + lane * 4;
    const int cw = col0 == 0 ? nx - 1 : col0 - 1;
    const int ce = (col0 + kPipeRow >= nx) ? 0 : col0 + kPipeRow;
    const int last_q = r1 - r0 + 1;  // rows q = 0 .. last_q are grid rows r0 - 1 .. r1
    auto slot = [&](int qq) { return ring + (size_t)((unsigned)qq % STAGES) * kRhsSlot; };
    auto issue = [&](int qq) {
      if (qq <= last_q) {
        const int ry = wrap_row(r0 - 1 + qq, ny);
        const double* row = u + (size_t)ry * nx;
        unsigned long long* sl = slot(qq);
        cp_async16(sl + 2 + lane * 4, row + c);
        cp_async16(sl + 4 + lane * 4, row + c + 2);
        if (lane == 0) cp_async8(sl + 1, row + cw);
        if (lane == 31) cp_async8(sl + 2 + kPipeRow, row + ce);
      }
      cp_commit();
    };
    for (int qq = 0; qq < STAGES - 1; ++qq) issue(qq);
    cp_wait<STAGES - 3>();
    __syncwarp();
    dfv ys[4], yc[4], yn[4];
    df_from_raw4<double>(slot(0) + 2 + lane * 4, 0, ys);
    df_from_raw4<double>(slot(1) + 2 + lane * 4, 0, yc);
    for (int qc = 1; qc < last_q; ++qc) {
      issue(qc + STAGES - 2);
      cp_wait<STAGES - 3>();
      __syncwarp();
      const unsigned long long* sn = slot(qc + 1);
      const unsigned long long* scn = slot(qc);
      df_from_raw4<double>(sn + 2 + lane * 4, 0, yn);
      dfv xw = shfl_up_df(yc[3]);
      dfv xe = shfl_down_df(yc[0]);
      if (lane == 0) xw = df_from_raw<double>(scn + 1, 0);
      if (lane == 31) xe = df_from_raw<double>(scn + 2 + kPipeRow, 0);
      float2 qo[4], ro[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const dfv ddx = df_add_loose(k == 3 ? xe : yc[k + 1], df_negv(k == 0 ? xw : yc[k - 1]));
        const dfv ddy = df_add_loose(yn[k], df_negv(ys[k]));
        const dfv grad = df_add_loose(df_mul(ddx, i2dx), df_mul(ddy, i2dy));
        const dfv qk = df_mul(yc[k], gx);
        const dfv rk = df_axpy(df_negv(ig), grad, wc0);  // wc0 - ig grad
        qo[k] = make_float2(qk.h, qk.l);
        ro[k] = make_float2(rk.h, rk.l);
      }
      const size_t ro_off = (size_t)(r0 - 1 + qc) * nx + c;
      *reinterpret_cast<float4*>(q + ro_off) = make_float4(qo[0].x, qo[0].y, qo[1].x, qo[1].y);
      *reinterpret_cast<float4*>(q + ro_off + 2) = make_float4(qo[2].x, qo[2].y, qo[3].x, qo[3].y);
      *reinterpret_cast<float4*>(r + ro_off) = make_float4(ro[0].x, ro[0].y, ro[1].x, ro[1].y);
      *reinterpret_cast<float4*>(r + ro_off + 2) = make_float4(ro[2].x, ro[2].y, ro[3].x, ro[3].y);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        ys[k] = yc[k];
        yc[k] = yn[k];
      }
      __syncwarp();
    }
    cp_wait<0>();
    __syncwarp();
  });
}

// Fields of an EXPRB32 step of the Burgers problem (central differences)
// in float-float on the FP32 pipe, written as doubles -- the counterparts
// of the FP64 rhs_kernel<1> and exprb32_stage_kernel<1>:
//   MODE 0: f_out = h (nu lap v - v (v_x + v_y)) [+ h src]   (h F(u), v = u)
//   MODE 1: f_out = -h v (v_x + v_y)   (the stage remainder h (F(a) - F(u))
//           of the quadratic term with v = p1 = a - u)
// lap and v_x + v_y by central differences.  Row strips with balanced row
// ranges, v rows (one-point halo) through a per-warp cp.async ring, each
// value split once (nx % 128 == 0, v and f_out 16-byte aligned).  cst as
// float pairs: h nu / dx^2, h nu / dy^2, 1/(2 dx), 1/(2 dy), -h, h.
struct BxField {
  float c[12];
};

template <int MODE, int STAGES>
__global__ void __launch_bounds__(kPipeThreads)
    burgers_field_df_kernel(int nx, int ny, const double* __restrict__ v, const double* __restrict__ src, BxField K,
                            double* __restrict__ f_out) {
  extern __shared__ __align__(16) unsigned long long bf_ring[];
  const dfv ax = {K.c[0], K.c[1]}, ay = {K.c[2], K.c[3]}, i2dx = {K.c[4], K.c[5]}, i2dy = {K.c[6], K.c[7]};
  const dfv mh = {K.c[8], K.c[9]}, hp = {K.c[10], K.c[11]};
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  unsigned long long* ring = bf_ring + (size_t)warp * STAGES * kRhsSlot;
  for_each_segment(nx, ny, 0, blockIdx.x * kPipeWarps + warp, gridDim.x * kPipeWarps, [&](int col0, int r0, int r1) {
    const int c = col0 + lane * 4;
    const int cw = col0 == 0 ? nx - 1 : col0 - 1;
    const int ce = (col0 + kPipeRow >= nx) ? 0 : col0 + kPipeRow;
    const int last_q = r1 - r0 + 1;  // rows q = 0 .. last_q are grid rows r0 - 1 .. r1
    auto slot = [&](int qq) { return ring + (size_t)((unsigned)qq % STAGES) * kRhsSlot; };
    auto issue = [&](int qq) {
      if (qq <= last_q) {
        const int ry = wrap_row(r0 - 1 + qq, ny);
        const double* row = v + (size_t)ry * nx;
        unsigned long long* sl = slot(qq);
        cp_async16(sl + 2 + lane * 4, row + c);
        cp_async16(sl + 4 + lane * 4, row + c + 2);
        if (lane == 0) cp_async8(sl + 1, row + cw);
        if (lane == 31) cp_async8(sl + 2 + kPipeRow, row + ce);
      }
      cp_commit();
    };
    for (int qq = 0; qq < STAGES - 1; ++qq) issue(qq);
    cp_wait<STAGES - 3>();
    __syncwarp();
    dfv ys[4], yc[4], yn[4];
    df_from_raw4<double>(slot(0) + 2 + lane * 4, 0, ys);
    df_from_raw4<double>(slot(1) + 2 + lane * 4, 0, yc);
    for (int qc = 1; qc < last_q; ++qc) {
      issue(qc + STAGES - 2);
      cp_wait<STAGES - 3>();
      __syncwarp();
      const unsigned long long* sn = slot(qc + 1);
      const unsigned long long* scn = slot(qc);
      df_from_raw4<double>(sn + 2 + lane * 4, 0, yn);
      dfv xw = shfl_up_df(yc[3]);
      dfv xe = shfl_down_df(yc[0]);
      if (lane == 0) xw = df_from_raw<double>(scn + 1, 0);
      if (lane == 31) xe = df_from_raw<double>(scn + 2 + kPipeRow, 0);
      const size_t o = (size_t)(r0 - 1 + qc) * nx + c;
      double res[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const dfv e = k == 3 ? xe : yc[k + 1], w = k == 0 ? xw : yc[k - 1];
        const dfv grad = df_add_loose(df_mul(df_add_loose(e, df_negv(w)), i2dx),
                                      df_mul(df_add_loose(yn[k], df_negv(ys[k])), i2dy));
        dfv f = df_mul(mh, df_mul(yc[k], grad));  // -h v (v_x + v_y)
        if constexpr (MODE == 0) {
          const dfv c2 = {2.f * yc[k].h, 2.f * yc[k].l};
          const dfv lxx = df_add_loose(df_add_loose(e, w), df_negv(c2));
          const dfv lyy = df_add_loose(df_add_loose(yn[k], ys[k]), df_negv(c2));
          f = df_add_loose(f, df_add_loose(df_mul(ax, lxx), df_mul(ay, lyy)));
          if (src) f = df_add_loose(f, df_mul(hp, df_split_scaled(__ldg(src + o + k), 0)));
        }
        res[k] = f2d_scaled(f.h, 0) + f2d_scaled(f.l, 0);  // both exact; one rounding to double
      }
      *reinterpret_cast<double2*>(f_out + o) = make_double2(res[0], res[1]);
      *reinterpret_cast<double2*>(f_out + o + 2) = make_double2(res[2], res[3]);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        ys[k] = yc[k];
        yc[k] = yn[k];
      }
      __syncwarp();
    }
    cp_wait<0>();
    __syncwarp();
  });
}

// Launch m (even) of the two-step loop for the Burgers Jacobian: y_m, p_m ->
// y_{m+2}, p_{m+2}; the launch protocol, buffers, scaling and stopping logic
// of leja_iter_df_pipe2_burgers_kernel.  SQ: the paired stencil, for square
// grids only (the host offers these instances only when nx == ny).
template <int MINB, int STAGES, bool SQ>
__global__ void __launch_bounds__(kPipeThreads, MINB)
    leja_iter_df_pipe2bx_kernel(const LoopArgs* __restrict__ Ap, LoopState* __restrict__ st,
                                double* __restrict__ partials, unsigned int* __restrict__ ticket,
                                cudaGraphConditionalHandle cond) {
  extern __shared__ __align__(16) unsigned long long pipe2bx_smem[];
  const LoopArgs& A = *Ap;
  const int m = __ldcg(&st->m);
  count_launch(st);
  if (__ldcg(&st->done)) return;
  const int kexp = __ldcg(&st->kscale);
  const int sig = __ldcg(&st->sig);
  const int dlt = __ldcg(&st->dlt);
  const int nx = A.nx, ny = A.ny;
  const int H = A.strip_h;
  const double dm1d = __ldg(A.d + m + 1);
  const double dm2d = __ldg(A.d + min(m + 2, A.kmax));  // unused when the loop ends at m+1 = kmax
  const double ys = pow2(sig + dlt - kexp);
  const dfv dm1 = df_from_double(dm1d * ys);
  const dfv dm2 = df_from_double(dm2d * ys);
  const dfv d0 = df_from_double(__ldg(A.d));
  const dfv xa = df_from_double(-__ldg(A.xi + m));
  const dfv xb = df_from_double(-__ldg(A.xi + m + 1));
  const float swf = (float)pow2(-dlt);
  const dfv lx = {A.bl[0], A.bl[1]}, ly = {A.bl[2], A.bl[3]}, rat = {A.bl[4], A.bl[5]};
  const int pass = m >> 1;
  float2* dst = reinterpret_cast<float2*>((pass & 1) ? A.y1 : A.y0);
  const float2* src = reinterpret_cast<const float2*>((pass & 1) ? A.y0 : A.y1);
  dfv acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  const int warp = threadIdx.x >> 5;
  unsigned long long* ring = pipe2bx_smem + (size_t)warp * STAGES * kSlotElemsBx;
  unsigned long long* hbuf =
      pipe2bx_smem + (size_t)kPipeWarps * STAGES * kSlotElemsBx + (size_t)warp * 32 * kHaloBx;
  for_each_segment(nx, ny, H, blockIdx.x * kPipeWarps + warp, gridDim.x * kPipeWarps, [&](int col0, int r0, int r1) {
    if (m == 0)
      bx_strip<STAGES, double, true, SQ>(A, A.w, dst, A.pdf, ring, hbuf, col0, r0, r1, lx, ly, rat, xa, xb, swf, d0,
                                         dm1, dm2, kexp, acc);
    else
      bx_strip<STAGES, float2, false, SQ>(A, src, dst, A.pdf, ring, hbuf, col0, r0, r1, lx, ly, rat, xa, xb, swf, d0,
                                          dm1, dm2, kexp, acc);
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
