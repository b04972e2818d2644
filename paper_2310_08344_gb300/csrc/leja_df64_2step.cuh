// Two Leja iterations per pass over memory (temporal blocking), float-float
// form, diffusion-advection operator.
//
// Each Newton step of Sec. 2.1 (Eq. 2) only needs the previous basis vector:
//   y_{m+1} = ((A - c)/gamma - xi_m) y_m,     p_{m+1} = p_m + d_{m+1} y_{m+1}.
// One launch of this kernel reads y_m and p_m once and writes y_{m+2} and
// p_{m+2}: every warp recomputes y_{m+1} on its rows plus a one-point halo
// (one extra row above and below its strip, one extra column on each side,
// from a two-point halo of y_m) and never stores it.  The HBM traffic per
// Leja iteration halves (16 instead of 32 bytes per point); the arithmetic
// per iteration grows by the halo recomputation only.
//
// The stopping test of Sec. 2.2 is still evaluated after every iteration: the
// launch accumulates ||y_{m+1}||, ||p_{m+1}||, ||y_{m+2}|| and ||p_{m+2}||,
// and the last block tests m+1 first.  If the loop stops there, p holds
// p_{m+2}; the loop records d_{m+2} and the output pass returns
// p_{m+1} = p_{m+2} - d_{m+2} y_{m+2} (y_{m+2} is in the basis buffer), so
// the result and the iteration count are those of the one-step loop up to
// float-float rounding.
//
// Scaling: the stored basis is renormalised by 2^-dlt once per launch (folded
// into the first step's weights and both Newton coefficients); the second
// step grows the stored values by at most the operator norm (< 8), far
// inside the float range.
#pragma once

#include "leja_df64.cuh"

namespace lexgb {

// Row index r in [-2, ny + 1] wrapped into [0, ny) without an integer
// division (a division per row would run through the conversion unit).
__device__ __forceinline__ int wrap_row(int r, int ny) {
  if (r < 0) r += ny;
  if (r < 0) r += ny;  // ny == 1
  if (r >= ny) r -= ny;
  if (r >= ny) r -= ny;
  return r;
}

// Ring slot: y_m row with two halo points per side, then the p_m row.
constexpr int kY2Slot = kPipeRow + 4;       // [w2 w1][128 points][e1 e2]
constexpr int kSlotElems2 = kY2Slot + kPipeRow;
template <int STAGES>
constexpr int pipe2_smem_bytes() {
  return kPipeWarps * STAGES * kSlotElems2 * 8;
}

// Sum of NV values over the grid in a fixed order (last block, thread 0).
template <int NV>
__device__ __forceinline__ void block_sum_n(double (&v)[NV]) {
  __shared__ double sh[NV][32];
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sh[i][warp] = v[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (int)(blockDim.x >> 5);
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double x = 0.0;
      for (int w = 0; w < nw; ++w) x += sh[i][w];
      v[i] = x;
    }
  }
  __syncthreads();
}

template <int NV>
__device__ __forceinline__ bool last_block_total_n(double (&v)[NV], double* __restrict__ partials,
                                                   unsigned int* __restrict__ ticket) {
  __shared__ int am_last;
  block_sum_n<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) partials[NV * blockIdx.x + i] = v[i];
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double x[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) x[i] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
    for (int i = 0; i < NV; ++i) x[i] += __ldcg(partials + NV * b + i);
  block_sum_n<NV>(x);
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = x[i];
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// One segment (rows r0..r1-1 of one 128-point column strip) of the two-step
// iteration.  S = double on the first launch (the caller's w), else float2.
// wa*: weights of step m (scaled by 2^-dlt), wb*: weights of step m+1.
// acc: float-float sums of y_{m+1}^2, p_{m+1}^2, y_{m+2}^2, p_{m+2}^2.
template <int STAGES, typename S, bool FIRST>
__device__ __forceinline__ void df2_strip(const LoopArgs& A, const S* __restrict__ src, float2* __restrict__ dst,
                                          float2* __restrict__ p, unsigned long long* ring, int col0, int r0, int r1,
                                          const float (&wah)[5], const float (&wal)[5], const float (&wbh)[5],
                                          const float (&wbl)[5], dfv d0, dfv dm1, dfv dm2, int sc, dfv (&acc)[4]) {
  const int lane = threadIdx.x & 31;
  const int nx = A.nx, ny = A.ny;
  const int c = col0 + lane * 4;
  const int cw = col0 == 0 ? nx - 2 : col0 - 2;                // first of the two west halo points
  const int ce = (col0 + kPipeRow >= nx) ? 0 : col0 + kPipeRow;  // first of the two east halo points
  const int nrows = r1 - r0;
  const int last_q = nrows + 3;  // y_m rows q = 0 .. nrows+3 are rows r0-2 .. r1+1
  auto slot = [&](int q) { return ring + (size_t)(q % STAGES) * kSlotElems2; };
  auto issue = [&](int q) {
    if (q <= last_q) {
      const int ry = wrap_row(r0 - 2 + q, ny);
      unsigned long long* s = slot(q);
      const S* row = src + (size_t)ry * nx;
      cp_async16(s + 2 + lane * 4, row + c);
      cp_async16(s + 4 + lane * 4, row + c + 2);
      if (lane == 0) cp_async16(s, row + cw);
      if (lane == 31) cp_async16(s + 2 + kPipeRow, row + ce);
      if constexpr (!FIRST) {
        // slot q also carries p_m of row r0 + q - 4 (the row finished when
        // slot q is the newest y_m row)
        if (q >= 4) {
          const float2* prow = p + (size_t)(r0 + q - 4) * nx;
          cp_async16(s + kY2Slot + lane * 4, prow + c);
          cp_async16(s + kY2Slot + lane * 4 + 2, prow + c + 2);
        }
      }
    }
    cp_commit();
  };
  for (int q = 0; q < STAGES - 1; ++q) issue(q);
  cp_wait<STAGES - 3>();
  __syncwarp();
  dfv ms[4], mc[4], mn[4];  // y_m rows a, a+1, a+2
  dfv bs[4], bc[4];         // y_{m+1} rows a-2, a-1 (as y_m row indices a-1, a)
  dfv hc = {0.f, 0.f};      // y_{m+1} halo point of row a-1 (lane 0: west, lane 31: east)
  df_from_raw4<S>(slot(0) + 2 + lane * 4, sc, ms);
  df_from_raw4<S>(slot(1) + 2 + lane * 4, sc, mc);
#pragma unroll
  for (int k = 0; k < 4; ++k) bs[k] = bc[k] = dfv{0.f, 0.f};
  const int hi = lane == 0 ? 1 : 2 + kPipeRow;  // slot index of this lane's halo point
  for (int a = 0; a <= nrows + 1; ++a) {
    issue(a + STAGES - 1);
    cp_wait<STAGES - 3>();
    __syncwarp();
    const unsigned long long* s0 = slot(a);
    const unsigned long long* s1 = slot(a + 1);
    const unsigned long long* s2 = slot(a + 2);
    df_from_raw4<S>(s2 + 2 + lane * 4, sc, mn);
    // step m: y_{m+1} on y_m row a+1 (grid row r0 - 1 + a)
    dfv xw = shfl_up_df(mc[3]);
    dfv xe = shfl_down_df(mc[0]);
    if (lane == 0) xw = df_from_raw<S>(s1 + 1, sc);
    if (lane == 31) xe = df_from_raw<S>(s1 + 2 + kPipeRow, sc);
    dfv ya[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const dfv t[5] = {k == 3 ? xe : mc[k + 1], k == 0 ? xw : mc[k - 1], mn[k], ms[k], mc[k]};
      ya[k] = df_dot5(wah, wal, t);
    }
    // and its halo point (west for lane 0, east for the others; used by
    // lanes 0 and 31)
    dfv ha;
    {
      const dfv t[5] = {df_from_raw<S>(s1 + hi + 1, sc), df_from_raw<S>(s1 + hi - 1, sc),
                        df_from_raw<S>(s2 + hi, sc), df_from_raw<S>(s0 + hi, sc), df_from_raw<S>(s1 + hi, sc)};
      ha = df_dot5(wah, wal, t);
    }
    if (a >= 2) {
      // step m+1: y_{m+2} on grid row r0 + a - 2 from y_{m+1} rows a-2 .. a
      dfv bw = shfl_up_df(bc[3]);
      dfv be = shfl_down_df(bc[0]);
      if (lane == 0) bw = hc;
      if (lane == 31) be = hc;
      dfv pold[4];
      if constexpr (FIRST) {
#pragma unroll
        for (int k = 0; k < 4; ++k) pold[k] = df_mul(d0, ms[k]);  // p_0 = d_0 y_0 on that row
      } else {
        df_from_raw4<float2>(s2 + kY2Slot + lane * 4, sc, pold);
      }
      dfv yb[4], pb[4];
      float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const dfv p1 = df_axpy(dm1, bc[k], pold[k]);
        const dfv t[5] = {k == 3 ? be : bc[k + 1], k == 0 ? bw : bc[k - 1], ya[k], bs[k], bc[k]};
        yb[k] = df_dot5(wbh, wbl, t);
        pb[k] = df_axpy(dm2, yb[k], p1);
        f0 = __fmaf_rn(bc[k].h, bc[k].h, f0);
        f1 = __fmaf_rn(p1.h, p1.h, f1);
        f2 = __fmaf_rn(yb[k].h, yb[k].h, f2);
        f3 = __fmaf_rn(pb[k].h, pb[k].h, f3);
      }
      df_acc(acc[0], f0);
      df_acc(acc[1], f1);
      df_acc(acc[2], f2);
      df_acc(acc[3], f3);
      const size_t ro = (size_t)(r0 + a - 2) * nx;
      df_store_row<4>(dst + ro, c, nx, yb);
      df_store_row<4>(p + ro, c, nx, pb);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ms[k] = mc[k];
      mc[k] = mn[k];
      bs[k] = bc[k];
      bc[k] = ya[k];
    }
    hc = ha;
    __syncwarp();
  }
  cp_wait<0>();
  __syncwarp();
}

// Launch m (even) of the two-step loop: y_m, p_m -> y_{m+2}, p_{m+2}.
// Basis buffers alternate per launch: launch m/2 writes y0 when m/2 is even.
template <int MINB, int STAGES>
__global__ void __launch_bounds__(kPipeThreads, MINB)
    leja_iter_df_pipe2_kernel(const LoopArgs* __restrict__ Ap, LoopState* __restrict__ st,
                              double* __restrict__ partials, unsigned int* __restrict__ ticket,
                              cudaGraphConditionalHandle cond) {
  extern __shared__ __align__(16) unsigned long long pipe2_smem[];
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
  unsigned long long* ring = pipe2_smem + (size_t)warp * STAGES * kSlotElems2;
  for_each_segment(nx, ny, H, blockIdx.x * kPipeWarps + warp, gridDim.x * kPipeWarps, [&](int col0, int r0, int r1) {
    if (m == 0)
      df2_strip<STAGES, double, true>(A, A.w, dst, A.pdf, ring, col0, r0, r1, wah, wal, wbh, wbl, d0, dm1, dm2, kexp,
                                      acc);
    else
      df2_strip<STAGES, float2, false>(A, src, dst, A.pdf, ring, col0, r0, r1, wah, wal, wbh, wbl, d0, dm1, dm2,
                                       kexp, acc);
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

namespace lexgb {

// ---------------------------------------------------------------------------
// Two Leja iterations per pass for the Burgers Jacobian J(u) (float-float).
// The point weights come from q = u/(2 dx gamma) and r (diagonal part) as in
// the one-step kernel: wE = lx - q, wW = lx + q, wN = ly - q dx/dy,
// wS = ly + q dx/dy, wC = r - xi.  The first step needs q and r on its rows
// and on the one-point column halo, the second on its output row, so each
// ring slot carries the y_m row (two-point halo), the q and r rows (one-point
// halo) and the p_m row.  Per Leja iteration the traffic falls from 48 to
// 24 bytes per point (q and r are read once per two iterations).
// ---------------------------------------------------------------------------
constexpr int kQSlot = kPipeRow + 4;  // [pad][w1][128][e1][pad]
constexpr int kSlotElems2B = kY2Slot + 2 * kQSlot + kPipeRow;
template <int STAGES>
constexpr int pipe2b_smem_bytes() {
  return kPipeWarps * STAGES * kSlotElems2B * 8;
}

// J(u) y at one point from its five neighbours and the point's q and r.
__device__ __forceinline__ dfv burgers_point(dfv ye, dfv yw, dfv yn, dfv ys, dfv yc, dfv q, dfv r, dfv xim, dfv lx,
                                             dfv ly, dfv rat, bool square) {
  const dfv wE = df_add(lx, df_neg(q)), wW = df_add(lx, q);
  const dfv wC = df_add(r, xim);
  if (square) {
    const float wh[3] = {wE.h, wW.h, wC.h};
    const float wl[3] = {wE.l, wW.l, wC.l};
    const dfv t[3] = {df_add(ye, yn), df_add(yw, ys), yc};
    return df_dot3(wh, wl, t);
  }
  const dfv qy = df_mul(q, rat);
  const dfv wN = df_add(ly, df_neg(qy)), wS = df_add(ly, qy);
  const float wh[5] = {wE.h, wW.h, wN.h, wS.h, wC.h};
  const float wl[5] = {wE.l, wW.l, wN.l, wS.l, wC.l};
  const dfv t[5] = {ye, yw, yn, ys, yc};
  return df_dot5(wh, wl, t);
}

template <int STAGES, typename S, bool FIRST>
__device__ __forceinline__ void df2_strip_burgers(const LoopArgs& A, const S* __restrict__ src,
                                                  float2* __restrict__ dst, float2* __restrict__ p,
                                                  unsigned long long* ring, int col0, int r0, int r1, dfv xa, dfv xb,
                                                  float swf, dfv d0, dfv dm1, dfv dm2, int sc, dfv (&acc)[4]) {
  const int lane = threadIdx.x & 31;
  const int nx = A.nx, ny = A.ny;
  const int c = col0 + lane * 4;
  const int cw = col0 == 0 ? nx - 2 : col0 - 2;
  const int ce = (col0 + kPipeRow >= nx) ? 0 : col0 + kPipeRow;
  const int qw = col0 == 0 ? nx - 1 : col0 - 1;  // one-point halo of q, r
  const int nrows = r1 - r0;
  const int last_q = nrows + 3;
  const dfv lx = {A.bl[0], A.bl[1]}, ly = {A.bl[2], A.bl[3]}, rat = {A.bl[4], A.bl[5]};
  const bool square = A.bl[4] == 1.0f && A.bl[5] == 0.0f && A.bl[0] == A.bl[2] && A.bl[1] == A.bl[3];
  auto slot = [&](int q) { return ring + (size_t)(q % STAGES) * kSlotElems2B; };
  auto issue = [&](int q) {
    if (q <= last_q) {
      const int ry = wrap_row(r0 - 2 + q, ny);
      unsigned long long* s = slot(q);
      const S* row = src + (size_t)ry * nx;
      cp_async16(s + 2 + lane * 4, row + c);
      cp_async16(s + 4 + lane * 4, row + c + 2);
      if (lane == 0) cp_async16(s, row + cw);
      if (lane == 31) cp_async16(s + 2 + kPipeRow, row + ce);
      // q and r of this row (with their one-point halo)
      const size_t ro = (size_t)ry * nx;
      unsigned long long* sq = s + kY2Slot;
      unsigned long long* sr = sq + kQSlot;
      cp_async16(sq + 2 + lane * 4, A.bq + ro + c);
      cp_async16(sq + 4 + lane * 4, A.bq + ro + c + 2);
      cp_async16(sr + 2 + lane * 4, A.br + ro + c);
      cp_async16(sr + 4 + lane * 4, A.br + ro + c + 2);
      if (lane == 0) {
        cp_async8(sq + 1, A.bq + ro + qw);
        cp_async8(sr + 1, A.br + ro + qw);
      }
      if (lane == 31) {
        cp_async8(sq + 2 + kPipeRow, A.bq + ro + ce);
        cp_async8(sr + 2 + kPipeRow, A.br + ro + ce);
      }
      if constexpr (!FIRST) {
        if (q >= 4) {
          const float2* prow = p + (size_t)(r0 + q - 4) * nx;
          unsigned long long* sp = sr + kQSlot;
          cp_async16(sp + lane * 4, prow + c);
          cp_async16(sp + lane * 4 + 2, prow + c + 2);
        }
      }
    }
    cp_commit();
  };
  for (int q = 0; q < STAGES - 1; ++q) issue(q);
  cp_wait<STAGES - 3>();
  __syncwarp();
  dfv ms[4], mc[4], mn[4];
  dfv bs[4], bc[4];
  dfv hc = {0.f, 0.f};
  df_from_raw4<S>(slot(0) + 2 + lane * 4, sc, ms);
  df_from_raw4<S>(slot(1) + 2 + lane * 4, sc, mc);
#pragma unroll
  for (int k = 0; k < 4; ++k) bs[k] = bc[k] = dfv{0.f, 0.f};
  const int hi = lane == 0 ? 1 : 2 + kPipeRow;
  for (int a = 0; a <= nrows + 1; ++a) {
    issue(a + STAGES - 1);
    cp_wait<STAGES - 3>();
    __syncwarp();
    const unsigned long long* s0 = slot(a);
    const unsigned long long* s1 = slot(a + 1);
    const unsigned long long* s2 = slot(a + 2);
    df_from_raw4<S>(s2 + 2 + lane * 4, sc, mn);
    // step m on y_m row a+1, with q and r of that row
    dfv q1[4], r1v[4];
    df_from_raw4<float2>(s1 + kY2Slot + 2 + lane * 4, 0, q1);
    df_from_raw4<float2>(s1 + kY2Slot + kQSlot + 2 + lane * 4, 0, r1v);
    dfv xw = shfl_up_df(mc[3]);
    dfv xe = shfl_down_df(mc[0]);
    if (lane == 0) xw = df_from_raw<S>(s1 + 1, sc);
    if (lane == 31) xe = df_from_raw<S>(s1 + 2 + kPipeRow, sc);
    dfv ya[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      dfv v = burgers_point(k == 3 ? xe : mc[k + 1], k == 0 ? xw : mc[k - 1], mn[k], ms[k], mc[k], q1[k], r1v[k], xa,
                            lx, ly, rat, square);
      v.h *= swf;
      v.l *= swf;
      ya[k] = v;
    }
    dfv ha;
    {
      const int qi = lane == 0 ? 1 : 2 + kPipeRow;  // q, r halo entry of this lane
      const dfv qh = df_from_raw<float2>(s1 + kY2Slot + qi, 0);
      const dfv rh = df_from_raw<float2>(s1 + kY2Slot + kQSlot + qi, 0);
      ha = burgers_point(df_from_raw<S>(s1 + hi + 1, sc), df_from_raw<S>(s1 + hi - 1, sc), df_from_raw<S>(s2 + hi, sc),
                         df_from_raw<S>(s0 + hi, sc), df_from_raw<S>(s1 + hi, sc), qh, rh, xa, lx, ly, rat, square);
      ha.h *= swf;
      ha.l *= swf;
    }
    if (a >= 2) {
      // step m+1 on grid row r0 + a - 2 (y_m slot a), q and r of that row
      dfv q0[4], r0v[4];
      df_from_raw4<float2>(s0 + kY2Slot + 2 + lane * 4, 0, q0);
      df_from_raw4<float2>(s0 + kY2Slot + kQSlot + 2 + lane * 4, 0, r0v);
      dfv bw = shfl_up_df(bc[3]);
      dfv be = shfl_down_df(bc[0]);
      if (lane == 0) bw = hc;
      if (lane == 31) be = hc;
      dfv pold[4];
      if constexpr (FIRST) {
#pragma unroll
        for (int k = 0; k < 4; ++k) pold[k] = df_mul(d0, ms[k]);
      } else {
        df_from_raw4<float2>(s2 + kY2Slot + 2 * kQSlot + lane * 4, 0, pold);
      }
      dfv yb[4], pb[4];
      float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const dfv p1 = df_axpy(dm1, bc[k], pold[k]);
        yb[k] = burgers_point(k == 3 ? be : bc[k + 1], k == 0 ? bw : bc[k - 1], ya[k], bs[k], bc[k], q0[k], r0v[k],
                              xb, lx, ly, rat, square);
        pb[k] = df_axpy(dm2, yb[k], p1);
        f0 = __fmaf_rn(bc[k].h, bc[k].h, f0);
        f1 = __fmaf_rn(p1.h, p1.h, f1);
        f2 = __fmaf_rn(yb[k].h, yb[k].h, f2);
        f3 = __fmaf_rn(pb[k].h, pb[k].h, f3);
      }
      df_acc(acc[0], f0);
      df_acc(acc[1], f1);
      df_acc(acc[2], f2);
      df_acc(acc[3], f3);
      const size_t ro = (size_t)(r0 + a - 2) * nx;
      df_store_row<4>(dst + ro, c, nx, yb);
      df_store_row<4>(p + ro, c, nx, pb);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ms[k] = mc[k];
      mc[k] = mn[k];
      bs[k] = bc[k];
      bc[k] = ya[k];
    }
    hc = ha;
    __syncwarp();
  }
  cp_wait<0>();
  __syncwarp();
}

template <int MINB, int STAGES>
__global__ void __launch_bounds__(kPipeThreads, MINB)
    leja_iter_df_pipe2_burgers_kernel(const LoopArgs* __restrict__ Ap, LoopState* __restrict__ st,
                                      double* __restrict__ partials, unsigned int* __restrict__ ticket,
                                      cudaGraphConditionalHandle cond) {
  extern __shared__ __align__(16) unsigned long long pipe2b_smem[];
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
  const int pass = m >> 1;
  float2* dst = reinterpret_cast<float2*>((pass & 1) ? A.y1 : A.y0);
  const float2* src = reinterpret_cast<const float2*>((pass & 1) ? A.y0 : A.y1);
  dfv acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  const int warp = threadIdx.x >> 5;
  unsigned long long* ring = pipe2b_smem + (size_t)warp * STAGES * kSlotElems2B;
  for_each_segment(nx, ny, H, blockIdx.x * kPipeWarps + warp, gridDim.x * kPipeWarps, [&](int col0, int r0, int r1) {
    if (m == 0)
      df2_strip_burgers<STAGES, double, true>(A, A.w, dst, A.pdf, ring, col0, r0, r1, xa, xb, swf, d0, dm1, dm2, kexp,
                                              acc);
    else
      df2_strip_burgers<STAGES, float2, false>(A, src, dst, A.pdf, ring, col0, r0, r1, xa, xb, swf, d0, dm1, dm2,
                                               kexp, acc);
  });
  double v[4] = {df_to_double(acc[0]), df_to_double(acc[1]), df_to_double(acc[2]), df_to_double(acc[3])};
  if (!last_block_total_n<4>(v, partials, ticket)) return;
  if (threadIdx.x == 0) {
    const double yscale = pow2(sig + dlt), pscale = pow2(kexp);
    leja_finalize(A, st, m, dm1d, v[0], v[1], yscale, pscale, cond);
    if (!st->done) {
      leja_finalize(A, st, m + 1, dm2d, v[2], v[3], yscale, pscale, cond);
    } else {
      st->fix = 1;
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
