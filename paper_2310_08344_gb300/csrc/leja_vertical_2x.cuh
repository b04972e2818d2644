// Vertical interpolation (Sec. 2.3: NP polynomials on one Newton basis, see
// leja_vertical.cuh) with two Leja iterations per pass over memory, float-
// float form, diffusion-advection operator: the issue-lean strip of
// leja_iter_df_pipe2x_kernel (paired stencil with carried pair sums on
// square grids, the column halo 16 rows at a time) carrying NP polynomials.
//
// One launch reads y_m and the NP polynomials p^(j)_m once and writes
// y_{m+2} and p^(j)_{m+2} = p^(j)_m + d^(j)_{m+1} y_{m+1} + d^(j)_{m+2} y_{m+2}
// (one compensated three-term sum each): 16 + 16 NP bytes per point per two
// iterations instead of per iteration.  The vertical stopping test runs
// after each of the two iterations (every polynomial must pass; the norms of
// p^(j)_{m+1} come from their leading floats); a loop that stops after the
// first leaves each p^(j) one term ahead, and the coefficient of that term,
// d^(j)_{m+2} times the storage scale, is recorded in V.fixd[j] for the
// output pass.
#pragma once

#include "leja_df64_2step_x.cuh"
#include "leja_vertical.cuh"
#include "lexgb_vertical.h"

namespace lexgb {

// Ring slot: y_m row with a two-point halo per side, then the p^(j)_m rows
// of the output row the slot serves.
template <int NP>
__host__ __device__ constexpr int vslot_elems() {
  return kY2Slot + NP * kPipeRow;
}
template <int STAGES, int NP>
constexpr int pipe2x_vert_smem_bytes() {
  return kPipeWarps * STAGES * vslot_elems<NP>() * 8 + kPipeWarps * 32 * 5 * 8;
}

// One segment (rows r0..r1-1 of one 128-point column strip): the walk of
// df2x_strip.  acc: sums of y_{m+1}^2, y_{m+2}^2, then per polynomial
// (p^(j)_{m+1})^2, (p^(j)_{m+2})^2.
template <int STAGES, typename S, bool FIRST, bool SQ, int NP>
__device__ __forceinline__ void df2x_vstrip(const LoopArgs& A, const VertArgs& V, const S* __restrict__ src,
                                            float2* __restrict__ dst, unsigned long long* ring,
                                            unsigned long long* hbuf, int col0, int r0, int r1,
                                            const float (&wah)[5], const float (&wal)[5], const float (&wbh)[5],
                                            const float (&wbl)[5], const dfv (&d0)[NP], const dfv (&dm1)[NP],
                                            const dfv (&dm2)[NP], int sc, dfv (&acc)[2 + 2 * NP]) {
  constexpr int SE = vslot_elems<NP>();
  const int lane = threadIdx.x & 31;
  const int nx = A.nx, ny = A.ny;
  const int c = col0 + lane * 4;
  const int cw = col0 == 0 ? nx - 2 : col0 - 2;                  // first of the two west halo points
  const int ce = (col0 + kPipeRow >= nx) ? 0 : col0 + kPipeRow;  // first of the two east halo points
  const int nrows = r1 - r0;
  const int last_q = nrows + 3;  // y_m rows q = 0 .. nrows+3 are rows r0-2 .. r1+1
  auto slot = [&](int q) { return ring + (size_t)((unsigned)q % STAGES) * SE; };
  auto issue = [&](int q) {
    // halo inputs of the next 16-row chunk, 8 rows before it is needed
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
        // slot q also carries the p^(j)_m rows of row r0 + q - 4
        if (q >= 4) {
          const size_t po = (size_t)(r0 + q - 4) * nx + c;
#pragma unroll
          for (int j = 0; j < NP; ++j) {
            cp_async16(s + kY2Slot + j * kPipeRow + lane * 4, V.pdf[j] + po);
            cp_async16(s + kY2Slot + j * kPipeRow + lane * 4 + 2, V.pdf[j] + po + 2);
          }
        }
      }
    }
    cp_commit();
  };
  df2x_halo_issue<S>(A, src, col0, r0, r1, hbuf);  // chunk 0, in the first commit group
  for (int q = 0; q < STAGES - 1; ++q) issue(q);
  cp_wait<STAGES - 3>();
  __syncwarp();
  dfv M0[4], M1[4], M2[4], B0[4], B1[4], B2[4];
  df_from_raw4<S>(slot(0) + 2 + lane * 4, sc, M0);
  df_from_raw4<S>(slot(1) + 2 + lane * 4, sc, M1);
#pragma unroll
  for (int k = 0; k < 4; ++k) B0[k] = B1[k] = dfv{0.f, 0.f};
  dfv qa[3], qb[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    qa[k] = df_add_loose(M0[k + 1], M1[k]);  // y_m row 0
    qb[k] = dfv{0.f, 0.f};
  }
  dfv hwin = {0.f, 0.f};
  float fs[2 + 2 * NP];
#pragma unroll
  for (int i = 0; i < 2 + 2 * NP; ++i) fs[i] = 0.f;
  auto flush = [&]() {
#pragma unroll
    for (int i = 0; i < 2 + 2 * NP; ++i) {
      df_acc(acc[i], fs[i]);
      fs[i] = 0.f;
    }
  };
  const int sl_base = lane == 0 ? 0 : 16;
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
        ya[k] = df_stencil<false>(wah, wal, k == 3 ? xe : mc[k + 1], k == 0 ? xw : mc[k - 1], mn[k], ms[k], mc[k]);
    }
    dfv senb[3];
    if constexpr (SQ) {
#pragma unroll
      for (int k = 0; k < 3; ++k) senb[k] = df_add_loose(bc[k + 1], ya[k]);
    }
    if (a >= 2) {
      // step m+1: y_{m+2} on output row r0 + t from y_{m+1} rows t-1 .. t+1
      const int t = a - 2;
      if ((t & 15) == 0) {
        flush();
        hwin = df2x_halo_compute<S, SQ>(hbuf, sc, wah, wal);
      }
      const int sl = sl_base + (t & 15);
      const dfv hv = {__shfl_sync(0xffffffffu, hwin.h, sl), __shfl_sync(0xffffffffu, hwin.l, sl)};
      dfv bw = shfl_up_df(bc[3]);
      dfv be = shfl_down_df(bc[0]);
      if (lane == 0) bw = hv;
      if (lane == 31) be = hv;
      dfv yb[4];
      if constexpr (SQ) {
        const dfv senb3 = df_add_loose(be, ya[3]);
        const dfv swsb0 = df_add_loose(bw, bs[0]);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          yb[k] = df_stencil_sq(wbh, wbl, k == 3 ? senb3 : senb[k], k == 0 ? swsb0 : qb[k - 1], bc[k]);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          yb[k] = df_stencil<false>(wbh, wbl, k == 3 ? be : bc[k + 1], k == 0 ? bw : bc[k - 1], ya[k], bs[k], bc[k]);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        fs[0] = __fmaf_rn(bc[k].h, bc[k].h, fs[0]);
        fs[1] = __fmaf_rn(yb[k].h, yb[k].h, fs[1]);
      }
      const size_t ro = (size_t)(r0 + t) * nx;
      df_store_row<4>(dst + ro, c, nx, yb);
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        dfv pold[4], pb[4];
        if constexpr (FIRST) {
#pragma unroll
          for (int k = 0; k < 4; ++k) pold[k] = df_mul(d0[j], ms[k]);  // p^(j)_0 = d^(j)_0 y_0 on that row
        } else {
          df_from_raw4<float2>(s2 + kY2Slot + j * kPipeRow + lane * 4, sc, pold);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          pb[k] = df_axpy2(dm1[j], bc[k], dm2[j], yb[k], pold[k]);
          const float p1h = __fmaf_rn(dm1[j].h, bc[k].h, pold[k].h);  // leading float of p^(j)_{m+1}
          fs[2 + 2 * j] = __fmaf_rn(p1h, p1h, fs[2 + 2 * j]);
          fs[3 + 2 * j] = __fmaf_rn(pb[k].h, pb[k].h, fs[3 + 2 * j]);
        }
        df_store_row<4>(V.pdf[j] + ro, c, nx, pb);
      }
    }
    if constexpr (SQ) {
#pragma unroll
      for (int k = 0; k < 3; ++k) qb[k] = senb[k];
    }
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
  flush();
  cp_wait<0>();
  __syncwarp();
}

// Launch m (even) of the two-step vertical loop; the scaling of the stored
// basis and of the polynomials is that of leja_iter_df_pipe2x_kernel.
template <int MINB, int STAGES, int NP>
__global__ void __launch_bounds__(kPipeThreads, MINB)
    leja_iter_df_vertical2x_kernel(const LoopArgs* __restrict__ Ap, const VertArgs* __restrict__ Vp,
                                   LoopState* __restrict__ st, double* __restrict__ partials,
                                   unsigned int* __restrict__ ticket, cudaGraphConditionalHandle cond) {
  extern __shared__ __align__(16) unsigned long long vert2x_smem[];
  const LoopArgs& A = *Ap;
  const VertArgs& V = *Vp;
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
  const double ys = pow2(sig + dlt - kexp);
  double dm1d[NP], dm2d[NP];
  dfv d0[NP], dm1[NP], dm2[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    dm1d[j] = __ldg(V.d[j] + m + 1);
    dm2d[j] = __ldg(V.d[j] + min(m + 2, A.kmax));  // unused when the loop ends at m+1 = kmax
    dm1[j] = df_from_double(dm1d[j] * ys);
    dm2[j] = df_from_double(dm2d[j] * ys);
    d0[j] = df_from_double(__ldg(V.d[j]));
  }
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
  dfv acc[2 + 2 * NP];
#pragma unroll
  for (int i = 0; i < 2 + 2 * NP; ++i) acc[i] = dfv{0.f, 0.f};
  const int warp = threadIdx.x >> 5;
  constexpr int SE = vslot_elems<NP>();
  unsigned long long* ring = vert2x_smem + (size_t)warp * STAGES * SE;
  unsigned long long* hbuf = vert2x_smem + (size_t)kPipeWarps * STAGES * SE + (size_t)warp * 32 * 5;
  const bool sq = nx == ny;  // the east and north weights coincide, and so do west and south
  for_each_segment(nx, ny, H, blockIdx.x * kPipeWarps + warp, gridDim.x * kPipeWarps, [&](int col0, int r0, int r1) {
    if (m == 0) {
      if (sq)
        df2x_vstrip<STAGES, double, true, true, NP>(A, V, A.w, dst, ring, hbuf, col0, r0, r1, wah, wal, wbh, wbl, d0,
                                                    dm1, dm2, kexp, acc);
      else
        df2x_vstrip<STAGES, double, true, false, NP>(A, V, A.w, dst, ring, hbuf, col0, r0, r1, wah, wal, wbh, wbl, d0,
                                                     dm1, dm2, kexp, acc);
    } else {
      if (sq)
        df2x_vstrip<STAGES, float2, false, true, NP>(A, V, src, dst, ring, hbuf, col0, r0, r1, wah, wal, wbh, wbl, d0,
                                                     dm1, dm2, kexp, acc);
      else
        df2x_vstrip<STAGES, float2, false, false, NP>(A, V, src, dst, ring, hbuf, col0, r0, r1, wah, wal, wbh, wbl,
                                                      d0, dm1, dm2, kexp, acc);
    }
  });
  double v[2 + 2 * NP];
#pragma unroll
  for (int i = 0; i < 2 + 2 * NP; ++i) v[i] = df_to_double(acc[i]);
  if (!last_block_total_n<2 + 2 * NP>(v, partials, ticket)) return;
  if (threadIdx.x == 0) {
    const double yscale = pow2(sig + dlt), pscale = pow2(kexp);
    double sp1[NP], sp2[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      sp1[j] = v[2 + 2 * j];
      sp2[j] = v[3 + 2 * j];
    }
    leja_finalize_vertical<NP>(A, st, m, dm1d, v[0], sp1, yscale, pscale, cond);
    if (!st->done) {
      leja_finalize_vertical<NP>(A, st, m + 1, dm2d, v[1], sp2, yscale, pscale, cond);
    } else {
      // every p^(j) holds p^(j)_{m+2}: the output pass subtracts
      // d^(j)_{m+2} y_{m+2} (coefficient V.fixd[j] per unit of the stored y)
      st->fix = 1;
      st->fix_buf = pass & 1;
#pragma unroll
      for (int j = 0; j < NP; ++j) V.fixd[j] = dm2d[j] * ys;
      st->fix_d = V.fixd[0];
    }
    const double rms = sqrt(v[1] / double(A.n));
    int e = 0;
    if (rms > 0.0 && isfinite(rms)) e = ilogb(rms);
    st->sig = sig + dlt;
    st->dlt = max(-100, min(100, e));
  }
}

// Before the output pass of polynomial j: its odd-stop coefficient (one
// thread; a loop that did not stop after an odd count leaves st->fix = 0).
static __global__ void vertical_select_fix_kernel(LoopState* st, const double* __restrict__ fixd, int j) {
  if (st->fix) st->fix_d = fixd[j];
}

}  // namespace lexgb
