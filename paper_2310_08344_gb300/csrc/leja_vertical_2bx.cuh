// Vertical interpolation (Sec. 2.3: NP polynomials on one Newton basis) with
// two Leja iterations per pass over memory, float-float form, Jacobian of
// the Burgers right-hand side (central differences): the walk of bx_strip
// (point weights q, r streamed with y; on square grids the paired stencil
// with carried pair sums; the column halo 16 rows at a time) carrying NP
// polynomials, as leja_vertical_2x.cuh does for the constant-coefficient
// operator (the same launch protocol, stopping test and odd-stop records).
#pragma once

#include "leja_df64_2step_bx.cuh"
#include "leja_vertical.cuh"
#include "lexgb_vertical.h"

namespace lexgb {

// Ring slot: y_m row with a two-point halo per side, the NP p^(j)_m rows of
// the output row the slot serves, then the q and r rows of the slot's row.
template <int NP>
__host__ __device__ constexpr int vbx_slot_elems() {
  return kY2Slot + NP * kPipeRow + 2 * kPipeRow;
}
template <int STAGES, int NP>
constexpr int pipe2bx_vert_smem_bytes() {
  return kPipeWarps * STAGES * vbx_slot_elems<NP>() * 8 + kPipeWarps * 32 * kHaloBx * 8;
}

template <int STAGES, typename S, bool FIRST, bool SQ, int NP>
__device__ __forceinline__ void bx_vstrip(const LoopArgs& A, const VertArgs& V, const S* __restrict__ src,
                                          float2* __restrict__ dst, unsigned long long* ring,
                                          unsigned long long* hbuf, int col0, int r0, int r1, dfv lx, dfv ly, dfv rat,
                                          dfv xa, dfv xb, float swf, const dfv (&d0)[NP], const dfv (&dm1)[NP],
                                          const dfv (&dm2)[NP], int sc, dfv (&acc)[2 + 2 * NP]) {
  constexpr int SE = vbx_slot_elems<NP>();
  constexpr int QO = kY2Slot + NP * kPipeRow;  // q row offset in a slot
  constexpr int RO = QO + kPipeRow;            // r row offset
  const int lane = threadIdx.x & 31;
  const int nx = A.nx, ny = A.ny;
  const int c = col0 + lane * 4;
  const int cw = col0 == 0 ? nx - 2 : col0 - 2;
  const int ce = (col0 + kPipeRow >= nx) ? 0 : col0 + kPipeRow;
  const int nrows = r1 - r0;
  const int last_q = nrows + 3;  // y_m rows q = 0 .. nrows+3 are rows r0-2 .. r1+1
  auto slot = [&](int q) { return ring + (size_t)((unsigned)q % STAGES) * SE; };
  auto issue = [&](int q) {
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
      cp_async16(s + QO + lane * 4, A.bq + ro + c);
      cp_async16(s + QO + lane * 4 + 2, A.bq + ro + c + 2);
      cp_async16(s + RO + lane * 4, A.br + ro + c);
      cp_async16(s + RO + lane * 4 + 2, A.br + ro + c + 2);
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
  bx_halo_issue<S>(A, src, col0, r0, r1, hbuf);  // chunk 0, in the first commit group
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
    const unsigned long long* s0 = slot(a);
    const unsigned long long* s1 = slot(a + 1);
    const unsigned long long* s2 = slot(a + 2);
    df_from_raw4<S>(s2 + 2 + lane * 4, sc, mn);
    {
      // step m: y_{m+1} on y_m row a+1, q and r of that row
      dfv qv[4], rv[4];
      df_from_raw4<float2>(s1 + QO + lane * 4, 0, qv);
      df_from_raw4<float2>(s1 + RO + lane * 4, 0, rv);
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
    dfv senb[3];
    if constexpr (SQ) {
#pragma unroll
      for (int k = 0; k < 3; ++k) senb[k] = df_add_loose(bc[k + 1], ya[k]);
    }
    if (a >= 2) {
      // step m+1: y_{m+2} on output row r0 + t, q and r of that row (slot a)
      const int t = a - 2;
      if ((t & 15) == 0) {
        flush();
        const dfv hv0 = bx_halo_compute<S, SQ>(hbuf, sc, lx, ly, rat, xa);
        hwin = {hv0.h * swf, hv0.l * swf};
      }
      const int sl = sl_base + (t & 15);
      const dfv hv = {__shfl_sync(0xffffffffu, hwin.h, sl), __shfl_sync(0xffffffffu, hwin.l, sl)};
      dfv bw = shfl_up_df(bc[3]);
      dfv be = shfl_down_df(bc[0]);
      if (lane == 0) bw = hv;
      if (lane == 31) be = hv;
      dfv q0[4], r0v[4];
      df_from_raw4<float2>(s0 + QO + lane * 4, 0, q0);
      df_from_raw4<float2>(s0 + RO + lane * 4, 0, r0v);
      dfv yb[4];
      if constexpr (SQ) {
        const dfv senb3 = df_add_loose(be, ya[3]);
        const dfv swsb0 = df_add_loose(bw, bs[0]);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          yb[k] = bx_point_sq(lx, q0[k], r0v[k], xb, k == 3 ? senb3 : senb[k], k == 0 ? swsb0 : qb[k - 1], bc[k]);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          yb[k] = bx_point5(lx, ly, rat, q0[k], r0v[k], xb, k == 3 ? be : bc[k + 1], k == 0 ? bw : bc[k - 1], ya[k],
                            bs[k], bc[k]);
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
          const float p1h = __fmaf_rn(dm1[j].h, bc[k].h, pold[k].h);
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

// Launch m (even) of the two-step vertical loop for the Burgers Jacobian;
// the scaling of leja_iter_df_pipe2bx_kernel, the stopping test and odd-stop
// records of leja_iter_df_vertical2x_kernel.
template <int MINB, int STAGES, int NP>
__global__ void __launch_bounds__(kPipeThreads, MINB)
    leja_iter_df_vertical2bx_kernel(const LoopArgs* __restrict__ Ap, const VertArgs* __restrict__ Vp,
                                    LoopState* __restrict__ st, double* __restrict__ partials,
                                    unsigned int* __restrict__ ticket, cudaGraphConditionalHandle cond) {
  extern __shared__ __align__(16) unsigned long long vert2bx_smem[];
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
  const dfv xa = df_from_double(-__ldg(A.xi + m));
  const dfv xb = df_from_double(-__ldg(A.xi + m + 1));
  const float swf = (float)pow2(-dlt);
  const dfv lx = {A.bl[0], A.bl[1]}, ly = {A.bl[2], A.bl[3]}, rat = {A.bl[4], A.bl[5]};
  const int pass = m >> 1;
  float2* dst = reinterpret_cast<float2*>((pass & 1) ? A.y1 : A.y0);
  const float2* src = reinterpret_cast<const float2*>((pass & 1) ? A.y0 : A.y1);
  dfv acc[2 + 2 * NP];
#pragma unroll
  for (int i = 0; i < 2 + 2 * NP; ++i) acc[i] = dfv{0.f, 0.f};
  const int warp = threadIdx.x >> 5;
  constexpr int SE = vbx_slot_elems<NP>();
  unsigned long long* ring = vert2bx_smem + (size_t)warp * STAGES * SE;
  unsigned long long* hbuf = vert2bx_smem + (size_t)kPipeWarps * STAGES * SE + (size_t)warp * 32 * kHaloBx;
  const bool sq = nx == ny;  // square grids: lx = ly and dx = dy
  for_each_segment(nx, ny, H, blockIdx.x * kPipeWarps + warp, gridDim.x * kPipeWarps, [&](int col0, int r0, int r1) {
    if (m == 0) {
      if (sq)
        bx_vstrip<STAGES, double, true, true, NP>(A, V, A.w, dst, ring, hbuf, col0, r0, r1, lx, ly, rat, xa, xb, swf,
                                                  d0, dm1, dm2, kexp, acc);
      else
        bx_vstrip<STAGES, double, true, false, NP>(A, V, A.w, dst, ring, hbuf, col0, r0, r1, lx, ly, rat, xa, xb, swf,
                                                   d0, dm1, dm2, kexp, acc);
    } else {
      if (sq)
        bx_vstrip<STAGES, float2, false, true, NP>(A, V, src, dst, ring, hbuf, col0, r0, r1, lx, ly, rat, xa, xb, swf,
                                                   d0, dm1, dm2, kexp, acc);
      else
        bx_vstrip<STAGES, float2, false, false, NP>(A, V, src, dst, ring, hbuf, col0, r0, r1, lx, ly, rat, xa, xb,
                                                    swf, d0, dm1, dm2, kexp, acc);
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

}  // namespace lexgb
