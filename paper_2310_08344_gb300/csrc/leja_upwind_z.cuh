// The product form of the upwind Burgers Jacobian in the pipelined float-
// float iteration and power pass (Problem III of Sec. 3); its own header and
// translation unit (lexgb_up3z.cu) so that it compiles in parallel with the
// rest.
#pragma once

#include "leja_upwind.cuh"

namespace lexgb {

// ---------------------------------------------------------------------------
// Pipelined float-float iteration for the upwind Burgers Jacobian, product
// form.  J(u) v = nu lap v + a (D_x + D_y)(u v) is linear in z = u v, so
// with q = u |a| / (6 dx gamma) (float pairs) and z = q y, one Newton step is
//   y' = lxs (yE + yW) + lys (yN + yS) + cc0 yC
//        + sum_o k_o z_{X(o s)} + rat sum_o k_o z_{Y(o s)}        (o = -1, 0, 1, 2)
// with constant weights: z is formed once per point as its row enters the
// register window (one float-float product), instead of seven point weights
// per point.  The y window holds rows r-1 .. r+2, the z window rows r-2 .. r+2;
// the ring keeps the y and q rows with their two-point halos (the centre
// row's halo gives yW, yE and the z halo points of lanes 0 and 31) and the p
// row of the output row.  STAGES ring slots: the previous centre row's, the
// centre row's through the newest row's (three), and STAGES - 4 rows in
// flight.
// ---------------------------------------------------------------------------

// Weights (as float pairs) of the twelve terms
// [yE, yW, yN, yS, yC, zX(-s), zX(s), zX(2s), zY(-s), zY(s), zY(2s), zC].
// POWER: one power-iteration pass instead of a Leja step -- w = J(u) v * sg
// (sg = 1 / ||v|| as a float pair), no polynomial, and sum w^2 accumulated
// to double accuracy (accy from the exact squares of the leading floats,
// small from their error terms and the cross terms).
// SQ (square grids with equal x and y coefficients: lxs = lys, rat = 1): the
// four y neighbours share one weight and z at the offsets o along x and y
// share k_o, so the twelve terms become six -- the four-point sum
// y_E + y_N + y_W + y_S, y_C, the pair sums z_X(o) + z_Y(o) for o = -s, s, 2s,
// and z_C.  The pairs (y_W + y_S) and (z_X(-1) + z_Y(-1)) at (r, i) are the
// pairs (y_E + y_N) and (z_X(1) + z_Y(1)) at (r - 1, i - 1) (the same two
// operands, so the same values): carried from the previous row.
template <typename S, bool FIRST, int SG, int STAGES, bool POWER = false, bool SQ = false>
__device__ __forceinline__ void df_strip_burgers_up3z(const LoopArgs& A, const S* __restrict__ src,
                                                      float2* __restrict__ dst, float2* __restrict__ p,
                                                      unsigned long long* ring, int col0, int r0, int r1,
                                                      const float (&wh)[12], const float (&wl)[12], float swf,
                                                      dfv d0, dfv dm1, int sc, dfv& accy, dfv& accp,
                                                      dfv sg = dfv{0.f, 0.f}, float* small = nullptr) {
  static_assert(STAGES >= 5, "the centre row through the newest row need three slots, plus rows in flight");
  constexpr int s = SG;
  const int lane = threadIdx.x & 31;
  const int nx = A.nx, ny = A.ny;
  const int c = col0 + lane * 4;
  const int cw = col0 == 0 ? nx - 2 : col0 - 2;
  const int ce = (col0 + kPipeRow >= nx) ? 0 : col0 + kPipeRow;
  const int nrows = r1 - r0;
  const int last_q = nrows + 3;  // rows q = 0 .. nrows+3 are r0-2 .. r1+1
  auto slot = [&](int q) { return ring + (size_t)(q % STAGES) * kSlotElemsUB; };
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
      if constexpr (!FIRST && !POWER) {
        if (q >= 4) {  // p of output row r0 + q - 4 arrives with the newest row
          const float2* prow = p + (size_t)(r0 + q - 4) * nx;
          unsigned long long* sp = sl + 2 * kY2Slot;
          cp_async16(sp + lane * 4, prow + c);
          cp_async16(sp + lane * 4 + 2, prow + c + 2);
        }
      }
    }
    cp_commit();
  };
  // z = q y at this lane's four points of the row in slot sl
  auto zrow = [&](const unsigned long long* sl, const dfv (&y)[4], dfv (&z)[4]) {
    dfv g[4];
    df_from_raw4<float2>(sl + kY2Slot + 2 + lane * 4, 0, g);
#pragma unroll
    for (int k = 0; k < 4; ++k) z[k] = df_mul(g[k], y[k]);
  };
  dfv y1[4], y2[4], y3[4], y4[4];          // y rows r-1 .. r+2
  dfv z0[4], z1[4], z2[4], z3[4], z4[4];   // z rows r-2 .. r+2
  for (int q = 0; q < STAGES; ++q) issue(q);
  cp_wait<STAGES - 4>();  // rows 0..3 complete
  __syncwarp();
  {
    dfv y0[4];
    df_from_raw4<S>(slot(0) + 2 + lane * 4, sc, y0);
    zrow(slot(0), y0, z0);
  }
  df_from_raw4<S>(slot(1) + 2 + lane * 4, sc, y1);
  df_from_raw4<S>(slot(2) + 2 + lane * 4, sc, y2);
  df_from_raw4<S>(slot(3) + 2 + lane * 4, sc, y3);
  zrow(slot(1), y1, z1);
  zrow(slot(2), y2, z2);
  zrow(slot(3), y3, z3);
  // halo indices of this lane in a slot: lane 0 takes the west points
  // (c-1, c-2), the others the east points (c+4, c+5 for lane 31)
  const int h1 = lane == 0 ? 1 : 2 + kPipeRow;
  const int h2 = lane == 0 ? 0 : 3 + kPipeRow;
  // square grids: weights of the six terms, and the (E,N) pair sums of y and
  // z on the row before the centre row at columns c .. c+2
  const float w6h[6] = {wh[0], wh[4], wh[5], wh[6], wh[7], wh[11]};
  const float w6l[6] = {wl[0], wl[4], wl[5], wl[6], wl[7], wl[11]};
  dfv cs[3], cz[3];
  if constexpr (SQ) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cs[k] = df_add_loose(y1[k + 1], y2[k]);
      cz[k] = df_add_loose(z1[k + 1], z2[k]);
    }
  }
  __syncwarp();  // every lane has read row 0 before its slot is refilled
  for (int a = 0; a < nrows; ++a) {
    issue(a + STAGES);      // into the slot of row a (its z is in registers)
    cp_wait<STAGES - 4>();  // rows up to a+4 complete
    __syncwarp();
    const unsigned long long* sn = slot(a + 4);
    const unsigned long long* sc2 = slot(a + 2);  // centre row
    df_from_raw4<S>(sn + 2 + lane * 4, sc, y4);
    zrow(sn, y4, z4);
    dfv pold[4];
    if constexpr (!FIRST && !POWER) df_from_raw4<float2>(sn + 2 * kY2Slot + lane * 4, 0, pold);
    // centre-row neighbours (shuffles outside any divergent branch)
    const dfv yu3 = shfl_up_df(y2[3]), yd0 = shfl_down_df(y2[0]);
    const dfv zu3 = shfl_up_df(z2[3]), zu2 = shfl_up_df(z2[2]);
    const dfv zd0 = shfl_down_df(z2[0]), zd1 = shfl_down_df(z2[1]);
    const dfv hy1 = df_from_raw<S>(sc2 + h1, sc), hy2 = df_from_raw<S>(sc2 + h2, sc);
    const dfv hz1 = df_mul(df_from_raw<float2>(sc2 + kY2Slot + h1, 0), hy1);
    const dfv hz2 = df_mul(df_from_raw<float2>(sc2 + kY2Slot + h2, 0), hy2);
    const dfv ym1 = lane == 0 ? hy1 : yu3, yp1 = lane == 31 ? hy1 : yd0;
    const dfv zm1 = lane == 0 ? hz1 : zu3, zm2 = lane == 0 ? hz2 : zu2;
    const dfv zp1 = lane == 31 ? hz1 : zd0, zp2 = lane == 31 ? hz2 : zd1;
    const dfv yxm1[4] = {ym1, y2[0], y2[1], y2[2]}, yxp1[4] = {y2[1], y2[2], y2[3], yp1};
    const dfv zxm1[4] = {zm1, z2[0], z2[1], z2[2]}, zxm2[4] = {zm2, zm1, z2[0], z2[1]};
    const dfv zxp1[4] = {z2[1], z2[2], z2[3], zp1}, zxp2[4] = {z2[2], z2[3], zp1, zp2};
    dfv y4s[4], zpp[4], zpm[4], z2s[4];  // square grids: the pair sums of this row
    if constexpr (SQ) {
      dfv sen[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        sen[k] = df_add_loose(yxp1[k], y3[k]);
        zpp[k] = df_add_loose(zxp1[k], z3[k]);
        z2s[k] = s > 0 ? df_add_loose(zxp2[k], z4[k]) : df_add_loose(zxm2[k], z0[k]);
      }
      const dfv sws0 = df_add_loose(yxm1[0], y1[0]);
      zpm[0] = df_add_loose(zxm1[0], z1[0]);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        y4s[k] = df_add_loose(sen[k], k == 0 ? sws0 : cs[k - 1]);
        if (k > 0) zpm[k] = cz[k - 1];
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        cs[k] = sen[k];
        cz[k] = zpp[k];
      }
    }
    dfv ynew[4], pnew[4];
    float fy = 0.f, fp = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      dfv v;
      if constexpr (SQ) {
        const dfv t6[6] = {y4s[k], y2[k], s > 0 ? zpm[k] : zpp[k], s > 0 ? zpp[k] : zpm[k], z2s[k], z2[k]};
        v = df_dot_n<6>(w6h, w6l, t6);
      } else {
        const dfv t[12] = {yxp1[k],
                           yxm1[k],
                           y3[k],
                           y1[k],
                           y2[k],
                           s > 0 ? zxm1[k] : zxp1[k],
                           s > 0 ? zxp1[k] : zxm1[k],
                           s > 0 ? zxp2[k] : zxm2[k],
                           s > 0 ? z1[k] : z3[k],
                           s > 0 ? z3[k] : z1[k],
                           s > 0 ? z4[k] : z0[k],
                           z2[k]};
        v = df_dot_n<12>(wh, wl, t);
      }
      if constexpr (POWER) {
        v = df_mul(sg, v);
        ynew[k] = v;
        float sq, se;
        two_prod(v.h, v.h, sq, se);
        df_acc(accy, sq);
        *small = __fmaf_rn(2.f * v.h, v.l, __fadd_rn(*small, se));
      } else {
        v.h *= swf;
        v.l *= swf;
        ynew[k] = v;
        const dfv po = FIRST ? df_mul(d0, y2[k]) : pold[k];
        pnew[k] = df_axpy(dm1, v, po);
        fy = __fmaf_rn(v.h, v.h, fy);
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
      y1[k] = y2[k];
      y2[k] = y3[k];
      y3[k] = y4[k];
      z0[k] = z1[k];
      z1[k] = z2[k];
      z2[k] = z3[k];
      z3[k] = z4[k];
    }
    __syncwarp();
  }
  cp_wait<0>();
  __syncwarp();
}

template <int MINB, int STAGES>
__global__ void __launch_bounds__(kPipeThreads, MINB)
    leja_iter_df_pipe_burgers_up3z_kernel(const LoopArgs* __restrict__ Ap, LoopState* __restrict__ st,
                                          double* __restrict__ partials, unsigned int* __restrict__ ticket,
                                          cudaGraphConditionalHandle cond) {
  extern __shared__ __align__(16) unsigned long long up3z_smem[];
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
  const double rat = o.gy / o.gx;
  const double wd[12] = {o.cxx * ig,
                         o.cxx * ig,
                         o.cyy * ig,
                         o.cyy * ig,
                         (-2.0 * o.cxx - 2.0 * o.cyy - A.up_c) * ig - xim,
                         kUp3Km,
                         kUp3K1,
                         kUp3K2,
                         kUp3Km * rat,
                         kUp3K1 * rat,
                         kUp3K2 * rat,
                         kUp3K0 * (1.0 + rat)};
  float wh[12], wl[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const dfv t = df_from_double(wd[k]);
    wh[k] = t.h;
    wl[k] = t.l;
  }
  float2* dst = reinterpret_cast<float2*>((m & 1) ? A.y1 : A.y0);
  const float2* src = reinterpret_cast<const float2*>(((m - 1) & 1) ? A.y1 : A.y0);
  dfv accy = {0.f, 0.f}, accp = {0.f, 0.f};
  const int warp = threadIdx.x >> 5;
  unsigned long long* ring = up3z_smem + (size_t)warp * STAGES * kSlotElemsUB;
  const bool sq = o.cxx == o.cyy && o.gx == o.gy;  // the six-term form (not on the first launch)
  for_each_segment(o.nx, o.ny, A.strip_h, blockIdx.x * kPipeWarps + warp, gridDim.x * kPipeWarps,
                   [&](int col0, int r0, int r1) {
    if (m == 0) {
      if (o.s > 0)
        df_strip_burgers_up3z<double, true, 1, STAGES>(A, A.w, dst, A.pdf, ring, col0, r0, r1, wh, wl, swf, d0, dm1,
                                                       kexp, accy, accp);
      else
        df_strip_burgers_up3z<double, true, -1, STAGES>(A, A.w, dst, A.pdf, ring, col0, r0, r1, wh, wl, swf, d0, dm1,
                                                        kexp, accy, accp);
    } else {
      if (sq) {
        if (o.s > 0)
          df_strip_burgers_up3z<float2, false, 1, STAGES, false, true>(A, src, dst, A.pdf, ring, col0, r0, r1, wh, wl,
                                                                       swf, d0, dm1, kexp, accy, accp);
        else
          df_strip_burgers_up3z<float2, false, -1, STAGES, false, true>(A, src, dst, A.pdf, ring, col0, r0, r1, wh, wl,
                                                                        swf, d0, dm1, kexp, accy, accp);
      } else {
        if (o.s > 0)
          df_strip_burgers_up3z<float2, false, 1, STAGES>(A, src, dst, A.pdf, ring, col0, r0, r1, wh, wl, swf, d0, dm1,
                                                          kexp, accy, accp);
        else
          df_strip_burgers_up3z<float2, false, -1, STAGES>(A, src, dst, A.pdf, ring, col0, r0, r1, wh, wl, swf, d0,
                                                           dm1, kexp, accy, accp);
      }
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

// One power-iteration pass (Sec. 2, Listing 7) on the upwind Burgers
// Jacobian in the pipelined product form: w = J(u) v / ||v||, rho_k = ||w||,
// the stop test of power_pass_finish.  q = u |a| / (6 dx) (gamma = 1); v is
// the caller's doubles on the first pass (vin_double), float pairs after.
// Needs nx % 128 == 0 and 16-byte aligned vectors; strip height 0
// (balanced row ranges).
template <int MINB, int STAGES>
__global__ void __launch_bounds__(kPipeThreads, MINB)
    power_pass_df_pipe_burgers_up3z_kernel(Up3Op o, const void* __restrict__ vin, int vin_double,
                                           float2* __restrict__ w, const float2* __restrict__ q,
                                           double* __restrict__ partials, unsigned int* __restrict__ ticket,
                                           LoopState* st) {
  extern __shared__ __align__(16) unsigned long long up3zp_smem[];
  if (__ldcg(&st->pdone)) return;
  const dfv sg = df_from_double(__ldcg(&st->sigma));
  const double rat = o.gy / o.gx;
  const double wd[12] = {o.cxx,  o.cxx,  o.cyy,        o.cyy,        -2.0 * o.cxx - 2.0 * o.cyy, kUp3Km,
                         kUp3K1, kUp3K2, kUp3Km * rat, kUp3K1 * rat, kUp3K2 * rat,               kUp3K0 * (1.0 + rat)};
  float wh[12], wl[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const dfv t = df_from_double(wd[k]);
    wh[k] = t.h;
    wl[k] = t.l;
  }
  LoopArgs A;
  A.nx = o.nx;
  A.ny = o.ny;
  A.bq = q;
  dfv acc = {0.f, 0.f}, unused = {0.f, 0.f};
  float small = 0.f;
  const dfv zero = {0.f, 0.f};
  const int warp = threadIdx.x >> 5;
  unsigned long long* ring = up3zp_smem + (size_t)warp * STAGES * kSlotElemsUB;
  const double* vd = reinterpret_cast<const double*>(vin);
  const float2* vf = reinterpret_cast<const float2*>(vin);
  const bool sq = o.cxx == o.cyy && o.gx == o.gy;  // the six-term form (not on the first pass)
  for_each_segment(o.nx, o.ny, 0, blockIdx.x * kPipeWarps + warp, gridDim.x * kPipeWarps,
                   [&](int col0, int r0, int r1) {
    if (vin_double) {
      if (o.s > 0)
        df_strip_burgers_up3z<double, true, 1, STAGES, true>(A, vd, w, nullptr, ring, col0, r0, r1, wh, wl, 1.f, zero,
                                                             zero, 0, acc, unused, sg, &small);
      else
        df_strip_burgers_up3z<double, true, -1, STAGES, true>(A, vd, w, nullptr, ring, col0, r0, r1, wh, wl, 1.f,
                                                              zero, zero, 0, acc, unused, sg, &small);
    } else {
      if (sq) {
        if (o.s > 0)
          df_strip_burgers_up3z<float2, false, 1, STAGES, true, true>(A, vf, w, nullptr, ring, col0, r0, r1, wh, wl,
                                                                      1.f, zero, zero, 0, acc, unused, sg, &small);
        else
          df_strip_burgers_up3z<float2, false, -1, STAGES, true, true>(A, vf, w, nullptr, ring, col0, r0, r1, wh, wl,
                                                                       1.f, zero, zero, 0, acc, unused, sg, &small);
      } else {
        if (o.s > 0)
          df_strip_burgers_up3z<float2, false, 1, STAGES, true>(A, vf, w, nullptr, ring, col0, r0, r1, wh, wl, 1.f,
                                                                zero, zero, 0, acc, unused, sg, &small);
        else
          df_strip_burgers_up3z<float2, false, -1, STAGES, true>(A, vf, w, nullptr, ring, col0, r0, r1, wh, wl, 1.f,
                                                                 zero, zero, 0, acc, unused, sg, &small);
      }
    }
  });
  double s = df_to_double(acc) + (double)small, dummy = 0.0;
  if (!last_block_total2(s, dummy, partials, ticket)) return;
  if (threadIdx.x == 0) power_pass_finish(st, s, o.n);
}

}  // namespace lexgb
