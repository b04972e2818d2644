// The float-float batch kernel (a translation unit of its own so that it
// compiles in parallel with the rest): many independent diffusion-advection
// instances of uneven sizes, two Leja iterations per pass, over a flat table
// of (instance, 128-column strip, H-row range) units; the batch's loop
// structure is described in leja_batch.cuh.
#include <cuda_runtime.h>

#include "leja_batch_state.h"
#include "leja_df64_2step_x.cuh"
#include "lexgb_df2x.h"

namespace lexgb {

// Two Leja iterations per pass for the float-float batch (the issue-lean
// two-step strip of the single-problem kernel, df2x_strip: the paired stencil
// with carried pair sums on square instances, the five-point form on the
// others, the column halo 16 rows at a time): launch m (even) takes every active instance
// from y_m, p_m to y_{m+2}, p_{m+2}, and each instance's stopping test runs
// after both iterations (four partial sums per strip).  An instance that
// stops after the first records the fix-up the output pass applies.
template <int MINB, int STAGES>
__global__ void __launch_bounds__(kPipeThreads, MINB)
    leja_batch_df_pipe2x_kernel(BatchInst* __restrict__ inst, const int* __restrict__ strip_inst,
                               BatchState* __restrict__ bs, double* __restrict__ partials,
                               unsigned int* __restrict__ tickets, unsigned int* __restrict__ block_ticket,
                               const double* __restrict__ xi, int H, int total_strips,
                               cudaGraphConditionalHandle cond, int use_cond) {
  extern __shared__ __align__(16) unsigned long long bpipe2x_smem[];
  const int m = __ldcg(&bs->m);
  if (m >= bs->mmax) return;  // host-driven launches past the end of the loop
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double xa = __ldg(xi + m), xb = __ldg(xi + m + 1);
  unsigned long long* ring = bpipe2x_smem + (size_t)warp * STAGES * kSlotElems2;
  unsigned long long* hbuf = bpipe2x_smem + (size_t)kPipeWarps * STAGES * kSlotElems2 + (size_t)warp * 32 * 5;
  for (int s = blockIdx.x * kPipeWarps + warp; s < total_strips; s += gridDim.x * kPipeWarps) {
    const int i = __ldg(strip_inst + s);
    BatchInst* I = inst + i;
    if (__ldcg(&I->done)) continue;
    LoopArgs A;
    A.nx = I->nx;
    A.ny = I->ny;
    const int kexp = __ldcg(&I->kscale), sig = __ldcg(&I->sig), dlt = __ldcg(&I->dlt);
    const int ncs = A.nx / 128;
    const int ls = s - I->first_strip;
    const int col0 = (ls % ncs) * 128;
    const int r0 = (ls / ncs) * H;
    const int r1 = min(r0 + H, A.ny);
    const double dm1d = __ldg(I->d + m + 1);
    const double dm2d = __ldg(I->d + min(m + 2, I->kmax));  // unused when the instance ends at m+1 = kmax
    const double ys = pow2(sig + dlt - kexp);
    const dfv dm1 = df_from_double(dm1d * ys), dm2 = df_from_double(dm2d * ys);
    const dfv d0 = df_from_double(__ldg(I->d));
    const double sw = pow2(-dlt);
    const float swf = (float)sw;
    const dfv wca = df_from_double((I->wc0 - xa) * sw), wcb = df_from_double(I->wc0 - xb);
    const float wah[5] = {I->wf[0] * swf, I->wf[2] * swf, I->wf[4] * swf, I->wf[6] * swf, wca.h};
    const float wal[5] = {I->wf[1] * swf, I->wf[3] * swf, I->wf[5] * swf, I->wf[7] * swf, wca.l};
    const float wbh[5] = {I->wf[0], I->wf[2], I->wf[4], I->wf[6], wcb.h};
    const float wbl[5] = {I->wf[1], I->wf[3], I->wf[5], I->wf[7], wcb.l};
    const int pass = m >> 1;
    float2* dst = (pass & 1) ? I->yf1 : I->yf0;
    dfv acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    const float2* src = (pass & 1) ? I->yf0 : I->yf1;
    const bool sq = A.nx == A.ny;  // the east and north weights coincide, and so do west and south
    if (m == 0) {
      if (sq)
        df2x_strip<STAGES, double, true, true>(A, I->w, dst, I->pf, ring, hbuf, col0, r0, r1, wah, wal, wbh, wbl, d0,
                                               dm1, dm2, kexp, acc);
      else
        df2x_strip<STAGES, double, true, false>(A, I->w, dst, I->pf, ring, hbuf, col0, r0, r1, wah, wal, wbh, wbl, d0,
                                                dm1, dm2, kexp, acc);
    } else {
      if (sq)
        df2x_strip<STAGES, float2, false, true>(A, src, dst, I->pf, ring, hbuf, col0, r0, r1, wah, wal, wbh, wbl, d0,
                                                dm1, dm2, kexp, acc);
      else
        df2x_strip<STAGES, float2, false, false>(A, src, dst, I->pf, ring, hbuf, col0, r0, r1, wah, wal, wbh, wbl, d0,
                                                 dm1, dm2, kexp, acc);
    }
    double v[4] = {df_to_double(acc[0]), df_to_double(acc[1]), df_to_double(acc[2]), df_to_double(acc[3])};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    unsigned last = 0;
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k) partials[4 * (size_t)s + k] = v[k];
      __threadfence();
      last = (atomicAdd(tickets + i, 1u) == (unsigned)I->nstrips - 1u) ? 1u : 0u;
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) continue;
    __threadfence();
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    for (int q = lane; q < I->nstrips; q += 32)
#pragma unroll
      for (int k = 0; k < 4; ++k) t[k] += __ldcg(partials + 4 * (size_t)(I->first_strip + q) + k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < 4; ++k) t[k] += __shfl_xor_sync(0xffffffffu, t[k], o);
    if (lane == 0) {
      const double inv_n = 1.0 / ((double)A.nx * (double)A.ny);
      const double yscale = pow2(sig + dlt), pscale = pow2(kexp);
      int status = 0, it = 0;
      bool done = false;
      // the stopping test of Sec. 2.2 after iteration m+1, then after m+2
      for (int q = 0; q < 2 && !done; ++q) {
        const double dd = q == 0 ? dm1d : dm2d;
        const double ynorm = sqrt(t[2 * q] * inv_n) * yscale, pnorm = sqrt(t[2 * q + 1] * inv_n) * pscale;
        const double e = fabs(dd) * ynorm;
        const int m1 = m + 1 + q;
        I->ynorm = ynorm;
        I->pnorm = pnorm;
        I->err = e;
        if (!isfinite(e) || !isfinite(pnorm)) {
          status = 5;
          done = true;
        } else if (e <= I->rtol * pnorm + I->atol) {
          done = true;
        } else if (m1 >= I->kmax) {
          status = 4;
          done = true;
        }
        it = m1;
        if (done && q == 0) {
          // p holds p_{m+2}: the output pass subtracts d_{m+2} y_{m+2}
          I->fix = 1;
          I->fix_d = dm2d * ys;
          I->fix_buf = pass & 1;
        }
      }
      const double rms = sqrt(t[2] * inv_n);
      int ex = 0;
      if (rms > 0.0 && isfinite(rms)) ex = ilogb(rms);
      I->sig = sig + dlt;
      I->dlt = max(-100, min(100, ex));
      tickets[i] = 0u;
      if (done) {
        I->status = status;
        I->iters = it;
        __threadfence();
        I->done = 1;
        if (atomicSub(&bs->active, 1) == 1 && use_cond) cudaGraphSetConditional(cond, 0);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(block_ticket, 1u) == gridDim.x - 1) {
      *block_ticket = 0u;
      bs->m = m + 2;
      if (m + 2 >= bs->mmax && use_cond) cudaGraphSetConditional(cond, 0);
    }
  }
}

const void* batch_df2x_kernel(int minb, int stages) {
  if (minb == 3 && stages == 5) return reinterpret_cast<const void*>(&leja_batch_df_pipe2x_kernel<3, 5>);
  if (minb == 4 && stages == 4) return reinterpret_cast<const void*>(&leja_batch_df_pipe2x_kernel<4, 4>);
  return nullptr;
}

int batch_df2x_smem_bytes(int stages) { return df2x_smem_bytes(stages); }

}  // namespace lexgb
