// Batched Leja interpolation: many independent diffusion-advection instances
// of uneven grid sizes in one launch per Leja iteration.
//
// The strips of all instances (32*VEC columns x H rows each) form one flat
// list; warps take strips with a grid stride, so small and large instances
// share every wave.  Each strip's partial sums go to its own slot; the warp
// that finishes the last strip of an instance (an arrival ticket per
// instance) adds that instance's partials in strip order, runs the stopping
// test of Sec. 2.2 for it and, when it has converged (or failed), marks it
// done: its strips are skipped by every later launch.  The last instance to
// finish ends the CUDA graph's while loop.  All instances advance together,
// so the iteration index m is global; the per-instance iteration counts are
// the m at which each stopped.
#pragma once

#include "leja_df64.cuh"
#include "leja_df64_2step.cuh"
#include "leja_batch_state.h"
#include "leja_kernels.cuh"

namespace lexgb {

template <int VEC>
__global__ void __launch_bounds__(kThreadsPerBlock)
    leja_batch_kernel(BatchInst* __restrict__ inst, const int* __restrict__ strip_inst, BatchState* __restrict__ bs,
                      double* __restrict__ partials, unsigned int* __restrict__ tickets,
                      unsigned int* __restrict__ block_ticket, const double* __restrict__ xi, int H,
                      int total_strips, cudaGraphConditionalHandle cond, int use_cond) {
  const int m = __ldcg(&bs->m);
  if (m >= bs->mmax) return;  // host-driven launches past the end of the loop
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double xim = __ldg(xi + m);
  for (int s = blockIdx.x * kWarpsPerBlock + warp; s < total_strips; s += gridDim.x * kWarpsPerBlock) {
    const int i = __ldg(strip_inst + s);
    BatchInst* I = inst + i;
    if (__ldcg(&I->done)) continue;
    LoopArgs A;
    A.nx = I->nx;
    A.ny = I->ny;
    A.wxp = I->wxp;
    A.wxm = I->wxm;
    A.wyp = I->wyp;
    A.wym = I->wym;
    A.u = nullptr;
    A.s = nullptr;
    const int ncs = (A.nx + 32 * VEC - 1) / (32 * VEC);
    const int ls = s - I->first_strip;
    const int col0 = (ls % ncs) * 32 * VEC;
    const int r0 = (ls / ncs) * H;
    const int r1 = min(r0 + H, A.ny);
    const double* d = I->d;
    const double dm1 = __ldg(d + m + 1);
    const double d0 = __ldg(d);
    const double wcm = I->wc0 - xim;
    double* dst = (m & 1) ? I->y1 : I->y0;
    double sy = 0.0, sp = 0.0;
    if (m == 0) {
      leja_strip<0, double, VEC, double, true>(A, I->w, dst, I->p, col0, r0, r1, wcm, d0, dm1, sy, sp);
    } else {
      const double* src = ((m - 1) & 1) ? I->y1 : I->y0;
      leja_strip<0, double, VEC, double, false>(A, src, dst, I->p, col0, r0, r1, wcm, d0, dm1, sy, sp);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
      sp += __shfl_xor_sync(0xffffffffu, sp, o);
    }
    unsigned last = 0;
    if (lane == 0) {
      partials[2 * (size_t)s] = sy;
      partials[2 * (size_t)s + 1] = sp;
      __threadfence();
      last = (atomicAdd(tickets + i, 1u) == (unsigned)I->nstrips - 1u) ? 1u : 0u;
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) continue;
    // this warp finalises instance i: fixed-order sum of its strip partials
    __threadfence();
    double ty = 0.0, tp = 0.0;
    for (int q = lane; q < I->nstrips; q += 32) {
      ty += __ldcg(partials + 2 * (size_t)(I->first_strip + q));
      tp += __ldcg(partials + 2 * (size_t)(I->first_strip + q) + 1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ty += __shfl_xor_sync(0xffffffffu, ty, o);
      tp += __shfl_xor_sync(0xffffffffu, tp, o);
    }
    if (lane == 0) {
      const double inv_n = 1.0 / ((double)A.nx * (double)A.ny);
      const double ynorm = sqrt(ty * inv_n), pnorm = sqrt(tp * inv_n);
      const double e = fabs(dm1) * ynorm;
      const int m1 = m + 1;
      int status = 0;
      bool done = false;
      if (!isfinite(e) || !isfinite(pnorm)) {
        status = 5;
        done = true;
      } else if (e <= I->rtol * pnorm + I->atol) {
        done = true;
      } else if (m1 >= I->kmax) {
        status = 4;
        done = true;
      }
      I->ynorm = ynorm;
      I->pnorm = pnorm;
      I->err = e;
      tickets[i] = 0u;
      if (done) {
        I->status = status;
        I->iters = m1;
        __threadfence();
        I->done = 1;
        if (atomicSub(&bs->active, 1) == 1 && use_cond) cudaGraphSetConditional(cond, 0);
      }
    }
  }
  // the last block to finish advances the global iteration index
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(block_ticket, 1u) == gridDim.x - 1) {
      *block_ticket = 0u;
      bs->m = m + 1;
      if (m + 1 >= bs->mmax && use_cond) cudaGraphSetConditional(cond, 0);
    }
  }
}

// ---------------------------------------------------------------------------
// Float-float batches (every instance nx % 128 == 0): the same strip list
// with 4 points per lane, the two-step pipelined strip of the one-context
// kernel, and a per-instance storage scaling.
// ---------------------------------------------------------------------------

// Largest biased exponent of |w| per instance (one warp per strip).
static __global__ void __launch_bounds__(kThreadsPerBlock)
    batch_df_scale_kernel(BatchInst* __restrict__ inst, const int* __restrict__ strip_inst, int H,
                          int total_strips) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int s = blockIdx.x * kWarpsPerBlock + warp; s < total_strips; s += gridDim.x * kWarpsPerBlock) {
    const int i = __ldg(strip_inst + s);
    BatchInst* I = inst + i;
    const int nx = I->nx, ny = I->ny;
    const int ncs = nx / 128;
    const int ls = s - I->first_strip;
    const int c = (ls % ncs) * 128 + lane * 4;
    const int r0 = (ls / ncs) * H, r1 = min(r0 + H, ny);
    int e = 0;
    for (int r = r0; r < r1; ++r)
#pragma unroll
      for (int k = 0; k < 4; ++k) e = max(e, (int)((__double2hiint(I->w[(size_t)r * nx + c + k]) >> 20) & 0x7ff));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if (lane == 0) atomicMax(&I->wexp, e);
  }
}

// kscale of every instance from its largest exponent (one thread each).
static __global__ void batch_df_scale_finish_kernel(BatchInst* __restrict__ inst, int B) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B; i += gridDim.x * blockDim.x) {
    BatchInst* I = inst + i;
    const int e = I->wexp;
    const int k = (e == 0) ? 0 : (e == 2047 ? 0 : e - 1023);
    I->kscale = max(-1000, min(1000, k));
    I->sig = I->kscale;
    I->dlt = 0;
  }
}

// p of every instance from float pairs to the caller's doubles (one warp per
// strip).
static __global__ void __launch_bounds__(kThreadsPerBlock)
    batch_df_output_kernel(const BatchInst* __restrict__ inst, const int* __restrict__ strip_inst, int H,
                           int total_strips) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int s = blockIdx.x * kWarpsPerBlock + warp; s < total_strips; s += gridDim.x * kWarpsPerBlock) {
    const int i = __ldg(strip_inst + s);
    const BatchInst* I = inst + i;
    const int nx = I->nx, ny = I->ny, k = I->kscale;
    const int ncs = nx / 128;
    const int ls = s - I->first_strip;
    const int c = (ls % ncs) * 128 + lane * 4;
    const int r0 = (ls / ncs) * H, r1 = min(r0 + H, ny);
    const int fix = I->fix;
    const dfv fd = df_from_double(-I->fix_d);
    const float2* yb = I->fix_buf ? I->yf1 : I->yf0;
    for (int r = r0; r < r1; ++r) {
      const size_t q = (size_t)r * nx + c;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 t = I->pf[q + j];
        dfv a = {t.x, t.y};
        if (fix) {
          const float2 y = yb[q + j];
          a = df_axpy(fd, dfv{y.x, y.y}, a);
        }
        I->p[q + j] = f2d_scaled(a.h, k) + f2d_scaled(a.l, k);
      }
    }
  }
}

// Resets the batch loop state (one thread).
static __global__ void batch_reset_kernel(BatchState* bs, int active, int mmax, unsigned int* block_ticket) {
  bs->m = 0;
  bs->active = active;
  bs->mmax = mmax;
  *block_ticket = 0u;
}

}  // namespace lexgb
