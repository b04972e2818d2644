// Instances of the issue-lean two-step float-float kernel for the Burgers
// Jacobian (a translation unit of their own so that they compile in parallel
// with the rest).
#include <cuda_runtime.h>

#include <algorithm>

#include "leja_df64_2step_bx.cuh"
#include "leja_vertical_2bx.cuh"
#include "lexgb_df2x.h"

namespace lexgb {

template <bool SQ>
const void* pick_bx(int minb, int stages) {
  if (minb == 3 && stages == 4) return reinterpret_cast<const void*>(&leja_iter_df_pipe2bx_kernel<3, 4, SQ>);
  if (minb == 2 && stages == 5) return reinterpret_cast<const void*>(&leja_iter_df_pipe2bx_kernel<2, 5, SQ>);
  return nullptr;
}

const void* df2bx_kernel(int minb, int stages, bool square) {
  return square ? pick_bx<true>(minb, stages) : pick_bx<false>(minb, stages);
}

cudaError_t burgers_weights_df(int nx, int ny, const double* u, double gx, double ig, double wc0, double dx,
                               double dy, float2* q, float2* r, int sm_count, cudaStream_t stream) {
  constexpr int kStages = 5;
  const double cv[5] = {gx, ig, wc0, 1.0 / (2 * dx), 1.0 / (2 * dy)};
  BxWeights W;
  for (int k = 0; k < 5; ++k) {
    W.c[2 * k] = (float)cv[k];
    W.c[2 * k + 1] = (float)(cv[k] - (double)W.c[2 * k]);
  }
  const int smem = kPipeWarps * kStages * kRhsSlot * 8;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, burgers_weights_df_kernel<kStages>,
                                                                kPipeThreads, smem);
  if (e != cudaSuccess) return e;
  const long long lines = (long long)(nx / kPipeRow) * ny;
  const long long want = (lines / 4 + kPipeWarps - 1) / kPipeWarps;
  const int grid = (int)std::max<long long>(1, std::min<long long>(want, (long long)std::max(per_sm, 1) * sm_count));
  burgers_weights_df_kernel<kStages><<<grid, kPipeThreads, smem, stream>>>(nx, ny, u, W, q, r);
  return cudaGetLastError();
}

cudaError_t burgers_field_df(int mode, int nx, int ny, const double* v, const double* src, double h, double nu,
                             double dx, double dy, double* f_out, int sm_count, cudaStream_t stream) {
  constexpr int kStages = 5;
  const double cv[6] = {h * nu / (dx * dx), h * nu / (dy * dy), 1.0 / (2 * dx), 1.0 / (2 * dy), -h, h};
  BxField K;
  for (int k = 0; k < 6; ++k) {
    K.c[2 * k] = (float)cv[k];
    K.c[2 * k + 1] = (float)(cv[k] - (double)K.c[2 * k]);
  }
  const int smem = kPipeWarps * kStages * kRhsSlot * 8;
  const void* fn = mode == 0 ? reinterpret_cast<const void*>(&burgers_field_df_kernel<0, kStages>)
                             : reinterpret_cast<const void*>(&burgers_field_df_kernel<1, kStages>);
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPipeThreads, smem);
  if (e != cudaSuccess) return e;
  const long long lines = (long long)(nx / kPipeRow) * ny;
  const long long want = (lines / 4 + kPipeWarps - 1) / kPipeWarps;
  const int grid = (int)std::max<long long>(1, std::min<long long>(want, (long long)std::max(per_sm, 1) * sm_count));
  if (mode == 0)
    burgers_field_df_kernel<0, kStages><<<grid, kPipeThreads, smem, stream>>>(nx, ny, v, src, K, f_out);
  else
    burgers_field_df_kernel<1, kStages><<<grid, kPipeThreads, smem, stream>>>(nx, ny, v, nullptr, K, f_out);
  return cudaGetLastError();
}

const void* vertical2bx_kernel(int np, int* smem) {
  // y, q, r and NP polynomial rows in the ring: two resident blocks up to
  // three polynomials
  switch (np) {
    case 1: *smem = pipe2bx_vert_smem_bytes<4, 1>(); return reinterpret_cast<const void*>(&leja_iter_df_vertical2bx_kernel<2, 4, 1>);
    case 2: *smem = pipe2bx_vert_smem_bytes<4, 2>(); return reinterpret_cast<const void*>(&leja_iter_df_vertical2bx_kernel<2, 4, 2>);
    case 3: *smem = pipe2bx_vert_smem_bytes<4, 3>(); return reinterpret_cast<const void*>(&leja_iter_df_vertical2bx_kernel<2, 4, 3>);
    default: *smem = 0; return nullptr;
  }
}

const void* df2bx_power_kernel() { return reinterpret_cast<const void*>(&power_pass_df_bx_kernel<5>); }

int df2bx_smem_bytes(int stages) {
  switch (stages) {
    case 4: return pipe2bx_smem_bytes<4>();
    case 5: return pipe2bx_smem_bytes<5>();
    default: return 0;
  }
}

}  // namespace lexgb
