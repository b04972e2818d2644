// Instances of the issue-lean two-step float-float kernel for the Burgers
// Jacobian (a translation unit of their own so that they compile in parallel
// with the rest).
#include <cuda_runtime.h>

#include "leja_df64_2step_bx.cuh"
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

const void* df2bx_power_kernel() { return reinterpret_cast<const void*>(&power_pass_df_bx_kernel<5>); }

int df2bx_smem_bytes(int stages) {
  switch (stages) {
    case 4: return pipe2bx_smem_bytes<4>();
    case 5: return pipe2bx_smem_bytes<5>();
    default: return 0;
  }
}

}  // namespace lexgb
