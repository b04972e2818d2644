// Instances of the issue-lean two-step float-float kernel for the paper's
// upwind diffusion-advection operator (a translation unit of their own so
// that they compile in parallel with the rest).
#include <cuda_runtime.h>

#include "leja_upwind_2step_x.cuh"
#include "lexgb_df2x.h"

namespace lexgb {

template <bool SQ>
const void* pick_up3x(int minb, int stages) {
  if (minb == 3 && stages == 6) return reinterpret_cast<const void*>(&leja_iter_df_pipe2x_up3_kernel<3, 6, SQ>);
  if (minb == 3 && stages == 5) return reinterpret_cast<const void*>(&leja_iter_df_pipe2x_up3_kernel<3, 5, SQ>);
  return nullptr;
}

const void* up3x_kernel(int minb, int stages, bool square) {
  return square ? pick_up3x<true>(minb, stages) : pick_up3x<false>(minb, stages);
}

int up3x_smem_bytes(int stages) {
  switch (stages) {
    case 5: return pipe2x_up3_smem_bytes<5>();
    case 6: return pipe2x_up3_smem_bytes<6>();
    default: return 0;
  }
}

}  // namespace lexgb
