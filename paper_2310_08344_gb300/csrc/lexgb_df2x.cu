// Instances of the issue-lean two-step float-float kernel (a translation unit
// of their own so that they compile in parallel with the rest).
#include <cuda_runtime.h>

#include "leja_df64_2step_x.cuh"
#include "lexgb_df2x.h"

namespace lexgb {

template <bool SQ>
const void* pick(int minb, int stages) {
  if (minb == 4 && stages == 4) return reinterpret_cast<const void*>(&leja_iter_df_pipe2x_kernel<4, 4, SQ>);
  if (minb == 4 && stages == 5) return reinterpret_cast<const void*>(&leja_iter_df_pipe2x_kernel<4, 5, SQ>);
  if (minb == 3 && stages == 5) return reinterpret_cast<const void*>(&leja_iter_df_pipe2x_kernel<3, 5, SQ>);
  // five blocks per SM: 96 registers (a few bytes of spills)
  if (minb == 5 && stages == 4) return reinterpret_cast<const void*>(&leja_iter_df_pipe2x_kernel<5, 4, SQ>);
  return nullptr;
}

const void* df2x_kernel(int minb, int stages, bool square) {
  return square ? pick<true>(minb, stages) : pick<false>(minb, stages);
}

int df2x_smem_bytes(int stages) {
  switch (stages) {
    case 4: return pipe2x_smem_bytes<4>();
    case 5: return pipe2x_smem_bytes<5>();
    default: return 0;
  }
}

}  // namespace lexgb
