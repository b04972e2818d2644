// Instances of the product-form kernels for the upwind Burgers Jacobian (a
// translation unit of their own so that they compile in parallel with the
// rest).
#include <cuda_runtime.h>

#include "leja_upwind_z.cuh"
#include "lexgb_df2x.h"

namespace lexgb {

const void* up3z_leja_kernel(int minb, int stages) {
  if (minb == 3 && stages == 5) return reinterpret_cast<const void*>(&leja_iter_df_pipe_burgers_up3z_kernel<3, 5>);
  if (minb == 2 && stages == 6) return reinterpret_cast<const void*>(&leja_iter_df_pipe_burgers_up3z_kernel<2, 6>);
  return nullptr;
}

const void* up3z_power_kernel() {
  return reinterpret_cast<const void*>(&power_pass_df_pipe_burgers_up3z_kernel<3, 5>);
}

}  // namespace lexgb
