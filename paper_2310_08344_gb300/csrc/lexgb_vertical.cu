// Kernels of the vertical Leja interpolation (one translation unit of their
// own so that their template instances compile in parallel with the rest).
#include <cuda_runtime.h>

#include "leja_vertical.cuh"
#include "lexgb.h"
#include "lexgb_vertical.h"

namespace lexgb {

namespace {

static __global__ void set_vertical_args_kernel(VertArgs v, VertArgs* dst) { *dst = v; }

template <int KIND, int NP>
const void* pick(int precision, bool wide) {
  if (precision == LX_DF64) return wide ? reinterpret_cast<const void*>(&leja_iter_df_vertical_kernel<KIND, NP>) : nullptr;
  if (precision == LX_MIXED)
    return wide ? reinterpret_cast<const void*>(&leja_iter_vertical_kernel<KIND, float, 2, NP>)
                : reinterpret_cast<const void*>(&leja_iter_vertical_kernel<KIND, float, 1, NP>);
  return wide ? reinterpret_cast<const void*>(&leja_iter_vertical_kernel<KIND, double, 2, NP>)
              : reinterpret_cast<const void*>(&leja_iter_vertical_kernel<KIND, double, 1, NP>);
}

template <int KIND>
const void* pick_np(int precision, bool wide, int np) {
  switch (np) {
    case 1: return pick<KIND, 1>(precision, wide);
    case 2: return pick<KIND, 2>(precision, wide);
    case 3: return pick<KIND, 3>(precision, wide);
    case 4: return pick<KIND, 4>(precision, wide);
    default: return nullptr;
  }
}

}  // namespace

const void* vertical_kernel(int kind, int precision, bool wide, int np) {
  return kind == LX_BURGERS ? pick_np<1>(precision, wide, np) : pick_np<0>(precision, wide, np);
}

cudaError_t upload_vertical_args(const VertArgs& v, VertArgs* dst, cudaStream_t stream) {
  set_vertical_args_kernel<<<1, 1, 0, stream>>>(v, dst);
  return cudaGetLastError();
}

}  // namespace lexgb
