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

template <bool BURGERS, int NP>
const void* pick_up3(int precision) {
  if (precision == LX_DF64) return reinterpret_cast<const void*>(&leja_iter_df_up3_vertical_kernel<BURGERS, NP>);
  if (precision == LX_MIXED) return reinterpret_cast<const void*>(&leja_iter_up3_vertical_kernel<BURGERS, float, NP>);
  return reinterpret_cast<const void*>(&leja_iter_up3_vertical_kernel<BURGERS, double, NP>);
}

template <bool BURGERS>
const void* pick_up3_np(int precision, int np) {
  switch (np) {
    case 1: return pick_up3<BURGERS, 1>(precision);
    case 2: return pick_up3<BURGERS, 2>(precision);
    case 3: return pick_up3<BURGERS, 3>(precision);
    case 4: return pick_up3<BURGERS, 4>(precision);
    default: return nullptr;
  }
}

}  // namespace

const void* vertical_kernel(int kind, int precision, bool wide, int np) {
  if (kind == LX_ADVDIFF_UP3) return pick_up3_np<false>(precision, np);
  if (kind == LX_BURGERS_UP3) return pick_up3_np<true>(precision, np);
  return kind == LX_BURGERS ? pick_np<1>(precision, wide, np) : pick_np<0>(precision, wide, np);
}


cudaError_t upload_vertical_args(const VertArgs& v, VertArgs* dst, cudaStream_t stream) {
  set_vertical_args_kernel<<<1, 1, 0, stream>>>(v, dst);
  return cudaGetLastError();
}

}  // namespace lexgb
