// Kernels of the vertical Leja interpolation (one translation unit of their
// own so that their template instances compile in parallel with the rest).
#include <cuda_runtime.h>

#include "leja_vertical.cuh"
#include "leja_vertical_2x.cuh"
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


const void* vertical2x_kernel(int np, int* smem) {
  // four resident blocks' worth of shared memory is not there for more than
  // two polynomials: 3 blocks per SM up to two, 2 beyond
  switch (np) {
    case 1: *smem = pipe2x_vert_smem_bytes<4, 1>(); return reinterpret_cast<const void*>(&leja_iter_df_vertical2x_kernel<3, 4, 1>);
    case 2: *smem = pipe2x_vert_smem_bytes<4, 2>(); return reinterpret_cast<const void*>(&leja_iter_df_vertical2x_kernel<3, 4, 2>);
    case 3: *smem = pipe2x_vert_smem_bytes<4, 3>(); return reinterpret_cast<const void*>(&leja_iter_df_vertical2x_kernel<2, 4, 3>);
    case 4: *smem = pipe2x_vert_smem_bytes<4, 4>(); return reinterpret_cast<const void*>(&leja_iter_df_vertical2x_kernel<2, 4, 4>);
    default: *smem = 0; return nullptr;
  }
}

cudaError_t select_vertical_fix(void* state, const double* fixd, int j, cudaStream_t stream) {
  vertical_select_fix_kernel<<<1, 1, 0, stream>>>(static_cast<LoopState*>(state), fixd, j);
  return cudaGetLastError();
}

cudaError_t upload_vertical_args(const VertArgs& v, VertArgs* dst, cudaStream_t stream) {
  set_vertical_args_kernel<<<1, 1, 0, stream>>>(v, dst);
  return cudaGetLastError();
}

}  // namespace lexgb
