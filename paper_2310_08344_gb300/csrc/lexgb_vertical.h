// Vertical Leja interpolation: the device argument block and the entry
// points of the translation unit that holds its kernels (lexgb_vertical.cu).
#pragma once

#include <cuda_runtime.h>

namespace lexgb {

constexpr int kMaxVertical = 4;

// Arguments of a vertical loop beyond LoopArgs (device resident).
struct VertArgs {
  int np;
  const double* d[kMaxVertical];  // divided differences of each polynomial
  double* p[kMaxVertical];        // FP64 / mixed: the caller's outputs
  float2* pdf[kMaxVertical];      // df64: polynomials as float pairs
  double* fixd;                   // two-step df64 loops: per-polynomial odd-stop coefficients (device)
};

// Fused vertical iteration kernel for (kind, precision, wide, np): wide means
// the vector-access class (FP64 / mixed: 2 points per lane and 16-byte
// aligned vectors; df64: 4 points per lane, nx % 128 == 0, the only df64
// class).  Kernel signature: (const LoopArgs*, const VertArgs*, LoopState*,
// double* partials, unsigned* ticket, cudaGraphConditionalHandle).  NULL if
// the combination has no kernel.
const void* vertical_kernel(int kind, int precision, bool wide, int np);

// The two-step float-float vertical kernel of the diffusion-advection
// operator for np polynomials (leja_iter_df_vertical2x_kernel; the same
// signature, 128 threads per block, dynamic shared memory *smem bytes,
// balanced row ranges), or NULL.
const void* vertical2x_kernel(int np, int* smem);

// Enqueues, before the output pass of polynomial j of a two-step vertical
// loop, the selection of its odd-stop coefficient fixd[j] into the loop
// state (one-thread kernel).
cudaError_t select_vertical_fix(void* state, const double* fixd, int j, cudaStream_t stream);

// Writes v to the device copy dst on `stream` (one-thread kernel).
cudaError_t upload_vertical_args(const VertArgs& v, VertArgs* dst, cudaStream_t stream);

}  // namespace lexgb
