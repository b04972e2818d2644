// Entry points of the translation units that hold the issue-lean two-step
// float-float kernels (lexgb_df2x.cu: diffusion-advection; lexgb_df2bx.cu:
// the Burgers Jacobian).
#pragma once

namespace lexgb {

// leja_iter_df_pipe2x_kernel<minb, stages, square> (signature of
// the fused iteration kernels: const LoopArgs*, LoopState*, double*
// partials, unsigned* ticket, cudaGraphConditionalHandle), or NULL if that
// instance is not built.  square: the instance with the paired stencil of
// a grid with nx == ny (east and north weights equal, west and south
// equal); the other instance takes any grid.  Its dynamic shared memory is
// df2x_smem_bytes(stages).
const void* df2x_kernel(int minb, int stages, bool square);
int df2x_smem_bytes(int stages);

// leja_iter_df_pipe2bx_kernel<minb, stages, square> (the Burgers Jacobian,
// same signature), or NULL if not built; square as above (nx == ny).  Its
// dynamic shared memory is df2bx_smem_bytes(stages).
const void* df2bx_kernel(int minb, int stages, bool square);
int df2bx_smem_bytes(int stages);

// leja_batch_df_pipe2x_kernel<minb, stages> (lexgb_batch_df.cu: the
// float-float batch, two Leja iterations per pass; signature BatchInst*,
// const int* strip_inst, BatchState*, double* partials, unsigned* tickets,
// unsigned* block_ticket, const double* xi, int H, int total_strips,
// cudaGraphConditionalHandle, int use_cond), or NULL if not built; its
// dynamic shared memory is batch_df2x_smem_bytes(stages).
const void* batch_df2x_kernel(int minb, int stages);
int batch_df2x_smem_bytes(int stages);

}  // namespace lexgb
