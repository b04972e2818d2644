// Entry points of the translation units that hold kernels compiled apart
// from the C ABI's own unit: the issue-lean two-step float-float kernels
// (lexgb_df2x.cu: diffusion-advection; lexgb_df2bx.cu: the Burgers Jacobian;
// lexgb_batch_df.cu: the float-float batch) and the product-form kernels of
// the upwind Burgers Jacobian (lexgb_up3z.cu).
#pragma once

#include <cuda_runtime.h>

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
// power_pass_df_bx_kernel<5>: the lean power pass of the Burgers Jacobian on
// square grids, with the arguments and shared memory of
// power_pass_df_rows_kernel<1, 5> (leja_df64.cuh).
const void* df2bx_power_kernel();
// leja_iter_df_vertical2bx_kernel for np = 1..3 polynomials (the two-step
// float-float vertical loop of the Burgers Jacobian; the signature of the
// vertical kernels, 128 threads, dynamic shared memory *smem), or NULL.
const void* vertical2bx_kernel(int np, int* smem);
// The point weights of the Burgers Jacobian as float pairs from u alone
// (burgers_weights_df_kernel): q = u gx, r = wc0 - (u_x + u_y) ig, central
// differences with spacings dx, dy; nx % 128 == 0 and u 16-byte aligned.
cudaError_t burgers_weights_df(int nx, int ny, const double* u, double gx, double ig, double wc0, double dx,
                               double dy, float2* q, float2* r, int sm_count, cudaStream_t stream);
// Fields of a Burgers EXPRB32 step in float-float, written as doubles
// (burgers_field_df_kernel): mode 0, f_out = h (nu lap v - v (v_x + v_y))
// (+ h src when src is not NULL); mode 1, f_out = -h v (v_x + v_y).  nx %
// 128 == 0; v, src and f_out 16-byte aligned.
cudaError_t burgers_field_df(int mode, int nx, int ny, const double* v, const double* src, double h, double nu,
                             double dx, double dy, double* f_out, int sm_count, cudaStream_t stream);

// leja_batch_df_pipe2x_kernel<minb, stages> (lexgb_batch_df.cu: the
// float-float batch, two Leja iterations per pass; signature BatchInst*,
// const int* strip_inst, BatchState*, double* partials, unsigned* tickets,
// unsigned* block_ticket, const double* xi, int H, int total_strips,
// cudaGraphConditionalHandle, int use_cond), or NULL if not built; its
// dynamic shared memory is batch_df2x_smem_bytes(stages).
const void* batch_df2x_kernel(int minb, int stages);
int batch_df2x_smem_bytes(int stages);

// leja_iter_df_pipe_burgers_up3z_kernel<minb, stages> (the fused iteration
// signature) for (3, 5) and (2, 6), or NULL; its dynamic shared memory is
// up3z_smem_bytes<stages>() (leja_upwind.cuh).
const void* up3z_leja_kernel(int minb, int stages);
// power_pass_df_pipe_burgers_up3z_kernel<3, 5>: (Up3Op, const void* vin,
// int vin_double, float2* w, const float2* q, double* partials, unsigned*
// ticket, LoopState*), dynamic shared memory up3z_smem_bytes<5>().
const void* up3z_power_kernel();

// leja_iter_df_pipe2x_up3_kernel<minb, stages, square> (lexgb_up3x.cu: the
// issue-lean two-step kernel of the upwind diffusion-advection operator;
// fused iteration signature) for minb 3, stages 5 or 6, or NULL; square:
// the paired stencil (nx == ny with equal x and y coefficients).  Its
// dynamic shared memory is up3x_smem_bytes(stages).
const void* up3x_kernel(int minb, int stages, bool square);
int up3x_smem_bytes(int stages);

}  // namespace lexgb
