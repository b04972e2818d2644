// Learned step-size / Leja-cost controller: a 5 -> 64 -> 64 -> 64 -> 2 ReLU
// MLP with BF16 weights and activations and FP32 accumulation on the tensor
// cores (mma.sync m16n8k16, operands staged through shared memory with
// ldmatrix).  The paper has no learned component; this network only proposes
// the next step size, and the embedded error test still accepts or rejects
// every step.
//
// Training step (mlp_train_step): one CTA per 128 batch rows runs the
// forward pass, the MSE loss and the full backward pass in shared memory and
// writes its partial gradients; a second kernel adds the partials in CTA
// order (deterministic) and applies Adam to the FP32 master weights, whose
// BF16 copies feed the next step.
//
// Parameter vector (FP32, kMlpParams floats): W1[5][64], b1[64], W2[64][64],
// b2[64], W3[64][64], b3[64], W4[64][2], b4[2]; W[i][j] connects input i to
// output j.  Inputs and targets are normalised with per-feature mean and
// standard deviation held by the model.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "lexgb_internal.h"

namespace {

constexpr int kIn = 5, kHid = 64, kOut = 2;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kIn * kHid, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid * kHid, kOffW4 = kOffB3 + kHid;
constexpr int kOffB4 = kOffW4 + kHid * kOut;
constexpr int kMlpParams = kOffB4 + kOut;  // 8834
constexpr int kRows = 128;                  // batch rows per CTA
constexpr int kMlpThreads = 256;            // 8 warps x 16 rows

// shared-memory strides (bf16 elements); padded so that the eight 16-byte
// rows of every ldmatrix fall into different banks
constexpr int kSX = 24;  // X: [128][16 used]
constexpr int kSH = 72;  // activations / gradients: [128][64 used]
constexpr int kSW = 72;  // W1 [16][64], W2, W3 [64][64]
constexpr int kSW4 = 24; // W4: [64][16 used, 2 non-zero]
constexpr int kSD = 24;  // dY: [128][16 used, 2 non-zero]

struct MlpSmem {
  __nv_bfloat16 x[kRows * kSX];
  __nv_bfloat16 h1[kRows * kSH], h2[kRows * kSH], h3[kRows * kSH];
  __nv_bfloat16 za[kRows * kSH], zb[kRows * kSH];
  __nv_bfloat16 dy[kRows * kSD];
  __nv_bfloat16 w1[16 * kSW], w2[kHid * kSW], w3[kHid * kSW], w4[kHid * kSW4];
  float b1[kHid], b2[kHid], b3[kHid], b4[8];
  float norm[2 * kIn + 2 * kOut];
  float loss[kMlpThreads / 32];
};

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x2(unsigned (&r)[2], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x2_t(unsigned (&r)[2], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(smem_addr(p)));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One 16 x 8 output tile: acc += sum over K of A(m0.., k) * B(k, n0..).
//  AT = false: A stored row-major [m][k] (stride lda);  AT = true: A is the
//  transpose of a row-major [k][m] array.  BT = false: B given as a
//  row-major [n][k] array;  BT = true: B stored row-major [k][n].
template <bool AT, bool BT>
__device__ __forceinline__ void tile_gemm(float (&acc)[4], const __nv_bfloat16* A, int lda, const __nv_bfloat16* B,
                                          int ldb, int m0, int n0, int K) {
  const int lane = threadIdx.x & 31;
  const int i = lane >> 3, r = lane & 7;
  const int lb = lane & 15;
  for (int k0 = 0; k0 < K; k0 += 16) {
    unsigned a[4], b[2];
    if (!AT)
      ldsm_x4(a, A + (size_t)(m0 + (i & 1) * 8 + r) * lda + k0 + (i >> 1) * 8);
    else
      ldsm_x4_t(a, A + (size_t)(k0 + (i >> 1) * 8 + r) * lda + m0 + (i & 1) * 8);
    if (!BT)
      ldsm_x2(b, B + (size_t)(n0 + (lb & 7)) * ldb + k0 + (lb >> 3) * 8);
    else
      ldsm_x2_t(b, B + (size_t)(k0 + (lb >> 3) * 8 + (lb & 7)) * ldb + n0);
    mma_bf16(acc, a, b);
  }
}

// Store a 16x8 accumulator tile (rows m0.., cols n0..) as bf16 after
// bias and optional ReLU, or multiplied by the ReLU mask of `mask`.
__device__ __forceinline__ void store_tile(const float (&acc)[4], __nv_bfloat16* out, int ldo, int m0, int n0,
                                           const float* bias, bool relu, const __nv_bfloat16* mask, int ldm) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, c = (lane & 3) * 2;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int row = m0 + g + 8 * h;
    float v0 = acc[2 * h], v1 = acc[2 * h + 1];
    if (bias) {
      v0 += bias[n0 + c];
      v1 += bias[n0 + c + 1];
    }
    if (relu) {
      v0 = fmaxf(v0, 0.f);
      v1 = fmaxf(v1, 0.f);
    }
    if (mask) {
      if (!(__bfloat162float(mask[(size_t)row * ldm + n0 + c]) > 0.f)) v0 = 0.f;
      if (!(__bfloat162float(mask[(size_t)row * ldm + n0 + c + 1]) > 0.f)) v1 = 0.f;
    }
    *reinterpret_cast<__nv_bfloat162*>(out + (size_t)row * ldo + n0 + c) = __floats2bfloat162_rn(v0, v1);
  }
}

// Write a 16x8 fp32 tile into a row-major [rows][ld] gradient block,
// keeping only rows < mrows and cols < ncols.
__device__ __forceinline__ void write_grad_tile(const float (&acc)[4], float* g, int ld, int m0, int n0, int mrows,
                                                int ncols) {
  const int lane = threadIdx.x & 31;
  const int gr = lane >> 2, c = (lane & 3) * 2;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int row = m0 + gr + 8 * h;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int col = n0 + c + e;
      if (row < mrows && col < ncols) g[(size_t)row * ld + col] = acc[2 * h + e];
    }
  }
}

__device__ void load_weights(MlpSmem& S, const __nv_bfloat16* __restrict__ wb, const float* __restrict__ wf,
                             const float* __restrict__ norm) {
  const int t = threadIdx.x;
  for (int q = t; q < 16 * kSW; q += blockDim.x) S.w1[q] = __float2bfloat16(0.f);
  for (int q = t; q < kHid * kSW4; q += blockDim.x) S.w4[q] = __float2bfloat16(0.f);
  __syncthreads();
  for (int q = t; q < kIn * kHid; q += blockDim.x) S.w1[(q / kHid) * kSW + q % kHid] = wb[kOffW1 + q];
  for (int q = t; q < kHid * kHid; q += blockDim.x) {
    S.w2[(q / kHid) * kSW + q % kHid] = wb[kOffW2 + q];
    S.w3[(q / kHid) * kSW + q % kHid] = wb[kOffW3 + q];
  }
  for (int q = t; q < kHid * kOut; q += blockDim.x) S.w4[(q / kOut) * kSW4 + q % kOut] = wb[kOffW4 + q];
  for (int q = t; q < kHid; q += blockDim.x) {
    S.b1[q] = wf[kOffB1 + q];
    S.b2[q] = wf[kOffB2 + q];
    S.b3[q] = wf[kOffB3 + q];
  }
  if (t < 8) S.b4[t] = t < kOut ? wf[kOffB4 + t] : 0.f;
  if (t < 2 * kIn + 2 * kOut) S.norm[t] = norm[t];
  __syncthreads();  // the normalisation and weights are read by every thread next
}

// Forward pass of the CTA's 128 rows: X (normalised, bf16) -> H1 -> H2 -> H3
// in shared memory; returns the output tile of this warp (16 x 8, cols 0..1).
__device__ void forward_cta(MlpSmem& S, const float* __restrict__ x, int B, int row0, float (&yacc)[4]) {
  const int t = threadIdx.x, warp = t >> 5;
  for (int q = t; q < kRows * 16; q += blockDim.x) {
    const int r = q / 16, c = q % 16;
    float v = 0.f;
    if (c < kIn && row0 + r < B) v = (x[(size_t)(row0 + r) * kIn + c] - S.norm[c]) / S.norm[kIn + c];
    S.x[r * kSX + c] = __float2bfloat16(v);
  }
  __syncthreads();
  const int m0 = warp * 16;
  for (int nt = 0; nt < kHid / 8; ++nt) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    tile_gemm<false, true>(acc, S.x, kSX, S.w1, kSW, m0, nt * 8, 16);
    store_tile(acc, S.h1, kSH, m0, nt * 8, S.b1, true, nullptr, 0);
  }
  __syncwarp();
  for (int nt = 0; nt < kHid / 8; ++nt) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    tile_gemm<false, true>(acc, S.h1, kSH, S.w2, kSW, m0, nt * 8, kHid);
    store_tile(acc, S.h2, kSH, m0, nt * 8, S.b2, true, nullptr, 0);
  }
  __syncwarp();
  for (int nt = 0; nt < kHid / 8; ++nt) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    tile_gemm<false, true>(acc, S.h2, kSH, S.w3, kSW, m0, nt * 8, kHid);
    store_tile(acc, S.h3, kSH, m0, nt * 8, S.b3, true, nullptr, 0);
  }
  __syncwarp();
  yacc[0] = yacc[1] = yacc[2] = yacc[3] = 0.f;
  tile_gemm<false, true>(yacc, S.h3, kSH, S.w4, kSW4, m0, 0, kHid);
  const int lane = t & 31, c = (lane & 3) * 2;
  yacc[0] += S.b4[c];
  yacc[1] += S.b4[c + 1];
  yacc[2] += S.b4[c];
  yacc[3] += S.b4[c + 1];
}

__global__ void __launch_bounds__(kMlpThreads) mlp_forward_kernel(const __nv_bfloat16* __restrict__ wb,
                                                                  const float* __restrict__ wf,
                                                                  const float* __restrict__ norm,
                                                                  const float* __restrict__ x, float* __restrict__ y,
                                                                  int B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem& S = *reinterpret_cast<MlpSmem*>(smem_raw);
  load_weights(S, wb, wf, norm);
  const int row0 = blockIdx.x * kRows;
  float yacc[4];
  forward_cta(S, x, B, row0, yacc);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, c = (lane & 3) * 2;
  if (c == 0) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = row0 + warp * 16 + g + 8 * h;
      if (row < B) {
        y[(size_t)row * kOut] = yacc[2 * h] * S.norm[2 * kIn + 2] + S.norm[2 * kIn];
        y[(size_t)row * kOut + 1] = yacc[2 * h + 1] * S.norm[2 * kIn + 3] + S.norm[2 * kIn + 1];
      }
    }
  }
}

// Forward + MSE loss + backward for 128 rows; partial gradients to
// gpart[blockIdx.x][kMlpParams + 1] (the last entry is the partial loss sum).
// Loss = sum over rows and outputs of (y_n - t_n)^2 / (2 B) on normalised
// outputs y_n and targets t_n.
__global__ void __launch_bounds__(kMlpThreads) mlp_grad_kernel(const __nv_bfloat16* __restrict__ wb,
                                                               const float* __restrict__ wf,
                                                               const float* __restrict__ norm,
                                                               const float* __restrict__ x,
                                                               const float* __restrict__ tgt, int B,
                                                               float* __restrict__ gpart) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem& S = *reinterpret_cast<MlpSmem*>(smem_raw);
  load_weights(S, wb, wf, norm);
  const int row0 = blockIdx.x * kRows;
  float yacc[4];
  forward_cta(S, x, B, row0, yacc);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int g = lane >> 2, c = (lane & 3) * 2;
  float* G = gpart + (size_t)blockIdx.x * (kMlpParams + 1);
  // dY (normalised outputs), zero outside the two outputs and the batch
  for (int q = t; q < kRows * kSD; q += blockDim.x) S.dy[q] = __float2bfloat16(0.f);
  __syncthreads();
  float lsum = 0.f;
  if (c == 0) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = warp * 16 + g + 8 * h, row = row0 + r;
      if (row < B) {
        const float t0 = (tgt[(size_t)row * kOut] - S.norm[2 * kIn]) / S.norm[2 * kIn + 2];
        const float t1 = (tgt[(size_t)row * kOut + 1] - S.norm[2 * kIn + 1]) / S.norm[2 * kIn + 3];
        const float e0 = yacc[2 * h] - t0, e1 = yacc[2 * h + 1] - t1;
        lsum += e0 * e0 + e1 * e1;
        S.dy[r * kSD] = __float2bfloat16(e0 / B);
        S.dy[r * kSD + 1] = __float2bfloat16(e1 / B);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0) S.loss[warp] = lsum;
  __syncthreads();
  if (t == 0) {
    float s = 0.f;
    for (int w = 0; w < kMlpThreads / 32; ++w) s += S.loss[w];
    G[kMlpParams] = s / (2.f * B);
  }
  // layer 4: dW4 = H3^T dY (64 x 2), db4, dH3 = dY W4^T masked by H3 > 0
  if (warp < 4) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    tile_gemm<true, true>(acc, S.h3, kSH, S.dy, kSD, warp * 16, 0, kRows);
    write_grad_tile(acc, G + kOffW4, kOut, warp * 16, 0, kHid, kOut);
  }
  if (t < kOut) {
    float s = 0.f;
    for (int r = 0; r < kRows; ++r) s += __bfloat162float(S.dy[r * kSD + t]);
    G[kOffB4 + t] = s;
  }
  for (int nt = 0; nt < kHid / 8; ++nt) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    tile_gemm<false, false>(acc, S.dy, kSD, S.w4, kSW4, warp * 16, nt * 8, 16);
    store_tile(acc, S.za, kSH, warp * 16, nt * 8, nullptr, false, S.h3, kSH);
  }
  __syncthreads();
  // layer 3: dW3 = H2^T dZ3, db3, dZ2 = (dZ3 W3^T) masked by H2 > 0
  for (int tile = warp; tile < 32; tile += 8) {
    const int mt = tile >> 3, nt = tile & 7;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    tile_gemm<true, true>(acc, S.h2, kSH, S.za, kSH, mt * 16, nt * 8, kRows);
    write_grad_tile(acc, G + kOffW3, kHid, mt * 16, nt * 8, kHid, kHid);
  }
  if (t < kHid) {
    float s = 0.f;
    for (int r = 0; r < kRows; ++r) s += __bfloat162float(S.za[r * kSH + t]);
    G[kOffB3 + t] = s;
  }
  for (int nt = 0; nt < kHid / 8; ++nt) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    tile_gemm<false, false>(acc, S.za, kSH, S.w3, kSW, warp * 16, nt * 8, kHid);
    store_tile(acc, S.zb, kSH, warp * 16, nt * 8, nullptr, false, S.h2, kSH);
  }
  __syncthreads();
  // layer 2: dW2 = H1^T dZ2, db2, dZ1 = (dZ2 W2^T) masked by H1 > 0
  for (int tile = warp; tile < 32; tile += 8) {
    const int mt = tile >> 3, nt = tile & 7;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    tile_gemm<true, true>(acc, S.h1, kSH, S.zb, kSH, mt * 16, nt * 8, kRows);
    write_grad_tile(acc, G + kOffW2, kHid, mt * 16, nt * 8, kHid, kHid);
  }
  if (t < kHid) {
    float s = 0.f;
    for (int r = 0; r < kRows; ++r) s += __bfloat162float(S.zb[r * kSH + t]);
    G[kOffB2 + t] = s;
  }
  __syncthreads();  // za is rewritten next
  for (int nt = 0; nt < kHid / 8; ++nt) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    tile_gemm<false, false>(acc, S.zb, kSH, S.w2, kSW, warp * 16, nt * 8, kHid);
    store_tile(acc, S.za, kSH, warp * 16, nt * 8, nullptr, false, S.h1, kSH);
  }
  __syncthreads();
  // layer 1: dW1 = X^T dZ1 (5 x 64), db1
  {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    tile_gemm<true, true>(acc, S.x, kSX, S.za, kSH, 0, warp * 8, kRows);
    write_grad_tile(acc, G + kOffW1, kHid, 0, warp * 8, kIn, kHid);
  }
  if (t < kHid) {
    float s = 0.f;
    for (int r = 0; r < kRows; ++r) s += __bfloat162float(S.za[r * kSH + t]);
    G[kOffB1 + t] = s;
  }
}

// Sum of the CTA partials in CTA order, then Adam on the FP32 masters and
// their BF16 copies.  adam = 0: only the summed gradient is written.
__global__ void mlp_reduce_adam_kernel(const float* __restrict__ gpart, int nparts, float* __restrict__ grad,
                                       float* __restrict__ w, float* __restrict__ mom, float* __restrict__ vel,
                                       __nv_bfloat16* __restrict__ wb, int adam, float lr, float b1, float b2,
                                       float eps, int step) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > kMlpParams) return;
  float s = 0.f;
  for (int k = 0; k < nparts; ++k) s += gpart[(size_t)k * (kMlpParams + 1) + p];
  grad[p] = s;
  if (!adam || p == kMlpParams) return;
  const float m = b1 * mom[p] + (1.f - b1) * s;
  const float v = b2 * vel[p] + (1.f - b2) * s * s;
  mom[p] = m;
  vel[p] = v;
  const float mh = m / (1.f - powf(b1, (float)step));
  const float vh = v / (1.f - powf(b2, (float)step));
  const float nw = w[p] - lr * mh / (sqrtf(vh) + eps);
  w[p] = nw;
  wb[p] = __float2bfloat16(nw);
}

__global__ void mlp_to_bf16_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kMlpParams) wb[p] = __float2bfloat16(w[p]);
}

bool ok(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return true;
  lexgb::set_last_error(what);
  return false;
}

}  // namespace

struct lx_mlp {
  int batch_max = 0;
  cudaStream_t stream = nullptr;
  float* d_w = nullptr;  // FP32 masters
  float* d_m = nullptr;
  float* d_v = nullptr;
  __nv_bfloat16* d_wb = nullptr;
  float* d_norm = nullptr;
  float* d_gpart = nullptr;
  float* d_grad = nullptr;  // kMlpParams + 1 (loss last)
  float* d_x = nullptr;     // staging for host-input calls
  float* d_y = nullptr;
  int step = 0;
};

extern "C" {

int mlp_param_count(void) { return kMlpParams; }

void mlp_destroy(lx_mlp* m) {
  if (!m) return;
  cudaFree(m->d_w);
  cudaFree(m->d_m);
  cudaFree(m->d_v);
  cudaFree(m->d_wb);
  cudaFree(m->d_norm);
  cudaFree(m->d_gpart);
  cudaFree(m->d_grad);
  cudaFree(m->d_x);
  cudaFree(m->d_y);
  delete m;
}

lx_status mlp_setup(int batch_max, const float* w_host, const float* norm_host, void* cuda_stream, lx_mlp** out) {
  if (!out || batch_max < 1 || batch_max > (1 << 22) || !w_host || !norm_host) return LX_E_INVAL;
  *out = nullptr;
  lx_mlp* m = new lx_mlp();
  m->batch_max = batch_max;
  m->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  const int parts = (batch_max + kRows - 1) / kRows;
  bool good = ok(cudaMalloc((void**)&m->d_w, sizeof(float) * kMlpParams), "cudaMalloc") &&
              ok(cudaMalloc((void**)&m->d_m, sizeof(float) * kMlpParams), "cudaMalloc") &&
              ok(cudaMalloc((void**)&m->d_v, sizeof(float) * kMlpParams), "cudaMalloc") &&
              ok(cudaMalloc((void**)&m->d_wb, sizeof(__nv_bfloat16) * kMlpParams), "cudaMalloc") &&
              ok(cudaMalloc((void**)&m->d_norm, sizeof(float) * (2 * kIn + 2 * kOut)), "cudaMalloc") &&
              ok(cudaMalloc((void**)&m->d_gpart, sizeof(float) * (size_t)parts * (kMlpParams + 1)), "cudaMalloc") &&
              ok(cudaMalloc((void**)&m->d_grad, sizeof(float) * (kMlpParams + 1)), "cudaMalloc") &&
              ok(cudaMalloc((void**)&m->d_x, sizeof(float) * kIn * 64), "cudaMalloc") &&
              ok(cudaMalloc((void**)&m->d_y, sizeof(float) * kOut * 64), "cudaMalloc");
  if (!good) {
    mlp_destroy(m);
    return LX_E_NOMEM;
  }
  good = ok(cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sizeof(MlpSmem)),
            "smem attr") &&
         ok(cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sizeof(MlpSmem)),
            "smem attr") &&
         ok(cudaMemcpy(m->d_w, w_host, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice), "upload w") &&
         ok(cudaMemcpy(m->d_norm, norm_host, sizeof(float) * (2 * kIn + 2 * kOut), cudaMemcpyHostToDevice),
            "upload norm") &&
         ok(cudaMemset(m->d_m, 0, sizeof(float) * kMlpParams), "memset") &&
         ok(cudaMemset(m->d_v, 0, sizeof(float) * kMlpParams), "memset");
  if (!good) {
    mlp_destroy(m);
    return LX_E_CUDA;
  }
  mlp_to_bf16_kernel<<<(kMlpParams + 255) / 256, 256, 0, m->stream>>>(m->d_w, m->d_wb);
  if (!ok(cudaStreamSynchronize(m->stream), "sync")) {
    mlp_destroy(m);
    return LX_E_CUDA;
  }
  *out = m;
  return LX_OK;
}

lx_status mlp_get_weights(lx_mlp* m, float* w_host) {
  if (!m || !w_host) return LX_E_INVAL;
  if (!ok(cudaMemcpyAsync(w_host, m->d_w, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, m->stream), "d2h") ||
      !ok(cudaStreamSynchronize(m->stream), "sync"))
    return LX_E_CUDA;
  return LX_OK;
}

lx_status mlp_forward(lx_mlp* m, const float* x_dev, float* y_dev, int B) {
  if (!m || !x_dev || !y_dev || B < 1) return LX_E_INVAL;
  const int grid = (B + kRows - 1) / kRows;
  mlp_forward_kernel<<<grid, kMlpThreads, sizeof(MlpSmem), m->stream>>>(m->d_wb, m->d_w, m->d_norm, x_dev, y_dev, B);
  if (!ok(cudaGetLastError(), "mlp_forward launch") || !ok(cudaStreamSynchronize(m->stream), "sync"))
    return LX_E_CUDA;
  return LX_OK;
}

lx_status mlp_forward_host(lx_mlp* m, const float* x_host, float* y_host, int B) {
  if (!m || !x_host || !y_host || B < 1 || B > 64) return LX_E_INVAL;
  if (!ok(cudaMemcpyAsync(m->d_x, x_host, sizeof(float) * kIn * B, cudaMemcpyHostToDevice, m->stream), "h2d"))
    return LX_E_CUDA;
  mlp_forward_kernel<<<1, kMlpThreads, sizeof(MlpSmem), m->stream>>>(m->d_wb, m->d_w, m->d_norm, m->d_x, m->d_y, B);
  if (!ok(cudaGetLastError(), "mlp_forward launch") ||
      !ok(cudaMemcpyAsync(y_host, m->d_y, sizeof(float) * kOut * B, cudaMemcpyDeviceToHost, m->stream), "d2h") ||
      !ok(cudaStreamSynchronize(m->stream), "sync"))
    return LX_E_CUDA;
  return LX_OK;
}

// adam = 0: compute the gradient only (grad_host receives kMlpParams
// floats); adam = 1: also take an Adam step.
lx_status mlp_train_step(lx_mlp* m, const float* x_dev, const float* t_dev, int B, int adam, float lr,
                         float* grad_host, float* loss) {
  if (!m || !x_dev || !t_dev || B < 1 || B > m->batch_max) return LX_E_INVAL;
  const int parts = (B + kRows - 1) / kRows;
  mlp_grad_kernel<<<parts, kMlpThreads, sizeof(MlpSmem), m->stream>>>(m->d_wb, m->d_w, m->d_norm, x_dev, t_dev, B,
                                                                       m->d_gpart);
  if (!ok(cudaGetLastError(), "mlp_grad launch")) return LX_E_CUDA;
  if (adam) m->step += 1;
  mlp_reduce_adam_kernel<<<(kMlpParams + 1 + 255) / 256, 256, 0, m->stream>>>(
      m->d_gpart, parts, m->d_grad, m->d_w, m->d_m, m->d_v, m->d_wb, adam, lr, 0.9f, 0.999f, 1e-8f,
      adam ? m->step : 1);
  if (!ok(cudaGetLastError(), "mlp_reduce launch")) return LX_E_CUDA;
  if (grad_host &&
      !ok(cudaMemcpyAsync(grad_host, m->d_grad, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, m->stream), "d2h"))
    return LX_E_CUDA;
  if (loss && !ok(cudaMemcpyAsync(loss, m->d_grad + kMlpParams, sizeof(float), cudaMemcpyDeviceToHost, m->stream),
                  "d2h"))
    return LX_E_CUDA;
  if (!ok(cudaStreamSynchronize(m->stream), "sync")) return LX_E_CUDA;
  return LX_OK;
}

}  // extern "C"
