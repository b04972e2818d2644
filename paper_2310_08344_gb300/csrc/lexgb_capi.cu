// Context, CUDA-graph Leja loop and C ABI of the engine (see include/lexgb.h).
//
// A context is the GB300 counterpart of the paper's struct Leja (Sec. 2.3,
// Listing 10): it owns the auxiliary device vectors from setup to destroy and
// runs the integrators.  Each Leja loop is one launch of a CUDA graph whose
// only node is a while-loop around the fused Leja-iteration kernel; the last
// block of each iteration decides convergence and ends the loop from the
// device, so the host synchronises once per API call instead of once per
// iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "leja_batch.cuh"
#include "leja_df64.cuh"
#include "leja_df64_2step.cuh"
#include "leja_upwind.cuh"
#include "leja_upwind_2step.cuh"
#include "leja_kernels.cuh"
#include "lexgb_df2x.h"
#include "lexgb_internal.h"
#include "lexgb_vertical.h"

using namespace lexgb;

namespace lexgb {
void set_last_error(const char* msg);
}

namespace {

thread_local std::string g_last_cuda_error;

bool cuda_ok(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return true;
  g_last_cuda_error = std::string(what) + ": " + cudaGetErrorString(e);
  return false;
}

}  // namespace

void lexgb::set_last_error(const char* msg) { g_last_cuda_error = msg; }

namespace {

#define LX_CUDA(call)                                   \
  do {                                                  \
    if (!cuda_ok((call), #call)) return LX_E_CUDA;      \
  } while (0)

constexpr int kMaxPower = 64;

struct CoefSlot {
  bool valid = false;
  int l = -1, count = 0;
  double h = 0, c = 0, gamma = 0;
  double* dev = nullptr;
  double* host = nullptr;  // pinned staging
};

// Kernel classes of the fused Leja iteration: "wide" (vector accesses; needs
// nx a multiple of the warp row and 16-byte aligned vectors) and "generic".
enum Variant { kVec2 = 0, kVec1 = 1, kNumVariants = 2 };

// One candidate implementation of the fused iteration.
struct Cand {
  const void* func;
  int threads;  // block size
  int smem;     // dynamic shared memory bytes
  int vec;      // points per lane (warp row = 32 * vec points)
  const char* name;
  int ipl = 1;  // Leja iterations per launch
  int strip = -1;  // default strip height when not autotuned (-1: by kind of kernel)
};

struct LoopGraph {
  bool built = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int grid = 0;
  Cand cand{};
  int strip_h = 32;
  int unroll = 1;
};

}  // namespace

struct lx_ctx {
  lx_problem prob{};
  int integrator = LX_ROS_EU;
  int K = 1000;
  cudaStream_t stream = nullptr;
  int device = 0;
  int sm_count = 0;
  long long n = 0;
  int strip_h = 32;
  Geo geo{};
  Up3Op up3{};  // constants of the upwind operators (kinds LX_*_UP3)

  double* d_xi = nullptr;
  CoefSlot coef[2];
  void* d_y[2] = {nullptr, nullptr};
  double* d_f = nullptr;   // h f(u), later R
  double* d_s = nullptr;   // u_x + u_y (Burgers)
  double* d_p3 = nullptr;  // phi_3 result (EXPRB32, EPIRK4s3A)
  double* d_ep[3] = {nullptr, nullptr, nullptr};  // EPIRK4s3A: stage increments, W3 / W4
  double* d_pw[2] = {nullptr, nullptr};  // power iteration ping-pong
  double* d_io[3] = {nullptr, nullptr, nullptr};  // staging for expint_step_host
  float2* d_pdf = nullptr;  // df64 form: polynomial as float pairs
  double* d_tune = nullptr; // autotuner: output vector of the timing runs
  float2* d_bq = nullptr;   // df64 Burgers: u / (2 dx gamma) per point
  float2* d_br = nullptr;   // df64 Burgers: diagonal weight per point
  float* d_uf = nullptr;    // mixed Burgers: u as floats
  float* d_sf = nullptr;    // mixed Burgers: u_x + u_y as floats
  // linearisation point, 1/gamma and c for which d_bq / d_br / d_uf / d_sf are
  // current within one call (the two loops of an EXPRB32 step share them);
  // cleared by every call and by every other writer of those buffers
  const double* prep_u = nullptr;
  double prep_ig = 0.0, prep_cc = 0.0;
  const double* d_src = nullptr;  // caller's time-independent source (borrowed), or NULL
  double* d_partials = nullptr;
  int partials_cap = 0;
  int stream_loop = 0;  // 1: launch the iterations from the host (profilers)
  int graph_unroll = 4; // fused-iteration kernel nodes per pass of the graph's while body
  int graph_iter_launches_pending = 0;  // a graph loop ran since the last end_call
  unsigned int* d_ticket = nullptr;
  LoopState* d_state = nullptr;
  LoopArgs* d_args = nullptr;
  LoopState* h_state = nullptr;  // pinned

  LoopGraph loop[kNumVariants];
  // vertical interpolation (lazily allocated): argument block, one
  // coefficient table of K doubles per polynomial, df64 polynomials beyond
  // the first (which uses d_pdf), and the loop graphs by class and count
  VertArgs* d_vargs = nullptr;
  double* d_vcoef = nullptr;
  double* d_vfix = nullptr;  // two-step df64 loops: per-polynomial odd-stop coefficients
  float2* d_pdfv[kMaxVertical] = {};
  LoopGraph vloop[kNumVariants][kMaxVertical];
  int aux_grid = 0;
  int pow_pipe_grid = 0;  // grid of the pipelined upwind power pass (0: not yet sized)

  cudaEvent_t ev[8] = {};
  int ev_used = 0;
  cudaEvent_t ev_pow[2] = {};
  lx_stats stats{};
};

namespace {

size_t basis_bytes(const lx_ctx* c) {
  return (size_t)c->n * (c->prob.precision == LX_MIXED ? sizeof(float) : sizeof(double));
}


template <int KIND, typename T, int VEC>
Cand iter_cand(const char* name) {
  return Cand{reinterpret_cast<const void*>(&leja_iter_kernel<KIND, T, VEC>), kThreadsPerBlock, 0, VEC, name};
}

bool is_burgers(int kind) { return kind == LX_BURGERS || kind == LX_BURGERS_UP3; }
bool is_up3(int kind) { return kind == LX_ADVDIFF_UP3 || kind == LX_BURGERS_UP3; }

// Candidates for (kind, precision, class); the first is the default.
std::vector<Cand> candidates(int kind, int precision, int cls, bool square = false) {
  const bool wide = cls == kVec2;
  std::vector<Cand> v;
  if (is_up3(kind)) {
    // point-wise kernels: one candidate, the same for both classes
    const bool b = kind == LX_BURGERS_UP3;
    const void* f = nullptr;
    const char* name = nullptr;
    if (precision == LX_DF64) {
      if (b && wide) {
        // product form first (z = q y formed once per point, constant
        // weights; 592 us per iteration at 8192^2 with balanced row ranges,
        // against 782 us for the point-weight form), then the point-weight form
        v.push_back(Cand{up3z_leja_kernel(3, 5), kPipeThreads,
                         up3z_smem_bytes<5>(), 4, "leja_iter_df_pipe_burgers_up3z_b3", 1, 0});
        v.push_back(Cand{up3z_leja_kernel(2, 6), kPipeThreads,
                         up3z_smem_bytes<6>(), 4, "leja_iter_df_pipe_burgers_up3z_b2", 1, 0});
        v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe_burgers_up3_kernel<2>), kPipeThreads,
                         kUpSmemBytesB, 4, "leja_iter_df_pipe_burgers_up3_b2"});
        v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe_burgers_up3_kernel<1>), kPipeThreads,
                         kUpSmemBytesB, 4, "leja_iter_df_pipe_burgers_up3_b1"});
      }
      if (!b && wide) {
        // pipelined (nx % 128 == 0, aligned vectors), then the point-wise form
        // two Leja iterations per pass first (379 us per iteration at 8192^2),
        // then one (390 us; 411 us with 8-row strips instead of balanced row
        // ranges): the kernels are issue-bound, so halving the traffic gains
        // only what the smaller instruction count per iteration gives
        // the issue-lean two-step form first (square grids get the paired
        // stencil), then the first two-step form
        v.push_back(Cand{up3x_kernel(3, 6, square), kPipeThreads, up3x_smem_bytes(6), 4, "leja_iter_df_pipe2x_up3_b3",
                         2, 0});
        v.push_back(Cand{up3x_kernel(3, 5, square), kPipeThreads, up3x_smem_bytes(5), 4,
                         "leja_iter_df_pipe2x_up3_b3_s5", 2, 0});
        v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe2_up3_kernel<3, 6>), kPipeThreads,
                         up3_2step_smem_bytes<6>(), 4, "leja_iter_df_pipe2_up3_b3", 2, 0});
        v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe_up3_kernel<3>), kPipeThreads,
                         kUpSmemBytes, 4, "leja_iter_df_pipe_up3_b3", 1, 0});
        v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe_up3_kernel<2>), kPipeThreads,
                         kUpSmemBytes, 4, "leja_iter_df_pipe_up3_b2", 1, 0});
        v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe2_up3_kernel<2, 6>), kPipeThreads,
                         up3_2step_smem_bytes<6>(), 4, "leja_iter_df_pipe2_up3_b2", 2, 0});
        v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe2_up3_kernel<4, 5>), kPipeThreads,
                         up3_2step_smem_bytes<5>(), 4, "leja_iter_df_pipe2_up3_b4", 2, 0});
      }
      if (!b) {
        f = reinterpret_cast<const void*>(&leja_iter_df_up3_kernel);
        name = "leja_iter_df_up3";
      }
    } else if (precision == LX_MIXED) {
      f = b ? reinterpret_cast<const void*>(&leja_iter_up3_kernel<true, float>)
            : reinterpret_cast<const void*>(&leja_iter_up3_kernel<false, float>);
      name = b ? "leja_iter_burgers_up3_mixed" : "leja_iter_advdiff_up3_mixed";
    } else {
      f = b ? reinterpret_cast<const void*>(&leja_iter_up3_kernel<true, double>)
            : reinterpret_cast<const void*>(&leja_iter_up3_kernel<false, double>);
      name = b ? "leja_iter_burgers_up3_f64" : "leja_iter_advdiff_up3_f64";
    }
    if (f) v.push_back(Cand{f, kThreadsPerBlock, 0, 1, name});
    return v;
  }
  if (precision == LX_DF64 && kind == LX_BURGERS) {
    if (wide) {
      // the issue-lean two-step form first (square grids get the paired
      // stencil): 34.0 us per Leja iteration at 2048^2 with a 5-row ring at 2
      // blocks/SM, 35.6 us with 4 rows at 3, against 47.7 us for the first
      // two-step form
      v.push_back(Cand{df2bx_kernel(2, 5, square), kPipeThreads, df2bx_smem_bytes(5), 4,
                       "leja_iter_df_pipe2bx_b2", 2});
      v.push_back(Cand{df2bx_kernel(3, 4, square), kPipeThreads, df2bx_smem_bytes(4), 4,
                       "leja_iter_df_pipe2bx_b3_s4", 2});
      v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe_burgers_kernel<1>), kPipeThreads,
                       kPipeSmemBytesB, 4, "leja_iter_df_pipe_burgers_b1"});
      v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe_burgers_kernel<2>), kPipeThreads,
                       kPipeSmemBytesB, 4, "leja_iter_df_pipe_burgers_b2"});
      v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe_burgers_kernel<3, 4>), kPipeThreads,
                       kPipeSmemBytesB4, 4, "leja_iter_df_pipe_burgers_b3_s4"});
      v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe2_burgers_kernel<1, 5>), kPipeThreads,
                       pipe2b_smem_bytes<5>(), 4, "leja_iter_df_pipe2_burgers_b1", 2});
      v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe2_burgers_kernel<2, 5>), kPipeThreads,
                       pipe2b_smem_bytes<5>(), 4, "leja_iter_df_pipe2_burgers_b2", 2});
      // more resident blocks with shorter rings (shared memory is the limit)
      v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe2_burgers_kernel<3, 4>), kPipeThreads,
                       pipe2b_smem_bytes<4>(), 4, "leja_iter_df_pipe2_burgers_b3_s4", 2});
      v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe_burgers_kernel<4, 3>), kPipeThreads,
                       kPipeWarps * 3 * kSlotElemsB * 8, 4, "leja_iter_df_pipe_burgers_b4_s3"});
    }
    return v;
  }
  if (precision == LX_DF64) {
    if (wide) {
      // default without autotuning: two iterations per pass at four blocks
      // per SM, issue-lean form
      // (square grids get the instances with the paired stencil built in)
      v.push_back(Cand{df2x_kernel(4, 4, square), kPipeThreads, df2x_smem_bytes(4), 4, "leja_iter_df_pipe2x_b4_s4",
                       2});
      v.push_back(Cand{df2x_kernel(4, 5, square), kPipeThreads, df2x_smem_bytes(5), 4, "leja_iter_df_pipe2x_b4", 2});
      v.push_back(Cand{df2x_kernel(3, 5, square), kPipeThreads, df2x_smem_bytes(5), 4, "leja_iter_df_pipe2x_b3", 2});
      v.push_back(Cand{df2x_kernel(5, 4, square), kPipeThreads, df2x_smem_bytes(4), 4, "leja_iter_df_pipe2x_b5_s4",
                       2});
      // the first two-step form (155 us per launch at 4096^2, four blocks per SM)
      v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe2_kernel<4, 4>), kPipeThreads,
                       pipe2_smem_bytes<4>(), 4, "leja_iter_df_pipe2_b4_s4", 2});
      v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe2_kernel<2, 6>), kPipeThreads,
                       pipe2_smem_bytes<6>(), 4, "leja_iter_df_pipe2_b2_s6", 2});
      v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe_kernel<2>), kPipeThreads, kPipeSmemBytes, 4,
                       "leja_iter_df_pipe_b2"});
      v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe_kernel<3>), kPipeThreads, kPipeSmemBytes, 4,
                       "leja_iter_df_pipe_b3"});
      v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe_kernel<4>), kPipeThreads, kPipeSmemBytes, 4,
                       "leja_iter_df_pipe_b4"});
      v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe_kernel<2, 8>), kPipeThreads,
                       kPipeSmemBytes8, 4, "leja_iter_df_pipe_b2_s8"});
      v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe_kernel<3, 8>), kPipeThreads,
                       kPipeSmemBytes8, 4, "leja_iter_df_pipe_b3_s8"});
      v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_advdiff_kernel<4>), kThreadsPerBlock, 0, 4,
                       "leja_iter_df_advdiff_v4"});
      v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe2_kernel<1, 5>), kPipeThreads,
                       pipe2_smem_bytes<5>(), 4, "leja_iter_df_pipe2_b1", 2});
      v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe2_kernel<2, 5>), kPipeThreads,
                       pipe2_smem_bytes<5>(), 4, "leja_iter_df_pipe2_b2", 2});
      v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe2_kernel<3, 5>), kPipeThreads,
                       pipe2_smem_bytes<5>(), 4, "leja_iter_df_pipe2_b3", 2});
      v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe2_kernel<3, 6>), kPipeThreads,
                       pipe2_smem_bytes<6>(), 4, "leja_iter_df_pipe2_b3_s6", 2});
      // four resident blocks per SM (127 registers, no spills)
      v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe2_kernel<4, 5>), kPipeThreads,
                       pipe2_smem_bytes<5>(), 4, "leja_iter_df_pipe2_b4", 2});
      // five (96 registers, a few bytes of spills)
      v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_pipe2_kernel<5, 4>), kPipeThreads,
                       pipe2_smem_bytes<4>(), 4, "leja_iter_df_pipe2_b5_s4", 2});
    } else {
      v.push_back(Cand{reinterpret_cast<const void*>(&leja_iter_df_advdiff_kernel<1>), kThreadsPerBlock, 0, 1,
                       "leja_iter_df_advdiff_v1"});
    }
    return v;
  }
  const bool mixed = precision == LX_MIXED;
  if (kind == LX_ADVDIFF) {
    if (!mixed)
      v.push_back(wide ? iter_cand<0, double, 2>("leja_iter_advdiff_f64_v2")
                       : iter_cand<0, double, 1>("leja_iter_advdiff_f64_v1"));
    else
      v.push_back(wide ? iter_cand<0, float, 2>("leja_iter_advdiff_mixed_v2")
                       : iter_cand<0, float, 1>("leja_iter_advdiff_mixed_v1"));
  } else {
    if (!mixed)
      v.push_back(wide ? iter_cand<1, double, 2>("leja_iter_burgers_f64_v2")
                       : iter_cand<1, double, 1>("leja_iter_burgers_f64_v1"));
    else
      v.push_back(wide ? iter_cand<1, float, 2>("leja_iter_burgers_mixed_v2")
                       : iter_cand<1, float, 1>("leja_iter_burgers_mixed_v1"));
  }
  return v;
}

int wide_vec(const lx_ctx* c) { return candidates(c->prob.kind, c->prob.precision, kVec2)[0].vec; }
bool is_square(const lx_problem& P) { return P.nx == P.ny; }

int grid_for(const lx_ctx* c, const Cand& k, int strip_h, int* grid) {
  if (k.smem > 48 * 1024 &&
      !cuda_ok(cudaFuncSetAttribute(k.func, cudaFuncAttributeMaxDynamicSharedMemorySize, k.smem), "smem attribute"))
    return LX_E_CUDA;
  const int ncs = (c->prob.nx + 32 * k.vec - 1) / (32 * k.vec);
  const int wpb = k.threads / 32;
  // strip_h == 0 (pipelined kernels only): one balanced row range per warp,
  // at least 4 rows each
  if (strip_h == 0 && k.smem == 0) return LX_E_INVAL;
  const long long units = strip_h > 0 ? (long long)ncs * ((c->prob.ny + strip_h - 1) / strip_h)
                                      : ((long long)ncs * c->prob.ny + 3) / 4;
  int per_sm = 0;
  if (!cuda_ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.func, k.threads, k.smem), "occupancy"))
    return LX_E_CUDA;
  per_sm = std::max(per_sm, 1);
  const int want = (int)std::min<long long>((units + wpb - 1) / wpb, 1 << 30);
  *grid = std::max(1, std::min(want, per_sm * c->sm_count));
  return *grid > c->partials_cap ? LX_E_INVAL : LX_OK;
}

void destroy_graph(LoopGraph& L) {
  if (L.exec) cudaGraphExecDestroy(L.exec);
  if (L.graph) cudaGraphDestroy(L.graph);
  L.exec = nullptr;
  L.graph = nullptr;
  L.built = false;
}

// (Re)build the while-loop graph of class `variant` around candidate k.
lx_status build_loop_graph(lx_ctx* c, int variant, const Cand& k, int strip_h) {
  LoopGraph& L = c->loop[variant];
  if (L.built && L.cand.func == k.func && L.strip_h == strip_h && L.unroll == c->graph_unroll) return LX_OK;
  destroy_graph(L);
  int grid = 0;
  int gs = grid_for(c, k, strip_h, &grid);
  if (gs != LX_OK) return (lx_status)gs;
  L.cand = k;
  L.strip_h = strip_h;
  L.unroll = c->graph_unroll;
  L.grid = grid;
  LX_CUDA(cudaGraphCreate(&L.graph, 0));
  cudaGraphConditionalHandle cond;
  LX_CUDA(cudaGraphConditionalHandleCreate(&cond, L.graph, 1, cudaGraphCondAssignDefault));
  // cudaGraphNodeParams holds a union without a default constructor: build it
  // in zeroed raw storage.
  alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
  std::memset(cp_raw, 0, sizeof(cp_raw));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  LX_CUDA(cudaGraphAddNode(&cnode, L.graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];

  const LoopArgs* args = c->d_args;
  LoopState* st = c->d_state;
  double* partials = c->d_partials;
  unsigned int* ticket = c->d_ticket;
  void* kargs[] = {(void*)&args, (void*)&st, (void*)&partials, (void*)&ticket, (void*)&cond};
  cudaKernelNodeParams kp;
  std::memset(&kp, 0, sizeof(kp));
  kp.func = const_cast<void*>(k.func);
  kp.gridDim = dim3(L.grid);
  kp.blockDim = dim3(k.threads);
  kp.sharedMemBytes = k.smem;
  kp.kernelParams = kargs;
  // `unroll` chained launches per pass of the body: the while condition is
  // evaluated once per pass; launches after the stop return at once.
  cudaGraphNode_t prev = nullptr;
  for (int u = 0; u < L.unroll; ++u) {
    cudaGraphNode_t knode;
    LX_CUDA(cudaGraphAddKernelNode(&knode, body, prev ? &prev : nullptr, prev ? 1 : 0, &kp));
    prev = knode;
  }
  LX_CUDA(cudaGraphInstantiate(&L.exec, L.graph, 0));
  L.built = true;
  return LX_OK;
}

int aux_blocks(const lx_ctx* c) {
  const long long want = (c->n + kThreadsPerBlock - 1) / kThreadsPerBlock;
  return (int)std::max<long long>(1, std::min<long long>(want, (long long)c->aux_grid));
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int choose_variant(const lx_ctx* c, const double* w, const double* out) {
  const int rowpts = 32 * wide_vec(c);
  if (c->prob.nx % rowpts != 0) return kVec1;
  if (c->prob.precision == LX_DF64)  // out is written by the conversion pass
    return aligned16(w) ? kVec2 : kVec1;
  if (aligned16(w) && aligned16(out) && aligned16(c->d_y[0]) && aligned16(c->d_y[1])) return kVec2;
  return kVec1;
}

// Selected candidate of a class (built on first use with the default).
lx_status ensure_graph(lx_ctx* c, int variant) {
  if (c->loop[variant].built) return LX_OK;
  const std::vector<Cand> cands = candidates(c->prob.kind, c->prob.precision, variant, is_square(c->prob));
  if (cands.empty()) {
    set_last_error("no kernel for this layout: the float-float Burgers form needs nx % 128 == 0 and 16-byte "
                   "aligned vectors");
    return LX_E_INVAL;
  }
  const Cand k = cands[0];
  // a candidate's own default strip height if it has one; otherwise
  // pipelined kernels (dynamic shared memory) default to 8-row strips (one
  // strip per warp then gives enough resident warps on mid-size grids), the
  // two-step kernel to balanced row ranges (its halo rows cost arithmetic)
  const int strip = k.strip >= 0 ? k.strip : (k.ipl == 2 ? 0 : (k.smem > 0 ? 8 : c->strip_h));
  return build_loop_graph(c, variant, k, strip);
}

lx_status ensure_coeffs(lx_ctx* c, int slot, int l, double h, double cc, double gamma) {
  CoefSlot& S = c->coef[slot];
  if (S.valid && S.l == l && S.h == h && S.c == cc && S.gamma == gamma) return LX_OK;
  const int count = leja_coeff_count(h, cc, gamma, c->K);
  std::vector<double> xi(count);
  leja_points(count, xi.data());
  int st = leja_coeffs(l, h, cc, gamma, xi.data(), count, S.host);
  if (st != LX_OK) return (lx_status)st;
  LX_CUDA(cudaMemcpyAsync(S.dev, S.host, sizeof(double) * count, cudaMemcpyHostToDevice, c->stream));
  S.valid = true;
  S.l = l;
  S.h = h;
  S.c = cc;
  S.gamma = gamma;
  S.count = count;
  return LX_OK;
}

// Loop arguments of one Leja loop (operator weights for the interval
// (c, gamma), tolerances, buffers) and the per-loop preparation kernels: the
// df64 Burgers point weights, the argument upload and state reset, and the
// df64 input scaling (wexp_known: the kernel that wrote w has already
// recorded its largest exponent).  d: divided differences with kmax + 1
// entries.
lx_status prepare_loop(lx_ctx* c, int strip_h, int kmax, const double* d, const double* u, const double* w,
                       double* out, double cc, double gamma, double rtol, double atol, bool wexp_known) {
  const lx_problem& P = c->prob;
  const double dx = 1.0 / P.nx, dy = 1.0 / P.ny;
  const double ig = 1.0 / gamma;
  LoopArgs a;
  std::memset(&a, 0, sizeof(a));
  a.nx = P.nx;
  a.ny = P.ny;
  a.n = c->n;
  a.strip_h = strip_h;
  a.kmax = kmax;
  a.w = w;
  a.y0 = c->d_y[0];
  a.y1 = c->d_y[1];
  a.p = out;
  a.u = u;
  a.s = c->d_s;
  a.xi = c->d_xi;
  a.d = d;
  const double nx2 = P.nu / (dx * dx), ny2 = P.nu / (dy * dy);
  if (P.kind == LX_ADVDIFF) {
    a.wxp = (nx2 + P.a / (2 * dx)) * ig;
    a.wxm = (nx2 - P.a / (2 * dx)) * ig;
    a.wyp = (ny2 + P.a / (2 * dy)) * ig;
    a.wym = (ny2 - P.a / (2 * dy)) * ig;
  } else {
    a.lx = nx2 * ig;
    a.ly = ny2 * ig;
    a.gx = ig / (2 * dx);
    a.gy = ig / (2 * dy);
    a.inv_gamma = ig;
  }
  a.wc0 = (-2.0 * nx2 - 2.0 * ny2 - cc) * ig;
  a.rtol = rtol;
  a.atol = atol;
  a.up = c->up3;
  a.up_c = cc;
  if (is_up3(P.kind)) a.inv_gamma = ig;
  const bool prep_current = c->prep_u == u && c->prep_ig == ig && c->prep_cc == cc;
  if (P.precision == LX_MIXED && P.kind == LX_BURGERS) {
    // the mixed form's float copies of u and u_x + u_y, once per loop
    a.uf = c->d_uf;
    a.sf = c->d_sf;
    if (!prep_current) {
      to_float_kernel<<<aux_blocks(c), kThreadsPerBlock, 0, c->stream>>>(c->n, u, c->d_uf);
      to_float_kernel<<<aux_blocks(c), kThreadsPerBlock, 0, c->stream>>>(c->n, c->d_s, c->d_sf);
      c->stats.kernels += 2;
      LX_CUDA(cudaGetLastError());
    }
  }
  if (P.precision == LX_DF64 && P.kind == LX_BURGERS_UP3) {
    // q = u |a| / (6 dx gamma) as float pairs for the point weights
    a.bq = c->d_bq;
    if (!prep_current) {
      up3_df_prep_kernel<<<aux_blocks(c), kThreadsPerBlock, 0, c->stream>>>(c->n, u, c->up3.gx * ig, c->d_bq);
      ++c->stats.kernels;
      LX_CUDA(cudaGetLastError());
    }
  }
  const double wd[4] = {a.wxp, a.wxm, a.wyp, a.wym};
  for (int k = 0; k < 4; ++k) {
    const float hi = (float)wd[k];
    a.wf[2 * k] = hi;
    a.wf[2 * k + 1] = (float)(wd[k] - (double)hi);
  }
  a.pdf = c->d_pdf;
  a.use_cond = c->stream_loop ? 0 : 1;
  const bool df = P.precision == LX_DF64;
  if (df && P.kind == LX_BURGERS) {
    const double blv[3] = {nx2 * ig, ny2 * ig, dx / dy};
    for (int k = 0; k < 3; ++k) {
      a.bl[2 * k] = (float)blv[k];
      a.bl[2 * k + 1] = (float)(blv[k] - (double)a.bl[2 * k]);
    }
    a.bq = c->d_bq;
    a.br = c->d_br;
    if (!prep_current) {
      if (P.nx % kPipeRow == 0 && aligned16(u))
        LX_CUDA(burgers_weights_df(P.nx, P.ny, u, ig / (2 * dx), ig, a.wc0, dx, dy, c->d_bq, c->d_br, c->sm_count,
                                   c->stream));
      else
        burgers_df_prep_kernel<<<aux_blocks(c), kThreadsPerBlock, 0, c->stream>>>(c->n, u, c->d_s, ig / (2 * dx),
                                                                                   ig, a.wc0, c->d_bq, c->d_br);
      ++c->stats.kernels;
      LX_CUDA(cudaGetLastError());
    }
  }
  c->prep_u = u;
  c->prep_ig = ig;
  c->prep_cc = cc;
  set_loop_args_kernel<<<1, 1, 0, c->stream>>>(a, c->d_args, c->d_state, c->d_ticket, wexp_known ? 0 : 1);
  ++c->stats.kernels;
  LX_CUDA(cudaGetLastError());
  if (df) {
    if (!wexp_known) {
      df_scale_kernel<<<aux_blocks(c), kThreadsPerBlock, 0, c->stream>>>(c->n, w, c->d_state);
      ++c->stats.kernels;
      LX_CUDA(cudaGetLastError());
    }
    df_scale_finish_kernel<<<1, 1, 0, c->stream>>>(c->d_state);
    ++c->stats.kernels;
    LX_CUDA(cudaGetLastError());
  }
  return LX_OK;
}

// One Leja loop.  df64 form only: `base` (may be NULL) is added to the
// output in the conversion pass, and wexp_known says that the kernel that
// wrote w has already recorded its largest exponent.
lx_status launch_loop(lx_ctx* c, int slot, int l, const double* u, const double* w, double* out, double cc,
                      double gamma, double h, double rtol, double atol, const double* base = nullptr,
                      bool wexp_known = false) {
  lx_status st = ensure_coeffs(c, slot, l, h, cc, gamma);
  if (st != LX_OK) return st;
  const int variant = choose_variant(c, w, out);
  st = ensure_graph(c, variant);
  if (st != LX_OK) return st;
  st = prepare_loop(c, c->loop[variant].strip_h, c->coef[slot].count - 1, c->coef[slot].dev, u, w, out, cc, gamma,
                    rtol, atol, wexp_known);
  if (st != LX_OK) return st;
  const bool df = c->prob.precision == LX_DF64;
  if (c->ev_used + 2 > 8) return LX_E_INVAL;
  LX_CUDA(cudaEventRecord(c->ev[c->ev_used], c->stream));
  if (!c->stream_loop) {
    LX_CUDA(cudaGraphLaunch(c->loop[variant].exec, c->stream));
    c->graph_iter_launches_pending = 1;
  } else {
    // Host-driven loop for profilers that cannot see kernels inside a
    // conditional graph: batches of launches, each kernel returning at once
    // after the device has set done.
    LoopGraph& L = c->loop[variant];
    const LoopArgs* args = c->d_args;
    LoopState* stp = c->d_state;
    double* partials = c->d_partials;
    unsigned int* ticket = c->d_ticket;
    cudaGraphConditionalHandle cond = 0;
    void* kargs[] = {(void*)&args, (void*)&stp, (void*)&partials, (void*)&ticket, (void*)&cond};
    for (int it = 0; it < c->coef[slot].count - 1; it += 8) {
      for (int k = 0; k < 8; ++k)
        LX_CUDA(cudaLaunchKernel(L.cand.func, dim3(L.grid), dim3(L.cand.threads), kargs, L.cand.smem, c->stream));
      c->stats.kernels += 8;
      LX_CUDA(cudaMemcpyAsync(c->h_state, c->d_state, sizeof(LoopState), cudaMemcpyDeviceToHost, c->stream));
      LX_CUDA(cudaStreamSynchronize(c->stream));
      if (c->h_state->done) break;
    }
  }
  LX_CUDA(cudaEventRecord(c->ev[c->ev_used + 1], c->stream));
  c->ev_used += 2;
  if (df && c->n % 2 == 0 && aligned16(out) && (!base || aligned16(base))) {
    const long long n2 = c->n / 2;
    const int G2 = (int)std::max<long long>(1, std::min<long long>((n2 + kThreadsPerBlock - 1) / kThreadsPerBlock,
                                                                   8LL * c->sm_count));
    df_output2_kernel<<<G2, kThreadsPerBlock, 0, c->stream>>>(
        n2, reinterpret_cast<const float4*>(c->d_pdf), reinterpret_cast<const double2*>(base),
        reinterpret_cast<double2*>(out), c->d_state, static_cast<const float4*>(c->d_y[0]),
        static_cast<const float4*>(c->d_y[1]));
    ++c->stats.kernels;
    LX_CUDA(cudaGetLastError());
  } else if (df) {
    df_output_kernel<<<aux_blocks(c), kThreadsPerBlock, 0, c->stream>>>(
        c->n, c->d_pdf, base, out, c->d_state, static_cast<const float2*>(c->d_y[0]),
        static_cast<const float2*>(c->d_y[1]));
    ++c->stats.kernels;
    LX_CUDA(cudaGetLastError());
  }
  return LX_OK;
}

lx_status begin_call(lx_ctx* c) {
  c->ev_used = 0;
  c->prep_u = nullptr;
  reset_call_kernel<<<1, 1, 0, c->stream>>>(c->d_state, c->d_ticket);
  ++c->stats.kernels;
  LX_CUDA(cudaGetLastError());
  return LX_OK;
}

// Synchronise, fold the loop timings into the statistics, fetch the state.
lx_status end_call(lx_ctx* c) {
  LX_CUDA(cudaMemcpyAsync(c->h_state, c->d_state, sizeof(LoopState), cudaMemcpyDeviceToHost, c->stream));
  LX_CUDA(cudaStreamSynchronize(c->stream));
  for (int k = 0; k + 1 < c->ev_used; k += 2) {
    float ms = 0.f;
    LX_CUDA(cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]));
    c->stats.loop_ms += ms;
    c->stats.loop_launches += 1;
  }
  c->stats.loop_iterations += c->h_state->iters_total;
  c->stats.kernels += c->graph_iter_launches_pending ? c->h_state->launches : 0;
  c->graph_iter_launches_pending = 0;
  c->ev_used = 0;
  return LX_OK;
}

bool valid_problem(const lx_problem* p) {
  if (!p) return false;
  if (p->nx < 1 || p->ny < 1) return false;
  if ((long long)p->nx * p->ny > (1LL << 31)) return false;
  if (p->kind != LX_ADVDIFF && p->kind != LX_BURGERS && p->kind != LX_ADVDIFF_UP3 && p->kind != LX_BURGERS_UP3)
    return false;
  if (p->precision == LX_DF64 && p->kind == LX_BURGERS_UP3 && p->nx % 128 != 0) return false;
  if (p->precision != LX_FP64 && p->precision != LX_MIXED && p->precision != LX_DF64) return false;
  if (p->precision == LX_DF64 && p->kind == LX_BURGERS && p->nx % 128 != 0) return false;
  if (!std::isfinite(p->nu) || !std::isfinite(p->a)) return false;
  return true;
}

}  // namespace

extern "C" {

const char* lx_status_str(lx_status s) {
  switch (s) {
    case LX_OK: return "ok";
    case LX_E_INVAL: return "invalid argument";
    case LX_E_NOMEM: return "out of memory";
    case LX_E_CUDA: return "CUDA error";
    case LX_E_NOCONV: return "Leja series did not converge";
    case LX_E_NONFINITE: return "non-finite value";
    case LX_E_TIMEOUT: return "device wait timed out";
    case LX_E_CALLBACK: return "right-hand side function failed";
  }
  return "unknown status";
}

const char* lx_last_cuda_error(void) { return g_last_cuda_error.c_str(); }

void leja_destroy(lx_ctx* c) {
  if (!c) return;
  for (auto& L : c->loop) destroy_graph(L);
  for (auto& row : c->vloop)
    for (auto& L : row) destroy_graph(L);
  cudaFree(c->d_vargs);
  cudaFree(c->d_vcoef);
  cudaFree(c->d_vfix);
  for (int j = 1; j < kMaxVertical; ++j) cudaFree(c->d_pdfv[j]);
  for (auto& S : c->coef) {
    if (S.dev) cudaFree(S.dev);
    if (S.host) cudaFreeHost(S.host);
  }
  cudaFree(c->d_xi);
  cudaFree(c->d_y[0]);
  cudaFree(c->d_y[1]);
  cudaFree(c->d_f);
  cudaFree(c->d_s);
  cudaFree(c->d_uf);
  cudaFree(c->d_sf);
  cudaFree(c->d_p3);
  for (auto* p : c->d_ep) cudaFree(p);
  cudaFree(c->d_pw[0]);
  cudaFree(c->d_pw[1]);
  for (auto* p : c->d_io) cudaFree(p);
  cudaFree(c->d_pdf);
  cudaFree(c->d_tune);
  cudaFree(c->d_bq);
  cudaFree(c->d_br);
  cudaFree(c->d_partials);
  cudaFree(c->d_ticket);
  cudaFree(c->d_state);
  cudaFree(c->d_args);
  if (c->h_state) cudaFreeHost(c->h_state);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : c->ev_pow)
    if (e) cudaEventDestroy(e);
  delete c;
}

lx_status leja_setup(const lx_problem* prob, int integrator, int max_leja, void* cuda_stream, lx_ctx** out) {
  if (!out) return LX_E_INVAL;
  *out = nullptr;
  if (!valid_problem(prob)) return LX_E_INVAL;
  if (integrator != LX_ROS_EU && integrator != LX_EXPRB32 && integrator != LX_EPIRK4S3A) return LX_E_INVAL;
  if (max_leja == 0) max_leja = 1000;
  if (max_leja < 16 || max_leja > 4096) return LX_E_INVAL;
  lx_ctx* c = new lx_ctx();
  c->prob = *prob;
  c->integrator = integrator;
  c->K = max_leja;
  c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  c->n = (long long)prob->nx * prob->ny;
  const double dx = 1.0 / prob->nx, dy = 1.0 / prob->ny;
  c->geo = Geo{prob->nx, prob->ny, c->n, 1.0 / (dx * dx), 1.0 / (dy * dy), 1.0 / (2 * dx), 1.0 / (2 * dy)};
  {
    // upwind operators on [-1,1)^2: spacing 2/n
    const double ux = 2.0 / prob->nx, uy = 2.0 / prob->ny;
    c->up3 = Up3Op{prob->nx, prob->ny, c->n, prob->a >= 0.0 ? 1 : -1, prob->nu / (ux * ux), prob->nu / (uy * uy),
                   std::fabs(prob->a) / (6.0 * ux), std::fabs(prob->a) / (6.0 * uy)};
  }
  auto fail = [&](lx_status s) {
    leja_destroy(c);
    return s;
  };
  if (!cuda_ok(cudaGetDevice(&c->device), "cudaGetDevice")) return fail(LX_E_CUDA);
  if (!cuda_ok(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device), "sm count"))
    return fail(LX_E_CUDA);
  std::vector<double> xi(c->K);
  if (leja_points(c->K, xi.data()) != LX_OK) return fail(LX_E_INVAL);

  const size_t nb = sizeof(double) * (size_t)c->n;
  auto dmalloc = [&](void** p, size_t bytes) { return cuda_ok(cudaMalloc(p, bytes), "cudaMalloc"); };
  if (!dmalloc((void**)&c->d_xi, sizeof(double) * c->K)) return fail(LX_E_NOMEM);
  for (auto& S : c->coef) {
    if (!dmalloc((void**)&S.dev, sizeof(double) * c->K)) return fail(LX_E_NOMEM);
    if (!cuda_ok(cudaMallocHost((void**)&S.host, sizeof(double) * c->K), "cudaMallocHost")) return fail(LX_E_NOMEM);
  }
  if (!dmalloc(&c->d_y[0], basis_bytes(c)) || !dmalloc(&c->d_y[1], basis_bytes(c))) return fail(LX_E_NOMEM);
  if (!dmalloc((void**)&c->d_f, nb) || !dmalloc((void**)&c->d_s, nb)) return fail(LX_E_NOMEM);
  if (integrator != LX_ROS_EU && !dmalloc((void**)&c->d_p3, nb)) return fail(LX_E_NOMEM);
  if (integrator == LX_EPIRK4S3A)
    for (auto*& p : c->d_ep)
      if (!dmalloc((void**)&p, nb)) return fail(LX_E_NOMEM);
  if (prob->precision == LX_DF64 && !dmalloc((void**)&c->d_pdf, sizeof(float2) * (size_t)c->n))
    return fail(LX_E_NOMEM);
  if (prob->precision == LX_MIXED && prob->kind == LX_BURGERS &&
      (!dmalloc((void**)&c->d_uf, sizeof(float) * (size_t)c->n) ||
       !dmalloc((void**)&c->d_sf, sizeof(float) * (size_t)c->n)))
    return fail(LX_E_NOMEM);
  if (prob->precision == LX_DF64 && (prob->kind == LX_BURGERS || prob->kind == LX_BURGERS_UP3) &&
      (!dmalloc((void**)&c->d_bq, sizeof(float2) * (size_t)c->n) ||
       !dmalloc((void**)&c->d_br, sizeof(float2) * (size_t)c->n)))
    return fail(LX_E_NOMEM);
  {
    const char* env = std::getenv("LEXGB_STREAM_LOOP");
    c->stream_loop = (env && env[0] == '1') ? 1 : 0;
  }
  c->partials_cap = 64 * c->sm_count;
  // up to 1 + kMaxVertical partial sums per block (vertical loops; the
  // two-step kernel uses four)
  if (!dmalloc((void**)&c->d_partials, sizeof(double) * (1 + kMaxVertical) * c->partials_cap))
    return fail(LX_E_NOMEM);
  if (!dmalloc((void**)&c->d_ticket, sizeof(unsigned int))) return fail(LX_E_NOMEM);
  if (!dmalloc((void**)&c->d_state, sizeof(LoopState))) return fail(LX_E_NOMEM);
  if (!dmalloc((void**)&c->d_args, sizeof(LoopArgs))) return fail(LX_E_NOMEM);
  if (!cuda_ok(cudaMallocHost((void**)&c->h_state, sizeof(LoopState)), "cudaMallocHost")) return fail(LX_E_NOMEM);
  for (auto& e : c->ev)
    if (!cuda_ok(cudaEventCreate(&e), "cudaEventCreate")) return fail(LX_E_CUDA);
  for (auto& e : c->ev_pow)
    if (!cuda_ok(cudaEventCreate(&e), "cudaEventCreate")) return fail(LX_E_CUDA);
  if (!cuda_ok(cudaMemsetAsync(c->d_ticket, 0, sizeof(unsigned int), c->stream), "memset") ||
      !cuda_ok(cudaMemsetAsync(c->d_state, 0, sizeof(LoopState), c->stream), "memset") ||
      !cuda_ok(cudaMemcpyAsync(c->d_xi, xi.data(), sizeof(double) * c->K, cudaMemcpyHostToDevice, c->stream),
               "upload xi"))
    return fail(LX_E_CUDA);
  // the auxiliary kernels use one resident wave of the aux kernels' blocks
  c->aux_grid = 4 * c->sm_count;
  for (int v = 0; v < kNumVariants; ++v) {
    if (v == kVec2 && prob->nx % (32 * wide_vec(c)) != 0) continue;
    if (candidates(prob->kind, prob->precision, v).empty()) continue;  // built on demand (and refused) later
    lx_status s = ensure_graph(c, v);
    if (s != LX_OK) return fail(s);
  }
  if (!cuda_ok(cudaStreamSynchronize(c->stream), "setup sync")) return fail(LX_E_CUDA);
  *out = c;
  return LX_OK;
}

// Grid of the pipelined upwind power pass: one balanced row range
// (at least four rows) per warp, at most the resident blocks of one wave.
lx_status size_pow_pipe_grid(lx_ctx* c) {
  const bool b = c->prob.kind == LX_BURGERS_UP3;
  const void* f = b ? up3z_power_kernel() : reinterpret_cast<const void*>(&power_pass_df_pipe_up3_kernel<3>);
  const int smem = b ? up3z_smem_bytes<5>() : kUpSmemBytes;
  LX_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int per_sm = 0;
  LX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kPipeThreads, smem));
  per_sm = std::max(per_sm, 1);
  const long long units = ((long long)(c->prob.nx / kPipeRow) * c->prob.ny + 3) / 4;
  const int want = (int)std::min<long long>((units + kPipeWarps - 1) / kPipeWarps, 1 << 30);
  c->pow_pipe_grid = std::max(1, std::min({want, per_sm * c->sm_count, c->partials_cap}));
  return LX_OK;
}

lx_status power_bound(lx_ctx* c, const double* u, const double* v0, int max_iters, double* rho, int* iters) {
  if (!c || !v0 || !rho || max_iters < 1 || max_iters > kMaxPower) return LX_E_INVAL;
  if (is_burgers(c->prob.kind) && !u) return LX_E_INVAL;
  const long long nb = sizeof(double) * c->n;
  if (!c->d_pw[0]) {
    if (!cuda_ok(cudaMalloc((void**)&c->d_pw[0], nb), "cudaMalloc") ||
        !cuda_ok(cudaMalloc((void**)&c->d_pw[1], nb), "cudaMalloc"))
      return LX_E_NOMEM;
  }
  const int G = aux_blocks(c);
  const lx_problem& P = c->prob;
  LX_CUDA(cudaEventRecord(c->ev_pow[0], c->stream));
  // float-float Burgers: the point weights straight from u on the FP32 pipe
  // (no FP64 gradient)
  const bool dfw = P.kind == LX_BURGERS && P.precision == LX_DF64 && P.nx % kPipeRow == 0 && aligned16(u);
  if (P.kind == LX_BURGERS && !dfw) {
    rhs_kernel<1><<<G, kThreadsPerBlock, 0, c->stream>>>(c->geo, P.nu, 0.0, 0.0, u, nullptr, c->d_s);
    ++c->stats.kernels;
    LX_CUDA(cudaGetLastError());
  }
  power_start_kernel<<<G, kThreadsPerBlock, 0, c->stream>>>(c->n, v0, max_iters, c->d_partials, c->d_ticket,
                                                             c->d_state);
  ++c->stats.kernels;
  LX_CUDA(cudaGetLastError());
  const bool dfp = P.precision == LX_DF64 && !is_up3(P.kind);
  const bool dfu = P.precision == LX_DF64 && is_up3(P.kind);  // float-float passes of the upwind kinds
  if (dfu && P.kind == LX_BURGERS_UP3) {
    // q = u |a| / (6 dx) as float pairs for the point weights of J(u)
    c->prep_u = nullptr;
    up3_df_prep_kernel<<<G, kThreadsPerBlock, 0, c->stream>>>(c->n, u, c->up3.gx, c->d_bq);
    ++c->stats.kernels;
    LX_CUDA(cudaGetLastError());
  }
  PowWeights PW;
  std::memset(&PW, 0, sizeof(PW));
  if (dfp) {
    const double dx = 1.0 / P.nx, dy = 1.0 / P.ny;
    const double nx2 = P.nu / (dx * dx), ny2 = P.nu / (dy * dy);
    if (P.kind == LX_ADVDIFF) {
      const double wd[5] = {nx2 + P.a / (2 * dx), nx2 - P.a / (2 * dx), ny2 + P.a / (2 * dy), ny2 - P.a / (2 * dy),
                            -2.0 * nx2 - 2.0 * ny2};
      for (int k = 0; k < 5; ++k) {
        PW.w[2 * k] = (float)wd[k];
        PW.w[2 * k + 1] = (float)(wd[k] - (double)PW.w[2 * k]);
      }
    } else {
      const double blv[3] = {nx2, ny2, dx / dy};
      for (int k = 0; k < 3; ++k) {
        PW.bl[2 * k] = (float)blv[k];
        PW.bl[2 * k + 1] = (float)(blv[k] - (double)PW.bl[2 * k]);
      }
      // q = u / (2 dx), r = -2 nu/dx^2 - 2 nu/dy^2 - (u_x + u_y)
      c->prep_u = nullptr;
      if (dfw)
        LX_CUDA(burgers_weights_df(P.nx, P.ny, u, 1.0 / (2 * dx), 1.0, -2.0 * nx2 - 2.0 * ny2, dx, dy, c->d_bq,
                                   c->d_br, c->sm_count, c->stream));
      else
        burgers_df_prep_kernel<<<G, kThreadsPerBlock, 0, c->stream>>>(c->n, u, c->d_s, 1.0 / (2 * dx), 1.0,
                                                                       -2.0 * nx2 - 2.0 * ny2, c->d_bq, c->d_br);
      ++c->stats.kernels;
      LX_CUDA(cudaGetLastError());
    }
  }
  for (int k = 1; k <= max_iters; ++k) {
    const double* in = (k == 1) ? v0 : c->d_pw[(k - 2) & 1];
    double* outv = c->d_pw[(k - 1) & 1];
    if (dfp) {
      float2* wf = reinterpret_cast<float2*>(outv);
      if (P.nx % kPipeRow == 0 && aligned16(in)) {
        // row-strip form with a cp.async ring
        constexpr int kPowStages = 5;
        const bool bk = P.kind != LX_ADVDIFF;
        // square Burgers grids: the lean pass (paired stencil, same arguments)
        const bool bsq = bk && P.nx == P.ny;
        const void* fn = bsq ? df2bx_power_kernel()
                             : (bk ? reinterpret_cast<const void*>(&power_pass_df_rows_kernel<1, kPowStages>)
                                   : reinterpret_cast<const void*>(&power_pass_df_rows_kernel<0, kPowStages>));
        const int smem = bk ? pow_rows_smem_bytes<1, kPowStages>() : pow_rows_smem_bytes<0, kPowStages>();
        LX_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        int per_sm = 0;
        LX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPipeThreads, smem));
        const long long lines = (long long)(P.nx / kPipeRow) * P.ny;
        const int GP = (int)std::max<long long>(1, std::min<long long>((lines / 4 + kPipeWarps - 1) / kPipeWarps,
                                                                         (long long)std::max(per_sm, 1) *
                                                                             c->sm_count));
        if (bsq) {
          int nx = P.nx, ny = P.ny, vin_double = k == 1 ? 1 : 0;
          long long n = c->n;
          const void* vin = in;
          float2* wout = wf;
          const float2* qq = c->d_bq;
          const float2* rr = c->d_br;
          double* partials = c->d_partials;
          unsigned int* ticket = c->d_ticket;
          LoopState* stp = c->d_state;
          void* args[] = {&nx, &ny, &n, &vin, &vin_double, &wout, &qq, &rr, &PW, &partials, &ticket, &stp};
          LX_CUDA(cudaLaunchKernel(fn, dim3(GP), dim3(kPipeThreads), args, (size_t)smem, c->stream));
        } else if (bk)
          power_pass_df_rows_kernel<1, kPowStages><<<GP, kPipeThreads, smem, c->stream>>>(
              P.nx, P.ny, c->n, in, k == 1 ? 1 : 0, wf, c->d_bq, c->d_br, PW, c->d_partials, c->d_ticket, c->d_state);
        else
          power_pass_df_rows_kernel<0, kPowStages><<<GP, kPipeThreads, smem, c->stream>>>(
              P.nx, P.ny, c->n, in, k == 1 ? 1 : 0, wf, nullptr, nullptr, PW, c->d_partials, c->d_ticket,
              c->d_state);
      } else if (P.kind == LX_ADVDIFF) {
        power_pass_df_kernel<0><<<G, kThreadsPerBlock, 0, c->stream>>>(c->geo, in, k == 1 ? 1 : 0, wf, nullptr,
                                                                       nullptr, PW, c->d_partials, c->d_ticket,
                                                                       c->d_state);
      } else {
        power_pass_df_kernel<1><<<G, kThreadsPerBlock, 0, c->stream>>>(c->geo, in, k == 1 ? 1 : 0, wf, c->d_bq,
                                                                       c->d_br, PW, c->d_partials, c->d_ticket,
                                                                       c->d_state);
      }
      ++c->stats.kernels;
      LX_CUDA(cudaGetLastError());
      continue;
    }
    if (dfu) {
      float2* wf = reinterpret_cast<float2*>(outv);
      const bool pipe = P.nx % kPipeRow == 0 && aligned16(in);
      if (pipe && c->pow_pipe_grid == 0) {
        lx_status gs = size_pow_pipe_grid(c);
        if (gs != LX_OK) return gs;
      }
      if (P.kind == LX_ADVDIFF_UP3 && pipe) {
        power_pass_df_pipe_up3_kernel<3><<<c->pow_pipe_grid, kPipeThreads, kUpSmemBytes, c->stream>>>(
            c->up3, in, k == 1 ? 1 : 0, wf, c->d_partials, c->d_ticket, c->d_state);
      } else if (P.kind == LX_ADVDIFF_UP3) {
        power_pass_df_up3_kernel<false><<<G, kThreadsPerBlock, 0, c->stream>>>(
            c->up3, in, k == 1 ? 1 : 0, wf, nullptr, c->d_partials, c->d_ticket, c->d_state);
      } else if (pipe) {
        // pipelined product form
        Up3Op op = c->up3;
        const void* vin = in;
        int vin_double = k == 1 ? 1 : 0;
        float2* wout = wf;
        const float2* q = c->d_bq;
        double* partials = c->d_partials;
        unsigned int* ticket = c->d_ticket;
        LoopState* st = c->d_state;
        void* args[] = {&op, &vin, &vin_double, &wout, &q, &partials, &ticket, &st};
        LX_CUDA(cudaLaunchKernel(up3z_power_kernel(), dim3(c->pow_pipe_grid), dim3(kPipeThreads), args,
                                 up3z_smem_bytes<5>(), c->stream));
      } else {
        power_pass_df_up3_kernel<true><<<G, kThreadsPerBlock, 0, c->stream>>>(
            c->up3, in, k == 1 ? 1 : 0, wf, c->d_bq, c->d_partials, c->d_ticket, c->d_state);
      }
      ++c->stats.kernels;
      LX_CUDA(cudaGetLastError());
      continue;
    }
    if (P.kind == LX_ADVDIFF_UP3)
      power_pass_up3_kernel<false><<<G, kThreadsPerBlock, 0, c->stream>>>(c->up3, nullptr, in, outv, c->d_partials,
                                                                          c->d_ticket, c->d_state);
    else if (P.kind == LX_BURGERS_UP3)
      power_pass_up3_kernel<true><<<G, kThreadsPerBlock, 0, c->stream>>>(c->up3, u, in, outv, c->d_partials,
                                                                         c->d_ticket, c->d_state);
    else if (P.kind == LX_ADVDIFF)
      power_pass_kernel<0><<<G, kThreadsPerBlock, 0, c->stream>>>(c->geo, P.nu, P.a, nullptr, nullptr, in, outv,
                                                                  c->d_partials, c->d_ticket, c->d_state);
    else
      power_pass_kernel<1><<<G, kThreadsPerBlock, 0, c->stream>>>(c->geo, P.nu, 0.0, u, c->d_s, in, outv,
                                                                  c->d_partials, c->d_ticket, c->d_state);
    ++c->stats.kernels;
    LX_CUDA(cudaGetLastError());
  }
  LX_CUDA(cudaEventRecord(c->ev_pow[1], c->stream));
  LX_CUDA(cudaMemcpyAsync(c->h_state, c->d_state, sizeof(LoopState), cudaMemcpyDeviceToHost, c->stream));
  LX_CUDA(cudaStreamSynchronize(c->stream));
  float ms = 0.f;
  LX_CUDA(cudaEventElapsedTime(&ms, c->ev_pow[0], c->ev_pow[1]));
  c->stats.power_ms += ms;
  *rho = c->h_state->rho;
  if (iters) *iters = c->h_state->pk;
  return (lx_status)c->h_state->pstatus;
}

lx_status phi_l_apply(lx_ctx* c, int l, const double* u, const double* w, double* out, double cc, double gamma,
                      double h, double rtol, double atol, int* iters) {
  if (!c || !w || !out || l < 0 || l > 8 || !(gamma != 0.0) || !std::isfinite(h) || !std::isfinite(cc) ||
      !std::isfinite(gamma) || !(rtol >= 0.0) || !(atol >= 0.0))
    return LX_E_INVAL;
  if ((const void*)out == (const void*)w || (u && (const void*)out == (const void*)u)) return LX_E_INVAL;
  if (is_burgers(c->prob.kind) && !u) return LX_E_INVAL;
  lx_status st = begin_call(c);
  if (st != LX_OK) return st;
  if (c->prob.kind == LX_BURGERS) {
    rhs_kernel<1><<<aux_blocks(c), kThreadsPerBlock, 0, c->stream>>>(c->geo, c->prob.nu, 0.0, 0.0, u, nullptr,
                                                                       c->d_s);
    ++c->stats.kernels;
    LX_CUDA(cudaGetLastError());
  }
  st = launch_loop(c, 0, l, u, w, out, cc, gamma, h, rtol, atol);
  if (st != LX_OK) return st;
  st = end_call(c);
  if (st != LX_OK) return st;
  if (iters) *iters = c->h_state->iters_total;
  return (lx_status)c->h_state->status_total;
}

lx_status phi_l_apply_vertical(lx_ctx* c, int l, int nc, const double* alpha, const double* u, const double* w,
                               double* const* out, double cc, double gamma, double h, double rtol, double atol,
                               int* iters) {
  if (!c || !w || !out || !alpha || nc < 1 || nc > kMaxVertical || l < 0 || l > 8 || !(gamma != 0.0) ||
      !std::isfinite(h) || !std::isfinite(cc) || !std::isfinite(gamma) || !(rtol >= 0.0) || !(atol >= 0.0))
    return LX_E_INVAL;
  for (int j = 0; j < nc; ++j) {
    if (!out[j] || !(alpha[j] > 0.0) || !std::isfinite(alpha[j])) return LX_E_INVAL;
    if ((const void*)out[j] == (const void*)w || (u && (const void*)out[j] == (const void*)u)) return LX_E_INVAL;
    for (int k = 0; k < j; ++k)
      if (out[k] == out[j]) return LX_E_INVAL;
  }
  const lx_problem& P = c->prob;
  if (is_burgers(P.kind) && !u) return LX_E_INVAL;
  const bool df = P.precision == LX_DF64;
  const bool up = is_up3(P.kind);  // point-wise kernels: no layout requirement
  bool wide;
  if (up) {
    wide = false;
  } else if (df) {
    if (P.nx % kPipeRow != 0 || !aligned16(w)) {
      set_last_error("vertical float-float interpolation needs nx % 128 == 0 and a 16-byte aligned w");
      return LX_E_INVAL;
    }
    wide = true;
  } else {
    wide = P.nx % 64 == 0 && aligned16(w) && aligned16(c->d_y[0]) && aligned16(c->d_y[1]);
    for (int j = 0; j < nc; ++j) wide = wide && aligned16(out[j]);
  }
  // float-float diffusion-advection: two Leja iterations per pass
  const bool two = df && (P.kind == LX_ADVDIFF || (P.kind == LX_BURGERS && nc <= 3));
  int smem2 = 0;
  const void* fn = !two ? vertical_kernel(P.kind, P.precision, wide, nc)
                        : (P.kind == LX_ADVDIFF ? vertical2x_kernel(nc, &smem2) : vertical2bx_kernel(nc, &smem2));
  if (!fn) return LX_E_INVAL;
  // lazily allocated vertical buffers
  if (!c->d_vargs && !cuda_ok(cudaMalloc((void**)&c->d_vargs, sizeof(VertArgs)), "cudaMalloc")) return LX_E_NOMEM;
  if (!c->d_vcoef &&
      !cuda_ok(cudaMalloc((void**)&c->d_vcoef, sizeof(double) * kMaxVertical * (size_t)c->K), "cudaMalloc"))
    return LX_E_NOMEM;
  if (two && !c->d_vfix && !cuda_ok(cudaMalloc((void**)&c->d_vfix, sizeof(double) * kMaxVertical), "cudaMalloc"))
    return LX_E_NOMEM;
  c->d_pdfv[0] = c->d_pdf;
  for (int j = 1; df && j < nc; ++j)
    if (!c->d_pdfv[j] && !cuda_ok(cudaMalloc((void**)&c->d_pdfv[j], sizeof(float2) * (size_t)c->n), "cudaMalloc"))
      return LX_E_NOMEM;
  lx_status st = begin_call(c);
  if (st != LX_OK) return st;
  if (P.kind == LX_BURGERS) {
    rhs_kernel<1><<<aux_blocks(c), kThreadsPerBlock, 0, c->stream>>>(c->geo, P.nu, 0.0, 0.0, u, nullptr, c->d_s);
    ++c->stats.kernels;
    LX_CUDA(cudaGetLastError());
  }
  // divided differences of phi_l(alpha_j h (c + gamma xi)) on a common table
  // long enough for the largest alpha_j
  int count = 2;
  for (int j = 0; j < nc; ++j) count = std::max(count, leja_coeff_count(alpha[j] * h, cc, gamma, c->K));
  std::vector<double> xi(count), dh((size_t)nc * count);
  leja_points(count, xi.data());
  for (int j = 0; j < nc; ++j) {
    const int cs = leja_coeffs(l, alpha[j] * h, cc, gamma, xi.data(), count, dh.data() + (size_t)j * count);
    if (cs != LX_OK) return (lx_status)cs;
    LX_CUDA(cudaMemcpyAsync(c->d_vcoef + (size_t)j * c->K, dh.data() + (size_t)j * count, sizeof(double) * count,
                            cudaMemcpyHostToDevice, c->stream));
  }
  LX_CUDA(cudaStreamSynchronize(c->stream));  // dh is host memory of this frame
  const int variant = wide ? kVec2 : kVec1;
  const int H = two ? 0 : ((df && !up) ? 8 : c->strip_h);
  LoopGraph& L = c->vloop[variant][nc - 1];
  if (!L.built || L.cand.func != fn) {
    destroy_graph(L);
    const Cand k = two ? Cand{fn, kPipeThreads, smem2, 4,
                              P.kind == LX_ADVDIFF ? "leja_iter_df_vertical2x" : "leja_iter_df_vertical2bx", 2, 0}
                       : Cand{fn, kThreadsPerBlock, 0, (df && !up) ? 4 : (wide ? 2 : 1), "leja_iter_vertical"};
    int grid = 0;
    const int gs = grid_for(c, k, H, &grid);
    if (gs != LX_OK) return (lx_status)gs;
    L.cand = k;
    L.strip_h = H;
    L.grid = grid;
    L.unroll = c->graph_unroll;
    LX_CUDA(cudaGraphCreate(&L.graph, 0));
    cudaGraphConditionalHandle cond;
    LX_CUDA(cudaGraphConditionalHandleCreate(&cond, L.graph, 1, cudaGraphCondAssignDefault));
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    std::memset(cp_raw, 0, sizeof(cp_raw));
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    LX_CUDA(cudaGraphAddNode(&cnode, L.graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    const LoopArgs* args = c->d_args;
    const VertArgs* vargs = c->d_vargs;
    LoopState* stp = c->d_state;
    double* partials = c->d_partials;
    unsigned int* ticket = c->d_ticket;
    void* kargs[] = {(void*)&args, (void*)&vargs, (void*)&stp, (void*)&partials, (void*)&ticket, (void*)&cond};
    cudaKernelNodeParams kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.func = const_cast<void*>(fn);
    kp.gridDim = dim3(L.grid);
    kp.blockDim = dim3(k.threads);
    kp.sharedMemBytes = (unsigned)k.smem;
    kp.kernelParams = kargs;
    cudaGraphNode_t prev = nullptr;
    for (int q = 0; q < L.unroll; ++q) {
      cudaGraphNode_t knode;
      LX_CUDA(cudaGraphAddKernelNode(&knode, body, prev ? &prev : nullptr, prev ? 1 : 0, &kp));
      prev = knode;
    }
    LX_CUDA(cudaGraphInstantiate(&L.exec, L.graph, 0));
    L.built = true;
  }
  st = prepare_loop(c, H, count - 1, c->d_vcoef, u, w, out[0], cc, gamma, rtol, atol, false);
  if (st != LX_OK) return st;
  VertArgs V;
  std::memset(&V, 0, sizeof(V));
  V.np = nc;
  for (int j = 0; j < nc; ++j) {
    V.d[j] = c->d_vcoef + (size_t)j * c->K;
    V.p[j] = out[j];
    V.pdf[j] = c->d_pdfv[j];
  }
  V.fixd = c->d_vfix;
  LX_CUDA(upload_vertical_args(V, c->d_vargs, c->stream));
  ++c->stats.kernels;
  if (c->ev_used + 2 > 8) return LX_E_INVAL;
  LX_CUDA(cudaEventRecord(c->ev[c->ev_used], c->stream));
  if (!c->stream_loop) {
    LX_CUDA(cudaGraphLaunch(L.exec, c->stream));
    c->graph_iter_launches_pending = 1;
  } else {
    const LoopArgs* args = c->d_args;
    const VertArgs* vargs = c->d_vargs;
    LoopState* stp = c->d_state;
    double* partials = c->d_partials;
    unsigned int* ticket = c->d_ticket;
    cudaGraphConditionalHandle cond = 0;
    void* kargs[] = {(void*)&args, (void*)&vargs, (void*)&stp, (void*)&partials, (void*)&ticket, (void*)&cond};
    for (int it = 0; it < count - 1; it += 8) {
      for (int q = 0; q < 8; ++q)
        LX_CUDA(cudaLaunchKernel(fn, dim3(L.grid), dim3(L.cand.threads), kargs, (size_t)L.cand.smem, c->stream));
      c->stats.kernels += 8;
      LX_CUDA(cudaMemcpyAsync(c->h_state, c->d_state, sizeof(LoopState), cudaMemcpyDeviceToHost, c->stream));
      LX_CUDA(cudaStreamSynchronize(c->stream));
      if (c->h_state->done) break;
    }
  }
  LX_CUDA(cudaEventRecord(c->ev[c->ev_used + 1], c->stream));
  c->ev_used += 2;
  if (df) {
    for (int j = 0; j < nc; ++j) {
      if (two) {
        // this polynomial's odd-stop coefficient into the loop state
        LX_CUDA(select_vertical_fix(c->d_state, c->d_vfix, j, c->stream));
        ++c->stats.kernels;
      }
      if (c->n % 2 == 0 && aligned16(out[j])) {
        const long long n2 = c->n / 2;
        const int G2 = (int)std::max<long long>(
            1, std::min<long long>((n2 + kThreadsPerBlock - 1) / kThreadsPerBlock, 8LL * c->sm_count));
        df_output2_kernel<<<G2, kThreadsPerBlock, 0, c->stream>>>(
            n2, reinterpret_cast<const float4*>(c->d_pdfv[j]), nullptr, reinterpret_cast<double2*>(out[j]),
            c->d_state, static_cast<const float4*>(c->d_y[0]), static_cast<const float4*>(c->d_y[1]));
      } else {
        df_output_kernel<<<aux_blocks(c), kThreadsPerBlock, 0, c->stream>>>(
            c->n, c->d_pdfv[j], nullptr, out[j], c->d_state, static_cast<const float2*>(c->d_y[0]),
            static_cast<const float2*>(c->d_y[1]));
      }
      ++c->stats.kernels;
      LX_CUDA(cudaGetLastError());
    }
  }
  st = end_call(c);
  if (st != LX_OK) return st;
  if (iters) *iters = c->h_state->iters_total;
  return (lx_status)c->h_state->status_total;
}

// EPIRK4s3A (the fourth-order exponential integrator of the paper's Table 2;
// its phi_1 stages by vertical interpolation, Sec. 2.3).  Coefficients: the
// ones the stiff order conditions sum b_i(z) c_i^2 = 2 phi_3(z) and
// sum b_i(z) c_i^3 = 6 phi_4(z) fix for the nodes c2 = 1/2, c3 = 2/3:
//   U_i = u + c_i P_i,  P_i = phi_1(c_i h J) h f(u),  R_i = h (F(U_i) - F(u)),
//   W3 = 32 R_2 - 27/2 R_3,  W4 = -144 R_2 + 81 R_3,
//   u_low  = u + P_1 + phi_3(h J) W3          (embedded, third order)
//   u_high = u_low + phi_4(h J) W4            (fourth order)
//   err = ||phi_4(h J) W4||.
// The engine's remainder kernels evaluate R_i from U_i - u (exactly
// -h p (p_x + p_y) for the quadratic central Burgers term, 0 for the
// linear operators).  The loops run through the public entry points (one
// vertical phi_1 loop with alpha = 1/2, 2/3, 1; one phi_3 and one phi_4
// loop), each synchronising once.
static lx_status epirk4s3a_step(lx_ctx* c, const double* u, double* u_low, double* u_high, double cc, double gamma,
                                double h, double rtol, double atol, double* err, int* iters) {
  const lx_problem& P = c->prob;
  const int G = aux_blocks(c);
  const bool burg = is_burgers(P.kind);
  // float-float central Burgers: h F(u) and the stage remainders on the FP32
  // pipe (as in expint_step)
  const bool dfb = P.precision == LX_DF64 && P.kind == LX_BURGERS && P.nx % kPipeRow == 0 && aligned16(u) &&
                   (!c->d_src || aligned16(c->d_src));
  const double c2 = 0.5, c3 = 2.0 / 3.0;
  const double b2 = 32.0, b3 = -13.5, e2 = -144.0, e3 = 81.0;
  double* E0 = c->d_ep[0];
  double* E1 = c->d_ep[1];
  double* T = c->d_ep[2];
  // h (f(u) + S) into d_f
  lx_status st = begin_call(c);
  if (st != LX_OK) return st;
  if (P.kind == LX_ADVDIFF)
    rhs_kernel<0><<<G, kThreadsPerBlock, 0, c->stream>>>(c->geo, P.nu, P.a, h, u, c->d_f, c->d_s, c->d_src);
  else if (P.kind == LX_BURGERS && dfb)
    LX_CUDA(burgers_field_df(0, P.nx, P.ny, u, c->d_src, h, P.nu, 1.0 / P.nx, 1.0 / P.ny, c->d_f, c->sm_count,
                             c->stream));
  else if (P.kind == LX_BURGERS)
    rhs_kernel<1><<<G, kThreadsPerBlock, 0, c->stream>>>(c->geo, P.nu, 0.0, h, u, c->d_f, c->d_s, c->d_src);
  else if (P.kind == LX_ADVDIFF_UP3)
    rhs_up3_kernel<false><<<G, kThreadsPerBlock, 0, c->stream>>>(c->up3, h, u, c->d_src, c->d_f);
  else
    rhs_up3_kernel<true><<<G, kThreadsPerBlock, 0, c->stream>>>(c->up3, h, u, c->d_src, c->d_f);
  ++c->stats.kernels;
  LX_CUDA(cudaGetLastError());
  st = end_call(c);
  if (st != LX_OK) return st;
  // P_2, P_3, P_1 from one Newton basis (P_1 into u_low)
  const double alpha[3] = {c2, c3, 1.0};
  double* outs[3] = {E0, E1, u_low};
  int it_v = 0, it3 = 0, it4 = 0;
  lx_status sv = phi_l_apply_vertical(c, 1, 3, alpha, burg ? u : nullptr, c->d_f, outs, cc, gamma, h, rtol, atol,
                                      &it_v);
  if (sv != LX_OK && sv != LX_E_NOCONV) return sv;
  // R_2 into d_f, R_3 into d_p3, then W3 into E0 and W4 into E1
  st = begin_call(c);
  if (st != LX_OK) return st;
  for (int i = 0; i < 2; ++i) {
    double* R = i == 0 ? c->d_f : c->d_p3;
    scale_kernel<<<G, kThreadsPerBlock, 0, c->stream>>>(c->n, alpha[i], i == 0 ? E0 : E1, T);
    if (P.kind == LX_ADVDIFF)
      exprb32_stage_kernel<0><<<G, kThreadsPerBlock, 0, c->stream>>>(c->geo, h, T, R);
    else if (P.kind == LX_BURGERS && dfb && aligned16(T) && aligned16(R))
      LX_CUDA(burgers_field_df(1, P.nx, P.ny, T, nullptr, h, P.nu, 1.0 / P.nx, 1.0 / P.ny, R, c->sm_count,
                               c->stream));
    else if (P.kind == LX_BURGERS)
      exprb32_stage_kernel<1><<<G, kThreadsPerBlock, 0, c->stream>>>(c->geo, h, T, R);
    else if (P.kind == LX_ADVDIFF_UP3)
      exprb32_stage_up3_kernel<false><<<G, kThreadsPerBlock, 0, c->stream>>>(c->up3, h, T, R);
    else
      exprb32_stage_up3_kernel<true><<<G, kThreadsPerBlock, 0, c->stream>>>(c->up3, h, T, R);
    c->stats.kernels += 2;
  }
  epirk_combine_kernel<<<G, kThreadsPerBlock, 0, c->stream>>>(c->n, c->d_f, c->d_p3, b2, b3, e2, e3, E0, E1);
  ++c->stats.kernels;
  LX_CUDA(cudaGetLastError());
  st = end_call(c);
  if (st != LX_OK) return st;
  // q3 = phi_3(h J) W3 into d_f, q4 = phi_4(h J) W4 into d_p3
  lx_status s3 = phi_l_apply(c, 3, burg ? u : nullptr, E0, c->d_f, cc, gamma, h, rtol, atol, &it3);
  if (s3 != LX_OK && s3 != LX_E_NOCONV) return s3;
  lx_status s4 = phi_l_apply(c, 4, burg ? u : nullptr, E1, c->d_p3, cc, gamma, h, rtol, atol, &it4);
  if (s4 != LX_OK && s4 != LX_E_NOCONV) return s4;
  st = begin_call(c);
  if (st != LX_OK) return st;
  epirk_final_kernel<<<G, kThreadsPerBlock, 0, c->stream>>>(c->n, u, u_low, c->d_f, c->d_p3, u_high, c->d_partials,
                                                             c->d_ticket, c->d_state);
  ++c->stats.kernels;
  LX_CUDA(cudaGetLastError());
  st = end_call(c);
  if (st != LX_OK) return st;
  if (err) *err = c->h_state->red;
  if (iters) *iters = it_v + it3 + it4;
  return sv != LX_OK ? sv : (s3 != LX_OK ? s3 : s4);
}

lx_status expint_step(lx_ctx* c, const double* u, double* u_low, double* u_high, double cc, double gamma, double h,
                      double rtol, double atol, double* err, int* iters) {
  if (!c || !u || !u_high || !(gamma != 0.0) || !std::isfinite(h) || !std::isfinite(cc) || !std::isfinite(gamma) ||
      !(rtol >= 0.0) || !(atol >= 0.0))
    return LX_E_INVAL;
  if ((const void*)u_high == (const void*)u) return LX_E_INVAL;
  if (c->integrator != LX_ROS_EU &&
      (!u_low || (const void*)u_low == (const void*)u || (const void*)u_low == (const void*)u_high))
    return LX_E_INVAL;
  if (c->integrator == LX_EPIRK4S3A) return epirk4s3a_step(c, u, u_low, u_high, cc, gamma, h, rtol, atol, err, iters);
  const lx_problem& P = c->prob;
  const int G = aux_blocks(c);
  lx_status st = begin_call(c);
  if (st != LX_OK) return st;
  if (P.precision == LX_DF64 && P.kind == LX_ADVDIFF && c->integrator == LX_ROS_EU) {
    // df64 Rosenbrock-Euler: h A u on the FP32 pipe (recording the input
    // scale), the Leja loop, and u + p fused into the loop's output pass
    const double dx = 1.0 / P.nx, dy = 1.0 / P.ny;
    const double nx2 = P.nu / (dx * dx), ny2 = P.nu / (dy * dy);
    RhsWeights W;
    W.wd[0] = h * (nx2 + P.a / (2 * dx));
    W.wd[1] = h * (nx2 - P.a / (2 * dx));
    W.wd[2] = h * (ny2 + P.a / (2 * dy));
    W.wd[3] = h * (ny2 - P.a / (2 * dy));
    W.wd[4] = h * (-2.0 * nx2 - 2.0 * ny2);
    for (int k = 0; k < 5; ++k) {
      W.wf[2 * k] = (float)W.wd[k];
      W.wf[2 * k + 1] = (float)(W.wd[k] - (double)W.wf[2 * k]);
    }
    if (P.nx % kPipeRow == 0 && aligned16(u) && (!c->d_src || aligned16(c->d_src))) {
      // row-window form with a cp.async ring: at most the resident blocks, at
      // least 4 rows per warp
      int per_sm = 0;
      constexpr int kRhsStages = 6;
      // square grids with equal east/north and west/south weights: the
      // paired stencil
      const bool sq = P.nx == P.ny && W.wd[0] == W.wd[2] && W.wd[1] == W.wd[3];
      const void* rk = sq ? reinterpret_cast<const void*>(&rhs_df_advdiff_ring_kernel<kRhsStages, true>)
                          : reinterpret_cast<const void*>(&rhs_df_advdiff_ring_kernel<kRhsStages, false>);
      LX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rk, kPipeThreads,
                                                            rhs_ring_smem_bytes<kRhsStages>()));
      const long long lines = (long long)(P.nx / kPipeRow) * P.ny;
      const int GR = (int)std::max<long long>(
          1, std::min<long long>((lines / 4 + kPipeWarps - 1) / kPipeWarps,
                                 (long long)std::max(per_sm, 1) * c->sm_count));
      if (sq)
        rhs_df_advdiff_ring_kernel<kRhsStages, true><<<GR, kPipeThreads, rhs_ring_smem_bytes<kRhsStages>(), c->stream>>>(
            P.nx, P.ny, u, W, c->d_f, c->d_state, c->d_src, h);
      else
        rhs_df_advdiff_ring_kernel<kRhsStages, false>
            <<<GR, kPipeThreads, rhs_ring_smem_bytes<kRhsStages>(), c->stream>>>(P.nx, P.ny, u, W, c->d_f,
                                                                                  c->d_state, c->d_src, h);
    } else {
      rhs_df_advdiff_kernel<<<G, kThreadsPerBlock, 0, c->stream>>>(c->geo, u, W, c->d_f, c->d_state, c->d_src, h);
    }
    ++c->stats.kernels;
    LX_CUDA(cudaGetLastError());
    st = launch_loop(c, 0, 1, u, c->d_f, u_high, cc, gamma, h, rtol, atol, u, true);
    if (st != LX_OK) return st;
    st = end_call(c);
    if (st != LX_OK) return st;
    if (err) *err = 0.0;
    if (iters) *iters = c->h_state->iters_total;
    return (lx_status)c->h_state->status_total;
  }
  const bool df_up3 = P.precision == LX_DF64 && is_up3(P.kind);
  // float-float central Burgers: h F(u) and the stage remainder on the FP32
  // pipe (the point weights come from u itself, so u_x + u_y is not needed)
  const bool dfb = P.precision == LX_DF64 && P.kind == LX_BURGERS && P.nx % kPipeRow == 0 && aligned16(u) &&
                   (!c->d_src || aligned16(c->d_src));
  if (df_up3 && c->integrator == LX_ROS_EU) {
    // the same for the upwind operators: h (f(u) + S) on the FP32 pipe, the
    // Leja loop, and u + p in the loop's output pass
    if (P.kind == LX_ADVDIFF_UP3)
      rhs_df_up3_kernel<<<G, kThreadsPerBlock, 0, c->stream>>>(c->up3, h, u, c->d_src, c->d_f, c->d_state);
    else
      burgers_up3_df_kernel<true><<<G, kThreadsPerBlock, 0, c->stream>>>(c->up3, h, u, c->d_src, c->d_f, c->d_state);
    ++c->stats.kernels;
    LX_CUDA(cudaGetLastError());
    st = launch_loop(c, 0, 1, u, c->d_f, u_high, cc, gamma, h, rtol, atol, u, true);
    if (st != LX_OK) return st;
    st = end_call(c);
    if (st != LX_OK) return st;
    if (err) *err = 0.0;
    if (iters) *iters = c->h_state->iters_total;
    return (lx_status)c->h_state->status_total;
  }
  // h f(u) and, for Burgers, u_x + u_y at the linearisation point
  if (P.kind == LX_ADVDIFF)
    rhs_kernel<0><<<G, kThreadsPerBlock, 0, c->stream>>>(c->geo, P.nu, P.a, h, u, c->d_f, c->d_s, c->d_src);
  else if (P.kind == LX_BURGERS && dfb)
    LX_CUDA(burgers_field_df(0, P.nx, P.ny, u, c->d_src, h, P.nu, 1.0 / P.nx, 1.0 / P.ny, c->d_f, c->sm_count,
                             c->stream));
  else if (P.kind == LX_BURGERS)
    rhs_kernel<1><<<G, kThreadsPerBlock, 0, c->stream>>>(c->geo, P.nu, 0.0, h, u, c->d_f, c->d_s, c->d_src);
  else if (df_up3 && P.kind == LX_ADVDIFF_UP3)
    rhs_df_up3_kernel<<<G, kThreadsPerBlock, 0, c->stream>>>(c->up3, h, u, c->d_src, c->d_f, c->d_state);
  else if (df_up3)
    burgers_up3_df_kernel<true><<<G, kThreadsPerBlock, 0, c->stream>>>(c->up3, h, u, c->d_src, c->d_f, c->d_state);
  else if (P.kind == LX_ADVDIFF_UP3)
    rhs_up3_kernel<false><<<G, kThreadsPerBlock, 0, c->stream>>>(c->up3, h, u, c->d_src, c->d_f);
  else
    rhs_up3_kernel<true><<<G, kThreadsPerBlock, 0, c->stream>>>(c->up3, h, u, c->d_src, c->d_f);
  ++c->stats.kernels;
  LX_CUDA(cudaGetLastError());
  if (c->integrator == LX_ROS_EU) {
    // p = phi_1(h J) h f(u) into u_high, then u_high = u + p
    st = launch_loop(c, 0, 1, u, c->d_f, u_high, cc, gamma, h, rtol, atol);
    if (st != LX_OK) return st;
    add_kernel<<<G, kThreadsPerBlock, 0, c->stream>>>(c->n, u, u_high);
    ++c->stats.kernels;
    LX_CUDA(cudaGetLastError());
    st = end_call(c);
    if (st != LX_OK) return st;
    if (err) *err = 0.0;
  } else {
    // p1 = phi_1(h J) h f(u) into u_low (the float-float upwind right-hand
    // sides have recorded the input exponent)
    st = launch_loop(c, 0, 1, u, c->d_f, u_low, cc, gamma, h, rtol, atol, nullptr, df_up3);
    if (st != LX_OK) return st;
    // R = h (F(a) - F(u)) into d_f (u_low keeps p1 until the final pass)
    if (P.kind == LX_ADVDIFF)
      exprb32_stage_kernel<0><<<G, kThreadsPerBlock, 0, c->stream>>>(c->geo, h, u_low, c->d_f);
    else if (P.kind == LX_BURGERS && dfb && aligned16(u_low))
      LX_CUDA(burgers_field_df(1, P.nx, P.ny, u_low, nullptr, h, P.nu, 1.0 / P.nx, 1.0 / P.ny, c->d_f, c->sm_count,
                               c->stream));
    else if (P.kind == LX_BURGERS)
      exprb32_stage_kernel<1><<<G, kThreadsPerBlock, 0, c->stream>>>(c->geo, h, u_low, c->d_f);
    else if (df_up3 && P.kind == LX_BURGERS_UP3)
      burgers_up3_df_kernel<false><<<G, kThreadsPerBlock, 0, c->stream>>>(c->up3, h, u_low, nullptr, c->d_f,
                                                                            c->d_state);
    else if (P.kind == LX_ADVDIFF_UP3)
      exprb32_stage_up3_kernel<false><<<G, kThreadsPerBlock, 0, c->stream>>>(c->up3, h, u_low, c->d_f);
    else
      exprb32_stage_up3_kernel<true><<<G, kThreadsPerBlock, 0, c->stream>>>(c->up3, h, u_low, c->d_f);
    ++c->stats.kernels;
    LX_CUDA(cudaGetLastError());
    // p3 = phi_3(h J) R
    st = launch_loop(c, 1, 3, u, c->d_f, c->d_p3, cc, gamma, h, rtol, atol);
    if (st != LX_OK) return st;
    // a = u + p1 into u_low, u_high = a + 2 p3, err = ||2 p3||
    exprb32_final_kernel<<<G, kThreadsPerBlock, 0, c->stream>>>(c->n, u, u_low, c->d_p3, u_high, c->d_partials,
                                                                 c->d_ticket, c->d_state);
    ++c->stats.kernels;
    LX_CUDA(cudaGetLastError());
    st = end_call(c);
    if (st != LX_OK) return st;
    if (err) *err = c->h_state->red;
  }
  if (iters) *iters = c->h_state->iters_total;
  return (lx_status)c->h_state->status_total;
}

lx_status expint_step_host(lx_ctx* c, const double* u_host, double* u_low_host, double* u_high_host, double cc,
                           double gamma, double h, double rtol, double atol, double* err, int* iters) {
  if (!c || !u_host || !u_high_host) return LX_E_INVAL;
  if (c->integrator != LX_ROS_EU && !u_low_host) return LX_E_INVAL;
  const size_t nb = sizeof(double) * (size_t)c->n;
  for (auto*& p : c->d_io)
    if (!p && !cuda_ok(cudaMalloc((void**)&p, nb), "cudaMalloc")) return LX_E_NOMEM;
  LX_CUDA(cudaMemcpyAsync(c->d_io[0], u_host, nb, cudaMemcpyHostToDevice, c->stream));
  lx_status st = expint_step(c, c->d_io[0], c->d_io[1], c->d_io[2], cc, gamma, h, rtol, atol, err, iters);
  if (st != LX_OK && st != LX_E_NOCONV) return st;
  LX_CUDA(cudaMemcpyAsync(u_high_host, c->d_io[2], nb, cudaMemcpyDeviceToHost, c->stream));
  if (c->integrator != LX_ROS_EU)
    LX_CUDA(cudaMemcpyAsync(u_low_host, c->d_io[1], nb, cudaMemcpyDeviceToHost, c->stream));
  LX_CUDA(cudaStreamSynchronize(c->stream));
  return st;
}

lx_status lx_ctx_stats(lx_ctx* c, lx_stats* out, int reset) {
  if (!c || !out) return LX_E_INVAL;
  *out = c->stats;
  if (reset) c->stats = lx_stats{};
  return LX_OK;
}

lx_status lx_ctx_set_loop_mode(lx_ctx* c, int stream_loop) {
  if (!c || (stream_loop != 0 && stream_loop != 1)) return LX_E_INVAL;
  c->stream_loop = stream_loop;
  return LX_OK;
}

lx_status lx_ctx_set_source(lx_ctx* c, const double* s_dev) {
  if (!c) return LX_E_INVAL;
  c->d_src = s_dev;
  return LX_OK;
}

lx_status lx_ctx_set_graph_unroll(lx_ctx* c, int unroll) {
  if (!c || unroll < 1 || unroll > 8) return LX_E_INVAL;
  c->graph_unroll = unroll;
  for (int v = 0; v < kNumVariants; ++v) {
    LoopGraph& L = c->loop[v];
    if (!L.built) continue;
    const lx_status st = build_loop_graph(c, v, L.cand, L.strip_h);
    if (st != LX_OK) return st;
  }
  return LX_OK;
}

lx_status lx_ctx_kernel_name(lx_ctx* c, char* buf, int len) {
  if (!c || !buf || len <= 0) return LX_E_INVAL;
  const int v = c->loop[kVec2].built ? kVec2 : kVec1;
  std::snprintf(buf, (size_t)len, "%s", c->loop[v].cand.name);
  return LX_OK;
}

int lx_ctx_iters_per_launch(lx_ctx* c) {
  if (!c) return 0;
  const int v = c->loop[kVec2].built ? kVec2 : kVec1;
  return c->loop[v].built ? c->loop[v].cand.ipl : 0;
}

}  // extern "C"

namespace {

std::string tune_key(const lx_ctx* c) {
  cudaDeviceProp prop;
  std::string dev = "unknown";
  if (cudaGetDeviceProperties(&prop, c->device) == cudaSuccess) dev = prop.name;
  for (auto& ch : dev)
    if (ch == ' ' || ch == '\t' || ch == '|') ch = '_';
  std::ostringstream k;
  k << dev << "|sm" << c->sm_count << "|" << c->prob.nx << "x" << c->prob.ny << "|kind" << c->prob.kind << "|prec"
    << c->prob.precision;
  return k.str();
}

// Average time per Leja iteration of candidate k with strip height H on the
// context's own buffers (zero data; stopping disabled).
lx_status tune_time(lx_ctx* c, const Cand& k, int H, int iters, double* us) {
  int grid = 0;
  int gs = grid_for(c, k, H, &grid);
  if (gs != LX_OK) return (lx_status)gs;
  const lx_problem& P = c->prob;
  LoopArgs a;
  std::memset(&a, 0, sizeof(a));
  a.nx = P.nx;
  a.ny = P.ny;
  a.n = c->n;
  a.strip_h = H;
  a.kmax = c->coef[0].count - 1;
  a.w = c->d_f;
  a.y0 = c->d_y[0];
  a.y1 = c->d_y[1];
  a.p = c->d_tune;
  a.u = c->d_f;
  a.s = c->d_s;
  a.uf = c->d_uf;  // (mixed Burgers; zeroed with the other buffers)
  a.sf = c->d_sf;
  a.xi = c->d_xi;
  a.d = c->coef[0].dev;
  a.up = c->up3;
  a.up_c = -20.0;
  a.wxp = a.wxm = a.wyp = a.wym = 0.25;
  a.lx = a.ly = a.gx = a.gy = a.inv_gamma = 0.25;
  a.wc0 = 1.0;
  for (int q = 0; q < 8; ++q) a.wf[q] = (q & 1) ? 0.f : 0.25f;
  for (int q = 0; q < 6; ++q) a.bl[q] = (q & 1) ? 0.f : 0.25f;
  a.pdf = c->d_pdf;
  a.bq = c->d_bq;  // df64 Burgers point weights (allocated for that form only)
  a.br = c->d_br;
  if (P.precision == LX_DF64 && P.kind == LX_BURGERS && (!a.bq || !a.br)) return LX_E_INVAL;
  a.rtol = 0.0;
  a.atol = -1.0;  // never converged: every launch does the full work
  a.use_cond = 0;
  set_loop_args_kernel<<<1, 1, 0, c->stream>>>(a, c->d_args, c->d_state, c->d_ticket);
  ++c->stats.kernels;
  LX_CUDA(cudaGetLastError());
  const LoopArgs* args = c->d_args;
  LoopState* stp = c->d_state;
  double* partials = c->d_partials;
  unsigned int* ticket = c->d_ticket;
  cudaGraphConditionalHandle cond = 0;
  void* kargs[] = {(void*)&args, (void*)&stp, (void*)&partials, (void*)&ticket, (void*)&cond};
  LX_CUDA(cudaLaunchKernel(k.func, dim3(grid), dim3(k.threads), kargs, k.smem, c->stream));  // m = 0 path
  LX_CUDA(cudaEventRecord(c->ev[0], c->stream));
  for (int i = 0; i < iters; ++i)
    LX_CUDA(cudaLaunchKernel(k.func, dim3(grid), dim3(k.threads), kargs, k.smem, c->stream));
  LX_CUDA(cudaEventRecord(c->ev[1], c->stream));
  LX_CUDA(cudaStreamSynchronize(c->stream));
  float ms = 0.f;
  LX_CUDA(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
  *us = 1e3 * ms / iters / k.ipl;  // per Leja iteration
  return LX_OK;
}

}  // namespace

extern "C" {

lx_status lx_ctx_select_kernel(lx_ctx* c, const char* name, int strip_h) {
  if (!c || !name || strip_h < 0) return LX_E_INVAL;
  for (int v = 0; v < kNumVariants; ++v)
    for (const Cand& k : candidates(c->prob.kind, c->prob.precision, v, is_square(c->prob)))
      if (std::strcmp(k.name, name) == 0) {
        if (v == kVec2 && c->prob.nx % (32 * k.vec) != 0) return LX_E_INVAL;
        return build_loop_graph(c, v, k, strip_h);
      }
  return LX_E_INVAL;
}

lx_status lx_ctx_autotune(lx_ctx* c, int iters, const char* cache_path, char* report, int len) {
  if (!c || iters < 1 || iters > 50) return LX_E_INVAL;
  const int v = (c->prob.nx % (32 * wide_vec(c)) == 0) ? kVec2 : kVec1;
  const std::string key = tune_key(c);
  std::ostringstream rep;
  rep << "{\"key\": \"" << key << "\", ";
  if (cache_path && cache_path[0]) {
    std::ifstream in(cache_path);
    std::string line, found_name;
    int found_h = 0;
    while (std::getline(in, line)) {
      std::istringstream ls(line);
      std::string k, nm;
      int hh = 0;
      if (ls >> k >> nm >> hh && k == key) {
        found_name = nm;
        found_h = hh;
      }
    }
    if (!found_name.empty() && lx_ctx_select_kernel(c, found_name.c_str(), found_h) == LX_OK) {
      rep << "\"cached\": true, \"selected\": {\"kernel\": \"" << found_name << "\", \"strip_h\": " << found_h
          << "}}";
      if (report && len > 0) std::snprintf(report, (size_t)len, "%s", rep.str().c_str());
      return LX_OK;
    }
  }
  const size_t nb = sizeof(double) * (size_t)c->n;
  if (!c->d_tune && !cuda_ok(cudaMalloc((void**)&c->d_tune, nb), "cudaMalloc")) return LX_E_NOMEM;
  LX_CUDA(cudaMemsetAsync(c->d_y[0], 0, basis_bytes(c), c->stream));
  LX_CUDA(cudaMemsetAsync(c->d_y[1], 0, basis_bytes(c), c->stream));
  LX_CUDA(cudaMemsetAsync(c->d_f, 0, nb, c->stream));
  LX_CUDA(cudaMemsetAsync(c->d_s, 0, nb, c->stream));
  LX_CUDA(cudaMemsetAsync(c->d_tune, 0, nb, c->stream));
  if (c->d_pdf) LX_CUDA(cudaMemsetAsync(c->d_pdf, 0, sizeof(float2) * (size_t)c->n, c->stream));
  c->prep_u = nullptr;
  if (c->d_bq) LX_CUDA(cudaMemsetAsync(c->d_bq, 0, sizeof(float2) * (size_t)c->n, c->stream));
  if (c->d_br) LX_CUDA(cudaMemsetAsync(c->d_br, 0, sizeof(float2) * (size_t)c->n, c->stream));
  if (c->d_uf) LX_CUDA(cudaMemsetAsync(c->d_uf, 0, sizeof(float) * (size_t)c->n, c->stream));
  if (c->d_sf) LX_CUDA(cudaMemsetAsync(c->d_sf, 0, sizeof(float) * (size_t)c->n, c->stream));
  lx_status st = ensure_coeffs(c, 0, 0, 1.0, -20.0, 10.0);
  if (st != LX_OK) return st;
  if (c->coef[0].count < 2 * iters + 4) return LX_E_INVAL;
  const int hs[] = {0, 8, 16, 32, 64, 128};
  double best = 1e30;
  Cand best_k{};
  int best_h = 32;
  rep << "\"cached\": false, \"timings\": [";
  bool first = true;
  for (const Cand& k : candidates(c->prob.kind, c->prob.precision, v, is_square(c->prob))) {
    for (int H : hs) {
      if (H > 2 * c->prob.ny && H != 8) continue;
      if (H == 0 && k.smem == 0) continue;  // balanced ranges: pipelined kernels only
      double us = 0.0;
      st = tune_time(c, k, H, iters, &us);
      if (st == LX_E_INVAL) continue;  // grid beyond the partials capacity
      if (st != LX_OK) return st;
      rep << (first ? "" : ", ") << "{\"kernel\": \"" << k.name << "\", \"strip_h\": " << H << ", \"us\": " << us
          << "}";
      first = false;
      if (us < best) {
        best = us;
        best_k = k;
        best_h = H;
      }
    }
  }
  if (!best_k.func) return LX_E_CUDA;
  st = build_loop_graph(c, v, best_k, best_h);
  if (st != LX_OK) return st;
  c->coef[0].valid = false;
  rep << "], \"selected\": {\"kernel\": \"" << best_k.name << "\", \"strip_h\": " << best_h << ", \"us\": " << best
      << "}}";
  if (cache_path && cache_path[0]) {
    std::ofstream out(cache_path, std::ios::app);
    if (out) out << key << "\t" << best_k.name << "\t" << best_h << "\t" << best << "\n";
  }
  if (report && len > 0) std::snprintf(report, (size_t)len, "%s", rep.str().c_str());
  return LX_OK;
}

}  // extern "C"

extern "C" {

double lx_controller_classical(double h, double err, double tol) {
  double f;
  if (!(err > 0.0)) {
    f = 2.0;
  } else {
    f = 0.9 * std::cbrt(tol / err);
    f = std::min(2.0, std::max(0.2, f));
  }
  return h * f;
}

lx_status mlp_forward_host(lx_mlp* m, const float* x_host, float* y_host, int B);

// Adaptive EXPRB32 loop shared by the classical and the learned controller.
static lx_status integrate_impl(lx_ctx* c, double* u, const double* v0, double t_final, double tol,
                                double leja_tol, int max_attempts, lx_integrate_info* info, lx_mlp* model,
                                double dt_ref) {
  if (!c || !u || !v0 || !info || !(tol > 0.0) || !(leja_tol > 0.0) || max_attempts < 1 || !(info->h > 0.0))
    return LX_E_INVAL;
  if (c->integrator != LX_EXPRB32) return LX_E_INVAL;
  if (model && !(dt_ref > 0.0)) return LX_E_INVAL;
  const size_t nb = sizeof(double) * (size_t)c->n;
  for (int k = 1; k < 3; ++k)
    if (!c->d_io[k] && !cuda_ok(cudaMalloc((void**)&c->d_io[k], nb), "cudaMalloc")) return LX_E_NOMEM;
  const int passes = info->power_iters > 0 ? info->power_iters : 10;
  double t = info->t, h = info->h;
  int steps = 0, rejected = 0, learned = 0;
  long long iters = 0;
  lx_status status = LX_OK;
  for (int att = 0; att < max_attempts && t < t_final; ++att) {
    const double hh = std::min(h, t_final - t);
    double rho = 0.0;
    lx_status st = power_bound(c, u, v0, passes, &rho, nullptr);
    if (st != LX_OK) {
      status = st;
      break;
    }
    double cc = 0.0, gamma = 0.0;
    st = lx_spectral_interval(rho, &cc, &gamma);
    if (st != LX_OK) {
      status = st;
      break;
    }
    double err = 0.0;
    int it = 0;
    st = expint_step(c, u, c->d_io[1], c->d_io[2], cc, gamma, hh, leja_tol, leja_tol, &err, &it);
    iters += it;
    if (st != LX_OK) {
      status = st;
      break;
    }
    info->last_err = err;
    const bool accept = err <= tol;
    double h_next = lx_controller_classical(hh, err, tol);
    if (model && accept) {
      // features of this attempt -> proposed log(h_next / h)
      vec_norm_kernel<<<aux_blocks(c), kThreadsPerBlock, 0, c->stream>>>(c->n, u, c->d_partials, c->d_ticket,
                                                                         c->d_state);
      ++c->stats.kernels;
      LX_CUDA(cudaGetLastError());
      LX_CUDA(cudaMemcpyAsync(c->h_state, c->d_state, sizeof(LoopState), cudaMemcpyDeviceToHost, c->stream));
      LX_CUDA(cudaStreamSynchronize(c->stream));
      const float x[5] = {(float)std::log(rho * hh), (float)std::log(hh / dt_ref), (float)(it / 100.0),
                          (float)std::log10(std::max(err, 1e-300) / tol), (float)c->h_state->red2};
      float y[2] = {0.f, 0.f};
      st = mlp_forward_host(model, x, y, 1);
      if (st != LX_OK) {
        status = st;
        break;
      }
      if (std::isfinite(y[0])) {
        const double f = std::exp(std::min(std::log(16.0), std::max(std::log(0.2), (double)y[0])));
        h_next = hh * f;
        ++learned;
      }
    }
    if (accept) {
      LX_CUDA(cudaMemcpyAsync(u, c->d_io[2], nb, cudaMemcpyDeviceToDevice, c->stream));
      t += hh;
      ++steps;
    } else {
      ++rejected;
    }
    h = h_next;
  }
  LX_CUDA(cudaStreamSynchronize(c->stream));
  info->t = t;
  info->h = h;
  info->steps = steps;
  info->rejected = rejected;
  info->leja_iters = iters;
  return status;
}

lx_status lx_integrate(lx_ctx* c, double* u, const double* v0, double t_final, double tol, double leja_tol,
                       int max_attempts, lx_integrate_info* info) {
  return integrate_impl(c, u, v0, t_final, tol, leja_tol, max_attempts, info, nullptr, 0.0);
}

lx_status lx_integrate_learned(lx_ctx* c, double* u, const double* v0, double t_final, double tol,
                               double leja_tol, int max_attempts, lx_mlp* model, double dt_ref,
                               lx_integrate_info* info) {
  if (!model) return LX_E_INVAL;
  return integrate_impl(c, u, v0, t_final, tol, leja_tol, max_attempts, info, model, dt_ref);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched instances (one launch per Leja iteration for all instances)
// ---------------------------------------------------------------------------

struct lx_batch {
  int B = 0;
  bool df = false;            // float-float batch (every nx % 128 == 0)
  float2* d_pbuf = nullptr;   // df: the polynomials as float pairs
  std::vector<size_t> poff;
  int K = 1000;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  int H = 32;
  std::vector<lx_problem> probs;
  std::vector<int> first_strip[2], nstrips[2];
  int total_strips[2] = {0, 0};
  int* d_strip_inst[2] = {nullptr, nullptr};
  BatchInst* d_inst = nullptr;
  BatchInst* h_inst = nullptr;  // pinned
  BatchState* d_bs = nullptr;
  // host-driven loop (profilers cannot see kernels inside a conditional
  // graph): the loop kernel and its launch shape per vector class
  int stream_loop = 0;
  const void* loop_fn[2] = {nullptr, nullptr};
  int loop_grid[2] = {0, 0}, loop_threads[2] = {0, 0}, loop_smem[2] = {0, 0};
  unsigned int* d_tickets = nullptr;
  unsigned int* d_block_ticket = nullptr;
  double* d_partials = nullptr;
  double* d_xi = nullptr;
  double* d_coef = nullptr;
  double* h_coef = nullptr;  // pinned, B x K
  struct Key {
    bool valid = false;
    int l = 0, count = 0;
    double h = 0, c = 0, g = 0;
  };
  std::vector<Key> keys;
  double* d_ybuf = nullptr;
  std::vector<size_t> yoff;
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  int grid[2] = {0, 0};
  cudaEvent_t ev[2] = {};
  lx_stats stats{};
};

namespace {

template <int VEC>
const void* batch_kernel_ptr() {
  return reinterpret_cast<const void*>(&leja_batch_kernel<VEC>);
}

// the float-float batch kernel's resident blocks per SM and ring depth
constexpr int kBatchDfMinBlocks = 3, kBatchDfStages = 5;

lx_status build_batch_graph(lx_batch* b, int v) {
  if (b->exec[v]) return LX_OK;
  const void* fn = v == 0 ? batch_kernel_ptr<2>() : batch_kernel_ptr<1>();
  int per_sm = 0;
  LX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreadsPerBlock, 0));
  const int want = (b->total_strips[v] + kWarpsPerBlock - 1) / kWarpsPerBlock;
  // grid of the auxiliary per-strip kernels (and of the FP64 iteration)
  b->grid[v] = std::max(1, std::min(want, std::max(per_sm, 1) * b->sm_count));
  int threads = kThreadsPerBlock, smem = 0, grid = b->grid[v];
  if (b->df) {
    // float-float: two Leja iterations per pass on the shared-memory-
    // pipelined strip, 4 warps per block
    fn = batch_df2x_kernel(kBatchDfMinBlocks, kBatchDfStages);
    threads = kPipeThreads;
    smem = batch_df2x_smem_bytes(kBatchDfStages);
    LX_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    LX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
    const int wantp = (b->total_strips[v] + kPipeWarps - 1) / kPipeWarps;
    grid = std::max(1, std::min(wantp, std::max(per_sm, 1) * b->sm_count));
  }
  LX_CUDA(cudaGraphCreate(&b->graph[v], 0));
  cudaGraphConditionalHandle cond;
  LX_CUDA(cudaGraphConditionalHandleCreate(&cond, b->graph[v], 1, cudaGraphCondAssignDefault));
  alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
  std::memset(cp_raw, 0, sizeof(cp_raw));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  LX_CUDA(cudaGraphAddNode(&cnode, b->graph[v], nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  BatchInst* inst = b->d_inst;
  const int* strip_inst = b->d_strip_inst[v];
  BatchState* bs = b->d_bs;
  double* partials = b->d_partials;
  unsigned int* tickets = b->d_tickets;
  unsigned int* bt = b->d_block_ticket;
  const double* xi = b->d_xi;
  int H = b->H, total = b->total_strips[v], use_cond = 1;
  void* kargs[] = {(void*)&inst, (void*)&strip_inst, (void*)&bs, (void*)&partials, (void*)&tickets, (void*)&bt,
                   (void*)&xi, (void*)&H, (void*)&total, (void*)&cond, (void*)&use_cond};
  cudaKernelNodeParams kp;
  std::memset(&kp, 0, sizeof(kp));
  b->loop_fn[v] = fn;
  b->loop_grid[v] = grid;
  b->loop_threads[v] = threads;
  b->loop_smem[v] = smem;
  kp.func = const_cast<void*>(fn);
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(threads);
  kp.sharedMemBytes = (unsigned)smem;
  kp.kernelParams = kargs;
  cudaGraphNode_t knode;
  LX_CUDA(cudaGraphAddKernelNode(&knode, body, nullptr, 0, &kp));
  LX_CUDA(cudaGraphInstantiate(&b->exec[v], b->graph[v], 0));
  return LX_OK;
}

}  // namespace

extern "C" {

void batch_destroy(lx_batch* b) {
  if (!b) return;
  for (int v = 0; v < 2; ++v) {
    if (b->exec[v]) cudaGraphExecDestroy(b->exec[v]);
    if (b->graph[v]) cudaGraphDestroy(b->graph[v]);
    cudaFree(b->d_strip_inst[v]);
  }
  cudaFree(b->d_inst);
  if (b->h_inst) cudaFreeHost(b->h_inst);
  cudaFree(b->d_bs);
  cudaFree(b->d_tickets);
  cudaFree(b->d_block_ticket);
  cudaFree(b->d_partials);
  cudaFree(b->d_xi);
  cudaFree(b->d_coef);
  if (b->h_coef) cudaFreeHost(b->h_coef);
  cudaFree(b->d_ybuf);
  cudaFree(b->d_pbuf);
  for (auto& e : b->ev)
    if (e) cudaEventDestroy(e);
  delete b;
}

lx_status batch_setup(int count, const lx_problem* probs, int max_leja, void* cuda_stream, lx_batch** out) {
  if (!out || count < 1 || !probs) return LX_E_INVAL;
  *out = nullptr;
  if (max_leja == 0) max_leja = 1000;
  if (max_leja < 16 || max_leja > 4096) return LX_E_INVAL;
  // one precision for the whole batch: FP64, or float-float with nx % 128 == 0
  const bool df = probs[0].precision == LX_DF64;
  for (int i = 0; i < count; ++i)
    if (!valid_problem(probs + i) || probs[i].kind != LX_ADVDIFF ||
        probs[i].precision != (df ? LX_DF64 : LX_FP64) || (df && probs[i].nx % 128 != 0))
      return LX_E_INVAL;
  lx_batch* b = new lx_batch();
  b->df = df;
  {
    const char* env = std::getenv("LEXGB_STREAM_LOOP");
    b->stream_loop = (env && env[0] == '1') ? 1 : 0;
  }
  auto fail = [&](lx_status s) {
    batch_destroy(b);
    return s;
  };
  b->B = count;
  // float-float: 64-row units (two 16-row halo chunks fewer per 128 rows and
  // half the two-row warm-ups of 32-row units; 19.6 against 20.6 ms per step
  // over the 256-instance workload, 21.6 ms with 96 rows)
  if (df) b->H = 64;
  b->K = max_leja;
  b->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  b->probs.assign(probs, probs + count);
  b->keys.resize(count);
  int dev = 0;
  if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice") ||
      !cuda_ok(cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev), "sm count"))
    return fail(LX_E_CUDA);
  // strip tables for the wide (VEC = 2; float-float: 4) and generic (VEC = 1)
  // kernels
  std::vector<int> table[2];
  for (int v = 0; v < 2; ++v) {
    const int vec = v == 0 ? (df ? 4 : 2) : 1;
    b->first_strip[v].resize(count);
    b->nstrips[v].resize(count);
    for (int i = 0; i < count; ++i) {
      const int ncs = (probs[i].nx + 32 * vec - 1) / (32 * vec);
      const int nrs = (probs[i].ny + b->H - 1) / b->H;
      b->first_strip[v][i] = (int)table[v].size();
      b->nstrips[v][i] = ncs * nrs;
      table[v].insert(table[v].end(), (size_t)ncs * nrs, i);
    }
    b->total_strips[v] = (int)table[v].size();
  }
  size_t ytot = 0, ptot = 0;
  for (int i = 0; i < count; ++i) {
    b->yoff.push_back(ytot);
    b->poff.push_back(ptot);
    const size_t n = (size_t)probs[i].nx * probs[i].ny;
    ytot += 2 * ((n + 31) / 32 * 32);
    ptot += (n + 31) / 32 * 32;
  }
  std::vector<double> xi(b->K);
  if (leja_points(b->K, xi.data()) != LX_OK) return fail(LX_E_INVAL);
  auto dm = [&](void** p, size_t bytes) { return cuda_ok(cudaMalloc(p, bytes), "cudaMalloc"); };
  if (!dm((void**)&b->d_inst, sizeof(BatchInst) * count) ||
      !cuda_ok(cudaMallocHost((void**)&b->h_inst, sizeof(BatchInst) * count), "cudaMallocHost") ||
      !dm((void**)&b->d_bs, sizeof(BatchState)) || !dm((void**)&b->d_tickets, sizeof(unsigned) * count) ||
      !dm((void**)&b->d_block_ticket, sizeof(unsigned)) ||
      !dm((void**)&b->d_partials, sizeof(double) * 4 * (size_t)std::max(b->total_strips[0], b->total_strips[1])) ||
      !dm((void**)&b->d_xi, sizeof(double) * b->K) || !dm((void**)&b->d_coef, sizeof(double) * b->K * count) ||
      !cuda_ok(cudaMallocHost((void**)&b->h_coef, sizeof(double) * b->K * count), "cudaMallocHost") ||
      !dm((void**)&b->d_ybuf, sizeof(double) * ytot) || (df && !dm((void**)&b->d_pbuf, sizeof(float2) * ptot)))
    return fail(LX_E_NOMEM);
  for (int v = 0; v < 2; ++v) {
    if (!dm((void**)&b->d_strip_inst[v], sizeof(int) * table[v].size())) return fail(LX_E_NOMEM);
    if (!cuda_ok(cudaMemcpy(b->d_strip_inst[v], table[v].data(), sizeof(int) * table[v].size(),
                            cudaMemcpyHostToDevice), "upload strips"))
      return fail(LX_E_CUDA);
  }
  if (!cuda_ok(cudaMemcpy(b->d_xi, xi.data(), sizeof(double) * b->K, cudaMemcpyHostToDevice), "upload xi"))
    return fail(LX_E_CUDA);
  for (auto& e : b->ev)
    if (!cuda_ok(cudaEventCreate(&e), "cudaEventCreate")) return fail(LX_E_CUDA);
  *out = b;
  return LX_OK;
}

lx_status batch_step(lx_batch* b, int l, const double* const* w, double* const* out, const double* cc,
                     const double* gamma, const double* h, double rtol, double atol, int* iters, int* status) {
  if (!b || !w || !out || !cc || !gamma || !h || l < 0 || l > 8 || !(rtol >= 0.0) || !(atol >= 0.0)) return LX_E_INVAL;
  bool wide = true;
  int mmax = 1;
  for (int i = 0; i < b->B; ++i) {
    if (!w[i] || !out[i] || w[i] == out[i] || !(gamma[i] != 0.0) || !std::isfinite(h[i] * cc[i]) ||
        !std::isfinite(h[i] * gamma[i]))
      return LX_E_INVAL;
    if (b->probs[i].nx % 64 != 0 || !aligned16(w[i]) || !aligned16(out[i])) wide = false;
  }
  if (b->df && !wide) return LX_E_INVAL;  // float-float batches need 16-byte aligned w and out
  const int v = wide ? 0 : 1;
  for (int i = 0; i < b->B; ++i) {
    lx_batch::Key& k = b->keys[i];
    double* hc = b->h_coef + (size_t)i * b->K;
    if (!(k.valid && k.l == l && k.h == h[i] && k.c == cc[i] && k.g == gamma[i])) {
      const int count = leja_coeff_count(h[i], cc[i], gamma[i], b->K);
      std::vector<double> xi(count);
      leja_points(count, xi.data());
      int st = leja_coeffs(l, h[i], cc[i], gamma[i], xi.data(), count, hc);
      if (st != LX_OK) return (lx_status)st;
      LX_CUDA(cudaMemcpyAsync(b->d_coef + (size_t)i * b->K, hc, sizeof(double) * count, cudaMemcpyHostToDevice,
                              b->stream));
      k.valid = true;
      k.l = l;
      k.h = h[i];
      k.c = cc[i];
      k.g = gamma[i];
      k.count = count;
    }
    const lx_problem& P = b->probs[i];
    const double dx = 1.0 / P.nx, dy = 1.0 / P.ny, ig = 1.0 / gamma[i];
    const double nx2 = P.nu / (dx * dx), ny2 = P.nu / (dy * dy);
    BatchInst& I = b->h_inst[i];
    std::memset(&I, 0, sizeof(I));
    I.nx = P.nx;
    I.ny = P.ny;
    I.first_strip = b->first_strip[v][i];
    I.nstrips = b->nstrips[v][i];
    I.kmax = k.count - 1;
    I.wxp = (nx2 + P.a / (2 * dx)) * ig;
    I.wxm = (nx2 - P.a / (2 * dx)) * ig;
    I.wyp = (ny2 + P.a / (2 * dy)) * ig;
    I.wym = (ny2 - P.a / (2 * dy)) * ig;
    I.wc0 = (-2.0 * nx2 - 2.0 * ny2 - cc[i]) * ig;
    I.rtol = rtol;
    I.atol = atol;
    I.w = w[i];
    const size_t n = (size_t)P.nx * P.ny;
    I.y0 = b->d_ybuf + b->yoff[i];
    I.y1 = I.y0 + (n + 31) / 32 * 32;
    I.p = out[i];
    I.d = b->d_coef + (size_t)i * b->K;
    if (b->df) {
      I.yf0 = reinterpret_cast<float2*>(I.y0);
      I.yf1 = reinterpret_cast<float2*>(I.y1);
      I.pf = b->d_pbuf + b->poff[i];
      const double wd[4] = {I.wxp, I.wxm, I.wyp, I.wym};
      for (int q = 0; q < 4; ++q) {
        I.wf[2 * q] = (float)wd[q];
        I.wf[2 * q + 1] = (float)(wd[q] - (double)I.wf[2 * q]);
      }
    }
    mmax = std::max(mmax, I.kmax);
  }
  lx_status st = build_batch_graph(b, v);
  if (st != LX_OK) return st;
  LX_CUDA(cudaMemcpyAsync(b->d_inst, b->h_inst, sizeof(BatchInst) * b->B, cudaMemcpyHostToDevice, b->stream));
  LX_CUDA(cudaMemsetAsync(b->d_tickets, 0, sizeof(unsigned) * b->B, b->stream));
  batch_reset_kernel<<<1, 1, 0, b->stream>>>(b->d_bs, b->B, mmax, b->d_block_ticket);
  LX_CUDA(cudaGetLastError());
  if (b->df) {
    // per-instance power-of-two input scaling
    batch_df_scale_kernel<<<b->grid[v], kThreadsPerBlock, 0, b->stream>>>(b->d_inst, b->d_strip_inst[v], b->H,
                                                                          b->total_strips[v]);
    LX_CUDA(cudaGetLastError());
    batch_df_scale_finish_kernel<<<(b->B + 255) / 256, 256, 0, b->stream>>>(b->d_inst, b->B);
    LX_CUDA(cudaGetLastError());
  }
  LX_CUDA(cudaEventRecord(b->ev[0], b->stream));
  if (!b->stream_loop) {
    LX_CUDA(cudaGraphLaunch(b->exec[v], b->stream));
  } else {
    // the same kernel launched from the host in batches of 8 (launches past
    // the end return at once)
    BatchInst* inst = b->d_inst;
    const int* strip_inst = b->d_strip_inst[v];
    BatchState* bs = b->d_bs;
    double* partials = b->d_partials;
    unsigned int* tickets = b->d_tickets;
    unsigned int* bt = b->d_block_ticket;
    const double* xi = b->d_xi;
    int H = b->H, total = b->total_strips[v], use_cond = 0;
    cudaGraphConditionalHandle cond = 0;
    void* kargs[] = {(void*)&inst, (void*)&strip_inst, (void*)&bs, (void*)&partials, (void*)&tickets, (void*)&bt,
                     (void*)&xi, (void*)&H, (void*)&total, (void*)&cond, (void*)&use_cond};
    for (int it = 0; it < mmax; it += 8) {
      for (int q = 0; q < 8; ++q)
        LX_CUDA(cudaLaunchKernel(b->loop_fn[v], dim3(b->loop_grid[v]), dim3(b->loop_threads[v]), kargs,
                                 (size_t)b->loop_smem[v], b->stream));
      BatchState hs0;
      LX_CUDA(cudaMemcpyAsync(&hs0, b->d_bs, sizeof(BatchState), cudaMemcpyDeviceToHost, b->stream));
      LX_CUDA(cudaStreamSynchronize(b->stream));
      if (hs0.active <= 0 || hs0.m >= mmax) break;
    }
  }
  LX_CUDA(cudaEventRecord(b->ev[1], b->stream));
  if (b->df) {
    batch_df_output_kernel<<<b->grid[v], kThreadsPerBlock, 0, b->stream>>>(b->d_inst, b->d_strip_inst[v], b->H,
                                                                           b->total_strips[v]);
    LX_CUDA(cudaGetLastError());
  }
  LX_CUDA(cudaMemcpyAsync(b->h_inst, b->d_inst, sizeof(BatchInst) * b->B, cudaMemcpyDeviceToHost, b->stream));
  BatchState hs;
  LX_CUDA(cudaMemcpyAsync(&hs, b->d_bs, sizeof(BatchState), cudaMemcpyDeviceToHost, b->stream));
  LX_CUDA(cudaStreamSynchronize(b->stream));
  float ms = 0.f;
  LX_CUDA(cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]));
  b->stats.loop_ms += ms;
  b->stats.loop_launches += 1;
  b->stats.loop_iterations += hs.m;
  lx_status first = LX_OK;
  for (int i = 0; i < b->B; ++i) {
    const BatchInst& I = b->h_inst[i];
    const int sti = I.done ? I.status : (int)LX_E_NOCONV;
    if (iters) iters[i] = I.done ? I.iters : hs.m;
    if (status) status[i] = sti;
    if (first == LX_OK && sti != LX_OK) first = (lx_status)sti;
  }
  return first;
}

lx_status batch_stats(lx_batch* b, lx_stats* out, int reset) {
  if (!b || !out) return LX_E_INVAL;
  *out = b->stats;
  if (reset) b->stats = lx_stats{};
  return LX_OK;
}

}  // extern "C"
