// phi_l_apply_noalloc: phi_l(hA)w for the diffusion-advection operator
// without any memory allocation by the library.
//
// Who needs this: callers that must not allocate device memory at the point
// of the call -- applications that hand the whole device to their own memory
// pool and forbid other allocators, plug-ins loaded into such a host
// application, and solvers embedded in time-critical loops where the
// implicit device synchronisation of cudaMalloc/cudaFree is unacceptable.
// They pass their input and output vectors, and all scratch (the two
// Newton-basis vectors, reduction partials, the loop state, the Leja points
// and coefficients) lives in one file-scope __device__ array of fixed size
// instead of in a context.
//
// Limits and rules:
//  * at most LX_NOALLOC_MAX_POINTS grid points and LX_NOALLOC_MAX_LEJA Leja
//    points; larger problems are rejected with LX_E_INVAL;
//  * the scratch array (about 4.2 MB) is part of the module and stays
//    resident on every GPU that loads the library until the process exits;
//  * every call uses the same array and leaves its contents behind: the
//    parts that must start at zero are cleared by each call, and two calls
//    whose GPU work overlaps (different streams, or different host threads
//    without ordering) race on the array and give wrong results;
//  * the call is driven from the host: it launches the fused iteration in
//    batches of 8, reads the loop state back and synchronises the stream
//    after each batch;
//  * set-up: the first call in the process computes the table of
//    LX_NOALLOC_MAX_LEJA Leja points on the host (the only host allocation,
//    made once), and the first call on each device, with that device
//    current, looks up the array's device address with cudaGetSymbolAddress
//    and uploads the point table with a synchronous copy; make that first
//    call before any stream capture begins.  Later calls allocate nothing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "leja_kernels.cuh"
#include "lexgb_internal.h"

using namespace lexgb;

namespace {

constexpr size_t kOffArgs = 0;
constexpr size_t kOffState = 512;
constexpr size_t kOffTicket = 1024;
constexpr size_t kMaxGrid = 4096;
constexpr size_t kOffPartials = 2048;
constexpr size_t kOffXi = kOffPartials + 2 * kMaxGrid * sizeof(double);
constexpr size_t kOffD = kOffXi + LX_NOALLOC_MAX_LEJA * sizeof(double) + 256;
constexpr size_t kOffY0 = (kOffD + LX_NOALLOC_MAX_LEJA * sizeof(double) + 255) / 256 * 256 + 256;
constexpr size_t kOffY1 = kOffY0 + (size_t)LX_NOALLOC_MAX_POINTS * sizeof(double);
constexpr size_t kScratchBytes = kOffY1 + (size_t)LX_NOALLOC_MAX_POINTS * sizeof(double);

static_assert(sizeof(LoopArgs) <= kOffState - kOffArgs, "LoopArgs does not fit its slot");
static_assert(sizeof(LoopState) <= kOffTicket - kOffState, "LoopState does not fit its slot");

// The scratch.  Host code must not use this name as a device address: in host
// code it is a host-side stand-in, and the real address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_dev_ptr[kMaxDevices] = {};
int g_grid[kMaxDevices][2] = {};

const void* noalloc_kernel(int vec2) {
  return vec2 ? reinterpret_cast<const void*>(&leja_iter_kernel<0, double, 2>)
              : reinterpret_cast<const void*>(&leja_iter_kernel<0, double, 1>);
}

// The Leja point table, computed once per process at its full length so
// that no later call grows it.
double g_xi[LX_NOALLOC_MAX_LEJA];
bool g_xi_ready = false;

// Once per device, with that device current: the scratch address, the
// resident grid sizes of the two kernel variants and the point table in the
// scratch.
lx_status device_setup(int dev, unsigned char** ptr, int* grid2) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_xi_ready) {
    if (leja_points(LX_NOALLOC_MAX_LEJA, g_xi) != LX_OK) return LX_E_INVAL;
    g_xi_ready = true;
  }
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_last_error("phi_l_apply_noalloc: cudaGetSymbolAddress failed");
      return LX_E_CUDA;
    }
    if (cudaMemcpy(static_cast<unsigned char*>(p) + kOffXi, g_xi, sizeof(g_xi), cudaMemcpyHostToDevice) !=
        cudaSuccess) {
      set_last_error("phi_l_apply_noalloc: upload of the Leja point table failed");
      return LX_E_CUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LX_E_CUDA;
    for (int v = 0; v < 2; ++v) {
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, noalloc_kernel(v), kThreadsPerBlock, 0) !=
          cudaSuccess)
        return LX_E_CUDA;
      g_grid[dev][v] = std::min<int>((int)kMaxGrid, std::max(1, per_sm) * sms);
    }
    g_dev_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *ptr = g_dev_ptr[dev];
  grid2[0] = g_grid[dev][0];
  grid2[1] = g_grid[dev][1];
  return LX_OK;
}

}  // namespace

extern "C" lx_status phi_l_apply_noalloc(const lx_problem* prob, int l, const double* w, double* out, double cc,
                                         double gamma, double h, double rtol, double atol, void* cuda_stream,
                                         int* iters) {
  if (!prob || !w || !out || l < 0 || l > 8 || !(gamma != 0.0) || !std::isfinite(h) || !std::isfinite(cc) ||
      !std::isfinite(gamma) || !(rtol >= 0.0) || !(atol >= 0.0) || (const void*)w == (const void*)out)
    return LX_E_INVAL;
  if (prob->kind != LX_ADVDIFF || prob->precision != LX_FP64 || prob->nx < 1 || prob->ny < 1 ||
      !std::isfinite(prob->nu) || !std::isfinite(prob->a)) {
    set_last_error("phi_l_apply_noalloc: only LX_ADVDIFF with LX_FP64 is supported");
    return LX_E_INVAL;
  }
  const long long n = (long long)prob->nx * prob->ny;
  if (n > LX_NOALLOC_MAX_POINTS) {
    set_last_error("phi_l_apply_noalloc: nx*ny exceeds LX_NOALLOC_MAX_POINTS (262144)");
    return LX_E_INVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LX_E_CUDA;
  unsigned char* base = nullptr;
  int grids[2];
  lx_status st = device_setup(dev, &base, grids);
  if (st != LX_OK) return st;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(cuda_stream);

  // Host side: Newton coefficients in stack buffers, at the points of the
  // table made at set-up (already in the scratch).
  const int count = leja_coeff_count(h, cc, gamma, LX_NOALLOC_MAX_LEJA);
  double d[LX_NOALLOC_MAX_LEJA];
  double ws[6 * (LX_NOALLOC_MAX_LEJA + 8)];
  st = (lx_status)leja_coeffs_ws(l, h, cc, gamma, g_xi, count, d, ws);
  if (st != LX_OK) return st;

  LoopArgs* d_args = reinterpret_cast<LoopArgs*>(base + kOffArgs);
  LoopState* d_state = reinterpret_cast<LoopState*>(base + kOffState);
  unsigned int* d_ticket = reinterpret_cast<unsigned int*>(base + kOffTicket);
  double* d_partials = reinterpret_cast<double*>(base + kOffPartials);
  double* d_xi = reinterpret_cast<double*>(base + kOffXi);
  double* d_d = reinterpret_cast<double*>(base + kOffD);
  double* y0 = reinterpret_cast<double*>(base + kOffY0);
  double* y1 = reinterpret_cast<double*>(base + kOffY1);
  if (cudaMemcpyAsync(d_d, d, sizeof(double) * count, cudaMemcpyHostToDevice, stream) != cudaSuccess)
    return LX_E_CUDA;

  const double dx = 1.0 / prob->nx, dy = 1.0 / prob->ny, ig = 1.0 / gamma;
  const double nx2 = prob->nu / (dx * dx), ny2 = prob->nu / (dy * dy);
  LoopArgs a;
  std::memset(&a, 0, sizeof(a));
  a.nx = prob->nx;
  a.ny = prob->ny;
  a.n = n;
  a.strip_h = 32;
  a.kmax = count - 1;
  a.w = w;
  a.y0 = y0;
  a.y1 = y1;
  a.p = out;
  a.xi = d_xi;
  a.d = d_d;
  a.wxp = (nx2 + prob->a / (2 * dx)) * ig;
  a.wxm = (nx2 - prob->a / (2 * dx)) * ig;
  a.wyp = (ny2 + prob->a / (2 * dy)) * ig;
  a.wym = (ny2 - prob->a / (2 * dy)) * ig;
  a.wc0 = (-2.0 * nx2 - 2.0 * ny2 - cc) * ig;
  a.rtol = rtol;
  a.atol = atol;
  a.use_cond = 0;
  // clears the loop state and the arrival ticket left by the previous call
  set_loop_args_kernel<<<1, 1, 0, stream>>>(a, d_args, d_state, d_ticket);
  reset_call_kernel<<<1, 1, 0, stream>>>(d_state, d_ticket);
  if (cudaGetLastError() != cudaSuccess) return LX_E_CUDA;

  const bool vec2 = prob->nx % 64 == 0 && (reinterpret_cast<uintptr_t>(w) & 15u) == 0 &&
                    (reinterpret_cast<uintptr_t>(out) & 15u) == 0;
  const int vec = vec2 ? 2 : 1;
  const int strips = ((prob->nx + 32 * vec - 1) / (32 * vec)) * ((prob->ny + 31) / 32);
  const int grid = std::max(1, std::min((strips + kWarpsPerBlock - 1) / kWarpsPerBlock, grids[vec2 ? 1 : 0]));
  const void* fn = noalloc_kernel(vec2 ? 1 : 0);
  const LoopArgs* kargs_a = d_args;
  cudaGraphConditionalHandle cond = 0;
  void* kargs[] = {(void*)&kargs_a, (void*)&d_state, (void*)&d_partials, (void*)&d_ticket, (void*)&cond};
  LoopState hs;
  std::memset(&hs, 0, sizeof(hs));
  for (int it = 0; it < a.kmax; it += 8) {
    for (int k = 0; k < 8; ++k)
      if (cudaLaunchKernel(fn, dim3(grid), dim3(kThreadsPerBlock), kargs, 0, stream) != cudaSuccess)
        return LX_E_CUDA;
    if (cudaMemcpyAsync(&hs, d_state, sizeof(LoopState), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
      return LX_E_CUDA;
    if (hs.done) break;
  }
  if (iters) *iters = hs.iters_total;
  return (lx_status)hs.status_total;
}
