// rb_static.cu -- rb_gepp_solve_static: the batched partial-pivot solve with no allocation.
//
// Some callers cannot allocate device memory at the time they solve: code held to a memory
// budget that forbids cudaMalloc, hosts that hand the library pre-allocated buffers only, or
// runtimes that must not take the allocator's locks on their hot path. For them this entry point takes device pointers to its inputs and outputs and uses, as
// the working copy of each matrix, a file-scope device array that exists for as long as the
// library is loaded. It calls no allocating CUDA or library routine.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "rb_ctx.h"

namespace rb {

// Working matrices of rb_gepp_solve_static: RB_STATIC_SCRATCH_BYTES (16 MiB) on every GPU on
// which the library's device code is loaded, held until the process exits.
constexpr size_t kStaticScratchDoubles = RB_STATIC_SCRATCH_BYTES / sizeof(double);
static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

namespace {
std::mutex g_static_mu;
constexpr int kMaxDevices = 64;
double *g_static_ptr[kMaxDevices] = {};
int g_static_sms[kMaxDevices] = {};
// Unique id of the context the cached address belongs to. A device reset (or a new primary
// context) reloads the module and may place the array elsewhere, so a changed id redoes the
// lookup instead of handing the kernel a stale address.
unsigned long long g_static_ctx[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// Id of the calling thread's current context (0 if the driver entry points are unavailable).
unsigned long long current_ctx_id() {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked = false;
  if (!looked) {  // called under g_static_mu
    looked = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_cur = (CtxGetCurrentFn)p;
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = (CtxGetIdFn)p;
  }
  if (!get_cur || !get_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_cur(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}
}  // namespace

// One system per CTA at a time: copy M_s into this CTA's slice of the scratch, eliminate there
// with the same block-cooperative partial pivoting as rb_gepp_solve, write x_s and status_s.
__global__ void __launch_bounds__(kThreads) k_gepp_static(const double *M, const double *rhs,
                                                          double *x, int *status, int n, int batch,
                                                          double *scratch) {
  extern __shared__ double sm[];
  double *b = sm, *red = sm + ((n + 1) & ~1);
  double *W = scratch + (size_t)blockIdx.x * n * n;
  const size_t nn = (size_t)n * n;
  for (int s = blockIdx.x; s < batch; s += gridDim.x) {
    const double *Ms = M + (size_t)s * nn;
    for (size_t e = threadIdx.x; e < nn; e += blockDim.x) W[e] = Ms[e];
    for (int i = threadIdx.x; i < n; i += blockDim.x) b[i] = rhs[(size_t)s * n + i];
    __syncthreads();
    const bool sing = gepp_solve_block<double>(W, n, n, b, red);
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[(size_t)s * n + i] = sing ? 0.0 : b[i];
    if (threadIdx.x == 0) status[s] = sing ? RB_Q_SINGULAR : 0;
    __syncthreads();
  }
}

}  // namespace rb

using namespace rb;

extern "C" int rb_gepp_solve_static(int n, int batch, const double *d_M, const double *d_rhs,
                                    double *d_x, int *d_status, void *cuda_stream) {
  if (n < 1 || n > RB_STATIC_N_MAX)
    return set_error(nullptr, RB_ERR_ARG, "rb_gepp_solve_static: n = %d outside 1..%d", n,
                     RB_STATIC_N_MAX);
  if (batch < 0) return set_error(nullptr, RB_ERR_ARG, "rb_gepp_solve_static: batch < 0");
  if (batch == 0) return RB_OK;
  if (!d_M || !d_rhs || !d_x || !d_status)
    return set_error(nullptr, RB_ERR_ARG, "rb_gepp_solve_static: NULL buffer");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "rb_gepp_solve_static: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_error(nullptr, RB_ERR_ARG, "device %d", dev);
  double *scratch;
  int sms;
  {
    // once per device (and again after a device reset), with that device current: the device
    // address of the scratch array
    std::lock_guard<std::mutex> lk(g_static_mu);
    const unsigned long long cid = current_ctx_id();
    if (!g_static_ptr[dev] || g_static_ctx[dev] != cid) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess) return cuda_fail(nullptr, e, "rb_gepp_solve_static: cudaGetSymbolAddress");
      int s = 0;
      e = cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return cuda_fail(nullptr, e, "rb_gepp_solve_static: SM count");
      g_static_ptr[dev] = (double *)p;
      g_static_sms[dev] = s;
      // the lookup made the device's context current on this thread if it was not yet
      g_static_ctx[dev] = cid ? cid : current_ctx_id();
    }
    scratch = g_static_ptr[dev];
    sms = g_static_sms[dev];
  }
  const size_t per_system = (size_t)n * n;
  int grid = (int)(kStaticScratchDoubles / per_system);
  grid = grid < batch ? grid : batch;
  grid = grid < 8 * sms ? grid : 8 * sms;
  const size_t smem = sizeof(double) * (((n + 1) & ~1) + 4 * kWarps);
  k_gepp_static<<<grid, kThreads, smem, (cudaStream_t)cuda_stream>>>(d_M, d_rhs, d_x, d_status, n,
                                                                    batch, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "rb_gepp_solve_static: launch");
  return RB_OK;
}
