// nnc_residual_noalloc: the FP64 residual r = y - NN(x) for callers that cannot allocate device
// memory.  Some host programs own the whole device memory budget themselves: a framework that
// hands out memory only from its own pool, or a control loop that must not call cudaMalloc
// because cudaMalloc can synchronise the device and its latency is unbounded.  Such a caller
// cannot create a net (nnc_load_weights allocates the packed weights), so it passes its own
// device buffers for the weights, x, y and r; the per-layer activations, which the net-based
// entry points keep in memory allocated by nnc_load_weights, live here in one file-scope device
// array instead.
//
// That array (kNoallocMaxWidth x 2 doubles = 1 MiB) is reserved on every GPU that loads the
// library and stays reserved until the process exits.  Every call shares it and it keeps the
// last call's contents, so calls whose kernels overlap on the GPU (on different streams, or
// from different host threads) race with each other; callers must order them.
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>
#include <string>

#include "../../include/nnc.h"
#include "common.cuh"

namespace nnc {

constexpr int kNoallocMaxWidth = 65536;                 // widest layer the array can hold
static __device__ __align__(256) double g_noalloc_act[2 * kNoallocMaxWidth];

// Host-side addresses of g_noalloc_act, one per device, resolved at the first call on that
// device (and again whenever the device's context has changed since: a context destroyed and
// created anew, e.g. after cudaDeviceReset, may load the module at another address).  In host
// code the symbol name itself is only a stand-in, not a device address.
constexpr int kMaxDevices = 64;
struct NoallocSlot {
  unsigned long long ctx_id;   // cuCtxGetId of the context the address belongs to
  double* ptr;
};
static NoallocSlot g_noalloc_slot[kMaxDevices] = {};
static std::mutex g_noalloc_mu;

// Identifier of the calling thread's current context (0 if none is current or the driver does
// not provide the query).  Host-side queries only: nothing is allocated.
static unsigned long long current_ctx_id() {
  static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_cur = (PFN_cuCtxGetCurrent_v4000)p;
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = (PFN_cuCtxGetId_v12000)p;
  });
  if (!get_cur || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_cur(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// One warp per output row: z = W_l a_in + b_l (FP64, W_l row-major with row stride k),
// a_out = sigma_l(z); on the last layer r = y - a_out instead.
__global__ void k_noalloc_layer(const double* __restrict__ W, const double* __restrict__ bias,
                                const double* __restrict__ a_in, int m, int k, int act,
                                double* __restrict__ a_out, const double* __restrict__ y,
                                double* __restrict__ r) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= m) return;
  const double* w = W + (size_t)row * k;
  double acc = 0.0;
  for (int j = lane; j < k; j += 32) acc = fma(w[j], a_in[j], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    double a, d1, d2;
    act_eval(act, acc + (bias ? bias[row] : 0.0), a, d1, d2);
    if (r) r[row] = y[row] - a;
    else a_out[row] = a;
  }
}

void note_launch(int n);
void set_last_error(const std::string& msg);

}  // namespace nnc

extern "C" int nnc_residual_noalloc(int n_layers, const int* widths, const int* act,
                                    const double* const* W, const double* const* b,
                                    const double* x, const double* y, double* r, void* stream) {
  using namespace nnc;
  if (n_layers < 1 || !widths || !act || !W || !x || !y || !r) {
    set_last_error("nnc_residual_noalloc: null argument or n_layers < 1");
    return NNC_ERR_ARG;
  }
  for (int l = 0; l <= n_layers; ++l)
    if (widths[l] < 1 || widths[l] > kNoallocMaxWidth) {
      set_last_error("nnc_residual_noalloc: layer width " + std::to_string(widths[l]) +
                     " outside [1, 65536], the size of its fixed scratch array");
      return NNC_ERR_ARG;
    }
  for (int l = 0; l < n_layers; ++l) {
    if (act[l] == NNC_SOFTMAX) {
      set_last_error("nnc_residual_noalloc: the softmax output layer is not supported here "
                     "(elementwise activations only); use nnc_residual on a loaded net");
      return NNC_ERR_UNSUPPORTED;
    }
    if (!W[l] || act[l] < NNC_IDENTITY || act[l] > NNC_GELU) {
      set_last_error("nnc_residual_noalloc: bad weight pointer or activation code");
      return NNC_ERR_ARG;
    }
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_last_error(std::string("nnc_residual_noalloc: no usable device: ") + cudaGetErrorString(e));
    return NNC_ERR_CUDA;
  }
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocSlot& slot = g_noalloc_slot[dev];
    const unsigned long long id = current_ctx_id();
    if (slot.ptr && id != 0 && slot.ctx_id == id) {
      base = slot.ptr;
    } else {
      // Set-up, with the device current: once per device and context (the first call on a
      // device; again only if its context was replaced).
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_act);
      if (e != cudaSuccess || !p) {
        set_last_error(std::string("nnc_residual_noalloc: cudaGetSymbolAddress failed: ") +
                       cudaGetErrorString(e));
        return NNC_ERR_CUDA;
      }
      // the lookup above makes the primary context current if it was not yet
      slot.ctx_id = current_ctx_id();
      slot.ptr = (double*)p;
      base = slot.ptr;
    }
  }
  double* buf[2] = {base, base + kNoallocMaxWidth};
  cudaStream_t st = (cudaStream_t)stream;
  const double* a_in = x;
  for (int l = 0; l < n_layers; ++l) {
    const int m = widths[l + 1], k = widths[l];
    const bool last = l == n_layers - 1;
    double* a_out = buf[l & 1];
    const int blocks = (m * 32 + 255) / 256;
    k_noalloc_layer<<<blocks, 256, 0, st>>>(W[l], b ? b[l] : nullptr, a_in, m, k, act[l], a_out,
                                             y, last ? r : nullptr);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_last_error(std::string("nnc_residual_noalloc: launch failed: ") + cudaGetErrorString(e));
      return NNC_ERR_CUDA;
    }
    a_in = a_out;
  }
  return NNC_OK;
}
