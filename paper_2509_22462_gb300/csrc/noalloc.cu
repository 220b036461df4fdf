// nnc_residual_noalloc: the FP64 residual r = y - NN(x) for callers that cannot allocate device
// memory, for example code running inside a CUDA-graph capture or inside another library's
// memory pool where cudaMalloc is not allowed, or a process whose allocator is owned by a host
// framework.  Such a caller passes its own device buffers for the weights, x, y and r; the
// per-layer activations, which the net-based entry points keep in memory allocated by
// nnc_load_weights, live here in one file-scope device array instead.
//
// That array (kNoallocMaxWidth x 2 doubles = 1 MiB) is reserved on every GPU that loads the
// library and stays reserved until the process exits.  Every call shares it and it keeps the
// last call's contents, so calls whose kernels overlap on the GPU (on different streams, or
// from different host threads) race with each other; callers must order them.
#include <cstring>
#include <string>

#include "../../include/nnc.h"
#include "common.cuh"

namespace nnc {

constexpr int kNoallocMaxWidth = 65536;                 // widest layer the array can hold
static __device__ __align__(256) double g_noalloc_act[2 * kNoallocMaxWidth];

// Host-side addresses of g_noalloc_act, one per device, resolved at the first call on that
// device.  In host code the symbol name itself is only a stand-in, not a device address.
constexpr int kMaxDevices = 64;
static double* g_noalloc_ptr[kMaxDevices] = {nullptr};

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
  for (int l = 0; l < n_layers; ++l)
    if (!W[l] || act[l] < NNC_IDENTITY || act[l] > NNC_GELU) {
      set_last_error("nnc_residual_noalloc: bad weight pointer or activation code");
      return NNC_ERR_ARG;
    }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_last_error(std::string("nnc_residual_noalloc: no usable device: ") + cudaGetErrorString(e));
    return NNC_ERR_CUDA;
  }
  if (!g_noalloc_ptr[dev]) {
    // Set-up, once per device, with that device current.
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_act);
    if (e != cudaSuccess || !p) {
      set_last_error(std::string("nnc_residual_noalloc: cudaGetSymbolAddress failed: ") +
                     cudaGetErrorString(e));
      return NNC_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = (double*)p;
  }
  double* buf[2] = {g_noalloc_ptr[dev], g_noalloc_ptr[dev] + kNoallocMaxWidth};
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
