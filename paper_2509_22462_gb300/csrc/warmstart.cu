// Learned warm start for the interior-point method: an MLP u -> GELU -> GELU -> linear that maps
// problem parameters (here the load vector of the SCOPF-shaped problem) to the solver's primal
// and dual starting point, trained by the library's own kernels:
//   forward   Z_1 = U W_1^T + b_1, H_1 = GELU(Z_1), Z_2 = H_1 W_2^T + b_2, H_2 = GELU(Z_2),
//             P = H_2 W_3^T + b_3                                   (GELU(z) = z Phi(z), erf form)
//   loss      L = mean((P - T)^2) over the batch, on standardized inputs and targets
//   backward  dP = 2 (P - T) / (B n_out); dW_l = dZ_l^T H_{l-1}; db_l = column sums of dZ_l;
//             dH_{l-1} = dZ_l W_l; dZ = dH * GELU'(Z)
//   Adam      (Kingma & Ba) on FP32 master weights, FP32 moments, BF16 operand copies.
// GEMMs: in the BF16 form the products run on the tcgen05 tensor cores (tc_plain: TMA-fed BF16
// operands, FP32 accumulation in tensor memory, bias / GELU fused into the epilogue, which also
// writes the transposed BF16 copy of each activation that the weight gradient dW = dZ^T H reads);
// the backward products take transposed operand copies written by the loss, GELU-derivative and
// Adam kernels.  Shapes the tensor cores cannot take (a batch that is not a multiple of 64 in the
// weight-gradient products, widths that are not multiples of 64) and the FP32 form use a
// shared-memory tiled CUDA-core kernel.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <random>
#include <string>
#include <vector>

#include "../../include/nnc.h"
#include "common.cuh"
#include "tc.cuh"

namespace nnc {
void set_last_error(const std::string& msg);
}
using namespace nnc;

namespace {

// C[m][n] = sum_k A(m, k) B(k, n) (+ bias[n]); A(m, k) = A[m * sam + k * sak] and likewise B,
// inputs of type T (BF16 or FP32), FP32 accumulation; optional GELU epilogue writes Z and H.
template <typename T>
__device__ __forceinline__ float ld(const T* p) {
  if constexpr (std::is_same<T, float>::value) return *p;
  else return __bfloat162float(*p);
}

template <typename T>
__global__ void __launch_bounds__(256) k_ws_gemm(const T* __restrict__ A, long sam, long sak,
                                                 const T* __restrict__ B, long sbk, long sbn, int M,
                                                 int N, int K, const float* __restrict__ bias,
                                                 float* __restrict__ C, int ldc, int gelu,
                                                 float* __restrict__ Hf, T* __restrict__ Hl,
                                                 int accumulate) {
  __shared__ float As[16][65];
  __shared__ float Bs[16][65];
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int i = threadIdx.x; i < 64 * 16; i += 256) {
      const int r = i >> 4, kk = i & 15;
      const int gm = m0 + r, gk = k0 + kk;
      As[kk][r] = (gm < M && gk < K) ? ld(A + gm * sam + gk * sak) : 0.f;
      const int gn = n0 + r;
      Bs[kk][r] = (gn < N && gk < K) ? ld(B + gk * sbk + gn * sbn) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + tx + 16 * i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + ty + 16 * j;
      if (n >= N) continue;
      float v = acc[i][j] + (bias ? bias[n] : 0.f);
      const size_t o = (size_t)m * ldc + n;
      if (accumulate) v += C[o];
      C[o] = v;
      if (gelu) {
        double a, d1, d2;
        act_eval(NNC_GELU, (double)v, a, d1, d2);
        Hf[o] = (float)a;
        if constexpr (std::is_same<T, float>::value) Hl[o] = (float)a;
        else Hl[o] = __float2bfloat16_rn((float)a);
      }
    }
  }
}

template <typename T>
void gemm(const T* A, long sam, long sak, const T* B, long sbk, long sbn, int M, int N, int K,
          const float* bias, float* C, int ldc, bool gelu, float* Hf, T* Hl, cudaStream_t st) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  k_ws_gemm<T><<<grid, 256, 0, st>>>(A, sam, sak, B, sbk, sbn, M, N, K, bias, C, ldc, gelu ? 1 : 0,
                                     Hf, Hl, 0);
  note_launch();
}

// dZ = dH * GELU'(Z), stored in FP32 and in the operand type.
template <typename T>
__global__ void k_ws_gelu_back(const float* __restrict__ dH, const float* __restrict__ Z, int n,
                               float* __restrict__ dZ, T* __restrict__ dZl, int cols,
                               __nv_bfloat16* __restrict__ dZt, int ldt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a, d1, d2;
  act_eval(NNC_GELU, (double)Z[i], a, d1, d2);
  const float v = dH[i] * (float)d1;
  dZ[i] = v;
  if constexpr (std::is_same<T, float>::value) dZl[i] = v;
  else dZl[i] = __float2bfloat16_rn(v);
  if (dZt) dZt[(size_t)(i % cols) * ldt + i / cols] = __float2bfloat16_rn(v);   // transposed copy
}

// dP = 2 (P - T) / (B n_out); loss partial sums per block into part[blockIdx.x].
template <typename T>
__global__ void k_ws_loss(const float* __restrict__ P, const float* __restrict__ Tt, int n,
                          float scale, float* __restrict__ dP, T* __restrict__ dPl,
                          double* __restrict__ part, int cols, __nv_bfloat16* __restrict__ dPp,
                          int ldp, __nv_bfloat16* __restrict__ dPt, int ldt) {
  __shared__ double red[256];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  if (i < n) {
    const float d = P[i] - Tt[i];
    s = (double)d * d;
    const float g = 2.f * d * scale;
    dP[i] = g;
    if constexpr (std::is_same<T, float>::value) dPl[i] = g;
    else dPl[i] = __float2bfloat16_rn(g);
    // tensor-core operands: dP with its row stride padded to a multiple of 64 (the padding stays
    // zero) and dP^T
    const int r = i / cols, c = i % cols;
    if (dPp) dPp[(size_t)r * ldp + c] = __float2bfloat16_rn(g);
    if (dPt) dPt[(size_t)c * ldt + r] = __float2bfloat16_rn(g);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// db[j] = sum_b dZ[b][j]
__global__ void k_ws_colsum(const float* __restrict__ dZ, int B, int N, float* __restrict__ db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += dZ[(size_t)b * N + j];
  db[j] = s;
}

// Adam on one flat parameter array; refreshes the operand copy (and, for a weight matrix of
// `cols` columns with wt given, its transposed BF16 copy, row stride ldt).
template <typename T>
__global__ void k_ws_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                          float* __restrict__ v, T* __restrict__ wl, int n, float lr, float b1,
                          float b2, float eps, float c1, float c2, int cols,
                          __nv_bfloat16* __restrict__ wt, int ldt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  if (wl) {
    if constexpr (std::is_same<T, float>::value) wl[i] = wi;
    else wl[i] = __float2bfloat16_rn(wi);
  }
  if (wt) wt[(size_t)(i % cols) * ldt + i / cols] = __float2bfloat16_rn(wi);
}

template <typename T>
__global__ void k_ws_gather(const float* __restrict__ src, const int* __restrict__ idx, int rows,
                            int cols, float* __restrict__ dst, T* __restrict__ dstl,
                            __nv_bfloat16* __restrict__ dstt = nullptr, int ldt = 0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  const int r = i / cols, c = i % cols;
  const float v = src[(size_t)idx[r] * cols + c];
  if (dst) dst[i] = v;
  if (dstl) {
    if constexpr (std::is_same<T, float>::value) dstl[i] = v;
    else dstl[i] = __float2bfloat16_rn(v);
  }
  if (dstt) dstt[(size_t)c * ldt + r] = __float2bfloat16_rn(v);
}

// dst = src in the operand type; with dstt also the transposed BF16 copy of a rows x cols matrix
template <typename T>
__global__ void k_ws_cast(const float* __restrict__ src, int n, T* __restrict__ dst, int cols = 1,
                          __nv_bfloat16* __restrict__ dstt = nullptr, int ldt = 0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if constexpr (std::is_same<T, float>::value) dst[i] = src[i];
  else dst[i] = __float2bfloat16_rn(src[i]);
  if (dstt) dstt[(size_t)(i % cols) * ldt + i / cols] = __float2bfloat16_rn(src[i]);
}

int wfail(int code, const std::string& m) {
  set_last_error(m);
  return code;
}
#define WCK(expr)                                                                            \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess) return wfail(NNC_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

struct nnc_ws {
  int n_in = 0, h1 = 0, h2 = 0, n_out = 0, prec = NNC_BF16;
  int sizes[6];
  float *w[6] = {}, *g[6] = {}, *m[6] = {}, *v[6] = {};
  void* wl[6] = {};                // operand copies (BF16 or FP32)
  std::vector<double> in_mean, in_std, out_mean, out_std;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<void*> allocs;
  long long step = 0;
  // batch workspace (capacity cap rows)
  int cap = 0;
  float *U = nullptr, *Tt = nullptr, *Z1 = nullptr, *H1 = nullptr, *Z2 = nullptr, *H2 = nullptr,
        *P = nullptr, *dP = nullptr, *dH = nullptr, *dZ = nullptr;
  void *Ul = nullptr, *H1l = nullptr, *H2l = nullptr, *dPl = nullptr, *dZl = nullptr;
  double* part = nullptr;
  int* idx = nullptr;
  float *Ud = nullptr, *Td = nullptr;   // standardized dataset on the device
  int nd = 0;
  // tensor-core path (BF16 form with n_in, h1, h2 multiples of 64): transposed BF16 operand copies
  // (row stride cap), dP with its row stride padded to n_out_p, W2^T and W3^T, and the plans of
  // the eight products (built for `plan_rows` batch rows)
  bool tc = false;
  int n_out_p = 0;
  __nv_bfloat16 *Ut = nullptr, *H1t = nullptr, *H2t = nullptr, *dPt = nullptr, *dZt = nullptr,
                *dPp = nullptr, *W2t = nullptr, *W3t = nullptr;
  int* d_err = nullptr;
  nnc::PlainPlan pl[8];
  int plan_rows = -1;
};

namespace {

template <typename X>
int walloc(nnc_ws* s, X** p, size_t n) {
  void* q = nullptr;
  if (cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(X)) != cudaSuccess) return wfail(NNC_ERR_OOM, "cudaMalloc failed");
  cudaMemsetAsync(q, 0, std::max<size_t>(n, 1) * sizeof(X), s->stream);
  s->allocs.push_back(q);
  *p = (X*)q;
  return NNC_OK;
}
#define WAL(p, n)                          \
  do {                                     \
    int r_ = walloc(s, &(p), (n));         \
    if (r_) return r_;                     \
  } while (0)

size_t esz(const nnc_ws* s) { return s->prec == NNC_FP32 ? 4 : 2; }

int ensure_cap(nnc_ws* s, int B) {
  if (B <= s->cap) return NNC_OK;
  if (s->tc) B = (B + 63) / 64 * 64;   // the transposed copies' row stride: a multiple of 64
  const int wmax = std::max(std::max(s->h1, s->h2), std::max(s->n_in, s->n_out));
  const size_t big = (size_t)B * wmax;
  WAL(s->U, big);
  WAL(s->Tt, big);
  WAL(s->Z1, big);
  WAL(s->H1, big);
  WAL(s->Z2, big);
  WAL(s->H2, big);
  WAL(s->P, big);
  WAL(s->dP, big);
  WAL(s->dH, big);
  WAL(s->dZ, big);
  unsigned char* q;
  WAL(q, big * esz(s)); s->Ul = q;
  WAL(q, big * esz(s)); s->H1l = q;
  WAL(q, big * esz(s)); s->H2l = q;
  WAL(q, big * esz(s)); s->dPl = q;
  WAL(q, big * esz(s)); s->dZl = q;
  WAL(s->part, (big + 255) / 256 + 1);
  WAL(s->idx, B);
  if (s->tc) {
    WAL(s->Ut, (size_t)s->n_in * B);
    WAL(s->H1t, (size_t)s->h1 * B);
    WAL(s->H2t, (size_t)s->h2 * B);
    WAL(s->dPt, (size_t)s->n_out * B);
    WAL(s->dZt, (size_t)std::max(s->h1, s->h2) * B);
    WAL(s->dPp, (size_t)B * s->n_out_p);
  }
  s->cap = B;
  s->plan_rows = -1;
  return NNC_OK;
}

// the eight tensor-core products for batches of B rows (tensor maps of the current buffers)
int make_plans(nnc_ws* s, int B) {
  if (s->plan_rows == B) return NNC_OK;
  using nnc::tc_plain_plan;
  const int cap = s->cap;
  const __nv_bfloat16* w1 = (const __nv_bfloat16*)s->wl[0];
  const __nv_bfloat16* w2 = (const __nv_bfloat16*)s->wl[2];
  const __nv_bfloat16* w3 = (const __nv_bfloat16*)s->wl[4];
  int r = tc_plain_plan(s->pl[0], s->Ul, B, s->n_in, w1, s->h1, s->n_in, B, s->h1, s->n_in);
  if (!r) r = tc_plain_plan(s->pl[1], s->H1l, B, s->h1, w2, s->h2, s->h1, B, s->h2, s->h1);
  if (!r) r = tc_plain_plan(s->pl[2], s->H2l, B, s->h2, w3, s->n_out, s->h2, B, s->n_out, s->h2);
  if (!r && B % 64 == 0) {
    r = tc_plain_plan(s->pl[3], s->dPt, s->n_out, cap, s->H2t, s->h2, cap, s->n_out, s->h2, B);
    if (!r) r = tc_plain_plan(s->pl[4], s->dPp, B, s->n_out_p, s->W3t, s->h2, s->n_out_p, B, s->h2, s->n_out_p);
    if (!r) r = tc_plain_plan(s->pl[5], s->dZt, s->h2, cap, s->H1t, s->h1, cap, s->h2, s->h1, B);
    if (!r) r = tc_plain_plan(s->pl[6], s->dZl, B, s->h2, s->W2t, s->h1, s->h2, B, s->h1, s->h2);
    if (!r) r = tc_plain_plan(s->pl[7], s->dZt, s->h1, cap, s->Ut, s->n_in, cap, s->h1, s->n_in, B);
  }
  if (r) return wfail(r, "warm start: tensor-core plan failed");
  s->plan_rows = B;
  return NNC_OK;
}
#define TCK(expr)                                                                            \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess) return wfail(NNC_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// forward on the first B rows of s->U (FP32) / s->Ul (operand type): P = net(U)
template <typename T>
int forward(nnc_ws* s, int B) {
  cudaStream_t st = s->stream;
  if constexpr (!std::is_same<T, float>::value) {
    if (s->tc) {
      int r = make_plans(s, B);
      if (r) return r;
      TCK(nnc::tc_plain(s->pl[0], s->w[1], s->Z1, s->h1, true, s->H1, s->H1l, s->H1t, s->cap, s->d_err, st));
      TCK(nnc::tc_plain(s->pl[1], s->w[3], s->Z2, s->h2, true, s->H2, s->H2l, s->H2t, s->cap, s->d_err, st));
      TCK(nnc::tc_plain(s->pl[2], s->w[5], s->P, s->n_out, false, nullptr, nullptr, nullptr, 0, s->d_err, st));
      return NNC_OK;
    }
  }
  T* Ul = (T*)s->Ul;
  gemm<T>(Ul, s->n_in, 1, (const T*)s->wl[0], 1, s->n_in, B, s->h1, s->n_in, s->w[1], s->Z1, s->h1,
          true, s->H1, (T*)s->H1l, st);
  gemm<T>((const T*)s->H1l, s->h1, 1, (const T*)s->wl[2], 1, s->h1, B, s->h2, s->h1, s->w[3], s->Z2,
          s->h2, true, s->H2, (T*)s->H2l, st);
  gemm<T>((const T*)s->H2l, s->h2, 1, (const T*)s->wl[4], 1, s->h2, B, s->n_out, s->h2, s->w[5], s->P,
          s->n_out, false, nullptr, (T*)nullptr, st);
  return NNC_OK;
}

// loss and gradients on the first B rows (targets in s->Tt); returns the loss through *loss
template <typename T>
int loss_grad(nnc_ws* s, int B, double* loss) {
  cudaStream_t st = s->stream;
  int rf = forward<T>(s, B);
  if (rf) return rf;
  const int nP = B * s->n_out;
  const int nb = (nP + 255) / 256;
  // tensor-core backward products need the batch (their K) to be a multiple of 64
  const bool tcb = !std::is_same<T, float>::value && s->tc && B % 64 == 0;
  k_ws_loss<T><<<nb, 256, 0, st>>>(s->P, s->Tt, nP, 1.f / (float)nP, s->dP, (T*)s->dPl, s->part,
                                   s->n_out, tcb ? s->dPp : nullptr, s->n_out_p,
                                   tcb ? s->dPt : nullptr, s->cap);
  note_launch();
  if (tcb) {
    // layer 3: dW3 = dP^T H2, db3 = colsum dP, dH2 = dP W3
    TCK(nnc::tc_plain(s->pl[3], nullptr, s->g[4], s->h2, false, nullptr, nullptr, nullptr, 0, s->d_err, st));
    k_ws_colsum<<<(s->n_out + 255) / 256, 256, 0, st>>>(s->dP, B, s->n_out, s->g[5]);
    TCK(nnc::tc_plain(s->pl[4], nullptr, s->dH, s->h2, false, nullptr, nullptr, nullptr, 0, s->d_err, st));
    k_ws_gelu_back<T><<<(B * s->h2 + 255) / 256, 256, 0, st>>>(s->dH, s->Z2, B * s->h2, s->dZ, (T*)s->dZl,
                                                              s->h2, s->dZt, s->cap);
    // layer 2
    TCK(nnc::tc_plain(s->pl[5], nullptr, s->g[2], s->h1, false, nullptr, nullptr, nullptr, 0, s->d_err, st));
    k_ws_colsum<<<(s->h2 + 255) / 256, 256, 0, st>>>(s->dZ, B, s->h2, s->g[3]);
    TCK(nnc::tc_plain(s->pl[6], nullptr, s->dH, s->h1, false, nullptr, nullptr, nullptr, 0, s->d_err, st));
    k_ws_gelu_back<T><<<(B * s->h1 + 255) / 256, 256, 0, st>>>(s->dH, s->Z1, B * s->h1, s->dZ, (T*)s->dZl,
                                                              s->h1, s->dZt, s->cap);
    // layer 1
    TCK(nnc::tc_plain(s->pl[7], nullptr, s->g[0], s->n_in, false, nullptr, nullptr, nullptr, 0, s->d_err, st));
    k_ws_colsum<<<(s->h1 + 255) / 256, 256, 0, st>>>(s->dZ, B, s->h1, s->g[1]);
    note_launch(5);
  } else {
  // layer 3: dW3 = dP^T H2, db3 = colsum dP, dH2 = dP W3
  gemm<T>((const T*)s->dPl, 1, s->n_out, (const T*)s->H2l, s->h2, 1, s->n_out, s->h2, B, nullptr,
          s->g[4], s->h2, false, nullptr, (T*)nullptr, st);
  k_ws_colsum<<<(s->n_out + 255) / 256, 256, 0, st>>>(s->dP, B, s->n_out, s->g[5]);
  gemm<T>((const T*)s->dPl, s->n_out, 1, (const T*)s->wl[4], s->h2, 1, B, s->h2, s->n_out, nullptr,
          s->dH, s->h2, false, nullptr, (T*)nullptr, st);
  k_ws_gelu_back<T><<<(B * s->h2 + 255) / 256, 256, 0, st>>>(s->dH, s->Z2, B * s->h2, s->dZ, (T*)s->dZl,
                                                            s->h2, nullptr, 0);
  // layer 2
  gemm<T>((const T*)s->dZl, 1, s->h2, (const T*)s->H1l, s->h1, 1, s->h2, s->h1, B, nullptr, s->g[2],
          s->h1, false, nullptr, (T*)nullptr, st);
  k_ws_colsum<<<(s->h2 + 255) / 256, 256, 0, st>>>(s->dZ, B, s->h2, s->g[3]);
  gemm<T>((const T*)s->dZl, s->h2, 1, (const T*)s->wl[2], s->h1, 1, B, s->h1, s->h2, nullptr, s->dH,
          s->h1, false, nullptr, (T*)nullptr, st);
  k_ws_gelu_back<T><<<(B * s->h1 + 255) / 256, 256, 0, st>>>(s->dH, s->Z1, B * s->h1, s->dZ, (T*)s->dZl,
                                                            s->h1, nullptr, 0);
  // layer 1
  gemm<T>((const T*)s->dZl, 1, s->h1, (const T*)s->Ul, s->n_in, 1, s->h1, s->n_in, B, nullptr, s->g[0],
          s->n_in, false, nullptr, (T*)nullptr, st);
  k_ws_colsum<<<(s->h1 + 255) / 256, 256, 0, st>>>(s->dZ, B, s->h1, s->g[1]);
  note_launch(5);
  }
  if (loss) {
    std::vector<double> h(nb);
    WCK(cudaMemcpyAsync(h.data(), s->part, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
    WCK(cudaStreamSynchronize(st));
    double t = 0;
    for (double x : h) t += x;
    *loss = t / nP;
  }
  return NNC_OK;
}

template <typename T>
void adam(nnc_ws* s, float lr, float b1, float b2, float eps) {
  s->step += 1;
  const float c1 = 1.f - std::pow(b1, (float)s->step), c2 = 1.f - std::pow(b2, (float)s->step);
  for (int i = 0; i < 6; ++i) {
    // W2^T and W3^T feed the tensor-core backward products
    __nv_bfloat16* wt = !s->tc ? nullptr : i == 2 ? s->W2t : i == 4 ? s->W3t : nullptr;
    const int cols = i == 2 ? s->h1 : i == 4 ? s->h2 : 1;
    const int ldt = i == 2 ? s->h2 : i == 4 ? s->n_out_p : 0;
    k_ws_adam<T><<<(s->sizes[i] + 255) / 256, 256, 0, s->stream>>>(
        s->w[i], s->g[i], s->m[i], s->v[i], (i % 2 == 0) ? (T*)s->wl[i] : (T*)nullptr, s->sizes[i], lr,
        b1, b2, eps, c1, c2, cols, wt, ldt);
  }
  note_launch(6);
}

template <typename T>
void stage_rows(nnc_ws* s, const float* U, const float* Tt, int B) {
  // U (B x n_in) and T (B x n_out) already on the device in standardized FP32
  if (U != s->U) cudaMemcpyAsync(s->U, U, sizeof(float) * B * s->n_in, cudaMemcpyDeviceToDevice, s->stream);
  if (Tt && Tt != s->Tt)
    cudaMemcpyAsync(s->Tt, Tt, sizeof(float) * B * s->n_out, cudaMemcpyDeviceToDevice, s->stream);
  k_ws_cast<T><<<(B * s->n_in + 255) / 256, 256, 0, s->stream>>>(s->U, B * s->n_in, (T*)s->Ul, s->n_in,
                                                                  s->tc ? s->Ut : nullptr, s->cap);
  note_launch();
}

int upload_std(nnc_ws* s, const double* U, const double* Tt, int N, bool with_t) {
  std::vector<float> hu((size_t)N * s->n_in), ht(with_t ? (size_t)N * s->n_out : 0);
  for (int r = 0; r < N; ++r) {
    for (int c = 0; c < s->n_in; ++c)
      hu[(size_t)r * s->n_in + c] = (float)((U[(size_t)r * s->n_in + c] - s->in_mean[c]) / s->in_std[c]);
    if (with_t)
      for (int c = 0; c < s->n_out; ++c)
        ht[(size_t)r * s->n_out + c] = (float)((Tt[(size_t)r * s->n_out + c] - s->out_mean[c]) / s->out_std[c]);
  }
  int r = ensure_cap(s, N);
  if (r) return r;
  WCK(cudaMemcpyAsync(s->U, hu.data(), sizeof(float) * hu.size(), cudaMemcpyHostToDevice, s->stream));
  if (with_t)
    WCK(cudaMemcpyAsync(s->Tt, ht.data(), sizeof(float) * ht.size(), cudaMemcpyHostToDevice, s->stream));
  WCK(cudaStreamSynchronize(s->stream));
  return NNC_OK;
}

// the tensor-core kernels' bounded waits record an error word; a set word fails the call
int check_ws_err(nnc_ws* s) {
  if (!s->d_err) return NNC_OK;
  int e = 0;
  WCK(cudaMemcpyAsync(&e, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  WCK(cudaStreamSynchronize(s->stream));
  if (e) {
    cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream);
    return wfail(NNC_ERR_TIMEOUT, "warm start: a bounded device-side wait ran out");
  }
  return NNC_OK;
}

}  // namespace

extern "C" {

int nnc_ws_create(nnc_ws** out, int n_in, int h1, int h2, int n_out, const double* const* params,
                  int prec, void* stream) {
  if (!out || n_in < 1 || h1 < 1 || h2 < 1 || n_out < 1 || !params || (prec != NNC_BF16 && prec != NNC_FP32))
    return wfail(NNC_ERR_ARG, "nnc_ws_create: bad arguments");
  *out = nullptr;
  nnc_ws* s = new nnc_ws();
  s->n_in = n_in;
  s->h1 = h1;
  s->h2 = h2;
  s->n_out = n_out;
  s->prec = prec;
  if (stream) s->stream = (cudaStream_t)stream;
  else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete s;
      return wfail(NNC_ERR_CUDA, "no CUDA device");
    }
    s->own_stream = true;
  }
  const int sz[6] = {h1 * n_in, h1, h2 * h1, h2, n_out * h2, n_out};
  s->tc = prec == NNC_BF16 && n_in % 64 == 0 && h1 % 64 == 0 && h2 % 64 == 0;
  s->n_out_p = (n_out + 63) / 64 * 64;
  if (s->tc) {
    int r = walloc(s, &s->W2t, (size_t)h1 * h2);
    if (!r) r = walloc(s, &s->W3t, (size_t)h2 * s->n_out_p);
    if (!r) r = walloc(s, &s->d_err, 1);
    if (r) {
      nnc_ws_free(s);
      return r;
    }
  }
  for (int i = 0; i < 6; ++i) {
    s->sizes[i] = sz[i];
    if (!params[i]) {
      nnc_ws_free(s);
      return wfail(NNC_ERR_ARG, "NULL parameter array");
    }
    int r = walloc(s, &s->w[i], sz[i]);
    if (!r) r = walloc(s, &s->g[i], sz[i]);
    if (!r) r = walloc(s, &s->m[i], sz[i]);
    if (!r) r = walloc(s, &s->v[i], sz[i]);
    unsigned char* q = nullptr;
    if (!r) r = walloc(s, &q, (size_t)sz[i] * esz(s));
    if (r) {
      nnc_ws_free(s);
      return r;
    }
    s->wl[i] = q;
    std::vector<float> h(params[i], params[i] + sz[i]);
    cudaMemcpyAsync(s->w[i], h.data(), sizeof(float) * sz[i], cudaMemcpyHostToDevice, s->stream);
    if (prec == NNC_FP32) k_ws_cast<float><<<(sz[i] + 255) / 256, 256, 0, s->stream>>>(s->w[i], sz[i], (float*)q);
    else {
      __nv_bfloat16* wt = !s->tc ? nullptr : i == 2 ? s->W2t : i == 4 ? s->W3t : nullptr;
      k_ws_cast<__nv_bfloat16><<<(sz[i] + 255) / 256, 256, 0, s->stream>>>(
          s->w[i], sz[i], (__nv_bfloat16*)q, i == 2 ? h1 : i == 4 ? h2 : 1, wt,
          i == 2 ? h2 : i == 4 ? s->n_out_p : 0);
    }
    note_launch();
    cudaStreamSynchronize(s->stream);
  }
  s->in_mean.assign(n_in, 0.0);
  s->in_std.assign(n_in, 1.0);
  s->out_mean.assign(n_out, 0.0);
  s->out_std.assign(n_out, 1.0);
  if (cudaGetLastError() != cudaSuccess) {
    nnc_ws_free(s);
    return wfail(NNC_ERR_CUDA, "nnc_ws_create: CUDA error");
  }
  *out = s;
  return NNC_OK;
}

void nnc_ws_free(nnc_ws* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (void* p : s->allocs) cudaFree(p);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

int nnc_ws_set_scaling(nnc_ws* s, const double* in_mean, const double* in_std,
                       const double* out_mean, const double* out_std) {
  if (!s || !in_mean || !in_std || !out_mean || !out_std) return wfail(NNC_ERR_ARG, "bad scaling");
  s->in_mean.assign(in_mean, in_mean + s->n_in);
  s->in_std.assign(in_std, in_std + s->n_in);
  s->out_mean.assign(out_mean, out_mean + s->n_out);
  s->out_std.assign(out_std, out_std + s->n_out);
  return NNC_OK;
}

int nnc_ws_loss_grad(nnc_ws* s, const double* U, const double* Tt, int B, double* loss,
                     double* const* grads) {
  if (!s || !U || !Tt || B < 1) return wfail(NNC_ERR_ARG, "nnc_ws_loss_grad: bad arguments");
  int r = upload_std(s, U, Tt, B, true);
  if (r) return r;
  if (s->prec == NNC_FP32) {
    stage_rows<float>(s, s->U, s->Tt, B);
    r = loss_grad<float>(s, B, loss);
  } else {
    stage_rows<__nv_bfloat16>(s, s->U, s->Tt, B);
    r = loss_grad<__nv_bfloat16>(s, B, loss);
  }
  if (r) return r;
  r = check_ws_err(s);
  if (r) return r;
  if (grads) {
    for (int i = 0; i < 6; ++i) {
      if (!grads[i]) continue;
      std::vector<float> h(s->sizes[i]);
      WCK(cudaMemcpyAsync(h.data(), s->g[i], sizeof(float) * s->sizes[i], cudaMemcpyDeviceToHost, s->stream));
      WCK(cudaStreamSynchronize(s->stream));
      for (int j = 0; j < s->sizes[i]; ++j) grads[i][j] = h[j];
    }
  }
  return NNC_OK;
}

int nnc_ws_adam_step(nnc_ws* s, double lr, double beta1, double beta2, double eps) {
  if (!s) return wfail(NNC_ERR_ARG, "ws is NULL");
  if (s->prec == NNC_FP32) adam<float>(s, (float)lr, (float)beta1, (float)beta2, (float)eps);
  else adam<__nv_bfloat16>(s, (float)lr, (float)beta1, (float)beta2, (float)eps);
  WCK(cudaGetLastError());
  return NNC_OK;
}

int nnc_ws_train(nnc_ws* s, const double* U, const double* Tt, int N, int epochs, int batch,
                 double lr, double beta1, double beta2, double eps, unsigned long long seed,
                 double* final_loss) {
  if (!s || !U || !Tt || N < 1 || epochs < 0 || batch < 1) return wfail(NNC_ERR_ARG, "nnc_ws_train: bad arguments");
  // standardize inputs and targets per coordinate over the data set
  for (int c = 0; c < s->n_in; ++c) {
    double mu = 0, sq = 0;
    for (int r = 0; r < N; ++r) mu += U[(size_t)r * s->n_in + c];
    mu /= N;
    for (int r = 0; r < N; ++r) sq += (U[(size_t)r * s->n_in + c] - mu) * (U[(size_t)r * s->n_in + c] - mu);
    s->in_mean[c] = mu;
    s->in_std[c] = std::max(std::sqrt(sq / N), 1e-12);
  }
  for (int c = 0; c < s->n_out; ++c) {
    double mu = 0, sq = 0;
    for (int r = 0; r < N; ++r) mu += Tt[(size_t)r * s->n_out + c];
    mu /= N;
    for (int r = 0; r < N; ++r) sq += (Tt[(size_t)r * s->n_out + c] - mu) * (Tt[(size_t)r * s->n_out + c] - mu);
    s->out_mean[c] = mu;
    s->out_std[c] = std::max(std::sqrt(sq / N), 1e-12);
  }
  // the standardized data set stays on the device; batches are gathered by index
  std::vector<float> hu((size_t)N * s->n_in), ht((size_t)N * s->n_out);
  for (int r = 0; r < N; ++r) {
    for (int c = 0; c < s->n_in; ++c)
      hu[(size_t)r * s->n_in + c] = (float)((U[(size_t)r * s->n_in + c] - s->in_mean[c]) / s->in_std[c]);
    for (int c = 0; c < s->n_out; ++c)
      ht[(size_t)r * s->n_out + c] = (float)((Tt[(size_t)r * s->n_out + c] - s->out_mean[c]) / s->out_std[c]);
  }
  if (N > s->nd) {
    int r = walloc(s, &s->Ud, hu.size());
    if (!r) r = walloc(s, &s->Td, ht.size());
    if (r) return r;
    s->nd = N;
  }
  WCK(cudaMemcpyAsync(s->Ud, hu.data(), sizeof(float) * hu.size(), cudaMemcpyHostToDevice, s->stream));
  WCK(cudaMemcpyAsync(s->Td, ht.data(), sizeof(float) * ht.size(), cudaMemcpyHostToDevice, s->stream));
  const int B = std::min(batch, N);
  int r = ensure_cap(s, B);
  if (r) return r;
  std::mt19937_64 rng(seed);
  std::vector<int> perm(N);
  std::iota(perm.begin(), perm.end(), 0);
  double last = 0.0;
  for (int e = 0; e < epochs; ++e) {
    std::shuffle(perm.begin(), perm.end(), rng);
    for (int b0 = 0; b0 + B <= N; b0 += B) {
      WCK(cudaMemcpyAsync(s->idx, perm.data() + b0, sizeof(int) * B, cudaMemcpyHostToDevice, s->stream));
      const bool want = (e == epochs - 1) && (b0 + 2 * B > N);
      if (s->prec == NNC_FP32) {
        k_ws_gather<float><<<(B * s->n_in + 255) / 256, 256, 0, s->stream>>>(s->Ud, s->idx, B, s->n_in, s->U, (float*)s->Ul);
        k_ws_gather<float><<<(B * s->n_out + 255) / 256, 256, 0, s->stream>>>(s->Td, s->idx, B, s->n_out, s->Tt, (float*)nullptr);
        note_launch(2);
        r = loss_grad<float>(s, B, want ? &last : nullptr);
        adam<float>(s, (float)lr, (float)beta1, (float)beta2, (float)eps);
      } else {
        k_ws_gather<__nv_bfloat16><<<(B * s->n_in + 255) / 256, 256, 0, s->stream>>>(
            s->Ud, s->idx, B, s->n_in, s->U, (__nv_bfloat16*)s->Ul, s->tc ? s->Ut : nullptr, s->cap);
        k_ws_gather<__nv_bfloat16><<<(B * s->n_out + 255) / 256, 256, 0, s->stream>>>(s->Td, s->idx, B, s->n_out, s->Tt, (__nv_bfloat16*)nullptr);
        note_launch(2);
        r = loss_grad<__nv_bfloat16>(s, B, want ? &last : nullptr);
        adam<__nv_bfloat16>(s, (float)lr, (float)beta1, (float)beta2, (float)eps);
      }
      if (r) return r;
    }
  }
  WCK(cudaStreamSynchronize(s->stream));
  WCK(cudaGetLastError());
  r = check_ws_err(s);
  if (r) return r;
  if (final_loss) *final_loss = last;
  return NNC_OK;
}

int nnc_ws_predict(nnc_ws* s, const double* U, int N, double* P) {
  if (!s || !U || !P || N < 1) return wfail(NNC_ERR_ARG, "nnc_ws_predict: bad arguments");
  int r = upload_std(s, U, nullptr, N, false);
  if (r) return r;
  if (s->prec == NNC_FP32) {
    stage_rows<float>(s, s->U, nullptr, N);
    r = forward<float>(s, N);
  } else {
    stage_rows<__nv_bfloat16>(s, s->U, nullptr, N);
    r = forward<__nv_bfloat16>(s, N);
  }
  if (r) return r;
  r = check_ws_err(s);
  if (r) return r;
  std::vector<float> h((size_t)N * s->n_out);
  WCK(cudaMemcpyAsync(h.data(), s->P, sizeof(float) * h.size(), cudaMemcpyDeviceToHost, s->stream));
  WCK(cudaStreamSynchronize(s->stream));
  for (int i = 0; i < N; ++i)
    for (int c = 0; c < s->n_out; ++c)
      P[(size_t)i * s->n_out + c] = h[(size_t)i * s->n_out + c] * s->out_std[c] + s->out_mean[c];
  return NNC_OK;
}

int nnc_ws_get_params(nnc_ws* s, double* const* params) {
  if (!s || !params) return wfail(NNC_ERR_ARG, "bad arguments");
  for (int i = 0; i < 6; ++i) {
    if (!params[i]) continue;
    std::vector<float> h(s->sizes[i]);
    WCK(cudaMemcpyAsync(h.data(), s->w[i], sizeof(float) * s->sizes[i], cudaMemcpyDeviceToHost, s->stream));
    WCK(cudaStreamSynchronize(s->stream));
    for (int j = 0; j < s->sizes[i]; ++j) params[i][j] = h[j];
  }
  return NNC_OK;
}

}  // extern "C"
