// The dense block of the interior-point KKT matrix (Eq. 2) factorized and solved on the GPU.
//
// In the reduced-space formulation the Newton matrix has one dense block, over the network
// inputs x:  K11 = W_DD + diag(sigma_D) + delta_w I  with  W_DD = s H + diag(h_f), where H is the
// n_in x n_in Hessian of lambda^T NN (Eq. 6) that the evaluation leaves in device memory, s its
// sign in the Lagrangian and h_f the objective's diagonal curvature.  The host driver works with
// the bordered matrix [[K11, .], [A_D, 0]] (A_D: the constraint rows restricted to x): a partial
// Cholesky of its leading n_in columns leaves L (K11 = L L^T), the rows Y^T = A_D L^-T and, in the
// bottom block, -A_D K11^-1 A_D^T (the Schur term of the multiplier system).  This file does the
// same on the device, so that neither H nor L leaves it:
//   1. assembly: K11 from H, s and the diagonal terms, scaled symmetrically by D = diag(K11)^-1/2
//      (a congruence: unit diagonal, so that the pivot test is scale-free and FP32 holds the
//      barrier terms of order 1e10 next to entries of order one), A_D scaled by D on the right;
//   2. right-looking blocked Cholesky in FP32 with 32-column panels: every CTA factorizes the
//      32 x 32 diagonal block in one warp's registers (the same arithmetic in every CTA, so all of
//      them take the same positive-definiteness decision), the panel rows below it are solved one
//      row per thread, the trailing lower triangle is updated in 64 x 64 tiles;
//   3. the border rows (Y^T and the bottom block; the scaling cancels there: Y^T = A_D D Lhat^-T,
//      with Lhat the factor of the scaled matrix) go to the host as FP64; L = D^-1 Lhat stays on
//      the device, and the two triangular solves of each Newton step run there
//      (L^-1 b = Lhat^-1 (D b), L^-T y = D Lhat^-T y), one CTA each, by 32-row blocks.
// The factorization is one cooperative launch (every CTA resident) with a grid barrier between
// the phases; every barrier wait is bounded (about two seconds of clock64), after which the
// kernel records an error and returns.  A pivot (before its square root) at or below kPivotMin of
// the unit diagonal means "not positive definite": the host then takes its indefinite paths with
// W_DD copied to it.  FP32 suffices where this is used: in the tensor-core forms H itself carries
// the relative error of its BF16 products, far above the factor's, and the interior-point
// convergence test uses the exact residual and gradient, not the factor.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "common.cuh"

namespace nnc {
void set_last_error(const std::string& msg);

namespace {

constexpr int kNB = 32;          // panel width
constexpr int kTile = 64;        // trailing-update tile
constexpr int kThreads = 256;
constexpr int kMaxGrid = 96;     // CTAs of the factorization (fewer CTAs: cheaper barriers)
constexpr int kSolveThreads = 512;
constexpr float kPivotMin = 1e-5f;
constexpr long long kBarrierCycles = 4000000000LL;   // about two seconds at GB300 clocks

struct KktArgs {
  int nd, m, N, ldp;
  const double* H;     // nd x nd, row stride nd
  double s;
  const double* dvec;  // nd: h_f + sigma + delta_w (+ eliminated pinning rows)
  const double* AD;    // m x nd
  double* sc;          // nd: D = diag(K11)^-1/2 (1 where the diagonal is not positive)
  float* A;            // N x ldp working matrix (lower triangle)
  double* border;      // m x N FP64: rows nd .. N-1 of the result
  int* flags;          // [0]: 1 + index of a failed pivot (0: positive definite), [1]: timeout
  unsigned* bar;       // [0]: arrivals, [1]: generation
};

// Grid barrier (generation counter): every CTA arrives once; the last one resets the arrival
// count and advances the generation.  Bounded: on expiry the CTA records the timeout and the
// caller returns.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* flags, volatile int* abort_sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (clock64() - t0 > kBarrierCycles) {
          atomicExch(flags + 1, 1);
          *abort_sh = 1;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *abort_sh == 0;
}

__global__ void __launch_bounds__(kThreads) k_kkt_chol(const KktArgs a) {
  __shared__ float Ls[kNB][kNB + 1];
  __shared__ float dinv[kNB];
  __shared__ float P[kTile][kNB + 1];
  __shared__ float Q[kTile][kNB + 1];
  __shared__ volatile int abort_sh;
  __shared__ int fail_sh;
  if (threadIdx.x == 0) abort_sh = 0;
  __syncthreads();
  const int nd = a.nd, N = a.N, ldp = a.ldp;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int gthreads = gridDim.x * blockDim.x;

  // 0. the scaling
  for (int i = gtid; i < nd; i += gthreads) {
    const double d = a.s * __ldcg(a.H + (size_t)i * nd + i) + __ldcg(a.dvec + i);
    __stcg(a.sc + i, d > 0.0 ? 1.0 / sqrt(d) : 1.0);
  }
  if (!grid_barrier(a.bar, a.flags, &abort_sh)) return;
  // 1. assembly of the scaled bordered matrix (lower triangle), a row per warp
  {
    const int warp = gtid >> 5, lane = threadIdx.x & 31, nwarps = gthreads >> 5;
    for (int i = warp; i < N; i += nwarps) {
      float* row = a.A + (size_t)i * ldp;
      if (i < nd) {
        const double si = __ldcg(a.sc + i);
        const double* h = a.H + (size_t)i * nd;
        for (int j = lane; j <= i; j += 32) {
          double v = a.s * __ldcg(h + j);
          if (i == j) v += __ldcg(a.dvec + i);
          __stcg(row + j, (float)(v * si * __ldcg(a.sc + j)));
        }
      } else {
        const double* ad = a.AD + (size_t)(i - nd) * nd;
        for (int j = lane; j <= i; j += 32)
          __stcg(row + j, j < nd ? (float)(__ldcg(ad + j) * __ldcg(a.sc + j)) : 0.f);
      }
    }
  }
  if (!grid_barrier(a.bar, a.flags, &abort_sh)) return;

  for (int kb = 0; kb < nd; kb += kNB) {
    const int nb = min(kNB, nd - kb);
    const int k1 = kb + nb;
    // 2a. diagonal block in warp 0's registers: lane r holds row r
    if (threadIdx.x == 0) fail_sh = 0;
    if (threadIdx.x < 32) {
      const int r = threadIdx.x;
      float v[kNB];
#pragma unroll
      for (int c = 0; c < kNB; ++c)
        v[c] = (r < nb && c <= r) ? __ldcg(a.A + (size_t)(kb + r) * ldp + kb + c) : (c == r ? 1.f : 0.f);
      int fail = 0;
      float mydiag = 1.f;   // L_rr (no dynamic index into v: it stays in registers)
#pragma unroll 32
      for (int j = 0; j < kNB; ++j) {
        const float piv = __shfl_sync(0xffffffffu, v[j], j);
        if (j < nb && !fail && !(piv > kPivotMin)) fail = kb + j + 1;
        const float d = sqrtf(fmaxf(piv, kPivotMin));
        if (r == j) mydiag = d;
        const float l = (r > j) ? v[j] / d : (r == j ? d : 0.f);
        v[j] = l;
#pragma unroll 31
        for (int k = j + 1; k < kNB; ++k) {
          const float lk = __shfl_sync(0xffffffffu, l, k);
          v[k] = (r >= k) ? v[k] - l * lk : v[k];
        }
      }
#pragma unroll
      for (int c = 0; c < kNB; ++c) Ls[r][c] = v[c];
      dinv[r] = 1.f / mydiag;
      if (r == 0) fail_sh = fail;
    }
    __syncthreads();
    if (fail_sh) {   // the same decision in every CTA
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(a.flags, fail_sh);
      return;
    }
    // 2b. panel rows below the block: x L11^T = a, one row per thread (right-looking)
    for (int i = k1 + gtid; i < N; i += gthreads) {
      float x[kNB];
      float* row = a.A + (size_t)i * ldp + kb;
#pragma unroll
      for (int k = 0; k < kNB; ++k) x[k] = k < nb ? __ldcg(row + k) : 0.f;
#pragma unroll
      for (int j = 0; j < kNB; ++j) {
        x[j] *= dinv[j];
#pragma unroll
        for (int k = j + 1; k < kNB; ++k) x[k] -= x[j] * Ls[k][j];
      }
#pragma unroll
      for (int k = 0; k < kNB; ++k)
        if (k < nb) __stcg(row + k, x[k]);
    }
    if (!grid_barrier(a.bar, a.flags, &abort_sh)) return;
    // the factored diagonal block goes back now that no CTA reads it any more (every CTA loaded
    // it before the barrier; the trailing update reads only rows >= k1)
    if (blockIdx.x == 0)
      for (int e = threadIdx.x; e < nb * kNB; e += blockDim.x) {
        const int r = e / kNB, c = e % kNB;
        if (c <= r) __stcg(a.A + (size_t)(kb + r) * ldp + kb + c, Ls[r][c]);
      }
    // 2c. trailing update of the lower triangle of rows / columns [k1, N)
    const int T = (N - k1 + kTile - 1) / kTile;
    const int ntiles = T * (T + 1) / 2;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      int I = (int)((sqrtf(8.f * t + 1.f) - 1.f) * 0.5f);
      while ((I + 1) * (I + 2) / 2 <= t) ++I;
      while (I * (I + 1) / 2 > t) --I;
      const int J = t - I * (I + 1) / 2;
      const int r0 = k1 + I * kTile, c0 = k1 + J * kTile;
      __syncthreads();
      for (int e = threadIdx.x; e < kTile * kNB; e += blockDim.x) {
        const int r = e / kNB, k = e % kNB;
        P[r][k] = (k < nb && r0 + r < N) ? __ldcg(a.A + (size_t)(r0 + r) * ldp + kb + k) : 0.f;
        Q[r][k] = (k < nb && c0 + r < N) ? __ldcg(a.A + (size_t)(c0 + r) * ldp + kb + k) : 0.f;
      }
      __syncthreads();
      float acc[4][4] = {};
#pragma unroll 8
      for (int k = 0; k < kNB; ++k) {
        float p[4], q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          p[u] = P[ty * 4 + u][k];
          q[u] = Q[tx * 4 + u][k];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int w = 0; w < 4; ++w) acc[u][w] += p[u] * q[w];
      }
      // all loads of the tile's old values first, then the stores (no load waits behind a store)
      float old[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = r0 + ty * 4 + u;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int j = c0 + tx * 4 + w;
          old[u][w] = (i < N && j <= i) ? __ldcg(a.A + (size_t)i * ldp + j) : 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = r0 + ty * 4 + u;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int j = c0 + tx * 4 + w;
          if (i < N && j <= i) __stcg(a.A + (size_t)i * ldp + j, old[u][w] - acc[u][w]);
        }
      }
    }
    if (!grid_barrier(a.bar, a.flags, &abort_sh)) return;
  }
  // 3. the border rows as FP64 (Y^T in the first nd columns, the bottom block after them)
  for (int e = gtid; e < a.m * N; e += gthreads) {
    const int r = e / N, j = e % N;
    const int i = nd + r;
    a.border[e] = j <= i ? (double)__ldcg(a.A + (size_t)i * ldp + j) : 0.0;
  }
}

// Triangular solves with L = D^-1 Lhat (Lhat: the FP32 factor in A, row stride ldp), one CTA of
// kSolveThreads: lower: x = L^-1 b = Lhat^-1 (D b); upper: x = L^-T b = D (Lhat^-T b).  By 32-row
// blocks: warp 0 solves the diagonal block with shuffles, then every thread updates its rows.
__global__ void __launch_bounds__(kSolveThreads, 1) k_kkt_lower(const float* __restrict__ A, int ldp,
                                                             int n, const double* __restrict__ sc,
                                                             double* __restrict__ xio) {
  extern __shared__ float xs[];   // n
  __shared__ float xb[kNB];
  for (int i = threadIdx.x; i < n; i += blockDim.x) xs[i] = (float)(xio[i] * sc[i]);
  __syncthreads();
  for (int kb = 0; kb < n; kb += kNB) {
    const int nb = min(kNB, n - kb);
    if (threadIdx.x < 32) {
      // lane r holds row r of the diagonal block and t_r
      const int r = threadIdx.x;
      float lrow[kNB];
#pragma unroll
      for (int c = 0; c < kNB; ++c)
        lrow[c] = (r < nb && c <= r) ? A[(size_t)(kb + r) * ldp + kb + c] : (c == r ? 1.f : 0.f);
      float t = r < nb ? xs[kb + r] : 0.f;
#pragma unroll 32
      for (int j = 0; j < kNB; ++j) {
        if (j < nb) {   // uniform over the warp
          const float xj = __shfl_sync(0xffffffffu, t / lrow[j], j);   // lane j: t_j / L_jj
          t = (r == j) ? xj : (r > j) ? t - lrow[j] * xj : t;
        }
      }
      if (r < nb) {
        xb[r] = t;
        xs[kb + r] = t;
      }
    }
    __syncthreads();
    for (int i = kb + nb + threadIdx.x; i < n; i += blockDim.x) {
      const float* li = A + (size_t)i * ldp + kb;
      float s = xs[i];
#pragma unroll 8
      for (int k = 0; k < nb; ++k) s -= li[k] * xb[k];
      xs[i] = s;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) xio[i] = (double)xs[i];
}

__global__ void __launch_bounds__(kSolveThreads, 1) k_kkt_upper(const float* __restrict__ A, int ldp,
                                                             int n, const double* __restrict__ sc,
                                                             double* __restrict__ xio) {
  extern __shared__ float xs[];   // n
  __shared__ float xb[kNB];
  for (int i = threadIdx.x; i < n; i += blockDim.x) xs[i] = (float)xio[i];
  __syncthreads();
  const int nblk = (n + kNB - 1) / kNB;
  for (int b = nblk - 1; b >= 0; --b) {
    const int kb = b * kNB, nb = min(kNB, n - kb);
    if (threadIdx.x < 32) {
      // Lhat_BB^T x_B = z_B, backwards: x_j = z_j / L_jj, then z_i -= L_ji x_j for i < j; lane r
      // holds column r of the diagonal block (lcol[j] = L_jr, j >= r) and t_r
      const int r = threadIdx.x;
      float lcol[kNB];
#pragma unroll
      for (int j = 0; j < kNB; ++j)
        lcol[j] = (r < nb && j < nb && j >= r) ? A[(size_t)(kb + j) * ldp + kb + r] : (j == r ? 1.f : 0.f);
      float t = r < nb ? xs[kb + r] : 0.f;
#pragma unroll 32
      for (int j = kNB - 1; j >= 0; --j) {
        if (j < nb) {   // uniform over the warp
          const float xj = __shfl_sync(0xffffffffu, t / lcol[j], j);   // lane j: t_j / L_jj
          t = (r == j) ? xj : (r < j) ? t - lcol[j] * xj : t;
        }
      }
      if (r < nb) {
        xb[r] = t;
        xs[kb + r] = t;
      }
    }
    __syncthreads();
    // z_i -= sum_{k in B} Lhat_ki x_k for i < kb (column segments of the block's rows)
    for (int i = threadIdx.x; i < kb; i += blockDim.x) {
      float s = xs[i];
#pragma unroll 8
      for (int k = 0; k < nb; ++k) s -= A[(size_t)(kb + k) * ldp + i] * xb[k];
      xs[i] = s;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) xio[i] = (double)xs[i] * sc[i];
}

// u = H x (FP64, one warp per row)
__global__ void k_kkt_matvec(const double* __restrict__ H, int n, const double* __restrict__ x,
                             double* __restrict__ u) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* h = H + (size_t)row * n;
  double acc = 0.0;
  for (int j = lane; j < n; j += 32) acc = fma(h[j], x[j], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) u[row] = acc;
}

// max |s H_ij + [i == j] h_i| over the matrix (non-negative doubles order like their bits)
__global__ void k_kkt_maxabs(const double* __restrict__ H, int n, double s,
                             const double* __restrict__ h, unsigned long long* out) {
  double mx = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)n * n;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    double v = s * H[e];
    if (i == j) v += h[i];
    mx = fmax(mx, fabs(v));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

}  // namespace

// ---------------------------------------------------------------- host side
struct DenseKktDev {
  int nd = 0, mmax = 0, ldp = 0, grid = 0, device = 0, m = 0;
  cudaStream_t st = nullptr;
  float* A = nullptr;
  double* sc = nullptr;
  double* border = nullptr;
  double* dvec = nullptr;
  double* AD = nullptr;
  double* vec = nullptr;        // nd: matvec / solve vector
  double* res = nullptr;        // nd: matvec output
  unsigned long long* mx = nullptr;
  int* flags = nullptr;
  unsigned* bar = nullptr;
  double* host_out = nullptr;   // pinned (nd + mmax)^2: the border rows at their offsets
  double* host_vec = nullptr;   // pinned 2 nd + 2
};

namespace {
bool ck(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return true;
  set_last_error(std::string("kkt on device: ") + what + ": " + cudaGetErrorString(e));
  return false;
}
}  // namespace

void dkkt_free(DenseKktDev* d) {
  if (!d) return;
  if (d->st) cudaStreamSynchronize(d->st);
  cudaFree(d->A);
  cudaFree(d->sc);
  cudaFree(d->border);
  cudaFree(d->dvec);
  cudaFree(d->AD);
  cudaFree(d->vec);
  cudaFree(d->res);
  cudaFree(d->mx);
  cudaFree(d->flags);
  cudaFree(d->bar);
  cudaFreeHost(d->host_out);
  cudaFreeHost(d->host_vec);
  delete d;
}

// Buffers for a dense block of nd rows with up to mmax border rows, on the current device.
DenseKktDev* dkkt_create(int nd, int mmax, cudaStream_t st) {
  DenseKktDev* d = new DenseKktDev;
  d->nd = nd;
  d->mmax = mmax;
  d->st = st;
  const int N = nd + mmax;
  d->ldp = (N + 3) / 4 * 4;
  cudaGetDevice(&d->device);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d->device);
  d->grid = std::max(1, std::min(sms, kMaxGrid));
  bool ok = ck(cudaMalloc(&d->A, sizeof(float) * (size_t)N * d->ldp), "alloc") &&
            ck(cudaMalloc(&d->sc, sizeof(double) * std::max(nd, 1)), "alloc") &&
            ck(cudaMalloc(&d->border, sizeof(double) * (size_t)std::max(mmax, 1) * N), "alloc") &&
            ck(cudaMalloc(&d->dvec, sizeof(double) * nd), "alloc") &&
            ck(cudaMalloc(&d->AD, sizeof(double) * (size_t)std::max(mmax, 1) * nd), "alloc") &&
            ck(cudaMalloc(&d->vec, sizeof(double) * nd), "alloc") &&
            ck(cudaMalloc(&d->res, sizeof(double) * nd), "alloc") &&
            ck(cudaMalloc(&d->mx, sizeof(unsigned long long)), "alloc") &&
            ck(cudaMalloc(&d->flags, sizeof(int) * 2), "alloc") &&
            ck(cudaMalloc(&d->bar, sizeof(unsigned) * 2), "alloc") &&
            ck(cudaMallocHost(&d->host_out, sizeof(double) * (size_t)N * N), "pinned alloc") &&
            ck(cudaMallocHost(&d->host_vec, sizeof(double) * (2 * (size_t)nd + 2 + (size_t)std::max(mmax, 1) * nd)),
               "pinned alloc") &&
            ck(cudaMemsetAsync(d->bar, 0, sizeof(unsigned) * 2, st), "memset") &&
            ck(cudaFuncSetAttribute(k_kkt_lower, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(sizeof(float) * std::max(nd, 1))), "attribute") &&
            ck(cudaFuncSetAttribute(k_kkt_upper, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(sizeof(float) * std::max(nd, 1))), "attribute");
  if (!ok) {
    dkkt_free(d);
    return nullptr;
  }
  return d;
}

// max |W_DD| with W_DD = s H + diag(hf) (hf: nd host doubles).  Returns NNC_OK or an error.
int dkkt_maxabs(DenseKktDev* d, const double* H, double s, const double* hf, double* out) {
  std::copy(hf, hf + d->nd, d->host_vec);
  if (!ck(cudaMemcpyAsync(d->dvec, d->host_vec, sizeof(double) * d->nd, cudaMemcpyHostToDevice, d->st), "copy") ||
      !ck(cudaMemsetAsync(d->mx, 0, sizeof(unsigned long long), d->st), "memset"))
    return NNC_ERR_CUDA;
  k_kkt_maxabs<<<148, 256, 0, d->st>>>(H, d->nd, s, d->dvec, d->mx);
  note_launch();
  unsigned long long bits = 0;
  if (!ck(cudaGetLastError(), "launch") ||
      !ck(cudaMemcpyAsync(d->host_vec, d->mx, sizeof(bits), cudaMemcpyDeviceToHost, d->st), "copy") ||
      !ck(cudaStreamSynchronize(d->st), "sync"))
    return NNC_ERR_CUDA;
  std::memcpy(&bits, d->host_vec, sizeof(bits));
  double v;
  std::memcpy(&v, &bits, sizeof(v));
  *out = v;
  return NNC_OK;
}

// u = H x (host vectors of nd doubles).
int dkkt_matvec(DenseKktDev* d, const double* H, const double* x, double* u) {
  std::copy(x, x + d->nd, d->host_vec);
  if (!ck(cudaMemcpyAsync(d->vec, d->host_vec, sizeof(double) * d->nd, cudaMemcpyHostToDevice, d->st), "copy"))
    return NNC_ERR_CUDA;
  k_kkt_matvec<<<(d->nd * 32 + 255) / 256, 256, 0, d->st>>>(H, d->nd, d->vec, d->res);
  note_launch();
  if (!ck(cudaGetLastError(), "launch") ||
      !ck(cudaMemcpyAsync(d->host_vec + d->nd, d->res, sizeof(double) * d->nd, cudaMemcpyDeviceToHost, d->st), "copy") ||
      !ck(cudaStreamSynchronize(d->st), "sync"))
    return NNC_ERR_CUDA;
  std::copy(d->host_vec + d->nd, d->host_vec + 2 * d->nd, u);
  return NNC_OK;
}

// Partial Cholesky of the bordered matrix [[s H + diag(dvec), .], [AD, 0]] (nd + m rows) on the
// device.  On NNC_OK, *pd says whether the dense block was positive definite; if so, *result
// points to a pinned host array with the layout of the host factorization (row-major, row
// stride nd + m) of which only the border rows are filled: Y^T = A_D L^-T in the first nd columns
// of rows nd .., -A_D K11^-1 A_D^T after them (lower triangle), valid until the next call.  L
// stays on the device for dkkt_solve_lower / dkkt_solve_upper.
int dkkt_factor(DenseKktDev* d, const double* H, double s, const double* dvec, const double* AD,
                int m, bool* pd, const double** result) {
  const int nd = d->nd, N = nd + m;
  if (m > d->mmax) {
    set_last_error("kkt on device: more border rows than allocated");
    return NNC_ERR_ARG;
  }
  double* hv = d->host_vec;
  std::copy(dvec, dvec + nd, hv);
  if (m > 0) std::copy(AD, AD + (size_t)m * nd, hv + 2 * (size_t)nd + 2);
  if (!ck(cudaMemcpyAsync(d->dvec, hv, sizeof(double) * nd, cudaMemcpyHostToDevice, d->st), "copy"))
    return NNC_ERR_CUDA;
  if (m > 0 && !ck(cudaMemcpyAsync(d->AD, hv + 2 * (size_t)nd + 2, sizeof(double) * (size_t)m * nd,
                                   cudaMemcpyHostToDevice, d->st), "copy"))
    return NNC_ERR_CUDA;
  if (!ck(cudaMemsetAsync(d->flags, 0, sizeof(int) * 2, d->st), "memset")) return NNC_ERR_CUDA;
  KktArgs args{nd, m, N, d->ldp, H, s, d->dvec, d->AD, d->sc, d->A, d->border, d->flags, d->bar};
  void* kargs[] = {&args};
  if (!ck(cudaLaunchCooperativeKernel((const void*)k_kkt_chol, dim3(d->grid), dim3(kThreads), kargs, 0, d->st),
          "cooperative launch"))
    return NNC_ERR_CUDA;
  note_launch();
  int* fl = (int*)(hv + nd);
  if (!ck(cudaMemcpyAsync(fl, d->flags, sizeof(int) * 2, cudaMemcpyDeviceToHost, d->st), "copy"))
    return NNC_ERR_CUDA;
  double* out_border = d->host_out + (size_t)nd * N;
  if (m > 0 && !ck(cudaMemcpyAsync(out_border, d->border, sizeof(double) * (size_t)m * N,
                                   cudaMemcpyDeviceToHost, d->st), "copy"))
    return NNC_ERR_CUDA;
  if (!ck(cudaStreamSynchronize(d->st), "sync")) return NNC_ERR_CUDA;
  if (fl[1]) {
    cudaMemsetAsync(d->bar, 0, sizeof(unsigned) * 2, d->st);
    set_last_error("kkt on device: a bounded grid-barrier wait ran out");
    return NNC_ERR_TIMEOUT;
  }
  d->m = m;
  *pd = fl[0] == 0;
  if (*pd) *result = d->host_out;
  return NNC_OK;
}

// x (nd host doubles) <- L^-1 x (lower != 0) or L^-T x with the last factorization's L.
int dkkt_solve(DenseKktDev* d, double* x, int lower) {
  const int nd = d->nd;
  std::copy(x, x + nd, d->host_vec);
  if (!ck(cudaMemcpyAsync(d->vec, d->host_vec, sizeof(double) * nd, cudaMemcpyHostToDevice, d->st), "copy"))
    return NNC_ERR_CUDA;
  const size_t smem = sizeof(float) * nd;
  if (lower) k_kkt_lower<<<1, kSolveThreads, smem, d->st>>>(d->A, d->ldp, nd, d->sc, d->vec);
  else k_kkt_upper<<<1, kSolveThreads, smem, d->st>>>(d->A, d->ldp, nd, d->sc, d->vec);
  note_launch();
  if (!ck(cudaGetLastError(), "launch") ||
      !ck(cudaMemcpyAsync(d->host_vec, d->vec, sizeof(double) * nd, cudaMemcpyDeviceToHost, d->st), "copy") ||
      !ck(cudaStreamSynchronize(d->st), "sync"))
    return NNC_ERR_CUDA;
  std::copy(d->host_vec, d->host_vec + nd, x);
  return NNC_OK;
}

}  // namespace nnc
