// CUDA-core GEMMs of the FP64 and FP32 forms: the forward tangent sweep of the Hessian
// (Zdot_l = W_l Adot_{l-1}, n_in tangent columns) and the per-layer symmetric product
// H += Zdot_l^T diag(c_l) Zdot_l.  GB300's FP64 rate is low, so the FP64 form is the accuracy
// reference of the GPU path rather than its fast path; the kernel is a plain shared-memory
// tiled GEMM with register micro-tiles.
#include "kernels.cuh"

namespace nnc {

enum { EPI_TANGENT = 0, EPI_SYRK = 1 };

// D[m][n] = sum_k A[m][k] B[n][k] on a (16*TM) x (16*TN) tile with 256 threads; thread (tx, ty)
// owns rows m0 + tx + 16 i and columns n0 + ty + 16 j.  K must be a multiple of 16 (all
// packed dimensions are multiples of 128).
template <typename T, int TM, int TN, int EPI>
__global__ void __launch_bounds__(256) k_simt_gemm(const T* __restrict__ A, int lda,
                                                   const T* __restrict__ B, int ldb, int M, int N,
                                                   int K, int k_per_split,
                                                   const double* __restrict__ s1,
                                                   const double* __restrict__ c,
                                                   T* __restrict__ At, T* __restrict__ Zt,
                                                   T* __restrict__ Yt, int ldo, int ldz,
                                                   double* __restrict__ Hp) {
  constexpr int BM = 16 * TM, BN = 16 * TN, BK = 16;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int bm = blockIdx.y, bn = blockIdx.x, split = blockIdx.z;
  if (EPI == EPI_SYRK && bn > bm) return;  // upper-triangle tiles are mirrored at the end
  const int m0 = bm * BM, n0 = bn * BN;
  const int kbeg = split * k_per_split;
  const int kend = min(K, kbeg + k_per_split);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    for (int i = threadIdx.x; i < BM * BK; i += 256) {
      const int r = i >> 4, kk = i & 15;
      const int gm = m0 + r;
      As[kk][r] = gm < M ? A[(size_t)gm * lda + k0 + kk] : T(0);
    }
    for (int i = threadIdx.x; i < BN * BK; i += 256) {
      const int r = i >> 4, kk = i & 15;
      const int gn = n0 + r;
      Bs[kk][r] = gn < N ? B[(size_t)gn * ldb + k0 + kk] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

  if (EPI == EPI_TANGENT) {
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int m = m0 + tx + 16 * i;
      if (m >= M) continue;
      const double sm = s1[m], cm = c[m];
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int n = n0 + ty + 16 * j;
        if (n >= N) continue;
        const double v = (double)acc[i][j];
        if (At) At[(size_t)n * ldo + m] = (T)(sm * v);
        if (Zt) {
          const size_t oz = (size_t)n * ldz + m;
          Zt[oz] = (T)v;
          Yt[oz] = (T)(cm * v);
        }
      }
    }
  } else {
    double* hp = Hp + (size_t)split * M * N;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int m = m0 + tx + 16 * i;
      if (m >= M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int n = n0 + ty + 16 * j;
        if (n >= N) continue;
        hp[(size_t)m * N + n] += (double)acc[i][j];
      }
    }
  }
}

cudaError_t launch_simt_tangent(bool fp64, const void* A, int lda, const void* B, int ldb, int M,
                                int N, int K, const double* s1, const double* c, void* At, int ldo,
                                void* Zt, void* Yt, int ldz, cudaStream_t st) {
  if (fp64) {
    dim3 grid((N + 63) / 64, (M + 63) / 64, 1);
    k_simt_gemm<double, 4, 4, EPI_TANGENT><<<grid, 256, 0, st>>>(
        (const double*)A, lda, (const double*)B, ldb, M, N, K, K, s1, c, (double*)At, (double*)Zt,
        (double*)Yt, ldo, ldz, nullptr);
  } else {
    dim3 grid((N + 127) / 128, (M + 127) / 128, 1);
    k_simt_gemm<float, 8, 8, EPI_TANGENT><<<grid, 256, 0, st>>>(
        (const float*)A, lda, (const float*)B, ldb, M, N, K, K, s1, c, (float*)At, (float*)Zt,
        (float*)Yt, ldo, ldz, nullptr);
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_simt_syrk(bool fp64, const void* Zt, const void* Yt, int ld, int n, int K,
                             int splits, double* Hp, cudaStream_t st) {
  const int kps = ((K + splits - 1) / splits + 15) / 16 * 16;
  if (fp64) {
    dim3 grid((n + 63) / 64, (n + 63) / 64, splits);
    k_simt_gemm<double, 4, 4, EPI_SYRK><<<grid, 256, 0, st>>>(
        (const double*)Zt, ld, (const double*)Yt, ld, n, n, K, kps, nullptr, nullptr, nullptr,
        nullptr, nullptr, 0, 0, Hp);
  } else {
    dim3 grid((n + 127) / 128, (n + 127) / 128, splits);
    k_simt_gemm<float, 8, 8, EPI_SYRK><<<grid, 256, 0, st>>>(
        (const float*)Zt, ld, (const float*)Yt, ld, n, n, K, kps, nullptr, nullptr, nullptr,
        nullptr, nullptr, 0, 0, Hp);
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace nnc
