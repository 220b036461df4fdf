// Bandwidth-bound kernels of libnnc: the forward value pass (Eq. 3), the reverse sweep with
// n_out (+1) seed columns that gives the Jacobian and the adjoints, the first-layer tangents,
// and the small reductions around them.  All read weights once, coalesced and vectorised.
#include <type_traits>

#include "async.cuh"
#include "kernels.cuh"

namespace nnc {

// ------------------------------------------------------------------ forward value pass
// One warp per output row.  FP32 weights are multiplied in FP32 with four independent
// partial sums per lane (32 terms each for k = 4096), which are summed in FP64.
template <typename TW>
__global__ void __launch_bounds__(256) k_gemv_fwd(const TW* __restrict__ W, int ldw,
                                                  const double* __restrict__ bias,
                                                  const void* __restrict__ a_in_v, int m, int k,
                                                  int act, double* __restrict__ a_out,
                                                  float* __restrict__ a_out_f,
                                                  double* __restrict__ s1, double* __restrict__ s2) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= m) return;
  double acc;
  if constexpr (std::is_same<TW, float>::value) {
    // FP32 weights meet the FP32 copy of the activations (no FP64 conversions in the loop).
    const float4* r4 = reinterpret_cast<const float4*>(W + (size_t)row * ldw);
    const float4* a4 = reinterpret_cast<const float4*>(a_in_v);
    const int nk4 = (k + 3) >> 2;
    float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll 8
    for (int j = lane; j < nk4; j += 32) {
      const float4 w = __ldg(r4 + j);
      const float4 a = a4[j];
      p0 = fmaf(w.x, a.x, p0);
      p1 = fmaf(w.y, a.y, p1);
      p2 = fmaf(w.z, a.z, p2);
      p3 = fmaf(w.w, a.w, p3);
    }
    acc = ((double)p0 + (double)p1) + ((double)p2 + (double)p3);
  } else {
    const double2* r2 = reinterpret_cast<const double2*>(W + (size_t)row * ldw);
    const double* a_in = reinterpret_cast<const double*>(a_in_v);
    const int nk2 = (k + 1) >> 1;
    double q0 = 0.0, q1 = 0.0;
#pragma unroll 4
    for (int j = lane; j < nk2; j += 32) {
      const double2 w = __ldg(r2 + j);
      const double2 a = *reinterpret_cast<const double2*>(a_in + 2 * j);
      q0 = fma(w.x, a.x, q0);
      q1 = fma(w.y, a.y, q1);
    }
    acc = q0 + q1;
  }
  acc = warp_sum(acc);
  if (lane == 0) {
    const double z = acc + (bias ? bias[row] : 0.0);
    double a, d1, d2;
    act_eval(act, z, a, d1, d2);
    a_out[row] = a;
    if (a_out_f) a_out_f[row] = (float)a;
    if (s1) s1[row] = d1;
    if (s2) s2[row] = d2;
  }
}

cudaError_t launch_gemv_fwd(bool fp64, const void* W, int ldw, const double* b, const void* a_in,
                            int m, int k, int act, double* a_out, float* a_out_f, double* s1,
                            double* s2, cudaStream_t st) {
  const int threads = 256;
  const int blocks = (m * 32 + threads - 1) / threads;
  if (fp64)
    k_gemv_fwd<double><<<blocks, threads, 0, st>>>((const double*)W, ldw, b, a_in, m, k, act, a_out,
                                                   a_out_f, s1, s2);
  else
    k_gemv_fwd<float><<<blocks, threads, 0, st>>>((const float*)W, ldw, b, a_in, m, k, act, a_out,
                                                  a_out_f, s1, s2);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ reverse sweep
// part[c][kk][s] = sum_{r in chunk c} W[r][kk] * Zbar[r][s]: the transposed product W^T Zbar of
// one reverse step.  A block of 256 threads covers 256 * VEC adjacent columns (VEC = 4 floats
// or 2 doubles per 16-byte load) and one chunk of kRevRows rows, whose seeds are staged in
// shared memory; many small blocks keep enough loads in flight to stream W at HBM rate.  FP32
// weights run in FP32 (seeds rounded to FP32), FP64 weights in FP64; partial sums are written
// in the same type and summed over chunks by k_rev_reduce.
constexpr int kRevRows = 64;     // rows per chunk
constexpr int kRevThreads = 256;

template <typename TW>
struct RevVec;
template <>
struct RevVec<float> {
  static constexpr int V = 4;
  __device__ static void load(const float* p, float (&w)[4]) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
  }
};
template <>
struct RevVec<double> {
  static constexpr int V = 2;
  __device__ static void load(const double* p, double (&w)[2]) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    w[0] = v.x; w[1] = v.y;
  }
};

template <typename TW, int SMAX>
__global__ void __launch_bounds__(kRevThreads) k_gemv_rev(const TW* __restrict__ W, int ldw, int m,
                                                          int kcols, const double* __restrict__ Zbar,
                                                          int S, TW* __restrict__ part) {
  constexpr int V = RevVec<TW>::V;
  __shared__ TW zs[kRevRows][SMAX];
  const int c0 = (blockIdx.x * kRevThreads + threadIdx.x) * V;
  const int r0 = blockIdx.y * kRevRows;
  const int nr = min(kRevRows, m - r0);
  for (int i = threadIdx.x; i < kRevRows * SMAX; i += kRevThreads) {
    const int r = i / SMAX, s = i % SMAX;
    zs[r][s] = (r < nr && s < S) ? (TW)Zbar[(size_t)(r0 + r) * S + s] : TW(0);
  }
  __syncthreads();
  if (c0 >= kcols) return;  // kcols is a multiple of 128, so a thread's V columns are all valid
  TW acc[V][SMAX];
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int s = 0; s < SMAX; ++s) acc[v][s] = TW(0);
  const TW* wp = W + (size_t)r0 * ldw + c0;
#pragma unroll 4
  for (int r = 0; r < nr; ++r) {
    TW w[V];
    RevVec<TW>::load(wp + (size_t)r * ldw, w);
#pragma unroll
    for (int s = 0; s < SMAX; ++s) {
      const TW z = zs[r][s];
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v][s] = fma(w[v], z, acc[v][s]);
    }
  }
  TW* out = part + ((size_t)blockIdx.y * kcols + c0) * S;
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int s = 0; s < SMAX; ++s)
      if (s < S) out[v * S + s] = acc[v][s];
}

int rev_chunks(int m, int kcols, int sm_count) {
  (void)kcols;
  (void)sm_count;
  return (m + kRevRows - 1) / kRevRows;
}

template <typename TW>
static void rev_dispatch(const TW* W, int ldw, int m, int kcols, const double* Zbar, int S,
                         int chunks, TW* part, cudaStream_t st) {
  constexpr int V = RevVec<TW>::V;
  dim3 grid((kcols + kRevThreads * V - 1) / (kRevThreads * V), chunks);
  if (S <= 1)
    k_gemv_rev<TW, 1><<<grid, kRevThreads, 0, st>>>(W, ldw, m, kcols, Zbar, S, part);
  else if (S <= 4)
    k_gemv_rev<TW, 4><<<grid, kRevThreads, 0, st>>>(W, ldw, m, kcols, Zbar, S, part);
  else if (S <= 12)
    k_gemv_rev<TW, 12><<<grid, kRevThreads, 0, st>>>(W, ldw, m, kcols, Zbar, S, part);
  else if (S <= 24)
    k_gemv_rev<TW, 24><<<grid, kRevThreads, 0, st>>>(W, ldw, m, kcols, Zbar, S, part);
  else
    k_gemv_rev<TW, 48><<<grid, kRevThreads, 0, st>>>(W, ldw, m, kcols, Zbar, S, part);
}

cudaError_t launch_gemv_rev(bool fp64, const void* W, int ldw, int m, int kcols, const double* Zbar,
                            int S, int chunks, void* part, cudaStream_t st) {
  if (S > 48) return cudaErrorInvalidValue;
  if (fp64)
    rev_dispatch<double>((const double*)W, ldw, m, kcols, Zbar, S, chunks, (double*)part, st);
  else
    rev_dispatch<float>((const float*)W, ldw, m, kcols, Zbar, S, chunks, (float*)part, st);
  note_launch();
  return cudaGetLastError();
}

template <typename TP>
__global__ void k_rev_reduce(const TP* __restrict__ part, int chunks, int kcols, int kvalid,
                             int S, const double* __restrict__ s1, const double* __restrict__ s2,
                             int lam_col, int nJ, double* __restrict__ Zbar_out,
                             double* __restrict__ c_out, float* __restrict__ c_out_f,
                             double* __restrict__ J_out, double* __restrict__ g_out) {
  async::griddep_launch();  // the next layer's streaming kernel may start fetching its weights
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kcols * S) return;
  const int kk = idx / S, s = idx % S;
  double v = 0.0;
  const size_t stride = (size_t)kcols * S;
  const TP* pp = part + idx;
#pragma unroll 8
  for (int c = 0; c < chunks; ++c) v += (double)pp[c * stride];
  if (Zbar_out) Zbar_out[idx] = s1 ? s1[kk] * v : v;
  if (s == lam_col) {
    if (c_out) c_out[kk] = s2[kk] * v;
    if (c_out_f) c_out_f[kk] = (float)(s2[kk] * v);
    if (g_out && kk < kvalid) g_out[kk] = v;
  }
  if (J_out && s < nJ && kk < kvalid) J_out[(size_t)s * kvalid + kk] = v;
}

cudaError_t launch_rev_reduce(bool fp64, const void* part, int chunks, int kcols, int kvalid, int S,
                              const double* s1, const double* s2, int lam_col, int nJ,
                              double* Zbar_out, double* c_out, float* c_out_f, double* J_out,
                              double* g_out, cudaStream_t st) {
  const int total = kcols * S;
  if (fp64)
    k_rev_reduce<double><<<(total + 255) / 256, 256, 0, st>>>(
        (const double*)part, chunks, kcols, kvalid, S, s1, s2, lam_col, nJ, Zbar_out, c_out,
        c_out_f, J_out, g_out);
  else
    k_rev_reduce<float><<<(total + 255) / 256, 256, 0, st>>>(
        (const float*)part, chunks, kcols, kvalid, S, s1, s2, lam_col, nJ, Zbar_out, c_out,
        c_out_f, J_out, g_out);
  note_launch();
  return cudaGetLastError();
}

// Seeds at the output layer (out_seed): zbar_L of every seed column, and the output layer's
// diagonal curvature c_L (the lambda column).  p: softmax probabilities, or NULL.
__global__ void k_rev_seed(int m, int S, int nJ, int lam_col, const double* __restrict__ s1,
                           const double* __restrict__ s2, const double* __restrict__ lam,
                           const double* __restrict__ p, double* __restrict__ Zbar,
                           double* __restrict__ c_out, float* __restrict__ c_out_f) {
  async::griddep_launch();
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * S) return;
  const int i = idx / S, s = idx % S;
  double c;
  Zbar[idx] = out_seed(i, s, m, nJ, lam_col, s1, s2, lam, p, &c);
  if (s == lam_col) {
    if (c_out) c_out[i] = c;
    if (c_out_f) c_out_f[i] = (float)c;
  }
}

cudaError_t launch_rev_seed(int m, int S, int nJ, int lam_col, const double* s1, const double* s2,
                            const double* lam, const double* p, double* Zbar, double* c_out,
                            float* c_out_f, cudaStream_t st) {
  const int total = m * S;
  k_rev_seed<<<(total + 255) / 256, 256, 0, st>>>(m, S, nJ, lam_col, s1, s2, lam, p, Zbar, c_out,
                                                  c_out_f);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ first-layer tangents
// Zdot_1 = W_1 I = W_1, so the tangents of layer 1 are a scaled transpose of W_1.  32 x 32
// tiles through shared memory keep both the read (along n) and the write (along m) coalesced.
// The FP32 copy of W_1 is used (FP64 for the FP64 form); the scaling runs in the same type.
template <Elem E>
__device__ __forceinline__ void put_tan(TanBuf b, size_t i, float v) {
  if constexpr (E == Elem::F32) {
    ((float*)b.hi)[i] = v;
  } else if constexpr (E == Elem::BF16) {
    ((__nv_bfloat16*)b.hi)[i] = __float2bfloat16_rn(v);
  } else {
    __nv_bfloat16 h, l;
    split_bf16(v, h, l);
    ((__nv_bfloat16*)b.hi)[i] = h;
    ((__nv_bfloat16*)b.lo)[i] = l;
  }
}

// ------------------------------------------------------------------ softmax output layer
// p = softmax(z) in place (the value pass computed the logits z = W_L a_{L-1} + b_L), with the
// maximum subtracted before exp.  m <= 64; one warp.
__global__ void k_softmax_head(int m, double* __restrict__ z) {
  const int lane = threadIdx.x;
  double v0 = lane < m ? z[lane] : -INFINITY, v1 = lane + 32 < m ? z[lane + 32] : -INFINITY;
  double mx = fmax(v0, v1);
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const double e0 = lane < m ? exp(v0 - mx) : 0.0, e1 = lane + 32 < m ? exp(v1 - mx) : 0.0;
  const double sum = warp_sum(e0 + e1);
  if (lane < m) z[lane] = e0 / sum;
  if (lane + 32 < m) z[lane + 32] = e1 / sum;
}

cudaError_t launch_softmax_head(int m, double* z, cudaStream_t st) {
  if (m > 64) return cudaErrorInvalidValue;
  k_softmax_head<<<1, 32, 0, st>>>(m, z);
  note_launch();
  return cudaGetLastError();
}

// The softmax layer's curvature grad_z^2(lambda^T p) = diag(p (lambda - lambar)) + U C U^T with
// U = [p, p lambda], C = [[2 lambar, -1], [-1, 0]], lambar = p^T lambda.  The diagonal part goes
// through the tangent epilogue like any layer; the rank-two part is written as two extra columns
// of the symmetric product's operands: with C's eigenvalues g_k = lambar +- sqrt(lambar^2 + 1)
// and u_k = p + (2 lambar - g_k) p lambda, U C U^T = sum_k g'_k u_k u_k^T,
// g'_k = g_k / (1 + (2 lambar - g_k)^2); column k of Zdot^T is w_k = Zdot_L^T u_k, of the scaled
// operand g'_k w_k, so the product adds sum_k g'_k w_k w_k^T to H.
template <Elem E>
__device__ __forceinline__ double get_tan(TanBuf b, size_t i) {
  if constexpr (E == Elem::F64) return ((const double*)b.hi)[i];
  else if constexpr (E == Elem::F32) return ((const float*)b.hi)[i];
  else if constexpr (E == Elem::BF16) return __bfloat162float(((const __nv_bfloat16*)b.hi)[i]);
  else
    return (double)__bfloat162float(((const __nv_bfloat16*)b.hi)[i]) +
           (double)__bfloat162float(((const __nv_bfloat16*)b.lo)[i]);
}

template <Elem E>
__device__ __forceinline__ void set_tan(TanBuf b, size_t i, double v) {
  if constexpr (E == Elem::F64) ((double*)b.hi)[i] = v;
  else put_tan<E>(b, i, (float)v);
}

template <Elem E>
__global__ void k_softmax_ext(int n, int m, const double* __restrict__ p, const double* __restrict__ lam,
                              TanBuf ZL, TanBuf Zx, TanBuf Yx, int ldz) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;   // tangent (row of Zdot^T)
  if (j >= n) return;
  double lb = 0.0;
  for (int i = 0; i < m; ++i) lb += lam[i] * p[i];
  const double r = sqrt(lb * lb + 1.0);
  const double g[2] = {lb + r, lb - r};
  double w[2] = {0.0, 0.0};
  for (int i = 0; i < m; ++i) {
    const double z = get_tan<E>(ZL, (size_t)j * ldz + i);
    const double pl = p[i] * lam[i];
#pragma unroll
    for (int k = 0; k < 2; ++k) w[k] += z * (p[i] + (2.0 * lb - g[k]) * pl);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const double t = 2.0 * lb - g[k];
    const size_t o = (size_t)j * ldz + k;
    set_tan<E>(Zx, o, w[k]);
    set_tan<E>(Yx, o, g[k] / (1.0 + t * t) * w[k]);
  }
}

cudaError_t launch_softmax_ext(Elem e, int n, int m, const double* p, const double* lam, TanBuf ZL,
                               TanBuf Zx, TanBuf Yx, int ldz, cudaStream_t st) {
  const int blocks = (n + 127) / 128;
  switch (e) {
    case Elem::F64: k_softmax_ext<Elem::F64><<<blocks, 128, 0, st>>>(n, m, p, lam, ZL, Zx, Yx, ldz); break;
    case Elem::F32: k_softmax_ext<Elem::F32><<<blocks, 128, 0, st>>>(n, m, p, lam, ZL, Zx, Yx, ldz); break;
    case Elem::BF16: k_softmax_ext<Elem::BF16><<<blocks, 128, 0, st>>>(n, m, p, lam, ZL, Zx, Yx, ldz); break;
    case Elem::BF16X3:
      k_softmax_ext<Elem::BF16X3><<<blocks, 128, 0, st>>>(n, m, p, lam, ZL, Zx, Yx, ldz);
      break;
  }
  note_launch();
  return cudaGetLastError();
}

template <Elem E, typename TW>
__global__ void k_first_tangent(const TW* __restrict__ W1, int ldw, int m_pad, int n,
                                const double* __restrict__ s1, const double* __restrict__ c,
                                TanBuf At, int lda, TanBuf Zt, TanBuf Yt, int ldz) {
  __shared__ TW tile[32][33];
  const int m0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int mm = m0 + r, nn = n0 + threadIdx.x;
    tile[r][threadIdx.x] = (mm < m_pad && nn < n) ? W1[(size_t)mm * ldw + nn] : TW(0);
  }
  __syncthreads();
  const int mm = m0 + threadIdx.x;
  if (mm >= m_pad) return;
  const TW sm = (TW)s1[mm], cm = (TW)c[mm];
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int nn = n0 + r;
    if (nn >= n) continue;
    const TW w = tile[threadIdx.x][r];
    if constexpr (E == Elem::F64) {
      if (At.hi) ((double*)At.hi)[(size_t)nn * lda + mm] = sm * w;
      if (Zt.hi) {
        ((double*)Zt.hi)[(size_t)nn * ldz + mm] = w;
        ((double*)Yt.hi)[(size_t)nn * ldz + mm] = cm * w;
      }
    } else {
      if (At.hi) put_tan<E>(At, (size_t)nn * lda + mm, sm * w);
      if (Zt.hi) {
        put_tan<E>(Zt, (size_t)nn * ldz + mm, w);
        put_tan<E>(Yt, (size_t)nn * ldz + mm, cm * w);
      }
    }
  }
}

// BF16 forms: 64 rows of W_1 x 32 tangents per block through a shared tile; a thread converts 8
// consecutive rows of one tangent and writes each output part as one 16-byte vector.
template <bool X3>
__global__ void __launch_bounds__(256) k_first_tangent_v(const float* __restrict__ W1, int ldw,
                                                         int m_pad, int n,
                                                         const double* __restrict__ s1,
                                                         const double* __restrict__ c, TanBuf At,
                                                         int lda, TanBuf Zt, TanBuf Yt, int ldz) {
  __shared__ float tile[64][33];
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 32;
  const int t = threadIdx.x, j = t / 8, q = t % 8;   // tangent n0 + j, rows m0 + 8q .. + 7
  const int nn = n0 + j, mb = m0 + 8 * q;
  // all global loads first (independent, so they are in flight together)
  float wv[8], sv[8], cv[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int mm = m0 + t / 32 + 8 * i, nc = n0 + (t & 31);
    wv[i] = (mm < m_pad && nc < n) ? __ldg(W1 + (size_t)mm * ldw + nc) : 0.f;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const bool in = mb + i < m_pad;
    sv[i] = in ? (float)__ldg(s1 + mb + i) : 0.f;
    cv[i] = in ? (float)__ldg(c + mb + i) : 0.f;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) tile[t / 32 + 8 * i][t & 31] = wv[i];
  __syncthreads();
  if (nn >= n || mb >= m_pad) return;
  uint32_t ah[4], al[4], zh[4], zl[4], yh[4], yl[4];
#pragma unroll
  for (int e = 0; e < 8; e += 2) {
    float a2[2], z2[2], y2[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const float w = tile[8 * q + e + u][j];
      z2[u] = w;
      a2[u] = sv[e + u] * w;
      y2[u] = cv[e + u] * w;
    }
    auto pk = [](float v0, float v1, uint32_t& hi, uint32_t& lo) {
      __nv_bfloat16 h0, l0, h1, l1;
      split_bf16(v0, h0, l0);
      split_bf16(v1, h1, l1);
      hi = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
      lo = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    };
    pk(a2[0], a2[1], ah[e / 2], al[e / 2]);
    pk(z2[0], z2[1], zh[e / 2], zl[e / 2]);
    pk(y2[0], y2[1], yh[e / 2], yl[e / 2]);
  }
  auto st16 = [](void* base, size_t idx, const uint32_t (&v)[4]) {
    *reinterpret_cast<uint4*>((__nv_bfloat16*)base + idx) = make_uint4(v[0], v[1], v[2], v[3]);
  };
  if (At.hi) {
    st16(At.hi, (size_t)nn * lda + mb, ah);
    if (X3) st16(At.lo, (size_t)nn * lda + mb, al);
  }
  if (Zt.hi) {
    st16(Zt.hi, (size_t)nn * ldz + mb, zh);
    if (X3) st16(Zt.lo, (size_t)nn * ldz + mb, zl);
  }
  if (Yt.hi) {
    st16(Yt.hi, (size_t)nn * ldz + mb, yh);
    if (X3) st16(Yt.lo, (size_t)nn * ldz + mb, yl);
  }
}

// BF16 forms, from the FP32 transpose W1T [n][ldt] of the first layer (made once at load): a
// thread takes eight consecutive rows m and kFtN tangents n (blockIdx.y), reads sigma' and c of its
// rows once for all of them, and per tangent reads W1T as two 16-byte loads and writes one 16-byte
// vector per output part.  Zdot_1 = W_1 does not depend on x, so its block of the symmetric
// product's operand is written once at load; per evaluation only Adot_1 = sigma_1' W_1^T (and
// c_1 W_1^T when Ydot is not deferred) is formed.
constexpr int kFtN = 4;
template <bool X3>
__global__ void __launch_bounds__(256) k_first_tangent_t(const float* __restrict__ W1T, int ldt,
                                                         int m_pad, int n,
                                                         const double* __restrict__ s1,
                                                         const double* __restrict__ c, TanBuf At,
                                                         int lda, TanBuf Yt, int ldz) {
  const int mb = 8 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (mb >= m_pad) return;
  const int n0 = blockIdx.y * kFtN;
  float sv[8], cv[8];
#pragma unroll
  for (int e = 0; e < 8; e += 2) {
    const double2 sp = __ldg(reinterpret_cast<const double2*>(s1 + mb + e));
    sv[e] = (float)sp.x;
    sv[e + 1] = (float)sp.y;
    if (Yt.hi) {
      const double2 cp = __ldg(reinterpret_cast<const double2*>(c + mb + e));
      cv[e] = (float)cp.x;
      cv[e + 1] = (float)cp.y;
    }
  }
  float4 w0[kFtN], w1[kFtN];
#pragma unroll
  for (int j = 0; j < kFtN; ++j)
    if (n0 + j < n) {
      w0[j] = __ldg(reinterpret_cast<const float4*>(W1T + (size_t)(n0 + j) * ldt + mb));
      w1[j] = __ldg(reinterpret_cast<const float4*>(W1T + (size_t)(n0 + j) * ldt + mb + 4));
    }
  auto pk = [](float v0, float v1, uint32_t& hi, uint32_t& lo) {
    __nv_bfloat16 h0, l0, h1, l1;
    split_bf16(v0, h0, l0);
    split_bf16(v1, h1, l1);
    hi = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
    lo = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
  };
  auto st16 = [](void* base, size_t idx, const uint32_t (&v)[4]) {
    *reinterpret_cast<uint4*>((__nv_bfloat16*)base + idx) = make_uint4(v[0], v[1], v[2], v[3]);
  };
#pragma unroll
  for (int j = 0; j < kFtN; ++j) {
    const int nn = n0 + j;
    if (nn >= n) break;
    const float w[8] = {w0[j].x, w0[j].y, w0[j].z, w0[j].w, w1[j].x, w1[j].y, w1[j].z, w1[j].w};
    if (At.hi) {
      uint32_t h[4], l[4];
#pragma unroll
      for (int e = 0; e < 8; e += 2) pk(sv[e] * w[e], sv[e + 1] * w[e + 1], h[e / 2], l[e / 2]);
      st16(At.hi, (size_t)nn * lda + mb, h);
      if (X3) st16(At.lo, (size_t)nn * lda + mb, l);
    }
    if (Yt.hi) {
      uint32_t h[4], l[4];
#pragma unroll
      for (int e = 0; e < 8; e += 2) pk(cv[e] * w[e], cv[e + 1] * w[e + 1], h[e / 2], l[e / 2]);
      st16(Yt.hi, (size_t)nn * ldz + mb, h);
      if (X3) st16(Yt.lo, (size_t)nn * ldz + mb, l);
    }
  }
}

// W^T (FP32): T[j][i] = W[i][j] for i < rows, j < cols, through 32 x 32 shared tiles.
__global__ void k_transpose_f32(const float* __restrict__ W, int ldw, int rows, int cols,
                                float* __restrict__ T, int ldt) {
  __shared__ float tile[32][33];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r, j = j0 + threadIdx.x;
    tile[r][threadIdx.x] = (i < rows && j < cols) ? W[(size_t)i * ldw + j] : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = j0 + r, i = i0 + threadIdx.x;
    if (j < cols && i < rows) T[(size_t)j * ldt + i] = tile[threadIdx.x][r];
  }
}

cudaError_t launch_transpose_f32(const float* W, int ldw, int rows, int cols, float* T, int ldt,
                                 cudaStream_t st) {
  dim3 g((cols + 31) / 32, (rows + 31) / 32), b(32, 8);
  k_transpose_f32<<<g, b, 0, st>>>(W, ldw, rows, cols, T, ldt);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_first_tangent_t(bool x3, const float* W1T, int ldt, int m_pad, int n,
                                   const double* s1, const double* c, TanBuf At, int lda,
                                   TanBuf Yt, int ldz, cudaStream_t st) {
  if (m_pad % 8 || ldt % 4 || lda % 8 || ldz % 8 || ((uintptr_t)W1T & 15)) return cudaErrorInvalidValue;
  const dim3 grid((m_pad / 8 + 255) / 256, (n + kFtN - 1) / kFtN);
  if (x3)
    k_first_tangent_t<true><<<grid, 256, 0, st>>>(W1T, ldt, m_pad, n, s1, c, At, lda, Yt, ldz);
  else
    k_first_tangent_t<false><<<grid, 256, 0, st>>>(W1T, ldt, m_pad, n, s1, c, At, lda, Yt, ldz);
  note_launch();
  return cudaGetLastError();
}

// Ydot = c * Zdot over the columns [k0, k1) of the n x ldz operand blocks of the symmetric
// product, c[k] per column (the curvature weight c_l of the layer owning column k):
// Y = split(c * (Z_hi + Z_lo)) in the split form, bf16(c * Z) otherwise.  Eight columns per
// thread (16-byte loads and stores).
template <bool X3>
__global__ void __launch_bounds__(256) k_scale_y(const __nv_bfloat16* __restrict__ Zh,
                                                 const __nv_bfloat16* __restrict__ Zl,
                                                 __nv_bfloat16* __restrict__ Yh,
                                                 __nv_bfloat16* __restrict__ Yl,
                                                 const float* __restrict__ c, int n, int ldz,
                                                 int k0, int k1) {
  const int per_row = (k1 - k0) / 8;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * per_row) return;
  const int row = (int)(t / per_row);
  const int k = k0 + 8 * (int)(t % per_row);
  const size_t o = (size_t)row * ldz + k;
  const uint4 zh = *reinterpret_cast<const uint4*>(Zh + o);
  uint4 zl = make_uint4(0, 0, 0, 0);
  if (X3) zl = *reinterpret_cast<const uint4*>(Zl + o);
  const float4 c0 = *reinterpret_cast<const float4*>(c + k);
  const float4 c1 = *reinterpret_cast<const float4*>(c + k + 4);
  const float cv[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
  const uint32_t zhw[4] = {zh.x, zh.y, zh.z, zh.w}, zlw[4] = {zl.x, zl.y, zl.z, zl.w};
  uint32_t yh[4], yl[4];
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    uint32_t h2 = 0, l2 = 0;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const float z = __bfloat162float(__ushort_as_bfloat16((unsigned short)(zhw[w] >> (16 * u)))) +
                      (X3 ? __bfloat162float(__ushort_as_bfloat16((unsigned short)(zlw[w] >> (16 * u)))) : 0.f);
      const float y = cv[2 * w + u] * z;
      __nv_bfloat16 hb, lb;
      if (X3) {
        split_bf16(y, hb, lb);
      } else {
        hb = __float2bfloat16_rn(y);
        lb = __float2bfloat16_rn(0.f);
      }
      h2 |= (uint32_t)__bfloat16_as_ushort(hb) << (16 * u);
      l2 |= (uint32_t)__bfloat16_as_ushort(lb) << (16 * u);
    }
    yh[w] = h2;
    yl[w] = l2;
  }
  *reinterpret_cast<uint4*>(Yh + o) = make_uint4(yh[0], yh[1], yh[2], yh[3]);
  if (X3) *reinterpret_cast<uint4*>(Yl + o) = make_uint4(yl[0], yl[1], yl[2], yl[3]);
}

cudaError_t launch_scale_y(bool x3, const void* Zh, const void* Zl, void* Yh, void* Yl,
                           const float* c, int n, int ldz, int k0, int k1, cudaStream_t st) {
  if (k1 <= k0) return cudaSuccess;
  if ((k0 | k1 | ldz) % 8 != 0) return cudaErrorInvalidValue;
  const long long threads = (long long)n * ((k1 - k0) / 8);
  const int blocks = (int)((threads + 255) / 256);
  if (x3)
    k_scale_y<true><<<blocks, 256, 0, st>>>((const __nv_bfloat16*)Zh, (const __nv_bfloat16*)Zl,
                                            (__nv_bfloat16*)Yh, (__nv_bfloat16*)Yl, c, n, ldz, k0, k1);
  else
    k_scale_y<false><<<blocks, 256, 0, st>>>((const __nv_bfloat16*)Zh, nullptr, (__nv_bfloat16*)Yh,
                                             nullptr, c, n, ldz, k0, k1);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_first_tangent(Elem e, const void* W1, int ldw, int m_pad, int n,
                                 const double* s1, const double* c, TanBuf At, int lda, TanBuf Zt,
                                 TanBuf Yt, int ldz, cudaStream_t st) {
  if ((e == Elem::BF16 || e == Elem::BF16X3) && m_pad % 64 == 0 && lda % 8 == 0 && ldz % 8 == 0) {
    // (Zt / Yt already point at the layer's column block, whose offset is a multiple of 128)
    dim3 g((n + 31) / 32, m_pad / 64);
    if (e == Elem::BF16X3)
      k_first_tangent_v<true><<<g, 256, 0, st>>>((const float*)W1, ldw, m_pad, n, s1, c, At, lda,
                                                 Zt, Yt, ldz);
    else
      k_first_tangent_v<false><<<g, 256, 0, st>>>((const float*)W1, ldw, m_pad, n, s1, c, At, lda,
                                                  Zt, Yt, ldz);
    note_launch();
    return cudaGetLastError();
  }
  dim3 grid((n + 31) / 32, (m_pad + 31) / 32), block(32, 8);
  const float* Wf = (const float*)W1;
  switch (e) {
    case Elem::F64:
      k_first_tangent<Elem::F64, double><<<grid, block, 0, st>>>((const double*)W1, ldw, m_pad, n, s1,
                                                                 c, At, lda, Zt, Yt, ldz);
      break;
    case Elem::F32:
      k_first_tangent<Elem::F32, float><<<grid, block, 0, st>>>(Wf, ldw, m_pad, n, s1, c, At, lda, Zt,
                                                                Yt, ldz);
      break;
    case Elem::BF16:
      k_first_tangent<Elem::BF16, float><<<grid, block, 0, st>>>(Wf, ldw, m_pad, n, s1, c, At, lda,
                                                                 Zt, Yt, ldz);
      break;
    case Elem::BF16X3:
      k_first_tangent<Elem::BF16X3, float><<<grid, block, 0, st>>>(Wf, ldw, m_pad, n, s1, c, At, lda,
                                                                   Zt, Yt, ldz);
      break;
  }
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Hessian finish
// H[i][j] = sum_s Hp[s][max(i,j)][min(i,j)]: the split partial sums hold the lower triangle; a
// 32 x 32 tile of H and its mirror tile are read coalesced and written coalesced.
template <typename TP>
__global__ void k_h_finish(const TP* __restrict__ Hp, int splits, int n, int ldp,
                           double* __restrict__ H) {
  __shared__ double t[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x;   // tile row / column of H
  const int i0 = bi * 32, j0 = bj * 32;
  // source tile: lower-triangle storage of block (max, min)
  const int r0 = bi >= bj ? i0 : j0, c0 = bi >= bj ? j0 : i0;
  for (int rr = threadIdx.y; rr < 32; rr += blockDim.y) {
    const int r = r0 + rr, c = c0 + threadIdx.x;
    double v = 0.0;
    if (r < n && c < n) {
      const int R = r >= c ? r : c, C = r >= c ? c : r;
#pragma unroll 4
      for (int s = 0; s < splits; ++s) v += (double)Hp[((size_t)s * n + R) * ldp + C];
    }
    t[rr][threadIdx.x] = v;
  }
  __syncthreads();
  for (int rr = threadIdx.y; rr < 32; rr += blockDim.y) {
    const int i = i0 + rr, j = j0 + threadIdx.x;
    if (i < n && j < n) H[(size_t)i * n + j] = bi >= bj ? t[rr][threadIdx.x] : t[threadIdx.x][rr];
  }
}

// FP32 partials (tensor-core forms): one block of 32 x 8 threads per lower 32 x 32 tile (bi >= bj)
// sums the splits in FP32 (GB300's FP64 rate is a small fraction of FP32's; the partials carry
// FP32 accuracy anyway), four rows per thread with every split's load issued before the adds,
// then writes the tile and its mirror, each coalesced.  Only R >= C entries of the partials are
// read (the upper triangle of a diagonal tile is not written by the product).
__global__ void __launch_bounds__(256) k_h_finish_f32(const float* __restrict__ Hp, int splits,
                                                      int n, int ldp, double* __restrict__ H) {
  __shared__ float t[32][33];
  int b = blockIdx.x, bi = 0;
  while (b > bi) b -= ++bi;          // lower-tile index -> (bi, bj), bj = b <= bi
  const int bj = b;
  const int i0 = bi * 32, j0 = bj * 32, x = threadIdx.x, y = threadIdx.y;
  const size_t plane = (size_t)n * ldp;
  const float* p[4];
  bool in[4];
  float v[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int r = i0 + y + 8 * k, c = j0 + x;
    in[k] = r < n && c < n;
    const int R = r >= c ? r : c, C = r >= c ? c : r;
    p[k] = Hp + (size_t)R * ldp + C;
    v[k] = 0.f;
  }
  for (int s = 0; s < splits; ++s)
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (in[k]) v[k] += __ldg(p[k] + s * plane);
#pragma unroll
  for (int k = 0; k < 4; ++k) t[y + 8 * k][x] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int rr = y + 8 * k;
    const int i = i0 + rr, j = j0 + x;
    if (i < n && j < n) H[(size_t)i * n + j] = (double)t[rr][x];
    if (bi != bj) {
      const int i2 = j0 + rr, j2 = i0 + x;   // mirror tile H[j0..][i0..]
      if (i2 < n && j2 < n) H[(size_t)i2 * n + j2] = (double)t[x][rr];
    }
  }
}

cudaError_t launch_h_finish(bool part_f32, const void* Hp, int splits, int n, int ldp, double* H,
                            cudaStream_t st) {
  const int T = (n + 31) / 32;
  if (part_f32) {
    k_h_finish_f32<<<T * (T + 1) / 2, dim3(32, 8), 0, st>>>((const float*)Hp, splits, n, ldp, H);
  } else {
    dim3 grid(T, T), block(32, 8);
    k_h_finish<double><<<grid, block, 0, st>>>((const double*)Hp, splits, n, ldp, H);
  }
  note_launch();
  return cudaGetLastError();
}

__global__ void k_sub(const double* y, const double* a, double* r, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = y[i] - a[i];
}

cudaError_t launch_sub(const double* y, const double* a, double* r, int n, cudaStream_t st) {
  k_sub<<<(n + 255) / 256, 256, 0, st>>>(y, a, r, n);
  note_launch();
  return cudaGetLastError();
}

__global__ void k_copy_pad(const double* src, double* dst, float2* dst2, int n, int n_pad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_pad) {
    const double v = i < n ? src[i] : 0.0;
    dst[i] = v;
    if (dst2) {
      const float h = (float)v;
      dst2[i] = make_float2(h, (float)(v - (double)h));
    }
  }
}

cudaError_t launch_copy_pad(const double* src, double* dst, void* dst2, int n, int n_pad,
                            cudaStream_t st) {
  k_copy_pad<<<(n_pad + 255) / 256, 256, 0, st>>>(src, dst, (float2*)dst2, n, n_pad);
  note_launch();
  return cudaGetLastError();
}

}  // namespace nnc

namespace nnc {

// ------------------------------------------------------------------ weight packing
// From the padded FP64 master copy: FP32 copy, and the BF16 split hi = bf16(w),
// lo = bf16(w - hi) used by the tensor-core forms.
__global__ void k_pack(const double* __restrict__ w64, size_t n, float* __restrict__ w32,
                       __nv_bfloat16* __restrict__ whi, __nv_bfloat16* __restrict__ wlo) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const double w = w64[i];
    if (w32) w32[i] = (float)w;
    if (whi) {
      __nv_bfloat16 h, l;
      split_bf16(w, h, l);
      whi[i] = h;
      if (wlo) wlo[i] = l;
    }
  }
}

cudaError_t launch_pack(const double* w64, size_t n, float* w32, __nv_bfloat16* whi,
                        __nv_bfloat16* wlo, cudaStream_t st) {
  size_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_pack<<<(unsigned)blocks, 256, 0, st>>>(w64, n, w32, whi, wlo);
  note_launch();
  return cudaGetLastError();
}

}  // namespace nnc

#include <cuda_fp8.h>

namespace nnc {

// ------------------------------------------------------------------ FP8 e4m3 packing
// Per output row r: s_r = max_k |W[r][k]| / 448 (448 = largest finite e4m3), W8 = e4m3(W / s_r).
// One block per row.
__global__ void k_pack_fp8_rows(const double* __restrict__ W, int ld, int cols,
                                unsigned char* __restrict__ W8, float* __restrict__ scale) {
  __shared__ float red[256];
  const int r = blockIdx.x;
  const double* w = W + (size_t)r * ld;
  float mx = 0.f;
  for (int k = threadIdx.x; k < cols; k += blockDim.x) mx = fmaxf(mx, fabsf((float)w[k]));
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  const float s = red[0] > 0.f ? red[0] / 448.f : 1.f;
  if (threadIdx.x == 0) scale[r] = s;
  const float inv = 1.f / s;
  for (int k = threadIdx.x; k < ld; k += blockDim.x)
    W8[(size_t)r * ld + k] = k < cols ? (unsigned char)__nv_cvt_float_to_fp8((float)w[k] * inv, __NV_SATFINITE, __NV_E4M3) : 0;
}

cudaError_t launch_pack_fp8(const double* W, int rows, int ld, int cols, unsigned char* W8,
                            float* scale, cudaStream_t st) {
  k_pack_fp8_rows<<<rows, 256, 0, st>>>(W, ld, cols, W8, scale);
  note_launch();
  return cudaGetLastError();
}

// Tangent rows to e4m3: for row n of A (BF16, n_rows x ld), t_n = max |A[n][:]| / 448 and
// A8[n][k] = e4m3(A[n][k] / t_n).
__global__ void k_quant_fp8_rows(const __nv_bfloat16* __restrict__ A, int ld,
                                 unsigned char* __restrict__ A8, float* __restrict__ t) {
  __shared__ float red[256];
  const int r = blockIdx.x;
  const __nv_bfloat16* a = A + (size_t)r * ld;
  float mx = 0.f;
  for (int k = threadIdx.x; k < ld; k += blockDim.x) mx = fmaxf(mx, fabsf(__bfloat162float(a[k])));
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  const float s = red[0] > 0.f ? red[0] / 448.f : 1.f;
  if (threadIdx.x == 0) t[r] = s;
  const float inv = 1.f / s;
  for (int k = threadIdx.x; k < ld; k += blockDim.x)
    A8[(size_t)r * ld + k] = (unsigned char)__nv_cvt_float_to_fp8(__bfloat162float(a[k]) * inv, __NV_SATFINITE, __NV_E4M3);
}

cudaError_t launch_quant_fp8(const void* A, int rows, int ld, unsigned char* A8, float* t,
                             cudaStream_t st) {
  k_quant_fp8_rows<<<rows, 256, 0, st>>>((const __nv_bfloat16*)A, ld, A8, t);
  note_launch();
  return cudaGetLastError();
}

}  // namespace nnc

namespace nnc {

// ------------------------------------------------------------------ tensor-core reverse sweep
// W_l^T packed as BF16 hi/lo (Wt[k][m] = W[m][k], K-major for the reverse GEMM; [kp][mp]).
__global__ void k_pack_t(const double* __restrict__ W, int mp, int kp, __nv_bfloat16* __restrict__ p0,
                         __nv_bfloat16* __restrict__ p1, __nv_bfloat16* __restrict__ p2) {
  __shared__ double tile[32][33];
  const int m0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int m = m0 + r, k = k0 + threadIdx.x;
    tile[r][threadIdx.x] = (m < mp && k < kp) ? W[(size_t)m * kp + k] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r, m = m0 + threadIdx.x;
    if (k < kp && m < mp) {
      __nv_bfloat16 a, b, c;
      split3_bf16(tile[threadIdx.x][r], a, b, c);
      const size_t o = (size_t)k * mp + m;
      p0[o] = a;
      p1[o] = b;
      p2[o] = c;
    }
  }
}

cudaError_t launch_pack_t(const double* W, int mp, int kp, __nv_bfloat16* p0, __nv_bfloat16* p1,
                          __nv_bfloat16* p2, cudaStream_t st) {
  dim3 grid((kp + 31) / 32, (mp + 31) / 32), block(32, 8);
  k_pack_t<<<grid, block, 0, st>>>(W, mp, kp, p0, p1, p2);
  note_launch();
  return cudaGetLastError();
}

// Output-layer seeds (out_seed), transposed for the reverse GEMM: Zb[s][i] = zbar_L[i][s] as three
// BF16 parts z0/z1/z2 (row stride ld); c_L of the lambda column.
__global__ void k_rev_seed_t(int m, int S, int nJ, int lam_col, const double* __restrict__ s1,
                             const double* __restrict__ s2, const double* __restrict__ lam,
                             const double* __restrict__ p, __nv_bfloat16* __restrict__ z0,
                             __nv_bfloat16* __restrict__ z1, __nv_bfloat16* __restrict__ z2, int ld,
                             double* __restrict__ c_out, float* __restrict__ c_f) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * S) return;
  const int i = idx / S, s = idx % S;
  double cv;
  const double zb = out_seed(i, s, m, nJ, lam_col, s1, s2, lam, p, &cv);
  __nv_bfloat16 a, b, c;
  split3_bf16(zb, a, b, c);
  const size_t o = (size_t)s * ld + i;
  z0[o] = a;
  z1[o] = b;
  z2[o] = c;
  if (s == lam_col) {
    if (c_out) c_out[i] = cv;
    if (c_f) c_f[i] = (float)cv;
  }
}

cudaError_t launch_rev_seed_t(int m, int S, int nJ, int lam_col, const double* s1, const double* s2,
                              const double* lam, const double* p, void* const z[3], int ld,
                              double* c_out, float* c_f, cudaStream_t st) {
  k_rev_seed_t<<<(m * S + 255) / 256, 256, 0, st>>>(m, S, nJ, lam_col, s1, s2, lam, p,
                                                    (__nv_bfloat16*)z[0], (__nv_bfloat16*)z[1],
                                                    (__nv_bfloat16*)z[2], ld, c_out, c_f);
  note_launch();
  return cudaGetLastError();
}

// Sum the split partials P[sp][k][0..bn) of W_l^T Zbar; then either the next seeds (transposed,
// three BF16 parts: Zb[s][k] = s1[k] * Abar[k][s]) and c = s2 * Abar[:, lam_col], or, on the first
// layer, J_out[s][k] (s < nJ) and g_out[k] (s = lam_col) for k < kvalid.
__global__ void k_rev_reduce_t(const float* __restrict__ P, int splits, int kcols, int bn, int S,
                               int kvalid, const double* __restrict__ s1,
                               const double* __restrict__ s2, int lam_col, int nJ,
                               __nv_bfloat16* __restrict__ z0, __nv_bfloat16* __restrict__ z1,
                               __nv_bfloat16* __restrict__ z2, int ld, double* __restrict__ c_out,
                               float* __restrict__ c_f,
                               double* __restrict__ J_out, double* __restrict__ g_out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kcols * S) return;
  const int k = idx / S, s = idx % S;
  double v = 0.0;
  for (int sp = 0; sp < splits; ++sp) v += (double)P[((size_t)sp * kcols + k) * bn + s];
  if (s1) {
    __nv_bfloat16 a, b, c;
    split3_bf16(s1[k] * v, a, b, c);
    const size_t o = (size_t)s * ld + k;
    z0[o] = a;
    z1[o] = b;
    z2[o] = c;
    if (s == lam_col) {
      if (c_out) c_out[k] = s2[k] * v;
      if (c_f) c_f[k] = (float)(s2[k] * v);
    }
  } else if (k < kvalid) {
    if (J_out && s < nJ) J_out[(size_t)s * kvalid + k] = v;
    if (g_out && s == lam_col) g_out[k] = v;
  }
}

cudaError_t launch_rev_reduce_t(const float* P, int splits, int kcols, int bn, int S, int kvalid,
                                const double* s1, const double* s2, int lam_col, int nJ,
                                void* const z[3], int ld, double* c_out, float* c_f, double* J_out,
                                double* g_out, cudaStream_t st) {
  __nv_bfloat16* z0 = z ? (__nv_bfloat16*)z[0] : nullptr;
  __nv_bfloat16* z1 = z ? (__nv_bfloat16*)z[1] : nullptr;
  __nv_bfloat16* z2 = z ? (__nv_bfloat16*)z[2] : nullptr;
  k_rev_reduce_t<<<(kcols * S + 255) / 256, 256, 0, st>>>(P, splits, kcols, bn, S, kvalid, s1, s2,
                                                          lam_col, nJ, z0, z1, z2, ld, c_out, c_f,
                                                          J_out, g_out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace nnc

namespace nnc {

// ------------------------------------------------------------------ double-float packing
// GB300's FP64 units are too slow for an FP64 GEMV to run at HBM speed, so the FP64-accurate value
// pass (k_stream.cu) runs in double-float arithmetic (Dekker 1971): a value is the unevaluated sum
// hi + lo of two FP32 numbers, hi = fl32(v), lo = fl32(v - hi).
// (hi, lo) float pairs of an FP64 array (weights at load time, the network input per call).
__global__ void k_split_df(const double* __restrict__ src, size_t n, float2* __restrict__ dst) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double v = src[i];
    const float h = (float)v;
    dst[i] = make_float2(h, (float)(v - (double)h));
  }
}

cudaError_t launch_split_df(const double* src, size_t n, void* dst, cudaStream_t st) {
  size_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_split_df<<<(unsigned)blocks, 256, 0, st>>>(src, n, (float2*)dst);
  note_launch();
  return cudaGetLastError();
}

}  // namespace nnc
