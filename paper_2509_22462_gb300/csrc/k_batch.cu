// Grouped bandwidth-bound kernels for a batch of networks with equal hidden widths and
// different input sizes (one stability-margin surrogate per contingency, Eq. 8 / Section 4.2).
// Every network's arrays are stacked: group g's rows of layer l start at g * mp_l; its input
// sits in row g of an n_max-padded block; its tangent rows start at boff[g] (n_g of them).
// One launch covers the same step of every network.
#include <algorithm>
#include <type_traits>

#include "batch.cuh"

namespace nnc {

__device__ __forceinline__ double bwarp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// x_cat (sum n_g, concatenated) -> xs[g][0..kp) (zero padded) in FP64 and FP32.
__global__ void k_bx_scatter(const double* __restrict__ xcat, const int* __restrict__ gn,
                             const int* __restrict__ goff, int kp, double* __restrict__ xs,
                             float* __restrict__ xf) {
  const int g = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= kp) return;
  const double v = j < gn[g] ? xcat[goff[g] + j] : 0.0;
  xs[(size_t)g * kp + j] = v;
  if (xf) xf[(size_t)g * kp + j] = (float)v;
}

cudaError_t launch_bx_scatter(const double* xcat, const int* gn, const int* goff, int kp, int groups,
                              double* xs, float* xf, cudaStream_t st) {
  dim3 grid((kp + 255) / 256, groups);
  k_bx_scatter<<<grid, 256, 0, st>>>(xcat, gn, goff, kp, xs, xf);
  note_launch();
  return cudaGetLastError();
}


// Reverse step of every group: part[g][c][kk][s] = sum_{r in chunk c} W_g[r][kk] Zbar_g[r][s]
// (FP32 weights, FP32 seeds), up to 256 threads x 4 columns per block (fewer for short rows, so
// that no thread of a block is idle), 64 rows per chunk.  Larger chunks cut the partial-sum
// traffic but leave too few blocks to stream the weights at full rate.
constexpr int kBRowsMax = 64;
__host__ __device__ constexpr int brev_rows(int) { return 64; }
template <int SMAX>
__global__ void __launch_bounds__(256) k_bgemv_rev(const float* __restrict__ W, int ldw, int mp,
                                                   int m, const double* __restrict__ Zbar, int S,
                                                   int chunks, float* __restrict__ part,
                                                   const int* __restrict__ gcols) {
  __shared__ float zs[kBRowsMax][SMAX];
  const int rows = brev_rows(ldw);
  const int g = blockIdx.z;
  const int c0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
  const int r0 = blockIdx.y * rows;
  const int nr = min(rows, m - r0);
  const double* zg = Zbar + (size_t)g * mp * S;
  for (int i = threadIdx.x; i < rows * SMAX; i += blockDim.x) {
    const int r = i / SMAX, s = i % SMAX;
    zs[r][s] = (r < nr && s < S) ? (float)zg[(size_t)(r0 + r) * S + s] : 0.f;
  }
  __syncthreads();
  if (c0 >= ldw) return;
  float* out = part + (((size_t)g * chunks + blockIdx.y) * ldw + c0) * S;
  // columns past the net's own (zero padding of a first layer): zero partials, no weight reads
  if (nr <= 0 || (gcols && c0 >= gcols[g])) {
    for (int i = 0; i < 4 * S; ++i) out[i] = 0.f;
    return;
  }
  float acc[4][SMAX];
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int s = 0; s < SMAX; ++s) acc[v][s] = 0.f;
  const float* wp = W + ((size_t)g * mp + r0) * ldw + c0;
#pragma unroll 4
  for (int r = 0; r < nr; ++r) {
    const float4 w = __ldg(reinterpret_cast<const float4*>(wp + (size_t)r * ldw));
#pragma unroll
    for (int s = 0; s < SMAX; ++s) {
      const float z = zs[r][s];
      acc[0][s] = fmaf(w.x, z, acc[0][s]);
      acc[1][s] = fmaf(w.y, z, acc[1][s]);
      acc[2][s] = fmaf(w.z, z, acc[2][s]);
      acc[3][s] = fmaf(w.w, z, acc[3][s]);
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int s = 0; s < SMAX; ++s)
      if (s < S) out[v * S + s] = acc[v][s];
}

cudaError_t launch_bgemv_rev(const float* W, int ldw, int mp, int m, int groups, const double* Zbar,
                             int S, float* part, cudaStream_t st, const int* gcols) {
  const int chunks = bgemv_rev_chunks(m, ldw);
  // threads: the row's 4-column groups, rounded up to whole warps, at most 256
  const int threads = std::min(256, (ldw / 4 + 31) / 32 * 32);
  dim3 grid((ldw + 4 * threads - 1) / (4 * threads), chunks, groups);
  if (S <= 2)
    k_bgemv_rev<2><<<grid, threads, 0, st>>>(W, ldw, mp, m, Zbar, S, chunks, part, gcols);
  else if (S <= 4)
    k_bgemv_rev<4><<<grid, threads, 0, st>>>(W, ldw, mp, m, Zbar, S, chunks, part, gcols);
  else
    return cudaErrorInvalidValue;
  note_launch();
  return cudaGetLastError();
}

int bgemv_rev_chunks(int m, int ldw) { return (m + brev_rows(ldw) - 1) / brev_rows(ldw); }

// Sum the chunks of every group; Zbar_out = s1 * Abar (next seeds), c = s2 * Abar[:, lam_col];
// on the first layer (s1 == NULL): J_cat[goff*nJ + s*n_g + kk] and grad_cat[goff + kk], kk < n_g.
__global__ void k_brev_reduce(const float* __restrict__ part, int chunks, int kcols, int mp_out,
                              int S, const double* __restrict__ s1, const double* __restrict__ s2,
                              int lam_col, int nJ, double* __restrict__ Zbar_out,
                              double* __restrict__ c_out, float* __restrict__ c_f,
                              const int* __restrict__ gn, const int* __restrict__ goff,
                              double* __restrict__ J_cat, double* __restrict__ g_cat) {
  const int g = blockIdx.y;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kcols * S) return;
  const int kk = idx / S, s = idx % S;
  const float* pp = part + (size_t)g * chunks * kcols * S + idx;
  // FP32 sums like the products (the reverse sweep is an FP32 recurrence); FP64 only for the
  // boundary products below, once per output
  float vf = 0.f;
#pragma unroll 8
  for (int c = 0; c < chunks; ++c) vf += pp[(size_t)c * kcols * S];
  const double v = (double)vf;
  if (s1) {
    const size_t gi = (size_t)g * mp_out + kk;
    if (kk < mp_out) Zbar_out[(size_t)g * mp_out * S + idx] = s1[gi] * v;
    if (s == lam_col && kk < mp_out) {
      c_out[gi] = s2[gi] * v;
      if (c_f) c_f[gi] = (float)(s2[gi] * v);
    }
  } else {
    const int n = gn[g];
    if (kk < n) {
      if (s < nJ && J_cat) J_cat[(size_t)goff[g] * nJ + (size_t)s * n + kk] = v;
      if (s == lam_col && g_cat) g_cat[goff[g] + kk] = v;
    }
  }
}

cudaError_t launch_brev_reduce(const float* part, int chunks, int kcols, int mp_out, int groups,
                               int S, const double* s1, const double* s2, int lam_col, int nJ,
                               double* Zbar_out, double* c_out, float* c_f, const int* gn,
                               const int* goff, double* J_cat, double* g_cat, cudaStream_t st) {
  dim3 grid((kcols * S + 255) / 256, groups);
  k_brev_reduce<<<grid, 256, 0, st>>>(part, chunks, kcols, mp_out, S, s1, s2, lam_col, nJ, Zbar_out,
                                      c_out, c_f, gn, goff, J_cat, g_cat);
  note_launch();
  return cudaGetLastError();
}

// Output-layer seeds of every group (m = n_out rows per group, stacked with stride mp).
__global__ void k_brev_seed(int m, int mp, int S, int nJ, int lam_col, const double* __restrict__ s1,
                            const double* __restrict__ s2, const double* __restrict__ lam,
                            double* __restrict__ Zbar, double* __restrict__ c_out,
                            float* __restrict__ c_f) {
  const int g = blockIdx.y;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * S) return;
  const int i = idx / S, s = idx % S;
  const size_t gi = (size_t)g * mp + i;
  double ab = 0.0;
  if (s == lam_col) ab = lam[(size_t)g * m + i];
  else if (s < nJ) ab = (s == i) ? 1.0 : 0.0;
  Zbar[(size_t)g * mp * S + idx] = s1[gi] * ab;
  if (s == lam_col) {
    c_out[gi] = s2[gi] * ab;
    if (c_f) c_f[gi] = (float)(s2[gi] * ab);
  }
}

cudaError_t launch_brev_seed(int m, int mp, int groups, int S, int nJ, int lam_col, const double* s1,
                             const double* s2, const double* lam, double* Zbar, double* c_out,
                             float* c_f, cudaStream_t st) {
  dim3 grid((m * S + 255) / 256, groups);
  k_brev_seed<<<grid, 256, 0, st>>>(m, mp, S, nJ, lam_col, s1, s2, lam, Zbar, c_out, c_f);
  note_launch();
  return cudaGetLastError();
}

// First-layer tangents of every group: At[boff+n][m] = s1[m] W1_g[m][n], Zt/Yt likewise at
// column offset 0 of the side-by-side array (row stride ldz), n < n_g.  A CTA transposes a
// 64-row x 32-column tile of W1_g through shared memory; a thread then owns one tangent column
// and eight consecutive rows, so every output is one 16-byte store of eight BF16 values (row
// strides and offsets are multiples of 8 elements, rows padded to a multiple of 64).
__global__ void __launch_bounds__(256) k_bfirst_tangent(const float* __restrict__ W1, int ldw, int mp,
                                                        const int* __restrict__ gn,
                                                        const int* __restrict__ goff,
                                                        const double* __restrict__ s1,
                                                        const double* __restrict__ c,
                                                        __nv_bfloat16* at_hi, __nv_bfloat16* at_lo,
                                                        int lda, __nv_bfloat16* zt_hi,
                                                        __nv_bfloat16* zt_lo, __nv_bfloat16* yt_hi,
                                                        __nv_bfloat16* yt_lo, int ldz, int x3) {
  __shared__ float tile[64][33];
  const int g = blockIdx.z;
  const int n_g = gn[g];
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 32;
  if (n0 >= n_g) return;   // the same for the whole CTA
  const float* Wg = W1 + (size_t)g * mp * ldw;
  const int t = threadIdx.x, j = t / 8, q = t % 8;   // tangent n0 + j, rows m0 + 8q .. + 7
  const int nn = n0 + j, mb = m0 + 8 * q;
  float wv[8], sv[8], cv[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int mm = m0 + t / 32 + 8 * i, nc = n0 + (t & 31);
    wv[i] = (mm < mp && nc < n_g) ? __ldg(Wg + (size_t)mm * ldw + nc) : 0.f;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const bool in = mb + i < mp;
    sv[i] = in ? (float)__ldg(s1 + (size_t)g * mp + mb + i) : 0.f;
    cv[i] = in ? (float)__ldg(c + (size_t)g * mp + mb + i) : 0.f;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) tile[t / 32 + 8 * i][t & 31] = wv[i];
  __syncthreads();
  if (nn >= n_g || mb >= mp) return;
  uint32_t ah[4], al[4], zh[4], zl[4], yh[4], yl[4];
  auto pk = [](float v0, float v1, uint32_t& hi, uint32_t& lo) {
    __nv_bfloat16 h0, l0, h1, l1;
    split_bf16(v0, h0, l0);
    split_bf16(v1, h1, l1);
    hi = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
    lo = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
  };
#pragma unroll
  for (int e = 0; e < 8; e += 2) {
    const float w0 = tile[8 * q + e][j], w1 = tile[8 * q + e + 1][j];
    pk(sv[e] * w0, sv[e + 1] * w1, ah[e / 2], al[e / 2]);
    pk(w0, w1, zh[e / 2], zl[e / 2]);
    pk(cv[e] * w0, cv[e + 1] * w1, yh[e / 2], yl[e / 2]);
  }
  auto st16 = [](__nv_bfloat16* base, size_t idx, const uint32_t (&v)[4]) {
    *reinterpret_cast<uint4*>(base + idx) = make_uint4(v[0], v[1], v[2], v[3]);
  };
  const size_t row = (size_t)goff[g] + nn;
  if (at_hi) {
    st16(at_hi, row * lda + mb, ah);
    if (x3) st16(at_lo, row * lda + mb, al);
  }
  if (zt_hi) {
    st16(zt_hi, row * ldz + mb, zh);
    if (x3) st16(zt_lo, row * ldz + mb, zl);
    st16(yt_hi, row * ldz + mb, yh);
    if (x3) st16(yt_lo, row * ldz + mb, yl);
  }
}

cudaError_t launch_bfirst_tangent(const float* W1, int ldw, int mp, int groups, int n_max,
                                  const int* gn, const int* goff, const double* s1, const double* c,
                                  void* at_hi, void* at_lo, int lda, void* zt_hi, void* zt_lo,
                                  void* yt_hi, void* yt_lo, int ldz, bool x3, cudaStream_t st) {
  // 16-byte stores: row strides and the outputs' element offsets must be multiples of 8
  auto al8 = [](const void* p) { return ((uintptr_t)p % 16) == 0; };
  if (mp % 64 || lda % 8 || ldz % 8 || !al8(at_hi) || !al8(at_lo) || !al8(zt_hi) || !al8(zt_lo) ||
      !al8(yt_hi) || !al8(yt_lo) || (zt_hi && !yt_hi))
    return cudaErrorInvalidValue;
  dim3 grid((n_max + 31) / 32, mp / 64, groups);
  k_bfirst_tangent<<<grid, 256, 0, st>>>(
      W1, ldw, mp, gn, goff, s1, c, (__nv_bfloat16*)at_hi, (__nv_bfloat16*)at_lo, lda,
      (__nv_bfloat16*)zt_hi, (__nv_bfloat16*)zt_lo, (__nv_bfloat16*)yt_hi, (__nv_bfloat16*)yt_lo, ldz,
      x3 ? 1 : 0);
  note_launch();
  return cudaGetLastError();
}

// H_g[i][j] = sum_s Hp[s][g][max][min] for every group (row-major n_g x n_g at hoff[g]).
__global__ void k_bh_finish(const float* __restrict__ Hp, int splits, long long ldh_split,
                            const int* __restrict__ gn, const long long* __restrict__ hoff,
                            double* __restrict__ H) {
  const int g = blockIdx.y;
  const int n = gn[g];
  const long long base = hoff[g];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * n;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    const int r = i > j ? i : j, cc = i > j ? j : i;
    double v = 0.0;
    for (int s = 0; s < splits; ++s) v += (double)Hp[s * ldh_split + base + (long long)r * n + cc];
    H[base + e] = v;
  }
}

cudaError_t launch_bh_finish(const float* Hp, int splits, long long ldh_split, int groups,
                             const int* gn, const long long* hoff, double* H, cudaStream_t st) {
  dim3 grid(32, groups);
  k_bh_finish<<<grid, 256, 0, st>>>(Hp, splits, ldh_split, gn, hoff, H);
  note_launch();
  return cudaGetLastError();
}

// r_cat[g*m + i] = y_cat[g*m + i] - a[g*mp + i]
__global__ void k_bsub(const double* y, const double* a, int m, int mp, int groups, double* r) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * groups) return;
  const int g = idx / m, i = idx % m;
  r[idx] = y[idx] - a[(size_t)g * mp + i];
}

cudaError_t launch_bsub(const double* y, const double* a, int m, int mp, int groups, double* r,
                        cudaStream_t st) {
  k_bsub<<<(m * groups + 255) / 256, 256, 0, st>>>(y, a, m, mp, groups, r);
  note_launch();
  return cudaGetLastError();
}

// y_cat[g*m + i] = a[g*mp + i]
__global__ void k_bgather(const double* a, int m, int mp, int groups, double* y) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * groups) return;
  y[idx] = a[(size_t)(idx / m) * mp + idx % m];
}

cudaError_t launch_bgather(const double* a, int m, int mp, int groups, double* y, cudaStream_t st) {
  k_bgather<<<(m * groups + 255) / 256, 256, 0, st>>>(a, m, mp, groups, y);
  note_launch();
  return cudaGetLastError();
}

}  // namespace nnc
