// Shared device helpers of libnnc: activations with their first and second derivatives,
// BF16 hi/lo splitting, launch bookkeeping.  Used by every kernel file of the library.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>

#include "../../include/nnc.h"

namespace nnc {

constexpr int kPad = 128;  // every packed dimension of weights and tangents is a multiple of this
inline int pad_up(int v, int p = kPad) { return (v + p - 1) / p * p; }

// Host-side launch counter (every kernel launch of the library goes through note_launch()).
void note_launch(int n = 1);

// sigma, sigma' and sigma'' of Eq. 3's activations, in FP64.  The derivatives follow from
// the definitions: tanh' = 1 - t^2, tanh'' = -2 t (1 - t^2); sigmoid' = s (1 - s),
// sigmoid'' = s (1 - s)(1 - 2 s); softplus' = sigmoid, softplus'' = sigmoid'; GELU(z) = z Phi(z),
// GELU' = Phi(z) + z phi(z), GELU'' = phi(z) (2 - z^2).
__device__ __forceinline__ void act_eval(int act, double z, double& a, double& d1, double& d2) {
  switch (act) {
    case NNC_TANH: {
      double t = tanh(z);
      a = t;
      d1 = 1.0 - t * t;
      d2 = -2.0 * t * d1;
      break;
    }
    case NNC_SIGMOID: {
      double s = 1.0 / (1.0 + exp(-z));
      a = s;
      d1 = s * (1.0 - s);
      d2 = d1 * (1.0 - 2.0 * s);
      break;
    }
    case NNC_SOFTPLUS: {
      double s = 1.0 / (1.0 + exp(-z));
      a = z > 0.0 ? z + log1p(exp(-z)) : log1p(exp(z));
      d1 = s;
      d2 = s * (1.0 - s);
      break;
    }
    case NNC_GELU: {
      const double kInvSqrt2 = 0.70710678118654752440;
      const double kInvSqrt2Pi = 0.39894228040143267794;
      double Phi = 0.5 * (1.0 + erf(z * kInvSqrt2));
      double phi = kInvSqrt2Pi * exp(-0.5 * z * z);
      a = z * Phi;
      d1 = Phi + z * phi;
      d2 = phi * (2.0 - z * z);
      break;
    }
    default:
      a = z;
      d1 = 1.0;
      d2 = 0.0;
  }
}

// Output-layer seed of the reverse sweep and the output layer's curvature for the Hessian.
// Seed column s is abar_L = e_s (s < nJ) or lambda (s = lam_col); zbar_L = D sigma_L(z_L)^T abar_L.
// Elementwise sigma_L: zbar_L[i] = sigma'_i abar_L[i] and the curvature grad_z^2(lambda^T a_L) is
// diag(sigma''_i lambda_i).  Softmax (p = the probabilities; D sigma = diag(p) - p p^T): zbar_L[i] =
// p_i (abar_L[i] - p^T abar_L), and the curvature is diag(p_i (lambda_i - lambar)) plus a rank-two
// part (handled by the caller), lambar = p^T lambda.  Returns zbar_L[i] of column s; *c = the
// diagonal curvature of row i (used with the lambda column).
__device__ __forceinline__ double out_seed(int i, int s, int m, int nJ, int lam_col,
                                           const double* s1, const double* s2, const double* lam,
                                           const double* p, double* c) {
  if (!p) {
    double ab = 0.0;
    if (s == lam_col) ab = lam[i];
    else if (s < nJ) ab = (s == i) ? 1.0 : 0.0;
    *c = s2[i] * (s == lam_col ? ab : 0.0);
    return s1[i] * ab;
  }
  if (s == lam_col) {
    double lb = 0.0;
    for (int j = 0; j < m; ++j) lb += lam[j] * p[j];
    *c = p[i] * (lam[i] - lb);
    return *c;
  }
  *c = 0.0;
  if (s < nJ) return p[i] * ((s == i ? 1.0 : 0.0) - p[s]);
  return 0.0;
}

// v ~ hi + lo with hi = bf16(v) and lo = bf16(v - hi): the split of the BF16x3 scheme
// (Henry, Tang & Heinecke 2019).  hi carries 8 significant bits, hi + lo about 16.
__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}
__device__ __forceinline__ void split_bf16(double v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __double2bfloat16(v);
  lo = __double2bfloat16(v - (double)__bfloat162float(hi));
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One step of a double-float dot product (hi, lo) += (wh + wl)(ah + al): TwoProduct of the
// leading terms with an FMA, the cross terms into the error part, TwoSum for the running sum
// (Dekker 1971).  The _rn intrinsics keep the compiler from contracting the error-free steps.
__device__ __forceinline__ void df_acc(float& hi, float& lo, float wh, float wl, float ah, float al) {
  const float p = __fmul_rn(wh, ah);
  const float pe = fmaf(wh, ah, -p);                  // exact error of p (TwoProduct)
  const float cross = fmaf(wh, al, __fmul_rn(wl, ah));
  const float s = __fadd_rn(hi, p);                    // TwoSum(hi, p)
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, __fadd_rn(pe, cross)));
}

// (h, l) += (bh, bl) in double-float arithmetic with FP32 operations only: TwoSum of the leading
// terms, the trailing terms and the rounding error added, then a TwoSum renormalisation.  GB300
// runs FP64 at a small fraction of its FP32 rate, so reductions of double-float sums stay in FP32.
__device__ __forceinline__ void df_add(float& h, float& l, float bh, float bl) {
  float s = __fadd_rn(h, bh);
  float bb = __fsub_rn(s, h);
  const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
  const float t = __fadd_rn(__fadd_rn(l, bl), e);
  h = __fadd_rn(s, t);
  bb = __fsub_rn(h, s);
  l = __fadd_rn(__fsub_rn(s, __fsub_rn(h, bb)), __fsub_rn(t, bb));
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void warp_sum_df(float& h, float& l) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o);
    const float ol = __shfl_xor_sync(0xffffffffu, l, o);
    df_add(h, l, oh, ol);
  }
}

// Three-way split v ~ p0 + p1 + p2, each part the BF16 rounding of what the earlier parts leave;
// the residual is below 2^-24 |v| (outside the BF16 underflow range).
__device__ __forceinline__ void split3_bf16(double v, __nv_bfloat16& p0, __nv_bfloat16& p1,
                                            __nv_bfloat16& p2) {
  p0 = __double2bfloat16(v);
  const double r1 = v - (double)__bfloat162float(p0);
  p1 = __double2bfloat16(r1);
  p2 = __double2bfloat16(r1 - (double)__bfloat162float(p1));
}

}  // namespace nnc
