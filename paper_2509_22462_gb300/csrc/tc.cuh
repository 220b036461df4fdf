// Tensor-core (tcgen05 / TMEM / TMA) GEMMs of the BF16 forms, host side.
//
// Both GEMMs compute D[m][n] = sum_k A[m][k] B[n][k] with A and B K-major BF16 in global memory
// (optionally split into hi and lo parts), FP32 accumulation in tensor memory, and a fused
// epilogue:
//   tangent : A = W_l (mp x kp), B = Adot_{l-1}^T (n x kp);  writes Adot_l^T = sigma_l' * D,
//             Zdot_l^T = D and Ydot_l^T = c_l * D (BF16 hi/lo), c_l = sigma_l'' * abar_l; the
//             Zdot / Ydot blocks of all layers sit side by side along K in one n x K_total array
//   syrk    : A = [Zdot_1 .. Zdot_L]^T, B = [Ydot_1 .. Ydot_L]^T (n x K_total): one product
//             H = sum_l Zdot_l^T diag(c_l) Zdot_l, split over K, lower-triangle tiles only.
#pragma once
#include <cuda.h>

#include "common.cuh"

namespace nnc {

enum { TC_TANGENT = 0, TC_SYRK = 1, TC_TANGENT_G = 2, TC_SYRK_G = 3, TC_REV = 4 };

struct TcPlan {
  CUtensorMap ta_hi, ta_lo, tb_hi, tb_lo;
  CUtensorMap ta_p2, tb_p2;   // third split parts (reverse sweep only)
  int kind = TC_TANGENT;
  int x3 = 0;           // split-BF16x3 products
  int M = 0, N = 0, K = 0;  // M: rows of A (multiple of 128), N: valid rows of B, K: multiple of 64
  int bn = 0;           // N tile
  int bk = 64;          // K block (elements) of a pipeline stage
  int mode = 0;         // 0 BF16, 1 split-BF16x3, 2 FP8 e4m3 (tangent GEMM only)
  int pair = 0;         // tangent GEMM on SM pairs (cta_group::2, 256-row tiles, bn = pair tile)
  int persistent = 0;   // grouped tangent GEMM: one CTA per SM over all (network, row block) tiles
  int sm_count = 0;
  int ntm = 0, ntn = 0; // tiles along M and N (pair plans: 256-row blocks)
  int splits = 1, kb_per_split = 0;
  bool ready = false;
};

// Tile code of a tangent plan: the N tile, negative for the SM-pair kernel.
inline int plan_code(const TcPlan& p) { return p.pair ? -p.bn : p.bn; }

// Choose tiles and split-K for one GEMM and encode its tensor maps.  a_rows / b_rows are the
// row counts of the A and B arrays (rows beyond them read as zero), ld_a / ld_b their row
// strides in elements.  Tangent GEMMs: force_bn > 0 pins a single-SM N tile, force_bn < 0 the
// SM-pair kernel with N tile -force_bn.  Returns NNC_OK or a negative status.
int tc_plan_make(TcPlan& p, int kind, int prec, const void* a_hi, const void* a_lo, int a_rows,
                 int ld_a, const void* b_hi, const void* b_lo, int b_rows, int ld_b, int M, int N,
                 int K, int sm_count, int force_bn = 0, int force_splits = 0,
                 const void* a_p2 = nullptr, const void* b_p2 = nullptr);

// at_* (row stride ldo) may be NULL on the last layer; zt_* / yt_* (row stride ldz) may be NULL
// for a layer without curvature, yt_* alone when c_l * Zdot_l is formed later (launch_scale_y).
// FP8 plans: A = W8 (e4m3, per-row scales wscale), B = tangents in e4m3 with per-row scales
// tscale; the outputs are BF16.
cudaError_t tc_tangent(const TcPlan& p, const double* s1, const float* c, void* at_hi, void* at_lo,
                       int ldo, void* zt_hi, void* zt_lo, void* yt_hi, void* yt_lo, int ldz,
                       int* err, cudaStream_t st, const float* wscale = nullptr,
                       const float* tscale = nullptr);

// The whole tangent chain of an evaluation in one persistent launch (BF16 and split-BF16x3 forms):
// plans[l] is layer l's single-SM tangent plan (every plan with the same N tile, mode and N),
// outs[l] its outputs as for tc_tangent; cnt: nl * ntn unsigned counters, zero at launch.
constexpr int kMaxChain = 12;
struct ChainOut {
  const double* s1;
  const float* c;
  void *at_hi, *at_lo;
  int ldo;
  void *zt_hi, *zt_lo, *yt_hi, *yt_lo;
};
cudaError_t tc_tangent_chain(const TcPlan* plans, const ChainOut* outs, int nl, unsigned* cnt,
                             int ldz, int* err, cudaStream_t st);

// Plain BF16 GEMM on the tensor cores (the learned warm start's layers): C[m][n] =
// sum_k A[m][k] B[n][k] (+ bias[n]) for m < M, n < N, A (a_rows x K, row stride lda) and B
// (b_rows x K, row stride ldb) K-major BF16, K a multiple of 64, strides multiples of 8; rows
// beyond a_rows / b_rows read as zero.  With gelu: Hf = GELU(C) (FP32, row stride ldc), Hl (BF16,
// row stride ldc) and, if Ht is not NULL, Ht[n][m] = GELU(C) (BF16, row stride ldt).
struct PlainPlan {
  CUtensorMap ta, tb;
  int M = 0, N = 0, K = 0, bn = 0, ntm = 0, ntn = 0;
  bool ready = false;
};
int tc_plain_plan(PlainPlan& p, const void* A, int a_rows, int lda, const void* B, int b_rows,
                  int ldb, int M, int N, int K);
cudaError_t tc_plain(const PlainPlan& p, const float* bias, float* C, int ldc, bool gelu, float* Hf,
                     void* Hl, void* Ht, int ldt, int* err, cudaStream_t st);

// Reverse sweep W_l^T Zbar with three-way split BF16 operands (six products, ~FP32 accuracy):
// A = W_l^T (parts 0/1/2, kp x mp, K-major), B = Zbar^T (parts, seeds x mp); writes
// part[split][k][0..bn) (FP32, bn = 16 or 48).
cudaError_t tc_rev(const TcPlan& p, float* part, int* err, cudaStream_t st);

// Hp: splits x N x N floats (row stride N); partial sums of the lower triangle are added.
cudaError_t tc_syrk(const TcPlan& p, float* Hp, int* err, cudaStream_t st);

// Grouped forms for a batch of networks of equal hidden widths (stacked buffers): group g's
// W_l rows start at g * M, its tangent rows at g_boff[g] (g_n[g] of them, <= the plan's N).
cudaError_t tc_tangent_grouped(const TcPlan& p, int groups, const int* g_n, const int* g_boff,
                               const double* s1, const float* c, void* at_hi, void* at_lo, int ldo,
                               void* zt_hi, void* zt_lo, void* yt_hi, void* yt_lo, int ldz,
                               int* err, cudaStream_t st);
// work[t] = (group, row tile, column tile, 0) over the lower-triangle tiles of every group;
// H_g (g_n[g]^2 floats, row-major) sits at Hp + split * ldh_split + g_hoff[g].
cudaError_t tc_syrk_grouped(const TcPlan& p, int n_tiles, const int4* work, const int* g_n,
                            const int* g_boff, const long long* g_hoff, long long ldh_split,
                            float* Hp, int* err, cudaStream_t st);

}  // namespace nnc
