// Launch wrappers of libnnc's kernels (host side).  Every wrapper queues work on `st` and
// returns the cudaError_t of the launch.
#pragma once
#include <cuda.h>

#include "common.cuh"

namespace nnc {

// Where a tangent-sweep epilogue writes one n x m tile set (row stride `ld`, in elements).
// For FP64/FP32 forms only `hi` is used (element type double/float); for BF16 forms hi and
// lo are __nv_bfloat16 arrays holding the split value (lo is ignored by single-pass BF16).
struct TanBuf {
  void* hi = nullptr;
  void* lo = nullptr;
};

enum class Elem { F64, F32, BF16, BF16X3 };

// ---- vector kernels (k_vector.cu)
// Forward layer: z = W a_in + b, a_out = sigma(z), s1 = sigma'(z), s2 = sigma''(z).
// a_in is double (fp64) or float (FP32 weights); a_out_f (may be NULL) receives a float copy.
cudaError_t launch_gemv_fwd(bool fp64, const void* W, int ldw, const double* b, const void* a_in,
                            int m, int k, int act, double* a_out, float* a_out_f, double* s1,
                            double* s2, cudaStream_t st);
// Reverse layer with S seed columns: part[c][kk][s] = sum over row chunk c of W[r][kk] Zbar[r][s]
// (part is double for FP64 weights, float for FP32 weights).
cudaError_t launch_gemv_rev(bool fp64, const void* W, int ldw, int m, int kcols, const double* Zbar,
                            int S, int chunks, void* part, cudaStream_t st);
int rev_chunks(int m, int kcols, int sm_count);
// Sum the chunks; then Zbar_out = s1 * Abar (if s1), c_out = s2 * Abar[:, lam_col] (if c_out),
// J_out[s][kk] = Abar[kk][s] for s < nJ (if J_out), g_out[kk] = Abar[kk][lam_col] (if g_out).
cudaError_t launch_rev_reduce(bool fp64, const void* part, int chunks, int kcols, int kvalid, int S,
                              const double* s1, const double* s2, int lam_col, int nJ,
                              double* Zbar_out, double* c_out, float* c_out_f, double* J_out,
                              double* g_out, cudaStream_t st);
// Softmax output layer (k_vector.cu): p = softmax(z) in place (m <= 64); and the rank-two part of
// its curvature as two extra columns of the symmetric product's operands: Zx[j][k] = w_k[j],
// Yx[j][k] = g'_k w_k[j] (k = 0, 1; row stride ldz), w_k = ZL^T u_k from the layer's tangent
// block ZL (element type e).
cudaError_t launch_softmax_head(int m, double* z, cudaStream_t st);
cudaError_t launch_softmax_ext(Elem e, int n, int m, const double* p, const double* lam, TanBuf ZL,
                               TanBuf Zx, TanBuf Yx, int ldz, cudaStream_t st);
// Seeds of the reverse sweep at the output layer (see k_vector.cu).
cudaError_t launch_rev_seed(int m, int S, int nJ, int lam_col, const double* s1, const double* s2,
                            const double* lam, const double* p, double* Zbar, double* c_out,
                            float* c_out_f, cudaStream_t st);
// First-layer tangents: Zdot_1 = W_1, so At[n][m] = s1[m] W1[m][n] (row stride lda), and
// Zt = W1^T, Yt[n][m] = c[m] W1[m][n] (row stride ldz; skipped if Zt.hi is NULL).  W1 is the
// FP32 copy of the first layer (the FP64 copy for the FP64 form).
// Ydot = c * Zdot over columns [k0, k1) of the n x ldz BF16 (hi, lo) operand blocks (k0, k1,
// ldz multiples of 8).
cudaError_t launch_scale_y(bool x3, const void* Zh, const void* Zl, void* Yh, void* Yl,
                           const float* c, int n, int ldz, int k0, int k1, cudaStream_t st);
cudaError_t launch_first_tangent(Elem e, const void* W1, int ldw, int m_pad, int n,
                                 const double* s1, const double* c, TanBuf At, int lda, TanBuf Zt,
                                 TanBuf Yt, int ldz, cudaStream_t st);
// The same for the BF16 forms from the FP32 transpose W1T [n][ldt] of W_1 (launch_transpose_f32):
// At[n][m] = s1[m] W1T[n][m] and, if Yt.hi, Yt[n][m] = c[m] W1T[n][m]; Zdot_1 is written once at
// load by launch_first_tangent with At and Yt empty.  m_pad, lda, ldz multiples of 8.
cudaError_t launch_first_tangent_t(bool x3, const float* W1T, int ldt, int m_pad, int n,
                                   const double* s1, const double* c, TanBuf At, int lda,
                                   TanBuf Yt, int ldz, cudaStream_t st);
// T[j][i] = W[i][j] (FP32) for i < rows, j < cols.
cudaError_t launch_transpose_f32(const float* W, int ldw, int rows, int cols, float* T, int ldt,
                                 cudaStream_t st);
// H[i][j] = sum_s Hp[s][max(i,j)][min(i,j)]  (exactly symmetric); Hp is double or float.
cudaError_t launch_h_finish(bool part_f32, const void* Hp, int splits, int n, int ldp, double* H,
                            cudaStream_t st);
// r = y - a  (FP64)
cudaError_t launch_sub(const double* y, const double* a, double* r, int n, cudaStream_t st);
// dst[i] = src[i] (double) for i < n; zero for n <= i < n_pad; dst2 (float2, may be NULL) its
// double-float (hi, lo) pairs
cudaError_t launch_copy_pad(const double* src, double* dst, void* dst2, int n, int n_pad,
                            cudaStream_t st);

// ---- CUDA-core GEMMs for the FP64 / FP32 forms (k_simt.cu)
// D[m][n] = sum_k A[m][k] B[n][k] (both K-major).
// Tangent epilogue: At[n][m] = s1[m] D (row stride ldo; At may be NULL), Zt[n][m] = D and
// Yt[n][m] = c[m] D (row stride ldz; both may be NULL)  for n < N.
cudaError_t launch_simt_tangent(bool fp64, const void* A, int lda, const void* B, int ldb, int M,
                                int N, int K, const double* s1, const double* c, void* At, int ldo,
                                void* Zt, void* Yt, int ldz, cudaStream_t st);
// Symmetric-product epilogue: Hp[s][i][j] += D over the lower-triangle tiles, split-K `splits`.
cudaError_t launch_simt_syrk(bool fp64, const void* Zt, const void* Yt, int ld, int n, int K,
                             int splits, double* Hp, cudaStream_t st);

}  // namespace nnc

namespace nnc {
cudaError_t launch_pack(const double* w64, size_t n, float* w32, __nv_bfloat16* whi,
                        __nv_bfloat16* wlo, cudaStream_t st);
}  // namespace nnc

namespace nnc {
// FP8 e4m3 with per-row scales (the FP8 form): W8[r][:] = e4m3(W[r][:] / s_r), s_r = max|W_r|/448.
cudaError_t launch_pack_fp8(const double* W, int rows, int ld, int cols, unsigned char* W8,
                            float* scale, cudaStream_t st);
// BF16 tangent rows to e4m3 with per-row scales t_n.
cudaError_t launch_quant_fp8(const void* A, int rows, int ld, unsigned char* A8, float* t,
                             cudaStream_t st);
}  // namespace nnc

namespace nnc {
// Bounded-wait self-tests: one CTA waits `limit` cycles on an mbarrier nothing arrives on and
// records `code` in *err (the streaming kernels' wait, and the tensor-core kernels' wait with its
// abort flag).
cudaError_t launch_wait_selftest_stream(int* err, long long limit, int code, cudaStream_t st);
cudaError_t launch_wait_selftest_tc(int* err, long long limit, int code, cudaStream_t st);
}  // namespace nnc

namespace nnc {
// Streaming value-pass layer in double-float arithmetic (k_stream.cu), launched with
// programmatic dependent launch: z = W a_in + b from (hi, lo) float2 weights and activations;
// a_out = sigma(z), a_df its (hi, lo) float2 copy, s1 = sigma'(z), s2 = sigma''(z) (each may be
// NULL).  ldw (elements per row) must be a multiple of 128.
cudaError_t launch_gemv_stream_df(const void* W2, int ldw, int m, const double* b, const void* a_in2,
                                  int act, double* a_out, void* a_df, double* s1, double* s2,
                                  int* err, int sm_count, cudaStream_t st);
// The same over `groups` networks stacked by rows (W2 [groups * mp][ldw], bias and outputs
// [groups * mp]): group g multiplies its own activations a_in2 + g * ld_in (float2 elements) and
// only its first m rows are computed (the padding rows' outputs are left as they are).  gcols
// (device, may be NULL): group g's weights have gcols[g] valid columns, the rest zero padding that
// is skipped in whole 512-byte groups.
cudaError_t launch_gemv_stream_df_grouped(const void* W2, int ldw, int groups, int mp, int m,
                                          const double* b, const void* a_in2, int ld_in, int act,
                                          double* a_out, void* a_df, double* s1, double* s2,
                                          int* err, int sm_count, cudaStream_t st,
                                          const int* gcols = nullptr);
}  // namespace nnc

namespace nnc {
// Streaming FP32 reverse sweep (k_rev.cu), up to 16 seed columns, programmatic dependent launch,
// thread-block clusters along the row blocks.  Seeds are FP32 with SM = rev_stream_sm(S) columns
// per row (zero past S).  One launch per layer: Abar[k][s] = sum_r W[r][k] Zf[r][s] (W through
// `map`, from rev_stream_map of the FP32 weights, mp x kp, kp a multiple of 128), then either the
// next seeds Zf_out[k][s] = s1n[k] Abar[k][s] and c = s2n * Abar[:, lam_col] (c_out / c_f_out may
// be NULL), or, with s1n NULL (first layer), J_out[s][k] (s < nJ) and g_out[k] (s = lam_col) for
// k < kvalid.  Geometry from rev_stream_geom (S: the most seeds of any call of the net); part holds
// (splits / cl) x kp x 16 floats, counters kp / 128 ints, zero before the first launch (each launch
// leaves them zero).
struct RevGeom {
  int rows = 0;     // rows per CTA (multiple of 32)
  int splits = 0;   // row blocks (CTAs per column strip), a multiple of cl
  int cl = 1;       // cluster size along the row blocks
};
int rev_stream_sm(int S);
bool rev_stream_map(CUtensorMap* map, const float* W, int mp, int kp);
RevGeom rev_stream_geom(int m, int kp, int S, int sm_count);
cudaError_t launch_rev_seed_f(int m, int S, int nJ, int lam_col, const double* s1, const double* s2,
                              const double* lam, const double* p, float* Zf, double* c_out,
                              float* c_f, cudaStream_t st);
cudaError_t launch_rev_stream(const CUtensorMap& map, int m, int kp, const float* Zf, int S,
                              const RevGeom& g, float* part, int* counters, int nJ, int lam_col,
                              int kvalid, const double* s1n, const double* s2n, float* Zf_out,
                              double* c_out, float* c_f_out, double* J_out, double* g_out, int* err,
                              cudaStream_t st);
}  // namespace nnc

namespace nnc {
// Tensor-core reverse sweep helpers (see k_vector.cu).
// Operands are split three ways into BF16 parts (W^T: p0/p1/p2; seeds: z[0..2]).
cudaError_t launch_pack_t(const double* W, int mp, int kp, __nv_bfloat16* p0, __nv_bfloat16* p1,
                          __nv_bfloat16* p2, cudaStream_t st);
cudaError_t launch_rev_seed_t(int m, int S, int nJ, int lam_col, const double* s1, const double* s2,
                              const double* lam, const double* p, void* const z[3], int ld,
                              double* c_out, float* c_f, cudaStream_t st);
cudaError_t launch_rev_reduce_t(const float* P, int splits, int kcols, int bn, int S, int kvalid,
                                const double* s1, const double* s2, int lam_col, int nJ,
                                void* const z[3], int ld, double* c_out, float* c_f, double* J_out,
                                double* g_out, cudaStream_t st);
}  // namespace nnc

namespace nnc {
cudaError_t launch_split_df(const double* src, size_t n, void* dst, cudaStream_t st);
}  // namespace nnc
