// Grouped launchers for a batch of networks (k_batch.cu); see batch.cu for the layout.
#pragma once
#include "common.cuh"
#include "kernels.cuh"

namespace nnc {

cudaError_t launch_bx_scatter(const double* xcat, const int* gn, const int* goff, int kp, int groups,
                              double* xs, float* xf, cudaStream_t st);
// gcols (device, may be NULL): group g's valid columns; the partials of the columns past them
// (a first layer's zero padding) are written as zero without reading the weights.
cudaError_t launch_bgemv_rev(const float* W, int ldw, int mp, int m, int groups, const double* Zbar,
                             int S, float* part, cudaStream_t st, const int* gcols = nullptr);
int bgemv_rev_chunks(int m, int ldw);   // row chunks of a reverse step (ldw: columns)
cudaError_t launch_brev_reduce(const float* part, int chunks, int kcols, int mp_out, int groups,
                               int S, const double* s1, const double* s2, int lam_col, int nJ,
                               double* Zbar_out, double* c_out, float* c_f, const int* gn,
                               const int* goff, double* J_cat, double* g_cat, cudaStream_t st);
cudaError_t launch_brev_seed(int m, int mp, int groups, int S, int nJ, int lam_col, const double* s1,
                             const double* s2, const double* lam, double* Zbar, double* c_out,
                             float* c_f, cudaStream_t st);
cudaError_t launch_bfirst_tangent(const float* W1, int ldw, int mp, int groups, int n_max,
                                  const int* gn, const int* goff, const double* s1, const double* c,
                                  void* at_hi, void* at_lo, int lda, void* zt_hi, void* zt_lo,
                                  void* yt_hi, void* yt_lo, int ldz, bool x3, cudaStream_t st);
cudaError_t launch_bh_finish(const float* Hp, int splits, long long ldh_split, int groups,
                             const int* gn, const long long* hoff, double* H, cudaStream_t st);
cudaError_t launch_bsub(const double* y, const double* a, int m, int mp, int groups, double* r,
                        cudaStream_t st);
cudaError_t launch_bgather(const double* a, int m, int mp, int groups, double* y, cudaStream_t st);

}  // namespace nnc
