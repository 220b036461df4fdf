// Host FP64 primal-dual interior-point driver (Eq. 1 with the Newton system of Eq. 2).
//
// The paper leaves the terms alpha and beta of Eq. 2 unstated; they are read as the barrier
// terms of IPOPT (Waechter & Biegler 2006): alpha = Sigma + delta_w I with
// Sigma = Z_L (V - L)^-1 + Z_U (U - V)^-1 and an inertia correction delta_w, beta the barrier
// gradient.  Steps per iteration: evaluate, scaled optimality error (s_max = 100) and barrier
// update (kappa_eps = 10, kappa_mu = 0.2, theta_mu = 1.5), inertia-corrected KKT factorization
// (inertia must be (n, m, 0)), Newton step, fraction to the boundary (tau = max(0.99, 1 - mu)),
// backtracking on the exact-penalty merit function (Armijo 1e-4), update and z safeguard
// (kappa_Sigma = 1e10).
//
// The network constraint makes the variables split into a dense block D (the network inputs x,
// whose Hessian block is the dense n_in x n_in matrix of Eq. 6) and a small block S (outputs,
// slacks) with diagonal Hessian.  The KKT matrix K = [[K11, K12], [K12^T, K22]] with
// K11 = W_DD + Sigma_D + delta_w I is factorized as: rows that pin one dense variable through
// slacks of their own eliminated first; a bordered blocked Cholesky of K11 (parallel on the host
// cores) that also leaves A_D L^-T and the Schur block -A_D K11^-1 A_D^T; Bunch-Kaufman LDL^T of
// the reduced multiplier system.  If K11 is positive definite, inertia(K) = (n_D, 0, 0) +
// inertia(Schur complement) (Haynsworth); otherwise Bunch-Kaufman of the dense block with the
// multipliers (positive small-block diagonals eliminated), or of the whole K.  Either way the
// inertia is exact.  The first trial point of each line search is evaluated together with its
// derivatives (problems that can), which the next iteration reuses when the step is accepted.
#include <cuda_runtime.h>
#include <omp.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "../../include/nnc.h"
#include "../../include/nnc_ipm.h"

// the dense block of the KKT matrix on the device (kkt_gpu.cu)
namespace nnc {
struct DenseKktDev;
DenseKktDev* dkkt_create(int nd, int mmax, cudaStream_t st);
void dkkt_free(DenseKktDev* d);
int dkkt_maxabs(DenseKktDev* d, const double* H, double s, const double* hf, double* out);
int dkkt_matvec(DenseKktDev* d, const double* H, const double* x, double* u);
int dkkt_factor(DenseKktDev* d, const double* H, double s, const double* dvec, const double* AD,
                int m, bool* pd, const double** result);
int dkkt_solve(DenseKktDev* d, double* x, int lower);
}  // namespace nnc

namespace {

using Clock = std::chrono::steady_clock;
double secs(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double>(b - a).count();
}

// Page-locked host array (device-to-host copies of the Hessian at link speed); plain heap memory
// if page-locked memory cannot be had.
struct PinnedVec {
  double* p = nullptr;
  bool pinned = false;
  PinnedVec() = default;
  PinnedVec(const PinnedVec&) = delete;
  PinnedVec& operator=(const PinnedVec&) = delete;
  ~PinnedVec() { release(); }
  void release() {
    if (p && pinned) cudaFreeHost(p);
    else delete[] p;
    p = nullptr;
  }
  void resize(size_t n) {
    release();
    pinned = cudaMallocHost((void**)&p, n * sizeof(double)) == cudaSuccess;
    if (!pinned) {
      cudaGetLastError();
      p = new double[n];
    }
  }
  double* data() { return p; }
  double& operator[](size_t i) { return p[i]; }
};

// ---------------------------------------------------------------- dense helpers (OpenMP)
double max_abs(const double* x, size_t n) {
  double m = 0.0;
#pragma omp parallel for reduction(max : m) schedule(static) if (n > 65536)
  for (long long i = 0; i < (long long)n; ++i) m = std::max(m, std::fabs(x[i]));
  return m;
}
bool all_finite(const double* x, size_t n) {
  int ok = 1;
#pragma omp parallel for reduction(&& : ok) schedule(static) if (n > 65536)
  for (long long i = 0; i < (long long)n; ++i) ok = ok && std::isfinite(x[i]);
  return ok != 0;
}
void par_zero(double* x, size_t n) {
#pragma omp parallel for schedule(static) if (n > 65536)
  for (long long i = 0; i < (long long)n; ++i) x[i] = 0.0;
}

// ---------------------------------------------------------------- dense linear algebra
// Two doubles as one SIMD value (GCC vector extension: NEON on Arm, SSE2 on x86); a scalar times
// a v2d multiplies both lanes.
typedef double v2d __attribute__((vector_size(16)));

// Diagonal block of the blocked Cholesky (rows and columns kb .. kb + nb of A, row stride n,
// fully updated),
// factorized transposed so that every update is a contiguous axpy: Dt[j * nb + c] = L[c][j]
// (c >= j), dinv[j] = 1 / L[j][j]; L is written back into A.  False on a pivot (before its square
// root) not above min_pivot.
bool chol_diag(int n, double* A, int kb, int nb, double* Dt, double* dinv, double min_pivot) {
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j <= i; ++j) Dt[(size_t)j * nb + i] = A[(size_t)(kb + i) * n + kb + j];
  for (int j = 0; j < nb; ++j) {
    double* cj = Dt + (size_t)j * nb;
    double d = cj[j];
    if (!(d > min_pivot) || !std::isfinite(d)) return false;
    d = std::sqrt(d);
    cj[j] = d;
    const double inv = 1.0 / d;
    dinv[j] = inv;
    for (int i = j + 1; i < nb; ++i) cj[i] *= inv;
    for (int c = j + 1; c < nb; ++c) {
      const double f = cj[c];
      double* cc = Dt + (size_t)c * nb;
      for (int i = c; i < nb; ++i) cc[i] -= f * cj[i];
    }
  }
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j <= i; ++j) A[(size_t)(kb + i) * n + kb + j] = Dt[(size_t)j * nb + i];
  return true;
}

// Partial Cholesky of a bordered matrix: A is N x N, row-major with row stride ld, lower triangle;
// its leading nc columns are factorized (the leading nc x nc block becomes L11, the rows below it
// L21 = A21 L11^-T) and the trailing block becomes A22 - L21 L21^T (nc = N: the plain Cholesky
// factor).  Returns false if the leading block is not positive definite, or if a pivot (before its
// square root) is not above min_pivot.  Right-looking, blocks of NB columns; per block, in one
// parallel region:
//  - panel L21 = A21 L11^-T, solved transposed (Pt[j][i] = L21[i][j], rows padded to a multiple of
//    8) in chunks of CH rows: 16 columns at a time by axpys, the later columns updated by a
//    4 x 8 register-tiled product (2-wide vectors);
//  - trailing update A22 -= L21 L21^T on the lower triangle in 8 x 4 tiles (16 two-wide vector
//    accumulators); the
//    row tiles of the next diagonal block go first to one thread, which then factorizes that block
//    while the others update the rest (the diagonal factorization leaves the critical path).
bool cholesky_bordered(int N, int nc, int ld, double* A, double min_pivot) {
  constexpr int NB = 48, CH = 32;   // measured on 16 Neoverse V2 cores: 0.85 ms for 784 + 19 rows
  std::vector<double> Dbuf[2] = {std::vector<double>((size_t)NB * NB), std::vector<double>((size_t)NB * NB)};
  std::vector<double> ibuf[2] = {std::vector<double>(NB), std::vector<double>(NB)};
  std::vector<double> Pt;
  int cur = 0;
  if (nc > 0 && !chol_diag(ld, A, 0, std::min(NB, nc), Dbuf[0].data(), ibuf[0].data(), min_pivot))
    return false;
  for (int kb = 0; kb < nc; kb += NB) {
    const int nb = std::min(NB, nc - kb);
    const int r0 = kb + nb;
    const int rem = N - r0;
    if (rem <= 0) break;
    const double* Dt = Dbuf[cur].data();
    const double* dinv = ibuf[cur].data();
    double* Dn = Dbuf[1 - cur].data();
    double* in = ibuf[1 - cur].data();
    const int nb2 = std::max(0, std::min(NB, nc - r0));   // next diagonal block (0: none)
    bool ok2 = true;
    const int rp = (rem + 7) / 8 * 8;
    Pt.resize((size_t)nb * rp);
    const int nch = (rp + CH - 1) / CH;
#pragma omp parallel
    {
#pragma omp for schedule(dynamic, 1)
      for (int ch = 0; ch < nch; ++ch) {
        const int i0 = ch * CH, i1 = std::min(rp, i0 + CH);
        for (int i = i0; i < i1; ++i) {
          if (i < rem) {
            const double* ai = A + (size_t)(r0 + i) * ld + kb;
            for (int j = 0; j < nb; ++j) Pt[(size_t)j * rp + i] = ai[j];
          } else {
            for (int j = 0; j < nb; ++j) Pt[(size_t)j * rp + i] = 0.0;
          }
        }
        for (int jb = 0; jb < nb; jb += 16) {
          const int je = std::min(nb, jb + 16);
          for (int j = jb; j < je; ++j) {
            double* pj = &Pt[(size_t)j * rp];
            const double inv = dinv[j];
            for (int i = i0; i < i1; ++i) pj[i] *= inv;
            const double* lj = Dt + (size_t)j * nb;
            for (int c = j + 1; c < je; ++c) {
              const double f = lj[c];
              double* pc = &Pt[(size_t)c * rp];
              for (int i = i0; i < i1; ++i) pc[i] -= f * pj[i];
            }
          }
          for (int c0 = je; c0 < nb; c0 += 4) {
            const int cn = std::min(4, nb - c0);
            for (int i = i0; i < i1; i += 8) {
              v2d acc[4][4];
              for (int v = 0; v < 4; ++v) acc[v][0] = acc[v][1] = acc[v][2] = acc[v][3] = v2d{0.0, 0.0};
              for (int j = jb; j < je; ++j) {
                const double* pj = &Pt[(size_t)j * rp + i];
                const double* lj = Dt + (size_t)j * nb + c0;
                v2d p4[4];
                std::memcpy(p4, pj, sizeof(p4));
                for (int v = 0; v < 4; ++v) {
                  const double l = v < cn ? lj[v] : 0.0;
                  for (int w = 0; w < 4; ++w) acc[v][w] += l * p4[w];
                }
              }
              for (int v = 0; v < cn; ++v) {
                double* pc = &Pt[(size_t)(c0 + v) * rp + i];
                for (int u = 0; u < 8; ++u) pc[u] -= acc[v][u >> 1][u & 1];
              }
            }
          }
        }
        for (int i = i0; i < std::min(i1, rem); ++i) {
          double* ai = A + (size_t)(r0 + i) * ld + kb;
          for (int j = 0; j < nb; ++j) ai[j] = Pt[(size_t)j * rp + i];
        }
      }
      const int nti = rp / 8;
      const int nd8 = (nb2 + 7) / 8;   // row tiles that hold the next diagonal block
      auto tile_row = [&](int ti) {
        const int i0 = ti * 8;
        for (int p0 = 0; p0 < i0 + 8; p0 += 4) {
          v2d acc[8][2];
          for (int u = 0; u < 8; ++u) acc[u][0] = acc[u][1] = v2d{0.0, 0.0};
          for (int q = 0; q < nb; ++q) {
            const double* c = Pt.data() + (size_t)q * rp;
            v2d b0, b1;
            std::memcpy(&b0, c + p0, sizeof(v2d));
            std::memcpy(&b1, c + p0 + 2, sizeof(v2d));
            for (int u = 0; u < 8; ++u) {
              const double a = c[i0 + u];
              acc[u][0] += a * b0;
              acc[u][1] += a * b1;
            }
          }
          for (int u = 0; u < 8 && i0 + u < rem; ++u) {
            double* ai = A + (size_t)(r0 + i0 + u) * ld + r0;
            for (int v = 0; v < 4 && p0 + v <= i0 + u; ++v) ai[p0 + v] -= acc[u][v >> 1][v & 1];
          }
        }
      };
#pragma omp single nowait
      if (nb2 > 0) {
        for (int ti = 0; ti < nd8; ++ti) tile_row(ti);
        ok2 = chol_diag(ld, A, r0, nb2, Dn, in, min_pivot);
      }
#pragma omp for schedule(dynamic, 1)
      for (int ti = nti - 1; ti >= nd8; --ti) tile_row(ti);   // long rows first
    }
    if (!ok2) return false;
    cur = 1 - cur;
  }
  return true;
}

// Plain Cholesky (row-major n x n, lower triangle), as above with no border.
bool cholesky(int n, double* A, double min_pivot = 0.0) {
  return cholesky_bordered(n, n, n, A, min_pivot);
}

// L^T x = y in place for one right-hand side.  Blocked by 64 rows from the end: the diagonal
// block is solved row by row, then the entries above it subtract its contribution in parallel.
void upper_solve_lt(int n, const double* L, double* x, int ld = 0) {
  if (ld == 0) ld = n;
  const int NB = 64;
  for (int k1 = n; k1 > 0; k1 -= NB) {
    const int k0 = std::max(0, k1 - NB);
    for (int i = k1 - 1; i >= k0; --i) {
      x[i] /= L[(size_t)i * ld + i];
      const double xi = x[i];
      const double* li = L + (size_t)i * ld;
      for (int j = k0; j < i; ++j) x[j] -= li[j] * xi;
    }
#pragma omp parallel for schedule(static) if (k0 >= 512)
    for (int j0 = 0; j0 < k0; j0 += 64) {
      const int j1 = std::min(k0, j0 + 64);
      for (int i = k0; i < k1; ++i) {
        const double xi = x[i];
        const double* li = L + (size_t)i * ld;
        for (int j = j0; j < j1; ++j) x[j] -= li[j] * xi;
      }
    }
  }
}

// Dot product with four partial sums (four independent multiply-add chains).
inline double dot4(const double* a, const double* b, int len) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int j = 0;
  for (; j + 4 <= len; j += 4) {
    s0 += a[j] * b[j];
    s1 += a[j + 1] * b[j + 1];
    s2 += a[j + 2] * b[j + 2];
    s3 += a[j + 3] * b[j + 3];
  }
  for (; j < len; ++j) s0 += a[j] * b[j];
  return (s0 + s1) + (s2 + s3);
}

// Y^T t for Y row-major nd x r: the rows of Y are added in order (contiguous, vectorizable).
inline std::vector<double> ytmul(int nd, int r, const double* Y, const double* t) {
  std::vector<double> out(r, 0.0);
  for (int i = 0; i < nd; ++i) {
    const double ti = t[i];
    const double* yi = Y + (size_t)i * r;
    for (int a = 0; a < r; ++a) out[a] += yi[a] * ti;
  }
  return out;
}

// L x = b in place for one right-hand side, blocked like upper_solve_lt.
void lower_solve1(int n, const double* L, double* x, int ld = 0) {
  if (ld == 0) ld = n;
  const int NB = 64;
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int k1 = std::min(n, k0 + NB);
    for (int i = k0; i < k1; ++i) {
      const double* li = L + (size_t)i * ld;
      x[i] = (x[i] - dot4(li + k0, x + k0, i - k0)) / li[i];
    }
#pragma omp parallel for schedule(static) if (n - k1 >= 512)
    for (int i = k1; i < n; ++i) x[i] -= dot4(L + (size_t)i * ld + k0, x + k0, k1 - k0);
  }
}

// Bunch-Kaufman symmetric indefinite factorization P A P^T = L D L^T (Golub & Van Loan,
// "Matrix Computations", Sec. 4.4), row-major.  The lower triangle of the input is read; the
// factorization keeps the whole symmetric matrix, so that the pivot column (= row k), the row of
// a candidate pivot and both rows of an interchange are contiguous.  Both triangles are updated
// with the same operand pairs (entry (i, j) and entry (j, i) take the same products), so the
// matrix stays exactly symmetric and the lower triangle follows the lower-triangle-only
// recurrence bit for bit.  On return the lower triangle
// holds L below the diagonal and D on it (and at (k + 1, k) for a 2 x 2 block); the pivot sequence
// and the inertia of A (Sylvester's law on the 1 x 1 / 2 x 2 blocks of D) are recorded.
struct BK {
  int n = 0;
  std::vector<double> A;     // factored in place: L below the diagonal, D on/near it
  std::vector<int> perm;     // row i of P A P^T is row perm[i] of A
  std::vector<int> step;     // 1 or 2 at the first index of each pivot block
  int npos = 0, nneg = 0, nzero = 0;
  bool factor(int n_, const double* src, double zero_tol) {
    n = n_;
    A.resize((size_t)n * n);
    for (int i = 0; i < n; ++i) {
      std::memcpy(&A[(size_t)i * n], src + (size_t)i * n, sizeof(double) * (i + 1));
      for (int j = 0; j < i; ++j) A[(size_t)j * n + i] = src[(size_t)i * n + j];
    }
    perm.resize(n);
    step.assign(n, 0);
    for (int i = 0; i < n; ++i) perm[i] = i;
    npos = nneg = nzero = 0;
    const double alpha = (1.0 + std::sqrt(17.0)) / 8.0;
    // w1, w2: the pivot row(s); g1, g2: the multipliers a D^-1 of every trailing index
    std::vector<double> w1(n, 0.0), w2(n, 0.0), g1(n, 0.0), g2(n, 0.0);
    // Shared state of the current step, written by the single thread that chooses the pivot:
    // kc the pivot index, ks its block size, zc a zero column, (sr, ss) the interchange (ss < 0:
    // none), the inverse of D's block (i11, i21, i22; 1 x 1: i11).  It is read only between the
    // single's barrier and the step's closing barrier; each thread advances its own copy k of the
    // pivot index there, so no thread can see a later step's value in the loop test.
    int kc = 0, ks = 1, sr = 0, ss = -1;
    bool zc = false;
    double i11 = 0.0, i21 = 0.0, i22 = 0.0;
    constexpr int kRows = 8;   // rows per ownership chunk: chunk c belongs to thread c % threads
    // One parallel region: per step the pivot choice and the interchange run on one thread (rows
    // only), then every thread applies the interchange's column swap to its own rows and updates
    // them; each row stays with one thread for the whole factorization (its cache).
#pragma omp parallel if (n > 256)
    {
      const int tid = omp_get_thread_num(), nt = omp_get_num_threads();
      int k = 0;
      while (k < n) {
#pragma omp single
        {
          kc = k;
          double* rk = &A[(size_t)k * n];
          const double absakk = std::fabs(rk[k]);
          int imax = k;
          double colmax = 0.0;
          for (int j = k + 1; j < n; ++j)
            if (std::fabs(rk[j]) > colmax) {
              colmax = std::fabs(rk[j]);
              imax = j;
            }
          ks = 1;
          ss = -1;
          zc = std::max(absakk, colmax) <= zero_tol;
          if (zc) {
            ++nzero;
            step[k] = 1;
            rk[k] = 0.0;
          } else {
            int kp = k;
            if (absakk < alpha * colmax) {
              const double* ri = &A[(size_t)imax * n];
              double rowmax = 0.0;   // largest off-diagonal of row imax inside the trailing block
              for (int j = k; j < n; ++j)
                if (j != imax) rowmax = std::max(rowmax, std::fabs(ri[j]));
              if (absakk >= alpha * colmax * (colmax / rowmax)) {
                kp = k;
              } else if (std::fabs(ri[imax]) >= alpha * rowmax) {
                kp = imax;
              } else {
                kp = imax;
                ks = 2;
              }
            }
            const int r = k + ks - 1;
            if (kp != r) {
              // symmetric interchange of r and kp: the two rows here (with their column swap),
              // the column swap of every other trailing row by its owner
              double* ar = &A[(size_t)r * n];
              double* as = &A[(size_t)kp * n];
              for (int j = 0; j < n; ++j) std::swap(ar[j], as[j]);
              std::swap(ar[r], ar[kp]);
              std::swap(as[r], as[kp]);
              if (ks == 2) std::swap(rk[r], rk[kp]);
              std::swap(perm[r], perm[kp]);
              sr = r;
              ss = kp;
            }
            step[k] = ks;
            if (ks == 1) {
              const double d = rk[k];
              if (std::fabs(d) <= zero_tol) ++nzero;
              else if (d > 0) ++npos;
              else ++nneg;
              i11 = d != 0.0 ? 1.0 / d : 0.0;
              std::memcpy(&w1[k + 1], &rk[k + 1], sizeof(double) * (n - k - 1));
              for (int j = k + 1; j < n; ++j) g1[j] = w1[j] * i11;
            } else {
              const double* rk1 = &A[(size_t)(k + 1) * n];
              const double d11 = rk[k], d21 = rk1[k], d22 = rk1[k + 1];
              const double det = d11 * d22 - d21 * d21;
              if (det < 0) {
                ++npos;
                ++nneg;
              } else if (std::fabs(det) <= zero_tol * zero_tol) {
                nzero += 2;
              } else if (d11 + d22 > 0) {
                npos += 2;
              } else {
                nneg += 2;
              }
              i11 = d22 / det;
              i22 = d11 / det;
              i21 = -d21 / det;
              std::memcpy(&w1[k + 2], &rk[k + 2], sizeof(double) * (n - k - 2));
              std::memcpy(&w2[k + 2], &rk1[k + 2], sizeof(double) * (n - k - 2));
              for (int j = k + 2; j < n; ++j) {
                g1[j] = w1[j] * i11 + w2[j] * i21;
                g2[j] = w1[j] * i21 + w2[j] * i22;
              }
            }
          }
        }
        // rows below the pivot block: pending column swap, multipliers L = a D^-1 (stored in the
        // pivot columns) and the trailing update of the whole row
        const int i_lo = kc + ks;
        for (int c = tid; c * kRows < n; c += nt) {
          const int c0 = std::max(c * kRows, i_lo), c1 = std::min(n, (c + 1) * kRows);
          for (int i = c0; i < c1; ++i) {
            double* ai = &A[(size_t)i * n];
            if (ss >= 0 && i != ss) std::swap(ai[sr], ai[ss]);
            if (zc) {
              ai[kc] = 0.0;
            } else if (ks == 1) {
              // (i, j), j <= i: a_ij -= g_i w_j;  (i, j), j > i: a_ij -= g_j w_i (= entry (j, i))
              const double f = g1[i], wi = ai[kc];
              ai[kc] = f;
              if (f != 0.0) {
                for (int j = kc + 1; j <= i; ++j) ai[j] -= f * w1[j];
                for (int j = i + 1; j < n; ++j) ai[j] -= g1[j] * wi;
              }
            } else {
              const double f1 = g1[i], f2 = g2[i], wi1 = ai[kc], wi2 = ai[kc + 1];
              ai[kc] = f1;
              ai[kc + 1] = f2;
              for (int j = kc + 2; j <= i; ++j) ai[j] -= f1 * w1[j] + f2 * w2[j];
              for (int j = i + 1; j < n; ++j) ai[j] -= g1[j] * wi1 + g2[j] * wi2;
            }
          }
        }
        k = kc + ks;
#pragma omp barrier
      }
    }
    return true;
  }
  // Solve A X = B for r right-hand sides at once (B: n x r row-major, overwritten by X): the same
  // three sweeps as solve, with every step a contiguous row operation on a block of columns of B;
  // in parallel over column blocks.
  void solve_multi(double* B, int r) const {
    if (r <= 0 || n == 0) return;
    std::vector<int> start(n);   // first index of each row's pivot block
    for (int k = 0; k < n;) {
      for (int c = k; c < k + step[k]; ++c) start[c] = k;
      k += step[k];
    }
    constexpr int kCols = 32;
#pragma omp parallel for schedule(dynamic, 1) if ((double)n * n * r > 1e6)
    for (int c0 = 0; c0 < r; c0 += kCols) {
      const int w = std::min(r, c0 + kCols) - c0;
      std::vector<double> Y((size_t)n * w);
      for (int i = 0; i < n; ++i)
        std::memcpy(&Y[(size_t)i * w], &B[(size_t)perm[i] * r + c0], sizeof(double) * w);
      // L y' = y: row i takes the columns of the pivot blocks before its own
      for (int i = 0; i < n; ++i) {
        const double* ai = &A[(size_t)i * n];
        double* yi = &Y[(size_t)i * w];
        for (int c = 0; c < start[i]; ++c) {
          const double l = ai[c];
          if (l == 0.0) continue;
          const double* yc = &Y[(size_t)c * w];
          for (int j = 0; j < w; ++j) yi[j] -= l * yc[j];
        }
      }
      // D z = y'
      for (int k = 0; k < n;) {
        double* y1 = &Y[(size_t)k * w];
        if (step[k] == 1) {
          const double d = A[(size_t)k * n + k];
          const double id = d != 0.0 ? 1.0 / d : 0.0;
          for (int j = 0; j < w; ++j) y1[j] *= id;
          k += 1;
        } else {
          double* y2 = &Y[(size_t)(k + 1) * w];
          const double d11 = A[(size_t)k * n + k], d21 = A[(size_t)(k + 1) * n + k],
                       d22 = A[(size_t)(k + 1) * n + k + 1];
          const double det = d11 * d22 - d21 * d21;
          for (int j = 0; j < w; ++j) {
            const double a = y1[j], b = y2[j];
            y1[j] = (d22 * a - d21 * b) / det;
            y2[j] = (-d21 * a + d11 * b) / det;
          }
          k += 2;
        }
      }
      // L^T x = z: rows from the last, each final row scattered into the earlier blocks' rows
      for (int i = n - 1; i >= 0; --i) {
        const double* ai = &A[(size_t)i * n];
        const double* yi = &Y[(size_t)i * w];
        for (int c = 0; c < start[i]; ++c) {
          const double l = ai[c];
          if (l == 0.0) continue;
          double* yc = &Y[(size_t)c * w];
          for (int j = 0; j < w; ++j) yc[j] -= l * yi[j];
        }
      }
      for (int i = 0; i < n; ++i)
        std::memcpy(&B[(size_t)perm[i] * r + c0], &Y[(size_t)i * w], sizeof(double) * w);
    }
  }
  // Solve A x = b (b overwritten by x).
  void solve(double* b) const {
    std::vector<double> y(n);
    for (int i = 0; i < n; ++i) y[i] = b[perm[i]];
    auto a = [&](int i, int j) { return A[(size_t)i * n + j]; };
    // L y' = y
    for (int k = 0; k < n;) {
      const int s = step[k];
      for (int c = k; c < k + s; ++c)
        for (int i = k + s; i < n; ++i) y[i] -= a(i, c) * y[c];
      k += s;
    }
    // D z = y'
    for (int k = 0; k < n;) {
      if (step[k] == 1) {
        const double d = a(k, k);
        y[k] = d != 0.0 ? y[k] / d : 0.0;
        k += 1;
      } else {
        const double d11 = a(k, k), d21 = a(k + 1, k), d22 = a(k + 1, k + 1);
        const double det = d11 * d22 - d21 * d21;
        const double y1 = y[k], y2 = y[k + 1];
        y[k] = (d22 * y1 - d21 * y2) / det;
        y[k + 1] = (-d21 * y1 + d11 * y2) / det;
        k += 2;
      }
    }
    // L^T x = z
    int k = n - 1;
    while (k >= 0) {
      const int k0 = (k >= 1 && step[k - 1] == 2) ? k - 1 : k;
      for (int c = k0; c <= k; ++c)
        for (int i = k + 1; i < n; ++i) y[c] -= a(i, c) * y[i];
      k = k0 - 1;
    }
    for (int i = 0; i < n; ++i) b[perm[i]] = y[i];
  }
};


// ---------------------------------------------------------------- block-tridiagonal sparse KKT
// LDL^T of the KKT matrix K = [[W + Sigma + dw I, A^T], [A, -dc I]] of a sparse problem whose
// unknowns (variables, then multipliers) are split into stages 0 .. S-1 such that every nonzero of
// W and A couples a stage with itself or with a neighbour (the full-space form of Eq. 4: per layer
// the affine multipliers, z_l, the activation multipliers, y_l, in a chain).  With F_0 = K_00 and
//   F_s = K_ss - C_s F_{s-1}^{-1} C_s^T,   C_s = K_{s,s-1},
// K = L diag(F_0, ..., F_{S-1}) L^T with L block unit lower bidiagonal, L_{s,s-1} = C_s F_{s-1}^{-1}.
// Each F_s (dense, the size of one layer) is factorized by Bunch-Kaufman with 1 x 1 and 2 x 2
// pivots, so zero diagonals (free variables without curvature, multipliers without dc) need no
// regularization, and inertia(K) = sum_s inertia(F_s) exactly (Sylvester's law on the block
// diagonal).  Only the nonzero rows of each coupling are solved for: X_s = F_{s-1}^{-1} C_s^T over
// those rows is kept for the solves.  A zero pivot of some F_s is reported through nzero (the
// driver then regularizes), as is a singular leading block of a nonsingular K, which this fixed
// stage order cannot pivot around.
struct StageKkt {
  int n = 0, m = 0, S = 0;
  std::vector<int> size;                  // unknowns per stage
  std::vector<int> ustage, ulocal;        // stage and local index of every unknown
  // destinations of the pattern entries: F_s(a, b) (b <= a, mirrored) or C_s(a, b)
  struct Dst { int s, a, b; bool coupling; };
  std::vector<Dst> wdst, jdst;            // for the W (lower) and A patterns
  std::vector<std::vector<int>> crow;     // per stage: local rows with a nonzero coupling
  std::vector<std::vector<int>> crow_of;  // per stage: local row -> index in crow, or -1
  std::vector<std::vector<double>> C, X;  // per stage: C_s rows (crow x size[s-1]), X_s (size[s-1] x crow)
  std::vector<std::vector<double>> F, R;  // F_s, then its equilibration R_s F_s R_s in place
  std::vector<BK> bk;
  int npos = 0, nneg = 0, nzero = 0;
  // F_s^{-1} B for r right-hand sides (B: size[s] x r row-major, overwritten)
  void apply_inv(int s, double* B, int r) const {
    const int k = size[s];
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < r; ++j) B[(size_t)i * r + j] *= R[s][i];
    bk[s].solve_multi(B, r);
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < r; ++j) B[(size_t)i * r + j] *= R[s][i];
  }

  // n variables with stages vstage, m constraints with stages cstage; W pattern (wr >= wc) and A
  // pattern (ar: constraint, ac: variable).  False if a nonzero couples non-neighbouring stages.
  bool setup(int n_, int m_, const int* vstage, const int* cstage, const std::vector<int>& wr,
             const std::vector<int>& wc, const std::vector<int>& ar, const std::vector<int>& ac) {
    n = n_;
    m = m_;
    S = 0;
    ustage.resize(n + m);
    ulocal.resize(n + m);
    for (int i = 0; i < n + m; ++i) {
      ustage[i] = i < n ? vstage[i] : cstage[i - n];
      if (ustage[i] < 0) return false;
      S = std::max(S, ustage[i] + 1);
    }
    size.assign(S, 0);
    for (int i = 0; i < n + m; ++i) ulocal[i] = size[ustage[i]]++;
    crow.assign(S, {});
    crow_of.assign(S, {});
    for (int s = 0; s < S; ++s) crow_of[s].assign(size[s], -1);
    auto place = [&](int u, int w, Dst& d) {
      const int su = ustage[u], sw = ustage[w];
      if (su == sw) {
        d = {su, std::max(ulocal[u], ulocal[w]), std::min(ulocal[u], ulocal[w]), false};
        return true;
      }
      if (std::abs(su - sw) != 1) return false;
      const int hi = su > sw ? u : w, lo = su > sw ? w : u;
      const int s = ustage[hi], a = ulocal[hi];
      if (crow_of[s][a] < 0) {
        crow_of[s][a] = (int)crow[s].size();
        crow[s].push_back(a);
      }
      d = {s, crow_of[s][a], ulocal[lo], true};
      return true;
    };
    wdst.resize(wr.size());
    for (size_t k = 0; k < wr.size(); ++k)
      if (!place(wr[k], wc[k], wdst[k])) return false;
    jdst.resize(ar.size());
    for (size_t k = 0; k < ar.size(); ++k)
      if (!place(n + ar[k], ac[k], jdst[k])) return false;
    C.assign(S, {});
    X.assign(S, {});
    F.assign(S, {});
    R.assign(S, {});
    bk.assign(S, BK{});
    return true;
  }

  // Each F_s is equilibrated (R_s F_s R_s, R_s = diag(1 / sqrt(max_j |F_s(i, j)|)), a congruence,
  // so the inertia is unchanged) before Bunch-Kaufman, whose zero test is then relative:
  // |pivot| <= rel_tol on rows of largest entry 1.  (An absolute test against the whole matrix's
  // scale would call the tiny but regular Schur complements of strongly active bounds zero.)
  void factor(const double* wv, const double* sig, const double* jv, double dw, double dc,
              double rel_tol) {
    npos = nneg = nzero = 0;
    for (int s = 0; s < S; ++s) {
      F[s].assign((size_t)size[s] * size[s], 0.0);
      C[s].assign(s > 0 ? crow[s].size() * (size_t)size[s - 1] : 0, 0.0);
    }
    for (int i = 0; i < n + m; ++i) {
      const int s = ustage[i], a = ulocal[i];
      F[s][(size_t)a * size[s] + a] += i < n ? sig[i] + dw : -dc;
    }
    auto add = [&](const Dst& d, double v) {
      if (d.coupling) {
        C[d.s][(size_t)d.a * size[d.s - 1] + d.b] += v;
      } else {
        F[d.s][(size_t)d.a * size[d.s] + d.b] += v;
        if (d.a != d.b) F[d.s][(size_t)d.b * size[d.s] + d.a] += v;
      }
    };
    for (size_t k = 0; k < wdst.size(); ++k) add(wdst[k], wv[k]);
    for (size_t k = 0; k < jdst.size(); ++k) add(jdst[k], jv[k]);
    for (int s = 0; s < S; ++s) {
      const int ns_ = size[s];
      if (s > 0 && !crow[s].empty()) {
        // X_s = F_{s-1}^{-1} C_s^T over the coupled rows, then F_s(rows) -= C_s X_s
        const int np = size[s - 1], r = (int)crow[s].size();
        std::vector<double>& Xs = X[s];
        Xs.assign((size_t)np * r, 0.0);
        for (int b = 0; b < r; ++b)
          for (int k = 0; k < np; ++k) Xs[(size_t)k * r + b] = C[s][(size_t)b * np + k];
        apply_inv(s - 1, Xs.data(), r);
        std::vector<double>& Fs = F[s];
        const std::vector<int>& rows = crow[s];
#pragma omp parallel for schedule(static) if ((double)r * r * np > 1e6)
        for (int a = 0; a < r; ++a) {
          const double* ca = &C[s][(size_t)a * np];
          std::vector<double> acc(r, 0.0);
          for (int k = 0; k < np; ++k) {
            const double c = ca[k];
            if (c == 0.0) continue;
            const double* xk = &Xs[(size_t)k * r];
            for (int b = 0; b < r; ++b) acc[b] += c * xk[b];
          }
          double* fa = &Fs[(size_t)rows[a] * ns_];
          for (int b = 0; b < r; ++b) fa[rows[b]] -= acc[b];
        }
      }
      std::vector<double>& Rs = R[s];
      Rs.assign(ns_, 1.0);
      for (int i = 0; i < ns_; ++i) {
        double mx = 0.0;
        const double* fi = &F[s][(size_t)i * ns_];
        for (int j = 0; j < ns_; ++j) mx = std::max(mx, std::fabs(fi[j]));
        if (mx > 0.0) Rs[i] = 1.0 / std::sqrt(mx);
      }
      for (int i = 0; i < ns_; ++i)
        for (int j = 0; j < ns_; ++j) F[s][(size_t)i * ns_ + j] *= Rs[i] * Rs[j];
      bk[s].factor(ns_, F[s].data(), rel_tol);
      npos += bk[s].npos;
      nneg += bk[s].nneg;
      nzero += bk[s].nzero;
    }
  }

  // x = K^{-1} b (b: variables, then multipliers; overwritten)
  void solve(double* b) const {
    std::vector<std::vector<double>> z(S);
    for (int s = 0; s < S; ++s) z[s].assign(size[s], 0.0);
    for (int i = 0; i < n + m; ++i) z[ustage[i]][ulocal[i]] = b[i];
    // forward: z_s -= X_s^T z_{s-1} on the coupled rows (z_{s-1} already final)
    for (int s = 1; s < S; ++s) {
      const int np = size[s - 1], r = (int)crow[s].size();
      for (int a = 0; a < r; ++a) {
        double t = 0.0;
        for (int k = 0; k < np; ++k) t += X[s][(size_t)k * r + a] * z[s - 1][k];
        z[s][crow[s][a]] -= t;
      }
    }
    for (int s = 0; s < S; ++s) {
      for (int i = 0; i < size[s]; ++i) z[s][i] *= R[s][i];
      bk[s].solve(z[s].data());
      for (int i = 0; i < size[s]; ++i) z[s][i] *= R[s][i];
    }
    // backward: x_s = w_s - X_{s+1} x_{s+1}(coupled rows)
    for (int s = S - 2; s >= 0; --s) {
      const int r = (int)crow[s + 1].size(), np = size[s];
      if (r == 0) continue;
      for (int k = 0; k < np; ++k) {
        double t = 0.0;
        const double* xk = &X[s + 1][(size_t)k * r];
        for (int a = 0; a < r; ++a) t += xk[a] * z[s + 1][crow[s + 1][a]];
        z[s][k] -= t;
      }
    }
    for (int i = 0; i < n + m; ++i) b[i] = z[ustage[i]][ulocal[i]];
  }
};

// ---------------------------------------------------------------- dense block on the device

// W_DD = s H + diag(hf) with H (nd x nd FP64) in device memory: the KKT solver assembles and
// factorizes the dense block there; host_wdd materializes W_DD on the host for the rare
// indefinite iterations.
struct DenseOnDevice {
  nnc::DenseKktDev* dk = nullptr;
  const double* H = nullptr;
  double s = 1.0;
  const double* hf = nullptr;
  std::function<const double*()> host_wdd;
};

// ---------------------------------------------------------------- structured KKT solver
// K = [[W_DD + diag(sig_D) + dw I, 0, A_D^T], [0, diag(W_SS + sig_S) + dw I, A_S^T],
//      [A_D, A_S, -dc I]], n = nd + ns primal rows and m constraint rows.
struct KktSolver {
  int nd = 0, ns = 0, m = 0, n = 0, r = 0, ldk = 0;
  std::vector<double> K11, Y, Sm, Kfull, tmp, Dinv, T, AS_;
  // the factored bordered matrix (row stride ldk): K11's storage, or the pinned copy of the
  // device factorization
  const double* Kp = nullptr;
  DenseOnDevice* dev = nullptr;   // dense block on the device (null: host)
  bool dev_factor = false;        // L of the current factorization is on the device
  int dev_error = 0;              // nnc_status of a failed device factorization or solve
  std::vector<double> dvec, pinadd;
  BK bkS, bkF, bkT, bkR;
  std::vector<int> zid;   // mode 3: small-block variables with a zero diagonal (free, no curvature)
  std::vector<double> R;
  // 0: Schur of the small block (BK); 1: whole matrix (BK); 2: diagonal small block; 3: diagonal
  // small block with zero entries kept next to the multipliers; 4: indefinite dense block (BK of
  // the dense block, the zero-diagonal variables and the multipliers)
  int mode = 0;
  bool t_chol = false;
  int npos = 0, nneg = 0, nzero = 0;

  // Rows eliminated before the rest ("pinning" rows, such as x_i - p_i + q_i = x_ref,i of the L1
  // problem): at most one nonzero in A_D, and slack columns with a positive diagonal that no
  // other row touches.  Eliminating the slacks leaves row j as a_j w_D[i_j] - e_j u_j = r~3_j with
  // e_j = dc + sum_c A_S[j,c]^2 / D_c > 0, and eliminating u_j adds a_j^2 / e_j to K11[i_j, i_j];
  // each such row adds one negative eigenvalue to the inertia (Haynsworth).
  struct PinTerm { int row, col; double a; };
  int m_all = 0, n_all = 0;
  std::vector<int> prow, pcol, orow;        // pinning rows, their A_D column (-1: none), other rows
  std::vector<double> palpha, pe, pD, r3t;
  std::vector<PinTerm> pterm;               // slack entries of the pinning rows
  std::vector<double> WDDp, ADo, ASo, core;
  void factor(int nd_, int ns_, int m_, const double* WDD, const double* WSS, const double* sig,
              const double* AD, const double* AS, double dw, double dc, double zero_tol) {
    dev_error = 0;
    m_all = m_;
    n_all = nd_ + ns_;
    prow.clear(); pcol.clear(); orow.clear(); palpha.clear(); pe.clear(); pterm.clear();
    pD.assign(ns_, 0.0);
    std::vector<int> ccount(ns_, 0);
    // column counts of A_S, in parallel over column blocks (each thread reads row segments)
#pragma omp parallel for schedule(static) if ((size_t)m_ * ns_ > 65536)
    for (int c0 = 0; c0 < ns_; c0 += 64) {
      const int c1 = std::min(ns_, c0 + 64);
      for (int j = 0; j < m_; ++j) {
        const double* r = AS + (size_t)j * ns_;
        for (int c = c0; c < c1; ++c) ccount[c] += r[c] != 0.0;
      }
    }
    for (int c = 0; c < ns_; ++c) pD[c] = WSS[c] + sig[nd_ + c] + dw;
    // per-row classification in parallel, then an ordered compaction
    std::vector<int> rcol(m_, -1);
    std::vector<double> re(m_, 0.0);
    std::vector<char> rpin(m_, 0);
#pragma omp parallel for schedule(static) if ((size_t)m_ * (nd_ + ns_) > 65536)
    for (int j = 0; j < m_; ++j) {
      int col = -1, nnz = 0;
      for (int i = 0; i < nd_ && nnz < 2; ++i)
        if (AD[(size_t)j * nd_ + i] != 0.0) { col = i; ++nnz; }
      bool pin = nnz <= 1;
      double e = dc;
      for (int c = 0; c < ns_ && pin; ++c) {
        const double a = AS[(size_t)j * ns_ + c];
        if (a == 0.0) continue;
        pin = ccount[c] == 1 && pD[c] > 0.0;
        e += a * a / pD[c];
      }
      rpin[j] = pin && e > 0.0;
      rcol[j] = col;
      re[j] = e;
    }
    for (int j = 0; j < m_; ++j) {
      const int col = rcol[j];
      const double e = re[j];
      if (rpin[j]) {
        prow.push_back(j);
        pcol.push_back(col);
        palpha.push_back(col >= 0 ? AD[(size_t)j * nd_ + col] : 0.0);
        pe.push_back(e);
        for (int c = 0; c < ns_; ++c)
          if (AS[(size_t)j * ns_ + c] != 0.0) pterm.push_back({(int)prow.size() - 1, c, AS[(size_t)j * ns_ + c]});
      } else {
        orow.push_back(j);
      }
    }
    if (prow.empty()) {
      pinadd.assign(nd_, 0.0);
      factor_core(nd_, ns_, m_, WDD, WSS, sig, AD, AS, dw, dc, zero_tol);
      return;
    }
    pinadd.assign(nd_, 0.0);
    for (size_t k = 0; k < prow.size(); ++k)
      if (pcol[k] >= 0) pinadd[pcol[k]] += palpha[k] * palpha[k] / pe[k];
    const int mo = (int)orow.size();
    ADo.assign((size_t)mo * nd_, 0.0);
    ASo.assign((size_t)mo * ns_, 0.0);
    for (int k = 0; k < mo; ++k) {
      std::memcpy(&ADo[(size_t)k * nd_], &AD[(size_t)orow[k] * nd_], sizeof(double) * nd_);
      std::memcpy(&ASo[(size_t)k * ns_], &AS[(size_t)orow[k] * ns_], sizeof(double) * ns_);
    }
    if (dev) {
      // the pinning terms enter the device assembly through pinadd; W_DD + pinadd is formed on the
      // host only if the device finds the dense block indefinite
      factor_core(nd_, ns_, mo, nullptr, WSS, sig, ADo.data(), ASo.data(), dw, dc, zero_tol);
      nneg += (int)prow.size();
      return;
    }
    WDDp.resize((size_t)nd_ * nd_);
#pragma omp parallel for schedule(static) if (nd_ >= 256)
    for (int i = 0; i < nd_; ++i)
      std::memcpy(&WDDp[(size_t)i * nd_], &WDD[(size_t)i * nd_], sizeof(double) * nd_);
    for (int i = 0; i < nd_; ++i) WDDp[(size_t)i * nd_ + i] += pinadd[i];
    factor_core(nd_, ns_, mo, WDDp.data(), WSS, sig, ADo.data(), ASo.data(), dw, dc, zero_tol);
    nneg += (int)prow.size();
  }

  // rhs (n + m) -> solution, in place
  void solve(double* rhs) {
    if (prow.empty()) {
      solve_core(rhs);
      return;
    }
    const int np = (int)prow.size(), mo = (int)orow.size();
    // r~3_j = r3_j - sum_c A_S[j,c] r2_c / D_c; r1 += a_j r~3_j / e_j
    r3t.assign(np, 0.0);
    for (int k = 0; k < np; ++k) r3t[k] = rhs[n_all + prow[k]];
    for (const PinTerm& t : pterm) r3t[t.row] -= t.a * rhs[nd + t.col] / pD[t.col];
    core.assign(rhs, rhs + n_all + mo);
    for (int k = 0; k < np; ++k)
      if (pcol[k] >= 0) core[pcol[k]] += palpha[k] * r3t[k] / pe[k];
    for (int k = 0; k < mo; ++k) core[n_all + k] = rhs[n_all + orow[k]];
    const std::vector<double> r2(rhs + nd, rhs + n_all);
    solve_core(core.data());
    std::vector<double> u(np);
    for (int k = 0; k < np; ++k)
      u[k] = ((pcol[k] >= 0 ? palpha[k] * core[pcol[k]] : 0.0) - r3t[k]) / pe[k];
    for (const PinTerm& t : pterm) core[nd + t.col] = (r2[t.col] - t.a * u[t.row]) / pD[t.col];
    std::copy(core.begin(), core.begin() + n_all, rhs);
    for (int k = 0; k < mo; ++k) rhs[n_all + orow[k]] = core[n_all + k];
    for (int k = 0; k < np; ++k) rhs[n_all + prow[k]] = u[k];
  }

  void factor_core(int nd_, int ns_, int m_, const double* WDD, const double* WSS, const double* sig,
                   const double* AD, const double* AS, double dw, double dc, double zero_tol) {
    nd = nd_;
    ns = ns_;
    m = m_;
    n = nd + ns;
    r = ns + m;
    // K11 with the constraint rows A_D below it (row stride ldk = nd + m): the partial Cholesky
    // of its leading nd columns leaves L, the rows Y^T = A_D L^-T and, in the bottom m x m block,
    // G = -A_D K11^-1 A_D^T
    ldk = nd + m;
    bool pd = nd == 0;
    bool host_factor = !dev || nd == 0;
    dev_factor = false;
    if (dev && nd > 0) {
      // assembly and partial Cholesky of the bordered matrix on the device (H stays there)
      dvec.resize(nd);
      for (int i = 0; i < nd; ++i) dvec[i] = dev->hf[i] + sig[i] + dw + pinadd[i];
      const double* res = nullptr;
      const int rc = nnc::dkkt_factor(dev->dk, dev->H, dev->s, dvec.data(), AD, m, &pd, &res);
      if (rc) {
        dev_error = rc;
        npos = nneg = nzero = 0;
        return;
      }
      if (pd) {
        Kp = res;   // border rows only; L stays on the device
        dev_factor = true;
      } else {
        // not positive definite in FP32 (or nearly singular): the FP64 host path decides, with
        // W_DD (+ the pinning terms) on the host
        const double* W = dev->host_wdd();
        if (!W) {
          dev_error = NNC_ERR_CUDA;
          npos = nneg = nzero = 0;
          return;
        }
        WDDp.assign(W, W + (size_t)nd * nd);
        for (int i = 0; i < nd; ++i) WDDp[(size_t)i * nd + i] += pinadd[i];
        WDD = WDDp.data();
        host_factor = true;
      }
    }
    if (host_factor) {
      K11.resize((size_t)ldk * ldk);
#pragma omp parallel for schedule(static) if (nd >= 256)
      for (int i = 0; i < ldk; ++i) {
        double* ki = &K11[(size_t)i * ldk];
        if (i < nd) {
          std::memcpy(ki, &WDD[(size_t)i * nd], sizeof(double) * nd);
          ki[i] += sig[i] + dw;
        } else {
          std::memcpy(ki, &AD[(size_t)(i - nd) * nd], sizeof(double) * nd);
          std::memset(ki + nd, 0, sizeof(double) * (i - nd + 1));
        }
      }
      pd = nd == 0 || cholesky_bordered(ldk, nd, ldk, K11.data(), 0.0);
      Kp = K11.data();
    }
    auto G = [&](int a, int b) { return Kp[(size_t)(nd + std::max(a, b)) * ldk + nd + std::min(a, b)]; };
    // Y = L^-1 A_D^T (nd x m) from the rows below L
    auto fill_y = [&](int cols, int off) {
      Y.assign((size_t)nd * cols, 0.0);
      for (int j = 0; j < m; ++j) {
        const double* yj = &Kp[(size_t)(nd + j) * ldk];
        for (int i = 0; i < nd; ++i) Y[(size_t)i * cols + off + j] = yj[i];
      }
    };
    bool diag_ok = pd && ns > 0;
    zid.clear();
    for (int a = 0; a < ns && diag_ok; ++a) {
      const double d = WSS[a] + sig[nd + a] + dw;
      diag_ok = d >= 0.0;
      if (d == 0.0) zid.push_back(a);
    }
    if (diag_ok && !zid.empty() && m == 0) diag_ok = false;
    const bool diag_pd = diag_ok && zid.empty();
    if (diag_ok && !zid.empty()) {
      // Zero-diagonal variables w_Z (free, no curvature) stay beside the multipliers: with the
      // dense block and the positive diagonal entries eliminated,
      //   R = [[0, A_Z^T], [A_Z, -T]],  T = dc I + A_D K11^-1 A_D^T + A_P D_P^-1 A_P^T,
      // and inertia(K) = (nd + |P|, 0, 0) + inertia(R).
      mode = 3;
      Dinv.assign(ns, 0.0);
      for (int a = 0; a < ns; ++a) {
        const double d = WSS[a] + sig[nd + a] + dw;
        Dinv[a] = d > 0.0 ? 1.0 / d : 0.0;
      }
      AS_.assign(AS, AS + (size_t)m * ns);
      fill_y(m, 0);
      const int nz = (int)zid.size(), nr = nz + m;
      R.assign((size_t)nr * nr, 0.0);
#pragma omp parallel for schedule(dynamic, 4) if (m >= 64)
      for (int a = 0; a < m; ++a) {
        for (int b = 0; b <= a; ++b) {
          double s = nd ? -G(a, b) : 0.0;   // (A_D K11^-1 A_D^T)[a][b]
          const double* ra = &AS_[(size_t)a * ns];
          const double* rb = &AS_[(size_t)b * ns];
          for (int c = 0; c < ns; ++c)
            if (ra[c] != 0.0 && rb[c] != 0.0) s += ra[c] * rb[c] * Dinv[c];
          const double t = -(s + (a == b ? dc : 0.0));
          R[(size_t)(nz + a) * nr + nz + b] = t;
          R[(size_t)(nz + b) * nr + nz + a] = t;
        }
      }
      for (int q = 0; q < nz; ++q)
        for (int j = 0; j < m; ++j) {
          const double v = AS[(size_t)j * ns + zid[q]];
          R[(size_t)q * nr + nz + j] = v;
          R[(size_t)(nz + j) * nr + q] = v;
        }
      bkR.factor(nr, R.data(), zero_tol);
      npos = nd + (ns - nz) + bkR.npos;
      nneg = bkR.nneg;
      nzero = bkR.nzero;
      return;
    }
    if (diag_pd) {
      // Eliminate the diagonal small block as well: T = -dc I - A_D K11^-1 A_D^T - A_S D^-1 A_S^T.
      // inertia(K) = (nd + ns, 0, 0) + inertia(T); T must be negative definite.
      mode = 2;
      Dinv.resize(ns);
      for (int a = 0; a < ns; ++a) Dinv[a] = 1.0 / (WSS[a] + sig[nd + a] + dw);
      AS_.assign(AS, AS + (size_t)m * ns);
      fill_y(m, 0);
      T.assign((size_t)m * m, 0.0);
#pragma omp parallel for schedule(dynamic, 4) if (m >= 64)
      for (int a = 0; a < m; ++a) {
        for (int b = 0; b <= a; ++b) {
          double s = nd ? -G(a, b) : 0.0;
          const double* ra = &AS_[(size_t)a * ns];
          const double* rb = &AS_[(size_t)b * ns];
          for (int c = 0; c < ns; ++c)
            if (ra[c] != 0.0 && rb[c] != 0.0) s += ra[c] * rb[c] * Dinv[c];
          // store -T (expected positive definite)
          T[(size_t)a * m + b] = s + (a == b ? dc : 0.0);
          T[(size_t)b * m + a] = T[(size_t)a * m + b];
        }
      }
      std::vector<double> Tc(T);
      // a pivot within the zero tolerance is left to Bunch-Kaufman, which reports it as zero
      t_chol = m == 0 || cholesky(m, Tc.data(), zero_tol);
      if (t_chol) {
        T.swap(Tc);
        npos = n;
        nneg = m;
        nzero = 0;
      } else {
        for (auto& v : T) v = -v;   // T itself, for the exact inertia
        bkT.factor(m, T.data(), zero_tol);
        npos = n + bkT.npos;
        nneg = bkT.nneg;
        nzero = bkT.nzero;
      }
      return;
    }
    if (!pd && m > 0) {
      bool nonneg = true;
      for (int a = 0; a < ns && nonneg; ++a) nonneg = WSS[a] + sig[nd + a] + dw >= 0.0;
      if (nonneg) {
        factor_indefinite(WDD, WSS, sig, AD, AS, dw, dc, zero_tol);
        return;
      }
    }
    if (pd) {
      fill_y(r, ns);   // Y = L^-1 K12, K12 = [0 | A_D^T] (nd x r)
      Sm.assign((size_t)r * r, 0.0);
      for (int a = 0; a < ns; ++a) Sm[(size_t)a * r + a] = WSS[a] + sig[nd + a] + dw;
      for (int j = 0; j < m; ++j)
        for (int a = 0; a < ns; ++a) {
          Sm[(size_t)(ns + j) * r + a] = AS[(size_t)j * ns + a];
          Sm[(size_t)a * r + ns + j] = AS[(size_t)j * ns + a];
        }
      for (int j = 0; j < m; ++j) Sm[(size_t)(ns + j) * r + ns + j] = -dc;
      // the rows and columns of the multipliers take G = -A_D K11^-1 A_D^T
      if (nd)
        for (int a = 0; a < m; ++a)
          for (int b = 0; b <= a; ++b) {
            Sm[(size_t)(ns + a) * r + ns + b] += G(a, b);
            if (b != a) Sm[(size_t)(ns + b) * r + ns + a] += G(a, b);
          }
      bkS.factor(r, Sm.data(), zero_tol);
      npos = nd + bkS.npos;
      nneg = bkS.nneg;
      nzero = bkS.nzero;
      mode = 0;
    } else {
      const int N = n + m;
      Kfull.assign((size_t)N * N, 0.0);
      for (int i = 0; i < nd; ++i)
        for (int j = 0; j < nd; ++j) Kfull[(size_t)i * N + j] = WDD[(size_t)i * nd + j];
      for (int i = 0; i < n; ++i) Kfull[(size_t)i * N + i] += sig[i] + dw + (i >= nd ? WSS[i - nd] : 0.0);
      for (int j = 0; j < m; ++j) {
        for (int i = 0; i < nd; ++i)
          Kfull[(size_t)(n + j) * N + i] = Kfull[(size_t)i * N + n + j] = AD[(size_t)j * nd + i];
        for (int a = 0; a < ns; ++a)
          Kfull[(size_t)(n + j) * N + nd + a] = Kfull[(size_t)(nd + a) * N + n + j] = AS[(size_t)j * ns + a];
        Kfull[(size_t)(n + j) * N + n + j] = -dc;
      }
      bkF.factor(N, Kfull.data(), zero_tol);
      npos = bkF.npos;
      nneg = bkF.nneg;
      nzero = bkF.nzero;
      mode = 1;
    }
  }
  // Mode 4: K11 is not positive definite but every small-block diagonal is >= 0.  The positive
  // ones (P) are eliminated; the dense block, the zero-diagonal variables (Z) and the multipliers
  // stay in one symmetric indefinite factorization of size nd + |Z| + m:
  //   M = [[K11, 0, A_D^T], [0, 0, A_Z^T], [A_D, A_Z, -(dc I + A_P D_P^-1 A_P^T)]],
  // inertia(K) = (|P|, 0, 0) + inertia(M).  Far smaller than the whole matrix when ns >> |Z|.
  BK bkM;
  void factor_indefinite(const double* WDD, const double* WSS, const double* sig, const double* AD,
                         const double* AS, double dw, double dc, double zero_tol) {
    mode = 4;
    Dinv.assign(ns, 0.0);
    zid.clear();
    for (int a = 0; a < ns; ++a) {
      const double d = WSS[a] + sig[nd + a] + dw;
      if (d > 0.0) Dinv[a] = 1.0 / d;
      else zid.push_back(a);
    }
    AS_.assign(AS, AS + (size_t)m * ns);
    const int nz = (int)zid.size(), N = nd + nz + m;
    std::vector<double> M((size_t)N * N, 0.0);
    for (int i = 0; i < nd; ++i) {
      std::memcpy(&M[(size_t)i * N], &WDD[(size_t)i * nd], sizeof(double) * nd);
      M[(size_t)i * N + i] += sig[i] + dw;
    }
    const int u0 = nd + nz;
    for (int j = 0; j < m; ++j)
      for (int i = 0; i < nd; ++i)
        M[(size_t)(u0 + j) * N + i] = M[(size_t)i * N + u0 + j] = AD[(size_t)j * nd + i];
    for (int q = 0; q < nz; ++q)
      for (int j = 0; j < m; ++j)
        M[(size_t)(u0 + j) * N + nd + q] = M[(size_t)(nd + q) * N + u0 + j] = AS[(size_t)j * ns + zid[q]];
    for (int j = 0; j < m; ++j)
      for (int k = 0; k <= j; ++k) {
        double t = j == k ? dc : 0.0;
        const double* rj = &AS[(size_t)j * ns];
        const double* rk = &AS[(size_t)k * ns];
        for (int c = 0; c < ns; ++c)
          if (rj[c] != 0.0 && rk[c] != 0.0) t += rj[c] * rk[c] * Dinv[c];
        M[(size_t)(u0 + j) * N + u0 + k] = M[(size_t)(u0 + k) * N + u0 + j] = -t;
      }
    bkM.factor(N, M.data(), zero_tol);
    npos = (ns - nz) + bkM.npos;
    nneg = bkM.nneg;
    nzero = bkM.nzero;
  }
  void solve_indefinite(double* rhs) {
    // [w_D; w_Z; u] = M^-1 [r1; r2_Z; r3 - A_P D_P^-1 r2_P]; w_P = D_P^-1 (r2_P - A_P^T u)
    const int nz = (int)zid.size(), N = nd + nz + m, u0 = nd + nz;
    std::vector<double> q(N);
    for (int i = 0; i < nd; ++i) q[i] = rhs[i];
    for (int k = 0; k < nz; ++k) q[nd + k] = rhs[nd + zid[k]];
    for (int j = 0; j < m; ++j) {
      double s = rhs[n + j];
      const double* ra = &AS_[(size_t)j * ns];
      for (int c = 0; c < ns; ++c)
        if (ra[c] != 0.0) s -= ra[c] * Dinv[c] * rhs[nd + c];
      q[u0 + j] = s;
    }
    bkM.solve(q.data());
    for (int c = 0; c < ns; ++c) {
      if (Dinv[c] == 0.0) continue;
      double s = rhs[nd + c];
      for (int j = 0; j < m; ++j) s -= AS_[(size_t)j * ns + c] * q[u0 + j];
      rhs[nd + c] = s * Dinv[c];
    }
    for (int k = 0; k < nz; ++k) rhs[nd + zid[k]] = q[nd + k];
    for (int i = 0; i < nd; ++i) rhs[i] = q[i];
    for (int j = 0; j < m; ++j) rhs[n + j] = q[u0 + j];
  }

  // L^-1 x and L^-T x with the current factorization's L (on the device or in Kp)
  void lsolve(double* x) {
    if (dev_factor) {
      const int rc = nnc::dkkt_solve(dev->dk, x, 1);
      if (rc) dev_error = rc;
    } else {
      lower_solve1(nd, Kp, x, ldk);
    }
  }
  void usolve(double* x) {
    if (dev_factor) {
      const int rc = nnc::dkkt_solve(dev->dk, x, 0);
      if (rc) dev_error = rc;
    } else {
      upper_solve_lt(nd, Kp, x, ldk);
    }
  }
  bool full() const { return mode == 1; }
  void solve_core(double* rhs) {
    if (mode == 4) {
      solve_indefinite(rhs);
      return;
    }
    if (mode == 1) {
      bkF.solve(rhs);
      return;
    }
    if (mode == 3) {
      // [w_Z; z] = R^-1 [r2_Z; r3 - A_D K11^-1 r1 - A_P D_P^-1 r2_P]; then u and w_P as in mode 2
      const int nz = (int)zid.size();
      tmp.assign(rhs, rhs + nd);
      if (nd) lsolve(tmp.data());
      std::vector<double> q(nz + m);
      for (int k = 0; k < nz; ++k) q[k] = rhs[nd + zid[k]];
      const std::vector<double> yt = ytmul(nd, m, Y.data(), tmp.data());   // A_D K11^-1 r1 = Y^T t
      for (int j = 0; j < m; ++j) {
        double s = rhs[n + j] - yt[j];
        const double* ra = &AS_[(size_t)j * ns];
        for (int c = 0; c < ns; ++c)
          if (ra[c] != 0.0) s -= ra[c] * Dinv[c] * rhs[nd + c];
        q[nz + j] = s;
      }
      bkR.solve(q.data());
      const double* z = q.data() + nz;
      // u = K11^-1 (r1 - A_D^T z) with L^-1 (r1 - A_D^T z) = t - Y z: one backward solve
      std::vector<double> u(nd);
      for (int i = 0; i < nd; ++i) u[i] = tmp[i] - dot4(&Y[(size_t)i * m], z, m);
      if (nd) usolve(u.data());
      for (int c = 0; c < ns; ++c) {
        double s = rhs[nd + c];
        for (int j = 0; j < m; ++j) s -= AS_[(size_t)j * ns + c] * z[j];
        rhs[nd + c] = s * Dinv[c];
      }
      for (int k = 0; k < nz; ++k) rhs[nd + zid[k]] = q[k];
      for (int i = 0; i < nd; ++i) rhs[i] = u[i];
      for (int j = 0; j < m; ++j) rhs[n + j] = z[j];
      return;
    }
    if (mode == 2) {
      // z = T^-1 (r3 - A_D K11^-1 r1 - A_S D^-1 r2); u = K11^-1 (r1 - A_D^T z); w = D^-1 (r2 - A_S^T z)
      tmp.assign(rhs, rhs + nd);
      if (nd) lsolve(tmp.data());     // t = L^-1 r1; A_D K11^-1 r1 = Y^T t
      std::vector<double> z(m);
      const std::vector<double> yt = ytmul(nd, m, Y.data(), tmp.data());
      for (int j = 0; j < m; ++j) {
        double s = rhs[n + j] - yt[j];
        const double* ra = &AS_[(size_t)j * ns];
        for (int c = 0; c < ns; ++c)
          if (ra[c] != 0.0) s -= ra[c] * Dinv[c] * rhs[nd + c];
        z[j] = s;
      }
      if (t_chol) {      // T = -(L_T L_T^T)
        lower_solve1(m, T.data(), z.data());
        upper_solve_lt(m, T.data(), z.data());
        for (double& v : z) v = -v;
      } else {
        bkT.solve(z.data());
      }
      // u = K11^-1 (r1 - A_D^T z) with L^-1 (r1 - A_D^T z) = t - Y z (Y = L^-1 A_D^T is stored)
      std::vector<double> u(nd);
      for (int i = 0; i < nd; ++i) u[i] = tmp[i] - dot4(&Y[(size_t)i * m], z.data(), m);
      if (nd) usolve(u.data());
      for (int c = 0; c < ns; ++c) {
        double s = rhs[nd + c];
        for (int j = 0; j < m; ++j) s -= AS_[(size_t)j * ns + c] * z[j];
        rhs[nd + c] = s * Dinv[c];
      }
      for (int i = 0; i < nd; ++i) rhs[i] = u[i];
      for (int j = 0; j < m; ++j) rhs[n + j] = z[j];
      return;
    }
    // [K11 K12; K12^T K22] [u; w] = [r1; r2]: w = S^-1 (r2 - Y^T L^-1 r1), u = K11^-1 (r1 - K12 w)
    tmp.assign(rhs, rhs + nd);
    if (nd) lsolve(tmp.data());
    std::vector<double> w(r);
    const std::vector<double> yt = ytmul(nd, r, Y.data(), tmp.data());
    for (int a = 0; a < r; ++a) w[a] = rhs[nd + a] - yt[a];
    bkS.solve(w.data());
    // u = K11^-1 (r1 - K12 w) with L^-1 (r1 - K12 w) = t - Y w (Y = L^-1 K12)
    for (int i = 0; i < nd; ++i) tmp[i] -= dot4(&Y[(size_t)i * r], w.data(), r);
    if (nd) usolve(tmp.data());
    for (int i = 0; i < nd; ++i) rhs[i] = tmp[i];
    for (int a = 0; a < r; ++a) rhs[nd + a] = w[a];
  }
};

// ---------------------------------------------------------------- problem interface
// min f(v) s.t. c(v) = 0, lb <= v <= ub;  v = [D block (nd) | S block (ns)].
struct IpmProblem {
  int nd = 0, ns = 0, m = 0;
  std::vector<double> lb, ub, v0;
  virtual ~IpmProblem() = default;
  virtual double f(const double* v) = 0;
  virtual void grad_f(const double* v, double* g) = 0;
  virtual int cons(const double* v, double* c) = 0;                         // "Function"
  virtual int jac(const double* v, double* AD, double* AS) = 0;             // m x nd, m x ns
  // W_DD (nd x nd, full) and diag(W_SS) (ns) of grad^2 f + sum_i lam_i grad^2 c_i
  virtual int hess(const double* v, const double* lam, double* WDD, double* WSS) = 0;
  // Jacobian and Hessian at one point from one network evaluation (problems that can); the driver
  // then takes both at the top of an iteration.
  virtual bool joint() const { return false; }
  virtual int jac_hess(const double* v, const double* lam, double* AD, double* AS, double* WDD,
                       double* WSS) {
    const int rc = jac(v, AD, AS);
    return rc ? rc : hess(v, lam, WDD, WSS);
  }
  // Trial points (joint problems that can): the constraint values at v together with the
  // Jacobian and Hessian there for the multipliers lam_t that v gets if the step is accepted, from
  // one network evaluation; jac_hess at exactly (v, lam_t) then reuses them.
  virtual bool speculative() const { return false; }
  virtual int cons_spec(const double* v, const double* lam_t, double* c) {
    (void)lam_t;
    return cons(v, c);
  }
  // true when jac_hess(v, lam) will reuse the derivatives of the last cons_spec
  virtual bool has_derivs(const double* v, const double* lam) const {
    (void)v;
    (void)lam;
    return false;
  }
  // Problems whose network Hessian can stay in device memory: W_DD = dense_scale() H +
  // diag(dense_diag()) with H = dense_dev() (nd x nd FP64, valid after jac_hess), on the CUDA
  // stream dense_stream().  After set_dense_on_device(true) their jac_hess leaves WDD unwritten,
  // and host_wdd() copies H back and forms W_DD on the host (null on failure).
  virtual bool dense_capable() const { return false; }
  virtual bool set_dense_on_device(bool on) { return !on; }
  virtual const double* dense_dev() const { return nullptr; }
  virtual double dense_scale() const { return 1.0; }
  virtual const double* dense_diag() const { return nullptr; }
  virtual cudaStream_t dense_stream() const { return nullptr; }
  virtual const double* host_wdd() { return nullptr; }
  // Sparse problems (the full-space form): nd = 0, ns = n; fixed patterns of the Jacobian
  // (constraint jr[k], variable jc[k]) and of the lower triangle of the Lagrangian Hessian
  // (hr[k] >= hc[k]), values from jac_sp / hess_sp in pattern order, and the stage of every
  // variable and constraint for the block-tridiagonal KKT factorization (StageKkt).  jac, hess
  // and jac_hess are not called for them.
  virtual bool sparse() const { return false; }
  std::vector<int> jr, jc, hr, hc, var_stage, con_stage;
  virtual int jac_sp(const double* v, double* vals) {
    (void)v;
    (void)vals;
    return NNC_ERR_UNSUPPORTED;
  }
  virtual int hess_sp(const double* v, const double* lam, double* vals) {
    (void)v;
    (void)lam;
    (void)vals;
    return NNC_ERR_UNSUPPORTED;
  }
};

// Derivatives kept from a trial-point evaluation, keyed by the point and the multipliers.
struct SpecCache {
  std::vector<double> v, lam;
  bool valid = false;
  void store(const double* v_, size_t nv, const double* lam_, size_t nl) {
    v.assign(v_, v_ + nv);
    lam.assign(lam_, lam_ + nl);
    valid = true;
  }
  bool match(const double* v_, const double* lam_) const {
    return valid && std::memcmp(v.data(), v_, sizeof(double) * v.size()) == 0 &&
           std::memcmp(lam.data(), lam_, sizeof(double) * lam.size()) == 0;
  }
};

struct Timers {
  double fn = 0, jac = 0, hess = 0, solver = 0;
  int n_fn = 0, n_jac = 0, n_hess = 0;
};

double inf_norm(const std::vector<double>& x) {
  double s = 0;
  for (double v : x) s = std::max(s, std::fabs(v));
  return s;
}

int ipm_solve(IpmProblem& p, const nnc_ipm_options& o, std::vector<double>& v_out,
              std::vector<double>& lam_out, nnc_ipm_result* res, const double* v_start = nullptr,
              const double* lam_start = nullptr) {
  const auto t_start = Clock::now();
  Timers T;
  const int nd = p.nd, ns = p.ns, n = nd + ns, m = p.m, r = ns + m;
  std::vector<char> hasL(n), hasU(n);
  std::vector<double> lb0(n, 0.0), ub0(n, 0.0);
  for (int i = 0; i < n; ++i) {
    hasL[i] = std::isfinite(p.lb[i]);
    hasU[i] = std::isfinite(p.ub[i]);
    if (hasL[i]) lb0[i] = p.lb[i];
    if (hasU[i]) ub0[i] = p.ub[i];
  }
  std::vector<double> v(p.v0);
  if (v_start) v.assign(v_start, v_start + n);
  for (int i = 0; i < n; ++i) {
    const double width = (hasL[i] && hasU[i]) ? ub0[i] - lb0[i] : INFINITY;
    if (hasL[i]) v[i] = std::max(v[i], lb0[i] + std::min(o.kappa1 * std::max(1.0, std::fabs(lb0[i])), o.kappa2 * width));
    if (hasU[i]) v[i] = std::min(v[i], ub0[i] - std::min(o.kappa1 * std::max(1.0, std::fabs(ub0[i])), o.kappa2 * width));
  }
  std::vector<double> zL(n), zU(n), lam(m, 0.0);
  for (int i = 0; i < n; ++i) {
    zL[i] = hasL[i] ? 1.0 : 0.0;
    zU[i] = hasU[i] ? 1.0 : 0.0;
  }
  double mu = o.mu0;
  if (v_start && lam_start) {
    // warm start: given multipliers, small barrier parameter, z = mu / slack
    mu = o.warm_mu0;
    for (int j = 0; j < m; ++j) lam[j] = lam_start[j];
    for (int i = 0; i < n; ++i) {
      zL[i] = hasL[i] ? mu / (v[i] - lb0[i]) : 0.0;
      zU[i] = hasU[i] ? mu / (ub0[i] - v[i]) : 0.0;
    }
  }
  double tau = std::max(o.tau_min, 1.0 - mu), nu = 1.0, delta_w_last = 0.0;
  int ls_fail = 0, status = NNC_IPM_MAX_ITER, it = 0;
  double E0 = INFINITY;
  // sparse problems: Jacobian and Hessian values in their patterns, the block-tridiagonal KKT
  // factorization over the problem's stages; no dense Jacobian blocks
  const bool sp = p.sparse();
  std::vector<double> g(n), c(m), AD(sp ? 0 : (size_t)m * nd), AS(sp ? 0 : (size_t)m * ns),
      WDD((size_t)nd * nd), WSS(sp ? 0 : ns), Jv(sp ? p.jr.size() : 0), Hv(sp ? p.hr.size() : 0),
      vt(n), ct(m), lam_t(m), rhs(n + m), sol(n + m), dv(n), dl(m), dzL(n), dzU(n), sL(n), sU(n),
      SigL(n), SigU(n), sig(n), gphi(n), atl(n);
  KktSolver kkt;
  StageKkt skkt;
  if (sp && (nd != 0 || (int)p.var_stage.size() != n || (int)p.con_stage.size() != m ||
             p.jc.size() != p.jr.size() || p.hc.size() != p.hr.size() ||
             !skkt.setup(n, m, p.var_stage.data(), p.con_stage.data(), p.hr, p.hc, p.jr, p.jc)))
    return NNC_ERR_UNSUPPORTED;
  // the dense block on the device (tensor-core forms of the single-network problems)
  DenseOnDevice dense;
  const bool dev_kkt = o.kkt_on_device && nd > 0 && p.dense_capable() && p.set_dense_on_device(true);
  if (dev_kkt) {
    dense.dk = nnc::dkkt_create(nd, m, p.dense_stream());
    if (!dense.dk) {
      p.set_dense_on_device(false);
      return NNC_ERR_CUDA;
    }
    dense.s = p.dense_scale();
    dense.hf = p.dense_diag();
    dense.host_wdd = [&p]() { return p.host_wdd(); };
    kkt.dev = &dense;
  }
  struct DenseGuard {
    DenseOnDevice& d;
    IpmProblem& p;
    bool on;
    ~DenseGuard() {
      if (d.dk) nnc::dkkt_free(d.dk);
      if (on) p.set_dense_on_device(false);
    }
  } dense_guard{dense, p, dev_kkt};
  // atl = A^T lam, row by row (contiguous reads of the dense Jacobian blocks)
  auto update_atl = [&]() {
    if (sp) {
      std::fill(atl.begin(), atl.end(), 0.0);
      for (size_t k = 0; k < Jv.size(); ++k) atl[p.jc[k]] += Jv[k] * lam[p.jr[k]];
      return;
    }
#pragma omp parallel for schedule(static) if ((size_t)m * n > 65536)
    for (int i0 = 0; i0 < n; i0 += 64) {   // column blocks, rows streamed
      const int i1 = std::min(n, i0 + 64);
      for (int i = i0; i < i1; ++i) atl[i] = 0.0;
      for (int j = 0; j < m; ++j) {
        const double l = lam[j];
        if (l == 0.0) continue;
        for (int i = i0; i < i1; ++i)
          atl[i] += (i < nd ? AD[(size_t)j * nd + i] : AS[(size_t)j * ns + i - nd]) * l;
      }
    }
  };
  (void)r;
  auto slackL = [&](const std::vector<double>& x, int i) { return hasL[i] ? x[i] - lb0[i] : 1.0; };
  auto slackU = [&](const std::vector<double>& x, int i) { return hasU[i] ? ub0[i] - x[i] : 1.0; };
  auto timed = [&](double& acc, int& cnt, auto fn) {
    const auto a = Clock::now();
    const int rc = fn();
    acc += secs(a, Clock::now());
    ++cnt;
    return rc;
  };
  auto errors = [&](double mu_) {
    int nb = 0;
    double sl = 0, sz = 0;
    for (int j = 0; j < m; ++j) sl += std::fabs(lam[j]);
    for (int i = 0; i < n; ++i) {
      nb += hasL[i] + hasU[i];
      sz += std::fabs(zL[i]) + std::fabs(zU[i]);
    }
    const double s_d = std::max(o.s_max, (sl + sz) / std::max(1, m + nb)) / o.s_max;
    const double s_c = std::max(o.s_max, sz / std::max(1, nb)) / o.s_max;
    double rd = 0, comp = 0, cinf = 0;
    for (int i = 0; i < n; ++i) {
      const double d = g[i] - zL[i] + zU[i] + atl[i];
      rd = std::max(rd, std::fabs(d));
      if (hasL[i]) comp = std::max(comp, std::fabs((v[i] - lb0[i]) * zL[i] - mu_));
      if (hasU[i]) comp = std::max(comp, std::fabs((ub0[i] - v[i]) * zU[i] - mu_));
    }
    for (int j = 0; j < m; ++j) cinf = std::max(cinf, std::fabs(c[j]));
    return std::max(std::max(rd / s_d, cinf), comp / s_c);
  };
  auto merit = [&](const std::vector<double>& x, double fx, const std::vector<double>& cx, double nu_) {
    double phi = fx;
    for (int i = 0; i < n; ++i) {
      if (hasL[i]) {
        const double s = x[i] - lb0[i];
        if (!(s > 0)) return (double)INFINITY;
        phi -= mu * std::log(s);
      }
      if (hasU[i]) {
        const double s = ub0[i] - x[i];
        if (!(s > 0)) return (double)INFINITY;
        phi -= mu * std::log(s);
      }
    }
    double c1 = 0;
    for (int j = 0; j < m; ++j) c1 += std::fabs(cx[j]);
    return phi + nu_ * c1;
  };

  bool have_c = false;
  for (it = 0; it <= o.max_iter; ++it) {
    const double fv = p.f(v.data());
    p.grad_f(v.data(), g.data());
    if (!have_c && m) {
      if (timed(T.fn, T.n_fn, [&] { return p.cons(v.data(), c.data()); })) { status = NNC_IPM_EVAL_ERROR; break; }
    }
    if (sp) {
      if (m && timed(T.jac, T.n_jac, [&] { return p.jac_sp(v.data(), Jv.data()); })) { status = NNC_IPM_EVAL_ERROR; break; }
    } else if (m && p.joint() && p.has_derivs(v.data(), lam.data())) {
      // taken with the residual at the accepted trial point (counted there)
      if (p.jac_hess(v.data(), lam.data(), AD.data(), AS.data(), WDD.data(), WSS.data())) {
        status = NNC_IPM_EVAL_ERROR;
        break;
      }
    } else if (m && p.joint()) {
      // J and the Hessian of the Lagrangian at (v, lam) in one evaluation (counted as both)
      ++T.n_jac;
      if (timed(T.hess, T.n_hess, [&] {
            return p.jac_hess(v.data(), lam.data(), AD.data(), AS.data(), WDD.data(), WSS.data());
          })) { status = NNC_IPM_EVAL_ERROR; break; }
    } else if (m && timed(T.jac, T.n_jac, [&] { return p.jac(v.data(), AD.data(), AS.data()); })) { status = NNC_IPM_EVAL_ERROR; break; }
    bool finite = std::isfinite(fv);
    for (double x : g) finite &= std::isfinite(x);
    for (double x : c) finite &= std::isfinite(x);
    finite &= all_finite(AD.data(), AD.size()) && all_finite(Jv.data(), Jv.size());
    if (!finite) { status = NNC_IPM_NONFINITE; break; }
    update_atl();
    E0 = errors(0.0);
    if (o.verbose)
      std::printf("iter %3d  f %.10e  inf_pr %.3e  E0 %.3e  mu %.1e\n", it, fv, m ? inf_norm(c) : 0.0, E0, mu);
    if (E0 <= o.tol) { status = NNC_IPM_OPTIMAL; break; }
    if (it == o.max_iter) break;
    double Emu = errors(mu);
    while (Emu <= o.kappa_eps * mu && mu > o.tol / 10.0) {
      mu = std::max(o.tol / 10.0, std::min(o.kappa_mu * mu, std::pow(mu, o.theta_mu)));
      tau = std::max(o.tau_min, 1.0 - mu);
      Emu = errors(mu);
    }
    if (sp) {
      if (timed(T.hess, T.n_hess, [&] { return p.hess_sp(v.data(), lam.data(), Hv.data()); })) { status = NNC_IPM_EVAL_ERROR; break; }
    } else if (!(m && p.joint()) &&
        timed(T.hess, T.n_hess, [&] { return p.hess(v.data(), lam.data(), WDD.data(), WSS.data()); })) { status = NNC_IPM_EVAL_ERROR; break; }
    const auto t_lin = Clock::now();
    for (int i = 0; i < n; ++i) {
      sL[i] = slackL(v, i);
      sU[i] = slackU(v, i);
      SigL[i] = hasL[i] ? zL[i] / sL[i] : 0.0;
      SigU[i] = hasU[i] ? zU[i] / sU[i] : 0.0;
      gphi[i] = g[i] - (hasL[i] ? mu / sL[i] : 0.0) + (hasU[i] ? mu / sU[i] : 0.0);
    }
    for (int i = 0; i < n; ++i) rhs[i] = -(gphi[i] + atl[i]);
    for (int j = 0; j < m; ++j) rhs[n + j] = -c[j];
    // --- inertia-corrected factorization
    double delta_w = 0.0, delta_c = 0.0;
    bool first = true, ok = false;
    double scale = 1.0;
    if (dev_kkt) {
      dense.H = p.dense_dev();
      double mx = 0.0;
      if (nnc::dkkt_maxabs(dense.dk, dense.H, dense.s, dense.hf, &mx)) { status = NNC_IPM_EVAL_ERROR; break; }
      scale = std::max(scale, mx);
    } else {
      scale = std::max(scale, max_abs(WDD.data(), WDD.size()));
    }
    for (int i = 0; i < n; ++i) {
      sig[i] = SigL[i] + SigU[i];
      scale = std::max(scale, sig[i]);
    }
    scale = std::max(scale, max_abs(AD.data(), AD.size()));
    scale = std::max(scale, max_abs(AS.data(), AS.size()));
    scale = std::max(scale, max_abs(Jv.data(), Jv.size()));
    scale = std::max(scale, max_abs(Hv.data(), Hv.size()));
    const double zero_tol = 1e-14 * scale;
    int tries = 0;
    const auto t_fac = Clock::now();
    while (true) {
      ++tries;
      if (sp)
        skkt.factor(Hv.data(), sig.data(), Jv.data(), delta_w, delta_c, 1e-14);
      else
        kkt.factor(nd, ns, m, WDD.data(), WSS.data(), sig.data(), AD.data(), AS.data(), delta_w,
                   delta_c, zero_tol);
      if (kkt.dev_error) break;
      const int npos = sp ? skkt.npos : kkt.npos, nneg = sp ? skkt.nneg : kkt.nneg,
                nzero = sp ? skkt.nzero : kkt.nzero;
      if (npos == n && nneg == m && nzero == 0) { ok = true; break; }
      if (nzero > 0 && delta_c == 0.0 && m) delta_c = 1e-8 * std::pow(mu, 0.25);
      if (first) {
        delta_w = delta_w_last == 0.0 ? o.delta_w0 : std::max(o.delta_w_min, o.kappa_w_minus * delta_w_last);
        first = false;
      } else {
        delta_w *= delta_w_last == 0.0 ? o.kappa_w_plus_bar : o.kappa_w_plus;
      }
      if (delta_w > o.delta_w_max) break;
    }
    if (kkt.dev_error) { status = NNC_IPM_EVAL_ERROR; T.solver += secs(t_lin, Clock::now()); break; }
    if (!ok) { status = NNC_IPM_INERTIA_FAILED; T.solver += secs(t_lin, Clock::now()); break; }
    if (delta_w > 0.0) delta_w_last = delta_w;
    const auto t_sol = Clock::now();
    sol = rhs;
    if (sp) skkt.solve(sol.data());
    else kkt.solve(sol.data());
    if (kkt.dev_error) { status = NNC_IPM_EVAL_ERROR; T.solver += secs(t_lin, Clock::now()); break; }
    const auto t_sol_end = Clock::now();
    for (int i = 0; i < n; ++i) dv[i] = sol[i];
    for (int j = 0; j < m; ++j) dl[j] = sol[n + j];
    for (int i = 0; i < n; ++i) {
      dzL[i] = hasL[i] ? mu / sL[i] - zL[i] - SigL[i] * dv[i] : 0.0;
      dzU[i] = hasU[i] ? mu / sU[i] - zU[i] + SigU[i] * dv[i] : 0.0;
    }
    // --- fraction to the boundary
    double a_max = 1.0, a_z = 1.0;
    for (int i = 0; i < n; ++i) {
      if (hasL[i] && dv[i] < 0) a_max = std::min(a_max, -tau * sL[i] / dv[i]);
      if (hasU[i] && dv[i] > 0) a_max = std::min(a_max, tau * sU[i] / dv[i]);
      if (hasL[i] && dzL[i] < 0) a_z = std::min(a_z, -tau * zL[i] / dzL[i]);
      if (hasU[i] && dzU[i] < 0) a_z = std::min(a_z, -tau * zU[i] / dzU[i]);
    }
    // --- penalty parameter and directional derivative
    double c1 = 0, dphi = 0;
    for (int j = 0; j < m; ++j) c1 += std::fabs(c[j]);
    for (int i = 0; i < n; ++i) dphi += gphi[i] * dv[i];
    if (m && c1 > 0) {
      // curvature dv^T (W + Sigma + delta_w I) dv
      double curv = 0;
      if (dev_kkt) {
        // dv_D^T W_DD dv_D = s dv^T (H dv) + sum_i hf_i dv_i^2, H dv on the device
        std::vector<double> hv(nd);
        if (nnc::dkkt_matvec(dense.dk, dense.H, dv.data(), hv.data())) { status = NNC_IPM_EVAL_ERROR; break; }
        for (int i = 0; i < nd; ++i) curv += dv[i] * (dense.s * hv[i] + dense.hf[i] * dv[i]);
      } else if (sp) {
        for (size_t k = 0; k < Hv.size(); ++k)
          curv += (p.hr[k] == p.hc[k] ? 1.0 : 2.0) * Hv[k] * dv[p.hr[k]] * dv[p.hc[k]];
      } else {
#pragma omp parallel for reduction(+ : curv) schedule(static)
        for (int i = 0; i < nd; ++i) {
          double s = 0;
          for (int j = 0; j < nd; ++j) s += WDD[(size_t)i * nd + j] * dv[j];
          curv += dv[i] * s;
        }
      }
      for (int i = 0; i < n; ++i)
        curv += (SigL[i] + SigU[i] + delta_w + (!sp && i >= nd ? WSS[i - nd] : 0.0)) * dv[i] * dv[i];
      double lmax = 0;
      for (int j = 0; j < m; ++j) lmax = std::max(lmax, std::fabs(lam[j] + dl[j]));
      const double nu_req = (dphi + 0.5 * std::max(curv, 0.0)) / (0.9 * c1);
      nu = std::max(nu, std::max(lmax + 1.0, nu_req + 1.0));
    }
    const double D = dphi - nu * c1;
    T.solver += secs(t_lin, Clock::now());
    if (o.verbose)
      std::printf("          kkt mode %d, %d factorization(s), delta_w %.1e: factor %.2f ms, solve %.2f ms, "
                  "step set-up %.2f ms\n", sp ? 5 : kkt.mode, tries, delta_w, 1e3 * secs(t_fac, t_sol),
                  1e3 * secs(t_sol, t_sol_end),
                  1e3 * (secs(t_lin, Clock::now()) - secs(t_fac, t_sol) - secs(t_sol, t_sol_end)));
    const double phi0 = merit(v, fv, c, nu);
    double alpha = a_max;
    bool accepted = false;
    bool spec_taken = false;   // the accepted point is the first trial, evaluated with lam_t
    for (int bt = 0; bt < o.max_backtracks; ++bt) {
      for (int i = 0; i < n; ++i) vt[i] = v[i] + alpha * dv[i];
      const double ft = p.f(vt.data());
      if (m && bt == 0 && p.speculative()) {
        // the first trial is usually accepted: evaluate it with its derivatives (one network
        // evaluation instead of a residual now and a full evaluation at the next iteration)
        for (int j = 0; j < m; ++j) lam_t[j] = lam[j] + alpha * dl[j];
        ++T.n_fn;
        ++T.n_jac;
        if (timed(T.hess, T.n_hess, [&] { return p.cons_spec(vt.data(), lam_t.data(), ct.data()); })) {
          status = NNC_IPM_EVAL_ERROR;
          break;
        }
      } else if (m && timed(T.fn, T.n_fn, [&] { return p.cons(vt.data(), ct.data()); })) {
        status = NNC_IPM_EVAL_ERROR;
        break;
      }
      const double phit = merit(vt, ft, ct, nu);
      if (std::isfinite(phit) && phit <= phi0 + o.eta * alpha * D) {
        accepted = true;
        spec_taken = bt == 0 && p.speculative();
        break;
      }
      alpha *= 0.5;
    }
    if (status == NNC_IPM_EVAL_ERROR) break;
    if (!accepted) {
      if (++ls_fail >= o.max_ls_failures) { status = NNC_IPM_LINESEARCH_FAILED; break; }
      for (int i = 0; i < n; ++i) vt[i] = v[i] + alpha * dv[i];
      if (m && timed(T.fn, T.n_fn, [&] { return p.cons(vt.data(), ct.data()); })) { status = NNC_IPM_EVAL_ERROR; break; }
    } else {
      ls_fail = 0;
    }
    v = vt;
    c = ct;
    have_c = true;
    if (spec_taken) lam = lam_t;   // bit for bit the multipliers the trial was evaluated with
    else
      for (int j = 0; j < m; ++j) lam[j] += alpha * dl[j];
    for (int i = 0; i < n; ++i) {
      zL[i] += a_z * dzL[i];
      zU[i] += a_z * dzU[i];
      const double s_l = slackL(v, i), s_u = slackU(v, i);
      zL[i] = hasL[i] ? std::max(std::min(zL[i], o.kappa_sigma * mu / s_l), mu / (o.kappa_sigma * s_l)) : 0.0;
      zU[i] = hasU[i] ? std::max(std::min(zU[i], o.kappa_sigma * mu / s_u), mu / (o.kappa_sigma * s_u)) : 0.0;
    }
  }
  v_out = v;
  lam_out = lam;
  if (res) {
    res->status = status;
    res->iters = it;
    res->obj = p.f(v.data());
    res->kkt_error = E0;
    res->solve_seconds = secs(t_start, Clock::now());
    res->t_function = T.fn;
    res->t_jacobian = T.jac;
    res->t_hessian = T.hess;
    res->t_solver = T.solver;
    res->n_function = T.n_fn;
    res->n_jacobian = T.n_jac;
    res->n_hessian = T.n_hess;
  }
  return NNC_OK;
}

// ---------------------------------------------------------------- device-resident evaluation
// One network evaluation at an iterate whose Hessian of lambda^T NN stays in device memory (for
// the device factorization of the KKT dense block): x, y, lambda go in through one pinned staging
// buffer, the residual r = y - NN(x) and J come back, H stays in `H`.  Its own stream orders the
// evaluation before the factorization.
struct DevEval {
  nnc_net* net = nullptr;
  int n_in = 0, n_out = 0;
  cudaStream_t st = nullptr;
  double* d = nullptr;          // x | y | lam | r | J | H
  PinnedVec stage;              // x | y | lam | r | J
  PinnedVec hh;                 // host copy of H (indefinite iterations only)
  double *x = nullptr, *y = nullptr, *lam = nullptr, *r = nullptr, *J = nullptr, *H = nullptr;
  ~DevEval() { release(); }
  void release() {
    if (st) cudaStreamSynchronize(st);
    if (d) cudaFree(d);
    if (st) cudaStreamDestroy(st);
    d = nullptr;
    st = nullptr;
  }
  bool init(nnc_net* net_, int n_in_, int n_out_) {
    net = net_;
    n_in = n_in_;
    n_out = n_out_;
    const size_t nstage = (size_t)n_in + 3 * n_out + (size_t)n_out * n_in;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return false;
    if (cudaMalloc(&d, sizeof(double) * (nstage + (size_t)n_in * n_in)) != cudaSuccess) {
      cudaGetLastError();
      release();
      return false;
    }
    x = d;
    y = x + n_in;
    lam = y + n_out;
    r = lam + n_out;
    J = r + n_out;
    H = J + (size_t)n_out * n_in;
    stage.resize(nstage);
    return true;
  }
  // r (when yh is given) and J at (xh, lamh); H on the device
  int eval(const double* xh, const double* yh, const double* lamh, double* rh, double* Jh) {
    double* s = stage.data();
    std::memcpy(s, xh, sizeof(double) * n_in);
    if (yh) std::memcpy(s + n_in, yh, sizeof(double) * n_out);
    std::memcpy(s + n_in + n_out, lamh, sizeof(double) * n_out);
    if (cudaMemcpyAsync(x, s, sizeof(double) * (n_in + 2 * n_out), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return NNC_ERR_CUDA;
    int rc = nnc_eval_kkt_dev(net, x, yh ? y : nullptr, lam, yh ? r : nullptr, J, H, nullptr, st);
    if (rc) return rc;
    double* back = s + n_in + 2 * n_out;
    const size_t nb = (size_t)n_out + (size_t)n_out * n_in;
    if (cudaMemcpyAsync(back, r, sizeof(double) * nb, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return NNC_ERR_CUDA;
    if (yh && rh) std::memcpy(rh, back, sizeof(double) * n_out);
    std::memcpy(Jh, back + n_out, sizeof(double) * (size_t)n_out * n_in);
    return NNC_OK;
  }
  const double* hess_host() {
    if (!hh.data()) hh.resize((size_t)n_in * n_in);
    if (cudaMemcpyAsync(hh.data(), H, sizeof(double) * (size_t)n_in * n_in, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return nullptr;
    return hh.data();
  }
};

// Tensor-core forms only: the FP64 and FP32 forms keep the host factorization (their Hessian is
// as exact as the FP64 factorization, and the FP64 form is the reference path).
bool tensor_core_form(nnc_net* net) {
  int L = 0, ni = 0, no = 0, prec = 0;
  return nnc_net_info(net, &L, &ni, &no, &prec) == NNC_OK &&
         (prec == NNC_BF16 || prec == NNC_BF16X3 || prec == NNC_FP8);
}

// ---------------------------------------------------------------- adversarial problem
// Variables v = (x in [0,1]^n_in | y free in R^n_out, s >= 0 in R^(n_out-1)).
// min ||x - x0||^2  s.t.  y - NN(x) = 0,  y_t - y_j - margin - s_j = 0 (j != t).
struct Adversarial : IpmProblem {
  nnc_net* net;
  int n_in, n_out, t;
  double margin;
  std::vector<double> x0, J, r;
  PinnedVec H;
  std::vector<int> others;
  Adversarial(nnc_net* net_, const double* x0_, int n_in_, int n_out_, int t_, double margin_)
      : net(net_), n_in(n_in_), n_out(n_out_), t(t_), margin(margin_), x0(x0_, x0_ + n_in_) {
    nd = n_in;
    ns = n_out + (n_out - 1);
    m = n_out + (n_out - 1);
    for (int j = 0; j < n_out; ++j)
      if (j != t) others.push_back(j);
    lb.assign(nd + ns, -INFINITY);
    ub.assign(nd + ns, INFINITY);
    for (int i = 0; i < n_in; ++i) {
      lb[i] = 0.0;
      ub[i] = 1.0;
    }
    for (int j = 0; j < n_out - 1; ++j) lb[n_in + n_out + j] = 0.0;
    J.resize((size_t)n_out * n_in);
    H.resize((size_t)n_in * n_in);
    r.resize(n_out);
  }
  int start() {
    std::vector<double> y(n_out);
    int rc = nnc_eval(net, x0.data(), y.data(), 1);
    if (rc) return rc;
    v0.assign(nd + ns, 0.0);
    for (int i = 0; i < n_in; ++i) v0[i] = x0[i];
    for (int j = 0; j < n_out; ++j) v0[n_in + j] = y[j];
    for (int k = 0; k < n_out - 1; ++k)
      v0[n_in + n_out + k] = std::max(y[t] - y[others[k]] - margin, 1e-2);
    return NNC_OK;
  }
  double f(const double* v) override {
    double s = 0;
    for (int i = 0; i < n_in; ++i) s += (v[i] - x0[i]) * (v[i] - x0[i]);
    return s;
  }
  void grad_f(const double* v, double* g) override {
    for (int i = 0; i < nd + ns; ++i) g[i] = i < n_in ? 2.0 * (v[i] - x0[i]) : 0.0;
  }
  SpecCache spec;
  void fill_cons(const double* v, double* c) {
    for (int j = 0; j < n_out; ++j) c[j] = r[j];
    const double* y = v + n_in;
    const double* s = v + n_in + n_out;
    for (int k = 0; k < n_out - 1; ++k) c[n_out + k] = y[t] - y[others[k]] - margin - s[k];
  }
  int cons(const double* v, double* c) override {
    // y - NN(x) with the FP64 weights (the FP64 residual at step acceptance)
    int rc = nnc_residual(net, v, v + n_in, r.data());
    if (rc) return rc;
    fill_cons(v, c);
    return NNC_OK;
  }
  bool speculative() const override { return true; }
  int cons_spec(const double* v, const double* lam_t, double* c) override {
    spec.valid = false;
    int rc = dense_on ? de.eval(v, v + n_in, lam_t, r.data(), J.data())
                      : nnc_eval_kkt(net, v, v + n_in, lam_t, r.data(), J.data(), H.data(), nullptr);
    if (rc) return rc;
    spec.store(v, nd + ns, lam_t, m);
    fill_cons(v, c);
    return NNC_OK;
  }
  // device-resident Hessian: W_DD = -H + 2 I
  DevEval de;
  bool dense_on = false;
  std::vector<double> hf, wdd;
  bool dense_capable() const override { return tensor_core_form(net); }
  bool set_dense_on_device(bool on) override {
    if (on && !de.d && !de.init(net, n_in, n_out)) return false;
    dense_on = on;
    spec.valid = false;
    hf.assign(n_in, 2.0);
    return true;
  }
  const double* dense_dev() const override { return de.H; }
  double dense_scale() const override { return -1.0; }
  const double* dense_diag() const override { return hf.data(); }
  cudaStream_t dense_stream() const override { return de.st; }
  const double* host_wdd() override {
    const double* Hh = de.hess_host();
    if (!Hh) return nullptr;
    wdd.resize((size_t)nd * nd);
#pragma omp parallel for schedule(static) if (nd >= 256)
    for (int i = 0; i < nd; ++i) {
      for (int j = 0; j < nd; ++j) wdd[(size_t)i * nd + j] = -Hh[(size_t)i * nd + j];
      wdd[(size_t)i * nd + i] += 2.0;
    }
    return wdd.data();
  }
  bool has_derivs(const double* v, const double* lam) const override { return spec.match(v, lam); }
  int jac(const double* v, double* AD, double* AS) override {
    int rc = nnc_jacobian(net, v, J.data());
    if (rc) return rc;
    fill_jac(AD, AS);
    return NNC_OK;
  }
  int hess(const double* v, const double* lam, double* WDD, double* WSS) override {
    // grad^2 f = 2 I on x; sum_i lam_i grad^2 c_i = -sum_{i < n_out} lam_i grad^2 NN_i (Eq. 6)
    int rc = nnc_hessian_lag(net, v, lam, H.data(), nullptr);
    if (rc) return rc;
    fill_wdd(WDD, WSS);
    return NNC_OK;
  }
  void fill_wdd(double* WDD, double* WSS) {
#pragma omp parallel for schedule(static) if (nd >= 256)
    for (int i = 0; i < nd; ++i) {
      for (int j = 0; j < nd; ++j) WDD[(size_t)i * nd + j] = -H[(size_t)i * nd + j];
      WDD[(size_t)i * nd + i] += 2.0;
    }
    std::fill(WSS, WSS + ns, 0.0);
  }
  void fill_jac(double* AD, double* AS) {
    par_zero(AD, (size_t)m * nd);
    par_zero(AS, (size_t)m * ns);
    for (int j = 0; j < n_out; ++j) {
      for (int i = 0; i < n_in; ++i) AD[(size_t)j * nd + i] = -J[(size_t)j * n_in + i];
      AS[(size_t)j * ns + j] = 1.0;
    }
    for (int k = 0; k < n_out - 1; ++k) {
      AS[(size_t)(n_out + k) * ns + t] = 1.0;
      AS[(size_t)(n_out + k) * ns + others[k]] = -1.0;
      AS[(size_t)(n_out + k) * ns + n_out + k] = -1.0;
    }
  }
  bool joint() const override { return true; }
  int jac_hess(const double* v, const double* lam, double* AD, double* AS, double* WDD,
               double* WSS) override {
    if (!spec.match(v, lam)) {   // else J and H are those of the accepted trial point
      int rc = dense_on ? de.eval(v, nullptr, lam, nullptr, J.data())
                        : nnc_eval_kkt(net, v, nullptr, lam, nullptr, J.data(), H.data(), nullptr);
      if (rc) return rc;
    }
    spec.valid = false;
    fill_jac(AD, AS);
    if (dense_on) std::fill(WSS, WSS + ns, 0.0);
    else fill_wdd(WDD, WSS);
    return NNC_OK;
  }
};

// ---------------------------------------------------------------- Eq. 7: the L1 adversarial problem
// The smallest L1 change to a reference image that makes the classifier's (softmax) probability of
// the target class at least conf.  The L1 norm through split variables x - x_ref = p - q:
// variables v = (x in [0,1]^n | p >= 0, q >= 0 in R^n, y in R^n_out with y_t >= conf),
//   min sum(p) + sum(q)  s.t.  x - p + q - x_ref = 0,  y - NN(x) = 0.
// The dense block is x (the network's curvature); p, q and y are the diagonal block (p, q carry
// only barrier terms, y is free except y_t, so its zero diagonal stays beside the multipliers).
struct AdversarialL1 : IpmProblem {
  nnc_net* net;
  int n_in, n_out, t;
  double conf;
  std::vector<double> xr, J, r;
  PinnedVec H;
  AdversarialL1(nnc_net* net_, const double* x_ref, int n_in_, int n_out_, int t_, double conf_)
      : net(net_), n_in(n_in_), n_out(n_out_), t(t_), conf(conf_), xr(x_ref, x_ref + n_in_) {
    nd = n_in;
    ns = 2 * n_in + n_out;
    m = n_in + n_out;
    lb.assign(nd + ns, 0.0);
    ub.assign(nd + ns, INFINITY);
    for (int i = 0; i < n_in; ++i) ub[i] = 1.0;
    for (int j = 0; j < n_out; ++j) lb[3 * n_in + j] = -INFINITY;
    lb[3 * n_in + t] = conf;
    J.resize((size_t)n_out * n_in);
    H.resize((size_t)n_in * n_in);
    r.resize(n_out);
  }
  int start() {
    std::vector<double> y(n_out);
    int rc = nnc_eval(net, xr.data(), y.data(), 1);
    if (rc) return rc;
    v0.assign(nd + ns, 0.0);
    for (int i = 0; i < n_in; ++i) v0[i] = xr[i];
    for (int j = 0; j < n_out; ++j) v0[3 * n_in + j] = y[j];
    return NNC_OK;
  }
  double f(const double* v) override {
    double s = 0;
    for (int i = n_in; i < 3 * n_in; ++i) s += v[i];
    return s;
  }
  void grad_f(const double* v, double* g) override {
    for (int i = 0; i < nd + ns; ++i) g[i] = (i >= n_in && i < 3 * n_in) ? 1.0 : 0.0;
  }
  SpecCache spec;
  int cons(const double* v, double* c) override {
    for (int i = 0; i < n_in; ++i) c[i] = v[i] - v[n_in + i] + v[2 * n_in + i] - xr[i];
    int rc = nnc_residual(net, v, v + 3 * n_in, r.data());   // y - NN(x), FP64-accurate
    if (rc) return rc;
    for (int j = 0; j < n_out; ++j) c[n_in + j] = r[j];
    return NNC_OK;
  }
  bool speculative() const override { return true; }
  int cons_spec(const double* v, const double* lam_t, double* c) override {
    spec.valid = false;
    for (int i = 0; i < n_in; ++i) c[i] = v[i] - v[n_in + i] + v[2 * n_in + i] - xr[i];
    int rc = dense_on ? de.eval(v, v + 3 * n_in, lam_t + n_in, r.data(), J.data())
                      : nnc_eval_kkt(net, v, v + 3 * n_in, lam_t + n_in, r.data(), J.data(), H.data(), nullptr);
    if (rc) return rc;
    for (int j = 0; j < n_out; ++j) c[n_in + j] = r[j];
    spec.store(v, nd + ns, lam_t, m);
    return NNC_OK;
  }
  // device-resident Hessian: W_DD = -H (the objective is linear)
  DevEval de;
  bool dense_on = false;
  std::vector<double> hf, wdd;
  bool dense_capable() const override { return tensor_core_form(net); }
  bool set_dense_on_device(bool on) override {
    if (on && !de.d && !de.init(net, n_in, n_out)) return false;
    dense_on = on;
    spec.valid = false;
    hf.assign(n_in, 0.0);
    return true;
  }
  const double* dense_dev() const override { return de.H; }
  double dense_scale() const override { return -1.0; }
  const double* dense_diag() const override { return hf.data(); }
  cudaStream_t dense_stream() const override { return de.st; }
  const double* host_wdd() override {
    const double* Hh = de.hess_host();
    if (!Hh) return nullptr;
    wdd.resize((size_t)nd * nd);
#pragma omp parallel for schedule(static) if (nd >= 256)
    for (int i = 0; i < nd; ++i)
      for (int j = 0; j < nd; ++j) wdd[(size_t)i * nd + j] = -Hh[(size_t)i * nd + j];
    return wdd.data();
  }
  bool has_derivs(const double* v, const double* lam) const override { return spec.match(v, lam); }
  void fill_jac(double* AD, double* AS) {
    par_zero(AD, (size_t)m * nd);
    par_zero(AS, (size_t)m * ns);
    for (int i = 0; i < n_in; ++i) {
      AD[(size_t)i * nd + i] = 1.0;
      AS[(size_t)i * ns + i] = -1.0;            // p_i
      AS[(size_t)i * ns + n_in + i] = 1.0;      // q_i
    }
    for (int j = 0; j < n_out; ++j) {
      for (int i = 0; i < n_in; ++i) AD[(size_t)(n_in + j) * nd + i] = -J[(size_t)j * n_in + i];
      AS[(size_t)(n_in + j) * ns + 2 * n_in + j] = 1.0;   // y_j
    }
  }
  void fill_wdd(double* WDD, double* WSS) {
#pragma omp parallel for schedule(static) if (nd >= 256)
    for (int i = 0; i < nd; ++i)
      for (int j = 0; j < nd; ++j) WDD[(size_t)i * nd + j] = -H[(size_t)i * nd + j];
    std::fill(WSS, WSS + ns, 0.0);
  }
  int jac(const double* v, double* AD, double* AS) override {
    int rc = nnc_jacobian(net, v, J.data());
    if (rc) return rc;
    fill_jac(AD, AS);
    return NNC_OK;
  }
  int hess(const double* v, const double* lam, double* WDD, double* WSS) override {
    // the objective is linear; sum_i lam_i grad^2 c_i = -sum_j lam_{n+j} grad^2 NN_j (Eq. 6)
    int rc = nnc_hessian_lag(net, v, lam + n_in, H.data(), nullptr);
    if (rc) return rc;
    fill_wdd(WDD, WSS);
    return NNC_OK;
  }
  bool joint() const override { return true; }
  int jac_hess(const double* v, const double* lam, double* AD, double* AS, double* WDD,
               double* WSS) override {
    if (!spec.match(v, lam)) {   // else J and H are those of the accepted trial point
      int rc = dense_on ? de.eval(v, nullptr, lam + n_in, nullptr, J.data())
                        : nnc_eval_kkt(net, v, nullptr, lam + n_in, nullptr, J.data(), H.data(), nullptr);
      if (rc) return rc;
    }
    spec.valid = false;
    fill_jac(AD, AS);
    if (dense_on) std::fill(WSS, WSS + ns, 0.0);
    else fill_wdd(WDD, WSS);
    return NNC_OK;
  }
};

// ---------------------------------------------------------------- Eq. 7 in the full space (Eq. 4)
// The network as per-layer variables and constraints: z_l - W_l y_{l-1} - b_l = 0 and
// y_l - sigma_l(z_l) = 0 (y_0 = x, y_L = y), with the objective, bounds and split variables of
// AdversarialL1.  Natural variable order v = (x, p, q, z_1, y_1, ..., z_L, y_L); constraints
// (link, then per layer the affine rows and the activation rows).  The Hessian of the Lagrangian
// is diagonal except for a softmax output (an n_out x n_out block on z_L).  Functions are affine
// maps and elementwise activations evaluated on the host (the paper evaluates its full-space
// model on the CPU too).  The Jacobian (the weights, sigma' and the identity links) and the
// Hessian stay sparse, and the KKT matrix, block tridiagonal over the chain of stages
// (p, q) | link multipliers | x | (affine multipliers, z_1) | (activation multipliers, y_1) | ...,
// is factorized stage by stage (StageKkt), where the paper uses a general sparse LDL^T (MA57).
namespace {
void host_act(int act, double z, double& a, double& d1, double& d2) {
  switch (act) {
    case NNC_TANH: {
      const double t = std::tanh(z);
      a = t;
      d1 = 1.0 - t * t;
      d2 = -2.0 * t * d1;
      return;
    }
    case NNC_SIGMOID: {
      const double e = std::exp(-std::fabs(z));
      const double sg = z >= 0 ? 1.0 / (1.0 + e) : e / (1.0 + e);
      a = sg;
      d1 = sg * (1.0 - sg);
      d2 = d1 * (1.0 - 2.0 * sg);
      return;
    }
    case NNC_SOFTPLUS: {
      const double e = std::exp(-std::fabs(z));
      a = (z > 0 ? z : 0.0) + std::log1p(e);
      const double sg = z >= 0 ? 1.0 / (1.0 + e) : e / (1.0 + e);
      d1 = sg;
      d2 = sg * (1.0 - sg);
      return;
    }
    case NNC_GELU: {
      const double phi = std::exp(-0.5 * z * z) / std::sqrt(2.0 * M_PI);
      const double Phi = 0.5 * (1.0 + std::erf(z / std::sqrt(2.0)));
      a = z * Phi;
      d1 = Phi + z * phi;
      d2 = phi * (2.0 - z * z);
      return;
    }
    default:
      a = z;
      d1 = 1.0;
      d2 = 0.0;
  }
}
void host_softmax(const double* z, int k, double* p) {
  double mx = z[0];
  for (int i = 1; i < k; ++i) mx = std::max(mx, z[i]);
  double s = 0;
  for (int i = 0; i < k; ++i) s += (p[i] = std::exp(z[i] - mx));
  for (int i = 0; i < k; ++i) p[i] /= s;
}
}  // namespace

struct AdversarialL1Full : IpmProblem {
  int n = 0, L = 0, t = 0, nv = 0;
  double conf = 0.6;
  std::vector<int> w, act, off_z, off_y, off_aff, off_act;
  std::vector<std::vector<double>> W, b;
  std::vector<double> xr, tmp;
  // Jacobian entries whose values change with v: act rows (sigma' or the softmax block)
  size_t j_act0 = 0;
  bool sparse() const override { return true; }
  int load(nnc_net* net, const double* x_ref, int target, double conf_) {
    int nl = 0, ni = 0, no = 0, prec = 0;
    int rc = nnc_net_info(net, &nl, &ni, &no, &prec);
    if (rc) return rc;
    L = nl;
    n = ni;
    t = target;
    conf = conf_;
    w.assign(1, n);
    act.resize(L);
    W.resize(L);
    b.resize(L);
    for (int l = 0; l < L; ++l) {
      int rows = 0, cols = 0;
      rc = nnc_layer_weights(net, l, nullptr, nullptr, &act[l], &rows, &cols);
      if (rc) return rc;
      W[l].resize((size_t)rows * cols);
      b[l].resize(rows);
      rc = nnc_layer_weights(net, l, W[l].data(), b[l].data(), nullptr, nullptr, nullptr);
      if (rc) return rc;
      w.push_back(rows);
    }
    for (int l = 0; l + 1 < L; ++l)
      if (act[l] == NNC_SOFTMAX) return NNC_ERR_UNSUPPORTED;
    // variables (x, p, q, z_1, y_1, ..., z_L, y_L); constraints (link rows, then per layer the
    // affine and the activation rows)
    int k = 3 * n, r = n;
    m = n;
    off_z.clear();
    off_y.clear();
    off_aff.clear();
    off_act.clear();
    for (int l = 0; l < L; ++l) {
      off_z.push_back(k);
      k += w[l + 1];
      off_y.push_back(k);
      k += w[l + 1];
      off_aff.push_back(r);
      r += w[l + 1];
      off_act.push_back(r);
      r += w[l + 1];
    }
    m = r;
    nv = k;
    nd = 0;
    ns = nv;
    // stages of the block-tridiagonal KKT factorization: (p, q) | link multipliers | x | then per
    // layer: (affine multipliers, z_l) | (activation multipliers, y_l).  Every nonzero couples a
    // stage with itself or a neighbour.  Each multiplier shares its stage with the variable it
    // links by an identity (z_l, y_l): alone, the affine multipliers of a layer wider than the one
    // before would form a singular block (W_l F^-1 W_l^T has the rank of the narrower layer).
    var_stage.assign(nv, 0);
    con_stage.assign(m, 0);
    for (int i = 0; i < n; ++i) var_stage[i] = 2;
    for (int l = 0; l < L; ++l) {
      const int s0 = 3 + 2 * l;
      for (int j = 0; j < w[l + 1]; ++j) {
        con_stage[off_aff[l] + j] = s0;
        var_stage[off_z[l] + j] = s0;
        con_stage[off_act[l] + j] = s0 + 1;
        var_stage[off_y[l] + j] = s0 + 1;
      }
    }
    for (int i = 0; i < n; ++i) con_stage[i] = 1;
    // Jacobian pattern: constant entries first, then the activation rows' entries
    jr.clear();
    jc.clear();
    auto ent = [&](int row, int col) {
      jr.push_back(row);
      jc.push_back(col);
    };
    for (int i = 0; i < n; ++i) {
      ent(i, i);
      ent(i, n + i);
      ent(i, 2 * n + i);
    }
    for (int l = 0; l < L; ++l) {
      const int kk = w[l + 1], kin = w[l], prev = l == 0 ? 0 : off_y[l - 1];
      for (int j = 0; j < kk; ++j) {
        ent(off_aff[l] + j, off_z[l] + j);
        for (int c = 0; c < kin; ++c) ent(off_aff[l] + j, prev + c);
      }
      for (int j = 0; j < kk; ++j) ent(off_act[l] + j, off_y[l] + j);
    }
    j_act0 = jr.size();
    for (int l = 0; l < L; ++l) {
      const int kk = w[l + 1];
      for (int j = 0; j < kk; ++j) {
        if (act[l] == NNC_SOFTMAX)
          for (int c = 0; c < kk; ++c) ent(off_act[l] + j, off_z[l] + c);
        else
          ent(off_act[l] + j, off_z[l] + j);
      }
    }
    // Hessian pattern (lower triangle): sigma'' on each z_l, the softmax block of z_L
    hr.clear();
    hc.clear();
    for (int l = 0; l < L; ++l) {
      const int kk = w[l + 1];
      for (int i = 0; i < kk; ++i) {
        if (act[l] == NNC_SOFTMAX) {
          for (int j = 0; j <= i; ++j) {
            hr.push_back(off_z[l] + i);
            hc.push_back(off_z[l] + j);
          }
        } else {
          hr.push_back(off_z[l] + i);
          hc.push_back(off_z[l] + i);
        }
      }
    }
    std::vector<double> lbn(nv, -INFINITY), ubn(nv, INFINITY);
    for (int i = 0; i < 3 * n; ++i) lbn[i] = 0.0;
    for (int i = 0; i < n; ++i) ubn[i] = 1.0;
    lbn[off_y[L - 1] + t] = conf;
    lb = lbn;
    ub = ubn;
    // start: x = x_ref, p = q = 0, (z_l, y_l) of the forward pass at x_ref
    xr.assign(x_ref, x_ref + n);
    v0.assign(nv, 0.0);
    for (int i = 0; i < n; ++i) v0[i] = xr[i];
    for (int l = 0; l < L; ++l) {
      const double* yp = l == 0 ? v0.data() : &v0[off_y[l - 1]];
      affine(l, yp, &v0[off_z[l]]);
      activate(l, &v0[off_z[l]], &v0[off_y[l]]);
    }
    return NNC_OK;
  }
  void affine(int l, const double* yp, double* z) const {
    const int rows = w[l + 1], cols = w[l];
#pragma omp parallel for schedule(static) if ((size_t)rows * cols > 65536)
    for (int r = 0; r < rows; ++r) {
      double s = b[l][r];
      const double* wr = &W[l][(size_t)r * cols];
      for (int c = 0; c < cols; ++c) s += wr[c] * yp[c];
      z[r] = s;
    }
  }
  void activate(int l, const double* z, double* y) const {
    if (act[l] == NNC_SOFTMAX) {
      host_softmax(z, w[l + 1], y);
      return;
    }
    double d1, d2;
    for (int r = 0; r < w[l + 1]; ++r) host_act(act[l], z[r], y[r], d1, d2);
  }
  double f(const double* v) override {
    double s = 0;
    for (int i = n; i < 3 * n; ++i) s += v[i];
    return s;
  }
  void grad_f(const double* v, double* g) override {
    (void)v;
    for (int i = 0; i < nv; ++i) g[i] = (i >= n && i < 3 * n) ? 1.0 : 0.0;
  }
  int cons(const double* v, double* c) override {
    for (int i = 0; i < n; ++i) c[i] = v[i] - v[n + i] + v[2 * n + i] - xr[i];
    for (int l = 0; l < L; ++l) {
      const int k = w[l + 1];
      const double* yp = l == 0 ? v : &v[off_y[l - 1]];
      tmp.resize(k);
      affine(l, yp, tmp.data());
      for (int j = 0; j < k; ++j) c[off_aff[l] + j] = v[off_z[l] + j] - tmp[j];
      activate(l, &v[off_z[l]], tmp.data());
      for (int j = 0; j < k; ++j) c[off_act[l] + j] = v[off_y[l] + j] - tmp[j];
    }
    return NNC_OK;
  }
  int jac(const double*, double*, double*) override { return NNC_ERR_UNSUPPORTED; }
  int hess(const double*, const double*, double*, double*) override { return NNC_ERR_UNSUPPORTED; }
  int jac_sp(const double* v, double* vals) override {
    size_t k = 0;
    for (int i = 0; i < n; ++i) {
      vals[k++] = 1.0;
      vals[k++] = -1.0;
      vals[k++] = 1.0;
    }
    for (int l = 0; l < L; ++l) {
      const int kk = w[l + 1], kin = w[l];
      for (int j = 0; j < kk; ++j) {
        vals[k++] = 1.0;
        const double* wr = &W[l][(size_t)j * kin];
        for (int c = 0; c < kin; ++c) vals[k++] = -wr[c];
      }
      for (int j = 0; j < kk; ++j) vals[k++] = 1.0;
    }
    for (int l = 0; l < L; ++l) {
      const int kk = w[l + 1];
      const double* z = &v[off_z[l]];
      if (act[l] == NNC_SOFTMAX) {
        tmp.resize(kk);
        host_softmax(z, kk, tmp.data());
        for (int j = 0; j < kk; ++j)
          for (int c = 0; c < kk; ++c) vals[k++] = -(tmp[j] * ((j == c) - tmp[c]));
      } else {
        for (int j = 0; j < kk; ++j) {
          double a, d1, d2;
          host_act(act[l], z[j], a, d1, d2);
          vals[k++] = -d1;
        }
      }
    }
    return k == jr.size() ? NNC_OK : NNC_ERR_ARG;
  }
  int hess_sp(const double* v, const double* lam, double* vals) override {
    // only y_l - sigma_l(z_l) is nonlinear: its multipliers mu give -grad^2 (mu^T sigma_l(z_l))
    size_t k = 0;
    for (int l = 0; l < L; ++l) {
      const int kk = w[l + 1];
      const double* mu = lam + off_act[l];
      const double* z = &v[off_z[l]];
      if (act[l] == NNC_SOFTMAX) {
        // sum_i mu_i grad^2 p_i = diag(p (mu - mubar)) - p (p mu)^T - (p mu) p^T + 2 mubar p p^T
        tmp.resize(kk);
        host_softmax(z, kk, tmp.data());
        double mb = 0;
        for (int i = 0; i < kk; ++i) mb += tmp[i] * mu[i];
        for (int i = 0; i < kk; ++i)
          for (int j = 0; j <= i; ++j) {
            double cij = -tmp[i] * tmp[j] * mu[j] - tmp[i] * mu[i] * tmp[j] + 2.0 * mb * tmp[i] * tmp[j];
            if (i == j) cij += tmp[i] * (mu[i] - mb);
            vals[k++] = -cij;
          }
      } else {
        for (int j = 0; j < kk; ++j) {
          double a, d1, d2;
          host_act(act[l], z[j], a, d1, d2);
          vals[k++] = -mu[j] * d2;
        }
      }
    }
    return k == hr.size() ? NNC_OK : NNC_ERR_ARG;
  }
};

// ---------------------------------------------------------------- SCOPF-shaped batch problem
// Variables v = (x in [0,1]^G | y in R^K, y >= 0).
// min sum_i c_i x_i^2  s.t.  y_k - (NN_k(x[S_k]) + shift_k) = 0,  sum_i x_i - D = 0.
// shift_k = delta_k - NN_k(xbar[S_k]) calibrates every margin to delta_k at xbar = D/G.
struct Scopf : IpmProblem {
  nnc_batch* b;
  int G, K, n_sum;
  long long h_sum;
  std::vector<int> sub, off, nk;
  std::vector<double> cost, shift, xc, yc, lc, Jc, Hc, rc;
  double D;
  Scopf(nnc_batch* b_, int G_, const int* subsets, const double* cost_, double D_)
      : b(b_), G(G_), D(D_) {
    int no = 0;
    nnc_batch_info(b, &K, &no, &n_sum, &h_sum);
    sub.assign(subsets, subsets + n_sum);
    cost.assign(cost_, cost_ + G);
    nd = G;
    ns = K;
    m = K + 1;
    lb.assign(nd + ns, 0.0);
    ub.assign(nd + ns, INFINITY);
    for (int i = 0; i < G; ++i) ub[i] = 1.0;
    xc.resize(n_sum);
    yc.resize(K);
    lc.resize(K);
    Jc.resize(n_sum);
    Hc.resize(h_sum);
    rc.resize(K);
    shift.assign(K, 0.0);
  }
  void set_offsets(const std::vector<int>& n_in) {
    nk = n_in;
    off.resize(K);
    int o = 0;
    for (int k = 0; k < K; ++k) {
      off[k] = o;
      o += nk[k];
    }
  }
  void gather(const double* v) {
    for (int j = 0; j < n_sum; ++j) xc[j] = v[sub[j]];
  }
  int start(const double* delta) {
    v0.assign(nd + ns, D / G);
    gather(v0.data());
    std::fill(yc.begin(), yc.end(), 0.0);
    int r = nnc_batch_residual(b, xc.data(), yc.data(), rc.data());  // r = -NN(xbar)
    if (r) return r;
    for (int k = 0; k < K; ++k) {
      shift[k] = delta[k] + rc[k];
      v0[G + k] = delta[k];
    }
    return NNC_OK;
  }
  double f(const double* v) override {
    double s = 0;
    for (int i = 0; i < G; ++i) s += cost[i] * v[i] * v[i];
    return s;
  }
  void grad_f(const double* v, double* g) override {
    for (int i = 0; i < nd + ns; ++i) g[i] = i < G ? 2.0 * cost[i] * v[i] : 0.0;
  }
  SpecCache spec;
  void fill_cons(const double* v, double* c) {
    double sx = 0;
    for (int i = 0; i < G; ++i) sx += v[i];
    for (int k = 0; k < K; ++k) c[k] = rc[k];
    c[K] = sx - D;
  }
  int cons(const double* v, double* c) override {
    gather(v);
    for (int k = 0; k < K; ++k) yc[k] = v[G + k] - shift[k];
    int r = nnc_batch_residual(b, xc.data(), yc.data(), rc.data());
    if (r) return r;
    fill_cons(v, c);
    return NNC_OK;
  }
  bool speculative() const override { return true; }
  int cons_spec(const double* v, const double* lam_t, double* c) override {
    spec.valid = false;
    gather(v);
    for (int k = 0; k < K; ++k) {
      yc[k] = v[G + k] - shift[k];
      lc[k] = lam_t[k];
    }
    int r = nnc_batch_eval_kkt(b, xc.data(), yc.data(), lc.data(), rc.data(), Jc.data(), Hc.data(), nullptr);
    if (r) return r;
    fill_cons(v, c);
    spec.store(v, nd + ns, lam_t, m);
    return NNC_OK;
  }
  bool has_derivs(const double* v, const double* lam) const override { return spec.match(v, lam); }
  int jac(const double* v, double* AD, double* AS) override {
    gather(v);
    int r = nnc_batch_eval(b, xc.data(), nullptr, nullptr, Jc.data(), nullptr, nullptr);
    if (r) return r;
    fill_jac(AD, AS);
    return NNC_OK;
  }
  void fill_jac(double* AD, double* AS) {
    par_zero(AD, (size_t)m * nd);
    par_zero(AS, (size_t)m * ns);
    for (int k = 0; k < K; ++k) {
      for (int j = 0; j < nk[k]; ++j) AD[(size_t)k * nd + sub[off[k] + j]] -= Jc[off[k] + j];
      AS[(size_t)k * ns + k] = 1.0;
    }
    for (int i = 0; i < G; ++i) AD[(size_t)K * nd + i] = 1.0;
  }
  int hess(const double* v, const double* lam, double* WDD, double* WSS) override {
    gather(v);
    for (int k = 0; k < K; ++k) lc[k] = lam[k];
    int r = nnc_batch_eval(b, xc.data(), lc.data(), nullptr, nullptr, Hc.data(), nullptr);
    if (r) return r;
    fill_wdd(WDD, WSS);
    return NNC_OK;
  }
  bool joint() const override { return true; }
  int jac_hess(const double* v, const double* lam, double* AD, double* AS, double* WDD,
               double* WSS) override {
    if (!spec.match(v, lam)) {   // else J and H are those of the accepted trial point
      gather(v);
      for (int k = 0; k < K; ++k) lc[k] = lam[k];
      int r = nnc_batch_eval(b, xc.data(), lc.data(), nullptr, Jc.data(), Hc.data(), nullptr);
      if (r) return r;
    }
    spec.valid = false;
    fill_jac(AD, AS);
    fill_wdd(WDD, WSS);
    return NNC_OK;
  }
  void fill_wdd(double* WDD, double* WSS) {
    std::fill(WDD, WDD + (size_t)nd * nd, 0.0);
    for (int i = 0; i < G; ++i) WDD[(size_t)i * nd + i] = 2.0 * cost[i];
    long long h = 0;
    for (int k = 0; k < K; ++k) {
      const int n = nk[k];
      const int* S = &sub[off[k]];
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) WDD[(size_t)S[i] * nd + S[j]] -= Hc[h + (long long)i * n + j];
      h += (long long)n * n;
    }
    std::fill(WSS, WSS + ns, 0.0);
  }
};

}  // namespace

extern "C" {

int nnc_ipm_scopf_warm(nnc_batch* batch, int G, const int* n_in, const int* subsets,
                       const double* cost, double demand, const double* delta,
                       const double* v_start, const double* lam_start, const nnc_ipm_options* opt,
                       double* v_out, double* lam_out, nnc_ipm_result* res) {
  int K = 0, no = 0, n_sum = 0;
  long long h_sum = 0;
  int rc = nnc_batch_info(batch, &K, &no, &n_sum, &h_sum);
  if (rc) return rc;
  if (G < 1 || !n_in || !subsets || !cost || !delta || no != 1) return NNC_ERR_ARG;
  int tot = 0;
  for (int k = 0; k < K; ++k) tot += n_in[k];
  if (tot != n_sum) return NNC_ERR_ARG;
  for (int j = 0; j < n_sum; ++j)
    if (subsets[j] < 0 || subsets[j] >= G) return NNC_ERR_ARG;
  nnc_ipm_options o;
  if (opt) o = *opt;
  else nnc_ipm_default_options(&o);
  Scopf p(batch, G, subsets, cost, demand);
  p.set_offsets(std::vector<int>(n_in, n_in + K));
  rc = p.start(delta);
  if (rc) return rc;
  std::vector<double> v, lam;
  rc = ipm_solve(p, o, v, lam, res, v_start, v_start ? lam_start : nullptr);
  if (rc) return rc;
  if (v_out) std::copy(v.begin(), v.end(), v_out);
  if (lam_out) std::copy(lam.begin(), lam.end(), lam_out);
  return NNC_OK;
}

int nnc_ipm_scopf(nnc_batch* batch, int G, const int* n_in, const int* subsets, const double* cost,
                  double demand, const double* delta, const nnc_ipm_options* opt, double* v_out,
                  double* lam_out, nnc_ipm_result* res) {
  return nnc_ipm_scopf_warm(batch, G, n_in, subsets, cost, demand, delta, nullptr, nullptr, opt,
                            v_out, lam_out, res);
}

int nnc_kkt_solve(int nd, int ns, int m, const double* WDD, const double* WSS, const double* sigma,
                  const double* AD, const double* AS, double delta_w, double delta_c,
                  double* rhs_sol, int* inertia) {
  if (nd < 0 || ns < 0 || m < 0 || (nd && !WDD) || (ns && !WSS) || !sigma || !rhs_sol ||
      (m && nd && !AD) || (m && ns && !AS))
    return NNC_ERR_ARG;
  const int n = nd + ns;
  double scale = 1.0;
  for (size_t i = 0; i < (size_t)nd * nd; ++i) scale = std::max(scale, std::fabs(WDD[i]));
  for (int i = 0; i < n; ++i) scale = std::max(scale, std::fabs(sigma[i]));
  for (size_t i = 0; i < (size_t)m * nd; ++i) scale = std::max(scale, std::fabs(AD[i]));
  for (size_t i = 0; i < (size_t)m * ns; ++i) scale = std::max(scale, std::fabs(AS[i]));
  std::vector<double> wss(WSS ? WSS : nullptr, WSS ? WSS + ns : nullptr);
  wss.resize(ns, 0.0);
  std::vector<double> ad(AD ? AD : nullptr, AD ? AD + (size_t)m * nd : nullptr);
  ad.resize((size_t)m * nd, 0.0);
  std::vector<double> as(AS ? AS : nullptr, AS ? AS + (size_t)m * ns : nullptr);
  as.resize((size_t)m * ns, 0.0);
  KktSolver k;
  k.factor(nd, ns, m, WDD, wss.data(), sigma, ad.data(), as.data(), delta_w, delta_c, 1e-14 * scale);
  if (inertia) {
    inertia[0] = k.npos;
    inertia[1] = k.nneg;
    inertia[2] = k.nzero;
    inertia[3] = k.full() ? 1 : 0;
  }
  if (k.nzero == 0) k.solve(rhs_sol);
  return NNC_OK;
}

int nnc_stage_kkt_solve(int n, int m, const int* var_stage, const int* con_stage, int nw,
                        const int* wr, const int* wc, const double* wv, int nj, const int* jr,
                        const int* jc, const double* jv, const double* sigma, double delta_w,
                        double delta_c, double* rhs_sol, int* inertia) {
  if (n < 0 || m < 0 || nw < 0 || nj < 0 || !var_stage || (m && !con_stage) || !sigma || !rhs_sol ||
      (nw && (!wr || !wc || !wv)) || (nj && (!jr || !jc || !jv)))
    return NNC_ERR_ARG;
  for (int k = 0; k < nw; ++k)
    if (wr[k] < 0 || wr[k] >= n || wc[k] < 0 || wc[k] > wr[k]) return NNC_ERR_ARG;
  for (int k = 0; k < nj; ++k)
    if (jr[k] < 0 || jr[k] >= m || jc[k] < 0 || jc[k] >= n) return NNC_ERR_ARG;
  std::vector<int> hr(wr, wr + nw), hc(wc, wc + nw), ar(jr, jr + nj), ac(jc, jc + nj);
  StageKkt k;
  if (!k.setup(n, m, var_stage, con_stage, hr, hc, ar, ac)) return NNC_ERR_UNSUPPORTED;
  k.factor(wv, sigma, jv, delta_w, delta_c, 1e-14);
  if (inertia) {
    inertia[0] = k.npos;
    inertia[1] = k.nneg;
    inertia[2] = k.nzero;
  }
  if (k.nzero == 0) k.solve(rhs_sol);
  return NNC_OK;
}

void nnc_ipm_default_options(nnc_ipm_options* o) {
  if (!o) return;
  o->tol = 1e-6;
  o->max_iter = 300;
  o->mu0 = 0.1;
  o->kappa_mu = 0.2;
  o->theta_mu = 1.5;
  o->kappa_eps = 10.0;
  o->tau_min = 0.99;
  o->kappa1 = 1e-2;
  o->kappa2 = 1e-2;
  o->s_max = 100.0;
  o->eta = 1e-4;
  o->delta_w0 = 1e-4;
  o->delta_w_min = 1e-20;
  o->delta_w_max = 1e40;
  o->kappa_w_plus = 8.0;
  o->kappa_w_plus_bar = 100.0;
  o->kappa_w_minus = 1.0 / 3.0;
  o->kappa_sigma = 1e10;
  o->max_backtracks = 40;
  o->max_ls_failures = 5;
  o->verbose = 0;
  o->warm_mu0 = 1e-3;
  o->kkt_on_device = 0;
}

int nnc_ipm_adversarial(nnc_net* net, const double* x0, int target, double margin,
                        const nnc_ipm_options* opt, double* v_out, double* lam_out,
                        nnc_ipm_result* res) {
  int L = 0, n_in = 0, n_out = 0, prec = 0;
  int rc = nnc_net_info(net, &L, &n_in, &n_out, &prec);
  if (rc) return rc;
  if (!x0 || target < 0 || target >= n_out || n_out < 2) return NNC_ERR_ARG;
  nnc_ipm_options o;
  if (opt) o = *opt;
  else nnc_ipm_default_options(&o);
  Adversarial p(net, x0, n_in, n_out, target, margin);
  rc = p.start();
  if (rc) return rc;
  std::vector<double> v, lam;
  rc = ipm_solve(p, o, v, lam, res);
  if (rc) return rc;
  if (v_out) std::copy(v.begin(), v.end(), v_out);
  if (lam_out) std::copy(lam.begin(), lam.end(), lam_out);
  return NNC_OK;
}

int nnc_ipm_adversarial_l1_fullspace(nnc_net* net, const double* x_ref, int target, double conf,
                                     const nnc_ipm_options* opt, double* v_out, double* lam_out,
                                     nnc_ipm_result* res) {
  int L = 0, n_in = 0, n_out = 0, prec = 0;
  int rc = nnc_net_info(net, &L, &n_in, &n_out, &prec);
  if (rc) return rc;
  if (!x_ref || target < 0 || target >= n_out || !(conf > 0.0 && conf < 1.0)) return NNC_ERR_ARG;
  nnc_ipm_options o;
  if (opt) o = *opt;
  else nnc_ipm_default_options(&o);
  AdversarialL1Full p;
  rc = p.load(net, x_ref, target, conf);
  if (rc) return rc;
  std::vector<double> v, lam;
  rc = ipm_solve(p, o, v, lam, res);
  if (rc) return rc;
  if (v_out) std::copy(v.begin(), v.end(), v_out);
  if (lam_out) std::copy(lam.begin(), lam.end(), lam_out);
  return NNC_OK;
}

int nnc_ipm_adversarial_l1(nnc_net* net, const double* x_ref, int target, double conf,
                           const nnc_ipm_options* opt, double* v_out, double* lam_out,
                           nnc_ipm_result* res) {
  int L = 0, n_in = 0, n_out = 0, prec = 0;
  int rc = nnc_net_info(net, &L, &n_in, &n_out, &prec);
  if (rc) return rc;
  if (!x_ref || target < 0 || target >= n_out || !(conf > 0.0 && conf < 1.0)) return NNC_ERR_ARG;
  nnc_ipm_options o;
  if (opt) o = *opt;
  else nnc_ipm_default_options(&o);
  AdversarialL1 p(net, x_ref, n_in, n_out, target, conf);
  rc = p.start();
  if (rc) return rc;
  std::vector<double> v, lam;
  rc = ipm_solve(p, o, v, lam, res);
  if (rc) return rc;
  if (v_out) std::copy(v.begin(), v.end(), v_out);
  if (lam_out) std::copy(lam.begin(), lam.end(), lam_out);
  return NNC_OK;
}

}  // extern "C"
