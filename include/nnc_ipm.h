/*
 * nnc_ipm.h -- host FP64 interior-point driver of libnnc for problems with an embedded network
 * constraint in the reduced-space form (Eq. 5): the network enters as y - NN(x) = 0 and its
 * value, Jacobian and Hessian of lambda^T NN come from the nnc_* oracles of nnc.h.
 *
 * The method is a primal-dual barrier method for Eq. 1 whose Newton system is Eq. 2 with the
 * unstated terms alpha, beta read as IPOPT's barrier terms (Waechter & Biegler 2006): inertia
 * correction delta_w, barrier parameter mu with monotone decrease, fraction to the boundary,
 * backtracking on an exact-penalty merit function.  The merit checks and all optimizer state stay
 * in FP64 on the host; so does the KKT factorization, except the dense block of the tensor-core
 * forms (opt->kkt_on_device).  The constraint residual y - NN(x) is always FP64-accurate
 * (nnc_residual), whatever the net's precision form.
 *
 * Ownership: all pointers are host memory owned by the caller.  Errors: negative nnc_status
 * for bad arguments or a failing oracle call; the solver's own outcome is in result->status.
 */
#ifndef NNC_IPM_H
#define NNC_IPM_H

#include "nnc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* result->status */
#define NNC_IPM_OPTIMAL 0           /* scaled KKT error <= tol */
#define NNC_IPM_MAX_ITER 1          /* iteration limit reached */
#define NNC_IPM_LINESEARCH_FAILED 2 /* max_ls_failures consecutive line searches failed */
#define NNC_IPM_NONFINITE 3         /* NaN or Inf in a function or derivative */
#define NNC_IPM_INERTIA_FAILED 4    /* delta_w exceeded delta_w_max */
#define NNC_IPM_EVAL_ERROR 5        /* an nnc_* oracle call failed (see nnc_last_error) */

typedef struct {
  double tol;              /* 1e-6, the paper's IPOPT tolerance (Section 5.1) */
  int max_iter;            /* 300 */
  double mu0;              /* 0.1 */
  double kappa_mu;         /* 0.2 */
  double theta_mu;         /* 1.5 */
  double kappa_eps;        /* 10 */
  double tau_min;          /* 0.99 */
  double kappa1, kappa2;   /* 1e-2: push of the start point into the bounds */
  double s_max;            /* 100: scaling of the optimality error */
  double eta;              /* 1e-4: Armijo constant */
  double delta_w0, delta_w_min, delta_w_max;         /* 1e-4, 1e-20, 1e40 */
  double kappa_w_plus, kappa_w_plus_bar, kappa_w_minus; /* 8, 100, 1/3 */
  double kappa_sigma;      /* 1e10: safeguard of the bound multipliers */
  int max_backtracks;      /* 40 */
  int max_ls_failures;     /* 5 */
  int verbose;             /* print one line per iteration */
  double warm_mu0;         /* 1e-3: barrier parameter of a warm start (z = warm_mu0 / slack) */
  int kkt_on_device;       /* 1: for the single-network problems in the tensor-core forms (NNC_BF16,
                            * NNC_BF16X3, NNC_FP8) the Hessian stays in device memory and the dense
                            * block of the KKT matrix is assembled, factorized and solved on the GPU
                            * (Jacobi-scaled FP32 blocked Cholesky of the bordered matrix in one
                            * cooperative launch, triangular solves on the device, only the border
                            * rows go to the host; an indefinite or nearly singular block, pivot
                            * <= 1e-5 of the unit diagonal, goes to the FP64 host path).  0 (default):
                            * everything on the host, which is faster at n_in = 784 on a 16-core
                            * host (the device factorization is latency-bound).  The FP64 and FP32
                            * forms and the SCOPF-shaped problem always factorize on the host. */
} nnc_ipm_options;

typedef struct {
  int status;              /* NNC_IPM_* */
  int iters;
  double obj;              /* objective at the returned point */
  double kkt_error;        /* scaled optimality error E_0 at the returned point */
  double solve_seconds;    /* wall time of the solve */
  /* breakdown of Table 4: Function (constraint residuals), Jacobian, Hessian, Solver
   * (factorization, solves, step computation); seconds and number of calls */
  double t_function, t_jacobian, t_hessian, t_solver;
  int n_function, n_jacobian, n_hessian;
} nnc_ipm_result;

void nnc_ipm_default_options(nnc_ipm_options* opt);

/* The KKT system of Eq. 2 in the structured form the driver factorizes (host FP64):
 *   K = [[W_DD + diag(sigma_D) + dw I, 0,                          A_D^T],
 *        [0,                           diag(W_SS + sigma_S) + dw I, A_S^T],
 *        [A_D,                         A_S,                         -dc I]]
 * with nd dense-block variables, ns small-block variables and m constraints (n = nd + ns).
 *   WDD : nd x nd row-major (symmetric);  WSS, sigma : ns and n entries;
 *   AD  : m x nd row-major;  AS : m x ns row-major (NULL = zero when the size is 0);
 *   rhs_sol : n + m doubles, the right-hand side on entry, the solution on return (left
 *             unchanged when K is singular);
 *   inertia : 4 ints (may be NULL): positive, negative and zero eigenvalue counts of K, and 1
 *             if the whole matrix had to be factorized (first block not positive definite and
 *             a negative small-block diagonal entry), else 0.
 * Factorization: rows that pin one dense variable through slack variables of their own (such
 * as x_i - p_i + q_i = x_ref,i) are eliminated first; then blocked Cholesky of the first block
 * and Bunch-Kaufman LDL^T of the reduced multiplier system, or, when the first block is
 * indefinite, Bunch-Kaufman of the dense block, the zero-diagonal variables and the multipliers
 * together (positive small-block diagonals eliminated), or of all of K.  The inertia is exact
 * in every form (Sylvester / Haynsworth). */
int nnc_kkt_solve(int nd, int ns, int m, const double* WDD, const double* WSS, const double* sigma,
                  const double* AD, const double* AS, double delta_w, double delta_c,
                  double* rhs_sol, int* inertia);

/* The sparse KKT solve of the full-space problems (host, FP64): K = [[W + diag(sigma) + delta_w I,
 * A^T], [A, -delta_c I]] with W (n x n, symmetric) given by its lower-triangle triplets
 * (wr[k] >= wc[k], values wv, repeated entries add up) and A (m x n) by triplets (constraint jr[k],
 * variable jc[k], values jv).  Every variable i has a stage var_stage[i] >= 0 and every constraint
 * j a stage con_stage[j]; every nonzero of W and A must couple a stage with itself or with the
 * next or previous one (K block tridiagonal over the stages).  K is factorized as L diag(F_s) L^T
 * with F_s = K_ss - K_{s,s-1} F_{s-1}^{-1} K_{s-1,s} (dense, Bunch-Kaufman with 1 x 1 and 2 x 2
 * pivots), so inertia(K) = sum_s inertia(F_s) exactly.  rhs_sol (n + m): the right-hand side,
 * overwritten by the solution when inertia[2] == 0 (else unchanged).  inertia (3 ints, may be
 * NULL): (positive, negative, zero) eigenvalue counts.  Each F_s is equilibrated (R F_s R with
 * R = diag(1 / sqrt(largest entry of each row)), which keeps its inertia) and a pivot of at most
 * 1e-14 there counts as zero; a zero is also reported when a leading block F_s is singular
 * although K is not (this solver pivots within stages only).  NNC_ERR_ARG for bad sizes, pointers or indices,
 * NNC_ERR_UNSUPPORTED when a nonzero couples stages that are not neighbours. */
int nnc_stage_kkt_solve(int n, int m, const int* var_stage, const int* con_stage, int nw,
                        const int* wr, const int* wc, const double* wv, int nj, const int* jr,
                        const int* jc, const double* jv, const double* sigma, double delta_w,
                        double delta_c, double* rhs_sol, int* inertia);

/* Eq. 7 itself: the smallest L1 change to the reference image x_ref that makes the classifier's
 * output t at least conf (a probability, for a softmax output layer: 0 < conf < 1).  Split
 * variables carry the L1 norm: v = (x in [0,1]^n_in, p >= 0, q >= 0 in R^n_in, y in R^n_out with
 * y_t >= conf),  min sum(p) + sum(q)  s.t.  x - p + q - x_ref = 0,  y - NN(x) = 0.
 * Start: x = x_ref, p = q = 0, y = NN(x_ref) (pushed into the bounds by the solver).
 *   v_out   : 3 n_in + n_out doubles (may be NULL);  lam_out : n_in + n_out doubles (may be NULL).
 *   result  : may be NULL. */
int nnc_ipm_adversarial_l1(nnc_net* net, const double* x_ref, int target, double conf,
                           const nnc_ipm_options* opt, double* v_out, double* lam_out,
                           nnc_ipm_result* result);

/* Eq. 7 with the network in the full space (Eq. 4): every layer's affine output z_l and
 * activation output y_l are variables, tied by z_l - W_l y_{l-1} - b_l = 0 and
 * y_l - sigma_l(z_l) = 0 (y_0 = x, y_L = y); objective, bounds and split variables as in
 * nnc_ipm_adversarial_l1, so both forms have the same optima.  Functions are evaluated on the host
 * from the net's FP64 weights; the Jacobian and the Hessian of the Lagrangian are kept sparse and
 * the KKT matrix is factorized stage by stage (nnc_stage_kkt_solve) over the chain
 * (p, q) | link multipliers | x | per layer: (affine multipliers, z_l) | (activation
 * multipliers, y_l), so memory and work grow with the sum over layers of (layer width)^3, not
 * with (variables + constraints)^3.
 *   v_out   : (x, p, q, z_1, y_1, ..., z_L, y_L): 3 n_in + 2 sum_l n_l doubles (may be NULL);
 *   lam_out : (link rows, then per layer the affine and the activation rows):
 *             n_in + 2 sum_l n_l doubles (may be NULL);  result : may be NULL. */
int nnc_ipm_adversarial_l1_fullspace(nnc_net* net, const double* x_ref, int target, double conf,
                                     const nnc_ipm_options* opt, double* v_out, double* lam_out,
                                     nnc_ipm_result* res);

/* The adversarial problem (a synthetic variant of Eq. 7): variables v = (x, y, s) with
 * x in [0,1]^n_in, y in R^n_out, s in R^(n_out-1), s >= 0;
 *   min ||x - x0||^2  s.t.  y - NN(x) = 0,  y_t - y_j - margin - s_j = 0 for j != t.
 * Start: x = x0, y = NN(x0) (FP64), s_j = max(y_t - y_j - margin, 1e-2).
 *   x0      : n_in doubles.      target : t in [0, n_out).     opt : NULL for defaults.
 *   v_out   : n_in + 2 n_out - 1 doubles (may be NULL), the final (x, y, s).
 *   lam_out : 2 n_out - 1 doubles (may be NULL), multipliers of (y - NN(x), margins).
 *   result  : may be NULL. */
int nnc_ipm_adversarial(nnc_net* net, const double* x0, int target, double margin,
                        const nnc_ipm_options* opt, double* v_out, double* lam_out,
                        nnc_ipm_result* result);

/* The SCOPF-shaped problem (a synthetic variant of Eq. 8), one surrogate per contingency in
 * `batch` (n_out = 1; see nnc_batch_create):  variables v = (x in [0,1]^G, y in R^K, y >= 0);
 *   min sum_i c_i x_i^2  s.t.  y_k - (NN_k(x[S_k]) + shift_k) = 0 (k < K),  sum_i x_i = demand,
 * where shift_k = delta_k - NN_k(xbar[S_k]) puts every margin at delta_k for the flat dispatch
 * xbar = demand / G (the start point).
 *   n_in    : K ints, the input count of each surrogate (must match the batch);
 *   subsets : sum_k n_in[k] ints, S_k concatenated (generator indices in [0, G));
 *   cost    : G doubles;  delta : K doubles (> 0);  opt : NULL for defaults;
 *   v_out   : G + K doubles (may be NULL);  lam_out : K + 1 doubles (may be NULL). */
int nnc_ipm_scopf(nnc_batch* batch, int G, const int* n_in, const int* subsets, const double* cost,
                  double demand, const double* delta, const nnc_ipm_options* opt, double* v_out,
                  double* lam_out, nnc_ipm_result* result);
/* The same problem from a predicted start (a learned warm start): v_start (G + K) is pushed into
 * the bounds like any start, the constraint multipliers start at lam_start (K + 1), the barrier
 * parameter at opt->warm_mu0 and every bound multiplier at warm_mu0 / slack. */
int nnc_ipm_scopf_warm(nnc_batch* batch, int G, const int* n_in, const int* subsets,
                       const double* cost, double demand, const double* delta,
                       const double* v_start, const double* lam_start, const nnc_ipm_options* opt,
                       double* v_out, double* lam_out, nnc_ipm_result* result);

#ifdef __cplusplus
}
#endif
#endif /* NNC_IPM_H */
