/*
 * nnc.h -- C ABI of libnnc: oracles for a neural-network constraint y = NN(x) embedded in a
 * nonlinear program, computed by hand-written CUDA kernels for sm_103a (GB300).
 *
 * The problem is Eq. 1 of the paper (min f(x) s.t. g(x) = 0, x >= 0).  In the reduced-space
 * ("gray-box") formulation of Section 3.2 the network appears as the single vector constraint
 * g(x, y) = y - NN(x) (Eq. 5), and an interior-point method (Eq. 2) asks at every iteration for
 *   - the value NN(x),
 *   - the dense Jacobian dNN/dx  (n_out x n_in),
 *   - the dense n_in x n_in matrix sum_i lambda_i d2 NN_i/dx2, the Hessian of the scalar
 *     lambda^T NN(x) (Eq. 6, Section 3.2.1).
 * NN is the multilayer perceptron of Eq. 3: z_l = W_l a_{l-1} + b_l, a_l = sigma_l(z_l),
 * a_0 = x, NN(x) = a_L, with W_l of shape d_l x d_{l-1} and d_0 = n_in, d_L = n_out.
 *
 * Conventions shared by every entry point
 *   - Return value: NNC_OK (0) on success, a negative nnc_status otherwise.  Nothing aborts or
 *     throws across this interface.  nnc_last_error() gives a message for the calling thread.
 *   - Host pointers ("const double* x"): owned by the caller, read or written during the call
 *     only; the call copies them to or from the device and returns after the device work and
 *     the copies have finished.  An output in page-locked memory (cudaHostAlloc,
 *     cudaHostRegister) is written in place by the kernel that forms it, without a copy.
 *   - Device pointers (entry points ending in _dev): owned by the caller, must stay valid
 *     until the work queued on `stream` has finished; the call returns once the work is
 *     queued (asynchronous).  `stream` is a cudaStream_t; NULL means the net's own stream.
 *   - All matrices are dense, row-major, FP64, without padding.
 *   - One net may be used by one host thread at a time; calls on one net are serialised on
 *     its stream.  Different nets are independent.
 *   - There is no CPU fallback: without a usable sm_103a device every call returns
 *     NNC_ERR_CUDA.
 */
#ifndef NNC_H
#define NNC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nnc_net nnc_net; /* opaque; the library owns all of its device memory */

typedef enum {
  NNC_OK = 0,
  NNC_ERR_ARG = -1,         /* bad argument: null pointer, bad size or code */
  NNC_ERR_CUDA = -2,        /* a CUDA call failed or no sm_103a device */
  NNC_ERR_NONFINITE = -3,   /* an input (x or lambda) holds NaN or Inf */
  NNC_ERR_TIMEOUT = -4,     /* a bounded device-side wait ran out; outputs are undefined */
  NNC_ERR_OOM = -5,         /* device allocation failed */
  NNC_ERR_UNSUPPORTED = -6  /* request not supported for this net (e.g. activation/precision) */
} nnc_status;

/* Number format of the network evaluation (Section 5.1 leaves it unstated).
 *   NNC_FP64   : every kernel in FP64 (value, Jacobian, Hessian).  The reference form.
 *   NNC_FP32   : FP32 weights and tangents on CUDA cores, FP32 products, FP64 outputs.
 *   NNC_BF16   : value/Jacobian/adjoint in FP32; Hessian sweep on tcgen05 tensor cores with
 *                BF16 operands and FP32 accumulation (one product per tile).
 *   NNC_BF16X3 : as NNC_BF16, but every tensor-core product is split-BF16x3 compensated:
 *                A*B ~ Ahi*Bhi + Ahi*Blo + Alo*Bhi, all three accumulated in one FP32 tile.
 *   NNC_FP8    : as NNC_BF16, but the Hessian sweep runs kind::f8f6f4 with e4m3 weights and
 *                per-output-row scales.  Reported, not held to the BF16 tolerances.
 * nnc_residual (and nnc_eval with fp64_residual != 0) is FP64 in the NNC_FP64 form; in every other
 * form it runs in double-float arithmetic (each value an unevaluated sum of two FP32 numbers, about
 * 48 significant bits) on (hi, lo) pairs of the FP64 weights, and is held to
 * |r - r_fp64| <= 1e-10 * max(1, |y|). */
typedef enum { NNC_FP64 = 0, NNC_FP32 = 1, NNC_BF16 = 2, NNC_BF16X3 = 3, NNC_FP8 = 4 } nnc_precision;

/* sigma_l of Eq. 3.  All are C^2, as interior-point methods require (Section 2). */
/* NNC_SOFTMAX: output layer only (n_out <= 64): p = softmax(z_L), the classifiers of Section 4.1.
 * Its second derivative couples the outputs; the library adds that coupling to H exactly. */
typedef enum {
  NNC_IDENTITY = 0, NNC_TANH = 1, NNC_SIGMOID = 2, NNC_SOFTPLUS = 3, NNC_GELU = 4, NNC_SOFTMAX = 5
} nnc_act;

/* Bits of `what` in nnc_eval_batched. */
#define NNC_WANT_Y 1u    /* value NN(x) */
#define NNC_WANT_J 2u    /* Jacobian dNN/dx */
#define NNC_WANT_H 4u    /* Hessian of lambda^T NN (needs lambda) */
#define NNC_WANT_G 8u    /* gradient lambda^T dNN/dx (needs lambda) */

/* Build a net on the current CUDA device from FP64 host weights (Eq. 3; the weights are
 * constant during optimisation, Section 3).
 *   out      : receives the new net (NULL on failure).
 *   n_layers : L >= 1.
 *   widths   : L+1 entries d_0..d_L, each in [1, 65536].
 *   act      : L entries of nnc_act, sigma_1..sigma_L.
 *   W        : L host pointers; W[l] is d_{l+1} x d_l row-major (layer l+1 of the paper).
 *   b        : L host pointers; b[l] has d_{l+1} entries; b itself or b[l] may be NULL (zero).
 *   prec     : nnc_precision of the Hessian / Jacobian / value kernels.
 *   stream   : cudaStream_t the net queues its work on; NULL creates a private stream.
 * The weights are copied and packed once (FP64 copy, FP32 copy, BF16 hi/lo split, FP8 with
 * per-row scales, as the precision needs); the caller may free W and b on return. */
int nnc_load_weights(nnc_net** out, int n_layers, const int* widths, const int* act,
                     const double* const* W, const double* const* b, int prec, void* stream);

/* y = NN(x) (Eq. 3).  x: n_in doubles; y: n_out doubles.  fp64_residual != 0 evaluates with the
 * FP64-accurate value pass whatever the precision form (the FP64 correction of the residual):
 * FP64 weights in the NNC_FP64 form, double-float (hi, lo) weight pairs in the others. */
int nnc_eval(nnc_net* net, const double* x, double* y, int fp64_residual);

/* r = y - NN(x) on the device, FP64-accurate: the residual of g(x, y) = y - NN(x) (Eq. 5) used
 * at step acceptance (FP64 in the NNC_FP64 form, double-float in the others, as stated above).
 * x: n_in, y: n_out, r: n_out doubles. */
int nnc_residual(nnc_net* net, const double* x, const double* y, double* r);

/* J = dNN/dx at x by a reverse sweep with n_out seed columns (the Jacobian oracle of
 * Section 2).  J: n_out x n_in row-major. */
int nnc_jacobian(nnc_net* net, const double* x, double* J);

/* H = sum_i lambda_i d2 NN_i/dx2 at x (Eq. 6): the Hessian of the scalar lambda^T NN(x),
 * computed without forming the third-order tensor.  H: n_in x n_in row-major, exactly
 * symmetric.  grad (may be NULL): the gradient lambda^T dNN/dx, n_in doubles.  The caller
 * applies the sign of g = y - NN and adds the objective's Hessian. */
int nnc_hessian_lag(nnc_net* net, const double* x, const double* lambda, double* H, double* grad);

/* Several nets (each with its own sizes) evaluated together: for k < K, the outputs selected
 * by `what` (NNC_WANT_* bits) for nets[k] at x[k] (and lambda[k]).  Arrays of K host pointers;
 * y[k], J[k], H[k] may be NULL when not requested (the whole array may be NULL if its bit is
 * not set).  All nets must share one precision and one CUDA device.  With K = 1 this is the
 * single-net "everything at one point" call of one interior-point iteration. */
int nnc_eval_batched(nnc_net* const* nets, int K, const double* const* x,
                     const double* const* lambda, double* const* y, double* const* J,
                     double* const* H, unsigned what);

/* Device-pointer twins (asynchronous on `stream`, NULL = the net's stream).  Same meanings as
 * above; every pointer is device memory of the stated size in doubles. */
int nnc_eval_dev(nnc_net* net, const double* x, double* y, int fp64_residual, void* stream);
int nnc_residual_dev(nnc_net* net, const double* x, const double* y, double* r, void* stream);
int nnc_jacobian_dev(nnc_net* net, const double* x, double* J, void* stream);
int nnc_hessian_lag_dev(nnc_net* net, const double* x, const double* lambda, double* H,
                        double* grad, void* stream);
/* One-net "everything" call on device pointers: y, J, H, grad may each be NULL (skipped). */
int nnc_eval_all_dev(nnc_net* net, const double* x, const double* lambda, double* y, double* J,
                     double* H, double* grad, void* stream);
/* What one interior-point iteration asks of the constraint y - NN(x) = 0 at the iterate (x, y)
 * (Eq. 2 with the constraint of Eq. 3, Hessian term of Eq. 6), from a single value pass: the
 * residual r = y - NN(x) at the accuracy of nnc_residual (FP64, or double-float with about 48
 * significant bits in the other forms), J = dNN/dx, H = sum_i lambda_i d2 NN_i/dx2 and
 * grad = lambda^T J.  Device pointers; r, J, H, grad may each be NULL (y is needed for r, lambda
 * for H and grad).  Asynchronous on `stream` (NULL = the net's stream). */
int nnc_eval_kkt_dev(nnc_net* net, const double* x, const double* y, const double* lambda,
                     double* r, double* J, double* H, double* grad, void* stream);
/* Host-pointer twin of nnc_eval_kkt_dev (copies in, evaluates, copies out, waits). */
int nnc_eval_kkt(nnc_net* net, const double* x, const double* y, const double* lambda, double* r,
                 double* J, double* H, double* grad);

/* ---- Grouped batch (many networks of equal hidden widths, different input sizes) ----------
 * One stability-margin surrogate per contingency of Eq. 8: K nets with the same depth, hidden
 * widths, activations and n_out (<= 3), each with its own n_in (<= 256), all BF16 or BF16X3.
 * nnc_batch_create stacks their packed weights (the nets stay valid and unchanged) so that
 * every step of the evaluation is one grouped launch for all K nets.  Concatenated layouts:
 *   x_cat      : sum_k n_in_k doubles, net k's input at offset off_k = sum_{j<k} n_in_j;
 *   lambda_cat : K x n_out;  y_cat, r_cat : K x n_out;  grad_cat : like x_cat;
 *   J_cat      : net k's n_out x n_in_k block (row-major) at offset off_k * n_out;
 *   H_cat      : net k's n_in_k x n_in_k block (row-major, symmetric) at offset
 *                hoff_k = sum_{j<k} n_in_j^2.
 * nnc_eval_batched uses this path (with a cached batch) when its nets qualify and evaluates
 * the nets one after another otherwise. */
typedef struct nnc_batch nnc_batch;
int nnc_batch_create(nnc_batch** out, nnc_net* const* nets, int K, void* stream);
void nnc_batch_free(nnc_batch* batch);
/* K, n_out, sum_k n_in_k, sum_k n_in_k^2 (any pointer may be NULL). */
int nnc_batch_info(const nnc_batch* batch, int* K, int* n_out, int* n_sum, long long* h_sum);
/* Replace the biases of one layer of every net: bias = K x d_{layer+1} host doubles (problem
 * data such as loads entering the first layer; the nets themselves are not changed). */
int nnc_batch_set_bias(nnc_batch* batch, int layer, const double* bias);
/* Split-K count of the batch's symmetric product (1..32; the CTAs of each lower-triangle tile
 * of sum_l Zdot_l^T diag(c_l) Zdot_l share its K = sum of the hidden widths; partial sums in FP32
 * planes, added in split order).  Pins the plan (reproducible profiles, tuning); drops a
 * captured graph.  NNC_ERR_ARG outside the range; the plan is unchanged on any error. */
int nnc_batch_tune_set(nnc_batch* batch, int syrk_splits);
/* The split-K count in use (0 when no layer has curvature). */
int nnc_batch_tuning(const nnc_batch* batch, int* syrk_splits);
/* Autotuner of a batch (no effect on results): times whole evaluations on the batch's own buffers
 * (CUDA events, no graph) for every grouped-tangent N tile that covers the widest network (112,
 * 128, 208, 256) and split-K counts 1 .. 3 of the symmetric product, and keeps the fastest.
 * cache_path (may be NULL) names a text file of earlier choices (one line per batch shape and
 * device: key, N tile, splits, microseconds), reused unless retune != 0 and appended to.  Reports
 * the choice in *tangent_bn, *syrk_splits (either may be NULL); drops a captured graph.  CUDA-core
 * forms and batches without curvature return NNC_OK with the current plan. */
int nnc_batch_autotune(nnc_batch* batch, const char* cache_path, int retune, int* tangent_bn,
                       int* syrk_splits);
/* Capture one evaluation in a CUDA graph on first use and replay it while the device pointers
 * passed to nnc_batch_eval_dev stay the same (enable = 0 drops the graph). */
int nnc_batch_use_graph(nnc_batch* batch, int enable);
/* Device pointers (any output may be NULL; lambda_cat needed for H or grad). */
int nnc_batch_eval_dev(nnc_batch* batch, const double* x_cat, const double* lambda_cat,
                       double* y_cat, double* J_cat, double* H_cat, double* grad_cat,
                       void* stream);
/* FP64-accurate residual r_cat = y_cat - NN(x_cat) of every net (double-float value pass),
 * device pointers. */
int nnc_batch_residual_dev(nnc_batch* batch, const double* x_cat, const double* y_cat,
                           double* r_cat, void* stream);
/* One interior-point iterate of every net from one value pass: the FP64-accurate residual
 * r_cat = y_cat - NN(x_cat) (r_cat may be NULL, then y_cat too), J, H and the gradient as in
 * nnc_batch_eval_dev (any may be NULL; lambda_cat needed for H or grad); captured in the CUDA
 * graph like nnc_batch_eval_dev. */
int nnc_batch_eval_kkt_dev(nnc_batch* batch, const double* x_cat, const double* y_cat,
                           const double* lambda_cat, double* r_cat, double* J_cat, double* H_cat,
                           double* grad_cat, void* stream);
/* Host-pointer twins (copy, run, copy back, wait). */
int nnc_batch_eval(nnc_batch* batch, const double* x_cat, const double* lambda_cat, double* y_cat,
                   double* J_cat, double* H_cat, double* grad_cat);
int nnc_batch_residual(nnc_batch* batch, const double* x_cat, const double* y_cat, double* r_cat);
/* Host-pointer twin of nnc_batch_eval_kkt_dev: copies x_cat (and y_cat, lambda_cat) in, returns
 * r_cat = y_cat - NN(x_cat), J_cat, H_cat and grad_cat (any output may be NULL; y_cat needed for
 * r_cat, lambda_cat for H_cat or grad_cat) from one value pass, and waits.  The same results as
 * nnc_batch_residual and nnc_batch_eval, bit for bit. */
int nnc_batch_eval_kkt(nnc_batch* batch, const double* x_cat, const double* y_cat,
                       const double* lambda_cat, double* r_cat, double* J_cat, double* H_cat,
                       double* grad_cat);

/* ---- Learned warm start ---------------------------------------------------------------------
 * An MLP n_in -> h1 -> h2 -> n_out with GELU hidden layers (GELU(z) = z Phi(z)) and a linear
 * output that maps problem parameters to an interior-point starting point, trained on the GPU
 * by the library's own forward, backward and Adam kernels.  Operands are BF16 (prec = NNC_BF16)
 * or FP32 (NNC_FP32) with FP32 accumulation; master weights and Adam moments are FP32.
 *   params : 6 host arrays W1 (h1 x n_in), b1, W2 (h2 x h1), b2, W3 (n_out x h2), b3 (row-major).
 * Inputs and targets are standardized per coordinate (nnc_ws_train sets the scaling from its
 * data; nnc_ws_set_scaling sets it directly); the loss is the mean squared error on
 * standardized targets; nnc_ws_predict returns de-standardized predictions. */
typedef struct nnc_ws nnc_ws;
int nnc_ws_create(nnc_ws** out, int n_in, int h1, int h2, int n_out, const double* const* params,
                  int prec, void* stream);
void nnc_ws_free(nnc_ws* ws);
int nnc_ws_set_scaling(nnc_ws* ws, const double* in_mean, const double* in_std,
                       const double* out_mean, const double* out_std);
/* Loss and gradients (6 host arrays like params, each may be NULL) on B rows U (B x n_in),
 * T (B x n_out) with the current weights; no update. */
int nnc_ws_loss_grad(nnc_ws* ws, const double* U, const double* T, int B, double* loss,
                     double* const* grads);
/* One Adam step (Kingma & Ba) with the gradients of the last nnc_ws_loss_grad. */
int nnc_ws_adam_step(nnc_ws* ws, double lr, double beta1, double beta2, double eps);
/* Mini-batch training: `epochs` passes over N rows in seeded random order, batch rows per step. */
int nnc_ws_train(nnc_ws* ws, const double* U, const double* T, int N, int epochs, int batch,
                 double lr, double beta1, double beta2, double eps, unsigned long long seed,
                 double* final_loss);
/* P (N x n_out) for U (N x n_in). */
int nnc_ws_predict(nnc_ws* ws, const double* U, int N, double* P);
/* Current FP32 master weights, widened to FP64 (6 host arrays, each may be NULL). */
int nnc_ws_get_params(nnc_ws* ws, double* const* params);

/* Free a net and all of its device memory (waits for its stream).  NULL is ignored. */
void nnc_free(nnc_net* net);

/* Message describing the last error on the calling thread ("" if none).  Valid until the
 * next call from the same thread. */
const char* nnc_last_error(void);

/* Query helpers (no device work). */
int nnc_net_info(const nnc_net* net, int* n_layers, int* n_in, int* n_out, int* prec);
/* Layer l (0-based) of the loaded net: its FP64 weights W (rows x cols, row-major, host, may be
 * NULL), bias b (rows, host, may be NULL; zeros if none was given), activation code, and shape
 * (rows = width of layer l+1, cols = width of layer l).  Synchronises the net's stream. */
int nnc_layer_weights(const nnc_net* net, int layer, double* W, double* b, int* act, int* rows,
                      int* cols);
/* Failure-detection self-test (no net): one CTA waits `cycles` clock cycles (1 .. 4e9) on an
 * mbarrier that nothing arrives on, with the bounded wait of the streaming kernels (which = 0) or
 * of the tensor-core kernels (which = 1, abort flag included).  The wait must give up: returns
 * NNC_ERR_TIMEOUT with the recorded wait code in *code (may be NULL), and the device stays usable. */
int nnc_selftest_bounded_wait(int which, long long cycles, int* code);
/* The same wait queued on the net's stream, recording its code in the net's own error word, as a
 * timed-out wait inside an evaluation would (no fault, nothing synchronised).  The net's next host
 * call (nnc_eval, nnc_eval_kkt, nnc_residual, ...) then returns NNC_ERR_TIMEOUT and clears the
 * word, and the call after it runs normally.  which and cycles as above; NNC_ERR_ARG otherwise. */
int nnc_selftest_net_wait(nnc_net* net, int which, long long cycles);
/* Number of kernel launches this library queued since load (all nets, this process). */
long long nnc_launch_count(void);

/* Autotuner for the tensor-core forms (no effect on results): times every N-tile width of each
 * tangent-GEMM shape, on one SM per tile and on SM pairs (tcgen05 cta_group::2, 256-row tiles;
 * layers with a multiple of 256 rows, BF16 forms), and every split-K count of the symmetric
 * product with 128- and 256-column tiles on the net's own buffers (CUDA events on its stream)
 * and keeps the fastest.
 * cache_path (may be NULL) names a JSON file of earlier choices, keyed by device, kind,
 * precision and shape; existing entries are reused unless retune != 0, and the file is
 * rewritten with the current choices.  CUDA-core forms return NNC_OK at once.  nnc_tuning
 * reports the current choice for one layer (a negative tangent tile is an SM-pair tile). */
int nnc_autotune(nnc_net* net, const char* cache_path, int retune);
int nnc_tuning(const nnc_net* net, int layer, int* tangent_bn, int* syrk_splits);
/* Pin the tensor-core tiling instead of tuning it (reproducible profiles): tangent_bn = the N tile
 * of every tangent GEMM (112, 128, 208 or 256 on one SM per tile; -128, -160, -208 or -256
 * on SM pairs, applied to the layers whose row count is a multiple of 256, not in the FP8 form;
 * 0 keeps the current one), syrk_splits = the split-K count of the symmetric product (1 .. the
 * count chosen at load; 0 keeps it).  No effect on the CUDA-core forms; NNC_ERR_ARG for other
 * values. */
int nnc_tune_set(nnc_net* net, int tangent_bn, int syrk_splits);

/* Per-kernel timing with CUDA events on the net's launch streams (no effect on results).
 * nnc_profile(net, 1) starts recording a pair of events around every launch (and clears what
 * was recorded); nnc_profile_read waits for the recorded work, then fills ms[k] (total
 * milliseconds) and count[k] (launches) for kernel kind k < n_kinds and clears the record:
 *   0 tangent GEMM, 1 symmetric product (Hessian accumulation), 2 forward layer,
 *   3 reverse layer, 4 other,
 *   5 tangent chain: one pair of events around all tangent GEMMs of an evaluation, counted as
 *     that many launches (its ms / count is the average launch time with the launches overlapping
 *     as they do unprofiled; recorded only when its own bit is set),
 *   6 value pass: likewise around the layers of the double-float value pass of an evaluation
 *     (non-FP64 forms), counted as its layers.
 * enable = 0 stops recording; enable = 1 records kinds 0 to 4; enable > 1 records only the kinds
 * whose bit (k + 1) is set, so that events do not sit between launches that overlap through
 * programmatic dependent launch. */
int nnc_profile(nnc_net* net, int enable);
int nnc_profile_read(nnc_net* net, double* ms, long long* count, int n_kinds);

/* r = y - NN(x) in FP64 without allocating any device memory.  The paper has no counterpart.
 * Some callers cannot call cudaMalloc: a host framework that owns the device memory budget and
 * hands out memory only from its own pool, or a control loop that must not call cudaMalloc
 * because it can synchronise the device and take unbounded time.  Such callers cannot create a
 * net with nnc_load_weights (it allocates the packed weights), so they pass every buffer:
 *   n_layers, widths (L+1 host ints, each in [1, 65536]), act (L host nnc_act codes, elementwise
 *   activations only: NNC_SOFTMAX returns NNC_ERR_UNSUPPORTED);
 *   W : L host pointers to device arrays, W[l] = d_{l+1} x d_l row-major FP64, no padding;
 *   b : NULL, or L host pointers to device arrays of d_{l+1} doubles (entries may be NULL);
 *   x (n_in), y (n_out), r (n_out): device arrays of doubles;  stream: cudaStream_t or NULL.
 * The layer activations go to one file-scope device array of 2 x 65536 doubles (1 MiB), which
 * every GPU that loads the library keeps until the process exits; a width above 65536 returns
 * NNC_ERR_ARG.  The first call on a device (and the first call after that device's context was
 * destroyed and created again) looks up the array's address with the device current, so make
 * that first call before any stream capture.  All calls share the array and it keeps the last
 * call's contents (every entry a call reads it has written first): calls whose work overlaps on
 * the GPU race and must be ordered by the caller.  The call is asynchronous on `stream`. */
int nnc_residual_noalloc(int n_layers, const int* widths, const int* act, const double* const* W,
                         const double* const* b, const double* x, const double* y, double* r,
                         void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NNC_H */
