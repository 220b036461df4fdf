// C ABI of libnnc (declared in include/nnc.h) and the host runtime behind it: the net object,
// weight packing, device workspaces and the order in which one oracle call runs its kernels.
//
// One interior-point iteration (Eq. 2) needs, at the same x:
//   forward value pass  z_l = W_l a_{l-1} + b_l, a_l = sigma_l(z_l)            (Eq. 3)
//   reverse sweep       abar_L = seeds, abar_{l-1} = W_l^T (sigma_l' * abar_l)  (Jacobian, adjoint)
//   tangent sweep       Zdot_1 = W_1, Zdot_l = W_l (sigma_{l-1}' * Zdot_{l-1})  (n_in tangents)
//   Hessian of lambda^T NN (Eq. 6) as  H = sum_l Zdot_l^T diag(sigma_l'' * abar_l) Zdot_l,
// which is what forward-over-reverse differentiation of lambda^T NN reduces to once the
// reverse tangents of the affine maps are unrolled.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "net.cuh"

namespace nnc {
static std::atomic<long long> g_launches{0};
void note_launch(int n) { g_launches += n; }
static thread_local std::string g_err;
static int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
void set_last_error(const std::string& msg) { g_err = msg; }
void* pinned_dev_ptr(void* host) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}
}  // namespace nnc

using namespace nnc;

namespace {

bool is_tc(int prec) { return prec == NNC_BF16 || prec == NNC_BF16X3 || prec == NNC_FP8; }

Elem tan_elem(int prec) {
  switch (prec) {
    case NNC_FP64: return Elem::F64;
    case NNC_FP32: return Elem::F32;
    case NNC_BF16: return Elem::BF16;
    case NNC_FP8: return Elem::BF16;
    default: return Elem::BF16X3;
  }
}

size_t elem_size(int prec) { return prec == NNC_FP64 ? 8 : prec == NNC_FP32 ? 4 : 2; }

#define CK(expr)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(e_ == cudaErrorMemoryAllocation ? NNC_ERR_OOM : NNC_ERR_CUDA,         \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));                  \
  } while (0)

template <typename T>
int dalloc(nnc_net* net, T** p, size_t n) {
  void* q = nullptr;
  const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess)
    return fail(NNC_ERR_OOM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " +
                                 cudaGetErrorString(e));
  e = cudaMemsetAsync(q, 0, bytes, net->stream);
  if (e != cudaSuccess) return fail(NNC_ERR_CUDA, cudaGetErrorString(e));
  net->allocs.push_back(q);
  net->bytes += bytes;
  *p = (T*)q;
  return NNC_OK;
}

#define AL(p, n)                                    \
  do {                                              \
    int r_ = dalloc(net, &(p), (n));                \
    if (r_ != NNC_OK) return r_;                    \
  } while (0)

int check_finite(const double* v, int n, const char* what) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return fail(NNC_ERR_NONFINITE, std::string(what) + " holds NaN or Inf");
  return NNC_OK;
}

// The error word e of the bounded waits, already read back: clear it and report a timeout.
int dev_err_status(nnc_net* net, int e) {
  if (e != 0) {
    int z = 0;
    cudaMemcpy(net->dev_err, &z, sizeof(int), cudaMemcpyHostToDevice);
    return fail(NNC_ERR_TIMEOUT, "a bounded device-side wait ran out (code " + std::to_string(e) + ")");
  }
  return NNC_OK;
}

// Host calls: queue the error word's copy behind the outputs into its pinned slot (the last
// element of h_stage), wait for the device once, then check it.
int sync_check(nnc_net* net, cudaStream_t st) {
  int* herr = reinterpret_cast<int*>(net->h_stage + net->h_stage_elems - 1);
  CK(cudaMemcpyAsync(herr, net->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return dev_err_status(net, *herr);
}

cudaStream_t pick(nnc_net* net, void* st) { return st ? (cudaStream_t)st : net->stream; }

// Kernel kinds of nnc_profile_read.
// PK_TAN_SPAN: one pair of events around the whole chain of tangent GEMMs of an evaluation (from
// before the first to after the last), counted as that many launches; PK_FWD_SPAN likewise around
// the layers of the value pass.  Both are recorded only when asked for by their own bits, so that
// no event sits between launches that overlap through programmatic dependent launch.
enum { PK_TANGENT = 0, PK_SYRK = 1, PK_FWD = 2, PK_REV = 3, PK_OTHER = 4, PK_TAN_SPAN = 5,
       PK_FWD_SPAN = 6, PK_N = 7 };

// Brackets one launch with a pair of events on its stream when profiling is on.
struct ProfScope {
  nnc_net* net;
  cudaStream_t st;
  bool on;
  size_t idx = 0;
  ProfScope(nnc_net* n, int kind, cudaStream_t s)
      : net(n), st(s), on(((n->prof_mask >> kind) & 1u) != 0) {
    if (!on) return;
    while (net->ev_used + 2 > net->ev_pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) {
        on = false;
        return;
      }
      net->ev_pool.push_back(e);
    }
    idx = net->ev_used;
    net->ev_used += 2;
    net->ev_kind.push_back(kind);
    net->ev_weight.push_back(1);
    cudaEventRecord(net->ev_pool[idx], st);
  }
  ~ProfScope() {
    if (on) cudaEventRecord(net->ev_pool[idx + 1], st);
  }
};
#define PROF(kind) ProfScope prof_scope_(net, kind, st)

// ---------------------------------------------------------------- forward value pass
// FP64 form: FP64 GEMV layers.  Other forms: one double-float streaming pass (about 48
// significant bits) whose sigma, sigma' and sigma'' feed the derivative sweeps; expects net->x and
// its pairs net->x2 (launch_copy_pad).
// Non-FP64 forms may run the layers [l0, l1) only (the output layer then goes to another stream).
int run_forward(nnc_net* net, bool fp64, cudaStream_t st, int l0 = 0, int l1 = -1) {
  if (l1 < 0) l1 = net->L;
  if (fp64) {
    const double* a_in = net->x;
    for (auto& Ly : net->layers) {
      PROF(PK_FWD);
      CK(launch_gemv_fwd(true, Ly.W64, Ly.kp, Ly.b, a_in, Ly.m, Ly.kp, Ly.act, Ly.a, nullptr, Ly.s1,
                         Ly.s2, st));
      a_in = Ly.a;
    }
    if (net->softmax) CK(launch_softmax_head(net->n_out, net->layers.back().a, st));
    return NNC_OK;
  }
  const void* a_in2 = l0 == 0 ? net->x2 : net->layers[l0 - 1].a2;
  {
    ProfScope span(net, PK_FWD_SPAN, st);   // the value pass's layers, counted as such
    if (span.on) net->ev_weight.back() = l1 - l0;
    for (int l = l0; l < l1; ++l) {
      LayerDev& Ly = net->layers[l];
      PROF(PK_FWD);
      CK(launch_gemv_stream_df(Ly.W2, Ly.kp, Ly.m, Ly.b, a_in2, Ly.act, Ly.a, Ly.a2, Ly.s1, Ly.s2,
                               net->dev_err, net->sm_count, st));
      a_in2 = Ly.a2;
    }
  }
  if (net->softmax && l1 == net->L) CK(launch_softmax_head(net->n_out, net->layers.back().a, st));
  return NNC_OK;
}

// FP64 value pass of the residual y - NN(x) from the raw device input x.  The FP64 form runs it
// in FP64; the other forms in double-float arithmetic (about 48 significant bits, HBM-bound).
int run_forward_fp64_values(nnc_net* net, const double* x, cudaStream_t st) {
  CK(launch_copy_pad(x, net->xr, net->prec == NNC_FP64 ? nullptr : net->xr2, net->n_in,
                     net->n_in_pad, st));
  if (net->prec == NNC_FP64) {
    const double* a_in = net->xr;
    for (auto& Ly : net->layers) {
      PROF(PK_FWD);
      CK(launch_gemv_fwd(true, Ly.W64, Ly.kp, Ly.b, a_in, Ly.m, Ly.kp, Ly.act, Ly.ra, nullptr,
                         nullptr, nullptr, st));
      a_in = Ly.ra;
    }
  } else {
    const void* a_in2 = net->xr2;
    for (auto& Ly : net->layers) {
      PROF(PK_FWD);
      CK(launch_gemv_stream_df(Ly.W2, Ly.kp, Ly.m, Ly.b, a_in2, Ly.act, Ly.ra, Ly.ra2, nullptr,
                               nullptr, net->dev_err, net->sm_count, st));
      a_in2 = Ly.ra2;
    }
  }
  if (net->softmax) CK(launch_softmax_head(net->n_out, net->layers.back().ra, st));
  return NNC_OK;
}

// ---------------------------------------------------------------- reverse sweep
// nJ Jacobian seeds (0 or n_out) and, if with_lam, one more seed column carrying lambda whose
// adjoints give c_l = sigma_l'' * abar_l for the Hessian and the gradient lambda^T J.
int run_reverse(nnc_net* net, bool fp64, int nJ, bool with_lam, const double* lam, double* J,
                double* g, cudaStream_t st) {
  const int S = nJ + (with_lam ? 1 : 0);
  if (S == 0) return NNC_OK;
  const int lam_col = with_lam ? nJ : -1;
  const bool tc = is_tc(net->prec);
  LayerDev& Lo = net->layers.back();
  const double* soft_p = net->softmax ? Lo.a : nullptr;   // softmax probabilities (value pass)
  if (net->tc_rev) {
    // seeds^T in three BF16 parts, then per layer: split-K tensor-core product W_l^T Zbar and a reduce
    // that forms the next seeds (or J and the gradient on the first layer)
    CK(launch_rev_seed_t(Lo.m, S, nJ, lam_col, Lo.s1, Lo.s2, lam, soft_p, net->Zb[0], Lo.mp,
                         with_lam ? Lo.c : nullptr, with_lam ? Lo.c_f : nullptr, st));
    for (int l = net->L - 1; l >= 0; --l) {
      LayerDev& Ly = net->layers[l];
      const int zn = (net->L - l) % 2;  // seeds of layer l-1
      PROF(PK_REV);
      CK(tc_rev(Ly.plan_rev, net->Prev, net->dev_err, st));
      if (l > 0) {
        LayerDev& Lp = net->layers[l - 1];
        CK(launch_rev_reduce_t(net->Prev, Ly.plan_rev.splits, Ly.kp, Ly.plan_rev.bn, S, Ly.k, Lp.s1,
                               Lp.s2, lam_col, nJ, net->Zb[zn], Ly.kp,
                               with_lam ? Lp.c : nullptr, with_lam ? Lp.c_f : nullptr, nullptr,
                               nullptr, st));
      } else {
        CK(launch_rev_reduce_t(net->Prev, Ly.plan_rev.splits, Ly.kp, Ly.plan_rev.bn, S, Ly.k, nullptr,
                               nullptr, lam_col, nJ, nullptr, 0, nullptr, nullptr, J, g, st));
      }
    }
    return NNC_OK;
  }
  if (net->rev_stream) {
    // FP32 weights streamed by TMA, one launch per layer (the layer boundary is fused in)
    CK(launch_rev_seed_f(Lo.m, S, nJ, lam_col, Lo.s1, Lo.s2, lam, soft_p, net->Zf[0],
                         with_lam ? Lo.c : nullptr, (with_lam && tc) ? Lo.c_f : nullptr, st));
    int cur = 0;
    for (int l = net->L - 1; l >= 0; --l) {
      LayerDev& Ly = net->layers[l];
      PROF(PK_REV);
      if (l > 0) {
        LayerDev& Lp = net->layers[l - 1];
        CK(launch_rev_stream(Ly.rev_map, Ly.m, Ly.kp, net->Zf[cur], S, Ly.rev_geom,
                             (float*)net->part, net->rev_cnt + Ly.rev_cnt_off, nJ, lam_col, Ly.k,
                             Lp.s1, Lp.s2, net->Zf[1 - cur], with_lam ? Lp.c : nullptr,
                             (with_lam && tc) ? Lp.c_f : nullptr, nullptr, nullptr, net->dev_err,
                             st));
      } else {
        CK(launch_rev_stream(Ly.rev_map, Ly.m, Ly.kp, net->Zf[cur], S, Ly.rev_geom,
                             (float*)net->part, net->rev_cnt + Ly.rev_cnt_off, nJ, lam_col, Ly.k,
                             nullptr, nullptr, nullptr, nullptr, nullptr, J, g, net->dev_err, st));
      }
      cur = 1 - cur;
    }
    return NNC_OK;
  }
  CK(launch_rev_seed(Lo.m, S, nJ, lam_col, Lo.s1, Lo.s2, lam, soft_p, net->Zbar[0],
                     with_lam ? Lo.c : nullptr, (with_lam && tc) ? Lo.c_f : nullptr, st));
  int cur = 0;
  for (int l = net->L - 1; l >= 0; --l) {
    LayerDev& Ly = net->layers[l];
    const int chunks = rev_chunks(Ly.m, Ly.kp, net->sm_count);
    PROF(PK_REV);
    CK(launch_gemv_rev(fp64, fp64 ? (const void*)Ly.W64 : (const void*)Ly.W32, Ly.kp, Ly.m, Ly.kp,
                       net->Zbar[cur], S, chunks, net->part, st));
    if (l > 0) {
      LayerDev& Lp = net->layers[l - 1];
      CK(launch_rev_reduce(fp64, net->part, chunks, Ly.kp, Ly.k, S, Lp.s1, Lp.s2, lam_col, nJ,
                           net->Zbar[1 - cur], with_lam ? Lp.c : nullptr,
                           (with_lam && tc) ? Lp.c_f : nullptr, nullptr, nullptr, st));
      cur = 1 - cur;
    } else {
      CK(launch_rev_reduce(fp64, net->part, chunks, Ly.kp, Ly.k, S, nullptr, nullptr, lam_col, nJ,
                           nullptr, nullptr, nullptr, J, g, st));
    }
  }
  return NNC_OK;
}

// ---------------------------------------------------------------- tangent sweep + H
// Forward tangents layer by layer (Zdot_1 = W_1 elementwise; Zdot_l = W_l Adot_{l-1} as a GEMM
// with the n_in tangents as columns), each layer's Zdot_l and c_l * Zdot_l stored side by side
// along K; then one symmetric product H = sum_l Zdot_l^T diag(c_l) Zdot_l.
// deferred: the tangent chain writes Zdot_l only (it does not need c_l, so the reverse sweep that
// produces c_l runs on the side stream meanwhile); after ev_join, one pass forms c_l * Zdot_l.
int run_hessian(nnc_net* net, const double* lam, double* H, cudaStream_t st, bool deferred) {
  const int n = net->n_in;
  const int prec = net->prec;
  const bool tc = is_tc(prec);
  const Elem e = tan_elem(prec);
  const size_t es = elem_size(prec);
  auto zoff = [&](void* base, int off) -> void* {
    return (base && off >= 0) ? (void*)((char*)base + (size_t)off * es) : nullptr;
  };
  LayerDev& L1 = net->layers[0];
  if (tc && net->use_chain && net->chain_nl > 0)
    CK(cudaMemsetAsync(net->chain_cnt, 0,
                       sizeof(unsigned) * (size_t)net->chain_nl * net->chain_plans[0].ntn, st));
  {
    PROF(PK_OTHER);
    TanBuf At0{net->At[0][0], net->At[0][1]};
    TanBuf Zt{zoff(net->Zt[0], L1.zy_off), zoff(net->Zt[1], L1.zy_off)};
    TanBuf Yt{deferred ? nullptr : zoff(net->Yt[0], L1.zy_off),
              deferred ? nullptr : zoff(net->Yt[1], L1.zy_off)};
    if (net->W1T)   // Zdot_1 was written at load
      CK(launch_first_tangent_t(e == Elem::BF16X3, net->W1T, L1.mp, L1.mp, n, L1.s1, L1.c,
                                net->L > 1 ? At0 : TanBuf{}, L1.mp, Yt, net->K_total, st));
    else
      CK(launch_first_tangent(e, prec == NNC_FP64 ? (const void*)L1.W64 : (const void*)L1.W32,
                              L1.kp, L1.mp, n, L1.s1, L1.c, net->L > 1 ? At0 : TanBuf{}, L1.mp, Zt,
                              Yt, net->K_total, st));
  }
  if (tc && net->use_chain && net->chain_nl > 0) {
    // every tangent GEMM in one persistent launch; its counters are cleared before the first
    // layer's kernel so that the chain still follows it by programmatic dependent launch
    std::vector<ChainOut> outs(net->chain_nl);
    for (int i = 0; i < net->chain_nl; ++i) {
      LayerDev& Ly = net->layers[i + 1];
      const bool last = i + 1 == net->L - 1;
      const int cur = i % 2;
      outs[i] = ChainOut{Ly.s1, Ly.c_f, last ? nullptr : net->At[1 - cur][0],
                         last ? nullptr : net->At[1 - cur][1], Ly.mp,
                         zoff(net->Zt[0], Ly.zy_off), zoff(net->Zt[1], Ly.zy_off),
                         deferred ? nullptr : zoff(net->Yt[0], Ly.zy_off),
                         deferred ? nullptr : zoff(net->Yt[1], Ly.zy_off)};
    }
    {
      ProfScope span(net, PK_TAN_SPAN, st);
      if (span.on) net->ev_weight.back() = net->chain_nl;
      PROF(PK_TANGENT);
      CK(tc_tangent_chain(net->chain_plans.data(), outs.data(), net->chain_nl, net->chain_cnt,
                          net->K_total, net->dev_err, st));
    }
  } else {
  int cur = 0;
  // span of the whole tangent chain (PK_TAN_SPAN), counted as its number of tangent GEMMs
  ProfScope span(net, PK_TAN_SPAN, st);
  int span_launches = 0;
  for (int l = 1; l < net->L; ++l) {
    LayerDev& Ly = net->layers[l];
    const bool last = (l == net->L - 1);
    if (last && Ly.zy_off < 0) break;  // a linear output layer adds nothing to H
    ++span_launches;
    void* Anext_hi = last ? nullptr : net->At[1 - cur][0];
    void* Anext_lo = last ? nullptr : net->At[1 - cur][1];
    if (prec == NNC_FP8) {
      PROF(PK_OTHER);
      CK(launch_quant_fp8(net->At[cur][0], n, Ly.kp, net->A8, net->tsc, st));
    }
    PROF(PK_TANGENT);
    if (tc) {
      CK(tc_tangent(Ly.plan_tan, Ly.s1, Ly.c_f, Anext_hi, Anext_lo, Ly.mp,
                    zoff(net->Zt[0], Ly.zy_off), zoff(net->Zt[1], Ly.zy_off),
                    deferred ? nullptr : zoff(net->Yt[0], Ly.zy_off),
                    deferred ? nullptr : zoff(net->Yt[1], Ly.zy_off), net->K_total,
                    net->dev_err, st, Ly.w8s, net->tsc));
    } else {
      CK(launch_simt_tangent(prec == NNC_FP64,
                             prec == NNC_FP64 ? (const void*)Ly.W64 : (const void*)Ly.W32, Ly.kp,
                             net->At[cur][0], Ly.kp, Ly.mp, n, Ly.kp, Ly.s1, Ly.c, Anext_hi, Ly.mp,
                             zoff(net->Zt[0], Ly.zy_off), zoff(net->Yt[0], Ly.zy_off),
                             net->K_total, st));
    }
    cur = 1 - cur;
  }
  if (span.on) {
    if (span_launches) {
      cudaEventRecord(net->ev_pool[span.idx + 1], st);
      net->ev_weight[net->ev_weight.size() - 1] = span_launches;
    } else {     // no tangent GEMM: drop the pair
      net->ev_used -= 2;
      net->ev_kind.pop_back();
      net->ev_weight.pop_back();
    }
    span.on = false;
  }
  }
  if (net->softmax) {
    // the rank-two part of the softmax layer's curvature as two extra operand columns
    LayerDev& Lo = net->layers.back();
    PROF(PK_OTHER);
    CK(launch_softmax_ext(e, n, net->n_out, Lo.a, lam,
                          TanBuf{zoff(net->Zt[0], Lo.zy_off), zoff(net->Zt[1], Lo.zy_off)},
                          TanBuf{zoff(net->Zt[0], net->ext_off), zoff(net->Zt[1], net->ext_off)},
                          TanBuf{zoff(net->Yt[0], net->ext_off), zoff(net->Yt[1], net->ext_off)},
                          net->K_total, st));
  }
  if (net->K_total == 0) {  // every layer is linear: H = 0
    CK(cudaMemsetAsync(H, 0, sizeof(double) * n * n, st));
    return NNC_OK;
  }
  if (deferred) {
    CK(cudaStreamWaitEvent(st, net->ev_join, 0));   // c_l of every layer is written
    PROF(PK_OTHER);
    CK(launch_scale_y(prec == NNC_BF16X3, net->Zt[0], net->Zt[1], net->Yt[0], net->Yt[1], net->cK,
                      n, net->K_total, 0, net->softmax ? net->ext_off : net->K_total, st));
  }
  {
    PROF(PK_SYRK);
    if (!tc)  // the tensor-core product stores its partials; the CUDA-core one adds to them
      CK(cudaMemsetAsync(net->Hp, 0, (size_t)net->h_splits * n * n * 8, st));
    if (tc)
      CK(tc_syrk(net->plan_syrk, (float*)net->Hp, net->dev_err, st));
    else
      CK(launch_simt_syrk(prec == NNC_FP64, net->Zt[0], net->Yt[0], net->K_total, n, net->K_total,
                          net->h_splits, (double*)net->Hp, st));
  }
  {
    PROF(PK_OTHER);
    // the tensor-core product writes exactly plan_syrk.splits planes (tuning may lower the count)
    const int planes = tc ? net->plan_syrk.splits : net->h_splits;
    CK(launch_h_finish(net->hp_f32, net->Hp, planes, n, n, H, st));
  }
  return NNC_OK;
}

// One value pass at x, then whatever is asked: y = NN(x), the residual rr = yv - NN(x), J, H and
// the gradient lambda^T J.
int eval_all(nnc_net* net, const double* x, const double* lam, double* y, double* J, double* H,
             double* g, cudaStream_t st, const double* yv = nullptr, double* rr = nullptr) {
  CK(launch_copy_pad(x, net->x, net->x2, net->n_in, net->n_in_pad, st));
  const bool fp64 = net->prec == NNC_FP64;
  // tensor-core forms: the reverse sweep (streaming, or on the tensor cores for more than 15
  // outputs) on the side stream, next to the tangent chain
  const bool fork = H && is_tc(net->prec) && (net->rev_stream || net->tc_rev) && net->side_stream;
  // With a linear output layer the tangent chain reads nothing of it, so that layer, y and the
  // residual go to the side stream ahead of the reverse sweep and the chain starts after layer
  // L - 1.  (Not while the value pass is timed as one span, nor with the persistent chain.)
  const bool tail = fork && !fp64 && net->L > 1 && net->layers.back().act == NNC_IDENTITY &&
                    !net->use_chain && !(net->prof_mask & (1u << PK_FWD_SPAN));
  int r = run_forward(net, fp64, st, 0, tail ? net->L - 1 : net->L);
  if (r != NNC_OK) return r;
  cudaStream_t vs = st;   // the stream of the output layer and of what reads its values
  if (fork) {
    CK(cudaEventRecord(net->ev_fork, st));
    CK(cudaStreamWaitEvent(net->side_stream, net->ev_fork, 0));
    if (tail) {
      vs = net->side_stream;
      r = run_forward(net, fp64, vs, net->L - 1, net->L);
      if (r != NNC_OK) return r;
    }
  }
  if (y)   // y may be the device address of page-locked host memory
    CK(cudaMemcpyAsync(y, net->layers.back().a, sizeof(double) * net->n_out, cudaMemcpyDefault,
                       vs));
  if (rr) CK(launch_sub(yv, net->layers.back().a, rr, net->n_out, vs));
  const bool need_lam = (H != nullptr) || (g != nullptr);
  if (fork) {
    r = run_reverse(net, fp64, J ? net->n_out : 0, true, lam, J, g, net->side_stream);
    if (r != NNC_OK) return r;
    CK(cudaEventRecord(net->ev_join, net->side_stream));
    r = run_hessian(net, lam, H, st, true);
    CK(cudaStreamWaitEvent(st, net->ev_join, 0));   // J and the gradient too, on every path
    return r;
  }
  if (J || need_lam) {
    r = run_reverse(net, fp64, J ? net->n_out : 0, need_lam, lam, J, g, st);
    if (r != NNC_OK) return r;
  }
  if (H) {
    r = run_hessian(net, lam, H, st, false);
    if (r != NNC_OK) return r;
  }
  return NNC_OK;
}

int check_net(const nnc_net* net) {
  if (!net) return fail(NNC_ERR_ARG, "net is NULL");
  return NNC_OK;
}

// Host-pointer wrapper: copy inputs in, run, copy outputs out, wait.  An output in page-locked
// memory is written there by the kernel that forms it (no device buffer, no transfer after it).
int host_call(nnc_net* net, const double* x, const double* lam, double* y, double* J, double* H,
              double* g, const double* yv = nullptr, double* rr = nullptr) {
  int r = check_net(net);
  if (r) return r;
  if (!x) return fail(NNC_ERR_ARG, "x is NULL");
  if ((H || g) && !lam) return fail(NNC_ERR_ARG, "lambda is NULL");
  r = check_finite(x, net->n_in, "x");
  if (r) return r;
  if (lam) {
    r = check_finite(lam, net->n_out, "lambda");
    if (r) return r;
  }
  CK(cudaSetDevice(net->device));
  cudaStream_t st = net->stream;
  double* hs = net->h_stage;
  std::memcpy(hs, x, sizeof(double) * net->n_in);
  double* hl = hs + net->n_in_pad;
  double* hy = hl + net->n_out;
  if (lam) std::memcpy(hl, lam, sizeof(double) * net->n_out);
  if (rr) std::memcpy(hy, yv, sizeof(double) * net->n_out);
  // one copy of the staging block up to the last input used (the device block has its layout)
  const size_t n_copy = rr ? (size_t)(hy - hs) + net->n_out
                        : lam ? (size_t)(hl - hs) + net->n_out : (size_t)net->n_in;
  CK(cudaMemcpyAsync(net->xin, hs, sizeof(double) * n_copy, cudaMemcpyHostToDevice, st));
  // each output: written in place if pinned, else through its device buffer and a copy
  auto direct = [](double* h) { return h ? (double*)pinned_dev_ptr(h) : nullptr; };
  double *y_d = direct(y), *J_d = direct(J), *H_d = direct(H), *g_d = direct(g), *r_d = direct(rr);
  r = eval_all(net, net->xin, lam ? net->lam : nullptr, y_d ? y_d : y ? net->ydev : nullptr,
               J_d ? J_d : J ? net->Jdev : nullptr, H_d ? H_d : H ? net->Hdev : nullptr,
               g_d ? g_d : g ? net->gdev : nullptr, st, rr ? net->yres : nullptr,
               r_d ? r_d : rr ? net->rdev : nullptr);
  if (r) return r;
  auto back = [&](double* h, double* d_direct, const double* dev, size_t n) -> cudaError_t {
    if (!h || d_direct) return cudaSuccess;
    return cudaMemcpyAsync(h, dev, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
  };
  CK(back(rr, r_d, net->rdev, net->n_out));
  CK(back(y, y_d, net->ydev, net->n_out));
  CK(back(J, J_d, net->Jdev, (size_t)net->n_out * net->n_in));
  CK(back(H, H_d, net->Hdev, (size_t)net->n_in * net->n_in));
  CK(back(g, g_d, net->gdev, net->n_in));
  return sync_check(net, st);   // the error word of the bounded waits comes back with the outputs
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

const char* nnc_last_error(void) { return g_err.c_str(); }

long long nnc_launch_count(void) { return g_launches.load(); }

int nnc_profile(nnc_net* net, int enable) {
  int r = check_net(net);
  if (r) return r;
  // 1: every kind; other nonzero values: a mask of kinds, bit (k + 1) for kind k
  net->prof_mask = enable == 0                ? 0u
                   : enable == 1              ? ~((1u << PK_TAN_SPAN) | (1u << PK_FWD_SPAN))
                                              : (unsigned)enable >> 1;
  net->ev_used = 0;
  net->ev_kind.clear();
  net->ev_weight.clear();
  return NNC_OK;
}

int nnc_profile_read(nnc_net* net, double* ms, long long* count, int n_kinds) {
  int r = check_net(net);
  if (r) return r;
  if (!ms || !count || n_kinds < 1) return fail(NNC_ERR_ARG, "bad profile buffers");
  for (int i = 0; i < n_kinds; ++i) {
    ms[i] = 0.0;
    count[i] = 0;
  }
  for (size_t i = 0; i < net->ev_kind.size(); ++i) {
    CK(cudaEventSynchronize(net->ev_pool[2 * i + 1]));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, net->ev_pool[2 * i], net->ev_pool[2 * i + 1]));
    const int k = net->ev_kind[i];
    if (k < n_kinds) {
      ms[k] += t;
      count[k] += net->ev_weight[i];
    }
  }
  net->ev_used = 0;
  net->ev_kind.clear();
  net->ev_weight.clear();
  return NNC_OK;
}

int nnc_net_info(const nnc_net* net, int* n_layers, int* n_in, int* n_out, int* prec) {
  if (!net) return fail(NNC_ERR_ARG, "net is NULL");
  if (n_layers) *n_layers = net->L;
  if (n_in) *n_in = net->n_in;
  if (n_out) *n_out = net->n_out;
  if (prec) *prec = net->prec;
  return NNC_OK;
}

int nnc_selftest_bounded_wait(int which, long long cycles, int* code) {
  if (code) *code = 0;
  if (which < 0 || which > 1 || cycles < 1 || cycles > 4000000000LL)
    return fail(NNC_ERR_ARG, "which must be 0 or 1, cycles in [1, 4e9]");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(NNC_ERR_CUDA, "no CUDA device");
  int* err = nullptr;
  CK(cudaMalloc(&err, sizeof(int)));
  cudaMemset(err, 0, sizeof(int));
  cudaError_t e = which == 0 ? launch_wait_selftest_stream(err, cycles, 91, nullptr)
                             : launch_wait_selftest_tc(err, cycles, 93, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(err);
  if (e != cudaSuccess) return fail(NNC_ERR_CUDA, cudaGetErrorString(e));
  if (code) *code = h;
  if (h) return fail(NNC_ERR_TIMEOUT, "a bounded device-side wait ran out (code " + std::to_string(h) + ")");
  return NNC_OK;
}

int nnc_selftest_net_wait(nnc_net* net, int which, long long cycles) {
  int r = check_net(net);
  if (r) return r;
  if (which < 0 || which > 1 || cycles < 1 || cycles > 4000000000LL)
    return fail(NNC_ERR_ARG, "which must be 0 or 1, cycles in [1, 4e9]");
  CK(cudaSetDevice(net->device));
  CK(which == 0 ? launch_wait_selftest_stream(net->dev_err, cycles, 91, net->stream)
                : launch_wait_selftest_tc(net->dev_err, cycles, 93, net->stream));
  return NNC_OK;
}

int nnc_layer_weights(const nnc_net* net, int layer, double* W, double* b, int* act, int* rows,
                      int* cols) {
  if (!net) return fail(NNC_ERR_ARG, "net is NULL");
  if (layer < 0 || layer >= net->L) return fail(NNC_ERR_ARG, "layer out of range");
  const LayerDev& Ly = net->layers[layer];
  if (act) *act = Ly.act;
  if (rows) *rows = Ly.m;
  if (cols) *cols = Ly.k;
  CK(cudaSetDevice(net->device));
  CK(cudaStreamSynchronize(net->stream));
  if (W)   // the padded rows of the FP64 master, unpadded on the host
    CK(cudaMemcpy2D(W, sizeof(double) * Ly.k, Ly.W64, sizeof(double) * Ly.kp, sizeof(double) * Ly.k,
                    Ly.m, cudaMemcpyDeviceToHost));
  if (b) {
    if (Ly.b) CK(cudaMemcpy(b, Ly.b, sizeof(double) * Ly.m, cudaMemcpyDeviceToHost));
    else std::memset(b, 0, sizeof(double) * Ly.m);
  }
  return NNC_OK;
}

void nnc_free(nnc_net* net) {
  if (!net) return;
  batch_cache_forget(net);
  cudaSetDevice(net->device);
  if (net->stream) cudaStreamSynchronize(net->stream);
  for (void* p : net->allocs) cudaFree(p);
  for (cudaEvent_t e : net->ev_pool) cudaEventDestroy(e);
  if (net->h_stage) cudaFreeHost(net->h_stage);
  if (net->side_stream) {
    cudaStreamSynchronize(net->side_stream);
    cudaStreamDestroy(net->side_stream);
  }
  if (net->ev_fork) cudaEventDestroy(net->ev_fork);
  if (net->ev_join) cudaEventDestroy(net->ev_join);
  if (net->own_stream && net->stream) cudaStreamDestroy(net->stream);
  delete net;
}

static int load_impl(nnc_net* net, int n_layers, const int* widths, const int* act,
                     const double* const* W, const double* const* b) {
  cudaDeviceProp prop;
  CK(cudaGetDevice(&net->device));
  CK(cudaGetDeviceProperties(&prop, net->device));
  if (prop.major != 10 || prop.minor != 3)
    return fail(NNC_ERR_CUDA, std::string("libnnc is built for sm_103a; device is ") + prop.name +
                                  " sm_" + std::to_string(prop.major * 10 + prop.minor));
  net->sm_count = prop.multiProcessorCount;
  net->L = n_layers;
  net->n_in = widths[0];
  net->n_out = widths[n_layers];
  net->n_in_pad = pad_up(net->n_in);
  net->S_max = net->n_out + 1;
  if (net->S_max > 48) return fail(NNC_ERR_UNSUPPORTED, "n_out > 47 is not supported");
  const int prec = net->prec;
  const bool tc = is_tc(prec);
  net->layers.resize(n_layers);
  int mp_max = net->n_in_pad;
  size_t part_max = 1;
  int rev_cnt_total = 0;
  for (int l = 0; l < n_layers; ++l) {
    LayerDev& Ly = net->layers[l];
    Ly.m = widths[l + 1];
    Ly.k = widths[l];
    Ly.act = act[l];
    Ly.mp = pad_up(Ly.m);
    Ly.kp = pad_up(Ly.k);
    mp_max = std::max(mp_max, Ly.mp);
    const size_t nw = (size_t)Ly.mp * Ly.kp;
    AL(Ly.W64, nw);
    CK(cudaMemcpy2DAsync(Ly.W64, sizeof(double) * Ly.kp, W[l], sizeof(double) * Ly.k,
                         sizeof(double) * Ly.k, Ly.m, cudaMemcpyHostToDevice, net->stream));
    if (prec != NNC_FP64) AL(Ly.W32, nw);
    if (tc && l > 0 && prec != NNC_FP8) {
      AL(Ly.Whi, nw);
      if (prec == NNC_BF16X3) AL(Ly.Wlo, nw);
    }
    CK(launch_pack(Ly.W64, nw, Ly.W32, Ly.Whi, Ly.Wlo, net->stream));
    // W^T in three BF16 parts for the tensor-core reverse sweep (nets with more than 15
    // outputs; the others stream the FP32 weights)
    if (tc && net->S_max > 16 && net->S_max <= 48) {
      AL(Ly.WThi, nw);
      AL(Ly.WTlo, nw);
      AL(Ly.WTp2, nw);
      CK(launch_pack_t(Ly.W64, Ly.mp, Ly.kp, Ly.WThi, Ly.WTlo, Ly.WTp2, net->stream));
    }
    if (prec == NNC_FP8 && l > 0) {
      AL(Ly.W8, nw);
      AL(Ly.w8s, Ly.mp);
      CK(launch_pack_fp8(Ly.W64, Ly.mp, Ly.kp, Ly.kp, Ly.W8, Ly.w8s, net->stream));
    }
    AL(Ly.b, Ly.mp);
    if (b && b[l])
      CK(cudaMemcpyAsync(Ly.b, b[l], sizeof(double) * Ly.m, cudaMemcpyHostToDevice, net->stream));
    AL(Ly.a, Ly.mp);
    AL(Ly.s1, Ly.mp);
    AL(Ly.s2, Ly.mp);
    AL(Ly.c, Ly.mp);
    AL(Ly.ra, Ly.mp);
    if (prec != NNC_FP64) {
      float2* a2;
      AL(a2, Ly.mp);
      Ly.a2 = a2;
      float2* w2;
      AL(w2, nw);
      Ly.W2 = w2;
      CK(launch_split_df(Ly.W64, nw, Ly.W2, net->stream));
      float2* r2;
      AL(r2, Ly.mp);
      Ly.ra2 = r2;
    }
    if (tc && Ly.act == NNC_IDENTITY) AL(Ly.c_f, Ly.mp);   // curvature layers: views of cK
    const int chunks = rev_chunks(Ly.m, Ly.kp, net->sm_count);
    part_max = std::max(part_max, (size_t)chunks * Ly.kp * net->S_max);
    if (prec != NNC_FP64 && net->S_max <= 16) {
      if (!rev_stream_map(&Ly.rev_map, Ly.W32, Ly.mp, Ly.kp))
        return fail(NNC_ERR_CUDA, "tensor map of the reverse sweep failed");
      Ly.rev_geom = rev_stream_geom(Ly.m, Ly.kp, net->S_max, net->sm_count);
      part_max = std::max(part_max, (size_t)(Ly.rev_geom.splits / Ly.rev_geom.cl) * Ly.kp * 16);
      Ly.rev_cnt_off = rev_cnt_total;
      rev_cnt_total += Ly.kp / kPad;
      net->rev_stream = true;
    }
  }
  net->mp_max = mp_max;
  AL(net->x, net->n_in_pad);
  // host-call inputs x | lambda | y in one block laid out as the pinned staging, so that one copy
  // moves them
  AL(net->xin, (size_t)net->n_in_pad + 2 * (size_t)net->n_out);
  net->lam = net->xin + net->n_in_pad;
  net->yres = net->lam + net->n_out;
  {
    float2* x2;
    AL(x2, net->n_in_pad);
    net->x2 = x2;
  }
  AL(net->xr, net->n_in_pad);
  {
    float2* x2;
    AL(x2, net->n_in_pad);
    net->xr2 = x2;
  }
  AL(net->ydev, net->n_out);
  AL(net->rdev, net->n_out);
  AL(net->Zbar[0], (size_t)mp_max * net->S_max);
  AL(net->Zbar[1], (size_t)mp_max * net->S_max);
  AL(net->part, part_max);
  if (net->rev_stream) {
    AL(net->Zf[0], (size_t)mp_max * 16);
    AL(net->Zf[1], (size_t)mp_max * 16);
    AL(net->rev_cnt, rev_cnt_total);
  }
  AL(net->Jdev, (size_t)net->n_out * net->n_in);
  AL(net->gdev, net->n_in_pad);
  AL(net->Hdev, (size_t)net->n_in * net->n_in);
  AL(net->dev_err, 1);
  // tangent buffers: Adot ping-pong (n_in x mp_max) and the side-by-side Zdot / Ydot blocks
  const int n = net->n_in;
  net->K_total = 0;
  for (auto& Ly : net->layers) {
    Ly.zy_off = Ly.act == NNC_IDENTITY ? -1 : net->K_total;
    if (Ly.zy_off >= 0) net->K_total += Ly.mp;
  }
  // softmax output: two more columns (one padded block) carry the rank-two part of its curvature
  net->softmax = net->layers.back().act == NNC_SOFTMAX;
  if (net->softmax) {
    net->ext_off = net->K_total;
    net->K_total += kPad;
  }
  if (tc) {
    AL(net->cK, std::max(net->K_total, kPad));
    for (auto& Ly : net->layers)
      if (Ly.zy_off >= 0) Ly.c_f = net->cK + Ly.zy_off;
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&net->side_stream, cudaStreamNonBlocking, lo) != cudaSuccess ||
        cudaEventCreateWithFlags(&net->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&net->ev_join, cudaEventDisableTiming) != cudaSuccess)
      return fail(NNC_ERR_CUDA, "side stream or events could not be created");
  }
  const size_t tan_elems = (size_t)n * mp_max;
  const size_t zy_elems = (size_t)n * std::max(net->K_total, kPad);
  const size_t es = elem_size(prec);
  const bool x3 = prec == NNC_BF16X3;
  unsigned char* p;
  for (int pp = 0; pp < 2; ++pp) {
    AL(p, tan_elems * es);
    net->At[pp][0] = p;
    if (x3) {
      AL(p, tan_elems * es);
      net->At[pp][1] = p;
    }
  }
  for (int part = 0; part < (x3 ? 2 : 1); ++part) {
    AL(p, zy_elems * es);
    net->Zt[part] = p;
    AL(p, zy_elems * es);
    net->Yt[part] = p;
  }
  if (prec == NNC_FP8) {
    AL(net->A8, tan_elems);
    AL(net->tsc, n);
  }
  if (tc) {
    // Zdot_1 = W_1 does not depend on x: its block of the symmetric product's operand is written
    // here once, and each evaluation forms Adot_1 = sigma_1' W_1^T from an FP32 copy of W_1^T
    LayerDev& L1 = net->layers[0];
    AL(net->W1T, (size_t)n * L1.mp);
    CK(launch_transpose_f32(L1.W32, L1.kp, L1.mp, n, net->W1T, L1.mp, net->stream));
    if (L1.zy_off >= 0) {
      const size_t off = (size_t)L1.zy_off * es;
      TanBuf Z1{(char*)net->Zt[0] + off, net->Zt[1] ? (char*)net->Zt[1] + off : nullptr};
      CK(launch_first_tangent(tan_elem(prec), L1.W32, L1.kp, L1.mp, n, L1.s1, L1.c, TanBuf{}, L1.mp,
                              Z1, TanBuf{}, net->K_total, net->stream));
    }
  }
  // split-K partial sums of H
  if (tc) {
    net->hp_f32 = true;
    for (int l = 1; l < n_layers; ++l) {
      LayerDev& Ly = net->layers[l];
      const int cur = (l - 1) % 2;
      int r = prec == NNC_FP8
                  ? tc_plan_make(Ly.plan_tan, TC_TANGENT, prec, Ly.W8, nullptr, Ly.mp, Ly.kp, net->A8,
                                 nullptr, n, Ly.kp, Ly.mp, n, Ly.kp, net->sm_count)
                  : tc_plan_make(Ly.plan_tan, TC_TANGENT, prec, Ly.Whi, Ly.Wlo, Ly.mp, Ly.kp,
                                 net->At[cur][0], net->At[cur][1], n, Ly.kp, Ly.mp, n, Ly.kp,
                                 net->sm_count);
      if (r != NNC_OK) return fail(r, "tensor-core tangent plan failed");
    }
    // the persistent chain: every tangent GEMM of an evaluation in one launch (not FP8, whose
    // tangent operand is re-quantized between layers)
    if (prec == NNC_BF16 || prec == NNC_BF16X3) {
      int nl = 0;
      for (int l = 1; l < n_layers; ++l) {
        if (l == n_layers - 1 && net->layers[l].zy_off < 0) break;
        ++nl;
      }
      if (nl >= 1 && nl <= kMaxChain) {
        net->chain_plans.assign(nl, TcPlan());
        const int bn = net->layers[1].plan_tan.pair ? 208 : net->layers[1].plan_tan.bn;
        bool ok = true;
        for (int i = 0; i < nl && ok; ++i) {
          LayerDev& Ly = net->layers[i + 1];
          const int cur = i % 2;
          ok = tc_plan_make(net->chain_plans[i], TC_TANGENT, prec, Ly.Whi, Ly.Wlo, Ly.mp, Ly.kp,
                            net->At[cur][0], net->At[cur][1], n, Ly.kp, Ly.mp, n, Ly.kp,
                            net->sm_count, bn) == NNC_OK;
        }
        if (ok) {
          unsigned* cnt;
          AL(cnt, (size_t)nl * net->chain_plans[0].ntn);
          net->chain_cnt = cnt;
          net->chain_nl = nl;
          net->use_chain = true;
        } else {
          net->chain_plans.clear();
        }
      }
    }
    // reverse sweep on the tensor cores (seed columns padded to 16 or 48)
    if (net->S_max > 16 && net->S_max <= 48) {
      size_t prev = 1;
      for (int pp = 0; pp < 2; ++pp)
        for (int part = 0; part < 3; ++part) {
          __nv_bfloat16* zb;
          AL(zb, (size_t)48 * mp_max);
          net->Zb[pp][part] = zb;
        }
      for (int l = 0; l < n_layers; ++l) {
        LayerDev& Ly = net->layers[l];
        const int zi = (n_layers - 1 - l) % 2;
        int r = tc_plan_make(Ly.plan_rev, TC_REV, prec, Ly.WThi, Ly.WTlo, Ly.kp, Ly.mp, net->Zb[zi][0],
                             net->Zb[zi][1], 48, Ly.mp, Ly.kp, net->S_max, Ly.mp, net->sm_count, 0, 0,
                             Ly.WTp2, net->Zb[zi][2]);
        if (r != NNC_OK) return fail(r, "tensor-core reverse plan failed");
        prev = std::max(prev, (size_t)Ly.plan_rev.splits * Ly.kp * Ly.plan_rev.bn);
      }
      AL(net->Prev, prev);
      net->tc_rev = true;
    }
    int splits = 1;
    if (net->K_total > 0) {
      int r = tc_plan_make(net->plan_syrk, TC_SYRK, prec, net->Zt[0], net->Zt[1], n, net->K_total,
                           net->Yt[0], net->Yt[1], n, net->K_total, n, n, net->K_total,
                           net->sm_count);
      if (r != NNC_OK) return fail(r, "tensor-core symmetric-product plan failed");
      splits = net->plan_syrk.splits;
      // room for the split partials of the 256-column tile too (the autotuner may pick it)
      TcPlan p256;
      if (tc_plan_make(p256, TC_SYRK, prec, net->Zt[0], net->Zt[1], n, net->K_total, net->Yt[0],
                       net->Yt[1], n, net->K_total, n, n, net->K_total, net->sm_count, 256) == NNC_OK)
        splits = std::max(splits, p256.splits);
    }
    net->h_splits = splits;
    float* hp;
    AL(hp, (size_t)splits * n * n);
    net->Hp = hp;
  } else {
    const int tile = prec == NNC_FP64 ? 64 : 128;
    const int T = (n + tile - 1) / tile;
    const int tiles = T * (T + 1) / 2;
    int splits = (2 * net->sm_count + tiles - 1) / tiles;
    splits = std::max(1, std::min(splits, std::max(net->K_total, kPad) / 256));
    net->h_splits = splits;
    net->hp_f32 = false;
    double* hp;
    AL(hp, (size_t)splits * n * n);
    net->Hp = hp;
  }
  // pinned staging of the host calls: x [n_in_pad] | lambda [n_out] | y [n_out] | error word
  net->h_stage_elems = (size_t)net->n_in_pad + 2 * (size_t)net->n_out + 1;
  CK(cudaMallocHost(&net->h_stage, sizeof(double) * net->h_stage_elems));
  CK(cudaStreamSynchronize(net->stream));
  return NNC_OK;
}

int nnc_load_weights(nnc_net** out, int n_layers, const int* widths, const int* act,
                     const double* const* W, const double* const* b, int prec, void* stream) {
  if (!out) return fail(NNC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n_layers < 1 || !widths || !act || !W) return fail(NNC_ERR_ARG, "bad layer description");
  for (int l = 0; l <= n_layers; ++l)
    if (widths[l] < 1 || widths[l] > 65536) return fail(NNC_ERR_ARG, "width out of range [1, 65536]");
  for (int l = 0; l < n_layers; ++l) {
    if (act[l] < NNC_IDENTITY || act[l] > NNC_SOFTMAX) return fail(NNC_ERR_ARG, "bad activation code");
    if (act[l] == NNC_SOFTMAX && (l != n_layers - 1 || widths[n_layers] > 64))
      return fail(NNC_ERR_ARG, "softmax is an output-layer activation with at most 64 outputs");
    if (!W[l]) return fail(NNC_ERR_ARG, "W[l] is NULL");
  }
  if (prec < NNC_FP64 || prec > NNC_FP8) return fail(NNC_ERR_ARG, "bad precision code");
  nnc_net* net = new nnc_net();
  net->prec = prec;
  if (stream) {
    net->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&net->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete net;
      return fail(NNC_ERR_CUDA, "no CUDA device or cudaStreamCreate failed");
    }
    net->own_stream = true;
  }
  int r = load_impl(net, n_layers, widths, act, W, b);
  if (r != NNC_OK) {
    std::string keep = g_err;
    nnc_free(net);
    g_err = keep;
    return r;
  }
  *out = net;
  return NNC_OK;
}

int nnc_eval(nnc_net* net, const double* x, double* y, int fp64_residual) {
  int r = check_net(net);
  if (r) return r;
  if (!x || !y) return fail(NNC_ERR_ARG, "x or y is NULL");
  if (!fp64_residual) return host_call(net, x, nullptr, y, nullptr, nullptr, nullptr);
  r = check_finite(x, net->n_in, "x");
  if (r) return r;
  CK(cudaSetDevice(net->device));
  cudaStream_t st = net->stream;
  std::memcpy(net->h_stage, x, sizeof(double) * net->n_in);
  CK(cudaMemcpyAsync(net->xin, net->h_stage, sizeof(double) * net->n_in, cudaMemcpyHostToDevice, st));
  r = run_forward_fp64_values(net, net->xin, st);
  if (r) return r;
  CK(cudaMemcpyAsync(y, net->layers.back().ra, sizeof(double) * net->n_out, cudaMemcpyDeviceToHost, st));
  return sync_check(net, st);   // the value pass's bounded waits too
}

int nnc_eval_dev(nnc_net* net, const double* x, double* y, int fp64_residual, void* stream) {
  int r = check_net(net);
  if (r) return r;
  if (!x || !y) return fail(NNC_ERR_ARG, "x or y is NULL");
  cudaStream_t st = pick(net, stream);
  if (fp64_residual) {
    r = run_forward_fp64_values(net, x, st);
  } else {
    CK(launch_copy_pad(x, net->x, net->x2, net->n_in, net->n_in_pad, st));
    r = run_forward(net, net->prec == NNC_FP64, st);
  }
  if (r) return r;
  const double* aL = fp64_residual ? net->layers.back().ra : net->layers.back().a;
  CK(cudaMemcpyAsync(y, aL, sizeof(double) * net->n_out, cudaMemcpyDeviceToDevice, st));
  return NNC_OK;
}

int nnc_residual_dev(nnc_net* net, const double* x, const double* y, double* rr, void* stream) {
  int r = check_net(net);
  if (r) return r;
  if (!x || !y || !rr) return fail(NNC_ERR_ARG, "x, y or r is NULL");
  cudaStream_t st = pick(net, stream);
  r = run_forward_fp64_values(net, x, st);
  if (r) return r;
  CK(launch_sub(y, net->layers.back().ra, rr, net->n_out, st));
  return NNC_OK;
}

int nnc_residual(nnc_net* net, const double* x, const double* y, double* rr) {
  int r = check_net(net);
  if (r) return r;
  if (!x || !y || !rr) return fail(NNC_ERR_ARG, "x, y or r is NULL");
  r = check_finite(x, net->n_in, "x");
  if (r) return r;
  CK(cudaSetDevice(net->device));
  cudaStream_t st = net->stream;
  std::memcpy(net->h_stage, x, sizeof(double) * net->n_in);
  double* hy = net->h_stage + net->n_in_pad + net->n_out;
  std::memcpy(hy, y, sizeof(double) * net->n_out);
  CK(cudaMemcpyAsync(net->xin, net->h_stage, sizeof(double) * net->n_in, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(net->yres, hy, sizeof(double) * net->n_out,
                     cudaMemcpyHostToDevice, st));
  r = nnc_residual_dev(net, net->xin, net->yres, net->rdev, st);
  if (r) return r;
  CK(cudaMemcpyAsync(rr, net->rdev, sizeof(double) * net->n_out, cudaMemcpyDeviceToHost, st));
  return sync_check(net, st);   // the value pass's bounded waits too
}

int nnc_jacobian(nnc_net* net, const double* x, double* J) {
  if (!J) return fail(NNC_ERR_ARG, "J is NULL");
  return host_call(net, x, nullptr, nullptr, J, nullptr, nullptr);
}

int nnc_jacobian_dev(nnc_net* net, const double* x, double* J, void* stream) {
  int r = check_net(net);
  if (r) return r;
  if (!x || !J) return fail(NNC_ERR_ARG, "x or J is NULL");
  return eval_all(net, x, nullptr, nullptr, J, nullptr, nullptr, pick(net, stream));
}

int nnc_hessian_lag(nnc_net* net, const double* x, const double* lambda, double* H, double* grad) {
  if (!H) return fail(NNC_ERR_ARG, "H is NULL");
  return host_call(net, x, lambda, nullptr, nullptr, H, grad);
}

int nnc_hessian_lag_dev(nnc_net* net, const double* x, const double* lambda, double* H,
                        double* grad, void* stream) {
  int r = check_net(net);
  if (r) return r;
  if (!x || !lambda || !H) return fail(NNC_ERR_ARG, "x, lambda or H is NULL");
  return eval_all(net, x, lambda, nullptr, nullptr, H, grad, pick(net, stream));
}

int nnc_eval_all_dev(nnc_net* net, const double* x, const double* lambda, double* y, double* J,
                     double* H, double* grad, void* stream) {
  int r = check_net(net);
  if (r) return r;
  if (!x) return fail(NNC_ERR_ARG, "x is NULL");
  if ((H || grad) && !lambda) return fail(NNC_ERR_ARG, "lambda is NULL");
  return eval_all(net, x, lambda, y, J, H, grad, pick(net, stream));
}

int nnc_eval_kkt(nnc_net* net, const double* x, const double* y, const double* lambda, double* r,
                 double* J, double* H, double* grad) {
  if (r && !y) return fail(NNC_ERR_ARG, "y is NULL");
  if (y) {
    const int rc = check_finite(y, net ? net->n_out : 0, "y");
    if (rc) return rc;
  }
  return host_call(net, x, lambda, nullptr, J, H, grad, y, r);
}

int nnc_eval_kkt_dev(nnc_net* net, const double* x, const double* y, const double* lambda,
                     double* r, double* J, double* H, double* grad, void* stream) {
  int rc = check_net(net);
  if (rc) return rc;
  if (!x) return fail(NNC_ERR_ARG, "x is NULL");
  if (r && !y) return fail(NNC_ERR_ARG, "y is NULL");
  if ((H || grad) && !lambda) return fail(NNC_ERR_ARG, "lambda is NULL");
  return eval_all(net, x, lambda, nullptr, J, H, grad, pick(net, stream), y, r);
}

int nnc_eval_batched(nnc_net* const* nets, int K, const double* const* x,
                     const double* const* lambda, double* const* y, double* const* J,
                     double* const* H, unsigned what) {
  if (K < 0 || (K > 0 && (!nets || !x))) return fail(NNC_ERR_ARG, "bad batch arguments");
  if ((what & NNC_WANT_Y) && !y) return fail(NNC_ERR_ARG, "y array is NULL");
  if ((what & NNC_WANT_J) && !J) return fail(NNC_ERR_ARG, "J array is NULL");
  if ((what & NNC_WANT_H) && (!H || !lambda)) return fail(NNC_ERR_ARG, "H or lambda array is NULL");
  if (K > 1 && !(what & NNC_WANT_G)) {
    // grouped path (one launch per step for all nets) when the nets qualify
    for (int k = 0; k < K; ++k) {
      if (!nets[k] || !x[k]) return fail(NNC_ERR_ARG, "NULL net or x");
      int r = check_finite(x[k], nets[k]->n_in, "x");
      if (r) return r;
      if (what & NNC_WANT_H) {
        if (!lambda[k]) return fail(NNC_ERR_ARG, "NULL lambda");
        r = check_finite(lambda[k], nets[k]->n_out, "lambda");
        if (r) return r;
      }
    }
    int r = eval_batched_grouped(nets, K, x, lambda, y, J, H, what);
    if (r != NNC_ERR_UNSUPPORTED) return r;
  }
  for (int k = 0; k < K; ++k) {
    int r = host_call(nets[k], x[k], (what & NNC_WANT_H) ? lambda[k] : nullptr,
                      (what & NNC_WANT_Y) ? y[k] : nullptr, (what & NNC_WANT_J) ? J[k] : nullptr,
                      (what & NNC_WANT_H) ? H[k] : nullptr, nullptr);
    if (r != NNC_OK) return r;
  }
  return NNC_OK;
}

}  // extern "C"
