// nnc_batch: many networks with the same hidden widths and activations but different input
// sizes (one stability-margin surrogate per contingency of Eq. 8), evaluated together.
//
// Layout: each layer's weights of all K networks are stacked (network g's rows start at g * mp_l;
// the first layer is padded to the widest input), so one grouped launch runs the same step of
// every network: the value pass, the reverse sweep (Jacobian + adjoint seeds), the first-layer
// tangents, one grouped tcgen05 tangent GEMM per hidden layer (the MMA N of each CTA set from
// its network's input count), one grouped symmetric product over the lower-triangle tiles of
// every network's Hessian, and the grouped finish.  The whole sequence can be captured once in
// a CUDA graph and replayed with fixed device buffers.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/nnc.h"
#include "batch.cuh"
#include "net.cuh"

namespace nnc {
void note_launch(int n);
}
using namespace nnc;

namespace {

struct BLayer {
  int m = 0, k = 0, act = 0, mp = 0, kp = 0, zy_off = -1;
  double* W64 = nullptr;
  float* W32 = nullptr;
  float2* W2 = nullptr;           // double-float (hi, lo) pairs of the weights (value passes)
  __nv_bfloat16 *Whi = nullptr, *Wlo = nullptr;
  double* b = nullptr;
  double *a = nullptr, *s1 = nullptr, *s2 = nullptr, *c = nullptr, *ra = nullptr;
  float2 *a2 = nullptr, *ra2 = nullptr;   // double-float pairs of a and ra (next layer's input)
  float* c_f = nullptr;
  TcPlan plan_tan;
};

int bfail(int code, const std::string& msg) {
  set_last_error(msg);
  return code;
}

}  // namespace

struct nnc_batch {
  int K = 0, L = 0, n_out = 0, prec = 0, n_sum = 0, n_max = 0, kp0 = 0, K_total = 0, S = 0;
  long long h_sum = 0;
  int device = 0, sm_count = 0;
  std::vector<int> n_k, boff;
  std::vector<long long> hoff;
  std::vector<nnc_net*> members;
  int *d_gn = nullptr, *d_goff = nullptr;
  long long* d_hoff = nullptr;
  int4* d_work = nullptr;
  int n_work = 0;
  std::vector<BLayer> layers;
  double *xs = nullptr, *lam = nullptr, *Zbar[2] = {nullptr, nullptr};
  float2* xs2 = nullptr;   // double-float pairs of the scattered inputs
  float* part = nullptr;
  void *At[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}}, *Zt[2] = {nullptr, nullptr},
       *Yt[2] = {nullptr, nullptr};
  float* Hp = nullptr;
  int hp_planes = 0;   // split-K planes Hp holds
  TcPlan plan_syrk;
  int* dev_err = nullptr;
  // device staging for the host-pointer calls
  double *x_in = nullptr, *lam_in = nullptr, *y_out = nullptr, *J_out = nullptr, *H_out = nullptr,
         *g_out = nullptr, *r_out = nullptr, *y_in = nullptr;
  double* h_stage = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<void*> allocs;
  size_t bytes = 0;
  // CUDA graph of one evaluation, keyed by its pointer arguments
  bool use_graph = false;
  cudaGraphExec_t gexec = nullptr;
  int g_kernels = 0;   // kernel nodes of the captured evaluation
  const void* gkey[9] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                         nullptr};
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

namespace {

#define BCK(expr)                                                                         \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return bfail(e_ == cudaErrorMemoryAllocation ? NNC_ERR_OOM : NNC_ERR_CUDA,          \
                   std::string(#expr) + ": " + cudaGetErrorString(e_));                   \
  } while (0)

template <typename T>
int balloc(nnc_batch* b, T** p, size_t n) {
  void* q = nullptr;
  const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) return bfail(NNC_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  e = cudaMemsetAsync(q, 0, bytes, b->stream);
  if (e != cudaSuccess) return bfail(NNC_ERR_CUDA, cudaGetErrorString(e));
  b->allocs.push_back(q);
  b->bytes += bytes;
  *p = (T*)q;
  return NNC_OK;
}
#define BAL(p, n)                     \
  do {                                \
    int r_ = balloc(b, &(p), (n));    \
    if (r_ != NNC_OK) return r_;      \
  } while (0)

bool is_tc_prec(int p) { return p == NNC_BF16 || p == NNC_BF16X3; }

// Value pass of every network in double-float arithmetic (one grouped streaming launch per layer):
// a (FP64-accurate), its pairs for the next layer and, for an evaluation, sigma' and sigma''.
int batch_value(nnc_batch* b, const double* x, bool residual, cudaStream_t st) {
  const int K = b->K;
  BCK(launch_bx_scatter(x, b->d_gn, b->d_goff, b->kp0, K, b->xs, nullptr, st));
  BCK(launch_split_df(b->xs, (size_t)K * b->kp0, b->xs2, st));
  const void* a_in = b->xs2;
  int ld_in = b->kp0;
  for (auto& Ly : b->layers) {
    // the first layer's rows hold each net's n_k inputs, padded to the widest: skip the padding
    BCK(launch_gemv_stream_df_grouped(Ly.W2, Ly.kp, K, Ly.mp, Ly.m, Ly.b, a_in, ld_in, Ly.act,
                                      residual ? Ly.ra : Ly.a, residual ? Ly.ra2 : Ly.a2,
                                      residual ? nullptr : Ly.s1, residual ? nullptr : Ly.s2,
                                      b->dev_err, b->sm_count, st,
                                      &Ly == &b->layers[0] ? b->d_gn : nullptr));
    a_in = residual ? Ly.ra2 : Ly.a2;
    ld_in = Ly.mp;
  }
  return NNC_OK;
}

int batch_eval(nnc_batch* b, const double* x, const double* lam, double* y, double* J, double* H,
               double* g, cudaStream_t st, const double* yv = nullptr, double* rr = nullptr) {
  const int K = b->K;
  const bool x3 = b->prec == NNC_BF16X3;
  int rv = batch_value(b, x, false, st);
  if (rv != NNC_OK) return rv;
  BLayer& Lo = b->layers.back();
  if (y) BCK(launch_bgather(Lo.a, b->n_out, Lo.mp, K, y, st));
  if (rr) BCK(launch_bsub(yv, Lo.a, b->n_out, Lo.mp, K, rr, st));   // y - NN(x), FP64-accurate
  if (!J && !H && !g) return NNC_OK;
  const int nJ = J ? b->n_out : 0;
  const bool with_lam = H || g;
  const int S = nJ + (with_lam ? 1 : 0);
  const int lam_col = with_lam ? nJ : -1;
  BCK(launch_brev_seed(b->n_out, Lo.mp, K, S, nJ, lam_col, Lo.s1, Lo.s2, lam, b->Zbar[0], Lo.c,
                       Lo.c_f, st));
  int cur = 0;
  for (int l = b->L - 1; l >= 0; --l) {
    BLayer& Ly = b->layers[l];
    BCK(launch_bgemv_rev(Ly.W32, Ly.kp, Ly.mp, Ly.m, K, b->Zbar[cur], S, b->part, st,
                         l == 0 ? b->d_gn : nullptr));
    const int chunks = bgemv_rev_chunks(Ly.m, Ly.kp);
    if (l > 0) {
      BLayer& Lp = b->layers[l - 1];
      BCK(launch_brev_reduce(b->part, chunks, Ly.kp, Lp.mp, K, S, Lp.s1, Lp.s2, lam_col, nJ,
                             b->Zbar[1 - cur], Lp.c, Lp.c_f, b->d_gn, b->d_goff, nullptr, nullptr, st));
      cur = 1 - cur;
    } else {
      BCK(launch_brev_reduce(b->part, chunks, Ly.kp, 0, K, S, nullptr, nullptr, lam_col, nJ, nullptr,
                             nullptr, nullptr, b->d_gn, b->d_goff, J, g, st));
    }
  }
  if (!H) return NNC_OK;
  BLayer& L1 = b->layers[0];
  auto zo = [&](void* base, int off) -> void* {
    return (base && off >= 0) ? (void*)((__nv_bfloat16*)base + off) : nullptr;
  };
  BCK(launch_bfirst_tangent(L1.W32, L1.kp, L1.mp, K, b->n_max, b->d_gn, b->d_goff, L1.s1, L1.c,
                            b->L > 1 ? b->At[0][0] : nullptr, b->At[0][1], L1.mp,
                            zo(b->Zt[0], L1.zy_off), zo(b->Zt[1], L1.zy_off), zo(b->Yt[0], L1.zy_off),
                            zo(b->Yt[1], L1.zy_off), b->K_total, x3, st));
  cur = 0;
  for (int l = 1; l < b->L; ++l) {
    BLayer& Ly = b->layers[l];
    const bool last = l == b->L - 1;
    if (last && Ly.zy_off < 0) break;
    BCK(tc_tangent_grouped(Ly.plan_tan, K, b->d_gn, b->d_goff, Ly.s1, Ly.c_f,
                           last ? nullptr : b->At[1 - cur][0], last ? nullptr : b->At[1 - cur][1],
                           Ly.mp, zo(b->Zt[0], Ly.zy_off), zo(b->Zt[1], Ly.zy_off),
                           zo(b->Yt[0], Ly.zy_off), zo(b->Yt[1], Ly.zy_off), b->K_total, b->dev_err,
                           st));
    cur = 1 - cur;
  }
  if (b->K_total == 0) {
    BCK(cudaMemsetAsync(H, 0, sizeof(double) * b->h_sum, st));
    return NNC_OK;
  }
  BCK(cudaMemsetAsync(b->Hp, 0, sizeof(float) * b->h_sum * b->plan_syrk.splits, st));
  BCK(tc_syrk_grouped(b->plan_syrk, b->n_work, b->d_work, b->d_gn, b->d_goff, b->d_hoff, b->h_sum,
                      b->Hp, b->dev_err, st));
  BCK(launch_bh_finish(b->Hp, b->plan_syrk.splits, b->h_sum, K, b->d_gn, b->d_hoff, H, st));
  return NNC_OK;
}

int batch_residual(nnc_batch* b, const double* x, const double* y, double* r, cudaStream_t st) {
  int rv = batch_value(b, x, true, st);
  if (rv != NNC_OK) return rv;
  BCK(launch_bsub(y, b->layers.back().ra, b->n_out, b->layers.back().mp, b->K, r, st));
  return NNC_OK;
}

int check_dev_err(nnc_batch* b) {
  int e = 0;
  BCK(cudaMemcpyAsync(&e, b->dev_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  if (e) {
    int z = 0;
    cudaMemcpy(b->dev_err, &z, sizeof(int), cudaMemcpyHostToDevice);
    return bfail(NNC_ERR_TIMEOUT, "a bounded device-side wait ran out (code " + std::to_string(e) + ")");
  }
  return NNC_OK;
}

// Host calls: queue the error word's copy behind the outputs into its pinned slot (the last
// element of h_stage), wait for the device once, then check it.
int sync_check(nnc_batch* b, cudaStream_t st) {
  int* herr = reinterpret_cast<int*>(b->h_stage + b->n_sum + 2 * (size_t)b->K * b->n_out);
  BCK(cudaMemcpyAsync(herr, b->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  BCK(cudaStreamSynchronize(st));
  if (*herr) {
    const int e = *herr;
    int z = 0;
    cudaMemcpy(b->dev_err, &z, sizeof(int), cudaMemcpyHostToDevice);
    return bfail(NNC_ERR_TIMEOUT, "a bounded device-side wait ran out (code " + std::to_string(e) + ")");
  }
  return NNC_OK;
}

int build(nnc_batch* b, nnc_net* const* nets, int K) {
  b->K = K;
  nnc_net* n0 = nets[0];
  b->L = n0->L;
  b->n_out = n0->n_out;
  b->prec = n0->prec;
  b->device = n0->device;
  b->sm_count = n0->sm_count;
  if (!is_tc_prec(b->prec)) return bfail(NNC_ERR_UNSUPPORTED, "batch needs a BF16 or BF16x3 net");
  if (nets[0]->softmax) return bfail(NNC_ERR_UNSUPPORTED, "batch members need an elementwise output layer");
  for (int k = 0; k < K; ++k) {
    nnc_net* n = nets[k];
    if (!n || n->L != b->L || n->n_out != b->n_out || n->prec != b->prec || n->device != b->device)
      return bfail(NNC_ERR_UNSUPPORTED, "batch members differ in depth, outputs, precision or device");
    for (int l = 0; l < b->L; ++l) {
      if (n->layers[l].act != n0->layers[l].act) return bfail(NNC_ERR_UNSUPPORTED, "activations differ");
      if (l > 0 && n->layers[l].k != n0->layers[l].k) return bfail(NNC_ERR_UNSUPPORTED, "hidden widths differ");
    }
    if (n->n_in > 256) return bfail(NNC_ERR_UNSUPPORTED, "batch members need n_in <= 256");
    b->members.push_back(n);
    b->n_k.push_back(n->n_in);
    b->boff.push_back(b->n_sum);
    b->hoff.push_back(b->h_sum);
    b->n_sum += n->n_in;
    b->h_sum += (long long)n->n_in * n->n_in;
    b->n_max = std::max(b->n_max, n->n_in);
  }
  b->S = b->n_out + 1;
  if (b->S > 4) return bfail(NNC_ERR_UNSUPPORTED, "batch members need n_out <= 3");
  b->kp0 = pad_up(b->n_max);
  const bool x3 = b->prec == NNC_BF16X3;
  // group metadata and the lower-triangle tile list of the symmetric product
  std::vector<int4> work;
  for (int k = 0; k < K; ++k) {
    const int t = (b->n_k[k] + 127) / 128;
    for (int tm = 0; tm < t; ++tm)
      for (int tn = 0; tn <= tm; ++tn) work.push_back(make_int4(k, tm, tn, 0));
  }
  b->n_work = (int)work.size();
  BAL(b->d_gn, K);
  BAL(b->d_goff, K);
  BAL(b->d_hoff, K);
  BAL(b->d_work, work.size());
  BCK(cudaMemcpyAsync(b->d_gn, b->n_k.data(), sizeof(int) * K, cudaMemcpyHostToDevice, b->stream));
  BCK(cudaMemcpyAsync(b->d_goff, b->boff.data(), sizeof(int) * K, cudaMemcpyHostToDevice, b->stream));
  BCK(cudaMemcpyAsync(b->d_hoff, b->hoff.data(), sizeof(long long) * K, cudaMemcpyHostToDevice, b->stream));
  BCK(cudaMemcpyAsync(b->d_work, work.data(), sizeof(int4) * work.size(), cudaMemcpyHostToDevice, b->stream));
  // stacked weights: copy every member's packed FP64 layer, then re-pack
  b->layers.resize(b->L);
  int mp_max = b->kp0;
  size_t part_max = 1;
  for (int l = 0; l < b->L; ++l) {
    BLayer& Ly = b->layers[l];
    const LayerDev& R = n0->layers[l];
    Ly.m = R.m;
    Ly.act = R.act;
    Ly.mp = R.mp;
    Ly.k = l == 0 ? b->n_max : R.k;
    Ly.kp = l == 0 ? b->kp0 : R.kp;
    mp_max = std::max(mp_max, Ly.mp);
    const size_t per = (size_t)Ly.mp * Ly.kp;
    BAL(Ly.W64, per * K);
    BAL(Ly.W32, per * K);
    BAL(Ly.W2, per * K);
    if (l > 0) {
      BAL(Ly.Whi, per * K);
      if (x3) BAL(Ly.Wlo, per * K);
    }
    BAL(Ly.b, (size_t)Ly.mp * K);
    for (int k = 0; k < K; ++k) {
      const LayerDev& S = nets[k]->layers[l];
      BCK(cudaMemcpy2DAsync(Ly.W64 + per * k, sizeof(double) * Ly.kp, S.W64, sizeof(double) * S.kp,
                            sizeof(double) * S.kp, S.mp, cudaMemcpyDeviceToDevice, b->stream));
      BCK(cudaMemcpyAsync(Ly.b + (size_t)Ly.mp * k, S.b, sizeof(double) * S.mp,
                          cudaMemcpyDeviceToDevice, b->stream));
    }
    BCK(launch_pack(Ly.W64, per * K, Ly.W32, Ly.Whi, Ly.Wlo, b->stream));
    BCK(launch_split_df(Ly.W64, per * K, Ly.W2, b->stream));
    BAL(Ly.a, (size_t)Ly.mp * K);
    BAL(Ly.a2, (size_t)Ly.mp * K);
    BAL(Ly.ra2, (size_t)Ly.mp * K);
    BAL(Ly.s1, (size_t)Ly.mp * K);
    BAL(Ly.s2, (size_t)Ly.mp * K);
    BAL(Ly.c, (size_t)Ly.mp * K);
    BAL(Ly.c_f, (size_t)Ly.mp * K);
    BAL(Ly.ra, (size_t)Ly.mp * K);
    part_max = std::max(part_max, (size_t)K * bgemv_rev_chunks(Ly.m, Ly.kp) * Ly.kp * b->S);
  }
  BAL(b->xs, (size_t)K * b->kp0);
  BAL(b->xs2, (size_t)K * b->kp0);
  BAL(b->Zbar[0], (size_t)K * mp_max * b->S);
  BAL(b->Zbar[1], (size_t)K * mp_max * b->S);
  BAL(b->part, part_max);
  BAL(b->dev_err, 1);
  b->K_total = 0;
  for (auto& Ly : b->layers) {
    Ly.zy_off = Ly.act == NNC_IDENTITY ? -1 : b->K_total;
    if (Ly.zy_off >= 0) b->K_total += Ly.mp;
  }
  const size_t tan = (size_t)b->n_sum * mp_max, zy = (size_t)b->n_sum * std::max(b->K_total, kPad);
  __nv_bfloat16* p;
  for (int pp = 0; pp < 2; ++pp) {
    BAL(p, tan);
    b->At[pp][0] = p;
    if (x3) {
      BAL(p, tan);
      b->At[pp][1] = p;
    }
  }
  for (int part = 0; part < (x3 ? 2 : 1); ++part) {
    BAL(p, zy);
    b->Zt[part] = p;
    BAL(p, zy);
    b->Yt[part] = p;
  }
  for (int l = 1; l < b->L; ++l) {
    BLayer& Ly = b->layers[l];
    const int cur = (l - 1) % 2;
    int r = tc_plan_make(Ly.plan_tan, TC_TANGENT_G, b->prec, Ly.Whi, Ly.Wlo, Ly.mp * K, Ly.kp,
                         b->At[cur][0], b->At[cur][1], b->n_sum, Ly.kp, Ly.mp, b->n_max, Ly.kp,
                         b->sm_count);
    if (r != NNC_OK) return bfail(r, "grouped tangent plan failed");
  }
  if (b->K_total > 0) {
    int r = tc_plan_make(b->plan_syrk, TC_SYRK_G, b->prec, b->Zt[0], b->Zt[1], b->n_sum, b->K_total,
                         b->Yt[0], b->Yt[1], b->n_sum, b->K_total, b->n_max, b->n_max, b->K_total,
                         b->sm_count);
    if (r != NNC_OK) return bfail(r, "grouped symmetric-product plan failed");
    BAL(b->Hp, (size_t)b->h_sum * b->plan_syrk.splits);
    b->hp_planes = b->plan_syrk.splits;
  }
  BAL(b->lam, (size_t)K * b->n_out);
  BAL(b->x_in, b->n_sum);
  BAL(b->lam_in, (size_t)K * b->n_out);
  BAL(b->y_out, (size_t)K * b->n_out);
  BAL(b->y_in, (size_t)K * b->n_out);
  BAL(b->r_out, (size_t)K * b->n_out);
  BAL(b->J_out, (size_t)b->n_sum * b->n_out);
  BAL(b->g_out, b->n_sum);
  BAL(b->H_out, b->h_sum);
  BCK(cudaMallocHost(&b->h_stage, sizeof(double) * (b->n_sum + 2 * (size_t)K * b->n_out + 1)));
  BCK(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
  BCK(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
  BCK(cudaStreamSynchronize(b->stream));
  return NNC_OK;
}

// The last batch built by nnc_eval_batched, reused while it is called with the same nets.
std::mutex g_cache_mu;
nnc_batch* g_cache = nullptr;

}  // namespace

namespace nnc {
// Called by nnc_free: drop the cached batch if it holds this net.
void batch_cache_forget(const nnc_net* net) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  if (!g_cache) return;
  for (auto* m : g_cache->members)
    if (m == net) {
      nnc_batch_free(g_cache);
      g_cache = nullptr;
      return;
    }
}
}  // namespace nnc

extern "C" {

int nnc_batch_create(nnc_batch** out, nnc_net* const* nets, int K, void* stream) {
  if (!out || !nets || K < 1) return bfail(NNC_ERR_ARG, "nnc_batch_create: bad arguments");
  *out = nullptr;
  nnc_batch* b = new nnc_batch();
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return bfail(NNC_ERR_CUDA, "cudaStreamCreate failed");
    }
    b->own_stream = true;
  }
  int r = build(b, nets, K);
  if (r != NNC_OK) {
    nnc_batch_free(b);
    return r;
  }
  *out = b;
  return NNC_OK;
}

void nnc_batch_free(nnc_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  for (void* p : b->allocs) cudaFree(p);
  if (b->h_stage) cudaFreeHost(b->h_stage);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

int nnc_batch_info(const nnc_batch* b, int* K, int* n_out, int* n_sum, long long* h_sum) {
  if (!b) return bfail(NNC_ERR_ARG, "batch is NULL");
  if (K) *K = b->K;
  if (n_out) *n_out = b->n_out;
  if (n_sum) *n_sum = b->n_sum;
  if (h_sum) *h_sum = b->h_sum;
  return NNC_OK;
}

int nnc_batch_set_bias(nnc_batch* b, int layer, const double* bias) {
  if (!b || !bias || layer < 0 || layer >= b->L) return bfail(NNC_ERR_ARG, "nnc_batch_set_bias: bad arguments");
  BLayer& Ly = b->layers[layer];
  BCK(cudaSetDevice(b->device));
  BCK(cudaMemcpy2DAsync(Ly.b, sizeof(double) * Ly.mp, bias, sizeof(double) * Ly.m, sizeof(double) * Ly.m,
                        b->K, cudaMemcpyHostToDevice, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  return NNC_OK;
}

int nnc_batch_tune_set(nnc_batch* b, int syrk_splits) {
  if (!b || syrk_splits < 1 || syrk_splits > 32) return bfail(NNC_ERR_ARG, "nnc_batch_tune_set: splits in [1, 32]");
  if (b->K_total == 0) return NNC_OK;
  BCK(cudaSetDevice(b->device));
  BCK(cudaStreamSynchronize(b->stream));
  TcPlan p;
  int r = tc_plan_make(p, TC_SYRK_G, b->prec, b->Zt[0], b->Zt[1], b->n_sum, b->K_total, b->Yt[0],
                       b->Yt[1], b->n_sum, b->K_total, b->n_max, b->n_max, b->K_total, b->sm_count,
                       0, syrk_splits);
  if (r != NNC_OK) return bfail(r, "grouped symmetric-product plan failed");
  if (p.splits > b->hp_planes) {
    float* hp = nullptr;
    BCK(cudaMalloc(&hp, sizeof(float) * (size_t)b->h_sum * p.splits));
    b->allocs.push_back(hp);   // the smaller buffer stays allocated until nnc_batch_free
    b->Hp = hp;
    b->hp_planes = p.splits;
  }
  b->plan_syrk = p;
  if (b->gexec) {   // the captured graph holds the old plan
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  return NNC_OK;
}

// Autotuner of a batch: times whole evaluations (value pass, reverse sweep, grouped tangent GEMMs,
// grouped symmetric product; CUDA events on the batch's stream, its own buffers, no graph) for
// every grouped-tangent N tile that covers the widest network and split-K counts 1 .. 3 of the
// symmetric product, and keeps the fastest; choices are cached in a text file (one line per
// batch shape: key, N tile, splits, microseconds).
int nnc_batch_autotune(nnc_batch* b, const char* cache_path, int retune, int* tangent_bn,
                       int* syrk_splits) {
  if (!b) return bfail(NNC_ERR_ARG, "batch is NULL");
  if (!(b->prec == NNC_BF16 || b->prec == NNC_BF16X3) || b->L < 2 || b->K_total == 0) {
    if (tangent_bn) *tangent_bn = b->L > 1 ? b->layers[1].plan_tan.bn : 0;
    if (syrk_splits) *syrk_splits = b->K_total > 0 ? b->plan_syrk.splits : 0;
    return NNC_OK;
  }
  BCK(cudaSetDevice(b->device));
  cudaDeviceProp prop;
  BCK(cudaGetDeviceProperties(&prop, b->device));
  char kb[256];
  std::snprintf(kb, sizeof kb, "batch-sm%d%d-%dsm-prec%d-K%d-nmax%d-hidden%d-depth%d", prop.major, prop.minor,
                prop.multiProcessorCount, b->prec, b->K, b->n_max, b->layers[1].mp, b->L);
  const std::string key = kb;
  int best_bn = 0, best_sp = 0;
  if (cache_path && !retune) {
    FILE* f = std::fopen(cache_path, "r");
    if (f) {
      char k[256];
      int bn = 0, sp = 0;
      double us = 0;
      while (std::fscanf(f, "%255s %d %d %lf", k, &bn, &sp, &us) == 4)
        if (key == k) {
          best_bn = bn;
          best_sp = sp;
        }
      std::fclose(f);
    }
  }
  auto apply = [&](int bn, int sp) -> int {
    for (int l = 1; l < b->L; ++l) {
      BLayer& Ly = b->layers[l];
      const int cur = (l - 1) % 2;
      TcPlan p;
      int r = tc_plan_make(p, TC_TANGENT_G, b->prec, Ly.Whi, Ly.Wlo, Ly.mp * b->K, Ly.kp, b->At[cur][0],
                           b->At[cur][1], b->n_sum, Ly.kp, Ly.mp, b->n_max, Ly.kp, b->sm_count, bn);
      if (r != NNC_OK) return r;
      Ly.plan_tan = p;
    }
    return nnc_batch_tune_set(b, sp);
  };
  double best_us = 1e30;
  if (!best_bn) {
    const int cands[4] = {112, 128, 208, 256};
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    for (int bn : cands) {
      if (bn < (b->n_max + 15) / 16 * 16) continue;   // one column tile per network
      for (int sp = 1; sp <= 3; ++sp) {
        if (apply(bn, sp) != NNC_OK) continue;
        auto run = [&] {
          return batch_eval(b, b->x_in, b->lam_in, nullptr, b->J_out, b->H_out, b->g_out, b->stream,
                            b->y_in, b->r_out);
        };
        if (run() != NNC_OK) continue;
        cudaEventRecord(e0, b->stream);
        bool ok = true;
        for (int i = 0; i < 3 && ok; ++i) ok = run() == NNC_OK;
        cudaEventRecord(e1, b->stream);
        if (!ok || cudaEventSynchronize(e1) != cudaSuccess) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double us = 1e3 * ms / 3;
        if (us < best_us) {
          best_us = us;
          best_bn = bn;
          best_sp = sp;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int r = check_dev_err(b);
    if (r) return r;
    if (!best_bn) return bfail(NNC_ERR_CUDA, "batch autotune: no candidate ran");
    if (cache_path) {
      FILE* f = std::fopen(cache_path, "a");
      if (f) {
        std::fprintf(f, "%s %d %d %.3f\n", key.c_str(), best_bn, best_sp, best_us);
        std::fclose(f);
      }
    }
  }
  int r = apply(best_bn, best_sp);
  if (r) return bfail(r, "batch autotune: the chosen tiling has no valid plan");
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  if (tangent_bn) *tangent_bn = best_bn;
  if (syrk_splits) *syrk_splits = best_sp;
  return NNC_OK;
}

int nnc_batch_tuning(const nnc_batch* b, int* syrk_splits) {
  if (!b) return bfail(NNC_ERR_ARG, "batch is NULL");
  if (syrk_splits) *syrk_splits = b->K_total > 0 ? b->plan_syrk.splits : 0;
  return NNC_OK;
}

int nnc_batch_use_graph(nnc_batch* b, int enable) {
  if (!b) return bfail(NNC_ERR_ARG, "batch is NULL");
  b->use_graph = enable != 0;
  if (!b->use_graph && b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  return NNC_OK;
}

static int batch_eval_dev(nnc_batch* b, const double* x, const double* yv, const double* lambda,
                          double* rr, double* y, double* J, double* H, double* grad, void* stream) {
  cudaStream_t st = stream ? (cudaStream_t)stream : b->stream;
  if (!b->use_graph) return batch_eval(b, x, lambda, y, J, H, grad, st, yv, rr);
  // Graph mode: capture once on the batch's own stream, replay while the pointers match.
  const void* key[9] = {x, lambda, y, J, H, grad, yv, rr, nullptr};
  if (b->gexec && std::memcmp(key, b->gkey, sizeof(key)) != 0) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  if (!b->gexec) {
    cudaGraph_t graph;
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int r = batch_eval(b, x, lambda, y, J, H, grad, b->stream, yv, rr);
    cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    if (r != NNC_OK) return r;
    BCK(e);
    size_t nn = 0;
    b->g_kernels = 0;
    if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess && nn) {
      std::vector<cudaGraphNode_t> nodes(nn);
      if (cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess)
        for (size_t i = 0; i < nn; ++i) {
          cudaGraphNodeType t;
          if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++b->g_kernels;
        }
    }
    e = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    BCK(e);
    std::memcpy(b->gkey, key, sizeof(key));
  }
  if (st != b->stream) {
    BCK(cudaEventRecord(b->ev_in, st));
    BCK(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
  }
  BCK(cudaGraphLaunch(b->gexec, b->stream));
  note_launch(b->g_kernels);
  if (st != b->stream) {
    BCK(cudaEventRecord(b->ev_out, b->stream));
    BCK(cudaStreamWaitEvent(st, b->ev_out, 0));
  }
  return NNC_OK;
}

int nnc_batch_eval_dev(nnc_batch* b, const double* x, const double* lambda, double* y, double* J,
                       double* H, double* grad, void* stream) {
  if (!b || !x || ((H || grad) && !lambda)) return bfail(NNC_ERR_ARG, "nnc_batch_eval_dev: bad arguments");
  return batch_eval_dev(b, x, nullptr, lambda, nullptr, y, J, H, grad, stream);
}

int nnc_batch_eval_kkt_dev(nnc_batch* b, const double* x, const double* y, const double* lambda,
                           double* r, double* J, double* H, double* grad, void* stream) {
  if (!b || !x || (r && !y) || ((H || grad) && !lambda))
    return bfail(NNC_ERR_ARG, "nnc_batch_eval_kkt_dev: bad arguments");
  return batch_eval_dev(b, x, y, lambda, r, nullptr, J, H, grad, stream);
}

int nnc_batch_residual_dev(nnc_batch* b, const double* x, const double* y, double* r, void* stream) {
  if (!b || !x || !y || !r) return bfail(NNC_ERR_ARG, "nnc_batch_residual_dev: bad arguments");
  return batch_residual(b, x, y, r, stream ? (cudaStream_t)stream : b->stream);
}

int nnc_batch_eval(nnc_batch* b, const double* x, const double* lambda, double* y, double* J,
                   double* H, double* grad) {
  if (!b || !x || ((H || grad) && !lambda)) return bfail(NNC_ERR_ARG, "nnc_batch_eval: bad arguments");
  BCK(cudaSetDevice(b->device));
  cudaStream_t st = b->stream;
  const size_t nl = (size_t)b->K * b->n_out;
  std::memcpy(b->h_stage, x, sizeof(double) * b->n_sum);
  BCK(cudaMemcpyAsync(b->x_in, b->h_stage, sizeof(double) * b->n_sum, cudaMemcpyHostToDevice, st));
  if (lambda) {
    std::memcpy(b->h_stage + b->n_sum, lambda, sizeof(double) * nl);
    BCK(cudaMemcpyAsync(b->lam_in, b->h_stage + b->n_sum, sizeof(double) * nl, cudaMemcpyHostToDevice, st));
  }
  int r = nnc_batch_eval_dev(b, b->x_in, lambda ? b->lam_in : nullptr, y ? b->y_out : nullptr,
                             J ? b->J_out : nullptr, H ? b->H_out : nullptr, grad ? b->g_out : nullptr, st);
  if (r) return r;
  if (y) BCK(cudaMemcpyAsync(y, b->y_out, sizeof(double) * nl, cudaMemcpyDeviceToHost, st));
  if (J) BCK(cudaMemcpyAsync(J, b->J_out, sizeof(double) * b->n_sum * b->n_out, cudaMemcpyDeviceToHost, st));
  if (H) BCK(cudaMemcpyAsync(H, b->H_out, sizeof(double) * b->h_sum, cudaMemcpyDeviceToHost, st));
  if (grad) BCK(cudaMemcpyAsync(grad, b->g_out, sizeof(double) * b->n_sum, cudaMemcpyDeviceToHost, st));
  return sync_check(b, st);
}

int nnc_batch_eval_kkt(nnc_batch* b, const double* x, const double* y, const double* lambda, double* r,
                       double* J, double* H, double* grad) {
  if (!b || !x || (r && !y) || ((H || grad) && !lambda))
    return bfail(NNC_ERR_ARG, "nnc_batch_eval_kkt: bad arguments");
  BCK(cudaSetDevice(b->device));
  cudaStream_t st = b->stream;
  const size_t nl = (size_t)b->K * b->n_out;
  double* hx = b->h_stage;
  double* hy = hx + b->n_sum;
  double* hl = hy + nl;
  std::memcpy(hx, x, sizeof(double) * b->n_sum);
  BCK(cudaMemcpyAsync(b->x_in, hx, sizeof(double) * b->n_sum, cudaMemcpyHostToDevice, st));
  if (r) {
    std::memcpy(hy, y, sizeof(double) * nl);
    BCK(cudaMemcpyAsync(b->y_in, hy, sizeof(double) * nl, cudaMemcpyHostToDevice, st));
  }
  if (lambda) {
    std::memcpy(hl, lambda, sizeof(double) * nl);
    BCK(cudaMemcpyAsync(b->lam_in, hl, sizeof(double) * nl, cudaMemcpyHostToDevice, st));
  }
  // outputs in page-locked memory are written in place by the kernels that form them
  auto direct = [](double* h) { return h ? (double*)pinned_dev_ptr(h) : nullptr; };
  double *r_d = direct(r), *J_d = direct(J), *H_d = direct(H), *g_d = direct(grad);
  int rc = nnc_batch_eval_kkt_dev(b, b->x_in, r ? b->y_in : nullptr, lambda ? b->lam_in : nullptr,
                                  r_d ? r_d : r ? b->r_out : nullptr, J_d ? J_d : J ? b->J_out : nullptr,
                                  H_d ? H_d : H ? b->H_out : nullptr,
                                  g_d ? g_d : grad ? b->g_out : nullptr, st);
  if (rc) return rc;
  if (r && !r_d) BCK(cudaMemcpyAsync(r, b->r_out, sizeof(double) * nl, cudaMemcpyDeviceToHost, st));
  if (J && !J_d)
    BCK(cudaMemcpyAsync(J, b->J_out, sizeof(double) * b->n_sum * b->n_out, cudaMemcpyDeviceToHost, st));
  if (H && !H_d) BCK(cudaMemcpyAsync(H, b->H_out, sizeof(double) * b->h_sum, cudaMemcpyDeviceToHost, st));
  if (grad && !g_d)
    BCK(cudaMemcpyAsync(grad, b->g_out, sizeof(double) * b->n_sum, cudaMemcpyDeviceToHost, st));
  return sync_check(b, st);
}

int nnc_batch_residual(nnc_batch* b, const double* x, const double* y, double* r) {
  if (!b || !x || !y || !r) return bfail(NNC_ERR_ARG, "nnc_batch_residual: bad arguments");
  BCK(cudaSetDevice(b->device));
  cudaStream_t st = b->stream;
  const size_t nl = (size_t)b->K * b->n_out;
  std::memcpy(b->h_stage, x, sizeof(double) * b->n_sum);
  std::memcpy(b->h_stage + b->n_sum, y, sizeof(double) * nl);
  BCK(cudaMemcpyAsync(b->x_in, b->h_stage, sizeof(double) * b->n_sum, cudaMemcpyHostToDevice, st));
  BCK(cudaMemcpyAsync(b->y_in, b->h_stage + b->n_sum, sizeof(double) * nl, cudaMemcpyHostToDevice, st));
  int rc = batch_residual(b, b->x_in, b->y_in, b->r_out, st);
  if (rc) return rc;
  BCK(cudaMemcpyAsync(r, b->r_out, sizeof(double) * nl, cudaMemcpyDeviceToHost, st));
  return sync_check(b, st);   // the value pass's bounded waits too
}

}  // extern "C"

namespace nnc {
// nnc_eval_batched's grouped path: reuse (or build) the cached batch for these nets and run it
// on host arrays.  Returns NNC_ERR_UNSUPPORTED when the nets cannot be grouped.
int eval_batched_grouped(nnc_net* const* nets, int K, const double* const* x,
                         const double* const* lambda, double* const* y, double* const* J,
                         double* const* H, unsigned what) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  bool same = g_cache && g_cache->K == K;
  for (int k = 0; same && k < K; ++k) same = g_cache->members[k] == nets[k];
  if (!same) {
    if (g_cache) nnc_batch_free(g_cache);
    g_cache = nullptr;
    nnc_batch* b = nullptr;
    int r = nnc_batch_create(&b, nets, K, nullptr);
    if (r != NNC_OK) return r;
    g_cache = b;
  }
  nnc_batch* b = g_cache;
  const int no = b->n_out;
  std::vector<double> xc(b->n_sum), lc((size_t)K * no), yc((size_t)K * no), Jc((size_t)b->n_sum * no),
      Hc(what & NNC_WANT_H ? b->h_sum : 0);
  for (int k = 0; k < K; ++k) {
    std::memcpy(xc.data() + b->boff[k], x[k], sizeof(double) * b->n_k[k]);
    if (what & NNC_WANT_H) std::memcpy(lc.data() + (size_t)k * no, lambda[k], sizeof(double) * no);
  }
  int r = nnc_batch_eval(b, xc.data(), (what & NNC_WANT_H) ? lc.data() : nullptr,
                         (what & NNC_WANT_Y) ? yc.data() : nullptr, (what & NNC_WANT_J) ? Jc.data() : nullptr,
                         (what & NNC_WANT_H) ? Hc.data() : nullptr, nullptr);
  if (r != NNC_OK) return r;
  for (int k = 0; k < K; ++k) {
    if (what & NNC_WANT_Y) std::memcpy(y[k], yc.data() + (size_t)k * no, sizeof(double) * no);
    if (what & NNC_WANT_J)
      std::memcpy(J[k], Jc.data() + (size_t)b->boff[k] * no, sizeof(double) * no * b->n_k[k]);
    if (what & NNC_WANT_H)
      std::memcpy(H[k], Hc.data() + b->hoff[k], sizeof(double) * b->n_k[k] * b->n_k[k]);
  }
  return NNC_OK;
}
}  // namespace nnc
