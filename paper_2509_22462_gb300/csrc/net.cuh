// Internal definitions shared by the library's translation units: the per-layer device state
// of a net and the net object behind the opaque nnc_net handle of include/nnc.h.
#pragma once
#include <string>
#include <vector>

#include "kernels.cuh"
#include "tc.cuh"

struct nnc_net;
namespace nnc {
void set_last_error(const std::string& msg);
// Device address of a host buffer in page-locked memory (cudaHostAlloc, cudaHostRegister), which
// kernels read and write directly through unified addressing; NULL for pageable memory.  Host
// calls let the kernels that form an output write such a buffer in place.
void* pinned_dev_ptr(void* host);
void batch_cache_forget(const nnc_net* net);
int eval_batched_grouped(nnc_net* const* nets, int K, const double* const* x,
                         const double* const* lambda, double* const* y, double* const* J,
                         double* const* H, unsigned what);
}

struct LayerDev {
  int m = 0, k = 0, act = 0, mp = 0, kp = 0;
  double* W64 = nullptr;          // [mp][kp], zero padded
  float* W32 = nullptr;           // [mp][kp]
  __nv_bfloat16* Whi = nullptr;   // [mp][kp]
  __nv_bfloat16* Wlo = nullptr;   // [mp][kp]
  unsigned char* W8 = nullptr;    // [mp][kp] e4m3 (FP8 form)
  __nv_bfloat16* WThi = nullptr;  // W_l^T [kp][mp] BF16 hi (tensor-core reverse sweep)
  __nv_bfloat16* WTlo = nullptr;  // W_l^T [kp][mp] BF16 second part
  __nv_bfloat16* WTp2 = nullptr;  // W_l^T [kp][mp] BF16 third part
  nnc::TcPlan plan_rev;           // tensor-core plan of this layer's reverse step
  float* w8s = nullptr;           // [mp] per-row scale of W8
  double* b = nullptr;            // [mp]
  double* a = nullptr;            // a_l [mp]
  double* s1 = nullptr;           // sigma_l'(z_l) [mp]
  double* s2 = nullptr;           // sigma_l''(z_l) [mp]
  double* c = nullptr;            // sigma_l''(z_l) * abar_l [mp]
  float* c_f = nullptr;           // FP32 copy of c for the tensor-core epilogue
  double* ra = nullptr;           // FP64-residual pass activations [mp]
  void* ra2 = nullptr;            // their double-float (hi, lo) pairs [mp] (float2)
  void* W2 = nullptr;             // double-float (hi, lo) pairs of W [mp][kp] (float2)
  void* a2 = nullptr;             // double-float (hi, lo) pairs of a_l [mp] (float2)
  nnc::TcPlan plan_tan;                // tensor-core plan of this layer's tangent GEMM
  CUtensorMap rev_map;            // TMA map of W32 for the streaming reverse layer
  nnc::RevGeom rev_geom;          // its launch geometry
  int rev_cnt_off = 0;            // offset of its strip counters in nnc_net::rev_cnt
  int zy_off = -1;                // column offset of this layer's Zdot / Ydot block (-1: none)
};

struct nnc_net {
  int L = 0, n_in = 0, n_out = 0, prec = 0, n_in_pad = 0, mp_max = 0, S_max = 0;
  std::vector<LayerDev> layers;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // tensor-core forms: the reverse sweep runs on side_stream next to the tangent chain (which no
  // longer needs its c_l); ev_fork / ev_join order it after the value pass and before the
  // symmetric product.  cK holds c_l of every curvature layer at its Zdot column offset.
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  float* cK = nullptr;
  int device = 0, sm_count = 0;
  std::vector<void*> allocs;
  double* x = nullptr;       // a_0 [n_in_pad]
  void* x2 = nullptr;        // double-float (hi, lo) pairs of a_0 [n_in_pad] (float2)
  double* xin = nullptr;     // host-call inputs: x [n_in_pad] | lambda | y, one block
  double* xr = nullptr;      // input of the FP64 residual pass [n_in_pad] (its own copy, so that
                             // a residual may run on another stream next to an evaluation)
  void* xr2 = nullptr;       // its double-float pairs (float2)
  double* yres = nullptr;    // y for the residual [n_out] (in the xin block)
  double* lam = nullptr;     // lambda [n_out] (in the xin block)
  double* ydev = nullptr;    // [n_out] staging
  double* rdev = nullptr;    // [n_out]
  double* Zbar[2] = {nullptr, nullptr};
  double* part = nullptr;
  double* Jdev = nullptr;    // [n_out][n_in]
  double* gdev = nullptr;    // [n_in]
  double* Hdev = nullptr;    // [n_in][n_in]
  void* At[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [ping-pong][hi, lo]
  void* Zt[2] = {nullptr, nullptr};  // [hi, lo]: Zdot_l^T of all curved layers, n x K_total
  void* Yt[2] = {nullptr, nullptr};  // [hi, lo]: (c_l * Zdot_l)^T, n x K_total
  int K_total = 0;                   // sum of mp_l over layers with sigma'' != 0 (+ 128: softmax)
  float* W1T = nullptr;              // tensor-core forms: FP32 W_1^T [n_in][mp_1] for Adot_1
  // persistent chain of tangent GEMMs (BF16 and split-BF16x3 forms; k_tc_chain): plans of layers
  // 1 .. chain_nl with one N tile, the chain's arrival counters, and whether evaluations use it
  // (chosen by the autotuner or nnc_tune_set)
  std::vector<nnc::TcPlan> chain_plans;
  int chain_nl = 0;
  unsigned* chain_cnt = nullptr;
  bool use_chain = false;
  bool softmax = false;              // softmax output layer
  int ext_off = -1;                  // its two rank-two curvature columns in the Zdot / Ydot arrays
  void* Zb[2][3] = {};  // reverse seeds^T [48][mp_max], ping-pong x three BF16 parts
  float* Prev = nullptr;             // split partials of the tensor-core reverse step
  bool tc_rev = false;               // reverse sweep on the tensor cores
  bool rev_stream = false;           // streaming FP32 reverse sweep (k_rev.cu)
  float* Zf[2] = {nullptr, nullptr}; // its FP32 seeds [mp_max][16], ping-pong
  int* rev_cnt = nullptr;            // its per-strip arrival counters
  unsigned char* A8 = nullptr;       // FP8 form: e4m3 copy of the current tangent operand
  float* tsc = nullptr;              // FP8 form: its per-row (per-tangent) scales
  nnc::TcPlan plan_syrk;                  // tensor-core plan of the one symmetric product
  void* Hp = nullptr;        // split partial sums of H (double for CUDA-core forms, float for TC)
  int h_splits = 1;
  bool hp_f32 = false;
  int* dev_err = nullptr;    // device error word of bounded waits
  double* h_stage = nullptr; // pinned host staging
  size_t h_stage_elems = 0;
  size_t bytes = 0;
  // optional per-kernel-kind CUDA-event timing (nnc_profile)
  unsigned prof_mask = 0;   // kernel kinds whose launches are bracketed by events
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<int> ev_kind;
  std::vector<int> ev_weight;   // launches each recorded event pair stands for
};

