// Streaming matrix-vector products of the value passes (Eq. 3): z = W a + b, a' = sigma(z).
//
// The weights are read once per pass and dominate the traffic.  A CTA owns a contiguous block of
// rows; its NW warps split every row into column slices of at most 4 KB (a whole number of
// 512-byte groups), and each warp streams its slice of successive rows through its own ring of
// shared-memory stages with bulk asynchronous copies (cp.async.bulk completing on an mbarrier),
// refilling a stage as soon as it has read it.  The warp's slice of the activation vector is
// held in registers for the whole kernel, so the inner loop is shared-memory loads and FMAs only.
// Per row each warp leaves one partial sum in shared memory; after every batch of up to 32 rows
// the CTA synchronises and warp 0 adds the partials (in a fixed order), applies the bias and the
// activation and writes the outputs.
//
// Launches use programmatic dependent launch: a layer's kernel issues its first weight copies
// (which depend on nothing computed in the step), then waits for the previous kernel's
// activations (griddepcontrol.wait), so one layer's ramp-up overlaps the previous layer's tail.
//
// Arithmetic: double-float weights and activations ((hi, lo) FP32 pairs, 8 bytes per weight, 16
// bytes of weights meet 16 bytes of activations), about 48 significant bits, with FP32 operations
// only (GB300 runs FP64 at a small fraction of its FP32 rate).  This is the value pass of every
// non-FP64 form: its sigma, sigma' and sigma'' feed the derivative sweeps and its output gives the
// FP64-accurate residual y - NN(x).
#include <algorithm>

#include "async.cuh"
#include "kernels.cuh"

namespace nnc {
namespace {

using namespace async;

constexpr int kSvGroup = 512;      // bytes of a row one warp instruction covers (32 lanes x 16 B)
constexpr int kSvMaxGroups = 8;    // groups per warp slice (4 KB)
constexpr int kSvMaxWarps = 16;
constexpr int kSvMaxStages = 4;
constexpr int kSvBatch = 32;       // rows between CTA-wide reductions
constexpr int kSvSlice = kSvMaxGroups * kSvGroup;

struct SvArgs {
  const void* W;        // [m][ldw] (hi, lo) float2 weights
  int ldw;              // elements per row, a multiple of 128 (padding columns are zero)
  int m;                // rows
  const double* bias;   // [m] or NULL
  const void* a_in;     // [ldw] (hi, lo) float2 activations, padding zero
  int act;
  double* a_out;        // [m] sigma(z), or NULL
  float2* a_df;         // [m] (hi, lo) copy of sigma(z) (input of the next DF layer), or NULL
  double* s1;           // [m] sigma'(z) or NULL
  double* s2;           // [m] sigma''(z) or NULL
  int* err;             // device error word (bounded waits)
  int nw;               // warps per CTA (= blockDim.x / 32)
  int gw;               // 512-byte groups per warp slice (<= kSvMaxGroups)
  int ns;               // ring stages per warp (<= kSvMaxStages)
  int rows_per_cta;
  // grouped rows (a batch of networks stacked by rows): rows [g group_rows, (g + 1) group_rows)
  // belong to group g, whose first group_m are valid and whose activation vector starts at
  // a_in + g ld_in (float2 elements); group_rows = 0: one vector for all rows
  int group_rows, group_m, ld_in;
  // grouped rows: valid columns of each group's weights (the rest of a row is zero padding and is
  // neither copied nor multiplied), or NULL (every row's ldw columns)
  const int* gcols;
};

__global__ void __launch_bounds__(kSvMaxWarps * 32) k_gemv_stream(const SvArgs p) {
  extern __shared__ __align__(128) unsigned char sv_smem[];
  __shared__ __align__(8) uint64_t full[kSvMaxWarps][kSvMaxStages];
  __shared__ double part[kSvBatch][kSvMaxWarps];
  __shared__ volatile int abort_flag;
  constexpr int EB = 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row_bytes = p.ldw * EB;
  const int groups = row_bytes / kSvGroup;
  const int g0 = warp * p.gw;
  const int r0 = blockIdx.x * p.rows_per_cta;
  int nrows = max(0, min(p.m, r0 + p.rows_per_cta) - r0);
  const int grp = p.group_rows ? r0 / p.group_rows : 0;   // rows_per_cta divides group_rows
  if (p.group_rows) nrows = max(0, min(nrows, p.group_m - (r0 - grp * p.group_rows)));
  // a group's rows end at its last 512-byte group holding a valid column
  const int groups_used =
      (p.group_rows && p.gcols) ? min(groups, (p.gcols[grp] * EB + kSvGroup - 1) / kSvGroup) : groups;
  const int ng = max(0, min(groups_used, g0 + p.gw) - g0);  // this warp's groups
  const int slice_bytes = ng * kSvGroup;
  unsigned char* ring = sv_smem + warp * (p.ns * kSvSlice);
  if (p.ns < 1 || p.ns > kSvMaxStages || p.nw * 32 != (int)blockDim.x || p.nw > kSvMaxWarps ||
      p.gw < 1 || p.gw > kSvMaxGroups)
    return;  // the launcher never builds such a configuration

  if (threadIdx.x == 0) abort_flag = 0;
  if (lane == 0) {
    for (int s = 0; s < p.ns; ++s) mbar_init(smem_u32(&full[warp][s]), 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto issue = [&](int i) {  // this warp's slice of row r0 + i into stage i % ns
    const int s = i % p.ns;
    const uint32_t bar = smem_u32(&full[warp][s]);
    mbar_expect_tx(bar, (uint32_t)slice_bytes);
    bulk_g2s(smem_u32(ring + s * kSvSlice),
             (const unsigned char*)p.W + (size_t)(r0 + i) * row_bytes + (size_t)g0 * kSvGroup,
             (uint32_t)slice_bytes, bar);
  };
  const int total = ng > 0 ? nrows : 0;
  int issued = 0;  // meaningful on lane 0 only
  if (lane == 0)
    for (; issued < total && issued < p.ns; ++issued) issue(issued);

  griddep_wait();    // the previous layer's activations are complete and visible
  griddep_launch();  // the next kernel in the stream may start issuing its own copies

  float4 act[kSvMaxGroups];
  const float4* a4 = reinterpret_cast<const float4*>(p.a_in) + (size_t)grp * (p.ld_in / 2) +
                     (size_t)g0 * 32 + lane;
#pragma unroll
  for (int g = 0; g < kSvMaxGroups; ++g)
    act[g] = g < ng ? __ldg(a4 + g * 32) : make_float4(0.f, 0.f, 0.f, 0.f);

  int i = 0;  // rows consumed by this warp
  for (int b0 = 0; b0 < nrows; b0 += kSvBatch) {
    const int nb = min(kSvBatch, nrows - b0);
    for (int r = 0; r < nb && !abort_flag; ++r) {
      float q0 = 0.f, q1 = 0.f, q2 = 0.f, q3 = 0.f;
      if (ng > 0) {
        const int s = i % p.ns;
        bool ok = mbar_wait(smem_u32(&full[warp][s]), (uint32_t)(i / p.ns) & 1u, p.err, 21);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
          abort_flag = 1;
          break;
        }
        const float4* w4 = reinterpret_cast<const float4*>(ring + s * kSvSlice) + lane;
#pragma unroll
        for (int g = 0; g < kSvMaxGroups; ++g) {
          if (g < ng) {
            const float4 w = w4[g * 32];  // two weights (hi, lo) meet two activations
            df_acc(q0, q1, w.x, w.y, act[g].x, act[g].y);
            df_acc(q2, q3, w.z, w.w, act[g].z, act[g].w);
          }
        }
        __syncwarp();
        ++i;
        if (lane == 0 && issued < total) {  // refill the stage just read
          fence_proxy_async();
          issue(issued);
          ++issued;
        }
      }
      // warp reduction of the two double-float sums (q0, q1), (q2, q3) in FP32 operations
      df_add(q0, q1, q2, q3);
      warp_sum_df(q0, q1);
      if (lane == 0) part[r][warp] = (double)q0 + (double)q1;
    }
    __syncthreads();
    if (abort_flag) break;
    if (warp == 0 && lane < nb) {
      const int row = r0 + b0 + lane;
      double z = p.bias ? p.bias[row] : 0.0;
      for (int w = 0; w < p.nw; ++w) z += part[lane][w];
      double a, d1, d2;
      act_eval(p.act, z, a, d1, d2);
      if (p.a_out) p.a_out[row] = a;
      if (p.a_df) {
        const float ah = (float)a;
        p.a_df[row] = make_float2(ah, (float)(a - (double)ah));
      }
      if (p.s1) p.s1[row] = d1;
      if (p.s2) p.s2[row] = d2;
    }
    __syncthreads();
  }
  if (abort_flag && lane == 0) {
    // a wait ran out: let this warp's copies still in flight land (short bound) before the
    // stages go away
    for (int k = i; k < issued; ++k)
      mbar_wait(smem_u32(&full[warp][k % p.ns]), (uint32_t)(k / p.ns) & 1u, p.err, 22,
                kWaitCycles / 8);
  }
}

cudaError_t launch_sv(SvArgs a, int sm_count, cudaStream_t st) {
  constexpr int EB = 8;
  const int groups = a.ldw * EB / kSvGroup;
  a.nw = (groups + kSvMaxGroups - 1) / kSvMaxGroups;
  if (a.nw < 1 || a.nw > kSvMaxWarps || a.m < 1) return cudaErrorInvalidValue;
  a.gw = (groups + a.nw - 1) / a.nw;
  // Two stages per warp suffice; what brings the stream to HBM speed is enough warps per SM
  // (3-4 CTAs): measured at 6.3 TB/s on a 1 GB matrix (6.6 TB/s with FP32 weights).  (Four stages
  // for one-warp CTAs, the 2 KB rows of a batch's first layer, measured slower: 216 against 154 us.)
  a.ns = 2;
  const int smem = a.nw * a.ns * kSvSlice;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_gemv_stream,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSvMaxWarps * 3 * kSvSlice);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_gemv_stream, cudaFuncAttributePreferredSharedMemoryCarveout,
                             100);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (smem > kSvMaxWarps * 3 * kSvSlice || a.ns > kSvMaxStages || a.gw > kSvMaxGroups)
    return cudaErrorInvalidValue;
  // CTAs per SM from shared memory (about 200 KB usable with the static part) and warps: layers
  // with short rows (few warps per CTA) get more CTAs per SM, so more copies are in flight
  const int per_sm = std::max(1, std::min({12, 200 * 1024 / smem, 48 / a.nw}));
  int used;
  if (a.group_rows > 0) {
    // grouped: rows per CTA a power of two dividing group_rows (a multiple of 128), chosen so
    // that the CTAs holding valid rows fill whole waves of resident CTAs best (larger on ties)
    const int groups = a.m / a.group_rows;
    const long long slots = (long long)per_sm * sm_count;
    int best = a.group_rows;
    double best_eff = -1.0;
    for (int p2 = a.group_rows; p2 >= 8; p2 /= 2) {
      const long long ctas = (long long)groups * ((a.group_m + p2 - 1) / p2);
      const long long waves = (ctas + slots - 1) / slots;
      const double eff = (double)ctas / (double)(waves * slots);
      if (eff > best_eff + 1e-9) {
        best_eff = eff;
        best = p2;
      }
    }
    a.rows_per_cta = best;
    used = a.m / best;
  } else {
    const int grid = std::max(1, std::min(a.m, per_sm * sm_count));
    a.rows_per_cta = (a.m + grid - 1) / grid;
    used = (a.m + a.rows_per_cta - 1) / a.rows_per_cta;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(used);
  cfg.blockDim = dim3(a.nw * 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_gemv_stream, a);
  note_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

// Self-test of the bounded wait: an mbarrier that nothing arrives on, waited for `limit` cycles;
// the wait must give up and record `code` in *err.
__global__ void k_wait_selftest(int* err, long long limit, int code) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(smem_u32(&bar), 0, err, code, limit);
  __syncthreads();
}

}  // namespace

cudaError_t launch_wait_selftest_stream(int* err, long long limit, int code, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(err, limit, code);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gemv_stream_df(const void* W2, int ldw, int m, const double* b, const void* a_in2,
                                  int act, double* a_out, void* a_df, double* s1, double* s2,
                                  int* err, int sm_count, cudaStream_t st) {
  if (ldw % kPad) return cudaErrorInvalidValue;
  SvArgs a{W2, ldw, m, b, a_in2, act, a_out, (float2*)a_df, s1, s2, err, 0, 0, 0, 0, 0, 0, 0,
           nullptr};
  return launch_sv(a, sm_count, st);
}

cudaError_t launch_gemv_stream_df_grouped(const void* W2, int ldw, int groups, int mp, int m,
                                          const double* b, const void* a_in2, int ld_in, int act,
                                          double* a_out, void* a_df, double* s1, double* s2,
                                          int* err, int sm_count, cudaStream_t st, const int* gcols) {
  if (ldw % kPad || mp % kPad || ld_in % kPad || groups < 1 || m < 1 || m > mp)
    return cudaErrorInvalidValue;
  SvArgs a{W2, ldw, groups * mp, b, a_in2, act, a_out, (float2*)a_df, s1, s2, err, 0, 0, 0, 0,
           mp, m, ld_in, gcols};
  return launch_sv(a, sm_count, st);
}

}  // namespace nnc
