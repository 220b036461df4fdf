// Reverse sweep of the non-FP64 forms (the adjoint recursion behind the Jacobian and Eq. 6): per
// layer l, Abar_{l-1} = W_l^T Zbar_l for up to 16 seed columns (n_out Jacobian seeds and the
// lambda column), with FP32 weights, FP32 products and FP32 sums (about 24 significant bits).
//
// The layer reads each FP32 weight once, so the kernel streams.  A CTA owns a strip of 128
// columns and a block of rows.  Each of its eight warps streams 8-row x 128-column boxes (4 KB,
// 2-D TMA) through a private two-stage ring and refills a stage as soon as it has read it (no
// CTA-wide hand-off); a lane takes four adjacent columns (one 16-byte shared load) times the row's
// seeds (broadcast loads): 4 x SM FMAs per 16 bytes of weights, issued as packed FP32 pairs
// (fma.rn.f32x2).  Measured on a 4096 x 4096 layer: 16 us (4.1 TB/s), against 19 us with four
// warps and scalar FMAs.  The seeds of the CTA's rows (FP32, SM per row) arrive with one bulk
// copy.
//
// Reduction over rows without a serial tail: the CTAs of one strip's row blocks form thread-block
// clusters of up to 8.  Each CTA adds its warps' partials in shared memory; after a cluster barrier
// every CTA adds a 1/8 slice of the strip's 128 x SM sums over the cluster's CTAs through
// distributed shared memory, in rank order (deterministic).  When a strip spans several clusters,
// the cluster sums go to global memory and the last CTA of the strip (an arrival counter) adds
// them.  The layer boundary is applied to the final sums: the next seeds
// Zbar_{l-1} = sigma'_{l-1} * Abar_{l-1} and c_{l-1} = sigma''_{l-1} * Abar_{l-1}[:, lambda], or on
// the first layer J and the gradient lambda^T J.
//
// Launched with programmatic dependent launch: the weight copies start while the previous layer is
// finishing; griddepcontrol.wait comes before the seeds are copied.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "async.cuh"
#include "kernels.cuh"

namespace nnc {
namespace {

using namespace async;

constexpr int kRvCols = 128;
constexpr int kRvBoxRows = 8;
constexpr int kRvBoxBytes = kRvCols * kRvBoxRows * 4;   // 4 KB
constexpr int kRvWarps = 8;
constexpr int kRvThreads = kRvWarps * 32;
constexpr int kRvStages = 2;
constexpr int kRvRing = kRvWarps * kRvStages * kRvBoxBytes;   // 64 KB
static_assert(kRvWarps * kRvCols * 16 * 4 <= kRvRing, "the cross-warp sums fit the ring");
constexpr int kRvMaxRows = 512;
constexpr int kRvMaxCluster = 8;

// Rows per CTA are capped so that the seed block stays within 24 KB.
constexpr int rv_max_rows(int sm) { return 6144 / sm < kRvMaxRows ? 6144 / sm / 32 * 32 : kRvMaxRows; }
constexpr int rv_smem(int sm, int rows) { return kRvRing + rows * sm * 4 + kRvCols * sm * 4; }

struct RvArgs {
  const float* Zf;      // [m][SM] seeds of the layer's rows (columns >= S zero)
  int m;                // rows with weights (the layer's outputs)
  int S;                // seed columns, <= SM
  int rows_per_cta;     // multiple of 32
  int kp;               // columns (a multiple of 128)
  int cl;               // cluster size along the row blocks (gridDim.y is a multiple)
  float* part;          // [gridDim.y / cl][kp][SM] cluster sums (strips spanning several clusters)
  int* counters;        // [kp / 128] arrival counters (zero between launches)
  // layer boundary
  int nJ, lam_col, kvalid;
  const double* s1n;    // sigma' of the layer below ([kp]), or NULL on the first layer
  const double* s2n;    // sigma'' of the layer below
  float* Zf_out;        // [kp][SM] next seeds
  double* c_out;        // [kp] c of the layer below (lambda column), or NULL
  float* c_f_out;       // its FP32 copy, or NULL
  double* J_out;        // first layer: J [nJ][kvalid], or NULL
  double* g_out;        // first layer: gradient [kvalid], or NULL
  int* err;
};

template <int SM>
__device__ __forceinline__ void rv_boundary(const RvArgs& a, int kk, int s, float v) {
  if (a.s1n) {
    a.Zf_out[(size_t)kk * SM + s] = s < a.S ? (float)(a.s1n[kk] * (double)v) : 0.f;
    if (s == a.lam_col) {
      const double cv = a.s2n[kk] * (double)v;
      if (a.c_out) a.c_out[kk] = cv;
      if (a.c_f_out) a.c_f_out[kk] = (float)cv;
    }
  } else if (kk < a.kvalid && s < a.S) {
    if (a.J_out && s < a.nJ) a.J_out[(size_t)s * a.kvalid + kk] = (double)v;
    if (a.g_out && s == a.lam_col) a.g_out[kk] = (double)v;
  }
}

template <int SM>
__global__ void __launch_bounds__(kRvThreads, SM <= 12 ? 2 : 1) k_rev_stream(const __grid_constant__ CUtensorMap tw,
                                                           const RvArgs a) {
  static_assert(SM % 4 == 0, "seed rows are read as float4");
  extern __shared__ __align__(128) unsigned char rv_smem_buf[];
  float* ring = reinterpret_cast<float*>(rv_smem_buf);
  float* zs = reinterpret_cast<float*>(rv_smem_buf + kRvRing);
  float* cpart = zs + (size_t)a.rows_per_cta * SM;   // [128][SM] this CTA's sums
  __shared__ __align__(8) uint64_t full[kRvWarps][kRvStages], zbar;
  __shared__ volatile int abort_flag;
  __shared__ int last_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k0 = blockIdx.x * kRvCols;
  const int r0 = blockIdx.y * a.rows_per_cta;
  const int nrows = max(0, min(a.m, r0 + a.rows_per_cta) - r0);   // 0 for padding CTAs
  const int nb = (nrows + kRvBoxRows - 1) / kRvBoxRows;           // 8-row boxes of the block
  const int nbw = warp < nb ? (nb - 1 - warp) / kRvWarps + 1 : 0;  // this warp's boxes
  float* my_ring = ring + warp * (kRvStages * kRvBoxBytes / 4);

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int w = 0; w < kRvWarps; ++w)
      for (int s = 0; s < kRvStages; ++s) mbar_init(smem_u32(&full[w][s]), 1);
    mbar_init(smem_u32(&zbar), 1);
    fence_mbar_init();
  }
  __syncthreads();
  // box j of this warp = box (warp + 8 j) of the block, rows r0 + 8 (warp + 8 j) ..
  auto issue = [&](int j) {
    const int s = j % kRvStages;
    mbar_expect_tx(smem_u32(&full[warp][s]), kRvBoxBytes);
    tma_load_2d(smem_u32(my_ring + s * (kRvBoxBytes / 4)), &tw, smem_u32(&full[warp][s]), k0,
                r0 + (warp + kRvWarps * j) * kRvBoxRows);
  };
  int issued = 0;  // lane 0 of each warp
  if (lane == 0)
    for (; issued < nbw && issued < kRvStages; ++issued) issue(issued);

  griddep_wait();  // the seeds of this layer are complete and visible
  griddep_launch();
  if (threadIdx.x == 0 && nrows > 0) {
    const uint32_t zb = (uint32_t)(nrows * SM * 4);
    mbar_expect_tx(smem_u32(&zbar), zb);
    bulk_g2s(smem_u32(zs), a.Zf + (size_t)r0 * SM, zb, smem_u32(&zbar));
  }
  // rows of the last box past the block's end meet zero seeds (their weights are zero too)
  for (int idx = nrows * SM + threadIdx.x; idx < nb * kRvBoxRows * SM; idx += kRvThreads)
    zs[idx] = 0.f;
  bool ok = nrows == 0 || mbar_wait_abort(smem_u32(&zbar), 0u, a.err, 34, &abort_flag);
  __syncthreads();
  ok = ok && !abort_flag;

  uint64_t acc2[4][SM / 2];   // packed FP32 pairs (seeds 2p, 2p + 1)
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int p = 0; p < SM / 2; ++p) acc2[v][p] = 0ull;
  int j = 0;
  for (; ok && j < nbw; ++j) {
    const int s = j % kRvStages;
    bool got = mbar_wait_abort(smem_u32(&full[warp][s]), (uint32_t)(j / kRvStages) & 1u, a.err, 32,
                               &abort_flag);
    got = __all_sync(0xffffffffu, got);
    if (!got) break;
    const float* box = my_ring + s * (kRvBoxBytes / 4);
    const float* zrow = zs + (size_t)(warp + kRvWarps * j) * kRvBoxRows * SM;
#pragma unroll 2
    for (int rr = 0; rr < kRvBoxRows; ++rr) {
      const float4 w = *reinterpret_cast<const float4*>(box + rr * kRvCols + lane * 4);
      const ulonglong2* z4 = reinterpret_cast<const ulonglong2*>(zrow + rr * SM);
      // packed FP32 FMAs (fma.rn.f32x2): one instruction updates two seeds of one column
      uint64_t wp[4];
      asm("mov.b64 %0, {%1, %1};" : "=l"(wp[0]) : "f"(w.x));
      asm("mov.b64 %0, {%1, %1};" : "=l"(wp[1]) : "f"(w.y));
      asm("mov.b64 %0, {%1, %1};" : "=l"(wp[2]) : "f"(w.z));
      asm("mov.b64 %0, {%1, %1};" : "=l"(wp[3]) : "f"(w.w));
#pragma unroll
      for (int q = 0; q < SM / 4; ++q) {
        const ulonglong2 z = z4[q];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc2[v][2 * q]) : "l"(wp[v]), "l"(z.x));
          asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc2[v][2 * q + 1]) : "l"(wp[v]), "l"(z.y));
        }
      }
    }
    __syncwarp();
    if (lane == 0 && issued < nbw) {  // refill the stage just read
      fence_proxy_async();
      issue(issued);
      ++issued;
    }
  }
  if (lane == 0) {
    // copies issued but not consumed (only after a wait ran out): let them land first
    for (int k = std::max(j, issued - kRvStages); k < issued; ++k)
      mbar_wait(smem_u32(&full[warp][k % kRvStages]), (uint32_t)(k / kRvStages) & 1u, a.err, 33,
                kWaitCycles / 8);
  }
  __syncthreads();  // every box consumed: the ring holds the warps' partials [warp][col][SM]
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int p = 0; p < SM / 2; ++p)
      *reinterpret_cast<uint64_t*>(ring + (warp * kRvCols + lane * 4 + v) * SM + 2 * p) = acc2[v][p];
  __syncthreads();
  for (int idx = threadIdx.x; idx < kRvCols * SM; idx += kRvThreads) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < kRvWarps; ++w) t += ring[w * kRvCols * SM + idx];
    cpart[idx] = t;
  }

  // cluster reduction: rank r adds slice r of the 128 x SM sums over the cluster's CTAs
  cluster_sync();
  const int cl = a.cl;
  const int rank = (int)cluster_rank();
  const int per = (kRvCols * SM + cl - 1) / cl;
  const int i0 = rank * per, i1 = min(kRvCols * SM, i0 + per);
  const int n_cl = gridDim.y / cl;
  const uint32_t cbase = smem_u32(cpart);
  for (int idx = i0 + threadIdx.x; idx < i1; idx += kRvThreads) {
    float v = 0.f;
    for (int q = 0; q < cl; ++q) v += ld_dsmem_f32(cbase + idx * 4, (uint32_t)q);
    if (n_cl == 1)
      rv_boundary<SM>(a, k0 + idx / SM, idx % SM, v);
    else
      a.part[((size_t)(blockIdx.y / cl) * a.kp + k0) * SM + idx] = v;
  }
  cluster_sync();  // no CTA leaves while another still reads its shared memory
  if (n_cl == 1) return;
  // several clusters per strip: the last CTA to arrive adds the cluster sums
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last_sh = atomicAdd(&a.counters[blockIdx.x], 1) == (int)gridDim.y - 1;
  __syncthreads();
  if (!last_sh) return;
  __threadfence();
  for (int idx = threadIdx.x; idx < kRvCols * SM; idx += kRvThreads) {
    float v = 0.f;
    for (int c = 0; c < n_cl; ++c) v += __ldcg(a.part + ((size_t)c * a.kp + k0) * SM + idx);
    rv_boundary<SM>(a, k0 + idx / SM, idx % SM, v);
  }
  if (threadIdx.x == 0) a.counters[blockIdx.x] = 0;  // ready for the next launch
}

// Output-layer seeds for the streaming sweep (out_seed): Zf[i][s] = zbar_L[i][s] in FP32 with SM
// columns per row (zero past S); c_L of the lambda column.  p: softmax probabilities or NULL.
__global__ void k_rev_seed_f(int m, int S, int SM, int nJ, int lam_col, const double* __restrict__ s1,
                             const double* __restrict__ s2, const double* __restrict__ lam,
                             const double* __restrict__ p, float* __restrict__ Zf,
                             double* __restrict__ c_out, float* __restrict__ c_f) {
  griddep_launch();
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * SM) return;
  const int i = idx / SM, s = idx % SM;
  double c = 0.0;
  const double zb = s < S ? out_seed(i, s, m, nJ, lam_col, s1, s2, lam, p, &c) : 0.0;
  Zf[idx] = (float)zb;
  if (s == lam_col) {
    if (c_out) c_out[i] = c;
    if (c_f) c_f[i] = (float)c;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

template <int SM>
cudaError_t launch_rv(const CUtensorMap& map, const RvArgs& a, dim3 grid, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_rev_stream<SM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         rv_smem(SM, rv_max_rows(SM)));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(kRvThreads);
  cfg.dynamicSmemBytes = rv_smem(SM, a.rows_per_cta);
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  at[1].id = cudaLaunchAttributeClusterDimension;
  at[1].val.clusterDim.x = 1;
  at[1].val.clusterDim.y = (unsigned)a.cl;
  at[1].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_rev_stream<SM>, map, a);
  note_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

int rev_stream_sm(int S) { return S <= 4 ? 4 : S <= 8 ? 8 : S <= 12 ? 12 : 16; }

bool rev_stream_map(CUtensorMap* map, const float* W, int mp, int kp) {
  auto enc = encode_fn();
  if (!enc || !W || kp % kRvCols) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)mp};
  cuuint64_t strides[1] = {(cuuint64_t)kp * 4};
  cuuint32_t box[2] = {(cuuint32_t)kRvCols, (cuuint32_t)kRvBoxRows};
  cuuint32_t es[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(W), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

RevGeom rev_stream_geom(int m, int kp, int S, int sm_count) {
  // row blocks per strip: as many as fit next to the strips in one wave of resident CTAs (two per
  // SM, one with more than 12 seeds), a multiple of the cluster size, with whole 32-row groups of
  // at most rv_max_rows rows
  const int strips = kp / kRvCols;
  const int slots = (rev_stream_sm(S) <= 12 ? 2 : 1) * sm_count;
  int splits = std::max(1, std::min(slots / std::max(1, strips), (m + 31) / 32));
  int cl = 1;
  while (cl * 2 <= std::min(kRvMaxCluster, splits)) cl *= 2;
  splits = std::max(cl, splits / cl * cl);
  int rows = (m + splits - 1) / splits;
  rows = std::min(rv_max_rows(rev_stream_sm(S)), (rows + 31) / 32 * 32);
  splits = (m + rows - 1) / rows;
  splits = (splits + cl - 1) / cl * cl;   // padding row blocks hold no rows
  return RevGeom{rows, splits, cl};
}

cudaError_t launch_rev_seed_f(int m, int S, int nJ, int lam_col, const double* s1, const double* s2,
                              const double* lam, const double* p, float* Zf, double* c_out,
                              float* c_f, cudaStream_t st) {
  const int SM = rev_stream_sm(S);
  k_rev_seed_f<<<(m * SM + 255) / 256, 256, 0, st>>>(m, S, SM, nJ, lam_col, s1, s2, lam, p, Zf,
                                                     c_out, c_f);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_rev_stream(const CUtensorMap& map, int m, int kp, const float* Zf, int S,
                              const RevGeom& g, float* part, int* counters, int nJ, int lam_col,
                              int kvalid, const double* s1n, const double* s2n, float* Zf_out,
                              double* c_out, float* c_f_out, double* J_out, double* g_out, int* err,
                              cudaStream_t st) {
  const int sm = rev_stream_sm(S);
  if (S < 1 || S > 16 || kp % kRvCols || g.rows % 32 || g.rows > rv_max_rows(sm) || g.rows < 32 ||
      g.cl < 1 || g.cl > kRvMaxCluster || g.splits % g.cl || (long long)g.rows * g.splits < m)
    return cudaErrorInvalidValue;
  RvArgs a{Zf, m, S, g.rows, kp, g.cl, part, counters, nJ, lam_col, kvalid, s1n, s2n, Zf_out,
           c_out, c_f_out, J_out, g_out, err};
  const dim3 grid(kp / kRvCols, g.splits);
  if (sm == 4) return launch_rv<4>(map, a, grid, st);
  if (sm == 8) return launch_rv<8>(map, a, grid, st);
  if (sm == 12) return launch_rv<12>(map, a, grid, st);
  return launch_rv<16>(map, a, grid, st);
}

}  // namespace nnc
