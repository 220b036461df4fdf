// tcgen05 / TMEM / TMA GEMMs of the BF16 and split-BF16x3 forms (sm_103a).
//
// One CTA computes a 128 x BN tile of D = A B^T (A: M x K, B: N x K, both K-major BF16):
//   warp 0     : TMA producer. 2-D tensor copies (128-byte swizzle) of the A and B k-blocks
//                (64 columns = 128 bytes) into a ring of shared-memory stages, each guarded by
//                a "full" and an "empty" mbarrier.
//   warp 1     : owns the tensor-memory allocation and issues tcgen05.mma (M = 128, N = BN,
//                K = 16 per instruction) from one thread; in the split-BF16x3 form each K step
//                issues Ahi*Bhi, Ahi*Blo and Alo*Bhi into the same FP32 accumulator.
//                tcgen05.commit frees a stage when its MMAs have read it, and signals the
//                epilogue after the last one.
//   warps 2..5 : epilogue. Each warp reads its 32 TMEM lanes (= 32 rows of the tile) with
//                tcgen05.ld and writes the fused outputs; the tangent outputs go through shared
//                memory 16 columns at a time and leave as whole 256-byte row segments
//                (tangent_epilogue_staged).
// Every mbarrier wait is bounded: on expiry the CTA records an error code in *err, stops its
// loops, waits (again bounded) for its own copies and MMAs in flight, frees its tensor memory
// and returns.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>

#include "kernels.cuh"
#include "tc.cuh"

namespace nnc {
namespace {

constexpr int BM = 128;
constexpr int kThreads = 192;
constexpr long long kWaitCycles = 4000000000LL;  // about two seconds at GB300 clocks

struct TcArgs {
  int M, N, K;
  int ntm, ntn, nkb, kb_per_split;
  const double* s1;
  const float* c;
  __nv_bfloat16 *at_hi, *at_lo, *zt_hi, *zt_lo, *yt_hi, *yt_lo;
  int ldo;   // row stride of at_*
  int ldz;   // row stride of zt_* / yt_*
  float* Hp;
  int* err;
  const float* wscale;   // FP8: per-row scale of W_l
  const float* tscale;   // FP8: per-row scale of the tangent operand
  // grouped modes: group g owns A rows [g * a_group_rows, ...) (tangent) and B / output rows
  // starting at g_boff[g]; g_n[g] valid columns; syrk: tile list `work` and H_g at g_hoff[g]
  const int* g_n;
  const int* g_boff;
  const long long* g_hoff;
  const int4* work;
  int a_group_rows;
  long long ldh_split;
  int vec_ok;   // tangent outputs: 16-byte aligned bases and row strides (staged epilogue)
};

// Per-layer description of the persistent tangent chain (k_tc_chain).
struct ChainLayer {
  int ntm, nkb, tile0;   // row blocks, K blocks, index of the layer's first tile
  const double* s1;
  const float* c;
  __nv_bfloat16 *at_hi, *at_lo;   // Adot_l^T (row stride ldo), NULL on the last layer
  int ldo;
  __nv_bfloat16 *zt_hi, *zt_lo, *yt_hi, *yt_lo;   // at the layer's column offset (row stride ldz)
};
struct ChainArgs {
  CUtensorMap ta_hi[kMaxChain], ta_lo[kMaxChain], tb_hi[kMaxChain], tb_lo[kMaxChain];
  ChainLayer L[kMaxChain];
  int nl, N, ntn, ldz, tiles;
  unsigned* cnt;   // [nl][ntn] arrival counters, zero at launch
  int* err;
};

// K-block of one pipeline stage, in elements: 64 (one 128-byte swizzled row) for single BF16; 32
// (64-byte swizzle) for split-BF16x3, whose stages carry four operand tiles, so that five stages
// fit in shared memory instead of two.
// The FP8 form (kind::f8f6f4, e4m3 operands) uses 128-element (128-byte) K blocks.
// MODE_BF16X6: three-way split v ~ p0 + p1 + p2 (about 24 significant bits) with the six products
// p_i q_j, i + j <= 2 -- FP32-level accuracy; used by the bandwidth-bound reverse sweep, whose
// Jacobian feeds the interior-point method's dual residual.
enum { MODE_BF16 = 0, MODE_BF16X3 = 1, MODE_FP8 = 2, MODE_BF16X6 = 3 };
constexpr int bk_for(int mode) {
  return (mode == MODE_BF16X3 || mode == MODE_BF16X6) ? 32 : mode == MODE_FP8 ? 128 : 64;
}

template <int BN, int MODE>
struct Cfg {
  static constexpr bool X6 = MODE == MODE_BF16X6;
  static constexpr bool X3 = MODE == MODE_BF16X3 || X6;   // has a second (lo) part
  static constexpr bool F8 = MODE == MODE_FP8;
  static constexpr int EB = F8 ? 1 : 2;                // bytes per element
  static constexpr int BKE = bk_for(MODE);
  static constexpr int ROWB = BKE * EB;                // bytes of one K-block row
  static constexpr int SWZ = ROWB == 128 ? 2 : 4;      // descriptor layout: SWIZZLE_128B / 64B
  static constexpr int SBO = 8 * ROWB;                 // bytes between 8-row core-matrix groups
  static constexpr int A_BYTES = BM * ROWB;
  static constexpr int B_BYTES = BN * ROWB;
  static constexpr int NPARTS = X6 ? 3 : X3 ? 2 : 1;
  static constexpr int STAGE_BYTES = NPARTS * (A_BYTES + B_BYTES);
  static constexpr int TX_BYTES = STAGE_BYTES;
  static constexpr int SMEM_BUDGET = 227 * 1024 - 2048;
  static constexpr int STAGES_FIT = SMEM_BUDGET / STAGE_BYTES;
  static constexpr int STAGES = STAGES_FIT > 8 ? 8 : STAGES_FIT;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
  static constexpr int TMEM_COLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
  // Instruction descriptor of tcgen05.mma kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
  // (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17, M >> 4 at bit 24.
  // kind::f16: A = B = BF16 (1 at bits 7-9 and 10-12); kind::f8f6f4: A = B = E4M3 (0).
  static constexpr uint32_t IDESC_NO_N =
      (1u << 4) | (F8 ? 0u : (1u << 7) | (1u << 10)) | ((uint32_t)(BM >> 4) << 24);
  static constexpr uint32_t IDESC = IDESC_NO_N | ((uint32_t)(BN >> 3) << 17);
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "UMMA N for M = 128");
  static_assert(B_BYTES % 1024 == 0, "stage parts must stay 1024-byte aligned");
  static_assert(STAGES >= 2, "at least two stages");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity.  Returns false if the CTA aborted or the
// wait ran out (then the error word and the CTA's abort flag are set).
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, int* err, int code,
                                          volatile int* abort_flag, long long limit = kWaitCycles) {
  if (mbar_try(a, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try(a, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) {
      atomicCAS(err, 0, code);
      *abort_flag = 1;
      return false;
    }
  }
}

// Programmatic dependent launch: wait until the preceding kernel of the stream has completed and
// its writes are visible; allow the next one to be scheduled.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t mbar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"((uint64_t)map), "r"(mbar), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor of tcgen05 for a K-major tile written by TMA with 128- or
// 64-byte swizzling: start address >> 4 (bits 0-13), stride between 8-row groups (SBO, >> 4 at
// bit 32), descriptor version 1 (bit 46), layout SWIZZLE_128B (2) or SWIZZLE_64B (4) at bits
// 61-63.  Moving along K inside a swizzled row is done by advancing the start address (32 bytes
// per K = 16).
template <int SWZ, int SBO>
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(SBO >> 4) << 32) | (1ull << 46) |
         ((uint64_t)SWZ << 61);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_f8(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// True on every thread of the four epilogue warps (named barrier 1, 128 threads) only if p is
// true on all of them, so that the barriers of the staged epilogue are reached by all or none.
__device__ __forceinline__ bool epi_all(bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.and.pred q, 1, 128, q;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)p)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

template <bool X3>
__device__ __forceinline__ void put(__nv_bfloat16* hi, __nv_bfloat16* lo, size_t o, float v) {
  if (X3) {
    __nv_bfloat16 h, l;
    split_bf16(v, h, l);
    hi[o] = h;
    lo[o] = l;
  } else {
    hi[o] = __float2bfloat16_rn(v);
  }
}

// Shared memory of the staged tangent epilogue: two buffers of [output][16 columns][128 rows] BF16
// for the outputs at_hi, zt_hi, yt_hi (and at_lo, zt_lo, yt_lo in the split form).
template <bool X3>
constexpr int staged_epi_bytes() {
  return 2 * (X3 ? 6 : 3) * 16 * BM * 2;
}

// Tangent epilogue of one 128-row tile, 16 accumulator columns at a time.  The four epilogue
// warps (thread `row` holds TMEM lane `row`) scale their row's values, write them as BF16 into
// shared memory as [output][column][row] (the pipeline stages are idle once every MMA has
// completed), meet at a named barrier, and store each output's 16 x 128 block as whole 256-byte
// row segments with 16-byte stores.  Stored one element per thread, the same outputs go out as
// 64-byte pieces, two store instructions per element, and their issue, not their bytes, set the
// epilogue's time.  Slices alternate between two buffers, so one barrier per slice suffices: a
// buffer is written again only after every thread has passed the barrier that follows its reads.
// Output row of column n: n, or b_row0 + n for a group of a batch; the column inside the row is
// m0 + row.  Needs args.vec_ok (16-byte aligned outputs and strides).
template <int MODE, int KIND>
__device__ __forceinline__ void tangent_epilogue_staged(const TcArgs& args, uint8_t* smem,
                                                        uint32_t tmem_q, int row, int m0, int n0,
                                                        int n_eff, int n_valid, int b_row0,
                                                        float sm, float cm, float wsc) {
  constexpr bool X3 = MODE == MODE_BF16X3;
  constexpr bool F8 = MODE == MODE_FP8;
  constexpr int NS = X3 ? 6 : 3;                 // output slots
  constexpr int SLOT = 16 * BM;                  // elements of one output's block
  __nv_bfloat16* stg = reinterpret_cast<__nv_bfloat16*>(smem);
  __nv_bfloat16* const outp[6] = {args.at_hi, args.zt_hi, args.yt_hi,
                                  args.at_lo, args.zt_lo, args.yt_lo};
  const bool has_a = args.at_hi != nullptr, has_z = args.zt_hi != nullptr,
             has_y = args.yt_hi != nullptr;
  int it = 0;
#pragma unroll 1
  for (int c0 = 0; c0 < n_eff; c0 += 16, ++it) {
    float v[16];
    tmem_ld16(tmem_q + (uint32_t)c0, v);
    __nv_bfloat16* buf = stg + (it & 1) * NS * SLOT;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      float x = v[j];
      if (F8) {
        const int n = n0 + c0 + j;
        x *= n < n_valid ? wsc * args.tscale[n] : 0.f;   // undo both FP8 scalings
      }
      const int o = j * BM + row;
      if (X3) {
        __nv_bfloat16 h, l;
        if (has_a) {
          split_bf16(sm * x, h, l);
          buf[0 * SLOT + o] = h;
          buf[3 * SLOT + o] = l;
        }
        if (has_z) {
          split_bf16(x, h, l);
          buf[1 * SLOT + o] = h;
          buf[4 * SLOT + o] = l;
        }
        if (has_y) {
          split_bf16(cm * x, h, l);
          buf[2 * SLOT + o] = h;
          buf[5 * SLOT + o] = l;
        }
      } else {
        if (has_a) buf[0 * SLOT + o] = __float2bfloat16_rn(sm * x);
        if (has_z) buf[1 * SLOT + o] = __float2bfloat16_rn(x);
        if (has_y) buf[2 * SLOT + o] = __float2bfloat16_rn(cm * x);
      }
    }
    epi_sync();
    // chunk c = row + 128 i of the slice: output i / 2, column (c / 16) % 16, 16-byte piece c % 16
#pragma unroll
    for (int i = 0; i < 2 * NS; ++i) {
      const int s = i >> 1;
      if ((s % 3 == 0 && !has_a) || (s % 3 == 1 && !has_z) || (s % 3 == 2 && !has_y)) continue;
      const int j = (row >> 4) + 8 * (i & 1), pc = row & 15;
      const int n = n0 + c0 + j;
      if (n < n_valid) {
        const size_t orow = (size_t)(KIND == TC_TANGENT_G ? b_row0 + n : n);
        const int ld = s % 3 == 0 ? args.ldo : args.ldz;
        *reinterpret_cast<uint4*>(outp[s] + orow * ld + m0 + pc * 8) =
            *reinterpret_cast<const uint4*>(buf + s * SLOT + j * BM + pc * 8);
      }
    }
  }
}

template <int BN, int MODE, int KIND>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap ta_hi, const __grid_constant__ CUtensorMap ta_lo,
              const __grid_constant__ CUtensorMap tb_hi, const __grid_constant__ CUtensorMap tb_lo,
              const __grid_constant__ CUtensorMap ta_p2, const __grid_constant__ CUtensorMap tb_p2,
              const TcArgs args) {
  using C = Cfg<BN, MODE>;
  constexpr bool X3 = C::X3;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + C::STAGES * C::STAGE_BYTES);
  uint64_t* empty = full + C::STAGES;
  uint64_t* accf = empty + C::STAGES;
  uint32_t* tmem_slot = (uint32_t*)(accf + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  volatile int* consumed_sh = (volatile int*)(tmem_slot + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int tm, tn, split, grp = 0, a_row0, b_row0, n_valid, n_eff = BN;
  if (KIND == TC_TANGENT) {
    // 1-D grid, full-width column tiles first (row-major over (tm, tn)), then one narrow tile per
    // row block for the N % BN remainder, whose MMA N is the remainder rounded up to 16
    const int nfull = args.N / BN;
    const int b = blockIdx.x;
    if (b < args.ntm * nfull) {
      tm = b / nfull;
      tn = b % nfull;
    } else {
      tm = b - args.ntm * nfull;
      tn = nfull;
    }
    split = 0;
    a_row0 = tm * BM;
    b_row0 = tn * BN;
    n_valid = args.N;
    n_eff = (min(BN, args.N - tn * BN) + 15) / 16 * 16;
  } else if (KIND == TC_SYRK) {
    tn = blockIdx.x % args.ntn;
    tm = blockIdx.x / args.ntn;
    split = blockIdx.y;
    if (tm * BM + BM - 1 < tn * BN) return;  // tile lies strictly above the diagonal
    a_row0 = tm * BM;
    b_row0 = tn * BN;
    n_valid = args.N;
  } else if (KIND == TC_REV) {
    tm = blockIdx.x;
    tn = 0;
    split = blockIdx.y;
    a_row0 = tm * BM;
    b_row0 = 0;
    n_valid = BN;
  } else if (KIND == TC_TANGENT_G) {
    tm = blockIdx.x;
    grp = blockIdx.y;
    tn = 0;
    split = 0;
    a_row0 = grp * args.a_group_rows + tm * BM;
    b_row0 = args.g_boff[grp];
    n_valid = args.g_n[grp];
  } else {
    const int4 w = args.work[blockIdx.x];
    grp = w.x;
    tm = w.y;
    tn = w.z;
    split = blockIdx.y;
    n_valid = args.g_n[grp];
    a_row0 = args.g_boff[grp] + tm * BM;
    b_row0 = args.g_boff[grp] + tn * BN;
  }
  if (KIND == TC_TANGENT_G || KIND == TC_SYRK_G) {
    // the MMA's N is chosen per CTA: the group's valid columns rounded up to 16
    const int cols = min(BN, n_valid - tn * BN);
    n_eff = (cols + 15) / 16 * 16;
    if (cols <= 0) return;
  }
  const uint32_t idesc = C::IDESC_NO_N | ((uint32_t)(n_eff >> 3) << 17);
  const int m0 = tm * BM, n0 = tn * BN;
  const int kb0 = split * args.kb_per_split;
  const int kb1 = min(args.nkb, kb0 + args.kb_per_split);
  const int nk = kb1 - kb0;
  if (nk <= 0) return;  // uniform over the CTA, before any barrier exists

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(accf), 1);
    *abort_flag = 0;
    *consumed_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // tangent chain (launched with programmatic dependent launch): the previous layer's outputs,
  // this layer's B operand, are complete before any copy or store of this CTA
  if (KIND == TC_TANGENT) griddep_wait();

  int issued = 0;  // producer only
  if (warp == 0) {
    if (lane == 0) {
      for (int i = 0; i < nk; ++i) {
        const int s = i % C::STAGES;
        const uint32_t ph = (uint32_t)(i / C::STAGES) & 1u;
        if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1u, args.err, 1, abort_flag)) break;
        uint8_t* st = smem + s * C::STAGE_BYTES;
        const uint32_t fb = smem_u32(&full[s]);
        mbar_expect_tx(fb, C::TX_BYTES);
        const int kx = (kb0 + i) * C::BKE;
        tma_load_2d(smem_u32(st), &ta_hi, fb, kx, a_row0);
        if (X3) tma_load_2d(smem_u32(st + C::A_BYTES), &ta_lo, fb, kx, a_row0);
        tma_load_2d(smem_u32(st + C::NPARTS * C::A_BYTES), &tb_hi, fb, kx, b_row0);
        if (X3) tma_load_2d(smem_u32(st + C::NPARTS * C::A_BYTES + C::B_BYTES), &tb_lo, fb, kx, b_row0);
        if (C::X6) {
          tma_load_2d(smem_u32(st + 2 * C::A_BYTES), &ta_p2, fb, kx, a_row0);
          tma_load_2d(smem_u32(st + C::NPARTS * C::A_BYTES + 2 * C::B_BYTES), &tb_p2, fb, kx, b_row0);
        }
        issued = i + 1;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int i = 0;
      for (; i < nk; ++i) {
        const int s = i % C::STAGES;
        const uint32_t ph = (uint32_t)(i / C::STAGES) & 1u;
        if (!mbar_wait(smem_u32(&full[s]), ph, args.err, 2, abort_flag)) break;
        tc_fence_after();
        const uint32_t st = smem_u32(smem + s * C::STAGE_BYTES);
        const uint32_t a_hi = st, a_lo = st + C::A_BYTES;
        const uint32_t b_hi = st + C::NPARTS * C::A_BYTES;
        const uint32_t b_lo = b_hi + C::B_BYTES;
#pragma unroll
        for (int kk = 0; kk < C::ROWB / 32; ++kk) {
          const uint32_t off = kk * 32;   // one MMA consumes 32 bytes of K: 16 BF16 or 32 E4M3
          constexpr int SW = C::SWZ, SB = C::SBO;
          if (C::F8)
            umma_f8(tmem, sdesc<SW, SB>(a_hi + off), sdesc<SW, SB>(b_hi + off), idesc,
                    (i > 0 || kk > 0) ? 1u : 0u);
          else
            umma_bf16(tmem, sdesc<SW, SB>(a_hi + off), sdesc<SW, SB>(b_hi + off), idesc,
                      (i > 0 || kk > 0) ? 1u : 0u);
          if (X3) {
            umma_bf16(tmem, sdesc<SW, SB>(a_hi + off), sdesc<SW, SB>(b_lo + off), idesc, 1u);
            umma_bf16(tmem, sdesc<SW, SB>(a_lo + off), sdesc<SW, SB>(b_hi + off), idesc, 1u);
          }
          if (C::X6) {
            const uint32_t a_p2 = a_hi + 2 * C::A_BYTES, b_p2 = b_hi + 2 * C::B_BYTES;
            umma_bf16(tmem, sdesc<SW, SB>(a_hi + off), sdesc<SW, SB>(b_p2 + off), idesc, 1u);
            umma_bf16(tmem, sdesc<SW, SB>(a_lo + off), sdesc<SW, SB>(b_lo + off), idesc, 1u);
            umma_bf16(tmem, sdesc<SW, SB>(a_p2 + off), sdesc<SW, SB>(b_hi + off), idesc, 1u);
          }
        }
        umma_commit(smem_u32(&empty[s]));
      }
      *consumed_sh = i;
      umma_commit(smem_u32(accf));  // arrives once every MMA issued above has completed
    }
  } else {
    const int q = warp & 3;  // TMEM lanes 32q .. 32q+31 belong to this warp
    const int row = q * 32 + lane;
    const bool ok = epi_all(mbar_wait(smem_u32(accf), 0, args.err, 3, abort_flag));
    tc_fence_after();
    // the next layer may be queued now: its CTAs take SMs as this grid's epilogues end
    if (KIND == TC_TANGENT && threadIdx.x == 64) griddep_launch();
    if (ok && KIND == TC_REV) {
      // split-K partial of W_l^T Zbar: P[split][k][0..BN) for row k of this tile
      const int k = m0 + row;
      float* out = args.Hp + ((size_t)split * args.M + k) * BN;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4*>(out + c0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
      }
    } else if (ok) {
      if (KIND == TC_TANGENT || KIND == TC_TANGENT_G) {
        const int m = m0 + row;                        // row of W_l inside the group
        const int ms = (KIND == TC_TANGENT_G ? grp * args.a_group_rows : 0) + m;
        const float sm = (float)args.s1[ms];
        const float cm = args.c[ms];
        const float wsc = C::F8 ? args.wscale[ms] : 1.f;   // FP8: per-row weight scale
        if (args.vec_ok) {
          static_assert(C::STAGES * C::STAGE_BYTES >= staged_epi_bytes<X3>(),
                        "staged epilogue fits in the pipeline stages");
          tangent_epilogue_staged<MODE, KIND>(args, smem, tmem + ((uint32_t)(q * 32) << 16), row,
                                              m0, n0, n_eff, n_valid, b_row0, sm, cm, wsc);
        } else {
#pragma unroll 1
          for (int c0 = 0; c0 < n_eff; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int n = n0 + c0 + j;
              if (C::F8 && n < n_valid) v[j] *= wsc * args.tscale[n];   // undo both FP8 scalings
              if (n < n_valid) {
                const size_t orow = (size_t)(KIND == TC_TANGENT_G ? b_row0 + n : n);
                if (args.at_hi) put<X3>(args.at_hi, args.at_lo, orow * args.ldo + m, sm * v[j]);
                if (args.zt_hi) put<X3>(args.zt_hi, args.zt_lo, orow * args.ldz + m, v[j]);
                if (args.yt_hi) put<X3>(args.yt_hi, args.yt_lo, orow * args.ldz + m, cm * v[j]);
              }
            }
          }
        }
      } else {
        const int i = m0 + row;
#pragma unroll 1
        for (int c0 = 0; c0 < n_eff; c0 += 16) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
          if (i < n_valid) {
            float* hp = KIND == TC_SYRK
                            ? args.Hp + ((size_t)split * args.N + i) * args.N
                            : args.Hp + split * args.ldh_split + args.g_hoff[grp] + (size_t)i * n_valid;
            // TC_SYRK: every (split, tile) has exactly one CTA and every split at least one K
            // block, so the partial is stored (the buffer needs no clearing); the grouped form
            // accumulates into a cleared buffer
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int n = n0 + c0 + j;
              if (n <= i) {
                if (KIND == TC_SYRK) hp[n] = v[j];
                else hp[n] += v[j];
              }
            }
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (*abort_flag) {
    // Drain: the producer waits for copies that the MMA warp never consumed, the MMA warp for
    // its outstanding MMAs, both with a short bound, before the memory goes away.
    if (warp == 0 && lane == 0) {
      for (int i = *consumed_sh; i < issued; ++i) {
        const int s = i % C::STAGES;
        const uint32_t ph = (uint32_t)(i / C::STAGES) & 1u;
        volatile int no_abort = 0;
        mbar_wait(smem_u32(&full[s]), ph, args.err, 4, &no_abort, kWaitCycles / 8);
      }
    }
    if (warp == 1 && lane == 0) {
      volatile int no_abort = 0;
      mbar_wait(smem_u32(accf), 0, args.err, 5, &no_abort, kWaitCycles / 8);
    }
    __syncthreads();
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(C::TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------- SM-pair tangent GEMM
// tcgen05 with cta_group::2: a cluster of two CTAs on two SMs computes a 256 x BNP tile.  Each
// CTA copies its own 128 rows of A and its half of the B tile (n / 2 rows) into its own shared
// memory; the copies of both CTAs complete on the even (leader) CTA's "full" barrier, whose
// producer expects the bytes of both.  The leader's MMA thread issues
// tcgen05.mma.cta_group::2 (M = 256): each SM's tensor core multiplies its own A rows by the
// whole B tile, taking one half of B from each SM's shared memory, so each SM stages and reads
// half of B instead of all of it (the single-SM kernel is bound by shared-memory traffic in the
// split form).  Commits arrive on both CTAs' barriers (multicast); each CTA's epilogue reads
// its own 128 accumulator lanes.  Waits are bounded as in k_tc_gemm; both CTAs reach the final
// cluster barrier on every path, so neither frees shared or tensor memory the other still uses.
template <int BNP, int MODE>
struct PairCfg {
  static constexpr bool X3 = MODE == MODE_BF16X3;
  static constexpr int BKE = bk_for(MODE);
  static constexpr int ROWB = BKE * 2;
  static constexpr int SWZ = ROWB == 128 ? 2 : 4;
  static constexpr int SBO = 8 * ROWB;
  static constexpr int BH = BNP / 2;                    // B rows per CTA (box height)
  static constexpr int BH_SLOT = (BH + 15) / 16 * 16;   // shared-memory rows, 1024-byte multiple
  static constexpr int A_BYTES = BM * ROWB;
  static constexpr int B_BYTES = BH_SLOT * ROWB;
  static constexpr int NPARTS = X3 ? 2 : 1;
  static constexpr int STAGE_BYTES = NPARTS * (A_BYTES + B_BYTES);
  static constexpr int TX_PAIR = 2 * NPARTS * (BM + BH) * ROWB;   // both CTAs' boxes
  static constexpr int SMEM_BUDGET = 227 * 1024 - 2048;
  static constexpr int STAGES_FIT = SMEM_BUDGET / STAGE_BYTES;
  static constexpr int STAGES = STAGES_FIT > 8 ? 8 : STAGES_FIT;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
  static constexpr int TMEM_COLS = BNP <= 32 ? 32 : BNP <= 64 ? 64 : BNP <= 128 ? 128 : 256;
  // kind::f16, D = F32, A = B = BF16, K-major, M = 256 (M >> 4 at bit 24)
  static constexpr uint32_t IDESC_NO_N =
      (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(256 >> 4) << 24);
  static_assert(MODE == MODE_BF16 || MODE == MODE_BF16X3, "pair kernel: BF16 forms");
  static_assert(BNP % 16 == 0 && BNP >= 32 && BNP <= 256, "UMMA N for M = 256");
  static_assert(A_BYTES % 1024 == 0 && B_BYTES % 1024 == 0, "1024-byte aligned stage parts");
  static_assert(STAGES >= 2, "at least two stages");
};

__device__ __forceinline__ uint32_t pair_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void pair_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
__device__ __forceinline__ uint32_t map_to_rank(uint32_t local, uint32_t rank) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
  return remote;
}
// 2-D tiled load into this CTA's shared memory whose completion is counted on an mbarrier that
// may sit in the peer CTA of the pair (the leader's "full" barrier).
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map,
                                                 uint32_t mbar_cluster, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"((uint64_t)map), "r"(mbar_cluster), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void umma_bf16_pair(uint32_t tmem_d, uint64_t a, uint64_t b,
                                               uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrives once on the mbarrier at this shared-memory offset in both CTAs of the pair when every
// MMA issued so far has completed.
__device__ __forceinline__ void umma_commit_pair(uint32_t mbar) {
  const uint16_t mask = 0x3;
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(mbar),
      "h"(mask)
      : "memory");
}

template <int BNP, int MODE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    k_tc_pair(const __grid_constant__ CUtensorMap ta_hi, const __grid_constant__ CUtensorMap ta_lo,
              const __grid_constant__ CUtensorMap tb_hi, const __grid_constant__ CUtensorMap tb_lo,
              const TcArgs args) {
  using C = PairCfg<BNP, MODE>;
  constexpr bool X3 = C::X3;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + C::STAGES * C::STAGE_BYTES);
  uint64_t* empty = full + C::STAGES;
  uint64_t* accf = empty + C::STAGES;
  uint32_t* tmem_slot = (uint32_t*)(accf + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  volatile int* consumed_sh = (volatile int*)(tmem_slot + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = pair_rank();   // 0: leader (issues the MMAs)
  // pair tiles: full-width column tiles first (row-major over (tm, tn)), then the remainder tile
  const int pr = blockIdx.x >> 1;
  const int nfull = args.N / BNP;
  int tm, tn;
  if (pr < args.ntm * nfull) {
    tm = pr / nfull;
    tn = pr % nfull;
  } else {
    tm = pr - args.ntm * nfull;
    tn = nfull;
  }
  const int n0 = tn * BNP;
  const int n_eff = (min(BNP, args.N - n0) + 15) / 16 * 16;   // MMA N of this pair
  const int a_row0 = tm * 2 * BM + (int)rank * BM;
  const int b_row0 = n0 + (int)rank * (n_eff / 2);
  const uint32_t idesc = C::IDESC_NO_N | ((uint32_t)(n_eff >> 3) << 17);
  const int nk = args.nkb;
  if (nk <= 0) return;  // uniform over both CTAs, before any barrier exists

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(accf), 1);
    *abort_flag = 0;
    *consumed_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  pair_sync();   // barriers of both CTAs initialised, tensor memory allocated in both
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  griddep_wait();   // programmatic dependent launch: the previous layer's outputs are complete
  const uint32_t full_leader = map_to_rank(smem_u32(full), 0);

  int issued = 0;  // producer only
  if (warp == 0) {
    if (lane == 0) {
      for (int i = 0; i < nk; ++i) {
        const int s = i % C::STAGES;
        const uint32_t ph = (uint32_t)(i / C::STAGES) & 1u;
        if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1u, args.err, 11, abort_flag)) break;
        uint8_t* st = smem + s * C::STAGE_BYTES;
        const uint32_t fb = full_leader + (uint32_t)(s * 8);
        if (rank == 0) mbar_expect_tx(smem_u32(&full[s]), C::TX_PAIR);
        const int kx = i * C::BKE;
        tma_load_2d_pair(smem_u32(st), &ta_hi, fb, kx, a_row0);
        if (X3) tma_load_2d_pair(smem_u32(st + C::A_BYTES), &ta_lo, fb, kx, a_row0);
        tma_load_2d_pair(smem_u32(st + C::NPARTS * C::A_BYTES), &tb_hi, fb, kx, b_row0);
        if (X3)
          tma_load_2d_pair(smem_u32(st + C::NPARTS * C::A_BYTES + C::B_BYTES), &tb_lo, fb, kx,
                           b_row0);
        issued = i + 1;
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      int i = 0;
      for (; i < nk; ++i) {
        const int s = i % C::STAGES;
        const uint32_t ph = (uint32_t)(i / C::STAGES) & 1u;
        if (!mbar_wait(smem_u32(&full[s]), ph, args.err, 12, abort_flag)) break;
        tc_fence_after();
        const uint32_t st = smem_u32(smem + s * C::STAGE_BYTES);
        const uint32_t a_hi = st, a_lo = st + C::A_BYTES;
        const uint32_t b_hi = st + C::NPARTS * C::A_BYTES;
        const uint32_t b_lo = b_hi + C::B_BYTES;
#pragma unroll
        for (int kk = 0; kk < C::ROWB / 32; ++kk) {
          const uint32_t off = kk * 32;   // one MMA consumes K = 16 (32 bytes)
          constexpr int SW = C::SWZ, SB = C::SBO;
          umma_bf16_pair(tmem, sdesc<SW, SB>(a_hi + off), sdesc<SW, SB>(b_hi + off), idesc,
                         (i > 0 || kk > 0) ? 1u : 0u);
          if (X3) {
            umma_bf16_pair(tmem, sdesc<SW, SB>(a_hi + off), sdesc<SW, SB>(b_lo + off), idesc, 1u);
            umma_bf16_pair(tmem, sdesc<SW, SB>(a_lo + off), sdesc<SW, SB>(b_hi + off), idesc, 1u);
          }
        }
        umma_commit_pair(smem_u32(&empty[s]));
      }
      *consumed_sh = i;
      umma_commit_pair(smem_u32(accf));   // both CTAs' epilogues start when every MMA is done
    }
  } else {
    const int q = warp & 3;  // TMEM lanes 32q .. 32q+31 belong to this warp
    const int row = q * 32 + lane;
    const bool ok = epi_all(mbar_wait(smem_u32(accf), 0, args.err, 13, abort_flag));
    tc_fence_after();
    if (threadIdx.x == 64) griddep_launch();
    if (ok && args.vec_ok) {
      static_assert(C::STAGES * C::STAGE_BYTES >= staged_epi_bytes<X3>(),
                    "staged epilogue fits in the pipeline stages");
      const int m = a_row0 + row;
      tangent_epilogue_staged<MODE, TC_TANGENT>(args, smem, tmem + ((uint32_t)(q * 32) << 16), row,
                                                a_row0, n0, n_eff, args.N, 0, (float)args.s1[m],
                                                args.c[m], 1.f);
    } else if (ok) {
      const int m = a_row0 + row;
      const float sm = (float)args.s1[m];
      const float cm = args.c[m];
#pragma unroll 1
      for (int c0 = 0; c0 < n_eff; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + c0 + j;
          if (n < args.N) {
            if (args.at_hi) put<X3>(args.at_hi, args.at_lo, (size_t)n * args.ldo + m, sm * v[j]);
            if (args.zt_hi) put<X3>(args.zt_hi, args.zt_lo, (size_t)n * args.ldz + m, v[j]);
            if (args.yt_hi) put<X3>(args.yt_hi, args.yt_lo, (size_t)n * args.ldz + m, cm * v[j]);
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (*abort_flag) {
    // Drain (bounded): the leader's producer waits for stages it expected but its MMA thread
    // never consumed, the MMA thread for its outstanding MMAs.
    if (rank == 0 && warp == 0 && lane == 0) {
      for (int i = *consumed_sh; i < issued; ++i) {
        const int s = i % C::STAGES;
        const uint32_t ph = (uint32_t)(i / C::STAGES) & 1u;
        volatile int no_abort = 0;
        mbar_wait(smem_u32(&full[s]), ph, args.err, 14, &no_abort, kWaitCycles / 8);
      }
    }
    if (rank == 0 && warp == 1 && lane == 0) {
      volatile int no_abort = 0;
      mbar_wait(smem_u32(accf), 0, args.err, 15, &no_abort, kWaitCycles / 8);
    }
    __syncthreads();
  }
  pair_sync();   // neither CTA releases memory the other's copies or MMAs may still use
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(C::TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------- persistent grouped tangent GEMM
// The grouped tangent GEMM of a batch (many networks, each with its own W_l and its own tangent
// count) as a persistent kernel: one CTA per SM takes the (network, 128-row block) tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...; the copy ring runs on across tiles, and two TMEM
// accumulators (2 x 256 columns) let the epilogue of one tile run while the MMAs of the next
// accumulate, so the short tiles of a batch (K = a hidden width) do not each pay a prologue and
// an unoverlapped epilogue.  Same operands and outputs as TC_TANGENT_G.
template <int BN, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_gtan(const __grid_constant__ CUtensorMap ta_hi, const __grid_constant__ CUtensorMap ta_lo,
              const __grid_constant__ CUtensorMap tb_hi, const __grid_constant__ CUtensorMap tb_lo,
              const TcArgs args, int groups) {
  using C = Cfg<BN, MODE>;
  constexpr bool X3 = C::X3;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + C::STAGES * C::STAGE_BYTES);
  uint64_t* empty = full + C::STAGES;
  uint64_t* accf = empty + C::STAGES;   // [2]: accumulator b holds a finished tile
  uint64_t* tfree = accf + 2;           // [2]: the epilogue has read accumulator b
  uint64_t* mdone = tfree + 2;          // every MMA issued has completed
  uint32_t* tmem_slot = (uint32_t*)(mdone + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  volatile int* consumed_sh = (volatile int*)(tmem_slot + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles = groups * args.ntm;
  const int nkb = args.nkb;
  if (nkb <= 0 || (int)blockIdx.x >= tiles) return;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&accf[b]), 1);
      mbar_init(smem_u32(&tfree[b]), 4);   // one arrival per epilogue warp
    }
    mbar_init(smem_u32(mdone), 1);
    *abort_flag = 0;
    *consumed_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  int issued = 0;  // producer only
  if (warp == 0) {
    if (lane == 0) {
      int i = 0;
      bool stop = false;
      for (int t = blockIdx.x; t < tiles && !stop; t += gridDim.x) {
        const int grp = t / args.ntm, tm = t % args.ntm;
        const int a_row0 = grp * args.a_group_rows + tm * BM;
        const int b_row0 = args.g_boff[grp];
        for (int kb = 0; kb < nkb; ++kb, ++i) {
          const int s = i % C::STAGES;
          const uint32_t ph = (uint32_t)(i / C::STAGES) & 1u;
          if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1u, args.err, 41, abort_flag)) {
            stop = true;
            break;
          }
          uint8_t* st = smem + s * C::STAGE_BYTES;
          const uint32_t fb = smem_u32(&full[s]);
          mbar_expect_tx(fb, C::TX_BYTES);
          const int kx = kb * C::BKE;
          tma_load_2d(smem_u32(st), &ta_hi, fb, kx, a_row0);
          if (X3) tma_load_2d(smem_u32(st + C::A_BYTES), &ta_lo, fb, kx, a_row0);
          tma_load_2d(smem_u32(st + C::NPARTS * C::A_BYTES), &tb_hi, fb, kx, b_row0);
          if (X3) tma_load_2d(smem_u32(st + C::NPARTS * C::A_BYTES + C::B_BYTES), &tb_lo, fb, kx, b_row0);
          issued = i + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int i = 0, pi = 0;
      bool stop = false;
      for (int t = blockIdx.x; t < tiles && !stop; t += gridDim.x, ++pi) {
        const int grp = t / args.ntm;
        const int b = pi & 1;
        if (pi >= 2 &&
            !mbar_wait(smem_u32(&tfree[b]), (uint32_t)((pi - 2) >> 1) & 1u, args.err, 42, abort_flag))
          break;
        tc_fence_after();
        const int n_eff = (min(BN, args.g_n[grp]) + 15) / 16 * 16;
        const uint32_t idesc = C::IDESC_NO_N | ((uint32_t)(n_eff >> 3) << 17);
        const uint32_t d = tmem + (uint32_t)(b * 256);
        for (int kb = 0; kb < nkb; ++kb, ++i) {
          const int s = i % C::STAGES;
          const uint32_t ph = (uint32_t)(i / C::STAGES) & 1u;
          if (!mbar_wait(smem_u32(&full[s]), ph, args.err, 43, abort_flag)) {
            stop = true;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(smem + s * C::STAGE_BYTES);
          const uint32_t a_hi = st, a_lo = st + C::A_BYTES;
          const uint32_t b_hi = st + C::NPARTS * C::A_BYTES;
          const uint32_t b_lo = b_hi + C::B_BYTES;
#pragma unroll
          for (int kk = 0; kk < C::ROWB / 32; ++kk) {
            const uint32_t off = kk * 32;
            constexpr int SW = C::SWZ, SB = C::SBO;
            umma_bf16(d, sdesc<SW, SB>(a_hi + off), sdesc<SW, SB>(b_hi + off), idesc,
                      (kb > 0 || kk > 0) ? 1u : 0u);
            if (X3) {
              umma_bf16(d, sdesc<SW, SB>(a_hi + off), sdesc<SW, SB>(b_lo + off), idesc, 1u);
              umma_bf16(d, sdesc<SW, SB>(a_lo + off), sdesc<SW, SB>(b_hi + off), idesc, 1u);
            }
          }
          umma_commit(smem_u32(&empty[s]));
        }
        if (!stop) umma_commit(smem_u32(&accf[b]));
      }
      *consumed_sh = i;
      umma_commit(smem_u32(mdone));
    }
  } else {
    const int q = warp & 3;  // TMEM lanes 32q .. 32q+31 belong to this warp
    const int row = q * 32 + lane;
    int pi = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++pi) {
      const int grp = t / args.ntm, tm = t % args.ntm;
      const int b = pi & 1;
      if (!mbar_wait(smem_u32(&accf[b]), (uint32_t)(pi >> 1) & 1u, args.err, 44, abort_flag)) break;
      tc_fence_after();
      const int n_valid = args.g_n[grp];
      const int n_eff = (min(BN, n_valid) + 15) / 16 * 16;
      const int b_row0 = args.g_boff[grp];
      const int m = tm * BM + row;                   // row of W_l inside the group
      const int ms = grp * args.a_group_rows + m;    // stacked row
      const float sm = (float)args.s1[ms];
      const float cm = args.c ? args.c[ms] : 0.f;
      const uint32_t dt = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * 256);
#pragma unroll 1
      for (int c0 = 0; c0 < n_eff; c0 += 16) {
        float v[16];
        tmem_ld16(dt + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = c0 + j;
          if (n < n_valid) {
            const size_t orow = (size_t)(b_row0 + n);
            if (args.at_hi) put<X3>(args.at_hi, args.at_lo, orow * args.ldo + m, sm * v[j]);
            if (args.zt_hi) put<X3>(args.zt_hi, args.zt_lo, orow * args.ldz + m, v[j]);
            if (args.yt_hi) put<X3>(args.yt_hi, args.yt_lo, orow * args.ldz + m, cm * v[j]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tfree[b]));
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1 && lane == 0) {
    // every MMA this CTA issued has completed before its memory goes away (bounded)
    volatile int no_abort = 0;
    mbar_wait(smem_u32(mdone), 0, args.err, 45, &no_abort, *abort_flag ? kWaitCycles / 8 : kWaitCycles);
  }
  if (*abort_flag && warp == 0 && lane == 0) {
    for (int i = *consumed_sh; i < issued; ++i) {
      const int s = i % C::STAGES;
      const uint32_t ph = (uint32_t)(i / C::STAGES) & 1u;
      volatile int no_abort = 0;
      mbar_wait(smem_u32(&full[s]), ph, args.err, 46, &no_abort, kWaitCycles / 8);
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                 : "memory");
  }
}

// ---------------------------------------------------------------- persistent tangent chain
// The whole chain of tangent GEMMs of one evaluation (Zdot_l = W_l Adot_{l-1} for every hidden
// layer, with the fused epilogue of TC_TANGENT) in one persistent launch: as many CTAs as one
// layer has tiles (at most one per SM; the remaining SMs stay free for the reverse sweep that runs
// next to the chain), CTA b taking the (layer, column block, row block) tiles b, b + gridDim.x, ...
// in that order.
// Layer l + 1's tiles of column block tn read Adot_l^T rows tn * BN .. (all of layer l's rows
// along K), so they wait (bounded) for an arrival counter that the epilogues of layer l's tiles
// of that column block advance: four arrivals (one per epilogue warp) per row block, released
// after the warp's stores, acquired by the producer before its first copy of the tile, with a
// proxy fence so that the tensor copies see the stores.  The same dependency covers the reuse of
// the ping-pong buffers: the writer of Adot_{l+1}^T rows tn waits for every reader of those rows
// (layer l's tiles of block tn).  A CTA only waits for tiles of a smaller index, which CTAs that
// are resident or finished hold, so the chain cannot dead-lock; the copy ring runs on across
// tiles and layers, and two TMEM accumulators overlap each epilogue with the next tile's MMAs.
// Programmatic dependent launch: the first layer's operand is complete after griddepcontrol.wait.
template <int BN, int MODE>
__global__ void __launch_bounds__(kThreads, 1) k_tc_chain(const __grid_constant__ ChainArgs args) {
  using C = Cfg<BN, MODE>;
  constexpr bool X3 = C::X3;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + C::STAGES * C::STAGE_BYTES);
  uint64_t* empty = full + C::STAGES;
  uint64_t* accf = empty + C::STAGES;   // [2]: accumulator b holds a finished tile
  uint64_t* tfree = accf + 2;           // [2]: the epilogue has read accumulator b
  uint64_t* mdone = tfree + 2;          // every MMA issued has completed
  uint32_t* tmem_slot = (uint32_t*)(mdone + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  volatile int* consumed_sh = (volatile int*)(tmem_slot + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles = args.tiles;
  if ((int)blockIdx.x >= tiles) return;
  // tile t -> (layer, column block, row block); layers in order, column blocks, then rows
  auto decode = [&](int t, int& li, int& tn, int& tm) {
    li = 0;
    while (li + 1 < args.nl && t >= args.L[li + 1].tile0) ++li;
    const int local = t - args.L[li].tile0;
    tn = local / args.L[li].ntm;
    tm = local % args.L[li].ntm;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&accf[b]), 1);
      mbar_init(smem_u32(&tfree[b]), 4);   // one arrival per epilogue warp
    }
    mbar_init(smem_u32(mdone), 1);
    *abort_flag = 0;
    *consumed_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  griddep_wait();   // the first layer's operand and the cleared counters are complete

  int issued = 0;  // producer only
  if (warp == 0) {
    if (lane == 0) {
      int i = 0;
      bool stop = false;
      for (int t = blockIdx.x; t < tiles && !stop; t += gridDim.x) {
        int li, tn, tm;
        decode(t, li, tn, tm);
        const ChainLayer& Ly = args.L[li];
        if (li > 0) {
          // every row block of the previous layer's column block tn is written (acquire)
          const unsigned* cnt = args.cnt + (size_t)(li - 1) * args.ntn + tn;
          const unsigned need = 4u * (unsigned)args.L[li - 1].ntm;
          unsigned v;
          asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(cnt) : "memory");
          if (v < need) {
            const long long t0 = clock64();
            while (true) {
              asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(cnt) : "memory");
              if (v >= need) break;
              if (*abort_flag) {
                stop = true;
                break;
              }
              if (clock64() - t0 > kWaitCycles) {
                atomicCAS(args.err, 0, 51);
                *abort_flag = 1;
                stop = true;
                break;
              }
            }
            if (stop) break;
          }
          asm volatile("fence.proxy.async.global;" ::: "memory");
        }
        const int a_row0 = tm * BM, b_row0 = tn * BN;
        for (int kb = 0; kb < Ly.nkb; ++kb, ++i) {
          const int s = i % C::STAGES;
          const uint32_t ph = (uint32_t)(i / C::STAGES) & 1u;
          if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1u, args.err, 52, abort_flag)) {
            stop = true;
            break;
          }
          uint8_t* st = smem + s * C::STAGE_BYTES;
          const uint32_t fb = smem_u32(&full[s]);
          mbar_expect_tx(fb, C::TX_BYTES);
          const int kx = kb * C::BKE;
          tma_load_2d(smem_u32(st), &args.ta_hi[li], fb, kx, a_row0);
          if (X3) tma_load_2d(smem_u32(st + C::A_BYTES), &args.ta_lo[li], fb, kx, a_row0);
          tma_load_2d(smem_u32(st + C::NPARTS * C::A_BYTES), &args.tb_hi[li], fb, kx, b_row0);
          if (X3)
            tma_load_2d(smem_u32(st + C::NPARTS * C::A_BYTES + C::B_BYTES), &args.tb_lo[li], fb, kx, b_row0);
          issued = i + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int i = 0, pi = 0;
      bool stop = false;
      for (int t = blockIdx.x; t < tiles && !stop; t += gridDim.x, ++pi) {
        int li, tn, tm;
        decode(t, li, tn, tm);
        const int b = pi & 1;
        if (pi >= 2 &&
            !mbar_wait(smem_u32(&tfree[b]), (uint32_t)((pi - 2) >> 1) & 1u, args.err, 53, abort_flag))
          break;
        tc_fence_after();
        const int n_eff = (min(BN, args.N - tn * BN) + 15) / 16 * 16;
        const uint32_t idesc = C::IDESC_NO_N | ((uint32_t)(n_eff >> 3) << 17);
        const uint32_t d = tmem + (uint32_t)(b * 256);
        const int nkb = args.L[li].nkb;
        for (int kb = 0; kb < nkb; ++kb, ++i) {
          const int s = i % C::STAGES;
          const uint32_t ph = (uint32_t)(i / C::STAGES) & 1u;
          if (!mbar_wait(smem_u32(&full[s]), ph, args.err, 54, abort_flag)) {
            stop = true;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(smem + s * C::STAGE_BYTES);
          const uint32_t a_hi = st, a_lo = st + C::A_BYTES;
          const uint32_t b_hi = st + C::NPARTS * C::A_BYTES;
          const uint32_t b_lo = b_hi + C::B_BYTES;
#pragma unroll
          for (int kk = 0; kk < C::ROWB / 32; ++kk) {
            const uint32_t off = kk * 32;
            constexpr int SW = C::SWZ, SB = C::SBO;
            umma_bf16(d, sdesc<SW, SB>(a_hi + off), sdesc<SW, SB>(b_hi + off), idesc,
                      (kb > 0 || kk > 0) ? 1u : 0u);
            if (X3) {
              umma_bf16(d, sdesc<SW, SB>(a_hi + off), sdesc<SW, SB>(b_lo + off), idesc, 1u);
              umma_bf16(d, sdesc<SW, SB>(a_lo + off), sdesc<SW, SB>(b_hi + off), idesc, 1u);
            }
          }
          umma_commit(smem_u32(&empty[s]));
        }
        if (!stop) umma_commit(smem_u32(&accf[b]));
      }
      *consumed_sh = i;
      umma_commit(smem_u32(mdone));
    }
  } else {
    const int q = warp & 3;  // TMEM lanes 32q .. 32q+31 belong to this warp
    const int row = q * 32 + lane;
    int pi = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++pi) {
      int li, tn, tm;
      decode(t, li, tn, tm);
      // the layer's fields in registers: a reference into the kernel parameters at a run-time
      // index would be re-read from memory at every store of the epilogue
      const ChainLayer Ly = args.L[li];
      const int b = pi & 1;
      if (!mbar_wait(smem_u32(&accf[b]), (uint32_t)(pi >> 1) & 1u, args.err, 55, abort_flag)) break;
      tc_fence_after();
      // the kernel after the chain may be queued once this CTA's last tile is in its epilogue
      if (t + (int)gridDim.x >= tiles && threadIdx.x == 64) griddep_launch();
      const int n0 = tn * BN;
      const int n_eff = (min(BN, args.N - n0) + 15) / 16 * 16;
      const int m = tm * BM + row;   // row of W_l
      const float sm = (float)Ly.s1[m];
      const float cm = Ly.c ? Ly.c[m] : 0.f;
      const uint32_t dt = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * 256);
#pragma unroll 1
      for (int c0 = 0; c0 < n_eff; c0 += 16) {
        float v[16];
        tmem_ld16(dt + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + c0 + j;
          if (n < args.N) {
            if (Ly.at_hi) put<X3>(Ly.at_hi, Ly.at_lo, (size_t)n * Ly.ldo + m, sm * v[j]);
            if (Ly.zt_hi) put<X3>(Ly.zt_hi, Ly.zt_lo, (size_t)n * args.ldz + m, v[j]);
            if (Ly.yt_hi) put<X3>(Ly.yt_hi, Ly.yt_lo, (size_t)n * args.ldz + m, cm * v[j]);
          }
        }
      }
      tc_fence_before();
      // release this warp's stores to the next layer's producers, then free the accumulator
      __threadfence();
      __syncwarp();
      if (lane == 0) {
        atomicAdd(args.cnt + (size_t)li * args.ntn + tn, 1u);
        mbar_arrive(smem_u32(&tfree[b]));
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1 && lane == 0) {
    volatile int no_abort = 0;
    mbar_wait(smem_u32(mdone), 0, args.err, 56, &no_abort, *abort_flag ? kWaitCycles / 8 : kWaitCycles);
  }
  if (*abort_flag && warp == 0 && lane == 0) {
    for (int i = *consumed_sh; i < issued; ++i) {
      const int s = i % C::STAGES;
      const uint32_t ph = (uint32_t)(i / C::STAGES) & 1u;
      volatile int no_abort = 0;
      mbar_wait(smem_u32(&full[s]), ph, args.err, 57, &no_abort, kWaitCycles / 8);
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                 : "memory");
  }
}

// ---------------------------------------------------------------- plain BF16 GEMM
// C = A B^T for the learned warm start's small dense layers (forward Z = X W^T, backward
// dH = dZ W and dW = dZ^T X with transposed operand copies): one 128 x BN tile per CTA, the
// producer / MMA / epilogue warps of k_tc_gemm, single BF16 product into an FP32 TMEM tile.
// Epilogue: C[m][n] = acc + bias[n] for m < M, n < N (FP32, row stride ldc); with gelu also
// Hf = GELU(C) (FP32), Hl = GELU(C) (BF16, row stride ldc) and, when Ht is given, the transposed
// BF16 copy Ht[n][m] (row stride ldt), the operand layout of the next backward product.
struct PlainArgs {
  int M, N, nkb, ntn;
  const float* bias;
  float* C;
  int ldc;
  int gelu;
  float* Hf;
  __nv_bfloat16* Hl;
  __nv_bfloat16* Ht;
  int ldt;
  int* err;
};

template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_plain(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
               const PlainArgs args) {
  using C = Cfg<BN, MODE_BF16>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + C::STAGES * C::STAGE_BYTES);
  uint64_t* empty = full + C::STAGES;
  uint64_t* accf = empty + C::STAGES;
  uint32_t* tmem_slot = (uint32_t*)(accf + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  volatile int* consumed_sh = (volatile int*)(tmem_slot + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tm = blockIdx.x / args.ntn, tn = blockIdx.x % args.ntn;
  const int m0 = tm * BM, n0 = tn * BN;
  const int n_eff = (min(BN, args.N - n0) + 15) / 16 * 16;
  const uint32_t idesc = C::IDESC_NO_N | ((uint32_t)(n_eff >> 3) << 17);
  const int nk = args.nkb;
  if (nk <= 0 || n_eff <= 0) return;   // uniform over the CTA, before any barrier exists

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(accf), 1);
    *abort_flag = 0;
    *consumed_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  int issued = 0;
  if (warp == 0) {
    if (lane == 0) {
      for (int i = 0; i < nk; ++i) {
        const int s = i % C::STAGES;
        const uint32_t ph = (uint32_t)(i / C::STAGES) & 1u;
        if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1u, args.err, 61, abort_flag)) break;
        uint8_t* st = smem + s * C::STAGE_BYTES;
        const uint32_t fb = smem_u32(&full[s]);
        mbar_expect_tx(fb, C::TX_BYTES);
        const int kx = i * C::BKE;
        tma_load_2d(smem_u32(st), &ta, fb, kx, m0);
        tma_load_2d(smem_u32(st + C::A_BYTES), &tb, fb, kx, n0);
        issued = i + 1;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int i = 0;
      for (; i < nk; ++i) {
        const int s = i % C::STAGES;
        const uint32_t ph = (uint32_t)(i / C::STAGES) & 1u;
        if (!mbar_wait(smem_u32(&full[s]), ph, args.err, 62, abort_flag)) break;
        tc_fence_after();
        const uint32_t st = smem_u32(smem + s * C::STAGE_BYTES);
#pragma unroll
        for (int kk = 0; kk < C::ROWB / 32; ++kk) {
          const uint32_t off = kk * 32;
          constexpr int SW = C::SWZ, SB = C::SBO;
          umma_bf16(tmem, sdesc<SW, SB>(st + off), sdesc<SW, SB>(st + C::A_BYTES + off), idesc,
                    (i > 0 || kk > 0) ? 1u : 0u);
        }
        umma_commit(smem_u32(&empty[s]));
      }
      *consumed_sh = i;
      umma_commit(smem_u32(accf));
    }
  } else {
    const int q = warp & 3;
    const int m = m0 + q * 32 + lane;
    const bool ok = mbar_wait(smem_u32(accf), 0, args.err, 63, abort_flag);
    tc_fence_after();
    if (ok) {
#pragma unroll 1
      for (int c0 = 0; c0 < n_eff; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
        if (m < args.M) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int n = n0 + c0 + j;
            if (n < args.N) {
              const float z = v[j] + (args.bias ? args.bias[n] : 0.f);
              const size_t o = (size_t)m * args.ldc + n;
              args.C[o] = z;
              if (args.gelu) {
                double a, d1, d2;
                act_eval(NNC_GELU, (double)z, a, d1, d2);
                args.Hf[o] = (float)a;
                const __nv_bfloat16 hb = __float2bfloat16_rn((float)a);
                args.Hl[o] = hb;
                if (args.Ht) args.Ht[(size_t)n * args.ldt + m] = hb;
              }
            }
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (*abort_flag) {
    if (warp == 0 && lane == 0) {
      for (int i = *consumed_sh; i < issued; ++i) {
        const int s = i % C::STAGES;
        const uint32_t ph = (uint32_t)(i / C::STAGES) & 1u;
        volatile int no_abort = 0;
        mbar_wait(smem_u32(&full[s]), ph, args.err, 64, &no_abort, kWaitCycles / 8);
      }
    }
    if (warp == 1 && lane == 0) {
      volatile int no_abort = 0;
      mbar_wait(smem_u32(accf), 0, args.err, 65, &no_abort, kWaitCycles / 8);
    }
    __syncthreads();
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(C::TMEM_COLS)
                 : "memory");
  }
}

// Self-test of the tensor-core kernels' bounded wait (with the CTA abort flag): an mbarrier that
// nothing arrives on; the wait gives up after `limit` cycles, records `code` and sets the flag,
// which a second wait then sees at once.
__global__ void k_tc_wait_selftest(int* err, long long limit, int code) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ volatile int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_wait(smem_u32(&bar), 0, err, code, &abort_flag, limit);
    if (abort_flag) mbar_wait(smem_u32(&bar), 0, err, code + 1, &abort_flag, limit);
  }
  __syncthreads();
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
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

// 2-D BF16 map: inner extent `cols` (K, contiguous), outer extent `rows`, row stride ld
// elements, box bk x box_rows with 128-byte (bk = 64) or 64-byte (bk = 32) swizzle, zero fill.
bool make_map(CUtensorMap* m, const void* base, int rows, int cols, int ld, int box_rows, int bk,
              int eb = 2) {
  if (!base) {
    memset(m, 0, sizeof(*m));
    return true;
  }
  auto enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * eb};
  cuuint32_t box[2] = {(cuuint32_t)bk, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, eb == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                   const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   bk * eb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int BN, int MODE, int KIND>
cudaError_t launch_t(const TcPlan& p, const TcArgs& a, dim3 grid, cudaStream_t st) {
  using C = Cfg<BN, MODE>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<BN, MODE, KIND>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (KIND == TC_TANGENT) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_tc_gemm<BN, MODE, KIND>, p.ta_hi, p.ta_lo,
                                             p.tb_hi, p.tb_lo, p.ta_p2, p.tb_p2, a);
    note_launch();
    return e;
  }
  k_tc_gemm<BN, MODE, KIND><<<grid, kThreads, C::SMEM, st>>>(p.ta_hi, p.ta_lo, p.tb_hi, p.tb_lo, p.ta_p2,
                                                             p.tb_p2, a);
  note_launch();
  return cudaGetLastError();
}

template <int BNP, int MODE>
cudaError_t launch_pair_t(const TcPlan& p, const TcArgs& a, int ctas, cudaStream_t st) {
  using C = PairCfg<BNP, MODE>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_pair<BNP, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = C::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_tc_pair<BNP, MODE>, p.ta_hi, p.ta_lo, p.tb_hi,
                                           p.tb_lo, a);
  note_launch();
  return e;
}

template <int BNP>
cudaError_t launch_pair_mode(const TcPlan& p, const TcArgs& a, int ctas, cudaStream_t st) {
  if (p.mode == MODE_BF16X3) return launch_pair_t<BNP, MODE_BF16X3>(p, a, ctas, st);
  if (p.mode == MODE_BF16) return launch_pair_t<BNP, MODE_BF16>(p, a, ctas, st);
  return cudaErrorInvalidValue;
}

constexpr int kPairTiles[4] = {128, 160, 208, 256};

cudaError_t launch_pair(const TcPlan& p, const TcArgs& a, int ctas, cudaStream_t st) {
  switch (p.bn) {
    case 128: return launch_pair_mode<128>(p, a, ctas, st);
    case 160: return launch_pair_mode<160>(p, a, ctas, st);
    case 208: return launch_pair_mode<208>(p, a, ctas, st);
    case 256: return launch_pair_mode<256>(p, a, ctas, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int KIND, int BN>
cudaError_t launch_mode(const TcPlan& p, const TcArgs& a, dim3 grid, cudaStream_t st) {
  if (p.mode == MODE_BF16X3) return launch_t<BN, MODE_BF16X3, KIND>(p, a, grid, st);
  if (p.mode == MODE_FP8) {
    if constexpr (KIND == TC_TANGENT) return launch_t<BN, MODE_FP8, KIND>(p, a, grid, st);
    return cudaErrorInvalidValue;
  }
  return launch_t<BN, MODE_BF16, KIND>(p, a, grid, st);
}

template <int KIND>
cudaError_t launch_any(const TcPlan& p, const TcArgs& a, dim3 grid, cudaStream_t st) {
  if constexpr (KIND == TC_REV) {
    if (p.bn == 16) return launch_t<16, MODE_BF16X6, KIND>(p, a, grid, st);
    if (p.bn == 48) return launch_t<48, MODE_BF16X6, KIND>(p, a, grid, st);
    return cudaErrorInvalidValue;
  }
  switch (p.bn) {
    case 112: return launch_mode<KIND, 112>(p, a, grid, st);
    case 128: return launch_mode<KIND, 128>(p, a, grid, st);
    case 208: return launch_mode<KIND, 208>(p, a, grid, st);
    case 256: return launch_mode<KIND, 256>(p, a, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

int count_lower_tiles(int ntm, int ntn, int bn) {
  int t = 0;
  for (int tm = 0; tm < ntm; ++tm)
    for (int tn = 0; tn < ntn; ++tn)
      if (tm * BM + BM - 1 >= tn * bn) ++t;
  return t;
}

}  // namespace

int tc_plan_make(TcPlan& p, int kind, int prec, const void* a_hi, const void* a_lo, int a_rows,
                 int ld_a, const void* b_hi, const void* b_lo, int b_rows, int ld_b, int M, int N,
                 int K, int sm_count, int force_bn, int force_splits, const void* a_p2,
                 const void* b_p2) {
  p = TcPlan();
  p.kind = kind;
  p.x3 = (prec == NNC_BF16X3 || kind == TC_REV) ? 1 : 0;
  p.M = M;
  p.N = N;
  p.K = K;
  p.mode = kind == TC_REV ? MODE_BF16X6
           : prec == NNC_BF16X3 ? MODE_BF16X3
           : (prec == NNC_FP8 && kind == TC_TANGENT) ? MODE_FP8 : MODE_BF16;
  p.bk = bk_for(p.mode);
  const int eb = p.mode == MODE_FP8 ? 1 : 2;
  if (K % 64 != 0 || K <= 0 || N <= 0 || M <= 0) return NNC_ERR_ARG;
  if ((kind == TC_TANGENT || kind == TC_TANGENT_G) && M % BM != 0) return NNC_ERR_ARG;
  const int nkb = K / p.bk;
  if (kind == TC_REV) {
    // reverse sweep: M = columns of W_l (rows of W_l^T), N = seed columns (16 or 48), split-K over
    // the rows of W_l so that about one CTA per SM runs
    if (N > 48) return NNC_ERR_UNSUPPORTED;
    p.bn = N <= 16 ? 16 : 48;
    p.ntm = M / BM;
    p.ntn = 1;
    int splits = force_splits ? force_splits : std::max(1, sm_count / std::max(1, p.ntm));
    splits = std::min(splits, nkb);
    p.kb_per_split = (nkb + splits - 1) / splits;
    p.splits = (nkb + p.kb_per_split - 1) / p.kb_per_split;
  } else if (kind == TC_TANGENT_G || kind == TC_SYRK_G) {
    // grouped: N is the widest group's column count (rounded to 16); the MMA N of each CTA is
    // chosen at run time from its group's width.
    int bn = (N + 15) / 16 * 16;
    if (force_bn) bn = force_bn;
    const int cands[4] = {112, 128, 208, 256};
    int pick = 256;
    for (int c : cands)
      if (c >= bn) {
        pick = c;
        break;
      }
    if (bn > 256) return NNC_ERR_UNSUPPORTED;
    p.bn = kind == TC_SYRK_G ? 128 : pick;
    p.ntm = kind == TC_TANGENT_G ? M / BM : 0;
    // grouped tangent GEMMs in the BF16 forms run persistently (one CTA per SM over the tiles)
    p.persistent = kind == TC_TANGENT_G && (p.mode == MODE_BF16 || p.mode == MODE_BF16X3);
    p.sm_count = sm_count;
    p.ntn = 1;
    p.splits = force_splits ? force_splits : 1;
    if (p.splits > nkb) p.splits = nkb;
    p.kb_per_split = (nkb + p.splits - 1) / p.splits;
    p.splits = (nkb + p.kb_per_split - 1) / p.kb_per_split;
  } else if (kind == TC_TANGENT && force_bn < 0) {
    // SM-pair kernel: 256-row tiles, N tile -force_bn
    bool ok = M % (2 * BM) == 0 && (p.mode == MODE_BF16 || p.mode == MODE_BF16X3);
    bool known = false;
    for (int t : kPairTiles) known |= t == -force_bn;
    if (!ok || !known) return NNC_ERR_ARG;
    p.pair = 1;
    p.bn = -force_bn;
    p.ntm = M / (2 * BM);
    p.ntn = (N + p.bn - 1) / p.bn;
    p.splits = 1;
    p.kb_per_split = nkb;
  } else if (kind == TC_TANGENT) {
    int best_bn = 208;
    double best = 1e30;
    const int cands[4] = {256, 208, 128, 112};
    const int ntm = M / BM;
    for (int bn : cands) {
      // waves of full tiles; the narrow remainder tile counts as a full one
      const int ctas = ntm * ((N + bn - 1) / bn);
      const double cost = (double)((ctas + sm_count - 1) / sm_count) * (bn + 24);
      if (cost < best - 1e-9) {
        best = cost;
        best_bn = bn;
      }
    }
    p.bn = force_bn ? force_bn : best_bn;
    p.ntm = ntm;
    p.ntn = (N + p.bn - 1) / p.bn;
    p.splits = 1;
    p.kb_per_split = nkb;
  } else {
    p.bn = force_bn ? force_bn : 128;
    p.ntm = (N + BM - 1) / BM;
    p.ntn = (N + p.bn - 1) / p.bn;
    const int tiles = count_lower_tiles(p.ntm, p.ntn, p.bn);
    int splits = force_splits ? force_splits : (sm_count + tiles / 2) / tiles;
    splits = splits < 1 ? 1 : splits > nkb ? nkb : splits;
    p.kb_per_split = (nkb + splits - 1) / splits;
    p.splits = (nkb + p.kb_per_split - 1) / p.kb_per_split;
  }
  const int a_box = BM;
  // REV: the seed rows of B beyond the plan's N read as zero; pair plans: each CTA's half of B
  const int b_box = p.pair ? p.bn / 2 : p.bn;
  if (!make_map(&p.ta_hi, a_hi, a_rows, K, ld_a, a_box, p.bk, eb)) return NNC_ERR_CUDA;
  if (!make_map(&p.ta_lo, p.x3 ? a_lo : nullptr, a_rows, K, ld_a, a_box, p.bk, eb)) return NNC_ERR_CUDA;
  if (!make_map(&p.tb_hi, b_hi, b_rows, K, ld_b, b_box, p.bk, eb)) return NNC_ERR_CUDA;
  if (!make_map(&p.tb_lo, p.x3 ? b_lo : nullptr, b_rows, K, ld_b, b_box, p.bk, eb)) return NNC_ERR_CUDA;
  const bool x6 = p.mode == MODE_BF16X6;
  if (x6 && (!a_p2 || !b_p2)) return NNC_ERR_ARG;
  if (!make_map(&p.ta_p2, x6 ? a_p2 : nullptr, a_rows, K, ld_a, a_box, p.bk, eb)) return NNC_ERR_CUDA;
  if (!make_map(&p.tb_p2, x6 ? b_p2 : nullptr, b_rows, K, ld_b, b_box, p.bk, eb)) return NNC_ERR_CUDA;
  p.ready = true;
  return NNC_OK;
}

cudaError_t launch_wait_selftest_tc(int* err, long long limit, int code, cudaStream_t st) {
  k_tc_wait_selftest<<<1, 32, 0, st>>>(err, limit, code);
  note_launch();
  return cudaGetLastError();
}

// The staged tangent epilogue stores 16-byte pieces: every output 16-byte aligned, row strides
// multiples of 8 elements.
int vec_outputs(const TcArgs& a) {
  auto al = [](const void* q) { return ((uintptr_t)q & 15) == 0; };
  return al(a.at_hi) && al(a.at_lo) && al(a.zt_hi) && al(a.zt_lo) && al(a.yt_hi) && al(a.yt_lo) &&
         a.ldo % 8 == 0 && a.ldz % 8 == 0;
}

cudaError_t tc_tangent(const TcPlan& p, const double* s1, const float* c, void* at_hi, void* at_lo,
                       int ldo, void* zt_hi, void* zt_lo, void* yt_hi, void* yt_lo, int ldz,
                       int* err, cudaStream_t st, const float* wscale, const float* tscale) {
  if (!p.ready || p.kind != TC_TANGENT) return cudaErrorInvalidValue;
  TcArgs a{};
  a.M = p.M;
  a.N = p.N;
  a.K = p.K;
  a.ntm = p.ntm;
  a.ntn = p.ntn;
  a.nkb = p.K / p.bk;
  a.kb_per_split = p.kb_per_split;
  a.s1 = s1;
  a.c = c;
  a.at_hi = (__nv_bfloat16*)at_hi;
  a.at_lo = (__nv_bfloat16*)at_lo;
  a.zt_hi = (__nv_bfloat16*)zt_hi;
  a.zt_lo = (__nv_bfloat16*)zt_lo;
  a.yt_hi = (__nv_bfloat16*)yt_hi;
  a.yt_lo = (__nv_bfloat16*)yt_lo;
  a.ldo = ldo;
  a.ldz = ldz;
  a.err = err;
  a.wscale = wscale;
  a.tscale = tscale;
  a.vec_ok = vec_outputs(a);
  if (p.pair) return launch_pair(p, a, 2 * p.ntm * p.ntn, st);
  return launch_any<TC_TANGENT>(p, a, dim3(p.ntn * p.ntm, 1, 1), st);
}

template <int BN, int MODE>
cudaError_t launch_gtan_t(const TcPlan& p, const TcArgs& a, int groups, int grid, cudaStream_t st) {
  using C = Cfg<BN, MODE>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_gtan<BN, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_tc_gtan<BN, MODE><<<grid, kThreads, C::SMEM, st>>>(p.ta_hi, p.ta_lo, p.tb_hi, p.tb_lo, a, groups);
  note_launch();
  return cudaGetLastError();
}

template <int BN>
cudaError_t launch_gtan_mode(const TcPlan& p, const TcArgs& a, int groups, int grid, cudaStream_t st) {
  if (p.mode == MODE_BF16X3) return launch_gtan_t<BN, MODE_BF16X3>(p, a, groups, grid, st);
  if (p.mode == MODE_BF16) return launch_gtan_t<BN, MODE_BF16>(p, a, groups, grid, st);
  return cudaErrorInvalidValue;
}

int tc_plain_plan(PlainPlan& p, const void* A, int a_rows, int lda, const void* B, int b_rows,
                  int ldb, int M, int N, int K) {
  p = PlainPlan();
  if (M <= 0 || N <= 0 || K <= 0 || K % 64 != 0 || lda % 8 != 0 || ldb % 8 != 0 || !A || !B)
    return NNC_ERR_ARG;
  p.M = M;
  p.N = N;
  p.K = K;
  p.bn = N <= 128 ? 128 : 256;
  p.ntm = (M + BM - 1) / BM;
  p.ntn = (N + p.bn - 1) / p.bn;
  if (!make_map(&p.ta, A, a_rows, K, lda, BM, 64) || !make_map(&p.tb, B, b_rows, K, ldb, p.bn, 64))
    return NNC_ERR_CUDA;
  p.ready = true;
  return NNC_OK;
}

template <int BN>
cudaError_t launch_plain_t(const PlainPlan& p, const PlainArgs& a, cudaStream_t st) {
  using C = Cfg<BN, MODE_BF16>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_plain<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_tc_plain<BN><<<p.ntm * p.ntn, kThreads, C::SMEM, st>>>(p.ta, p.tb, a);
  note_launch();
  return cudaGetLastError();
}

cudaError_t tc_plain(const PlainPlan& p, const float* bias, float* Cout, int ldc, bool gelu, float* Hf,
                     void* Hl, void* Ht, int ldt, int* err, cudaStream_t st) {
  if (!p.ready || !Cout || (gelu && (!Hf || !Hl))) return cudaErrorInvalidValue;
  PlainArgs a{p.M, p.N, p.K / 64, p.ntn, bias, Cout, ldc, gelu ? 1 : 0, Hf, (__nv_bfloat16*)Hl,
              (__nv_bfloat16*)Ht, ldt, err};
  return p.bn == 128 ? launch_plain_t<128>(p, a, st) : launch_plain_t<256>(p, a, st);
}

template <int BN, int MODE>
cudaError_t launch_chain_t(const ChainArgs& a, int grid, cudaStream_t st) {
  using C = Cfg<BN, MODE>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_chain<BN, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = C::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_tc_chain<BN, MODE>, a);
  note_launch();
  return e;
}

template <int BN>
cudaError_t launch_chain_mode(int mode, const ChainArgs& a, int grid, cudaStream_t st) {
  if (mode == MODE_BF16X3) return launch_chain_t<BN, MODE_BF16X3>(a, grid, st);
  if (mode == MODE_BF16) return launch_chain_t<BN, MODE_BF16>(a, grid, st);
  return cudaErrorInvalidValue;
}

cudaError_t tc_tangent_chain(const TcPlan* plans, const ChainOut* outs, int nl, unsigned* cnt,
                             int ldz, int* err, cudaStream_t st) {
  if (nl < 1 || nl > kMaxChain || !cnt) return cudaErrorInvalidValue;
  ChainArgs a{};
  const TcPlan& p0 = plans[0];
  int tiles = 0;
  for (int l = 0; l < nl; ++l) {
    const TcPlan& p = plans[l];
    if (!p.ready || p.kind != TC_TANGENT || p.pair || p.bn != p0.bn || p.mode != p0.mode ||
        p.N != p0.N || p.splits != 1)
      return cudaErrorInvalidValue;
    a.ta_hi[l] = p.ta_hi;
    a.ta_lo[l] = p.ta_lo;
    a.tb_hi[l] = p.tb_hi;
    a.tb_lo[l] = p.tb_lo;
    ChainLayer& L = a.L[l];
    L.ntm = p.ntm;
    L.nkb = p.K / p.bk;
    L.tile0 = tiles;
    L.s1 = outs[l].s1;
    L.c = outs[l].c;
    L.at_hi = (__nv_bfloat16*)outs[l].at_hi;
    L.at_lo = (__nv_bfloat16*)outs[l].at_lo;
    L.ldo = outs[l].ldo;
    L.zt_hi = (__nv_bfloat16*)outs[l].zt_hi;
    L.zt_lo = (__nv_bfloat16*)outs[l].zt_lo;
    L.yt_hi = (__nv_bfloat16*)outs[l].yt_hi;
    L.yt_lo = (__nv_bfloat16*)outs[l].yt_lo;
    tiles += p.ntm * p.ntn;
  }
  a.nl = nl;
  a.N = p0.N;
  a.ntn = p0.ntn;
  a.ldz = ldz;
  a.tiles = tiles;
  a.cnt = cnt;
  a.err = err;
  const int grid = std::min({p0.sm_count > 0 ? p0.sm_count : 148, tiles, p0.ntm * p0.ntn});
  switch (p0.bn) {
    case 112: return launch_chain_mode<112>(p0.mode, a, grid, st);
    case 128: return launch_chain_mode<128>(p0.mode, a, grid, st);
    case 208: return launch_chain_mode<208>(p0.mode, a, grid, st);
    case 256: return launch_chain_mode<256>(p0.mode, a, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t tc_tangent_grouped(const TcPlan& p, int groups, const int* g_n, const int* g_boff,
                               const double* s1, const float* c, void* at_hi, void* at_lo, int ldo,
                               void* zt_hi, void* zt_lo, void* yt_hi, void* yt_lo, int ldz,
                               int* err, cudaStream_t st) {
  if (!p.ready || p.kind != TC_TANGENT_G) return cudaErrorInvalidValue;
  TcArgs a{};
  a.M = p.M;
  a.N = p.N;
  a.K = p.K;
  a.ntm = p.ntm;
  a.ntn = 1;
  a.nkb = p.K / p.bk;
  a.kb_per_split = a.nkb;
  a.s1 = s1;
  a.c = c;
  a.at_hi = (__nv_bfloat16*)at_hi;
  a.at_lo = (__nv_bfloat16*)at_lo;
  a.zt_hi = (__nv_bfloat16*)zt_hi;
  a.zt_lo = (__nv_bfloat16*)zt_lo;
  a.yt_hi = (__nv_bfloat16*)yt_hi;
  a.yt_lo = (__nv_bfloat16*)yt_lo;
  a.ldo = ldo;
  a.ldz = ldz;
  a.err = err;
  a.g_n = g_n;
  a.g_boff = g_boff;
  a.a_group_rows = p.M;
  a.vec_ok = vec_outputs(a);
  if (p.persistent) {
    const int grid = std::min(p.sm_count, groups * p.ntm);
    switch (p.bn) {
      case 112: return launch_gtan_mode<112>(p, a, groups, grid, st);
      case 128: return launch_gtan_mode<128>(p, a, groups, grid, st);
      case 208: return launch_gtan_mode<208>(p, a, groups, grid, st);
      case 256: return launch_gtan_mode<256>(p, a, groups, grid, st);
      default: return cudaErrorInvalidValue;
    }
  }
  return launch_any<TC_TANGENT_G>(p, a, dim3(p.ntm, groups, 1), st);
}

cudaError_t tc_syrk_grouped(const TcPlan& p, int n_tiles, const int4* work, const int* g_n,
                            const int* g_boff, const long long* g_hoff, long long ldh_split,
                            float* Hp, int* err, cudaStream_t st) {
  if (!p.ready || p.kind != TC_SYRK_G) return cudaErrorInvalidValue;
  TcArgs a{};
  a.K = p.K;
  a.nkb = p.K / p.bk;
  a.kb_per_split = p.kb_per_split;
  a.Hp = Hp;
  a.err = err;
  a.g_n = g_n;
  a.g_boff = g_boff;
  a.g_hoff = g_hoff;
  a.work = work;
  a.ldh_split = ldh_split;
  return launch_any<TC_SYRK_G>(p, a, dim3(n_tiles, p.splits, 1), st);
}

cudaError_t tc_rev(const TcPlan& p, float* part, int* err, cudaStream_t st) {
  if (!p.ready || p.kind != TC_REV) return cudaErrorInvalidValue;
  TcArgs a{};
  a.M = p.M;
  a.N = p.N;
  a.K = p.K;
  a.ntm = p.ntm;
  a.ntn = 1;
  a.nkb = p.K / p.bk;
  a.kb_per_split = p.kb_per_split;
  a.Hp = part;
  a.err = err;
  return launch_any<TC_REV>(p, a, dim3(p.ntm, p.splits, 1), st);
}

cudaError_t tc_syrk(const TcPlan& p, float* Hp, int* err, cudaStream_t st) {
  if (!p.ready || p.kind != TC_SYRK) return cudaErrorInvalidValue;
  TcArgs a{};
  a.M = p.M;
  a.N = p.N;
  a.K = p.K;
  a.ntm = p.ntm;
  a.ntn = p.ntn;
  a.nkb = p.K / p.bk;
  a.kb_per_split = p.kb_per_split;
  a.Hp = Hp;
  a.err = err;
  return launch_any<TC_SYRK>(p, a, dim3(p.ntm * p.ntn, p.splits, 1), st);
}

}  // namespace nnc
