// Thick-restart rotation X = U Y on the tensor cores (tcgen05), FP32 data.
//
// Algorithm 1's restart forms X = U Y(:, 1:p_hat) (likewise A U Y, B U Y): a
// dense (n x w) (w x k) product, w <= 64, k <= 32.  Each 128-row tile of U is
// a set of tcgen05.mma problems D (128 x N) = A (128 x K) B^T with A = the U
// tile, B = Y^T (K = w rounded up to 16), accumulated in FP32 in tensor
// memory.  The operands are BF16: every FP32 value u is split exactly into
// three BF16 parts u = u0 + u1 + u2 (8 significant bits each: u0 = bf16(u),
// u1 = bf16(u - u0), u2 = u - u0 - u1), Y (FP64) likewise to FP32 accuracy,
// and the six products u_a y_b with a + b <= 2 are summed, smallest first;
// the three dropped ones are below 2^-24 of the product.  The parts of Y^T are
// stacked along N (Np = k rounded up to 16): u0 [y0 y1 y2], u1 [y0 y1] and
// u2 y0 are three MMAs per K step, each into its own columns.  The result keeps
// FP32 accuracy, while the CUDA cores only split and store (about six
// instructions per element of U instead of k FMAs).
//
// Per CTA (one per SM), warp-specialised, every hand-off an mbarrier:
//  * a producer warp stages tiles of U (128 rows x w columns) with one 2D
//    tensor copy each into STAGES shared buffers (full/empty);
//  * eight split warps (two threads per tile row, alternate eight-column
//    chunks) split the staged tile into one of three operand sets (three
//    K-major BF16 parts each; opfull), after the MMAs of the tile that last
//    used that set have completed (opempty);
//  * an MMA warp (one elected lane) issues the tile's products into one of
//    two FP32 accumulators in tensor memory, once the epilogue has drained it
//    (accempty), and commits them to opempty and mmadone;
//  * four epilogue warps (warp 8 + q <-> tensor-memory lanes 32q..32q+31)
//    read the accumulator back, sum its six column blocks and store X,
//    column by column, coalesced.
// So the split of tile i+1, the MMAs of tile i and the epilogue of tile i-1
// overlap, and the copies run STAGES tiles ahead.  Shared-memory operands use
// the canonical K-major layout without swizzle: 8-row x 16-byte core
// matrices, 128 bytes apart along K, rows of core matrices K/8 * 128 bytes
// apart.  Every wait is bounded; a CTA that gives up sets kFlagTimeout,
// drains its copies and MMAs, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "launch.h"
#include "tallskinny.cuh"

namespace trplk {

namespace {

constexpr int kRotRows = 128;               // rows per tile (MMA M)
constexpr int kSplitWarps = 8, kEpiWarps = 4;   // two split threads per tile row
constexpr int kOpBufs = 3;                      // operand sets in flight
constexpr int kProdWarp = kSplitWarps + kEpiWarps, kMmaWarp = kProdWarp + 1;
constexpr int kRotThreads = (kMmaWarp + 1) * 32;
constexpr int kRotMaxStages = 8;
constexpr uint32_t kTmemCols = 512;         // two FP32 accumulators of 6 Np <= 192 columns, 256 apart
constexpr size_t kRotSmemFloor = 120 * 1024; // more than half an SM's shared memory: one CTA per SM

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  // start address, leading (K) and stride (M/N) byte offsets in 16-byte units,
  // descriptor version 1 at bits 46-48, no swizzle
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// K-major offset (bytes) of element (r, c) in a buffer of rows x Kp bf16
__device__ __forceinline__ uint32_t kmaj(int r, int c, int Kp) {
  return (uint32_t)((r >> 3) * (Kp / 8) * 128 + (c >> 3) * 128 + (r & 7) * 16 + (c & 7) * 2);
}

// (u0, u1) -> three packed BF16 pairs with u = p0 + p1 + p2 exactly: each
// part is the round-to-nearest BF16 of what the earlier parts leave, and
// every remainder is exact in FP32.  Word layout: u0 in the low half (the
// lower K index comes first in memory).
__device__ __forceinline__ void split3x2(float u0, float u1, uint32_t& p0, uint32_t& p1, uint32_t& p2) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(u0, u1);
  const float r0 = u0 - __low2float(h), r1 = u1 - __high2float(h);
  const __nv_bfloat162 m = __floats2bfloat162_rn(r0, r1);
  const __nv_bfloat162 l = __floats2bfloat162_rn(r0 - __low2float(m), r1 - __high2float(m));
  p0 = *reinterpret_cast<const uint32_t*>(&h);
  p1 = *reinterpret_cast<const uint32_t*>(&m);
  p2 = *reinterpret_cast<const uint32_t*>(&l);
}

// 32 consecutive FP32 columns of tensor memory, this warp's 32 lanes (one
// row each), into r; complete after tcgen05.wait::ld
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

struct RotArgs {
  const float* U;
  int64_t ld;
  int w, k, ntiles, stages, Kp, Np;
  const double* Y;
  int ldY;
  float* X;
  int* status;
  uint32_t polls;
};

__global__ void __launch_bounds__(kRotThreads, 1) rotate_tc_kernel(const __grid_constant__ CUtensorMap umap, RotArgs a) {
  grid_dependency_wait();
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kRotMaxStages], empty[kRotMaxStages], opfull[kOpBufs], opempty[kOpBufs],
      mmadone[2], accempty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int w = a.w, Kp = a.Kp, Np = a.Np, S = a.stages;
  const uint32_t abytes = (uint32_t)kRotRows * Kp * 2, bbytes = (uint32_t)Np * Kp * 2;
  unsigned char* Aop = smem;                       // kOpBufs operand sets, three parts each, K-major
  unsigned char* Bop = smem + 3 * kOpBufs * abytes;   // three parts of Y^T, K-major
  unsigned char* stage0 = Bop + 3 * bbytes;        // U tiles as staged: column c at c * 512 bytes
  const uint32_t stage_bytes = (uint32_t)w * kRotRows * 4;

  // Y^T parts: B row n = output column n, K index c = basis column c; the
  // FP64 y through its FP32 rounding plus the FP32 remainder's first part
  for (int e = tid; e < Np * Kp; e += blockDim.x) {
    const int n = e / Kp, c = e - n * Kp;
    const double yd = (n < a.k && c < w) ? a.Y[(int64_t)n * a.ldY + c] : 0.0;
    const __nv_bfloat16 y0 = __float2bfloat16_rn((float)yd);
    const double r1 = yd - (double)__bfloat162float(y0);
    const __nv_bfloat16 y1 = __float2bfloat16_rn((float)r1);
    const __nv_bfloat16 y2 = __float2bfloat16_rn((float)(r1 - (double)__bfloat162float(y1)));
    const uint32_t off = kmaj(n, c, Kp);
    *reinterpret_cast<__nv_bfloat16*>(Bop + off) = y0;
    *reinterpret_cast<__nv_bfloat16*>(Bop + bbytes + off) = y1;
    *reinterpret_cast<__nv_bfloat16*>(Bop + 2 * bbytes + off) = y2;
  }
  if (tid == 0) {
    s_abort = 0;
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kSplitWarps);
    }
    for (int b = 0; b < kOpBufs; ++b) {
      mbar_init(&opfull[b], kSplitWarps);
      mbar_init(&opempty[b], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&mmadone[b], 1);
      mbar_init(&accempty[b], kEpiWarps);
    }
    fence_mbar_init();
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the B parts, for the tensor core
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  volatile int* abort_flag = &s_abort;

  const int my_tiles = (a.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  int issued = 0, mma_issued = 0;
  bool fail = false;
  if (warp == kProdWarp) {
    for (int it = 0; it < my_tiles; ++it) {
      const int s = it % S;
      if (it >= S && !mbar_warp_wait(&empty[s], (uint32_t)(((it / S) - 1) & 1), a.polls, abort_flag)) {
        fail = true;
        break;
      }
      // one 2D tensor copy: rows row0..row0+127 of all w columns, column-major
      const int row0 = (int)((blockIdx.x + it * gridDim.x) * kRotRows);
      if (lane == 0) {
        mbar_arrive_expect_tx(&full[s], stage_bytes);
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
            "[%4];" ::"r"(smem_addr(stage0 + (size_t)s * stage_bytes)),
            "l"(reinterpret_cast<uint64_t>(&umap)), "r"(row0), "r"(0), "r"(smem_addr(&full[s]))
            : "memory");
      }
      __syncwarp();
      issued = it + 1;
    }
  } else if (warp < kSplitWarps) {
    const int m = tid & (kRotRows - 1), half = tid >> 7;   // tile row; which eight-column chunks
    for (int it = 0; it < my_tiles; ++it) {
      const int s = it % S, ob = it % kOpBufs;
      if (!mbar_warp_wait(&full[s], (uint32_t)((it / S) & 1), a.polls, abort_flag) ||
          (it >= kOpBufs &&
           !mbar_warp_wait(&opempty[ob], (uint32_t)(((it / kOpBufs) - 1) & 1), a.polls, abort_flag))) {
        fail = true;
        break;
      }
      const float* st = reinterpret_cast<const float*>(stage0 + (size_t)s * stage_bytes) + m;
      unsigned char* Ab = Aop + (size_t)ob * 3 * abytes;
      // this row's values into the three K-major parts, eight columns at a time
      for (int c0 = 8 * half; c0 < Kp; c0 += 16) {
        float u[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) u[q] = c0 + q < w ? st[(c0 + q) * kRotRows] : 0.f;
        uint32_t p0[4], p1[4], p2[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) split3x2(u[2 * q], u[2 * q + 1], p0[q], p1[q], p2[q]);
        const uint32_t off = kmaj(m, c0, Kp);
        *reinterpret_cast<uint4*>(Ab + off) = make_uint4(p0[0], p0[1], p0[2], p0[3]);
        *reinterpret_cast<uint4*>(Ab + abytes + off) = make_uint4(p1[0], p1[1], p1[2], p1[3]);
        *reinterpret_cast<uint4*>(Ab + 2 * abytes + off) = make_uint4(p2[0], p2[1], p2[2], p2[3]);
      }
      // the operands, for the tensor core; the stage is free again
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&empty[s]);
        mbar_arrive(&opfull[ob]);
      }
    }
  } else if (warp == kMmaWarp) {
    const uint32_t sbo = (uint32_t)(Kp / 8) * 128;
    // u0 [y0 y1 y2], u1 [y0 y1] and u2 y0, each in its own columns: the three
    // parts of Y^T are stacked along N in one K-major buffer, so each part of U
    // is one MMA per K step, and the six products u_a y_b with a + b <= 2 land
    // in six column blocks, which the epilogue sums smallest first
    const uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kRotRows >> 4) << 24);
    for (int it = 0; it < my_tiles; ++it) {
      const int b = it & 1, ob = it % kOpBufs;
      if (!mbar_warp_wait(&opfull[ob], (uint32_t)((it / kOpBufs) & 1), a.polls, abort_flag) ||
          (it >= 2 && !mbar_warp_wait(&accempty[b], (uint32_t)(((it >> 1) - 1) & 1), a.polls, abort_flag))) {
        fail = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (lane == 0) {
        const uint32_t abase = smem_addr(Aop + (size_t)ob * 3 * abytes);
        const uint64_t bd0 = smem_desc(smem_addr(Bop), 128, sbo);
        for (int g = 0; g < 3; ++g) {
          // part g of U times the first 3 - g parts of Y^T, in its own columns
          const uint32_t dcol = tmem + (uint32_t)b * 256 + (uint32_t)(g == 0 ? 0 : g == 1 ? 3 * Np : 5 * Np);
          const uint32_t idesc = idesc0 | ((uint32_t)(((3 - g) * Np) >> 3) << 17);
          const uint64_t ad0 = smem_desc(abase + g * abytes, 128, sbo);
          for (int kk = 0; kk < Kp / 16; ++kk) {
            // 256 bytes along K = 16 in the start-address field
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
                "l"(ad0 + (uint64_t)(kk * 16)), "l"(bd0 + (uint64_t)(kk * 16)), "r"(idesc), "r"(kk > 0 ? 1u : 0u));
          }
        }
        // operand set free (for the split), accumulator full (for the epilogue)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_addr(&opempty[ob]))
                     : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_addr(&mmadone[b]))
                     : "memory");
      }
      __syncwarp();
      mma_issued = it + 1;
    }
  } else {
    const int q = warp - kSplitWarps;   // tensor-memory lanes 32q..32q+31 = tile rows
    for (int it = 0; it < my_tiles; ++it) {
      const int b = it & 1;
      if (!mbar_warp_wait(&mmadone[b], (uint32_t)((it >> 1) & 1), a.polls, abort_flag)) {
        fail = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // column blocks (Np wide): A0 A1 A2 = u0 y0, u0 y1, u0 y2; B0 B1 = u1 y0,
      // u1 y1; C0 = u2 y0; x = ((C0 + B1) + A2) + (B0 + A1)) + A0
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)b * 256;
      float x[32];
      uint32_t r0[32], r1[32], r2[32];
      if (Np == 32) {
        tmem_ld32(taddr + 160, r0);   // C0
        tmem_ld32(taddr + 128, r1);   // B1
        tmem_ld32(taddr + 64, r2);    // A2
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 32; ++j)
          x[j] = (__uint_as_float(r0[j]) + __uint_as_float(r1[j])) + __uint_as_float(r2[j]);
        tmem_ld32(taddr + 96, r0);    // B0
        tmem_ld32(taddr + 32, r1);    // A1
        tmem_ld32(taddr, r2);         // A0
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 32; ++j)
          x[j] = (x[j] + (__uint_as_float(r0[j]) + __uint_as_float(r1[j]))) + __uint_as_float(r2[j]);
      } else {
        tmem_ld32(taddr + 64, r0);    // B1, C0
        tmem_ld32(taddr + 32, r1);    // A2, B0
        tmem_ld32(taddr, r2);         // A0, A1
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j)
          x[j] = (((__uint_as_float(r0[16 + j]) + __uint_as_float(r0[j])) + __uint_as_float(r1[j])) +
                  (__uint_as_float(r1[16 + j]) + __uint_as_float(r2[16 + j]))) +
                 __uint_as_float(r2[j]);
      }
      // the accumulator is free for the tile after next
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&accempty[b]);
      float* xp = a.X + (int64_t)(blockIdx.x + it * gridDim.x) * kRotRows + q * 32 + lane;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        if (j < a.k) *xp = x[j];
        xp += a.ld;
      }
    }
  }
  grid_dependents_launch();
  // agree on a timeout; drain the copies and the MMAs in flight; free tensor memory
  if (fail) *abort_flag = 1;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (*abort_flag) {
    if (tid == 0) atomicOr(a.status, kFlagTimeout);
    if (warp == kProdWarp && lane == 0) {
      for (int it = issued - S; it < issued; ++it) {
        if (it < 0) continue;
        if (!mbar_wait_bounded(&full[it % S], (uint32_t)((it / S) & 1), kDrainPolls)) atomicOr(a.status, kFlagDrain);
      }
    }
    if (warp == kMmaWarp && lane == 0 && mma_issued > 0) {
      const int it = mma_issued - 1;   // the last commit tracks every earlier MMA
      if (!mbar_wait_bounded(&mmadone[it & 1], (uint32_t)((it >> 1) & 1), kDrainPolls))
        atomicOr(a.status, kFlagDrain);
    }
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == kMmaWarp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

}  // namespace

// The driver's tensor-map encoder, through the runtime (no link against the
// driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

bool rotate_tc_fits(int w, int k) { return w >= 1 && w <= kMaxQ && k >= 1 && k <= 32; }

// The CUDA-core rotation spends k FMAs per element of U, the tensor-core one
// a fixed split (about six instructions per element) and 3 w/16 MMAs per
// 128-row tile.  Measured on GB300 (microseconds per launch, tensor against
// CUDA cores): n = 4,117,504: w = 40, k = 20: 232 / 365; w = 64, k = 32: 289 /
// 946; w = 24, k = 16: 216 / 188; n = 2,097,152: w = 39, k = 15: 118 / 175;
// w = 16, k = 6: 91 / 40; n = 884,736, w = 50, k = 25: 67 / 150.  The tensor
// cores win once w k >= 480.
bool rotate_tc_preferred(int w, int k) { return rotate_tc_fits(w, k) && w * k >= 480; }

void rotate_tc(const Ctx& c, int64_t ld, int w, int k, const float* U, const double* Y, int ldY, float* X) {
  if (!rotate_tc_fits(w, k) || ld % kRotRows != 0) throw Error(TRPLK_EINVAL, "tensor-core rotation: bad shape");
  RotArgs a;
  a.U = U;
  a.ld = ld;
  a.w = w;
  a.k = k;
  a.ntiles = (int)(ld / kRotRows);
  a.Kp = (w + 15) / 16 * 16;
  a.Np = k <= 16 ? 16 : 32;
  a.Y = Y;
  a.ldY = ldY;
  a.X = X;
  a.status = c.status;
  a.polls = c.wait_polls;
  const size_t fixed = 3 * kOpBufs * (size_t)kRotRows * a.Kp * 2 + 3 * (size_t)a.Np * a.Kp * 2;
  const size_t stage = (size_t)w * kRotRows * 4;
  constexpr size_t kSmemMax = 232448 - 2048;
  // one CTA per SM; as many staged tiles as fit (at least two, at most kRotMaxStages)
  a.stages = (int)std::min<size_t>(kRotMaxStages, (kSmemMax - fixed) / stage);
  if (a.stages < 2) throw Error(TRPLK_EINVAL, "tensor-core rotation: tile does not fit");
  const size_t smem = std::max(fixed + (size_t)a.stages * stage, kRotSmemFloor);
  smem_optin<rotate_tc_kernel>((int)kSmemMax, c.device);
  // U as a 2D tensor: ld rows (innermost, FP32) by w columns, tiles of 128 rows
  // by w columns; rows and column strides are multiples of 16 bytes (ld is a
  // multiple of 256), and every tile starts at a multiple of 128 rows
  CUtensorMap umap;
  const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  const cuuint64_t gdim[2] = {(cuuint64_t)ld, (cuuint64_t)w};
  const cuuint64_t gstride[1] = {(cuuint64_t)ld * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kRotRows, (cuuint32_t)w};
  const cuuint32_t estride[2] = {1, 1};
  if (!encode ||
      encode(&umap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(U), gdim, gstride, box, estride,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    throw Error(TRPLK_EINVAL, "tensor-core rotation: tensor map for U rejected");
  const int grid = (int)std::min<int64_t>(a.ntiles, (int64_t)c.sms);
  // algorithmic bytes: U's w columns read once, X's k columns written once
  ProfScope ps(c, prof_kind<float>(PK_TS_ROT), (double)(w + k) * ld * sizeof(float));
  launch_dependent(rotate_tc_kernel, dim3(grid), dim3(kRotThreads), smem, c.stream, umap, a);
  check_launch("rotate_tc_kernel");
}

}  // namespace trplk
