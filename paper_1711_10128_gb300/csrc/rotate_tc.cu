// Thick-restart rotation X = U Y on the tensor cores (tcgen05), FP32 data.
//
// Algorithm 1's restart forms X = U Y(:, 1:p_hat) (likewise A U Y, B U Y): a
// dense (n x w) (w x k) product, w <= 64, k <= 32.  Each 128-row tile of U is
// one tcgen05.mma problem D (128 x N) = A (128 x K) B^T with A = the U tile,
// B = Y^T (N = k rounded up to 16, K = w rounded up to 16), accumulated in
// FP32 in tensor memory.  The operands are BF16: every FP32 value u is split
// exactly into three BF16 parts u = u0 + u1 + u2 (8 significant bits each:
// u0 = bf16(u), u1 = bf16(u - u0), u2 = u - u0 - u1), Y (FP64) likewise to
// FP32 accuracy, and the six products u_a y_b with a + b <= 2 are summed,
// smallest first; the three dropped ones are below 2^-24 of the product.  The
// result keeps FP32 accuracy, while the CUDA cores only split and store (about
// eight instructions per element of U instead of k FMAs).
//
// Per CTA: one producer warp stages tiles of U with 1D bulk copies (one
// 512-byte copy per column segment) into STAGES shared buffers (full/empty
// mbarriers); four consumer warps (thread t <-> tile row t) split the tile
// into the three K-major operand buffers, thread 0 issues the MMAs and
// commits them to an mbarrier, and the four warps read D back from tensor
// memory (warp w owns lanes 32w..32w+31 = rows) and store X, column by
// column, coalesced.  Shared-memory operands use the canonical K-major layout
// without swizzle: 8-row x 16-byte core matrices, 128 bytes apart along K,
// rows of core matrices K/8 * 128 bytes apart.  Every wait is bounded; a CTA
// that gives up sets kFlagTimeout, drains its copies and MMAs, frees its
// tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "launch.h"
#include "tallskinny.cuh"

namespace trplk {

namespace {

constexpr int kRotRows = 128;               // rows per tile (MMA M)
constexpr int kRotThreads = kRotRows + 32;  // four consumer warps and a producer warp
constexpr int kRotMaxStages = 4;
constexpr uint32_t kTmemCols = 32;          // FP32 accumulator columns (N <= 32)

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

__device__ __forceinline__ void split3(float u, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  a = __float2bfloat16_rn(u);
  const float r = u - __bfloat162float(a);
  b = __float2bfloat16_rn(r);
  c = __float2bfloat16_rn(r - __bfloat162float(b));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
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

__global__ void __launch_bounds__(kRotThreads, 4) rotate_tc_kernel(RotArgs a) {
  grid_dependency_wait();
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kRotMaxStages], empty[kRotMaxStages], mma_bar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool producer = warp == 4;
  const int w = a.w, Kp = a.Kp, Np = a.Np;
  const uint32_t abytes = (uint32_t)kRotRows * Kp * 2, bbytes = (uint32_t)Np * Kp * 2;
  unsigned char* Abuf = smem;                      // the U tile's 3 parts, K-major
  unsigned char* Bbuf = smem + 3 * abytes;         // 3 parts of Y^T, K-major
  unsigned char* stage0 = Bbuf + 3 * bbytes;       // U tiles as staged: column c at c * 512 bytes
  const uint32_t stage_bytes = (uint32_t)w * kRotRows * 4;

  // Y^T parts: B row n = output column n, K index c = basis column c
  for (int e = tid; e < Np * Kp; e += blockDim.x) {
    const int n = e / Kp, c = e - n * Kp;
    const float y = (n < a.k && c < w) ? (float)a.Y[(int64_t)n * a.ldY + c] : 0.f;
    // FP64 y to three BF16 parts through its FP32 rounding plus the FP32 remainder's first part
    const double yd = (n < a.k && c < w) ? a.Y[(int64_t)n * a.ldY + c] : 0.0;
    const __nv_bfloat16 y0 = __float2bfloat16_rn(y);
    const double r1 = yd - (double)__bfloat162float(y0);
    const __nv_bfloat16 y1 = __float2bfloat16_rn((float)r1);
    const __nv_bfloat16 y2 = __float2bfloat16_rn((float)(r1 - (double)__bfloat162float(y1)));
    const uint32_t off = kmaj(n, c, Kp);
    *reinterpret_cast<__nv_bfloat16*>(Bbuf + off) = y0;
    *reinterpret_cast<__nv_bfloat16*>(Bbuf + bbytes + off) = y1;
    *reinterpret_cast<__nv_bfloat16*>(Bbuf + 2 * bbytes + off) = y2;
  }
  if (tid == 0) {
    s_abort = 0;
    for (int s = 0; s < a.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 4);
    }
    mbar_init(&mma_bar[0], 1);
    mbar_init(&mma_bar[1], 1);
    fence_mbar_init();
  }
  if (warp == 0) {
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
  int issued_upto = 0, mma_issued[2] = {0, 0};
  bool fail = false;
  if (producer) {
    for (int it = 0; it < my_tiles; ++it) {
      const int s = it % a.stages;
      if (it >= a.stages) {
        int ok = 1;
        if (lane == 0) {
          ok = 0;
          const uint32_t par = (uint32_t)(((it / a.stages) - 1) & 1);
          for (uint32_t i = 0; i < a.polls; ++i) {
            if (mbar_try_wait(&empty[s], par)) { ok = 1; break; }
            if (*abort_flag) break;
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          if (lane == 0) *abort_flag = 1;
          fail = true;
          break;
        }
      }
      const int64_t row0 = (int64_t)(blockIdx.x + it * gridDim.x) * kRotRows;
      unsigned char* st = stage0 + (size_t)s * stage_bytes;
      if (lane == 0) mbar_arrive_expect_tx(&full[s], stage_bytes);
      __syncwarp();
      for (int c = lane; c < w; c += 32)
        bulk_g2s(st + (size_t)c * kRotRows * 4, a.U + (int64_t)c * a.ld + row0, kRotRows * 4, &full[s]);
      issued_upto = it + 1;
    }
  } else {
    const int m = tid;   // tile row
    const uint32_t sbo = (uint32_t)(Kp / 8) * 128;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(Np >> 3) << 17) | ((uint32_t)(kRotRows >> 4) << 24);
    bool mma_bad = false;   // this warp gave up waiting for a tile's MMAs
    // split tile `it` (stage it % stages) into operand set `buf`, agree on
    // failure, issue its MMAs into accumulator `buf`; false: stop
    auto stage_and_issue = [&](int it, int buf) -> bool {   // buf: accumulator / barrier slot (0)
      const int s = it % a.stages;
      const bool ok = mbar_warp_wait(&full[s], (uint32_t)((it / a.stages) & 1), a.polls, abort_flag);
      const unsigned char* st = stage0 + (size_t)s * stage_bytes;
      unsigned char* Ab = Abuf;
      if (ok) {
        // this row's w values into the three K-major parts, eight columns at a time
        for (int c0 = 0; c0 < Kp; c0 += 8) {
          uint32_t p0[4], p1[4], p2[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = c0 + 2 * q;
            const float u0 = c < w ? reinterpret_cast<const float*>(st)[c * kRotRows + m] : 0.f;
            const float u1 = c + 1 < w ? reinterpret_cast<const float*>(st)[(c + 1) * kRotRows + m] : 0.f;
            __nv_bfloat16 a0, b0, c0_, a1, b1, c1;
            split3(u0, a0, b0, c0_);
            split3(u1, a1, b1, c1);
            p0[q] = pack2(a0, a1);
            p1[q] = pack2(b0, b1);
            p2[q] = pack2(c0_, c1);
          }
          const uint32_t off = kmaj(m, c0, Kp);
          *reinterpret_cast<uint4*>(Ab + off) = make_uint4(p0[0], p0[1], p0[2], p0[3]);
          *reinterpret_cast<uint4*>(Ab + abytes + off) = make_uint4(p1[0], p1[1], p1[2], p1[3]);
          *reinterpret_cast<uint4*>(Ab + 2 * abytes + off) = make_uint4(p2[0], p2[1], p2[2], p2[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      // release the stage; agree on failure; order the writes (and earlier
      // tensor-memory reads of this accumulator) before the MMAs
      __syncwarp();
      if (ok && lane == 0) mbar_arrive(&empty[s]);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      if (consumer_sync_or<kRotRows>(!ok || mma_bad)) {
        if (!ok && lane == 0) *abort_flag = 1;
        return false;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (m == 0) {
        // products u_a y_b, a + b <= 2, smallest first
        const int pa[6] = {1, 2, 0, 1, 0, 0}, pb[6] = {1, 0, 2, 0, 1, 0};
        const uint32_t dcol = tmem;
        bool first = true;
        for (int t = 0; t < 6; ++t)
          for (int kk = 0; kk < Kp / 16; ++kk) {
            const uint64_t ad = smem_desc(smem_addr(Ab + pa[t] * abytes) + kk * 256, 128, sbo);
            const uint64_t bd = smem_desc(smem_addr(Bbuf + pb[t] * bbytes) + kk * 256, 128, sbo);
            const uint32_t acc = first ? 0u : 1u;
            first = false;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
          }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_addr(&mma_bar[buf]))
                     : "memory");
      }
      ++mma_issued[buf];
      return true;
    };
    // one tile at a time: split, MMAs, drain (the CTAs sharing an SM overlap
    // one another's latencies).  `stop` comes only from the tiles' barriers,
    // so every consumer warp leaves the loop at the same tile; a warp that
    // gave up an MMA wait reports it at the next barrier (or ends with the
    // last tile)
    bool stop = false;
    for (int it = 0; it < my_tiles && !stop; ++it) {
      if (!stage_and_issue(it, 0)) {
        fail = true;
        stop = true;
        break;
      }
      if (!mbar_warp_wait(&mma_bar[0], (uint32_t)(it & 1), a.polls, abort_flag)) {
        if (lane == 0) *abort_flag = 1;
        mma_bad = true;
        fail = true;
        continue;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint32_t r[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const int64_t row0 = (int64_t)(blockIdx.x + it * gridDim.x) * kRotRows;
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < a.k) a.X[(int64_t)j * a.ld + row0 + m] = __uint_as_float(r[j]);
    }
  }
  grid_dependents_launch();
  // agree on a timeout; drain the copies and the MMAs in flight; free tensor memory
  if (fail) *abort_flag = 1;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (*abort_flag) {
    if (tid == 0) atomicOr(a.status, kFlagTimeout);
    if (producer && lane == 0) {
      for (int it = issued_upto - a.stages; it < issued_upto; ++it) {
        if (it < 0) continue;
        if (!mbar_wait_bounded(&full[it % a.stages], (uint32_t)((it / a.stages) & 1), kDrainPolls))
          atomicOr(a.status, kFlagDrain);
      }
    }
    for (int b = 0; b < 2; ++b)
      if (tid == 0 && mma_issued[b] > 0 &&
          !mbar_wait_bounded(&mma_bar[b], (uint32_t)((mma_issued[b] - 1) & 1), kDrainPolls))
        atomicOr(a.status, kFlagDrain);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

}  // namespace

bool rotate_tc_fits(int w, int k) { return w >= 1 && w <= kMaxQ && k >= 1 && k <= 32; }

// The CUDA-core rotation spends k FMAs per element of U, the tensor-core one
// a fixed split (about eight instructions per element) plus per-tile latency:
// measured on GB300, the tensor cores win once k >= 24 (k = 25: 123 against
// 150 us at n = 884,736, w = 50; k = 15..20: the CUDA cores win).
bool rotate_tc_preferred(int w, int k) { return rotate_tc_fits(w, k) && k >= 24; }

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
  const size_t fixed = 3 * (size_t)kRotRows * a.Kp * 2 + 3 * (size_t)a.Np * a.Kp * 2;
  const size_t stage = (size_t)w * kRotRows * 4;
  constexpr size_t kSmemMax = 232448 - 2048;
  // the most CTAs per SM (up to 4) that keep two stages each, then as many
  // stages as fit (up to kRotMaxStages)
  int per_sm = 1;
  for (int cand = 4; cand >= 1; --cand)
    if (fixed + 2 * stage + 2048 <= 233472 / cand) { per_sm = cand; break; }
  const size_t budget = std::min<size_t>(kSmemMax, 233472 / per_sm - 2048);
  a.stages = (int)std::min<size_t>(kRotMaxStages, (budget - fixed) / stage);
  if (a.stages < 1) throw Error(TRPLK_EINVAL, "tensor-core rotation: tile does not fit");
  const size_t smem = fixed + (size_t)a.stages * stage;
  smem_optin<rotate_tc_kernel>((int)kSmemMax, c.device);
  const int grid = (int)std::min<int64_t>(a.ntiles, (int64_t)c.sms * per_sm);
  // algorithmic bytes: U's w columns read once, X's k columns written once
  ProfScope ps(c, prof_kind<float>(PK_TS_ROT), (double)(w + k) * ld * sizeof(float));
  launch_dependent(rotate_tc_kernel, dim3(grid), dim3(kRotThreads), smem, c.stream, a);
  check_launch("rotate_tc_kernel");
}

}  // namespace trplk
