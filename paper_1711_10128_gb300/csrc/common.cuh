// Internal helpers shared by the CUDA translation units of libtrplk.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdio>
#include <mutex>
#include <string>
#include <utility>

#include "trplk.h"

namespace trplk {

// ----------------------------------------------------------------- constants
constexpr int kMaxQ = 64;          // largest supported basis size q
constexpr int kMaxK = 32;          // largest supported thick-restart size p_hat
constexpr int kMaxPartials = 1024; // CTA partial sums a reduction may hold

// Error flags a kernel may raise in the device status word.
enum : int {
  kFlagTimeout = 1,     // a bounded wait on an mbarrier ran out
  kFlagNaN = 2,         // a NaN/Inf reached a reduction
  kFlagBreakdown = 4,   // Lanczos vector fell into the span of the basis
  kFlagNotSPD = 8,      // x^T B x <= 0 seen
  kFlagJacobi = 16,     // Rayleigh-Ritz eigensolver did not converge
  kFlagDrain = 32,      // after a timeout, an issued bulk copy did not land within kDrainPolls
};

// Polls of one bounded mbarrier wait in the streaming passes (the default;
// a handle may lower it to exercise the timeout path), and of the wait for
// the copies still in flight when a CTA gives up.  Copies from valid device
// memory always land, so the second bound is a backstop only.
constexpr uint32_t kWaitPolls = 1u << 22;
constexpr uint32_t kDrainPolls = 1u << 26;

// Storage traits.  Rows are tiled in TR-row tiles; a CTA has TR threads so a
// thread owns one row of a tile.  One tile column is TR * sizeof(S) = 1 KiB.
template <typename S> struct Tile;
template <> struct Tile<double> { static constexpr int TR = 128; };
template <> struct Tile<float> { static constexpr int TR = 256; };

__host__ __device__ inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// ----------------------------------------------------------------- host errors
struct Status {
  trplk_status code = TRPLK_OK;
  std::string msg;
};

#define TRPLK_CUDA_TRY(expr)                                                      \
  do {                                                                            \
    cudaError_t _e = (expr);                                                      \
    if (_e != cudaSuccess) {                                                      \
      char _b[512];                                                               \
      snprintf(_b, sizeof(_b), "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), \
               __FILE__, __LINE__);                                               \
      throw ::trplk::Error(TRPLK_ECUDA, _b);                                      \
    }                                                                             \
  } while (0)

struct Error {
  trplk_status code;
  std::string msg;
  Error(trplk_status c, std::string m) : code(c), msg(std::move(m)) {}
};

// Opt kernel `Kernel` into `bytes` of dynamic shared memory on `device`, once
// per (kernel, device): the attribute is kept per device, and a process may
// hold handles on several GPUs.  Lock-free after the first call.
template <auto Kernel>
void smem_optin(int bytes, int device) {
  static std::atomic<unsigned long long> done{0};
  static std::mutex mu;
  const unsigned long long bit = 1ull << (device & 63);
  if (done.load(std::memory_order_acquire) & bit) return;
  std::lock_guard<std::mutex> g(mu);
  if (done.load(std::memory_order_relaxed) & bit) return;
  const cudaError_t e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(TRPLK_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
  }
  done.fetch_or(bit, std::memory_order_release);
}

inline void check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    throw Error(TRPLK_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  }
}

// ----------------------------------------------------------------- device: compensated dot product
// FP64-class accumulation of products of floats on the FP32 pipes (the FP64
// pipe of this GPU runs at 1/58 of the FP32 rate).  This is Dot2 of Ogita,
// Rump and Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 26,
// 2005): each product is split exactly into h + r by an FMA, h enters the
// running sum p through Knuth's error-free TwoSum, and all rounding errors are
// gathered in a second float s.  The value p + s is read out in FP64, so the
// error is about (n u)^2 sum|a_i b_i| with u = 2^-24, n the terms per thread.
// The streaming passes use its blocked form fma4 (below), which rounds four
// products together before the exact TwoSum.
// The _rn intrinsics keep the compiler from contracting these operations into
// FMAs, which would break the error-free transforms.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  float t = __fadd_rn(a, b);
  float bb = __fsub_rn(t, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(t, bb)), __fsub_rn(b, bb));
  s = t;
}

// ----------------------------------------------------------------- accumulators
// Acc<S>: FP64-class accumulation of products of S values.
template <typename S> struct Acc;
template <> struct Acc<double> {
  double v;
  __device__ __forceinline__ void zero() { v = 0.0; }
  __device__ __forceinline__ void fma(double a, double b) { v = ::fma(a, b, v); }
  __device__ __forceinline__ void fma4(double a0, double b0, double a1, double b1, double a2, double b2, double a3,
                                       double b3) {
    v = ::fma(a0, b0, v);
    v = ::fma(a1, b1, v);
    v = ::fma(a2, b2, v);
    v = ::fma(a3, b3, v);
  }
  __device__ __forceinline__ void add(double a) { v += a; }
  __device__ __forceinline__ double value() const { return v; }
  __device__ __forceinline__ void shfl_down_add(int off) { v += __shfl_down_sync(0xffffffffu, v, off); }
};
template <> struct Acc<float> {
  float p, s;
  __device__ __forceinline__ void zero() { p = 0.f; s = 0.f; }
  __device__ __forceinline__ void fma(float a, float b) {
    float h = __fmul_rn(a, b);
    float r = __fmaf_rn(a, b, -h);
    float q;
    two_sum(p, h, p, q);
    s = __fadd_rn(s, __fadd_rn(q, r));
  }
  __device__ __forceinline__ void add(float a) {
    float q;
    two_sum(p, a, p, q);
    s += q;
  }
  // Four consecutive products: their sum in FP32 (a block of four roundings),
  // added exactly by TwoSum.  11 instructions for four products instead of
  // 40; the block errors are at most 4u times the block's sum of |a b|, and
  // random in sign across the many blocks of a long dot product, so the sum
  // keeps FP64-class accuracy in practice (worst case 4u sum |a b|).
  __device__ __forceinline__ void fma4(float a0, float b0, float a1, float b1, float a2, float b2, float a3,
                                       float b3) {
    float blk = __fmul_rn(a0, b0);
    blk = __fmaf_rn(a1, b1, blk);
    blk = __fmaf_rn(a2, b2, blk);
    blk = __fmaf_rn(a3, b3, blk);
    add(blk);
  }
  __device__ __forceinline__ double value() const { return (double)p + (double)s; }
  __device__ __forceinline__ void shfl_down_add(int off) {
    float po = __shfl_down_sync(0xffffffffu, p, off);
    float so = __shfl_down_sync(0xffffffffu, s, off);
    float q;
    two_sum(p, po, p, q);
    s += so + q;
  }
};

// AccFast<S>: plain accumulation in S.  Used only for the first CGS pass of
// the FP32 path, whose rounding errors the second (compensated) pass removes.
template <typename S> struct AccFast;
template <> struct AccFast<double> : Acc<double> {};
template <> struct AccFast<float> {
  float p;
  __device__ __forceinline__ void zero() { p = 0.f; }
  __device__ __forceinline__ void fma(float a, float b) { p = fmaf(a, b, p); }
  __device__ __forceinline__ void fma4(float a0, float b0, float a1, float b1, float a2, float b2, float a3,
                                       float b3) {
    p = fmaf(a0, b0, p);
    p = fmaf(a1, b1, p);
    p = fmaf(a2, b2, p);
    p = fmaf(a3, b3, p);
  }
  __device__ __forceinline__ double value() const { return (double)p; }
  __device__ __forceinline__ void shfl_down_add(int off) { p += __shfl_down_sync(0xffffffffu, p, off); }
};

// Part<S>: one CTA's partial sum of a projection, as the grid reduction
// moves it.  FP64 path: the double.  FP32 path: the compensated pair (p, s)
// itself, packed into the 8 bytes of a double slot, and added pairwise by
// TwoSum in FP32 -- the last CTA's sum over every CTA then runs on the FP32
// pipe instead of the FP64 pipe (64 times slower on this GPU); its rounding
// (about u^2 times the sum of |p|) stays far below the partials' own.
template <typename S> struct Part;
template <> struct Part<double> {
  double v;
  __device__ __forceinline__ void zero() { v = 0.0; }
  __device__ __forceinline__ void add(const Part& o) { v += o.v; }
  __device__ __forceinline__ double value() const { return v; }
  __device__ __forceinline__ void store(double* slot) const { *slot = v; }
  __device__ __forceinline__ void load(const double* slot) { v = *slot; }
  __device__ __forceinline__ void shfl_down_add(int off) { v += __shfl_down_sync(0xffffffffu, v, off); }
  __device__ __forceinline__ static Part of(const Acc<double>& a) { return Part{a.v}; }
};
template <> struct Part<float> {
  float p, s;
  __device__ __forceinline__ void zero() { p = 0.f; s = 0.f; }
  __device__ __forceinline__ void add(const Part& o) {
    float e;
    two_sum(p, o.p, p, e);
    s = __fadd_rn(s, __fadd_rn(e, o.s));
  }
  __device__ __forceinline__ double value() const { return (double)p + (double)s; }
  __device__ __forceinline__ void store(double* slot) const { *reinterpret_cast<float2*>(slot) = make_float2(p, s); }
  __device__ __forceinline__ void load(const double* slot) {
    const float2 v = *reinterpret_cast<const float2*>(slot);
    p = v.x;
    s = v.y;
  }
  __device__ __forceinline__ void shfl_down_add(int off) {
    Part o;
    o.p = __shfl_down_sync(0xffffffffu, p, off);
    o.s = __shfl_down_sync(0xffffffffu, s, off);
    add(o);
  }
  __device__ __forceinline__ static Part of(const Acc<float>& a) { return Part{a.p, a.s}; }
  __device__ __forceinline__ static Part of(const AccFast<float>& a) { return Part{a.p, 0.f}; }
};

// ----------------------------------------------------------------- device: mbarrier + bulk copy
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: gives up after `limit` polls (each poll itself suspends for a
// hardware-chosen time) and reports false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit = kWaitPolls) {
  for (uint32_t i = 0; i < limit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
  }
  return false;
}

// Warp-uniform bounded wait: every lane polls until all lanes have seen the
// phase complete (true), any lane sees *abort set, or `limit` rounds have
// passed (false).  All lanes leave after the same round with the same result,
// so the warp stays converged whether the wait succeeds or gives up.  A
// completed phase stays visible until the waiting warp itself releases the
// stage, so a lane that has seen it need not poll again.
__device__ __forceinline__ bool mbar_warp_wait(uint64_t* bar, uint32_t parity, uint32_t limit,
                                               const volatile int* abort) {
  bool done = false;
  for (uint32_t i = 0; i < limit; ++i) {
    if (!done) done = mbar_try_wait(bar, parity);
    if (__all_sync(0xffffffffu, done)) return true;
    if (__any_sync(0xffffffffu, *abort != 0)) return false;
  }
  return false;
}

// 1D bulk copy global -> shared (TMA engine), completion counted on `bar`.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// ----------------------------------------------------------------- device: dependent launch
// Kernels launched with launch_dependent() may start before the previous
// kernel of the stream has finished; they must call grid_dependency_wait()
// before touching global memory (it returns once that kernel has completed
// and its writes are visible).  grid_dependents_launch() lets the next such
// kernel be scheduled as this one's CTAs exit.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependents_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch `kernel` on `stream` as a programmatic dependent of the stream's
// previous kernel (the kernel must begin with grid_dependency_wait()).
template <typename... KArgs, typename... Args>
void launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                      Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// The same launch in plain stream order (the kernel starts after the previous
// one has finished).
template <typename... KArgs, typename... Args>
void launch_plain(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                  Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cfg.numAttrs = 0;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ----------------------------------------------------------------- device: grid reduction
// Deterministic two-stage reduction: every CTA writes `n` partial values, the
// last CTA to finish sums them in CTA order.  `counter` must be zero on entry
// and is reset by the last CTA.  Returns true in the last CTA (all threads).
__device__ __forceinline__ bool last_block_arrive(unsigned int* counter) {
  __shared__ unsigned int s_ticket;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_ticket = atomicAdd(counter, 1u);
  __syncthreads();
  bool last = (s_ticket == gridDim.x - 1);
  if (last) __threadfence();
  return last;
}

}  // namespace trplk
