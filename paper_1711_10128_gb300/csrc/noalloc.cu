// trplk_project_noalloc: the projection h = BU^T v with no device allocation.
//
// Some callers cannot let a library allocate device memory.  A serving
// process that has planned the whole device in advance (its own pool holds
// all free memory, so a cudaMalloc would fail or fragment that plan) is one;
// a latency-critical loop that cannot afford the device-wide synchronisation
// a cudaMalloc or cudaFree may imply is another.  For them this entry point
// runs the same projection kernel as trplk_project, but its reduction scratch
// (per-CTA partial sums, the last-CTA ticket and a status word) lives in one
// file-scope __device__ array of fixed size, so the call needs no handle and
// allocates nothing.
//
// Limits and sharing: the array holds partial sums for at most
// kNoAllocCtas = 256 CTAs of 128 doubles each (256 KiB, plus 256 bytes for
// the ticket and status).  The call never launches more CTAs than that, so
// any n fits; w above 64 is rejected.  Every GPU that loads the library keeps
// this array until the process exits.  All calls share it and it keeps the
// previous call's contents: the ticket and status are cleared at the start
// of every call, and two calls whose kernels overlap on the GPU (different
// streams, or different host threads) race on it -- serialise them.
//
// The device address of the array is looked up once per device, on the first
// call with that device current (cudaGetSymbolAddress); make that first call
// before any stream capture begins.  Under lazy module loading (the CUDA
// runtime's default since 12.2) that first call is also what loads this
// file's module, and the load places the array and the kernels' code in
// device memory: the first call must come before the caller's pool takes the
// device's free memory (or the process runs with CUDA_MODULE_LOADING=EAGER).
// Later calls allocate nothing.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "launch.h"
#include "tallskinny.cuh"

namespace {

using namespace trplk;

constexpr int kNoAllocCtas = 256;
constexpr size_t kPartialDoubles = (size_t)kNoAllocCtas * kPartialStride;
constexpr size_t kScratchDoubles = kPartialDoubles + 32;   // + ticket and status words

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
double* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set-up once).
trplk_status scratch_address(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return TRPLK_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return TRPLK_ECUDA;
    }
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return TRPLK_OK;
}

constexpr size_t kSmemMax = 232448 - 1024;
constexpr size_t kSmemPerSM = 233472;

// One launch of the projection kernel instantiated for bases of at most MAXW
// columns (narrower instantiations keep their accumulators in registers).
template <typename S, int MAXW>
trplk_status launch_project(TSArgs<S>& a, cudaStream_t stream, int sms) {
  constexpr int TR = Tile<S>::TR;
  constexpr int kThreads = TR + 32;
  auto kern = ts_kernel<S, TS_PROJ, MAXW>;
  const size_t fixed = ts_smem_fixed<S>(0);
  const size_t stage = ts_stage_bytes<S>(1, a.w, 1);
  const int stages = (int)std::min<size_t>(4, (kSmemMax - fixed) / stage);
  if (stages < 1) return TRPLK_EINVAL;
  a.stages = stages;
  const size_t smem = fixed + (size_t)stages * stage;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax) != cudaSuccess) {
    cudaGetLastError();
    return TRPLK_ECUDA;
  }
  // CTAs per SM: the fewest allowed by shared memory, registers and threads
  const int by_smem = (int)std::max<size_t>(1, kSmemPerSM / (smem + 1024));
  const int by_regs = std::max(1, 65536 / (std::max(fa.numRegs, 1) * kThreads));
  const int per_sm = std::min(std::min(by_smem, by_regs), 2048 / kThreads);
  int grid = (int)std::min<int64_t>(a.ntiles, (int64_t)sms * per_sm);
  grid = std::min(grid, kNoAllocCtas);
  kern<<<grid, kThreads, smem, stream>>>(a);
  return cudaGetLastError() == cudaSuccess ? TRPLK_OK : TRPLK_ECUDA;
}

template <typename S>
trplk_status project_noalloc(int64_t ld, int w, const S* BU, const S* v, double* hout, cudaStream_t stream,
                             double* scratch) {
  constexpr int TR = Tile<S>::TR;
  TSArgs<S> a;
  memset(&a, 0, sizeof(a));
  a.mat[0] = BU;
  a.nmat = 1;
  a.vec[0] = v;
  a.nvec = 1;
  a.w = w;
  a.ld = ld;
  a.out0 = hout;
  a.ntiles = (int)(ld / TR);
  a.partials = scratch;
  a.pstride = kPartialStride;
  a.counter = reinterpret_cast<unsigned int*>(scratch + kPartialDoubles);
  a.status = reinterpret_cast<int*>(scratch + kPartialDoubles + 1);
  a.polls = kWaitPolls;
  a.kind = TS_PROJ;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return TRPLK_ECUDA;
  }
  // ticket and status start at zero on every call (the array keeps old contents)
  if (cudaMemsetAsync(scratch + kPartialDoubles, 0, 32 * sizeof(double), stream) != cudaSuccess) {
    cudaGetLastError();
    return TRPLK_ECUDA;
  }
  trplk_status st;
  if (w <= kMaxQ / 2)
    st = launch_project<S, kMaxQ / 2>(a, stream, sms);
  else if (w <= 3 * kMaxQ / 4)
    st = launch_project<S, 3 * kMaxQ / 4>(a, stream, sms);
  else
    st = launch_project<S, kMaxQ>(a, stream, sms);
  if (st != TRPLK_OK) return st;
  int flags = 0;
  if (cudaMemcpyAsync(&flags, a.status, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess) {
    cudaGetLastError();
    return TRPLK_ECUDA;
  }
  if (flags & kFlagTimeout) return TRPLK_ETIMEOUT;
  if (flags & kFlagNaN) return TRPLK_NAN;
  return TRPLK_OK;
}

}  // namespace

extern "C" trplk_status trplk_project_noalloc(int dtype, int64_t n, int64_t ld, int w, const void* BU, const void* v,
                                              double* hout, void* cuda_stream) {
  if (n < 1 || ld < n || ld % 256 != 0 || w < 1 || w > trplk::kMaxQ || !BU || !v || !hout) return TRPLK_EINVAL;
  if (dtype != TRPLK_F64 && dtype != TRPLK_F32) return TRPLK_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return TRPLK_ECUDA;
  }
  double* scratch = nullptr;
  trplk_status st = scratch_address(dev, &scratch);
  if (st != TRPLK_OK) return st;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  if (dtype == TRPLK_F64)
    return project_noalloc<double>(ld, w, static_cast<const double*>(BU), static_cast<const double*>(v), hout, stream,
                                   scratch);
  return project_noalloc<float>(ld, w, static_cast<const float*>(BU), static_cast<const float*>(v), hout, stream,
                                scratch);
}
