// The library handle: device context, workspace cache and host read-back
// buffer, shared by the translation units that implement the C ABI.
#pragma once
#include <algorithm>
#include <map>
#include <string>

#include "launch.h"

using namespace trplk;

// ---------------------------------------------------------------- handle
struct trplk_handle {
  Ctx ctx;
  Profiler prof;
  bool own_stream = false;
  std::string err;
  struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
  };
  std::map<std::string, Buf> bufs;
  std::map<std::string, std::string> layouts;   // workspace group -> layout key
  double* pinned = nullptr;   // host read-back area
  size_t pinned_bytes = 0;

  // A named device buffer of at least `bytes`, zero-filled when (re)allocated
  // or when `zero` is set.
  void* get(const std::string& name, size_t bytes, bool zero = false) {
    bytes = std::max<size_t>(bytes, 256);
    Buf& b = bufs[name];
    if (b.bytes < bytes) {
      if (b.p) cudaFree(b.p);
      b.p = nullptr;
      b.bytes = 0;
      cudaError_t e = cudaMalloc(&b.p, bytes);
      if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(TRPLK_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes for " + name + " failed");
      }
      b.bytes = bytes;
      TRPLK_CUDA_TRY(cudaMemsetAsync(b.p, 0, bytes, ctx.stream));
    } else if (zero) {
      TRPLK_CUDA_TRY(cudaMemsetAsync(b.p, 0, bytes, ctx.stream));
    }
    return b.p;
  }
  double* host(size_t count) {
    size_t bytes = count * sizeof(double);
    if (pinned_bytes < bytes) {
      if (pinned) cudaFreeHost(pinned);
      pinned = nullptr;
      TRPLK_CUDA_TRY(cudaMallocHost(&pinned, bytes));
      pinned_bytes = bytes;
    }
    return pinned;
  }
  void sync() { TRPLK_CUDA_TRY(cudaStreamSynchronize(ctx.stream)); }
  int read_status() {
    int s = 0;
    TRPLK_CUDA_TRY(cudaMemcpyAsync(&s, ctx.status, sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
    sync();
    return s;
  }
  void clear_status() { TRPLK_CUDA_TRY(cudaMemsetAsync(ctx.status, 0, sizeof(int), ctx.stream)); }
};


// SELL-32 copy of a device CSR (solver.cu); see attach_sell there.
void attach_sell(trplk_handle* h, DevCsr<double>& d, const std::string& tag, DevCsr<float>* f32);

// Run an ABI entry point body: set the device, map exceptions to statuses.
template <typename F>
trplk_status guarded(trplk_handle* h, F&& f) {
  if (!h) return TRPLK_EINVAL;
  h->err.clear();
  try {
    TRPLK_CUDA_TRY(cudaSetDevice(h->ctx.device));
    return f();
  } catch (const Error& e) {
    h->err = e.msg;
    if (e.code == TRPLK_ECUDA) cudaGetLastError();
    return e.code;
  } catch (const std::exception& e) {
    h->err = e.what();
    return TRPLK_ECUDA;
  }
}

// Preconditioner on A's lower pattern for trplk_solve (fsai.cu): kind 0
// classical FSAI, 1 learned FSAI (MLP weights on the host, 7-point grid
// dims), both M = G^T G; kind 2 IC(0), M = P_s^T P_s (ic0_apply).
struct FsaiPrecond {
  DevCsr<double> G, GT;
  DevCsr<float> Gf, GTf;
  bool ok = false;
  // kind 2: the IC(0) factor L (in G, L^T in GT), applied by Jacobi sweeps
  // with the reciprocal of its diagonal
  bool ic0 = false;
  double* dinv = nullptr;
  float* dinvf = nullptr;
};
FsaiPrecond build_fsai_precond(trplk_handle* h, const DevCsr<double>& A, int kind, const int32_t* dims,
                               const float* weights_host, bool bf16, bool need32);
