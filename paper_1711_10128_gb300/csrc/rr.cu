// Rayleigh-Ritz eigensolver for the small projection T (Algorithm 1,
// 'compute eigenpairs of T, T = Y Theta Y^T').
//
// One CTA, T (w <= 64) in shared memory.  The cyclic Jacobi method with the
// round-robin (tournament) ordering: each round rotates w/2 disjoint index
// pairs at once -- three parallel phases (rotation angles, column updates
// A J and V J, row updates J^T A) -- and w - 1 rounds make a sweep over all
// pairs.  Rotations use the symmetric 2x2 Schur decomposition of Golub and
// Van Loan (Sec. 8.5); the rotated pair's off-diagonal entry is set to zero.
// Off-diagonal norms are summed directly, never as a difference of norms.
//
// The FP64 pipe of this GPU retires 2 FMAs per clock per SM (the FP32 pipe
// 128), so the sweeps run in two precisions:
//  1. FP32 sweeps on fp32(T) until its off-diagonal norm is <= 1e-6 ||T||_F,
//     accumulating the rotations into V (orthogonal to about 1e-7);
//  2. V is promoted to FP64 and re-orthonormalised by two Gram-Schmidt passes
//     per column, then B = V^T T V is formed in FP64 (an exact orthogonal
//     similarity up to FP64 rounding) -- nearly diagonal;
//  3. FP64 sweeps on B (quadratic convergence: usually one or two) until its
//     off-diagonal norm is <= 1e-15 ||T||_F, accumulating into V.
// Eigenvalues are then sorted ascending (stable rank sort) and every
// eigenvector is signed so its largest-magnitude entry, the first such, is
// positive.
#include <cmath>

#include "launch.h"

namespace trplk {

namespace {

constexpr int kThreads = 256;

template <typename T>
__device__ __forceinline__ void sym_schur2(T app, T aqq, T apq, T skip, T& c, T& s) {
  if (!(fabs(apq) > skip)) {
    c = 1;
    s = 0;
    return;
  }
  const T tau = (aqq - app) / (2 * apq);
  const T t = tau >= 0 ? 1 / (tau + sqrt(1 + tau * tau)) : -1 / (-tau + sqrt(1 + tau * tau));
  c = 1 / sqrt(1 + t * t);
  s = t * c;
}

struct RotShared {
  int p[kMaxQ / 2], q[kMaxQ / 2];
  double c[kMaxQ / 2], s[kMaxQ / 2];
  double red[kThreads / 32];
  double val;
};

// sum over the CTA; result valid in every thread
__device__ double block_sum(double v, RotShared& sh) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh.red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kThreads / 32; ++i) t += sh.red[i];
    sh.val = t;
  }
  __syncthreads();
  return sh.val;
}

template <typename T>
__device__ double off_norm(const T* A, int w, int ld, RotShared& sh) {
  double o = 0.0;
  for (int e = threadIdx.x; e < w * w; e += kThreads) {
    const int i = e / w, j = e - i * w;
    if (i != j) {
      const double a = (double)A[i * ld + j];
      o += a * a;
    }
  }
  return sqrt(block_sum(o, sh));
}

// Jacobi sweeps on the symmetric A (row-major, ld), rotations accumulated into
// V.  Stops when the off-diagonal norm is <= tol * fro.  Returns true if it did.
template <typename T>
__device__ bool jacobi_sweeps(T* A, T* V, int w, int ld, double fro, double tol, double skip_rel, int max_sweeps,
                              RotShared& sh) {
  const int tid = threadIdx.x;
  const int wp = w + (w & 1);   // even number of slots; slot w (if any) is a dummy
  const int npairs = wp / 2;
  const T skip = (T)(skip_rel * fro);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (off_norm(A, w, ld, sh) <= tol * fro) return true;
    for (int round = 0; round < wp - 1; ++round) {
      if (tid < npairs) {
        // tournament ordering: slot 0 fixed, slots 1..wp-1 rotate
        auto slot = [&](int i) { return i == 0 ? 0 : 1 + (i - 1 + round) % (wp - 1); };
        int p = slot(tid), q = slot(wp - 1 - tid);
        if (p > q) { const int tmp = p; p = q; q = tmp; }
        T c = 1, s = 0;
        if (q < w) sym_schur2<T>(A[p * ld + p], A[q * ld + q], A[p * ld + q], skip, c, s);
        sh.p[tid] = p;
        sh.q[tid] = q;
        sh.c[tid] = (double)c;
        sh.s[tid] = (double)s;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int e = tid; e < npairs * w; e += kThreads) {
        const int k = e / w, i = e - k * w;
        const T s = (T)sh.s[k];
        if (s == 0) continue;
        const T c = (T)sh.c[k];
        const int p = sh.p[k], q = sh.q[k];
        const T aip = A[i * ld + p], aiq = A[i * ld + q];
        A[i * ld + p] = c * aip - s * aiq;
        A[i * ld + q] = s * aip + c * aiq;
        const T vip = V[i * ld + p], viq = V[i * ld + q];
        V[i * ld + p] = c * vip - s * viq;
        V[i * ld + q] = s * vip + c * viq;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int e = tid; e < npairs * w; e += kThreads) {
        const int k = e / w, j = e - k * w;
        const T s = (T)sh.s[k];
        if (s == 0) continue;
        const T c = (T)sh.c[k];
        const int p = sh.p[k], q = sh.q[k];
        const T apj = A[p * ld + j], aqj = A[q * ld + j];
        A[p * ld + j] = c * apj - s * aqj;
        A[q * ld + j] = s * apj + c * aqj;
      }
      __syncthreads();
      if (tid < npairs && sh.s[tid] != 0.0) {
        A[sh.p[tid] * ld + sh.q[tid]] = 0;
        A[sh.q[tid] * ld + sh.p[tid]] = 0;
      }
      __syncthreads();
    }
  }
  return off_norm(A, w, ld, sh) <= tol * fro;
}

__global__ void __launch_bounds__(kThreads) rr_kernel(int w, const double* __restrict__ T, int ldT,
                                                      double* __restrict__ theta, double* __restrict__ Y, int* status) {
  extern __shared__ __align__(16) double sh_d[];
  __shared__ RotShared sh;
  __shared__ int s_rank[kMaxQ];
  const int ld = w + 1;   // padded rows (bank spread)
  double* A = sh_d;                       // T, then B = V^T T V (FP64)
  double* V = A + w * ld;                 // eigenvectors (FP64)
  double* W = V + w * ld;                 // scratch (FP64): T V
  float* A32 = reinterpret_cast<float*>(W + w * ld);
  float* V32 = A32 + w * ld;
  const int tid = threadIdx.x;

  for (int e = tid; e < w * w; e += kThreads) {
    const int i = e / w, j = e - i * w;
    const int r = i < j ? i : j, cc = i < j ? j : i;
    const double a = T[(int64_t)cc * ldT + r];
    A[i * ld + j] = a;
    A32[i * ld + j] = (float)a;
    V32[i * ld + j] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  double f = 0.0;
  for (int e = tid; e < w * w; e += kThreads) {
    const double a = A[(e / w) * ld + (e % w)];
    f += a * a;
  }
  const double fro = sqrt(block_sum(f, sh));

  bool ok = true;
  if (w > 1 && fro > 0.0) {
    // 1. FP32 sweeps
    jacobi_sweeps<float>(A32, V32, w, ld, fro, 1e-6, 1e-9, 20, sh);
    // 2. promote V, re-orthonormalise (two Gram-Schmidt passes per column)
    for (int e = tid; e < w * w; e += kThreads) V[(e / w) * ld + (e % w)] = (double)V32[(e / w) * ld + (e % w)];
    __syncthreads();
    for (int j = 0; j < w; ++j) {
      for (int pass = 0; pass < 2; ++pass) {
        // h_i = V[:, i] . V[:, j] for i < j, one warp per coefficient
        for (int i = tid >> 5; i < j; i += kThreads / 32) {
          double d = 0.0;
          for (int r = tid & 31; r < w; r += 32) d += V[r * ld + i] * V[r * ld + j];
          for (int off = 16; off > 0; off >>= 1) d += __shfl_down_sync(0xffffffffu, d, off);
          if ((tid & 31) == 0) W[i] = d;
        }
        __syncthreads();
        for (int r = tid; r < w; r += kThreads) {
          double s = 0.0;
          for (int i = 0; i < j; ++i) s += V[r * ld + i] * W[i];
          V[r * ld + j] -= s;
        }
        __syncthreads();
      }
      double nn = 0.0;
      for (int r = tid; r < w; r += kThreads) nn += V[r * ld + j] * V[r * ld + j];
      const double inv = 1.0 / sqrt(block_sum(nn, sh));
      for (int r = tid; r < w; r += kThreads) V[r * ld + j] *= inv;
      __syncthreads();
    }
    // 3. B = V^T T V in FP64 (W = T V, then A = V^T W)
    for (int e = tid; e < w * w; e += kThreads) {
      const int i = e / w, j = e - i * w;
      double s = 0.0;
      for (int r = 0; r < w; ++r) s += A[i * ld + r] * V[r * ld + j];
      W[i * ld + j] = s;
    }
    __syncthreads();
    for (int e = tid; e < w * w; e += kThreads) {
      const int i = e / w, j = e - i * w;
      if (j < i) continue;
      double s = 0.0;
      for (int r = 0; r < w; ++r) s += V[r * ld + i] * W[r * ld + j];
      A[i * ld + j] = s;
      A[j * ld + i] = s;
    }
    __syncthreads();
    // 4. FP64 polishing sweeps
    ok = jacobi_sweeps<double>(A, V, w, ld, fro, 1e-15, 1e-18, 30, sh);
  } else if (w == 1) {
    if (tid == 0) V[0] = 1.0;
    __syncthreads();
  } else {
    for (int e = tid; e < w * w; e += kThreads) V[(e / w) * ld + (e % w)] = (e / w == e % w) ? 1.0 : 0.0;
    __syncthreads();
  }
  if (!ok && tid == 0) atomicOr(status, kFlagJacobi);

  // stable ascending rank of the eigenvalues
  for (int i = tid; i < w; i += kThreads) {
    const double di = A[i * ld + i];
    int r = 0;
    for (int j = 0; j < w; ++j) {
      const double dj = A[j * ld + j];
      r += (dj < di) || (dj == di && j < i);
    }
    s_rank[i] = r;
  }
  __syncthreads();
  for (int i = tid; i < w; i += kThreads) {
    const int r = s_rank[i];
    theta[r] = A[i * ld + i];
    // sign rule: largest |entry| (first such) positive
    int im = 0;
    double am = -1.0;
    for (int j = 0; j < w; ++j) {
      const double a = fabs(V[j * ld + i]);
      if (a > am) { am = a; im = j; }
    }
    const double sg = V[im * ld + i] < 0.0 ? -1.0 : 1.0;
    for (int j = 0; j < w; ++j) Y[(int64_t)r * w + j] = sg * V[j * ld + i];
    if (!isfinite(theta[r])) atomicOr(status, kFlagNaN);
  }
}

}  // namespace

void rayleigh_ritz(const Ctx& c, int w, const double* T, int ldT, double* theta, double* Y) {
  if (w < 1 || w > kMaxQ) throw Error(TRPLK_EINVAL, "Rayleigh-Ritz size out of range");
  auto bytes = [](int ww) { return (size_t)ww * (ww + 1) * (3 * sizeof(double) + 2 * sizeof(float)); };
  static bool cfg = false;
  if (!cfg) {
    TRPLK_CUDA_TRY(cudaFuncSetAttribute(rr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes(kMaxQ)));
    cfg = true;
  }
  ProfScope ps(c, PK_RR, 0.0);
  rr_kernel<<<1, kThreads, bytes(w), c.stream>>>(w, T, ldT, theta, Y, c.status);
  check_launch("rr_kernel");
}

}  // namespace trplk
