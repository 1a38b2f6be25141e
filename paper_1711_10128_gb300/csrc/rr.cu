// Rayleigh-Ritz eigensolver for the small projection T (Algorithm 1,
// 'compute eigenpairs of T, T = Y Theta Y^T').
//
// One CTA, FP64, T and the eigenvector matrix V held in shared memory.  The
// cyclic Jacobi method with the round-robin (tournament) ordering: each round
// rotates w/2 disjoint index pairs at once, so a round is three parallel
// phases (rotation angles, column updates A J and V J, row updates J^T A),
// and w - 1 rounds make a sweep over all pairs.  Rotations use the
// symmetric 2x2 Schur decomposition of Golub and Van Loan (Sec. 8.5);
// the rotated pair's off-diagonal entry is set to zero exactly.  Sweeps stop
// when the off-diagonal Frobenius norm (summed directly, never as a
// difference of norms) is <= 1e-15 times ||T||_F.  Then eigenvalues are
// sorted ascending (stable rank sort) and every eigenvector is signed so its
// largest-magnitude entry, the first such, is positive.
#include <cmath>

#include "launch.h"

namespace trplk {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void sym_schur2(double app, double aqq, double apq, double& c, double& s) {
  if (apq == 0.0 || fabs(aqq - app) > 1e300 * fabs(apq)) {
    c = 1.0;
    s = 0.0;
    return;
  }
  const double tau = (aqq - app) / (2.0 * apq);
  const double t = tau >= 0.0 ? 1.0 / (tau + hypot(1.0, tau)) : -1.0 / (-tau + hypot(1.0, tau));
  c = 1.0 / hypot(1.0, t);
  s = t * c;
}

__global__ void __launch_bounds__(kThreads) rr_jacobi_kernel(int w, const double* __restrict__ T, int ldT,
                                                             double* __restrict__ theta, double* __restrict__ Y,
                                                             int* status) {
  extern __shared__ __align__(16) double sh[];
  const int ld = w + 1;                      // padded row length (bank spread)
  double* A = sh;                            // A[i * ld + j]
  double* V = sh + w * ld;
  __shared__ int s_p[kMaxQ / 2], s_q[kMaxQ / 2];
  __shared__ double s_c[kMaxQ / 2], s_s[kMaxQ / 2];
  __shared__ double s_red[kThreads / 32];
  __shared__ double s_fro, s_off;
  __shared__ int s_rank[kMaxQ];
  const int tid = threadIdx.x;

  for (int e = tid; e < w * w; e += kThreads) {
    const int i = e / w, j = e - i * w;
    const int r = i < j ? i : j, cc = i < j ? j : i;
    A[i * ld + j] = T[(int64_t)cc * ldT + r];
    V[i * ld + j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();

  auto block_sum = [&](double v) -> double {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((tid & 31) == 0) s_red[tid >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (tid == 0) {
      for (int i = 0; i < kThreads / 32; ++i) t += s_red[i];
    }
    __syncthreads();
    return t;   // valid in thread 0
  };

  {
    double f = 0.0;
    for (int e = tid; e < w * w; e += kThreads) {
      const double a = A[(e / w) * ld + (e % w)];
      f += a * a;
    }
    const double t = block_sum(f);
    if (tid == 0) s_fro = sqrt(t);
    __syncthreads();
  }

  const int wp = w + (w & 1);   // even number of slots; slot w (if any) is a dummy
  const int npairs = wp / 2;
  bool converged = (w <= 1);
  for (int sweep = 0; sweep < 60 && !converged; ++sweep) {
    // convergence test on the off-diagonal norm
    double o = 0.0;
    for (int e = tid; e < w * w; e += kThreads) {
      const int i = e / w, j = e - i * w;
      if (i != j) {
        const double a = A[i * ld + j];
        o += a * a;
      }
    }
    const double t = block_sum(o);
    if (tid == 0) s_off = sqrt(t);
    __syncthreads();
    if (s_off <= 1e-15 * s_fro) {
      converged = true;
      break;
    }
    for (int round = 0; round < wp - 1; ++round) {
      if (tid < npairs) {
        // tournament ordering: slot 0 fixed, slots 1..wp-1 rotate
        auto slot = [&](int i) { return i == 0 ? 0 : 1 + (i - 1 + round) % (wp - 1); };
        int p = slot(tid), q = slot(wp - 1 - tid);
        if (p > q) { const int tmp = p; p = q; q = tmp; }
        double c = 1.0, s = 0.0;
        if (q < w) sym_schur2(A[p * ld + p], A[q * ld + q], A[p * ld + q], c, s);
        s_p[tid] = p;
        s_q[tid] = q;
        s_c[tid] = c;
        s_s[tid] = s;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int e = tid; e < npairs * w; e += kThreads) {
        const int k = e / w, i = e - k * w;
        const double s = s_s[k];
        if (s == 0.0) continue;
        const double c = s_c[k];
        const int p = s_p[k], q = s_q[k];
        const double aip = A[i * ld + p], aiq = A[i * ld + q];
        A[i * ld + p] = c * aip - s * aiq;
        A[i * ld + q] = s * aip + c * aiq;
        const double vip = V[i * ld + p], viq = V[i * ld + q];
        V[i * ld + p] = c * vip - s * viq;
        V[i * ld + q] = s * vip + c * viq;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int e = tid; e < npairs * w; e += kThreads) {
        const int k = e / w, j = e - k * w;
        const double s = s_s[k];
        if (s == 0.0) continue;
        const double c = s_c[k];
        const int p = s_p[k], q = s_q[k];
        const double apj = A[p * ld + j], aqj = A[q * ld + j];
        A[p * ld + j] = c * apj - s * aqj;
        A[q * ld + j] = s * apj + c * aqj;
      }
      __syncthreads();
      if (tid < npairs && s_s[tid] != 0.0) {
        A[s_p[tid] * ld + s_q[tid]] = 0.0;
        A[s_q[tid] * ld + s_p[tid]] = 0.0;
      }
      __syncthreads();
    }
  }
  if (!converged && tid == 0) atomicOr(status, kFlagJacobi);

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
  const size_t smem = 2 * (size_t)w * (w + 1) * sizeof(double);
  static bool cfg = false;
  if (!cfg) {
    TRPLK_CUDA_TRY(cudaFuncSetAttribute(rr_jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        2 * kMaxQ * (kMaxQ + 1) * (int)sizeof(double)));
    cfg = true;
  }
  ProfScope ps(c, PK_RR, 0.0);
  rr_jacobi_kernel<<<1, kThreads, smem, c.stream>>>(w, T, ldT, theta, Y, c.status);
  check_launch("rr_jacobi_kernel");
}

}  // namespace trplk
