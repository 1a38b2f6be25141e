// Rayleigh-Ritz eigensolver for the small projection T (Algorithm 1,
// 'compute eigenpairs of T, T = Y Theta Y^T').
//
// One CTA, T (w <= 64) in shared memory, padded to an even order wp with a
// zero row and column.  The cyclic Jacobi method with the round-robin
// (tournament) ordering: each round rotates the wp/2 disjoint index pairs at
// once.  Rotations use the symmetric 2x2 Schur decomposition of Golub and Van
// Loan (Sec. 8.5).  A round is two phases: the rotation angles, then the
// similarity A <- J^T A J applied block by block -- the 2x2 block of rows
// (p_K, q_K) and columns (p_L, q_L) becomes R_K^T A_KL R_L, each block (and its
// mirror) owned by one thread -- together with V <- V J.  The rotated pairs'
// off-diagonal entries are set to zero.  Off-diagonal norms are summed
// directly, never as a difference of norms.
//
// The FP64 pipe of this GPU retires 2 FMAs per clock per SM (the FP32 pipe
// 128), so the sweeps run in two precisions:
//  1. FP32 sweeps on fp32(T) until its off-diagonal norm is <= 1e-6 ||T||_F,
//     accumulating the rotations into V (orthogonal to about 1e-7);
//  2. V is promoted to FP64 and made orthogonal to FP64 rounding by two
//     Newton-Schulz steps V <- V (3 I - V^T V) / 2 (each squares the
//     departure from orthogonality), then B = V^T T V is formed in FP64 (an
//     orthogonal similarity up to FP64 rounding) -- nearly diagonal;
//  3. FP64 sweeps on B (quadratic convergence: usually one or two; the second
//     skips the rotations already below 1e-16 ||T||_F) until its
//     off-diagonal norm is <= 3e-15 ||T||_F, accumulating into V.
// Eigenvalues are then sorted ascending (stable rank sort) and every
// eigenvector is signed so its largest-magnitude entry, the first such, is
// positive.
#include <cmath>

#include "launch.h"

namespace trplk {

namespace {

constexpr int kThreads = 512;
constexpr int kMaxPairs = kMaxQ / 2;
constexpr int kMaxBlocks = kMaxPairs * (kMaxPairs + 1) / 2;

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
  int p[kMaxPairs], q[kMaxPairs];
  double c[kMaxPairs], s[kMaxPairs];
  float cf[kMaxPairs], sf[kMaxPairs];
  unsigned char bk[kMaxBlocks], bl[kMaxBlocks];   // block b -> pairs (K, L), K <= L
  unsigned char sp[kMaxQ - 1][kMaxPairs], sq[kMaxQ - 1][kMaxPairs];   // round -> pair -> (p, q), p < q
  double red[kThreads / 32];
  double val;
};

template <typename T> __device__ __forceinline__ T rot_c(const RotShared& sh, int k);
template <> __device__ __forceinline__ double rot_c<double>(const RotShared& sh, int k) { return sh.c[k]; }
template <> __device__ __forceinline__ float rot_c<float>(const RotShared& sh, int k) { return sh.cf[k]; }
template <typename T> __device__ __forceinline__ T rot_s(const RotShared& sh, int k);
template <> __device__ __forceinline__ double rot_s<double>(const RotShared& sh, int k) { return sh.s[k]; }
template <> __device__ __forceinline__ float rot_s<float>(const RotShared& sh, int k) { return sh.sf[k]; }

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

// Jacobi sweeps on the symmetric A (wp x wp, row-major, ld, zero beyond w),
// rotations accumulated into V.  Stops when the off-diagonal norm is
// <= tol * fro.  Returns true if it did.
template <typename T>
__device__ bool jacobi_sweeps(T* A, T* V, int w, int wp, int ld, double fro, double tol, double skip_rel,
                              int max_sweeps, RotShared& sh) {
  const int tid = threadIdx.x;
  const int npairs = wp / 2;
  const int nblk = npairs * (npairs + 1) / 2;
  int lgw = 0;   // V tasks: row i = e & (2^lgw - 1), pair L = e >> lgw (rows >= w idle)
  while ((1 << lgw) < w) ++lgw;
  const int ntask = nblk + (npairs << lgw);   // A blocks, then (row of V, pair) tasks
  const T skip = (T)(skip_rel * fro);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (off_norm(A, w, ld, sh) <= tol * fro) return true;
    for (int round = 0; round < wp - 1; ++round) {
      if (tid < npairs) {
        const int p = sh.sp[round][tid], q = sh.sq[round][tid];
        T c = 1, s = 0;
        sym_schur2<T>(A[p * ld + p], A[q * ld + q], A[p * ld + q], skip, c, s);
        sh.p[tid] = p;
        sh.q[tid] = q;
        if (sizeof(T) == 8) { sh.c[tid] = (double)c; sh.s[tid] = (double)s; }
        else { sh.cf[tid] = (float)c; sh.sf[tid] = (float)s; }
      }
      __syncthreads();
      for (int t = tid; t < ntask; t += kThreads) {
        if (t < nblk) {
          const int K = sh.bk[t], L = sh.bl[t];
          const T sK = rot_s<T>(sh, K), sL = rot_s<T>(sh, L);
          if (sK == 0 && sL == 0) continue;
          const T cK = rot_c<T>(sh, K), cL = rot_c<T>(sh, L);
          const int pK = sh.p[K], qK = sh.q[K], pL = sh.p[L], qL = sh.q[L];
          const T x00 = A[pK * ld + pL], x01 = A[pK * ld + qL], x10 = A[qK * ld + pL], x11 = A[qK * ld + qL];
          // Y = X R_L (columns), Z = R_K^T Y (rows)
          const T y00 = cL * x00 - sL * x01, y01 = sL * x00 + cL * x01;
          const T y10 = cL * x10 - sL * x11, y11 = sL * x10 + cL * x11;
          const T z00 = cK * y00 - sK * y10, z10 = sK * y00 + cK * y10;
          const T z01 = cK * y01 - sK * y11, z11 = sK * y01 + cK * y11;
          if (K == L) {
            A[pK * ld + pK] = z00;
            A[qK * ld + qK] = z11;
            A[pK * ld + qK] = 0;
            A[qK * ld + pK] = 0;
          } else {
            A[pK * ld + pL] = z00;
            A[pK * ld + qL] = z01;
            A[qK * ld + pL] = z10;
            A[qK * ld + qL] = z11;
            A[pL * ld + pK] = z00;
            A[qL * ld + pK] = z01;
            A[pL * ld + qK] = z10;
            A[qL * ld + qK] = z11;
          }
        } else {
          const int e = t - nblk;
          const int L = e >> lgw, i = e & ((1 << lgw) - 1);
          if (i >= w) continue;
          const T sL = rot_s<T>(sh, L);
          if (sL == 0) continue;
          const T cL = rot_c<T>(sh, L);
          const int pL = sh.p[L], qL = sh.q[L];
          const T vp = V[i * ld + pL], vq = V[i * ld + qL];
          V[i * ld + pL] = cL * vp - sL * vq;
          V[i * ld + qL] = sL * vp + cL * vq;
        }
      }
      __syncthreads();
    }
  }
  return off_norm(A, w, ld, sh) <= tol * fro;
}

// X = V (3 I - V^T V) / 2 for the w x w V (FP64); M, X scratch.
__device__ void newton_schulz(const double* V, double* M, double* X, int w, int ld) {
  for (int e = threadIdx.x; e < w * w; e += kThreads) {
    const int i = e / w, j = e - i * w;
    double s = 0.0;
    for (int r = 0; r < w; ++r) s = fma(V[r * ld + i], V[r * ld + j], s);
    M[i * ld + j] = (i == j ? 1.5 : 0.0) - 0.5 * s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < w * w; e += kThreads) {
    const int i = e / w, j = e - i * w;
    double s = 0.0;
    for (int r = 0; r < w; ++r) s = fma(V[i * ld + r], M[r * ld + j], s);
    X[i * ld + j] = s;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads) rr_kernel(int w, const double* __restrict__ T, int ldT,
                                                      double* __restrict__ theta, double* __restrict__ Y, int* status) {
  extern __shared__ __align__(16) double sh_d[];
  __shared__ RotShared sh;
  __shared__ int s_rank[kMaxQ];
  const int wp = w + (w & 1);   // even order; index w (if any) is a zero dummy
  const int ld = wp + 1;        // padded rows (bank spread)
  double* A = sh_d;                       // T, then B = V^T T V (FP64)
  double* V = A + wp * ld;                // eigenvectors (FP64)
  double* W = V + wp * ld;                // scratch (FP64)
  double* X = W + wp * ld;                // scratch (FP64)
  float* A32 = reinterpret_cast<float*>(X + wp * ld);
  float* V32 = A32 + wp * ld;
  const int tid = threadIdx.x;

  for (int e = tid; e < wp * wp; e += kThreads) {
    const int i = e / wp, j = e - i * wp;
    const int r = i < j ? i : j, cc = i < j ? j : i;
    const double a = (i < w && j < w) ? T[(int64_t)cc * ldT + r] : 0.0;
    A[i * ld + j] = a;
    A32[i * ld + j] = (float)a;
    V32[i * ld + j] = (i == j && i < w) ? 1.f : 0.f;
  }
  {
    const int np = wp / 2;
    // tournament ordering: slot 0 fixed, slots 1..wp-1 rotate one place per round
    for (int e = tid; e < (wp - 1) * np; e += kThreads) {
      const int round = e / np, k = e - round * np;
      int p = k == 0 ? 0 : 1 + (k - 1 + round) % (wp - 1);
      int q = 1 + (wp - 2 - k + round) % (wp - 1);
      if (p > q) { const int tmp = p; p = q; q = tmp; }
      sh.sp[round][k] = (unsigned char)p;
      sh.sq[round][k] = (unsigned char)q;
    }
    for (int b = tid; b < np * (np + 1) / 2; b += kThreads) {
      int K = 0, rem = b;   // row K of the upper triangle holds np - K blocks
      while (rem >= np - K) { rem -= np - K; ++K; }
      sh.bk[b] = (unsigned char)K;
      sh.bl[b] = (unsigned char)(K + rem);
    }
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
    jacobi_sweeps<float>(A32, V32, w, wp, ld, fro, 1e-6, 1e-9, 20, sh);
    // 2. promote V, two Newton-Schulz steps (V <-> X ping-pong)
    for (int e = tid; e < wp * wp; e += kThreads) V[(e / wp) * ld + (e % wp)] = (double)V32[(e / wp) * ld + (e % wp)];
    __syncthreads();
    newton_schulz(V, W, X, w, ld);
    newton_schulz(X, W, V, w, ld);
    // 3. B = V^T T V in FP64 (W = T V, then A = V^T W)
    for (int e = tid; e < w * w; e += kThreads) {
      const int i = e / w, j = e - i * w;
      double s = 0.0;
      for (int r = 0; r < w; ++r) s = fma(A[i * ld + r], V[r * ld + j], s);
      W[i * ld + j] = s;
    }
    __syncthreads();
    for (int e = tid; e < w * w; e += kThreads) {
      const int i = e / w, j = e - i * w;
      if (j < i) continue;
      double s = 0.0;
      for (int r = 0; r < w; ++r) s = fma(V[r * ld + i], W[r * ld + j], s);
      A[i * ld + j] = s;
      A[j * ld + i] = s;
    }
    __syncthreads();
    // 4. FP64 polishing sweeps.  Rotations with |a_pq| <= 1e-16 ||T||_F are
    // skipped (their effect on eigenvalues is below a_pq^2 / gap), so the
    // stopping norm is 3e-15 ||T||_F >= sqrt(w^2 / 2) * 1e-16 ||T||_F.
    ok = jacobi_sweeps<double>(A, V, w, wp, ld, fro, 3e-15, 1e-16, 30, sh);
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
  auto bytes = [](int ww) {
    const size_t wp = (size_t)(ww + (ww & 1));
    return wp * (wp + 1) * (4 * sizeof(double) + 2 * sizeof(float));
  };
  smem_optin<rr_kernel>((int)bytes(kMaxQ), c.device);
  ProfScope ps(c, PK_RR, 0.0);
  rr_kernel<<<1, kThreads, bytes(w), c.stream>>>(w, T, ldT, theta, Y, c.status);
  check_launch("rr_kernel");
}

}  // namespace trplk
