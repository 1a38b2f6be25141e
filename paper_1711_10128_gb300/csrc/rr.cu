// Rayleigh-Ritz eigensolver for the small projection T (Algorithm 1,
// 'compute eigenpairs of T, T = Y Theta Y^T').
//
// One CTA of (wp/2)^2 threads (whole warps, 64 to 1024); T (w <= 64) padded
// to an even order wp with a zero row and column.  The cyclic Jacobi method with the round-robin (tournament)
// ordering: each round rotates the wp/2 disjoint index pairs at once
// (index 0 stays, indices 1..wp-1 move one place per round).  Rotations use
// the symmetric 2x2 Schur decomposition of Golub and Van Loan (Sec. 8.5).
// The similarity A <- J^T A J is applied block by block: the 2x2 block of rows
// (p_K, q_K) and columns (p_L, q_L) becomes R_K^T A_KL R_L, and V <- V J.
//
// The FP64 pipe of this GPU retires 2 FMAs per clock per SM (the FP32 pipe
// 128), so the sweeps run in two precisions:
//  1. FP32 sweeps on fp32(T) until its off-diagonal norm is <= 1e-6 ||T||_F.
//     Thread (K, L) keeps in registers the block (K, L) of the matrix (only
//     for K <= L; it also writes the mirror) and rows (2K, 2K+1) x columns
//     (p_L, q_L) of V; it computes both rotations it needs from the pairs'
//     diagonal blocks (every thread that needs a rotation computes it from
//     the same values with the same operations, so all agree bit for bit),
//     rotates, and writes its entries to the other of two shared buffers.
//     After one barrier it reads its next round's entries: one barrier per
//     round, and no round waits on a rotation computed by another thread.
//  2. V is promoted to FP64 and made orthogonal to FP64 rounding by two
//     Newton-Schulz steps V <- V (3 I - V^T V) / 2 (each squares the departure
//     from orthogonality), then B = V^T T V is formed in FP64 (an orthogonal
//     similarity up to FP64 rounding) -- nearly diagonal.
//  3. FP64 sweeps on B (quadratic convergence: usually one or two; rotations
//     below 1e-16 ||T||_F are skipped) until its off-diagonal norm is
//     <= 3e-15 ||T||_F, in place in shared memory: one thread per pair forms
//     its rotation, then one thread per block (K <= L, with its mirror) and
//     one per (row pair, pair) of V apply them.  These sweeps are bound by the
//     FP64 pipe.
// For a T projected from FP32 data (the FP32 phase of the mixed path) the
// eigenpairs need only be far more accurate than that data (about 1e-7
// relative): one Newton-Schulz step (V orthogonal to about 1e-12) and FP64
// sweeps down to an off-diagonal norm of 1e-10 ||T||_F (usually one sweep;
// the eigenvalues then carry errors of order 1e-20 ||T||_F^2 / gap).
// Eigenvalues are then sorted ascending (stable rank sort) and every
// eigenvector is signed so its largest-magnitude entry, the first such, is
// positive.
#include <algorithm>
#include <cmath>

#include "launch.h"

namespace trplk {

namespace {

constexpr int kThreads = 1024;
constexpr int kMaxPairs = kMaxQ / 2;

// Round-robin slot: the pair (p < q) that slot k holds in the current round,
// over wp = m + 1 indices.  Index 0 stays in slot 0; positions a, b of the
// others advance by one (mod m) per round.
struct Slot {
  int k, m, a, b;
  __device__ __forceinline__ void init(int k_, int m_) {
    k = k_;
    m = m_;
    a = k == 0 ? 0 : k - 1;
    b = m - 1 - k;
  }
  __device__ __forceinline__ void next() {
    a = a + 1 == m ? 0 : a + 1;
    b = b + 1 == m ? 0 : b + 1;
  }
  __device__ __forceinline__ int p() const {
    const int x = k == 0 ? 0 : 1 + a, y = 1 + b;
    return x < y ? x : y;
  }
  __device__ __forceinline__ int q() const {
    const int x = k == 0 ? 0 : 1 + a, y = 1 + b;
    return x < y ? y : x;
  }
};

// Rotation of a pair's 2x2 block from d = a_qq - a_pp and e = 2 a_pq (both
// scaled by 1 / ||T||_F, so squares neither overflow nor underflow):
// t = tan(angle) = sign(d) e / (|d| + sqrt(d^2 + e^2)), the smaller root, free
// of cancellation; c = 1 / sqrt(1 + t^2), s = t c.  Computed in FP32 with the
// fast reciprocal and reciprocal square root (every op is a single hardware
// approximation, 2 ulp at most): c^2 + s^2 = 1 to a few FP32 ulp, and the
// rotated a_pq falls by about 1e7.
__device__ __forceinline__ void rot_f32(float d, float e, float& c, float& s) {
  const float q = fmaf(d, d, e * e);
  const float h = q * rsqrtf(q);
  const float t = __fdividef(d >= 0.f ? e : -e, fabsf(d) + h);
  c = rsqrtf(fmaf(t, t, 1.f));
  s = t * c;
}

__device__ __forceinline__ void schur2_f32(float app, float aqq, float apq, float skip, float inv_fro, float& c,
                                           float& s) {
  if (!(fabsf(apq) > skip)) {
    c = 1.f;
    s = 0.f;
    return;
  }
  rot_f32((aqq - app) * inv_fro, 2.f * apq * inv_fro, c, s);
}

// FP64 rotation: the angle from rot_f32 (FP32-accurate, so the rotated a_pq
// is not zero but about 1e-7 of its size, and is kept), made orthogonal to
// FP64 rounding: with the FP32 pair (c0, s0) exact in FP64 and
// delta = c0^2 + s0^2 - 1 (|delta| ~ 1e-7), (c, s) = (c0, s0) (1 - delta/2 +
// 3 delta^2/8), the series of (1 + delta)^(-1/2) to an error of about
// delta^3.  The FP64 pipe's long latency (an FP64 division or square root
// costs hundreds of clocks on this GPU) stays off the round's critical path.
__device__ __forceinline__ void schur2_f64(double app, double aqq, double apq, double skip, double inv_fro, double& c,
                                           double& s) {
  if (!(fabs(apq) > skip)) {
    c = 1.0;
    s = 0.0;
    return;
  }
  float c0, s0;
  rot_f32((float)((aqq - app) * inv_fro), (float)(2.0 * apq * inv_fro), c0, s0);
  const double cd = c0, sd = s0;
  const double delta = fma(cd, cd, fma(sd, sd, -1.0));
  const double f = fma(delta, fma(delta, 0.375, -0.5), 1.0);
  c = cd * f;
  s = sd * f;
}

struct RrShared {
  int p[kMaxPairs], q[kMaxPairs];
  double c[kMaxPairs], s[kMaxPairs];
  double red[kThreads / 32];
  double val;
  int rank[kMaxQ];
};

// Sum over the CTA (blockDim.x a multiple of 32); result valid in every
// thread.  Warps reduce by shuffles, warp 0 sums the warps' partials (a
// single FP64 add chain per lane instead of one per thread).
template <typename F>
__device__ F block_sum(F v, RrShared& sh) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) sh.red[threadIdx.x >> 5] = (double)v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? sh.red[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
    if (threadIdx.x == 0) sh.val = t;
  }
  __syncthreads();
  return (F)sh.val;
}

__device__ double off_norm_f64(const double* A, int w, int ld, RrShared& sh) {
  double o = 0.0;
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
    const int i = e / w, j = e - i * w;
    if (i != j) o = fma(A[i * ld + j], A[i * ld + j], o);
  }
  return sqrt(block_sum(o, sh));
}

// FP32 sweeps (step 1).  A0/A1 and V0/V1: double buffers of wp x wp (ld),
// A0 = fp32(T), V0 = identity on entry.  Returns the buffer index holding V.
__device__ int jacobi_f32(float* A0, float* A1, float* V0, float* V1, int w, int wp, int ld, double fro, double tol,
                          float skip, int max_sweeps, RrShared& sh) {
  const int tid = threadIdx.x;
  const float tol32 = (float)(tol * fro);
  const float inv_fro = (float)(1.0 / fro);
  const int np = wp / 2, m = wp - 1;
  const bool active = tid < np * np;
  const int K = active ? tid / np : 0, L = active ? tid - (tid / np) * np : 0;
  const bool upper = active && K <= L;
  int cur = 0;
  Slot sK, sL;
  sK.init(K, m);
  sL.init(L, m);
  const int r0 = 2 * K, r1 = 2 * K + 1;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int round = 0; round < m; ++round) {
      const float* A = cur ? A1 : A0;
      const float* V = cur ? V1 : V0;
      const int pK = sK.p(), qK = sK.q(), pL = sL.p(), qL = sL.q();
      float x00 = 0.f, x01 = 0.f, x10 = 0.f, x11 = 0.f, v00 = 0.f, v01 = 0.f, v10 = 0.f, v11 = 0.f;
      float kpp = 0.f, kqq = 0.f, kpq = 0.f, lpp = 0.f, lqq = 0.f, lpq = 0.f;
      if (active) {
        lpp = A[pL * ld + pL];
        lqq = A[qL * ld + qL];
        lpq = A[pL * ld + qL];
        v00 = V[r0 * ld + pL];
        v01 = V[r0 * ld + qL];
        v10 = V[r1 * ld + pL];
        v11 = V[r1 * ld + qL];
        if (upper) {
          kpp = A[pK * ld + pK];
          kqq = A[qK * ld + qK];
          kpq = A[pK * ld + qK];
          x00 = A[pK * ld + pL];
          x01 = A[pK * ld + qL];
          x10 = A[qK * ld + pL];
          x11 = A[qK * ld + qL];
        }
      }
      if (round == 0) {
        // off-diagonal norm at the start of the sweep, from the upper blocks
        // (a block off the diagonal counts twice, for its mirror)
        const float o = K == L ? 2.f * x01 * x01 : 2.f * (x00 * x00 + x01 * x01 + x10 * x10 + x11 * x11);
        if (sqrtf(block_sum(upper ? o : 0.f, sh)) <= tol32) return cur;
      }
      float cL, sLr;
      schur2_f32(lpp, lqq, lpq, skip, inv_fro, cL, sLr);
      float* An = cur ? A0 : A1;
      float* Vn = cur ? V0 : V1;
      if (active) {
        Vn[r0 * ld + pL] = cL * v00 - sLr * v01;
        Vn[r0 * ld + qL] = sLr * v00 + cL * v01;
        Vn[r1 * ld + pL] = cL * v10 - sLr * v11;
        Vn[r1 * ld + qL] = sLr * v10 + cL * v11;
      }
      if (upper) {
        float cK, sKr;
        schur2_f32(kpp, kqq, kpq, skip, inv_fro, cK, sKr);
        // Y = X R_L (columns), Z = R_K^T Y (rows)
        const float y00 = cL * x00 - sLr * x01, y01 = sLr * x00 + cL * x01;
        const float y10 = cL * x10 - sLr * x11, y11 = sLr * x10 + cL * x11;
        const float z00 = cK * y00 - sKr * y10, z10 = sKr * y00 + cK * y10;
        const float z01 = cK * y01 - sKr * y11, z11 = sKr * y01 + cK * y11;
        if (K == L) {
          const bool rot = sKr != 0.f;
          An[pK * ld + pK] = z00;
          An[qK * ld + qK] = z11;
          An[pK * ld + qK] = rot ? 0.f : z01;
          An[qK * ld + pK] = rot ? 0.f : z10;
        } else {
          An[pK * ld + pL] = z00;
          An[pK * ld + qL] = z01;
          An[qK * ld + pL] = z10;
          An[qK * ld + qL] = z11;
          An[pL * ld + pK] = z00;
          An[qL * ld + pK] = z01;
          An[pL * ld + qK] = z10;
          An[qL * ld + qK] = z11;
        }
      }
      __syncthreads();
      cur ^= 1;
      sK.next();
      sL.next();
    }
  }
  return cur;
}

// FP64 sweeps (step 3) in place on A (wp x wp, ld), rotations accumulated into
// V.  Stops when the off-diagonal norm is <= tol * fro; returns true if it did.
__device__ bool jacobi_f64(double* A, double* V, int w, int wp, int ld, double fro, double tol, double skip,
                           int max_sweeps, RrShared& sh) {
  const int tid = threadIdx.x;
  const double inv_fro = 1.0 / fro;
  const int np = wp / 2, m = wp - 1;
  const int nb = np * (np + 1) / 2;
  // this thread's block (K <= L) of the upper triangle, if any
  int K = 0, L = 0;
  if (tid < nb) {
    int rem = tid;
    while (rem >= np - K) { rem -= np - K; ++K; }
    L = K + rem;
  }
  // this thread's (row pair, pair) of V, if any
  const int nvr = (w + 1) / 2;
  const bool vtask = tid < nvr * np;
  const int vr = vtask ? 2 * (tid / np) : 0, vL = vtask ? tid - (tid / np) * np : 0;
  Slot slot;
  slot.init(tid < np ? tid : 0, m);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (off_norm_f64(A, w, ld, sh) <= tol * fro) return true;
    for (int round = 0; round < m; ++round) {
      if (tid < np) {
        const int p = slot.p(), q = slot.q();
        double c, s;
        schur2_f64(A[p * ld + p], A[q * ld + q], A[p * ld + q], skip, inv_fro, c, s);
        sh.p[tid] = p;
        sh.q[tid] = q;
        sh.c[tid] = c;
        sh.s[tid] = s;
        slot.next();
      }
      __syncthreads();
      if (tid < nb) {
        const double sK = sh.s[K], sL = sh.s[L];
        if (sK != 0.0 || sL != 0.0) {
          const double cK = sh.c[K], cL = sh.c[L];
          const int pK = sh.p[K], qK = sh.q[K], pL = sh.p[L], qL = sh.q[L];
          const double x00 = A[pK * ld + pL], x01 = A[pK * ld + qL], x10 = A[qK * ld + pL], x11 = A[qK * ld + qL];
          const double y00 = cL * x00 - sL * x01, y01 = sL * x00 + cL * x01;
          const double y10 = cL * x10 - sL * x11, y11 = sL * x10 + cL * x11;
          const double z00 = cK * y00 - sK * y10, z10 = sK * y00 + cK * y10;
          const double z01 = cK * y01 - sK * y11, z11 = sK * y01 + cK * y11;
          if (K == L) {   // symmetric: z10 equals z01 up to rounding
            A[pK * ld + pK] = z00;
            A[qK * ld + qK] = z11;
            A[pK * ld + qK] = z01;
            A[qK * ld + pK] = z01;
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
        }
      }
      if (vtask) {
        const double sL = sh.s[vL];
        if (sL != 0.0) {
          const double cL = sh.c[vL];
          const int pL = sh.p[vL], qL = sh.q[vL];
          const double a0 = V[vr * ld + pL], b0 = V[vr * ld + qL];
          const double a1 = V[(vr + 1) * ld + pL], b1 = V[(vr + 1) * ld + qL];
          V[vr * ld + pL] = cL * a0 - sL * b0;
          V[vr * ld + qL] = sL * a0 + cL * b0;
          V[(vr + 1) * ld + pL] = cL * a1 - sL * b1;
          V[(vr + 1) * ld + qL] = sL * a1 + cL * b1;
        }
      }
      __syncthreads();
    }
  }
  return off_norm_f64(A, w, ld, sh) <= tol * fro;
}

// X = V (3 I - V^T V) / 2 for the w x w V (FP64); M, X scratch.
__device__ void newton_schulz(const double* V, double* M, double* X, int w, int ld) {
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
    const int i = e / w, j = e - i * w;
    if (j < i) continue;
    double s = 0.0;
    for (int r = 0; r < w; ++r) s = fma(V[r * ld + i], V[r * ld + j], s);
    const double v = (i == j ? 1.5 : 0.0) - 0.5 * s;
    M[i * ld + j] = v;
    M[j * ld + i] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
    const int i = e / w, j = e - i * w;
    double s = 0.0;
    for (int r = 0; r < w; ++r) s = fma(V[i * ld + r], M[r * ld + j], s);
    X[i * ld + j] = s;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads) rr_kernel(int w, const double* __restrict__ T, int ldT,
                                                      double* __restrict__ theta, double* __restrict__ Y, int* status,
                                                      int fp32_data) {
  extern __shared__ __align__(16) double sh_d[];
  __shared__ RrShared sh;
  const int wp = w + (w & 1);   // even order; index w (if any) is a zero dummy
  const int ld = wp + 1;        // padded rows (bank spread)
  double* A = sh_d;             // T, then B = V^T T V (FP64)
  double* V = A + wp * ld;      // eigenvectors (FP64)
  double* W = V + wp * ld;      // scratch (FP64); the FP32 matrix buffers during step 1
  double* X = W + wp * ld;      // scratch (FP64); the FP32 V buffers during step 1
  float* A32a = reinterpret_cast<float*>(W);
  float* A32b = A32a + wp * ld;
  float* V32a = reinterpret_cast<float*>(X);
  float* V32b = V32a + wp * ld;
  const int tid = threadIdx.x;

  double f = 0.0;
  for (int e = tid; e < wp * wp; e += blockDim.x) {
    const int i = e / wp, j = e - i * wp;
    const int r = i < j ? i : j, cc = i < j ? j : i;
    const double a = (i < w && j < w) ? T[(int64_t)cc * ldT + r] : 0.0;
    A[i * ld + j] = a;
    A32a[i * ld + j] = (float)a;
    V32a[i * ld + j] = (i == j && i < w) ? 1.f : 0.f;
    f += a * a;
  }
  const double fro = sqrt(block_sum(f, sh));   // (its barriers also publish the buffers)

  bool ok = true;
  if (w > 1 && fro > 0.0) {
    // 1. FP32 sweeps
    const int vb = jacobi_f32(A32a, A32b, V32a, V32b, w, wp, ld, fro, 1e-6, (float)(1e-9 * fro), 20, sh);
    // 2. promote V, two Newton-Schulz steps (V -> X -> V)
    const float* V32 = vb ? V32b : V32a;
    for (int e = tid; e < wp * wp; e += blockDim.x) V[(e / wp) * ld + (e % wp)] = (double)V32[(e / wp) * ld + (e % wp)];
    __syncthreads();
    newton_schulz(V, W, X, w, ld);
    if (fp32_data) {   // one step: orthogonal to about 1e-12, far below FP32 data
      for (int e = tid; e < wp * wp; e += blockDim.x) V[(e / wp) * ld + (e % wp)] = X[(e / wp) * ld + (e % wp)];
      __syncthreads();
    } else {
      newton_schulz(X, W, V, w, ld);
    }
    // 3. B = V^T T V in FP64 (W = T V, then A = V^T W)
    for (int e = tid; e < w * w; e += blockDim.x) {
      const int i = e / w, j = e - i * w;
      double s = 0.0;
      for (int r = 0; r < w; ++r) s = fma(A[i * ld + r], V[r * ld + j], s);
      W[i * ld + j] = s;
    }
    __syncthreads();
    for (int e = tid; e < w * w; e += blockDim.x) {
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
    ok = jacobi_f64(A, V, w, wp, ld, fro, fp32_data ? 1e-10 : 3e-15, 1e-16 * fro, 30, sh);
  } else if (w == 1) {
    if (tid == 0) V[0] = 1.0;
    __syncthreads();
  } else {
    for (int e = tid; e < w * w; e += blockDim.x) V[(e / w) * ld + (e % w)] = (e / w == e % w) ? 1.0 : 0.0;
    __syncthreads();
  }
  if (!ok && tid == 0) atomicOr(status, kFlagJacobi);

  // stable ascending rank of the eigenvalues
  for (int i = tid; i < w; i += blockDim.x) {
    const double di = A[i * ld + i];
    int r = 0;
    for (int j = 0; j < w; ++j) {
      const double dj = A[j * ld + j];
      r += (dj < di) || (dj == di && j < i);
    }
    sh.rank[i] = r;
  }
  __syncthreads();
  // theta, and each eigenvector signed so its largest |entry| (first such) is
  // positive: one warp per eigenvector
  const int warp = tid >> 5, lane = tid & 31;
  for (int i = warp; i < w; i += blockDim.x >> 5) {
    const int r = sh.rank[i];
    double am = -1.0;
    int im = 0;
    for (int j = lane; j < w; j += 32) {
      const double a = fabs(V[j * ld + i]);
      if (a > am) { am = a; im = j; }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const double ao = __shfl_xor_sync(0xffffffffu, am, off);
      const int io = __shfl_xor_sync(0xffffffffu, im, off);
      if (ao > am || (ao == am && io < im)) { am = ao; im = io; }
    }
    const double sg = V[im * ld + i] < 0.0 ? -1.0 : 1.0;
    for (int j = lane; j < w; j += 32) Y[(int64_t)r * w + j] = sg * V[j * ld + i];
    if (lane == 0) {
      theta[r] = A[i * ld + i];
      if (!isfinite(A[i * ld + i])) atomicOr(status, kFlagNaN);
    }
  }
}

}  // namespace

void rayleigh_ritz(const Ctx& c, int w, const double* T, int ldT, double* theta, double* Y, bool fp32_data) {
  if (w < 1 || w > kMaxQ) throw Error(TRPLK_EINVAL, "Rayleigh-Ritz size out of range");
  auto bytes = [](int ww) {
    const size_t wp = (size_t)(ww + (ww & 1));
    return wp * (wp + 1) * 4 * sizeof(double);
  };
  smem_optin<rr_kernel>((int)bytes(kMaxQ), c.device);
  ProfScope ps(c, PK_RR, 0.0);
  // one thread per 2x2 block of the FP32 sweeps ((wp / 2)^2), whole warps,
  // at least two; every later phase strides over the same threads
  const int np = (w + (w & 1)) / 2;
  const int threads = std::max(64, (np * np + 31) / 32 * 32);
  rr_kernel<<<1, threads, bytes(w), c.stream>>>(w, T, ldT, theta, Y, c.status, fp32_data ? 1 : 0);
  check_launch("rr_kernel");
}

}  // namespace trplk
