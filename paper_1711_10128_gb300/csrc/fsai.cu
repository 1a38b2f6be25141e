// Factorised sparse approximate inverse (FSAI) preconditioner M = G^T G,
// classical and learned, with the training of its MLP on the GPU.
//
// The paper (Sec. 3) allows any preconditioner approximating (A - rho I)^-1
// and uses ILU/LDL in its experiments (Sec. 5); the factorised sparse
// approximate inverse here is this library's data-parallel preconditioner:
//  * G is lower triangular on the pattern P of A's lower triangle (with the
//    diagonal); M x = G^T (G x) is two sparse matvecs (G, and G^T stored as
//    CSR on A's upper pattern, its values gathered through a permutation);
//  * classical FSAI (Kolotilina-Yeremin): row i of G solves
//    A[P_i, P_i] g = e_i, scaled so that (G A G^T)_ii = 1 -- one thread per
//    row, FP64 Cholesky of the |P_i| x |P_i| block (|P_i| <= 16);
//  * learned FSAI, for 7-point operators on an Nx x Ny x Nz grid: an MLP
//    8 -> 64 -> 64 -> 7 (ReLU) maps per-row features of A (log a_ii, the
//    scaled couplings a_ij/sqrt(a_ii a_jj), diagonal dominance) to G's row:
//    g_ii = softplus(o_c)/sqrt(a_ii), g_ij = o_dir/sqrt(a_jj) -- variables in
//    which classical FSAI is a smooth function of the features; weights and
//    activations in BF16 (or FP32 for reference runs), FP32 accumulation;
//  * training loss over solver vectors v (the residuals A x - theta x of Ritz
//    vectors from capped Jacobi TRPL+K runs -- the vectors M acts on inside
//    the solver): c_v [(Mv)^T A (Mv) - 2 ||Gv||^2]
//    (the energy-norm error of Mv against A^-1 v less a constant),
//    c_v = 1/(v^T D^-1 v), plus gamma times the Kaporin measure
//    log(mean_i (G A G^T)_ii) - (2/n) sum_i log g_ii; analytic gradients with
//    respect to G, through the MLP (recomputing activations) to the weights,
//    reduced deterministically; Adam updates.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "handle.h"
#include "tallskinny.cuh"

namespace trplk {

constexpr int kH = 64;
constexpr int OFF_W1 = 0, OFF_B1 = 512, OFF_W2 = 576, OFF_B2 = 4672, OFF_W3 = 4736, OFF_B3 = 5184;
constexpr int kNParams = 5191;
constexpr int kMaxP = 16;

// ---------------------------------------------------------------- pattern
__global__ void tri_count_kernel(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                 int64_t* __restrict__ cl, int64_t* __restrict__ cu) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t a = 0, b = 0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      a += col[e] <= i;
      b += col[e] >= i;
    }
    cl[i] = a;
    cu[i] = b;
  }
}

// in-place exclusive scan of one 1024-element chunk per block; block totals out
__global__ void scan_chunks_kernel(int64_t n, int64_t* __restrict__ x, int64_t* __restrict__ totals) {
  __shared__ int64_t s[1024];
  const int64_t i = blockIdx.x * 1024LL + threadIdx.x;
  s[threadIdx.x] = i < n ? x[i] : 0;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int64_t t = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  const int64_t incl = s[threadIdx.x];
  const int64_t excl = threadIdx.x ? s[threadIdx.x - 1] : 0;
  if (i < n) x[i] = excl;
  if (threadIdx.x == 1023) totals[blockIdx.x] = incl;
  (void)incl;
}

__global__ void add_offsets_kernel(int64_t n, int64_t* __restrict__ x, const int64_t* __restrict__ offs) {
  const int64_t i = blockIdx.x * 1024LL + threadIdx.x;
  if (i < n) x[i] += offs[blockIdx.x];
}

__global__ void fill_lower_kernel(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                  const int64_t* __restrict__ rpL, int32_t* __restrict__ colL) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = rpL[i];
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
      if (col[e] <= i) colL[p++] = col[e];
  }
}

__global__ void fill_upper_kernel(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                  const int64_t* __restrict__ rpL, const int32_t* __restrict__ colL,
                                  const int64_t* __restrict__ rpU, int32_t* __restrict__ colU,
                                  int64_t* __restrict__ perm, int* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = rpU[i];
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      const int32_t j = col[e];
      if (j < i) continue;
      int64_t q = -1;
      for (int64_t f = rpL[j]; f < rpL[j + 1]; ++f)
        if (colL[f] == i) { q = f; break; }
      if (q < 0) { atomicOr(status, 64); q = rpL[j]; }   // pattern not symmetric
      colU[p] = j;
      perm[p] = q;
      ++p;
    }
  }
}

__global__ void gather_kernel(int64_t m, const int64_t* __restrict__ perm, const double* __restrict__ src,
                              double* __restrict__ dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = src[perm[e]];
}

// ---------------------------------------------------------------- A[P_i, P_i]
// value a_jk from row j of A (sorted columns), 0 if absent
__device__ __forceinline__ double a_at(const int64_t* rp, const int32_t* col, const double* val, int64_t j, int32_t k) {
  int64_t lo = rp[j], hi = rp[j + 1];
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (col[mid] < k) lo = mid + 1; else hi = mid;
  }
  return (lo < rp[j + 1] && col[lo] == k) ? val[lo] : 0.0;
}

__global__ void fsai_classic_kernel(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                    const double* __restrict__ val, const int64_t* __restrict__ rpL,
                                    const int32_t* __restrict__ colL, double* __restrict__ g, int* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = rpL[i];
    const int m = (int)(rpL[i + 1] - s);
    if (m < 1 || m > kMaxP) { atomicOr(status, 64); continue; }
    double L[kMaxP * kMaxP];
    for (int a = 0; a < m; ++a)
      for (int b = 0; b <= a; ++b) L[a * kMaxP + b] = a_at(rp, col, val, colL[s + a], colL[s + b]);
    bool ok = true;
    for (int c = 0; c < m && ok; ++c) {   // Cholesky, lower triangle in place
      double d = L[c * kMaxP + c];
      for (int k = 0; k < c; ++k) d -= L[c * kMaxP + k] * L[c * kMaxP + k];
      if (!(d > 0.0)) { ok = false; break; }
      d = sqrt(d);
      L[c * kMaxP + c] = d;
      for (int r = c + 1; r < m; ++r) {
        double t = L[r * kMaxP + c];
        for (int k = 0; k < c; ++k) t -= L[r * kMaxP + k] * L[c * kMaxP + k];
        L[r * kMaxP + c] = t / d;
      }
    }
    if (!ok) { atomicOr(status, kFlagNotSPD); continue; }
    // solve L L^T x = e_last: L y = e_last gives y = (0,..,0, 1/L_mm); then L^T x = y
    double x[kMaxP];
    for (int a = 0; a < m; ++a) x[a] = 0.0;
    x[m - 1] = 1.0 / L[(m - 1) * kMaxP + (m - 1)];
    for (int r = m - 1; r >= 0; --r) {
      double t = x[r];
      for (int k = r + 1; k < m; ++k) t -= L[k * kMaxP + r] * x[k];
      x[r] = t / L[r * kMaxP + r];
    }
    const double sc = 1.0 / sqrt(x[m - 1]);
    for (int a = 0; a < m; ++a) g[s + a] = x[a] * sc;
  }
}

// ---------------------------------------------------------------- features and MLP
__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
template <typename WT> __device__ __forceinline__ WT from_f(float x);
template <> __device__ __forceinline__ float from_f<float>(float x) { return x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <typename WT> __device__ __forceinline__ float rnd(float x) { return to_f(from_f<WT>(x)); }

// features of row i (order: log a_ii, then the scaled couplings
// a_ij / sqrt(a_ii a_jj) towards -x, +x, -y, +y, -z, +z, then the diagonal
// dominance (a_ii - sum |a_ij|) / a_ii); `diag` holds A's diagonal
__device__ __forceinline__ void row_features(int64_t i, const int64_t* rp, const int32_t* col, const double* val,
                                             const double* diag, int64_t nx, int64_t nxy, float f[8], double& aii) {
  const double d = diag[i];
  double offabs = 0.0, nb[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
    const int64_t j = col[e];
    if (j == i) continue;
    const double a = val[e];
    offabs += fabs(a);
    const double c = a / sqrt(d * diag[j]);
    const int64_t o = j - i;
    if (o == -1) nb[0] = c;
    else if (o == 1) nb[1] = c;
    else if (o == -nx) nb[2] = c;
    else if (o == nx) nb[3] = c;
    else if (o == -nxy) nb[4] = c;
    else if (o == nxy) nb[5] = c;
  }
  aii = d;
  f[0] = (float)log(d);
  for (int k = 0; k < 6; ++k) f[1 + k] = (float)nb[k];
  f[7] = (float)((d - offabs) / d);
}

__global__ void diag_kernel(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const double* __restrict__ val, double* __restrict__ diag, int* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
      if (col[e] == i) d = val[e];
    if (!(d > 0.0)) atomicOr(status, kFlagNotSPD);
    diag[i] = d;
  }
}

__device__ __forceinline__ int slot_of(int64_t off, int64_t nx, int64_t nxy) {
  return off == -nxy ? 0 : off == -nx ? 1 : off == -1 ? 2 : off == 0 ? 3 : -1;
}

__device__ __forceinline__ double softplus_d(double x) { return x > 30.0 ? x : log1p(exp(x)); }
__device__ __forceinline__ double sigmoid_d(double x) { return 1.0 / (1.0 + exp(-x)); }

template <typename WT>
struct MlpShared {
  WT W1[512], W2[4096], W3[448];
  float b1[64], b2[64], b3[8];
};

template <typename WT>
__device__ void load_mlp(MlpShared<WT>& m, const float* __restrict__ P) {
  for (int e = threadIdx.x; e < 512; e += blockDim.x) m.W1[e] = from_f<WT>(P[OFF_W1 + e]);
  for (int e = threadIdx.x; e < 4096; e += blockDim.x) m.W2[e] = from_f<WT>(P[OFF_W2 + e]);
  for (int e = threadIdx.x; e < 448; e += blockDim.x) m.W3[e] = from_f<WT>(P[OFF_W3 + e]);
  for (int e = threadIdx.x; e < 64; e += blockDim.x) {
    m.b1[e] = P[OFF_B1 + e];
    m.b2[e] = P[OFF_B2 + e];
  }
  for (int e = threadIdx.x; e < 7; e += blockDim.x) m.b3[e] = P[OFF_B3 + e];
  __syncthreads();
}

// Forward pass fused with the construction of G's row: G values (FP64) and
// the raw outputs o (n x 7, FP32) for the backward pass.
template <typename WT>
__global__ void __launch_bounds__(128) mlp_g_kernel(int64_t n, const int64_t* __restrict__ rp,
                                                    const int32_t* __restrict__ col, const double* __restrict__ val,
                                                    const double* __restrict__ diag,
                                                    int64_t nx, int64_t nxy, const float* __restrict__ P,
                                                    const int64_t* __restrict__ rpL, const int32_t* __restrict__ colL,
                                                    double* __restrict__ g, float* __restrict__ O) {
  __shared__ MlpShared<WT> m;
  load_mlp(m, P);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float f[8];
    double aii;
    row_features(i, rp, col, val, diag, nx, nxy, f, aii);
#pragma unroll
    for (int c = 0; c < 8; ++c) f[c] = rnd<WT>(f[c]);
    float h1[kH];
#pragma unroll
    for (int k = 0; k < kH; ++k) {
      float a = m.b1[k];
#pragma unroll
      for (int c = 0; c < 8; ++c) a = fmaf(to_f(m.W1[k * 8 + c]), f[c], a);
      h1[k] = rnd<WT>(fmaxf(a, 0.f));
    }
    float o[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) o[q] = m.b3[q];
    for (int k = 0; k < kH; ++k) {
      float a = m.b2[k];
#pragma unroll
      for (int j = 0; j < kH; ++j) a = fmaf(to_f(m.W2[k * kH + j]), h1[j], a);
      const float h2 = rnd<WT>(fmaxf(a, 0.f));
#pragma unroll
      for (int q = 0; q < 7; ++q) o[q] = fmaf(to_f(m.W3[q * kH + k]), h2, o[q]);
    }
    if (O)
#pragma unroll
      for (int q = 0; q < 7; ++q) O[i * 7 + q] = o[q];
    for (int64_t e = rpL[i]; e < rpL[i + 1]; ++e) {
      const int sl = slot_of((int64_t)colL[e] - i, nx, nxy);
      double v = 0.0;
      if (sl == 3) v = softplus_d((double)o[3]) / sqrt(aii);
      else if (sl >= 0) v = (double)o[sl] / sqrt(diag[colL[e]]);
      g[e] = v;
    }
  }
}

// ---------------------------------------------------------------- loss pieces
// out[0..2] = sum a0*b0, sum a1*b1, sum a2*a2*w2 (a null b or w counts as 1);
// deterministic two-stage reduction
__global__ void dot3_kernel(int64_t n, const double* __restrict__ a0, const double* __restrict__ b0,
                            const double* __restrict__ a1, const double* __restrict__ b1,
                            const double* __restrict__ a2, const double* __restrict__ w2,
                            double* __restrict__ partials, unsigned int* counter, double* __restrict__ out) {
  double s0 = 0, s1 = 0, s2 = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (a0) s0 += a0[i] * (b0 ? b0[i] : 1.0);
    if (a1) s1 += a1[i] * (b1 ? b1[i] : 1.0);
    if (a2) s2 += a2[i] * a2[i] * (w2 ? w2[i] : 1.0);
  }
  __shared__ double red[3][32];
  for (int off = 16; off > 0; off >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, off);
    s1 += __shfl_down_sync(0xffffffffu, s1, off);
    s2 += __shfl_down_sync(0xffffffffu, s2, off);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { red[0][warp] = s0; red[1][warp] = s1; red[2][warp] = s2; }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0;
    for (int k = 0; k < (int)(blockDim.x / 32); ++k) t += red[threadIdx.x][k];
    partials[blockIdx.x * 3 + threadIdx.x] = t;
  }
  if (!last_block_arrive(counter)) return;
  if (threadIdx.x < 3) {
    double t = 0;
    for (unsigned b = 0; b < gridDim.x; ++b) t += partials[b * 3 + threadIdx.x];
    out[threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0u;
}

// gG[e] += scale * (2 s_i w_j + 2 t_i v_j - 4 s_i v_j), scale = wgt / dots[2]
__global__ void grad_energy_kernel(int64_t n, const int64_t* __restrict__ rpL, const int32_t* __restrict__ colL,
                                   const double* __restrict__ s, const double* __restrict__ w,
                                   const double* __restrict__ t, const double* __restrict__ v,
                                   const double* __restrict__ dots, double wgt, double* __restrict__ gG) {
  const double sc = wgt / dots[2];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double si = s[i], ti = t[i];
    for (int64_t e = rpL[i]; e < rpL[i + 1]; ++e) {
      const int32_t j = colL[e];
      gG[e] += sc * (2.0 * si * w[j] + 2.0 * ti * v[j] - 4.0 * si * v[j]);
    }
  }
}

// per row: d_i = (G A G^T)_ii, GA_e = (G A)_ij on the pattern, logg_i = log g_ii
__global__ void kaporin_rows_kernel(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                    const double* __restrict__ val, const int64_t* __restrict__ rpL,
                                    const int32_t* __restrict__ colL, const double* __restrict__ g,
                                    double* __restrict__ d, double* __restrict__ GA, double* __restrict__ logg,
                                    int* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = rpL[i];
    const int m = (int)(rpL[i + 1] - s);
    double di = 0.0;
    for (int a = 0; a < m; ++a) {
      double t = 0.0;
      for (int b = 0; b < m; ++b) t += a_at(rp, col, val, colL[s + a], colL[s + b]) * g[s + b];
      GA[s + a] = t;
      di += g[s + a] * t;
    }
    d[i] = di;
    const double gii = g[rpL[i + 1] - 1];   // the diagonal is the last lower entry
    if (!(gii > 0.0)) atomicOr(status, kFlagNaN);
    logg[i] = log(gii);
  }
}

// gG[e] += gamma * (2 GA_e / (n md) - [diag] 2 / (n g_ii)), md = sums[0]/n
__global__ void grad_kaporin_kernel(int64_t n, const int64_t* __restrict__ rpL, const double* __restrict__ g,
                                    const double* __restrict__ GA, const double* __restrict__ sums, double gamma,
                                    double* __restrict__ gG) {
  const double md = sums[0] / (double)n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e1 = rpL[i + 1];
    for (int64_t e = rpL[i]; e < e1; ++e) {
      double v = 2.0 * GA[e] / ((double)n * md);
      if (e == e1 - 1) v -= 2.0 / ((double)n * g[e]);
      gG[e] += gamma * v;
    }
  }
}

// ---------------------------------------------------------------- IC(0)
// The no-fill incomplete Cholesky factor L on the lower pattern of A (the
// paper preconditions with no-fill incomplete factorizations, Sec. 5.4-5.5).
// The left-looking recurrence s = a_ij - sum_{k<j} l_ik l_jk, l_ij = s / l_jj,
// l_ii = sqrt(s) is solved as a fixed point: every sweep recomputes all
// entries in parallel from the previous sweep's values (so the result does
// not depend on thread order) until no entry moves; the fixed point is the
// IC(0) factor, reached exactly after at most the depth of the dependency
// graph and, for these operators, after a few tens of sweeps.

// starting values l_ij = a_ij / sqrt(a_jj), l_ii = sqrt(a_ii)
__global__ void ic0_init_kernel(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                const double* __restrict__ val, const double* __restrict__ diag,
                                const int64_t* __restrict__ rpL, const int32_t* __restrict__ colL,
                                double* __restrict__ l) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int64_t e = rpL[i]; e < rpL[i + 1]; ++e) {
      const int32_t j = colL[e];
      l[e] = j == i ? sqrt(diag[i]) : a_at(rp, col, val, i, j) / sqrt(diag[j]);
    }
}

// One fixed-point sweep lnew = F(lold); stats[0] = max |lnew - lold|,
// stats[1] = max |lnew| (non-negative doubles compare as their bit patterns);
// strict: a non-positive pivot raises kFlagNotSPD (IC(0) breakdown).
__global__ void __launch_bounds__(256) ic0_sweep_kernel(int64_t n, const int64_t* __restrict__ rp,
                                                        const int32_t* __restrict__ col,
                                                        const double* __restrict__ val,
                                                        const int64_t* __restrict__ rpL,
                                                        const int32_t* __restrict__ colL,
                                                        const double* __restrict__ lold, double* __restrict__ lnew,
                                                        unsigned long long* stats, int strict, int* status) {
  double dmax = 0.0, vmax = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r0 = rpL[i];
    for (int64_t e = r0; e < rpL[i + 1]; ++e) {
      const int32_t j = colL[e];
      double s = a_at(rp, col, val, i, j);
      // sum over k < j of l_ik l_jk: merge row i (entries before e) with row j
      // (entries before its diagonal, which is the last of the row)
      int64_t pi = r0, pj = rpL[j];
      const int64_t ej = rpL[j + 1] - 1;
      while (pi < e && pj < ej) {
        const int32_t ci = colL[pi], cj = colL[pj];
        if (ci == cj) {
          s -= lold[pi] * lold[pj];
          ++pi;
          ++pj;
        } else if (ci < cj) {
          ++pi;
        } else {
          ++pj;
        }
      }
      double v;
      if (j < i) {
        v = s / lold[ej];
      } else {
        if (!(s > 0.0)) {
          if (strict) atomicOr(status, kFlagNotSPD);
          s = 1e-300;
        }
        v = sqrt(s);
      }
      lnew[e] = v;
      dmax = fmax(dmax, fabs(v - lold[e]));
      vmax = fmax(vmax, fabs(v));
    }
  }
  __shared__ double red[2][8];
  for (int off = 16; off > 0; off >>= 1) {
    dmax = fmax(dmax, __shfl_down_sync(0xffffffffu, dmax, off));
    vmax = fmax(vmax, __shfl_down_sync(0xffffffffu, vmax, off));
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = dmax;
    red[1][threadIdx.x >> 5] = vmax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      dmax = fmax(dmax, red[0][w]);
      vmax = fmax(vmax, red[1][w]);
    }
    atomicMax(stats, (unsigned long long)__double_as_longlong(dmax));
    atomicMax(stats + 1, (unsigned long long)__double_as_longlong(vmax));
  }
}

// dinv[i] = 1 / l_ii (the diagonal is the last entry of each lower row)
__global__ void lower_diag_inv_kernel(int64_t n, const int64_t* __restrict__ rpL, const double* __restrict__ l,
                                      double* __restrict__ dinv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dinv[i] = 1.0 / l[rpL[i + 1] - 1];
}

// ---------------------------------------------------------------- MLP backward
// One tile = 64 rows: threads 0..63 recompute their row's activations and
// back-propagate dL/do into shared memory; then all 128 threads accumulate
// the weight gradients of the tile (each owns fixed entries, so sums are in a
// fixed order); per-CTA partials are summed in CTA order by the last CTA.
constexpr int kBR = 64;               // rows per tile
constexpr int kRowF = 8 + 64 + 64 + 8 + 64 + 64;   // f, h1, h2, dO(7+pad), dh2, dh1
constexpr int kEntPerThread = (kNParams + 127) / 128;

template <typename WT>
__global__ void __launch_bounds__(128) mlp_backward_kernel(
    int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const double* __restrict__ val,
    const double* __restrict__ diag, int64_t nx, int64_t nxy, const float* __restrict__ P,
    const int64_t* __restrict__ rpL,
    const int32_t* __restrict__ colL, const float* __restrict__ O, const double* __restrict__ gG,
    double* __restrict__ partials, unsigned int* counter, double* __restrict__ grad) {
  __shared__ MlpShared<WT> m;
  extern __shared__ float rows[];   // [kBR][kRowF]
  load_mlp(m, P);
  const int tid = threadIdx.x;
  float acc[kEntPerThread];
#pragma unroll
  for (int q = 0; q < kEntPerThread; ++q) acc[q] = 0.f;
  const int64_t ntiles = (n + kBR - 1) / kBR;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t i = tile * kBR + tid;
    if (tid < kBR) {
      float* R = rows + tid * kRowF;
      float* f = R;
      float* h1 = R + 8;
      float* h2 = R + 72;
      float* dO = R + 136;
      float* dh2 = R + 144;
      float* dh1 = R + 208;
      if (i < n) {
        double aii;
        float ff[8];
        row_features(i, rp, col, val, diag, nx, nxy, ff, aii);
        for (int c = 0; c < 8; ++c) f[c] = rnd<WT>(ff[c]);
        for (int k = 0; k < kH; ++k) {
          float a = m.b1[k];
          for (int c = 0; c < 8; ++c) a = fmaf(to_f(m.W1[k * 8 + c]), f[c], a);
          h1[k] = rnd<WT>(fmaxf(a, 0.f));
        }
        for (int k = 0; k < kH; ++k) {
          float a = m.b2[k];
          for (int j = 0; j < kH; ++j) a = fmaf(to_f(m.W2[k * kH + j]), h1[j], a);
          h2[k] = rnd<WT>(fmaxf(a, 0.f));
        }
        // dL/do from dL/dG (g_ii = softplus(o_c)/sqrt(a_ii), g_ij = o_dir/sqrt(a_ii))
        for (int q = 0; q < 8; ++q) dO[q] = 0.f;
        for (int64_t e = rpL[i]; e < rpL[i + 1]; ++e) {
          const int sl = slot_of((int64_t)colL[e] - i, nx, nxy);
          if (sl == 3) dO[3] += (float)(gG[e] * sigmoid_d((double)O[i * 7 + 3]) / sqrt(aii));
          else if (sl >= 0) dO[sl] += (float)(gG[e] / sqrt(diag[colL[e]]));
        }
        for (int k = 0; k < kH; ++k) {
          float a = 0.f;
          for (int q = 0; q < 7; ++q) a = fmaf(to_f(m.W3[q * kH + k]), dO[q], a);
          dh2[k] = h2[k] > 0.f ? a : 0.f;
        }
        for (int j = 0; j < kH; ++j) {
          float a = 0.f;
          for (int k = 0; k < kH; ++k) a = fmaf(to_f(m.W2[k * kH + j]), dh2[k], a);
          dh1[j] = h1[j] > 0.f ? a : 0.f;
        }
      } else {
        for (int c = 0; c < kRowF; ++c) R[c] = 0.f;
      }
    }
    __syncthreads();
    // weight-gradient entries owned by this thread: e = tid + 128 q (the entry
    // loop is unrolled so acc stays in registers; the row loops are not, which
    // keeps the kernel small -- the order of every sum is the same either way)
#pragma unroll
    for (int q = 0; q < kEntPerThread; ++q) {
      const int e = tid + 128 * q;
      if (e >= kNParams) break;
      float s = 0.f;
      if (e < OFF_B1) {                 // W1[k][c]: dh1_k f_c
        const int k = e >> 3, c = e & 7;
#pragma unroll 1
        for (int r = 0; r < kBR; ++r) s = fmaf(rows[r * kRowF + 208 + k], rows[r * kRowF + c], s);
      } else if (e < OFF_W2) {          // b1[k]
        const int k = e - OFF_B1;
#pragma unroll 1
        for (int r = 0; r < kBR; ++r) s += rows[r * kRowF + 208 + k];
      } else if (e < OFF_B2) {          // W2[k][j]: dh2_k h1_j
        const int k = (e - OFF_W2) >> 6, j = (e - OFF_W2) & 63;
#pragma unroll 1
        for (int r = 0; r < kBR; ++r) s = fmaf(rows[r * kRowF + 144 + k], rows[r * kRowF + 8 + j], s);
      } else if (e < OFF_W3) {          // b2[k]
        const int k = e - OFF_B2;
#pragma unroll 1
        for (int r = 0; r < kBR; ++r) s += rows[r * kRowF + 144 + k];
      } else if (e < OFF_B3) {          // W3[q][k]: dO_q h2_k
        const int qq = (e - OFF_W3) >> 6, k = (e - OFF_W3) & 63;
#pragma unroll 1
        for (int r = 0; r < kBR; ++r) s = fmaf(rows[r * kRowF + 136 + qq], rows[r * kRowF + 72 + k], s);
      } else {                          // b3[q]
        const int qq = e - OFF_B3;
#pragma unroll 1
        for (int r = 0; r < kBR; ++r) s += rows[r * kRowF + 136 + qq];
      }
      acc[q] += s;
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < kEntPerThread; ++q) {
    const int e = tid + 128 * q;
    if (e < kNParams) partials[(size_t)blockIdx.x * kNParams + e] = (double)acc[q];
  }
  if (!last_block_arrive(counter)) return;
  for (int e = tid; e < kNParams; e += blockDim.x) {
    double t = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) t += partials[(size_t)b * kNParams + e];
    grad[e] = t;
  }
  __syncthreads();
  if (tid == 0) *counter = 0u;
}

// Adam (Kingma and Ba, 2015) on the FP32 master weights
__global__ void adam_kernel(int np, float* __restrict__ P, float* __restrict__ mom, float* __restrict__ vel,
                            const double* __restrict__ g, float lr, float b1, float b2, float eps, int step) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= np) return;
  const float gr = (float)g[e];
  const float m1 = b1 * mom[e] + (1.f - b1) * gr;
  const float v1 = b2 * vel[e] + (1.f - b2) * gr * gr;
  mom[e] = m1;
  vel[e] = v1;
  const float mh = m1 / (1.f - powf(b1, (float)step));
  const float vh = v1 / (1.f - powf(b2, (float)step));
  P[e] -= lr * mh / (sqrtf(vh) + eps);
}

inline unsigned blocks_for(const Ctx& c, int64_t n) {
  const int64_t g = (n + 255) / 256, cap = (int64_t)c.sms * 8;
  return (unsigned)std::max<int64_t>(1, std::min(g, cap));
}

}  // namespace trplk

// ================================================================ host side
namespace {

using namespace trplk;

// The pattern of G (lower triangle of A with the diagonal) and of G^T.
struct FsaiOp {
  int64_t n = 0, nnzL = 0, nnzU = 0;
  const int64_t* rp = nullptr;
  const int32_t* col = nullptr;
  const double* val = nullptr;
  double* diag = nullptr;
  int64_t *rpL = nullptr, *rpU = nullptr, *perm = nullptr;
  int32_t *colL = nullptr, *colU = nullptr;
};

void exclusive_scan(trplk_handle* h, int64_t* x, int64_t n, const std::string& tag, int64_t* total) {
  const Ctx& c = h->ctx;
  const int64_t nb = (n + 1023) / 1024;
  auto* tot = static_cast<int64_t*>(h->get(tag + ".scan", nb * sizeof(int64_t)));
  {
    ProfScope ps(c, PK_OTHER, 0.0);
    scan_chunks_kernel<<<(unsigned)nb, 1024, 0, c.stream>>>(n, x, tot);
    check_launch("scan_chunks");
  }
  std::vector<int64_t> ht(nb);
  TRPLK_CUDA_TRY(cudaMemcpyAsync(ht.data(), tot, nb * sizeof(int64_t), cudaMemcpyDeviceToHost, c.stream));
  h->sync();
  int64_t run = 0;
  for (int64_t b = 0; b < nb; ++b) {
    const int64_t t = ht[b];
    ht[b] = run;
    run += t;
  }
  TRPLK_CUDA_TRY(cudaMemcpyAsync(tot, ht.data(), nb * sizeof(int64_t), cudaMemcpyHostToDevice, c.stream));
  {
    ProfScope ps(c, PK_OTHER, 0.0);
    add_offsets_kernel<<<(unsigned)nb, 1024, 0, c.stream>>>(n, x, tot);
    check_launch("add_offsets");
  }
  h->sync();
  *total = run;
}

FsaiOp build_pattern(trplk_handle* h, int64_t n, const int64_t* rp, const int32_t* col, const double* val,
                     const std::string& tag) {
  const Ctx& c = h->ctx;
  FsaiOp op;
  op.n = n;
  op.rp = rp;
  op.col = col;
  op.val = val;
  op.rpL = static_cast<int64_t*>(h->get(tag + ".rpL", (n + 1) * sizeof(int64_t)));
  op.rpU = static_cast<int64_t*>(h->get(tag + ".rpU", (n + 1) * sizeof(int64_t)));
  {
    ProfScope ps(c, PK_OTHER, 0.0);
    tri_count_kernel<<<blocks_for(c, n), 256, 0, c.stream>>>(n, rp, col, op.rpL, op.rpU);
    check_launch("tri_count");
  }
  exclusive_scan(h, op.rpL, n, tag + ".L", &op.nnzL);
  exclusive_scan(h, op.rpU, n, tag + ".U", &op.nnzU);
  TRPLK_CUDA_TRY(cudaMemcpyAsync(op.rpL + n, &op.nnzL, sizeof(int64_t), cudaMemcpyHostToDevice, c.stream));
  TRPLK_CUDA_TRY(cudaMemcpyAsync(op.rpU + n, &op.nnzU, sizeof(int64_t), cudaMemcpyHostToDevice, c.stream));
  op.colL = static_cast<int32_t*>(h->get(tag + ".colL", op.nnzL * sizeof(int32_t)));
  op.colU = static_cast<int32_t*>(h->get(tag + ".colU", op.nnzU * sizeof(int32_t)));
  op.perm = static_cast<int64_t*>(h->get(tag + ".perm", op.nnzU * sizeof(int64_t)));
  h->clear_status();
  {
    ProfScope ps(c, PK_OTHER, 0.0);
    fill_lower_kernel<<<blocks_for(c, n), 256, 0, c.stream>>>(n, rp, col, op.rpL, op.colL);
    check_launch("fill_lower");
  }
  {
    ProfScope ps(c, PK_OTHER, 0.0);
    fill_upper_kernel<<<blocks_for(c, n), 256, 0, c.stream>>>(n, rp, col, op.rpL, op.colL, op.rpU, op.colU, op.perm,
                                                             c.status);
    check_launch("fill_upper");
  }
  op.diag = static_cast<double*>(h->get(tag + ".diag", n * sizeof(double)));
  {
    ProfScope ps(c, PK_OTHER, 0.0);
    diag_kernel<<<blocks_for(c, n), 256, 0, c.stream>>>(n, rp, col, val, op.diag, c.status);
    check_launch("diag");
  }
  const int st = h->read_status();
  if (st & 64) throw Error(TRPLK_EINVAL, "FSAI needs a structurally symmetric matrix");
  if (st & kFlagNotSPD) throw Error(TRPLK_NOT_SPD_B, "FSAI needs a positive diagonal");
  return op;
}

void check_dims(const FsaiOp& op, const int32_t* dims) {
  if (!dims || dims[0] < 2 || dims[1] < 2 || dims[2] < 1 ||
      (int64_t)dims[0] * dims[1] * dims[2] != op.n)
    throw Error(TRPLK_EINVAL, "learned FSAI needs grid dims (nx, ny, nz >= 2, 2, 1) with nx*ny*nz = n");
}

// G values (FP64, lower pattern order): classical, or from the MLP weights
// `P` (device FP32 packed; bf16 selects BF16 weights/activations).
void fsai_values(trplk_handle* h, const FsaiOp& op, int kind, const int32_t* dims, const float* P, bool bf16,
                 double* g, float* O) {
  const Ctx& c = h->ctx;
  h->clear_status();
  if (kind == 0) {
    ProfScope ps(c, PK_OTHER, 0.0);
    fsai_classic_kernel<<<blocks_for(c, op.n), 128, 0, c.stream>>>(op.n, op.rp, op.col, op.val, op.rpL, op.colL, g,
                                                                   c.status);
    check_launch("fsai_classic");
  } else {
    check_dims(op, dims);
    const int64_t nx = dims[0], nxy = (int64_t)dims[0] * dims[1];
    ProfScope ps(c, PK_OTHER, 0.0);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((op.n + 127) / 128, (int64_t)c.sms * 8));
    if (bf16)
      mlp_g_kernel<__nv_bfloat16><<<grid, 128, 0, c.stream>>>(op.n, op.rp, op.col, op.val, op.diag, nx, nxy, P,
                                                              op.rpL, op.colL, g, O);
    else
      mlp_g_kernel<float><<<grid, 128, 0, c.stream>>>(op.n, op.rp, op.col, op.val, op.diag, nx, nxy, P, op.rpL,
                                                      op.colL, g, O);
    check_launch("mlp_g");
  }
  const int st = h->read_status();
  if (st & 64) throw Error(TRPLK_EINVAL, "FSAI pattern row longer than 16 entries");
  if (st & kFlagNotSPD) throw Error(TRPLK_NOT_SPD_B, "classical FSAI: a principal block of A is not SPD");
}

struct LossOut {
  double L = 0, E = 0, K = 0;
};

// Loss and gradient w.r.t. the MLP weights for one operator and its vectors
// V (device, n x nv column-major, ld = n).  grad: device double[kNParams].
LossOut loss_grad(trplk_handle* h, const FsaiOp& op, const int32_t* dims, const float* P, bool bf16, const double* V,
                  int nv, double gamma, double* grad, const std::string& tag) {
  const Ctx& c = h->ctx;
  const int64_t n = op.n;
  double* g = static_cast<double*>(h->get(tag + ".g", op.nnzL * sizeof(double)));
  double* gT = static_cast<double*>(h->get(tag + ".gT", op.nnzU * sizeof(double)));
  float* O = static_cast<float*>(h->get(tag + ".O", n * 7 * sizeof(float)));
  double* gG = static_cast<double*>(h->get(tag + ".gG", op.nnzL * sizeof(double)));
  double* GA = static_cast<double*>(h->get(tag + ".GA", op.nnzL * sizeof(double)));
  double* s = static_cast<double*>(h->get(tag + ".s", n * sizeof(double)));
  double* u = static_cast<double*>(h->get(tag + ".u", n * sizeof(double)));
  double* w = static_cast<double*>(h->get(tag + ".w", n * sizeof(double)));
  double* t = static_cast<double*>(h->get(tag + ".t", n * sizeof(double)));
  double* dv = static_cast<double*>(h->get(tag + ".dinv", n * sizeof(double)));
  double* dk = static_cast<double*>(h->get(tag + ".d", n * sizeof(double)));
  double* lg = static_cast<double*>(h->get(tag + ".logg", n * sizeof(double)));
  double* dots = static_cast<double*>(h->get(tag + ".dots", 8 * sizeof(double)));
  fsai_values(h, op, 1, dims, P, bf16, g, O);
  {
    ProfScope ps(c, PK_OTHER, 0.0);
    gather_kernel<<<blocks_for(c, op.nnzU), 256, 0, c.stream>>>(op.nnzU, op.perm, g, gT);
    check_launch("gather");
  }
  DevCsr<double> G{n, op.nnzL, op.rpL, op.colL, g};
  DevCsr<double> GT{n, op.nnzU, op.rpU, op.colU, gT};
  DevCsr<double> A{n, 0, op.rp, op.col, op.val};
  DevCsr<double> Ad{n, 0, op.rp, op.col, op.val};
  jacobi_dinv<double>(c, Ad, dv);
  TRPLK_CUDA_TRY(cudaMemsetAsync(gG, 0, op.nnzL * sizeof(double), c.stream));
  const unsigned nb = std::min<unsigned>(blocks_for(c, n), (unsigned)kMaxPartials);
  LossOut out;
  double* hp = h->host(8);
  for (int k = 0; k < nv; ++k) {
    const double* v = V + (size_t)k * n;
    spmv<double>(c, G, v, s);
    spmv<double>(c, GT, s, u);
    spmv<double>(c, A, u, w);
    spmv<double>(c, G, w, t);
    {
      ProfScope ps(c, PK_OTHER, 0.0);
      dot3_kernel<<<nb, 256, 0, c.stream>>>(n, u, w, s, s, v, dv, c.partials, c.counter, dots);
      check_launch("dot3");
    }
    {
      ProfScope ps(c, PK_OTHER, 0.0);
      grad_energy_kernel<<<blocks_for(c, n), 256, 0, c.stream>>>(n, op.rpL, op.colL, s, w, t, v, dots, 1.0 / nv, gG);
      check_launch("grad_energy");
    }
    TRPLK_CUDA_TRY(cudaMemcpyAsync(hp, dots, 3 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    h->sync();
    out.E += (hp[0] - 2.0 * hp[1]) / hp[2] / nv;
  }
  h->clear_status();
  {
    ProfScope ps(c, PK_OTHER, 0.0);
    kaporin_rows_kernel<<<blocks_for(c, n), 256, 0, c.stream>>>(n, op.rp, op.col, op.val, op.rpL, op.colL, g, dk, GA,
                                                                lg, c.status);
    check_launch("kaporin_rows");
  }
  {
    ProfScope ps(c, PK_OTHER, 0.0);
    dot3_kernel<<<nb, 256, 0, c.stream>>>(n, dk, nullptr, lg, nullptr, nullptr, nullptr, c.partials, c.counter, dots);
    check_launch("dot3");
  }
  {
    ProfScope ps(c, PK_OTHER, 0.0);
    grad_kaporin_kernel<<<blocks_for(c, n), 256, 0, c.stream>>>(n, op.rpL, g, GA, dots, gamma, gG);
    check_launch("grad_kaporin");
  }
  TRPLK_CUDA_TRY(cudaMemcpyAsync(hp, dots, 3 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  h->sync();
  if (h->read_status() & kFlagNaN) throw Error(TRPLK_NAN, "FSAI diagonal not positive");
  out.K = std::log(hp[0] / (double)n) - 2.0 * hp[1] / (double)n;
  out.L = out.E + gamma * out.K;
  // back through the MLP to the weights
  const unsigned gb = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>({(n + kBR - 1) / kBR, (int64_t)c.sms * 2, (int64_t)kMaxPartials}));
  double* part = static_cast<double*>(h->get("fsai.bwd.partials", (size_t)gb * kNParams * sizeof(double)));
  const size_t smem = (size_t)kBR * kRowF * sizeof(float);
  const int64_t nx = dims[0], nxy = (int64_t)dims[0] * dims[1];
  {
    ProfScope ps(c, PK_OTHER, 0.0);
    if (bf16) {
      TRPLK_CUDA_TRY(cudaFuncSetAttribute(mlp_backward_kernel<__nv_bfloat16>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      mlp_backward_kernel<__nv_bfloat16><<<gb, 128, smem, c.stream>>>(n, op.rp, op.col, op.val, op.diag, nx, nxy, P,
                                                                       op.rpL, op.colL, O, gG, part, c.counter, grad);
    } else {
      TRPLK_CUDA_TRY(cudaFuncSetAttribute(mlp_backward_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
      mlp_backward_kernel<float><<<gb, 128, smem, c.stream>>>(n, op.rp, op.col, op.val, op.diag, nx, nxy, P, op.rpL,
                                                              op.colL, O, gG, part, c.counter, grad);
    }
    check_launch("mlp_backward");
  }
  return out;
}

// IC(0) values (lower pattern order) into l: fixed-point sweeps from the
// starting values until the largest change is <= 4 u max |l| (u = 2^-53),
// read back every 4 sweeps; a last strict sweep checks every pivot.
void ic0_values(trplk_handle* h, const FsaiOp& op, double* l) {
  const Ctx& c = h->ctx;
  double* l2 = static_cast<double*>(h->get("ic0.l2", op.nnzL * sizeof(double)));
  auto* stats = static_cast<unsigned long long*>(h->get("ic0.stats", 2 * sizeof(unsigned long long)));
  h->clear_status();
  {
    ProfScope ps(c, PK_OTHER, 0.0);
    ic0_init_kernel<<<blocks_for(c, op.n), 256, 0, c.stream>>>(op.n, op.rp, op.col, op.val, op.diag, op.rpL,
                                                               op.colL, l);
    check_launch("ic0_init");
  }
  constexpr int kMaxSweeps = 4000;
  double* cur = l;
  double* nxt = l2;
  bool done = false;
  for (int sw = 1; sw <= kMaxSweeps && !done; ++sw) {
    const bool check = (sw % 4) == 0 || sw == kMaxSweeps;
    if (check) TRPLK_CUDA_TRY(cudaMemsetAsync(stats, 0, 2 * sizeof(unsigned long long), c.stream));
    {
      ProfScope ps(c, PK_OTHER, 0.0);
      ic0_sweep_kernel<<<blocks_for(c, op.n), 256, 0, c.stream>>>(op.n, op.rp, op.col, op.val, op.rpL, op.colL, cur,
                                                                  nxt, stats, 0, c.status);
      check_launch("ic0_sweep");
    }
    std::swap(cur, nxt);
    if (check) {
      unsigned long long hs[2];
      TRPLK_CUDA_TRY(cudaMemcpyAsync(hs, stats, sizeof(hs), cudaMemcpyDeviceToHost, c.stream));
      h->sync();
      double dmax, vmax;
      memcpy(&dmax, &hs[0], 8);
      memcpy(&vmax, &hs[1], 8);
      if (!(dmax == dmax) || !(vmax == vmax)) throw Error(TRPLK_NAN, "IC(0) sweeps produced NaN");
      done = dmax <= 4.0 * 1.1102230246251565e-16 * vmax;
    }
  }
  if (!done) throw Error(TRPLK_EINVAL, "IC(0) fixed-point sweeps did not converge");
  // one more sweep from the converged values, strict about the pivots
  {
    ProfScope ps(c, PK_OTHER, 0.0);
    ic0_sweep_kernel<<<blocks_for(c, op.n), 256, 0, c.stream>>>(op.n, op.rp, op.col, op.val, op.rpL, op.colL, cur, nxt,
                                                                stats, 1, c.status);
    check_launch("ic0_sweep");
  }
  if (nxt != l) TRPLK_CUDA_TRY(cudaMemcpyAsync(l, nxt, op.nnzL * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
  if (h->read_status() & kFlagNotSPD) throw Error(TRPLK_NOT_SPD_B, "IC(0) breakdown: a pivot is not positive");
}

void upload_weights(trplk_handle* h, const float* host, float* dev) {
  TRPLK_CUDA_TRY(cudaMemcpyAsync(dev, host, kNParams * sizeof(float), cudaMemcpyHostToDevice, h->ctx.stream));
}

}  // namespace

// Preconditioner for trplk_solve (declared in handle.h).
FsaiPrecond build_fsai_precond(trplk_handle* h, const DevCsr<double>& A, int kind, const int32_t* dims,
                               const float* weights_host, bool bf16, bool need32) {
  const Ctx& c = h->ctx;
  FsaiPrecond pc;
  FsaiOp op = build_pattern(h, A.n, A.rowptr, A.col, A.val, "precond");
  double* g = static_cast<double*>(h->get("precond.g", op.nnzL * sizeof(double)));
  double* gT = static_cast<double*>(h->get("precond.gT", op.nnzU * sizeof(double)));
  float* P = nullptr;
  if (kind == 1) {
    if (!weights_host) throw Error(TRPLK_EINVAL, "learned FSAI needs MLP weights");
    P = static_cast<float*>(h->get("precond.mlp", kNParams * sizeof(float)));
    upload_weights(h, weights_host, P);
  }
  if (kind == 2)
    ic0_values(h, op, g);
  else
    fsai_values(h, op, kind, dims, P, bf16, g, nullptr);
  {
    ProfScope ps(c, PK_OTHER, 0.0);
    gather_kernel<<<blocks_for(c, op.nnzU), 256, 0, c.stream>>>(op.nnzU, op.perm, g, gT);
    check_launch("gather");
  }
  if (kind == 2) {
    const int64_t ld = round_up(op.n, 256);
    pc.ic0 = true;
    pc.dinv = static_cast<double*>(h->get("precond.dinv", ld * sizeof(double), true));
    {
      ProfScope ps(c, PK_OTHER, 0.0);
      lower_diag_inv_kernel<<<blocks_for(c, op.n), 256, 0, c.stream>>>(op.n, op.rpL, g, pc.dinv);
      check_launch("lower_diag_inv");
    }
    if (need32) {
      pc.dinvf = static_cast<float*>(h->get("precond.dinvf", ld * sizeof(float), true));
      convert<float, double>(c, ld, pc.dinv, pc.dinvf);
    }
  }
  pc.G = DevCsr<double>{op.n, op.nnzL, op.rpL, op.colL, g};
  pc.GT = DevCsr<double>{op.n, op.nnzU, op.rpU, op.colU, gT};
  if (need32) {
    float* gf = static_cast<float*>(h->get("precond.gf", op.nnzL * sizeof(float)));
    float* gTf = static_cast<float*>(h->get("precond.gTf", op.nnzU * sizeof(float)));
    convert<float, double>(c, op.nnzL, g, gf);
    convert<float, double>(c, op.nnzU, gT, gTf);
    pc.Gf = DevCsr<float>{op.n, op.nnzL, op.rpL, op.colL, gf};
    pc.GTf = DevCsr<float>{op.n, op.nnzU, op.rpU, op.colU, gTf};
  }
  attach_sell(h, pc.G, "precond.G", need32 ? &pc.Gf : nullptr);
  attach_sell(h, pc.GT, "precond.GT", need32 ? &pc.GTf : nullptr);
  pc.ok = true;
  return pc;
}

// ================================================================ C ABI
namespace {
DevCsr<double> dev64(const trplk_csr* M) {
  if (!M || !M->on_device || M->dtype != TRPLK_F64 || M->n < 1)
    throw Error(TRPLK_EINVAL, "FSAI calls take a device CSR with F64 values");
  return DevCsr<double>{M->n, M->nnz, M->rowptr, M->col, static_cast<const double*>(M->val)};
}
}  // namespace

extern "C" {

int trplk_mlp_param_count(void) { return kNParams; }

trplk_status trplk_fsai_mlp_init(float* weights, uint64_t seed) {
  if (!weights) return TRPLK_EINVAL;
  // SplitMix64 (Steele, Lea, Flood 2014) on a counter, 53-bit uniforms in
  // (0, 1], standard normals by the Box-Muller transform
  uint64_t ctr = 0;
  auto uniform = [&]() {
    uint64_t z = (seed ^ ctr++) + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return ((z >> 11) + 1) * (1.0 / 9007199254740992.0);
  };
  auto normal = [&]() {
    const double u1 = uniform(), u2 = uniform();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  };
  float* P = weights;
  for (int i = 0; i < kNParams; ++i) P[i] = 0.0f;
  for (int i = 0; i < 64 * 8; ++i) P[i] = (float)(normal() * std::sqrt(2.0 / 8.0));               // W1
  for (int i = 0; i < 64 * 64; ++i) P[576 + i] = (float)(normal() * std::sqrt(2.0 / 64.0));      // W2
  P[kNParams - 7 + 3] = (float)std::log(std::expm1(1.0));                                          // b3[c]
  return TRPLK_OK;
}

trplk_status trplk_fsai_values(trplk_handle* h, const trplk_csr* A, int kind, const int32_t* dims,
                               const float* weights, int bf16, double* g, int64_t* nnz_lower) {
  return guarded(h, [&]() -> trplk_status {
    if (kind < 0 || kind > 2) throw Error(TRPLK_EINVAL, "kind must be 0 (classical), 1 (learned) or 2 (IC(0))");
    DevCsr<double> a = dev64(A);
    FsaiOp op = build_pattern(h, a.n, a.rowptr, a.col, a.val, "step.fsai");
    if (nnz_lower) *nnz_lower = op.nnzL;
    if (!g) return TRPLK_OK;
    if (kind == 2) {
      ic0_values(h, op, g);
      h->sync();
      return TRPLK_OK;
    }
    float* P = nullptr;
    if (kind == 1) {
      if (!weights) throw Error(TRPLK_EINVAL, "learned FSAI needs MLP weights");
      P = static_cast<float*>(h->get("step.fsai.mlp", kNParams * sizeof(float)));
      upload_weights(h, weights, P);
    }
    fsai_values(h, op, kind, dims, P, bf16 != 0, g, nullptr);
    h->sync();
    return TRPLK_OK;
  });
}

trplk_status trplk_fsai_apply(trplk_handle* h, const trplk_csr* A, const double* g, const double* x, double* y) {
  return guarded(h, [&]() -> trplk_status {
    if (!g || !x || !y || x == y) throw Error(TRPLK_EINVAL, "bad FSAI apply arguments");
    DevCsr<double> a = dev64(A);
    const Ctx& c = h->ctx;
    FsaiOp op = build_pattern(h, a.n, a.rowptr, a.col, a.val, "step.fsai");
    double* gT = static_cast<double*>(h->get("step.fsai.gT", op.nnzU * sizeof(double)));
    double* t = static_cast<double*>(h->get("step.fsai.t", op.n * sizeof(double)));
    {
      ProfScope ps(c, PK_OTHER, 0.0);
      gather_kernel<<<blocks_for(c, op.nnzU), 256, 0, c.stream>>>(op.nnzU, op.perm, g, gT);
      check_launch("gather");
    }
    DevCsr<double> G{op.n, op.nnzL, op.rpL, op.colL, g};
    DevCsr<double> GT{op.n, op.nnzU, op.rpU, op.colU, gT};
    attach_sell(h, G, "step.fsai.G", nullptr);
    attach_sell(h, GT, "step.fsai.GT", nullptr);
    spmv<double>(c, G, x, t);
    spmv<double>(c, GT, t, y);
    h->sync();
    return TRPLK_OK;
  });
}

trplk_status trplk_ic0_apply(trplk_handle* h, const trplk_csr* A, const double* l, const double* x, double* y) {
  return guarded(h, [&]() -> trplk_status {
    if (!l || !x || !y || x == y) throw Error(TRPLK_EINVAL, "bad IC(0) apply arguments");
    DevCsr<double> a = dev64(A);
    const Ctx& c = h->ctx;
    FsaiOp op = build_pattern(h, a.n, a.rowptr, a.col, a.val, "step.fsai");
    const int64_t ld = round_up(op.n, 256);
    double* lT = static_cast<double*>(h->get("step.fsai.gT", op.nnzU * sizeof(double)));
    double* dv = static_cast<double*>(h->get("step.ic0.dinv", ld * sizeof(double), true));
    double* in = static_cast<double*>(h->get("step.ic0.in", ld * sizeof(double), true));
    double* out = static_cast<double*>(h->get("step.ic0.out", ld * sizeof(double), true));
    double* t[3];
    for (int i = 0; i < 3; ++i)
      t[i] = static_cast<double*>(h->get("step.ic0.t" + std::to_string(i), ld * sizeof(double), true));
    {
      ProfScope ps(c, PK_OTHER, 0.0);
      gather_kernel<<<blocks_for(c, op.nnzU), 256, 0, c.stream>>>(op.nnzU, op.perm, l, lT);
      check_launch("gather");
    }
    {
      ProfScope ps(c, PK_OTHER, 0.0);
      lower_diag_inv_kernel<<<blocks_for(c, op.n), 256, 0, c.stream>>>(op.n, op.rpL, l, dv);
      check_launch("lower_diag_inv");
    }
    DevCsr<double> L{op.n, op.nnzL, op.rpL, op.colL, l};
    DevCsr<double> LT{op.n, op.nnzU, op.rpU, op.colU, lT};
    attach_sell(h, L, "step.ic0.L", nullptr);
    attach_sell(h, LT, "step.ic0.LT", nullptr);
    TRPLK_CUDA_TRY(cudaMemcpyAsync(in, x, op.n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    ic0_apply<double>(c, ld, L, LT, dv, kIc0Sweeps, in, out, t[0], t[1], t[2]);
    TRPLK_CUDA_TRY(cudaMemcpyAsync(y, out, op.n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    h->sync();
    return TRPLK_OK;
  });
}

trplk_status trplk_fsai_loss_grad(trplk_handle* h, const trplk_csr* A, const int32_t* dims, const float* weights,
                                  int bf16, const double* V, int nv, double gamma, double* loss, double* grad) {
  return guarded(h, [&]() -> trplk_status {
    if (!weights || !V || nv < 1 || !loss || !grad) throw Error(TRPLK_EINVAL, "bad FSAI loss arguments");
    DevCsr<double> a = dev64(A);
    FsaiOp op = build_pattern(h, a.n, a.rowptr, a.col, a.val, "step.fsai");
    check_dims(op, dims);
    float* P = static_cast<float*>(h->get("step.fsai.mlp", kNParams * sizeof(float)));
    double* gr = static_cast<double*>(h->get("step.fsai.grad", kNParams * sizeof(double)));
    upload_weights(h, weights, P);
    LossOut lo = loss_grad(h, op, dims, P, bf16 != 0, V, nv, gamma, gr, "step.fsai.lg");
    TRPLK_CUDA_TRY(cudaMemcpyAsync(grad, gr, kNParams * sizeof(double), cudaMemcpyDeviceToHost, h->ctx.stream));
    h->sync();
    loss[0] = lo.L;
    loss[1] = lo.E;
    loss[2] = lo.K;
    return TRPLK_OK;
  });
}

trplk_status trplk_fsai_train(trplk_handle* h, const trplk_csr* ops, const int32_t* dims, int nops,
                              const trplk_train_params* tp, float* weights, double* losses) {
  return guarded(h, [&]() -> trplk_status {
    if (!ops || !dims || nops < 1 || !tp || !weights) throw Error(TRPLK_EINVAL, "bad training arguments");
    if (tp->iters < 0 || tp->vectors < 1 || tp->harvest_cycles < 1 || !(tp->lr > 0.0))
      throw Error(TRPLK_EINVAL, "bad training parameters");
    const Ctx& c = h->ctx;
    // 1. harvest solver vectors: Jacobi TRPL+K (mixed path) capped at
    //    harvest_cycles cycles; the residuals of its Ritz vectors are the
    //    training vectors
    std::vector<double*> Vs(nops);
    for (int o = 0; o < nops; ++o) {
      const int64_t n = ops[o].n;
      Vs[o] = static_cast<double*>(h->get("train.V" + std::to_string(o), (size_t)n * tp->vectors * sizeof(double)));
      double* ev = static_cast<double*>(h->get("train.ev", 64 * sizeof(double)));
      double* rs = static_cast<double*>(h->get("train.rs", 64 * sizeof(double)));
      trplk_params sp;
      memset(&sp, 0, sizeof(sp));
      sp.p = tp->vectors;
      sp.q = tp->q;
      sp.k = tp->k;
      sp.l = tp->l;
      sp.tol = 1e-12;
      sp.max_cycles = tp->harvest_cycles;
      sp.seed = tp->seed + (uint64_t)o;
      sp.which = TRPLK_SMALLEST;
      sp.precond = TRPLK_PRECOND_JACOBI;
      sp.precision = TRPLK_PRECISION_MIXED;
      sp.outputs_on_device = 1;
      sp.mixed_tol = 1e-12;
      trplk_info inf;
      double* X = static_cast<double*>(h->get("train.X", (size_t)n * tp->vectors * sizeof(double)));
      const trplk_status st = trplk_solve(h, &ops[o], nullptr, &sp, nullptr, ev, X, rs, &inf);
      if (st != TRPLK_OK && st != TRPLK_NOT_CONVERGED) throw Error(st, std::string("harvest solve: ") + h->err);
      h->err.clear();
      // the training vectors are the residuals r_i = A x_i - theta_i x_i: the
      // vectors M is applied to inside TRPL+K
      std::vector<double> th(tp->vectors);
      TRPLK_CUDA_TRY(cudaMemcpyAsync(th.data(), ev, tp->vectors * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
      h->sync();
      DevCsr<double> A{n, ops[o].nnz, ops[o].rowptr, ops[o].col, static_cast<const double*>(ops[o].val)};
      double* ax = static_cast<double*>(h->get("train.ax", n * sizeof(double)));
      for (int j = 0; j < tp->vectors; ++j) {
        spmv<double>(c, A, X + (size_t)j * n, ax);
        axpby_shift<double>(c, n, ax, X + (size_t)j * n, th[j], Vs[o] + (size_t)j * n);
      }
    }
    // 2. Adam over the operators in turn
    float* P = static_cast<float*>(h->get("train.P", kNParams * sizeof(float)));
    float* mom = static_cast<float*>(h->get("train.m", kNParams * sizeof(float), true));
    float* vel = static_cast<float*>(h->get("train.v", kNParams * sizeof(float), true));
    double* gr = static_cast<double*>(h->get("train.grad", kNParams * sizeof(double)));
    upload_weights(h, weights, P);
    std::vector<FsaiOp> pats(nops);
    for (int o = 0; o < nops; ++o) {
      pats[o] = build_pattern(h, ops[o].n, ops[o].rowptr, ops[o].col, static_cast<const double*>(ops[o].val),
                              "train.op" + std::to_string(o));
      check_dims(pats[o], dims + 3 * o);
    }
    for (int it = 0; it < tp->iters; ++it) {
      const int o = it % nops;
      LossOut lo = loss_grad(h, pats[o], dims + 3 * o, P, tp->bf16 != 0, Vs[o], tp->vectors, tp->gamma, gr,
                             "train.lg");
      if (losses) losses[it] = lo.L;
      ProfScope ps(c, PK_OTHER, 0.0);
      adam_kernel<<<(kNParams + 255) / 256, 256, 0, c.stream>>>(kNParams, P, mom, vel, gr, (float)tp->lr, 0.9f,
                                                                 0.999f, 1e-8f, it + 1);
      check_launch("adam");
    }
    TRPLK_CUDA_TRY(cudaMemcpyAsync(weights, P, kNParams * sizeof(float), cudaMemcpyDeviceToHost, c.stream));
    h->sync();
    return TRPLK_OK;
  });
}

}  // extern "C"
