// Sparse matrix-vector products and small elementwise kernels.
//
// SpMV (eq. (UpdateT), z = A g).  Operators whose entries lie on a few
// diagonals (stencils, structured FEM) are converted to DIA at set-up
// (dia_spmv_kernel: no column indices).  Other operators whose rows have
// similar lengths are converted to SELL-32 and multiplied by
// sell_spmv_kernel below.  Operators with very unequal rows (power-law graphs)
// get the hybrid form of the same kernel: rows sorted by length class, short
// rows in SELL-32 slices, long rows one warp each, the longest one CTA each.
// CSR-stream, one thread per row, serves matrices with neither copy.  A CTA owns
// 256 consecutive rows; it streams the values and column indices of those
// rows into shared memory with coalesced loads (the rows are contiguous in
// CSR, so the whole block is one contiguous range), then each thread forms its
// row's dot product from shared memory, gathering x through the read-only
// cache (for the stencil and FEM operators the gathered x lines are reused
// from L1/L2 by the neighbouring rows).  The matvecs are launched in plain
// stream order: launched as programmatic dependents they cost 4-10% of the
// Chung-Lu solve (their many-CTA grids were held back by resident CTAs of the
// neighbouring kernels), while the streaming passes gain from it.  They still
// begin with grid_dependency_wait() (a no-op in plain order), so either launch
// is correct.
// No warp-shuffle reductions: on this
// GPU a shuffle-and-add tree in FP64 costs more FP64 instructions than the
// products themselves.  A block whose rows hold more nonzeros than the
// shared-memory chunk is processed in chunks.
#include <utility>

#include "launch.h"
#include "tallskinny.cuh"

namespace trplk {

namespace {
constexpr int kRows = 256;
template <typename S> struct Chunk;
template <> struct Chunk<double> { static constexpr int CH = 4096; };   // 48 KiB of (val, col)
template <> struct Chunk<float> { static constexpr int CH = 4096; };    // 32 KiB

template <typename S, bool SCALED>
__global__ void __launch_bounds__(kRows) spmv_kernel(int64_t n, const int64_t* __restrict__ rowptr,
                                                     const int32_t* __restrict__ col,
                                                     const S* __restrict__ val, const S* __restrict__ x,
                                                     S* __restrict__ y, const double* __restrict__ scale,
                                                     S* __restrict__ g, const S* __restrict__ bx,
                                                     S* __restrict__ bg) {
  grid_dependency_wait();
  constexpr int CH = Chunk<S>::CH;
  extern __shared__ __align__(16) unsigned char sm[];
  S* s_val = reinterpret_cast<S*>(sm);
  int32_t* s_col = reinterpret_cast<int32_t*>(sm + CH * sizeof(S));
  const int64_t r0 = (int64_t)blockIdx.x * kRows;
  const int64_t r1 = r0 + kRows < n ? r0 + kRows : n;
  const int64_t row = r0 + threadIdx.x;
  const int64_t base = rowptr[r0];
  const int64_t end = rowptr[r1];
  const int64_t my_s = row < n ? rowptr[row] : end;
  const int64_t my_e = row < n ? rowptr[row + 1] : end;
  constexpr int PER = CH / kRows;   // elements each thread stages per chunk
  S sum = 0;
  for (int64_t c0 = base; c0 < end; c0 += CH) {
    const int cnt = (int)(end - c0 < CH ? end - c0 : CH);
    // issue every load of the chunk before the first shared-memory store
    S vv[PER];
    int32_t cc[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = threadIdx.x + u * kRows;
      if (e < cnt) {
        vv[u] = val[c0 + e];
        cc[u] = col[c0 + e];
      }
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = threadIdx.x + u * kRows;
      if (e < cnt) {
        s_val[e] = vv[u];
        s_col[e] = cc[u];
      }
    }
    __syncthreads();
    const int lo = (int)((my_s > c0 ? my_s : c0) - c0);
    const int hi = (int)((my_e < c0 + cnt ? my_e : c0 + cnt) - c0);
    int e = lo;
    for (; e + 4 <= hi; e += 4) {   // four independent gathers in flight
      const S x0 = __ldg(&x[s_col[e]]), x1 = __ldg(&x[s_col[e + 1]]);
      const S x2 = __ldg(&x[s_col[e + 2]]), x3 = __ldg(&x[s_col[e + 3]]);
      sum = fmaS(s_val[e], x0, sum);
      sum = fmaS(s_val[e + 1], x1, sum);
      sum = fmaS(s_val[e + 2], x2, sum);
      sum = fmaS(s_val[e + 3], x3, sum);
    }
    for (; e < hi; ++e) sum = fmaS(s_val[e], __ldg(&x[s_col[e]]), sum);
    __syncthreads();
  }
  if (row < n) {
    if (SCALED) {
      const S s = (S)(*scale);
      y[row] = s * sum;
      g[row] = s * x[row];
      if (bx) bg[row] = s * bx[row];
    } else {
      y[row] = sum;
    }
  }
}

template <typename S, bool SCALED>
__device__ __forceinline__ void spmv_finish(int64_t row, S sum, const S* __restrict__ x, S* __restrict__ y,
                                            const double* __restrict__ scale, S* __restrict__ g,
                                            const S* __restrict__ bx, S* __restrict__ bg) {
  if (SCALED) {
    const S s = (S)(*scale);
    y[row] = s * sum;
    g[row] = s * x[row];
    if (bx) bg[row] = s * bx[row];
  } else {
    y[row] = sum;
  }
}

// One long CSR row: entries e0 + t, e0 + t + step, ... with four independent
// chains (fixed order, so the result is deterministic).
template <typename S>
__device__ __forceinline__ S row_segment(int64_t e, int64_t re, int step, const int32_t* __restrict__ col,
                                         const S* __restrict__ val, const S* __restrict__ x) {
  S s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  for (; e + 3 * (int64_t)step < re; e += 4 * (int64_t)step) {
    const int32_t c0 = __ldg(col + e), c1 = __ldg(col + e + step);
    const int32_t c2 = __ldg(col + e + 2 * step), c3 = __ldg(col + e + 3 * step);
    const S v0 = __ldg(val + e), v1 = __ldg(val + e + step), v2 = __ldg(val + e + 2 * step);
    const S v3 = __ldg(val + e + 3 * step);
    s0 = fmaS(v0, __ldg(x + c0), s0);
    s1 = fmaS(v1, __ldg(x + c1), s1);
    s2 = fmaS(v2, __ldg(x + c2), s2);
    s3 = fmaS(v3, __ldg(x + c3), s3);
  }
  for (; e < re; e += step) s0 = fmaS(__ldg(val + e), __ldg(x + __ldg(col + e)), s0);
  return (s0 + s1) + (s2 + s3);
}

template <typename S>
__device__ __forceinline__ S warp_sum(S v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// SELL-32 matvec: one warp per 32-row slice, one lane per row.  The slice's
// entries are stored column-major, so every load of values and column indices
// is one coalesced 128/256-byte transaction and independent of the others;
// no row-pointer chase and no shared-memory staging.
// HYB: the grid starts with n_cta blocks that each own one of the longest
// rows (256 threads stride the row, block reduction in a fixed order), then
// blocks of 8 warps that each own one long row (lanes stride the row, xor
// butterfly), then the SELL slices of the remaining rows, whose positions map
// to rows through perm.  Heavy rows come first so they start first.
template <typename S, bool SCALED, bool HYB>
__global__ void __launch_bounds__(256) sell_spmv_kernel(
    int64_t m, int64_t nslices, const int64_t* __restrict__ sl_ptr, const int32_t* __restrict__ sl_col,
    const S* __restrict__ sl_val, const int32_t* __restrict__ perm, const int32_t* __restrict__ long_rows,
    int64_t n_cta, int64_t n_warp, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const S* __restrict__ val, const S* __restrict__ x, S* __restrict__ y, const double* __restrict__ scale,
    S* __restrict__ g, const S* __restrict__ bx, S* __restrict__ bg) {
  grid_dependency_wait();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t b = blockIdx.x;
  if (HYB) {
    if (b < n_cta) {   // one CTA per row
      __shared__ S red[8];
      const int64_t row = long_rows[b];
      const S v = warp_sum(row_segment<S>(rowptr[row] + threadIdx.x, rowptr[row + 1], 256, col, val, x));
      if (lane == 0) red[warp] = v;
      __syncthreads();
      if (threadIdx.x == 0) {
        S t = red[0];
#pragma unroll
        for (int w = 1; w < 8; ++w) t += red[w];
        spmv_finish<S, SCALED>(row, t, x, y, scale, g, bx, bg);
      }
      return;
    }
    b -= n_cta;
    const int64_t wblocks = (n_warp + 7) / 8;
    if (b < wblocks) {   // one warp per row
      const int64_t w = b * 8 + warp;
      if (w >= n_warp) return;
      const int64_t row = long_rows[n_cta + w];
      const S v = warp_sum(row_segment<S>(rowptr[row] + lane, rowptr[row + 1], 32, col, val, x));
      if (lane == 0) spmv_finish<S, SCALED>(row, v, x, y, scale, g, bx, bg);
      return;
    }
    b -= wblocks;
  }
  const int64_t slice = b * 8 + warp;
  if (slice >= nslices) return;
  const int64_t base = sl_ptr[slice];
  const int len = (int)((sl_ptr[slice + 1] - base) >> 5);
  const S* vp = sl_val + base + lane;
  const int32_t* cp = sl_col + base + lane;
  S sum = 0;
  int j = 0;
  for (; j + 4 <= len; j += 4) {
    const int32_t c0 = __ldg(cp + 32 * j), c1 = __ldg(cp + 32 * (j + 1));
    const int32_t c2 = __ldg(cp + 32 * (j + 2)), c3 = __ldg(cp + 32 * (j + 3));
    const S v0 = __ldg(vp + 32 * j), v1 = __ldg(vp + 32 * (j + 1));
    const S v2 = __ldg(vp + 32 * (j + 2)), v3 = __ldg(vp + 32 * (j + 3));
    const S x0 = __ldg(x + c0), x1 = __ldg(x + c1), x2 = __ldg(x + c2), x3 = __ldg(x + c3);
    sum = fmaS(v0, x0, sum);
    sum = fmaS(v1, x1, sum);
    sum = fmaS(v2, x2, sum);
    sum = fmaS(v3, x3, sum);
  }
  if (j < len) {   // remainder of 1..3 entries, loads issued together
    const int r = len - j;
    const int32_t c0 = __ldg(cp + 32 * j);
    const int32_t c1 = r > 1 ? __ldg(cp + 32 * (j + 1)) : c0;
    const int32_t c2 = r > 2 ? __ldg(cp + 32 * (j + 2)) : c0;
    const S v0 = __ldg(vp + 32 * j);
    const S v1 = r > 1 ? __ldg(vp + 32 * (j + 1)) : (S)0;
    const S v2 = r > 2 ? __ldg(vp + 32 * (j + 2)) : (S)0;
    const S x0 = __ldg(x + c0), x1 = __ldg(x + c1), x2 = __ldg(x + c2);
    sum = fmaS(v0, x0, sum);
    if (r > 1) sum = fmaS(v1, x1, sum);
    if (r > 2) sum = fmaS(v2, x2, sum);
  }
  const int64_t pos = slice * 32 + lane;
  if (pos < m) spmv_finish<S, SCALED>(HYB ? (int64_t)perm[pos] : pos, sum, x, y, scale, g, bx, bg);
}

struct DiaOff {
  int off[kMaxDiag];
};

// DIA matvec: thread per row, one coalesced load of each diagonal's value and
// of the shifted x window (x stays in L2); no index traffic.
template <typename S, bool SCALED>
__global__ void __launch_bounds__(256) dia_spmv_kernel(int64_t n, int64_t ld, int ndiag, const DiaOff off,
                                                       const S* __restrict__ dval, const S* __restrict__ x,
                                                       S* __restrict__ y, const double* __restrict__ scale,
                                                       S* __restrict__ g, const S* __restrict__ bx,
                                                       S* __restrict__ bg) {
  grid_dependency_wait();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  S s0 = 0, s1 = 0;
  int d = 0;
  for (; d + 1 < ndiag; d += 2) {
    const int64_t j0 = i + off.off[d], j1 = i + off.off[d + 1];
    const S a0 = __ldg(dval + (int64_t)d * ld + i), a1 = __ldg(dval + (int64_t)(d + 1) * ld + i);
    if ((uint64_t)j0 < (uint64_t)n) s0 = fmaS(a0, __ldg(x + j0), s0);
    if ((uint64_t)j1 < (uint64_t)n) s1 = fmaS(a1, __ldg(x + j1), s1);
  }
  if (d < ndiag) {
    const int64_t j0 = i + off.off[d];
    if ((uint64_t)j0 < (uint64_t)n) s0 = fmaS(__ldg(dval + (int64_t)d * ld + i), __ldg(x + j0), s0);
  }
  spmv_finish<S, SCALED>(i, s0 + s1, x, y, scale, g, bx, bg);
}

template <typename S>
void spmv_launch(const Ctx& c, const DevCsr<S>& A, const S* x, S* y, const double* scale, S* g,
                 const S* bx, S* bg, bool scaled) {
  if (A.n == 0) return;
  if (A.dia_val) {
    DiaOff off;
    for (int d = 0; d < kMaxDiag; ++d) off.off[d] = d < A.ndiag ? A.dia_off[d] : 0;
    // algorithmic bytes: the diagonals' values, x once, y (and the scaled copies) once
    double bytes = (double)A.ndiag * A.n * sizeof(S) + 2.0 * A.n * sizeof(S);
    if (scaled) bytes += (double)A.n * sizeof(S) * (bx ? 3 : 1);
    ProfScope ps(c, prof_kind<S>(scaled ? PK_SPMV_SCALED : PK_SPMV), bytes);
    const unsigned gb = (unsigned)((A.n + 255) / 256);
    if (scaled)
      launch_plain(dia_spmv_kernel<S, true>, dim3(gb), dim3(256), 0, c.stream, A.n, A.dia_ld, A.ndiag, off,
                       A.dia_val, x, y, scale, g, bx, bg);
    else
      launch_plain(dia_spmv_kernel<S, false>, dim3(gb), dim3(256), 0, c.stream, A.n, A.dia_ld, A.ndiag, off,
                       A.dia_val, x, y, (const double*)nullptr, (S*)nullptr, (const S*)nullptr, (S*)nullptr);
    check_launch("dia_spmv_kernel");
    return;
  }
  if (A.sl_ptr) {
    const bool hyb = A.sl_perm || A.long_rows;
    const int64_t m = hyb ? A.sl_rows : A.n;
    const int64_t nslices = (m + 31) / 32;
    const int64_t nlong = A.n_long_cta + A.n_long_warp;
    const int64_t blocks = (hyb ? A.n_long_cta + (A.n_long_warp + 7) / 8 : 0) + (nslices + 7) / 8;
    if (blocks > 0x7fffffff) throw Error(TRPLK_EINVAL, "matrix too large");
    // algorithmic bytes: values + column indices once, slice offsets, row
    // map and long-row pointers, x once, y (and the scaled copies) once
    double bytes = (double)A.nnz * (sizeof(S) + 4) + (double)(nslices + 1) * 8 + 2.0 * A.n * sizeof(S);
    if (hyb) bytes += (double)m * 4 + (double)nlong * 20;
    if (scaled) bytes += (double)A.n * sizeof(S) * (bx ? 3 : 1);
    ProfScope ps(c, prof_kind<S>(scaled ? PK_SPMV_SCALED : PK_SPMV), bytes);
    const unsigned gb = (unsigned)(blocks > 0 ? blocks : 1);
#define TRPLK_SELL(SC, HY)                                                                                  \
  launch_plain(sell_spmv_kernel<S, SC, HY>, dim3(gb), dim3(256), 0, c.stream, m, nslices, A.sl_ptr,      \
                   A.sl_col, A.sl_val, A.sl_perm, A.long_rows, A.n_long_cta, A.n_long_warp, A.rowptr, A.col,  \
                   A.val, x, y, scale, g, bx, bg)
    if (scaled) {
      if (hyb) TRPLK_SELL(true, true); else TRPLK_SELL(true, false);
    } else {
      if (hyb) TRPLK_SELL(false, true); else TRPLK_SELL(false, false);
    }
#undef TRPLK_SELL
    check_launch("sell_spmv_kernel");
    return;
  }
  constexpr int CH = Chunk<S>::CH;
  const size_t smem = CH * (sizeof(S) + sizeof(int32_t));
  const int64_t blocks = (A.n + kRows - 1) / kRows;
  if (blocks > 0x7fffffff) throw Error(TRPLK_EINVAL, "matrix too large");
  // algorithmic bytes: values + column indices + row pointers, x once, y (and
  // the scaled copies) written once
  double bytes = (double)A.nnz * (sizeof(S) + 4) + (double)(A.n + 1) * 8 + 2.0 * A.n * sizeof(S);
  if (scaled) bytes += (double)A.n * sizeof(S) * (bx ? 3 : 1);
  ProfScope ps(c, prof_kind<S>(scaled ? PK_SPMV_SCALED : PK_SPMV), bytes);
  if (scaled) {
    smem_optin<spmv_kernel<S, true>>((int)smem, c.device);
    launch_plain(spmv_kernel<S, true>, dim3((unsigned)blocks), dim3(kRows), smem, c.stream, A.n, A.rowptr, A.col,
                     A.val, x, y, scale, g, bx, bg);
  } else {
    smem_optin<spmv_kernel<S, false>>((int)smem, c.device);
    launch_plain(spmv_kernel<S, false>, dim3((unsigned)blocks), dim3(kRows), smem, c.stream, A.n, A.rowptr,
                     A.col, A.val, x, y, (const double*)nullptr, (S*)nullptr, (const S*)nullptr, (S*)nullptr);
  }
  check_launch("spmv_kernel");
}

// ---- elementwise kernels
template <typename S>
__global__ void restart_vector_kernel(int64_t ld, const S* __restrict__ ax, const S* __restrict__ bx,
                                      const double* __restrict__ theta_t, const S* __restrict__ dinv,
                                      int pmode, S* __restrict__ v) {
  const S th = (S)(*theta_t);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ld; i += (int64_t)gridDim.x * blockDim.x) {
    S r = ax[i] - th * bx[i];
    if (pmode == PM_JACOBI) r *= dinv[i];
    v[i] = r;
  }
}

template <typename D, typename S>
__global__ void convert_kernel(int64_t count, const S* __restrict__ src, D* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (D)src[i];
}

template <typename S>
__global__ void axpby_shift_kernel(int64_t ld, const S* __restrict__ x, const S* __restrict__ y, double rho,
                                   S* __restrict__ r) {
  const S rr = (S)rho;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ld; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = x[i] - rr * y[i];
}

// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): one generator step on the state seed ^ counter.
__device__ __forceinline__ uint64_t splitmix64(uint64_t s) {
  uint64_t z = s + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void start_block_kernel(int64_t n, int64_t ld, int k, uint64_t seed, double* __restrict__ X) {
  const int64_t total = ld * (int64_t)k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / ld, i = e - c * ld;
    double v = 0.0;
    if (i < n) {
      const uint64_t z = splitmix64(seed ^ (uint64_t)(c * n + i));
      v = 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
    }
    X[e] = v;
  }
}

// The diagonal entry of row i (the last one if the row stores it twice; 0 if
// none), read by the 32 lanes of a warp striding the row; every lane returns it.
template <typename S>
__device__ __forceinline__ S row_diag_warp(int64_t i, const int64_t* __restrict__ rowptr,
                                           const int32_t* __restrict__ col, const S* __restrict__ val, int lane) {
  const int64_t a = rowptr[i], b = rowptr[i + 1];
  int64_t at = -1;
  S d = 0;
  for (int64_t e = a + lane; e < b; e += 32)
    if (col[e] == i) {
      at = e;
      d = val[e];
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int64_t at2 = __shfl_xor_sync(0xffffffffu, at, o);
    const S d2 = __shfl_xor_sync(0xffffffffu, d, o);
    if (at2 > at) {
      at = at2;
      d = d2;
    }
  }
  return d;
}

template <typename S>
__global__ void jacobi_dinv_kernel(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                   const S* __restrict__ val, S* __restrict__ dinv, int* status) {
  // one warp per row (coalesced reads; a power-law row does not hold up a thread)
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    const S d = row_diag_warp<S>(i, rowptr, col, val, lane);
    if (lane == 0) {
      if (!(d != 0)) atomicOr(status, kFlagNaN);
      dinv[i] = d != 0 ? (S)1 / d : (S)0;
    }
  }
}

// out = d .* x
template <typename S>
__global__ void scale_kernel(int64_t ld, const S* __restrict__ d, const S* __restrict__ x, S* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ld; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = d[i] * x[i];
}

// one Jacobi sweep's update: out = x + d .* (b - t), t = L x
template <typename S>
__global__ void sweep_update_kernel(int64_t ld, const S* __restrict__ x, const S* __restrict__ d,
                                    const S* __restrict__ b, const S* __restrict__ t, S* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ld; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = x[i] + d[i] * (b[i] - t[i]);
}

// diag[i] = a_ii (0 where the row has no diagonal entry)
__global__ void diag_of_kernel(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const double* __restrict__ val, double* __restrict__ diag) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    const double d = row_diag_warp<double>(i, rowptr, col, val, lane);
    if (lane == 0) diag[i] = d;
  }
}

// The per-cycle shifted Jacobi preconditioner (Sec. 3: M may change every
// cycle to approximate (A - rho_i B)^-1): dinv_j = 1 / max(a_jj - rho b_jj,
// 1e-3 a_jj), b_jj = 1 without B; formed in FP64, stored in S; rows >= n 0.
template <typename S>
__global__ void shifted_jacobi_kernel(int64_t n, int64_t ld, const double* __restrict__ dA,
                                      const double* __restrict__ dB, const double* __restrict__ rho_p,
                                      S* __restrict__ dinv) {
  const double rho = *rho_p;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ld; i += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (i < n) {
      const double a = dA[i];
      const double d = fmax(a - rho * (dB ? dB[i] : 1.0), 1e-3 * a);
      v = 1.0 / d;
    }
    dinv[i] = (S)v;
  }
}

__global__ void sell_lengths_kernel(int64_t m, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ perm,
                                    int32_t* __restrict__ lens) {
  const int64_t slice = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t pos = slice * 32 + lane;
  int len = 0;
  if (pos < m) {
    const int64_t row = perm ? (int64_t)perm[pos] : pos;
    len = (int)(rowptr[row + 1] - rowptr[row]);
  }
  for (int off = 16; off > 0; off >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, off));
  if (lane == 0 && slice * 32 < m) lens[slice] = len;
}

template <typename S>
__global__ void sell_fill_kernel(int64_t m, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                 const double* __restrict__ val, const int32_t* __restrict__ perm,
                                 const int64_t* __restrict__ sl_ptr, int32_t* __restrict__ sl_col,
                                 S* __restrict__ sl_val) {
  const int64_t slice = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (slice * 32 >= m) return;
  const int64_t pos = slice * 32 + lane;
  const int64_t row = pos < m ? (perm ? (int64_t)perm[pos] : pos) : -1;
  const int64_t base = sl_ptr[slice];
  const int len = (int)((sl_ptr[slice + 1] - base) >> 5);
  const int64_t rs = row >= 0 ? rowptr[row] : 0;
  const int rl = row >= 0 ? (int)(rowptr[row + 1] - rs) : 0;
  const int32_t pad_col = (int32_t)(row >= 0 ? row : 0);
  for (int j = 0; j < len; ++j) {
    const int64_t o = base + 32 * (int64_t)j + lane;
    if (j < rl) {
      if (sl_col) sl_col[o] = col[rs + j];
      sl_val[o] = (S)val[rs + j];
    } else {
      if (sl_col) sl_col[o] = pad_col;
      sl_val[o] = (S)0;
    }
  }
}

// kDiaSamples rows along a Weyl sequence (fractional parts of k times the
// golden ratio, so no sample lines up with the grid boundaries of a
// power-of-two stencil); their first kMaxDiag column offsets
__global__ void dia_sample_kernel(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                  int32_t* __restrict__ out) {
  const int k = threadIdx.x;
  if (k >= kDiaSamples) return;
  const uint64_t frac = (uint64_t)(uint32_t)((uint64_t)(k + 1) * 2654435769ull);   // 2^32 frac(k phi)
  const int64_t i = (int64_t)((frac * (uint64_t)n) >> 32);
  int32_t* o = out + k * (kMaxDiag + 1);
  const int64_t rs = rowptr[i], re = rowptr[i + 1];
  const int cnt = (int)(re - rs < kMaxDiag ? re - rs : kMaxDiag);
  o[0] = re - rs > kMaxDiag ? -1 : cnt;   // -1: too many entries for DIA
  for (int e = 0; e < cnt; ++e) o[1 + e] = (int32_t)((int64_t)col[rs + e] - i);
}

struct DiaOffSorted {
  int off[kMaxDiag];
};

template <typename S>
__global__ void dia_fill_kernel(int64_t n, int64_t ld, const int64_t* __restrict__ rowptr,
                                const int32_t* __restrict__ col, const double* __restrict__ val, int ndiag,
                                const DiaOffSorted off, S* __restrict__ dval, int* __restrict__ missing) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int64_t o = (int64_t)col[e] - i;
      int lo = 0, hi = ndiag - 1, d = -1;
      while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        if (off.off[mid] == o) { d = mid; break; }
        if (off.off[mid] < o) lo = mid + 1; else hi = mid - 1;
      }
      if (d < 0) { atomicOr(missing, 1); continue; }
      dval[(int64_t)d * ld + i] = (S)val[e];
    }
  }
}

// length class of a row: the longest first.  [0, 22): more than kWarpRow
// entries, by descending floor(log2 len); [22, 28): kShortRow+1 .. kWarpRow,
// likewise; [28, 61): 0 .. kShortRow entries, by descending length.
__device__ __forceinline__ int hyb_bucket(int64_t len) {
  const int lg = 63 - __clzll((unsigned long long)(len > 0 ? len : 1));
  if (len > kWarpRow) return lg >= 31 ? 0 : 31 - lg;
  if (len > kShortRow) return 22 + (10 - lg);
  return 28 + (kShortRow - (int)len);
}

// one warp per chunk of kHybChunk rows: class counts of the chunk
__global__ void __launch_bounds__(256) hyb_hist_kernel(int64_t n, const int64_t* __restrict__ rowptr,
                                                       int32_t* __restrict__ hist) {
  __shared__ int cnt[8][64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t chunk = (int64_t)blockIdx.x * 8 + warp;
  for (int b = lane; b < 64; b += 32) cnt[warp][b] = 0;
  __syncwarp();
  const int64_t r0 = chunk * kHybChunk;
  for (int i = lane; i < kHybChunk; i += 32) {
    const int64_t row = r0 + i;
    if (row < n) atomicAdd(&cnt[warp][hyb_bucket(rowptr[row + 1] - rowptr[row])], 1);
  }
  __syncwarp();
  if (r0 < n)
    for (int b = lane; b < kHybBuckets; b += 32) hist[chunk * kHybBuckets + b] = cnt[warp][b];
}

// stable scatter: rows of a chunk are visited in order 32 at a time; lanes of
// one class find their rank among themselves with a match + popcount
__global__ void __launch_bounds__(256) hyb_scatter_kernel(int64_t n, const int64_t* __restrict__ rowptr,
                                                          const int32_t* __restrict__ offs,
                                                          int32_t* __restrict__ order) {
  __shared__ int off[8][64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t chunk = (int64_t)blockIdx.x * 8 + warp;
  const int64_t r0 = chunk * kHybChunk;
  if (r0 >= n) return;   // warp-uniform
  for (int b = lane; b < kHybBuckets; b += 32) off[warp][b] = offs[chunk * kHybBuckets + b];
  __syncwarp();
  for (int i = 0; i < kHybChunk; i += 32) {
    const int64_t row = r0 + i + lane;
    const int b = row < n ? hyb_bucket(rowptr[row + 1] - rowptr[row]) : 63;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (row < n) order[off[warp][b] + rank] = (int32_t)row;
    __syncwarp();
    if (row < n && rank == 0) off[warp][b] += __popc(peers);
    __syncwarp();
  }
}

inline unsigned grid_for(const Ctx& c, int64_t count) {
  int64_t g = (count + 255) / 256;
  int64_t cap = (int64_t)c.sms * 8;
  return (unsigned)(g < cap ? (g > 0 ? g : 1) : cap);
}

}  // namespace

template <typename S>
void spmv(const Ctx& c, const DevCsr<S>& A, const S* x, S* y) {
  spmv_launch<S>(c, A, x, y, nullptr, nullptr, nullptr, nullptr, false);
}

template <typename S>
void spmv_scaled(const Ctx& c, const DevCsr<S>& A, const S* x, const double* scale, S* y, S* g,
                 const S* bx, S* bg) {
  spmv_launch<S>(c, A, x, y, scale, g, bx, bg, true);
}

template <typename S>
void restart_vector(const Ctx& c, int64_t ld, const S* ax, const S* bx, const double* theta_t,
                    const S* dinv, int pmode, S* v) {
  ProfScope ps(c, PK_OTHER, 0.0);
  restart_vector_kernel<S><<<grid_for(c, ld), 256, 0, c.stream>>>(ld, ax, bx, theta_t, dinv, pmode, v);
  check_launch("restart_vector");
}

template <typename D, typename S>
void convert(const Ctx& c, int64_t count, const S* src, D* dst) {
  if (count == 0) return;
  ProfScope ps(c, PK_OTHER, 0.0);
  convert_kernel<D, S><<<grid_for(c, count), 256, 0, c.stream>>>(count, src, dst);
  check_launch("convert");
}

void start_block(const Ctx& c, int64_t n, int64_t ld, int k, uint64_t seed, double* X) {
  ProfScope ps(c, PK_OTHER, 0.0);
  start_block_kernel<<<grid_for(c, ld * k), 256, 0, c.stream>>>(n, ld, k, seed, X);
  check_launch("start_block");
}

template <typename S>
void jacobi_dinv(const Ctx& c, const DevCsr<S>& A, S* dinv) {
  ProfScope ps(c, PK_OTHER, 0.0);
  jacobi_dinv_kernel<S><<<grid_for(c, A.n * 32), 256, 0, c.stream>>>(A.n, A.rowptr, A.col, A.val, dinv, c.status);
  check_launch("jacobi_dinv");
}

template <typename S>
void axpby_shift(const Ctx& c, int64_t ld, const S* x, const S* y, double rho, S* r) {
  ProfScope ps(c, PK_OTHER, 0.0);
  axpby_shift_kernel<S><<<grid_for(c, ld), 256, 0, c.stream>>>(ld, x, y, rho, r);
  check_launch("axpby_shift");
}

// IC(0) preconditioner M b = P_s^T (P_s b): P_s b by `sweeps` Jacobi sweeps
// x <- x + D^-1 (b - L x) from x = D^-1 b (L with its diagonal D: the same
// iterate as x <- D^-1 (b - L_strict x)), then the same on L^T.
template <typename S>
void ic0_apply(const Ctx& c, int64_t ld, const DevCsr<S>& L, const DevCsr<S>& LT, const S* dinv, int sweeps,
               const S* in, S* out, S* t0, S* t1, S* t2) {
  auto scale = [&](const S* x, S* o) {
    ProfScope ps(c, PK_OTHER, 0.0);
    scale_kernel<S><<<grid_for(c, ld), 256, 0, c.stream>>>(ld, dinv, x, o);
    check_launch("scale");
  };
  auto update = [&](const S* x, const S* b, const S* t, S* o) {
    ProfScope ps(c, PK_OTHER, 0.0);
    sweep_update_kernel<S><<<grid_for(c, ld), 256, 0, c.stream>>>(ld, x, dinv, b, t, o);
    check_launch("sweep_update");
  };
  // forward: the result ends in f (t0 or t2)
  S* f = t0;
  S* g = t2;
  scale(in, f);
  for (int s = 0; s < sweeps; ++s) {
    spmv<S>(c, L, f, t1);
    update(f, in, t1, g);
    std::swap(f, g);
  }
  // backward on L^T with right-hand side f; iterates alternate between out
  // and g, starting where the last one lands in out
  S* y = (sweeps % 2 == 0) ? out : g;
  S* z = (sweeps % 2 == 0) ? g : out;
  scale(f, y);
  for (int s = 0; s < sweeps; ++s) {
    spmv<S>(c, LT, y, t1);
    update(y, f, t1, z);
    std::swap(y, z);
  }
}
template void ic0_apply<double>(const Ctx&, int64_t, const DevCsr<double>&, const DevCsr<double>&, const double*,
                                int, const double*, double*, double*, double*, double*);
template void ic0_apply<float>(const Ctx&, int64_t, const DevCsr<float>&, const DevCsr<float>&, const float*, int,
                               const float*, float*, float*, float*, float*);

void diag_of(const Ctx& c, int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, double* diag) {
  ProfScope ps(c, PK_OTHER, 0.0);
  diag_of_kernel<<<grid_for(c, n * 32), 256, 0, c.stream>>>(n, rowptr, col, val, diag);
  check_launch("diag_of");
}

template <typename S>
void shifted_jacobi(const Ctx& c, int64_t n, int64_t ld, const double* dA, const double* dB, const double* rho,
                    S* dinv) {
  ProfScope ps(c, PK_OTHER, 0.0);
  shifted_jacobi_kernel<S><<<grid_for(c, ld), 256, 0, c.stream>>>(n, ld, dA, dB, rho, dinv);
  check_launch("shifted_jacobi");
}
template void shifted_jacobi<double>(const Ctx&, int64_t, int64_t, const double*, const double*, const double*,
                                     double*);
template void shifted_jacobi<float>(const Ctx&, int64_t, int64_t, const double*, const double*, const double*,
                                    float*);

void sell_lengths(const Ctx& c, int64_t m, const int64_t* rowptr, const int32_t* perm, int32_t* lens) {
  const int64_t nslices = (m + 31) / 32;
  if (nslices == 0) return;
  ProfScope ps(c, PK_OTHER, 0.0);
  sell_lengths_kernel<<<(unsigned)((nslices * 32 + 255) / 256), 256, 0, c.stream>>>(m, rowptr, perm, lens);
  check_launch("sell_lengths");
}

template <typename S>
void sell_fill(const Ctx& c, int64_t m, const int64_t* rowptr, const int32_t* col, const double* val,
               const int32_t* perm, const int64_t* sl_ptr, int32_t* sl_col, S* sl_val) {
  const int64_t nslices = (m + 31) / 32;
  if (nslices == 0) return;
  ProfScope ps(c, PK_OTHER, 0.0);
  sell_fill_kernel<S><<<(unsigned)((nslices * 32 + 255) / 256), 256, 0, c.stream>>>(m, rowptr, col, val, perm,
                                                                                    sl_ptr, sl_col, sl_val);
  check_launch("sell_fill");
}

void dia_sample(const Ctx& c, int64_t n, const int64_t* rowptr, const int32_t* col, int32_t* out) {
  ProfScope ps(c, PK_OTHER, 0.0);
  dia_sample_kernel<<<1, kDiaSamples, 0, c.stream>>>(n, rowptr, col, out);
  check_launch("dia_sample");
}

template <typename S>
void dia_fill(const Ctx& c, int64_t n, int64_t ld, const int64_t* rowptr, const int32_t* col, const double* val,
              int ndiag, const int* off, S* dia_val, int* missing) {
  DiaOffSorted o;
  for (int d = 0; d < kMaxDiag; ++d) o.off[d] = d < ndiag ? off[d] : 0;
  ProfScope ps(c, PK_OTHER, 0.0);
  dia_fill_kernel<S><<<grid_for(c, n), 256, 0, c.stream>>>(n, ld, rowptr, col, val, ndiag, o, dia_val, missing);
  check_launch("dia_fill");
}
template void dia_fill<double>(const Ctx&, int64_t, int64_t, const int64_t*, const int32_t*, const double*, int,
                               const int*, double*, int*);
template void dia_fill<float>(const Ctx&, int64_t, int64_t, const int64_t*, const int32_t*, const double*, int,
                              const int*, float*, int*);

void hyb_hist(const Ctx& c, int64_t n, const int64_t* rowptr, int32_t* hist) {
  const int64_t chunks = (n + kHybChunk - 1) / kHybChunk;
  ProfScope ps(c, PK_OTHER, 0.0);
  hyb_hist_kernel<<<(unsigned)((chunks + 7) / 8), 256, 0, c.stream>>>(n, rowptr, hist);
  check_launch("hyb_hist");
}

void hyb_scatter(const Ctx& c, int64_t n, const int64_t* rowptr, const int32_t* offs, int32_t* order) {
  const int64_t chunks = (n + kHybChunk - 1) / kHybChunk;
  ProfScope ps(c, PK_OTHER, 0.0);
  hyb_scatter_kernel<<<(unsigned)((chunks + 7) / 8), 256, 0, c.stream>>>(n, rowptr, offs, order);
  check_launch("hyb_scatter");
}

template void sell_fill<double>(const Ctx&, int64_t, const int64_t*, const int32_t*, const double*, const int32_t*,
                                const int64_t*, int32_t*, double*);
template void sell_fill<float>(const Ctx&, int64_t, const int64_t*, const int32_t*, const double*, const int32_t*,
                               const int64_t*, int32_t*, float*);
template void spmv<double>(const Ctx&, const DevCsr<double>&, const double*, double*);
template void spmv<float>(const Ctx&, const DevCsr<float>&, const float*, float*);
template void spmv_scaled<double>(const Ctx&, const DevCsr<double>&, const double*, const double*, double*,
                                  double*, const double*, double*);
template void spmv_scaled<float>(const Ctx&, const DevCsr<float>&, const float*, const double*, float*, float*,
                                 const float*, float*);
template void restart_vector<double>(const Ctx&, int64_t, const double*, const double*, const double*,
                                     const double*, int, double*);
template void restart_vector<float>(const Ctx&, int64_t, const float*, const float*, const double*, const float*,
                                    int, float*);
template void convert<float, double>(const Ctx&, int64_t, const double*, float*);
template void convert<double, float>(const Ctx&, int64_t, const float*, double*);
template void convert<double, double>(const Ctx&, int64_t, const double*, double*);
template void jacobi_dinv<double>(const Ctx&, const DevCsr<double>&, double*);
template void jacobi_dinv<float>(const Ctx&, const DevCsr<float>&, float*);
template void axpby_shift<double>(const Ctx&, int64_t, const double*, const double*, double, double*);
template void axpby_shift<float>(const Ctx&, int64_t, const float*, const float*, double, float*);

}  // namespace trplk
