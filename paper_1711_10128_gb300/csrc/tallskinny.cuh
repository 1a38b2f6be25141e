// Tall-skinny streaming kernels over the basis U (n x w, column-major).
//
// Every pass of the inner step, the +K block and the restart streams U (and
// A U or B U) from HBM once.  The kernels share one engine:
//  * persistent CTAs, grid = SMs x CTAs-per-SM (never more than the tiles);
//  * a CTA has TR threads and walks TR-row tiles with stride gridDim.x;
//  * one warp stages each tile into shared memory with 1D bulk copies (the
//    TMA engine, cp.async.bulk): one 1 KiB copy per column segment and per
//    vector segment, completion counted on an mbarrier; up to 4 stages are in
//    flight so HBM latency is hidden behind the compute of earlier tiles;
//  * compute reads shared memory only: thread-per-row for the updates
//    v <- v - U h, column-per-warp for the projections U^T v;
//  * projections accumulate in FP64 (double data) or Dot2-compensated FP32
//    (float data), are reduced per CTA and then summed in CTA order by the
//    last CTA to finish (deterministic, no floating-point atomics).
// Rows n..ld-1 of every array are zero, so whole tiles are always copied.
#pragma once
#include "common.cuh"

namespace trplk {

enum TSKind : int {
  TS_PROJ = 0,     // out0 = mat0^T vec0                                   (1 RHS)
  TS_INNER = 1,    // v = M(z - rho bg); out0 = mat0^T z; out1 = mat1^T v  (2 RHS)
  TS_UPDPROJ = 2,  // v' = v - mat0 h; out0 = mat1^T v'
  TS_UPDNORM = 3,  // v' = v - mat0 h; out0 = ||v'||^2 -> beta, 1/beta, breakdown test
  TS_UPD = 4,      // v' = v - mat0 h
  TS_ROT = 5,      // xout = mat0 Y                                        (k outputs)
  TS_RESID = 6,    // rnorm_j = ||mat1_j - theta_j mat2_j||, xnorm_j = ||mat0_j||
  TS_DOT = 7,      // out0 = vec0^T vec1 -> beta, 1/beta, breakdown test
};

// Inner-step preconditioner modes of TS_INNER.
enum : int { PM_IDENTITY = 0, PM_JACOBI = 1, PM_GIVEN = 2 };

__device__ __forceinline__ double fmaS(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ float fmaS(float a, float b, float c) { return fmaf(a, b, c); }

template <typename S>
struct TSArgs {
  const S* mat[3];     // staged matrices, w columns each (ld)
  int nmat;            // number of distinct staged matrices
  int matsel[3];       // which staged matrix plays operand 0/1/2 of the kind
  const S* vec[3];     // staged vectors
  int nvec;
  int w;               // columns of each staged matrix
  int64_t ld;
  int ntiles;
  int stages;
  int kind;
  int pmode;           // TS_INNER preconditioner mode
  double rho;
  const double* hcoef;   // [w] update coefficients (device)
  const double* haux;    // [w] first-pass coefficients for the beta0 of UPDNORM
  const double* Y;       // rotation coefficients (device, w x k, ldY)
  int ldY, k;
  const double* theta;   // [k] for TS_RESID
  S* vout;               // updated / preconditioned vector (ld)
  S* xout;               // rotation output (ld)
  double* partials;      // per-CTA partial sums [gridDim.x][pstride]
  int pstride;
  unsigned int* counter; // zero on entry, reset by the last CTA
  double* out0;          // final reductions
  double* out1;
  double* scale_out;     // 1/beta for UPDNORM / DOT
  double eps_breakdown;
  int* status;           // device status word (flags)
};

template <typename S>
__device__ __forceinline__ void ts_issue_tile(const TSArgs<S>& a, unsigned char* stage, uint64_t* bar,
                                              int tile) {
  constexpr int TR = Tile<S>::TR;
  constexpr uint32_t colbytes = TR * sizeof(S);
  const int lane = threadIdx.x & 31;
  const int nmc = a.nmat * a.w;
  const int ncopies = nmc + a.nvec;
  if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)ncopies * colbytes);
  __syncwarp();
  const int64_t row0 = (int64_t)tile * TR;
  for (int c = lane; c < ncopies; c += 32) {
    const S* src;
    if (c < nmc) {
      const int m = c / a.w, col = c - m * a.w;
      src = a.mat[m] + (int64_t)col * a.ld + row0;
    } else {
      src = a.vec[c - nmc] + row0;
    }
    bulk_g2s(stage + (size_t)c * colbytes, src, colbytes, bar);
  }
}

// Shared memory layout (bytes): [bars 64][hcoef 512][Y w*k doubles][vtile TR*S][red 2*TR*8][stages]
template <typename S>
inline size_t ts_smem_fixed(int w, int k) {
  constexpr int TR = Tile<S>::TR;
  size_t ybytes = round_up((size_t)kMaxQ * (size_t)(k > 0 ? k : 1) * sizeof(double), 128);
  (void)w;
  return 64 + 512 + ybytes + TR * sizeof(S) + 2 * TR * sizeof(double) + 128;
}

template <typename S, int KIND>
__global__ void __launch_bounds__(Tile<S>::TR) ts_kernel(TSArgs<S> a) {
  constexpr int TR = Tile<S>::TR;
  constexpr int NW = TR / 32;            // warps per CTA
  constexpr int RPL = TR / 32;           // rows per lane in column-parallel phases
  constexpr int MAXJ = kMaxQ / NW;       // columns per warp (upper bound)
  constexpr int KMAX = kMaxK;
  constexpr uint32_t colbytes = TR * sizeof(S);

  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  S* s_h = reinterpret_cast<S*>(smem + 64);          // update coefficients, as S
  S* s_y = reinterpret_cast<S*>(smem + 64 + 512);    // rotation coefficients / theta, as S
  const size_t ybytes = round_up((size_t)kMaxQ * (size_t)(a.k > 0 ? a.k : 1) * sizeof(double), 128);
  S* s_v = reinterpret_cast<S*>(smem + 64 + 512 + ybytes);
  double* s_red = reinterpret_cast<double*>(smem + 64 + 512 + ybytes + TR * sizeof(S));
  unsigned char* stages = smem + round_up(64 + 512 + ybytes + TR * sizeof(S) + 2 * TR * sizeof(double), 128);
  const size_t stage_bytes = (size_t)(a.nmat * a.w + a.nvec) * colbytes;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int w = a.w;

  // coefficients into shared memory
  if (KIND == TS_UPDPROJ || KIND == TS_UPDNORM || KIND == TS_UPD) {
    for (int c = tid; c < w; c += TR) s_h[c] = (S)a.hcoef[c];
  }
  if (KIND == TS_ROT) {
    for (int e = tid; e < w * a.k; e += TR) {
      int c = e / a.k, j = e - c * a.k;
      s_y[e] = (S)a.Y[(int64_t)j * a.ldY + c];
    }
  }
  if (KIND == TS_RESID) {
    for (int j = tid; j < a.k; j += TR) s_y[j] = (S)a.theta[j];
  }
  if (tid == 0) {
    for (int s = 0; s < a.stages; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  const int my_tiles = (a.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  if (warp == 0) {
    const int pre = my_tiles < a.stages ? my_tiles : a.stages;
    for (int s = 0; s < pre; ++s) ts_issue_tile(a, stages + s * stage_bytes, &bars[s], blockIdx.x + s * gridDim.x);
  }

  // per-thread accumulators
  Acc<S> acc0[MAXJ], acc1[MAXJ];
#pragma unroll
  for (int j = 0; j < MAXJ; ++j) { acc0[j].zero(); acc1[j].zero(); }
  Acc<S> racc;
  racc.zero();
  bool timed_out = false;
  int consumed = 0;

  for (int it = 0; it < my_tiles; ++it) {
    const int s = it % a.stages;
    const uint32_t parity = (uint32_t)((it / a.stages) & 1);
    bool ok = mbar_wait_bounded(&bars[s], parity);
    if (!__syncthreads_and(ok)) { timed_out = true; break; }
    consumed = it + 1;
    const int tile = blockIdx.x + it * gridDim.x;
    const int64_t row = (int64_t)tile * TR + tid;
    const S* st = reinterpret_cast<const S*>(stages + s * stage_bytes);
    const S* m0 = st + (size_t)a.matsel[0] * w * TR;
    const S* m1 = st + (size_t)a.matsel[1] * w * TR;
    const S* m2 = st + (size_t)a.matsel[2] * w * TR;
    const S* vst = st + (size_t)a.nmat * w * TR;   // staged vectors

    if (KIND == TS_PROJ) {
#pragma unroll
      for (int j = 0; j < MAXJ; ++j) {
        const int c = warp + NW * j;
        if (c < w) {
#pragma unroll
          for (int r = 0; r < RPL; ++r) acc0[j].fma(m0[c * TR + lane + 32 * r], vst[lane + 32 * r]);
        }
      }
    } else if (KIND == TS_INNER) {
      // prologue: v = M (z - rho bg), thread per row
      const S z = vst[tid];
      S v;
      if (a.pmode == PM_GIVEN) {
        v = vst[TR + tid];
      } else {
        const S bg = vst[TR + tid];
        v = z - (S)a.rho * bg;
        if (a.pmode == PM_JACOBI) v *= vst[2 * TR + tid];
        a.vout[row] = v;
      }
      s_v[tid] = v;
      __syncthreads();
#pragma unroll
      for (int j = 0; j < MAXJ; ++j) {
        const int c = warp + NW * j;
        if (c < w) {
#pragma unroll
          for (int r = 0; r < RPL; ++r) {
            const int i = lane + 32 * r;
            acc0[j].fma(m0[c * TR + i], vst[i]);
            acc1[j].fma(m1[c * TR + i], s_v[i]);
          }
        }
      }
    } else if (KIND == TS_UPDPROJ || KIND == TS_UPDNORM || KIND == TS_UPD) {
      // v' = v - U h, thread per row
      S dot = 0;
      for (int c = 0; c < w; ++c) dot = fmaS(m0[c * TR + tid], s_h[c], dot);
      const S vn = vst[tid] - dot;
      a.vout[row] = vn;
      if (KIND == TS_UPDNORM) racc.fma(vn, vn);
      if (KIND == TS_UPDPROJ) {
        s_v[tid] = vn;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < MAXJ; ++j) {
          const int c = warp + NW * j;
          if (c < w) {
#pragma unroll
            for (int r = 0; r < RPL; ++r) acc0[j].fma(m1[c * TR + lane + 32 * r], s_v[lane + 32 * r]);
          }
        }
      }
    } else if (KIND == TS_ROT) {
      S out[KMAX];
#pragma unroll
      for (int j = 0; j < KMAX; ++j) out[j] = 0;
      for (int c = 0; c < w; ++c) {
        const S u = m0[c * TR + tid];
#pragma unroll
        for (int j = 0; j < KMAX; ++j)
          if (j < a.k) out[j] = fmaS(u, s_y[c * a.k + j], out[j]);
      }
#pragma unroll
      for (int j = 0; j < KMAX; ++j)
        if (j < a.k) a.xout[(int64_t)j * a.ld + row] = out[j];
    } else if (KIND == TS_RESID) {
#pragma unroll
      for (int j = 0; j < MAXJ; ++j) {
        const int c = warp + NW * j;
        if (c < w) {
          const S th = s_y[c];
#pragma unroll
          for (int r = 0; r < RPL; ++r) {
            const int i = lane + 32 * r;
            const S x = m0[c * TR + i];
            const S rr = m1[c * TR + i] - th * m2[c * TR + i];
            acc0[j].fma(rr, rr);
            acc1[j].fma(x, x);
          }
        }
      }
    } else if (KIND == TS_DOT) {
      racc.fma(vst[tid], vst[TR + tid]);
    }

    __syncthreads();   // everyone is done with stage s
    if (warp == 0 && it + a.stages < my_tiles)
      ts_issue_tile(a, stages + s * stage_bytes, &bars[s], blockIdx.x + (it + a.stages) * gridDim.x);
  }

  if (timed_out) {
    // drain copies still in flight into our shared memory, then report
    if (tid == 0) atomicOr(a.status, kFlagTimeout);
    for (int it = consumed; it < my_tiles && it < consumed + a.stages; ++it) {
      const int s = it % a.stages;
      mbar_wait_bounded(&bars[s], (uint32_t)((it / a.stages) & 1));
    }
    __syncthreads();
  }

  // ---------------- per-CTA partials
  double* part = a.partials + (size_t)blockIdx.x * a.pstride;
  if (KIND == TS_PROJ || KIND == TS_INNER || KIND == TS_UPDPROJ || KIND == TS_RESID) {
#pragma unroll
    for (int j = 0; j < MAXJ; ++j) {
      const int c = warp + NW * j;
      if (c < w) {  // warp-uniform
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          acc0[j].shfl_down_add(off);
          if (KIND == TS_INNER || KIND == TS_RESID) acc1[j].shfl_down_add(off);
        }
        if (lane == 0) {
          part[c] = acc0[j].value();
          if (KIND == TS_INNER || KIND == TS_RESID) part[kMaxQ + c] = acc1[j].value();
        }
      }
    }
  } else if (KIND == TS_UPDNORM || KIND == TS_DOT) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) racc.shfl_down_add(off);
    if (lane == 0) s_red[warp] = racc.value();
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int i = 0; i < NW; ++i) t += s_red[i];
      part[0] = t;
    }
  }
  if (KIND == TS_UPD || KIND == TS_ROT) return;

  // ---------------- last CTA: sum partials in CTA order
  // Each warp owns four outputs at a time; lane l sums CTAs l, l+32, ... in
  // order, then a fixed shuffle tree combines the lanes (deterministic).
  if (!last_block_arrive(a.counter)) return;
  const int nb = gridDim.x;
  if (KIND == TS_PROJ || KIND == TS_INNER || KIND == TS_UPDPROJ || KIND == TS_RESID) {
    const bool two = (KIND == TS_INNER || KIND == TS_RESID);
    const int nout = two ? 2 * w : w;   // outputs o < w -> out0[o], else out1[o - w]
    for (int o0 = warp * 4; o0 < nout; o0 += NW * 4) {
      double t[4] = {0.0, 0.0, 0.0, 0.0};
      int col[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int o = o0 + u;
        col[u] = o < w ? o : kMaxQ + (o - w);
      }
      for (int b = lane; b < nb; b += 32) {
        const double* pb = a.partials + (size_t)b * a.pstride;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (o0 + u < nout) t[u] += pb[col[u]];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        for (int off = 16; off > 0; off >>= 1) t[u] += __shfl_down_sync(0xffffffffu, t[u], off);
      if (lane == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int o = o0 + u;
          if (o >= nout) continue;
          double v = t[u];
          if (KIND == TS_RESID) v = sqrt(v);
          if (!isfinite(v)) atomicOr(a.status, kFlagNaN);
          if (o < w) a.out0[o] = v; else a.out1[o - w] = v;
        }
      }
    }
  } else {  // UPDNORM, DOT: beta = sqrt(sum), beta0 by Pythagoras (warp 0)
    if (warp == 0) {
      double t = 0.0, hh = 0.0;
      for (int b = lane; b < nb; b += 32) t += a.partials[(size_t)b * a.pstride];
      for (int c = lane; c < w; c += 32) {
        if (a.haux) hh += a.haux[c] * a.haux[c];
        if (a.hcoef) hh += a.hcoef[c] * a.hcoef[c];
      }
      for (int off = 16; off > 0; off >>= 1) {
        t += __shfl_down_sync(0xffffffffu, t, off);
        hh += __shfl_down_sync(0xffffffffu, hh, off);
      }
      if (lane == 0) {
        if (t < 0.0) atomicOr(a.status, kFlagNotSPD);
        const double tt = t > 0.0 ? t : 0.0;
        const double beta = sqrt(tt);
        const double b0 = sqrt(tt + hh);
        a.out0[0] = beta;
        a.out0[1] = b0;
        if (!isfinite(beta) || !isfinite(b0)) atomicOr(a.status, kFlagNaN);
        const bool broke = !(beta > a.eps_breakdown * b0);
        if (broke) atomicOr(a.status, kFlagBreakdown);
        if (a.scale_out) *a.scale_out = broke ? 0.0 : 1.0 / beta;
      }
    }
  }
  __syncthreads();
  if (tid == 0) *a.counter = 0u;
}

}  // namespace trplk
