// Tall-skinny streaming kernels over the basis U (n x w, column-major).
//
// Every pass of the inner step, the +K block and the restart streams U (and
// A U or B U) from HBM once.  The kernels share one engine:
//  * persistent CTAs, grid = SMs x CTAs-per-SM (never more than the tiles);
//    a CTA walks TR-row tiles with stride gridDim.x;
//  * warp specialisation: one producer warp stages each tile into shared
//    memory with 1D bulk copies (the TMA engine, cp.async.bulk) -- one 1 KiB
//    copy per column segment and per vector segment -- and NW = TR/32
//    consumer warps compute on it; every stage has a "full" mbarrier
//    (transaction bytes) and an "empty" mbarrier (one arrival per consumer
//    warp), so consumers run ahead by up to STAGES (<= 8) tiles and the producer
//    refills a stage as soon as the last consumer has left it;
//  * compute reads shared memory only: thread-per-row for the updates
//    v <- v - U h, and balanced (column, row-slice) tasks for the projections
//    U^T v, each task with its own accumulator;
//  * projections accumulate in FP64 (double data) or compensated FP32 (float
//    data: each lane's four consecutive products summed in FP32, the block
//    sums added exactly by TwoSum) -- except the first CGS pass of the float
//    path, accumulated plainly in FP32 because the second, compensated pass
//    removes its error --
//    are reduced per CTA and then summed in CTA order by the last CTA to
//    finish (deterministic, no floating-point atomics).
// Rows n..ld-1 of every array are zero, so whole tiles are always copied.
// Every wait is bounded (a.polls polls) and also ends when another warp of
// the CTA has given up (a flag in shared memory); every wait's outcome is
// warp-uniform, and the consumer warps of TS_UPDPROJ, which meet at a named
// barrier once per tile, decide together at that barrier.  A CTA that gives
// up sets kFlagTimeout, waits until every bulk copy it issued has landed (so
// no copy writes into the shared memory of an exited CTA), still takes part
// in the grid reduction's ticket, and returns; the host reads the flag.
#pragma once
#include <type_traits>

#include "common.cuh"

namespace trplk {

enum TSKind : int {
  TS_PROJ = 0,     // out0 = mat0^T vec0                                   (1 RHS)
  TS_INNER = 1,    // v = M(zs - rho bs); out0 = mat0^T z; out1 = mat1^T v  (2 RHS;
                   // zs, bs = z, bg, or the staged vectors vsrc, bsrc in block TRPL+K)
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

// Four consecutive values of S (one 128-bit shared load for float, two for
// double).  Addresses are 16-byte aligned: a lane's rows start at 4*lane.
template <typename S> struct V4 { S x, y, z, w; };
__device__ __forceinline__ V4<float> ld4(const float* p) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  return {q.x, q.y, q.z, q.w};
}
__device__ __forceinline__ V4<double> ld4(const double* p) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void st4(float* p, const V4<float>& v) {
  *reinterpret_cast<float4*>(p) = make_float4(v.x, v.y, v.z, v.w);
}
__device__ __forceinline__ void st4(double* p, const V4<double>& v) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v.x, v.y);
  reinterpret_cast<double2*>(p)[1] = make_double2(v.z, v.w);
}

template <typename S>
struct TSArgs {
  const S* mat[3];     // staged matrices, w columns each (ld)
  int nmat;            // number of distinct staged matrices
  int matsel[3];       // which staged matrix plays operand 0/1/2 of the kind
  const S* vec[5];     // staged vectors
  int nvec;
  int vsrc, bsrc;      // TS_INNER: staged vectors the new Lanczos vector is formed from (0, 1: z and bg)
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
  uint32_t polls;        // bound of every mbarrier wait (kWaitPolls unless lowered for a test)
};

// Row slices per tile for the projection tasks: a task is (column, slice)
// and a lane covers RPS = TR / (32 NQ) rows of its slice.
template <typename S> struct Slices;
template <> struct Slices<double> { static constexpr int NQ = 1; };
template <> struct Slices<float> { static constexpr int NQ = 2; };

template <typename S>
struct TSLayout {
  static constexpr int TR = Tile<S>::TR;
  static constexpr int NW = TR / 32;              // consumer warps
  static constexpr int NQ = Slices<S>::NQ;
  static constexpr int RPS = TR / (32 * NQ);      // rows per lane per task (4)
  static constexpr uint32_t COLB = TR * sizeof(S);
};

// Shared memory (bytes): [full/empty bars 128][h 512][Y 64*k doubles]
// [task partials 2*NQ*64 doubles][red 64 doubles][stage 0 | stage 1 | ...],
// a stage = staged columns and vectors, then one TR-vector scratch (s_v).
template <typename S>
__host__ __device__ inline size_t ts_smem_fixed(int k) {
  using L = TSLayout<S>;
  const size_t ybytes = (size_t)kMaxQ * (size_t)(k > 0 ? k : 1) * sizeof(double);
  const size_t fixed = 128 + 512 + ybytes + 2 * L::NQ * kMaxQ * sizeof(double) + 64 * sizeof(double);
  return (fixed + 127) / 128 * 128;
}
template <typename S>
__host__ __device__ inline size_t ts_stage_bytes(int nmat, int w, int nvec) {
  return (size_t)(nmat * w + nvec + 1) * TSLayout<S>::COLB;
}

template <typename S>
__device__ __forceinline__ void ts_issue_tile(const TSArgs<S>& a, unsigned char* stage, uint64_t* full,
                                              int tile, int lane) {
  constexpr uint32_t colbytes = TSLayout<S>::COLB;
  constexpr int TR = TSLayout<S>::TR;
  const int nmc = a.nmat * a.w;
  const int ncopies = nmc + a.nvec;
  if (lane == 0) mbar_arrive_expect_tx(full, (uint32_t)ncopies * colbytes);
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
    bulk_g2s(stage + (size_t)c * colbytes, src, colbytes, full);
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

template <int NTHREADS>
__device__ __forceinline__ void consumer_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(NTHREADS) : "memory");
}

// Named barrier 1 over the consumer threads that also ORs a predicate across
// them: true in every consumer thread if any passed `flag` != 0.
template <int NTHREADS>
__device__ __forceinline__ bool consumer_sync_or(bool flag) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n bar.red.or.pred po, 1, %2, pi;\n"
      " selp.u32 %0, 1, 0, po;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)flag), "n"(NTHREADS)
      : "memory");
  return r != 0;
}

// Two CTAs per SM for the float path (<= 113 registers), where the FP32
// pipes need the extra warps to hide the compensated-sum latency chains.
template <typename S> struct MinBlocks { static constexpr int value = 1; };
template <> struct MinBlocks<float> { static constexpr int value = 2; };

// MAXW: the widest basis the instantiation serves; its accumulators (MAXT
// tasks per warp) live in registers for the whole kernel, so narrow bases get
// their own instantiation with a third of them (no spills, see the launcher).
template <typename S, int KIND, int MAXW = kMaxQ>
__global__ void __launch_bounds__(Tile<S>::TR + 32, MinBlocks<S>::value) ts_kernel(TSArgs<S> a) {
  using L = TSLayout<S>;
  constexpr int TR = L::TR, NW = L::NW, NQ = L::NQ, RPS = L::RPS;
  constexpr int MAXT = NQ * MAXW / NW;
  constexpr int SLICE = TR / NQ;
  static_assert(RPS == 4, "the task phase maps four consecutive rows to a lane");
  constexpr bool TASKS = (KIND == TS_PROJ || KIND == TS_INNER || KIND == TS_UPDPROJ || KIND == TS_RESID);
  constexpr bool TWO = (KIND == TS_INNER || KIND == TS_RESID);

  // launched as a programmatic dependent of the previous kernel on the
  // stream: wait until it has finished and its writes are visible before any
  // global access
  grid_dependency_wait();
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + 8;
  S* s_h = reinterpret_cast<S*>(smem + 128);
  S* s_y = reinterpret_cast<S*>(smem + 128 + 512);
  const size_t ybytes = (size_t)kMaxQ * (size_t)(a.k > 0 ? a.k : 1) * sizeof(double);
  double* s_task = reinterpret_cast<double*>(smem + 128 + 512 + ybytes);   // [2][NQ * kMaxQ]
  double* s_red = s_task + 2 * NQ * kMaxQ;
  unsigned char* stages = smem + ts_smem_fixed<S>(a.k);
  const size_t stage_bytes = ts_stage_bytes<S>(a.nmat, a.w, a.nvec);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool producer = (warp == NW);
  const int w = a.w;
  // Projection tasks: task (c, h) sums column c over row slice h of every
  // tile.  Consumer warp `warp` takes slice hs = warp / WPS and the columns
  // cls, cls + WPS, cls + 2 WPS, ... of it (its j-th task is column
  // cls + WPS j), so every task of a warp reads the same rows of the staged
  // vectors; a lane owns the four consecutive rows i0 .. i0 + 3 of the slice.
  constexpr int WPS = NW / NQ;
  const int hs = warp / WPS, cls = warp - hs * WPS;
  const int i0 = hs * SLICE + 4 * lane;

  if (KIND == TS_UPDPROJ || KIND == TS_UPDNORM || KIND == TS_UPD)
    for (int c = tid; c < w; c += blockDim.x) s_h[c] = (S)a.hcoef[c];
  if (KIND == TS_ROT)
    for (int e = tid; e < w * a.k; e += blockDim.x) {
      const int c = e / a.k, j = e - c * a.k;
      s_y[e] = (S)a.Y[(int64_t)j * a.ldY + c];
    }
  if (KIND == TS_RESID)
    for (int j = tid; j < a.k; j += blockDim.x) s_y[j] = (S)a.theta[j];
  __shared__ int s_abort;   // set by the first warp that gives up a wait
  if (tid == 0) {
    s_abort = 0;
    for (int s = 0; s < a.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NW);
    }
    fence_mbar_init();
  }
  __syncthreads();
  volatile int* abort_flag = &s_abort;

  const int my_tiles = (a.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  // TS_INNER's second right-hand side is the first CGS pass: plain
  // accumulation (its error is removed by the compensated second pass)
  using Acc1 = typename std::conditional<KIND == TS_INNER, AccFast<S>, Acc<S>>::type;
  Acc<S> acc0[MAXT];
  Acc1 acc1[MAXT];
#pragma unroll
  for (int j = 0; j < MAXT; ++j) { acc0[j].zero(); acc1[j].zero(); }
  Acc<S> racc;
  racc.zero();
  int issued_upto = 0;   // producer: tiles issued
  bool fail = false;

  if (producer) {
    // ---------------- producer warp: keep STAGES tiles in flight
    for (int it = 0; it < my_tiles; ++it) {
      const int s = it % a.stages;
      if (it >= a.stages) {
        int ok = 1;
        if (lane == 0) {
          ok = 0;
          const uint32_t par = (uint32_t)(((it / a.stages) - 1) & 1);
          for (uint32_t i = 0; i < a.polls; ++i) {
            if (mbar_try_wait(&empty[s], par)) { ok = 1; break; }
            if (*abort_flag) break;
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          if (lane == 0) *abort_flag = 1;
          fail = true;
          break;
        }
      }
      ts_issue_tile(a, stages + s * stage_bytes, &full[s], blockIdx.x + it * gridDim.x, lane);
      issued_upto = it + 1;
    }
  } else {
    // ---------------- consumer warps
    for (int it = 0; it < my_tiles; ++it) {
      const int s = it % a.stages;
      const bool ok = mbar_warp_wait(&full[s], (uint32_t)((it / a.stages) & 1), a.polls, abort_flag);
      if (!ok) {
        if (lane == 0) *abort_flag = 1;
        // TS_UPDPROJ's consumers meet at a named barrier in every tile: a
        // warp that gave up still goes there once, where all of them learn it
        if (KIND == TS_UPDPROJ) consumer_sync_or<TR>(true);
        fail = true;
        break;
      }
      const int tile = blockIdx.x + it * gridDim.x;
      const int64_t row0 = (int64_t)tile * TR;
      const S* st = reinterpret_cast<const S*>(stages + s * stage_bytes);
      const S* m0 = st + (size_t)a.matsel[0] * w * TR;
      const S* m1 = st + (size_t)a.matsel[1] * w * TR;
      const S* m2 = st + (size_t)a.matsel[2] * w * TR;
      const S* vst = st + (size_t)a.nmat * w * TR;                          // staged vectors
      S* s_v = const_cast<S*>(st) + (size_t)(a.nmat * w + a.nvec) * TR;     // per-stage scratch

      if (KIND == TS_PROJ || KIND == TS_INNER || KIND == TS_RESID) {
        // Row mapping of the task phase: the warp's tasks all lie in its row
        // slice hs, where a lane owns the four consecutive rows i0 .. i0+3,
        // read with 128-bit shared loads; the staged vector (and, for
        // TS_INNER, the preconditioned vector) of those rows stays in
        // registers for the whole tile.
        const V4<S> zq = ld4(vst + i0);
        V4<S> vq = zq;
        if (KIND == TS_INNER) {
          // no barrier: each warp forms the preconditioned vector for its
          // slice; the lanes whose rows fall in row block `warp` store it
          if (a.pmode == PM_GIVEN) {
            vq = ld4(vst + TR + i0);
          } else {
            // the source of the new vector: the just-multiplied column (z, bg)
            // or, in block TRPL+K, the column of the same sequence b back
            const V4<S> zs = a.vsrc ? ld4(vst + a.vsrc * TR + i0) : zq;
            const V4<S> bg = ld4(vst + a.bsrc * TR + i0);
            const S rho = (S)a.rho;
            V4<S> v;
            v.x = zs.x - rho * bg.x;
            v.y = zs.y - rho * bg.y;
            v.z = zs.z - rho * bg.z;
            v.w = zs.w - rho * bg.w;
            if (a.pmode == PM_JACOBI) {
              const V4<S> dv = ld4(vst + 2 * TR + i0);
              v.x *= dv.x;
              v.y *= dv.y;
              v.z *= dv.z;
              v.w *= dv.w;
            }
            if ((i0 >> 5) == warp) st4(a.vout + row0 + i0, v);
            vq = v;
          }
        }
        const bool alias = (a.matsel[1] == a.matsel[0]);
        // Tasks go in pairs (columns c, c + WPS) so two independent
        // accumulation chains per right-hand side interleave; the second of
        // the last pair may be idle.
#pragma unroll
        for (int j = 0; j < MAXT; j += 2) {
          const int c = cls + WPS * j;
          if (c >= w) break;   // warp-uniform branch
          const bool two = c + WPS < w;
          const int off = c * TR + i0;
          const int off2 = two ? off + WPS * TR : off;
          const V4<S> u = ld4(m0 + off);
          const V4<S> u2 = ld4(m0 + off2);
          const V4<S>& z = zq;
          if (KIND == TS_PROJ) {
            acc0[j].fma4(u.x, z.x, u.y, z.y, u.z, z.z, u.w, z.w);
            if (two) acc0[j + 1].fma4(u2.x, z.x, u2.y, z.y, u2.z, z.z, u2.w, z.w);
            continue;
          }
          if (KIND == TS_INNER) {
            const V4<S>& v = vq;
            const V4<S> b = alias ? u : ld4(m1 + off);
            const V4<S> b2 = alias ? u2 : ld4(m1 + off2);
            acc0[j].fma4(u.x, z.x, u.y, z.y, u.z, z.z, u.w, z.w);
            acc1[j].fma4(b.x, v.x, b.y, v.y, b.z, v.z, b.w, v.w);
            if (two) {
              acc0[j + 1].fma4(u2.x, z.x, u2.y, z.y, u2.z, z.z, u2.w, z.w);
              acc1[j + 1].fma4(b2.x, v.x, b2.y, v.y, b2.z, v.z, b2.w, v.w);
            }
            continue;
          }
          {  // TS_RESID: ||AX_c - theta_c BX_c||^2 and ||X_c||^2 (second task handled alone below)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              if (q == 1 && !two) break;
              const int cc = q ? c + WPS : c, oo = q ? off2 : off;
              const V4<S> uu = q ? u2 : u;
              const S th = s_y[cc];
              const V4<S> ax = ld4(m1 + oo), bx = ld4(m2 + oo);
              const S r0 = ax.x - th * bx.x, r1 = ax.y - th * bx.y, r2 = ax.z - th * bx.z, r3 = ax.w - th * bx.w;
              acc0[j + q].fma4(r0, r0, r1, r1, r2, r2, r3, r3);
              acc1[j + q].fma4(uu.x, uu.x, uu.y, uu.y, uu.z, uu.z, uu.w, uu.w);
            }
          }
        }
      } else if (KIND == TS_UPDPROJ || KIND == TS_UPDNORM || KIND == TS_UPD) {
        // v' = v - U h, thread per row, two chains
        // (even columns into d0, odd into d1; coefficients read four at a time)
        S d0 = 0, d1 = 0;
        int c = 0;
        for (; c + 3 < w; c += 4) {
          const V4<S> hc = ld4(s_h + c);
          d0 = fmaS(m0[c * TR + tid], hc.x, d0);
          d1 = fmaS(m0[(c + 1) * TR + tid], hc.y, d1);
          d0 = fmaS(m0[(c + 2) * TR + tid], hc.z, d0);
          d1 = fmaS(m0[(c + 3) * TR + tid], hc.w, d1);
        }
        for (; c + 1 < w; c += 2) {
          d0 = fmaS(m0[c * TR + tid], s_h[c], d0);
          d1 = fmaS(m0[(c + 1) * TR + tid], s_h[c + 1], d1);
        }
        if (c < w) d0 = fmaS(m0[c * TR + tid], s_h[c], d0);
        const S vn = vst[tid] - (d0 + d1);
        a.vout[row0 + tid] = vn;
        if (KIND == TS_UPDNORM) racc.fma(vn, vn);
        if (KIND == TS_UPDPROJ) {
          s_v[tid] = vn;
          // the tile's barrier; it also tells every consumer whether another
          // consumer warp gave up its wait for this tile
          if (consumer_sync_or<TR>(false)) { fail = true; break; }
          const V4<S> v = ld4(s_v + i0);
#pragma unroll
          for (int j = 0; j < MAXT; j += 2) {
            const int cc = cls + WPS * j;
            if (cc >= w) break;
            const bool two = cc + WPS < w;
            const V4<S> b = ld4(m1 + cc * TR + i0);
            const V4<S> b2 = ld4(m1 + (two ? cc + WPS : cc) * TR + i0);
            acc0[j].fma4(b.x, v.x, b.y, v.y, b.z, v.z, b.w, v.w);
            if (two) acc0[j + 1].fma4(b2.x, v.x, b2.y, v.y, b2.z, v.z, b2.w, v.w);
          }
        }
      } else if (KIND == TS_ROT) {
        // outputs in chunks of KC so no FMA is spent on columns past k
        constexpr int KC = 4;
        for (int j0 = 0; j0 < a.k; j0 += KC) {
          if (j0 + KC <= a.k) {
            S out[KC];
#pragma unroll
            for (int u = 0; u < KC; ++u) out[u] = 0;
            for (int c = 0; c < w; ++c) {
              const S uu = m0[c * TR + tid];
#pragma unroll
              for (int u = 0; u < KC; ++u) out[u] = fmaS(uu, s_y[c * a.k + j0 + u], out[u]);
            }
#pragma unroll
            for (int u = 0; u < KC; ++u) a.xout[(int64_t)(j0 + u) * a.ld + row0 + tid] = out[u];
          } else {
            for (int j = j0; j < a.k; ++j) {
              S o = 0;
              for (int c = 0; c < w; ++c) o = fmaS(m0[c * TR + tid], s_y[c * a.k + j], o);
              a.xout[(int64_t)j * a.ld + row0 + tid] = o;
            }
          }
        }
      } else if (KIND == TS_DOT) {
        racc.fma(vst[tid], vst[TR + tid]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
  }

  // The tiles are done: the next kernel's CTAs may now be scheduled as ours
  // exit (only the reductions below remain).  Triggered this late so that
  // they never hold SM resources while this kernel still streams.
  grid_dependents_launch();

  // ---------------- agree on a timeout, drain, report
  // Tiles older than issued_upto - stages have landed: the producer issued
  // each later tile only after every consumer warp had released the older
  // one's stage, which it did after seeing that tile's full barrier complete.
  // The last `stages` issued tiles may still be in flight.
  if (fail) *abort_flag = 1;
  __syncthreads();
  if (*abort_flag) {
    if (tid == 0) atomicOr(a.status, kFlagTimeout);
    if (producer && lane == 0) {
      for (int it = issued_upto - a.stages; it < issued_upto; ++it) {
        if (it < 0) continue;
        const int s = it % a.stages;
        if (!mbar_wait_bounded(&full[s], (uint32_t)((it / a.stages) & 1), kDrainPolls))
          atomicOr(a.status, kFlagDrain);
      }
    }
  }
  __syncthreads();

  // ---------------- per-CTA partials
  double* part = a.partials + (size_t)blockIdx.x * a.pstride;
  if (TASKS) {
    if (!producer) {
#pragma unroll
      for (int j = 0; j < MAXT; ++j) {
        const int c = cls + WPS * j;
        if (c >= w) break;
        const int t = c * NQ + hs;   // slot of task (c, hs)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          acc0[j].shfl_down_add(off);
          if (TWO) acc1[j].shfl_down_add(off);
        }
        if (lane == 0) {
          Part<S>::of(acc0[j]).store(&s_task[t]);
          if (TWO) Part<S>::of(acc1[j]).store(&s_task[NQ * kMaxQ + t]);
        }
      }
    }
    __syncthreads();
    for (int o = tid; o < (TWO ? 2 : 1) * w; o += blockDim.x) {
      const int r = o / w, c = o - r * w;
      Part<S> t, x;
      t.load(&s_task[r * NQ * kMaxQ + c * NQ]);
#pragma unroll
      for (int h = 1; h < NQ; ++h) {
        x.load(&s_task[r * NQ * kMaxQ + c * NQ + h]);
        t.add(x);
      }
      t.store(&part[r * kMaxQ + c]);
    }
  } else if (KIND == TS_UPDNORM || KIND == TS_DOT) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) racc.shfl_down_add(off);
    if (lane == 0) s_red[warp] = producer ? 0.0 : racc.value();
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
  const int nwarps = blockDim.x / 32;
  if (TASKS) {
    const int nout = TWO ? 2 * w : w;   // outputs o < w -> out0[o], else out1[o - w]
    for (int o0 = warp * 4; o0 < nout; o0 += nwarps * 4) {
      Part<S> t[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) t[u].zero();
      int col[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int o = o0 + u;
        col[u] = o < w ? o : kMaxQ + (o - w);
      }
      // the loads of eight CTAs' partials are issued before they are added
      // (in the same order as one at a time: the sums are unchanged)
      for (int b0 = lane; b0 < nb; b0 += 32 * 8) {
        Part<S> pv[8][4];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int b = b0 + 32 * q;
          const double* pb = a.partials + (size_t)b * a.pstride;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (b < nb && o0 + u < nout) pv[q][u].load(pb + col[u]);
            else pv[q][u].zero();
          }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (b0 + 32 * q < nb) t[u].add(pv[q][u]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        for (int off = 16; off > 0; off >>= 1) t[u].shfl_down_add(off);
      if (lane == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int o = o0 + u;
          if (o >= nout) continue;
          double v = t[u].value();
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
