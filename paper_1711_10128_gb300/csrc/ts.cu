// Launchers of the tall-skinny streaming kernels (see tallskinny.cuh).
#include <algorithm>
#include <atomic>
#include <cstring>

#include "launch.h"
#include "tallskinny.cuh"

namespace trplk {

namespace {

constexpr size_t kSmemMax = 232448 - 1024;   // opt-in shared memory per CTA less static use
constexpr size_t kSmemPerSM = 233472;        // shared memory per SM

// CTAs of one instantiation that fit on an SM by registers and threads (the
// same on every device of this architecture); opts the kernel into the full
// shared memory on `device`.
template <typename S, int KIND, int MAXW>
int regs_limit(int device) {
  static std::atomic<int> lim{0};
  int l = lim.load(std::memory_order_relaxed);
  if (!l) {
    cudaFuncAttributes fa;
    TRPLK_CUDA_TRY(cudaFuncGetAttributes(&fa, ts_kernel<S, KIND, MAXW>));
    const int threads = Tile<S>::TR + 32;
    const int regs = std::max(fa.numRegs, 1) * threads;
    l = std::max(1, std::min(65536 / regs, 2048 / threads));
    lim.store(l, std::memory_order_relaxed);
  }
  smem_optin<ts_kernel<S, KIND, MAXW>>((int)kSmemMax, device);
  return l;
}

template <typename S, int KIND, int MAXW>
void launch_kind(const Ctx& c, TSArgs<S>& a, size_t fixed, size_t stage, double bytes) {
  // Most CTAs per SM that still keep >= 2 stages each (measured: a second
  // producer/consumer group per SM hides more latency than deeper pipelines
  // of one group, e.g. 56.7 us against 87.5 us for the FP32 update+norm pass
  // at n = 2^21, w = 32), then as many stages as fit, up to 8.
  const int lim = regs_limit<S, KIND, MAXW>(c.device);
  int per_sm = 1, stages = 0;
  for (int cand = lim; cand >= 1; --cand) {
    const size_t per_cta = std::min<size_t>(kSmemMax, kSmemPerSM / cand - 1024);
    if (per_cta <= fixed) continue;
    const int st = (int)std::min<size_t>(8, (per_cta - fixed) / stage);
    if (st >= 2 || (cand == 1 && st >= 1)) {
      per_sm = cand;
      stages = st;
      break;
    }
  }
  if (stages < 1) throw Error(TRPLK_EINVAL, "tile does not fit in shared memory");
  a.stages = stages;
  const size_t smem = fixed + (size_t)stages * stage;
  int grid = (int)std::min<int64_t>(a.ntiles, (int64_t)c.sms * per_sm);
  grid = std::min(grid, kMaxPartials);
  ProfScope ps(c, prof_kind<S>(PK_TS_PROJ + KIND), bytes);
  launch_dependent(ts_kernel<S, KIND, MAXW>, dim3(grid), dim3(Tile<S>::TR + 32), smem, c.stream, a);
  check_launch("ts_kernel");
}

// Kinds with per-warp projection tasks get instantiations sized for the
// basis width (w <= 32, <= 48, <= 64): the accumulators of the widest one
// spilled inside its task loop (measured at w = 23).
template <typename S, int KIND>
void launch_tasks(const Ctx& c, TSArgs<S>& a, size_t fixed, size_t stage, double bytes) {
  if (a.w <= kMaxQ / 2)
    launch_kind<S, KIND, kMaxQ / 2>(c, a, fixed, stage, bytes);
  else if (a.w <= 3 * kMaxQ / 4)
    launch_kind<S, KIND, 3 * kMaxQ / 4>(c, a, fixed, stage, bytes);
  else
    launch_kind<S, KIND, kMaxQ>(c, a, fixed, stage, bytes);
}

template <typename S>
void run(const Ctx& c, TSArgs<S> a, int kind) {
  constexpr int TR = Tile<S>::TR;
  if (a.ld % TR != 0) throw Error(TRPLK_EINVAL, "leading dimension must be a multiple of 256");
  if (a.w < 0 || a.w > kMaxQ) throw Error(TRPLK_EINVAL, "basis width out of range");
  a.ntiles = (int)(a.ld / TR);
  if (a.ntiles == 0) return;
  const size_t fixed = ts_smem_fixed<S>(a.k);
  const size_t stage = ts_stage_bytes<S>(a.nmat, a.w, a.nvec);
  a.partials = c.partials;
  a.pstride = kPartialStride;
  a.counter = c.counter;
  a.status = c.status;
  a.polls = c.wait_polls;
  a.kind = kind;
  // algorithmic bytes: every staged column and vector once, plus the outputs
  double bytes = (double)(a.nmat * a.w + a.nvec) * a.ld * sizeof(S);
  if (kind == TS_INNER && a.pmode != PM_GIVEN) bytes += (double)a.ld * sizeof(S);
  if (kind == TS_UPDPROJ || kind == TS_UPDNORM || kind == TS_UPD) bytes += (double)a.ld * sizeof(S);
  if (kind == TS_ROT) bytes += (double)a.k * a.ld * sizeof(S);
  switch (kind) {
    case TS_PROJ: launch_tasks<S, TS_PROJ>(c, a, fixed, stage, bytes); break;
    case TS_INNER: launch_tasks<S, TS_INNER>(c, a, fixed, stage, bytes); break;
    case TS_UPDPROJ: launch_tasks<S, TS_UPDPROJ>(c, a, fixed, stage, bytes); break;
    case TS_UPDNORM: launch_kind<S, TS_UPDNORM, kMaxQ>(c, a, fixed, stage, bytes); break;
    case TS_UPD: launch_kind<S, TS_UPD, kMaxQ>(c, a, fixed, stage, bytes); break;
    case TS_ROT: launch_kind<S, TS_ROT, kMaxQ>(c, a, fixed, stage, bytes); break;
    case TS_RESID: launch_tasks<S, TS_RESID>(c, a, fixed, stage, bytes); break;
    case TS_DOT: launch_kind<S, TS_DOT, kMaxQ>(c, a, fixed, stage, bytes); break;
    default: throw Error(TRPLK_EINVAL, "unknown tall-skinny kind");
  }
}

template <typename S>
TSArgs<S> blank() {
  TSArgs<S> a;
  memset(&a, 0, sizeof(a));
  a.matsel[0] = 0;
  a.matsel[1] = 0;
  a.matsel[2] = 0;
  a.vsrc = 0;
  a.bsrc = 1;
  return a;
}

}  // namespace

template <typename S>
void ts_project(const Ctx& c, int64_t ld, int w, const S* BU, const S* v, double* hout) {
  if (w == 0) return;
  TSArgs<S> a = blank<S>();
  a.mat[0] = BU; a.nmat = 1;
  a.vec[0] = v; a.nvec = 1;
  a.w = w; a.ld = ld; a.out0 = hout;
  run(c, a, TS_PROJ);
}

template <typename S>
void ts_inner(const Ctx& c, int64_t ld, int w, const S* U, const S* BU, const S* z, const S* bg,
              const S* dinv, int pmode, double rho, S* v, double* tcol, double* h1, const S* zsrc,
              const S* bsrc) {
  TSArgs<S> a = blank<S>();
  a.mat[0] = U;
  if (BU == U) { a.nmat = 1; a.matsel[1] = 0; }
  else { a.mat[1] = BU; a.nmat = 2; a.matsel[1] = 1; }
  a.vec[0] = z;
  if (pmode == PM_GIVEN) { a.vec[1] = v; a.nvec = 2; }
  else {
    a.vec[1] = bg;
    a.nvec = 2;
    if (pmode == PM_JACOBI) { a.vec[2] = dinv; a.nvec = 3; }
    if (zsrc) {   // block TRPL+K: the new vector comes from another column
      if (pmode != PM_JACOBI) a.vec[2] = z;   // placeholder at the Jacobi slot
      a.vec[3] = zsrc;
      a.vec[4] = bsrc;
      a.nvec = 5;
      a.vsrc = 3;
      a.bsrc = 4;
    }
  }
  a.pmode = pmode; a.rho = rho; a.vout = v;
  a.w = w; a.ld = ld; a.out0 = tcol; a.out1 = h1;
  run(c, a, TS_INNER);
}

template <typename S>
void ts_update_project(const Ctx& c, int64_t ld, int w, const S* U, const S* BU, const double* h,
                       S* v, double* hout) {
  TSArgs<S> a = blank<S>();
  a.mat[0] = U;
  if (BU == U) { a.nmat = 1; a.matsel[1] = 0; }
  else { a.mat[1] = BU; a.nmat = 2; a.matsel[1] = 1; }
  a.vec[0] = v; a.nvec = 1;
  a.hcoef = h; a.vout = v;
  a.w = w; a.ld = ld; a.out0 = hout;
  run(c, a, TS_UPDPROJ);
}

template <typename S>
void ts_update_norm(const Ctx& c, int64_t ld, int w, const S* U, const double* h, const double* haux,
                    S* v, double* beta2, double* scale, double eps_breakdown) {
  TSArgs<S> a = blank<S>();
  a.mat[0] = U; a.nmat = w > 0 ? 1 : 0;
  a.vec[0] = v; a.nvec = 1;
  a.hcoef = w > 0 ? h : nullptr; a.haux = w > 0 ? haux : nullptr; a.vout = v;
  a.w = w; a.ld = ld; a.out0 = beta2; a.scale_out = scale; a.eps_breakdown = eps_breakdown;
  run(c, a, TS_UPDNORM);
}

template <typename S>
void ts_update(const Ctx& c, int64_t ld, int w, const S* U, const double* h, S* v) {
  if (w == 0) return;
  TSArgs<S> a = blank<S>();
  a.mat[0] = U; a.nmat = 1;
  a.vec[0] = v; a.nvec = 1;
  a.hcoef = h; a.vout = v;
  a.w = w; a.ld = ld;
  run(c, a, TS_UPD);
}

template <typename S>
void ts_dot_norm(const Ctx& c, int64_t ld, const S* v, const S* bv, const double* h1,
                 const double* h2, int w, double* beta2, double* scale, double eps_breakdown) {
  TSArgs<S> a = blank<S>();
  a.nmat = 0;
  a.vec[0] = v; a.vec[1] = bv; a.nvec = 2;
  a.w = w; a.ld = ld; a.hcoef = w > 0 ? h2 : nullptr; a.haux = w > 0 ? h1 : nullptr;
  a.out0 = beta2; a.scale_out = scale; a.eps_breakdown = eps_breakdown;
  run(c, a, TS_DOT);
}

template <typename S>
void ts_rotate(const Ctx& c, int64_t ld, int w, int k, const S* U, const double* Y, int ldY, S* X,
               bool tensor_cores) {
  if (k > kMaxK) throw Error(TRPLK_EINVAL, "rotation width exceeds 32");
  if constexpr (sizeof(S) == 4) {
    if (tensor_cores && rotate_tc_preferred(w, k)) {
      rotate_tc(c, ld, w, k, U, Y, ldY, X);
      return;
    }
  }
  TSArgs<S> a = blank<S>();
  a.mat[0] = U; a.nmat = 1;
  a.nvec = 0;
  a.Y = Y; a.ldY = ldY; a.k = k; a.xout = X;
  a.w = w; a.ld = ld;
  run(c, a, TS_ROT);
}

template <typename S>
void ts_resid(const Ctx& c, int64_t ld, int k, const S* X, const S* AX, const S* BX,
              const double* theta, double* rnorm, double* xnorm) {
  TSArgs<S> a = blank<S>();
  a.mat[0] = X; a.mat[1] = AX; a.matsel[0] = 0; a.matsel[1] = 1;
  if (BX == nullptr || BX == X) { a.nmat = 2; a.matsel[2] = 0; }
  else { a.mat[2] = BX; a.nmat = 3; a.matsel[2] = 2; }
  a.nvec = 0;
  a.theta = theta; a.k = k;
  a.w = k; a.ld = ld; a.out0 = rnorm; a.out1 = xnorm;
  run(c, a, TS_RESID);
}

#define TRPLK_INST(S)                                                                                 \
  template void ts_project<S>(const Ctx&, int64_t, int, const S*, const S*, double*);                 \
  template void ts_inner<S>(const Ctx&, int64_t, int, const S*, const S*, const S*, const S*,         \
                            const S*, int, double, S*, double*, double*, const S*, const S*);         \
  template void ts_update_project<S>(const Ctx&, int64_t, int, const S*, const S*, const double*, S*, \
                                     double*);                                                        \
  template void ts_update_norm<S>(const Ctx&, int64_t, int, const S*, const double*, const double*,   \
                                  S*, double*, double*, double);                                      \
  template void ts_update<S>(const Ctx&, int64_t, int, const S*, const double*, S*);                  \
  template void ts_dot_norm<S>(const Ctx&, int64_t, const S*, const S*, const double*, const double*, \
                               int, double*, double*, double);                                        \
  template void ts_rotate<S>(const Ctx&, int64_t, int, int, const S*, const double*, int, S*, bool);  \
  template void ts_resid<S>(const Ctx&, int64_t, int, const S*, const S*, const S*, const double*,    \
                            double*, double*);

TRPLK_INST(double)
TRPLK_INST(float)

}  // namespace trplk
