// Host driver of TRPL+K (Algorithm 1 of Wu, Xue and Stathopoulos, Sec. 3) and
// the C ABI of libtrplk.
//
// The cycle loop runs on the host and enqueues every vector operation on the
// handle's stream; the only device->host traffic is a small read-back per
// cycle (Ritz values, residual norms, Lanczos norms, status flags: under
// 2 KB).  The projection T, the Ritz coefficients Y and all n-vectors stay in
// device memory.  Storage type S is double (FP64 path) or float (FP32 phase
// of the mixed path); coefficients, T, Ritz values and norms are always FP64.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "launch.h"
#include "tallskinny.cuh"

using namespace trplk;

#include "handle.h"

// Build the SELL-32 copy of a device CSR (values from the FP64 array; an
// FP32 copy too when f32 != nullptr) unless padding would add more than 25%.
namespace {
// SELL-32 over the m rows perm[0..m) (perm null: rows 0..m-1): slice offsets
// from the slice lengths, then column indices and FP64 (and FP32) values.
void build_sell(trplk_handle* h, DevCsr<double>& d, const std::string& tag, DevCsr<float>* f32, int64_t m,
                const int32_t* perm, const std::vector<int64_t>& ptr) {
  const Ctx& c = h->ctx;
  const int64_t nslices = (m + 31) / 32;
  const int64_t padded = ptr[nslices];
  auto* sp = static_cast<int64_t*>(h->get(tag + ".sl_ptr", (nslices + 1) * sizeof(int64_t)));
  auto* sc = static_cast<int32_t*>(h->get(tag + ".sl_col", std::max<int64_t>(padded, 1) * sizeof(int32_t)));
  auto* sv = static_cast<double*>(h->get(tag + ".sl_val", std::max<int64_t>(padded, 1) * sizeof(double)));
  TRPLK_CUDA_TRY(cudaMemcpyAsync(sp, ptr.data(), (nslices + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c.stream));
  sell_fill<double>(c, m, d.rowptr, d.col, d.val, perm, sp, sc, sv);
  d.sl_ptr = sp;
  d.sl_col = sc;
  d.sl_val = sv;
  if (f32) {
    auto* svf = static_cast<float*>(h->get(tag + ".sl_valf", std::max<int64_t>(padded, 1) * sizeof(float)));
    sell_fill<float>(c, m, d.rowptr, d.col, d.val, perm, sp, nullptr, svf);
    f32->sl_ptr = sp;
    f32->sl_col = sc;
    f32->sl_val = svf;
  }
  h->sync();   // ptr (host vector) must stay alive until its copy finished
}

std::vector<int64_t> slice_offsets(trplk_handle* h, const std::string& tag, int64_t m, const int64_t* rowptr,
                                   const int32_t* perm) {
  const Ctx& c = h->ctx;
  const int64_t nslices = (m + 31) / 32;
  std::vector<int64_t> ptr(nslices + 1, 0);
  if (nslices == 0) return ptr;
  auto* lens = static_cast<int32_t*>(h->get(tag + ".sl_len", nslices * sizeof(int32_t)));
  sell_lengths(c, m, rowptr, perm, lens);
  std::vector<int32_t> hl(nslices);
  TRPLK_CUDA_TRY(cudaMemcpyAsync(hl.data(), lens, nslices * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
  h->sync();
  for (int64_t s = 0; s < nslices; ++s) ptr[s + 1] = ptr[s] + 32 * (int64_t)hl[s];
  return ptr;
}
}  // namespace

// DIA copy when the entries lie on at most kMaxDiag diagonals and the zero
// padding stays under 30%: candidate offsets from kDiaSamples sample rows, every entry
// placed by binary search among them (any entry off them: no DIA).
static bool try_dia(trplk_handle* h, DevCsr<double>& d, const std::string& tag, DevCsr<float>* f32) {
  const Ctx& c = h->ctx;
  const int64_t n = d.n;
  if (n < 64 || d.nnz == 0) return false;
  auto* smp = static_cast<int32_t*>(h->get(tag + ".dia_smp", kDiaSamples * (kMaxDiag + 1) * sizeof(int32_t)));
  dia_sample(c, n, d.rowptr, d.col, smp);
  std::vector<int32_t> hs(kDiaSamples * (kMaxDiag + 1));
  TRPLK_CUDA_TRY(cudaMemcpyAsync(hs.data(), smp, hs.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
  h->sync();
  std::vector<int> offs;
  for (int k = 0; k < kDiaSamples; ++k) {
    const int cnt = hs[k * (kMaxDiag + 1)];
    if (cnt < 0) return false;
    for (int e = 0; e < cnt; ++e) offs.push_back(hs[k * (kMaxDiag + 1) + 1 + e]);
  }
  std::sort(offs.begin(), offs.end());
  offs.erase(std::unique(offs.begin(), offs.end()), offs.end());
  const int nd = (int)offs.size();
  if (nd == 0 || nd > kMaxDiag) return false;
  if ((double)nd * (double)n > 1.3 * (double)d.nnz) return false;
  const int64_t ld = round_up(n, 256);
  auto* miss = static_cast<int*>(h->get(tag + ".dia_miss", sizeof(int), true));
  auto* dv = static_cast<double*>(h->get(tag + ".dia_val", (size_t)nd * ld * sizeof(double), true));
  dia_fill<double>(c, n, ld, d.rowptr, d.col, d.val, nd, offs.data(), dv, miss);
  int hm = 0;
  TRPLK_CUDA_TRY(cudaMemcpyAsync(&hm, miss, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  h->sync();
  if (hm) return false;
  d.dia_val = dv;
  d.dia_ld = ld;
  d.ndiag = nd;
  for (int k = 0; k < nd; ++k) d.dia_off[k] = offs[k];
  if (f32) {
    auto* dvf = static_cast<float*>(h->get(tag + ".dia_valf", (size_t)nd * ld * sizeof(float)));
    convert<float, double>(c, (int64_t)nd * ld, dv, dvf);
    f32->dia_val = dvf;
    f32->dia_ld = ld;
    f32->ndiag = nd;
    for (int k = 0; k < nd; ++k) f32->dia_off[k] = offs[k];
  }
  return true;
}

// SELL-32 copy of a device CSR (or the DIA copy, see try_dia).  When plain slices would pad the entries by
// more than 25% (rows of very unequal length), the hybrid form is built
// instead: rows ordered by length class (a stable counting sort: per-chunk
// class counts on the device, their prefix sums here), the longest rows
// handled by a CTA or a warp each from the CSR arrays, the rest in slices.
void attach_sell(trplk_handle* h, DevCsr<double>& d, const std::string& tag, DevCsr<float>* f32) {
  const Ctx& c = h->ctx;
  const int64_t n = d.n;
  if (try_dia(h, d, tag, f32)) return;
  std::vector<int64_t> ptr = slice_offsets(h, tag, n, d.rowptr, nullptr);
  const int64_t nslices = (n + 31) / 32;
  if ((double)ptr[nslices] <= 1.25 * (double)d.nnz + 32.0 * nslices) {
    build_sell(h, d, tag, f32, n, nullptr, ptr);
    return;
  }
  const int64_t chunks = (n + kHybChunk - 1) / kHybChunk;
  auto* hist = static_cast<int32_t*>(h->get(tag + ".hyb_hist", chunks * kHybBuckets * sizeof(int32_t)));
  auto* order = static_cast<int32_t*>(h->get(tag + ".hyb_order", n * sizeof(int32_t)));
  hyb_hist(c, n, d.rowptr, hist);
  std::vector<int32_t> hh(chunks * kHybBuckets);
  TRPLK_CUDA_TRY(cudaMemcpyAsync(hh.data(), hist, hh.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
  h->sync();
  // offsets[chunk][b] = rows of classes < b + rows of class b in earlier chunks
  std::vector<int64_t> total(kHybBuckets, 0);
  for (int64_t ch = 0; ch < chunks; ++ch)
    for (int b = 0; b < kHybBuckets; ++b) total[b] += hh[ch * kHybBuckets + b];
  std::vector<int64_t> start(kHybBuckets + 1, 0);
  for (int b = 0; b < kHybBuckets; ++b) start[b + 1] = start[b] + total[b];
  std::vector<int32_t> offs(hh.size());
  for (int b = 0; b < kHybBuckets; ++b) {
    int64_t run = start[b];
    for (int64_t ch = 0; ch < chunks; ++ch) {
      offs[ch * kHybBuckets + b] = (int32_t)run;
      run += hh[ch * kHybBuckets + b];
    }
  }
  TRPLK_CUDA_TRY(cudaMemcpyAsync(hist, offs.data(), offs.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream));
  hyb_scatter(c, n, d.rowptr, hist, order);
  h->sync();   // offs (host vector) must stay alive until its copy finished
  const int64_t n_cta = start[hyb_class_end_cta()];
  const int64_t n_long = start[hyb_class_end_warp()];
  const int64_t m = n - n_long;
  const int32_t* perm = order + n_long;
  std::vector<int64_t> hptr = slice_offsets(h, tag, m, d.rowptr, perm);
  build_sell(h, d, tag, f32, m, perm, hptr);
  d.sl_perm = perm;
  d.sl_rows = m;
  d.long_rows = order;
  d.n_long_cta = n_cta;
  d.n_long_warp = n_long - n_cta;
  if (f32) {
    f32->sl_perm = perm;
    f32->sl_rows = m;
    f32->long_rows = order;
    f32->n_long_cta = n_cta;
    f32->n_long_warp = n_long - n_cta;
  }
}


namespace {

constexpr double kEpsBreakdown64 = 1e-12;
constexpr double kEpsBreakdown32 = 1e-5;
constexpr double kEpsDependent = 1e-10;
constexpr double kBlockNear = 100.0;  // refinement block: pairs within this factor of tol

trplk_status status_from_flags(int f) {
  if (f & kFlagTimeout) return TRPLK_ETIMEOUT;
  if (f & kFlagNaN) return TRPLK_NAN;
  if (f & kFlagNotSPD) return TRPLK_NOT_SPD_B;
  return TRPLK_OK;
}

void check_flags(trplk_handle* h, int mask_ignore = kFlagBreakdown) {
  int f = h->read_status() & ~mask_ignore;
  if (f) {
    trplk_status s = status_from_flags(f);
    if (s == TRPLK_OK) s = TRPLK_ECUDA;
    std::string m = "device status flags 0x" + std::to_string(f);
    if (f & kFlagTimeout) m += " (a bounded mbarrier wait gave up)";
    if (f & kFlagDrain) m += " (a bulk copy had not landed when its CTA gave up waiting for it)";
    throw Error(s, m);
  }
}

// ---------------------------------------------------------------- device matrices
struct Operator {
  int64_t n = 0, nnz = 0;
  DevCsr<double> d;   // FP64 values (always present)
  DevCsr<float> f;    // FP32 values (mixed path only)
  double norm1 = 0.0;
};

// Row pointers (thread per row) and column indices (thread per entry, so
// every read is coalesced and no long row holds up a thread).
__global__ void validate_csr_kernel(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                                    int* status) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  bool bad = false;
  for (int64_t i = t0; i < n; i += stride) {
    const int64_t a = rowptr[i], b = rowptr[i + 1];
    bad |= a > b || a < 0 || b > nnz;
  }
  for (int64_t e = t0; e < nnz; e += stride) bad |= col[e] < 0 || col[e] >= n;
  if (bad) atomicOr(status, 64);
}

template <typename S>
__global__ void row_abs_sum_kernel(int64_t n, const int64_t* rowptr, const S* val, double* out) {
  // out[blockIdx.x] = max over the block's rows of sum_j |a_ij|; one warp per
  // row, lanes striding it
  __shared__ double s_m[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  double m = 0.0;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    double s = 0.0;
    for (int64_t e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) s += fabs((double)val[e]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    m = s > m ? s : m;
  }
  if (lane == 0) s_m[warp] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, s_m[w]);
    out[blockIdx.x] = t;
  }
}

__global__ void set_diag_block_kernel(double* T, int ldT, int k, const double* theta) {
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int j = e / k, i = e - j * k;
    T[(int64_t)j * ldT + i] = (i == j) ? theta[i] : 0.0;
  }
}

// Upload or wrap a caller's CSR; `tag` names the workspace slots.
Operator make_operator(trplk_handle* h, const trplk_csr* M, const std::string& tag, bool need_f32) {
  Operator op;
  if (!M) return op;
  if (M->n <= 0 || M->nnz < 0 || !M->rowptr || !M->col || !M->val)
    throw Error(TRPLK_EINVAL, tag + ": empty or null CSR");
  if (M->dtype != TRPLK_F64) throw Error(TRPLK_EINVAL, tag + ": solver matrices must have F64 values");
  op.n = M->n;
  op.nnz = M->nnz;
  const Ctx& c = h->ctx;
  if (M->on_device) {
    op.d.rowptr = M->rowptr;
    op.d.col = M->col;
    op.d.val = static_cast<const double*>(M->val);
  } else {
    // host arrays: validate cheaply on the host, then copy
    if (M->rowptr[0] != 0 || M->rowptr[M->n] != M->nnz) throw Error(TRPLK_EINVAL, tag + ": bad row pointers");
    auto* rp = static_cast<int64_t*>(h->get(tag + ".rowptr", (M->n + 1) * sizeof(int64_t)));
    auto* cl = static_cast<int32_t*>(h->get(tag + ".col", M->nnz * sizeof(int32_t)));
    auto* vl = static_cast<double*>(h->get(tag + ".val", M->nnz * sizeof(double)));
    TRPLK_CUDA_TRY(cudaMemcpyAsync(rp, M->rowptr, (M->n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c.stream));
    TRPLK_CUDA_TRY(cudaMemcpyAsync(cl, M->col, M->nnz * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream));
    TRPLK_CUDA_TRY(cudaMemcpyAsync(vl, M->val, M->nnz * sizeof(double), cudaMemcpyHostToDevice, c.stream));
    op.d.rowptr = rp;
    op.d.col = cl;
    op.d.val = vl;
  }
  op.d.n = op.n;
  op.d.nnz = op.nnz;
  // structural validation on the device (column range, monotone rows)
  h->clear_status();
  ProfScope ps1(c, PK_OTHER, 0.0);
  validate_csr_kernel<<<std::max(1, std::min<int>((int)((op.nnz + 255) / 256), c.sms * 8)), 256, 0, c.stream>>>(
      op.n, op.nnz, op.d.rowptr, op.d.col, c.status);
  check_launch("validate_csr");
  // no kernel reads the rows before their pointers are known to be in range
  if (h->read_status() & 64) throw Error(TRPLK_EINVAL, tag + ": row pointers or column indices out of range");
  const int nb = std::max(1, std::min<int>((int)((op.n + 255) / 256), 1024));
  auto* part = static_cast<double*>(h->get("norm1.part", 1024 * sizeof(double)));
  ProfScope ps2(c, PK_OTHER, 0.0);
  row_abs_sum_kernel<double><<<nb, 256, 0, c.stream>>>(op.n, op.d.rowptr, op.d.val, part);
  check_launch("row_abs_sum");
  double* hp = h->host(1024);
  TRPLK_CUDA_TRY(cudaMemcpyAsync(hp, part, nb * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  h->sync();
  op.norm1 = 0.0;
  for (int i = 0; i < nb; ++i) op.norm1 = std::max(op.norm1, hp[i]);
  if (need_f32) {
    auto* vf = static_cast<float*>(h->get(tag + ".valf", op.nnz * sizeof(float)));
    convert<float, double>(c, op.nnz, op.d.val, vf);
    op.f = DevCsr<float>{op.n, op.nnz, op.d.rowptr, op.d.col, vf};
  }
  attach_sell(h, op.d, tag, need_f32 ? &op.f : nullptr);
  return op;
}

template <typename S> const DevCsr<S>& pick(const Operator& o);
template <> const DevCsr<double>& pick<double>(const Operator& o) { return o.d; }
template <> const DevCsr<float>& pick<float>(const Operator& o) { return o.f; }

// ---------------------------------------------------------------- the solver
struct SolveOut {
  int cycles = 0;
  int64_t mvA = 0, mvB = 0, prec = 0;
  bool converged = false;
  bool breakdown = false;
  std::vector<double> theta;   // k Ritz values at exit (locked ones first under hard locking)
  int cur = 0;                 // basis buffer holding X at exit
  int locked = 0;              // pairs locked (hard locking)
};

template <typename S>
struct Solver {
  trplk_handle* h;
  const Ctx& c;
  int64_t n, ld;
  int p, q, k, l;
  double tol;
  int max_cycles;
  bool hasB;
  bool skip_converged;          // refinement phase: targets skip converged pairs
  bool check_start = false;     // replace dependent start columns (refinement phase)
  bool block_refine = false;    // refinement phase: cycles start from all unconverged residuals
  int stall_window = 0;         // >0: stop when the target residual stagnates
  bool stalled = false;
  // Hard locking: columns [0, nq) of every basis buffer hold the locked Ritz
  // vectors; T, the Rayleigh-Ritz step and the restart act on the active
  // columns [nq, ...) while every orthogonalisation also covers the locked
  // ones.  The active Ritz values sit at theta + toff until the next RR.
  int blk = 1;                  // block TRPL+K: targets per cycle (1: Algorithm 1)
  bool hard_lock = false;
  int nq = 0, toff = 0;
  std::vector<double> lam_q;    // locked Ritz values
  double* theta_out = nullptr;  // [p] final Ritz values in basis-column order
  // Per-cycle shifted Jacobi M_i = diag(A - rho_i B)^-1: FP64 diagonals of
  // A and B (B null: identity); the solver rewrites dinv at every cycle
  const double* diagA = nullptr;
  const double* diagB = nullptr;
  S* dinv_var = nullptr;
  double* tmp64 = nullptr;
  const Operator& Aop;
  const Operator& Bop;
  const DevCsr<S>& A;
  const DevCsr<S>* B;
  const S* dinv;
  int pmode;
  const DevCsr<S>* MG = nullptr;    // FSAI factor G (M = G^T G) when set; IC(0) factor L when ic0_dinv is set
  const DevCsr<S>* MGT = nullptr;
  const S* ic0_dinv = nullptr;      // IC(0): 1 / diag(L); M = P_s^T P_s by Jacobi sweeps
  S* itmp[2] = {nullptr, nullptr};
  S* rtmp = nullptr;
  S* ttmp = nullptr;
  double normA;
  double eps_breakdown;
  // workspace
  S* U[2];
  S* AU[2];
  S* BU[2];
  S *v, *bv;
  double *T, *theta, *Y, *h1, *h2, *betas, *scale, *rn, *xn;
  int ldT;

  Solver(trplk_handle* h_, const std::string& tag, int64_t n_, int p_, int q_, int k_, int l_, double tol_,
         int maxc, const Operator& A_, const Operator& B_, bool hasB_, const S* dinv_, int pmode_)
      : h(h_), c(h_->ctx), n(n_), p(p_), q(q_), k(k_), l(l_), tol(tol_), max_cycles(maxc), hasB(hasB_),
        skip_converged(false), Aop(A_), Bop(B_), A(pick<S>(A_)), B(hasB_ ? &pick<S>(B_) : nullptr),
        dinv(dinv_), pmode(pmode_) {
    ld = round_up(n, 256);
    normA = Aop.norm1;
    eps_breakdown = sizeof(S) == 8 ? kEpsBreakdown64 : kEpsBreakdown32;
    // Rows n..ld-1 of every n-vector must be zero.  Buffers are zeroed when
    // first allocated and whenever the problem layout changes.
    const std::string key = std::to_string(n) + "/" + std::to_string(q) + "/" + std::to_string(hasB);
    const bool fresh = h->layouts[tag] != key;
    h->layouts[tag] = key;
    const size_t basis = (size_t)ld * q * sizeof(S);
    for (int b = 0; b < 2; ++b) {
      U[b] = static_cast<S*>(h->get(tag + ".U" + std::to_string(b), basis, fresh));
      AU[b] = static_cast<S*>(h->get(tag + ".AU" + std::to_string(b), basis, fresh));
      BU[b] = hasB ? static_cast<S*>(h->get(tag + ".BU" + std::to_string(b), basis, fresh)) : U[b];
    }
    v = static_cast<S*>(h->get(tag + ".v", ld * sizeof(S), fresh));
    bv = hasB ? static_cast<S*>(h->get(tag + ".bv", ld * sizeof(S), fresh)) : v;
    ldT = q;
    T = static_cast<double*>(h->get(tag + ".T", (size_t)q * q * sizeof(double)));
    theta = static_cast<double*>(h->get(tag + ".theta", kMaxQ * sizeof(double)));
    Y = static_cast<double*>(h->get(tag + ".Y", (size_t)kMaxQ * kMaxQ * sizeof(double)));
    h1 = static_cast<double*>(h->get(tag + ".h1", kMaxQ * sizeof(double)));
    h2 = static_cast<double*>(h->get(tag + ".h2", kMaxQ * sizeof(double)));
    betas = static_cast<double*>(h->get(tag + ".betas", 2 * (kMaxQ + 8) * sizeof(double)));
    scale = static_cast<double*>(h->get(tag + ".scale", 8 * sizeof(double)));
    rn = static_cast<double*>(h->get(tag + ".rn", kMaxQ * sizeof(double)));
    tmp64 = static_cast<double*>(h->get(tag + ".tmp64", ld * sizeof(double), fresh));
    rtmp = static_cast<S*>(h->get(tag + ".rtmp", ld * sizeof(S), fresh));
    ttmp = static_cast<S*>(h->get(tag + ".ttmp", ld * sizeof(S), fresh));
    xn = static_cast<double*>(h->get(tag + ".xn", kMaxQ * sizeof(double)));
    theta_out = static_cast<double*>(h->get(tag + ".theta_out", kMaxQ * sizeof(double)));
  }

  S* col(S* M, int j) { return M + (size_t)j * ld; }

  // out = M in: G^T (G in) (FSAI, two sparse matvecs) or P_s^T (P_s in)
  // (IC(0), Jacobi sweeps with L and L^T)
  void apply_fsai(const S* in, S* out) {
    if (ic0_dinv) {
      for (int i = 0; i < 2; ++i)
        if (!itmp[i])
          itmp[i] = static_cast<S*>(h->get(std::string(sizeof(S) == 8 ? "f64" : "f32") + ".itmp" + std::to_string(i),
                                           ld * sizeof(S), true));
      ic0_apply<S>(c, ld, *MG, *MGT, ic0_dinv, kIc0Sweeps, in, out, ttmp, itmp[0], itmp[1]);
      return;
    }
    spmv<S>(c, *MG, in, ttmp);
    spmv<S>(c, *MGT, ttmp, out);
  }

  // v <- CGS2(v) against the w columns of (U, BU) given h1 = BU^T v; leaves
  // v unnormalised, bv = B v, betas[slot] = (beta, beta0), *scale = 1/beta.
  void orthonormalize_tail(int cur, int w, int slot, SolveOut& out) {
    ts_update_project<S>(c, ld, w, U[cur], BU[cur], h1, v, h2);
    if (hasB) {
      ts_update<S>(c, ld, w, U[cur], h2, v);
      spmv<S>(c, *B, v, bv);
      out.mvB++;
      ts_dot_norm<S>(c, ld, v, bv, h1, h2, w, betas + 2 * slot, scale, eps_breakdown);
    } else {
      ts_update_norm<S>(c, ld, w, U[cur], h2, h1, v, betas + 2 * slot, scale, eps_breakdown);
    }
  }

  // v = M (A x_i - theta_i B x_i) from the stored images (Algorithm 1,
  // restart); i counts active pairs (column nq + i, Ritz value theta[toff + i])
  void precond_residual(int cur, int i) {
    const int c0 = nq + i;
    if (MG) {
      restart_vector<S>(c, ld, col(AU[cur], c0), col(BU[cur], c0), theta + toff + i, nullptr, PM_IDENTITY, rtmp);
      apply_fsai(rtmp, v);
    } else {
      restart_vector<S>(c, ld, col(AU[cur], c0), col(BU[cur], c0), theta + toff + i, dinv, pmode, v);
    }
  }

  // normalise v into column w of (U, BU) and form column w of AU (one A matvec)
  void append(int cur, int w, SolveOut& out) {
    spmv_scaled<S>(c, A, v, scale, col(AU[cur], w), col(U[cur], w), hasB ? bv : nullptr,
                   hasB ? col(BU[cur], w) : nullptr);
    out.mvA++;
  }

  void read_back(int count, std::vector<double>& th, std::vector<double>& r, std::vector<double>& x,
                 std::vector<double>* bet, int nbet) {
    double* hp = h->host(4 * kMaxQ + 2 * (kMaxQ + 8));
    TRPLK_CUDA_TRY(cudaMemcpyAsync(hp, theta, count * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    TRPLK_CUDA_TRY(cudaMemcpyAsync(hp + kMaxQ, rn, count * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    TRPLK_CUDA_TRY(cudaMemcpyAsync(hp + 2 * kMaxQ, xn, count * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    if (bet && nbet > 0)
      TRPLK_CUDA_TRY(cudaMemcpyAsync(hp + 4 * kMaxQ, betas, 2 * nbet * sizeof(double), cudaMemcpyDeviceToHost,
                                     c.stream));
    h->sync();
    th.assign(hp, hp + count);
    r.assign(hp + kMaxQ, hp + kMaxQ + count);
    x.assign(hp + 2 * kMaxQ, hp + 2 * kMaxQ + count);
    if (bet) bet->assign(hp + 4 * kMaxQ, hp + 4 * kMaxQ + 2 * nbet);
  }

  // Rayleigh-Ritz on T[0:w,0:w], rotate (U, AU, BU)[cur] into the other
  // buffer, residual norms of the k new Ritz vectors.  Returns the new cur.
  // Under hard locking all of this acts on the active columns [nq, w).
  int rr_and_restart(int cur, int w) {
    const int wa = w - nq, ka = k - nq;
    const size_t o = (size_t)nq * ld;
    rayleigh_ritz(c, wa, T + (size_t)nq * ldT + nq, ldT, theta, Y, sizeof(S) == 4);
    toff = 0;
    const int nx = 1 - cur;
    // The tensor-core rotation (FP32 data, B = I): on the Q1 pencil the FP32
    // phase with it left the FP64 refinement 37 cycles instead of 21
    // (n = 884,736, w = 50, k = 25), so pencils keep the CUDA-core rotation.
    ts_rotate<S>(c, ld, wa, ka, U[cur] + o, Y, wa, U[nx] + o, !hasB);
    ts_rotate<S>(c, ld, wa, ka, AU[cur] + o, Y, wa, AU[nx] + o, !hasB);
    if (hasB) ts_rotate<S>(c, ld, wa, ka, BU[cur] + o, Y, wa, BU[nx] + o, false);
    ts_resid<S>(c, ld, ka, U[nx] + o, AU[nx] + o, hasB ? BU[nx] + o : nullptr, theta, rn, xn);
    return nx;
  }

  // Lock the first s active pairs of buffer `cur` (hard locking): they stay
  // where they are, a copy goes to the same columns of the other buffer (the
  // next restart writes only the active columns), their values are kept.
  void lock(int cur, int s, std::vector<double>& th) {
    const int other = 1 - cur;
    const size_t bytes = (size_t)s * ld * sizeof(S);
    TRPLK_CUDA_TRY(cudaMemcpyAsync(col(U[other], nq), col(U[cur], nq), bytes, cudaMemcpyDeviceToDevice, c.stream));
    TRPLK_CUDA_TRY(cudaMemcpyAsync(col(AU[other], nq), col(AU[cur], nq), bytes, cudaMemcpyDeviceToDevice, c.stream));
    if (hasB)
      TRPLK_CUDA_TRY(cudaMemcpyAsync(col(BU[other], nq), col(BU[cur], nq), bytes, cudaMemcpyDeviceToDevice, c.stream));
    for (int i = 0; i < s; ++i) lam_q.push_back(th[i]);
    th.erase(th.begin(), th.begin() + s);
    nq += s;
    toff += s;
  }

  // theta_out[0:p] = the p returned Ritz values in the order of the basis
  // columns 0..p-1 (locked values first under hard locking)
  void finish_theta(int pp) {
    if (nq > 0)
      TRPLK_CUDA_TRY(cudaMemcpyAsync(theta_out, lam_q.data(), std::min(nq, pp) * sizeof(double),
                                     cudaMemcpyHostToDevice, c.stream));
    if (pp > nq)
      TRPLK_CUDA_TRY(cudaMemcpyAsync(theta_out + nq, theta + toff, (pp - nq) * sizeof(double),
                                     cudaMemcpyDeviceToDevice, c.stream));
    h->sync();   // lam_q (host) must stay alive until its copy finished
  }

  // Algorithm 1.  X0: double n x k (ld) on the device.  On return
  // theta_out[0:p] holds the Ritz values of basis columns 0..p-1 of U[cur].
  SolveOut run(const double* X0) {
    SolveOut out = run_cycles(X0);
    out.locked = nq;
    finish_theta(p);
    return out;
  }

  SolveOut run_cycles(const double* X0) {
    SolveOut out;
    int cur = 0;
    h->clear_status();
    // start block into U[0][:, :k] (as S)
    if (sizeof(S) == 8) {
      TRPLK_CUDA_TRY(cudaMemcpyAsync(U[0], X0, (size_t)ld * k * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    } else {
      convert<S, double>(c, (int64_t)ld * k, X0, U[0]);
    }
    // B-orthonormalise column by column (CGS2) and form A X (Algorithm 1 input).
    // A column that is (numerically) in the span of the previous ones is
    // replaced by a fresh SplitMix64 column once; the replacement matters when
    // the start block comes from a lower-precision phase.
    for (int j = 0; j < k; ++j) {
      for (int attempt = 0; attempt < 2; ++attempt) {
        TRPLK_CUDA_TRY(cudaMemcpyAsync(v, col(U[0], j), ld * sizeof(S), cudaMemcpyDeviceToDevice, c.stream));
        ts_project<S>(c, ld, j, BU[0], v, h1);
        orthonormalize_tail(0, j, j, out);
        if (!check_start) break;
        double* hb = h->host(2);
        TRPLK_CUDA_TRY(cudaMemcpyAsync(hb, betas + 2 * j, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
        h->sync();
        if (hb[0] > eps_breakdown * hb[1]) break;
        if (attempt == 1) throw Error(TRPLK_EINVAL, "start block is numerically rank deficient");
        start_block(c, n, ld, 1, 0x5DEECE66Dull ^ (uint64_t)(j + 1) * 0x9E3779B97F4A7C15ull, tmp64);
        convert<S, double>(c, ld, tmp64, col(U[0], j));
      }
      append(0, j, out);
    }
    // T = X^T A X (upper triangle), initial RR
    for (int j = 0; j < k; ++j) ts_project<S>(c, ld, j + 1, U[0], col(AU[0], j), T + (size_t)j * ldT);
    cur = rr_and_restart(0, k);
    std::vector<double> th, r, x, bet;
    read_back(k, th, r, x, &bet, k);
    check_flags(h, kFlagBreakdown);
    if (!check_start)
      for (int j = 0; j < k; ++j)
        if (!(bet[2 * j] > eps_breakdown * bet[2 * j + 1]))
          throw Error(TRPLK_EINVAL, "start block is numerically rank deficient");

    auto converged_vec = [&](const std::vector<double>& rr, const std::vector<double>& xx) {
      std::vector<char> cv(rr.size());
      for (size_t i = 0; i < rr.size(); ++i) cv[i] = rr[i] <= tol * normA * xx[i];
      return cv;
    };
    int t = 0;
    std::vector<char> cvec = converged_vec(r, x);
    if (skip_converged) {
      const auto& cv = cvec;
      while (t < p && cv[t]) ++t;
      if (t >= p) {
        out.converged = true;
        out.theta = th;
        out.cur = cur;
        return out;
      }
    }
    // X_prev: columns [xp_start, xp_start + xp_count) of U[xp_buf]
    int xp_buf = -1, xp_start = 0, xp_count = 0;
    std::vector<double> hist;   // stagnation detection
    int hist_t = -1;

    for (int cycle = 1; cycle <= max_cycles; ++cycle) {
      out.cycles = cycle;
      const double rho = th[t];
      h->clear_status();
      {
        ProfScope ps(c, PK_OTHER, 0.0);
        set_diag_block_kernel<<<1, 256, 0, c.stream>>>(T + (size_t)nq * ldT + nq, ldT, k - nq, theta + toff);
      }
      check_launch("set_diag_block");
      // per-cycle preconditioner M_i = diag(A - rho_i B)^-1 (Sec. 3)
      if (dinv_var) shifted_jacobi<S>(c, n, ld, diagA, diagB, theta + toff + t, dinv_var);
      const int nprev = (xp_buf >= 0) ? xp_count : 0;
      // refinement: first the preconditioned residuals of the other
      // unconverged pairs already near tol (relative residual <= kBlockNear
      // tol), each B-orthonormalised against the basis (a block Davidson step
      // for all of them), dropped when dependent; pairs further away wait for
      // their turn as the target, whose Krylov steps converge them faster
      int w0 = k;
      if (block_refine) {
        std::vector<int> blk;
        for (int i = 0; i < p; ++i)
          if (i != t && !cvec[i] && r[i] <= kBlockNear * tol * normA * x[i]) blk.push_back(i);
        const int room = std::max(0, q - k - nprev - 1);
        if ((int)blk.size() > room) blk.resize(room);
        for (int i : blk) {
          precond_residual(cur, i);
          out.prec++;
          ts_project<S>(c, ld, w0, BU[cur], v, h1);
          orthonormalize_tail(cur, w0, kMaxQ, out);
          double* hp = h->host(2);
          TRPLK_CUDA_TRY(cudaMemcpyAsync(hp, betas + 2 * kMaxQ, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
          h->sync();
          if (!(hp[0] > eps_breakdown * hp[1])) continue;
          append(cur, w0, out);
          ++w0;
          ts_project<S>(c, ld, w0, U[cur], col(AU[cur], w0 - 1), T + (size_t)(w0 - 1) * ldT);
        }
      }
      // the cycle's targets t .. t+b-1 (capped at p_hat - 1) and their shifts
      // (block TRPL+K; b = 1 is Algorithm 1)
      int tg[kMaxK];
      double rhos[kMaxK];
      for (int i = 0; i < blk; ++i) {
        tg[i] = std::min(t + i, k - nq - 1);
        rhos[i] = th[tg[i]];
      }
      // first Lanczos vector u = M (A x_t - rho B x_t)  (Algorithm 1, restart)
      precond_residual(cur, tg[0]);
      out.prec++;
      ts_project<S>(c, ld, w0, BU[cur], v, h1);
      orthonormalize_tail(cur, w0, 0, out);
      const int m = q - w0 - nprev;
      int w = w0;
      // inner preconditioned Lanczos with the T update (eq. (UpdateT)); with
      // b > 1 the first b vectors are the targets' preconditioned residuals
      // and column a >= b is formed from column a - b with the shift of its
      // sequence a mod b
      for (int j = 0; j < m; ++j) {
        append(cur, w, out);
        ++w;
        if (j < m - 1) {
          const int a1 = j + 1;   // the next column of the cycle
          double* tcol = T + (size_t)(w - 1) * ldT;
          if (a1 < blk) {   // restart vector of the next target; the pass forms column w-1's T entries
            precond_residual(cur, tg[a1]);
            ts_inner<S>(c, ld, w, U[cur], BU[cur], col(AU[cur], w - 1), col(BU[cur], w - 1), nullptr, PM_GIVEN, 0.0,
                        v, tcol, h1);
          } else {
            const int src = w0 + a1 - blk;   // == w - 1 when b = 1
            const double shift = rhos[a1 % blk];
            if (MG) {   // M = G^T G (or IC(0)), then the fused pass with the preconditioned vector given
              axpby_shift<S>(c, ld, col(AU[cur], src), col(BU[cur], src), shift, rtmp);
              apply_fsai(rtmp, v);
              ts_inner<S>(c, ld, w, U[cur], BU[cur], col(AU[cur], w - 1), col(BU[cur], w - 1), nullptr, PM_GIVEN,
                          shift, v, tcol, h1);
            } else if (src == w - 1) {
              ts_inner<S>(c, ld, w, U[cur], BU[cur], col(AU[cur], w - 1), col(BU[cur], w - 1), dinv, pmode, shift, v,
                          tcol, h1);
            } else {
              ts_inner<S>(c, ld, w, U[cur], BU[cur], col(AU[cur], w - 1), col(BU[cur], w - 1), dinv, pmode, shift, v,
                          tcol, h1, col(AU[cur], src), col(BU[cur], src));
            }
          }
          out.prec++;
          orthonormalize_tail(cur, w, j + 1, out);
        } else {
          ts_project<S>(c, ld, w, U[cur], col(AU[cur], w - 1), T + (size_t)(w - 1) * ldT);
        }
      }
      // breakdown: find the first Lanczos norm that collapsed (slots 0..m-1)
      {
        double* hp = h->host(2 * (kMaxQ + 8));
        TRPLK_CUDA_TRY(cudaMemcpyAsync(hp, betas, 2 * m * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
        h->sync();
        int good = m;
        for (int j = 0; j < m; ++j)
          if (!(hp[2 * j] > eps_breakdown * hp[2 * j + 1])) { good = j; break; }
        if (good < m) {
          out.breakdown = true;
          w = w0 + good;
          if (good == 0 && nprev == 0 && w0 == k) {
            out.theta = th;
            out.cur = cur;
            return out;
          }
        }
      }
      // +K: orthogonalise X_prev against [X, G] and complete T (Algorithm 1)
      for (int i = 0; i < nprev; ++i) {
        TRPLK_CUDA_TRY(cudaMemcpyAsync(v, col(U[xp_buf], xp_start + i), ld * sizeof(S), cudaMemcpyDeviceToDevice,
                                       c.stream));
        ts_project<S>(c, ld, w, BU[cur], v, h1);
        orthonormalize_tail(cur, w, kMaxQ, out);
        double* hp = h->host(2);
        TRPLK_CUDA_TRY(cudaMemcpyAsync(hp, betas + 2 * kMaxQ, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
        h->sync();
        if (!(hp[0] > kEpsDependent)) continue;   // X_prev columns have unit B-norm
        append(cur, w, out);
        ++w;
        ts_project<S>(c, ld, w, U[cur], col(AU[cur], w - 1), T + (size_t)(w - 1) * ldT);
      }
      // X_prev for the next cycle: x_t .. x_min(t+l-1, p) of this cycle's X
      // (active pairs; their columns start at nq)
      const int nxt_start = nq + t, nxt_count = std::max(0, std::min(t + l, p - nq) - t);
      const int old = cur;
      cur = rr_and_restart(cur, w);
      read_back(k - nq, th, r, x, nullptr, 0);
      check_flags(h, kFlagBreakdown);
      cvec = converged_vec(r, x);
      const auto& cv = cvec;
      if (stall_window > 0) {
        // the target's relative residual, tracked while the target is unchanged
        const double rel = r[t] / (normA * x[t]);
        if (hist_t != t) {
          hist.clear();
          hist_t = t;
        }
        hist.push_back(rel);
        // not halved over stall_window cycles below 1e-6 (where FP32 rounding
        // can hold a residual up), or over 4 stall_window cycles at any level
        // (a guard: the FP64 continuation then takes over)
        auto flat = [&](int win) { return (int)hist.size() > win && rel > 0.5 * hist[hist.size() - 1 - win]; };
        if (!cv[t] && ((rel < 1e-6 && flat(stall_window)) || flat(4 * stall_window))) {
          stalled = true;
          out.theta = th;
          out.cur = cur;
          return out;
        }
      }
      xp_buf = old;
      xp_start = nxt_start;
      xp_count = nxt_count;
      if (hard_lock) {
        // lock the leading run of converged active pairs; drop as many X_prev
        // columns (their copies of the locked vectors); the target stays the
        // smallest active pair
        int sl = 0;
        while (sl < p - nq && cv[sl]) ++sl;
        if (sl > 0) {
          const int drop = std::min(sl, xp_count);
          xp_start += drop;
          xp_count -= drop;
          lock(cur, sl, th);
          r.erase(r.begin(), r.begin() + sl);
          x.erase(x.begin(), x.begin() + sl);
          cvec.erase(cvec.begin(), cvec.begin() + sl);
        }
        if (nq >= p) {
          out.converged = true;
          break;
        }
        continue;
      }
      if (cv[t]) {   // Algorithm 1: flag, drop x_1^prev, advance the target
        ++t;
        if (xp_count > 0) { ++xp_start; --xp_count; }
        if (skip_converged) while (t < p && cv[t]) ++t;
      }
      if (t >= p) {
        int fail = -1;
        for (int i = 0; i < p; ++i)
          if (!cv[i]) { fail = i; break; }
        if (fail < 0) {
          out.converged = true;
          break;
        }
        t = fail;
      }
    }
    out.theta = th;
    out.cur = cur;
    return out;
  }
};

// Final FP64 check with fresh matvecs: resid[i] = ||A x - theta B x|| / (||A||_1 ||x||).
void check_residuals_fp64(trplk_handle* h, const Operator& Aop, const Operator* Bop, int64_t ld, int p,
                          const double* X, const double* theta_dev, double normA, double* resid_host) {
  const Ctx& c = h->ctx;
  double* ax = static_cast<double*>(h->get("check.ax", ld * sizeof(double), true));
  double* bx = static_cast<double*>(h->get("check.bx", ld * sizeof(double), true));
  double* rn = static_cast<double*>(h->get("check.rn", kMaxQ * sizeof(double)));
  double* xn = static_cast<double*>(h->get("check.xn", kMaxQ * sizeof(double)));
  for (int i = 0; i < p; ++i) {
    const double* xi = X + (size_t)i * ld;
    spmv<double>(c, Aop.d, xi, ax);
    if (Bop) spmv<double>(c, Bop->d, xi, bx);
    ts_resid<double>(c, ld, 1, xi, ax, Bop ? bx : nullptr, theta_dev + i, rn + i, xn + i);
  }
  double* hp = h->host(2 * kMaxQ);
  TRPLK_CUDA_TRY(cudaMemcpyAsync(hp, rn, p * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  TRPLK_CUDA_TRY(cudaMemcpyAsync(hp + kMaxQ, xn, p * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  h->sync();
  for (int i = 0; i < p; ++i) resid_host[i] = hp[i] / (normA * hp[kMaxQ + i]);
}

void validate_params(const trplk_params* P, int64_t n) {
  if (!P) throw Error(TRPLK_EINVAL, "params is NULL");
  if (P->which != TRPLK_SMALLEST) throw Error(TRPLK_EINVAL, "only which = TRPLK_SMALLEST is supported");
  if (P->p < 1 || P->k < P->p) throw Error(TRPLK_EINVAL, "need 1 <= p <= k");
  if (P->k > kMaxK) throw Error(TRPLK_EINVAL, "k (thick-restart size) must be <= 32");
  if (P->l < 0) throw Error(TRPLK_EINVAL, "l must be >= 0");
  if (P->q < P->k + std::max(P->l, 1) + 1) throw Error(TRPLK_EINVAL, "need q >= k + max(l,1) + 1");
  if (P->q > kMaxQ) throw Error(TRPLK_EINVAL, "q must be <= 64");
  if (P->q > n) throw Error(TRPLK_EINVAL, "q must be <= n");
  if (!(P->tol > 0.0)) throw Error(TRPLK_EINVAL, "tol must be > 0");
  if (P->max_cycles < 1) throw Error(TRPLK_EINVAL, "max_cycles must be >= 1");
  if (P->precond < TRPLK_PRECOND_NONE || P->precond > TRPLK_PRECOND_IC0)
    throw Error(TRPLK_EINVAL, "unsupported preconditioner");
  if (P->locking != TRPLK_LOCKING_SOFT && P->locking != TRPLK_LOCKING_HARD)
    throw Error(TRPLK_EINVAL, "unknown locking mode");
  const int blk = P->block < 1 ? 1 : P->block;
  if (blk > P->k || P->k + blk + P->l > P->q) throw Error(TRPLK_EINVAL, "need block <= k and k + block + l <= q");
  if (blk > 1 && P->locking == TRPLK_LOCKING_HARD) throw Error(TRPLK_EINVAL, "block TRPL+K runs with soft locking");
  if (P->precond == TRPLK_PRECOND_FSAI_LEARNED && !P->mlp_weights)
    throw Error(TRPLK_EINVAL, "learned FSAI needs mlp_weights");
  if (P->precision != TRPLK_PRECISION_FP64 && P->precision != TRPLK_PRECISION_MIXED)
    throw Error(TRPLK_EINVAL, "unknown precision");
}

DevCsr<double> dev_csr64(const trplk_csr* M) {
  if (!M || !M->on_device) throw Error(TRPLK_EINVAL, "step-level calls take device CSR matrices");
  if (M->dtype != TRPLK_F64) throw Error(TRPLK_EINVAL, "expected F64 values");
  return DevCsr<double>{M->n, M->nnz, M->rowptr, M->col, static_cast<const double*>(M->val)};
}

void check_ld(int64_t n, int64_t ld) {
  if (n < 1 || ld < n || ld % 256 != 0) throw Error(TRPLK_EINVAL, "need n >= 1, ld >= n, ld % 256 == 0");
}

}  // namespace

// ================================================================ C ABI
extern "C" {

int trplk_abi_version(void) { return TRPLK_ABI_VERSION; }

trplk_status trplk_create(trplk_handle** out, int device, void* stream) {
  if (!out) return TRPLK_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return TRPLK_EINVAL;
  }
  auto* h = new trplk_handle();
  try {
    h->ctx.device = device;
    h->ctx.prof = &h->prof;
    TRPLK_CUDA_TRY(cudaSetDevice(device));
    TRPLK_CUDA_TRY(cudaDeviceGetAttribute(&h->ctx.sms, cudaDevAttrMultiProcessorCount, device));
    if (stream) {
      h->ctx.stream = static_cast<cudaStream_t>(stream);
    } else {
      TRPLK_CUDA_TRY(cudaStreamCreateWithFlags(&h->ctx.stream, cudaStreamNonBlocking));
      h->own_stream = true;
    }
    h->ctx.partials = static_cast<double*>(h->get("ctx.partials", (size_t)kMaxPartials * kPartialStride * sizeof(double)));
    h->ctx.counter = static_cast<unsigned int*>(h->get("ctx.counter", 64));
    h->ctx.status = static_cast<int*>(h->get("ctx.status", 64));
    h->sync();
  } catch (const Error& e) {
    trplk_destroy(h);
    return e.code;
  }
  *out = h;
  return TRPLK_OK;
}

trplk_status trplk_destroy(trplk_handle* h) {
  if (!h) return TRPLK_OK;
  cudaSetDevice(h->ctx.device);
  if (h->ctx.stream) cudaStreamSynchronize(h->ctx.stream);
  for (auto& kv : h->bufs)
    if (kv.second.p) cudaFree(kv.second.p);
  if (h->pinned) cudaFreeHost(h->pinned);
  if (h->own_stream && h->ctx.stream) cudaStreamDestroy(h->ctx.stream);
  delete h;
  return TRPLK_OK;
}

const char* trplk_last_error(const trplk_handle* h) { return h ? h->err.c_str() : "null handle"; }

trplk_status trplk_solve(trplk_handle* h, const trplk_csr* A, const trplk_csr* B, const trplk_params* P,
                         const double* X0, double* evals, double* evecs, double* resid, trplk_info* info) {
  return guarded(h, [&]() -> trplk_status {
    auto t0 = std::chrono::steady_clock::now();
    const int64_t launches0 = h->prof.launches;
    if (!A) throw Error(TRPLK_EINVAL, "A is NULL");
    if (!evals || !evecs || !resid) throw Error(TRPLK_EINVAL, "output pointer is NULL");
    validate_params(P, A->n);
    if (B && (B->n != A->n || B->on_device != A->on_device)) throw Error(TRPLK_EINVAL, "A and B differ in n or location");
    const bool mixed = P->precision == TRPLK_PRECISION_MIXED;
    const Ctx& c = h->ctx;
    Operator Aop = make_operator(h, A, "A", mixed);
    Operator Bop = make_operator(h, B, "B", mixed);
    const bool hasB = B != nullptr;
    const int64_t n = A->n, ld = round_up(n, 256);
    // preconditioner
    const bool shifted = P->precond == TRPLK_PRECOND_JACOBI_SHIFTED;
    const int pmode = (P->precond == TRPLK_PRECOND_JACOBI || shifted) ? PM_JACOBI : PM_IDENTITY;
    double* dinv64 = nullptr;
    float* dinv32 = nullptr;
    double* diagA = nullptr;
    double* diagB = nullptr;
    if (shifted) {   // M_i rebuilt by every cycle from the diagonals of A and B
      dinv64 = static_cast<double*>(h->get("dinv64", ld * sizeof(double), true));
      diagA = static_cast<double*>(h->get("diagA", ld * sizeof(double), true));
      diag_of(c, n, Aop.d.rowptr, Aop.d.col, Aop.d.val, diagA);
      if (hasB) {
        diagB = static_cast<double*>(h->get("diagB", ld * sizeof(double), true));
        diag_of(c, n, Bop.d.rowptr, Bop.d.col, Bop.d.val, diagB);
      }
      if (mixed) dinv32 = static_cast<float*>(h->get("dinv32", ld * sizeof(float), true));
    } else if (pmode == PM_JACOBI) {
      dinv64 = static_cast<double*>(h->get("dinv64", ld * sizeof(double), true));
      jacobi_dinv<double>(c, Aop.d, dinv64);
      if (mixed) {
        dinv32 = static_cast<float*>(h->get("dinv32", ld * sizeof(float), true));
        convert<float, double>(c, ld, dinv64, dinv32);
      }
    }
    const bool hard = P->locking == TRPLK_LOCKING_HARD;
    FsaiPrecond fsai;
    if (P->precond == TRPLK_PRECOND_FSAI || P->precond == TRPLK_PRECOND_FSAI_LEARNED ||
        P->precond == TRPLK_PRECOND_IC0)
      fsai = build_fsai_precond(h, Aop.d,
                                P->precond == TRPLK_PRECOND_FSAI ? 0 : P->precond == TRPLK_PRECOND_IC0 ? 2 : 1, P->grid,
                                P->mlp_weights, P->mlp_bf16 != 0, mixed);
    // start block (double, ld)
    double* X0d = static_cast<double*>(h->get("X0", (size_t)ld * P->k * sizeof(double), X0 != nullptr));
    if (X0) {
      TRPLK_CUDA_TRY(cudaMemcpy2DAsync(X0d, ld * sizeof(double), X0, n * sizeof(double), n * sizeof(double), P->k,
                                       cudaMemcpyDefault, c.stream));
    } else {
      start_block(c, n, ld, P->k, P->seed, X0d);
    }
    trplk_info inf;
    memset(&inf, 0, sizeof(inf));
    inf.normA = Aop.norm1;
    SolveOut res;
    const double* Xfinal = nullptr;
    const double* theta_dev = nullptr;
    bool breakdown = false;
    if (!mixed) {
      Solver<double> S(h, "f64", n, P->p, P->q, P->k, P->l, P->tol, P->max_cycles, Aop, Bop, hasB, dinv64, pmode);
      if (fsai.ok) { S.MG = &fsai.G; S.MGT = &fsai.GT; S.ic0_dinv = fsai.dinv; }
      S.hard_lock = hard;
      S.blk = P->block < 1 ? 1 : P->block;
      if (shifted) { S.diagA = diagA; S.diagB = diagB; S.dinv_var = dinv64; }
      res = S.run(X0d);
      inf.cycles = res.cycles;
      inf.mv_A = res.mvA;
      inf.mv_B = res.mvB;
      inf.prec_apply = res.prec;
      inf.locked = res.locked;
      Xfinal = S.U[res.cur];
      theta_dev = S.theta_out;
      breakdown = res.breakdown && !res.converged;
    } else {
      // FP32 phase: to mixed_tol, by default max(tol, 3e-8) -- about half the
      // FP32 unit roundoff, the level at which Ritz vectors stored in FP32 stop
      // improving; a target stuck below 1e-6 for 30 cycles, or not halving its
      // residual in 120 cycles at any level, also ends the phase
      const double tol32 = P->mixed_tol > 0.0 ? P->mixed_tol : std::max(P->tol, 3e-8);
      Solver<float> S32(h, "f32", n, P->p, P->q, P->k, P->l, std::max(tol32, P->tol), P->max_cycles, Aop, Bop, hasB,
                        dinv32, pmode);
      S32.stall_window = 30;
      if (fsai.ok) { S32.MG = &fsai.Gf; S32.MGT = &fsai.GTf; S32.ic0_dinv = fsai.dinvf; }
      S32.hard_lock = hard;
      S32.blk = P->block < 1 ? 1 : P->block;
      if (shifted) { S32.diagA = diagA; S32.diagB = diagB; S32.dinv_var = dinv32; }
      SolveOut r32 = S32.run(X0d);
      inf.locked = r32.locked;
      // promote the k Ritz vectors and refine in FP64 from them
      double* Xr = static_cast<double*>(h->get("Xrefine", (size_t)ld * P->k * sizeof(double)));
      convert<double, float>(c, (int64_t)ld * P->k, S32.U[r32.cur], Xr);
      // The refinement only lifts pairs from about 3e-8 to tol.  Each of its
      // cycles starts from the preconditioned residuals of all unconverged
      // pairs (a block step for every pair at once), then kRefineKrylov
      // Krylov steps on the target, so its basis is
      // q_ref = p_hat + (p - 1) + 1 + kRefineKrylov + l, at most q.
      constexpr int kRefineKrylov = 4;
      const int q_ref = std::min(P->q, P->k + P->p + kRefineKrylov + P->l);
      Solver<double> S64(h, "f64", n, P->p, q_ref, P->k, P->l, P->tol, std::max(1, P->max_cycles - r32.cycles), Aop,
                         Bop, hasB, dinv64, pmode);
      S64.skip_converged = true;
      S64.check_start = true;
      S64.block_refine = true;
      if (fsai.ok) { S64.MG = &fsai.G; S64.MGT = &fsai.GT; S64.ic0_dinv = fsai.dinv; }
      if (shifted) { S64.diagA = diagA; S64.diagB = diagB; S64.dinv_var = dinv64; }
      SolveOut r64 = S64.run(Xr);
      inf.cycles = r32.cycles;
      inf.refine_cycles = r64.cycles;
      inf.mv_A = r32.mvA + r64.mvA;
      inf.mv_B = r32.mvB + r64.mvB;
      inf.prec_apply = r32.prec + r64.prec;
      Xfinal = S64.U[r64.cur];
      theta_dev = S64.theta_out;
      res = r64;
      breakdown = r64.breakdown && !r64.converged;
    }
    // final FP64 check with fresh matvecs
    std::vector<double> rh(P->p);
    check_residuals_fp64(h, Aop, hasB ? &Bop : nullptr, ld, P->p, Xfinal, theta_dev, Aop.norm1, rh.data());
    inf.mv_check = (int64_t)P->p * (hasB ? 2 : 1);
    inf.nconv = 0;
    inf.max_resid = 0.0;
    for (int i = 0; i < P->p; ++i) {
      inf.nconv += rh[i] <= P->tol;
      inf.max_resid = std::max(inf.max_resid, rh[i]);
    }
    // outputs, ascending (hard locking can return the locked pairs out of
    // order): evals and resid permuted on the host, evecs column by column
    std::vector<double> thf(P->p);
    TRPLK_CUDA_TRY(cudaMemcpyAsync(thf.data(), theta_dev, P->p * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    h->sync();
    std::vector<int> ord(P->p);
    for (int i = 0; i < P->p; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return thf[a] < thf[b]; });
    std::vector<double> evs(P->p), rs(P->p);
    for (int i = 0; i < P->p; ++i) {
      evs[i] = thf[ord[i]];
      rs[i] = rh[ord[i]];
    }
    const cudaMemcpyKind k2o = P->outputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const cudaMemcpyKind h2o = P->outputs_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    TRPLK_CUDA_TRY(cudaMemcpyAsync(evals, evs.data(), P->p * sizeof(double), h2o, c.stream));
    bool identity = true;
    for (int i = 0; i < P->p; ++i) identity = identity && ord[i] == i;
    if (identity) {
      TRPLK_CUDA_TRY(cudaMemcpy2DAsync(evecs, n * sizeof(double), Xfinal, ld * sizeof(double), n * sizeof(double),
                                       P->p, k2o, c.stream));
    } else {
      for (int i = 0; i < P->p; ++i)
        TRPLK_CUDA_TRY(cudaMemcpyAsync(evecs + (size_t)i * n, Xfinal + (size_t)ord[i] * ld, n * sizeof(double), k2o,
                                       c.stream));
    }
    TRPLK_CUDA_TRY(cudaMemcpyAsync(resid, rs.data(), P->p * sizeof(double), h2o, c.stream));
    h->sync();
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    inf.launches = h->prof.launches - launches0;
    if (info) *info = inf;
    if (inf.nconv == P->p) return TRPLK_OK;
    if (breakdown) {
      h->err = "Krylov space became invariant (breakdown)";
      return TRPLK_BREAKDOWN;
    }
    h->err = "not converged within max_cycles";
    return TRPLK_NOT_CONVERGED;
  });
}

// ---------------------------------------------------------------- step-level entry points
trplk_status trplk_spmv(trplk_handle* h, const trplk_csr* A, const void* x, void* y) {
  return guarded(h, [&]() -> trplk_status {
    if (!A || !A->on_device || !x || !y || A->n < 1) throw Error(TRPLK_EINVAL, "bad spmv arguments");
    if (x == y) throw Error(TRPLK_EINVAL, "y must not alias x");
    if (A->dtype == TRPLK_F64) {
      DevCsr<double> a = dev_csr64(A);
      attach_sell(h, a, "step.spmv", nullptr);
      spmv<double>(h->ctx, a, static_cast<const double*>(x), static_cast<double*>(y));
    } else if (A->dtype == TRPLK_F32) {
      DevCsr<float> a{A->n, A->nnz, A->rowptr, A->col, static_cast<const float*>(A->val)};
      // the FP32 SELL copy is built from an FP64 view of the same values
      double* v64 = static_cast<double*>(h->get("step.spmv.v64", A->nnz * sizeof(double)));
      convert<double, float>(h->ctx, A->nnz, static_cast<const float*>(A->val), v64);
      DevCsr<double> d{A->n, A->nnz, A->rowptr, A->col, v64};
      attach_sell(h, d, "step.spmv", &a);
      spmv<float>(h->ctx, a, static_cast<const float*>(x), static_cast<float*>(y));
    } else {
      throw Error(TRPLK_EINVAL, "bad dtype");
    }
    h->sync();
    return TRPLK_OK;
  });
}

#define TRPLK_DISPATCH(dtype, ...)                                    \
  do {                                                                \
    if ((dtype) == TRPLK_F64) {                                       \
      using S = double;                                               \
      __VA_ARGS__;                                                    \
    } else if ((dtype) == TRPLK_F32) {                                \
      using S = float;                                                \
      __VA_ARGS__;                                                    \
    } else {                                                          \
      throw Error(TRPLK_EINVAL, "bad dtype");                         \
    }                                                                 \
  } while (0)

trplk_status trplk_inner_project(trplk_handle* h, int dtype, int64_t n, int64_t ld, int w, const void* U,
                                 const void* BU, const void* z, const void* bg, const void* dinv, double rho,
                                 void* v, double* tcol, double* h1) {
  return guarded(h, [&]() -> trplk_status {
    check_ld(n, ld);
    if (w < 1 || w > kMaxQ || !U || !BU || !z || !bg || !v || !tcol || !h1) throw Error(TRPLK_EINVAL, "bad arguments");
    h->clear_status();
    TRPLK_DISPATCH(dtype, ts_inner<S>(h->ctx, ld, w, (const S*)U, (const S*)BU, (const S*)z, (const S*)bg,
                                      (const S*)dinv, dinv ? PM_JACOBI : PM_IDENTITY, rho, (S*)v, tcol, h1));
    check_flags(h, 0);
    return TRPLK_OK;
  });
}

trplk_status trplk_project(trplk_handle* h, int dtype, int64_t n, int64_t ld, int w, const void* BU, const void* v,
                           double* hout) {
  return guarded(h, [&]() -> trplk_status {
    check_ld(n, ld);
    if (w < 1 || w > kMaxQ || !BU || !v || !hout) throw Error(TRPLK_EINVAL, "bad arguments");
    h->clear_status();
    TRPLK_DISPATCH(dtype, ts_project<S>(h->ctx, ld, w, (const S*)BU, (const S*)v, hout));
    check_flags(h, 0);
    return TRPLK_OK;
  });
}

trplk_status trplk_cgs2(trplk_handle* h, int dtype, int64_t n, int64_t ld, int w, const void* U, const void* BU,
                        const trplk_csr* B, const double* h1, void* v, void* Bv, double* beta) {
  return guarded(h, [&]() -> trplk_status {
    check_ld(n, ld);
    if (w < 0 || w > kMaxQ || !U || !BU || !v || !beta || (w > 0 && !h1)) throw Error(TRPLK_EINVAL, "bad arguments");
    if (B && (!Bv || !B->on_device || B->dtype != dtype)) throw Error(TRPLK_EINVAL, "bad B arguments");
    h->clear_status();
    const Ctx& c = h->ctx;
    double* h2 = static_cast<double*>(h->get("step.h2", kMaxQ * sizeof(double)));
    double* sc = static_cast<double*>(h->get("step.scale", 8 * sizeof(double)));
    TRPLK_DISPATCH(dtype, {
      const double eps = sizeof(S) == 8 ? kEpsBreakdown64 : kEpsBreakdown32;
      ts_update_project<S>(c, ld, w, (const S*)U, (const S*)BU, h1, (S*)v, h2);
      if (B) {
        DevCsr<S> b{B->n, B->nnz, B->rowptr, B->col, static_cast<const S*>(B->val)};
        ts_update<S>(c, ld, w, (const S*)U, h2, (S*)v);
        spmv<S>(c, b, (const S*)v, (S*)Bv);
        ts_dot_norm<S>(c, ld, (const S*)v, (const S*)Bv, h1, h2, w, beta, sc, eps);
      } else {
        ts_update_norm<S>(c, ld, w, (const S*)U, h2, h1, (S*)v, beta, sc, eps);
      }
    });
    check_flags(h, kFlagBreakdown);
    return TRPLK_OK;
  });
}

trplk_status trplk_rayleigh_ritz(trplk_handle* h, int w, const double* T, int ldT, double* theta, double* Y) {
  return guarded(h, [&]() -> trplk_status {
    if (w < 1 || w > kMaxQ || ldT < w || !T || !theta || !Y) throw Error(TRPLK_EINVAL, "bad arguments");
    h->clear_status();
    rayleigh_ritz(h->ctx, w, T, ldT, theta, Y);
    check_flags(h, 0);
    return TRPLK_OK;
  });
}

trplk_status trplk_rotate(trplk_handle* h, int dtype, int64_t n, int64_t ld, int w, int k, const void* U,
                          const double* Y, int ldY, void* Xout) {
  return guarded(h, [&]() -> trplk_status {
    check_ld(n, ld);
    if (w < 1 || w > kMaxQ || k < 1 || k > kMaxK || ldY < w || !U || !Y || !Xout || U == Xout)
      throw Error(TRPLK_EINVAL, "bad arguments");
    h->clear_status();
    TRPLK_DISPATCH(dtype, ts_rotate<S>(h->ctx, ld, w, k, (const S*)U, Y, ldY, (S*)Xout));
    check_flags(h, 0);
    return TRPLK_OK;
  });
}

trplk_status trplk_rotate_tc(trplk_handle* h, int64_t n, int64_t ld, int w, int k, const float* U, const double* Y,
                             int ldY, float* Xout) {
  return guarded(h, [&]() -> trplk_status {
    check_ld(n, ld);
    if (!rotate_tc_fits(w, k) || ldY < w || !U || !Y || !Xout || (const void*)U == (const void*)Xout)
      throw Error(TRPLK_EINVAL, "bad arguments");
    h->clear_status();
    rotate_tc(h->ctx, ld, w, k, U, Y, ldY, Xout);
    check_flags(h, 0);
    return TRPLK_OK;
  });
}

trplk_status trplk_residual_norms(trplk_handle* h, int dtype, int64_t n, int64_t ld, int k, const void* X,
                                  const void* AX, const void* BX, const double* theta, double* rnorm, double* xnorm) {
  return guarded(h, [&]() -> trplk_status {
    check_ld(n, ld);
    if (k < 1 || k > kMaxQ || !X || !AX || !theta || !rnorm || !xnorm) throw Error(TRPLK_EINVAL, "bad arguments");
    h->clear_status();
    TRPLK_DISPATCH(dtype, ts_resid<S>(h->ctx, ld, k, (const S*)X, (const S*)AX, (const S*)BX, theta, rnorm, xnorm));
    check_flags(h, 0);
    return TRPLK_OK;
  });
}

trplk_status trplk_start_block(trplk_handle* h, int64_t n, int64_t ld, int k, uint64_t seed, double* X) {
  return guarded(h, [&]() -> trplk_status {
    check_ld(n, ld);
    if (k < 1 || !X) throw Error(TRPLK_EINVAL, "bad arguments");
    start_block(h->ctx, n, ld, k, seed, X);
    h->sync();
    return TRPLK_OK;
  });
}

trplk_status trplk_check_residuals(trplk_handle* h, const trplk_csr* A, const trplk_csr* B, int64_t ld, int p,
                                   const double* X, const double* theta, double normA, double* resid) {
  return guarded(h, [&]() -> trplk_status {
    if (!A || !X || !theta || !resid || p < 1 || p > kMaxQ) throw Error(TRPLK_EINVAL, "bad arguments");
    check_ld(A->n, ld);
    Operator Aop;
    Aop.n = A->n;
    Aop.d = dev_csr64(A);
    Operator Bop;
    if (B) {
      Bop.n = B->n;
      Bop.d = dev_csr64(B);
    }
    h->clear_status();
    std::vector<double> rh(p);
    check_residuals_fp64(h, Aop, B ? &Bop : nullptr, ld, p, X, theta, normA, rh.data());
    TRPLK_CUDA_TRY(cudaMemcpy(resid, rh.data(), p * sizeof(double), cudaMemcpyHostToDevice));
    check_flags(h, 0);
    return TRPLK_OK;
  });
}

trplk_status trplk_set_wait_limit(trplk_handle* h, int64_t polls) {
  return guarded(h, [&]() -> trplk_status {
    h->sync();
    h->ctx.wait_polls = polls < 0 ? kWaitPolls : (uint32_t)std::min<int64_t>(polls, 1ll << 31);
    return TRPLK_OK;
  });
}

static const char* kProfNames[kProfKinds] = {
    "spmv", "spmv_scaled", "ts_project", "ts_inner", "ts_update_project", "ts_update_norm", "ts_update",
    "ts_rotate", "ts_resid", "ts_dot", "rayleigh_ritz", "other",
    "spmv_f64", "spmv_scaled_f64", "ts_project_f64", "ts_inner_f64", "ts_update_project_f64", "ts_update_norm_f64",
    "ts_update_f64", "ts_rotate_f64", "ts_resid_f64", "ts_dot_f64", "rayleigh_ritz_f64", "other_f64"};

trplk_status trplk_profile(trplk_handle* h, int enable) {
  return guarded(h, [&]() -> trplk_status {
    h->sync();
    h->prof.reset();
    h->prof.on = enable != 0;
    return TRPLK_OK;
  });
}

const char* trplk_profile_kind_name(int kind) {
  return (kind >= 0 && kind < kProfKinds) ? kProfNames[kind] : nullptr;
}

trplk_status trplk_profile_read(trplk_handle* h, int kind, int64_t* launches, double* milliseconds,
                                double* bytes) {
  return guarded(h, [&]() -> trplk_status {
    if (kind < 0 || kind >= kProfKinds || !launches || !milliseconds || !bytes)
      throw Error(TRPLK_EINVAL, "bad profile query");
    h->sync();
    int64_t n = 0;
    double ms = 0.0, by = 0.0;
    for (const auto& r : h->prof.recs) {
      if (r.kind != kind) continue;
      float t = 0.f;
      TRPLK_CUDA_TRY(cudaEventElapsedTime(&t, h->prof.pool[r.e0], h->prof.pool[r.e1]));
      ++n;
      ms += t;
      by += r.bytes;
    }
    *launches = n;
    *milliseconds = ms;
    *bytes = by;
    return TRPLK_OK;
  });
}

}  // extern "C"
