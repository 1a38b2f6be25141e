// Host-side launch wrappers shared by the translation units of libtrplk.
#pragma once
#include <vector>

#include "common.cuh"

namespace trplk {

// Kernel families timed by the optional per-launch profiler.
enum ProfKind : int {
  PK_SPMV = 0, PK_SPMV_SCALED, PK_TS_PROJ, PK_TS_INNER, PK_TS_UPDPROJ, PK_TS_UPDNORM, PK_TS_UPD,
  PK_TS_ROT, PK_TS_RESID, PK_TS_DOT, PK_RR, PK_OTHER, PK_COUNT
};
// Families of launches on FP64 data are counted apart from their FP32 twins
// (kinds PK_COUNT + base): the two bind on different units.
constexpr int kProfKinds = 2 * PK_COUNT;
template <typename S>
constexpr int prof_kind(int base) { return sizeof(S) == 8 ? PK_COUNT + base : base; }

// Counts every kernel launch; when `on`, brackets each launch with CUDA
// events on the launching stream and records its algorithmic bytes.
struct Profiler {
  bool on = false;
  int64_t launches = 0;
  std::vector<cudaEvent_t> pool;
  size_t next = 0;
  struct Rec {
    int kind;
    size_t e0, e1;
    double bytes;
  };
  std::vector<Rec> recs;
  size_t take() {
    if (next == pool.size()) {
      cudaEvent_t e;
      TRPLK_CUDA_TRY(cudaEventCreate(&e));
      pool.push_back(e);
    }
    return next++;
  }
  void reset() {
    next = 0;
    recs.clear();
  }
  ~Profiler() {
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// Per-handle device context: stream, SM count and the small scratch every
// reduction kernel shares (kernels on one stream run one after another).
struct Ctx {
  cudaStream_t stream = nullptr;
  int device = 0;
  int sms = 0;
  double* partials = nullptr;      // [kMaxPartials][kPartialStride]
  unsigned int* counter = nullptr; // last-CTA ticket, kept at zero between kernels
  int* status = nullptr;           // device status word (kFlag*)
  Profiler* prof = nullptr;
  uint32_t wait_polls = kWaitPolls;  // bound of the streaming passes' mbarrier waits
};

// RAII bracket of one kernel launch for the profiler.
struct ProfScope {
  const Ctx& c;
  int kind;
  double bytes;
  size_t e0 = (size_t)-1;
  ProfScope(const Ctx& c_, int kind_, double bytes_) : c(c_), kind(kind_), bytes(bytes_) {
    if (!c.prof) return;
    c.prof->launches++;
    if (c.prof->on) {
      e0 = c.prof->take();
      TRPLK_CUDA_TRY(cudaEventRecord(c.prof->pool[e0], c.stream));
    }
  }
  ~ProfScope() {
    if (!c.prof || e0 == (size_t)-1) return;
    try {
      size_t e1 = c.prof->take();
      if (cudaEventRecord(c.prof->pool[e1], c.stream) == cudaSuccess) c.prof->recs.push_back({kind, e0, e1, bytes});
    } catch (...) {
      // a failed event never hides the error of the launch itself
    }
  }
};
constexpr int kPartialStride = 2 * kMaxQ;

// Device CSR in the library's own layout.
template <typename S>
struct DevCsr {
  int64_t n = 0, nnz = 0;
  const int64_t* rowptr = nullptr;
  const int32_t* col = nullptr;
  const S* val = nullptr;
  // optional SELL-32 copy (slices of 32 rows, entries column-major within a
  // slice, padded with zeros); used by the matvec when present
  const int64_t* sl_ptr = nullptr;   // [nslices + 1], multiples of 32
  const int32_t* sl_col = nullptr;
  const S* sl_val = nullptr;
  // hybrid layout for rows of very unequal length (power-law graphs): the
  // SELL slices cover only the rows listed in sl_perm (rows of at most
  // kShortRow entries, sorted by descending length; null = all rows in
  // order); long_rows lists the others, longest first: the first n_long_cta
  // (more than kWarpRow entries) get a CTA each, the next n_long_warp a warp
  // each, both reading the CSR arrays above
  const int32_t* sl_perm = nullptr;
  int64_t sl_rows = 0;               // rows in the SELL part (n without sl_perm)
  const int32_t* long_rows = nullptr;
  int64_t n_long_cta = 0, n_long_warp = 0;
  // optional diagonal (DIA) copy for operators whose entries lie on at most
  // kMaxDiag diagonals (stencils, structured FEM): values dia_val[d * ld + i]
  // of a_{i, i + dia_off[d]} (zero where absent), ld = n rounded up to 256;
  // used by the matvec when present (no column indices to read)
  const S* dia_val = nullptr;
  int64_t dia_ld = 0;
  int ndiag = 0;
  int dia_off[64] = {};
};

constexpr int kMaxDiag = 64;     // most diagonals of the DIA form
constexpr int kDiaSamples = 64;  // rows sampled for the DIA offsets
constexpr int kShortRow = 32;    // longest row kept in the SELL part of a hybrid
constexpr int kWarpRow = 1024;   // longest row given one warp; longer: one CTA
constexpr int kHybBuckets = 61;  // length classes of the hybrid's row sort
constexpr int kHybChunk = 1024;  // rows per warp in the sort kernels

// ---- SpMV (spmv.cu)
// y = A x.
template <typename S>
void spmv(const Ctx& c, const DevCsr<S>& A, const S* x, S* y);
// s = *scale; y = s (A x); g = s x; if bx: bg = s bx  (normalisation folded
// into the next matvec).  Rows >= n of y, g, bg are left untouched.
template <typename S>
void spmv_scaled(const Ctx& c, const DevCsr<S>& A, const S* x, const double* scale, S* y, S* g,
                 const S* bx, S* bg);

// SELL-32 construction over the m rows perm[0..m) (perm null: rows 0..m-1):
// lens[s] = longest row of slice s; then, given the slice offsets, scatter
// column indices (when sl_col != nullptr) and values.
void sell_lengths(const Ctx& c, int64_t m, const int64_t* rowptr, const int32_t* perm, int32_t* lens);
// DIA construction: up to kMaxDiag column offsets (col - row) of kDiaSamples
// rows spread over the matrix into out[k * (kMaxDiag + 1)] (count first); then
// dia_val[d * ld + i] = a_{i, i + off[d]} for every entry, *missing set when
// an entry's offset is not among the ndiag sorted offsets.
void dia_sample(const Ctx& c, int64_t n, const int64_t* rowptr, const int32_t* col, int32_t* out);
template <typename S>
void dia_fill(const Ctx& c, int64_t n, int64_t ld, const int64_t* rowptr, const int32_t* col, const double* val,
              int ndiag, const int* off, S* dia_val, int* missing);
// Hybrid row order: per chunk of kHybChunk rows, counts of every length class
// (hist[chunk * kHybBuckets + b]); then, from per-chunk starting offsets, the
// stable counting-sort scatter order[pos] = row.
void hyb_hist(const Ctx& c, int64_t n, const int64_t* rowptr, int32_t* hist);
void hyb_scatter(const Ctx& c, int64_t n, const int64_t* rowptr, const int32_t* offs, int32_t* order);
// length class of a row: [0, 22) one CTA, [22, 28) one warp, [28, 61) SELL
inline int hyb_class_end_cta() { return 22; }
inline int hyb_class_end_warp() { return 28; }
template <typename S>
void sell_fill(const Ctx& c, int64_t m, const int64_t* rowptr, const int32_t* col, const double* val,
               const int32_t* perm, const int64_t* sl_ptr, int32_t* sl_col, S* sl_val);

// ---- tall-skinny passes (ts.cu).  All vectors have ld rows (zero padded).
template <typename S>
void ts_project(const Ctx& c, int64_t ld, int w, const S* BU, const S* v, double* hout);
// zsrc, bsrc (block TRPL+K): form v = M(zsrc - rho bsrc) instead of M(z - rho bg)
template <typename S>
void ts_inner(const Ctx& c, int64_t ld, int w, const S* U, const S* BU, const S* z, const S* bg,
              const S* dinv, int pmode, double rho, S* v, double* tcol, double* h1, const S* zsrc = nullptr,
              const S* bsrc = nullptr);
template <typename S>
void ts_update_project(const Ctx& c, int64_t ld, int w, const S* U, const S* BU, const double* h,
                       S* v, double* hout);
template <typename S>
void ts_update_norm(const Ctx& c, int64_t ld, int w, const S* U, const double* h, const double* haux,
                    S* v, double* beta2, double* scale, double eps_breakdown);
template <typename S>
void ts_update(const Ctx& c, int64_t ld, int w, const S* U, const double* h, S* v);
template <typename S>
void ts_dot_norm(const Ctx& c, int64_t ld, const S* v, const S* bv, const double* h1,
                 const double* h2, int w, double* beta2, double* scale, double eps_breakdown);
template <typename S>
void ts_rotate(const Ctx& c, int64_t ld, int w, int k, const S* U, const double* Y, int ldY, S* X,
               bool tensor_cores = true);
template <typename S>
void ts_resid(const Ctx& c, int64_t ld, int k, const S* X, const S* AX, const S* BX,
              const double* theta, double* rnorm, double* xnorm);

// ---- restart rotation on the tensor cores (rotate_tc.cu): X = U Y(:, 0:k),
// FP32 U and X, FP64 Y, w <= 64, k <= 32, ld % 128 == 0
bool rotate_tc_fits(int w, int k);
void rotate_tc(const Ctx& c, int64_t ld, int w, int k, const float* U, const double* Y, int ldY, float* X);
// whether ts_rotate<float> takes the tensor-core path for this shape
bool rotate_tc_preferred(int w, int k);

// ---- small kernels (misc.cu)
// v = M (AX[:, t] - theta_t BX[:, t]); pmode PM_* ; theta_t read from device.
template <typename S>
void restart_vector(const Ctx& c, int64_t ld, const S* ax, const S* bx, const double* theta_t,
                    const S* dinv, int pmode, S* v);
template <typename D, typename S>
void convert(const Ctx& c, int64_t count, const S* src, D* dst);
void start_block(const Ctx& c, int64_t n, int64_t ld, int k, uint64_t seed, double* X);
template <typename S>
void jacobi_dinv(const Ctx& c, const DevCsr<S>& A, S* dinv);
// IC(0) preconditioner out = P_s^T (P_s in): `sweeps` Jacobi sweeps with the
// factor L (diagonal included; dinv = 1 / diag(L)), then with LT = L^T;
// t0, t1, t2 scratch vectors (ld rows); out distinct from in and the scratch
template <typename S>
void ic0_apply(const Ctx& c, int64_t ld, const DevCsr<S>& L, const DevCsr<S>& LT, const S* dinv, int sweeps,
               const S* in, S* out, S* t0, S* t1, S* t2);
constexpr int kIc0Sweeps = 2;   // Jacobi sweeps per triangular solve of the IC(0) preconditioner
// diag[i] = a_ii (FP64)
void diag_of(const Ctx& c, int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, double* diag);
// dinv = 1 / max(dA - rho dB, 1e-3 dA) (dB null: 1), rho read from device; rows >= n zero
template <typename S>
void shifted_jacobi(const Ctx& c, int64_t n, int64_t ld, const double* dA, const double* dB, const double* rho,
                    S* dinv);
// r = x - rho * y   (elementwise, ld rows)
template <typename S>
void axpby_shift(const Ctx& c, int64_t ld, const S* x, const S* y, double rho, S* r);

// ---- Rayleigh-Ritz (rr.cu): eigenpairs of the w x w symmetric T (upper
// triangle read), theta ascending, Y (ld = w) sign-normalised; fp32_data: T
// comes from FP32 data, eigenpairs to 1e-10 ||T||_F instead of FP64 rounding.
void rayleigh_ritz(const Ctx& c, int w, const double* T, int ldT, double* theta, double* Y, bool fp32_data = false);

}  // namespace trplk
