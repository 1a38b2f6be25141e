"""Thin ctypes binding of libtrplk (the C ABI declared in include/trplk.h).

Argument marshalling only: every function forwards to the entry point of the
same name in ``libtrplk.so``; all computation happens in the library's CUDA
kernels.  Arrays are passed as torch tensors (device memory, for the
step-level calls and device-resident solves) or numpy arrays (host memory).
Importing this module loads the library and raises if it is missing -- there
is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtrplk.so")

OK, EINVAL, ENOMEM, ECUDA, NOT_CONVERGED, BREAKDOWN, NOT_SPD_B, NAN, ETIMEOUT = range(9)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "NOT_CONVERGED", 5: "BREAKDOWN",
                6: "NOT_SPD_B", 7: "NAN", 8: "ETIMEOUT"}
F64, F32 = 0, 1
SMALLEST = 0
PRECOND_NONE, PRECOND_JACOBI, PRECOND_FSAI, PRECOND_FSAI_LEARNED, PRECOND_JACOBI_SHIFTED, PRECOND_IC0 = range(6)
LOCKING_SOFT, LOCKING_HARD = 0, 1
ABI_VERSION = 2
MLP_PARAMS = 5191
PRECISION_FP64, PRECISION_MIXED = 0, 1


class trplk_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("dtype", C.c_int), ("on_device", C.c_int)]


class trplk_params(C.Structure):
    _fields_ = [("p", C.c_int), ("q", C.c_int), ("k", C.c_int), ("l", C.c_int), ("tol", C.c_double),
                ("max_cycles", C.c_int), ("seed", C.c_uint64), ("which", C.c_int), ("precond", C.c_int),
                ("precision", C.c_int), ("outputs_on_device", C.c_int), ("mlp_weights", C.c_void_p),
                ("grid", C.c_int * 3), ("mlp_bf16", C.c_int), ("mixed_tol", C.c_double), ("locking", C.c_int),
                ("block", C.c_int)]


class trplk_train_params(C.Structure):
    _fields_ = [("iters", C.c_int), ("lr", C.c_double), ("vectors", C.c_int), ("harvest_cycles", C.c_int),
                ("q", C.c_int), ("k", C.c_int), ("l", C.c_int), ("seed", C.c_uint64), ("bf16", C.c_int),
                ("gamma", C.c_double)]


class trplk_info(C.Structure):
    _fields_ = [("cycles", C.c_int), ("refine_cycles", C.c_int), ("mv_A", C.c_int64), ("mv_B", C.c_int64),
                ("prec_apply", C.c_int64), ("mv_check", C.c_int64), ("seconds", C.c_double),
                ("nconv", C.c_int), ("normA", C.c_double), ("max_resid", C.c_double), ("launches", C.c_int64),
                ("locked", C.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class TrplkError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing; build it with `python -m paper_1711_10128_gb300.build`")
    lib = C.CDLL(LIB_PATH)
    vp, i64, i32, dbl, st = C.c_void_p, C.c_int64, C.c_int, C.c_double, C.c_int
    sigs = {
        "trplk_abi_version": (C.c_int, []),
        "trplk_create": (st, [C.POINTER(vp), i32, vp]),
        "trplk_destroy": (st, [vp]),
        "trplk_last_error": (C.c_char_p, [vp]),
        "trplk_solve": (st, [vp, C.POINTER(trplk_csr), C.POINTER(trplk_csr), C.POINTER(trplk_params), vp, vp, vp,
                             vp, C.POINTER(trplk_info)]),
        "trplk_spmv": (st, [vp, C.POINTER(trplk_csr), vp, vp]),
        "trplk_inner_project": (st, [vp, i32, i64, i64, i32, vp, vp, vp, vp, vp, dbl, vp, vp, vp]),
        "trplk_project": (st, [vp, i32, i64, i64, i32, vp, vp, vp]),
        "trplk_cgs2": (st, [vp, i32, i64, i64, i32, vp, vp, C.POINTER(trplk_csr), vp, vp, vp, vp]),
        "trplk_rayleigh_ritz": (st, [vp, i32, vp, i32, vp, vp]),
        "trplk_rotate": (st, [vp, i32, i64, i64, i32, i32, vp, vp, i32, vp]),
        "trplk_residual_norms": (st, [vp, i32, i64, i64, i32, vp, vp, vp, vp, vp, vp]),
        "trplk_rotate_tc": (st, [vp, i64, i64, i32, i32, vp, vp, i32, vp]),
        "trplk_start_block": (st, [vp, i64, i64, i32, C.c_uint64, vp]),
        "trplk_check_residuals": (st, [vp, C.POINTER(trplk_csr), C.POINTER(trplk_csr), i64, i32, vp, vp, dbl, vp]),
        "trplk_project_noalloc": (st, [i32, i64, i64, i32, vp, vp, vp, vp]),
        "trplk_set_wait_limit": (st, [vp, i64]),
        "trplk_mlp_param_count": (C.c_int, []),
        "trplk_fsai_mlp_init": (st, [vp, C.c_uint64]),
        "trplk_fsai_values": (st, [vp, C.POINTER(trplk_csr), i32, vp, vp, i32, vp, C.POINTER(C.c_int64)]),
        "trplk_fsai_apply": (st, [vp, C.POINTER(trplk_csr), vp, vp, vp]),
        "trplk_ic0_apply": (st, [vp, C.POINTER(trplk_csr), vp, vp, vp]),
        "trplk_fsai_loss_grad": (st, [vp, C.POINTER(trplk_csr), vp, vp, i32, vp, i32, dbl, vp, vp]),
        "trplk_fsai_train": (st, [vp, C.POINTER(trplk_csr), vp, i32, C.POINTER(trplk_train_params), vp, vp]),
        "trplk_profile": (st, [vp, i32]),
        "trplk_profile_read": (st, [vp, i32, C.POINTER(C.c_int64), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "trplk_profile_kind_name": (C.c_char_p, [i32]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()
if LIB.trplk_abi_version() != ABI_VERSION:
    raise ImportError("libtrplk ABI version mismatch")


def exported_symbols():
    return [n for n in dir(LIB) if n.startswith("trplk_")]


# ---------------------------------------------------------------- marshalling helpers
def ptr(a):
    """Raw pointer of a torch tensor / numpy array / None."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    raise TypeError(f"cannot take the address of {type(a)}")


def _is_device(a):
    return hasattr(a, "is_cuda") and a.is_cuda


def make_csr(rowptr, col, val):
    """trplk_csr from three arrays (all torch CUDA tensors or all numpy)."""
    dev = _is_device(val)
    dt = F32 if str(val.dtype) in ("torch.float32", "float32") else F64
    n = int(rowptr.shape[0]) - 1
    nnz = int(col.shape[0])
    s = trplk_csr(n, nnz, ptr(rowptr), ptr(col), ptr(val), dt, 1 if dev else 0)
    s._keep = (rowptr, col, val)
    return s


class Handle:
    """Owns one trplk_handle (one CUDA device, one stream)."""

    def __init__(self, device: int = 0, stream=None):
        h = C.c_void_p()
        rc = LIB.trplk_create(C.byref(h), device, stream)
        if rc != OK:
            raise TrplkError(rc, "trplk_create failed")
        self.h = h

    def close(self):
        if self.h:
            LIB.trplk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc, allow=(OK,)):
        if rc not in allow:
            raise TrplkError(rc, LIB.trplk_last_error(self.h).decode())
        return rc


# ---------------------------------------------------------------- the C ABI, same names
def trplk_create(device=0, stream=None) -> Handle:
    return Handle(device, stream)


def trplk_destroy(h: Handle):
    h.close()


def trplk_last_error(h: Handle) -> str:
    return LIB.trplk_last_error(h.h).decode()


def trplk_solve(h: Handle, A: trplk_csr, B, params: trplk_params, X0, evals, evecs, resid, info=None):
    """Status code of trplk_solve; raises on anything but OK / NOT_CONVERGED."""
    info = info if info is not None else trplk_info()
    rc = LIB.trplk_solve(h.h, C.byref(A), C.byref(B) if B is not None else None, C.byref(params), ptr(X0),
                         ptr(evals), ptr(evecs), ptr(resid), C.byref(info))
    h.check(rc, allow=(OK, NOT_CONVERGED))
    return rc


def trplk_spmv(h: Handle, A: trplk_csr, x, y):
    return h.check(LIB.trplk_spmv(h.h, C.byref(A), ptr(x), ptr(y)))


def trplk_inner_project(h, dtype, n, ld, w, U, BU, z, bg, dinv, rho, v, tcol, h1):
    return h.check(LIB.trplk_inner_project(h.h, dtype, n, ld, w, ptr(U), ptr(BU), ptr(z), ptr(bg), ptr(dinv),
                                           float(rho), ptr(v), ptr(tcol), ptr(h1)))


def trplk_project(h, dtype, n, ld, w, BU, v, hout):
    return h.check(LIB.trplk_project(h.h, dtype, n, ld, w, ptr(BU), ptr(v), ptr(hout)))


def trplk_cgs2(h, dtype, n, ld, w, U, BU, B, h1, v, Bv, beta):
    return h.check(LIB.trplk_cgs2(h.h, dtype, n, ld, w, ptr(U), ptr(BU), C.byref(B) if B is not None else None,
                                  ptr(h1), ptr(v), ptr(Bv), ptr(beta)))


def trplk_rayleigh_ritz(h, w, T, ldT, theta, Y):
    return h.check(LIB.trplk_rayleigh_ritz(h.h, w, ptr(T), ldT, ptr(theta), ptr(Y)))


def trplk_rotate(h, dtype, n, ld, w, k, U, Y, ldY, X):
    return h.check(LIB.trplk_rotate(h.h, dtype, n, ld, w, k, ptr(U), ptr(Y), ldY, ptr(X)))


def trplk_rotate_tc(h, n, ld, w, k, U, Y, ldY, X):
    return h.check(LIB.trplk_rotate_tc(h.h, n, ld, w, k, ptr(U), ptr(Y), ldY, ptr(X)))


def trplk_residual_norms(h, dtype, n, ld, k, X, AX, BX, theta, rnorm, xnorm):
    return h.check(LIB.trplk_residual_norms(h.h, dtype, n, ld, k, ptr(X), ptr(AX), ptr(BX), ptr(theta),
                                            ptr(rnorm), ptr(xnorm)))


def trplk_start_block(h, n, ld, k, seed, X):
    return h.check(LIB.trplk_start_block(h.h, n, ld, k, C.c_uint64(seed), ptr(X)))


def trplk_check_residuals(h, A, B, ld, p, X, theta, normA, resid):
    return h.check(LIB.trplk_check_residuals(h.h, C.byref(A), C.byref(B) if B is not None else None, ld, p, ptr(X),
                                             ptr(theta), float(normA), ptr(resid)))


def trplk_project_noalloc(dtype, n, ld, w, BU, v, hout, stream=None):
    """h = BU^T v without any device allocation (status code; raises on error)."""
    rc = LIB.trplk_project_noalloc(dtype, n, ld, w, ptr(BU), ptr(v), ptr(hout), stream)
    if rc != OK:
        raise TrplkError(rc, "trplk_project_noalloc failed")
    return rc


def trplk_set_wait_limit(h, polls):
    """Failure-injection hook: bound the streaming passes' waits to `polls`
    polls (0: give up at once; negative: the default)."""
    return h.check(LIB.trplk_set_wait_limit(h.h, int(polls)))


def trplk_fsai_values(h, A, kind, dims=None, weights=None, bf16=0, g=None):
    """G values on A's lower pattern (device tensor g) -> nnz of the pattern."""
    nnz = C.c_int64()
    d = (C.c_int32 * 3)(*dims) if dims is not None else None
    h.check(LIB.trplk_fsai_values(h.h, C.byref(A), kind, d, ptr(weights), int(bf16), ptr(g), C.byref(nnz)))
    return nnz.value


def trplk_ic0_apply(h, A, l, x, y):
    return h.check(LIB.trplk_ic0_apply(h.h, C.byref(A), ptr(l), ptr(x), ptr(y)))


def trplk_fsai_apply(h, A, g, x, y):
    return h.check(LIB.trplk_fsai_apply(h.h, C.byref(A), ptr(g), ptr(x), ptr(y)))


def trplk_fsai_loss_grad(h, A, dims, weights, bf16, V, nv, gamma=0.1):
    """(loss[3], grad[MLP_PARAMS]) as numpy arrays."""
    loss = np.zeros(3)
    grad = np.zeros(MLP_PARAMS)
    d = (C.c_int32 * 3)(*dims)
    h.check(LIB.trplk_fsai_loss_grad(h.h, C.byref(A), d, ptr(weights), int(bf16), ptr(V), int(nv), float(gamma),
                                     ptr(loss), ptr(grad)))
    return loss, grad


def trplk_fsai_train(h, ops, dims, tp, weights, iters=None):
    """Train in place: ops list of device trplk_csr, dims list of (nx, ny, nz),
    weights float32 numpy array (MLP_PARAMS); returns the loss history."""
    arr = (trplk_csr * len(ops))(*ops)
    d = (C.c_int32 * (3 * len(ops)))(*[int(x) for t in dims for x in t])
    losses = np.zeros(max(tp.iters, 1))
    h.check(LIB.trplk_fsai_train(h.h, arr, d, len(ops), C.byref(tp), ptr(weights), ptr(losses)))
    return losses[:tp.iters]


def trplk_fsai_mlp_init(seed=0):
    """Starting MLP weights (FP32 packed) from the library's initialiser."""
    w = np.zeros(MLP_PARAMS, np.float32)
    rc = LIB.trplk_fsai_mlp_init(ptr(w), int(seed))
    if rc != OK:
        raise TrplkError(rc, "trplk_fsai_mlp_init failed")
    return w


def pack_mlp(p):
    """Pack a dict of MLP arrays (W1, b1, W2, b2, W3, b3) into the FP32 layout."""
    return np.concatenate([np.asarray(p[k], np.float32).ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def unpack_mlp(w):
    w = np.asarray(w, np.float64)
    return dict(W1=w[0:512].reshape(64, 8), b1=w[512:576], W2=w[576:4672].reshape(64, 64), b2=w[4672:4736],
                W3=w[4736:5184].reshape(7, 64), b3=w[5184:5191])


def trplk_profile(h, enable):
    return h.check(LIB.trplk_profile(h.h, int(enable)))


def trplk_profile_read(h, kind):
    """(launches, milliseconds, algorithmic bytes) of one kernel family."""
    n, ms, by = C.c_int64(), C.c_double(), C.c_double()
    h.check(LIB.trplk_profile_read(h.h, kind, C.byref(n), C.byref(ms), C.byref(by)))
    return n.value, ms.value, by.value


def trplk_profile_kind_name(kind):
    r = LIB.trplk_profile_kind_name(kind)
    return r.decode() if r else None


def profile_summary(h):
    """{family name: (launches, ms, bytes)} for every family with launches."""
    out = {}
    k = 0
    while True:
        name = trplk_profile_kind_name(k)
        if name is None:
            break
        n, ms, by = trplk_profile_read(h, k)
        if n:
            out[name] = (n, ms, by)
        k += 1
    return out


# ---------------------------------------------------------------- convenience
def make_params(p, q, k, l, tol=1e-8, max_cycles=5000, seed=0, precond=PRECOND_JACOBI,
                precision=PRECISION_FP64, outputs_on_device=0, mixed_tol=0.0, mlp_weights=None, grid=(0, 0, 0),
                mlp_bf16=1, locking=LOCKING_SOFT, block=1):
    prm = trplk_params(p, q, k, l, tol, max_cycles, seed, SMALLEST, precond, precision, outputs_on_device,
                       ptr(mlp_weights), (C.c_int * 3)(*grid), int(mlp_bf16), mixed_tol, int(locking), int(block))
    prm._keep = mlp_weights
    return prm


def solve(h: Handle, A: trplk_csr, B=None, *, p, q, k, l, tol=1e-8, X0=None, max_cycles=5000, seed=0,
          precond=PRECOND_JACOBI, precision=PRECISION_FP64, mixed_tol=0.0, mlp_weights=None, grid=(0, 0, 0),
          mlp_bf16=1, locking=LOCKING_SOFT, block=1):
    """Solve with host outputs (numpy); returns (evals, evecs, resid, status, info dict)."""
    n = A.n
    evals = np.zeros(p)
    evecs = np.zeros((p, n))       # column-major n x p == row-major p x n
    resid = np.zeros(p)
    info = trplk_info()
    params = make_params(p, q, k, l, tol, max_cycles, seed, precond, precision, 0, mixed_tol, mlp_weights, grid,
                         mlp_bf16, locking, block)
    X0c = None
    if X0 is not None:
        X0c = X0 if _is_device(X0) else np.ascontiguousarray(np.asarray(X0, np.float64).T)
    rc = trplk_solve(h, A, B, params, X0c, evals, evecs, resid, info)
    return evals, evecs.T.copy(), resid, rc, info.as_dict()
