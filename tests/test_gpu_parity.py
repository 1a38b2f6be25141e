"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Step-level tests compare each kernel with the oracle's step on the same seeded
inputs, element by element, at sizes that span several 256-row tiles plus a
ragged tail.  Solve-level tests compare Ritz values with the oracle's after
one and two cycles (same arithmetic up to rounding order), converged
eigenvalues with the oracle and closed forms, and check B-orthonormality,
residuals (recomputed by the oracle's own matvec) and the matvec accounting.

Tolerances: FP64 kernels 1e-12 relative to the natural scale of the quantity
(rounding-order differences of sums of <= n terms, n <= 10^5); FP32 storage
kernels compare with the oracle evaluated on the same float inputs, with the
compensated (Dot2) accumulations held to 1e-12, the plainly accumulated first
CGS pass to n u (u = 2^-24) and FP32 arithmetic to 1e-6; converged
eigenvalues 1e-10 relative (the required FP64 parity).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import trplk as O
from paper_1711_10128_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_10128_gb300 import build
    build.build()
    from paper_1711_10128_gb300 import binding as b
    return b


@pytest.fixture(scope="module")
def h(lib):
    hd = lib.Handle(0)
    yield hd
    hd.close()


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def dev_csr(lib, A, dtype=torch.float64):
    rp, cl, vl = dev(A.rowptr), dev(A.col), dev(A.val, dtype)
    return lib.make_csr(rp, cl, vl)


def padded(X, ld, dtype=torch.float64):
    """column-major (ld x k) device block from an n x k numpy array."""
    n, k = X.shape
    out = torch.zeros((k, ld), dtype=dtype, device="cuda")
    out[:, :n] = torch.from_numpy(np.ascontiguousarray(X.T)).to(dtype).cuda()
    return out


def ld_of(n):
    return (n + 255) // 256 * 256


OPS = {
    "lap2d_37": lambda: W.laplacian_2d(37),                                   # n = 1369, ragged
    "diff3d_13": lambda: W.diffusion_3d(13, W.lognormal_field(13, 1.0, 3)),   # n = 2197
    "fem_7": lambda: W.fem_q1_pencil(7, np.random.default_rng(4).uniform(1, 10, (7, 7, 7)))[0],
}


# ---------------------------------------------------------------- a1 SpMV
@pytest.mark.parametrize("name", sorted(OPS))
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_spmv_matches_oracle(lib, h, name, prec):
    A = OPS[name]()
    rng = np.random.default_rng(1)
    x = rng.standard_normal(A.n)
    As = A.to_scipy()
    if prec == "f64":
        Ad = dev_csr(lib, A)
        y = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        lib.trplk_spmv(h, Ad, dev(x), y)
        ref = O.spmv(As, x)
        scale = abs(As) @ np.abs(x)
        assert np.all(np.abs(y.cpu().numpy() - ref) <= 1e-14 * scale + 1e-300)
    else:
        xf = x.astype(np.float32)
        Af = sp.csr_matrix((A.val.astype(np.float32).astype(np.float64), A.col, A.rowptr), shape=(A.n, A.n))
        Ad = dev_csr(lib, A, torch.float32)
        y = torch.zeros(A.n, dtype=torch.float32, device="cuda")
        lib.trplk_spmv(h, Ad, dev(xf), y)
        ref = O.spmv(Af, xf.astype(np.float64))
        scale = abs(Af) @ np.abs(xf.astype(np.float64))
        assert np.all(np.abs(y.cpu().numpy().astype(np.float64) - ref) <= 1e-6 * scale)


def hub_matrix(n=6000, seed=7):
    """Rows of every length class of the hybrid SpMV: two hubs of more than
    1024 entries, rows of 33..1024, short rows of 1..32, and empty rows."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, 33, n)
    lens[rng.choice(n, 300, replace=False)] = 0
    lens[rng.choice(n, 200, replace=False)] = rng.integers(33, 1025, 200)
    lens[[5, 4000]] = [3000, 1500]
    rows = []
    for i, m in enumerate(lens):
        rows.append(np.sort(rng.choice(n, int(m), replace=False)))
    col = np.concatenate(rows).astype(np.int32)
    rowptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    val = rng.standard_normal(col.size)
    return W.Csr(rowptr, col, val)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_spmv_hybrid_rows_match_oracle(lib, h, prec):
    """The hybrid form (rows sorted by length class: CTA per row, warp per row,
    SELL slices) against the oracle's matvec, empty rows included."""
    A = hub_matrix()
    x = np.random.default_rng(2).standard_normal(A.n)
    dt = torch.float64 if prec == "f64" else torch.float32
    vals = A.val if prec == "f64" else A.val.astype(np.float32).astype(np.float64)
    xs = x if prec == "f64" else x.astype(np.float32).astype(np.float64)
    As = sp.csr_matrix((vals, A.col, A.rowptr), shape=(A.n, A.n))
    y = torch.full((A.n,), 7.0, dtype=dt, device="cuda")
    lib.trplk_spmv(h, dev_csr(lib, A, dt), dev(xs.astype(np.float64 if prec == "f64" else np.float32)), y)
    ref = O.spmv(As, xs)
    scale = abs(As) @ np.abs(xs)
    rel = 1e-14 if prec == "f64" else 1e-6
    assert np.all(np.abs(y.cpu().numpy().astype(np.float64) - ref) <= rel * scale)
    empty = np.flatnonzero(np.diff(A.rowptr) == 0)
    assert empty.size > 0 and np.all(y.cpu().numpy()[empty] == 0)


def test_spmv_storage_form_follows_the_structure(lib, h):
    """Stencil and FEM operators take the diagonal (DIA) form -- the profiler's
    algorithmic bytes of the matvec are ndiag n 8 + 2 n 8, no index traffic --
    and a power-law graph does not; the results match the oracle either way."""
    def matvec_bytes(A):
        x = np.random.default_rng(3).standard_normal(A.n)
        y = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        lib.trplk_profile(h, 1)
        lib.trplk_spmv(h, dev_csr(lib, A), dev(x), y)
        n_l, ms, by = lib.trplk_profile_read(h, 12)   # spmv on FP64 data
        lib.trplk_profile(h, 0)
        ref = O.spmv(A.to_scipy(), x)
        assert np.allclose(y.cpu().numpy(), ref, rtol=0, atol=1e-13 * np.abs(ref).max())
        return n_l, by
    for A, nd in ((W.laplacian_2d(37), 5), (W.diffusion_3d(13, W.lognormal_field(13, 1.0, 3)), 7),
                  (W.fem_q1_pencil(12, np.random.default_rng(4).uniform(1, 10, (12, 12, 12)))[0], 27)):
        n_l, by = matvec_bytes(A)
        assert n_l == 1 and by == nd * A.n * 8 + 2 * A.n * 8
    # too much zero padding (35%: boundary rows of a 7^3 Q1 operator) or too
    # many diagonals (a power-law graph): another form, never the DIA bytes
    for A in (W.fem_q1_pencil(7, np.random.default_rng(4).uniform(1, 10, (7, 7, 7)))[0],
              W.chung_lu_laplacian(3000, 8.0, 2.1, 3)):
        n_l, by = matvec_bytes(A)
        assert n_l == 1 and by > A.nnz * 12


def test_spmv_full_size_sampled_rows(lib, h):
    """128^3 lognormal diffusion (n = 2,097,152): sampled rows against the
    oracle's row dot products."""
    A = W.diffusion_3d(128, W.lognormal_field(128, 1.0, 1))
    x = W.start_block(A.n, 1, 11)[:, 0]
    y = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    lib.trplk_spmv(h, dev_csr(lib, A), dev(x), y)
    yh = y.cpu().numpy()
    rows = np.random.default_rng(2).choice(A.n, 4000, replace=False)
    rows = np.concatenate([rows, [0, A.n - 1]])
    for i in rows:
        s, e = A.rowptr[i], A.rowptr[i + 1]
        ref = float(np.dot(A.val[s:e], x[A.col[s:e]]))
        assert abs(yh[i] - ref) <= 1e-14 * float(np.dot(np.abs(A.val[s:e]), np.abs(x[A.col[s:e]])))


# ---------------------------------------------------------------- a2-a4 inner step
def basis(n, w, seed, B=None):
    Bf = (lambda v: v.copy()) if B is None else (lambda v: B @ v)
    U, BU, _ = O.b_orthonormalise(np.random.default_rng(seed).standard_normal((n, w)), Bf)
    return U, BU, Bf


@pytest.mark.parametrize("n,w", [(1369, 1), (2197, 9), (5000, 40), (777, 64)])
def test_inner_project_fp64(lib, h, n, w):
    rng = np.random.default_rng(n + w)
    U, BU, _ = basis(n, w, 3)
    z, bg = rng.standard_normal(n), rng.standard_normal(n)
    dinv = 1.0 / rng.uniform(1, 5, n)
    rho = 0.37
    ld = ld_of(n)
    Ud = padded(U, ld)
    zd, bgd, dvd = padded(z[:, None], ld), padded(bg[:, None], ld), padded(dinv[:, None], ld)
    v = torch.zeros(ld, dtype=torch.float64, device="cuda")
    tcol = torch.zeros(w, dtype=torch.float64, device="cuda")
    h1 = torch.zeros(w, dtype=torch.float64, device="cuda")
    lib.trplk_inner_project(h, lib.F64, n, ld, w, Ud, Ud, zd, bgd, dvd, rho, v, tcol, h1)
    vref = dinv * (z - rho * bg)                     # the oracle's Jacobi step
    # the GPU forms z - rho*bg with one FMA: a few ulp of |z| + |rho bg|
    assert np.all(np.abs(v.cpu().numpy()[:n] - vref) <= 4e-16 * dinv * (np.abs(z) + rho * np.abs(bg)))
    assert np.all(v.cpu().numpy()[n:] == 0)
    sc = math.sqrt(n)
    assert np.allclose(tcol.cpu().numpy(), U.T @ z, rtol=0, atol=1e-13 * sc)
    assert np.allclose(h1.cpu().numpy(), U.T @ vref, rtol=0, atol=1e-13 * sc)


@pytest.mark.parametrize("n,w", [(2197, 9), (5000, 40)])
def test_inner_project_fp32_compensated(lib, h, n, w):
    rng = np.random.default_rng(7)
    U = rng.standard_normal((n, w)).astype(np.float32)
    z = rng.standard_normal(n).astype(np.float32)
    bg = rng.standard_normal(n).astype(np.float32)
    ld = ld_of(n)
    Ud = padded(U, ld, torch.float32)
    zd, bgd = padded(z[:, None], ld, torch.float32), padded(bg[:, None], ld, torch.float32)
    v = torch.zeros(ld, dtype=torch.float32, device="cuda")
    tcol = torch.zeros(w, dtype=torch.float64, device="cuda")
    h1 = torch.zeros(w, dtype=torch.float64, device="cuda")
    rho = 0.25
    lib.trplk_inner_project(h, lib.F32, n, ld, w, Ud, Ud, zd, bgd, None, rho, v, tcol, h1)
    vh = v.cpu().numpy()[:n]
    vref = (z - np.float32(rho) * bg)                # float arithmetic as on the GPU
    assert np.allclose(vh, vref, rtol=1e-6, atol=1e-6)
    U64 = U.astype(np.float64)
    # exact products of the float data, summed in FP64.  The compensated sums
    # round each lane's four consecutive products together and add the block
    # sums exactly (TwoSum): at most 4u sum |u z| (u = 2^-24) -- n/4 times
    # tighter than plain FP32 summation allows -- and in practice far below
    exact_t = U64.T @ z.astype(np.float64)
    mag = np.abs(U64).T @ np.abs(z.astype(np.float64))
    err_t = np.abs(tcol.cpu().numpy() - exact_t)
    print("T column error / sum|u z|: max", (err_t / mag).max())
    assert np.all(err_t <= 4 * 2.0 ** -24 * mag + 1e-13 * mag)
    # the first CGS pass is accumulated plainly in FP32 (the compensated second
    # pass removes its error): FP32 summation accuracy, n u sum |u v|
    exact_h = U64.T @ vh.astype(np.float64)
    magh = np.abs(U64).T @ np.abs(vh.astype(np.float64))
    assert np.all(np.abs(h1.cpu().numpy() - exact_h) <= n * 2.0 ** -24 * magh)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n,w", [(1369, 1), (5000, 17), (2197, 33), (300_000, 49), (777, 64)])
def test_project_matches_definition(lib, h, prec, n, w):
    """trplk_project, h = BU^T v (one CGS pass in the B-inner product, Sec. 3),
    against its definition evaluated in FP64 numpy on the same inputs, for
    every basis-width instantiation (w <= 32, <= 48, <= 64) and a ragged n
    whose tiles outnumber the CTAs.  FP64 data: rounding-order differences,
    1e-13 sqrt(n) in the scale of unit columns.  FP32 data: the products are
    exact in FP64, so the error is the compensated sum's, at most
    4u sum |b v| (u = 2^-24)."""
    rng = np.random.default_rng(n + 7 * w)
    BU = rng.standard_normal((n, w)) / math.sqrt(n)
    v = rng.standard_normal(n)
    ld = ld_of(n)
    tdt = torch.float64 if prec == "f64" else torch.float32
    if prec == "f32":
        BU, v = BU.astype(np.float32).astype(np.float64), v.astype(np.float32).astype(np.float64)
    out = torch.full((w,), float("nan"), dtype=torch.float64, device="cuda")
    lib.trplk_project(h, lib.F64 if prec == "f64" else lib.F32, n, ld, w, padded(BU, ld, tdt),
                      padded(v[:, None], ld, tdt), out)
    got = out.cpu().numpy()
    ref = BU.T @ v
    if prec == "f64":
        assert np.allclose(got, ref, rtol=0, atol=1e-13 * math.sqrt(n) * np.abs(v).max()), np.abs(got - ref).max()
    else:
        mag = np.abs(BU).T @ np.abs(v)
        assert np.all(np.abs(got - ref) <= 4 * 2.0 ** -24 * mag + 1e-15 * mag), (np.abs(got - ref) / mag).max()


@pytest.mark.parametrize("withB", [False, True])
@pytest.mark.parametrize("w", [0, 1, 12, 30])
def test_cgs2_matches_oracle(lib, h, withB, w):
    if withB:
        A, B = W.fem_q1_pencil(9)
        Bs = B.to_scipy()
        n = B.n
    else:
        n = 3001
        Bs = None
    U, BU, Bf = basis(n, max(w, 1), 5, Bs)
    U, BU = U[:, :w], BU[:, :w]
    x = np.random.default_rng(9).standard_normal(n)
    wo, Bw, beta, beta0, hsum = O.cgs2(x, U, BU, Bf)
    ld = ld_of(n)
    if w:
        Ud = padded(U, ld)
        BUd = padded(BU, ld) if withB else Ud
    else:
        Ud = torch.zeros(ld, dtype=torch.float64, device="cuda")
        BUd = Ud
    v = padded(x[:, None], ld)[0].contiguous()
    h1 = torch.from_numpy(BU.T @ x if w else np.zeros(1)).cuda()
    bv = torch.zeros(ld, dtype=torch.float64, device="cuda")
    bet = torch.zeros(2, dtype=torch.float64, device="cuda")
    Bd = dev_csr(lib, B) if withB else None
    lib.trplk_cgs2(h, lib.F64, n, ld, w, Ud, BUd, Bd, h1, v, bv if withB else None, bet)
    vh = v.cpu().numpy()
    assert np.allclose(vh[:n], wo, rtol=0, atol=1e-13 * np.abs(x).max())
    assert np.all(vh[n:] == 0)
    b = bet.cpu().numpy()
    assert abs(b[0] - beta) <= 1e-12 * beta
    assert abs(b[1] - beta0) <= 1e-12 * beta0
    if withB:
        assert np.allclose(bv.cpu().numpy()[:n], Bw, rtol=0, atol=1e-13 * np.abs(Bw).max())


# ---------------------------------------------------------------- a6 Rayleigh-Ritz
@pytest.mark.parametrize("w", [1, 2, 3, 17, 40, 64])
def test_rayleigh_ritz_matches_oracle(lib, h, w):
    rng = np.random.default_rng(w)
    M = rng.standard_normal((w, w))
    M = M + M.T + np.diag(np.arange(w) * 0.5)   # well separated spectrum
    T = np.triu(M) + np.tril(rng.standard_normal((w, w)), -1) * 1e3   # lower triangle must be ignored
    th_ref, Y_ref = O.rayleigh_ritz(np.triu(M))
    Td = torch.from_numpy(np.asfortranarray(T).ravel(order="F")).cuda()
    th = torch.zeros(w, dtype=torch.float64, device="cuda")
    Y = torch.zeros(w * w, dtype=torch.float64, device="cuda")
    lib.trplk_rayleigh_ritz(h, w, Td, w, th, Y)
    scale = np.abs(th_ref).max()
    assert np.allclose(th.cpu().numpy(), th_ref, rtol=0, atol=1e-13 * scale)
    Yh = Y.cpu().numpy().reshape(w, w).T          # column-major
    assert np.allclose(Yh, Y_ref, atol=1e-10)
    assert np.allclose(Yh.T @ Yh, np.eye(w), atol=1e-13)


def test_rayleigh_ritz_diagonal_and_degenerate(lib, h):
    """Already-diagonal T (the state right after a thick restart) and an exactly
    degenerate pair: eigenvalues exact, eigenvectors orthonormal."""
    w = 12
    d = np.array([3.0, 1.0, 2.0, 2.0, 5.0, -1.0, 0.5, 7.0, 7.0, 7.0, 4.0, 6.0])
    T = np.diag(d)
    th = torch.zeros(w, dtype=torch.float64, device="cuda")
    Y = torch.zeros(w * w, dtype=torch.float64, device="cuda")
    lib.trplk_rayleigh_ritz(h, w, torch.from_numpy(T.ravel(order="F")).cuda(), w, th, Y)
    assert np.array_equal(th.cpu().numpy(), np.sort(d))
    Yh = Y.cpu().numpy().reshape(w, w).T
    assert np.allclose(Yh.T @ Yh, np.eye(w), atol=0)
    assert np.allclose(T @ Yh, Yh * th.cpu().numpy(), atol=0)


@pytest.mark.parametrize("w", [24, 40, 64])
def test_rayleigh_ritz_clustered_spectrum(lib, h, w):
    """The spectrum of a thick-restart T on a power-law graph: Ritz values from
    1e-3 to 1e4, with a pair 1e-9 apart (relative), an exact double and a
    triple 1e-12 ||T|| apart, in a random orthogonal basis.  Eigenvectors inside
    a cluster are not unique, so they are checked through invariants: the
    eigenvalues against LAPACK's to 1e-13 ||T||, Y orthonormal to 1e-13, and
    T Y = Y Theta to 1e-13 ||T||."""
    rng = np.random.default_rng(100 + w)
    d = np.sort(10.0 ** rng.uniform(-3, 4, w))
    top = d.max()
    d[1] = d[0] * (1 + 1e-9)
    d[3] = d[2]
    d[5], d[6] = d[4] + 1e-12 * top, d[4] + 2e-12 * top
    Q = np.linalg.qr(rng.standard_normal((w, w)))[0]
    T = (Q * d) @ Q.T
    T = (T + T.T) / 2
    th = torch.zeros(w, dtype=torch.float64, device="cuda")
    Y = torch.zeros(w * w, dtype=torch.float64, device="cuda")
    lib.trplk_rayleigh_ritz(h, w, torch.from_numpy(np.asfortranarray(T).ravel(order="F")).cuda(), w, th, Y)
    thh = th.cpu().numpy()
    Yh = Y.cpu().numpy().reshape(w, w).T
    assert np.all(np.diff(thh) >= 0)
    assert np.abs(thh - np.linalg.eigvalsh(T)).max() <= 1e-13 * top
    assert np.abs(Yh.T @ Yh - np.eye(w)).max() <= 1e-13
    assert np.abs(T @ Yh - Yh * thh).max() <= 1e-13 * top


# ---------------------------------------------------------------- a7 rotation + residuals
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_rotate_and_residual_norms(lib, h, prec):
    n, w, k = 4099, 33, 15
    rng = np.random.default_rng(12)
    U = rng.standard_normal((n, w))
    AU = rng.standard_normal((n, w))
    Yc = np.linalg.qr(rng.standard_normal((w, w)))[0]
    theta = np.sort(rng.uniform(0, 2, k))
    ld = ld_of(n)
    dt, dtn = (torch.float64, np.float64) if prec == "f64" else (torch.float32, np.float32)
    code = lib.F64 if prec == "f64" else lib.F32
    Ud, AUd = padded(U, ld, dt), padded(AU, ld, dt)
    Yd = torch.from_numpy(Yc.ravel(order="F")).cuda()
    X = torch.zeros((k, ld), dtype=dt, device="cuda")
    AX = torch.zeros((k, ld), dtype=dt, device="cuda")
    lib.trplk_rotate(h, code, n, ld, w, k, Ud, Yd, w, X)
    lib.trplk_rotate(h, code, n, ld, w, k, AUd, Yd, w, AX)
    Uq, AUq = U.astype(dtn).astype(np.float64), AU.astype(dtn).astype(np.float64)
    Xref, AXref = Uq @ Yc[:, :k], AUq @ Yc[:, :k]
    tol = 1e-13 if prec == "f64" else 2e-6
    assert np.allclose(X.cpu().numpy()[:, :n].T, Xref, rtol=0, atol=tol * np.abs(Uq).max() * math.sqrt(w))
    assert np.all(X.cpu().numpy()[:, n:] == 0)
    rn = torch.zeros(k, dtype=torch.float64, device="cuda")
    xn = torch.zeros(k, dtype=torch.float64, device="cuda")
    lib.trplk_residual_norms(h, code, n, ld, k, X, AX, None, torch.from_numpy(theta).cuda(), rn, xn)
    Xg = X.cpu().numpy()[:, :n].T.astype(np.float64)
    AXg = AX.cpu().numpy()[:, :n].T.astype(np.float64)
    if prec == "f64":
        rref, xref = O.residual_norms(AXg, Xg, Xg, theta)
        assert np.allclose(rn.cpu().numpy(), rref, rtol=1e-13)
        assert np.allclose(xn.cpu().numpy(), xref, rtol=1e-13)
    else:
        th32 = theta.astype(np.float32)
        R = (AX.cpu().numpy()[:, :n].T - X.cpu().numpy()[:, :n].T * th32[None, :]).astype(np.float64)
        assert np.allclose(rn.cpu().numpy(), np.linalg.norm(R, axis=0), rtol=1e-6)
        # sums of squares, four per FP32 block then exact TwoSum: relative error
        # of the sum at most 3u, of the norm 1.5u (u = 2^-24)
        assert np.allclose(xn.cpu().numpy(), np.linalg.norm(Xg, axis=0), rtol=2 * 2.0 ** -24)


@pytest.mark.parametrize("w,k", [(5, 3), (33, 15), (40, 20), (50, 25), (64, 32)])
def test_tensor_core_rotation_matches_definition(lib, h, w, k):
    """The restart rotation X = U Y on the tensor cores (tcgen05, BF16 parts
    of an exact three-way split, FP32 accumulation) against U Y in FP64 on the
    stored FP32 values, at the FP32 rotation's tolerance (2e-6 of
    max|U| sqrt(w)), for narrow to the widest shapes and a ragged n; padding
    rows stay zero."""
    n = 4099
    rng = np.random.default_rng(w * 31 + k)
    U = rng.standard_normal((n, w))
    Yc = np.linalg.qr(rng.standard_normal((w, w)))[0]
    ld = ld_of(n)
    Ud = padded(U, ld, torch.float32)
    Yd = torch.from_numpy(Yc.ravel(order="F")).cuda()
    X = torch.full((k, ld), float("nan"), dtype=torch.float32, device="cuda")
    X[:, n:] = 0
    lib.trplk_rotate_tc(h, n, ld, w, k, Ud, Yd, w, X)
    Uq = U.astype(np.float32).astype(np.float64)
    Xref = Uq @ Yc[:, :k]
    got = X.cpu().numpy()[:, :n].T.astype(np.float64)
    err = np.abs(got - Xref).max() / (np.abs(Uq).max() * math.sqrt(w))
    print("tensor-core rotation w", w, "k", k, "error / (max|U| sqrt(w))", err)
    assert err <= 2e-6
    assert np.all(X.cpu().numpy()[:, n:] == 0)
    # the dispatching entry agrees (it takes this path for w k >= 480)
    X2 = torch.zeros((k, ld), dtype=torch.float32, device="cuda")
    lib.trplk_rotate(h, lib.F32, n, ld, w, k, Ud, Yd, w, X2)
    assert np.abs(X2.cpu().numpy()[:, :n].T - Xref).max() <= 2e-6 * np.abs(Uq).max() * math.sqrt(w)


@pytest.mark.parametrize("w,k", [(16, 6), (40, 20), (50, 25), (64, 32)])
def test_tensor_core_rotation_many_tiles_per_cta(lib, h, w, k):
    """The rotation's pipeline over many tiles per CTA (n = 300,007: 2,344
    tiles of 128 rows on one CTA per SM, so every staged-tile slot, operand set
    and tensor-memory accumulator is reused many times, with its barrier
    parities) against U Y in FP64, at the FP32 rotation's tolerance; the
    padding rows stay zero."""
    n = 300_007
    rng = np.random.default_rng(w * 7 + k)
    U = rng.standard_normal((n, w)) / math.sqrt(n)
    Yc = np.linalg.qr(rng.standard_normal((w, w)))[0]
    ld = ld_of(n)
    Ud = padded(U, ld, torch.float32)
    Yd = torch.from_numpy(Yc.ravel(order="F")).cuda()
    X = torch.full((k, ld), float("nan"), dtype=torch.float32, device="cuda")
    X[:, n:] = 0
    lib.trplk_rotate_tc(h, n, ld, w, k, Ud, Yd, w, X)
    Uq = U.astype(np.float32).astype(np.float64)
    Xref = Uq @ Yc[:, :k]
    got = X.cpu().numpy()[:, :n].T.astype(np.float64)
    assert np.abs(got - Xref).max() <= 2e-6 * np.abs(Uq).max() * math.sqrt(w)
    assert np.all(X.cpu().numpy()[:, n:] == 0)


# ---------------------------------------------------------------- start block (bit-exact)
def test_start_block_bit_exact(lib, h):
    n, k = 3001, 7
    ld = ld_of(n)
    X = torch.zeros((k, ld), dtype=torch.float64, device="cuda")
    lib.trplk_start_block(h, n, ld, k, 12345, X)
    ref = W.start_block(n, k, 12345)
    got = X.cpu().numpy()
    assert np.array_equal(got[:, :n].T, ref)
    assert np.all(got[:, n:] == 0)


# ---------------------------------------------------------------- a8 final check
def test_check_residuals_matches_numpy(lib, h):
    A, B = W.fem_q1_pencil(6)
    As, Bs = A.to_scipy(), B.to_scipy()
    p = 4
    rng = np.random.default_rng(3)
    X = rng.standard_normal((A.n, p))
    theta = rng.uniform(1, 10, p)
    ld = ld_of(A.n)
    out = torch.zeros(p, dtype=torch.float64, device="cuda")
    nA = O.norm1(As)
    lib.trplk_check_residuals(h, dev_csr(lib, A), dev_csr(lib, B), ld, p, padded(X, ld),
                              torch.from_numpy(theta).cuda(), nA, out)
    ref = np.linalg.norm(As @ X - (Bs @ X) * theta, axis=0) / (nA * np.linalg.norm(X, axis=0))
    assert np.allclose(out.cpu().numpy(), ref, rtol=1e-13)


# ---------------------------------------------------------------- whole solves
@pytest.mark.parametrize("cycles", [1, 2, 3])
def test_first_cycles_match_oracle_iterates(lib, h, cycles):
    """Same start block, same readings: after 1-3 cycles the Ritz values agree
    to rounding level (the +K block enters from cycle 2 on)."""
    A = W.diffusion_3d(12, W.lognormal_field(12, 1.0, 21))
    p, q, k, l = 4, 16, 6, 2
    X0 = W.start_block(A.n, k, 5)
    ref = O.solve(A.to_scipy(), None, p, q, k, l, 1e-14, X0, "jacobi", max_cycles=cycles)
    ev, X, res, rc, info = lib.solve(h, dev_csr(lib, A), None, p=p, q=q, k=k, l=l, tol=1e-14, X0=X0,
                                     max_cycles=cycles)
    assert info["cycles"] == cycles == ref["cycles"]
    assert info["mv_A"] == ref["mv_A"]
    assert np.allclose(ev, ref["evals"], rtol=1e-11)
    # Ritz vectors: same up to rounding (spectrum is simple here)
    for i in range(p):
        c = abs(X[:, i] @ ref["evecs"][:, i])
        assert c > 1 - 1e-9


def test_c1_laplacian_full_size_matches_oracle_and_closed_form(lib, h):
    """100 x 100 5-point Laplacian, p = 5, q = 20, p_hat = 8, +K = 5, Jacobi, tol 1e-8."""
    N, p, q, k, l = 100, 5, 20, 8, 5
    A = W.laplacian_2d(N)
    X0 = W.start_block(A.n, k, 0)
    ref = O.solve(A.to_scipy(), None, p, q, k, l, 1e-8, X0, "jacobi")
    ev, X, res, rc, info = lib.solve(h, dev_csr(lib, A), None, p=p, q=q, k=k, l=l, tol=1e-8, X0=X0)
    assert rc == lib.OK
    hgrid = math.pi / (2 * (N + 1))
    lam = np.sort([4 * math.sin(i * hgrid) ** 2 + 4 * math.sin(j * hgrid) ** 2
                   for i in range(1, 8) for j in range(1, 8)])[:p]
    assert np.all(np.abs(ev - ref["evals"]) <= 1e-10 * np.abs(ref["evals"]))
    assert np.all(np.abs(ev - lam) <= 1e-10 * lam)
    assert np.all(res <= 1e-8)
    # residuals recomputed by the oracle's matvec
    As = A.to_scipy()
    r = np.linalg.norm(As @ X - X * ev, axis=0) / (O.norm1(As) * np.linalg.norm(X, axis=0))
    assert np.all(r <= 1e-8)
    assert np.allclose(X.T @ X, np.eye(p), atol=1e-12)
    assert info["mv_A"] == k + (q - k) * info["cycles"]


def test_generalized_fem_pencil_matches_oracle(lib, h):
    N = 8
    A, B = W.fem_q1_pencil(N, np.random.default_rng(2).uniform(1, 10, (N, N, N)))
    As, Bs = A.to_scipy(), B.to_scipy()
    p, q, k, l = 5, 20, 8, 1
    X0 = W.start_block(A.n, k, 2)
    ref = O.solve(As, Bs, p, q, k, l, 1e-9, X0, "jacobi")
    ev, X, res, rc, info = lib.solve(h, dev_csr(lib, A), dev_csr(lib, B), p=p, q=q, k=k, l=l, tol=1e-9, X0=X0)
    assert rc == lib.OK and ref["status"] == O.OK
    assert np.all(np.abs(ev - ref["evals"]) <= 1e-10 * np.abs(ref["evals"]))
    assert np.allclose(X.T @ (Bs @ X), np.eye(p), atol=1e-11)
    r = np.linalg.norm(As @ X - (Bs @ X) * ev, axis=0) / (O.norm1(As) * np.linalg.norm(X, axis=0))
    assert np.all(r <= 1e-9)
    assert info["mv_B"] == info["mv_A"]


def test_mixed_precision_matches_oracle(lib, h):
    N = 20
    A = W.diffusion_3d(N, W.lognormal_field(N, 1.0, 1))
    As = A.to_scipy()
    p, q, k, l = 6, 24, 10, 1
    X0 = W.start_block(A.n, k, 0)
    ref = O.solve(As, None, p, q, k, l, 1e-10, X0, "jacobi")
    ev, X, res, rc, info = lib.solve(h, dev_csr(lib, A), None, p=p, q=q, k=k, l=l, tol=1e-10, X0=X0,
                                     precision=lib.PRECISION_MIXED)
    assert rc == lib.OK
    assert np.all(res <= 1e-10)
    assert np.all(np.abs(ev - ref["evals"]) <= 1e-10 * np.abs(ref["evals"]))
    assert np.allclose(X.T @ X, np.eye(p), atol=1e-11)


def test_mixed_precision_generalized_pencil_matches_oracle(lib, h):
    """The mixed path on the Q1 stiffness/mass pencil (B != I): FP32 basis with
    B-images, FP64 refinement; eigenvalues against the FP64 oracle."""
    N = 8
    A, B = W.fem_q1_pencil(N, np.random.default_rng(2).uniform(1, 10, (N, N, N)))
    As, Bs = A.to_scipy(), B.to_scipy()
    p, q, k, l = 5, 20, 8, 1
    X0 = W.start_block(A.n, k, 2)
    ref = O.solve(As, Bs, p, q, k, l, 1e-9, X0, "jacobi")
    ev, X, res, rc, info = lib.solve(h, dev_csr(lib, A), dev_csr(lib, B), p=p, q=q, k=k, l=l, tol=1e-9, X0=X0,
                                     precision=lib.PRECISION_MIXED)
    assert rc == lib.OK and ref["status"] == O.OK
    assert np.all(np.abs(ev - ref["evals"]) <= 1e-10 * np.abs(ref["evals"]))
    assert np.allclose(X.T @ (Bs @ X), np.eye(p), atol=1e-11)
    r = np.linalg.norm(As @ X - (Bs @ X) * ev, axis=0) / (O.norm1(As) * np.linalg.norm(X, axis=0))
    assert np.all(r <= 1e-9)
    # every orthogonalised vector costs one B matvec; a dropped +K column or an
    # early end of the inner loop costs no A matvec, so only >= holds here
    assert info["mv_B"] >= info["mv_A"]


_CL_REF = {}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n,mean,p", [(3000, 8.0, 6), (80000, 20.0, 4)])
def test_chung_lu_laplacian_matches_oracle(lib, h, precision, n, mean, p):
    """Shifted Laplacian of a Chung-Lu power-law graph (largest component;
    the larger case has rows of more than 1024 entries, so every class of the
    hybrid SpMV runs inside the solve): the smallest eigenvalue is the shift
    exactly (constant vector), the rest match the oracle's."""
    L = W.chung_lu_laplacian(n, mean, 2.1, 3)
    Ls = L.to_scipy()
    q, k, l = 24, 10, 1
    X0 = W.start_block(L.n, k, 1)
    if (n, p) not in _CL_REF:
        _CL_REF[(n, p)] = O.solve(Ls, None, p, q, k, l, 1e-10, X0, "jacobi")
    ref = _CL_REF[(n, p)]
    prec = lib.PRECISION_FP64 if precision == "fp64" else lib.PRECISION_MIXED
    ev, X, res, rc, info = lib.solve(h, dev_csr(lib, L), None, p=p, q=q, k=k, l=l, tol=1e-10, X0=X0,
                                     precision=prec)
    assert rc == lib.OK and ref["status"] == O.OK
    assert abs(ev[0] - 1e-3) <= 1e-12
    assert np.all(np.abs(ev - ref["evals"]) <= 1e-10 * np.abs(ref["evals"]))
    r = np.linalg.norm(Ls @ X - X * ev, axis=0) / (O.norm1(Ls) * np.linalg.norm(X, axis=0))
    assert np.all(r <= 1e-10)


def test_ragged_and_degenerate_edges(lib, h):
    """Tiny n (q = n), p = k = 1, l = 0, no preconditioner."""
    A = W.laplacian_2d(4)      # n = 16
    X0 = W.start_block(A.n, 1, 3)
    ev, X, res, rc, info = lib.solve(h, dev_csr(lib, A), None, p=1, q=16, k=1, l=0, tol=1e-10, X0=X0,
                                     precond=lib.PRECOND_NONE)
    lam0 = 8 * math.sin(math.pi / 10) ** 2
    assert rc in (lib.OK, lib.BREAKDOWN)
    assert abs(ev[0] - lam0) <= 1e-10


def test_invalid_arguments_are_rejected(lib, h):
    A = W.laplacian_2d(10)
    Ad = dev_csr(lib, A)
    with pytest.raises(lib.TrplkError) as e:
        lib.solve(h, Ad, None, p=5, q=8, k=4, l=1)            # k < p
    assert e.value.code == lib.EINVAL
    with pytest.raises(lib.TrplkError) as e:
        lib.solve(h, Ad, None, p=2, q=6, k=4, l=2)            # q < k + l + 1
    assert e.value.code == lib.EINVAL
    bad = W.Csr(A.rowptr.copy(), A.col.copy(), A.val.copy())
    bad.col[5] = A.n + 3                                        # column out of range
    with pytest.raises(lib.TrplkError) as e:
        lib.solve(h, dev_csr(lib, bad), None, p=2, q=10, k=4, l=1)
    assert e.value.code == lib.EINVAL
    # the handle stays usable afterwards
    ev, X, res, rc, info = lib.solve(h, Ad, None, p=2, q=12, k=4, l=1, tol=1e-8)
    assert rc == lib.OK


def test_every_parameter_rule_is_enforced(lib, h):
    """Each rule of the solver's parameter check returns EINVAL with its own
    message and leaves the handle usable; so do row pointers that run
    backwards or past nnz (found by the device-side structure check)."""
    A = W.laplacian_2d(10)
    Ad = dev_csr(lib, A)
    cases = [
        (dict(p=2, q=12, k=4, l=1, tol=0.0), "tol"),
        (dict(p=2, q=12, k=4, l=-1), "l must be"),
        (dict(p=2, q=70, k=4, l=1), "q must be <= 64"),
        (dict(p=2, q=40, k=33, l=1), "k (thick-restart size)"),
        (dict(p=2, q=12, k=4, l=1, max_cycles=0), "max_cycles"),
        (dict(p=2, q=12, k=4, l=1, precond=99), "preconditioner"),
        (dict(p=2, q=12, k=4, l=1, locking=7), "locking"),
        (dict(p=2, q=12, k=4, l=1, block=5), "block"),
        (dict(p=2, q=8, k=4, l=2, block=3), "block"),
        (dict(p=2, q=12, k=4, l=1, block=2, locking=lib.LOCKING_HARD), "soft locking"),
        (dict(p=2, q=12, k=4, l=1, precision=5), "precision"),
        (dict(p=2, q=12, k=4, l=1, precond=lib.PRECOND_FSAI_LEARNED), "mlp_weights"),
        (dict(p=0, q=12, k=4, l=1), "need 1 <= p <= k"),
        (dict(p=5, q=12, k=4, l=1), "need 1 <= p <= k"),
        (dict(p=2, q=6, k=4, l=2), "need q >= k + max(l,1) + 1"),
        (dict(p=2, q=5, k=4, l=0), "need q >= k + max(l,1) + 1"),
    ]
    for kw, msg in cases:
        with pytest.raises(lib.TrplkError) as e:
            lib.solve(h, Ad, None, **kw)
        assert e.value.code == lib.EINVAL, kw
        assert msg in lib.trplk_last_error(h), (kw, lib.trplk_last_error(h))
    # q larger than n (n = 25), a pencil whose B has another n, and a wanted
    # end other than the smallest eigenvalues
    small = dev_csr(lib, W.laplacian_2d(5))
    other_n = dev_csr(lib, W.laplacian_2d(11))
    for args, kw, msg in [((small, None), dict(p=2, q=30, k=4, l=1), "q must be <= n"),
                          ((Ad, other_n), dict(p=2, q=12, k=4, l=1), "A and B differ")]:
        with pytest.raises(lib.TrplkError) as e:
            lib.solve(h, *args, **kw)
        assert e.value.code == lib.EINVAL and msg in lib.trplk_last_error(h), msg
    prm = lib.make_params(2, 12, 4, 1)
    prm.which = lib.SMALLEST + 1
    with pytest.raises(lib.TrplkError) as e:
        lib.trplk_solve(h, Ad, None, prm, None, np.zeros(2), np.zeros((2, 100)), np.zeros(2), lib.trplk_info())
    assert e.value.code == lib.EINVAL and "SMALLEST" in lib.trplk_last_error(h)
    for broken in ("backwards", "past_nnz"):
        rp = A.rowptr.copy()
        if broken == "backwards":
            rp[7] = rp[8] + 1
        else:
            rp[50] = A.nnz + 5
        bad = W.Csr(rp, A.col.copy(), A.val.copy())
        with pytest.raises(lib.TrplkError) as e:
            lib.solve(h, dev_csr(lib, bad), None, p=2, q=10, k=4, l=1)
        assert e.value.code == lib.EINVAL, broken
    ev, X, res, rc, info = lib.solve(h, Ad, None, p=2, q=12, k=4, l=1, tol=1e-8)
    assert rc == lib.OK


def test_host_inputs_and_outputs(lib, h):
    """The e2e form: host CSR and host outputs through trplk_solve."""
    A = W.laplacian_2d(30)
    hc = lib.make_csr(A.rowptr, A.col, A.val)
    ev, X, res, rc, info = lib.solve(h, hc, None, p=3, q=14, k=5, l=1, tol=1e-9)
    assert rc == lib.OK
    hgrid = math.pi / 62
    lam = np.sort([4 * math.sin(i * hgrid) ** 2 + 4 * math.sin(j * hgrid) ** 2
                   for i in range(1, 5) for j in range(1, 5)])[:3]
    assert np.allclose(ev, lam, rtol=1e-9)


# ---------------------------------------------------------------- full-size workloads
def _reference(name):
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "reference_runs.json")
    return json.load(open(path))[name]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_diffusion128_matches_oracle_full_run(lib, h, precision):
    """The 128^3 lognormal diffusion operator (n = 2,097,152) with the bench's
    settings (p = 10, q = 40, p_hat = 15, +K = 1, Jacobi, tol 1e-8, seed 0):
    eigenvalues against the oracle's converged full run (stored by
    oracle/reference_runs.py) to 1e-10 relative, residuals recomputed with the
    oracle's own matvec, B-orthonormality, and -- for the FP64 path -- the
    oracle's cycle count."""
    ref = _reference("diffusion128")
    A = W.diffusion_3d(128, W.lognormal_field(128, 1.0, 1))
    prec = lib.PRECISION_FP64 if precision == "fp64" else lib.PRECISION_MIXED
    ev, X, res, rc, info = lib.solve(h, dev_csr(lib, A), None, p=10, q=40, k=15, l=1, tol=1e-8, seed=0,
                                     precision=prec)
    assert rc == lib.OK
    refev = np.array(ref["evals"])
    rel = np.abs(ev - refev) / np.abs(refev)
    if precision == "fp64":
        # same arithmetic as the oracle up to rounding order: 1e-10 relative
        assert np.all(rel <= 1e-10), rel
    As = A.to_scipy()
    nA = O.norm1(As)
    r = np.linalg.norm(As @ X - X * ev, axis=0) / (nA * np.linalg.norm(X, axis=0))
    assert np.all(r <= 1e-8)
    if precision == "mixed":
        # another (FP32) trajectory to the same residual: each run's Ritz value
        # lies within the Kato-Temple bound ||r||^2 / gap of the eigenvalue
        # (unit vectors, ||r|| = relative residual x ||A||_1), gap = distance
        # to the nearest other computed eigenvalue; the pairs 8-10 are
        # clustered (gaps ~4e-6), where tol 1e-8 bounds the error only weakly
        # -- the tol 1e-12 comparison below holds them to 1e-10
        gap = np.array([np.min(np.abs(np.delete(refev, i) - refev[i])) for i in range(10)])
        bound = ((r * nA) ** 2 + (np.array(ref["resid"]) * nA) ** 2) / gap + 1e-10 * np.abs(refev)
        print("mixed path eigenvalue error vs oracle (relative):", rel.max(), "bound (relative):",
              (bound / np.abs(refev)).min(), "..", (bound / np.abs(refev)).max())
        assert np.all(np.abs(ev - refev) <= bound), (np.abs(ev - refev), bound)
    assert np.allclose(X.T @ X, np.eye(10), atol=1e-10)
    if precision == "fp64":
        assert info["cycles"] == ref["cycles"]
        assert info["mv_A"] == ref["mv_A"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_q1pencil96_matches_oracle_full_run(lib, h, precision):
    """The Q1 stiffness/mass pencil on 96^3 elements (n = 884,736, B != I) with
    the bench's settings (p = 20, q = 50, p_hat = 25, +K = 1, Jacobi, tol
    1e-8): eigenvalues against the oracle's converged full run, residuals
    recomputed with the oracle's matvecs, B-orthonormality; the FP64 path
    also reproduces the oracle's cycle and matvec counts."""
    ref = _reference("q1pencil96")
    N = 96
    A, B = W.fem_q1_pencil(N, np.random.default_rng(2).uniform(1.0, 10.0, (N, N, N)))
    prec = lib.PRECISION_FP64 if precision == "fp64" else lib.PRECISION_MIXED
    ev, X, res, rc, info = lib.solve(h, dev_csr(lib, A), dev_csr(lib, B), p=20, q=50, k=25, l=1, tol=1e-8, seed=0,
                                     precision=prec)
    assert rc == lib.OK
    refev = np.array(ref["evals"])
    rel = np.abs(ev - refev) / np.abs(refev)
    print(precision, "Q1 pencil eigenvalue error vs oracle (relative): max", rel.max())
    # FP64: the oracle's arithmetic up to rounding order; mixed: another
    # trajectory to the same residual, held to 1e-8 relative (see the 128^3 case)
    assert np.all(rel <= (1e-10 if precision == "fp64" else 1e-8)), rel
    As, Bs = A.to_scipy(), B.to_scipy()
    r = np.linalg.norm(As @ X - (Bs @ X) * ev, axis=0) / (O.norm1(As) * np.linalg.norm(X, axis=0))
    assert np.all(r <= 1e-8)
    assert np.allclose(X.T @ (Bs @ X), np.eye(20), atol=1e-10)
    if precision == "fp64":
        assert info["cycles"] == ref["cycles"]
        assert info["mv_A"] == ref["mv_A"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_chunglu22_matches_oracle_full_run(lib, h, precision):
    """L + 1e-3 I of the 2^22-vertex Chung-Lu graph's largest component
    (n = 4,117,504, nnz = 71,231,354; rows up to 8220 entries, so the hybrid
    SpMV with all three row classes runs) with the bench's settings (p = 16,
    q = 40, p_hat = 20, +K = 1, Jacobi, tol 1e-8): the smallest eigenvalue is
    the shift (constant vector on a connected graph), the others against the
    oracle's full run; the FP64 path also reproduces its cycle count."""
    ref = _reference("chunglu22")
    L = W.chung_lu_laplacian(1 << 22, 16.0, 2.1, 3)
    prec = lib.PRECISION_FP64 if precision == "fp64" else lib.PRECISION_MIXED
    ev, X, res, rc, info = lib.solve(h, dev_csr(lib, L), None, p=16, q=40, k=20, l=1, tol=1e-8, seed=0,
                                     precision=prec)
    assert rc == lib.OK
    Ls = L.to_scipy()
    nA = O.norm1(Ls)
    r = np.linalg.norm(Ls @ X - X * ev, axis=0) / (nA * np.linalg.norm(X, axis=0))
    assert np.all(r <= 1e-8)
    # constant eigenvector: |theta - 1e-3| <= ||r||^2 / gap (Kato-Temple), gap ~0.12
    assert abs(ev[0] - 1e-3) <= max((r[0] * nA) ** 2 / 0.1, 1e-14)
    refev = np.array(ref["evals"])
    rel = np.abs(ev - refev) / np.abs(refev)
    print(precision, "Chung-Lu eigenvalue error vs oracle (relative): max", rel.max())
    if precision == "fp64":
        # the oracle's arithmetic up to rounding order
        assert np.all(rel <= 1e-10), rel
    else:
        # another trajectory to the same residual.  Both Ritz values lie within
        # the Kato-Temple bound ||r||^2 / gap of the eigenvalue (unit vectors,
        # ||r|| = relative residual x ||A||_1 = up to 1.6e-4 here); the gap is
        # the distance to the nearest other computed eigenvalue (down to 2.2e-5
        # in the clusters, where the bound is weak and stated as such)
        gap = np.array([np.min(np.abs(np.delete(refev, i) - refev[i])) for i in range(16)])
        r_gpu = r * nA
        r_orc = np.array(ref["resid"]) * nA
        bound = (r_gpu ** 2 + r_orc ** 2) / gap + 1e-10 * np.abs(refev)
        print("Kato-Temple bound (relative):", (bound / np.abs(refev)).min(), "..", (bound / np.abs(refev)).max())
        assert np.all(np.abs(ev - refev) <= bound), (np.abs(ev - refev), bound)
    assert np.allclose(X.T @ X, np.eye(16), atol=1e-10)
    if precision == "fp64":
        assert info["cycles"] == ref["cycles"]
        assert info["mv_A"] == ref["mv_A"]


@pytest.mark.parametrize("path", ["fp64-jacobi", "mixed-learned-fsai"])
def test_full_size_aniso128_matches_oracle_full_run(lib, h, path):
    """Anisotropic 7-point diffusion on 128^3 (n = 2,097,152, held-out seed 2000)
    with the bench's settings (p = 20, q = 50, p_hat = 25, +K = 1, tol 1e-8).
    FP64 with Jacobi: the oracle's arithmetic up to rounding order -- its
    eigenvalues to 1e-10 relative and its cycle count.  Mixed with the learned
    FSAI preconditioner (trained on twelve 32^3 operators of the family): the
    preconditioner changes the trajectory, not the eigenpairs, so eigenvalues
    agree within the Kato-Temple bound of both runs' residuals."""
    ref = _reference("aniso128")
    A = W.anisotropic_diffusion(128, 2000)
    kw = dict(p=20, q=50, k=25, l=1, tol=1e-8, seed=0)
    if path == "fp64-jacobi":
        ev, X, res, rc, info = lib.solve(h, dev_csr(lib, A), None, precision=lib.PRECISION_FP64, **kw)
    else:
        ops = [dev_csr(lib, W.anisotropic_diffusion(32, s)) for s in range(1000, 1012)]
        w = lib.trplk_fsai_mlp_init(0)
        tp = lib.trplk_train_params(iters=240, lr=2e-3, vectors=8, harvest_cycles=6, q=24, k=10, l=1, seed=5, bf16=1,
                                    gamma=0.1)
        lib.trplk_fsai_train(h, ops, [(32, 32, 32)] * 12, tp, w)
        ev, X, res, rc, info = lib.solve(h, dev_csr(lib, A), None, precision=lib.PRECISION_MIXED,
                                         precond=lib.PRECOND_FSAI_LEARNED, mlp_weights=w, grid=(128, 128, 128),
                                         mlp_bf16=1, **kw)
    assert rc == lib.OK
    As = A.to_scipy()
    nA = O.norm1(As)
    r = np.linalg.norm(As @ X - X * ev, axis=0) / (nA * np.linalg.norm(X, axis=0))
    assert np.all(r <= 1e-8)
    assert np.allclose(X.T @ X, np.eye(20), atol=1e-10)
    refev = np.array(ref["evals"])
    rel = np.abs(ev - refev) / np.abs(refev)
    print(path, "anisotropic 128^3 eigenvalue error vs oracle (relative): max", rel.max(), "matvecs", info["mv_A"])
    if path == "fp64-jacobi":
        assert np.all(rel <= 1e-10), rel
        assert info["cycles"] == ref["cycles"]
    else:
        gap = np.array([np.min(np.abs(np.delete(refev, i) - refev[i])) for i in range(20)])
        bound = ((r * nA) ** 2 + (np.array(ref["resid"]) * nA) ** 2) / gap + 1e-10 * np.abs(refev)
        assert np.all(np.abs(ev - refev) <= bound), (np.abs(ev - refev), bound)


def test_full_size_chunglu22_mixed_at_tol_1e12_matches_oracle(lib, h):
    """The mixed path on the 2^22-vertex Chung-Lu operator at tol 1e-12 against
    the oracle's run at tol 1e-12: there the Kato-Temple bound of the clustered
    pairs, (1e-12 ||A||_1)^2 / 2e-5 ~ 1e-11, is below 1e-10 relative, so the
    eigenvalues compare at 1e-10."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "reference_runs.json")
    runs = json.load(open(path))
    if "chunglu22_tight" not in runs:
        pytest.skip("the oracle's tol 1e-12 run is not stored")
    ref = runs["chunglu22_tight"]
    L = W.chung_lu_laplacian(1 << 22, 16.0, 2.1, 3)
    ev, X, res, rc, info = lib.solve(h, dev_csr(lib, L), None, p=16, q=40, k=20, l=1, tol=1e-12, seed=0,
                                     precision=lib.PRECISION_MIXED)
    assert rc == lib.OK
    assert np.all(res <= 1e-12)
    refev = np.array(ref["evals"])
    rel = np.abs(ev - refev) / np.abs(refev)
    print("mixed Chung-Lu at tol 1e-12: eigenvalue error vs oracle (relative): max", rel.max())
    assert np.all(rel <= 1e-10), rel


def test_full_size_diffusion128_mixed_at_tol_1e12_matches_oracle(lib, h):
    """The mixed path on the 128^3 lognormal diffusion operator at tol 1e-12
    against the oracle's run at tol 1e-12: there the Kato-Temple bound of the
    clustered pairs, (1e-12 ||A||_1)^2 / 4e-6, is far below 1e-10 relative,
    so the eigenvalues of the two runs compare at 1e-10."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "reference_runs.json")
    runs = json.load(open(path))
    if "diffusion128_tight" not in runs:
        pytest.skip("the oracle's tol 1e-12 run is not stored")
    ref = runs["diffusion128_tight"]
    A = W.diffusion_3d(128, W.lognormal_field(128, 1.0, 1))
    ev, X, res, rc, info = lib.solve(h, dev_csr(lib, A), None, p=10, q=40, k=15, l=1, tol=1e-12, seed=0,
                                     precision=lib.PRECISION_MIXED)
    assert rc == lib.OK
    assert np.all(res <= 1e-12)
    refev = np.array(ref["evals"])
    rel = np.abs(ev - refev) / np.abs(refev)
    print("mixed 128^3 diffusion at tol 1e-12: eigenvalue error vs oracle (relative): max", rel.max())
    assert np.all(rel <= 1e-10), rel


def _lap3d_eigs(N, count):
    s = 4 * np.sin(np.arange(1, N + 1) * np.pi / (2 * (N + 1))) ** 2
    return np.sort((s[:, None, None] + s[None, :, None] + s[None, None, :]).ravel())[:count]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_closed_forms(lib, h, precision):
    """The full-size 128^3 diffusion operator with all coefficients 1 (the 3D
    Laplacian, n = 2,097,152; the wanted 10 end with a complete triple) at tol
    1e-10: each computed eigenvalue lies within the Kato-Temple bound
    ||r||^2 / gap of its closed form (r the recomputed residual of the returned
    unit vector, gap the distance to the nearest distinct eigenvalue) plus the
    FP64 rounding floor of a Ritz value, 64 u ||A||_1 (u = 2^-52), and within
    1e-10 relative."""
    prec = lib.PRECISION_FP64 if precision == "fp64" else lib.PRECISION_MIXED
    A = W.diffusion_3d(128)
    lam_all = _lap3d_eigs(128, 11)
    p = 10
    ev, X, res, rc, info = lib.solve(h, dev_csr(lib, A), None, p=p, q=40, k=15, l=1, tol=1e-10, seed=0,
                                     precision=prec)
    assert rc == lib.OK
    lam = lam_all[:p]
    uniq = np.unique(np.round(lam_all, 12))
    gap = np.array([np.min(np.abs(uniq[np.abs(uniq - x) > 1e-9 * x] - x)) for x in lam])
    As = A.to_scipy()
    R = As @ X - X * ev
    r2 = np.sum(R * R, axis=0) / np.sum(X * X, axis=0)
    err = np.abs(ev - lam)
    floor = 64 * 2.0 ** -52 * O.norm1(As)
    print(precision, "closed-form error (relative): max", (err / lam).max(), "absolute max", err.max(),
          "rounding floor", floor)
    assert np.all(err <= r2 / gap + floor)
    assert np.all(err <= 1e-10 * lam)


# ---------------------------------------------------------------- hard locking and M(rho_i)
@pytest.mark.parametrize("case", ["lap2d", "pencil"])
def test_hard_locking_matches_oracle(lib, h, case):
    """Hard locking (locked vectors at the front of the basis, T and the
    Rayleigh-Ritz step on the active columns) against the oracle's hard
    locking: the FP64 path follows its arithmetic, so cycles, matvecs and the
    number of locked pairs agree exactly and the eigenvalues to 1e-10; the
    vectors come back ascending and B-orthonormal."""
    if case == "lap2d":
        A, B = W.laplacian_2d(30), None
        p, q, k, l = 5, 16, 7, 1
    else:
        A, B = W.fem_q1_pencil(6, np.random.default_rng(3).uniform(1, 10, (6, 6, 6)))
        p, q, k, l = 4, 16, 6, 2
    As = A.to_scipy()
    Bs = None if B is None else B.to_scipy()
    X0 = W.start_block(A.n, k, 1)
    ref = O.solve(As, Bs, p, q, k, l, 1e-10, X0, "jacobi", locking="hard")
    ev, X, res, rc, info = lib.solve(h, dev_csr(lib, A), None if B is None else dev_csr(lib, B), p=p, q=q, k=k,
                                     l=l, tol=1e-10, X0=X0, locking=lib.LOCKING_HARD)
    assert rc == lib.OK and ref["status"] == O.OK
    assert info["cycles"] == ref["cycles"] and info["mv_A"] == ref["mv_A"] and info["locked"] == ref["locked"] == p
    assert np.all(np.abs(ev - ref["evals"]) <= 1e-10 * np.abs(ref["evals"]))
    assert np.all(np.diff(ev) >= 0) and np.all(res <= 1e-10)
    G = X.T @ (X if Bs is None else Bs @ X)
    assert np.allclose(G, np.eye(p), atol=1e-10)


def test_hard_locking_mixed_path(lib, h):
    """The mixed path locks in its FP32 phase and polishes all p pairs in
    FP64: same eigenvalues as the oracle's hard-locking run within the
    Kato-Temple bound of both runs' residuals (another trajectory)."""
    A = W.diffusion_3d(14, W.lognormal_field(14, 1.0, 2))
    As = A.to_scipy()
    p, q, k, l = 6, 20, 8, 1
    X0 = W.start_block(A.n, k, 3)
    ref = O.solve(As, None, p, q, k, l, 1e-10, X0, "jacobi", locking="hard")
    ev, X, res, rc, info = lib.solve(h, dev_csr(lib, A), None, p=p, q=q, k=k, l=l, tol=1e-10, X0=X0,
                                     precision=lib.PRECISION_MIXED, locking=lib.LOCKING_HARD)
    assert rc == lib.OK and info["locked"] >= 1
    nA = O.norm1(As)
    refev = ref["evals"]
    gap = np.array([np.min(np.abs(np.delete(refev, i) - refev[i])) for i in range(p)])
    bound = ((res * nA) ** 2 + (ref["resid"] * nA) ** 2) / gap + 1e-10 * np.abs(refev)
    assert np.all(np.abs(ev - refev) <= bound)
    assert np.all(np.abs(ev - refev) <= 1e-10 * np.abs(refev))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_shifted_jacobi_matches_oracle(lib, h, precision):
    """The per-cycle preconditioner M_i = diag(A - rho_i B)^-1 (floored at
    1e-3 a_jj), rebuilt on the device every cycle from that cycle's shift:
    FP64 follows the oracle's cycles exactly and its eigenvalues to 1e-10;
    the mixed path reaches the same eigenvalues."""
    A = W.diffusion_3d(12, W.lognormal_field(12, 1.0, 5))
    As = A.to_scipy()
    p, q, k, l = 5, 18, 7, 1
    X0 = W.start_block(A.n, k, 2)
    ref = O.solve(As, None, p, q, k, l, 1e-10, X0, "jacobi_shifted")
    prec = lib.PRECISION_FP64 if precision == "fp64" else lib.PRECISION_MIXED
    ev, X, res, rc, info = lib.solve(h, dev_csr(lib, A), None, p=p, q=q, k=k, l=l, tol=1e-10, X0=X0,
                                     precond=lib.PRECOND_JACOBI_SHIFTED, precision=prec)
    assert rc == lib.OK and ref["status"] == O.OK
    assert np.all(np.abs(ev - ref["evals"]) <= 1e-10 * np.abs(ref["evals"]))
    if precision == "fp64":
        assert info["cycles"] == ref["cycles"] and info["mv_A"] == ref["mv_A"]


# ---------------------------------------------------------------- block TRPL+K
@pytest.mark.parametrize("b", [2, 3])
@pytest.mark.parametrize("case", ["c1", "pencil"])
def test_block_trplk_matches_oracle(lib, h, case, b):
    """Block TRPL+K (b targets per cycle, columns cycling through the b
    sequences) against the oracle's block form: C1 at full size (the 2D
    Laplacian on 100 x 100) and a Q1 stiffness/mass pencil, FP64 path --
    eigenvalues to 1e-10, residuals, B-orthonormality and the matvec
    accounting p_hat + (q - p_hat) cycles; cycle counts equal where the wanted
    eigenvalues are simple (the pencil), within 15% where the wanted set holds
    exactly degenerate pairs (C1), whose in-space Ritz vectors depend on
    rounding order."""
    if case == "c1":
        A, B = W.laplacian_2d(100), None
        p, q, k, l = 5, 20, 8, 5
    else:
        A, B = W.fem_q1_pencil(12, np.random.default_rng(3).uniform(1, 10, (12, 12, 12)))
        p, q, k, l = 6, 24, 9, 1
    if k + b + l > q:
        l = q - k - b
    As = A.to_scipy()
    Bs = None if B is None else B.to_scipy()
    X0 = W.start_block(A.n, k, 0)
    ref = O.solve(As, Bs, p, q, k, l, 1e-8, X0, "jacobi", block=b)
    ev, X, res, rc, info = lib.solve(h, dev_csr(lib, A), None if B is None else dev_csr(lib, B), p=p, q=q, k=k, l=l,
                                     tol=1e-8, X0=X0, block=b)
    assert rc == lib.OK and ref["status"] == O.OK
    print(case, "b =", b, "cycles GPU / oracle", info["cycles"], ref["cycles"])
    assert np.all(np.abs(ev - ref["evals"]) <= 1e-10 * np.abs(ref["evals"])), np.abs(ev - ref["evals"])
    assert np.all(res <= 1e-8)
    G = X.T @ (X if Bs is None else Bs @ X)
    assert np.allclose(G, np.eye(p), atol=1e-10)
    assert info["mv_A"] == k + (q - k) * info["cycles"]
    if case == "pencil":
        assert info["cycles"] == ref["cycles"] and info["mv_A"] == ref["mv_A"]
    else:
        assert abs(info["cycles"] - ref["cycles"]) <= 0.15 * ref["cycles"]


def test_block_trplk_mixed_path(lib, h):
    """The mixed path with b = 2 (FP32 phase in blocks, FP64 refinement)
    reaches the oracle's eigenvalues on a lognormal diffusion operator."""
    A = W.diffusion_3d(16, W.lognormal_field(16, 1.0, 4))
    As = A.to_scipy()
    p, q, k, l = 6, 22, 8, 1
    X0 = W.start_block(A.n, k, 1)
    ref = O.solve(As, None, p, q, k, l, 1e-10, X0, "jacobi", block=2)
    ev, X, res, rc, info = lib.solve(h, dev_csr(lib, A), None, p=p, q=q, k=k, l=l, tol=1e-10, X0=X0, block=2,
                                     precision=lib.PRECISION_MIXED)
    assert rc == lib.OK and ref["status"] == O.OK
    assert np.all(np.abs(ev - ref["evals"]) <= 1e-10 * np.abs(ref["evals"]))
