"""Failure detection, driven from the host (no GPU fault, trap or hang): a NaN
in A's values, an indefinite B, and too few cycles.  Each returns its status
code through the C ABI and leaves the handle usable."""
import numpy as np
import pytest

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


def dev_csr(lib, A):
    return lib.make_csr(torch.from_numpy(A.rowptr).cuda(), torch.from_numpy(A.col).cuda(),
                        torch.from_numpy(A.val).cuda())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nan_in_matrix_returns_nan_status(lib, h, precision):
    A = W.laplacian_2d(20)
    bad = W.Csr(A.rowptr.copy(), A.col.copy(), A.val.copy())
    bad.val[7] = np.nan
    prec = lib.PRECISION_FP64 if precision == "fp64" else lib.PRECISION_MIXED
    with pytest.raises(lib.TrplkError) as e:
        lib.solve(h, dev_csr(lib, bad), None, p=2, q=12, k=4, l=1, tol=1e-8, precision=prec)
    assert e.value.code == lib.NAN
    ev, X, res, rc, info = lib.solve(h, dev_csr(lib, A), None, p=2, q=12, k=4, l=1, tol=1e-8, precision=prec)
    assert rc == lib.OK


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_indefinite_b_returns_not_spd(lib, h, precision):
    A = W.laplacian_2d(20)
    n = A.n
    B = W.Csr(np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), -np.ones(n))
    prec = lib.PRECISION_FP64 if precision == "fp64" else lib.PRECISION_MIXED
    with pytest.raises(lib.TrplkError) as e:
        lib.solve(h, dev_csr(lib, A), dev_csr(lib, B), p=2, q=12, k=4, l=1, tol=1e-8, precision=prec)
    assert e.value.code == lib.NOT_SPD_B


def test_max_cycles_returns_not_converged_with_best_pairs(lib, h):
    A = W.laplacian_2d(30)
    ev, X, res, rc, info = lib.solve(h, dev_csr(lib, A), None, p=3, q=14, k=5, l=1, tol=1e-12, max_cycles=2)
    assert rc == lib.NOT_CONVERGED
    assert info["cycles"] == 2 and info["nconv"] < 3
    assert np.all(np.isfinite(ev)) and np.all(np.diff(ev) >= 0) and np.all(np.isfinite(res))
    assert np.allclose(X.T @ X, np.eye(3), atol=1e-10)


def test_wait_timeout_returns_etimeout_and_the_handle_recovers(lib, h):
    """The bounded waits of the streaming passes, made to run out on purpose:
    with the handle's wait limit at 0 polls every mbarrier wait gives up at
    once.  The pass must agree on it across the CTA (the update-and-project
    pass meets at a named barrier every tile), wait for the bulk copies it
    already issued, return TRPLK_ETIMEOUT through the status word -- never a
    hang or a fault -- and leave the handle usable: the same calls with the
    default limit then give the definition's answers and a solve converges."""
    n = 300_000   # 1172 FP32 tiles: more than the CTAs, several stages in flight per CTA
    ld = (n + 255) // 256 * 256
    w = 20
    rng = np.random.default_rng(5)
    U = np.linalg.qr(rng.standard_normal((n, w)))[0]
    v = rng.standard_normal(n)
    Ud = torch.zeros((w, ld), dtype=torch.float32, device="cuda")
    Ud[:, :n] = torch.from_numpy(np.ascontiguousarray(U.T)).float().cuda()
    vd = torch.zeros(ld, dtype=torch.float32, device="cuda")
    vd[:n] = torch.from_numpy(v).float().cuda()
    hout = torch.zeros(w, dtype=torch.float64, device="cuda")
    beta = torch.zeros(2, dtype=torch.float64, device="cuda")
    A = W.laplacian_2d(40)
    lib.trplk_set_wait_limit(h, 0)
    try:
        with pytest.raises(lib.TrplkError) as e:
            lib.trplk_project(h, lib.F32, n, ld, w, Ud, vd, hout)
        assert e.value.code == lib.ETIMEOUT
        with pytest.raises(lib.TrplkError) as e:      # update + projection, then update + norm
            lib.trplk_cgs2(h, lib.F32, n, ld, w, Ud, Ud, None, hout, vd.clone(), None, beta)
        assert e.value.code == lib.ETIMEOUT
        for precision in (lib.PRECISION_FP64, lib.PRECISION_MIXED):
            with pytest.raises(lib.TrplkError) as e:
                lib.solve(h, dev_csr(lib, A), None, p=2, q=12, k=4, l=1, tol=1e-8, precision=precision)
            assert e.value.code == lib.ETIMEOUT
            assert "gave up" in lib.trplk_last_error(h)
    finally:
        lib.trplk_set_wait_limit(h, -1)
    lib.trplk_project(h, lib.F32, n, ld, w, Ud, vd, hout)
    Uf = Ud[:, :n].double().cpu().numpy()
    vf = vd[:n].double().cpu().numpy()
    ref = Uf @ vf
    mag = np.abs(Uf) @ np.abs(vf)
    assert np.all(np.abs(hout.cpu().numpy() - ref) <= 4 * 2.0 ** -24 * mag + 1e-13)
    ev, X, res, rc, info = lib.solve(h, dev_csr(lib, A), None, p=2, q=12, k=4, l=1, tol=1e-8,
                                     precision=lib.PRECISION_MIXED)
    assert rc == lib.OK and np.all(res <= 1e-8)


def test_tensor_core_rotation_timeout_returns_etimeout_and_recovers(lib, h):
    """The tensor-core rotation's bounded waits made to run out (wait limit 0):
    every warp role gives up at its first wait, the CTA agrees on it through
    shared memory, waits for the tensor copies its producer already issued,
    frees its tensor memory and reports TRPLK_ETIMEOUT -- no hang, no fault --
    and the same call with the default limit then gives U Y."""
    n, w, k = 300_000, 40, 20
    ld = (n + 255) // 256 * 256
    rng = np.random.default_rng(9)
    U = rng.standard_normal((n, w)) / np.sqrt(n)
    Yc = np.linalg.qr(rng.standard_normal((w, w)))[0]
    Ud = torch.zeros((w, ld), dtype=torch.float32, device="cuda")
    Ud[:, :n] = torch.from_numpy(np.ascontiguousarray(U.T)).float().cuda()
    Yd = torch.from_numpy(Yc.ravel(order="F")).cuda()
    X = torch.zeros((k, ld), dtype=torch.float32, device="cuda")
    lib.trplk_set_wait_limit(h, 0)
    try:
        with pytest.raises(lib.TrplkError) as e:
            lib.trplk_rotate_tc(h, n, ld, w, k, Ud, Yd, w, X)
        assert e.value.code == lib.ETIMEOUT
    finally:
        lib.trplk_set_wait_limit(h, -1)
    lib.trplk_rotate_tc(h, n, ld, w, k, Ud, Yd, w, X)
    Uq = Ud[:, :n].double().cpu().numpy().T
    ref = Uq @ Yc[:, :k]
    assert np.abs(X.cpu().numpy()[:, :n].T - ref).max() <= 2e-6 * np.abs(Uq).max() * np.sqrt(w)
