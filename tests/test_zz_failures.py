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
