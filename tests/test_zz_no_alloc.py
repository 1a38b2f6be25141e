"""GPU test of trplk_project_noalloc, the projection entry point that
allocates no device memory.  It exists for callers that cannot let a library
call cudaMalloc: processes whose own pool has already planned all device
memory (an allocation would fail or break the plan) and latency-critical loops
that cannot take the device synchronisation an allocation may cause.

Checked here: on two calls in a row (the second reuses the scratch array the
first left behind) it gives the coefficients of trplk_project, within the
tolerance of the projection tests, and of the definition BU^T v evaluated in
FP64 numpy; it does the same on a non-default stream; once warmed up, a call
leaves the device's free memory unchanged; a basis wider than the limit is
rejected.  Collected last on purpose; runs alone in a fresh process too."""
import math

import numpy as np
import pytest

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


def _inputs(n, w, seed, tdt):
    ld = (n + 255) // 256 * 256
    g = torch.Generator().manual_seed(seed)
    BU = torch.zeros((w, ld), dtype=torch.float64)
    BU[:, :n] = torch.randn((w, n), generator=g, dtype=torch.float64)
    v = torch.zeros(ld, dtype=torch.float64)
    v[:n] = torch.randn(n, generator=g, dtype=torch.float64)
    BU, v = BU.to(tdt), v.to(tdt)
    # the definition on the stored (possibly FP32) values, in FP64
    ref = BU[:, :n].double().numpy() @ v[:n].double().numpy()
    mag = np.abs(BU[:, :n].double().numpy()) @ np.abs(v[:n].double().numpy())
    return ld, BU.cuda(), v.cuda(), ref, mag


def _tol(dtype, n, mag):
    # FP64: rounding order, 1e-13 sqrt(n) (the projection tests' tolerance);
    # FP32: the compensated sum's bound 4u sum |b v|, u = 2^-24
    return 1e-13 * math.sqrt(n) if dtype == "f64" else 4 * 2.0 ** -24 * mag + 1e-13


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_projection_matches_handle_projection_twice(lib, dtype):
    tdt = torch.float64 if dtype == "f64" else torch.float32
    code = lib.F64 if dtype == "f64" else lib.F32
    h = lib.Handle(0)
    try:
        # 300,000 rows: more tiles than the 256 CTAs the scratch holds; the
        # widths reach every instantiation (w <= 32, <= 48, <= 64)
        for call, (n, w, seed) in enumerate([(300_000, 37, 1), (2_000, 64, 2), (70_001, 5, 3)]):
            ld, BUd, vd, ref, mag = _inputs(n, w, seed, tdt)
            base = torch.zeros(w, dtype=torch.float64, device="cuda")
            got = torch.full((w,), float("nan"), dtype=torch.float64, device="cuda")
            lib.trplk_project(h, code, n, ld, w, BUd, vd, base)
            lib.trplk_project_noalloc(code, n, ld, w, BUd, vd, got, None)
            torch.cuda.synchronize()
            g, b = got.cpu().numpy(), base.cpu().numpy()
            tol = _tol(dtype, n, mag)
            assert np.all(np.abs(g - b) <= tol), (call, np.abs(g - b).max())
            assert np.all(np.abs(g - ref) <= tol), (call, np.abs(g - ref).max())
    finally:
        h.close()


def test_noalloc_on_a_side_stream_and_without_allocating(lib):
    n, w = 123_457, 40
    ld, BUd, vd, ref, mag = _inputs(n, w, 11, torch.float32)
    out = torch.full((w,), float("nan"), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    # first call on this stream, width class and dtype: may load code
    lib.trplk_project_noalloc(lib.F32, n, ld, w, BUd, vd, out, s.cuda_stream)
    s.synchronize()
    assert np.all(np.abs(out.cpu().numpy() - ref) <= _tol("f32", n, mag))
    out.fill_(float("nan"))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    lib.trplk_project_noalloc(lib.F32, n, ld, w, BUd, vd, out, s.cuda_stream)
    s.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert np.all(np.abs(out.cpu().numpy() - ref) <= _tol("f32", n, mag))


def test_noalloc_rejects_oversized_basis(lib):
    x = torch.zeros(256, dtype=torch.float64, device="cuda")
    out = torch.zeros(65, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.TrplkError) as e:
        lib.trplk_project_noalloc(lib.F64, 256, 256, 65, x, x, out, None)
    assert e.value.code == lib.EINVAL
