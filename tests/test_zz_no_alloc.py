"""GPU test of trplk_project_noalloc, the projection entry point that
allocates no device memory (for callers whose device memory is fully planned
by their own pool, or whose hot loop cannot take an allocation's device
synchronisation).  It must give the same coefficients as trplk_project,
within the tolerance of the projection tests, on two calls in a row (the
second call reuses the scratch the first one left behind).  Collected last on
purpose; runs alone in a fresh process too."""
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


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_projection_matches_handle_projection_twice(lib, dtype):
    tdt = torch.float64 if dtype == "f64" else torch.float32
    code = lib.F64 if dtype == "f64" else lib.F32
    h = lib.Handle(0)
    try:
        # 300,000 rows: more tiles than the 256 CTAs the scratch holds
        for call, (n, w, seed) in enumerate([(300_000, 37, 1), (2_000, 64, 2)]):
            ld = (n + 255) // 256 * 256
            g = torch.Generator().manual_seed(seed)
            BU = torch.zeros((w, ld), dtype=torch.float64)
            BU[:, :n] = torch.randn((w, n), generator=g, dtype=torch.float64)
            v = torch.zeros(ld, dtype=torch.float64)
            v[:n] = torch.randn(n, generator=g, dtype=torch.float64)
            BUd, vd = BU.to(tdt).cuda(), v.to(tdt).cuda()
            ref = torch.zeros(w, dtype=torch.float64, device="cuda")
            got = torch.full((w,), float("nan"), dtype=torch.float64, device="cuda")
            lib.trplk_project(h, code, n, ld, w, BUd, vd, ref)
            lib.trplk_project_noalloc(code, n, ld, w, BUd, vd, got, None)
            torch.cuda.synchronize()
            tol = 1e-13 * math.sqrt(n)   # projection tolerance of the parity tests
            assert np.allclose(got.cpu().numpy(), ref.cpu().numpy(), rtol=0, atol=tol), call
    finally:
        h.close()


def test_noalloc_rejects_oversized_basis(lib):
    x = torch.zeros(256, dtype=torch.float64, device="cuda")
    out = torch.zeros(65, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.TrplkError) as e:
        lib.trplk_project_noalloc(lib.F64, 256, 256, 65, x, x, out, None)
    assert e.value.code == lib.EINVAL
