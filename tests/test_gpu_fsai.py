"""Parity of the FSAI preconditioner kernels (classical and learned), the
training loss and its gradient, FSAI-preconditioned solves, and the gain of
the trained network over the unpreconditioned-by-learning (Jacobi) method.

Tolerances: classical FSAI and M x in FP64 to 1e-12 relative; the MLP in its
FP32 mode (FP32 weights, activations and accumulation) against the FP64
oracle to 2e-4 relative, the BF16 mode to 3e-2 (BF16 keeps 8 mantissa bits);
loss 1e-5 and weight gradients 2e-3 relative to their largest entry (FP32
forward/backward); converged eigenvalues 1e-10."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fsai as F
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


def dcsr(lib, A):
    return lib.make_csr(torch.from_numpy(A.rowptr).cuda(), torch.from_numpy(A.col).cuda(),
                        torch.from_numpy(A.val).cuda())


def aniso(N, seed):
    return W.anisotropic_diffusion(N, seed)


def random_mlp(seed, scale=0.3):
    p = F.init_mlp(seed)
    rng = np.random.default_rng(seed + 1)
    p["W3"] = scale * rng.standard_normal(p["W3"].shape)
    p["b3"] = p["b3"] + 0.1 * rng.standard_normal(7)
    return p


def test_classical_fsai_values_match_oracle(lib, h):
    for A in (aniso(11, 3), W.fem_q1_pencil(6, np.random.default_rng(1).uniform(1, 10, (6, 6, 6)))[0]):
        As = A.to_scipy()
        Gref = F.classical_fsai(As)
        nnz = lib.trplk_fsai_values(h, dcsr(lib, A), 0)
        assert nnz == Gref.nnz
        g = torch.zeros(nnz, dtype=torch.float64, device="cuda")
        lib.trplk_fsai_values(h, dcsr(lib, A), 0, g=g)
        assert np.allclose(g.cpu().numpy(), Gref.data, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("bf16,tol", [(0, 2e-4), (1, 3e-2)])
def test_learned_fsai_values_match_oracle(lib, h, bf16, tol):
    N = 9
    A = aniso(N, 5)
    As = A.to_scipy()
    p = random_mlp(2)
    o, _ = F.mlp_forward(p, F.features_7pt(As, (N, N, N)))
    Gref = F.g_from_outputs(As, (N, N, N), o)
    w = lib.pack_mlp(p)
    nnz = lib.trplk_fsai_values(h, dcsr(lib, A), 1, (N, N, N), w, bf16)
    g = torch.zeros(nnz, dtype=torch.float64, device="cuda")
    lib.trplk_fsai_values(h, dcsr(lib, A), 1, (N, N, N), w, bf16, g)
    got = g.cpu().numpy()
    assert np.all(np.abs(got - Gref.data) <= tol * np.abs(Gref.data).max())


def test_fsai_apply_matches_oracle(lib, h):
    A = aniso(10, 8)
    As = A.to_scipy()
    G = F.classical_fsai(As)
    x = np.random.default_rng(3).standard_normal(A.n)
    y = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    lib.trplk_fsai_apply(h, dcsr(lib, A), torch.from_numpy(G.data).cuda(), torch.from_numpy(x).cuda(), y)
    ref = F.apply_M(G, x)
    assert np.allclose(y.cpu().numpy(), ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())


@pytest.mark.parametrize("bf16", [0, 1])
def test_loss_and_gradient_match_oracle(lib, h, bf16):
    """Training loss and its gradient against the oracle (F5; F6 for BF16).
    FP32 mode against the FP64 oracle: loss 1e-5, gradient 2e-3 of its largest
    entry.  BF16 mode (the mode training runs in) against the oracle's BF16
    mode, which rounds the same quantities at the same points (features,
    W1..W3, both hidden activations) and computes the rest in FP64: the two
    differ by FP32 against FP64 accumulation (sums of <= 64 terms, ~1e-6
    relative) and by the rare bfloat16 rounding decisions that this moves
    across a tie (one activation by 2^-8 relative, out of n x 128); held to
    1e-5 on the loss and 1e-3 of the largest entry on the gradient.  The
    gradient must also differ from the FP64 oracle's by less than its own
    bfloat16 rounding allows (0.1 of the largest entry)."""
    N = 8
    A = aniso(N, 9)
    As = A.to_scipy()
    p = random_mlp(4, 0.2)
    V = np.random.default_rng(6).standard_normal((A.n, 3))
    Lref, gref, parts = F.loss_and_grad_mlp(p, As, (N, N, N), V, quant="bf16" if bf16 else None)
    Vd = torch.from_numpy(np.ascontiguousarray(V.T)).cuda()        # column-major n x nv
    loss, grad = lib.trplk_fsai_loss_grad(h, dcsr(lib, A), (N, N, N), lib.pack_mlp(p), bf16, Vd, 3, F.GAMMA)
    assert abs(loss[0] - Lref) <= 1e-5 * abs(Lref)
    assert abs(loss[1] - parts["E"]) <= 1e-5 * abs(parts["E"])
    assert abs(loss[2] - parts["K"]) <= 1e-5 * max(1.0, abs(parts["K"]))
    gr = lib.pack_mlp(gref).astype(np.float64)
    err = np.abs(grad - gr).max() / np.abs(gr).max()
    print("bf16" if bf16 else "fp32", "mode: gradient error / largest entry", err)
    assert err <= (1e-3 if bf16 else 2e-3)
    if bf16:
        g64 = lib.pack_mlp(F.loss_and_grad_mlp(p, As, (N, N, N), V)[1]).astype(np.float64)
        assert np.abs(grad - g64).max() <= 0.1 * np.abs(g64).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_classical_fsai_solve_matches_oracle(lib, h, precision):
    N = 12
    A = aniso(N, 11)
    As = A.to_scipy()
    G = F.classical_fsai(As)
    p, q, k, l = 4, 18, 6, 1
    X0 = W.start_block(A.n, k, 1)
    ref = O.solve(As, None, p, q, k, l, 1e-10, X0, lambda v: F.apply_M(G, v))
    prec = lib.PRECISION_FP64 if precision == "fp64" else lib.PRECISION_MIXED
    ev, X, res, rc, info = lib.solve(h, dcsr(lib, A), None, p=p, q=q, k=k, l=l, tol=1e-10, X0=X0,
                                     precond=lib.PRECOND_FSAI, precision=prec)
    assert rc == lib.OK and ref["status"] == O.OK
    assert np.all(np.abs(ev - ref["evals"]) <= 1e-10 * np.abs(ref["evals"]))
    if precision == "fp64":
        assert info["cycles"] == ref["cycles"]


def test_training_reduces_loss_and_learned_fsai_beats_jacobi(lib, h):
    """Train on 12 anisotropic operators (24^3), test on 2 held-out ones: the
    loss falls, and the learned preconditioner needs fewer matvecs than Jacobi
    to the same tolerance (the gain of the network over the method without it)."""
    N = 24
    train = [aniso(N, 1000 + s) for s in range(12)]
    held = [aniso(N, 2000 + s) for s in range(2)]
    ops = [dcsr(lib, A) for A in train]
    w = lib.pack_mlp(F.init_mlp(0))
    tp = lib.trplk_train_params(iters=240, lr=2e-3, vectors=8, harvest_cycles=6, q=24, k=10, l=1, seed=5, bf16=1,
                                gamma=0.1)
    losses = lib.trplk_fsai_train(h, ops, [(N, N, N)] * 12, tp, w)
    first, last = losses[:12].mean(), losses[-12:].mean()
    print("training loss", first, "->", last)
    assert last < first
    gains = []
    for A in held:
        kw = dict(p=6, q=24, k=10, l=1, tol=1e-8, seed=0, precision=lib.PRECISION_MIXED)
        _, _, rj, rcj, ij = lib.solve(h, dcsr(lib, A), None, precond=lib.PRECOND_JACOBI, **kw)
        _, _, rl, rcl, il = lib.solve(h, dcsr(lib, A), None, precond=lib.PRECOND_FSAI_LEARNED, mlp_weights=w,
                                      grid=(N, N, N), mlp_bf16=1, **kw)
        _, _, rc_, rcc, ic = lib.solve(h, dcsr(lib, A), None, precond=lib.PRECOND_FSAI, **kw)
        assert rcj == lib.OK and rcl == lib.OK and rcc == lib.OK
        print("matvecs jacobi / learned / classical FSAI:", ij["mv_A"], il["mv_A"], ic["mv_A"])
        gains.append(ij["mv_A"] / il["mv_A"])
    print("matvec gain of the learned FSAI over Jacobi on held-out operators:", gains)
    assert min(gains) > 1.0


# ---------------------------------------------------------------- IC(0)
def test_ic0_factor_matches_oracle(lib, h):
    """The IC(0) factor from the device's fixed-point sweeps (run to
    convergence) against the oracle's left-looking recurrence, to 1e-12."""
    from oracle import ic0 as I
    for A in (aniso(11, 3), W.fem_q1_pencil(6, np.random.default_rng(1).uniform(1, 10, (6, 6, 6)))[0],
              W.chung_lu_laplacian(3000, 8.0, 2.1, 4)):
        Lref = I.ic0(A.to_scipy())
        nnz = lib.trplk_fsai_values(h, dcsr(lib, A), 2)
        assert nnz == Lref.nnz
        l = torch.zeros(nnz, dtype=torch.float64, device="cuda")
        lib.trplk_fsai_values(h, dcsr(lib, A), 2, g=l)
        assert np.allclose(l.cpu().numpy(), Lref.data, rtol=1e-12, atol=1e-13 * np.abs(Lref.data).max())


def test_ic0_apply_matches_oracle(lib, h):
    """M x = P^T (P x) with two Jacobi sweeps per triangular solve, to 1e-12."""
    from oracle import ic0 as I
    A = aniso(10, 8)
    L = I.ic0(A.to_scipy())
    x = np.random.default_rng(3).standard_normal(A.n)
    y = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    lib.trplk_ic0_apply(h, dcsr(lib, A), torch.from_numpy(L.data).cuda(), torch.from_numpy(x).cuda(), y)
    ref = I.apply_M(L, x, 2)
    assert np.allclose(y.cpu().numpy(), ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ic0_solve_matches_oracle(lib, h, precision):
    """TRPL+K preconditioned by IC(0): the FP64 path follows the oracle's
    cycles and its eigenvalues to 1e-10; the mixed path reaches the same
    eigenvalues."""
    from oracle import ic0 as I
    N = 12
    A = aniso(N, 11)
    As = A.to_scipy()
    p, q, k, l = 4, 18, 6, 1
    X0 = W.start_block(A.n, k, 1)
    ref = O.solve(As, None, p, q, k, l, 1e-10, X0, I.preconditioner(As, 2))
    prec = lib.PRECISION_FP64 if precision == "fp64" else lib.PRECISION_MIXED
    ev, X, res, rc, info = lib.solve(h, dcsr(lib, A), None, p=p, q=q, k=k, l=l, tol=1e-10, X0=X0,
                                     precond=lib.PRECOND_IC0, precision=prec)
    assert rc == lib.OK and ref["status"] == O.OK
    assert np.all(np.abs(ev - ref["evals"]) <= 1e-10 * np.abs(ref["evals"]))
    if precision == "fp64":
        assert info["cycles"] == ref["cycles"]
