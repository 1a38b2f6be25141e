"""Pins of the FSAI oracle (oracle/fsai.py): exact inverse factors on full
patterns, the normalisation and Kaporin-minimality of classical FSAI, the
energy-norm identity of the loss, finite-difference gradients, known features
and the Jacobi starting point of the MLP."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fsai as F
from paper_1711_10128_gb300 import workloads as W


def test_classical_fsai_full_pattern_is_exact_inverse_factor():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((6, 6))
    A = X @ X.T + 6 * np.eye(6)
    G = F.classical_fsai(sp.csr_matrix(A)).toarray()   # lower pattern = full lower triangle
    assert np.allclose(G @ A @ G.T, np.eye(6), atol=1e-12)
    assert np.allclose(G.T @ G, np.linalg.inv(A), atol=1e-12)


def test_classical_fsai_diagonal_and_normalisation():
    A = W.diffusion_3d(5, W.lognormal_field(5, 1.0, 3)).to_scipy()
    G = F.classical_fsai(A)
    d = np.asarray((G @ A).multiply(G).sum(axis=1)).ravel()
    assert np.allclose(d, 1.0, atol=1e-12)          # (G A G^T)_ii = 1
    D = sp.diags(np.arange(1.0, 9.0))
    Gd = F.classical_fsai(D).toarray()
    assert np.allclose(Gd, np.diag(1 / np.sqrt(np.arange(1.0, 9.0))), atol=1e-15)


def test_classical_fsai_minimises_kaporin_on_its_pattern():
    A = W.diffusion_3d(4, W.lognormal_field(4, 1.0, 5), axis=(1.0, 7.0, 30.0)).to_scipy()
    G = F.classical_fsai(A)
    k0 = F.kaporin(G, A)
    rng = np.random.default_rng(1)
    for _ in range(20):
        P = G.copy()
        P.data = P.data * (1 + 1e-2 * rng.standard_normal(P.nnz))
        assert F.kaporin(P, A) > k0 - 1e-14
    # scaling G does not change K (it is scale invariant)
    assert abs(F.kaporin(3.0 * G, A) - k0) < 1e-12


def test_energy_term_equals_error_in_A_norm_minus_constant():
    A = W.diffusion_3d(4, W.lognormal_field(4, 1.0, 6)).to_scipy()
    Ad = A.toarray()
    G = F.classical_fsai(A)
    rng = np.random.default_rng(2)
    v = rng.standard_normal(A.shape[0])
    Mv = F.apply_M(G, v)
    E = Mv @ (A @ Mv) - 2 * np.linalg.norm(G @ v) ** 2
    x = np.linalg.solve(Ad, v)
    assert abs(E - ((x - Mv) @ Ad @ (x - Mv) - v @ x)) <= 1e-10 * abs(v @ x)


def test_loss_gradient_in_G_matches_finite_differences():
    A = W.diffusion_3d(4, W.lognormal_field(4, 1.0, 7)).to_scipy()
    G = F.classical_fsai(A)
    rng = np.random.default_rng(3)
    G.data = G.data * (1 + 0.1 * rng.standard_normal(G.nnz))
    V = rng.standard_normal((A.shape[0], 3))
    L, g, _ = F.loss_and_grad_G(G, A, V)
    for e in rng.choice(G.nnz, 12, replace=False):
        h = 1e-6 * max(1.0, abs(G.data[e]))
        Gp, Gm = G.copy(), G.copy()
        Gp.data[e] += h
        Gm.data[e] -= h
        fd = (F.loss_and_grad_G(Gp, A, V)[0] - F.loss_and_grad_G(Gm, A, V)[0]) / (2 * h)
        assert abs(fd - g[e]) <= 1e-6 * max(1.0, abs(fd)), (e, fd, g[e])


def test_mlp_gradient_matches_finite_differences():
    dims = (4, 4, 4)
    A = W.diffusion_3d(4, W.lognormal_field(4, 1.0, 8), axis=(1.0, 3.0, 9.0)).to_scipy()
    p = F.init_mlp(4, hidden=8)
    rng = np.random.default_rng(5)
    p["W3"] = 0.1 * rng.standard_normal(p["W3"].shape)
    p["b2"] = 0.1 * rng.standard_normal(p["b2"].shape)
    V = rng.standard_normal((A.shape[0], 2))
    L, g, _ = F.loss_and_grad_mlp(p, A, dims, V)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = p[name].ravel()
        for idx in rng.choice(flat.size, min(4, flat.size), replace=False):
            h = 1e-6
            old = flat[idx]
            flat[idx] = old + h
            lp = F.loss_and_grad_mlp(p, A, dims, V)[0]
            flat[idx] = old - h
            lm = F.loss_and_grad_mlp(p, A, dims, V)[0]
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].ravel()[idx]
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(fd)), (name, idx, fd, an)
    assert np.all(g["W3"][4:] == 0) and np.all(g["b3"][4:] == 0)   # unused upper outputs


def test_features_of_constant_laplacian_and_jacobi_start():
    N = 4
    A = W.diffusion_3d(N).to_scipy()
    Fe = F.features_7pt(A, (N, N, N))
    interior = (1 * N + 1) * N + 1                     # cell (1,1,1)
    assert np.allclose(Fe[interior], [np.log(6), -1 / 6, -1 / 6, -1 / 6, -1 / 6, -1 / 6, -1 / 6, 0.0])
    corner = 0                                          # boundary faces add to the diagonal only
    assert np.allclose(Fe[corner], [np.log(6), 0, -1 / 6, 0, -1 / 6, 0, -1 / 6, 0.5])
    # scaled couplings use both diagonals: a_ij / sqrt(a_ii a_jj)
    B = W.diffusion_3d(N, W.lognormal_field(N, 1.0, 2)).to_scipy()
    Fb = F.features_7pt(B, (N, N, N))
    i = interior
    assert np.isclose(Fb[i, 1], B[i, i - 1] / np.sqrt(B[i, i] * B[i - 1, i - 1]))
    p = F.init_mlp(0)
    o, _ = F.mlp_forward(p, Fe)
    G = F.g_from_outputs(A, (N, N, N), o)
    assert np.allclose(G.toarray(), np.diag(1 / np.sqrt(A.diagonal())), atol=1e-14)


def test_classical_fsai_is_representable_by_the_output_map():
    """With the scaled couplings of F3 and the 1/sqrt(a_jj) scaling of F4,
    classical FSAI of a 7-point operator is o_dir = -c_dir / sqrt(1 - s),
    softplus(o_c) = 1 / sqrt(1 - s), s = sum of the squared lower couplings."""
    N = 5
    A = W.anisotropic_diffusion(N, 1003).to_scipy()
    Fe = F.features_7pt(A, (N, N, N))
    c = Fe[:, [5, 3, 1]]                      # lower couplings (-z, -y, -x)
    s = (c ** 2).sum(axis=1)
    o = np.zeros((A.shape[0], 7))
    o[:, 0:3] = -c / np.sqrt(1 - s)[:, None]
    o[:, 3] = np.log(np.expm1(1 / np.sqrt(1 - s)))
    G = F.g_from_outputs(A, (N, N, N), o)
    assert np.allclose(G.toarray(), F.classical_fsai(A).toarray(), atol=1e-12)


def test_bf16_rounding_matches_the_library_conversion():
    """F6's rounding (through FP32, nearest, ties to even) against torch's
    float32 -> bfloat16 conversion, on random values of many magnitudes and on
    exact ties (low 16 bits 0x8000) with both parities of the kept bit."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = rng.standard_normal(20000) * np.exp(rng.uniform(-30, 30, 20000))
    bits = rng.integers(0, 2 ** 31, 4000, dtype=np.uint64).astype(np.uint32)
    ties = ((bits & np.uint32(0x7F7F0000)) | np.uint32(0x8000)).view(np.float32).astype(np.float64)
    for v in (x, ties, -ties, np.array([0.0, 1.0, -2.5, 3.0e38, 1.0e-38])):
        ref = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
        assert np.array_equal(F.bf16_round(v), ref)


def test_bf16_mode_b3_gradient_matches_finite_differences():
    """The BF16 mode (F6): b3 is not rounded and enters after the last rounded
    activation, so the rounded network's loss is smooth in b3 and its analytic
    gradient must match central differences.  The BF16 loss stays within the
    rounding's reach of the FP64 loss (8 significant bits: a few 2^-8)."""
    dims = (4, 4, 4)
    A = W.diffusion_3d(4, W.lognormal_field(4, 1.0, 8), axis=(1.0, 3.0, 9.0)).to_scipy()
    p = F.init_mlp(4, hidden=8)
    rng = np.random.default_rng(6)
    p["W3"] = 0.1 * rng.standard_normal(p["W3"].shape)
    p["b2"] = 0.1 * rng.standard_normal(p["b2"].shape)
    V = rng.standard_normal((A.shape[0], 2))
    L, g, _ = F.loss_and_grad_mlp(p, A, dims, V, quant="bf16")
    for idx in range(4):
        h = 1e-6
        old = p["b3"][idx]
        p["b3"][idx] = old + h
        lp = F.loss_and_grad_mlp(p, A, dims, V, quant="bf16")[0]
        p["b3"][idx] = old - h
        lm = F.loss_and_grad_mlp(p, A, dims, V, quant="bf16")[0]
        p["b3"][idx] = old
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g["b3"][idx]) <= 1e-5 * max(1.0, abs(fd)), (idx, fd, g["b3"][idx])
    L64, g64, _ = F.loss_and_grad_mlp(p, A, dims, V)
    assert L != L64 and abs(L - L64) <= 4 * 2.0 ** -8 * abs(L64)
    for name in g:
        assert np.all(np.abs(g[name] - g64[name]) <= 0.1 * np.abs(g64[name]).max() + 1e-300), name


def test_loss_scales_each_vector_by_its_jacobi_energy():
    """F5: the energy part of the loss is the mean over the vectors of
    c_v E_v with c_v = 1 / (v^T D^-1 v) and E_v from the A-norm identity
    (computed here by a dense solve)."""
    A = W.diffusion_3d(4, W.lognormal_field(4, 1.0, 9)).to_scipy()
    Ad = A.toarray()
    G = F.classical_fsai(A)
    rng = np.random.default_rng(11)
    V = rng.standard_normal((A.shape[0], 3)) * np.array([1.0, 10.0, 0.1])
    d = np.diag(Ad)
    want = 0.0
    for c in range(V.shape[1]):
        v = V[:, c]
        x = np.linalg.solve(Ad, v)
        Mv = F.apply_M(G, v)
        want += ((x - Mv) @ Ad @ (x - Mv) - v @ x) / (v @ (v / d))
    want /= V.shape[1]
    _, _, parts = F.loss_and_grad_G(G, A, V)
    assert abs(parts["E"] - want) <= 1e-10 * abs(want)


@pytest.mark.parametrize("quant", [None, "bf16"])
def test_first_layer_gradient_uses_the_features_the_network_saw(quant):
    """dL/dW1[:, f] = x_f dL/db1 for a feature f that has the same value x_f
    in every row (the chain rule through z1 = W1 x + b1): on the
    constant-coefficient operator every diagonal is 6, so feature 0 is log 6
    in FP64 and its bfloat16 rounding in the BF16 mode (F6)."""
    dims = (4, 4, 4)
    A = W.diffusion_3d(4).to_scipy()
    p = F.init_mlp(2, hidden=8)
    rng = np.random.default_rng(12)
    p["W3"] = 0.1 * rng.standard_normal(p["W3"].shape)
    p["b1"] = 0.1 * rng.standard_normal(p["b1"].shape)
    V = rng.standard_normal((A.shape[0], 2))
    _, g, _ = F.loss_and_grad_mlp(p, A, dims, V, quant=quant)
    x0 = np.log(6.0) if quant is None else F.bf16_round(np.log(6.0))
    assert np.abs(g["b1"]).max() > 0
    assert np.allclose(g["W1"][:, 0], x0 * g["b1"], rtol=1e-12, atol=1e-14 * np.abs(g["b1"]).max())
    assert quant is None or abs(x0 - np.log(6.0)) > 1e-4   # the rounding is visible at this tolerance


def test_kaporin_closed_form_and_the_loss_weight():
    """K(D^-1/2) = log a for a constant diagonal a (G A G^T has unit diagonal);
    the loss is E + 0.1 K with the same K as the stand-alone measure (F5)."""
    A = W.diffusion_3d(4).to_scipy()                 # every diagonal entry is 6
    G = sp.diags(1.0 / np.sqrt(A.diagonal())).tocsr()
    assert abs(F.kaporin(G, A) - np.log(6.0)) <= 1e-14
    B = W.diffusion_3d(4, W.lognormal_field(4, 1.0, 3)).to_scipy()
    Gc = F.classical_fsai(B)
    V = np.random.default_rng(4).standard_normal((B.shape[0], 2))
    L, _, parts = F.loss_and_grad_G(Gc, B, V)
    assert abs(parts["K"] - F.kaporin(Gc, B)) <= 1e-12 * abs(parts["K"])
    assert abs(L - (parts["E"] + 0.1 * parts["K"])) <= 1e-14 * max(1.0, abs(L))


def _mlp_case(seed):
    dims = (4, 4, 4)
    A = W.diffusion_3d(4, W.lognormal_field(4, 1.0, 8), axis=(1.0, 3.0, 9.0)).to_scipy()
    p = F.init_mlp(seed, hidden=8)
    rng = np.random.default_rng(seed + 10)
    p["W3"] = 0.1 * rng.standard_normal(p["W3"].shape)
    p["b1"] = 0.1 * rng.standard_normal(p["b1"].shape)
    p["b2"] = 0.1 * rng.standard_normal(p["b2"].shape)
    V = rng.standard_normal((A.shape[0], 2))
    return A, dims, p, V


def test_bf16_mode_sees_only_the_rounded_weights():
    """F6: the rounded network uses W1, W2, W3 only through their bfloat16
    roundings, forward and backward alike, so moving every weight inside its
    rounding interval changes neither the loss nor any gradient."""
    A, dims, p, V = _mlp_case(5)
    L, g, _ = F.loss_and_grad_mlp(p, A, dims, V, quant="bf16")
    q = dict(p)
    for name in ("W1", "W2", "W3"):
        w = p[name]
        moved = w * (1.0 + 1e-5) + 1e-30        # far inside an interval of relative width 2^-8
        keep = F.bf16_round(moved) == F.bf16_round(w)
        q[name] = np.where(keep, moved, w)
        assert keep.mean() > 0.9 and np.any(q[name] != w)
    L2, g2, _ = F.loss_and_grad_mlp(q, A, dims, V, quant="bf16")
    assert L2 == L
    for name in g:
        assert np.array_equal(g2[name], g[name]), name


def test_bf16_forward_rounds_where_the_reading_says():
    """F6 composed independently with torch's bfloat16 conversion: features
    through FP32, W1..W3 and both hidden activations rounded, biases not,
    products and sums in FP64."""
    torch = pytest.importorskip("torch")
    A, dims, p, _ = _mlp_case(6)
    Fe = F.features_7pt(A, dims)
    bf = lambda a: torch.from_numpy(np.asarray(a, np.float64).astype(np.float32)).to(torch.bfloat16).to(
        torch.float64).numpy()
    h1 = bf(np.maximum(bf(Fe) @ bf(p["W1"]).T + p["b1"], 0.0))
    h2 = bf(np.maximum(h1 @ bf(p["W2"]).T + p["b2"], 0.0))
    o = h2 @ bf(p["W3"]).T + p["b3"]
    got, _ = F.mlp_forward(p, Fe, quant="bf16")
    assert np.allclose(got, o, rtol=1e-13, atol=1e-15)
    plain, _ = F.mlp_forward(p, Fe)
    assert not np.allclose(plain, o, rtol=1e-6)      # the roundings are visible
