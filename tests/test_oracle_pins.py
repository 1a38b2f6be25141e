"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle (``oracle/``) against something other than
itself: closed-form spectra, a brute-force dense eigensolve, the optimal
line-search step of Lemma 3 (Sec. 4), the special cases the paper names
(TRLan for M = I and l = 0, Sec. 5.2; LOPCG for one inner step, Sec. 5.1;
the Krylov space for a single restart vector, Sec. 4.2), the matvec
accounting behind Tables 2-5, and invariants (B-orthonormality,
T = U^T A U, monotone Ritz values).
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse as sp

from oracle import dense
from oracle import trplk as O
from paper_1711_10128_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def lap2d_eigs(N, count):
    h = math.pi / (2 * (N + 1))
    ev = sorted(4 * math.sin(i * h) ** 2 + 4 * math.sin(j * h) ** 2
                for i in range(1, N + 1) for j in range(1, N + 1))
    return np.array(ev[:count])


def lap3d_eigs(N, count):
    s = 4 * np.sin(np.arange(1, N + 1) * np.pi / (2 * (N + 1))) ** 2
    return np.sort((s[:, None, None] + s[None, :, None] + s[None, None, :]).ravel())[:count]


def fem_eigs(N, count):
    h = 1.0 / N
    t = (2 * np.arange(1, N + 1) - 1) * np.pi / (2 * N)
    mu = (6 / h ** 2) * (1 - np.cos(t)) / (2 + np.cos(t))
    return np.sort((mu[:, None, None] + mu[None, :, None] + mu[None, None, :]).ravel())[:count]


def test_norm_is_the_largest_absolute_row_sum():
    """R1: ||A||_1 is the largest absolute row sum (for symmetric A also the
    largest column sum): 8 for the 5-point Laplacian, and a hand-made
    matrix whose largest row sum needs the absolute values."""
    assert O.norm1(W.laplacian_2d(6).to_scipy()) == 8.0
    M = sp.csr_matrix(np.array([[2.0, -3.0, 0.0], [-3.0, 1.0, 0.5], [0.0, 0.5, -4.0]]))
    assert O.norm1(M) == 5.0
    r = O.solve(W.laplacian_2d(12).to_scipy(), None, 2, 10, 4, 1, 1e-8, W.start_block(144, 4, 1), "jacobi")
    assert r["normA"] == 8.0


# ---------------------------------------------------------------- dense pieces
@pytest.mark.parametrize("n", [1, 2, 7, 31])
def test_jacobi_eigh_tridiagonal_closed_form(n):
    T = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    w, V = dense.jacobi_eigh(T)
    ref = 2 - 2 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
    assert np.allclose(w, np.sort(ref), atol=1e-13)
    assert np.allclose(T @ V, V * w, atol=1e-12)
    assert np.allclose(V.T @ V, np.eye(n), atol=1e-13)


def test_jacobi_eigh_matches_lapack_random():
    rng = np.random.default_rng(5)
    for n in (3, 16, 50):
        M = rng.standard_normal((n, n))
        M = M + M.T
        w, V = dense.jacobi_eigh(M)
        assert np.allclose(w, np.linalg.eigvalsh(M), atol=1e-12 * np.abs(w).max())
        assert np.allclose(M @ V, V * w, atol=1e-12 * np.abs(w).max())


def test_rayleigh_ritz_against_dense_jacobi_and_sign_rule():
    rng = np.random.default_rng(7)
    M = rng.standard_normal((12, 12))
    M = M + M.T
    theta, Y = O.rayleigh_ritz(np.triu(M))     # only the upper triangle is read
    w, V = dense.jacobi_eigh(M)
    assert np.allclose(theta, w, atol=1e-12)
    for c in range(12):
        i = np.argmax(np.abs(Y[:, c]))
        assert Y[i, c] > 0
        assert abs(abs(V[:, c] @ Y[:, c]) - 1) < 1e-10


def test_two_vector_rayleigh_ritz_matches_lemma3_optimal_step():
    """Lemma 3 (Sec. 4): min over span{x, d} of the Rayleigh quotient of
    (A, B) is reached at x + alpha* d, alpha* the smaller positive (or the
    unique) root of a alpha^2 + b alpha + c = 0."""
    A, B = W.fem_q1_pencil(4)
    A, B = A.to_scipy().toarray(), B.to_scipy().toarray()
    rng = np.random.default_rng(3)
    v1 = sl.eigh(A, B)[1][:, 0]
    x = v1 + 0.05 * rng.standard_normal(v1.size)
    x /= math.sqrt(x @ B @ x)
    rho = x @ A @ x
    grad = A @ x - rho * B @ x
    d = -grad + 0.1 * rng.standard_normal(x.size)        # a descent direction
    assert d @ grad < 0
    a = (d @ A @ d) * (d @ B @ x) - (d @ B @ d) * (d @ A @ x)
    b = (d @ A @ d) * (x @ B @ x) - (d @ B @ d) * (x @ A @ x)
    c = (d @ A @ x) * (x @ B @ x) - (d @ B @ x) * (x @ A @ x)
    roots = np.roots([a, b, c]) if abs(a) > 0 else np.array([-c / b])
    roots = np.real(roots[np.isreal(roots)])
    alpha = roots[roots > 0].min()
    y = x + alpha * d
    rq_opt = (y @ A @ y) / (y @ B @ y)
    # the oracle's pieces: B-orthonormalise [x, d], project, Rayleigh-Ritz
    Bfun = lambda v: B @ v
    Q, BQ, _ = O.b_orthonormalise(np.stack([x, d], axis=1), Bfun)
    T = Q.T @ A @ Q
    theta, _ = O.rayleigh_ritz(T)
    assert abs(theta[0] - rq_opt) <= 1e-12 * abs(rq_opt)


def test_cgs2_b_orthogonality_and_norm():
    A, B = W.fem_q1_pencil(5)
    Bs = B.to_scipy()
    rng = np.random.default_rng(11)
    n = Bs.shape[0]
    Bfun = lambda v: Bs @ v
    U, BU, _ = O.b_orthonormalise(rng.standard_normal((n, 9)), Bfun)
    assert np.allclose(U.T @ (Bs @ U), np.eye(9), atol=1e-13)
    w = rng.standard_normal(n)
    wo, Bw, beta, beta0, h = O.cgs2(w, U, BU, Bfun)
    assert np.abs(U.T @ (Bs @ wo)).max() <= 1e-13 * beta
    assert abs(beta - math.sqrt(wo @ (Bs @ wo))) <= 1e-13 * beta
    assert abs(beta0 - math.sqrt(w @ (Bs @ w))) <= 1e-12 * beta0
    # w = U h + wo exactly (up to rounding)
    assert np.allclose(U @ h + wo, w, atol=1e-12 * np.abs(w).max())


# ---------------------------------------------------------------- whole solves
def kato_temple_ok(theta, lam, rnorm, gap):
    return abs(theta - lam) <= rnorm ** 2 / gap + 1e-14 * abs(lam) + rnorm * 1e-8


@pytest.mark.parametrize("N,p,q,k,l", [(30, 5, 20, 8, 5), (24, 3, 12, 4, 1)])
def test_solve_2d_laplacian_closed_form(N, p, q, k, l):
    A = W.laplacian_2d(N)
    As = A.to_scipy()
    X0 = W.start_block(A.n, k, 0)
    r = O.solve(As, None, p, q, k, l, 1e-10, X0, "jacobi")
    assert r["status"] == O.OK
    lam = lap2d_eigs(N, p + 1)
    gap = lam[p] - lam[p - 1] if lam[p] > lam[p - 1] else lam[p] - lam[0]
    rabs = r["resid"] * r["normA"]
    for i in range(p):
        assert abs(r["evals"][i] - lam[i]) <= 1e-9 * lam[i]
        # Krylov-Weinstein: |theta - lambda| <= ||r|| for B = I
        assert np.min(np.abs(lap2d_eigs(N, 2 * p + 2) - r["evals"][i])) <= rabs[i] + 1e-15
    assert np.all(r["resid"] <= 1e-10)
    X = r["evecs"]
    assert np.allclose(X.T @ X, np.eye(p), atol=1e-12)
    # matvec accounting of Tables 2-5: p_hat + (q - p_hat) * cycles
    assert r["mv_A"] == k + (q - k) * r["cycles"]


def test_full_size_2d_laplacian_100():
    """The 100 x 100 Laplacian with p = 5, q = 20, p_hat = 8, +K = 5, tol 1e-8."""
    N, p, q, k, l = 100, 5, 20, 8, 5
    A = W.laplacian_2d(N)
    r = O.solve(A.to_scipy(), None, p, q, k, l, 1e-8, W.start_block(A.n, k, 0), "jacobi")
    assert r["status"] == O.OK
    lam = lap2d_eigs(N, p)
    # error bounded by ||r||^2 / gap (Kato-Temple) with ||r|| <= 1e-8 * ||A||_1
    assert np.all(np.abs(r["evals"] - lam) <= (8e-8) ** 2 / 1e-3 + 1e-13)
    assert np.all(r["resid"] <= 1e-8)
    assert r["mv_A"] == k + (q - k) * r["cycles"]


def test_solve_3d_isotropic_closed_form():
    N = 12
    A = W.diffusion_3d(N)
    p, q, k, l = 4, 16, 6, 1
    r = O.solve(A.to_scipy(), None, p, q, k, l, 1e-10, W.start_block(A.n, k, 1), "jacobi")
    assert r["status"] == O.OK
    lam = lap3d_eigs(N, p)
    assert np.all(np.abs(r["evals"] - lam) <= 1e-9 * lam)


def test_solve_generalized_fem_pencil_closed_form_and_brute_force():
    N = 6
    A, B = W.fem_q1_pencil(N)
    As, Bs = A.to_scipy(), B.to_scipy()
    p, q, k, l = 5, 18, 8, 1
    r = O.solve(As, Bs, p, q, k, l, 1e-10, W.start_block(A.n, k, 2), "jacobi")
    assert r["status"] == O.OK
    lam = fem_eigs(N, p)
    brute = sl.eigh(As.toarray(), Bs.toarray(), eigvals_only=True)[:p]
    assert np.allclose(lam, brute, rtol=1e-11)
    assert np.all(np.abs(r["evals"] - lam) <= 1e-9 * lam)
    X = r["evecs"]
    assert np.allclose(X.T @ (Bs @ X), np.eye(p), atol=1e-11)
    assert r["mv_A"] == k + (q - k) * r["cycles"]
    assert r["mv_B"] == r["mv_A"]


def test_solve_variable_coefficient_brute_force():
    N = 10
    A = W.diffusion_3d(N, W.lognormal_field(N, 1.0, 4))
    As = A.to_scipy()
    p, q, k, l = 6, 20, 8, 2
    r = O.solve(As, None, p, q, k, l, 1e-10, W.start_block(A.n, k, 3), "jacobi")
    assert r["status"] == O.OK
    brute = np.linalg.eigvalsh(As.toarray())[:p]
    assert np.all(np.abs(r["evals"] - brute) <= 1e-9 * brute)


def test_invariants_T_equals_UtAU_and_b_orthonormal_basis():
    N = 5
    A, B = W.fem_q1_pencil(N, np.random.default_rng(0).uniform(1, 10, (N, N, N)))
    As, Bs = A.to_scipy(), B.to_scipy()
    r = O.solve(As, Bs, 3, 14, 5, 2, 1e-10, W.start_block(A.n, 5, 9), "jacobi",
                max_cycles=4, record=True)
    for tr in r["trace"]:
        U = tr["U"]
        assert np.allclose(U.T @ (Bs @ U), np.eye(U.shape[1]), atol=1e-12)
        TA = U.T @ (As @ U)
        assert np.allclose(tr["T"], TA, atol=1e-11 * np.abs(TA).max())
        assert np.allclose(tr["AU"], As @ U, atol=1e-12 * np.abs(tr["AU"]).max())
        assert np.allclose(tr["BU"], Bs @ U, atol=1e-12 * np.abs(tr["BU"]).max())
    # after restart T(1:p_hat, 1:p_hat) = diag(theta) (Sec. 3)
    T1 = r["trace"][1]["T"]
    th0 = r["trace"][0]["theta"][:5]
    assert np.allclose(T1[:5, :5], np.diag(th0), atol=1e-12 * np.abs(th0).max())


def test_target_advance_and_recheck_follow_the_recorded_residuals():
    """R9 on a solve whose soft-locked pairs drift: in every cycle the target
    advances by one exactly when its residual (recorded after the cycle's
    Rayleigh-Ritz step) is below tol; when the last target converges while an
    earlier pair has drifted above tol, the next cycle targets the first such
    pair.  This run (2D Laplacian 14 x 14, p = 5, l = 2) has such a return."""
    A = W.laplacian_2d(14).to_scipy()
    p, q, k, l, tol = 5, 14, 6, 2, 1e-8
    r = O.solve(A, None, p, q, k, l, tol, W.start_block(A.shape[0], k, 32), "jacobi")
    assert r["status"] == O.OK
    h = r["history"]
    returns = 0
    for a, b in zip(h[:-1], h[1:]):
        t, res = a["t"], a["resid"]
        if res[t] > tol:
            assert b["t"] == t
        elif t + 1 < p:
            assert b["t"] == t + 1
        else:   # the last target converged: back to the first pair above tol
            assert np.any(res > tol)
            assert b["t"] == int(np.flatnonzero(res > tol)[0])
            returns += 1
    assert returns >= 1
    assert np.all(h[-1]["resid"] <= tol)


def test_ritz_values_never_increase():
    """The restart space contains the previous p_hat Ritz vectors, so by the
    Courant-Fischer minimax property every kept Ritz value can only decrease."""
    A = W.diffusion_3d(9, W.lognormal_field(9, 1.0, 6))
    r = O.solve(A.to_scipy(), None, 4, 14, 6, 1, 1e-12, W.start_block(A.n, 6, 4), "jacobi",
                max_cycles=30)
    th = np.array([h["theta"] for h in r["history"]])
    assert np.all(np.diff(th, axis=0) <= 1e-12 * np.abs(th).max())


def test_trlan_special_case_tridiagonal_g_block():
    """M = I and l = 0: TRPL+K reduces to thick-restart Lanczos (Sec. 5.2), so the
    G-G block of T obeys the Lanczos three-term relation (is tridiagonal)."""
    A = W.diffusion_3d(8, W.lognormal_field(8, 1.0, 2))
    k = 4
    r = O.solve(A.to_scipy(), None, 2, 14, k, 0, 1e-12, W.start_block(A.n, k, 5), "none",
                max_cycles=3, record=True)
    for tr in r["trace"]:
        G = tr["T"][k:, k:]
        scale = np.abs(G).max()
        off = np.abs(np.triu(G, 2)).max()
        assert off <= 1e-10 * scale
        assert np.abs(np.diag(G, 1)).min() > 1e-6 * scale


def test_single_vector_basis_is_preconditioned_krylov_space():
    """p_hat = 1: span{x, G} = K_{m+1}(M (A - rho B), x) (Sec. 4.2)."""
    A = W.diffusion_3d(7, W.lognormal_field(7, 1.0, 8))
    As = A.to_scipy()
    dinv = 1.0 / As.diagonal()
    q = 7
    r = O.solve(As, None, 1, q, 1, 1, 1e-14, W.start_block(A.n, 1, 6), "jacobi",
                max_cycles=1, record=True)
    tr = r["trace"][0]
    U, rho = tr["U"], tr["rho"]
    x = U[:, 0]
    K = [x]
    for _ in range(q - 1):
        v = dinv * (As @ K[-1] - rho * K[-1])
        K.append(v / np.linalg.norm(v))
    Qk, _ = np.linalg.qr(np.stack(K, axis=1))
    s = np.linalg.svd(Qk.T @ U, compute_uv=False)
    assert s.min() > 1 - 1e-8


def test_lopcg_special_case():
    """p_hat = 1, one inner step and l = 1: the space is span{x_i, M r_i, x_(i-1)},
    LOPCG's (Sec. 5.1; eq. (subspace_lobpcg) with p = 1).  An independent loop
    using Gram matrices of the raw vectors reproduces the Ritz values."""
    A = W.diffusion_3d(8, W.lognormal_field(8, 0.5, 12))
    As = A.to_scipy()
    dinv = 1.0 / As.diagonal()
    x0 = W.start_block(A.n, 1, 7)[:, 0]
    r = O.solve(As, None, 1, 3, 1, 1, 1e-30, x0[:, None], "jacobi", max_cycles=12)
    ours = [h["theta"][0] for h in r["history"]]

    def rr(V):
        G = V.T @ V
        H = V.T @ (As @ V)
        w, Y = sl.eigh(H, G)
        y = V @ Y[:, 0]
        return w[0], y / np.linalg.norm(y)

    x = x0 / np.linalg.norm(x0)
    rho = x @ (As @ x)
    # first cycle: no previous vector yet, two inner steps (m = q - p_hat = 2)
    g1 = dinv * (As @ x - rho * x)
    g2 = dinv * (As @ g1 - rho * g1)
    th, xn = rr(np.stack([x, g1, g2], axis=1))
    ref = [th]
    xprev, x = x, xn
    for _ in range(11):
        rho = x @ (As @ x)
        g1 = dinv * (As @ x - rho * x)
        th, xn = rr(np.stack([x, g1, xprev], axis=1))
        ref.append(th)
        xprev, x = x, xn
    ours, ref = np.array(ours), np.array(ref)
    assert np.allclose(ours, ref, rtol=1e-9, atol=1e-12)


def test_paper_matvec_counts_follow_restart_accounting():
    """Every TRPL+K MV count printed in Tables 2-5 equals p_hat + (q - p_hat) c
    for an integer cycle count c, with p_hat = 8, q = 18 (Sec. 5 setup): the
    accounting the oracle's counter follows."""
    rows = [line.split() for line in open(os.path.join(GOLDEN, "paper_mv_counts.txt"))
            if line.strip() and not line.startswith("#")]
    assert len(rows) == 22
    for table, name, p, mv in rows:
        assert (int(mv) - 8) % 10 == 0, (table, name, mv)


def test_closed_form_values_c1():
    """The 2D formula evaluated for the 100 x 100 grid (checks its transcription)."""
    lam = lap2d_eigs(100, 6)
    assert abs(lam[0] - 1.934870832047740e-3) < 1e-17
    assert abs(lam[1] - lam[2]) < 1e-17 and abs(lam[3] - 7.737611465622606e-3) < 1e-17
    brute = np.linalg.eigvalsh(W.laplacian_2d(12).to_scipy().toarray())[:6]
    assert np.allclose(brute, lap2d_eigs(12, 6), rtol=1e-13)


def test_closed_form_values_full_size_c2_c3():
    """The 3D Laplacian (128^3, all coefficients 1) and the constant-E Q1 pencil
    (96^3 elements) formulas at full size, against the values computed
    independently for these configurations: smallest and last-wanted eigenvalue
    and the multiplicities that end each wanted set."""
    lam = lap3d_eigs(128, 12)
    assert abs(lam[0] - 1.779180929164e-3) < 1e-15
    assert abs(lam[9] - 6.521553292339e-3) < 1e-15
    assert abs(lam[7] - lam[9]) < 1e-17 and lam[10] > lam[9] + 1e-4   # (1,1,3) triple closes the 10
    mu = fem_eigs(96, 21)
    assert abs(mu[0] - 7.4023684517) < 1e-9
    assert abs(mu[19] - 1.0614157990e2) < 1e-7
    assert abs(mu[17] - mu[19]) < 1e-9 and mu[20] > mu[19] + 1.0      # (2,2,3) triple closes the 20


def test_breakdown_on_an_invariant_krylov_space_still_gives_exact_eigenpairs():
    """Reading R5: with three distinct eigenvalues (multiplicity 4 each) and
    M = I the Krylov space of one start vector is invariant after at most
    three steps; the inner loop ends early and the Rayleigh-Ritz step still
    yields the smallest eigenvalue exactly."""
    rng = np.random.default_rng(5)
    lam = np.repeat([1.0, 2.5, 4.0], 4)
    Q = np.linalg.qr(rng.standard_normal((12, 12)))[0]
    A = sp.csr_matrix((Q * lam) @ Q.T)
    r = O.solve(A, None, 1, 10, 1, 0, 1e-12, W.start_block(12, 1, 3), None)
    assert r["status"] in (O.OK, O.BREAKDOWN)
    assert r["cycles"] == 1 and r["mv_A"] < 1 + (10 - 1)   # the cycle stopped before its 9 inner steps
    assert abs(r["evals"][0] - 1.0) <= 1e-12
    x = r["evecs"][:, 0]
    assert np.linalg.norm(A @ x - x) <= 1e-10


def test_breakdown_status_when_the_restart_vector_lies_in_the_start_space():
    """R5: a preconditioner that maps every residual into span(X) makes the
    cycle's first Lanczos vector vanish under CGS2; nothing new can enter the
    basis, so the solve stops in its first cycle with status breakdown (the
    start block is no eigenspace: its residuals are not small)."""
    A = W.laplacian_2d(10).to_scipy()
    n, p, k = A.shape[0], 2, 4
    X0 = W.start_block(n, k, 5)
    Qx = np.linalg.qr(X0)[0]
    r = O.solve(A, None, p, 12, k, 1, 1e-10, X0, lambda v: Qx @ (Qx.T @ v), max_cycles=50)
    assert r["status"] == O.BREAKDOWN and r["cycles"] == 1
    assert r["mv_A"] == k and np.all(r["resid"] > 1e-3)


def test_rank_deficient_start_block_is_rejected_and_counters_match_the_operator():
    """R2: a start block with a dependent column cannot be B-orthonormalised
    (error); with B = I no B matvec is counted, with a pencil the start block's
    k B matvecs are."""
    A = W.laplacian_2d(10).to_scipy()
    X0 = W.start_block(100, 4, 5)
    X0[:, 3] = 2.0 * X0[:, 1] - X0[:, 0]
    with pytest.raises(ValueError):
        O.solve(A, None, 2, 12, 4, 1, 1e-8, X0, "jacobi")
    r = O.solve(A, None, 2, 12, 4, 1, 1e-8, W.start_block(100, 4, 5), "jacobi")
    assert r["mv_B"] == 0
    N = 4
    Ap, Bp = W.fem_q1_pencil(N, np.ones((N, N, N)))
    rp = O.solve(Ap.to_scipy(), Bp.to_scipy(), 2, 12, 4, 1, 1e-8, W.start_block(Ap.n, 4, 5), "jacobi", max_cycles=1)
    assert rp["mv_B"] == 4 + (rp["mv_A"] - 4)   # the start block, then one B matvec per new vector


# ---------------------------------------------------------------- hard locking (R13), M(rho_i) (R14)
@pytest.mark.parametrize("precond", ["jacobi", "jacobi_shifted"])
def test_hard_locking_closed_form_accounting_and_locked_orthogonality(precond):
    """Hard locking (R13) on the 2D Laplacian: the locked and returned pairs
    meet the closed form within Krylov-Weinstein (|theta - lambda| <= ||r||),
    the locked vectors stay B-orthogonal to every active basis they sit beside
    (Q^T B U = 0 in each cycle), the output is orthonormal, and every cycle
    still costs q - p_hat matvecs (Tables 2-5's accounting)."""
    N, p, q, k, l = 24, 5, 16, 7, 1
    A = W.laplacian_2d(N)
    As = A.to_scipy()
    r = O.solve(As, None, p, q, k, l, 1e-10, W.start_block(A.n, k, 1), precond, record=True, locking="hard")
    assert r["status"] == O.OK and r["locked"] == p
    lam = lap2d_eigs(N, 2 * p + 2)
    rabs = r["resid"] * r["normA"]
    assert np.all(np.diff(r["evals"]) >= 0)
    for i in range(p):
        assert np.min(np.abs(lam - r["evals"][i])) <= rabs[i] + 1e-15
        assert abs(r["evals"][i] - lam[i]) <= 1e-9 * lam[i]
    X = r["evecs"]
    assert np.allclose(X.T @ X, np.eye(p), atol=1e-10)
    assert r["mv_A"] == k + (q - k) * r["cycles"]
    assert any(tr["nq"] > 0 for tr in r["trace"])
    for tr in r["trace"]:
        if tr["nq"]:
            assert np.abs(tr["QtBU"]).max() <= 1e-12


def test_hard_locking_locks_each_leading_converged_run_and_trims_x_prev():
    """R13 cycle by cycle against the recorded residuals: a cycle locks
    exactly the leading run of its active pairs below tol (several at once
    when they converge together), and the next cycle's X_prev holds the
    min(l, active wanted) leading Ritz vectors less the ones just locked."""
    p, q, k, l, tol = 6, 16, 8, 2, 1e-10
    A = W.diffusion_3d(7, W.lognormal_field(7, 1.0, 5)).to_scipy()   # distinct eigenvalues
    # three start columns within 1e-12 of eigenvectors: those pairs converge together
    X0 = W.start_block(A.shape[0], k, 1).copy()
    V = np.linalg.eigh(A.toarray())[1]
    X0[:, :3] = V[:, :3] + 1e-12 * X0[:, :3]
    r = O.solve(A, None, p, q, k, l, tol, X0, "jacobi", record=True, locking="hard")
    assert r["status"] == O.OK
    h, tr = r["history"], r["trace"]
    multi = 0
    for c in range(len(h) - 1):
        res, nq = h[c]["resid"], h[c]["nq"]
        run = 0
        while run < res.size and res[run] <= tol:
            run += 1
        s = h[c + 1]["nq"] - nq
        assert s == run, c
        multi += s >= 2
        assert tr[c + 1]["nprev"] == max(0, min(l, p - nq) - s), c
    assert multi >= 1


def test_returned_pairs_are_ritz_pairs_when_the_cycle_limit_stops_the_solve():
    """Every returned value is the Rayleigh quotient of its returned vector
    (B-normalised), also when max_cycles ends a solve with some pairs locked
    and some still active (hard locking) or unconverged (soft locking)."""
    N = 24
    A = W.laplacian_2d(N).to_scipy()
    for locking, cycles in (("hard", 30), ("soft", 4)):
        r = O.solve(A, None, 6, 16, 8, 2, 1e-10, W.start_block(A.shape[0], 8, 1), "jacobi", max_cycles=cycles,
                    locking=locking)
        assert r["status"] == O.NOT_CONVERGED
        if locking == "hard":
            assert 0 < r["locked"] < 6
        X = r["evecs"]
        assert np.allclose(X.T @ X, np.eye(6), atol=1e-10)
        assert np.abs(np.einsum("ij,ij->j", X, A @ X) - r["evals"]).max() <= 1e-10 * r["normA"]


def test_x_prev_holds_the_targets_up_to_p():
    """R7 with a +K block larger than the wanted pairs left: the next cycle's
    X_prev is x_t .. x_min(t+l-1, p) of this cycle's start, less x_t when the
    target converged (checked cycle by cycle against the recorded residuals)."""
    A = W.laplacian_2d(20).to_scipy()
    p, q, k, l, tol = 4, 16, 6, 3, 1e-10
    r = O.solve(A, None, p, q, k, l, tol, W.start_block(A.shape[0], k, 3), "jacobi", record=True)
    assert r["status"] == O.OK
    h, tr = r["history"], r["trace"]
    near_end = 0
    for c in range(len(h) - 1):
        t = h[c]["t"]
        adv = 1 if h[c]["resid"][t] <= tol else 0
        assert tr[c + 1]["nprev"] == min(t + l, p) - t - adv, c
        near_end += t + l > p
    assert near_end >= 1


def test_hard_locking_cycle_before_any_lock_is_the_soft_cycle():
    """R13 on a pencil: until a pair is locked the active basis is the whole
    basis, so each hard-locking cycle is an Algorithm 1 cycle with the
    smallest pair as target -- the same Ritz values as the soft path, cycle
    by cycle, as long as both target the first pair."""
    N = 5
    A, B = W.fem_q1_pencil(N, np.random.default_rng(7).uniform(1, 10, (N, N, N)))
    As, Bs = A.to_scipy(), B.to_scipy()
    p, q, k, l = 3, 16, 6, 1
    X0 = W.start_block(A.n, k, 8)
    rs = O.solve(As, Bs, p, q, k, l, 1e-10, X0, "jacobi", record=True)
    rh = O.solve(As, Bs, p, q, k, l, 1e-10, X0, "jacobi", record=True, locking="hard")
    same = 0
    for hs, hh, ts, th in zip(rs["history"], rh["history"], rs["trace"], rh["trace"]):
        if hs["t"] != 0 or hh["nq"] != 0:
            break
        assert np.allclose(th["theta"], ts["theta"], rtol=1e-12, atol=0)
        same += 1
    assert same >= 3


def test_hard_locking_generalized_pencil_brute_force():
    """Hard locking on the Q1 stiffness/mass pencil against a dense
    generalized eigensolve (B-inner products throughout, R3 + R13)."""
    N = 5
    A, B = W.fem_q1_pencil(N, np.random.default_rng(3).uniform(1, 10, (N, N, N)))
    As, Bs = A.to_scipy(), B.to_scipy()
    p, q, k, l = 4, 16, 6, 1
    r = O.solve(As, Bs, p, q, k, l, 1e-10, W.start_block(A.n, k, 2), "jacobi", locking="hard")
    assert r["status"] == O.OK
    brute = sl.eigh(As.toarray(), Bs.toarray(), eigvals_only=True)[:p]
    assert np.all(np.abs(r["evals"] - brute) <= 1e-9 * brute)
    X = r["evecs"]
    assert np.allclose(X.T @ (Bs @ X), np.eye(p), atol=1e-10)


def test_hard_locking_with_one_wanted_pair_is_soft_locking():
    """With p = 1 nothing is locked before the solve ends, so hard locking
    must reproduce Algorithm 1's iterates exactly: same cycles, matvecs and
    Ritz values cycle by cycle."""
    A = W.diffusion_3d(8, W.lognormal_field(8, 1.0, 2))
    As = A.to_scipy()
    X0 = W.start_block(A.n, 4, 5)
    soft = O.solve(As, None, 1, 12, 4, 1, 1e-10, X0, "jacobi")
    hard = O.solve(As, None, 1, 12, 4, 1, 1e-10, X0, "jacobi", locking="hard")
    assert soft["cycles"] == hard["cycles"] and soft["mv_A"] == hard["mv_A"]
    for hs, hh in zip(soft["history"], hard["history"]):
        assert np.allclose(hs["theta"][:1], hh["theta"][:1], rtol=1e-13, atol=0)
    assert np.allclose(soft["evals"], hard["evals"], rtol=1e-13, atol=0)


def test_shifted_jacobi_on_a_constant_diagonal_is_the_unpreconditioned_method():
    """R14 on the 2D Laplacian (constant diagonal 4, B = I): M_i is the scalar
    1/(4 - rho_i), which does not change the Krylov space, the CGS2 basis or
    any Ritz value -- the iterates must be those of M = I, cycle by cycle."""
    A = W.laplacian_2d(20)
    As = A.to_scipy()
    X0 = W.start_block(A.n, 6, 7)
    none = O.solve(As, None, 3, 14, 6, 1, 1e-10, X0, "none")
    shif = O.solve(As, None, 3, 14, 6, 1, 1e-10, X0, "jacobi_shifted")
    assert none["cycles"] == shif["cycles"] and none["mv_A"] == shif["mv_A"]
    for a, b in zip(none["history"], shif["history"]):
        assert np.allclose(a["theta"], b["theta"], rtol=1e-11, atol=0)


def test_shifted_jacobi_preconditioner_definition_and_floor():
    """M_i = diag(max(a_jj - rho b_jj, 1e-3 a_jj))^-1 (R14), with and without B."""
    A = sp.diags([2.0, 5.0, 10.0]).tocsr()
    B = sp.diags([1.0, 2.0, 0.5]).tocsr()
    v = np.array([1.0, 1.0, 1.0])
    assert np.allclose(O.shifted_jacobi_preconditioner(A, None, 1.0)(v), [1.0, 1 / 4.0, 1 / 9.0])
    # rho = 3: a - rho b = (-1, -1, 8.5) -> floored to (2e-3, 5e-3, 8.5)
    assert np.allclose(O.shifted_jacobi_preconditioner(A, B, 3.0)(v), [500.0, 200.0, 1 / 8.5])


# ---------------------------------------------------------------- parameter studies (Sec. 5.2, Figs. 1-3)
def test_unrestarted_lanczos_closed_form_and_quasi_optimality():
    """The unrestarted Lanczos yardstick reaches the closed-form smallest
    eigenvalue of the 2D Laplacian (Kato-Temple at its residual), and TRPL+K
    with the paper's small basis (q = 18, p_hat = 8, l = 1, no
    preconditioner) needs no more than 1.5 times its matvecs (Sec. 5.2:
    close to optimal with a very small basis)."""
    N = 40
    A = W.laplacian_2d(N)
    As = A.to_scipy()
    x0 = W.start_block(A.n, 8, 12)
    th, mv = O.lanczos_unrestarted(As, x0[:, 0], 1e-9)
    lam = lap2d_eigs(N, 2)
    assert abs(th - lam[0]) <= (1e-9 * O.norm1(As)) ** 2 / (lam[1] - lam[0]) + 1e-14
    r = O.solve(As, None, 1, 18, 8, 1, 1e-9, x0, "none")
    assert r["status"] == O.OK
    assert mv <= r["mv_A"] <= 1.5 * mv


def test_unrestarted_lanczos_stops_when_its_krylov_space_is_invariant():
    """With two distinct eigenvalues the Krylov space of any start vector is
    invariant after two steps: the residual identity gives zero there, so the
    yardstick stops after exactly two matvecs with the smallest eigenvalue."""
    rng = np.random.default_rng(13)
    Q = np.linalg.qr(rng.standard_normal((30, 30)))[0]
    lam = np.r_[np.full(10, 0.5), np.full(20, 3.0)]
    A = sp.csr_matrix((Q * lam) @ Q.T)
    th, mv = O.lanczos_unrestarted(A, rng.standard_normal(30), 1e-12)
    assert mv == 2 and abs(th - 0.5) <= 1e-12


def test_one_preconditioner_application_per_new_lanczos_vector():
    """Accounting of Algorithm 1's M applications: each cycle applies M to
    the restart residual and after each inner matvec but the last, i.e. once
    per new Lanczos vector.  With l = 0 every matvec after the start block
    belongs to an inner step, so the counts agree; +K vectors take matvecs
    but no M."""
    A = W.diffusion_3d(6, W.lognormal_field(6, 1.0, 4)).to_scipy()
    X0 = W.start_block(A.shape[0], 6, 2)
    r0 = O.solve(A, None, 3, 16, 6, 0, 1e-8, X0, "jacobi")
    assert r0["status"] == O.OK and r0["prec"] == r0["mv_A"] - 6
    r1 = O.solve(A, None, 3, 16, 6, 1, 1e-8, X0, "jacobi")
    assert r1["status"] == O.OK and r1["mv_A"] - 6 - r1["cycles"] < r1["prec"] < r1["mv_A"] - 6


def test_one_previous_vector_cuts_matvecs_for_five_pairs():
    """Fig. 3's trend without a preconditioner, p = 5: l = 1 needs clearly
    fewer matvecs than l = 0 (TRLan, Sec. 5.2) on the 2D Laplacian."""
    A = W.laplacian_2d(60)
    As = A.to_scipy()
    x0 = W.start_block(A.n, 8, 12)
    mv = {l: O.solve(As, None, 5, 18, 8, l, 1e-8, x0, "none")["mv_A"] for l in (0, 1)}
    assert mv[1] < 0.9 * mv[0], mv


# ---------------------------------------------------------------- block TRPL+K (R15)
def test_block_first_cycle_spans_the_block_krylov_space():
    """With M = I and no +K vectors, the first cycle of block TRPL+K (b = 2)
    builds span [X, R, C R, C^2 R, ...] with R the residuals of the two
    targets and C = (I - X X^T) A the projected operator of Sec. 3 (the block
    Krylov space; the shifts do not change it): every basis column lies in the
    explicitly built space, column block by column block."""
    A = W.diffusion_3d(7, W.lognormal_field(7, 1.0, 2)).to_scipy()
    n = A.shape[0]
    p, q, k, b = 2, 14, 4, 2
    X0 = W.start_block(n, k, 3)
    r = O.solve(A, None, p, q, k, 0, 1e-14, X0, "none", max_cycles=1, record=True, block=b)
    tr = r["trace"][0]
    U = tr["U"]
    X, AX, _, theta, _, _ = O.initial_rayleigh_ritz(A, lambda v: v.copy(), X0)
    R = AX[:, :b] - X[:, :b] * theta[:b]
    blocks = [X, R]
    while sum(Z.shape[1] for Z in blocks) < U.shape[1]:
        Z = A @ blocks[-1]
        blocks.append(Z - X @ (X.T @ Z))
    Kall = np.hstack(blocks)
    assert U.shape[1] == q
    for c in range(k, q + 1):
        K = np.linalg.qr(Kall[:, :c])[0]
        assert np.linalg.norm(U[:, :c] - K @ (K.T @ U[:, :c])) <= 1e-9 * np.sqrt(c), c


def test_block_sequences_keep_their_own_shifts():
    """With a preconditioner that is not a multiple of I the shift of each
    sequence shapes its Krylov space.  On a block-diagonal operator whose two
    targets lie in different blocks (start columns supported on one block
    each, so X, the residuals and Jacobi's M all respect the blocks), the two
    sequences of block TRPL+K (b = 2) never mix: the first cycle's basis must
    lie in span[X, K(C_1, P M r_1), K(C_2, P M r_2)] with
    C_i = P M (A - theta_i I) and P = I - X X^T, each Krylov space built
    explicitly with its own sequence's shift (R15)."""
    N = 5
    A1 = W.diffusion_3d(N, W.lognormal_field(N, 1.0, 11)).to_scipy()
    A2 = W.diffusion_3d(N, W.lognormal_field(N, 1.0, 12)).to_scipy()
    A = sp.block_diag([A1, A2]).tocsr()
    m = A1.shape[0]
    n = 2 * m
    p, q, k, b = 2, 14, 4, 2
    R0 = W.start_block(n, k, 7)
    X0 = np.zeros((n, k))
    for c in range(k):   # columns alternate between the two blocks
        h = c % 2
        X0[h * m:(h + 1) * m, c] = R0[h * m:(h + 1) * m, c]
    X, AX, _, theta, _, _ = O.initial_rayleigh_ritz(A, lambda v: v.copy(), X0)
    side = [int(np.linalg.norm(X[m:, c]) > np.linalg.norm(X[:m, c])) for c in range(b)]
    assert sorted(side) == [0, 1] and theta[0] != theta[1]   # the targets sit in different blocks
    r = O.solve(A, None, p, q, k, 0, 1e-14, X0, "jacobi", max_cycles=1, record=True, block=b)
    U = r["trace"][0]["U"]
    dinv = 1.0 / A.diagonal()
    P = lambda v: v - X @ (X.T @ v)
    per = (q - k) // b
    seqs = []
    for i in range(b):   # orthonormal basis of K(C_i, P M r_i), grown one vector at a time
        v = P(dinv * (AX[:, i] - theta[i] * X[:, i]))
        Q = [v / np.linalg.norm(v)]
        while len(Q) < per:
            z = P(dinv * (A @ Q[-1] - theta[i] * Q[-1]))
            for _ in range(2):
                for u in Q:
                    z = z - u * (u @ z)
            Q.append(z / np.linalg.norm(z))
        seqs.append(np.array(Q).T)
    for c in range(k + 1, q + 1):
        counts = [len([a for a in range(k, c) if (a - k) % b == i]) for i in range(b)]
        K = np.linalg.qr(np.hstack([X] + [seqs[i][:, :counts[i]] for i in range(b)]))[0]
        assert np.linalg.norm(U[:, :c] - K @ (K.T @ U[:, :c])) <= 1e-9 * np.sqrt(c), c


def test_block_step_taken_as_one_block_gives_the_same_basis():
    """R15 builds the block basis column by column; since the b new vectors of
    a block come from the previous block's matvecs alone, the same basis is
    reached block by block: B-orthogonalise all b vectors against the basis
    at once (two passes), orthonormalise them within the block (CGS2 column
    by column), then take their b matvecs together.  Gram-Schmidt with
    positive normalisation is unique, so both orders give the same vectors
    (here: the first cycle on the Q1 pencil, Jacobi, b = 3, to rounding)."""
    N = 5
    A, B = W.fem_q1_pencil(N, np.random.default_rng(9).uniform(1, 10, (N, N, N)))
    As, Bs = A.to_scipy(), B.to_scipy()
    n = A.n
    p, q, k, b = 3, 18, 6, 3
    X0 = W.start_block(n, k, 6)
    r = O.solve(As, Bs, p, q, k, 0, 1e-14, X0, "jacobi", max_cycles=1, record=True, block=b)
    U_ref = r["trace"][0]["U"]
    applyB = lambda v: Bs @ v
    X, AX, BX, theta, _, _ = O.initial_rayleigh_ritz(As, applyB, X0)
    dinv = 1.0 / As.diagonal()
    U, BU = X.copy(), BX.copy()
    V = np.column_stack([dinv * (AX[:, i] - theta[i] * BX[:, i]) for i in range(b)])
    while U.shape[1] < q:
        V = V[:, : q - U.shape[1]]
        for _ in range(2):                      # the block against the basis
            V = V - U @ (BU.T @ V)
        new, Bnew = [], []
        for c in range(V.shape[1]):             # within the block
            v = V[:, c]
            for _ in range(2):
                for u, Bu in zip(new, Bnew):
                    v = v - u * (Bu @ v)
            Bv = applyB(v)
            beta = np.sqrt(v @ Bv)
            new.append(v / beta)
            Bnew.append(Bv / beta)
        Unew, BUnew = np.column_stack(new), np.column_stack(Bnew)
        Z = As @ Unew                            # the block's b matvecs together
        V = np.column_stack([dinv * (Z[:, i] - theta[i] * BUnew[:, i]) for i in range(Unew.shape[1])])
        U, BU = np.hstack([U, Unew]), np.hstack([BU, BUnew])
    assert U.shape == U_ref.shape
    assert np.abs(U - U_ref).max() <= 1e-12 * np.abs(U_ref).max()
    assert np.abs(U.T @ (Bs @ U) - np.eye(q)).max() <= 1e-10


def test_block_closed_form_degenerate_pairs_and_accounting():
    """Block TRPL+K (b = 2) on the 2D Laplacian, whose wanted set holds
    exactly degenerate pairs: closed-form eigenvalues, orthonormal vectors,
    and p_hat + (q - p_hat) matvecs per cycle."""
    N = 24
    A = W.laplacian_2d(N).to_scipy()
    p, q, k, l = 6, 20, 8, 1
    r = O.solve(A, None, p, q, k, l, 1e-10, W.start_block(A.shape[0], k, 2), "jacobi", block=2)
    assert r["status"] == O.OK
    lam = lap2d_eigs(N, p)
    assert np.all(np.abs(r["evals"] - lam) <= 1e-9 * lam)
    X = r["evecs"]
    assert np.allclose(X.T @ X, np.eye(p), atol=1e-10)
    assert r["mv_A"] == k + (q - k) * r["cycles"]


def test_block_generalized_pencil_brute_force():
    N = 5
    A, B = W.fem_q1_pencil(N, np.random.default_rng(5).uniform(1, 10, (N, N, N)))
    As, Bs = A.to_scipy(), B.to_scipy()
    p, q, k, l = 4, 18, 6, 1
    r = O.solve(As, Bs, p, q, k, l, 1e-10, W.start_block(A.n, k, 4), "jacobi", block=3)
    assert r["status"] == O.OK
    brute = sl.eigh(As.toarray(), Bs.toarray(), eigvals_only=True)[:p]
    assert np.all(np.abs(r["evals"] - brute) <= 1e-9 * brute)
    X = r["evecs"]
    assert np.allclose(X.T @ (Bs @ X), np.eye(p), atol=1e-10)
