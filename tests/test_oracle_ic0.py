"""Pins of the IC(0) oracle (oracle/ic0.py) against the mathematics: the
defining property (L L^T)_ij = a_ij on the lower pattern, exact Cholesky for
a tridiagonal matrix (no fill exists), Jacobi-sweep triangular solves equal to
the truncated Neumann series and, once the sweeps reach the depth of the
dependency graph, to an exact triangular solve; the preconditioner is
symmetric positive definite and, with exact solves, (L L^T)^-1."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from oracle import ic0 as I
from paper_1711_10128_gb300 import workloads as W


def test_factor_matches_a_on_the_lower_pattern():
    ops = [W.anisotropic_diffusion(8, 2004).to_scipy(),
           W.fem_q1_pencil(5, np.random.default_rng(1).uniform(1, 10, (5, 5, 5)))[0].to_scipy(),
           W.chung_lu_laplacian(600, 6.0, 2.1, 2).to_scipy()]
    for A in ops:
        L = I.ic0(A)
        T = sp.tril(A).tocsr()
        P = (L @ L.T).tocsr()
        rows = np.repeat(np.arange(A.shape[0]), np.diff(T.indptr))
        got = np.asarray(P[rows, T.indices]).ravel()
        assert np.allclose(got, T.data, rtol=1e-12, atol=1e-12 * np.abs(T.data).max())
        assert np.all(L.diagonal() > 0)
        # the pattern is A's lower triangle: no fill
        assert L.nnz == T.nnz and np.array_equal(L.indices, T.indices)


def test_tridiagonal_factor_is_the_exact_cholesky_factor():
    n = 40
    A = sp.diags([-np.ones(n - 1), 2.5 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
    L = I.ic0(A).toarray()
    assert np.allclose(L, np.linalg.cholesky(A.toarray()), rtol=0, atol=1e-14)


def test_sweeps_are_the_truncated_neumann_series_and_converge_to_the_exact_solve():
    A = W.laplacian_2d(10).to_scipy()
    L = I.ic0(A)
    d = L.diagonal()
    Ls = (L - sp.diags(d)).toarray()
    Dinv = np.diag(1.0 / d)
    b = np.random.default_rng(0).standard_normal(A.shape[0])
    for s in (0, 1, 2, 3):
        Ps = sum(np.linalg.matrix_power(-Dinv @ Ls, t) for t in range(s + 1)) @ Dinv
        assert np.allclose(I.sweep_solve(L, b, s), Ps @ b, rtol=1e-12, atol=1e-12)
        assert np.allclose(I.sweep_solve(L, b, s, transpose=True), Ps.T @ b, rtol=1e-12, atol=1e-12)
    # the dependency graph of the 10 x 10 grid is 19 levels deep: 19 sweeps are exact
    exact = sla.spsolve_triangular(L, b, lower=True)
    assert np.allclose(I.sweep_solve(L, b, 19), exact, rtol=1e-12, atol=1e-13)
    exactT = sla.spsolve_triangular(L.T.tocsr(), b, lower=False)
    assert np.allclose(I.sweep_solve(L, b, 19, transpose=True), exactT, rtol=1e-12, atol=1e-13)


def test_preconditioner_is_spd_and_tends_to_the_inverse_of_the_factor_product():
    A = W.diffusion_3d(5, W.lognormal_field(5, 1.0, 3)).to_scipy()
    L = I.ic0(A)
    n = A.shape[0]
    E = np.eye(n)
    M2 = np.column_stack([I.apply_M(L, E[:, j], 2) for j in range(n)])
    assert np.allclose(M2, M2.T, rtol=0, atol=1e-13 * np.abs(M2).max())
    assert np.linalg.eigvalsh(M2).min() > 0
    Mx = np.column_stack([I.apply_M(L, E[:, j], 3 * 5) for j in range(n)])   # depth 13 on the 5^3 grid
    LLt = (L @ L.T).toarray()
    assert np.allclose(Mx @ LLt, np.eye(n), atol=1e-10)


def test_non_positive_pivot_is_a_breakdown():
    """I1: a symmetric matrix that is not positive definite on its pattern has
    a non-positive pivot, which is raised, not taken."""
    with pytest.raises(ValueError):
        I.ic0(sp.csr_matrix(np.array([[1.0, 2.0], [2.0, 1.0]])))


def test_preconditioner_applies_the_truncated_series_with_its_sweep_count():
    """I3 as the solver sees it: preconditioner(A, s) applies P_s^T P_s with
    P_s the explicit truncated Neumann series of s sweeps."""
    A = W.diffusion_3d(5, W.lognormal_field(5, 1.0, 3)).to_scipy()
    L = I.ic0(A)
    d = L.diagonal()
    Ls = (L - sp.diags(d)).toarray()
    Dinv = np.diag(1.0 / d)
    b = np.random.default_rng(1).standard_normal(A.shape[0])
    for s in (1, 2, 3):
        Ps = sum(np.linalg.matrix_power(-Dinv @ Ls, t) for t in range(s + 1)) @ Dinv
        assert np.allclose(I.preconditioner(A, s)(b), Ps.T @ (Ps @ b), rtol=1e-12, atol=1e-14)
