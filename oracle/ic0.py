"""Incomplete Cholesky IC(0) preconditioner -- TEST INFRASTRUCTURE ONLY (see
``oracle``).

The paper preconditions with incomplete factorizations: ILU(0) without fill
for the standard problems (Sec. 5.4, Tables 4-5) and incomplete LDL^T for the
pencils (Sec. 5.5).  For symmetric positive definite A the no-fill
factorization is IC(0).  Plain FP64 numpy; readings (also in the design
notes):

I1 Pattern: L is lower triangular on the pattern of A's lower triangle with
   the diagonal (no fill).  IC(0) is the textbook left-looking recurrence over
   that pattern, row by row, columns ascending:
     s = a_ij - sum_{k < j, k in P_i and P_j} l_ik l_jk,
     l_ij = s / l_jj (j < i),  l_ii = sqrt(s);
   equivalently (L L^T)_ij = a_ij for every (i, j) of the pattern.
   A non-positive pivot s is a breakdown (raised).
I2 Triangular solves by Jacobi sweeps (the form a GPU applies without a
   sequence of dependent levels): with D = diag(L) and L_s = L - D,
     x_0 = D^-1 b,  x_{t+1} = D^-1 (b - L_s x_t)  (t = 0..s-1),
   i.e. x_s = P_s b with P_s = sum_{t=0..s} (-D^-1 L_s)^t D^-1, the
   truncated Neumann series of L^-1 (exact once s reaches the depth of the
   dependency graph: D^-1 L_s is nilpotent).  The transposed solve sweeps
   with L^T the same way and equals P_s^T.
I3 The preconditioner is M = P_s^T P_s: symmetric positive definite for every
   s (P_s is lower triangular with the positive diagonal D^-1), and
   (L L^T)^-1 in the limit of exact solves.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def lower_pattern_csr(A):
    """tril(A) with the diagonal, columns ascending, as CSR (I1)."""
    L = sp.tril(sp.csr_matrix(A)).tocsr()
    L.sort_indices()
    return L


def ic0(A):
    """The IC(0) factor L (CSR on A's lower pattern) of SPD A (I1)."""
    T = lower_pattern_csr(A)
    n = T.shape[0]
    rp, cl, av = T.indptr, T.indices, T.data
    lv = np.zeros_like(av)
    row = [dict() for _ in range(n)]       # row[i][k] = l_ik (computed so far)
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            j = int(cl[e])
            Ri, Rj = row[i], row[j]
            s = av[e] - sum(v * Rj[k] for k, v in Ri.items() if k < j and k in Rj)
            if j < i:
                lij = s / row[j][j]
            else:
                if not s > 0.0:
                    raise ValueError(f"IC(0) breakdown at row {i}: pivot {s}")
                lij = np.sqrt(s)
            Ri[j] = lij
            lv[e] = lij
    return sp.csr_matrix((lv, cl.copy(), rp.copy()), shape=(n, n))


def sweep_solve(L, b, sweeps, transpose=False):
    """x = P_s b (or P_s^T b) by `sweeps` Jacobi sweeps on L (I2)."""
    L = sp.csr_matrix(L)
    d = L.diagonal()
    Ls = (L - sp.diags(d)).tocsr()
    if transpose:
        Ls = Ls.T.tocsr()
    x = b / d
    for _ in range(sweeps):
        x = (b - Ls @ x) / d
    return x


def apply_M(L, b, sweeps):
    """M b = P_s^T (P_s b) (I3)."""
    return sweep_solve(L, sweep_solve(L, b, sweeps), sweeps, transpose=True)


def preconditioner(A, sweeps):
    """The IC(0) preconditioner of A with `sweeps` Jacobi sweeps per solve,
    as a function for oracle.trplk.solve."""
    L = ic0(A)
    return lambda v: apply_M(L, v, sweeps)
