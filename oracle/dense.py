"""Cyclic Jacobi eigensolver for small dense symmetric matrices -- TEST
INFRASTRUCTURE ONLY (see ``oracle``).

The textbook row-cyclic Jacobi method (Golub and Van Loan, Matrix
Computations, Sec. 8.5): sweep over the pairs (i, j), i < j, in row order;
for each, the symmetric 2x2 Schur decomposition gives the rotation that
zeroes A[i, j]; apply it on both sides and accumulate it into V.  Stops when
the off-diagonal Frobenius norm is <= tol * ||A||_F.  Pure Python loops, so
only for tiny matrices (the brute-force check of the Rayleigh-Ritz step and
of whole spectra of tiny operators).
"""
from __future__ import annotations

import math

import numpy as np


def _sym_schur2(app, aqq, apq):
    """(c, s) with [c s; -s c]^T [app apq; apq aqq] [c s; -s c] diagonal."""
    app, aqq, apq = float(app), float(aqq), float(apq)
    if apq == 0.0 or abs(aqq - app) > 1e300 * abs(apq):
        return 1.0, 0.0
    tau = (aqq - app) / (2.0 * apq)
    if tau >= 0.0:
        t = 1.0 / (tau + math.hypot(1.0, tau))
    else:
        t = -1.0 / (-tau + math.hypot(1.0, tau))
    c = 1.0 / math.hypot(1.0, t)
    return c, t * c


def jacobi_eigh(A, tol=1e-15, max_sweeps=100):
    """Eigenvalues (ascending) and orthonormal eigenvectors of symmetric A."""
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    V = np.eye(n)
    fro = np.linalg.norm(A)
    for _ in range(max_sweeps):
        off = float(np.linalg.norm(A - np.diag(np.diag(A))))
        if off <= tol * fro:
            break
        for i in range(n - 1):
            for j in range(i + 1, n):
                c, s = _sym_schur2(A[i, i], A[j, j], A[i, j])
                if s == 0.0:
                    continue
                # A <- J^T A J with J = I except J[i,i]=J[j,j]=c, J[i,j]=s, J[j,i]=-s
                ai, aj = A[:, i].copy(), A[:, j].copy()
                A[:, i] = c * ai - s * aj
                A[:, j] = s * ai + c * aj
                ai, aj = A[i, :].copy(), A[j, :].copy()
                A[i, :] = c * ai - s * aj
                A[j, :] = s * ai + c * aj
                vi, vj = V[:, i].copy(), V[:, j].copy()
                V[:, i] = c * vi - s * vj
                V[:, j] = s * vi + c * vj
    w = np.diag(A).copy()
    order = np.argsort(w, kind="stable")
    return w[order], V[:, order]
