"""Factorised sparse approximate inverse (FSAI) preconditioners, classical and
MLP-predicted, with the training loss and its gradient -- TEST INFRASTRUCTURE
ONLY (see ``oracle``).

The paper (Sec. 3) allows any preconditioner M approximating (A - rho I)^-1;
its experiments use ILU/LDL (Sec. 5).  This module restates the factorised
form M = G^T G with G sparse lower triangular on the pattern of A's lower
triangle, which is the learned preconditioner of this repository (not a
method of the paper).  Plain FP64 numpy; every function follows its
definition literally.

Readings (also in the design notes):
F1 Pattern P_i of row i: the columns j <= i with a_ij != 0 (A's lower
   triangle with the diagonal).
F2 Classical FSAI (Kolotilina and Yeremin): g_hat_i = A[P_i, P_i]^-1 e_i,
   g_i = g_hat_i / sqrt(g_hat_ii).  It minimises the Kaporin measure
   K(G) = log(mean_i d_i) - (2/n) sum_i log g_ii, d_i = (G A G^T)_ii,
   over G with that pattern (the pin of this module).
F3 7-point operators on an Nx x Ny x Nz grid (x fastest): neighbour
   directions by column offset (-1, +1, -Nx, +Nx, -NxNy, +NxNy); features
   [log a_ii, c_{-x}, c_{+x}, c_{-y}, c_{+y}, c_{-z}, c_{+z},
   (a_ii - sum_j |a_ij|)/a_ii] with the symmetrically scaled couplings
   c_j = a_ij / sqrt(a_ii a_jj), 0 where missing.
F4 MLP 8 -> 64 -> 64 -> 7, ReLU hidden layers; outputs map to the
   directions (-z, -y, -x, c, +x, +y, +z); g_ii = softplus(o_c)/sqrt(a_ii),
   g_ij = o_dir/sqrt(a_jj) for the lower neighbours j; the upper three
   outputs are unused (their gradient is zero).  In these variables classical
   FSAI of a 7-point operator is a smooth function of the features
   (o_dir = -c_dir / sqrt(1 - sum_lower c^2), softplus(o_c) =
   1 / sqrt(1 - sum_lower c^2)), which the network can represent; row-local
   ratios a_ij/a_ii and a 1/sqrt(a_ii) scaling could not, since classical
   FSAI depends on the neighbours' diagonals.
F5 Loss over solver vectors v (columns of V): the energy-norm error of Mv as
   an approximation of A^-1 v, less its G-independent part,
   E_v = (Mv)^T A (Mv) - 2 ||Gv||^2 = ||A^-1 v - Mv||_A^2 - v^T A^-1 v,
   scaled by c_v = 1/(v^T D^-1 v) (D = diag A) and averaged over v; plus
   gamma = 0.1 times the Kaporin measure K(G).
F6 BF16 mode (quant="bf16"): the network of F4 with the features (first
   rounded to FP32), the weight matrices W1, W2, W3 and both hidden
   activations rounded to bfloat16 (round to nearest, ties to even, through
   FP32), everything else in FP64; biases are not rounded.  Its backward is
   the F4/F5 chain rule evaluated at the rounded values (the rounding has zero
   derivative almost everywhere, so this is the gradient the rounded network
   is trained with).  Pins: the rounding against a library's bfloat16
   conversion; the gradient with respect to b3, on which the rounded loss
   depends smoothly, against finite differences.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

GAMMA = 0.1
DIRS = ("-z", "-y", "-x", "c", "+x", "+y", "+z")


def lower_pattern(A):
    """CSR (rowptr, col) of the lower triangle of A with the diagonal (F1)."""
    L = sp.tril(sp.csr_matrix(A)).tocsr()
    L.sort_indices()
    return L.indptr.astype(np.int64), L.indices.astype(np.int32)


def classical_fsai(A):
    """G values on A's lower pattern (F2), as a CSR matrix."""
    A = sp.csr_matrix(A)
    rp, cl = lower_pattern(A)
    n = A.shape[0]
    Ad = A.toarray() if n <= 4000 else None
    vals = np.zeros(cl.size)
    for i in range(n):
        P = cl[rp[i]:rp[i + 1]]
        sub = Ad[np.ix_(P, P)] if Ad is not None else A[P][:, P].toarray()
        e = np.zeros(P.size)
        e[-1] = 1.0                      # the diagonal is the last column of the lower pattern
        gh = np.linalg.solve(sub, e)
        vals[rp[i]:rp[i + 1]] = gh / np.sqrt(gh[-1])
    return sp.csr_matrix((vals, cl, rp), shape=(n, n))


def kaporin(G, A):
    """K(G) = log(mean_i (G A G^T)_ii) - (2/n) sum_i log g_ii (F2)."""
    G = sp.csr_matrix(G)
    d = np.asarray((G @ sp.csr_matrix(A)).multiply(G).sum(axis=1)).ravel()
    return float(np.log(d.mean()) - 2.0 * np.mean(np.log(G.diagonal())))


def features_7pt(A, dims):
    """Per-row features of a 7-point operator (F3), shape (n, 8)."""
    A = sp.csr_matrix(A)
    nx, ny, nz = dims
    n = A.shape[0]
    offs = {-1: 1, 1: 2, -nx: 3, nx: 4, -nx * ny: 5, nx * ny: 6}
    diag = A.diagonal()
    F = np.zeros((n, 8))
    for i in range(n):
        s, e = A.indptr[i], A.indptr[i + 1]
        aii = diag[i]
        off_sum = 0.0
        for jj in range(s, e):
            j, a = A.indices[jj], A.data[jj]
            if j != i:
                off_sum += abs(a)
                F[i, offs[j - i]] = a / np.sqrt(aii * diag[j])
        F[i, 0] = np.log(aii)
        F[i, 7] = (aii - off_sum) / aii
    return F


def init_mlp(seed=0, hidden=64):
    """Weights whose G starts at D^-1/2 (M = Jacobi): W3 = 0, b3 = softplus^-1(1) on c."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((hidden, 8)) * np.sqrt(2.0 / 8)
    W2 = rng.standard_normal((hidden, hidden)) * np.sqrt(2.0 / hidden)
    W3 = np.zeros((7, hidden))
    b1 = np.zeros(hidden)
    b2 = np.zeros(hidden)
    b3 = np.zeros(7)
    b3[3] = np.log(np.expm1(1.0))
    return dict(W1=W1, b1=b1, W2=W2, b2=b2, W3=W3, b3=b3)


def bf16_round(x):
    """x rounded to bfloat16 (F6): to FP32 first (nearest), then to the nearest
    value with 8 significant bits, ties to even, returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _quantiser(quant):
    if quant is None:
        return lambda x: x
    if quant == "bf16":
        return bf16_round
    raise ValueError(f"unknown quantisation {quant!r}")


def mlp_forward(p, F, quant=None):
    """o = W3 relu(W2 relu(W1 f + b1) + b2) + b3 for every row (F4); with
    quant = "bf16" the features, W1..W3 and the hidden activations are
    rounded to bfloat16 (F6)."""
    q = _quantiser(quant)
    F = q(F)
    z1 = F @ q(p["W1"]).T + p["b1"]
    h1 = q(np.maximum(z1, 0.0))
    z2 = h1 @ q(p["W2"]).T + p["b2"]
    h2 = q(np.maximum(z2, 0.0))
    o = h2 @ q(p["W3"]).T + p["b3"]
    return o, (F, z1, h1, z2, h2)


def softplus(x):
    return np.logaddexp(0.0, x)


def sigmoid(x):
    return 0.5 * (1.0 + np.tanh(0.5 * x))


def g_from_outputs(A, dims, o):
    """G (CSR on A's lower pattern) from the MLP outputs (F4)."""
    A = sp.csr_matrix(A)
    nx, ny, nz = dims
    rp, cl = lower_pattern(A)
    n = A.shape[0]
    d = A.diagonal()
    slot = {-nx * ny: 0, -nx: 1, -1: 2, 0: 3}
    vals = np.zeros(cl.size)
    for i in range(n):
        for jj in range(rp[i], rp[i + 1]):
            k = slot[int(cl[jj]) - i]
            vals[jj] = softplus(o[i, 3]) / np.sqrt(d[i]) if k == 3 else o[i, k] / np.sqrt(d[cl[jj]])
    return sp.csr_matrix((vals, cl, rp), shape=(n, n))


def loss_and_grad_G(G, A, V):
    """Loss (F5) and its gradient w.r.t. the values of G (same pattern).

    E_v = (Mv)^T A (Mv) - 2 ||Gv||^2, M = G^T G.  With s = G v, u = G^T s,
    w = A u, t = G w:  dE_v/dG_ij = 2 s_i w_j + 2 t_i v_j - 4 s_i v_j.
    K(G) gradient: dK/dg_ij = 2 (A_{P_i} g_i)_j / (n mean d) - 2 [i == j]/(n g_ii).
    """
    G = sp.csr_matrix(G)
    A = sp.csr_matrix(A)
    n = A.shape[0]
    dinv = 1.0 / A.diagonal()
    rows = np.repeat(np.arange(n), np.diff(G.indptr))
    cols = G.indices
    gE = np.zeros(G.nnz)
    E = 0.0
    nv = V.shape[1]
    for c in range(nv):
        v = V[:, c]
        cv = 1.0 / float(v @ (dinv * v))
        s = G @ v
        u = G.T @ s
        w = A @ u
        t = G @ w
        E += cv * (u @ w - 2.0 * s @ s)
        gE += cv * (2.0 * s[rows] * w[cols] + 2.0 * t[rows] * v[cols] - 4.0 * s[rows] * v[cols])
    E /= nv
    gE /= nv
    # Kaporin term
    GA = G @ A
    d = np.asarray(GA.multiply(G).sum(axis=1)).ravel()
    md = d.mean()
    K = float(np.log(md) - 2.0 * np.mean(np.log(G.diagonal())))
    # (A_{P_i} g_i)_j for j in P_i equals (G A)_ij restricted to the pattern
    GAv = np.asarray(GA[rows, cols]).ravel()
    gK = 2.0 * GAv / (n * md)
    diag = rows == cols
    gK[diag] -= 2.0 / (n * G.data[diag])
    return E + GAMMA * K, gE + GAMMA * gK, dict(E=E, K=K)


def loss_and_grad_mlp(p, A, dims, V, quant=None):
    """Loss of the MLP-predicted G and the gradient w.r.t. every weight (F4, F5;
    F6 with quant = "bf16")."""
    A = sp.csr_matrix(A)
    q = _quantiser(quant)
    F = features_7pt(A, dims)
    o, (F_, z1, h1, z2, h2) = mlp_forward(p, F, quant)
    G = g_from_outputs(A, dims, o)
    L, gG, parts = loss_and_grad_G(G, A, V)
    # dL/do from dL/dG (F4 chain rule)
    nx, ny, nz = dims
    n = A.shape[0]
    rows = np.repeat(np.arange(n), np.diff(G.indptr))
    cols = G.indices
    sq = np.sqrt(A.diagonal())
    slot = {-nx * ny: 0, -nx: 1, -1: 2, 0: 3}
    dO = np.zeros((n, 7))
    for e in range(G.nnz):
        i, j = rows[e], cols[e]
        k = slot[int(j) - int(i)]
        if k == 3:
            dO[i, 3] += gG[e] * sigmoid(o[i, 3]) / sq[i]
        else:
            dO[i, k] += gG[e] / sq[j]
    # back through the MLP
    g = {}
    g["W3"] = dO.T @ h2
    g["b3"] = dO.sum(axis=0)
    dh2 = dO @ q(p["W3"]) * (z2 > 0)
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(axis=0)
    dh1 = dh2 @ q(p["W2"]) * (z1 > 0)
    g["W1"] = dh1.T @ F_
    g["b1"] = dh1.sum(axis=0)
    return L, g, parts


def apply_M(G, x):
    """M x = G^T (G x)."""
    G = sp.csr_matrix(G)
    return G.T @ (G @ x)
