"""Plain FP64 TRPL+K on the CPU -- TEST INFRASTRUCTURE ONLY (see ``oracle``).

Follows Algorithm 1 of Wu, Xue and Stathopoulos (arXiv 1711.10128, Sec. 3)
step by step, extended to the pencil (A, B) with B symmetric positive definite
as the paper says it can be (end of Sec. 3; Algorithm 2 of Sec. 4 shows the
B-normalised form).  Library primitives serve as steps: scipy's CSR
matrix-vector product for the matvecs, numpy matrix products for the
projections and numpy's symmetric eigensolver for the small Rayleigh-Ritz
problem.  Nothing is blocked, fused or reordered beyond what the algorithm
states.

Readings where the paper is silent, ambiguous or garbled (each one is also
recorded in the design notes of the repository):

R1  Norm in the stopping rule: ||A|| is the 1-norm (largest absolute row sum),
    not the Frobenius norm of eq. (stop_criterion); the test is
    ||A x - theta B x||_2 <= tol * ||A||_1 * ||x||_2.
R2  Start block: Algorithm 1 takes p (here p_hat) orthonormal initial vectors;
    the caller's X0 (n x p_hat) is B-orthonormalised column by column by CGS2.
R3  Generalized pencil: every inner product is the B-inner product, the
    projector is (I - X X^T B), T = U^T A U, residual r = A x - theta B x.
    B-images of the basis (BU) are stored, so U^T B w is formed as (BU)^T w.
R4  Inner step (eq. (UpdateT) and the sentence after it): the next Lanczos
    vector is M(z - rho B g_j), not M(z - rho x_1) as printed; the printed
    form does not generate the Krylov space of C = (I - XX^T B) M (A - rho B)
    that Sec. 3 describes.  It is orthogonalised by two full classical
    Gram-Schmidt passes (CGS2) against all current basis columns.
R5  Breakdown: if the B-norm after CGS2 is <= 1e-12 times the B-norm before
    it, the inner loop stops early.
R6  Inner steps per cycle: m = q - p_hat - |X_prev| (first cycle m = q - p_hat),
    so each cycle costs q - p_hat matvecs and residuals use the stored images
    A U, B U (no extra matvec) -- the accounting behind the matvec counts of
    Tables 2-5.
R7  +K block: X_prev holds copies of x_t .. x_min(t+l-1, p) taken at the
    start of the cycle (before its RR, as in Algorithm 1); next cycle it is
    orthogonalised against [X, G] by block CGS2, then column by column
    within itself (CGS2); a column whose B-norm falls to <= 1e-10 (X_prev
    columns have unit B-norm) is dropped.  On convergence of the target the
    first X_prev column is removed.
R8  Rayleigh-Ritz: T is kept as its upper triangle (column c holds
    u_r^T A u_c for r <= c) and mirrored; eigenvalues ascending; each
    eigenvector is signed so its entry of largest magnitude (the first
    such) is positive.
R9  Convergence: one target advance per cycle at most (the IF of
    Algorithm 1); when t passes p all p residuals are re-checked and t
    returns to the first failing index if any has drifted above tol.
R10 Restart: X = U Y(:, 1:p_hat) (likewise AX, BX), T = diag(theta_1..p_hat),
    rho = theta_t, first Lanczos vector u = M r_t.  M is fixed across cycles
    (Jacobi: M = diag(A)^-1; the paper builds its ILU on A, Sec. 5.4).
R13 Hard locking (locking="hard"; Sec. 3 says it can replace the soft locking
    of Algorithm 1 but does not spell it out): after a cycle's Rayleigh-Ritz
    step, the leading run of converged Ritz pairs of the active basis is
    locked -- their vectors move to a locked block Q (kept, never rotated
    again), their Ritz values are final.  The locked vectors count against
    the memory budget: with |Q| locked the active search uses basis
    q - |Q|, restart size p_hat - |Q| and seeks the p - |Q| smallest pairs;
    every new basis vector (Lanczos, restart and +K vectors) is
    B-orthogonalised against [Q, U] by CGS2, while T and the Rayleigh-Ritz
    step cover the active basis only.  The target is always the smallest
    active pair; locking s pairs drops the first s columns of X_prev.  The
    solve ends when p pairs are locked.  Outputs are sorted by value.  Each
    cycle still costs q - p_hat matvecs, so the accounting of R6 holds.
R15 Block TRPL+K (block=b; the paper leaves a block TRPL+K to future work,
    Sec. 5.5): each cycle works on the b targets t .. t+b-1 (capped at
    p_hat - 1) with shifts rho_i = theta_{t+i}; the cycle's first b Lanczos
    vectors are M r_{t+i}, and every later one is M(A g - rho_i B g) from the
    vector g appended b steps earlier (so the columns cycle through the b
    sequences), each B-orthogonalised by CGS2 against every column already in
    the basis -- block Gram-Schmidt taken column by column, so the basis
    after each block spans the block Krylov space.  The target advances as in
    Algorithm 1 (R9); +K and the restart are unchanged, and each cycle still
    costs q - p_hat matvecs.  block = 1 is Algorithm 1.
R14 Per-cycle preconditioner (precond="jacobi_shifted"; Sec. 3 notes that M
    may change every cycle to approximate (A - rho_i B)^-1): the shifted
    Jacobi preconditioner M_i = diag(d)^-1 with
    d_j = max(a_jj - rho_i b_jj, 1e-3 a_jj), rebuilt at the start of every
    cycle from that cycle's rho_i (the floor keeps M_i positive definite when
    rho_i passes a diagonal ratio a_jj / b_jj).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

EPS_BREAKDOWN = 1e-12
EPS_DEPENDENT = 1e-10

OK, NOT_CONVERGED, BREAKDOWN = "ok", "not_converged", "breakdown"


def as_csr(rowptr, col, val, n):
    """CSR arrays -> scipy matrix (the matvec primitive)."""
    return sp.csr_matrix((np.asarray(val, np.float64), np.asarray(col), np.asarray(rowptr)), shape=(n, n))


def norm1(A) -> float:
    """||A||_1 = largest absolute row sum (reading R1); A symmetric."""
    return float(np.asarray(abs(A).sum(axis=1)).max())


def spmv(A, x):
    """y = A x (the matvec of Sec. 3, eq. (UpdateT))."""
    return A @ x


def jacobi_preconditioner(A):
    """M = diag(A)^-1 applied elementwise (reading R10)."""
    dinv = 1.0 / A.diagonal()
    return lambda v: dinv * v


def shifted_jacobi_preconditioner(A, B, rho):
    """M_i = diag(max(a_jj - rho b_jj, 1e-3 a_jj))^-1 (reading R14)."""
    a = A.diagonal()
    b = np.ones_like(a) if B is None else B.diagonal()
    d = np.maximum(a - rho * b, 1e-3 * a)
    dinv = 1.0 / d
    return lambda v: dinv * v


def make_preconditioner(A, precond):
    if precond is None or precond == "none":
        return lambda v: v.copy()
    if precond == "jacobi":
        return jacobi_preconditioner(A)
    if callable(precond):
        return precond
    raise ValueError(f"unknown preconditioner {precond!r}")


def cgs2(w, U, BU, applyB):
    """Orthogonalise w against the B-orthonormal columns of U (BU = B U) by two
    classical Gram-Schmidt passes in the B-inner product (readings R3, R4).

    Returns (w_out, B w_out, beta = ||w_out||_B, beta0 = ||w_in||_B, h1 + h2);
    beta0 is taken by Pythagoras from the two coefficient vectors and beta, so
    no extra matvec with B is spent.  w_out is NOT normalised.
    """
    h1 = BU.T @ w
    w = w - U @ h1
    h2 = BU.T @ w
    w = w - U @ h2
    Bw = applyB(w)
    beta = float(np.sqrt(max(w @ Bw, 0.0)))
    beta0 = float(np.sqrt(h1 @ h1 + h2 @ h2 + beta * beta))
    return w, Bw, beta, beta0, h1 + h2


def mirror_upper(T):
    """Symmetric matrix from its upper triangle (reading R8)."""
    return np.triu(T) + np.triu(T, 1).T


def rayleigh_ritz(T):
    """T = Y Theta Y^T (Algorithm 1, 'compute eigenpairs of T'), from the
    upper triangle of T; ascending Theta; sign rule of reading R8."""
    theta, Y = np.linalg.eigh(mirror_upper(np.asarray(T, np.float64)))
    for c in range(Y.shape[1]):
        i = int(np.argmax(np.abs(Y[:, c])))
        if Y[i, c] < 0:
            Y[:, c] = -Y[:, c]
    return theta, Y


def b_orthonormalise(X0, applyB):
    """B-orthonormalise the columns of X0 one by one with CGS2 (reading R2).
    Returns (X, BX, number of B matvecs)."""
    n, k = X0.shape
    X = np.zeros((n, k))
    BX = np.zeros((n, k))
    for c in range(k):
        w, Bw, beta, beta0, _ = cgs2(X0[:, c].astype(np.float64), X[:, :c], BX[:, :c], applyB)
        if beta <= EPS_BREAKDOWN * beta0:
            raise ValueError("start block is numerically rank deficient")
        X[:, c] = w / beta
        BX[:, c] = Bw / beta
    return X, BX, k


def initial_rayleigh_ritz(A, applyB, X0):
    """Algorithm 1, first two steps: RR on the B-orthonormal start block.
    Returns X, AX, BX (rotated to Ritz vectors), theta and matvec counts."""
    X, BX, mvB = b_orthonormalise(X0, applyB)
    AX = A @ X
    k = X.shape[1]
    T = np.zeros((k, k))
    for c in range(k):
        T[: c + 1, c] = X[:, : c + 1].T @ AX[:, c]
    theta, Y = rayleigh_ritz(T)
    return X @ Y, AX @ Y, BX @ Y, theta, k, mvB


def residual_norms(AX, BX, X, theta):
    """||A x_i - theta_i B x_i||_2 and ||x_i||_2 from stored images (R6)."""
    R = AX - BX * theta[None, :]
    return np.linalg.norm(R, axis=0), np.linalg.norm(X, axis=0)


def solve(A, B, p, q, k, l, tol, X0, precond="jacobi", max_cycles=5000, record=False, locking="soft", block=1):
    """TRPL+K (Algorithm 1) for the p smallest eigenpairs of (A, B).

    A, B: scipy CSR (B None means identity); q: maximum basis size; k: thick
    restart size p_hat >= p; l: maximum number of +K vectors; X0: n x k start
    block; precond: "jacobi", "none", "jacobi_shifted" (R14) or a function;
    locking: "soft" (Algorithm 1) or "hard" (R13); block: the block size of
    R15 (1: Algorithm 1; soft locking only).  Returns a dict with
    evals, evecs (B-orthonormal), resid (final FP64 check with fresh matvecs,
    relative to ||A||_1 ||x||_2), status, cycles, matvec counters and a
    per-cycle history.
    """
    if locking == "hard":
        if block != 1:
            raise ValueError("block TRPL+K is defined with soft locking")
        return _solve_hard(A, B, p, q, k, l, tol, X0, precond, max_cycles, record)
    if locking != "soft":
        raise ValueError(f"unknown locking {locking!r}")
    A = sp.csr_matrix(A)
    n = A.shape[0]
    if not (1 <= p <= k and k + max(l, 1) + 1 <= q <= n):
        raise ValueError("need 1 <= p <= k and k + max(l,1) + 1 <= q <= n")
    if not (1 <= block <= k and k + block + l <= q):
        raise ValueError("need 1 <= block <= k and k + block + l <= q")
    Bm = None if B is None else sp.csr_matrix(B)
    applyB = (lambda x: x.copy()) if Bm is None else (lambda x: Bm @ x)
    shifted = precond == "jacobi_shifted"
    Mapply = None if shifted else make_preconditioner(A, precond)
    normA = norm1(A)
    cnt = dict(mv_A=0, mv_B=0, prec=0, mv_check=0)

    # Algorithm 1: RR on the start block, target t = 1, rho = theta_1, X_prev = []
    X, AX, BX, theta, mvA, mvB = initial_rayleigh_ritz(A, applyB, np.asarray(X0, np.float64))
    cnt["mv_A"] += mvA
    cnt["mv_B"] += mvB if Bm is not None else 0
    t = 0
    Xprev = np.zeros((n, 0))
    U = np.zeros((n, q))
    AU = np.zeros((n, q))
    BU = np.zeros((n, q))
    T = np.zeros((q, q))
    history = []
    trace = []
    status = NOT_CONVERGED
    cycle = 0
    for cycle in range(1, max_cycles + 1):
        rho = theta[t]
        if shifted:   # M_i from this cycle's shift (R14)
            Mapply = shifted_jacobi_preconditioner(A, Bm, rho)
        U[:] = 0.0
        AU[:] = 0.0
        BU[:] = 0.0
        T[:] = 0.0
        U[:, :k], AU[:, :k], BU[:, :k] = X, AX, BX
        T[:k, :k] = np.diag(theta[:k])
        # the cycle's targets and shifts (R15; block = 1: Algorithm 1)
        tg = [min(t + i, k - 1) for i in range(block)]
        rhos = [theta[i] for i in tg]
        # first Lanczos vectors: u_i = M (A x_ti - rho_i B x_ti)   (Algorithm 1, restart)
        pend = [Mapply(AX[:, i] - theta[i] * BX[:, i]) for i in tg]
        cnt["prec"] += len(pend)
        nprev = Xprev.shape[1]
        m = q - k - nprev
        w = k
        broke = False
        # inner preconditioned Lanczos building G and T (eq. (UpdateT)); with
        # block > 1 the columns cycle through the b sequences (R15)
        for j in range(m):
            v = pend.pop(0)
            g, Bg, beta, beta0, _ = cgs2(v, U[:, :w], BU[:, :w], applyB)
            if Bm is not None:
                cnt["mv_B"] += 1
            if beta <= EPS_BREAKDOWN * beta0:
                broke = True
                break
            U[:, w] = g / beta
            BU[:, w] = Bg / beta
            z = A @ U[:, w]
            cnt["mv_A"] += 1
            AU[:, w] = z
            T[: w + 1, w] = U[:, : w + 1].T @ z
            w += 1
            if j + len(pend) < m - 1:
                pend.append(Mapply(z - rhos[j % block] * BU[:, w - 1]))
                cnt["prec"] += 1
        if broke and w == k and nprev == 0:
            status = BREAKDOWN
            break
        # +K: orthogonalise X_prev against [X, G], then within itself (R7)
        if nprev > 0:
            W = Xprev.copy()
            for _ in range(2):
                C = BU[:, :w].T @ W
                W = W - U[:, :w] @ C
            w0 = w
            for c in range(nprev):
                wv, Bw, beta, _, _ = cgs2(W[:, c], U[:, w0:w], BU[:, w0:w], applyB)
                if Bm is not None:
                    cnt["mv_B"] += 1
                if beta <= EPS_DEPENDENT:
                    continue
                U[:, w] = wv / beta
                BU[:, w] = Bw / beta
                w += 1
            # l matvecs complete T = U^T A U (Algorithm 1, 'compute the remaining T')
            for c in range(w0, w):
                z = A @ U[:, c]
                cnt["mv_A"] += 1
                AU[:, c] = z
                T[: c + 1, c] = U[:, : c + 1].T @ z
        # X_prev for the next cycle: x_t .. x_min(t+l-1, p) of this cycle's start
        Xprev_next = X[:, t: min(t + l, p)].copy()
        # Rayleigh-Ritz and the thick restart rotation (Algorithm 1, R8, R10)
        theta_all, Y = rayleigh_ritz(T[:w, :w])
        if record:
            trace.append(dict(T=mirror_upper(T[:w, :w]).copy(), theta=theta_all.copy(), w=w, m=m,
                              nprev=nprev, rho=rho, U=U[:, :w].copy(), AU=AU[:, :w].copy(),
                              BU=BU[:, :w].copy()))
        Yk = Y[:, :k]
        X = U[:, :w] @ Yk
        AX = AU[:, :w] @ Yk
        BX = BU[:, :w] @ Yk
        theta = theta_all[:k]
        rn, xn = residual_norms(AX, BX, X, theta)
        conv = rn <= tol * normA * xn
        # convergence test on the target, one advance per cycle (R9)
        t_before = t
        if conv[t]:
            t += 1
            Xprev_next = Xprev_next[:, 1:]
        history.append(dict(cycle=cycle, t=t_before, rho=rho, theta=theta[:p].copy(),
                            resid=(rn / (normA * xn))[:p].copy(), mv_A=cnt["mv_A"]))
        Xprev = Xprev_next
        if t >= p:
            failing = np.flatnonzero(~conv[:p])
            if failing.size == 0:
                status = OK
                break
            t = int(failing[0])
    # final FP64 check with fresh matvecs
    evecs = X[:, :p].copy()
    evals = theta[:p].copy()
    AXf = A @ evecs
    BXf = applyB(evecs) if Bm is None else Bm @ evecs
    cnt["mv_check"] += p
    rf = np.linalg.norm(AXf - BXf * evals[None, :], axis=0) / (normA * np.linalg.norm(evecs, axis=0))
    if status == OK and not np.all(rf <= tol):
        status = NOT_CONVERGED
    out = dict(evals=evals, evecs=evecs, resid=rf, status=status, cycles=cycle, normA=normA,
               history=history, **cnt)
    if record:
        out["trace"] = trace
    return out


def _solve_hard(A, B, p, q, k, l, tol, X0, precond, max_cycles, record):
    """TRPL+K with hard locking (reading R13); the steps of a cycle are those
    of `solve`, on the active basis, with every orthogonalisation also
    against the locked block Q."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    if not (1 <= p <= k and k + max(l, 1) + 1 <= q <= n):
        raise ValueError("need 1 <= p <= k and k + max(l,1) + 1 <= q <= n")
    Bm = None if B is None else sp.csr_matrix(B)
    applyB = (lambda x: x.copy()) if Bm is None else (lambda x: Bm @ x)
    shifted = precond == "jacobi_shifted"
    Mapply = None if shifted else make_preconditioner(A, precond)
    normA = norm1(A)
    cnt = dict(mv_A=0, mv_B=0, prec=0, mv_check=0)

    X, AX, BX, theta, mvA, mvB = initial_rayleigh_ritz(A, applyB, np.asarray(X0, np.float64))
    cnt["mv_A"] += mvA
    cnt["mv_B"] += mvB if Bm is not None else 0
    Q = np.zeros((n, 0))          # locked vectors
    BQ = np.zeros((n, 0))
    lam_q = []                    # their Ritz values
    Xprev = np.zeros((n, 0))
    history = []
    trace = []
    status = NOT_CONVERGED
    cycle = 0
    for cycle in range(1, max_cycles + 1):
        nq = Q.shape[1]
        qa, ka, pa = q - nq, k - nq, p - nq          # active basis, restart size, wanted
        rho = theta[0]                                # the target: smallest active pair
        if shifted:
            Mapply = shifted_jacobi_preconditioner(A, Bm, rho)
        U = np.zeros((n, qa))
        AU = np.zeros((n, qa))
        BU = np.zeros((n, qa))
        T = np.zeros((qa, qa))
        U[:, :ka], AU[:, :ka], BU[:, :ka] = X, AX, BX
        T[:ka, :ka] = np.diag(theta[:ka])
        v = Mapply(AX[:, 0] - rho * BX[:, 0])
        cnt["prec"] += 1
        nprev = Xprev.shape[1]
        m = qa - ka - nprev
        w = ka
        broke = False
        for j in range(m):
            # CGS2 against [Q, U] in the B-inner product
            g, Bg, beta, beta0, _ = cgs2(v, np.hstack([Q, U[:, :w]]), np.hstack([BQ, BU[:, :w]]), applyB)
            if Bm is not None:
                cnt["mv_B"] += 1
            if beta <= EPS_BREAKDOWN * beta0:
                broke = True
                break
            U[:, w] = g / beta
            BU[:, w] = Bg / beta
            z = A @ U[:, w]
            cnt["mv_A"] += 1
            AU[:, w] = z
            T[: w + 1, w] = U[:, : w + 1].T @ z
            w += 1
            if j < m - 1:
                v = Mapply(z - rho * BU[:, w - 1])
                cnt["prec"] += 1
        if broke and w == ka and nprev == 0:
            status = BREAKDOWN
            break
        if nprev > 0:
            QU = np.hstack([Q, U[:, :w]])
            BQU = np.hstack([BQ, BU[:, :w]])
            W = Xprev.copy()
            for _ in range(2):
                C = BQU.T @ W
                W = W - QU @ C
            w0 = w
            for c in range(nprev):
                wv, Bw, beta, _, _ = cgs2(W[:, c], U[:, w0:w], BU[:, w0:w], applyB)
                if Bm is not None:
                    cnt["mv_B"] += 1
                if beta <= EPS_DEPENDENT:
                    continue
                U[:, w] = wv / beta
                BU[:, w] = Bw / beta
                w += 1
            for c in range(w0, w):
                z = A @ U[:, c]
                cnt["mv_A"] += 1
                AU[:, c] = z
                T[: c + 1, c] = U[:, : c + 1].T @ z
        Xprev_next = X[:, 0: min(l, pa)].copy()
        theta_all, Y = rayleigh_ritz(T[:w, :w])
        if record:
            trace.append(dict(theta=theta_all.copy(), w=w, m=m, nprev=nprev, rho=rho, nq=nq,
                              QtBU=(BQ.T @ U[:, :w]).copy() if nq else np.zeros((0, w))))
        Yk = Y[:, :ka]
        X = U[:, :w] @ Yk
        AX = AU[:, :w] @ Yk
        BX = BU[:, :w] @ Yk
        theta = theta_all[:ka]
        rn, xn = residual_norms(AX, BX, X, theta)
        conv = rn <= tol * normA * xn
        history.append(dict(cycle=cycle, t=nq, rho=rho, nq=nq, theta=theta[:pa].copy(),
                            resid=(rn / (normA * xn))[:pa].copy(), mv_A=cnt["mv_A"]))
        # lock the leading run of converged active pairs (R13)
        s = 0
        while s < pa and conv[s]:
            s += 1
        if s > 0:
            Q = np.hstack([Q, X[:, :s]])
            BQ = np.hstack([BQ, BX[:, :s]])
            lam_q.extend(float(x) for x in theta[:s])
            X, AX, BX, theta = X[:, s:], AX[:, s:], BX[:, s:], theta[s:]
            Xprev_next = Xprev_next[:, min(s, Xprev_next.shape[1]):]
        Xprev = Xprev_next
        if Q.shape[1] >= p:
            status = OK
            break
    # outputs: locked pairs, then the active ones still wanted, sorted by value
    nq = Q.shape[1]
    evecs = np.hstack([Q, X[:, : max(0, p - nq)]])[:, :p]
    evals = np.concatenate([np.asarray(lam_q), theta[: max(0, p - nq)]])[:p]
    order = np.argsort(evals, kind="stable")
    evals, evecs = evals[order], evecs[:, order]
    AXf = A @ evecs
    BXf = applyB(evecs) if Bm is None else Bm @ evecs
    cnt["mv_check"] += p
    rf = np.linalg.norm(AXf - BXf * evals[None, :], axis=0) / (normA * np.linalg.norm(evecs, axis=0))
    if status == OK and not np.all(rf <= tol):
        status = NOT_CONVERGED
    out = dict(evals=evals, evecs=evecs, resid=rf, status=status, cycles=cycle, normA=normA,
               history=history, locked=nq, **cnt)
    if record:
        out["trace"] = trace
    return out


def lanczos_unrestarted(A, x0, tol, max_mv=5000):
    """Unrestarted Lanczos for the smallest eigenpair of A (B = I, M = I):
    the yardstick of the quasi-optimality discussion (Sec. 4; Fig. 1 of
    Sec. 5.1 compares TRPL+K with it).  The Krylov basis is kept in full and
    every new vector is re-orthogonalised against all of it by CGS2, so T_j is
    the exact projection; after each step the smallest Ritz pair of T_j is
    tested with the residual identity ||A x - theta x|| = beta_{j+1} |y_j|
    (last component of its eigenvector), against tol ||A||_1.  Returns
    (theta, matvecs); matvecs counts A x0 as the first."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    normA = norm1(A)
    Q = np.zeros((n, min(max_mv, n) + 1))
    q = np.asarray(x0, np.float64)
    Q[:, 0] = q / np.linalg.norm(q)
    T = np.zeros((Q.shape[1], Q.shape[1]))
    theta = None
    for j in range(min(max_mv, n)):
        z = A @ Q[:, j]
        T[: j + 1, j] = Q[:, : j + 1].T @ z
        T[j, : j + 1] = T[: j + 1, j]
        w, _, beta, _, _ = cgs2(z, Q[:, : j + 1], Q[:, : j + 1], lambda v: v.copy())
        th, Y = np.linalg.eigh(T[: j + 1, : j + 1])
        theta = th[0]
        if beta * abs(Y[j, 0]) <= tol * normA or beta == 0.0:
            return float(theta), j + 1
        Q[:, j + 1] = w / beta
    return float(theta), min(max_mv, n)
