"""The oracle's pins catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of an oracle module -- a dropped term
or pass, a wrong sign, index or operand, a missing mirror or rotation -- the
kind a restatement of Algorithm 1 (or of the FSAI and IC(0) definitions) can
plausibly contain.  A child process loads the planted copy in place of the
module and runs that module's pin tests (tests/test_oracle_pins.py,
test_oracle_fsai.py, test_oracle_ic0.py); at least one pin must fail.  The
mistake is planted in the oracle on the CPU only; nothing here touches the
CUDA path.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PINS = {
    "trplk": "tests/test_oracle_pins.py",
    "dense": "tests/test_oracle_pins.py",
    "ic0": "tests/test_oracle_ic0.py",
    "fsai": "tests/test_oracle_fsai.py",
}

# (module, mistake, text in the module, planted text); the first occurrence is replaced
MUTANTS = [
    ("trplk", "CGS pass 2 projects in the Euclidean, not the B-inner product",
     "    h2 = BU.T @ w\n", "    h2 = U.T @ w\n"),
    ("trplk", "CGS second pass dropped",
     "    h2 = BU.T @ w\n    w = w - U @ h2\n", "    h2 = 0.0 * h1\n"),
    ("trplk", "residual A x + theta B x",
     "R = AX - BX * theta[None, :]", "R = AX + BX * theta[None, :]"),
    ("trplk", "inner step shifted by + rho",
     "pend.append(Mapply(z - rhos[j % block] * BU[:, w - 1]))",
     "pend.append(Mapply(z + rhos[j % block] * BU[:, w - 1]))"),
    ("trplk", "upper triangle of T not mirrored",
     "return np.triu(T) + np.triu(T, 1).T", "return np.triu(T) + np.triu(T, 1)"),
    ("trplk", "T column stored as a row (transposed index)",
     "T[: w + 1, w] = U[:, : w + 1].T @ z", "T[w, : w + 1] = U[:, : w + 1].T @ z"),
    ("trplk", "X_prev taken one index late",
     "Xprev_next = X[:, t: min(t + l, p)].copy()", "Xprev_next = X[:, t + 1: min(t + 1 + l, p)].copy()"),
    ("trplk", "restart T without the Ritz values on its diagonal",
     "T[:k, :k] = np.diag(theta[:k])", "T[:k, :k] = 0.0"),
    ("trplk", "start block not rotated to Ritz vectors",
     "return X @ Y, AX @ Y, BX @ Y, theta, k, mvB", "return X, AX, BX, theta, k, mvB"),
    ("trplk", "restart rotates U, not B U, into B X",
     "BX = BU[:, :w] @ Yk", "BX = U[:, :w] @ Yk"),
    ("trplk", "Jacobi preconditioner D instead of D^-1",
     "dinv = 1.0 / A.diagonal()\n    return lambda v: dinv * v", "dinv = A.diagonal()\n    return lambda v: dinv * v"),
    ("trplk", "shift always theta_1, not the target's",
     "rho = theta[t]", "rho = theta[0]"),
    ("trplk", "eigenvector sign rule inverted",
     "if Y[i, c] < 0:", "if Y[i, c] > 0:"),
    ("trplk", "hard locking: new vectors not orthogonalised against the locked block",
     "cgs2(v, np.hstack([Q, U[:, :w]]), np.hstack([BQ, BU[:, :w]]), applyB)", "cgs2(v, U[:, :w], BU[:, :w], applyB)"),
    ("trplk", "block TRPL+K: every sequence shifted by the first target",
     "rhos[j % block]", "rhos[0]"),
    ("trplk", "shifted Jacobi without its floor",
     "d = np.maximum(a - rho * b, 1e-3 * a)", "d = a - rho * b"),
    ("trplk", "unrestarted Lanczos: T not mirrored",
     "T[j, : j + 1] = T[: j + 1, j]", "T[j, : j] = 0.0"),
    ("trplk", "norm of A: smallest instead of largest absolute row sum",
     "abs(A).sum(axis=1)).max()", "abs(A).sum(axis=1)).min()"),
    ("trplk", "recheck returns to the first pair, not the first failing one",
     "t = int(failing[0])", "t = 0"),
    ("trplk", "+K vectors orthogonalised against X only, not [X, G]",
     "C = BU[:, :w].T @ W\n                W = W - U[:, :w] @ C", "C = BU[:, :k].T @ W\n                W = W - U[:, :k] @ C"),
    ("trplk", "restart keeps p_hat - 1 vectors",
     "Yk = Y[:, :k]", "Yk = Y[:, :k - 1]"),
    ("trplk", "shifted Jacobi ignores B",
     "b = np.ones_like(a) if B is None else B.diagonal()", "b = np.ones_like(a)"),
    ("trplk", "breakdown in the first inner step not reported",
     "            status = BREAKDOWN\n            break\n        # +K", "            pass\n        # +K"),
    ("trplk", "rank-deficient start block accepted",
     "        if beta <= EPS_BREAKDOWN * beta0:\n            raise ValueError(\"start block is numerically rank deficient\")\n", ""),
    ("trplk", "B matvecs counted for B = I",
     "    cnt[\"mv_B\"] += mvB if Bm is not None else 0\n    t = 0", "    cnt[\"mv_B\"] += mvB\n    t = 0"),
    ("trplk", "unrestarted Lanczos: matvec count off by one",
     "            return float(theta), j + 1", "            return float(theta), j + 2"),
    ("trplk", "restart vectors' preconditioner applications not counted",
     '        cnt["prec"] += len(pend)\n', '        cnt["prec"] += 0\n'),
    ("trplk", "hard locking: X_prev not trimmed when pairs are locked",
     "            Xprev_next = Xprev_next[:, min(s, Xprev_next.shape[1]):]", "            Xprev_next = Xprev_next[:, 0:]"),
    ("trplk", "hard locking: at most one pair locked per cycle",
     "        while s < pa and conv[s]:\n            s += 1", "        while s < min(pa, 1) and conv[s]:\n            s += 1"),
    ("trplk", "hard locking: active outputs shifted by one vector",
     "    evecs = np.hstack([Q, X[:, : max(0, p - nq)]])[:, :p]",
     "    evecs = np.hstack([Q, X[:, 1: max(0, p - nq) + 1]])[:, :p]"),
    ("trplk", "X_prev capped at p_hat instead of p",
     "        Xprev_next = X[:, t: min(t + l, p)].copy()", "        Xprev_next = X[:, t: min(t + l, k)].copy()"),
    ("trplk", "hard locking: inner step shifted by rho g, not rho B g",
     "                v = Mapply(z - rho * BU[:, w - 1])", "                v = Mapply(z - rho * U[:, w - 1])"),
    ("dense", "Jacobi rotation with the wrong sign on one side",
     "A[:, j] = s * ai + c * aj", "A[:, j] = -s * ai + c * aj"),
    ("dense", "2x2 Schur step: tau of the wrong sign",
     "tau = (aqq - app) / (2.0 * apq)", "tau = (app - aqq) / (2.0 * apq)"),
    ("ic0", "off-diagonal factor entry divided by sqrt(l_jj)",
     "lij = s / row[j][j]", "lij = s / np.sqrt(row[j][j])"),
    ("ic0", "sweep adds the off-diagonal part",
     "x = (b - Ls @ x) / d", "x = (b + Ls @ x) / d"),
    ("ic0", "non-positive pivot taken",
     "                if not s > 0.0:\n                    raise ValueError(f\"IC(0) breakdown at row {i}: pivot {s}\")\n", ""),
    ("ic0", "the solver's preconditioner takes one sweep more",
     "    return lambda v: apply_M(L, v, sweeps)", "    return lambda v: apply_M(L, v, sweeps + 1)"),
    ("fsai", "classical FSAI row scaled by g_ii, not sqrt(g_ii)",
     "vals[rp[i]:rp[i + 1]] = gh / np.sqrt(gh[-1])", "vals[rp[i]:rp[i + 1]] = gh / gh[-1]"),
    ("fsai", "energy gradient with a wrong coefficient",
     "- 4.0 * s[rows] * v[cols])", "- 2.0 * s[rows] * v[cols])"),
    ("fsai", "Kaporin gradient: diagonal term halved",
     "gK[diag] -= 2.0 / (n * G.data[diag])", "gK[diag] -= 1.0 / (n * G.data[diag])"),
    ("fsai", "MLP backward gated by the wrong layer",
     'dh2 = dO @ q(p["W3"]) * (z2 > 0)', 'dh2 = dO @ q(p["W3"]) * (z1 > 0)'),
    ("fsai", "diagonal-dominance feature with the wrong sign",
     "F[i, 7] = (aii - off_sum) / aii", "F[i, 7] = (aii + off_sum) / aii"),
    ("fsai", "softplus derivative dropped",
     "dO[i, 3] += gG[e] * sigmoid(o[i, 3]) / sq[i]", "dO[i, 3] += gG[e] / sq[i]"),
    ("fsai", "loss vectors not scaled by their Jacobi energy",
     "cv = 1.0 / float(v @ (dinv * v))", "cv = 1.0"),
    ("fsai", "BF16 first-layer gradient from the unrounded features",
     'g["W1"] = dh1.T @ F_', 'g["W1"] = dh1.T @ F'),
    ("fsai", "BF16 mode: second hidden activation not rounded",
     "    h2 = q(np.maximum(z2, 0.0))", "    h2 = np.maximum(z2, 0.0)"),
    ("fsai", "BF16 mode: W2 not rounded in the forward pass",
     'z2 = h1 @ q(p["W2"]).T + p["b2"]', 'z2 = h1 @ p["W2"].T + p["b2"]'),
    ("fsai", "BF16 mode: backward through the unrounded W3",
     'dh2 = dO @ q(p["W3"]) * (z2 > 0)', 'dh2 = dO @ p["W3"] * (z2 > 0)'),
    ("fsai", "BF16 mode: backward through the unrounded W2",
     'dh1 = dh2 @ q(p["W2"]) * (z1 > 0)', 'dh1 = dh2 @ p["W2"] * (z1 > 0)'),
    ("fsai", "Kaporin weight 0.2 instead of 0.1",
     "GAMMA = 0.1", "GAMMA = 0.2"),
    ("fsai", "Kaporin measure with the sum instead of the mean",
     "    return float(np.log(d.mean()) - 2.0 * np.mean(np.log(G.diagonal())))",
     "    return float(np.log(d.sum()) - 2.0 * np.mean(np.log(G.diagonal())))"),
    ("fsai", "bfloat16 rounding without ties to even",
     "(b + 0x7FFF + ((b >> 16) & 1))", "(b + 0x8000)"),
]

BOOT = r"""
import sys, types
root, name, old, new, pins = sys.argv[1:6]
sys.path.insert(0, root)
import oracle
path = f"{root}/oracle/{name}.py"
src = open(path).read()
assert old in src, "mutation text not found"
mod = types.ModuleType("oracle." + name)
mod.__file__ = path
exec(compile(src.replace(old, new, 1), path, "exec"), mod.__dict__)
sys.modules["oracle." + name] = mod
setattr(oracle, name, mod)
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", f"{root}/{pins}"]))
"""


def _run(mutant):
    name, _, old, new = mutant
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", BOOT, ROOT, name, old, new, PINS[name]], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:] + r.stderr[-2000:]


def test_every_mutation_text_occurs_in_its_module():
    for name, what, old, _ in MUTANTS:
        assert old in open(os.path.join(ROOT, "oracle", f"{name}.py")).read(), what


def test_pins_catch_every_planted_mistake():
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        results = list(ex.map(_run, MUTANTS))
    survivors = []
    for (name, what, _, _), (rc, out) in zip(MUTANTS, results):
        # pytest exit code 1: tests ran and at least one failed (not a crash or collection error)
        if rc != 1:
            survivors.append(f"{name}: {what} (exit {rc})\n{out}")
    assert not survivors, "\n\n".join(survivors)


@pytest.mark.parametrize("name", sorted(set(PINS)))
def test_unmutated_modules_pass_their_pins_through_the_same_loader(name):
    rc, out = _run((name, "none", "from __future__ import annotations", "from __future__ import annotations"))
    assert rc == 0, out
