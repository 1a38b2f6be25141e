"""Parameter studies of TRPL+K on the GPU (Sec. 5.2 of Wu, Xue and
Stathopoulos): the maximum basis size q and the number of previous vectors l.

Sec. 5.2 varies q (with l = 1, p = 1) to compare TRPL+K with TRLan (TRPL+K
with l = 0 and no preconditioner) as the basis grows, and varies l from 0 to
5 (p = 5, q = 18, p_hat = 8, no preconditioner) to show that l = 1 gives the
benefit of +K.  The paper's matrices are not available here; the studies run
on seeded synthetic operators of this package (2D Laplacian, 3D lognormal
diffusion, a Chung-Lu graph Laplacian) through the C ABI, FP64 path, and
report matvecs, cycles and seconds per setting.  The basis is capped at
q = 64 (the library's largest), so the paper's q = 128...512 are not run.

Readings: the q sweep keeps p_hat = min(8, q - 3) (the paper's restart size,
reduced where q is too small to hold it with one +K vector and one Lanczos
step); the l sweep uses the paper's q = 18, p_hat = 8.

Usage: python -m paper_1711_10128_gb300.studies [--quick] > studies.json
"""
from __future__ import annotations

import argparse
import json
import time

Q_SWEEP = (8, 12, 16, 24, 32, 48, 64)
L_SWEEP = (0, 1, 2, 3, 4, 5)


def operators(quick=False):
    """Seeded synthetic operators (name -> Csr) the studies run on."""
    from . import workloads as W
    if quick:
        return {"laplace2d_40": W.laplacian_2d(40),
                "diffusion3d_12": W.diffusion_3d(12, W.lognormal_field(12, 1.0, 7))}
    return {"laplace2d_100": W.laplacian_2d(100),
            "diffusion3d_32": W.diffusion_3d(32, W.lognormal_field(32, 1.0, 7)),
            "chunglu_20000": W.chung_lu_laplacian(20000, 8.0, 2.1, 5)}


def restart_size(q):
    """p_hat of the q sweep: the paper's 8, or q - 3 for small q."""
    return min(8, q - 3)


def run_one(lib, h, Ad, n, p, q, k, l, tol, seed, precond):
    import numpy as np
    from . import workloads as W
    X0 = W.start_block(n, k, seed)
    t0 = time.perf_counter()
    ev, X, res, rc, info = lib.solve(h, Ad, None, p=p, q=q, k=k, l=l, tol=tol, X0=X0, max_cycles=20000,
                                     precond=precond, precision=lib.PRECISION_FP64)
    secs = time.perf_counter() - t0
    return {"p": p, "q": q, "k": k, "l": l, "status": lib.STATUS_NAMES.get(rc, rc), "mv_A": info["mv_A"],
            "cycles": info["cycles"], "seconds": secs, "max_resid": float(np.max(res)),
            "evals": [float(x) for x in ev]}


def q_sweep(lib, h, Ad, n, tol=1e-8, seed=12, qs=Q_SWEEP):
    """TRPL+K (l = 1) and TRLan (l = 0), p = 1, no preconditioner, for each q."""
    out = []
    for q in qs:
        for l in (1, 0):
            out.append(run_one(lib, h, Ad, n, 1, q, restart_size(q), l, tol, seed, lib.PRECOND_NONE))
    return out


def l_sweep(lib, h, Ad, n, tol=1e-8, seed=12, ls=L_SWEEP, p=5, q=18, k=8):
    """p = 5, q = 18, p_hat = 8, no preconditioner, for each l."""
    return [run_one(lib, h, Ad, n, p, q, k, l, tol, seed, lib.PRECOND_NONE) for l in ls]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="small operators only")
    ap.add_argument("--tol", type=float, default=1e-8)
    args = ap.parse_args()
    import torch
    from . import binding as lib
    h = lib.Handle(0)
    res = {}
    try:
        for name, A in operators(args.quick).items():
            Ad = lib.make_csr(torch.from_numpy(A.rowptr).cuda(), torch.from_numpy(A.col).cuda(),
                              torch.from_numpy(A.val).cuda())
            res[name] = {"n": A.n, "nnz": A.nnz, "q_sweep": q_sweep(lib, h, Ad, A.n, args.tol),
                         "l_sweep": l_sweep(lib, h, Ad, A.n, args.tol)}
    finally:
        h.close()
    print(json.dumps(res))


if __name__ == "__main__":
    main()
