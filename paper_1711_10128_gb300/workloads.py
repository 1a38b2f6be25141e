"""Seeded synthetic inputs for the TRPL+K eigensolver.

This module only builds inputs: sparse symmetric operators (A, B) in CSR form,
seeded coefficient fields and the counter-based start block.  It holds none of
the eigensolver's arithmetic, so both the CUDA path and the CPU oracle may take
their inputs from here.

Operators (the paper measures on SuiteSparse / Matrix Market / FEAP matrices,
Tables 1 and 6; these synthetic families stand in for them):

* ``laplacian_2d(N)``      -- 5-point Dirichlet Laplacian on an N x N grid.
* ``diffusion_3d(N, ...)``  -- cell-centred 7-point finite-volume diffusion on
  N^3 cells, harmonic-mean face coefficients, Dirichlet ghost cells.  With all
  coefficients 1 it is exactly the textbook 7-point Laplacian.
* ``fem_q1_pencil(N, E)``   -- trilinear (Q1) hexahedral stiffness K and
  consistent mass M on N^3 elements of the unit cube, Dirichlet on the faces
  x=0, y=0, z=0 (so n = N^3 free nodes), 27-point stencil.
* ``chung_lu_laplacian``    -- shifted graph Laplacian L + shift*I of a
  Chung-Lu power-law random graph restricted to its largest component.

Ordering is lexicographic with x fastest.  Every CSR is returned as
``(rowptr int64[n+1], col int32[nnz], val float64[nnz])`` with sorted columns.
"""
from __future__ import annotations

import numpy as np

GOLDEN64 = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


class Csr:
    """A symmetric sparse matrix in CSR form (host, numpy)."""

    def __init__(self, rowptr, col, val):
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)
        self.n = self.rowptr.size - 1
        self.nnz = int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))

    def diagonal(self):
        rows = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.rowptr))
        d = np.zeros(self.n)
        m = rows == self.col
        d[rows[m]] = self.val[m]
        return d


def _csr_from_offsets(shape, offsets, coeffs):
    """Build CSR from a structured stencil.

    ``shape`` is the grid (nz, ny, nx); ``offsets`` a list of (dz, dy, dx);
    ``coeffs[k]`` an array of ``shape`` with the coupling of each point to its
    neighbour at ``offsets[k]`` (entries whose neighbour lies outside the grid
    are ignored).  Offsets must be listed in increasing linear-index order so
    that each row's columns come out sorted.
    """
    nz, ny, nx = shape
    n = nz * ny * nx
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cols, vals, masks = [], [], []
    for (dz, dy, dx), c in zip(offsets, coeffs):
        jz, jy, jx = iz + dz, iy + dy, ix + dx
        inside = (jz >= 0) & (jz < nz) & (jy >= 0) & (jy < ny) & (jx >= 0) & (jx < nx)
        cols.append(((jz * ny + jy) * nx + jx).reshape(-1))
        vals.append(np.asarray(c, dtype=np.float64).reshape(-1))
        masks.append(inside.reshape(-1))
    cols = np.stack(cols, axis=1)
    vals = np.stack(vals, axis=1)
    masks = np.stack(masks, axis=1)
    counts = masks.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return Csr(rowptr, cols[masks].astype(np.int32), vals[masks])


def laplacian_2d(N: int) -> Csr:
    """5-point Dirichlet Laplacian (diagonal 4, neighbours -1) on N x N.

    Eigenvalues 4 sin^2(i pi / (2(N+1))) + 4 sin^2(j pi / (2(N+1))).
    """
    shape = (1, N, N)
    one = np.ones(shape)
    offs = [(0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1), (0, 1, 0)]
    return _csr_from_offsets(shape, offs, [-one, -one, 4 * one, -one, -one])


def lognormal_field(N: int, sigma: float, seed: int) -> np.ndarray:
    """Per-cell coefficients exp(sigma * xi), xi ~ N(0,1), shape (N, N, N)."""
    rng = np.random.default_rng(seed)
    return np.exp(sigma * rng.standard_normal((N, N, N)))


def diffusion_3d(N: int, coef: np.ndarray | None = None, axis=(1.0, 1.0, 1.0)) -> Csr:
    """Cell-centred 7-point diffusion operator on N^3 cells (no h^2 scaling).

    The coupling across the face between cells i and j in direction d is
    ``-axis[d] * 2 c_i c_j / (c_i + c_j)``; a boundary face adds
    ``axis[d] * c_i`` to the diagonal (Dirichlet ghost value 0).  ``axis`` is
    (x, y, z).  With ``coef`` = 1 and ``axis`` = 1 the eigenvalues are
    sum_d 4 sin^2(i_d pi / (2(N+1))).
    """
    if coef is None:
        coef = np.ones((N, N, N))
    c = np.asarray(coef, dtype=np.float64)
    ax, ay, az = (float(a) for a in axis)
    diag = np.zeros_like(c)
    faces = {}
    for name, axis_idx, f in (("x", 2, ax), ("y", 1, ay), ("z", 0, az)):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[axis_idx] = slice(0, N - 1)
        hi[axis_idx] = slice(1, N)
        ci, cj = c[tuple(lo)], c[tuple(hi)]
        h = f * 2.0 * ci * cj / (ci + cj)
        minus = np.zeros_like(c)   # coupling of a cell to its -d neighbour
        plus = np.zeros_like(c)    # coupling of a cell to its +d neighbour
        plus[tuple(lo)] = -h
        minus[tuple(hi)] = -h
        faces[name] = (minus, plus)
        diag[tuple(lo)] += h
        diag[tuple(hi)] += h
        first = [slice(None)] * 3
        last = [slice(None)] * 3
        first[axis_idx] = slice(0, 1)
        last[axis_idx] = slice(N - 1, N)
        diag[tuple(first)] += f * c[tuple(first)]
        diag[tuple(last)] += f * c[tuple(last)]
    offs = [(-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0)]
    coeffs = [faces["z"][0], faces["y"][0], faces["x"][0], diag,
              faces["x"][1], faces["y"][1], faces["z"][1]]
    return _csr_from_offsets((N, N, N), offs, coeffs)


def anisotropic_axes(seed: int, lo: float = 1.0, hi: float = 100.0):
    """Axis factors (1, r_y, r_z) with r log-uniform on [lo, hi]."""
    rng = np.random.default_rng(seed)
    r = np.exp(rng.uniform(np.log(lo), np.log(hi), size=2))
    return (1.0, float(r[0]), float(r[1]))


def anisotropic_diffusion(N: int, seed: int, sigma: float = 1.5) -> Csr:
    """One member of the anisotropic diffusion family: axis factors
    log-uniform on [1, 100], coefficients lognormal(0, sigma), both seeded."""
    axes = anisotropic_axes(seed)
    coef = lognormal_field(N, sigma, seed + 7919)
    return diffusion_3d(N, coef, axes)


def _q1_1d(h):
    k1 = np.array([[1.0, -1.0], [-1.0, 1.0]]) / h
    m1 = np.array([[2.0, 1.0], [1.0, 2.0]]) * (h / 6.0)
    return k1, m1


def fem_q1_pencil(N: int, E: np.ndarray | None = None):
    """Trilinear hexahedral stiffness A and consistent mass B on N^3 elements.

    Element e contributes E_e (K1 x M1 x M1 + M1 x K1 x M1 + M1 x M1 x K1) to A
    and M1 x M1 x M1 to B, with the 1D linear-element matrices
    K1 = (1/h)[[1,-1],[-1,1]], M1 = (h/6)[[2,1],[1,2]], h = 1/N.  Nodes on the
    faces x=0, y=0, z=0 are fixed (Dirichlet); the rest (natural boundary) are
    free, giving n = N^3 unknowns.  With E = 1 the eigenvalues are sums of the
    1D Dirichlet-Neumann values mu_k = (6/h^2)(1-cos t_k)/(2+cos t_k),
    t_k = (2k-1) pi / (2N).
    """
    if E is None:
        E = np.ones((N, N, N))
    E = np.asarray(E, dtype=np.float64)
    h = 1.0 / N
    k1, m1 = _q1_1d(h)
    P = N + 1  # nodes per direction, node (iz, iy, ix) with 0..N
    offs = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    off_index = {o: i for i, o in enumerate(offs)}
    ca = np.zeros((27, P, P, P))
    cb = np.zeros((27, P, P, P))
    # local node a = (az, ay, ax) in {0,1}^3; element (ez, ey, ex) touches nodes
    # (ez+az, ey+ay, ex+ax).  Coupling of node a to node b is added at node a
    # under offset b - a.
    for az in (0, 1):
        for ay in (0, 1):
            for ax in (0, 1):
                for bz in (0, 1):
                    for by in (0, 1):
                        for bx in (0, 1):
                            kval = (k1[ax, bx] * m1[ay, by] * m1[az, bz]
                                    + m1[ax, bx] * k1[ay, by] * m1[az, bz]
                                    + m1[ax, bx] * m1[ay, by] * k1[az, bz])
                            mval = m1[ax, bx] * m1[ay, by] * m1[az, bz]
                            o = off_index[(bz - az, by - ay, bx - ax)]
                            sl = (o, slice(az, az + N), slice(ay, ay + N), slice(ax, ax + N))
                            ca[sl] += E * kval
                            cb[sl] += mval
    # keep only free nodes (index >= 1 in every direction)
    free = (slice(1, P), slice(1, P), slice(1, P))
    A = _csr_from_offsets((N, N, N), offs, [ca[(i,) + free] for i in range(27)])
    B = _csr_from_offsets((N, N, N), offs, [cb[(i,) + free] for i in range(27)])
    return A, B


def chung_lu_laplacian(n: int, mean_degree: float, gamma: float, seed: int,
                       shift: float = 1e-3, largest_component: bool = True) -> Csr:
    """Shifted graph Laplacian L + shift*I of a Chung-Lu random graph.

    Expected-degree weights w_i proportional to (i + i0)^(-1/(gamma-1)),
    scaled to the requested mean degree; edge (i, j), i < j, is present with
    probability min(1, w_i w_j / sum(w)).  Edges are drawn with the
    Miller-Hagberg geometric-skip method (O(n + m)), vectorised over rows in
    rounds.  No self loops, unit weights.  If ``largest_component`` is set the
    graph is restricted (and relabelled) to its largest connected component.
    """
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    rng = np.random.default_rng(seed)
    beta = 1.0 / (gamma - 1.0)
    idx = np.arange(n, dtype=np.float64)

    def weights(i0):
        w = (idx + i0) ** (-beta)
        return w * (mean_degree * n / w.sum())

    # choose the offset i0 so that the largest expected degree is sqrt(sum w),
    # the usual Chung-Lu condition that keeps w_i w_j / S <= 1
    lo, hi = 0.0, float(n)
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        w = weights(mid)
        if w[0] > np.sqrt(w.sum()):
            lo = mid
        else:
            hi = mid
    w = weights(hi)
    S = w.sum()
    # Weights are sorted non-increasing; for row i walk j = i+1.. with
    # geometric skips under the running bound q = min(1, w_i w_j / S).
    rows_out, cols_out = [], []
    active = np.arange(n - 1, dtype=np.int64)
    j = active + 1
    q = np.minimum(1.0, w[active] * w[np.minimum(j, n - 1)] / S)
    while active.size:
        r = rng.random(active.size)
        with np.errstate(divide="ignore"):
            skip = np.where(q < 1.0, np.floor(np.log(r) / np.log1p(-q)), 0.0)
        skip = np.minimum(skip, n)  # avoid overflow
        j = j + skip.astype(np.int64)
        ok = j < n
        active, j, q = active[ok], j[ok], q[ok]
        if not active.size:
            break
        pij = np.minimum(1.0, w[active] * w[j] / S)
        accept = rng.random(active.size) < pij / q
        rows_out.append(active[accept])
        cols_out.append(j[accept])
        q = pij
        j = j + 1
        ok = j < n
        active, j, q = active[ok], j[ok], q[ok]
    ri = np.concatenate(rows_out) if rows_out else np.zeros(0, np.int64)
    ci = np.concatenate(cols_out) if cols_out else np.zeros(0, np.int64)
    W = sp.coo_matrix((np.ones(ri.size), (ri, ci)), shape=(n, n)).tocsr()
    W = W + W.T
    W.data[:] = 1.0
    if largest_component:
        ncomp, lab = connected_components(W, directed=False)
        big = np.argmax(np.bincount(lab))
        keep = np.flatnonzero(lab == big)
        W = W[keep][:, keep]
    deg = np.asarray(W.sum(axis=1)).ravel()
    L = sp.diags(deg + shift) - W
    L = L.tocsr()
    L.sort_indices()
    return Csr(L.indptr, L.indices, L.data)


def splitmix64_uniform(seed: int, counters: np.ndarray) -> np.ndarray:
    """uniform[-1, 1) values from one SplitMix64 step per counter.

    SplitMix64 (Steele, Lea and Flood, 2014): state s = seed XOR counter;
    z = s + 0x9E3779B97F4A7C15; z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB; z ^= z >> 31.  The top 53 bits
    give u in [0, 1) and the value is 2u - 1.
    """
    with np.errstate(over="ignore"):
        z = np.uint64(seed) ^ counters.astype(np.uint64)
        z = z + GOLDEN64
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        z = z ^ (z >> np.uint64(31))
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0


def start_block(n: int, k: int, seed: int) -> np.ndarray:
    """The n x k start block, column-major: element (i, c) uses counter c*n + i."""
    c = np.arange(n * k, dtype=np.uint64)
    return splitmix64_uniform(seed, c).reshape(k, n).T.copy(order="F")
