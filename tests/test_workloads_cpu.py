"""The seeded input generators shared by the oracle and the CUDA path: sizes
of the full-size operators, symmetry, the graph Laplacian's row sums, the
start block's determinism and range."""
import numpy as np
import scipy.sparse as sp

from paper_1711_10128_gb300 import workloads as W


def _symmetric(M):
    M = M.tocsr()
    D = (M - M.T).tocsr()
    return D.nnz == 0 or np.abs(D.data).max() <= 1e-14 * np.abs(M.data).max()


def test_diffusion_128_sizes_and_structure():
    A = W.diffusion_3d(128, W.lognormal_field(128, 1.0, 1))
    assert (A.n, A.nnz) == (2_097_152, 14_581_760)
    As = A.to_scipy()
    assert _symmetric(As)
    d = As.diagonal()
    off = np.asarray(abs(As).sum(axis=1)).ravel() - d
    assert np.all(d > 0) and np.all(d >= off - 1e-12 * d)   # weakly diagonally dominant (Dirichlet ghosts)
    assert np.all(As.data[As.indices != np.repeat(np.arange(A.n), np.diff(A.rowptr))] < 0)


def test_q1_pencil_96_sizes_and_structure():
    A, B = W.fem_q1_pencil(96, np.random.default_rng(2).uniform(1.0, 10.0, (96, 96, 96)))
    assert (A.n, A.nnz, B.nnz) == (884_736, 23_393_656, 23_393_656)
    assert _symmetric(A.to_scipy()) and _symmetric(B.to_scipy())
    assert np.all(B.to_scipy().diagonal() > 0)


def test_chung_lu_laplacian_full_size():
    L = W.chung_lu_laplacian(1 << 22, 16.0, 2.1, 3)
    assert (L.n, L.nnz) == (4_117_504, 71_231_354)
    Ls = L.to_scipy()
    assert _symmetric(Ls)
    assert np.allclose(Ls @ np.ones(L.n), 1e-3, rtol=0, atol=1e-9)   # (L + 1e-3 I) 1 = 1e-3 1
    deg = np.rint(Ls.diagonal() - 1e-3)                             # integer degrees
    assert deg.min() >= 1 and deg.sum() == L.nnz - L.n and deg.max() == np.diff(L.rowptr).max() - 1
    assert abs(deg.mean() - 16.0) < 0.5                              # mean degree of the component ~ 16
    ncomp, _ = sp.csgraph.connected_components(Ls, directed=False)
    assert ncomp == 1


def test_anisotropic_family_is_symmetric_with_axis_factors_in_range():
    for seed in (1000, 2000):
        ax = np.asarray(W.anisotropic_axes(seed), dtype=float)
        assert np.all(ax >= 1.0) and np.all(ax <= 100.0)
        assert _symmetric(W.anisotropic_diffusion(12, seed).to_scipy())


def test_start_block_is_deterministic_and_uniform():
    X = W.start_block(5000, 3, 17)
    assert X.shape == (5000, 3) and np.array_equal(X, W.start_block(5000, 3, 17))
    assert not np.array_equal(X, W.start_block(5000, 3, 18))
    assert X.min() >= -1.0 and X.max() < 1.0 and abs(X.mean()) < 0.05
    assert np.linalg.matrix_rank(X) == 3
